"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and
compare with the FP64 oracle."""
import numpy as np

from paper_1208_2407_gb300 import trotter


def ensure_library():
    from paper_1208_2407_gb300 import build
    build.build()
    return trotter.load()


def run_gpu(re, im, V, dt, theta, steps, dtype="f32", path="fused", K=0, observe=False):
    ny, nx = re.shape
    g = trotter.Grid(nx, ny, dtype)
    try:
        g.set_state(re, im)
        g.set_potential(V, dt, theta)
        if path == "fused":
            g.evolve(steps, K)
        elif path == "plain":
            g.evolve_plain(steps)
        else:
            raise ValueError(path)
        out = g.get_state(np.float64)
        obs = g.observe() if observe else None
    finally:
        g.close()
    return out, obs


def rel_l2(are, aim, bre, bim):
    num = np.sqrt(np.sum((are - bre) ** 2 + (aim - bim) ** 2))
    den = np.sqrt(np.sum(bre ** 2 + bim ** 2))
    return float(num / den) if den > 0 else float(num)


def random_state(rng, nx, ny):
    re = rng.standard_normal((ny, nx))
    im = rng.standard_normal((ny, nx))
    s = np.sqrt(np.sum(re * re + im * im))
    return re / s, im / s


def grid_plane(g, index):
    """A view of plane `index` of a grid's slab (0/1 state pair A, 2/3 pair B,
    4 gamma_V, 5 s_V, 6 V) as an (ny, nx) tensor of the grid's dtype."""
    import torch
    L = g.layout
    es = 8 if g.dtype == trotter.TS_F64 else 4
    tdt = torch.float64 if es == 8 else torch.float32
    start = index * int(L.plane_bytes)
    raw = g.slab[start:start + int(L.pitch) * g.ny * es]
    return raw.view(tdt).reshape(g.ny, int(L.pitch))[:, :g.nx]
