"""The method's variants at the sizes the benchmark times, on sampled windows:
fourth-order steps and the time-dependent potential on 8192^2, the 3-D
lattice on 512^3.  A site after s sweeps-and-phase substeps depends only on
sites within 2s per axis (windows start on even coordinates), so the oracle
evolves small windows exactly; only sites outside the window's light cone of
its artificial edges are compared.  Tolerance 1e-6 relative L2 (a few steps
of FP32 rounding).
"""
import numpy as np
import pytest

import oracle
from paper_1208_2407_gb300 import trotter
from paper_1208_2407_gb300 import workloads as wl

from gpu_helpers import ensure_library, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def _windows(rng, shape, half, count):
    """Window origins (even) and ends for `count` centres: the corners, edge
    midpoints and random points."""
    dims = len(shape)
    centres = []
    for corner in range(2 ** dims):
        centres.append(tuple((shape[a] - 1) if (corner >> a) & 1 else 0 for a in range(dims)))
    while len(centres) < count:
        centres.append(tuple(int(rng.integers(0, shape[a])) for a in range(dims)))
    out = []
    for c in centres:
        lo = [max(0, (c[a] - half) & ~1) for a in range(dims)]
        hi = [min(shape[a], lo[a] + 2 * half + 2) for a in range(dims)]
        out.append((lo, hi))
    return out


def _inner(lo, hi, shape, margin):
    """Slices (in window coordinates) of the sites the window's own edges do
    not reach."""
    sl = []
    for a in range(len(shape)):
        b0 = 0 if lo[a] == 0 else margin
        b1 = (hi[a] - lo[a]) if hi[a] == shape[a] else (hi[a] - lo[a]) - margin
        sl.append(slice(b0, b1))
    return tuple(sl)


def _compare(gpu_re, gpu_im, re0, im0, shape, margin, count, seed, evolve_window):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for lo, hi in _windows(rng, shape, margin + 6, count):
        box = tuple(slice(lo[a], hi[a]) for a in range(len(shape)))
        ore, oim = evolve_window(re0[box].double().cpu().numpy(),
                                 im0[box].double().cpu().numpy(), box)
        inner = _inner(lo, hi, shape, margin)
        gbox = tuple(slice(box[a].start + inner[a].start, box[a].start + inner[a].stop)
                     for a in range(len(shape)))
        err = rel_l2(gpu_re[gbox].double().cpu().numpy(), gpu_im[gbox].double().cpu().numpy(),
                     ore[inner], oim[inner])
        worst = max(worst, err)
    return worst


def _random_state(shape, seed):
    import torch
    gen = torch.Generator(device="cuda").manual_seed(seed)
    re = torch.randn(shape, generator=gen, device="cuda", dtype=torch.float32)
    im = torch.randn(shape, generator=gen, device="cuda", dtype=torch.float32)
    return re, im


def test_fourth_order_8192_sampled_windows():
    n, steps = 8192, 2                       # 10 second-order substeps
    re0, im0 = _random_state((n, n), 31)
    V = wl.random_gaussians_potential(np.random.default_rng(31), n, n)
    g = trotter.Grid(n, n, "f32")
    try:
        g.set_state(re0, im0)
        g.set_potential(V, wl.DT, wl.THETA, order=4)
        g.evolve(steps)
        out_re, out_im = g.get_state(np.float32, device=True)
    finally:
        g.close()
    worst = _compare(out_re, out_im, re0, im0, (n, n), 2 * 5 * steps + 2, 24, 31,
                     lambda wr, wi, box: oracle.evolve(wr, wi, V[box], wl.DT, wl.THETA, steps,
                                                       order=4))
    assert worst < 1e-6, worst


def test_drive_8192_sampled_windows():
    n, steps = 8192, 8
    re0, im0 = _random_state((n, n), 32)
    V = wl.random_gaussians_potential(np.random.default_rng(32), n, n)
    V1 = (np.arange(n) - n / 2.0)[None, :] * np.ones((n, 1)) * 1e-3
    a = 0.5 + 0.3 * np.sin(0.7 * (np.arange(steps) + 0.5) * wl.DT)
    g = trotter.Grid(n, n, "f32")
    try:
        g.set_state(re0, im0)
        g.set_potential(V, wl.DT, wl.THETA)
        g.set_drive(V1, a)
        g.evolve(steps)
        out_re, out_im = g.get_state(np.float32, device=True)
    finally:
        g.close()
    worst = _compare(out_re, out_im, re0, im0, (n, n), 2 * steps + 2, 24, 32,
                     lambda wr, wi, box: oracle.evolve_driven(wr, wi, V[box], V1[box], a, wl.DT,
                                                              wl.THETA))
    assert worst < 1e-6, worst


def test_3d_512_sampled_windows():
    import torch
    n, steps = 512, 4
    re0, im0 = _random_state((n, n, n), 33)
    V = wl.harmonic_potential3(n, n, n, 1e-2)
    g = trotter.Grid(n, n, "f32", nz=n)
    try:
        g.set_state(re0, im0)
        g.set_potential(torch.from_numpy(V).cuda(), wl.DT, wl.THETA)
        g.evolve(steps)
        out_re, out_im = g.get_state(np.float32, device=True)
    finally:
        g.close()
    worst = _compare(out_re, out_im, re0, im0, (n, n, n), 2 * steps + 2, 16, 33,
                     lambda wr, wi, box: oracle.evolve3(wr, wi, V[box], wl.DT, wl.THETA, steps))
    assert worst < 1e-6, worst
