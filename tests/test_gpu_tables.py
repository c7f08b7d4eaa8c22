"""Table preparation on the GPU against FP64-then-round (host numpy).

FP32 grids evaluate gamma_V = 2 sin^2(V dt / 2) and s_V = sin(V dt) in
double-float arithmetic (V dt carried to ~2^-46 relative) and round once.
Each entry must be within one ulp of the FP64 value rounded to FP32, or --
near a zero of sin, where the FP64 value itself is only as accurate as the
rounded argument -- within 2^-44 |V dt| of it; a mismatch is rare.  In the
FP32 subnormal range (values below ~1e-36) a few ulps are allowed.
"""
import numpy as np
import pytest

from paper_1208_2407_gb300 import trotter

from gpu_helpers import ensure_library, grid_plane, random_state, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def _ulps(a, b):
    ai = a.astype(np.float32).view(np.int32).astype(np.int64)
    bi = b.astype(np.float32).view(np.int32).astype(np.int64)
    # map to a monotone integer line
    ai = np.where(ai < 0, -(ai & 0x7fffffff), ai)
    bi = np.where(bi < 0, -(bi & 0x7fffffff), bi)
    return np.abs(ai - bi)


@pytest.mark.parametrize("dt", [0.05, 0.013, 1.0])
def test_phase_table_matches_fp64_then_round(dt):
    rng = np.random.default_rng(int(dt * 1000))
    nx, ny = 301, 207
    mag = 10.0 ** rng.uniform(-25, np.log10(100.0 / dt), (ny, nx))
    V = mag * rng.choice([-1.0, 1.0], (ny, nx))
    V[0, :10] = 0.0
    V[1, :5] = [1e-300, -5e-70, 3.0 * np.pi / dt, 150.0 / dt, -2000.0 / dt]   # last two: FP64 path
    g = trotter.Grid(nx, ny, "f32")
    try:
        g.set_potential(V, dt, dt / 2)
        pg = grid_plane(g, 4).cpu().numpy()
        ps = grid_plane(g, 5).cpu().numpy()
        vp = grid_plane(g, 6).cpu().numpy()
    finally:
        g.close()
    h = 0.5 * V * dt
    want_pg = (2.0 * np.sin(h) ** 2).astype(np.float32)
    want_ps = np.sin(V * dt).astype(np.float32)
    want_vp = V.astype(np.float32)
    arg_err = 2.0 ** -44 * np.abs(V * dt)
    for name, got, want in (("gamma", pg, want_pg), ("s", ps, want_ps), ("V", vp, want_vp)):
        u = _ulps(got, want)
        normal = np.abs(want) >= 1e-36
        close = (u <= 1) | (np.abs(got.astype(np.float64) - want) <= arg_err)
        assert close[normal].all(), (name, V[normal & ~close][:5], got[normal & ~close][:5],
                                     want[normal & ~close][:5])
        assert np.mean(u[normal] > 0) < 1e-3, name
        assert u[~normal].max(initial=0) <= 4, name


def test_large_theta_runs_the_plain_path():
    rng = np.random.default_rng(2)
    re, im = random_state(rng, 40, 30)
    V = rng.uniform(-0.5, 0.5, (30, 40))
    dt, theta = 2.0, 1.0        # theta > pi/4: the fused kernel's lifting form does not apply
    (a_re, a_im), _ = run_gpu(re, im, V, dt, theta, 5, K=4)
    (b_re, b_im), _ = run_gpu(re, im, V, dt, theta, 5, path="plain")
    assert np.array_equal(a_re, b_re) and np.array_equal(a_im, b_im)
