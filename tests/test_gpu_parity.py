"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 grids (plain path) 1e-12 relative L2; FP32 grids 1e-5
relative L2 (the stated FP32 bar; the FP32 rounding budget after ~9000
sweeps is a few 1e-6).  Observables are compared against the oracle's
compensated sums of the same (rounded) state.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1208_2407_gb300 import trotter
from paper_1208_2407_gb300 import workloads as wl

from gpu_helpers import ensure_library, random_state, rel_l2, run_gpu

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-12
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


# ---------------------------------------------------------------------------
# the 256^2 FP64 workload: plain FP64 path, psi, norm, <x>, <y>
# ---------------------------------------------------------------------------
def test_plain_fp64_workload_matches_oracle():
    c = wl.plain_fp64_256()
    (gre, gim), obs = run_gpu(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"],
                              dtype="f64", path="plain", observe=True)
    ore, oim = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    assert rel_l2(gre, gim, ore, oim) < FP64_TOL
    m = oracle.moments(ore, oim)
    assert abs(obs["norm"] - m[0]) < 1e-13
    assert abs(obs["x"] - m[1] / m[0]) < 1e-10
    assert abs(obs["y"] - m[2] / m[0]) < 1e-10
    assert abs(obs["norm"] - 1.0) < 1e-12


def test_fp64_default_evolve_on_the_workload():
    """ts_evolve on an FP64 grid merges the sweeps where steps meet (one sweep
    per launch, 6 n + 2 sweeps and n phases for n steps, lifting form):
    within FP64 rounding of the oracle and of the literal plain sequence."""
    c = wl.plain_fp64_256()
    (a_re, a_im), _ = run_gpu(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"],
                              dtype="f64", path="fused", K=0)
    (b_re, b_im), _ = run_gpu(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"],
                              dtype="f64", path="plain")
    ore, oim = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    assert rel_l2(a_re, a_im, ore, oim) < FP64_TOL
    assert rel_l2(a_re, a_im, b_re, b_im) < FP64_TOL


@pytest.mark.parametrize("steps,expected", [(1, 9), (2, 16), (7, 51)])
def test_fp64_default_evolve_launch_count(steps, expected):
    rng = np.random.default_rng(3)
    re, im = random_state(rng, 40, 24)
    g = trotter.Grid(40, 24, "f64")
    try:
        g.set_state(re, im)
        g.set_potential(None, 0.05, 0.025)
        trotter.ts_launch_count(reset=True)
        g.evolve(steps)
        assert trotter.ts_launch_count() == expected      # 7 n + 2
        trotter.ts_launch_count(reset=True)
        g.evolve_plain(steps)
        assert trotter.ts_launch_count() == 9 * steps
    finally:
        g.close()


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 2), (3, 5), (17, 33), (1, 64), (64, 1),
                                   (257, 131), (113, 1000)])
@pytest.mark.parametrize("dt,theta", [(0.05, 0.025), (-0.05, -0.025), (2.0, 1.3)])
def test_small_grids_fp64_default(nx, ny, dt, theta):
    """Merged sweeps at every angle range: theta = 1.3 puts the merged angle
    2.6 beyond pi/2, where those sweeps take the versine form."""
    rng = np.random.default_rng(nx * 31 + ny)
    re, im = random_state(rng, nx, ny)
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    (gre, gim), _ = run_gpu(re, im, V, dt, theta, 11, dtype="f64")
    ore, oim = oracle.evolve(re, im, V, dt, theta, 11)
    assert rel_l2(gre, gim, ore, oim) < FP64_TOL


# ---------------------------------------------------------------------------
# small and ragged grids: every path, every fused depth
# ---------------------------------------------------------------------------
SIZES = [(1, 1), (2, 2), (3, 5), (17, 33), (130, 66), (1, 64), (64, 1), (257, 131),
         (121, 9), (240, 242), (113, 1000)]


@pytest.mark.parametrize("nx,ny", SIZES)
def test_small_grids_plain_fp64(nx, ny):
    rng = np.random.default_rng(nx * 7919 + ny)
    re, im = random_state(rng, nx, ny)
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    (gre, gim), _ = run_gpu(re, im, V, 0.05, 0.025, 11, dtype="f64", path="plain")
    ore, oim = oracle.evolve(re, im, V, 0.05, 0.025, 11)
    assert rel_l2(gre, gim, ore, oim) < FP64_TOL


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("K", [None, 1, 2, 3, 4, 5, 6, 7, 8])
def test_small_grids_fp32(nx, ny, K):
    rng = np.random.default_rng(nx * 104729 + ny)
    re, im = random_state(rng, nx, ny)
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    steps = 13
    path = "plain" if K is None else "fused"
    (gre, gim), _ = run_gpu(re, im, V, 0.05, 0.025, steps, dtype="f32", path=path, K=K or 0)
    ore, oim = oracle.evolve(re, im, V, 0.05, 0.025, steps)
    err = rel_l2(gre, gim, ore, oim)
    assert err < 2e-6, err          # 13 steps: far inside the 1e-5 bar


@pytest.mark.parametrize("K", [1, 2, 3, 4, 8])
def test_fused_matches_plain_fp32_on_a_packet(K):
    c = wl.harmonic_2048(seed=3, n=300, steps=24)
    (a_re, a_im), _ = run_gpu(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"], K=K)
    (b_re, b_im), _ = run_gpu(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"],
                              path="plain")
    assert rel_l2(a_re, a_im, b_re, b_im) < 2e-6


# ---------------------------------------------------------------------------
# the 2048^2 FP32 precision workload, 1000 steps, vs the FP64 oracle
# ---------------------------------------------------------------------------
# Norm drift bound: the lifting and versine forms keep each sweep's defect
# |c^2 + s^2 - 1| near 1e-10 (tables rounded once from FP64), so 1000 steps of
# ~7 sweeps drift the norm by at most ~1e-6 even if every defect had one sign;
# FP32 rounding itself is unbiased and adds ~1e-8.
NORM_DRIFT_TOL = 1e-6
# The energy of the Trotter map itself oscillates at O(dt^2), so the GPU's
# energy drift is compared with the oracle's drift on the same packet: FP32
# state errors of ~4e-6 rel-L2 move <psi|H|psi> by ~1e-5 of |E| at most.
ENERGY_DRIFT_TOL = 2e-5


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_harmonic_2048_fp32_vs_fp64_oracle(seed):
    c = wl.harmonic_2048(seed=seed)
    g = trotter.Grid(c["nx"], c["ny"], "f32")
    try:
        g.set_state(c["re"], c["im"])
        g.set_potential(c["V"], c["dt"], c["theta"])
        obs0 = g.observe()
        g.evolve(c["steps"])
        obs = g.observe()
        gre, gim = g.get_state(np.float64)
    finally:
        g.close()
    ore, oim = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"],
                             nthreads=NTHREADS)
    err = rel_l2(gre, gim, ore, oim)
    assert err < FP32_TOL, err
    norm_drift = abs(obs["norm"] - obs0["norm"])
    assert norm_drift < NORM_DRIFT_TOL, norm_drift
    e0 = sum(oracle.energy(c["re"], c["im"], c["V"]))
    e_oracle = sum(oracle.energy(ore, oim, c["V"]))
    e_gpu0 = obs0["e_kin"] + obs0["e_pot"]
    e_gpu = obs["e_kin"] + obs["e_pot"]
    scale = max(1e-12, abs(e0))
    drift_gpu = (e_gpu - e_gpu0) / scale
    drift_oracle = (e_oracle - e0) / scale
    assert abs(drift_gpu - drift_oracle) < ENERGY_DRIFT_TOL, (drift_gpu, drift_oracle)
    assert abs(e_gpu - e_oracle) < 1e-4 * max(1.0, abs(e_oracle))
    print("config 2 seed %d: rel-L2 %.3e, norm drift %.2e, energy drift %.3e (oracle %.3e)"
          % (seed, err, norm_drift, drift_gpu, drift_oracle))


# ---------------------------------------------------------------------------
# full size, the launch configuration the benchmark times: sampled windows.
# A site after n steps depends only on sites within 2n per axis (for a window
# whose origin is even), so the oracle evolves small windows exactly.
# ---------------------------------------------------------------------------
def _window_parity(n, steps, K, count, seed):
    import torch
    gen = torch.Generator(device="cuda").manual_seed(seed)
    re_d = torch.randn((n, n), generator=gen, device="cuda", dtype=torch.float32)
    im_d = torch.randn((n, n), generator=gen, device="cuda", dtype=torch.float32)
    rng = np.random.default_rng(seed)
    V = wl.random_gaussians_potential(rng, n, n)
    g = trotter.Grid(n, n, "f32")
    try:
        g.set_state(re_d, im_d)
        g.set_potential(V, wl.DT, wl.THETA)
        g.evolve(steps, K)
        out_re, out_im = g.get_state(np.float32, device=True)
    finally:
        g.close()
    margin = 2 * steps + 2
    half = margin + 6
    centers = [(0, 0), (n - 1, 0), (0, n - 1), (n - 1, n - 1), (n // 2, 0), (0, n // 2),
               (n - 1, n // 2), (n // 2, n - 1)]
    for v in (120, 112, 104):          # strip boundaries of the fused geometry
        centers += [(v * 3 + d, int(rng.integers(0, n))) for d in (-1, 0, 1)]
    while len(centers) < count:
        centers.append((int(rng.integers(0, n)), int(rng.integers(0, n))))
    worst = 0.0
    for xc, yc in centers:
        xa = max(0, (xc - half) & ~1)
        ya = max(0, (yc - half) & ~1)
        xb = min(n, xa + 2 * half + 2)
        yb = min(n, ya + 2 * half + 2)
        wre = re_d[ya:yb, xa:xb].double().cpu().numpy()
        wim = im_d[ya:yb, xa:xb].double().cpu().numpy()
        ore, oim = oracle.evolve(wre, wim, V[ya:yb, xa:xb], wl.DT, wl.THETA, steps)
        # sites unaffected by the window's artificial edges
        x0 = 0 if xa == 0 else margin
        y0 = 0 if ya == 0 else margin
        x1 = (xb - xa) if xb == n else (xb - xa) - margin
        y1 = (yb - ya) if yb == n else (yb - ya) - margin
        gre = out_re[ya + y0:ya + y1, xa + x0:xa + x1].double().cpu().numpy()
        gim = out_im[ya + y0:ya + y1, xa + x0:xa + x1].double().cpu().numpy()
        err = rel_l2(gre, gim, ore[y0:y1, x0:x1], oim[y0:y1, x0:x1])
        worst = max(worst, err)
    return worst


@pytest.mark.parametrize("K", [0, 1, 2, 3, 8])
def test_full_size_8192_sampled_windows(K):
    worst = _window_parity(8192, 8, K, 48, seed=11 + K)
    assert worst < 1e-6, worst


def test_full_size_16384_sampled_windows():
    worst = _window_parity(16384, 8, 0, 32, seed=5)
    assert worst < 1e-6, worst


# ---------------------------------------------------------------------------
# observables against the oracle's compensated sums of the same state
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_observables_match_oracle(dtype):
    rng = np.random.default_rng(21)
    nx, ny = 130, 67
    re, im = random_state(rng, nx, ny)
    V = rng.uniform(-1, 1, (ny, nx))
    if dtype == "f32":      # the oracle sums the state the grid actually holds
        re, im = re.astype(np.float32).astype(np.float64), im.astype(np.float32).astype(np.float64)
        Vr = V.astype(np.float32).astype(np.float64)
    else:
        Vr = V
    g = trotter.Grid(nx, ny, dtype)
    try:
        g.set_state(re, im)
        g.set_potential(V, 0.05, 0.025)
        obs = g.observe()
        nrm = g.norm()
    finally:
        g.close()
    m = oracle.moments(re, im)
    kin, pot = oracle.energy(re, im, Vr, 1.0)
    assert obs["norm"] == pytest.approx(m[0], rel=1e-14)
    assert nrm == pytest.approx(m[0], rel=1e-14)
    assert obs["x"] == pytest.approx(m[1] / m[0], rel=1e-13)
    assert obs["y"] == pytest.approx(m[2] / m[0], rel=1e-13)
    assert obs["x2"] == pytest.approx(m[3] / m[0], rel=1e-13)
    assert obs["y2"] == pytest.approx(m[4] / m[0], rel=1e-13)
    assert obs["e_kin"] == pytest.approx(kin, rel=1e-12, abs=1e-15)
    assert obs["e_pot"] == pytest.approx(pot, rel=1e-12, abs=1e-15)


# ---------------------------------------------------------------------------
# boundary behaviour: round trips, batching, argument errors, launch counts
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_state_round_trip_host_and_device(dtype):
    import torch
    rng = np.random.default_rng(4)
    re, im = random_state(rng, 77, 45)
    g = trotter.Grid(77, 45, dtype)
    try:
        g.set_state(re, im)
        a_re, a_im = g.get_state(np.float64)
        b_re, b_im = g.get_state(np.float32, device=True)
        g.set_state(b_re.contiguous(), b_im.contiguous())
        c_re, c_im = g.get_state(np.float32)
    finally:
        g.close()
    tol = 0.0 if dtype == "f64" else 1e-7
    assert np.max(np.abs(a_re - re)) <= tol * np.max(np.abs(re))
    assert np.array_equal(b_re.cpu().numpy(), re.astype(np.float32))
    assert np.array_equal(c_re, b_re.cpu().numpy())


def test_batched_equals_individual():
    """FP32 grids share one multi-grid launch sequence; an FP64 grid in the
    batch runs its own sequence (K applies to FP32 grids only)."""
    rng = np.random.default_rng(8)
    shapes = [(64, 40, "f32"), (130, 66, "f32"), (33, 257, "f32"), (50, 30, "f64")]
    steps = [5, 9, 12, 7]
    grids, inputs = [], []
    for (nx, ny, dtype) in shapes:
        re, im = random_state(rng, nx, ny)
        V = rng.uniform(-0.5, 0.5, (ny, nx))
        g = trotter.Grid(nx, ny, dtype)
        g.set_state(re, im)
        g.set_potential(V, 0.05, 0.025)
        grids.append(g)
        inputs.append((re, im, V, dtype))
    try:
        trotter.evolve_batched(grids, steps, K=3)
        outs = [g.get_state(np.float64) for g in grids]
    finally:
        for g in grids:
            g.close()
    for (re, im, V, dtype), s, (gre, gim) in zip(inputs, steps, outs):
        K = 3 if dtype == "f32" else 0
        (b_re, b_im), _ = run_gpu(re, im, V, 0.05, 0.025, s, dtype=dtype, K=K)
        assert np.array_equal(gre, b_re) and np.array_equal(gim, b_im)


def test_argument_errors_and_launch_count():
    g = trotter.Grid(40, 30, "f32")
    try:
        with pytest.raises(trotter.TrotterError) as e:
            g.evolve(3, K=9)
        assert e.value.status == trotter.TS_ERR_ARG
        with pytest.raises(trotter.TrotterError) as e:
            g.evolve(-1)
        assert e.value.status == trotter.TS_ERR_ARG
        g.set_potential(None, 0.05, 0.025)
        trotter.ts_launch_count(reset=True)
        g.evolve(10, K=4)           # 4 + 4 + 2
        assert trotter.ts_launch_count() == 3
        trotter.ts_launch_count(reset=True)
        g.evolve(10)                # the default depth
        d = trotter.ts_fused_default_depth()
        assert 1 <= d <= 8 and trotter.ts_launch_count() == (10 + d - 1) // d
        trotter.ts_launch_count(reset=True)
        g.evolve(10, K=4)
        g.evolve_plain(2)
        assert trotter.ts_launch_count() == 3 + 18
    finally:
        g.close()
    g64 = trotter.Grid(40, 30, "f64")
    try:
        with pytest.raises(trotter.TrotterError) as e:
            g64.evolve(2, K=2)
        assert e.value.status == trotter.TS_ERR_UNSUPPORTED
    finally:
        g64.close()


def test_zero_potential_identity_step_and_zero_steps():
    rng = np.random.default_rng(1)
    re, im = random_state(rng, 50, 20)
    g = trotter.Grid(50, 20, "f32")
    try:
        g.set_state(re, im)
        g.evolve(0)
        a_re, _ = g.get_state(np.float64)
        assert np.array_equal(a_re, re.astype(np.float32).astype(np.float64))
        g.set_potential(None, 0.0, 0.0)       # identity step
        g.evolve(6, K=3)
        b_re, b_im = g.get_state(np.float64)
        assert np.array_equal(b_re, a_re)
    finally:
        g.close()
