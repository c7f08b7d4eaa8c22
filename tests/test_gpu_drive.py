"""Time-dependent potential V0 + a(t) V1 on the GPU vs the FP64 oracle's
driven evolution, through the C ABI.

The drive phase exp(-i a_n dt V1) is computed on the device per site and
step; the static table, the sweeps and the rest of the step are those of the
time-independent path.  Tolerances: FP64 1e-12, FP32 1e-5 relative L2.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate

import oracle
from paper_1208_2407_gb300 import trotter
from paper_1208_2407_gb300 import workloads as wl

from gpu_helpers import ensure_library, random_state, rel_l2

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-12
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def drive_inputs(rng, nx, ny, steps, dt=0.05):
    re, im = random_state(rng, nx, ny)
    V0 = rng.uniform(-0.5, 0.5, (ny, nx))
    V1 = rng.uniform(-1.0, 1.0, (ny, nx))
    a = 0.6 * np.sin(1.3 * (np.arange(steps) + 0.5) * dt) + 0.2
    return re, im, V0, V1, a


def run_driven(re, im, V0, V1, a, dt, theta, dtype="f32", path="fused", K=0, chunks=None):
    ny, nx = re.shape
    g = trotter.Grid(nx, ny, dtype)
    try:
        g.set_state(re, im)
        g.set_potential(V0, dt, theta)
        g.set_drive(V1, a)
        for n in (chunks or [len(a)]):
            if path == "fused":
                g.evolve(n, K)
            else:
                g.evolve_plain(n)
        return g.get_state(np.float64)
    finally:
        g.close()


@pytest.mark.parametrize("nx,ny", [(3, 5), (130, 66), (257, 131)])
@pytest.mark.parametrize("path", ["fused", "plain"])
def test_fp64_matches_oracle(nx, ny, path):
    rng = np.random.default_rng(nx + 3 * ny)
    re, im, V0, V1, a = drive_inputs(rng, nx, ny, 9)
    gre, gim = run_driven(re, im, V0, V1, a, 0.05, 0.025, dtype="f64", path=path)
    ore, oim = oracle.evolve_driven(re, im, V0, V1, a, 0.05, 0.025)
    assert rel_l2(gre, gim, ore, oim) < FP64_TOL


@pytest.mark.parametrize("nx,ny", [(1, 64), (257, 131), (240, 242), (113, 1000)])
@pytest.mark.parametrize("K", [0, 1, 2, 3, 4, 8])
def test_fp32_fused_matches_oracle(nx, ny, K):
    rng = np.random.default_rng(nx * 5 + ny)
    re, im, V0, V1, a = drive_inputs(rng, nx, ny, 11)
    gre, gim = run_driven(re, im, V0, V1, a, 0.05, 0.025, K=K)
    ore, oim = oracle.evolve_driven(re, im, V0, V1, a, 0.05, 0.025, nthreads=NTHREADS)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL


def test_fp32_plain_and_large_angles():
    """FP32 plain path; and drive angles beyond the short series' range
    (|a V1 dt| up to 3), where the kernel first reduces the angle by a
    multiple of pi."""
    rng = np.random.default_rng(12)
    re, im, V0, V1, a = drive_inputs(rng, 200, 90, 9)
    gre, gim = run_driven(re, im, V0, V1, a, 0.05, 0.025, path="plain")
    ore, oim = oracle.evolve_driven(re, im, V0, V1, a, 0.05, 0.025)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL
    big = 60.0 * np.cos(0.3 * np.arange(9))
    gre, gim = run_driven(re, im, V0, V1, big, 0.05, 0.025, K=3)
    ore, oim = oracle.evolve_driven(re, im, V0, V1, big, 0.05, 0.025)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL


def test_amplitudes_consumed_across_calls():
    """Steps split over several evolve calls use consecutive amplitudes."""
    rng = np.random.default_rng(13)
    re, im, V0, V1, a = drive_inputs(rng, 150, 77, 17)
    gre, gim = run_driven(re, im, V0, V1, a, 0.05, 0.025, K=3, chunks=[5, 1, 11])
    ore, oim = oracle.evolve_driven(re, im, V0, V1, a, 0.05, 0.025)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL


def test_fp64_amplitudes_consumed_across_calls():
    rng = np.random.default_rng(17)
    re, im, V0, V1, a = drive_inputs(rng, 70, 45, 12)
    gre, gim = run_driven(re, im, V0, V1, a, 0.05, 0.025, dtype="f64", chunks=[1, 6, 5])
    ore, oim = oracle.evolve_driven(re, im, V0, V1, a, 0.05, 0.025)
    assert rel_l2(gre, gim, ore, oim) < FP64_TOL


def test_running_out_of_amplitudes_launches_nothing():
    rng = np.random.default_rng(14)
    re, im, V0, V1, a = drive_inputs(rng, 64, 40, 4)
    g = trotter.Grid(64, 40, "f32")
    try:
        g.set_state(re, im)
        g.set_potential(V0, 0.05, 0.025)
        g.set_drive(V1, a)
        g.evolve(3)
        before = g.get_state(np.float64)
        trotter.ts_launch_count(reset=True)
        with pytest.raises(trotter.TrotterError) as e:
            g.evolve(2)
        assert e.value.status == trotter.TS_ERR_ARG
        assert trotter.ts_launch_count() == 0
        after = g.get_state(np.float64)
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
        g.evolve(1)       # the last amplitude is still there
    finally:
        g.close()


def test_set_potential_and_clear_end_the_drive():
    """After clear_drive, or a new set_potential, steps use V0 alone: the same
    result bit for bit as a grid that never had a drive."""
    rng = np.random.default_rng(15)
    re, im, V0, V1, a = drive_inputs(rng, 96, 64, 6)
    plain = trotter.Grid(96, 64, "f32")
    g = trotter.Grid(96, 64, "f32")
    try:
        plain.set_state(re, im)
        plain.set_potential(V0, 0.05, 0.025)
        plain.evolve(5)
        ref = plain.get_state(np.float64)
        for end in ("clear", "set_potential"):
            g.set_state(re, im)
            g.set_potential(V0, 0.05, 0.025)
            g.set_drive(V1, a)
            if end == "clear":
                g.clear_drive()
            else:
                g.set_potential(V0, 0.05, 0.025)
            g.evolve(5)
            out = g.get_state(np.float64)
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
    finally:
        plain.close()
        g.close()


def test_refusals():
    g = trotter.Grid(64, 64, "f32")
    try:
        g.set_potential(None, 0.05, 0.025)
        with pytest.raises(trotter.TrotterError) as e:
            g.set_drive(None, [0.1, float("nan")])
        assert e.value.status == trotter.TS_ERR_ARG
        g.set_drive(None, [0.1] * 4)
        t = np.zeros((64, 64))
        with pytest.raises(trotter.TrotterError) as e:
            trotter.adjoint_fidelity_grad(g, t, t, 4, 2)
        assert e.value.status == trotter.TS_ERR_UNSUPPORTED
        g.set_potential(None, 0.05, 0.025, order=4)
        with pytest.raises(trotter.TrotterError) as e:
            g.set_drive(None, [0.1])
        assert e.value.status == trotter.TS_ERR_UNSUPPORTED
    finally:
        g.close()


def test_harmonic_2048_with_oscillating_field():
    """The 2048^2 harmonic workload plus a uniform field along x oscillating
    in time (V1 = x - cx, a = F0 cos(w t)), 1000 steps."""
    c = wl.harmonic_2048(seed=2)
    n, dt, steps = c["nx"], c["dt"], c["steps"]
    V1 = (np.arange(n) - n / 2.0)[None, :] * np.ones((n, 1))
    a = 2e-3 * np.cos(0.05 * (np.arange(steps) + 0.5) * dt)
    gre, gim = run_driven(c["re"], c["im"], c["V"], V1, a, dt, c["theta"])
    ore, oim = oracle.evolve_driven(c["re"], c["im"], c["V"], V1, a, dt, c["theta"],
                                    nthreads=NTHREADS)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL


def test_uniform_force_drift_closed_form_on_the_gpu():
    """The exact lattice drift of a packet under a uniform force a(t) along x
    (the Bloch-wave quasi-momentum follows k - int a), FP32 fused path."""
    nx, ny, sigma, T, dt, k0 = 256, 32, 6.0, 8.0, 0.025, 0.6
    x0 = nx / 2.0
    re, im = wl.gaussian_packet(nx, ny, x0, ny / 2.0, sigma, k0, 0.0)
    V1 = (np.arange(nx) - x0)[None, :] * np.ones((ny, 1))
    F0, w = 0.15, 0.7
    n = int(round(T / dt))
    a = F0 * np.cos(w * (np.arange(n) + 0.5) * dt)
    gre, gim = run_driven(re, im, None, V1, a, dt, dt / 2)
    damp = math.exp(-1.0 / (8.0 * sigma * sigma))
    drift, _ = scipy.integrate.quad(
        lambda t: 2 * math.sin(k0 - F0 * math.sin(w * t) / w) * damp, 0.0, T,
        epsabs=1e-13, epsrel=1e-13)
    m = oracle.moments(gre, gim)
    assert abs(m[1] / m[0] - (x0 + drift)) < 2e-3


@pytest.mark.parametrize("scale", [1e-3, 1.0, 10.0, 40.0, 3000.0])
def test_drive_phase_alone_against_closed_form(scale):
    """theta = 0 and V0 = 0 leave only the drive phases: psi_T = psi_0
    exp(-i dt V1 sum_n a_n) per site.  Angles from 1e-5 to ~1e4 rad per step
    cover the series (angles up to 0.8: scale 10 puts warps near that edge)
    and the reduced path; the per-site error bound is about 1e-6 per step
    (series, reduction and the phase update in FP32)."""
    rng = np.random.default_rng(16)
    nx, ny, steps, dt = 160, 40, 8, 0.05
    re, im = random_state(rng, nx, ny)
    V1 = rng.uniform(-1.0, 1.0, (ny, nx)) * scale
    a = rng.uniform(0.5, 1.5, steps)
    for path in ("fused", "plain"):
        gre, gim = run_driven(re, im, None, V1, a, dt, 0.0, path=path)
        expect = (re + 1j * im) * np.exp(-1j * dt * V1 * np.sum(a))
        err = np.abs((gre + 1j * gim) - expect) / np.maximum(np.abs(re + 1j * im), 1e-30)
        # FP32 V1 and a_n dt carry a relative rounding of ~1e-7 into the angle
        bound = 1e-5 + 2.4e-7 * dt * np.abs(V1) * np.sum(a)
        assert np.all(err < bound), (path, float(np.max(err / bound)))
