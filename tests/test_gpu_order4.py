"""Fourth-order Suzuki steps (Sec. 2, Eq. fourthorder) on the GPU vs the FP64
oracle's order-4 evolution, through the C ABI.

U4(dt) = U2(p dt)^2 U2((1-4p) dt) U2(p dt)^2 with p = 1/(4 - 4^(1/3)).  With
K = 0 the GPU applies each U4 step in one launch of the fused kernel (five
substeps, two phase tables in one box); with K >= 1 it runs the p dt substeps
of neighbouring steps as fused launches of depth <= K and each (1-4p) dt
substep as a depth-1 launch.  Tolerances as for the second-order path: FP64
1e-12, FP32 1e-5 relative L2.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1208_2407_gb300 import trotter
from paper_1208_2407_gb300 import workloads as wl

from gpu_helpers import ensure_library, random_state, rel_l2
from test_oracle_pins import cplx, exact_evolve

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-12
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def run4(re, im, V, dt, theta, steps, dtype="f32", path="fused", K=0):
    ny, nx = re.shape
    g = trotter.Grid(nx, ny, dtype)
    try:
        g.set_state(re, im)
        g.set_potential(V, dt, theta, order=4)
        if path == "fused":
            g.evolve(steps, K)
        else:
            g.evolve_plain(steps)
        return g.get_state(np.float64)
    finally:
        g.close()


@pytest.mark.parametrize("nx,ny", [(3, 5), (130, 66), (257, 131)])
@pytest.mark.parametrize("path", ["fused", "plain"])
def test_fp64_matches_oracle(nx, ny, path):
    """FP64 grids: ts_evolve merges the sweeps where substeps meet (angles
    2a and a + b there), ts_evolve_plain runs every substep in full."""
    rng = np.random.default_rng(nx * 31 + ny)
    re, im = random_state(rng, nx, ny)
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    gre, gim = run4(re, im, V, 0.05, 0.025, 7, dtype="f64", path=path)
    ore, oim = oracle.evolve(re, im, V, 0.05, 0.025, 7, order=4)
    assert rel_l2(gre, gim, ore, oim) < FP64_TOL


@pytest.mark.parametrize("nx,ny", [(1, 64), (257, 131), (240, 242), (113, 1000)])
@pytest.mark.parametrize("K", [0, 1, 2, 3, 4, 5, 8])
def test_fp32_fused_matches_oracle(nx, ny, K):
    rng = np.random.default_rng(nx * 7 + ny)
    re, im = random_state(rng, nx, ny)
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    gre, gim = run4(re, im, V, 0.05, 0.025, 9, K=K)
    ore, oim = oracle.evolve(re, im, V, 0.05, 0.025, 9, order=4, nthreads=NTHREADS)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL


def test_fp32_plain_matches_oracle():
    rng = np.random.default_rng(5)
    re, im = random_state(rng, 257, 131)
    V = rng.uniform(-0.5, 0.5, (131, 257))
    gre, gim = run4(re, im, V, 0.05, 0.025, 9, path="plain")
    ore, oim = oracle.evolve(re, im, V, 0.05, 0.025, 9, order=4)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL


def test_free_evolution_and_large_angle():
    """V = None; and theta large enough that the (1-4p) substep angle exceeds
    pi/4, where ts_evolve takes the plain path for every substep."""
    rng = np.random.default_rng(6)
    re, im = random_state(rng, 96, 80)
    gre, gim = run4(re, im, None, 0.05, 0.025, 6)
    ore, oim = oracle.evolve(re, im, None, 0.05, 0.025, 6, order=4)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL
    V = rng.uniform(-0.5, 0.5, (80, 96))
    gre, gim = run4(re, im, V, 2.0, 1.3, 3)
    ore, oim = oracle.evolve(re, im, V, 2.0, 1.3, 3, order=4)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL


def test_harmonic_2048_matches_oracle():
    c = wl.harmonic_2048(seed=0, steps=200)
    gre, gim = run4(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    ore, oim = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"],
                             order=4, nthreads=NTHREADS)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL


def test_fourth_order_convergence_on_the_gpu():
    """The FP64 GPU path against exp(-iHT) from a dense eigendecomposition:
    the error falls ~16x when dt is halved, and is far below second order's."""
    nx, ny, T = 12, 10, 1.6
    rng = np.random.default_rng(11)
    re, im = wl.gaussian_packet(nx, ny, 5.3, 4.6, 1.7, 0.6, -0.4)
    V = 0.3 * np.sin(0.7 * np.arange(nx))[None, :] * np.cos(0.5 * np.arange(ny))[:, None]
    V = V + 0.05 * rng.standard_normal((ny, nx))
    exact = exact_evolve(nx, ny, V, T, cplx(re, im))
    errs = []
    for dt in (0.2, 0.1, 0.05):
        n = int(round(T / dt))
        gre, gim = run4(re, im, V, dt, dt / 2, n, dtype="f64")
        errs.append(np.linalg.norm(cplx(gre, gim) - exact))
    assert 13.0 < errs[1] / errs[2] < 19.0 and errs[0] / errs[1] > 10.0, errs
    g = trotter.Grid(nx, ny, "f64")
    try:
        g.set_state(re, im)
        g.set_potential(V, 0.05, 0.025)
        g.evolve(int(round(T / 0.05)))
        e2re, e2im = g.get_state(np.float64)
    finally:
        g.close()
    assert errs[2] < 0.05 * np.linalg.norm(cplx(e2re, e2im) - exact)


@pytest.mark.parametrize("K,steps,expected", [(0, 5, 5), (4, 5, 11), (4, 1, 3), (3, 5, 15),
                                               (2, 3, 9)])
def test_launch_sequence(K, steps, expected):
    """K = 0: one launch per step (all five substeps fused).  K >= 1: per run
    of a substeps ceil(r / K) launches, plus one per b substep: depth 4 gives
    1 + 2 n launches for n steps, depth 3 gives 3 n."""
    rng = np.random.default_rng(8)
    re, im = random_state(rng, 64, 64)
    g = trotter.Grid(64, 64, "f32")
    try:
        g.set_state(re, im)
        g.set_potential(None, 0.05, 0.025, order=4)
        trotter.ts_launch_count(reset=True)
        g.evolve(steps, K)
        assert trotter.ts_launch_count() == expected
    finally:
        g.close()


def test_batched_and_reset_to_second_order():
    """An order-4 grid inside ts_evolve_batched gives its solo result bit for
    bit, and setting order 2 again on the same grid restores U2 exactly."""
    rng = np.random.default_rng(9)
    re, im = random_state(rng, 200, 150)
    V = rng.uniform(-0.5, 0.5, (150, 200))
    solo = run4(re, im, V, 0.05, 0.025, 4)
    grids = [trotter.Grid(200, 150, "f32") for _ in range(2)]
    try:
        for i, g in enumerate(grids):
            g.set_state(re, im)
            g.set_potential(V, 0.05, 0.025, order=4 if i == 0 else 2)
        trotter.evolve_batched(grids, [4, 4])
        b4 = grids[0].get_state(np.float64)
        b2 = grids[1].get_state(np.float64)
        assert np.array_equal(b4[0], solo[0]) and np.array_equal(b4[1], solo[1])
        grids[0].set_state(re, im)
        grids[0].set_potential(V, 0.05, 0.025, order=2)
        grids[0].evolve(4)
        r2 = grids[0].get_state(np.float64)
        assert np.array_equal(r2[0], b2[0]) and np.array_equal(r2[1], b2[1])
    finally:
        for g in grids:
            g.close()


def test_refusals():
    g = trotter.Grid(64, 64, "f32")
    try:
        with pytest.raises(trotter.TrotterError) as e:
            g.set_potential(None, 0.05, 0.025, order=3)
        assert e.value.status == trotter.TS_ERR_ARG
        g.set_potential(None, 0.05, 0.025, order=4)
        t = np.zeros((64, 64))
        with pytest.raises(trotter.TrotterError) as e:
            trotter.adjoint_fidelity_grad(g, t, t, 4, 2)
        assert e.value.status == trotter.TS_ERR_UNSUPPORTED
    finally:
        g.close()
