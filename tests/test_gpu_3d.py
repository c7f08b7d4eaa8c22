"""Three-dimensional lattices on the GPU vs the FP64 oracle's 3-D step,
through the C ABI.  FP32 grids run one fused launch per step (a CTA per
block of 16 slabs, two per warp, 12 of them stored, trading rows for the odd
Z sweeps);
FP64 and ts_evolve_plain run one kernel per sweep.  Tolerances: FP64 1e-12,
FP32 1e-5 relative L2.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1208_2407_gb300 import trotter
from paper_1208_2407_gb300 import workloads as wl

from gpu_helpers import ensure_library, rel_l2

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-12
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def rand3(rng, nx, ny, nz):
    re = rng.standard_normal((nz, ny, nx))
    im = rng.standard_normal((nz, ny, nx))
    s = np.sqrt(np.sum(re * re + im * im))
    return re / s, im / s


def run3(re, im, V, dt, theta, steps, dtype="f32", path="fused"):
    nz, ny, nx = re.shape
    g = trotter.Grid(nx, ny, dtype, nz=nz)
    try:
        g.set_state(re, im)
        g.set_potential(V, dt, theta)
        if path == "fused":
            g.evolve(steps)
        else:
            g.evolve_plain(steps)
        return g.get_state(np.float64), g.observe()
    finally:
        g.close()


@pytest.mark.parametrize("nx,ny,nz", [(3, 5, 2), (17, 6, 9), (40, 33, 12)])
@pytest.mark.parametrize("path", ["fused", "plain"])
def test_fp64_matches_oracle(nx, ny, nz, path):
    """FP64: ts_evolve merges the sweeps where steps meet (9 n + 3 sweeps in
    lifting form); ts_evolve_plain runs all 12 per step."""
    rng = np.random.default_rng(nx + 7 * ny + 31 * nz)
    re, im = rand3(rng, nx, ny, nz)
    V = rng.uniform(-0.5, 0.5, (nz, ny, nx))
    (gre, gim), _ = run3(re, im, V, 0.05, 0.025, 6, dtype="f64", path=path)
    ore, oim = oracle.evolve3(re, im, V, 0.05, 0.025, 6)
    assert rel_l2(gre, gim, ore, oim) < FP64_TOL


def test_fp64_launch_count():
    rng = np.random.default_rng(23)
    re, im = rand3(rng, 64, 16, 12)
    g = trotter.Grid(64, 16, "f64", nz=12)
    try:
        g.set_state(re, im)
        g.set_potential(None, 0.05, 0.025)
        trotter.ts_launch_count(reset=True)
        g.evolve(5)
        assert trotter.ts_launch_count() == 10 * 5 + 3     # 9 n + 3 sweeps, n phases
        trotter.ts_launch_count(reset=True)
        g.evolve_plain(5)
        assert trotter.ts_launch_count() == 13 * 5
    finally:
        g.close()


# nz across the z-blocks of 20 stored slabs (19, 20, 21, 40, 41, 150) and of
# 12 (11, 12, 13, 24, 25), odd and even ny (1 and 2 included), strips of 120
# columns with a ragged last one (121, 241, 257)
@pytest.mark.parametrize("nx,ny,nz", [(96, 64, 40), (130, 66, 17), (33, 2, 9), (257, 130, 5),
                                      (64, 32, 150), (20, 8, 2), (5, 11, 7), (121, 7, 13),
                                      (40, 9, 3), (3, 1, 25), (241, 5, 24), (17, 12, 11),
                                      (16, 3, 12), (9, 4, 19), (48, 10, 20), (35, 6, 21),
                                      (24, 5, 41)])
@pytest.mark.parametrize("path", ["fused", "plain"])
def test_fp32_matches_oracle(nx, ny, nz, path):
    """Every side length and block edge of the fused 3-D step against the
    oracle, and the plain path on the same lattices."""
    rng = np.random.default_rng(nx * 3 + ny * 5 + nz)
    re, im = rand3(rng, nx, ny, nz)
    V = rng.uniform(-0.5, 0.5, (nz, ny, nx))
    (gre, gim), _ = run3(re, im, V, 0.05, 0.025, 7, path=path)
    ore, oim = oracle.evolve3(re, im, V, 0.05, 0.025, 7, nthreads=NTHREADS)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL


def test_observables_3d():
    rng = np.random.default_rng(21)
    re, im = rand3(rng, 48, 20, 14)
    V = rng.uniform(-0.5, 0.5, (14, 20, 48))
    (gre, gim), obs = run3(re, im, V, 0.05, 0.025, 5, dtype="f64")
    m = oracle.moments3(gre, gim)
    kin, pot = oracle.energy3(gre, gim, V)
    assert abs(obs["norm"] - m[0]) < 1e-13
    for key, q in (("x", 1), ("y", 2), ("z", 3), ("x2", 4), ("y2", 5), ("z2", 6)):
        assert abs(obs[key] - m[q] / m[0]) < 1e-10 * max(1.0, abs(m[q] / m[0])), key
    assert abs(obs["e_kin"] - kin) < 1e-12 and abs(obs["e_pot"] - pot) < 1e-12


def test_launch_sequence_and_refusals():
    rng = np.random.default_rng(22)
    re, im = rand3(rng, 64, 16, 12)
    g = trotter.Grid(64, 16, "f32", nz=12)
    try:
        g.set_state(re, im)
        g.set_potential(None, 0.05, 0.025)
        trotter.ts_launch_count(reset=True)
        g.evolve(5)
        assert trotter.ts_launch_count() == 5          # one fused launch per step
        with pytest.raises(trotter.TrotterError) as e:
            g.set_potential(None, 0.05, 0.025, order=4)
        assert e.value.status == trotter.TS_ERR_UNSUPPORTED
        g.set_potential(None, 0.05, 0.025)
        with pytest.raises(trotter.TrotterError) as e:
            g.set_drive(None, [0.1])
        assert e.value.status == trotter.TS_ERR_UNSUPPORTED
    finally:
        g.close()
    with pytest.raises(trotter.TrotterError) as e:
        trotter.ts_grid_layout3(64, 1 << 16, 1 << 15)
    assert e.value.status == trotter.TS_ERR_ARG


def test_harmonic_128_cubed():
    c = wl.harmonic_3d(n=128, steps=200)
    (gre, gim), obs = run3(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    ore, oim = oracle.evolve3(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"],
                              nthreads=NTHREADS)
    assert rel_l2(gre, gim, ore, oim) < FP32_TOL
    assert abs(obs["norm"] - 1.0) < 1e-6
