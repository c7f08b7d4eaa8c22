"""Edge cases of the grid geometry on the GPU against the FP64 oracle: the
largest side the library accepts (2^20) along either axis, a single row and
a single column, and 3-D lattices with one slab per axis degenerate."""
import numpy as np
import pytest

import oracle
from paper_1208_2407_gb300 import trotter

from gpu_helpers import ensure_library, random_state, rel_l2

pytestmark = pytest.mark.gpu
MAX_SIDE = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


@pytest.mark.parametrize("nx,ny", [(MAX_SIDE, 3), (3, MAX_SIDE), (MAX_SIDE, 1), (1, MAX_SIDE)])
@pytest.mark.parametrize("K", [0, 4])
def test_longest_side(nx, ny, K):
    rng = np.random.default_rng(nx % 97 + ny % 89 + K)
    re, im = random_state(rng, nx, ny)
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    g = trotter.Grid(nx, ny, "f32")
    try:
        g.set_state(re, im)
        g.set_potential(V, 0.05, 0.025)
        g.evolve(5, K)
        gre, gim = g.get_state(np.float64)
        norm = g.norm()
    finally:
        g.close()
    ore, oim = oracle.evolve(re, im, V, 0.05, 0.025, 5, nthreads=8)
    assert rel_l2(gre, gim, ore, oim) < 1e-5
    assert abs(norm - 1.0) < 1e-6


def test_sides_beyond_the_limit_are_refused():
    for nx, ny in ((MAX_SIDE + 1, 2), (2, MAX_SIDE + 1), (0, 5), (5, 0)):
        with pytest.raises(trotter.TrotterError) as e:
            trotter.ts_grid_layout(nx, ny)
        assert e.value.status == trotter.TS_ERR_ARG


@pytest.mark.parametrize("nx,ny,nz", [(1, 2, 64), (64, 2, 1), (2, 64, 3), (1, 1, 50)])
def test_degenerate_3d(nx, ny, nz):
    rng = np.random.default_rng(nx + ny + nz)
    re = rng.standard_normal((nz, ny, nx))
    im = rng.standard_normal((nz, ny, nx))
    s = np.sqrt(np.sum(re * re + im * im))
    re, im = re / s, im / s
    V = rng.uniform(-0.5, 0.5, (nz, ny, nx))
    g = trotter.Grid(nx, ny, "f32", nz=nz)
    try:
        # nz = 1 is a 2-D grid: its arrays have shape (ny, nx)
        g.set_state(re.reshape(g.shape), im.reshape(g.shape))
        g.set_potential(V.reshape(g.shape), 0.05, 0.025)
        g.evolve(6)
        gre, gim = (a.reshape(re.shape) for a in g.get_state(np.float64))
    finally:
        g.close()
    ore, oim = oracle.evolve3(re, im, V, 0.05, 0.025, 6)
    assert rel_l2(gre, gim, ore, oim) < 1e-5
