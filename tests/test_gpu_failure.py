"""The failure path of the bounded device waits, made to run on the GPU
without a fault: a warp waits on an mbarrier that nothing completes, the
wait gives up after a short limit and sets the grid's error word, and the
next syncing call reports TS_ERR_TIMEOUT.  The context stays usable: the
state is untouched, the error word is cleared, and evolution afterwards
matches the FP64 oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_1208_2407_gb300 import trotter

from gpu_helpers import ensure_library, random_state, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def test_bounded_wait_gives_up_and_is_reported():
    import torch
    rng = np.random.default_rng(41)
    re, im = random_state(rng, 150, 90)
    V = rng.uniform(-0.5, 0.5, (90, 150))
    g = trotter.Grid(150, 90, "f32")
    try:
        g.set_state(re, im)
        g.set_potential(V, 0.05, 0.025)
        g.evolve(5)
        before = g.get_state(np.float64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        trotter.ts_check_wait_timeout(g.handle, 20_000_000, trotter.current_stream_ptr())
        with pytest.raises(trotter.TrotterError) as e:
            g.get_state(np.float64)
        waited = time.perf_counter() - t0
        assert e.value.status == trotter.TS_ERR_TIMEOUT
        assert 0.015 < waited < 5.0, waited          # the 20 ms limit ran out, then it returned
        after = g.get_state(np.float64)              # word cleared; state untouched
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
        g.evolve(6)                                  # the context still evolves correctly
        gre, gim = g.get_state(np.float64)
        assert g.norm() == pytest.approx(1.0, abs=1e-5)
    finally:
        g.close()
    ore, oim = oracle.evolve(re, im, V, 0.05, 0.025, 11)
    assert rel_l2(gre, gim, ore, oim) < 1e-5


def test_limit_out_of_range_is_refused():
    g = trotter.Grid(32, 32, "f32")
    try:
        for bad in (0, 999, 2_000_000_001):
            with pytest.raises(trotter.TrotterError) as e:
                trotter.ts_check_wait_timeout(g.handle, bad, trotter.current_stream_ptr())
            assert e.value.status == trotter.TS_ERR_ARG
        trotter.ts_launch_count(reset=True)
        g.norm()
        assert trotter.ts_launch_count() == 2         # nothing else was queued
    finally:
        g.close()
