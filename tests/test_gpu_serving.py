"""The continuous-batching server: results equal solo evolutions bit for bit,
admission by the HBM budget, refusal of requests that can never fit,
cancellation, bounded waits and statistics."""
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


def _requests(count, seed, sides=(64, 96, 128, 200, 256), steps=(3, 61)):
    reqs = wl.serving_requests(count=count, mean_gap_s=1e-4, seed=seed, sides=sides,
                               steps_range=steps)
    out = []
    for r in reqs:
        re, im, V = r.inputs()
        out.append((r, re, im, V))
    return out


def _solo(r, re, im, V, K=4):
    g = trotter.Grid(r.nx, r.ny, "f32")
    try:
        g.set_state(re, im)
        g.set_potential(V, r.dt, r.theta)
        g.evolve(r.steps, K)
        return g.get_state(np.float64)
    finally:
        g.close()


def test_results_in_the_mix_equal_solo_runs():
    items = _requests(14, seed=7)
    srv = trotter.Server(hbm_budget_bytes=8 << 30, max_slots=16, K=4, max_epoch_steps=12)
    try:
        tickets = [srv.submit(r.nx, r.ny, r.steps, r.dt, r.theta, V, re, im)
                   for (r, re, im, V) in items]
        for t in tickets:
            assert srv.wait(t, 60000).status == 0
        stats = srv.stats()
        assert stats["completed"] == len(items)
        assert stats["epochs"] >= 2
        for (r, re, im, V), t in zip(items, tickets):
            got = srv.fetch(t, r.ny, r.nx)
            want = _solo(r, re, im, V)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), r
            srv.release(t)
        # and against the FP64 oracle for two of them
        for (r, re, im, V) in items[:2]:
            ore, oim = oracle.evolve(re, im, V, r.dt, r.theta, r.steps)
            w = _solo(r, re, im, V)
            assert rel_l2(w[0], w[1], ore, oim) < 1e-5
        assert srv.stats()["bytes_in_use"] == 0
    finally:
        srv.close()


@pytest.mark.parametrize("K", [1, 2, 3])
def test_mix_equals_solo_at_each_depth(K):
    """The server at depths 1-3 (graph-captured epochs and remainder
    launches at every depth below K): each result equals its solo run at the
    same depth bit for bit."""
    items = _requests(6, seed=20 + K)
    srv = trotter.Server(hbm_budget_bytes=8 << 30, max_slots=8, K=K, max_epoch_steps=10)
    try:
        tickets = [srv.submit(r.nx, r.ny, r.steps, r.dt, r.theta, V, re, im)
                   for (r, re, im, V) in items]
        for t in tickets:
            assert srv.wait(t, 60000).status == 0
        for (r, re, im, V), t in zip(items, tickets):
            got = srv.fetch(t, r.ny, r.nx)
            want = _solo(r, re, im, V, K=K)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), r
            srv.release(t)
    finally:
        srv.close()


def test_admission_respects_the_budget():
    items = _requests(6, seed=3, sides=(256,), steps=(20, 40))
    per = trotter.ts_grid_layout(256, 256, trotter.TS_F32).slab_bytes
    srv = trotter.Server(hbm_budget_bytes=2 * per + 1024, max_slots=8, K=4)
    try:
        tickets = [srv.submit(r.nx, r.ny, r.steps, r.dt, r.theta, V, re, im)
                   for (r, re, im, V) in items]
        for t in tickets:
            assert srv.wait(t, 60000).status == 0
            srv.release(t)        # frees memory for the next admission
        st = srv.stats()
        assert st["completed"] == 6
        assert st["peak_bytes"] <= 2 * per + 1024
    finally:
        srv.close()


def test_a_request_that_can_never_fit_is_refused():
    srv = trotter.Server(hbm_budget_bytes=1 << 20, max_slots=4)
    try:
        re = np.zeros((512, 512))
        with pytest.raises(trotter.TrotterError) as e:
            srv.submit(512, 512, 10, 0.05, 0.025, None, re, re)
        assert e.value.status == trotter.TS_ERR_BUSY
    finally:
        srv.close()


def test_cancel_pending_and_bounded_wait():
    items = _requests(4, seed=11, sides=(512,), steps=(1500, 2000))
    per = trotter.ts_grid_layout(512, 512, trotter.TS_F32).slab_bytes
    srv = trotter.Server(hbm_budget_bytes=per + 1024, max_slots=1, K=4)
    try:
        tickets = [srv.submit(r.nx, r.ny, r.steps, r.dt, r.theta, V, re, im)
                   for (r, re, im, V) in items]
        srv.cancel(tickets[-1])            # still queued behind the budget
        with pytest.raises(trotter.TrotterError) as e:
            srv.wait(tickets[-1], 1000)
        assert e.value.status == trotter.TS_ERR_STATE
        with pytest.raises(trotter.TrotterError) as e:
            srv.wait(tickets[2], 0)        # not done yet: the wait gives up
        assert e.value.status == trotter.TS_ERR_TIMEOUT
        for t in tickets[:-1]:
            assert srv.wait(t, 120000).status == 0
            srv.release(t)
        srv.release(tickets[-1])
        st = srv.stats()
        assert st["completed"] == 3 and st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
        assert st["bytes_in_use"] == 0
    finally:
        srv.close()


def test_zero_steps_returns_the_input_state():
    rng = np.random.default_rng(0)
    re = rng.standard_normal((40, 70))
    im = rng.standard_normal((40, 70))
    srv = trotter.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    try:
        t = srv.submit(70, 40, 0, 0.05, 0.025, None, re, im)
        assert srv.wait(t, 10000).status == 0
        got = srv.fetch(t, 40, 70)
        assert np.array_equal(got[0], re.astype(np.float32).astype(np.float64))
        srv.release(t)
    finally:
        srv.close()
