"""Grids driven from several host threads at once (one grid per thread, each
on its own stream): results equal the same evolutions run one after another,
bit for bit.  The first launch of a depth sets up that kernel's occupancy
once; here several threads race to it."""
import threading

import numpy as np
import pytest

from paper_1208_2407_gb300 import trotter

from gpu_helpers import ensure_library, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def _job(seed, nx, ny, steps, K, order):
    rng = np.random.default_rng(seed)
    re, im = random_state(rng, nx, ny)
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    return re, im, V, steps, K, order


def _run(job, stream=None):
    import torch
    re, im, V, steps, K, order = job
    ny, nx = re.shape
    g = trotter.Grid(nx, ny, "f32")
    try:
        st = trotter._VP(stream.cuda_stream) if stream is not None else None
        g.set_state(re, im, stream=st)
        g.set_potential(V, 0.05, 0.025, stream=st, order=order)
        g.evolve(steps, K, stream=st)
        return g.get_state(np.float64, stream=st)
    finally:
        if stream is not None:
            stream.synchronize()
        g.close()


def test_concurrent_threads_match_sequential():
    import torch
    # depths 5-7 (and the fourth-order kernel) are launched here first
    jobs = [_job(100 + i, 300 + 37 * i, 200 + 11 * i, 13 + i, K, order)
            for i, (K, order) in enumerate([(5, 2), (6, 2), (7, 2), (0, 4), (5, 2), (7, 2)])]
    results = [None] * len(jobs)
    errors = []

    def worker(i):
        try:
            s = torch.cuda.Stream()
            results[i] = _run(jobs[i], s)
        except Exception as e:       # reported below
            errors.append(e)

    ths = [threading.Thread(target=worker, args=(i,)) for i in range(len(jobs))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errors, errors
    for i, job in enumerate(jobs):
        want = _run(job)
        assert np.array_equal(results[i][0], want[0]) and np.array_equal(results[i][1], want[1]), i
