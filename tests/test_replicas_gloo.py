"""The multi-rank path of bench.py (independent replicas, no data-path
collective) on CPU: two gloo ranks each evolve their own grid; the job's
throughput is the ranks' total work over the slowest rank's time, and each
rank's result equals a single-process run of the same input."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import time

    import bench
    import oracle
    from paper_1208_2407_gb300 import workloads as wl

    dist = bench.Dist(world, rank, "gloo")
    c = wl.harmonic_2048(seed=rank, n=48, steps=20)     # each replica: its own input
    dist.barrier()
    t0 = time.perf_counter()
    re, im = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    if rank == 1:
        time.sleep(0.2)                                 # the slow rank sets the job time
    el = time.perf_counter() - t0
    dist.barrier()
    value = bench.replica_throughput(dist, 48 * 48 * 20, el)
    np.save(os.path.join(outdir, "re%d.npy" % rank), re)
    with open(os.path.join(outdir, "r%d.json" % rank), "w") as f:
        json.dump({"value": value, "el": el}, f)
    dist.close()


def test_two_gloo_replicas(tmp_path):
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / ("r%d.json" % k))) for k in range(2)]
    slowest = max(x["el"] for x in r)
    assert r[1]["el"] > r[0]["el"]
    for x in r:
        assert x["value"] == pytest.approx(2 * 48 * 48 * 20 / slowest, rel=1e-9)
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1208_2407_gb300 import workloads as wl
    for k in range(2):
        c = wl.harmonic_2048(seed=k, n=48, steps=20)
        re, _ = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
        assert np.array_equal(np.load(tmp_path / ("re%d.npy" % k)), re)
