"""ts_norm_noalloc: the norm for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: their device memory is already fully
reserved by another allocator (a framework's caching pool, a serving process
with a fixed HBM budget), or they run a loop that must not take the
synchronising path of a fresh allocation.  ts_norm_noalloc gives them the
norm reduction with its scratch in a fixed array inside the library, so the
call allocates nothing.  These tests check it through the C ABI against the
regular ts_norm and against the FP64 oracle's sum of the same (rounded)
state, on two calls in a row (different grid sizes, so the second call starts
with the first call's leftovers in the shared scratch); that a call changes
neither the device's free memory nor torch's allocated bytes; and that
arguments it cannot serve safely are refused before any kernel runs.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_1208_2407_gb300 import trotter

from gpu_helpers import ensure_library, random_state

pytestmark = pytest.mark.gpu


def _norm_both(nx, ny, dtype, seed):
    import torch
    rng = np.random.default_rng(seed)
    re, im = random_state(rng, nx, ny)
    re, im = 3.0 * re, 0.5 * im          # a norm away from 1
    g = trotter.Grid(nx, ny, dtype)
    try:
        g.set_state(re, im)
        want = g.norm()
        re_p, im_p, pitch = g.state_planes()
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        code = trotter.TS_F64 if dtype == "f64" else trotter.TS_F32
        trotter.ts_norm_noalloc(trotter._VP(re_p), trotter._VP(im_p), code, nx, ny, pitch,
                                trotter._VP(out.data_ptr()), trotter.current_stream_ptr())
        torch.cuda.synchronize()
        got = float(out.item())
        # the state as the grid holds it (FP32 grids: rounded once), exactly in FP64
        sre, sim = g.get_state(np.float64)
    finally:
        g.close()
    return got, want, oracle.norm(sre, sim)


def test_norm_noalloc_matches_ts_norm_on_two_calls_in_a_row():
    ensure_library()
    assert trotter.ts_norm_noalloc_scratch_bytes() == 1024 * 7 * 8
    got1, want1, ora1 = _norm_both(2048, 1500, "f32", seed=1)   # many reduction blocks
    got2, want2, ora2 = _norm_both(70, 33, "f64", seed=2)       # few blocks, stale scratch above
    assert got1 == pytest.approx(want1, rel=1e-14)
    assert got2 == pytest.approx(want2, rel=1e-14)
    # both sums are compensated: against the oracle's Neumaier sum to 1e-14
    assert got1 == pytest.approx(ora1, rel=1e-14)
    assert got2 == pytest.approx(ora2, rel=1e-14)


def test_norm_noalloc_allocates_nothing():
    ensure_library()
    import torch
    nx, ny = 1000, 700
    re, im = random_state(np.random.default_rng(3), nx, ny)
    g = trotter.Grid(nx, ny, "f32")
    try:
        g.set_state(re, im)
        re_p, im_p, pitch = g.state_planes()
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        args = (trotter._VP(re_p), trotter._VP(im_p), trotter.TS_F32, nx, ny, pitch,
                trotter._VP(out.data_ptr()), trotter.current_stream_ptr())
        trotter.ts_norm_noalloc(*args)       # the first call on a device looks up the scratch
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        trotter.ts_launch_count(True)
        trotter.ts_norm_noalloc(*args)
        launches = trotter.ts_launch_count()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        alloc1 = torch.cuda.memory_allocated()
    finally:
        g.close()
    assert launches == 2                     # the block pass and the final pass
    assert free1 == free0
    assert alloc1 == alloc0


def test_norm_noalloc_rejects_sizes_beyond_its_limits():
    ensure_library()
    import torch
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(64, dtype=torch.float32, device="cuda")
    p = trotter._VP(dummy.data_ptr())
    with pytest.raises(trotter.TrotterError) as e:
        trotter.ts_norm_noalloc(p, p, trotter.TS_F32, (1 << 20) + 1, 1, (1 << 20) + 32,
                                trotter._VP(out.data_ptr()), trotter.current_stream_ptr())
    assert e.value.status == trotter.TS_ERR_ARG and "2^20" in str(e.value)
    with pytest.raises(trotter.TrotterError) as e:
        trotter.ts_norm_noalloc(p, p, trotter.TS_F32, 64, 1, 32,
                                trotter._VP(out.data_ptr()), trotter.current_stream_ptr())
    assert e.value.status == trotter.TS_ERR_ARG
    # FP32 rows of 70 floats: the 16-byte loads of odd rows would be misaligned
    with pytest.raises(trotter.TrotterError) as e:
        trotter.ts_norm_noalloc(p, p, trotter.TS_F32, 70, 1, 70,
                                trotter._VP(out.data_ptr()), trotter.current_stream_ptr())
    assert e.value.status == trotter.TS_ERR_ARG and "multiple of 4" in str(e.value)
    # planes 4 bytes off a 16-byte boundary (FP32) or off an 8-byte one (FP64)
    p4 = trotter._VP(dummy.data_ptr() + 4)
    with pytest.raises(trotter.TrotterError) as e:
        trotter.ts_norm_noalloc(p4, p, trotter.TS_F32, 8, 1, 8,
                                trotter._VP(out.data_ptr()), trotter.current_stream_ptr())
    assert e.value.status == trotter.TS_ERR_ARG and "aligned" in str(e.value)
    with pytest.raises(trotter.TrotterError) as e:
        trotter.ts_norm_noalloc(p, p4, trotter.TS_F64, 4, 1, 4,
                                trotter._VP(out.data_ptr()), trotter.current_stream_ptr())
    assert e.value.status == trotter.TS_ERR_ARG and "aligned" in str(e.value)
