"""Adjoint gradient of the fidelity on the GPU: against the FP64 oracle
adjoint, against central finite differences in FP64, invariants, autograd.

Tolerance: the FP32 adjoint differs from FP64 gradients by the FP32 rounding
of the forward and costate evolutions (~1e-6 relative); the bar is 1e-4
relative L2 over the compared sites.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1208_2407_gb300 import trotter
from paper_1208_2407_gb300 import workloads as wl

from gpu_helpers import ensure_library, random_state

pytestmark = pytest.mark.gpu
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def gpu_adjoint(c, steps, ckpt, K=0):
    g = trotter.Grid(c["nx"], c["ny"], "f32")
    try:
        g.set_state(c["re"], c["im"])
        g.set_potential(c["V"], c["dt"], c["theta"])
        F, grad = trotter.adjoint_fidelity_grad(g, c["target_re"], c["target_im"], steps, ckpt,
                                                K=K)
        grad = grad.double().cpu().numpy()
    finally:
        g.close()
    return F, grad


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# segments of 7 steps (depth 3 and 4 leave ragged launches), one segment of
# 41 steps, and segments of one step (every launch at depth 1)
@pytest.mark.parametrize("K", [1, 2, 3, 4])
@pytest.mark.parametrize("nx,ny,steps,ckpt", [(64, 48, 30, 7), (130, 67, 41, 50), (33, 129, 12, 1)])
def test_adjoint_matches_fp64_oracle_small(nx, ny, steps, ckpt, K):
    rng = np.random.default_rng(nx + ny)
    re, im = random_state(rng, nx, ny)
    tre, tim = random_state(rng, nx, ny)
    # correlate target and initial state so that F is not tiny
    tre, tim = 0.6 * re + 0.4 * tre, 0.6 * im + 0.4 * tim
    s = np.sqrt(np.sum(tre ** 2 + tim ** 2))
    tre, tim = tre / s, tim / s
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    c = dict(nx=nx, ny=ny, re=re, im=im, target_re=tre, target_im=tim, V=V, dt=0.05, theta=0.025)
    F, g = gpu_adjoint(c, steps, ckpt, K)
    og, oF, _ = oracle.adjoint_grad(re, im, tre, tim, V, 0.05, 0.025, steps)
    assert abs(F - oF) < 1e-5 * max(1.0, oF)
    assert rel(g, og) < 1e-4, rel(g, og)
    assert abs(g.sum()) < 1e-4 * np.abs(g).sum()


def _f64_fidelity(c, V, steps, g64):
    g64.set_state(c["re"], c["im"])
    g64.set_potential(V, c["dt"], c["theta"])
    g64.evolve_plain(steps)
    re, im = g64.get_state(np.float64)
    z = np.vdot(c["target_re"] + 1j * c["target_im"], re + 1j * im)
    return abs(z) ** 2


@pytest.fixture(scope="module")
def adj1024():
    """The 1024^2 FP32 workload (500 steps, checkpoints every 50) and its FP64
    references: central differences (h = 1e-3) on 64 sites inside the
    support, evaluated with the FP64 GPU path, and the FP64 oracle adjoint
    over the whole grid."""
    c = wl.adjoint_pair(n=1024, steps=500, seed=0)
    steps = c["steps"]
    rng = np.random.default_rng(123)
    weight = c["re"] ** 2 + c["im"] ** 2 + c["target_re"] ** 2 + c["target_im"] ** 2
    cand = np.flatnonzero(weight.ravel() > 1e-3 * weight.max())
    sites = rng.choice(cand, 64, replace=False)
    h = 1e-3
    g64 = trotter.Grid(c["nx"], c["ny"], "f64")
    fd = np.zeros(len(sites))
    try:
        for i, j in enumerate(sites):
            Vp = c["V"].copy()
            Vm = c["V"].copy()
            Vp.flat[j] += h
            Vm.flat[j] -= h
            fd[i] = (_f64_fidelity(c, Vp, steps, g64) - _f64_fidelity(c, Vm, steps, g64)) / (2 * h)
    finally:
        g64.close()
    og, oF, _ = oracle.adjoint_grad(c["re"], c["im"], c["target_re"], c["target_im"], c["V"],
                                    c["dt"], c["theta"], steps, nthreads=NTHREADS)
    return c, sites, fd, og, oF


@pytest.mark.parametrize("K", [0, 1, 2, 4])
def test_adjoint_1024_500_steps_vs_fd_and_oracle(adj1024, K):
    """The gradient at the default backward depth and at depths 1, 2 and 4
    against both FP64 references (1e-4 relative L2)."""
    c, sites, fd, og, oF = adj1024
    F, g = gpu_adjoint(c, c["steps"], 50, K)
    assert 0.05 < F < 0.95, F
    err_fd = rel(g.ravel()[sites], fd)
    assert err_fd < 1e-4, err_fd
    assert abs(F - oF) < 1e-5
    assert rel(g, og) < 1e-4, rel(g, og)


def test_autograd_function_matches_direct_call():
    import torch
    from paper_1208_2407_gb300.autograd import fidelity
    c = wl.adjoint_pair(n=160, steps=60, seed=4)
    F0, g0 = gpu_adjoint(c, 60, 16)
    V = torch.tensor(c["V"], dtype=torch.float64, requires_grad=True)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    F = fidelity(V, t(c["re"]), t(c["im"]), t(c["target_re"]), t(c["target_im"]), c["dt"],
                 c["theta"], 60, 16)
    F.backward()
    assert abs(F.item() - F0) < 1e-12
    assert np.array_equal(V.grad.numpy().astype(np.float32), g0.astype(np.float32))


def test_backward_depth_out_of_range_is_rejected():
    import torch
    c = wl.adjoint_pair(n=64, steps=4, seed=1)
    g = trotter.Grid(64, 64, "f32")
    try:
        g.set_state(c["re"], c["im"])
        g.set_potential(c["V"], c["dt"], c["theta"])
        nbytes = trotter.ts_adjoint_workspace(g.handle, 4, 2)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        grad = torch.empty((64, 64), dtype=torch.float32, device="cuda")
        tre = torch.tensor(c["target_re"], dtype=torch.float64, device="cuda")
        tim = torch.tensor(c["target_im"], dtype=torch.float64, device="cuda")
        trotter.ts_adjoint_forward(g.handle, trotter._VP(tre.data_ptr()),
                                   trotter._VP(tim.data_ptr()), trotter.TS_F64,
                                   trotter.TS_DEVICE, 4, 2, trotter._VP(ws.data_ptr()), nbytes,
                                   trotter.current_stream_ptr())
        for K in (-1, 5):
            with pytest.raises(trotter.TrotterError) as e:
                trotter.ts_adjoint_backward_depth(g.handle, trotter._VP(ws.data_ptr()), nbytes,
                                                  K, trotter._VP(grad.data_ptr()),
                                                  trotter.current_stream_ptr())
            assert e.value.status == trotter.TS_ERR_ARG
    finally:
        g.close()


def test_backward_without_forward_is_rejected():
    import torch
    g = trotter.Grid(32, 32, "f32")
    try:
        ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
        grad = torch.empty((32, 32), dtype=torch.float32, device="cuda")
        with pytest.raises(trotter.TrotterError) as e:
            trotter.ts_adjoint_backward(g.handle, trotter._VP(ws.data_ptr()), ws.numel(),
                                        trotter._VP(grad.data_ptr()),
                                        trotter.current_stream_ptr())
        assert e.value.status == trotter.TS_ERR_STATE
    finally:
        g.close()
