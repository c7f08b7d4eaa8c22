"""torch.autograd.Function for the fidelity of a Trotter-Suzuki evolution.

``FidelityLoss.apply(V, psi0_re, psi0_im, target_re, target_im, dt, theta,
steps, ckpt_every)`` returns F = |<target|U2(dt)^steps psi0>|^2 as a 0-d
tensor; ``F.backward()`` fills ``V.grad`` with dF/dV from the library's
adjoint kernels (checkpointed backward evolution with the conjugate sweeps).
All computation runs in libtrotter.so; this module only allocates the grid
and the workspace with torch and keeps them between forward and backward.
"""
from __future__ import annotations

import torch

from . import trotter


class FidelityLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, psi0_re, psi0_im, target_re, target_im, dt, theta, steps,
                ckpt_every=50):
        ny, nx = V.shape
        grid = trotter.Grid(nx, ny, "f32")
        st = trotter.current_stream_ptr()
        grid.set_state(psi0_re.contiguous(), psi0_im.contiguous(), stream=st)
        Vd = V.detach().to(device="cuda", dtype=torch.float64).contiguous()
        grid.set_potential(Vd, float(dt), float(theta), stream=st)
        tre = target_re.contiguous()
        tim = target_im.contiguous()
        tp, tdt, tw, _ = trotter._array_ptr(tre, grid.shape)
        ip, _, _, _ = trotter._array_ptr(tim, grid.shape)
        nbytes = trotter.ts_adjoint_workspace(grid.handle, int(steps), int(ckpt_every))
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        F, c = trotter.ts_adjoint_forward(grid.handle, tp, ip, tdt, tw, int(steps),
                                          int(ckpt_every), trotter._VP(ws.data_ptr()), nbytes,
                                          st)
        ctx.grid, ctx.ws, ctx.nbytes = grid, ws, nbytes
        ctx.keep = (tre, tim)
        ctx.V_meta = (V.dtype, V.device)
        ctx.overlap = c
        return torch.tensor(F, dtype=V.dtype, device=V.device)

    @staticmethod
    def backward(ctx, gF):
        grid = ctx.grid
        grad = torch.empty(grid.shape, dtype=torch.float32, device="cuda")
        trotter.ts_adjoint_backward(grid.handle, trotter._VP(ctx.ws.data_ptr()), ctx.nbytes,
                                    trotter._VP(grad.data_ptr()), trotter.current_stream_ptr())
        dtype, device = ctx.V_meta
        gV = gF * grad.to(device=device, dtype=dtype)
        grid.close()
        ctx.grid = ctx.ws = None
        return gV, None, None, None, None, None, None, None, None


def fidelity(V, psi0_re, psi0_im, target_re, target_im, dt, theta, steps, ckpt_every=50):
    return FidelityLoss.apply(V, psi0_re, psi0_im, target_re, target_im, dt, theta, steps,
                              ckpt_every)
