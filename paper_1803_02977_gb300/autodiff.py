"""torch.autograd.Function over nsteps time steps, differentiated by the
library's hand-written adjoint (lem_adjoint): gradients of a scalar loss of
the final elevations with respect to the per-cell uplift field U, the
erodibility K and the initial elevations h0.

Forward runs lem_step on a copy of h0 (FP64).  Backward recomputes the
forward from checkpoints kept every `ckpt_every` steps and sweeps each step's
frozen receiver graph donors-first; nothing of the forward is stored between
the two passes except h0, U and K.
"""
from __future__ import annotations

import torch

from . import lem


class LemRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h0, U, K, nsteps, ckpt_every, dx, m, dt):
        if h0.dtype != torch.float64 or U.dtype != torch.float64:
            raise ValueError("LemRun differentiates FP64 runs")
        Kv = float(K)
        h = h0.detach().clone().contiguous()
        mdl = lem.Model(h, dx=dx, K=Kv, m=m, U=0.0, dt=dt)
        mdl.set_uplift_field(U.detach())
        mdl.step(nsteps)
        mdl.sync()
        mdl.close()
        ctx.save_for_backward(h0.detach().contiguous(), U.detach().contiguous())
        ctx.params = (Kv, int(nsteps), int(ckpt_every), float(dx), float(m), float(dt))
        return h

    @staticmethod
    def backward(ctx, grad_hT):
        h0, U = ctx.saved_tensors
        Kv, nsteps, ckpt, dx, m, dt = ctx.params
        mdl = lem.Model(h0.clone(), dx=dx, K=Kv, m=m, U=0.0, dt=dt)
        mdl.set_uplift_field(U)
        dU = torch.empty_like(U)
        lam0 = torch.empty_like(h0)
        dK = lem.lem_adjoint(mdl.ctx, h0, grad_hT.contiguous(), nsteps, ckpt, dU, lam0)
        mdl.close()
        gK = torch.tensor(dK, dtype=torch.float64, device=h0.device)
        return lam0, dU, gK, None, None, None, None, None


def run(h0, U, K, nsteps, ckpt_every=10, dx=100.0, m=0.5, dt=1000.0):
    """Differentiable nsteps-step run: returns h_T (FP64, same shape as h0)."""
    return LemRun.apply(h0, U, K, nsteps, ckpt_every, dx, m, dt)
