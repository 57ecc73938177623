"""Differentiable reduced AL objective: F(u, pd, qd, s) as a torch.autograd.Function.

Forward: Newton-Raphson power flow at (u, pd, qd) and the value of the scaled
AL functional F (Sec. IV-A); the states x [B, n_x] are kept for the backward
pass.  Backward: each scenario's power flow restarts from its kept state (it
converges at once: the factors at x, no Newton iteration), then the adjoint
gradient (Prop. 1) gives dF/du = d_u F + lambda^T G_u, dF/dpd and dF/dqd
(total derivatives through g and the slack generation) and dF/ds = -phi'.
All arithmetic runs in libopf through the C ABI (opf_objective_batched: the
power flows and adjoint solves of the scenarios spread over a pool of
contexts of the network, each on its own stream); this module only moves
tensors and applies the upstream gradient.

Batched form: u [B, n_u], pd/qd [B, n_bus], s [B, m] -> F [B]; every scenario
is warm-started from the same nominal state.
"""
from __future__ import annotations

import torch

from paper_2110_02590_b300 import OPFContext, objective_batched


class _ReducedObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, pd, qd, s, obj):
        x = torch.empty((u.shape[0], obj.x0.numel()), dtype=torch.float64, device=u.device)
        out = objective_batched(obj.pool, obj.al, u.detach().contiguous(), pd.detach().contiguous(),
                                qd.detach().contiguous(), s.detach().contiguous(), obj.x0, grads=False, x_out=x)
        ctx.save_for_backward(u, pd, qd, s)
        ctx.obj = obj
        ctx.x = x  # the converged states (restart points of the backward pass)
        return out["F"]

    @staticmethod
    def backward(ctx, gF):
        u, pd, qd, s = ctx.saved_tensors
        obj = ctx.obj
        g = objective_batched(obj.pool, obj.al, u.detach().contiguous(), pd.detach().contiguous(),
                              qd.detach().contiguous(), s.detach().contiguous(), ctx.x, grads=True, x_out=ctx.x)
        w = gF.reshape(-1, 1)
        return w * g["grad_u"], w * g["grad_pd"], w * g["grad_qd"], w * g["grad_s"], None


class ReducedObjective(torch.nn.Module):
    """F(u, pd, qd, s) for a batch of scenarios of one network.

    `al` holds sigma_f, rho, sigma_c and y (the multiplier state of the AL
    outer loop); the slack s is an input so that its gradient is available.
    `pool` contexts of the network (each with a stream of its own, driven by a
    host thread of its own) share the scenarios; the default takes one per host
    core up to 16 (on a 16-core host with a 2,000-bus net: 8 contexts 1.76k,
    16 contexts 2.20k, 32 contexts 1.94k scenarios/s, forward and backward).
    opf_ctx is only read for its network and device.
    """

    def __init__(self, opf_ctx, al: dict, pool: int = 0):
        import os
        if pool <= 0:
            pool = max(1, min(16, os.cpu_count() or 1))
        super().__init__()
        self.al = {k: v for k, v in al.items() if k in ("sigma_f", "rho", "sigma_c", "y")}
        self.pool = []
        for _ in range(max(1, int(pool))):
            c = OPFContext(opf_ctx.net, device=opf_ctx.device.index)
            c.use_own_stream()
            self.pool.append(c)
        dev = opf_ctx.device
        self.x0 = torch.cat([torch.zeros(opf_ctx.npv + opf_ctx.npq, dtype=torch.float64, device=dev),
                             torch.ones(opf_ctx.npq, dtype=torch.float64, device=dev)])

    def set_warm_start(self, x0):
        self.x0 = x0.detach().clone()

    def forward(self, u, pd, qd, s):
        squeeze = u.dim() == 1
        if squeeze:
            u, pd, qd, s = u[None], pd[None], qd[None], s[None]
        F = _ReducedObjective.apply(u, pd, qd, s, self)
        return F[0] if squeeze else F
