"""Differentiable reduced AL objective: F(u, pd, qd, s) as a torch.autograd.Function.

Forward: Newton-Raphson power flow at (u, pd, qd) and the value of the scaled
AL functional F (Sec. IV-A).  Backward: the power flow is re-solved from the
saved inputs (the state x is recomputed, not stored across the batch), then the
adjoint gradient (Prop. 1) gives dF/du = d_u F + lambda^T G_u, dF/dpd and
dF/dqd (total derivatives through g and the slack generation) and dF/ds = -phi'.
All arithmetic runs in libopf through the C ABI (opf_powerflow,
opf_reduced_gradient); this module only moves tensors.

Batched form: u [B, n_u], pd/qd [B, n_bus], s [B, m] -> F [B]; the scenarios are
solved one after another on one context, each warm-started from the context's
nominal state.
"""
from __future__ import annotations

import torch


class _ReducedObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, pd, qd, s, opf, al, x0):
        B = u.shape[0]
        F = torch.empty(B, dtype=torch.float64, device=u.device)
        for b in range(B):
            opf.powerflow(u[b].contiguous(), pd=pd[b].contiguous(), qd=qd[b].contiguous(), x0=x0)
            F[b] = opf.reduced_gradient(dict(al, s=s[b].contiguous()))["F"][0]
        ctx.save_for_backward(u, pd, qd, s)
        ctx.opf, ctx.al, ctx.x0 = opf, al, x0
        return F

    @staticmethod
    def backward(ctx, gF):
        u, pd, qd, s = ctx.saved_tensors
        opf, al, x0 = ctx.opf, ctx.al, ctx.x0
        gu, gpd, gqd, gs = (torch.empty_like(t) for t in (u, pd, qd, s))
        for b in range(u.shape[0]):
            opf.powerflow(u[b].contiguous(), pd=pd[b].contiguous(), qd=qd[b].contiguous(), x0=x0)
            g = opf.reduced_gradient(dict(al, s=s[b].contiguous()))
            gu[b] = gF[b] * g["grad_u"]
            gpd[b] = gF[b] * g["grad_pd"]
            gqd[b] = gF[b] * g["grad_qd"]
            gs[b] = gF[b] * g["grad_s"]
        return gu, gpd, gqd, gs, None, None, None


class ReducedObjective(torch.nn.Module):
    """F(u, pd, qd, s) for a batch of scenarios of one network.

    `al` holds sigma_f, rho, sigma_c and y (the multiplier state of the AL
    outer loop); the slack s is an input so that its gradient is available.
    """

    def __init__(self, opf_ctx, al: dict):
        super().__init__()
        self.opf = opf_ctx
        self.al = {k: v for k, v in al.items() if k in ("sigma_f", "rho", "sigma_c", "y")}
        u0 = torch.zeros(opf_ctx.nu, dtype=torch.float64, device=opf_ctx.device)
        self.x0 = torch.cat([torch.zeros(opf_ctx.npv + opf_ctx.npq, dtype=torch.float64, device=opf_ctx.device),
                             torch.ones(opf_ctx.npq, dtype=torch.float64, device=opf_ctx.device)])
        del u0

    def set_warm_start(self, x0):
        self.x0 = x0.detach().clone()

    def forward(self, u, pd, qd, s):
        squeeze = u.dim() == 1
        if squeeze:
            u, pd, qd, s = u[None], pd[None], qd[None], s[None]
        F = _ReducedObjective.apply(u, pd, qd, s, self.opf, self.al, self.x0)
        return F[0] if squeeze else F
