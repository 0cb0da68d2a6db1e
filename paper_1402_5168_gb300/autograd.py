"""torch.autograd wrappers around the library's forward and adjoint steps.

The n-step evolution u_n = G^n u_0 (G = one application of R(tau L), a real
linear map) is differentiated with the library's own transposed sweeps
(``Operator.apply_adjoint``): for a loss of u_n the gradient with respect to
u_0 is (G^T)^n dL/du_n.  For a loss that reads every intermediate state, such
as a misfit at sensor nodes after each step,

    L = sum_{t=1..n} || S u_t - d_t ||^2,

the gradient is the backward recursion lam_n = 2 S^T r_n,
lam_t = G^T lam_{t+1} + 2 S^T r_t, dL/du_0 = G^T lam_1 with r_t = S u_t - d_t.
The forward pass keeps every k-th state (checkpoints); the backward pass
recomputes the states of one segment at a time from its checkpoint with the
forward step, so memory holds at most n/k + k states.

Only argument marshalling and the recursion's bookkeeping live here: every
step, forward or transposed, runs in the library.
"""
from __future__ import annotations

import torch


class Evolve(torch.autograd.Function):
    """u_n = G^n u_0 with gradient (G^T)^n g."""

    @staticmethod
    def forward(ctx, u0, op, n_steps):
        ctx.op, ctx.n = op, int(n_steps)
        u = u0.detach().clone().contiguous()
        op.apply(u, ctx.n)
        return u

    @staticmethod
    def backward(ctx, g):
        y = g.detach().clone().contiguous()
        ctx.op.apply_adjoint(y, ctx.n)
        return y, None, None


def evolve(op, u0: torch.Tensor, n_steps: int) -> torch.Tensor:
    """Differentiable G^n u0 (u0: CUDA float64 [fields, n_nodes] or [n_rhs, fields, n_nodes])."""
    return Evolve.apply(u0, op, n_steps)


class SensorMisfit(torch.autograd.Function):
    """L = sum_{t=1..n} ||u_t[field, idx] - data[t-1]||^2 with checkpointed adjoint."""

    @staticmethod
    def forward(ctx, u0, op, n_steps, field, idx, data, every):
        n, k = int(n_steps), max(1, int(every))
        u = u0.detach().clone().contiguous()
        ckpt = {0: u.clone()}
        loss = torch.zeros((), dtype=u.dtype, device=u.device)
        for t in range(1, n + 1):
            op.apply(u, 1)
            r = u[..., field, idx] - data[t - 1]
            loss = loss + (r * r).sum()
            if t % k == 0 and t < n:
                ckpt[t] = u.clone()
        ctx.op, ctx.n, ctx.k, ctx.field = op, n, k, field
        ctx.ckpt = ckpt
        ctx.save_for_backward(idx, data)
        return loss

    @staticmethod
    def backward(ctx, gl):
        idx, data = ctx.saved_tensors
        op, n, k, field = ctx.op, ctx.n, ctx.k, ctx.field
        lam = None
        # segments [c, c + k) of steps, last segment first
        starts = sorted(ctx.ckpt.keys(), reverse=True)
        for c in starts:
            end = min(c + k, n)
            u = ctx.ckpt[c].clone()
            states = []
            for _ in range(c + 1, end + 1):
                op.apply(u, 1)
                states.append(u.clone())
            for t in range(end, c, -1):
                ut = states[t - c - 1]
                seed = torch.zeros_like(ut)
                seed[..., field, idx] = 2.0 * (ut[..., field, idx] - data[t - 1])
                lam = seed if lam is None else lam + seed
                lam = lam.contiguous()
                op.apply_adjoint(lam, 1)       # lam <- G^T lam: now the seed for u_{t-1}
        ctx.ckpt = None
        return gl * lam, None, None, None, None, None, None


def sensor_misfit(op, u0: torch.Tensor, n_steps: int, field: int, idx: torch.Tensor, data: torch.Tensor,
                  checkpoint_every: int = 10) -> torch.Tensor:
    """Differentiable sum over steps t = 1..n of ||u_t[field, idx] - data[t-1]||^2.

    idx: LongTensor of node indices (sensors); data: [n_steps, len(idx)] (or with a
    leading rhs axis matching u0).  The backward pass keeps one state per
    ``checkpoint_every`` steps and recomputes the rest."""
    return SensorMisfit.apply(u0, op, n_steps, field, idx, data, checkpoint_every)
