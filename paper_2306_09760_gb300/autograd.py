"""Gradients through TVD-RK3 rollouts of the WCNS-FE scheme.

`rollout(u0, solver, dt, nsteps)` advances `u0` (a [nvar, ny, nx] CUDA tensor) by
`nsteps` fixed-size TVD-RK3 steps with the library and is differentiable: the backward
pass calls the hand-written adjoint once per step, from the last step to the first.
With `stages=True` (the default) the forward keeps RK-stage checkpoints -- the state
and the two intermediate stage states of every step, written by `wcns_step_stages` --
and the backward runs `wcns_adjoint_step_stages` on them; with `stages=False` it keeps
one checkpoint of the state per step (a third of the memory) and `wcns_adjoint_step`
recomputes the two intermediate stages from it.  Both give the same gradient bit for
bit.  All arithmetic of the forward and reverse sweeps runs in the library's kernels;
this module only orders streams and copies between the caller's [nvar, ny, nx] view and
the library's padded rows.
"""
from __future__ import annotations

import torch

from . import wcns


class WcnsRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0: torch.Tensor, solver: "wcns.Solver", dt: float, nsteps: int, stages: bool = True):
        if not u0.is_cuda:
            raise ValueError("u0 must be a CUDA tensor")
        g = solver.grid
        cur = torch.cuda.current_stream()
        st = solver.stream if solver.stream is not None else cur
        st.wait_stream(cur)
        with torch.cuda.stream(st):
            u = solver.alloc()
            u[:, :, : g.nx].copy_(u0.detach().to(solver.tdtype))
            ckpts = []
            for _ in range(int(nsteps)):
                un = u.clone()
                if stages:
                    u1, u2 = solver.alloc(), solver.alloc()
                    wcns.wcns_step_stages(solver.ctx, u, float(dt), u1, u2)
                    ckpts.append((un, u1, u2))
                else:
                    wcns.wcns_step(solver.ctx, u, float(dt), 1, 0.0)
                    ckpts.append((un,))
            out = u[:, :, : g.nx].clone()
        cur.wait_stream(st)
        ctx.solver = solver
        ctx.dt = float(dt)
        ctx.ckpts = ckpts
        ctx.in_dtype = u0.dtype
        return out.to(u0.dtype)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        solver = ctx.solver
        g = solver.grid
        cur = torch.cuda.current_stream()
        st = solver.stream if solver.stream is not None else cur
        st.wait_stream(cur)
        with torch.cuda.stream(st):
            lam = solver.alloc()
            lam[:, :, : g.nx].copy_(grad_out.to(solver.tdtype))
            for ck in reversed(ctx.ckpts):
                if len(ck) == 3:
                    wcns.wcns_adjoint_step_stages(solver.ctx, ck[0], ck[1], ck[2], ctx.dt, lam, lam)
                else:
                    wcns.wcns_adjoint_step(solver.ctx, ck[0], ctx.dt, lam, lam)
            grad = lam[:, :, : g.nx].clone()
        cur.wait_stream(st)
        ctx.ckpts = None
        return grad.to(ctx.in_dtype), None, None, None, None


def rollout(u0: torch.Tensor, solver: "wcns.Solver", dt: float, nsteps: int, stages: bool = True) -> torch.Tensor:
    return WcnsRollout.apply(u0, solver, dt, nsteps, stages)
