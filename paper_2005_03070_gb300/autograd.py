"""Differentiable two-grid solve for the variable-coefficient operator.

x(kappa) solves -div(kappa grad x) + beta x_x = b on the (N+2)^2 node field kappa.  The
forward pass is the two-grid deflated solve (coarse GMRES-DR, prolongation, BiCGStab-Proj);
the backward pass solves A^T lambda = dL/dx with the same two-grid deflation built from
coarse GMRES-DR on A_c^T (left eigenvectors), then contracts lambda and x over the
faces: dL/dkappa_p = -1/2 sum_{faces touching p} (lambda_a - lambda_b)(x_a - x_b) / h^2.
Every numerical step runs in libtg.so; this module only wires it into autograd.

With ``recompute=True`` the forward solution is not kept: the backward pass solves the
forward problem again before the adjoint (memory for time).
"""
from __future__ import annotations

import torch

from . import tg


class _Cfg:
    def __init__(self, N, beta, m, k, nev, rtolev, rtol, ncyc, restart_mvps, precision, recompute):
        self.N, self.beta, self.m, self.k, self.nev, self.rtolev = N, beta, m, k, nev, rtolev
        self.rtol, self.ncyc, self.restart_mvps, self.precision, self.recompute = (
            rtol, ncyc, restart_mvps, precision, recompute)


def _forward_solve(op, b, c):
    xc, defl, _, _ = op.coarse_gmresdr(b, c.m, c.k, nev=c.nev, rtolev=c.rtolev, precision=c.precision)
    x = op.prolong(xc)
    status, st = op.solve(b, x, defl, precision=c.precision, rtol=c.rtol, ncyc=c.ncyc,
                          restart_mvps=c.restart_mvps)
    if status != tg.TG_OK:
        raise tg.TgError(status, "forward two-grid solve")
    return x


class TwoGridSolve(torch.autograd.Function):
    """x = A(kappa)^{-1} b, differentiable with respect to kappa and b (dL/db is the
    adjoint solution lambda)."""

    @staticmethod
    def forward(ctx, kappa: torch.Tensor, b: torch.Tensor, cfg: _Cfg):
        op = tg.Operator("vark2d", cfg.N, (cfg.beta,), kappa=kappa.contiguous())
        x = _forward_solve(op, b, cfg)
        ctx.cfg = cfg
        ctx.op = op
        if cfg.recompute:
            ctx.save_for_backward(kappa, b)
        else:
            ctx.save_for_backward(kappa, b, x)
        return x

    @staticmethod
    def backward(ctx, grad_x: torch.Tensor):
        cfg = ctx.cfg
        op = ctx.op
        if cfg.recompute:
            kappa, b = ctx.saved_tensors
            x = _forward_solve(op, b, cfg)
        else:
            kappa, b, x = ctx.saved_tensors
        g = grad_x.contiguous()
        _, defl_l, _, _ = op.coarse_gmresdr(g, cfg.m, cfg.k, nev=cfg.nev, rtolev=cfg.rtolev, transpose=True,
                                            precision=cfg.precision, want_xc=False)
        lam = torch.zeros_like(g)
        dk = torch.empty_like(kappa)
        status, st = op.adjoint_solve(defl_l, g, lam, x=x, dkappa=dk, rtol=cfg.rtol, ncyc=cfg.ncyc,
                                      restart_mvps=cfg.restart_mvps, precision=cfg.precision)
        if status != tg.TG_OK:
            raise tg.TgError(status, "adjoint two-grid solve")
        # x = A^{-1} b, so dL/db = A^{-T} dL/dx = lambda
        return dk, (lam if ctx.needs_input_grad[1] else None), None


def two_grid_solve(kappa, b, N, beta=1.0, m=40, k=20, nev=None, rtolev=1e-2, rtol=1e-8, ncyc=20,
                   restart_mvps=0, precision="f32_ir", recompute=False):
    """x = A(kappa)^{-1} b with a hand-written adjoint (autograd on kappa)."""
    cfg = _Cfg(N, beta, m, k, k if nev is None else nev, rtolev, rtol, ncyc, restart_mvps, precision, recompute)
    return TwoGridSolve.apply(kappa, b, cfg)
