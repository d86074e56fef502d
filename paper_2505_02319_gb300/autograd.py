"""Differentiation of the linear response drho(dV) = E^-1 chi0 dV.

Forward: b = chi0 dV (all Sternheimer equations solved tightly), then
E drho = b by Algorithm 1.  Backward, for an upstream gradient g = dL/d drho:
E^T lambda = g by the same solver on the transpose E^T = 1 - K chi0 (chi0 and K
are symmetric, Sec. 2.2), then dL/d dV = chi0^T lambda = chi0 lambda.  The
backward pass recomputes everything it needs (no orbital responses dphi_n are
kept from the forward pass), so its memory is that of one more solve.
Both solves run in the library; this module only wires them into autograd.
A batch dV of shape (nrhs, Ng) (several perturbations, e.g. the 32 of the
differentiated batch) is solved in lockstep: one ikr_solve_response and one
ikr_solve_response_adjoint over all rows, each row scaled to unit norm so that
tau_rel is relative per row.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ikr


def _chi0(ctx: ikr.Context, v: torch.Tensor, rel_tol: float, precision: int) -> torch.Tensor:
    """chi0 v with every Sternheimer residual below rel_tol ||v|| (linearity of chi0)."""
    n = float(torch.linalg.norm(v))
    if n == 0.0:
        return torch.zeros_like(v)
    nsys = int(ctx.groundstate_nsys)
    out, _ = ctx.apply_chi0((v / n).contiguous(), tol=np.full(nsys, rel_tol), precision=precision)
    return out * n


def _chi0_rows(ctx, v, rel_tol, precision):
    if v.dim() == 1:
        return _chi0(ctx, v, rel_tol, precision)
    return torch.stack([_chi0(ctx, row, rel_tol, precision) for row in v])


def _solve(ctx, rhs, adjoint, tau_rel, opts):
    """E x = rhs (or E^T x = rhs) with every row scaled to unit norm: the rows
    of a batch advance in lockstep in one library call."""
    rows = rhs.reshape(-1, rhs.shape[-1])
    n = torch.linalg.norm(rows, dim=1, keepdim=True)
    live = n.squeeze(1) > 0
    x = torch.zeros_like(rows)
    rep = None
    if bool(live.any()):
        fn = ctx.solve_response_adjoint if adjoint else ctx.solve_response
        sub = (rows[live] / n[live]).contiguous()
        xs, rep = fn(sub if rhs.dim() > 1 else sub[0], tau=tau_rel, **opts)
        x[live] = xs.reshape(-1, rows.shape[1]) * n[live]
    return x.reshape(rhs.shape), rep


class DysonResponse(torch.autograd.Function):
    """drho = E^-1 chi0 dV on a context with ground state; differentiable in dV
    ((Ng,) or a batch (nrhs, Ng))."""

    @staticmethod
    def forward(fctx, dV, ctx, tau_rel=1e-10, chi0_rel=1e-12, opts=None):
        opts = dict(opts or {})
        prec = opts.get("precision", ikr.FP64)
        prec = {"fp64": ikr.FP64, "mixed": ikr.MIXED}.get(prec, prec)
        b = _chi0_rows(ctx, dV.detach(), chi0_rel, ikr.FP64)
        x, rep = _solve(ctx, b, False, tau_rel, opts)
        fctx.ctx, fctx.tau_rel, fctx.chi0_rel, fctx.opts, fctx.prec = ctx, tau_rel, chi0_rel, opts, prec
        fctx.report = rep
        return x

    @staticmethod
    def backward(fctx, g):
        lam, _ = _solve(fctx.ctx, g.detach().contiguous(), True, fctx.tau_rel, fctx.opts)
        grad = _chi0_rows(fctx.ctx, lam, fctx.chi0_rel, ikr.FP64)
        return grad, None, None, None, None


def dyson_response(dV, ctx, tau_rel=1e-10, chi0_rel=1e-12, **opts):
    """Differentiable drho = E^-1 chi0 dV (see DysonResponse)."""
    return DysonResponse.apply(dV, ctx, tau_rel, chi0_rel, opts)
