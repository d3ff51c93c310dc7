"""A QCP solution as a differentiable torch function of the problem data.

``qcp_layer(plan, P_vals, A_vals, q, b)`` returns the solution (x, y, s) the
plan was built at, as tensors that depend on the data: reverse mode
(``loss.backward()``) runs the library's VJP (Sec. 3.2), forward mode
(``torch.func.jvp`` / ``torch.autograd.forward_ad``) its JVP (Sec. 3.1).
Nothing here computes a derivative itself: both directions go through the C
ABI (qcp_derivative_vjp / qcp_derivative_jvp), batch plans included, so a
layer over B problems takes concatenated data and gives concatenated
solutions.

Gradients are with respect to the STORED values.  P is stored as its upper
triangle; a stored off-diagonal value p_ij stands for both P_ij and P_ji, so
its gradient is twice the entry of the symmetric adjoint the VJP returns
(diagonal entries once).  The derivative is taken at the plan's point: the
tensors passed in must hold the data the plan was built from (their values
are not read again).
"""
from __future__ import annotations

import torch

from . import api


def _offdiag_weight(plan: api.Plan) -> torch.Tensor:
    """2 for stored off-diagonal P entries, 1 on the diagonal (concatenated
    over the plan's problems)."""
    parts = []
    for pt in plan.problems:
        rows = torch.repeat_interleave(torch.arange(pt.n, device=pt.P_indptr.device),
                                       (pt.P_indptr[1:] - pt.P_indptr[:-1]))
        parts.append(torch.where(rows == pt.P_indices.to(torch.int64), 1.0, 2.0))
    return torch.cat(parts).to(plan.dtype)


class QCPSolution(torch.autograd.Function):
    """(P_vals, A_vals, q, b) -> (x, y, s) at the plan's point."""

    @staticmethod
    def forward(plan, opts, P_vals, A_vals, q, b):
        sol = [torch.cat([getattr(pt, f) for pt in plan.problems]) for f in ("x", "y", "s")]
        return tuple(t.clone() for t in sol)

    @staticmethod
    def setup_context(ctx, inputs, output):
        ctx.plan, ctx.opts = inputs[0], inputs[1]

    @staticmethod
    def backward(ctx, gx, gy, gs):
        plan = ctx.plan
        z = lambda g, n: g if g is not None else torch.zeros(n, device=plan.device, dtype=plan.dtype)
        gx, gy, gs = z(gx, plan.n_total), z(gy, plan.m_total), z(gs, plan.m_total)
        dP, dA, dq, db, _ = api.qcp_derivative_vjp(plan, gx.contiguous(), gy.contiguous(), gs.contiguous(),
                                                   ctx.opts)
        return None, None, dP * _offdiag_weight(plan), dA, dq, db

    @staticmethod
    def jvp(ctx, _plan, _opts, dP, dA, dq, db):
        plan = ctx.plan
        z = lambda t, n: t if t is not None else torch.zeros(n, device=plan.device, dtype=plan.dtype)
        dx, dy, ds, _ = api.qcp_derivative_jvp(plan, z(dP, plan.nnzP_total), z(dA, plan.nnzA_total),
                                               z(dq, plan.n_total), z(db, plan.m_total), ctx.opts)
        return dx, dy, ds


def qcp_layer(plan: api.Plan, P_vals, A_vals, q, b, opts=None):
    """(x, y, s) of the plan's problem(s) as a differentiable function of the
    stored data (see the module docstring)."""
    return QCPSolution.apply(plan, opts, P_vals, A_vals, q, b)
