"""Helpers for the GPU tests: run the library through its C ABI (via the
thin ctypes binding) and compare with the CPU oracle."""
import numpy as np
import torch

import qcpgen as g
from conftest import rel_err


def lib():
    import __graft_entry__ as ge
    ge.build()
    import paper_2508_17522_gb300 as q
    return q


def to_np(*ts):
    return [t.detach().cpu().numpy().astype(np.float64) for t in ts]


def gpu_jvp(q, plan, d, opts):
    dx, dy, ds, info = q.qcp_derivative_jvp(plan, d.dP, d.dA, d.dq, d.db, opts)
    return to_np(dx, dy, ds), info


def gpu_vjp(q, plan, d, opts):
    dP, dA, dq, db, info = q.qcp_derivative_vjp(plan, d.wx, d.wy, d.ws, opts)
    return to_np(dP, dA, dq, db), info


def adjoint_gap(prob, d, jvp_out, vjp_out):
    """|<JVP(dtheta), w> - <dtheta, VJP(w)>| / scale, weight 2 on stored
    off-diagonal P entries (the VJP returns symmetric-matrix entries)."""
    dx, dy, ds = jvp_out
    gP, gA, gq, gb = vjp_out
    c = np.where(prob.P.row_ids() == prob.P.indices, 1.0, 2.0)
    lhs = dx @ d.wx + dy @ d.wy + ds @ d.ws
    rhs = (c * d.dP) @ gP + d.dA @ gA + d.dq @ gq + d.db @ gb
    scale = (np.linalg.norm(np.concatenate([dx, dy, ds])) * np.linalg.norm(np.concatenate([d.wx, d.wy, d.ws]))
             + 1e-300)
    return abs(lhs - rhs) / scale


__all__ = ["lib", "to_np", "gpu_jvp", "gpu_vjp", "adjoint_gap", "rel_err", "g", "torch"]
