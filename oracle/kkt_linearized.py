"""Residuals of the differentiated optimality conditions (a property check).

At a strictly complementary optimum the derivative (dx, dy, ds) of the
solution map along d theta satisfies the optimality conditions of Sec. 2.1
differentiated at fixed active structure:
    dP x + P dx + dA^T y + A^T dy + dq = 0           (stationarity)
    dA x + A dx + ds - db = 0                        (primal feasibility)
and, block by block (Appendix A cones):
    zero cone:            ds = 0
    R+ row with s = 0:    ds_i = 0;   with y = 0:  dy_i = 0
    SOC with s = 0:       ds = 0;     with y = 0:  dy = 0
    SOC with y, s on opposite boundary rays y = a(1, u), s = b(1, -u):
        y stays on the boundary:  y_u^T dy_u - y_t dy_t = 0
        s stays opposite to y:    (s_t ds_u - ds_t s_u)/s_t^2 + (y_t dy_u - dy_t y_u)/y_t^2 = 0
These equations need only sparse products, so they check a JVP at any size;
together they determine the derivative when the active constraints have full
rank (the generator's regularity), which makes them a pin independent of the
homogeneous embedding.
"""
import numpy as np
import scipy.sparse as sp

ZERO, NONNEG, SOC = 0, 1, 2


def residuals(prob, d, dx, dy, ds):
    """Return (stationarity, feasibility, complementarity) residual vectors."""
    U = prob.P.to_scipy()
    Pf = (U + sp.triu(U, k=1).T).tocsr()
    A = prob.A.to_scipy()
    dU = sp.csr_matrix((d.dP, prob.P.indices, prob.P.indptr), shape=U.shape)
    dPf = (dU + sp.triu(dU, k=1).T).tocsr()
    dA = sp.csr_matrix((d.dA, prob.A.indices, prob.A.indptr), shape=A.shape)
    x, y, s = prob.x, prob.y, prob.s
    e1 = dPf @ x + Pf @ dx + dA.T @ y + A.T @ dy + d.dq
    e2 = dA @ x + A @ dx + ds - d.db
    comp = []
    r = 0
    for t, k in prob.cones:
        yb, sb, dyb, dsb = y[r:r + k], s[r:r + k], dy[r:r + k], ds[r:r + k]
        if t == ZERO:
            comp.append(dsb)
        elif t == NONNEG:
            comp.append(np.where(sb == 0.0, dsb, dyb))
        else:
            ys, ss = np.any(yb != 0.0), np.any(sb != 0.0)
            if ys and not ss:
                comp.append(dsb)
            elif ss and not ys:
                comp.append(dyb)
            elif ys and ss:
                comp.append(np.array([yb[1:] @ dyb[1:] - yb[0] * dyb[0]]))
                comp.append((sb[0] * dsb[1:] - dsb[0] * sb[1:]) / sb[0] ** 2
                            + (yb[0] * dyb[1:] - dyb[0] * yb[1:]) / yb[0] ** 2)
        r += k
    e3 = np.concatenate(comp) if comp else np.zeros(0)
    return e1, e2, e3


def relative_residual(prob, d, dx, dy, ds):
    """max of the three residual norms, each relative to the size of the
    terms that enter it (so that 1e-12 means agreement to rounding)."""
    e1, e2, e3 = residuals(prob, d, dx, dy, ds)
    U = prob.P.to_scipy()
    scale1 = (np.linalg.norm(d.dq) + np.linalg.norm(dx) * max(1.0, float(np.max(np.abs(U.data), initial=0.0)))
              + np.linalg.norm(dy) * max(1.0, abs(prob.A.data).max(initial=0.0)) + 1e-300)
    scale2 = np.linalg.norm(d.db) + np.linalg.norm(ds) + np.linalg.norm(dx) * max(
        1.0, abs(prob.A.data).max(initial=0.0)) + 1e-300
    scale3 = np.linalg.norm(dy) + np.linalg.norm(ds) + 1e-300
    return max(np.linalg.norm(e1) / scale1, np.linalg.norm(e2) / scale2,
               (np.linalg.norm(e3) / scale3) if e3.size else 0.0)
