"""Projections onto the dual cone K* and their derivatives (Appendix A).

The cone K is a product of blocks (type, dim) listed in row order.  The
derivative method projects z_y = y - s onto the DUAL cone K*; the dual of the
zero cone {0} is the whole line R (projection = identity, derivative = I),
the nonnegative orthant and the second-order cone are self-dual.

Kinks (Appendix A leaves the derivative undefined there) are broken as
follows: R+ uses the indicator 1{z > 0}; the SOC cases are tested in the
order the projection lists them, with non-strict inequalities:
||u|| <= -t gives 0, else ||u|| <= t gives the identity, else the formula.
"""
import numpy as np

ZERO, NONNEG, SOC = 0, 1, 2


def proj_soc(z):
    """Euclidean projection onto {(t, u): ||u||_2 <= t} (Appendix A, SOC)."""
    t, u = z[0], z[1:]
    r = np.linalg.norm(u)
    if r <= -t:
        return np.zeros_like(z)
    if r <= t:
        return z.copy()
    out = np.empty_like(z)
    out[0] = r
    out[1:] = u
    return 0.5 * (1.0 + t / r) * out


def dproj_soc(z):
    """Jacobian of proj_soc at z as a dense matrix (Appendix A, SOC).

    Off the two boundary cases, D[(dt, du)] =
    (1/(2 r)) (r dt + u^T du,  u dt + (t + r) du - (t / r^2)(u^T du) u),
    r = ||u||.
    """
    d = z.shape[0]
    t, u = z[0], z[1:]
    r = np.linalg.norm(u)
    if r <= -t:
        return np.zeros((d, d))
    if r <= t:
        return np.eye(d)
    J = np.empty((d, d))
    J[0, 0] = r / (2.0 * r)
    J[0, 1:] = u / (2.0 * r)
    J[1:, 0] = u / (2.0 * r)
    J[1:, 1:] = ((t + r) / (2.0 * r)) * np.eye(d - 1) - (t / (2.0 * r ** 3)) * np.outer(u, u)
    return J


def proj_dual_block(ctype, z):
    if ctype == ZERO:
        return z.copy()                   # dual of {0} is R
    if ctype == NONNEG:
        return np.maximum(z, 0.0)
    if ctype == SOC:
        return proj_soc(z)
    raise ValueError(ctype)


def dproj_dual_block(ctype, z):
    d = z.shape[0]
    if ctype == ZERO:
        return np.eye(d)
    if ctype == NONNEG:
        return np.diag((z > 0.0).astype(np.float64))
    if ctype == SOC:
        return dproj_soc(z)
    raise ValueError(ctype)


def proj_primal_block(ctype, z):
    """Projection onto the block of K itself (used by the Moreau pin)."""
    if ctype == ZERO:
        return np.zeros_like(z)
    return proj_dual_block(ctype, z)      # R+ and SOC are self-dual


def _blocks(cones):
    r = 0
    for t, d in cones:
        yield t, r, r + d
        r += d


def proj_dual(cones, z):
    out = np.empty_like(z)
    for t, a, b in _blocks(cones):
        out[a:b] = proj_dual_block(t, z[a:b])
    return out


def proj_primal(cones, z):
    out = np.empty_like(z)
    for t, a, b in _blocks(cones):
        out[a:b] = proj_primal_block(t, z[a:b])
    return out


def dproj_dual(cones, z):
    """Block-diagonal dense Jacobian of the projection onto K* at z."""
    m = z.shape[0]
    D = np.zeros((m, m))
    for t, a, b in _blocks(cones):
        D[a:b, a:b] = dproj_dual_block(t, z[a:b])
    return D


def dproj_dual_sparse(cones, z):
    """Same Jacobian as a scipy sparse block-diagonal matrix."""
    import scipy.sparse as sp
    blocks = [sp.csr_matrix(dproj_dual_block(t, z[a:b])) for t, a, b in _blocks(cones)]
    if not blocks:
        return sp.csr_matrix((0, 0))
    return sp.block_diag(blocks, format="csr")


def kink_margin(cones, z):
    """Distance (in the quantities the case tests compare) to the nearest
    point where the projection is not differentiable."""
    best = np.inf
    for t, a, b in _blocks(cones):
        zb = z[a:b]
        if t == NONNEG and zb.size:
            best = min(best, float(np.min(np.abs(zb))))
        elif t == SOC:
            r = np.linalg.norm(zb[1:])
            best = min(best, abs(r - abs(zb[0])) if (r > 0 or zb[0] != 0) else 0.0)
    return best
