"""Projections onto the dual cone K* and their derivatives (Appendix A).

The cone K is a product of blocks (type, dim) listed in row order.  The
derivative method projects z_y = y - s onto the DUAL cone K*; the dual of the
zero cone {0} is the whole line R (projection = identity, derivative = I),
the nonnegative orthant, the second-order cone and the positive
semidefinite cone are self-dual.

Kinks (Appendix A leaves the derivative undefined there) are broken as
follows: R+ uses the indicator 1{z > 0}; the SOC cases are tested in the
order the projection lists them, with non-strict inequalities:
||u|| <= -t gives 0, else ||u|| <= t gives the identity, else the formula;
the PSD cone treats an eigenvalue as positive only when it is > 0.

A PSD block of order k holds a symmetric k x k matrix X as its scaled
upper triangle, column by column (dim = k (k + 1) / 2):
    svec(X) = (X_11, sqrt2 X_12, X_22, sqrt2 X_13, sqrt2 X_23, X_33, ...),
so that <svec(X), svec(Y)> = trace(X Y).
"""
import numpy as np

ZERO, NONNEG, SOC, PSD, EXP, POW = 0, 1, 2, 3, 4, 5


def psd_order(d):
    """k with k (k + 1) / 2 = d."""
    k = int(round((np.sqrt(8 * d + 1) - 1) / 2))
    if k * (k + 1) // 2 != d:
        raise ValueError(f"{d} is not a triangular number")
    return k


def smat(v):
    """The symmetric matrix of a PSD block's entries (inverse of svec)."""
    k = psd_order(v.shape[0])
    X = np.empty((k, k))
    i = 0
    for j in range(k):           # column j of the upper triangle
        for a in range(j + 1):   # row a <= j
            X[a, j] = X[j, a] = v[i] if a == j else v[i] / np.sqrt(2.0)
            i += 1
    return X


def svec(X):
    k = X.shape[0]
    out = np.empty(k * (k + 1) // 2)
    i = 0
    for j in range(k):
        for a in range(j + 1):
            out[i] = X[a, j] if a == j else np.sqrt(2.0) * X[a, j]
            i += 1
    return out


def proj_psd(z):
    """Projection onto the PSD cone (Appendix A): keep the nonnegative part
    of the eigendecomposition, sum_i max(lambda_i, 0) v_i v_i^T."""
    lam, V = np.linalg.eigh(smat(z))
    return svec((V * np.maximum(lam, 0.0)) @ V.T)


def psd_B(lam):
    """The symmetric weights of D Pi_psd: the divided differences of
    max(., 0) over the eigenvalues (Appendix A; 1 where both are positive,
    0 where both are not, lambda_i / (lambda_i - lambda_j) for lambda_i > 0
    >= lambda_j)."""
    k = lam.shape[0]
    B = np.empty((k, k))
    for i in range(k):
        for j in range(k):
            pi, pj = lam[i] > 0.0, lam[j] > 0.0
            if pi and pj:
                B[i, j] = 1.0
            elif not pi and not pj:
                B[i, j] = 0.0
            elif pi:
                B[i, j] = lam[i] / (lam[i] - lam[j])
            else:
                B[i, j] = lam[j] / (lam[j] - lam[i])
    return B


def dproj_psd(z):
    """Jacobian of proj_psd at z in svec coordinates (Appendix A):
    D[dZ] = V (B o (V^T dZ V)) V^T, column by column."""
    lam, V = np.linalg.eigh(smat(z))
    B = psd_B(lam)
    d = z.shape[0]
    J = np.empty((d, d))
    for c in range(d):
        e = np.zeros(d)
        e[c] = 1.0
        J[:, c] = svec(V @ (B * (V.T @ smat(e) @ V)) @ V.T)
    return J


# ------------------------------------------------------------ exponential cone
# K_exp = cl{(x, y, z): y > 0, y exp(x / y) <= z} (Appendix A).  Its
# boundary away from the face {(x, 0, z): x <= 0, z >= 0} is the family of
# rays t a(r), a(r) = (r, 1, exp(r)), t > 0.

def in_exp(p, tol=0.0):
    x, y, z = p
    if abs(y) <= tol and x <= tol and z >= -tol:   # the face {(x, 0, z): x <= 0, z >= 0}
        return True
    if y > 0:
        return y * np.exp(x / y) <= z + tol
    return False


def in_exp_dual(q, tol=0.0):
    """K_exp* = cl{(u, v, w): u < 0, -u exp(v / u) <= e w} (Appendix A)."""
    u, v, w = q
    if abs(u) <= tol and v >= -tol and w >= -tol:  # the face {(0, v, w): v, w >= 0}
        return True
    if u < 0:
        return -u * np.exp(v / u) <= np.e * w + tol
    return False


def proj_exp(p):
    """Euclidean projection onto K_exp (Appendix A): p itself inside K, 0
    inside the polar cone -K*, (x, 0, max(z, 0)) when x < 0 and y < 0, else
    the nearest point of the boundary.  The last case is computed as its
    definition: over the rays a(r), the nearest point of each ray is
    max(<a, p>, 0) / |a|^2 a, and the best ray maximises <a, p>^2 / |a|^2 with
    <a, p> > 0 (a grid over r, then scipy's bounded scalar minimiser); the
    face {(x, 0, z): x <= 0, z >= 0} is a candidate too.  The best ray is
    refined to full precision as the root of the stationarity condition
    <a', p> |a|^2 - <a, p> <a', a> = 0 (a' = (1, 0, exp(r))) inside the grid
    cell of the minimum."""
    from scipy.optimize import brentq, minimize_scalar
    p = np.asarray(p, np.float64)
    x, y, z = p
    if in_exp(p):
        return p.copy()
    if in_exp_dual(-p):
        return np.zeros(3)
    if x < 0 and y < 0:
        return np.array([x, 0.0, max(z, 0.0)])
    a = lambda r: np.array([r, 1.0, np.exp(r)])

    def dist2(r):
        ar = a(r)
        t = max(ar @ p, 0.0) / (ar @ ar)
        return float(np.sum((t * ar - p) ** 2))

    def stat(r):
        ar, da = a(r), np.array([1.0, 0.0, np.exp(r)])
        return (da @ p) * (ar @ ar) - (ar @ p) * (da @ ar)

    # rays toward the face need very negative r (r = x / y when y > 0 is
    # the ray straight above p); exp(r) stays representable down to -700
    grid = np.concatenate([np.linspace(-700.0, -40.0, 6601)[:-1], np.linspace(-40.0, 40.0, 8001)])
    if y > 0 and -700.0 < x / y < 40.0:
        grid = np.sort(np.append(grid, x / y))
    A = np.stack([grid, np.ones_like(grid), np.exp(grid)], 1)
    tg = np.maximum(A @ p, 0.0) / np.sum(A * A, 1)
    vals = np.sum((tg[:, None] * A - p) ** 2, 1)
    i = int(np.argmin(vals))
    lo, hi = grid[max(i - 1, 0)], grid[min(i + 1, grid.size - 1)]
    if stat(lo) * stat(hi) < 0:
        rstar = brentq(stat, lo, hi, xtol=1e-16, rtol=4 * np.finfo(float).eps, maxiter=500)
    else:
        rstar = minimize_scalar(dist2, bounds=(lo, hi), method="bounded",
                                options={"xatol": 1e-14, "maxiter": 500}).x
    ar = a(rstar)
    best = max(ar @ p, 0.0) / (ar @ ar) * ar
    face = np.array([min(x, 0.0), 0.0, max(z, 0.0)])
    return face if np.sum((face - p) ** 2) < np.sum((best - p) ** 2) else best


def dproj_exp(p):
    """Jacobian of proj_exp at p (Appendix A): I inside K, 0 inside the polar
    cone, diag(1, 0, 1{z > 0}) when x < 0 and y < 0, else the leading 3 x 3
    block of J^-1 with J the Jacobian of the projection's optimality
    conditions at the projected point (x*, y*, z*) and multiplier
    mu* = z* - z."""
    p = np.asarray(p, np.float64)
    x, y, z = p
    if in_exp(p):
        return np.eye(3)
    if in_exp_dual(-p):
        return np.zeros((3, 3))
    if x < 0 and y < 0:
        return np.diag([1.0, 0.0, 1.0 if z > 0 else 0.0])
    xs, ys, zs = proj_exp(p)
    return np.linalg.inv(exp_kkt_jacobian(xs, ys, zs - z))[:3, :3]


def exp_kkt_jacobian(xs, ys, mu):
    """J of Appendix A: the Jacobian of the optimality conditions of the
    projection onto the boundary z = y exp(x / y), at the projected point
    (xs, ys) with multiplier mu.  The printed (2, 2) entry is garbled; it is
    read as 1 + mu xs^2 exp(xs / ys) / ys^3, the matching entry of the
    Hessian of y exp(x / y) - z."""
    e = np.exp(xs / ys)
    return np.array([
        [1.0 + mu * e / ys, -mu * xs * e / ys ** 2, 0.0, e],
        [-mu * xs * e / ys ** 2, 1.0 + mu * xs ** 2 * e / ys ** 3, 0.0, (1.0 - xs / ys) * e],
        [0.0, 0.0, 1.0, -1.0],
        [e, (1.0 - xs / ys) * e, -1.0, 0.0]])


def proj_exp_dual(q):
    """Projection onto K_exp* by the Moreau decomposition (Appendix A):
    Pi_{K*}(q) = q + Pi_K(-q)."""
    q = np.asarray(q, np.float64)
    return q + proj_exp(-q)


def dproj_exp_dual(q):
    return np.eye(3) - dproj_exp(-np.asarray(q, np.float64))


# ------------------------------------------------------------------ power cone
# K_pow,a = {(x, y, z): x, y >= 0, x^a y^(1-a) >= |z|}, 0 < a < 1 (Appendix A).

def in_pow(p, a, tol=0.0):
    x, y, z = p
    if x < -tol or y < -tol:
        return False
    return max(x, 0.0) ** a * max(y, 0.0) ** (1 - a) >= abs(z) - tol


def in_pow_dual(q, a, tol=0.0):
    u, v, w = q
    if u < -tol or v < -tol:
        return False
    return (max(u, 0.0) / a) ** a * (max(v, 0.0) / (1 - a)) ** (1 - a) >= abs(w) - tol


def _pow_f(x, y, z, a, r):
    fx = 0.5 * (x + np.sqrt(x * x + 4 * a * r * (abs(z) - r)))
    fy = 0.5 * (y + np.sqrt(y * y + 4 * (1 - a) * r * (abs(z) - r)))
    return fx, fy


def _pow_r(x, y, z, a):
    """The root r in (0, |z|) of r = f_x(r)^a f_y(r)^(1-a) (Appendix A).
    r = 0 solves the equation too whenever x <= 0 or y <= 0, so the bracket
    starts at the largest of |z| 10^-k (k = 1, 2, ...) where the residual is
    positive (it is negative at |z|)."""
    from scipy.optimize import brentq
    g = lambda r: (lambda f: f[0] ** a * f[1] ** (1 - a))(_pow_f(x, y, z, a, r)) - r
    az = abs(z)
    lo = None
    for k in range(1, 300):
        if g(az * 10.0 ** -k) > 0:
            lo = az * 10.0 ** -k
            break
    if lo is None:
        return 0.0
    return brentq(g, lo, az, xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=1000)


def proj_pow(p, a):
    """Projection onto K_pow,a (Appendix A): p inside K, 0 inside the polar
    cone, (x+, y+, 0) for z = 0, else (f_x(r), f_y(r), sign(z) r)."""
    p = np.asarray(p, np.float64)
    x, y, z = p
    if in_pow(p, a):
        return p.copy()
    if in_pow_dual(-p, a):
        return np.zeros(3)
    if z == 0.0:
        return np.array([max(x, 0.0), max(y, 0.0), 0.0])
    r = _pow_r(x, y, z, a)
    fx, fy = _pow_f(x, y, z, a, r)
    return np.array([fx, fy, np.sign(z) * r])


def dproj_pow(p, a):
    """Jacobian of proj_pow (Appendix A, from Hien 2015 Theorem 3.1)."""
    p = np.asarray(p, np.float64)
    x, y, z = p
    if in_pow(p, a):
        return np.eye(3)
    if in_pow_dual(-p, a):
        return np.zeros((3, 3))
    if z == 0.0:
        if x > 0 and y < 0:
            d = 1.0 if a > 0.5 else (0.0 if a < 0.5 else x / (2 * abs(y) + x))
        elif y > 0 and x < 0:
            d = 1.0 if a < 0.5 else (0.0 if a > 0.5 else y / (2 * abs(x) + y))
        else:
            d = 0.0
        return np.diag([1.0 if x > 0 else 0.0, 1.0 if y > 0 else 0.0, d])
    r = _pow_r(x, y, z, a)
    fx, fy = _pow_f(x, y, z, a, r)
    az, sz = abs(z), np.sign(z)
    gx, gy = 2 * fx - x, 2 * fy - y
    T = -(a * x / gx + (1 - a) * y / gy)
    L = 2 * (az - r) / (az + (az - 2 * r) * (a * x / gx + (1 - a) * y / gy))
    J = np.empty((3, 3))
    J[0, 0] = 0.5 + x / (2 * gx) + a * a * (az - 2 * r) * r * L / gx ** 2
    J[0, 1] = J[1, 0] = (a - a * a) * (az - 2 * r) * r * L / (gx * gy)
    J[0, 2] = J[2, 0] = sz * a * r * L / gx
    J[1, 1] = 0.5 + y / (2 * gy) + (1 - a) ** 2 * (az - 2 * r) * r * L / gy ** 2
    J[1, 2] = J[2, 1] = sz * (1 - a) * r * L / gy
    J[2, 2] = r / az + r / az * T * L
    return J


def proj_pow_dual(q, a):
    q = np.asarray(q, np.float64)
    return q + proj_pow(-q, a)


def dproj_pow_dual(q, a):
    return np.eye(3) - dproj_pow(-np.asarray(q, np.float64), a)


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


def proj_dual_block(ctype, z, a=None):
    """Projection onto the dual of one block (a: the power cone's exponent)."""
    if ctype == ZERO:
        return z.copy()                   # dual of {0} is R
    if ctype == NONNEG:
        return np.maximum(z, 0.0)
    if ctype == SOC:
        return proj_soc(z)
    if ctype == PSD:
        return proj_psd(z)
    if ctype == EXP:
        return proj_exp_dual(z)           # the exponential and power cones are not self-dual
    if ctype == POW:
        return proj_pow_dual(z, a)
    raise ValueError(ctype)


def dproj_dual_block(ctype, z, a=None):
    d = z.shape[0]
    if ctype == ZERO:
        return np.eye(d)
    if ctype == NONNEG:
        return np.diag((z > 0.0).astype(np.float64))
    if ctype == SOC:
        return dproj_soc(z)
    if ctype == PSD:
        return dproj_psd(z)
    if ctype == EXP:
        return dproj_exp_dual(z)
    if ctype == POW:
        return dproj_pow_dual(z, a)
    raise ValueError(ctype)


def proj_primal_block(ctype, z, a=None):
    """Projection onto the block of K itself (used by the Moreau pin)."""
    if ctype == ZERO:
        return np.zeros_like(z)
    if ctype == EXP:
        return proj_exp(z)
    if ctype == POW:
        return proj_pow(z, a)
    return proj_dual_block(ctype, z)      # R+, SOC and PSD are self-dual


def _blocks(cones):
    """(type, first row, end row, parameter) per block; cones holds (type,
    dim) or (type, dim, parameter) entries (the parameter: the power cone's
    exponent)."""
    r = 0
    for c in cones:
        t, d = c[0], c[1]
        yield t, r, r + d, (c[2] if len(c) > 2 else None)
        r += d


def cone_list(prob):
    """(type, dim, parameter) per block of a problem (parameter 0 unless a
    power cone)."""
    par = getattr(prob, "cone_param", None)
    if par is None:
        par = np.zeros(len(prob.cone_type))
    return [(int(t), int(d), float(a)) for t, d, a in zip(prob.cone_type, prob.cone_dim, par)]


def proj_dual(cones, z):
    out = np.empty_like(z)
    for t, a, b, par in _blocks(cones):
        out[a:b] = proj_dual_block(t, z[a:b], par)
    return out


def proj_primal(cones, z):
    out = np.empty_like(z)
    for t, a, b, par in _blocks(cones):
        out[a:b] = proj_primal_block(t, z[a:b], par)
    return out


def dproj_dual(cones, z):
    """Block-diagonal dense Jacobian of the projection onto K* at z."""
    m = z.shape[0]
    D = np.zeros((m, m))
    for t, a, b, par in _blocks(cones):
        D[a:b, a:b] = dproj_dual_block(t, z[a:b], par)
    return D


def dproj_dual_sparse(cones, z):
    """Same Jacobian as a scipy sparse block-diagonal matrix.  The zero and
    R+ blocks are diagonal, so they are built as sparse diagonals (the same
    entries as dproj_dual_block) and never stored densely."""
    import scipy.sparse as sp

    def block(t, zb, par):
        if t == ZERO:
            return sp.identity(zb.shape[0], format="csr")
        if t == NONNEG:
            Db = sp.diags((zb > 0.0).astype(np.float64), format="csr")
            Db.eliminate_zeros()
            return Db
        return sp.csr_matrix(dproj_dual_block(t, zb, par))

    blocks = [block(t, z[a:b], par) for t, a, b, par in _blocks(cones)]
    if not blocks:
        return sp.csr_matrix((0, 0))
    return sp.block_diag(blocks, format="csr")


def kink_margin(cones, z):
    """Distance (in the quantities the case tests compare) to the nearest
    point where the projection is not differentiable."""
    best = np.inf
    for t, a, b, _ in _blocks(cones):
        zb = z[a:b]
        if t == NONNEG and zb.size:
            best = min(best, float(np.min(np.abs(zb))))
        elif t == SOC:
            r = np.linalg.norm(zb[1:])
            best = min(best, abs(r - abs(zb[0])) if (r > 0 or zb[0] != 0) else 0.0)
        elif t == PSD:
            best = min(best, float(np.min(np.abs(np.linalg.eigvalsh(smat(zb))))))
    return best
