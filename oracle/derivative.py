"""JVP and VJP of the QCP solution map (Sec. 3.1 and 3.2).

Forward (Sec. 3.1):  z = (x, y - s, 1);  dN = D_theta N(z)[d theta];
  dz solves F dz = -dN;  (dx, dy, ds) = D phi(z) dz.
Adjoint (Sec. 3.2):  g = D phi(z)^T (dx, dy, ds);  r solves F^T r = -g;
  d theta = D_theta N(z)^T [r], kept on the patterns of P (upper) and A.

F is singular at every root: R is positively homogeneous (Sec. 2.3), so
F z = R(z) = 0.  Sec. 2.4 assumes F invertible; the reading used here is
that both linear systems are consistent (dN lies in the range of F because
N(s(theta), theta) = 0 along the solution map, and g is orthogonal to z
because D phi(z) z = 0), and that any solution gives the same outputs,
since D phi(z) z = 0 and D_theta N^T annihilates the null space of F^T.

Two ways to solve, both plain:
  * dense: LU with partial pivoting of the bordered (N+1) x (N+1) matrix
    [[F, beta], [e_N^T, 0]] (beta a fixed random unit vector, e_N fixes
    dz_N = 0); the same factors solve the adjoint system.  The extra
    unknown (lambda / mu) must come out ~0: it is a built-in consistency
    alarm.
  * matrix-free: LSMR, as Sec. 3.1 prescribes, on the least-squares problems
    min ||F dz + dN|| and min ||F^T r + g||, with products by F and F^T
    formed from sparse P, A and the block-diagonal D Pi.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import cones as C
from . import embedding as E


def _beta(N, seed=20250824):
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(N)
    return v / np.linalg.norm(v)


class DenseFactor:
    """Dense F at the constructed root and the LU of its bordered form."""

    def __init__(self, prob, z=None):
        self.prob = prob
        self.z = E.solution_to_z(prob) if z is None else z
        self.F = E.F_dense(prob, self.z)
        N = self.F.shape[0]
        B = np.zeros((N + 1, N + 1))
        B[:N, :N] = self.F
        B[:N, N] = _beta(N)
        B[N, N - 1] = 1.0
        self.lu = sla.lu_factor(B, check_finite=True)
        piv = np.abs(np.diag(self.lu[0]))
        self.pivot_ratio = float(piv.min() / piv.max())
        self.N = N

    def solve(self, rhs, trans=0):
        sol = sla.lu_solve(self.lu, np.concatenate([rhs, [0.0]]), trans=trans)
        return sol[:self.N], float(sol[self.N])


def d_theta_N(prob, z, dP, dA, dq, db):
    """D_theta N(z)[d theta] = D_theta Q(Pi z)[d theta] / |z_N|  (Sec. 2.4)."""
    return E.DthetaQ(prob, E.proj_K(prob, z), dP, dA, dq, db) / abs(z[-1])


def d_theta_N_T(prob, z, w):
    """D_theta N(z)^T [w] on the stored patterns: (dP vals, dA vals, dq, db)."""
    Pt, At, qt, bt = E.DthetaQ_T_dense(prob, E.proj_K(prob, z), w / abs(z[-1]))
    dPv, dAv = E.restrict_to_patterns(prob, Pt, At)
    return dPv, dAv, qt, bt


def jvp_dense(prob, d, fac=None):
    """(dx, dy, ds) = D phi(z) (-F^{-1}) D_theta N(z)[d theta]  (Sec. 3.1)."""
    fac = fac or DenseFactor(prob)
    z = fac.z
    big = fac.N > 3000
    dN = (d_theta_N_sparse if big else d_theta_N)(prob, z, d.dP, d.dA, d.dq, d.db)
    dz, lam = fac.solve(-dN)
    res = np.linalg.norm(fac.F @ dz + dN) / max(np.linalg.norm(dN), 1e-300)
    info = {"lambda": lam, "pivot_ratio": fac.pivot_ratio, "rel_residual": float(res)}
    if big:   # D phi applied without forming it (pinned equal to the dense D phi)
        dx, dy, ds = _phi_apply(prob, z, dz)
        return dx, dy, ds, info
    out = E.Dphi(prob, z) @ dz
    n, m = prob.n, prob.m
    return out[:n], out[n:n + m], out[n + m:], info


def vjp_dense(prob, d, fac=None):
    """d theta = D_theta N(z)^T (-F^{-T}) D phi(z)^T w  (Sec. 3.2)."""
    fac = fac or DenseFactor(prob)
    z = fac.z
    big = fac.N > 3000
    if big:
        g = _phi_apply_T(prob, z, d.wx, d.wy, d.ws)
    else:
        g = E.Dphi(prob, z).T @ np.concatenate([d.wx, d.wy, d.ws])
    r, mu = fac.solve(-g, trans=1)
    res = np.linalg.norm(fac.F.T @ r + g) / max(np.linalg.norm(g), 1e-300)
    dPv, dAv, dq, db = (d_theta_N_T_sparse if big else d_theta_N_T)(prob, z, r)
    info = {"mu": mu, "pivot_ratio": fac.pivot_ratio, "rel_residual": float(res)}
    return dPv, dAv, dq, db, info


# ---------------------------------------------------------------- matrix-free
class FOperator:
    """Products with F = (1/z_N)(D_u Q(Pi z) D Pi(z) - D Pi(z) + I) and F^T
    from sparse P, A and a sparse block-diagonal D Pi_{K*}."""

    def __init__(self, prob, z=None):
        self.prob = prob
        self.z = E.solution_to_z(prob) if z is None else z
        n, m = prob.n, prob.m
        self.n, self.m = n, m
        self.P = E.P_full_sparse(prob)
        self.A = prob.A.to_scipy()
        self.AT = self.A.T.tocsr()
        zx, zy, zN = E.split(prob, self.z)
        pz = E.proj_K(prob, self.z)
        self.x, self.y, self.tau = E.split(prob, pz)
        self.Dy = C.dproj_dual_sparse(C.cone_list(prob), zy)
        self.dtau = 1.0 if zN > 0 else 0.0
        self.zN = zN
        self.Px = self.P @ self.x
        self.last_x = (-2.0 / self.tau) * self.Px - prob.q     # row N of D_u Q, x part
        self.last_t = (1.0 / self.tau ** 2) * (self.x @ self.Px)
        self.N = n + m + 1

    def _DPi(self, v):
        n, m = self.n, self.m
        return np.concatenate([v[:n], self.Dy @ v[n:n + m], [self.dtau * v[-1]]])

    def _DPi_T(self, v):
        n, m = self.n, self.m
        return np.concatenate([v[:n], self.Dy.T @ v[n:n + m], [self.dtau * v[-1]]])

    def _DuQ(self, w):
        n, m = self.n, self.m
        wx, wy, wt = w[:n], w[n:n + m], w[-1]
        p = self.prob
        return np.concatenate([
            self.P @ wx + self.AT @ wy + p.q * wt,
            -(self.A @ wx) + p.b * wt,
            [self.last_x @ wx - p.b @ wy + self.last_t * wt],
        ])

    def _DuQ_T(self, r):
        n, m = self.n, self.m
        r1, r2, r3 = r[:n], r[n:n + m], r[-1]
        p = self.prob
        return np.concatenate([
            self.P @ r1 - self.AT @ r2 + self.last_x * r3,
            self.A @ r1 - p.b * r3,
            [p.q @ r1 + p.b @ r2 + self.last_t * r3],
        ])

    def matvec(self, v):
        dv = self._DPi(v)
        return (self._DuQ(dv) - dv + v) / self.zN

    def rmatvec(self, u):
        return (self._DPi_T(self._DuQ_T(u)) - self._DPi_T(u) + u) / self.zN

    def sparse(self):
        """F assembled as a scipy CSR matrix from the same pieces (D_u Q with
        its dense tau row and column, the block-diagonal D Pi), for the
        column-scaled LSMR below."""
        import scipy.sparse as sp
        p, n, m = self.prob, self.n, self.m
        DuQ = sp.bmat([[self.P, self.AT, sp.csr_matrix(p.q.reshape(-1, 1))],
                       [-self.A, None, sp.csr_matrix(p.b.reshape(-1, 1))],
                       [sp.csr_matrix(self.last_x.reshape(1, -1)), sp.csr_matrix(-p.b.reshape(1, -1)),
                        sp.csr_matrix([[self.last_t]])]], format="csr")
        DPi = sp.block_diag([sp.identity(n), self.Dy, sp.csr_matrix([[self.dtau]])], format="csr")
        return ((DuQ @ DPi - DPi + sp.identity(self.N)) / self.zN).tocsr()

    def linear_operator(self, transpose=False):
        mv, rmv = (self.rmatvec, self.matvec) if transpose else (self.matvec, self.rmatvec)
        return spla.LinearOperator((self.N, self.N), matvec=mv, rmatvec=rmv, dtype=np.float64)


def d_theta_N_sparse(prob, z, dP, dA, dq, db):
    """D_theta N(z)[d theta] with sparse dP, dA (same formula as d_theta_N)."""
    import scipy.sparse as sp
    U = sp.csr_matrix((dP, prob.P.indices, prob.P.indptr), shape=(prob.n, prob.n))
    dPs = (U + sp.triu(U, k=1).T).tocsr()
    dAs = sp.csr_matrix((dA, prob.A.indices, prob.A.indptr), shape=(prob.m, prob.n))
    x, y, tau = E.split(prob, E.proj_K(prob, z))
    out = np.concatenate([
        dPs @ x + dAs.T @ y + tau * dq,
        -(dAs @ x) + tau * db,
        [(-1.0 / tau) * (x @ (dPs @ x)) - dq @ x - db @ y],
    ])
    return out / abs(z[-1])


def d_theta_N_T_sparse(prob, z, w):
    """D_theta N(z)^T [w] evaluated only at the stored pattern positions."""
    x, y, tau = E.split(prob, E.proj_K(prob, z))
    w = w / abs(z[-1])
    w1, w2, wN = E.split(prob, w)
    pi, pj = prob.P.row_ids(), prob.P.indices
    ai, aj = prob.A.row_ids(), prob.A.indices
    dP = 0.5 * (w1[pi] * x[pj] + x[pi] * w1[pj]) - (wN / tau) * x[pi] * x[pj]
    dA = y[ai] * w1[aj] - w2[ai] * x[aj]
    return dP, dA, tau * w1 - wN * x, tau * w2 - wN * y


def _phi_apply(prob, z, dz):
    """D phi(z) dz without forming D phi."""
    n, m = prob.n, prob.m
    zx, zy, zN = E.split(prob, z)
    py = C.proj_dual(C.cone_list(prob), zy)
    D = C.dproj_dual_sparse(C.cone_list(prob), zy)
    dzx, dzy, dzN = dz[:n], dz[n:n + m], dz[-1]
    Ddy = D @ dzy
    return ((dzx - dzN * zx / zN) / zN, (Ddy - dzN * py / zN) / zN,
            (Ddy - dzy - dzN * (py - zy) / zN) / zN)


def _phi_apply_T(prob, z, wx, wy, ws):
    """D phi(z)^T (wx, wy, ws) without forming D phi."""
    zx, zy, zN = E.split(prob, z)
    py = C.proj_dual(C.cone_list(prob), zy)
    D = C.dproj_dual_sparse(C.cone_list(prob), zy)
    gy = (D.T @ (wy + ws) - ws) / zN
    gN = -(zx @ wx + py @ wy + (py - zy) @ ws) / zN ** 2
    return np.concatenate([wx / zN, gy, [gN]])


def _ruiz(F, sweeps=16):
    """Row and column scalings (r, c) of a sparse matrix by Ruiz's iterated
    equilibration in the 2-norm (Ruiz 2001): each sweep divides every row
    of diag(r) F diag(c) by the square root of its norm, then every column
    likewise.  Both linear systems are consistent, so the scaled problem
    min ||diag(r) (F diag(c) y - b)|| has the same solution dz = c y; only
    the Krylov iterates change."""
    import scipy.sparse as sp
    F = sp.csr_matrix(F)
    r = np.ones(F.shape[0])
    c = np.ones(F.shape[1])
    for _ in range(sweeps):
        G = sp.diags(r) @ F @ sp.diags(c)
        rn = np.sqrt(np.asarray(G.multiply(G).sum(axis=1)).ravel())
        r = r / np.sqrt(np.where(rn > 0, rn, 1.0))
        G = sp.diags(r) @ F @ sp.diags(c)
        cn = np.sqrt(np.asarray(G.multiply(G).sum(axis=0)).ravel())
        c = c / np.sqrt(np.where(cn > 0, cn, 1.0))
    return r, c


def _scaled_lsmr(F, b, rtol, maxiter):
    """LSMR on diag(r) F diag(c) y = diag(r) b (Ruiz scalings), x = c y."""
    import scipy.sparse as sp
    r, c = _ruiz(F)
    res = spla.lsmr(sp.diags(r) @ F @ sp.diags(c), r * b, atol=0.0, btol=rtol, conlim=0.0, maxiter=maxiter)
    return c * res[0], res


def jvp_lsmr(prob, d, rtol=1e-10, maxiter=None, op=None, scale=False):
    """Matrix-free JVP: LSMR on min ||F dz + dN|| (Sec. 3.1).  scale=True
    runs it on the assembled sparse F with Ruiz's row and column scalings
    (dz = C y; F dz = -dN is consistent, so the solution is the same).  rtol
    bounds the scaled problem's residual; info reports the true one."""
    op = op or FOperator(prob)
    z = op.z
    dN = d_theta_N_sparse(prob, z, d.dP, d.dA, d.dq, d.db)
    if scale:
        dz, res = _scaled_lsmr(op.sparse(), -dN, rtol, maxiter or 20 * op.N)
    else:
        res = spla.lsmr(op.linear_operator(), -dN, atol=0.0, btol=rtol, conlim=0.0,
                        maxiter=maxiter or 20 * op.N)
        dz = res[0]
    true_res = np.linalg.norm(op.matvec(dz) + dN) / max(np.linalg.norm(dN), 1e-300)
    dx, dy, ds = _phi_apply(prob, z, dz)
    return dx, dy, ds, {"iters": int(res[2]), "istop": int(res[1]), "rel_residual": float(true_res)}


def vjp_lsmr(prob, d, rtol=1e-10, maxiter=None, op=None, scale=False):
    """Matrix-free VJP: LSMR on min ||F^T r + g|| (Sec. 3.2); scale=True as
    in jvp_lsmr, on F^T."""
    op = op or FOperator(prob)
    z = op.z
    g = _phi_apply_T(prob, z, d.wx, d.wy, d.ws)
    if scale:
        r, res = _scaled_lsmr(op.sparse().T.tocsr(), -g, rtol, maxiter or 20 * op.N)
    else:
        res = spla.lsmr(op.linear_operator(transpose=True), -g, atol=0.0, btol=rtol, conlim=0.0,
                        maxiter=maxiter or 20 * op.N)
        r = res[0]
    true_res = np.linalg.norm(op.rmatvec(r) + g) / max(np.linalg.norm(g), 1e-300)
    dPv, dAv, dq, db = d_theta_N_T_sparse(prob, z, r)
    return dPv, dAv, dq, db, {"iters": int(res[2]), "istop": int(res[1]),
                              "rel_residual": float(true_res)}
