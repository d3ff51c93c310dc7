"""The homogeneous embedding, its residual map and their derivatives.

Everything here is written for a general point z with z_N != 0 and a
general tau = (Pi z)_N, exactly as Sec. 2.1-2.4 state it; nothing assumes
the simplifications tau = z_N = 1 that hold at a constructed root.

  Q(u)           Sec. 2.1, "embedding": Q1 = P x + A^T y + tau q,
                 Q2 = -A x + tau b, Q3 = -(1/tau) x^T P x - q^T x - b^T y
  Pi             projection onto K = R^n x K* x R+ (Sec. 2.1 / 2.3)
  R(z)           Sec. 2.3, eq. residual-map: Q(Pi z) - Pi z + z
  N(z)           Sec. 2.3, eq. normalized-residual: R(z) / |z_N|
  D_u Q          Sec. 2.4, the Jacobian of Q in u
  F = D_z N      Sec. 2.4 / 3.1: (1/z_N)(D_u Q(Pi z) D Pi(z) - D Pi(z) + I)
  D_theta Q      Sec. 2.4 and its adjoint (the tuple printed there lists
                 b~ twice; it is read as (P~, A~, q~, b~))
  phi, D phi     Sec. 2.4, "Solution construction"
"""
import numpy as np
import scipy.sparse as sp

from . import cones as C


# ---------------------------------------------------------------- data views
def P_full(prob):
    """Dense symmetric P from its stored upper triangle."""
    U = prob.P.to_scipy().toarray()
    return U + np.triu(U, 1).T


def P_full_sparse(prob):
    U = prob.P.to_scipy()
    return (U + sp.triu(U, k=1).T).tocsr()


def sym_from_upper_values(prob, vals):
    """Dense symmetric matrix whose upper triangle holds `vals` on P's pattern."""
    n = prob.n
    M = np.zeros((n, n))
    rows = prob.P.row_ids()
    cols = prob.P.indices
    M[rows, cols] = vals
    M[cols, rows] = vals
    return M


def dense_on_A_pattern(prob, vals):
    M = np.zeros((prob.m, prob.n))
    M[prob.A.row_ids(), prob.A.indices] = vals
    return M


def A_dense(prob):
    return prob.A.to_scipy().toarray()


def split(prob, v):
    n, m = prob.n, prob.m
    return v[:n], v[n:n + m], v[n + m]


# ---------------------------------------------------------------- root
def solution_to_z(prob, x=None, y=None, s=None):
    """Sec. 3.1: z = M^{-1}(u, v) = u - v, u = (x, y, 1), v = (0, s, 0)."""
    x = prob.x if x is None else x
    y = prob.y if y is None else y
    s = prob.s if s is None else s
    return np.concatenate([x, y - s, [1.0]])


# ---------------------------------------------------------------- Q and Pi
def Q(prob, u, P=None, A=None, q=None, b=None):
    """Q(u, theta) of eq. (embedding); theta defaults to the problem's."""
    P = P_full(prob) if P is None else P
    A = A_dense(prob) if A is None else A
    q = prob.q if q is None else q
    b = prob.b if b is None else b
    x, y, tau = split(prob, u)
    return np.concatenate([
        P @ x + A.T @ y + tau * q,
        -A @ x + tau * b,
        [-(1.0 / tau) * (x @ P @ x) - q @ x - b @ y],
    ])


def proj_K(prob, z):
    """Pi onto K = R^n x K* x R+."""
    zx, zy, zN = split(prob, z)
    return np.concatenate([zx, C.proj_dual(C.cone_list(prob), zy), [max(zN, 0.0)]])


def dproj_K(prob, z):
    """D Pi(z) = blkdiag(I_n, D Pi_{K*}(z_y), 1{z_N > 0}) as a dense matrix."""
    n, m = prob.n, prob.m
    zx, zy, zN = split(prob, z)
    D = np.zeros((n + m + 1, n + m + 1))
    D[:n, :n] = np.eye(n)
    D[n:n + m, n:n + m] = C.dproj_dual(C.cone_list(prob), zy)
    D[-1, -1] = 1.0 if zN > 0 else 0.0
    return D


def residual_map(prob, z, theta=None):
    """R(z) = Q(Pi z) - Pi z + z  (eq. residual-map)."""
    th = theta or {}
    pz = proj_K(prob, z)
    return Q(prob, pz, **th) - pz + z


def normalized_residual(prob, z, theta=None):
    """N(z) = R(z) / |z_N|  (eq. normalized-residual)."""
    return residual_map(prob, z, theta) / abs(z[-1])


# ---------------------------------------------------------------- D_u Q and F
def DuQ(prob, u):
    """The Jacobian of Q with respect to u (Sec. 2.4)."""
    n, m = prob.n, prob.m
    P = P_full(prob)
    A = A_dense(prob)
    x, y, tau = split(prob, u)
    J = np.zeros((n + m + 1, n + m + 1))
    J[:n, :n] = P
    J[:n, n:n + m] = A.T
    J[:n, -1] = prob.q
    J[n:n + m, :n] = -A
    J[n:n + m, -1] = prob.b
    J[-1, :n] = (-2.0 / tau) * (P @ x) - prob.q
    J[-1, n:n + m] = -prob.b
    J[-1, -1] = (1.0 / tau ** 2) * (x @ P @ x)
    return J


def F_dense(prob, z, dense_limit=3000):
    """F = D_z N(z) = (1/z_N)(D_u Q(Pi z) D Pi(z) - D Pi(z) + I)  (Sec. 3.1).
    Above dense_limit rows the product D_u Q D Pi is formed with D Pi held
    sparse; both forms give the same matrix (pinned against each other)."""
    pz = proj_K(prob, z)
    DP = dproj_K(prob, z)
    N = z.shape[0]
    if N <= dense_limit:
        prod = DuQ(prob, pz) @ DP
    else:
        # the same product, with D Pi held sparse (it is block diagonal)
        prod = np.asarray((sp.csr_matrix(DP).T @ DuQ(prob, pz).T).T)
    return (prod - DP + np.eye(N)) / z[-1]


# ---------------------------------------------------------------- D_theta Q
def DthetaQ(prob, u, dP_vals, dA_vals, dq, db):
    """D_theta Q(u)[d theta] (Sec. 2.4); dP is the symmetric matrix whose
    upper triangle holds dP_vals on P's pattern, dA lives on A's pattern."""
    dP = sym_from_upper_values(prob, dP_vals)
    dA = dense_on_A_pattern(prob, dA_vals)
    x, y, tau = split(prob, u)
    return np.concatenate([
        dP @ x + dA.T @ y + tau * dq,
        -dA @ x + tau * db,
        [(-1.0 / tau) * (x @ dP @ x) - dq @ x - db @ y],
    ])


def DthetaQ_T_dense(prob, u, w):
    """D_theta Q(u)^T [w] as full dense matrices (Sec. 2.4):
    P~ = (1/2)(w1 x^T + x w1^T) - (w_N / tau) x x^T,  A~ = y w1^T - w2 x^T,
    q~ = tau w1 - w_N x,  b~ = tau w2 - w_N y."""
    x, y, tau = split(prob, u)
    w1, w2, wN = split(prob, w)
    Pt = 0.5 * (np.outer(w1, x) + np.outer(x, w1)) - (wN / tau) * np.outer(x, x)
    At = np.outer(y, w1) - np.outer(w2, x)
    qt = tau * w1 - wN * x
    bt = tau * w2 - wN * y
    return Pt, At, qt, bt


def restrict_to_patterns(prob, Pt, At):
    """Keep only the entries on the stored patterns of P (upper) and A
    (Sec. 3.2: only the non-explicit-zero entries are formed)."""
    return (Pt[prob.P.row_ids(), prob.P.indices],
            At[prob.A.row_ids(), prob.A.indices])


# ---------------------------------------------------------------- phi
def phi(prob, z):
    """phi(z) = (z_x, Pi_{K*}(z_y), Pi_{K*}(z_y) - z_y) / z_N."""
    zx, zy, zN = split(prob, z)
    py = C.proj_dual(C.cone_list(prob), zy)
    return np.concatenate([zx, py, py - zy]) / zN


def Dphi(prob, z):
    """Jacobian of phi at z (reduces to the matrix printed in Sec. 2.4 when
    z_N = 1: columns -x, -y, -s in the last position)."""
    n, m = prob.n, prob.m
    zx, zy, zN = split(prob, z)
    py = C.proj_dual(C.cone_list(prob), zy)
    D = C.dproj_dual(C.cone_list(prob), zy)
    J = np.zeros((n + 2 * m, n + m + 1))
    J[:n, :n] = np.eye(n) / zN
    J[n:n + m, n:n + m] = D / zN
    J[n + m:, n:n + m] = (D - np.eye(m)) / zN
    J[:, -1] = -np.concatenate([zx, py, py - zy]) / zN ** 2
    return J
