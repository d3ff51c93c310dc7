"""Closed-form derivatives of a strictly complementary QP (a pin).

For a QP (cone = {0}^p x R+^k) whose optimum is strictly complementary and
whose active rows are linearly independent, the active set is locally
constant, so the optimality conditions of Sec. 2.1 reduce to the linear
KKT system of an equality-constrained QP:
    [P  A_a^T] [x  ]   [-q  ]
    [A_a  0  ] [y_a] = [ b_a],   y_i = 0 off the active set, s = b - A x,
with a = zero rows plus R+ rows where y > 0.  Differentiating it gives the
reduced-KKT derivative
    [P  A_a^T] [dx  ]   [-dq - dP x - dA_a^T y_a]
    [A_a  0  ] [dy_a] = [ db_a - dA_a x         ],
    dy_i = 0 (inactive), ds_a = 0, ds_i = db_i - dA_i x - A_i dx.
These are textbook facts about QPs, independent of the homogeneous
embedding, which is what makes them a pin for the oracle.
"""
import numpy as np

from . import embedding as E

ZERO, NONNEG = 0, 1


def active_rows(prob):
    act = np.zeros(prob.m, bool)
    r = 0
    for t, d in prob.cones:
        if t == ZERO:
            act[r:r + d] = True
        elif t == NONNEG:
            act[r:r + d] = prob.y[r:r + d] > 0.0
        else:
            raise ValueError("closed form covers QPs only (zero and R+ blocks)")
        r += d
    return act


def kkt_solve(P, A, q, b, act):
    """Solve the equality-constrained QP with the active set fixed."""
    n = P.shape[0]
    Aa = A[act]
    k = Aa.shape[0]
    K = np.zeros((n + k, n + k))
    K[:n, :n] = P
    K[:n, n:] = Aa.T
    K[n:, :n] = Aa
    sol = np.linalg.solve(K, np.concatenate([-q, b[act]]))
    x = sol[:n]
    y = np.zeros(A.shape[0])
    y[act] = sol[n:]
    s = b - A @ x
    s[act] = 0.0
    return x, y, s


def jvp_kkt(prob, d):
    """Reduced-KKT derivative of (x, y, s) along d theta."""
    act = active_rows(prob)
    P = E.P_full(prob)
    A = E.A_dense(prob)
    dP = E.sym_from_upper_values(prob, d.dP)
    dA = E.dense_on_A_pattern(prob, d.dA)
    x, y = prob.x, prob.y
    n = prob.n
    Aa, dAa = A[act], dA[act]
    k = Aa.shape[0]
    K = np.zeros((n + k, n + k))
    K[:n, :n] = P
    K[:n, n:] = Aa.T
    K[n:, :n] = Aa
    rhs = np.concatenate([-d.dq - dP @ x - dAa.T @ y[act], d.db[act] - dAa @ x])
    sol = np.linalg.solve(K, rhs)
    dx = sol[:n]
    dy = np.zeros(prob.m)
    dy[act] = sol[n:]
    ds = d.db - dA @ x - A @ dx
    ds[act] = 0.0
    return dx, dy, ds


def jvp_fd(prob, d, h=1e-6):
    """Central differences of the fixed-active-set KKT solution."""
    act = active_rows(prob)
    P = E.P_full(prob)
    A = E.A_dense(prob)
    dP = E.sym_from_upper_values(prob, d.dP)
    dA = E.dense_on_A_pattern(prob, d.dA)
    plus = kkt_solve(P + h * dP, A + h * dA, prob.q + h * d.dq, prob.b + h * d.db, act)
    minus = kkt_solve(P - h * dP, A - h * dA, prob.q - h * d.dq, prob.b - h * d.db, act)
    return tuple((p - mi) / (2 * h) for p, mi in zip(plus, minus))


def jacobian_kkt(prob):
    """Dense Jacobian of theta -> (x, y, s) by the closed form, one column per
    stored value of P (upper; an off-diagonal value moves P_ij and P_ji),
    then A's stored values, q, b."""
    from qcpgen.problems import Directions
    nP, nA, n, m = prob.P.nnz, prob.A.nnz, prob.n, prob.m
    cols = []
    z = lambda k: np.zeros(k)
    for k in range(nP):
        e = z(nP); e[k] = 1.0
        cols.append(np.concatenate(jvp_kkt(prob, Directions(e, z(nA), z(n), z(m), 0, 0, 0))))
    for k in range(nA):
        e = z(nA); e[k] = 1.0
        cols.append(np.concatenate(jvp_kkt(prob, Directions(z(nP), e, z(n), z(m), 0, 0, 0))))
    for k in range(n):
        e = z(n); e[k] = 1.0
        cols.append(np.concatenate(jvp_kkt(prob, Directions(z(nP), z(nA), e, z(m), 0, 0, 0))))
    for k in range(m):
        e = z(m); e[k] = 1.0
        cols.append(np.concatenate(jvp_kkt(prob, Directions(z(nP), z(nA), z(n), e, 0, 0, 0))))
    return np.stack(cols, axis=1)


def vjp_kkt(prob, d):
    """Adjoint of the closed form, in the library's convention: the values
    returned for P are entries of a symmetric matrix at the stored upper
    positions, so the gradient with respect to a stored off-diagonal value
    is twice the returned entry."""
    J = jacobian_kkt(prob)
    w = np.concatenate([d.wx, d.wy, d.ws])
    g = J.T @ w
    nP, nA, n = prob.P.nnz, prob.A.nnz, prob.n
    diag = prob.P.row_ids() == prob.P.indices
    gP = g[:nP] / np.where(diag, 1.0, 2.0)
    return gP, g[nP:nP + nA], g[nP + nA:nP + nA + n], g[nP + nA + n:]
