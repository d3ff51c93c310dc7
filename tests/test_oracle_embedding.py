"""Pins for the oracle's embedding, residual map and derivative operators.

  * R(z) = 0 at the constructed root (Sec. 2.3: N(z) = 0 iff z solves the pair)
  * F z = 0: R is positively homogeneous (Sec. 2.3), so F z = R(z) = 0
  * F equals the finite-difference Jacobian of N (Sec. 2.4 defines F = D_z N)
    -- also at points away from the root, with tau != 1 and z_N != 1
  * D_theta N is exact: N is affine in theta (Sec. 2.4), so
    N(z, theta + dtheta) - N(z, theta) = D_theta N[dtheta] to rounding
  * the printed adjoint D_theta Q^T is the adjoint of D_theta Q
  * D phi equals the finite-difference Jacobian of phi, and D phi(z) z = 0
  * the matrix-free operator agrees with the dense F and F^T
"""
import numpy as np
import pytest

import qcpgen as g
from oracle import derivative as D
from oracle import embedding as E


def _problems():
    return [g.config1(0), g.small_qcp(1, 9, 2, 4, (3, 4)), g.small_qcp(2, 14, 0, 6, (3, 5, 2, 6)),
            g.unconstrained_qp(0, 6), g.equality_qp(3, 8, 5)]


@pytest.fixture(scope="module", params=range(5))
def prob(request):
    return _problems()[request.param]


def test_root_and_null_vector(prob):
    z = E.solution_to_z(prob)
    assert np.linalg.norm(E.residual_map(prob, z)) < 1e-12 * max(1, np.linalg.norm(z))
    F = E.F_dense(prob, z)
    assert np.linalg.norm(F @ z) < 1e-12 * np.linalg.norm(F) * np.linalg.norm(z)


def _fd_jac(fun, z, h=1e-6):
    return np.column_stack([(fun(z + h * e) - fun(z - h * e)) / (2 * h) for e in np.eye(z.size)])


def test_F_is_jacobian_of_normalized_residual(prob):
    """At roots (the constructed one and a scaled copy, tau = z_N != 1) F is
    the Jacobian of N; anywhere Pi is differentiable z_N F is the Jacobian of
    R by the chain rule (the two differ by R(z) e_N^T / z_N^2, zero at roots)."""
    rng = np.random.default_rng(0)
    z0 = E.solution_to_z(prob)
    for pt in range(3):
        z = z0 * (1.0 if pt == 0 else rng.uniform(0.5, 2.0))
        if pt == 2:
            z = z + 0.05 * rng.standard_normal(z.size)
            z[-1] = abs(z[-1])
        F = E.F_dense(prob, z)
        if pt < 2:
            J = _fd_jac(lambda v: E.normalized_residual(prob, v), z)
            assert np.max(np.abs(F - J)) < 1e-6 * max(1.0, np.max(np.abs(F)))
        J = _fd_jac(lambda v: E.residual_map(prob, v), z)
        assert np.max(np.abs(z[-1] * F - J)) < 1e-6 * max(1.0, np.max(np.abs(J)))


def test_dtheta_N_is_exact_difference(prob):
    d = g.make_directions(prob, 5)
    rng = np.random.default_rng(1)
    z = E.solution_to_z(prob) * rng.uniform(0.5, 2.0)
    th0 = {"P": E.P_full(prob), "A": E.A_dense(prob), "q": prob.q, "b": prob.b}
    th1 = {"P": th0["P"] + E.sym_from_upper_values(prob, d.dP),
           "A": th0["A"] + E.dense_on_A_pattern(prob, d.dA),
           "q": prob.q + d.dq, "b": prob.b + d.db}
    diff = E.normalized_residual(prob, z, th1) - E.normalized_residual(prob, z, th0)
    lin = D.d_theta_N(prob, z, d.dP, d.dA, d.dq, d.db)
    np.testing.assert_allclose(lin, diff, atol=1e-11 * max(1, np.max(np.abs(diff))))
    np.testing.assert_allclose(D.d_theta_N_sparse(prob, z, d.dP, d.dA, d.dq, d.db), lin,
                               atol=1e-12 * max(1, np.max(np.abs(lin))))


def test_dtheta_adjoint(prob):
    """<D_theta N[dtheta], w> = <dtheta, D_theta N^T[w]> with the Frobenius
    product of the full symmetric dP (weight 2 on stored off-diagonals)."""
    d = g.make_directions(prob, 6)
    rng = np.random.default_rng(2)
    z = E.solution_to_z(prob) * rng.uniform(0.5, 2.0)
    w = rng.standard_normal(prob.N)
    lhs = D.d_theta_N(prob, z, d.dP, d.dA, d.dq, d.db) @ w
    gP, gA, gq, gb = D.d_theta_N_T(prob, z, w)
    c = np.where(prob.P.row_ids() == prob.P.indices, 1.0, 2.0)
    rhs = (c * d.dP) @ gP + d.dA @ gA + d.dq @ gq + d.db @ gb
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))
    sP, sA, sq, sb = D.d_theta_N_T_sparse(prob, z, w)
    np.testing.assert_allclose(np.concatenate([sP, sA, sq, sb]),
                               np.concatenate([gP, gA, gq, gb]), atol=1e-12)


def test_dphi(prob):
    z = E.solution_to_z(prob)
    J = E.Dphi(prob, z)
    np.testing.assert_allclose(J, _fd_jac(lambda v: E.phi(prob, v), z), atol=1e-7)
    assert np.linalg.norm(J @ z) < 1e-12 * np.linalg.norm(z)
    # phi(z) returns the optimum at the constructed root
    np.testing.assert_allclose(E.phi(prob, z), np.concatenate([prob.x, prob.y, prob.s]), atol=1e-14)
    dz = np.random.default_rng(3).standard_normal(z.size)
    np.testing.assert_allclose(np.concatenate(D._phi_apply(prob, z, dz)), J @ dz, atol=1e-12)
    w = np.random.default_rng(4).standard_normal(prob.n + 2 * prob.m)
    n, m = prob.n, prob.m
    np.testing.assert_allclose(D._phi_apply_T(prob, z, w[:n], w[n:n + m], w[n + m:]), J.T @ w,
                               atol=1e-12)


def test_matrix_free_operator(prob):
    rng = np.random.default_rng(9)
    z = E.solution_to_z(prob)
    F = E.F_dense(prob, z)
    op = D.FOperator(prob)
    for _ in range(3):
        v = rng.standard_normal(prob.N)
        np.testing.assert_allclose(op.matvec(v), F @ v, atol=1e-12 * np.linalg.norm(F) * np.linalg.norm(v))
        np.testing.assert_allclose(op.rmatvec(v), F.T @ v, atol=1e-12 * np.linalg.norm(F) * np.linalg.norm(v))


def test_F_dense_sparse_branch():
    """Above 3000 rows F_dense forms D_u Q D Pi with D Pi held sparse; on a
    problem just above that size (N = 3101, SOC and R+ blocks) it equals the
    dense product, F z = 0 at the root, and a point off the root (another
    D Pi pattern) agrees too."""
    prob = g.small_qcp(5, 1000, 100, 1500, (10,) * 40 + (20,) * 5)
    z = E.solution_to_z(prob)
    assert z.size == 3101
    Fs = E.F_dense(prob, z)                    # the sparse branch (N > 3000)
    Fd = E.F_dense(prob, z, dense_limit=10 ** 9)
    assert np.max(np.abs(Fs - Fd)) <= 1e-14 * np.max(np.abs(Fd))
    assert np.linalg.norm(Fs @ z) < 1e-12 * np.linalg.norm(Fs) * np.linalg.norm(z)
    zp = z + 0.3 * np.random.default_rng(1).standard_normal(z.size)
    zp[-1] = 1.0
    assert np.max(np.abs(E.F_dense(prob, zp) - E.F_dense(prob, zp, dense_limit=10 ** 9))) <= \
        1e-14 * np.max(np.abs(E.F_dense(prob, zp, dense_limit=10 ** 9)))
