"""Pins for the oracle's JVP and VJP of the solution map (Sec. 3.1, 3.2).

  * strictly complementary QPs: the reduced-KKT closed form, and central
    finite differences that re-solve the KKT system with the active set fixed
  * the VJP of a QP equals the transpose of the closed-form Jacobian
  * unconstrained QP: dx = -P^{-1}(dP x + dq); equality-only QP: textbook KKT
  * SOC problems: central finite differences of the solution map, re-solved
    by Newton on the residual map alone
  * the adjoint identity <JVP(dtheta), w> = <dtheta, VJP(w)> (weight 2 on
    stored off-diagonal entries of the symmetric dP)
  * LSMR (the paper's solver) agrees with the dense bordered LU, and the
    bordering unknowns come out ~0 (both systems are consistent)
  * a mistake planted in the oracle (a flipped sign) is caught by the pins
"""
import numpy as np
import pytest

import qcpgen as g
from oracle import derivative as D
from oracle import embedding as E
from oracle import newton_fd as NF
from oracle import qp_kkt as K
from conftest import rel_err


QPS = [lambda: g.config1(0), lambda: g.config1(1),
       lambda: g.small_qcp(11, 12, 3, 10, ()), lambda: g.small_qcp(12, 20, 0, 30, (), nnz_per_row=5),
       # the paper's example shape (Sec. 4): P singular on x, a zero block after the R+ block
       lambda: g.paper_example(0, m=40, n=20)]
SOCS = [lambda: g.small_qcp(21, 10, 2, 5, (3, 4, 5)),
        lambda: g.small_qcp(22, 16, 0, 6, (3, 3, 6, 8), soc_mix=(0.5, 0.25)),
        lambda: g.small_qcp(23, 12, 1, 0, (2, 5, 7), soc_mix=(0.34, 0.33)),
        # PSD blocks (Appendix A): orders 3 and 2 with s of rank 1 and 0, and
        # orders 4 and 3 with ranks 2 and 3
        lambda: g.small_qcp(24, 14, 1, 4, (3,), psd_orders=(3, 2), psd_ranks=(1, 0)),
        lambda: g.small_qcp(25, 18, 0, 3, (), psd_orders=(4, 3), psd_ranks=(2, 3)),
        # exponential-cone blocks (Appendix A): boundary pairs and both interiors
        lambda: g.small_qcp(31, 12, 1, 3, (3,), exp_kinds=("ray", "ray", "sint", "yint")),
        # power-cone blocks of several exponents
        lambda: g.small_qcp(41, 12, 1, 3, (3,), pow_blocks=(("ray", 0.3), ("ray", 0.5), ("sint", 0.7),
                                                           ("yint", 0.4)))]


@pytest.mark.parametrize("mk", QPS)
def test_qp_closed_form_and_kkt_fd(mk):
    p = mk()
    for k in range(2):
        d = g.make_directions(p, 100 + k)
        dx, dy, ds, info = D.jvp_dense(p, d)
        kk = K.jvp_kkt(p, d)
        assert rel_err((dx, dy, ds), kk) < 1e-10
        assert rel_err(K.jvp_fd(p, d), kk) < 1e-7
        assert abs(info["lambda"]) < 1e-9


@pytest.mark.parametrize("mk", QPS[:3])
def test_qp_vjp_is_transpose_of_closed_form(mk):
    p = mk()
    d = g.make_directions(p, 7)
    got = D.vjp_dense(p, d)
    assert rel_err(got[:4], K.vjp_kkt(p, d)) < 1e-10
    assert abs(got[4]["mu"]) < 1e-9


def test_unconstrained_qp():
    p = g.unconstrained_qp(1, 7)
    d = g.make_directions(p, 1)
    dx, dy, ds, _ = D.jvp_dense(p, d)
    P = E.P_full(p)
    dP = E.sym_from_upper_values(p, d.dP)
    np.testing.assert_allclose(dx, -np.linalg.solve(P, dP @ p.x + d.dq), rtol=1e-11, atol=1e-12)
    assert dy.size == 0 and ds.size == 0
    # the adjoint: dq = -P^{-1} wx, dP = sym outer product
    gP, gA, gq, gb, _ = D.vjp_dense(p, d)
    lam = np.linalg.solve(P, d.wx)
    np.testing.assert_allclose(gq, -lam, rtol=1e-11, atol=1e-12)
    full = -0.5 * (np.outer(lam, p.x) + np.outer(p.x, lam))
    np.testing.assert_allclose(gP, full[p.P.row_ids(), p.P.indices], rtol=1e-10, atol=1e-12)


def test_equality_qp_textbook_kkt():
    p = g.equality_qp(5, 9, 4)
    d = g.make_directions(p, 2)
    P, A = E.P_full(p), E.A_dense(p)
    dP = E.sym_from_upper_values(p, d.dP)
    dA = E.dense_on_A_pattern(p, d.dA)
    Kmat = np.block([[P, A.T], [A, np.zeros((4, 4))]])
    sol = np.linalg.solve(Kmat, np.concatenate([-d.dq - dP @ p.x - dA.T @ p.y, d.db - dA @ p.x]))
    dx, dy, ds, _ = D.jvp_dense(p, d)
    np.testing.assert_allclose(dx, sol[:9], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dy, sol[9:], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(ds, 0.0, atol=1e-12)


@pytest.mark.parametrize("mk", SOCS)
def test_soc_jvp_against_newton_fd(mk):
    p = mk()
    d = g.make_directions(p, 3)
    dx, dy, ds, info = D.jvp_dense(p, d)
    fx, fy, fs, finfo = NF.jvp_fd(p, d, h=1e-6)
    assert finfo["res_plus"] < 1e-11 and finfo["res_minus"] < 1e-11
    assert rel_err((dx, dy, ds), (fx, fy, fs)) < 1e-7


@pytest.mark.parametrize("mk", QPS[:2] + SOCS)
def test_adjoint_identity(mk):
    p = mk()
    fac = D.DenseFactor(p)
    for k in range(3):
        d = g.make_directions(p, 50 + k)
        dx, dy, ds, _ = D.jvp_dense(p, d, fac)
        gP, gA, gq, gb, _ = D.vjp_dense(p, d, fac)
        c = np.where(p.P.row_ids() == p.P.indices, 1.0, 2.0)
        lhs = dx @ d.wx + dy @ d.wy + ds @ d.ws
        rhs = (c * d.dP) @ gP + d.dA @ gA + d.dq @ gq + d.db @ gb
        assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


@pytest.mark.parametrize("mk", [QPS[0], SOCS[0], SOCS[1]])
def test_lsmr_matches_dense(mk):
    p = mk()
    d = g.make_directions(p, 9)
    fac = D.DenseFactor(p)
    jd = D.jvp_dense(p, d, fac)
    jl = D.jvp_lsmr(p, d, rtol=1e-13)
    assert jl[3]["rel_residual"] < 1e-10
    assert rel_err(jl[:3], jd[:3]) < 1e-8
    vd = D.vjp_dense(p, d, fac)
    vl = D.vjp_lsmr(p, d, rtol=1e-13)
    assert rel_err(vl[:4], vd[:4]) < 1e-8


def test_planted_sign_error_is_caught(monkeypatch):
    """Flip the sign of the A~ term in D_theta Q^T: the QP pin must fail."""
    p = g.config1(0)
    d = g.make_directions(p, 7)
    good = D.vjp_dense(p, d)
    ref = K.vjp_kkt(p, d)
    assert rel_err(good[:4], ref) < 1e-10
    orig = E.DthetaQ_T_dense

    def bad(prob, u, w):
        Pt, At, qt, bt = orig(prob, u, w)
        x, y, tau = E.split(prob, u)
        w1, w2, wN = E.split(prob, w)
        return Pt, np.outer(y, w1) + np.outer(w2, x), qt, bt

    monkeypatch.setattr(E, "DthetaQ_T_dense", bad)
    assert rel_err(D.vjp_dense(p, d)[:4], ref) > 1e-3


def test_planted_transposed_operand_is_caught(monkeypatch):
    """Use D Pi^T D_u Q instead of D_u Q D Pi in F: the SOC Newton pin fails."""
    p = SOCS[0]()
    d = g.make_directions(p, 3)
    ref = NF.jvp_fd(p, d)[:3]

    def bad_F(prob, z):
        pz = E.proj_K(prob, z)
        DP = E.dproj_K(prob, z)
        return (DP.T @ E.DuQ(prob, pz) - DP + np.eye(z.size)) / z[-1]

    monkeypatch.setattr(E, "F_dense", bad_F)
    assert rel_err(D.jvp_dense(p, d)[:3], ref) > 1e-3


@pytest.mark.parametrize("mk", QPS[:2] + SOCS[:3])   # the linearised KKT system covers R+ and SOC blocks
def test_linearized_kkt_pins_dense_jvp(mk):
    """The dense JVP satisfies the differentiated optimality conditions, and
    a perturbed answer does not (so the check has teeth)."""
    from oracle import kkt_linearized as KL
    p = mk()
    d = g.make_directions(p, 17)
    dx, dy, ds, _ = D.jvp_dense(p, d)
    assert KL.relative_residual(p, d, dx, dy, ds) < 1e-11
    rng = np.random.default_rng(0)
    bad = dy + 1e-4 * np.linalg.norm(dy) * rng.standard_normal(dy.size) / np.sqrt(dy.size)
    assert KL.relative_residual(p, d, dx, bad, ds) > 1e-7


@pytest.mark.parametrize("mk", [lambda: g.config1(0), lambda: g.small_qcp(2, 14, 0, 6, (3, 5, 2, 6)),
                                lambda: g.small_qcp(25, 60, 3, 10, (40, 5), soc_mix=(0.5, 0.0))])
def test_assembled_F_and_scaled_lsmr(mk):
    """The matrix-free oracle's assembled sparse F equals the dense F (at the
    root and off it), and its Ruiz-scaled LSMR reaches the dense-LU JVP and
    VJP: the scaling changes the iterates, not the solution of the
    consistent systems.  This is the oracle the large GPU parity cases use."""
    from oracle import embedding as E
    prob = mk()
    z = E.solution_to_z(prob)
    op = D.FOperator(prob)
    assert np.max(np.abs(op.sparse().toarray() - E.F_dense(prob, z))) < 1e-13 * max(1.0, np.abs(E.F_dense(prob, z)).max())
    zp = z + 0.3 * np.random.default_rng(5).standard_normal(z.size)
    zp[-1] = 1.0
    opp = D.FOperator(prob, zp)
    assert np.max(np.abs(opp.sparse().toarray() - E.F_dense(prob, zp))) < 1e-12 * max(1.0, np.abs(E.F_dense(prob, zp)).max())
    d = g.make_directions(prob, 8)
    fac = D.DenseFactor(prob)
    rj = D.jvp_dense(prob, d, fac)[:3]
    rv = D.vjp_dense(prob, d, fac)[:4]
    j = D.jvp_lsmr(prob, d, rtol=1e-13, scale=True, op=op)
    v = D.vjp_lsmr(prob, d, rtol=1e-13, scale=True, op=op)
    for a, b in zip(j[:3], rj):
        assert np.linalg.norm(a - b) <= 1e-9 * max(np.linalg.norm(b), 1e-300)
    for a, b in zip(v[:4], rv):
        assert np.linalg.norm(a - b) <= 1e-9 * max(np.linalg.norm(b), 1e-300)
