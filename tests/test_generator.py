"""The seeded generator: optimality conditions hold by construction, the
active constraints have full rank, layouts are consistent, and draws are
reproducible."""
import numpy as np
import pytest

import qcpgen as g
from qcpgen.problems import _constraint_rows


def _check(p):
    Pu = p.P.to_scipy()
    assert np.all(p.P.row_ids() <= p.P.indices), "P must be upper"
    for M in (p.P, p.A, p.AT):
        assert np.all(np.diff(M.indptr) >= 0)
        for r in range(min(M.nrows, 300)):
            c = M.indices[M.indptr[r]:M.indptr[r + 1]]
            assert np.all(np.diff(c) > 0)
    np.testing.assert_array_equal(p.AT.data, p.A.data[p.AT_perm])
    assert np.array_equal(p.A.to_scipy().T.toarray() if p.m * p.n < 4e6 else 0,
                          p.AT.to_scipy().toarray() if p.m * p.n < 4e6 else 0)
    assert int(p.cone_dim.sum()) == p.m
    Pf = Pu + __import__("scipy.sparse", fromlist=["triu"]).triu(Pu, k=1).T
    A = p.A.to_scipy()
    np.testing.assert_allclose(A @ p.x + p.s, p.b, atol=1e-12 * max(1, np.abs(p.b).max(initial=0)))
    np.testing.assert_allclose(Pf @ p.x + A.T @ p.y, -p.q, atol=1e-11 * max(1, np.abs(p.q).max(initial=0)))
    assert abs(p.s @ p.y) < 1e-12 * max(1.0, np.linalg.norm(p.s) * np.linalg.norm(p.y))
    r = 0
    for bi, (t, d) in enumerate(p.cones):
        yb, sb = p.y[r:r + d], p.s[r:r + d]
        if t == g.ZERO:
            assert np.all(sb == 0)
        elif t == g.NONNEG:
            assert np.all(yb >= 0) and np.all(sb >= 0)
            assert np.all((yb > 0) ^ (sb > 0)), "strict complementarity"
        elif t == g.POW:
            from oracle.cones import in_pow, in_pow_dual
            a = p.cone_param[bi]
            assert in_pow(sb, a, 1e-12) and in_pow_dual(yb, a, 1e-12)
        elif t == g.EXP:
            from oracle.cones import in_exp, in_exp_dual
            assert in_exp(sb, 1e-12) and in_exp_dual(yb, 1e-12)
            assert np.any(yb != 0) or np.any(sb != 0)
        elif t == g.PSD:
            from oracle.cones import smat   # the oracle's own convention, as an independent check
            ly, ls = np.linalg.eigvalsh(smat(yb)), np.linalg.eigvalsh(smat(sb))
            assert ly.min() > -1e-12 and ls.min() > -1e-12
            tol = 1e-9
            assert int((ly > tol).sum()) + int((ls > tol).sum()) == ly.size, "strict complementarity"
        else:
            assert np.linalg.norm(yb[1:]) <= yb[0] + 1e-12
            assert np.linalg.norm(sb[1:]) <= sb[0] + 1e-12
            assert (yb[0] > 0) or (sb[0] > 0)
        r += d


def test_config1():
    p = g.config1(0)
    assert (p.n, p.m, p.P.nnz) == (50, 80, 1275)
    _check(p)
    C = _constraint_rows(p.A, p.cones, p.y, p.s)
    assert C.shape[0] == 50 and np.linalg.matrix_rank(C.toarray()) == 50
    q = g.config1(0)
    np.testing.assert_array_equal(p.A.data, q.A.data)
    np.testing.assert_array_equal(p.q, q.q)


@pytest.mark.slow
def test_config2():
    p = g.config2(0)
    assert (p.n, p.m) == (2000, 5500) and p.A.nnz == 44000
    assert len(p.cones) == 302
    _check(p)


def test_config3_scaled_and_small():
    p = g.config3(0, scale=0.02)
    _check(p)
    assert max(d for t, d in p.cones if t == g.SOC) <= 200
    assert min(d for t, d in p.cones if t == g.SOC) >= 3
    for p in [g.small_qcp(1, 12, 3, 6, (3, 4, 5)), g.unconstrained_qp(0, 5), g.equality_qp(2, 8, 3)]:
        _check(p)


def test_config4_subset():
    ps = g.config4(0, n_problems=3, n_range=(50, 120))
    for p in ps:
        _check(p)
        assert 1.5 * p.n - 1 <= p.m <= 3 * p.n + 1
    # problem i is drawn from its own stream
    q = g.config4(0, n_problems=1, n_range=(50, 120), first=1)[0]
    np.testing.assert_array_equal(q.q, ps[1].q)


def test_config5_family_small():
    fam = g.config5_family(0, scale=0.02)
    a, b = fam.instance(0), fam.instance(1)
    _check(a)
    _check(b)
    assert a.P is b.P and a.A is b.A
    assert not np.array_equal(a.q, b.q)


def test_fp32_rounding():
    p = g.config1(0)
    r = g.round_to_fp32(p)
    assert np.all(r.A.data == r.A.data.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(r.q - p.q)) <= 1e-6 * np.max(np.abs(p.q))


def test_paper_example_shape():
    p = g.paper_example(0, m=60, n=30)
    _check(p)
    assert (p.n, p.m) == (90, 91)
    assert p.cones == [(g.ZERO, 60), (g.NONNEG, 30), (g.ZERO, 1)]
    assert p.P.nnz == 60 and np.all(p.P.indices >= 30)         # r^T P r: diagonal on r only
    assert p.A.nnz == 60 * 30 + 60 + 30 + 30                   # [C D; E 0; f^T 0]
    assert np.all(p.x[:30] >= 0) and np.allclose(p.b[60:90], 0.0)   # x >= 0 as in the example
    C = _constraint_rows(p.A, p.cones, p.y, p.s)
    assert np.linalg.matrix_rank(C.toarray()) == C.shape[0] <= p.n


def test_psd_blocks():
    from oracle.cones import smat
    for ranks in [(1, 0), (0, 2), (3, 1), (2, 2)]:
        p = g.small_qcp(31, 14, 1, 4, (3,), psd_orders=(3, 2), psd_ranks=ranks)
        _check(p)
        assert p.cones[-2:] == [(g.PSD, 6), (g.PSD, 3)]
        C = _constraint_rows(p.A, p.cones, p.y, p.s)
        # every active direction: 1 zero row, the active R+ rows, the SOC block's,
        # and (k - r)(k - r + 1)/2 per PSD block
        assert np.linalg.matrix_rank(C.toarray()) == C.shape[0]
        # y s = 0 as matrices, not only in trace
        r = p.m - 9
        for d in (6, 3):
            assert np.allclose(smat(p.y[r:r + d]) @ smat(p.s[r:r + d]), 0.0, atol=1e-12)
            r += d


def test_exp_blocks():
    p = g.small_qcp(31, 12, 1, 3, (3,), exp_kinds=("ray", "ray", "sint", "yint"))
    _check(p)
    assert p.cones[-4:] == [(g.EXP, 3)] * 4
    C = _constraint_rows(p.A, p.cones, p.y, p.s)
    # 1 zero row, the active R+ rows, the SOC block's, 1 per boundary pair, 3 for y inside K_exp*
    assert np.linalg.matrix_rank(C.toarray()) == C.shape[0] <= p.n


def test_pow_blocks():
    p = g.small_qcp(41, 12, 1, 3, (3,), pow_blocks=(("ray", 0.3), ("ray", 0.5), ("sint", 0.7), ("yint", 0.4)))
    _check(p)
    assert p.cones[-4:] == [(g.POW, 3)] * 4 and list(p.cone_param[-4:]) == [0.3, 0.5, 0.7, 0.4]
