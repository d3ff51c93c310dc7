"""Pins for the oracle's cone projections and their derivatives (Appendix A).

Each check uses a property fixed by the mathematics, not the oracle's own
formula: the Moreau decomposition z = Pi_{K*}(z) - Pi_K(-z) (Sec. 2.3),
membership and orthogonality of the two parts, finite differences of the
projection, symmetry of the derivative, and D Pi(z) z = Pi(z) (Pi is
positively homogeneous).
"""
import numpy as np
import pytest

from oracle import cones as C


def _soc_in(z, tol=1e-12):
    return np.linalg.norm(z[1:]) <= z[0] + tol


@pytest.mark.parametrize("d", [1, 2, 3, 7, 40])
def test_soc_moreau_and_optimality(d):
    rng = np.random.default_rng(d)
    for _ in range(200):
        z = rng.standard_normal(d) * rng.uniform(0.1, 5)
        p = C.proj_soc(z)
        pol = z - p                       # the part in the polar cone -K
        assert _soc_in(p)
        assert _soc_in(-pol)
        assert abs(p @ pol) <= 1e-12 * max(1.0, z @ z)
        # Moreau for a self-dual cone: z = Pi(z) - Pi(-z)
        np.testing.assert_allclose(p - C.proj_soc(-z), z, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3, 9])
def test_soc_projection_is_nearest_point(d):
    """Brute force: no sampled cone point is closer to z than Pi(z)."""
    rng = np.random.default_rng(100 + d)
    for _ in range(30):
        z = rng.standard_normal(d)
        p = C.proj_soc(z)
        dist = np.linalg.norm(z - p)
        u = rng.standard_normal((5000, d - 1))
        t = np.linalg.norm(u, axis=1) + np.abs(rng.standard_normal(5000)) * rng.uniform(0, 1)
        pts = np.column_stack([t, u])
        assert np.min(np.linalg.norm(pts - z, axis=1)) >= dist - 1e-12


@pytest.mark.parametrize("d", [2, 3, 5, 20])
def test_soc_derivative_matches_finite_differences(d):
    rng = np.random.default_rng(7 * d)
    h = 1e-6
    for case in range(60):
        z = rng.standard_normal(d)
        r = np.linalg.norm(z[1:])
        if abs(r - abs(z[0])) < 1e-2:
            continue
        J = C.dproj_soc(z)
        Jfd = np.column_stack([(C.proj_soc(z + h * e) - C.proj_soc(z - h * e)) / (2 * h)
                               for e in np.eye(d)])
        np.testing.assert_allclose(J, Jfd, atol=1e-7)
        np.testing.assert_allclose(J, J.T, atol=1e-15)
        np.testing.assert_allclose(J @ z, C.proj_soc(z), atol=1e-12)


def test_soc_kink_tie_break():
    """On the boundaries the cases are tested in order, non-strictly."""
    assert np.all(C.dproj_soc(np.array([0.0, 0.0, 0.0])) == 0.0)      # ||u|| <= -t, u=0, t=0
    assert np.all(C.dproj_soc(np.array([-5.0, 3.0, 4.0])) == 0.0)     # ||u|| = -t
    np.testing.assert_array_equal(C.dproj_soc(np.array([5.0, 3.0, 4.0])), np.eye(3))  # ||u|| = t
    np.testing.assert_array_equal(C.proj_soc(np.array([5.0, 3.0, 4.0])), [5.0, 3.0, 4.0])


def test_nonneg_and_zero_blocks():
    z = np.array([-2.0, -0.0, 0.0, 1e-300, 3.0])
    np.testing.assert_array_equal(C.proj_dual_block(C.NONNEG, z), [0, 0, 0, 1e-300, 3.0])
    np.testing.assert_array_equal(np.diag(C.dproj_dual_block(C.NONNEG, z)), [0, 0, 0, 1, 1])
    # the dual of {0} is R: identity projection and derivative
    np.testing.assert_array_equal(C.proj_dual_block(C.ZERO, z), z)
    np.testing.assert_array_equal(C.dproj_dual_block(C.ZERO, z), np.eye(5))
    # primal {0}: projection 0 (Appendix A, zero cone), Moreau with its dual
    np.testing.assert_array_equal(C.proj_primal_block(C.ZERO, z), 0 * z)


def test_product_cone_moreau_blockwise():
    rng = np.random.default_rng(3)
    cones = [(C.ZERO, 3), (C.NONNEG, 4), (C.SOC, 5), (C.SOC, 1), (C.NONNEG, 2), (C.SOC, 3)]
    m = sum(d for _, d in cones)
    for _ in range(50):
        z = rng.standard_normal(m)
        np.testing.assert_allclose(C.proj_dual(cones, z) - C.proj_primal(cones, -z), z, atol=1e-13)
        D = C.dproj_dual(cones, z)
        Ds = C.dproj_dual_sparse(cones, z).toarray()
        np.testing.assert_array_equal(D, Ds)
        np.testing.assert_allclose(D @ z, C.proj_dual(cones, z), atol=1e-12)


# ----------------------------------------------------------------- PSD cone
def _rand_sym_entries(rng, k, scale=1.0):
    X = rng.standard_normal((k, k)) * scale
    return C.svec((X + X.T) / 2)


def test_psd_svec_is_an_isometry():
    rng = np.random.default_rng(7)
    for k in (1, 2, 3, 5):
        a, b = _rand_sym_entries(rng, k), _rand_sym_entries(rng, k)
        assert abs(a @ b - np.trace(C.smat(a) @ C.smat(b))) <= 1e-12 * (1 + abs(a @ b))
        np.testing.assert_allclose(C.svec(C.smat(a)), a, atol=1e-15)
    # the layout: (X11, sqrt2 X12, X22, sqrt2 X13, sqrt2 X23, X33)
    X = np.array([[1.0, 2.0, 4.0], [2.0, 3.0, 5.0], [4.0, 5.0, 6.0]])
    r2 = np.sqrt(2.0)
    np.testing.assert_allclose(C.svec(X), [1.0, 2 * r2, 3.0, 4 * r2, 5 * r2, 6.0])


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_psd_moreau_and_optimality(k):
    rng = np.random.default_rng(300 + k)
    for _ in range(100):
        z = _rand_sym_entries(rng, k, rng.uniform(0.1, 5))
        p = C.proj_psd(z)
        pol = z - p
        assert np.linalg.eigvalsh(C.smat(p)).min() >= -1e-12
        assert np.linalg.eigvalsh(C.smat(-pol)).min() >= -1e-12
        assert abs(p @ pol) <= 1e-12 * max(1.0, z @ z)
        np.testing.assert_allclose(p - C.proj_psd(-z), z, atol=1e-12)


@pytest.mark.parametrize("k", [2, 3])
def test_psd_projection_is_nearest_point(k):
    """Brute force over sampled PSD matrices: none is closer than Pi(z)."""
    rng = np.random.default_rng(400 + k)
    for _ in range(20):
        z = _rand_sym_entries(rng, k)
        dist = np.linalg.norm(z - C.proj_psd(z))
        G = rng.standard_normal((4000, k, k))
        cand = np.einsum("nij,nkj->nik", G, G) * rng.uniform(0, 2, (4000, 1, 1))
        dists = [np.linalg.norm(z - C.svec(M)) for M in cand]
        assert min(dists) >= dist - 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_psd_derivative_fd_symmetry_homogeneity(k):
    rng = np.random.default_rng(500 + k)
    for _ in range(20):
        z = _rand_sym_entries(rng, k)
        lam = np.linalg.eigvalsh(C.smat(z))
        if np.min(np.abs(lam)) < 1e-3:
            continue
        J = C.dproj_psd(z)
        h = 1e-6
        for _ in range(3):
            v = rng.standard_normal(z.shape[0])
            fd = (C.proj_psd(z + h * v) - C.proj_psd(z - h * v)) / (2 * h)
            np.testing.assert_allclose(J @ v, fd, atol=2e-7 * (1 + np.abs(fd).max()))
        np.testing.assert_allclose(J, J.T, atol=1e-13)
        np.testing.assert_allclose(J @ z, C.proj_psd(z), atol=1e-12 * (1 + np.abs(z).max()))


def test_psd_derivative_special_cases():
    """Diagonal Z: D maps the (a, b) entry to B_ab times itself, with B the
    divided differences of max(., 0); a PSD Z gives the identity, a negative
    definite Z gives 0."""
    lam = np.array([2.0, -1.0, 0.5])
    z = C.svec(np.diag(lam))
    J = C.dproj_psd(z)
    i = 0
    for j in range(3):
        for a in range(j + 1):
            li, lj = lam[a], lam[j]
            pa, pj = max(li, 0), max(lj, 0)
            want = 1.0 if li == lj and li > 0 else (pa - pj) / (li - lj) if li != lj else 0.0
            assert abs(J[i, i] - want) < 1e-13, (a, j, J[i, i], want)
            assert np.allclose(np.delete(J[i], i), 0.0, atol=1e-13)
            i += 1
    rng = np.random.default_rng(3)
    G = rng.standard_normal((4, 4))
    np.testing.assert_allclose(C.dproj_psd(C.svec(G @ G.T + 0.1 * np.eye(4))), np.eye(10), atol=1e-12)
    np.testing.assert_allclose(C.dproj_psd(C.svec(-(G @ G.T + 0.1 * np.eye(4)))), np.zeros((10, 10)), atol=1e-12)


# ------------------------------------------------------- exponential cone
def test_exp_projection_characterised():
    """Pi(p) in K_exp, Pi(p) - p in K_exp* (p - Pi(p) in the polar cone) and
    the two orthogonal: the conditions that define the projection onto a
    closed convex cone; and the same for the dual cone's projection."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        p = rng.standard_normal(3) * rng.uniform(0.1, 4)
        P = C.proj_exp(p)
        s = max(1.0, np.linalg.norm(p))
        assert C.in_exp(P, 1e-9 * s), (p, P)
        assert C.in_exp_dual(P - p, 1e-9 * s), (p, P)
        assert abs(P @ (P - p)) <= 1e-10 * s * s
        Q = C.proj_exp_dual(p)
        assert C.in_exp_dual(Q, 1e-9 * s) and C.in_exp(Q - p, 1e-9 * s)
        assert abs(Q @ (Q - p)) <= 1e-10 * s * s


def test_exp_projection_is_nearest_point():
    """Brute force over sampled points of K_exp (its rays and its face)."""
    rng = np.random.default_rng(12)
    r = rng.uniform(-6, 6, 20000)
    t = rng.exponential(2.0, 20000)
    pts = np.stack([t * r, t, t * np.exp(r)], 1)
    face = np.stack([-rng.exponential(2.0, 5000), np.zeros(5000), rng.exponential(2.0, 5000)], 1)
    cand = np.concatenate([pts, face])
    for _ in range(30):
        p = rng.standard_normal(3) * 2
        d = np.linalg.norm(C.proj_exp(p) - p)
        assert np.min(np.linalg.norm(cand - p, axis=1)) >= d - 1e-9


def test_exp_derivative_fd_symmetry_homogeneity():
    rng = np.random.default_rng(13)
    seen = 0
    for _ in range(200):
        p = rng.standard_normal(3) * 2
        if C.in_exp(p, 1e-3) or C.in_exp_dual(-p, 1e-3) or (p[0] < 0 and p[1] < 0):
            continue
        seen += 1
        J = C.dproj_exp(p)
        h = 1e-6
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            fd = (C.proj_exp(p + e) - C.proj_exp(p - e)) / (2 * h)
            np.testing.assert_allclose(J[:, k], fd, atol=1e-6 * (1 + np.abs(fd).max()))
        np.testing.assert_allclose(J, J.T, atol=1e-9)
        np.testing.assert_allclose(J @ p, C.proj_exp(p), atol=1e-9 * (1 + np.abs(p).max()))
        Jd = C.dproj_exp_dual(p)
        fd = np.stack([(C.proj_exp_dual(p + h * e) - C.proj_exp_dual(p - h * e)) / (2 * h) for e in np.eye(3)], 1)
        np.testing.assert_allclose(Jd, fd, atol=1e-6 * (1 + np.abs(fd).max()))
    assert seen > 50


def _exp_by_construction(t, r, mu):
    """A point with a known projection onto K_exp and the exact Jacobian of
    that projection, from the boundary parametrisation alone.

    a(r) = (r, 1, e^r) spans a boundary ray of K_exp and n(r) = (-e^r,
    (r - 1) e^r, 1) lies on the boundary of K_exp* with <a, n> = 0, so for
    t, mu > 0 the point p = t a(r) - mu n(r) projects to t a(r) (it meets the
    three conditions of a projection onto a closed convex cone).  Along the
    map theta = (t, r, mu) -> p the projection is theta -> t a(r), so
    D Pi(p) = [dPi/dtheta] [dp/dtheta]^-1 exactly."""
    e = np.exp(r)
    a, n = np.array([r, 1.0, e]), np.array([-e, (r - 1.0) * e, 1.0])
    da, dn = np.array([1.0, 0.0, e]), np.array([-e, r * e, 0.0])
    dp = np.stack([a, t * da - mu * dn, -n], 1)
    dpi = np.stack([a, t * da, np.zeros(3)], 1)
    return t * a - mu * n, t * a, dpi @ np.linalg.inv(dp), dp


def test_exp_projection_and_derivative_by_construction():
    """Exact values, not finite differences: the oracle's Pi and D Pi (its
    ray search and the J of Appendix A) agree with the boundary
    parametrisation to rounding.  The parametrisation's own derivative is
    checked by differences first."""
    rng = np.random.default_rng(14)
    for lo, hi in ((-30.0, -4.0), (-4.0, 3.0), (3.0, 8.0)):
        for _ in range(60):
            th = np.array([np.exp(rng.uniform(-3, 3)), rng.uniform(lo, hi), np.exp(rng.uniform(-3, 3))])
            p, P, D, dp = _exp_by_construction(*th)
            h = 1e-6 * (1 + np.abs(th))
            fd = np.stack([(_exp_by_construction(*(th + h[k] * e))[0] -
                            _exp_by_construction(*(th - h[k] * e))[0]) / (2 * h[k]) for k, e in enumerate(np.eye(3))], 1)
            np.testing.assert_allclose(fd, dp, atol=1e-6 * (1 + np.abs(dp).max()))
            np.testing.assert_allclose(C.proj_exp(p), P, atol=1e-12 * (1 + np.abs(P).max()))
            np.testing.assert_allclose(C.dproj_exp(p), D, atol=1e-10)
            # the dual cone by the Moreau decomposition: -p projects onto K* at mu n
            np.testing.assert_allclose(C.dproj_exp_dual(-p), np.eye(3) - D, atol=1e-10)


def test_exp_special_cases():
    """Inside K: identity; inside the polar cone: 0; x, y < 0: (x, 0, z+)."""
    p_in = np.array([0.0, 1.0, 2.0])            # 1 * exp(0) = 1 <= 2
    np.testing.assert_allclose(C.proj_exp(p_in), p_in)
    np.testing.assert_allclose(C.dproj_exp(p_in), np.eye(3))
    p_pol = -np.array([-1.0, 0.0, 1.0])          # -(u, v, w) with u < 0, -u exp(v/u) = 1 <= e
    np.testing.assert_allclose(C.proj_exp(p_pol), np.zeros(3))
    np.testing.assert_allclose(C.dproj_exp(p_pol), np.zeros((3, 3)))
    p_neg = np.array([-2.0, -1.0, 3.0])
    assert not C.in_exp(p_neg) and not C.in_exp_dual(-p_neg)
    np.testing.assert_allclose(C.proj_exp(p_neg), [-2.0, 0.0, 3.0])
    np.testing.assert_allclose(C.dproj_exp(p_neg), np.diag([1.0, 0.0, 1.0]))


# ------------------------------------------------------------ power cone
@pytest.mark.parametrize("a", [0.2, 0.5, 0.75])
def test_pow_projection_characterised(a):
    rng = np.random.default_rng(int(100 * a))
    for _ in range(200):
        p = rng.standard_normal(3) * rng.uniform(0.1, 4)
        s = max(1.0, np.linalg.norm(p))
        P = C.proj_pow(p, a)
        assert C.in_pow(P, a, 1e-9 * s) and C.in_pow_dual(P - p, a, 1e-9 * s), (p, P)
        assert abs(P @ (P - p)) <= 1e-10 * s * s
        Q = C.proj_pow_dual(p, a)
        assert C.in_pow_dual(Q, a, 1e-9 * s) and C.in_pow(Q - p, a, 1e-9 * s)


def test_pow_projection_is_nearest_point():
    rng = np.random.default_rng(21)
    a = 0.35
    u = rng.exponential(2.0, (30000, 2))
    cand = np.concatenate([u, (u[:, :1] ** a * u[:, 1:] ** (1 - a)) * rng.uniform(-1, 1, (30000, 1))], 1)
    for _ in range(30):
        p = rng.standard_normal(3) * 2
        d = np.linalg.norm(C.proj_pow(p, a) - p)
        assert np.min(np.linalg.norm(cand - p, axis=1)) >= d - 1e-9


@pytest.mark.parametrize("a", [0.2, 0.5, 0.75])
def test_pow_derivative_fd_symmetry_homogeneity(a):
    rng = np.random.default_rng(int(1000 * a))
    seen = 0
    for _ in range(200):
        p = rng.standard_normal(3) * 2
        if C.in_pow(p, a, 1e-3) or C.in_pow_dual(-p, a, 1e-3) or abs(p[2]) < 1e-3:
            continue
        seen += 1
        J = C.dproj_pow(p, a)
        h = 1e-6
        fd = np.stack([(C.proj_pow(p + h * e, a) - C.proj_pow(p - h * e, a)) / (2 * h) for e in np.eye(3)], 1)
        np.testing.assert_allclose(J, fd, atol=2e-6 * (1 + np.abs(fd).max()))
        np.testing.assert_allclose(J, J.T, atol=1e-12)
        np.testing.assert_allclose(J @ p, C.proj_pow(p, a), atol=1e-9 * (1 + np.abs(p).max()))
    assert seen > 50


def _pow_by_construction(u, v, mu, a):
    """The power cone's analogue of _exp_by_construction: b(u, v) = (u, v,
    w), w = u^a v^(1-a), is on the boundary of K_pow,a; n(u, v) = (a w / u,
    (1 - a) w / v, -1) is on the boundary of K_pow,a* with <b, n> = 0; so
    p = b - mu n projects to b, and D Pi(p) = [dPi/dtheta] [dp/dtheta]^-1
    along theta = (u, v, mu)."""
    w = u ** a * v ** (1 - a)
    b = np.array([u, v, w])
    n = np.array([a * w / u, (1 - a) * w / v, -1.0])
    bu, bv = np.array([1.0, 0.0, a * w / u]), np.array([0.0, 1.0, (1 - a) * w / v])
    nu = np.array([a * (a - 1) * w / u ** 2, a * (1 - a) * w / (u * v), 0.0])
    nv = np.array([a * (1 - a) * w / (u * v), -a * (1 - a) * w / v ** 2, 0.0])
    dp = np.stack([bu - mu * nu, bv - mu * nv, -n], 1)
    dpi = np.stack([bu, bv, np.zeros(3)], 1)
    return b - mu * n, b, dpi @ np.linalg.inv(dp), dp


@pytest.mark.parametrize("a", [0.1, 0.35, 0.5, 0.9])
def test_pow_projection_and_derivative_by_construction(a):
    """Exact values for the root search and Hien's formula, on both signs of
    z (the cone is symmetric under z -> -z)."""
    rng = np.random.default_rng(int(1000 * a) + 7)
    S = np.diag([1.0, 1.0, -1.0])
    for _ in range(60):
        th = np.exp(rng.uniform(-3, 3, 3))
        p, P, D, dp = _pow_by_construction(*th, a)
        h = 1e-6 * th
        fd = np.stack([(_pow_by_construction(*(th + h[k] * e), a)[0] -
                        _pow_by_construction(*(th - h[k] * e), a)[0]) / (2 * h[k]) for k, e in enumerate(np.eye(3))], 1)
        np.testing.assert_allclose(fd, dp, atol=1e-6 * (1 + np.abs(dp).max()))
        np.testing.assert_allclose(C.proj_pow(p, a), P, atol=1e-12 * (1 + np.abs(P).max()))
        np.testing.assert_allclose(C.dproj_pow(p, a), D, atol=1e-11)
        np.testing.assert_allclose(C.proj_pow(S @ p, a), S @ P, atol=1e-12 * (1 + np.abs(P).max()))
        np.testing.assert_allclose(C.dproj_pow(S @ p, a), S @ D @ S, atol=1e-11)


def test_pow_special_cases():
    a = 0.5
    np.testing.assert_allclose(C.dproj_pow(np.array([1.0, 4.0, 1.0]), a), np.eye(3))   # 1^.5 4^.5 = 2 >= 1
    np.testing.assert_allclose(C.dproj_pow(np.array([-1.0, -4.0, 0.5]), a), np.zeros((3, 3)))
    # z = 0 off both cones: (x+, y+, 0); d from the case table, d_x = x / (2|y| + x) at a = 1/2
    p = np.array([2.0, -1.0, 0.0])
    np.testing.assert_allclose(C.proj_pow(p, a), [2.0, 0.0, 0.0])
    np.testing.assert_allclose(C.dproj_pow(p, a), np.diag([1.0, 0.0, 2.0 / 4.0]))
    h = 1e-6
    fd = (C.proj_pow(p + [0, 0, h], a) - C.proj_pow(p - [0, 0, h], a)) / (2 * h)
    np.testing.assert_allclose(fd, [0.0, 0.0, 0.5], atol=1e-4)     # the case table's d_x, by differences
    np.testing.assert_allclose(C.dproj_pow(p, 0.7), np.diag([1.0, 0.0, 1.0]))
    np.testing.assert_allclose(C.dproj_pow(p, 0.3), np.diag([1.0, 0.0, 0.0]))
    for aa, want in ((0.7, 1.0), (0.3, 0.0)):
        fd = (C.proj_pow(p + [0, 0, h], aa) - C.proj_pow(p - [0, 0, h], aa)) / (2 * h)
        assert abs(fd[2] - want) < 1e-3, (aa, fd)
