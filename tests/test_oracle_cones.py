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
