"""Mistakes planted in the oracle's cone code are caught by the cone pins.

Each test swaps one plausible error into `oracle.cones` (a dropped term, a
wrong index, a flipped sign, a lost scale factor, the other reading of a
garbled entry) and runs an unchanged pin from test_oracle_cones.py, which
must then fail.  The pins are properties fixed by the mathematics (finite
differences, the conditions that define a projection, the isometry of the
PSD layout, exact values built from a cone's boundary), so a pin that let
one of these through would be too weak to certify the oracle.
"""
import numpy as np
import pytest

import test_oracle_cones as pins
from oracle import cones as C


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


# ------------------------------------------------------------------ SOC
def test_soc_dropped_rank_one_term(monkeypatch):
    """D Pi_soc without its -(t / r^2)(u^T du) u term (Appendix A)."""
    orig = C.dproj_soc

    def bad(z):
        J = orig(z)
        t, u = z[0], z[1:]
        r = np.linalg.norm(u)
        if r > abs(t):
            J[1:, 1:] += (t / (2.0 * r ** 3)) * np.outer(u, u)
        return J

    monkeypatch.setattr(C, "dproj_soc", bad)
    _fails(pins.test_soc_derivative_matches_finite_differences, 3)


def test_soc_sign_of_t(monkeypatch):
    """(r - t) in place of (t + r) on the identity part of D Pi_soc."""
    orig = C.dproj_soc

    def bad(z):
        J = orig(z)
        t, u = z[0], z[1:]
        r = np.linalg.norm(u)
        if r > abs(t):
            J[1:, 1:] -= (t / r) * np.eye(z.shape[0] - 1)
        return J

    monkeypatch.setattr(C, "dproj_soc", bad)
    _fails(pins.test_soc_derivative_matches_finite_differences, 5)


# ------------------------------------------------------------------ PSD
def test_psd_wrong_index_in_B(monkeypatch):
    """lambda_j / (lambda_i - lambda_j) in place of lambda_i / (lambda_i -
    lambda_j) for a positive lambda_i and a nonpositive lambda_j."""
    def bad(lam):
        k = lam.shape[0]
        B = np.empty((k, k))
        for i in range(k):
            for j in range(k):
                pi, pj = lam[i] > 0.0, lam[j] > 0.0
                if pi == pj:
                    B[i, j] = 1.0 if pi else 0.0
                elif pi:
                    B[i, j] = lam[j] / (lam[i] - lam[j])
                else:
                    B[i, j] = lam[i] / (lam[j] - lam[i])
        return B

    monkeypatch.setattr(C, "psd_B", bad)
    _fails(pins.test_psd_derivative_fd_symmetry_homogeneity, 3)


def test_psd_layout_without_sqrt2(monkeypatch):
    """The upper triangle stored without the sqrt2 on off-diagonal entries:
    still a consistent pair of maps, but no longer an isometry, so the
    projection it induces is not orthogonal."""
    def svec(X):
        k = X.shape[0]
        return np.array([X[a, j] for j in range(k) for a in range(j + 1)])

    def smat(v):
        k = C.psd_order(v.shape[0])
        X = np.empty((k, k))
        i = 0
        for j in range(k):
            for a in range(j + 1):
                X[a, j] = X[j, a] = v[i]
                i += 1
        return X

    monkeypatch.setattr(C, "svec", svec)
    monkeypatch.setattr(C, "smat", smat)
    _fails(pins.test_psd_svec_is_an_isometry)
    _fails(pins.test_psd_moreau_and_optimality, 3)


# ---------------------------------------------------------- exponential cone
def test_exp_other_reading_of_the_garbled_entry(monkeypatch):
    """The printed (2, 2) entry of J reads "1 + -"; taking it as
    1 - mu x^2 e^{x/y} / y^3 fails the finite differences and the exact
    values, which the oracle's reading (the Hessian entry, with a plus)
    passes."""
    orig = C.exp_kkt_jacobian

    def bad(xs, ys, mu):
        J = orig(xs, ys, mu)
        J[1, 1] = 2.0 - J[1, 1]
        return J

    monkeypatch.setattr(C, "exp_kkt_jacobian", bad)
    _fails(pins.test_exp_derivative_fd_symmetry_homogeneity)
    _fails(pins.test_exp_projection_and_derivative_by_construction)


def test_exp_dual_moreau_sign(monkeypatch):
    """D Pi_{K*}(q) = I + D Pi_K(-q) in place of I - D Pi_K(-q)."""
    monkeypatch.setattr(C, "dproj_exp_dual",
                        lambda q: np.eye(3) + C.dproj_exp(-np.asarray(q, np.float64)))
    _fails(pins.test_exp_derivative_fd_symmetry_homogeneity)


def test_exp_multiplier_sign(monkeypatch):
    """The multiplier taken as z - z* instead of z* - z."""
    orig = C.exp_kkt_jacobian
    monkeypatch.setattr(C, "exp_kkt_jacobian", lambda xs, ys, mu: orig(xs, ys, -mu))
    _fails(pins.test_exp_derivative_fd_symmetry_homogeneity)
    _fails(pins.test_exp_projection_and_derivative_by_construction)


# --------------------------------------------------------------- power cone
def test_pow_exponents_swapped_in_f_y(monkeypatch):
    """f_y built with a in place of 1 - a: the projection leaves the cone or
    stops being orthogonal."""
    def bad(x, y, z, a, r):
        fx = 0.5 * (x + np.sqrt(x * x + 4 * a * r * (abs(z) - r)))
        fy = 0.5 * (y + np.sqrt(y * y + 4 * a * r * (abs(z) - r)))
        return fx, fy

    monkeypatch.setattr(C, "_pow_f", bad)
    _fails(pins.test_pow_projection_characterised, 0.2)
    _fails(pins.test_pow_projection_and_derivative_by_construction, 0.35)


def test_pow_dropped_sign_of_z(monkeypatch):
    """The derivative's (x, z) and (y, z) entries without their sign(z)."""
    orig = C.dproj_pow

    def bad(p, a):
        J = orig(p, a)
        s = np.sign(p[2]) if p[2] != 0.0 else 1.0
        J[0, 2] *= s
        J[2, 0] *= s
        J[1, 2] *= s
        J[2, 1] *= s
        return J

    monkeypatch.setattr(C, "dproj_pow", bad)
    _fails(pins.test_pow_derivative_fd_symmetry_homogeneity, 0.5)
    _fails(pins.test_pow_projection_and_derivative_by_construction, 0.5)
