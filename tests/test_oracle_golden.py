"""The oracle against hand-derived closed forms stored in tests/golden.

The paper prints no numerical example; these fixtures are small problems
whose solution map has a closed form (derivations inside the JSON file):
SOC projections (Appendix A), scalar QPs with an active and an inactive
constraint (Sec. 2.1), and a QCP whose solution is a projection onto the SOC.
"""
import json
import os

import numpy as np

from qcpgen.problems import Directions, NONNEG, SOC
from oracle import cones as C
from oracle import derivative as D
from handmade import qcp_from_dense

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


def test_soc_projection_golden():
    g = GOLD["soc_projection"]
    for case in g["cases"]:
        np.testing.assert_allclose(C.proj_soc(np.array(case["z"])), case["proj"], atol=1e-15)
    np.testing.assert_allclose(C.dproj_soc(np.array(g["dproj_at"])), g["dproj"], atol=1e-15)


def _scalar(gq):
    return qcp_from_dense([[gq["P"]]], [[gq["A"]]], [gq["q"]], [gq["b"]], [(NONNEG, 1)],
                          [gq["x"]], [gq["y"]], [gq["s"]])


def test_scalar_qp_active_golden():
    gq = GOLD["scalar_qp_active"]
    p = _scalar(gq)
    dt = gq["dtheta"]
    d = Directions(np.array([dt["dP"]]), np.array([dt["dA"]]), np.array([dt["dq"]]),
                   np.array([dt["db"]]), np.array([gq["w"]["wx"]]), np.array([gq["w"]["wy"]]),
                   np.array([gq["w"]["ws"]]))
    dx, dy, ds, _ = D.jvp_dense(p, d)
    np.testing.assert_allclose([dx[0], dy[0], ds[0]], [gq["jvp"]["dx"], gq["jvp"]["dy"], gq["jvp"]["ds"]],
                               atol=1e-12)
    gP, gA, gq_, gb, _ = D.vjp_dense(p, d)
    v = gq["vjp"]
    np.testing.assert_allclose([gP[0], gA[0], gq_[0], gb[0]], [v["dP"], v["dA"], v["dq"], v["db"]],
                               atol=1e-12)


def test_scalar_qp_inactive_golden():
    gq = GOLD["scalar_qp_inactive"]
    p = _scalar(gq)
    dt = gq["dtheta"]
    d = Directions(np.array([dt["dP"]]), np.array([dt["dA"]]), np.array([dt["dq"]]),
                   np.array([dt["db"]]), np.zeros(1), np.zeros(1), np.zeros(1))
    dx, dy, ds, _ = D.jvp_dense(p, d)
    np.testing.assert_allclose([dx[0], dy[0], ds[0]], [gq["jvp"]["dx"], gq["jvp"]["dy"], gq["jvp"]["ds"]],
                               atol=1e-12)


def test_soc_projection_problem_golden():
    gq = GOLD["soc_projection_problem"]
    p = qcp_from_dense(np.eye(3), -np.eye(3), gq["q"], [0.0, 0.0, 0.0], [(SOC, 3)],
                       gq["x"], gq["y"], gq["s"])
    d = Directions(np.zeros(p.P.nnz), np.zeros(p.A.nnz), np.array(gq["dq"]), np.zeros(3),
                   np.zeros(3), np.zeros(3), np.zeros(3))
    dx, dy, ds, _ = D.jvp_dense(p, d)
    j = gq["jvp"]
    np.testing.assert_allclose(dx, j["dx"], atol=1e-12)
    np.testing.assert_allclose(dy, j["dy"], atol=1e-12)
    np.testing.assert_allclose(ds, j["ds"], atol=1e-12)


def test_psd_projection_golden():
    g = GOLD["psd_projection"]
    np.testing.assert_allclose(C.proj_psd(np.array(g["z"])), g["proj"], atol=1e-14)
    np.testing.assert_allclose(C.dproj_psd(np.array(g["z"])) @ np.array(g["dproj_dir"]), g["dproj_times_dir"],
                               atol=1e-14)
    np.testing.assert_allclose(C.dproj_psd(np.array(g["z_diag"])), g["dproj_diag"], atol=1e-14)


def test_exp_projection_golden():
    """Hand-derived values on the exponential cone (fixture: its derivation)."""
    g = GOLD["exp_projection"]
    p = np.array(g["p"])
    np.testing.assert_allclose(C.proj_exp(p), g["proj"], atol=1e-14)
    np.testing.assert_allclose(C.dproj_exp(p), g["dproj"], atol=1e-13)
    # the dual cone by the Moreau decomposition: -p projects onto K_exp* at mu n
    np.testing.assert_allclose(C.proj_exp_dual(-p), -p + np.array(g["proj"]), atol=1e-14)
    np.testing.assert_allclose(C.dproj_exp_dual(-p), np.eye(3) - np.array(g["dproj"]), atol=1e-13)


def test_pow_projection_golden():
    """Hand-derived values on the power cone at a = 1/2, both signs of z."""
    g = GOLD["pow_projection"]
    p, a = np.array(g["p"]), g["a"]
    S = np.diag([1.0, 1.0, -1.0])
    np.testing.assert_allclose(C.proj_pow(p, a), g["proj"], atol=1e-14)
    np.testing.assert_allclose(C.dproj_pow(p, a), g["dproj"], atol=1e-13)
    np.testing.assert_allclose(C.proj_pow(S @ p, a), S @ np.array(g["proj"]), atol=1e-14)
    np.testing.assert_allclose(C.dproj_pow(S @ p, a), S @ np.array(g["dproj"]) @ S, atol=1e-13)


def test_kink_margin_golden():
    """Hand-computed distances to the kinks of D Pi (fixture: the reason for
    each value); among them both boundary rays of the second-order cone."""
    for case in GOLD["kink_margin"]["cases"]:
        cones = [tuple(c) for c in case["cones"]]
        got = C.kink_margin(cones, np.array(case["z"]))
        assert abs(got - case["margin"]) <= 1e-14, (case, got)
