"""Failure statuses of the library, reached without any GPU fault.

  * QCP_ERR_TIMEOUT: the persistent engine's grid barrier gives up after a
    bounded number of polls.  CTA 0 is held (by the global timer, bounded)
    before its first barrier, so the others' short waits run out; every CTA
    returns, the call reports the timeout, and the plan still gives the
    oracle's results afterwards.
  * QCP_BREAKDOWN: a non-finite value in a right-hand side (a NaN planted in
    the host-built direction) or in the problem data (a NaN in q, which
    enters F through its tau column and row, Sec. 2.4) makes a Krylov scalar
    non-finite; every engine reports it.
  * QCP_WARN_NEAR_KINK: a solution whose distance to a kink of D Pi
    (Appendix A) is known by construction is flagged exactly when kink_tol
    is above that distance.
"""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import g, gpu_jvp, gpu_vjp, lib, rel_err, torch
from oracle import cones as C
from oracle import derivative as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    return lib()


def _plan(q, prob, dtype=torch.float64):
    return q.qcp_plan_create(q.problem_tensors(prob, "cuda", dtype), dtype)


def test_persistent_barrier_timeout(q):
    from paper_2508_17522_gb300._native import QCPError
    prob = g.config3(0, scale=0.01)
    d = g.make_directions(prob, 41)
    ref = D.jvp_dense(prob, d)[:3]
    plan = _plan(q, prob)
    opts = q.options(rtol=1e-10, maxiter=100000, precond="equilibrate", engine="persistent")
    plan.set_barrier_wait(polls=16, hold_ns=5_000_000)
    for _ in range(2):
        with pytest.raises(QCPError, match="ERR_TIMEOUT"):
            gpu_jvp(q, plan, d, opts)
        with pytest.raises(QCPError, match="ERR_TIMEOUT"):
            gpu_vjp(q, plan, d, opts)
    # the context and the plan stay usable
    plan.set_barrier_wait(0, 0)
    jv, ji = gpu_jvp(q, plan, d, opts)
    assert ji[0]["status"] == "QCP_OK" and rel_err(jv, ref) < 1e-6, ji
    with pytest.raises(QCPError, match="ERR_ARG"):
        plan.set_barrier_wait(-1, 0)
    with pytest.raises(QCPError, match="ERR_ARG"):
        plan.set_barrier_wait(16, 2_000_000_000)
    plan.close()


@pytest.mark.parametrize("engine", ["passes", "persistent", "cluster", "stream", "auto"])
def test_nan_direction_breaks_down(q, engine):
    from paper_2508_17522_gb300._native import QCPError
    prob = g.small_qcp(43, 20, 2, 10, (3, 5))
    d = g.make_directions(prob, 42)
    bad = dataclasses.replace(d, dq=d.dq.copy(), ws=d.ws.copy())
    bad.dq[3] = np.nan
    bad.ws[1] = np.nan
    plan = _plan(q, prob)
    opts = q.options(rtol=1e-10, maxiter=2000, engine=engine)
    with pytest.raises(QCPError, match="BREAKDOWN"):
        gpu_jvp(q, plan, bad, opts)
    with pytest.raises(QCPError, match="BREAKDOWN"):
        gpu_vjp(q, plan, bad, opts)
    # the next call on the same plan is unaffected
    jv, ji = gpu_jvp(q, plan, d, opts)
    assert ji[0]["status"] == "QCP_OK" and rel_err(jv, D.jvp_dense(prob, d)[:3]) < 1e-6
    plan.close()


@pytest.mark.parametrize("engine", ["passes", "persistent", "cluster"])
@pytest.mark.parametrize("precond", ["none", "equilibrate"])
def test_nan_in_problem_data_breaks_down(q, engine, precond):
    from paper_2508_17522_gb300._native import QCPError
    prob = g.small_qcp(44, 20, 2, 10, (3, 5))
    badq = prob.q.copy()
    badq[5] = np.nan
    bad = dataclasses.replace(prob, q=badq)
    d = g.make_directions(prob, 43)
    plan = _plan(q, bad)
    opts = q.options(rtol=1e-10, maxiter=500, engine=engine, precond=precond)
    with pytest.raises(QCPError, match="BREAKDOWN"):
        gpu_jvp(q, plan, d, opts)
    with pytest.raises(QCPError, match="BREAKDOWN"):
        gpu_vjp(q, plan, d, opts)
    plan.close()


def test_near_kink_warning(q):
    """R+ rows and SOC blocks at chosen distances from their kinks: the
    reported margin is the oracle's (pinned by hand-computed cases), and the
    status turns to QCP_WARN_NEAR_KINK exactly above it, outputs unchanged."""
    prob = g.small_qcp(45, 20, 2, 10, (3, 5))
    zy = prob.y - prob.s
    want = C.kink_margin(C.cone_list(prob), zy)
    assert want > 0.1
    d = g.make_directions(prob, 44)
    ref = D.jvp_dense(prob, d)[:3]
    plan = _plan(q, prob)
    jv, ji = gpu_jvp(q, plan, d, q.options(rtol=1e-11, kink_tol=0.99 * want))
    assert ji[0]["status"] == "QCP_OK", ji
    assert abs(ji[0]["kink_margin"] - want) <= 1e-12 * want, (ji[0]["kink_margin"], want)
    for engine in ("passes", "persistent", "cluster", "stream"):
        wv, wi = gpu_jvp(q, plan, d, q.options(rtol=1e-11, kink_tol=1.01 * want, engine=engine))
        assert wi[0]["status"] == "QCP_WARN_NEAR_KINK", (engine, wi)
        assert rel_err(wv, ref) < 1e-6
        _, vi = gpu_vjp(q, plan, d, q.options(rtol=1e-11, kink_tol=1.01 * want, engine=engine))
        assert vi[0]["status"] == "QCP_WARN_NEAR_KINK", (engine, vi)
    plan.close()


def test_near_kink_margin_constructed(q):
    """An R+ row moved to |z_i| = 1e-3 and an SOC block with t - ||u|| = 2e-3
    by construction (complementarity kept): the plan reports 1e-3, the
    oracle's margin, and warns above it."""
    prob = g.small_qcp(46, 20, 0, 6, (3,), soc_mix=(0.0, 1.0))
    y, s = prob.y.copy(), prob.s.copy()
    if y[0] > 0:          # keep the row's side of the complementarity
        y[0] = 1e-3
    else:
        s[0] = 1e-3
    assert np.all(s[6:9] == 0.0)   # the SOC block holds s = 0, y interior
    u = y[7:9] / np.linalg.norm(y[7:9])
    y[6], y[7:9] = 1.0, (1.0 - 2e-3) * u
    mod = g.with_optimum(prob, prob.x, y, s)
    want = C.kink_margin(C.cone_list(mod), mod.y - mod.s)
    assert abs(want - 1e-3) < 1e-15, want
    d = g.make_directions(mod, 45)
    ref = D.jvp_dense(mod, d)[:3]
    plan = _plan(q, mod)
    jv, ji = gpu_jvp(q, plan, d, q.options(rtol=1e-10, kink_tol=1.5e-3))
    assert ji[0]["status"] == "QCP_WARN_NEAR_KINK", ji
    assert abs(ji[0]["kink_margin"] - 1e-3) < 1e-15, ji
    assert rel_err(jv, ref) < 1e-6
    _, ji = gpu_jvp(q, plan, d, q.options(rtol=1e-10, kink_tol=0.5e-3))
    assert ji[0]["status"] == "QCP_OK", ji
    plan.close()
