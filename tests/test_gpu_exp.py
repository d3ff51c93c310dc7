"""The exponential and power cones (Appendix A) on the GPU: D Pi onto the
dual cone made at plan time per block (Moreau: I - D Pi_K(-z); the
exponential cone's nearest boundary ray by a scan and bisection and its
derivative from the optimality conditions' Jacobian; the power cone's root
r by bisection and the printed derivative formula) and applied as a dense
3 x 3 per pass, on the pass, persistent, stream and cluster engines (the
last two in double-float), against the CPU FP64 oracle (its own searches, pinned by membership, orthogonality and finite
differences)."""
import numpy as np
import pytest

from gpu_helpers import adjoint_gap, g, gpu_jvp, gpu_vjp, lib, rel_err, to_np, torch
from oracle import derivative as D

pytestmark = pytest.mark.gpu

TOL64 = 1e-6

EXPS = [
    ("exp4", lambda: g.small_qcp(31, 12, 1, 3, (3,), exp_kinds=("ray", "ray", "sint", "yint"))),
    ("exp_rays", lambda: g.small_qcp(32, 20, 0, 4, (), exp_kinds=("ray",) * 5)),
    ("exp_psd_soc", lambda: g.small_qcp(33, 24, 1, 4, (4,), psd_orders=(3,), psd_ranks=(1,),
                                        exp_kinds=("ray", "yint", "sint"))),
    ("pow4", lambda: g.small_qcp(41, 12, 1, 3, (3,), pow_blocks=(("ray", 0.3), ("ray", 0.5), ("sint", 0.7),
                                                                ("yint", 0.4)))),
    ("pow_exp", lambda: g.small_qcp(42, 20, 0, 3, (), exp_kinds=("ray", "ray"),
                                    pow_blocks=(("ray", 0.25), ("ray", 0.6), ("yint", 0.5)))),
]


@pytest.fixture(scope="module")
def q():
    return lib()


@pytest.mark.parametrize("precond", ["none", "equilibrate"])
@pytest.mark.parametrize("name,mk", EXPS, ids=[e[0] for e in EXPS])
def test_exp_jvp_vjp_match_oracle(q, name, mk, precond):
    prob = mk()
    d = g.make_directions(prob, 23)
    fac = D.DenseFactor(prob)
    rj = D.jvp_dense(prob, d, fac)[:3]
    rv = D.vjp_dense(prob, d, fac)[:4]
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
    for engine in ("auto", "persistent", "stream", "cluster"):
        for solver in ("lsqr", "lsmr"):
            opts = q.options(rtol=1e-11, precond=precond, engine=engine, solver=solver)
            jv, ji = gpu_jvp(q, plan, d, opts)
            vv, vi = gpu_vjp(q, plan, d, opts)
            # auto: the cluster engine (these problems fit it); the stream
            # and cluster engines apply the cones' D Pi as stored dense
            # matrices in df64
            want = {"persistent": "persistent", "stream": "stream"}.get(engine, "cluster")
            assert plan.last_engine() == want, (engine, solver, plan.last_engine())
            assert rel_err(jv, rj) < TOL64, (engine, solver, rel_err(jv, rj), ji)
            assert rel_err(vv, rv) < TOL64, (engine, solver, rel_err(vv, rv), vi)
            assert adjoint_gap(prob, d, jv, vv) < 1e-8
    with pytest.raises(RuntimeError):  # the FP64 cluster kernel has no dense D Pi
        gpu_jvp(q, plan, d, q.options(engine="cluster_fp64"))
    plan.close()


def test_exp_in_a_batch(q):
    probs = [EXPS[0][1](), g.config1(0), EXPS[2][1](), EXPS[3][1]()]
    dirs = [g.make_directions(p, 9) for p in probs]
    plan = q.qcp_batch_plan_create([q.problem_tensors(p, "cuda") for p in probs], torch.float64)
    cat = lambda name: np.concatenate([getattr(dd, name) for dd in dirs])
    opts = q.options(rtol=1e-12)
    dx, dy, ds, ji = q.qcp_derivative_jvp(plan, cat("dP"), cat("dA"), cat("dq"), cat("db"), opts)
    gP, gA, gq, gb, vi = q.qcp_derivative_vjp(plan, cat("wx"), cat("wy"), cat("ws"), opts)
    dx, dy, ds, gP, gA, gq, gb = to_np(dx, dy, ds, gP, gA, gq, gb)
    on = om = op = oa = 0
    for p, dd in zip(probs, dirs):
        fac = D.DenseFactor(p)
        assert rel_err((dx[on:on + p.n], dy[om:om + p.m], ds[om:om + p.m]), D.jvp_dense(p, dd, fac)[:3]) < TOL64
        assert rel_err((gP[op:op + p.P.nnz], gA[oa:oa + p.A.nnz], gq[on:on + p.n], gb[om:om + p.m]),
                       D.vjp_dense(p, dd, fac)[:4]) < TOL64
        on, om, op, oa = on + p.n, om + p.m, op + p.P.nnz, oa + p.A.nnz
    plan.close()


def test_pow_exponent_required(q):
    prob = EXPS[3][1]()
    bad = prob.with_values(cone_param=np.where(prob.cone_param > 0, 1.5, 0.0))
    with pytest.raises(RuntimeError):
        q.qcp_plan_create(q.problem_tensors(bad, "cuda"), torch.float64)
