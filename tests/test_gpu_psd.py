"""The positive semidefinite cone (Appendix A) on the GPU: D Pi_psd = V (B o
(V^T dZ V)) V^T with the eigendecomposition made at plan time, on the pass
and persistent engines, and on the stream and cluster engines as the dense
matrix of that map (made at plan time from the same V and B, applied in
double-float), against the CPU FP64 oracle (which uses its own
eigendecomposition and the same formula, and is pinned by finite
differences of re-solves)."""
import numpy as np
import pytest

from gpu_helpers import adjoint_gap, g, gpu_jvp, gpu_vjp, lib, rel_err, to_np, torch
from oracle import derivative as D

pytestmark = pytest.mark.gpu

TOL64 = 1e-6

PSDS = [
    ("psd3_psd2", lambda: g.small_qcp(24, 14, 1, 4, (3,), psd_orders=(3, 2), psd_ranks=(1, 0))),
    ("psd4_psd3", lambda: g.small_qcp(25, 18, 0, 3, (), psd_orders=(4, 3), psd_ranks=(2, 3))),
    ("psd1_to_6", lambda: g.small_qcp(26, 30, 2, 6, (4,), psd_orders=(1, 2, 5, 6), psd_ranks=(0, 1, 2, 4))),
    ("psd_order_12", lambda: g.small_qcp(27, 60, 0, 4, (), psd_orders=(12,), psd_ranks=(7,))),
]


@pytest.fixture(scope="module")
def q():
    return lib()


@pytest.mark.parametrize("precond", ["none", "equilibrate", "jacobi"])
@pytest.mark.parametrize("name,mk", PSDS, ids=[p[0] for p in PSDS])
def test_psd_jvp_vjp_match_oracle(q, name, mk, precond):
    prob = mk()
    d = g.make_directions(prob, 21)
    fac = D.DenseFactor(prob)
    rj = D.jvp_dense(prob, d, fac)[:3]
    rv = D.vjp_dense(prob, d, fac)[:4]
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
    for engine in ("auto", "persistent", "stream", "cluster"):
        for solver in ("lsqr", "lsmr"):
            if engine == "stream" and precond == "jacobi":
                continue  # the stream engine runs unscaled or equilibrated
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
            for inf in (ji[0], vi[0]):
                assert inf["status"] in ("QCP_OK", "QCP_NOT_CONVERGED"), inf
                assert inf["rel_residual"] <= (1e-11 if inf["status"] == "QCP_OK" else 1e-8), inf
                assert inf["kink_margin"] > 0.0
            assert adjoint_gap(prob, d, jv, vv) < 1e-8
    plan.close()


def test_psd_plan_rules(q):
    """The FP64 cluster kernel refuses PSD plans, the kink margin is the smallest
    |eigenvalue| of z_y on the PSD blocks (or a smaller R+/SOC margin), and
    malformed PSD sizes are rejected."""
    from oracle import cones as C
    prob = PSDS[0][1]()
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
    d = g.make_directions(prob, 3)
    with pytest.raises(RuntimeError):
        gpu_jvp(q, plan, d, q.options(engine="cluster_fp64"))
    _, info = gpu_jvp(q, plan, d, q.options(rtol=1e-10))
    zy = prob.y - prob.s
    want = C.kink_margin(prob.cones, zy)
    assert abs(info[0]["kink_margin"] - want) <= 1e-12 * max(1.0, want), (info[0]["kink_margin"], want)
    plan.close()
    bad = prob.with_values(cone_dim=np.array([1, 4, 3, 5, 4], np.int32))  # 5 and 4 are not k (k + 1) / 2
    with pytest.raises(RuntimeError):
        q.qcp_plan_create(q.problem_tensors(bad, "cuda"), torch.float64)


def test_psd_in_a_batch_with_other_problems(q):
    probs = [PSDS[1][1](), g.config1(0), g.small_qcp(42, 33, 0, 20, (4, 4, 12), soc_mix=(0.5, 0.2)), PSDS[2][1]()]
    dirs = [g.make_directions(p, 9) for p in probs]
    plan = q.qcp_batch_plan_create([q.problem_tensors(p, "cuda") for p in probs], torch.float64)
    cat = lambda name: np.concatenate([getattr(dd, name) for dd in dirs])
    opts = q.options(rtol=1e-12, precond="equilibrate")
    dx, dy, ds, ji = q.qcp_derivative_jvp(plan, cat("dP"), cat("dA"), cat("dq"), cat("db"), opts)
    gP, gA, gq, gb, vi = q.qcp_derivative_vjp(plan, cat("wx"), cat("wy"), cat("ws"), opts)
    dx, dy, ds, gP, gA, gq, gb = to_np(dx, dy, ds, gP, gA, gq, gb)
    on = om = op = oa = 0
    for p, dd in zip(probs, dirs):
        fac = D.DenseFactor(p)
        rj = D.jvp_dense(p, dd, fac)[:3]
        rv = D.vjp_dense(p, dd, fac)[:4]
        assert rel_err((dx[on:on + p.n], dy[om:om + p.m], ds[om:om + p.m]), rj) < TOL64
        assert rel_err((gP[op:op + p.P.nnz], gA[oa:oa + p.A.nnz], gq[on:on + p.n], gb[om:om + p.m]), rv) < TOL64
        on, om, op, oa = on + p.n, om + p.m, op + p.P.nnz, oa + p.A.nnz
    plan.close()
