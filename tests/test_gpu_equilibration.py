"""Iterated row/column equilibration (qcp_plan_set_equilibration) on the GPU.

Both linear systems of the method (Sec. 3.1 and 3.2) are consistent, so a
row scaling W and a column scaling C of F change the Krylov iterates but not
the outputs (dx, dy, ds) or (dP, dA, dq, db).  These tests run 3, 8 and 16
sweeps of the scaling on every engine and compare with the dense oracle:
FP64 storage within 1e-6, FP32 storage within 1e-4 of the oracle run on the
FP32-rounded data.  Each output block is checked on its own as well as the
concatenation.
"""
import numpy as np
import pytest

from gpu_helpers import adjoint_gap, g, gpu_jvp, gpu_vjp, lib, rel_err, to_np, torch
from oracle import derivative as D

pytestmark = pytest.mark.gpu

TOL64 = 1e-6
TOL32 = 1e-4

PROBS = [
    ("config1", lambda: g.config1(0)),
    ("soc_mix", lambda: g.small_qcp(21, 10, 2, 5, (3, 4, 5))),
    ("soc_big_block", lambda: g.small_qcp(25, 60, 3, 10, (40, 5), soc_mix=(0.5, 0.0))),
    ("config3_scaled", lambda: g.config3(0, scale=0.004)),
]


@pytest.fixture(scope="module")
def q():
    return lib()


def _plan(q, prob, dtype=torch.float64, max_rhs=1, sweeps=16):
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda", dtype), dtype, max_rhs=max_rhs)
    plan.set_equilibration(sweeps)
    return plan


def _check_blocks(got, ref, tol, what):
    assert rel_err(got, ref) < tol, (what, rel_err(got, ref))
    for i, (a, b) in enumerate(zip(got, ref)):
        nb = np.linalg.norm(b)
        if nb > 0:
            assert np.linalg.norm(np.asarray(a) - b) / nb < tol, (what, "block", i)
        else:
            assert np.linalg.norm(np.asarray(a)) < tol, (what, "block", i)


@pytest.mark.parametrize("sweeps", [3, 8, 16])
@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_sweeps_match_oracle_every_engine(q, name, mk, sweeps):
    prob = mk()
    d = g.make_directions(prob, 31)
    fac = D.DenseFactor(prob)
    ref_j = D.jvp_dense(prob, d, fac)[:3]
    ref_v = D.vjp_dense(prob, d, fac)[:4]
    plan = _plan(q, prob, sweeps=sweeps)
    for engine in ("passes", "persistent", "cluster", "cluster_fp64"):
        opts = q.options(rtol=1e-11, maxiter=200000, precond="equilibrate", engine=engine)
        jv, ji = gpu_jvp(q, plan, d, opts)
        vv, vi = gpu_vjp(q, plan, d, opts)
        _check_blocks(jv, ref_j, TOL64, (name, sweeps, engine, "jvp", ji))
        _check_blocks(vv, ref_v, TOL64, (name, sweeps, engine, "vjp", vi))
        for inf in (ji[0], vi[0]):
            assert inf["status"] in ("QCP_OK", "QCP_NOT_CONVERGED"), inf
            assert inf["rel_residual"] <= (1e-11 if inf["status"] == "QCP_OK" else 1e-8), inf
        assert adjoint_gap(prob, d, jv, vv) < 1e-8
    plan.close()


@pytest.mark.parametrize("sweeps", [8])
@pytest.mark.parametrize("name,mk", PROBS[1:3], ids=[p[0] for p in PROBS[1:3]])
def test_sweeps_fp32_storage(q, name, mk, sweeps):
    prob = mk()
    r = g.round_to_fp32(prob)
    d = g.make_directions(prob, 32)
    d32 = g.Directions(*[np.asarray(a, np.float32).astype(np.float64) for a in
                         (d.dP, d.dA, d.dq, d.db, d.wx, d.wy, d.ws)])
    fac = D.DenseFactor(r)
    ref_j = D.jvp_dense(r, d32, fac)[:3]
    ref_v = D.vjp_dense(r, d32, fac)[:4]
    plan = _plan(q, prob, torch.float32, sweeps=sweeps)
    for engine in ("passes", "cluster"):
        opts = q.options(rtol=1e-8, maxiter=200000, precond="equilibrate", engine=engine)
        jv, _ = gpu_jvp(q, plan, d32, opts)
        vv, _ = gpu_vjp(q, plan, d32, opts)
        _check_blocks(jv, ref_j, TOL32, (name, engine, "jvp"))
        _check_blocks(vv, ref_v, TOL32, (name, engine, "vjp"))
    plan.close()


def test_sweeps_config2_four_directions(q):
    """Configuration 2 at rtol 1e-10 with 8 sweeps, the combined call on the
    cluster engine (the benchmark's call) and the pass engine."""
    prob = g.config2(0)
    dirs = g.make_directions_batch(prob, 5, 4)
    fac = D.DenseFactor(prob)
    ref_j = [D.jvp_dense(prob, d, fac)[:3] for d in dirs]
    ref_v = [D.vjp_dense(prob, d, fac)[:4] for d in dirs]
    k = len(dirs)
    n, m, nP, nA = prob.n, prob.m, prob.P.nnz, prob.A.nnz
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs])
    plan = _plan(q, prob, max_rhs=2 * k, sweeps=8)
    for engine in ("cluster", "passes"):
        opts = q.options(rtol=1e-10, maxiter=200000, precond="equilibrate", engine=engine)
        (dx, dy, ds), (gP, gA, gq, gb), info = q.qcp_derivative_jvp_vjp_multi(
            plan, k, cat("dP"), cat("dA"), cat("dq"), cat("db"), k, cat("wx"), cat("wy"), cat("ws"), opts)
        assert all(i["status"] == "QCP_OK" for i in info), (engine, info)
        dx, dy, ds, gP, gA, gq, gb = to_np(dx, dy, ds, gP, gA, gq, gb)
        for i in range(k):
            _check_blocks((dx[i * n:(i + 1) * n], dy[i * m:(i + 1) * m], ds[i * m:(i + 1) * m]), ref_j[i], TOL64,
                          (engine, "jvp", i))
            _check_blocks((gP[i * nP:(i + 1) * nP], gA[i * nA:(i + 1) * nA], gq[i * n:(i + 1) * n],
                           gb[i * m:(i + 1) * m]), ref_v[i], TOL64, (engine, "vjp", i))
    plan.close()


def test_more_sweeps_fewer_iterations(q):
    """On a scaled-down configuration 3 (N = 3201) repeated sweeps cut the
    LSQR iterations of both solves, and the outputs stay the oracle's."""
    prob = g.config3(0, scale=0.01)
    d = g.make_directions(prob, 33)
    fac = D.DenseFactor(prob)
    ref_j = D.jvp_dense(prob, d, fac)[:3]
    its = {}
    for sweeps in (1, 8):
        plan = _plan(q, prob, sweeps=sweeps)
        opts = q.options(rtol=1e-8, maxiter=400000, precond="equilibrate", engine="passes")
        jv, ji = gpu_jvp(q, plan, d, opts)
        _, vi = gpu_vjp(q, plan, d, opts)
        assert rel_err(jv, ref_j) < TOL64, (sweeps, rel_err(jv, ref_j))
        its[sweeps] = ji[0]["iters"] + vi[0]["iters"]
        plan.close()
    assert its[8] < 0.5 * its[1], its


def test_set_equilibration_rules(q):
    """Out-of-range sweeps are refused and leave the plan as it was; the
    setting is refused once the plan has run a derivative call; a plan
    starts with 16 sweeps (setting 16 again changes nothing)."""
    from paper_2508_17522_gb300._native import QCPError
    prob = g.small_qcp(21, 10, 2, 5, (3, 4, 5))
    d = g.make_directions(prob, 34)
    fac = D.DenseFactor(prob)
    ref_j = D.jvp_dense(prob, d, fac)[:3]
    plan = _plan(q, prob)
    for bad in (0, 65, -3):
        with pytest.raises(QCPError, match="ERR_ARG"):
            plan.set_equilibration(bad)
    plan.set_equilibration(4)
    opts = q.options(rtol=1e-11, precond="equilibrate", engine="passes")
    jv, _ = gpu_jvp(q, plan, d, opts)
    assert rel_err(jv, ref_j) < TOL64
    with pytest.raises(QCPError, match="ERR_ARG"):
        plan.set_equilibration(8)
    jv2, _ = gpu_jvp(q, plan, d, opts)
    for a, b in zip(jv, jv2):
        assert np.array_equal(a, b)
    plan.close()
