"""The stream engine (QCP_ENGINE_STREAM) against the CPU oracle.

The engine cuts every problem's rows into warp-sized units: SELL-32 slices
of x-rows and of zero-cone / R+ rows with 1 to 32 lanes per row, packed
second-order-cone blocks of at most 32 rows (segmented warp sums for D Pi,
Appendix A), single blocks of 33 to 256 rows, and 512-entry chunks of
longer rows (a row of several chunks is completed by whichever chunk
finishes last).  The problems below reach each kind: SOC mixes with blocks
of dimension 1 to 200, dense P rows of 1300+ entries (three chunks),
power-law columns (config 3, scaled), m = 0.
Tolerances: FP64 1e-6, FP32 storage 1e-4 against the oracle on the
FP32-rounded data; every output block is checked on its own.
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
    ("soc_dims_1_2", lambda: g.small_qcp(24, 14, 1, 3, (1, 2, 2, 7, 1), soc_mix=(0.4, 0.3))),
    ("soc_big_block", lambda: g.small_qcp(25, 60, 3, 10, (40, 5), soc_mix=(0.5, 0.0))),
    ("soc_200_block", lambda: g.small_qcp(26, 260, 10, 40, (200, 33, 31, 32, 9), soc_mix=(0.4, 0.3),
                                          nnz_per_row=3)),
    ("dense_P_long_rows", lambda: g.small_qcp(27, 1300, 100, 400, (10,) * 10, nnz_per_row=6)),
    ("unconstrained", lambda: g.unconstrained_qp(2, 9)),
    ("equality", lambda: g.equality_qp(4, 12, 7)),
    ("config3_scaled", lambda: g.config3(0, scale=0.01)),
]


@pytest.fixture(scope="module")
def q():
    return lib()


def _plan(q, prob, dtype=torch.float64, max_rhs=1):
    return q.qcp_plan_create(q.problem_tensors(prob, "cuda", dtype), dtype, max_rhs=max_rhs)


def _check_blocks(got, ref, tol, what):
    assert rel_err(got, ref) < tol, (what, rel_err(got, ref))
    for i, (a, b) in enumerate(zip(got, ref)):
        nb = np.linalg.norm(b)
        err = np.linalg.norm(np.asarray(a) - b) / (nb if nb > 0 else 1.0)
        assert err < tol, (what, "block", i, err)


@pytest.mark.parametrize("precond", ["none", "equilibrate"])
@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_stream_matches_oracle(q, name, mk, precond):
    prob = mk()
    d = g.make_directions(prob, 51)
    fac = D.DenseFactor(prob)
    ref_j = D.jvp_dense(prob, d, fac)[:3]
    ref_v = D.vjp_dense(prob, d, fac)[:4]
    plan = _plan(q, prob)
    opts = q.options(rtol=1e-11, maxiter=400000, precond=precond, engine="stream")
    jv, ji = gpu_jvp(q, plan, d, opts)
    assert plan.last_engine() == "stream"
    vv, vi = gpu_vjp(q, plan, d, opts)
    _check_blocks(jv, ref_j, TOL64, (name, precond, "jvp", ji))
    _check_blocks(vv, ref_v, TOL64, (name, precond, "vjp", vi))
    for inf in (ji[0], vi[0]):
        assert inf["status"] in ("QCP_OK", "QCP_NOT_CONVERGED"), inf
        assert inf["rel_residual"] <= (1e-11 if inf["status"] == "QCP_OK" else 1e-8), inf
    assert adjoint_gap(prob, d, jv, vv) < 1e-8
    # the same bits on a second call (fixed work split, fixed summation order)
    jv2, _ = gpu_jvp(q, plan, d, opts)
    for a, b in zip(jv, jv2):
        assert np.array_equal(a, b)
    plan.close()


@pytest.mark.parametrize("precond", ["none", "equilibrate"])
@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_stream_lsmr_matches_oracle(q, name, mk, precond):
    """LSMR (Fong & Saunders 2011) on the stream engine: the deferred
    (hbar, x, h) updates in the u-passes, the last ones in a stopped
    system's final u-pass; the oracle per output block, and the same bits on
    a second call."""
    prob = mk()
    d = g.make_directions(prob, 53)
    fac = D.DenseFactor(prob)
    ref_j = D.jvp_dense(prob, d, fac)[:3]
    ref_v = D.vjp_dense(prob, d, fac)[:4]
    plan = _plan(q, prob)
    opts = q.options(rtol=1e-11, maxiter=400000, precond=precond, engine="stream", solver="lsmr")
    jv, ji = gpu_jvp(q, plan, d, opts)
    assert plan.last_engine() == "stream"
    vv, vi = gpu_vjp(q, plan, d, opts)
    _check_blocks(jv, ref_j, TOL64, (name, precond, "jvp", ji))
    _check_blocks(vv, ref_v, TOL64, (name, precond, "vjp", vi))
    for inf in (ji[0], vi[0]):
        assert inf["status"] in ("QCP_OK", "QCP_NOT_CONVERGED"), inf
        assert inf["rel_residual"] <= (1e-11 if inf["status"] == "QCP_OK" else 1e-8), inf
    assert adjoint_gap(prob, d, jv, vv) < 1e-8
    jv2, _ = gpu_jvp(q, plan, d, opts)
    for a, b in zip(jv, jv2):
        assert np.array_equal(a, b)
    plan.close()


@pytest.mark.parametrize("name,mk", [PROBS[1], PROBS[3], PROBS[5]], ids=[PROBS[1][0], PROBS[3][0], PROBS[5][0]])
def test_stream_fp32_storage(q, name, mk):
    prob = mk()
    r = g.round_to_fp32(prob)
    d = g.make_directions(prob, 52)
    d32 = g.Directions(*[np.asarray(a, np.float32).astype(np.float64) for a in
                         (d.dP, d.dA, d.dq, d.db, d.wx, d.wy, d.ws)])
    fac = D.DenseFactor(r)
    plan = _plan(q, prob, torch.float32)
    opts = q.options(rtol=1e-8, maxiter=400000, precond="equilibrate", engine="stream")
    jv, _ = gpu_jvp(q, plan, d32, opts)
    vv, _ = gpu_vjp(q, plan, d32, opts)
    _check_blocks(jv, D.jvp_dense(r, d32, fac)[:3], TOL32, (name, "jvp"))
    _check_blocks(vv, D.vjp_dense(r, d32, fac)[:4], TOL32, (name, "vjp"))
    plan.close()


def test_stream_config2_directions_and_pair_call(q):
    """Several systems per launch (gridDim.y), the JVP+VJP call, warm starts."""
    prob = g.config2(0)
    dirs = g.make_directions_batch(prob, 5, 3)
    fac = D.DenseFactor(prob)
    k = len(dirs)
    n, m, nP, nA = prob.n, prob.m, prob.P.nnz, prob.A.nnz
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs])
    plan = _plan(q, prob, max_rhs=2 * k)
    opts = q.options(rtol=1e-10, maxiter=400000, precond="equilibrate", engine="stream")
    (dx, dy, ds), (gP, gA, gq, gb), info = q.qcp_derivative_jvp_vjp_multi(
        plan, k, cat("dP"), cat("dA"), cat("dq"), cat("db"), k, cat("wx"), cat("wy"), cat("ws"), opts)
    assert all(i["status"] == "QCP_OK" for i in info), info
    dx, dy, ds, gP, gA, gq, gb = to_np(dx, dy, ds, gP, gA, gq, gb)
    for i, d in enumerate(dirs):
        _check_blocks((dx[i * n:(i + 1) * n], dy[i * m:(i + 1) * m], ds[i * m:(i + 1) * m]),
                      D.jvp_dense(prob, d, fac)[:3], TOL64, ("jvp", i))
        _check_blocks((gP[i * nP:(i + 1) * nP], gA[i * nA:(i + 1) * nA], gq[i * n:(i + 1) * n],
                       gb[i * m:(i + 1) * m]), D.vjp_dense(prob, d, fac)[:4], TOL64, ("vjp", i))
    # a single-direction call reproduces direction 0 of the multi call
    j0, _ = gpu_jvp(q, plan, dirs[0], opts)
    mx, _, _, _ = q.qcp_derivative_jvp_multi(plan, k, cat("dP"), cat("dA"), cat("dq"), cat("db"), opts)
    assert rel_err(j0[0], to_np(mx)[0][:n]) < 1e-9
    # a warm start anywhere still reaches the oracle
    N = prob.N
    ws = torch.tensor(np.random.default_rng(4).standard_normal(N), device="cuda")
    jw, _ = gpu_jvp(q, plan, dirs[1], q.options(rtol=1e-10, precond="equilibrate", engine="stream", warm_start=ws))
    _check_blocks(jw, D.jvp_dense(prob, dirs[1], fac)[:3], TOL64, "warm")
    plan.close()


def test_stream_batched_uneven_problems(q):
    probs = [g.config1(0), g.small_qcp(41, 17, 2, 8, (3, 6)), g.unconstrained_qp(5, 4),
             g.small_qcp(42, 33, 0, 20, (4, 4, 12), soc_mix=(0.5, 0.2)), g.config3(1, scale=0.003),
             g.small_qcp(25, 60, 3, 10, (40, 5), soc_mix=(0.5, 0.0))]
    dirs = [g.make_directions(p, 9) for p in probs]
    plan = q.qcp_batch_plan_create([q.problem_tensors(p, "cuda") for p in probs], torch.float64)
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs])
    opts = q.options(rtol=1e-12, precond="equilibrate", engine="stream")
    dx, dy, ds, ji = q.qcp_derivative_jvp(plan, cat("dP"), cat("dA"), cat("dq"), cat("db"), opts)
    gP, gA, gq, gb, vi = q.qcp_derivative_vjp(plan, cat("wx"), cat("wy"), cat("ws"), opts)
    dx, dy, ds, gP, gA, gq, gb = to_np(dx, dy, ds, gP, gA, gq, gb)
    on = om = op = oa = 0
    for p, d, a, b in zip(probs, dirs, ji, vi):
        fac = D.DenseFactor(p)
        _check_blocks((dx[on:on + p.n], dy[om:om + p.m], ds[om:om + p.m]), D.jvp_dense(p, d, fac)[:3], TOL64, a)
        _check_blocks((gP[op:op + p.P.nnz], gA[oa:oa + p.A.nnz], gq[on:on + p.n], gb[om:om + p.m]),
                      D.vjp_dense(p, d, fac)[:4], TOL64, b)
        on, om, op, oa = on + p.n, om + p.m, op + p.P.nnz, oa + p.A.nnz
    plan.close()


def test_stream_engine_rules(q):
    """auto runs the stream engine when a system does not fit the cluster
    engine (LSQR and LSMR); the stream engine refuses the diagonal
    preconditioner and PSD blocks of more than 256 entries, and agrees with
    the pass engine on a larger problem."""
    from paper_2508_17522_gb300._native import QCPError
    prob = g.config3(3, scale=0.1)
    d = g.make_directions(prob, 4)
    plan = _plan(q, prob)
    opts = q.options(rtol=1e-10, maxiter=400000, precond="equilibrate")
    a, ai = gpu_jvp(q, plan, d, opts)
    assert plan.last_engine() == "stream", plan.last_engine()
    b, bi = gpu_jvp(q, plan, d, q.options(rtol=1e-10, maxiter=400000, precond="equilibrate", engine="passes"))
    assert ai[0]["status"] == "QCP_OK" and bi[0]["status"] == "QCP_OK", (ai, bi)
    assert rel_err(a, b) < 1e-7, rel_err(a, b)
    # LSMR runs on the stream engine too, and auto picks it for LSMR here
    c, ci = gpu_jvp(q, plan, d, q.options(rtol=1e-10, maxiter=400000, precond="equilibrate", solver="lsmr"))
    assert plan.last_engine() == "stream", plan.last_engine()
    assert ci[0]["status"] == "QCP_OK", ci
    assert rel_err(c, b) < 1e-7, rel_err(c, b)
    N = prob.N
    with pytest.raises(QCPError, match="ERR_ARG"):
        gpu_jvp(q, plan, d, q.options(precond="diag", precond_d=torch.ones(N, device="cuda", dtype=torch.float64),
                                      engine="stream"))
    plan.close()
    # a PSD block of order 23 (276 entries) is beyond the engine's 256-row blocks
    psd = g.small_qcp(31, 300, 0, 4, (3,), psd_orders=(23,))
    pl = _plan(q, psd)
    with pytest.raises(QCPError, match="ERR_ARG"):
        gpu_jvp(q, pl, g.make_directions(psd, 1), q.options(engine="stream"))
    pl.close()


@pytest.mark.slow
def test_config3_tenth_against_matrix_free_oracle(q):
    """Configuration 3's structure at a tenth of its size (N = 32 001: power-law
    columns, lognormal SOC blocks, 1000+-entry rows), too large for the dense
    oracle: the outputs of the stream and pass engines against the oracle's
    own matrix-free solve (Ruiz-scaled LSMR on the assembled sparse F, to a
    relative residual of 1e-12), element by element in every output block."""
    prob = g.config3(0, scale=0.1)
    d = g.make_directions(prob, 61)
    op = D.FOperator(prob)
    rj = D.jvp_lsmr(prob, d, rtol=1e-12, scale=True, maxiter=40000, op=op)
    rv = D.vjp_lsmr(prob, d, rtol=1e-12, scale=True, maxiter=40000, op=op)
    assert rj[3]["rel_residual"] < 1e-10 and rv[4]["rel_residual"] < 1e-10, (rj[3], rv[4])
    plan = _plan(q, prob)
    for engine in ("stream", "passes"):
        opts = q.options(rtol=1e-11, maxiter=400000, precond="equilibrate", engine=engine)
        jv, ji = gpu_jvp(q, plan, d, opts)
        vv, vi = gpu_vjp(q, plan, d, opts)
        assert plan.last_engine() == engine
        _check_blocks(jv, rj[:3], TOL64, (engine, "jvp", ji))
        _check_blocks(vv, rv[:4], TOL64, (engine, "vjp", vi))
    plan.close()
