"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances: FP64 storage, relative error <= 1e-6 over the concatenated
outputs; FP32 storage, <= 1e-4 against the oracle run on the FP32-rounded
problem promoted to FP64 (rounding the data moves theta by ~6e-8, which a
conditioned solve can amplify, so the oracle sees the same rounded data).
"""
import numpy as np
import pytest

from gpu_helpers import adjoint_gap, g, gpu_jvp, gpu_vjp, lib, rel_err, to_np, torch
from oracle import derivative as D
from oracle import kkt_linearized as KL

pytestmark = pytest.mark.gpu

TOL64 = 1e-6
TOL32 = 1e-4


@pytest.fixture(scope="module")
def q():
    return lib()


def _plan(q, prob, dtype=torch.float64, max_rhs=1):
    return q.qcp_plan_create(q.problem_tensors(prob, "cuda", dtype), dtype, max_rhs=max_rhs)


SMALL = [
    ("config1", lambda: g.config1(0)),
    ("config1_seed3", lambda: g.config1(3)),
    ("soc_mix", lambda: g.small_qcp(21, 10, 2, 5, (3, 4, 5))),
    ("soc_rays", lambda: g.small_qcp(22, 16, 0, 6, (3, 3, 6, 8), soc_mix=(0.5, 0.25))),
    ("soc_dims_1_2", lambda: g.small_qcp(24, 14, 1, 3, (1, 2, 2, 7, 1), soc_mix=(0.4, 0.3))),
    ("soc_big_block", lambda: g.small_qcp(25, 60, 3, 10, (40, 5), soc_mix=(0.5, 0.0))),
    ("unconstrained", lambda: g.unconstrained_qp(2, 9)),
    ("equality", lambda: g.equality_qp(4, 12, 7)),
    ("config3_scaled", lambda: g.config3(0, scale=0.004)),
    ("config5_scaled", lambda: g.config5_family(0, scale=0.01).instance(0)),
]


@pytest.mark.parametrize("precond", ["none", "equilibrate"])
@pytest.mark.parametrize("name,mk", SMALL, ids=[s[0] for s in SMALL])
def test_jvp_vjp_fp64_small(q, name, mk, precond):
    prob = mk()
    d = g.make_directions(prob, 11)
    fac = D.DenseFactor(prob)
    ref_j = D.jvp_dense(prob, d, fac)[:3]
    ref_v = D.vjp_dense(prob, d, fac)[:4]
    plan = _plan(q, prob)
    opts = q.options(rtol=1e-11, maxiter=100000, precond=precond)
    jv, ji = gpu_jvp(q, plan, d, opts)
    vv, vi = gpu_vjp(q, plan, d, opts)
    assert rel_err(jv, ref_j) < TOL64, (rel_err(jv, ref_j), ji)
    assert rel_err(vv, ref_v) < TOL64, (rel_err(vv, ref_v), vi)
    # the status is OK unless rounding stalls the true residual above rtol,
    # in which case it says so and the residual is still small
    for inf in (ji[0], vi[0]):
        assert inf["status"] in ("QCP_OK", "QCP_NOT_CONVERGED"), inf
        assert inf["rel_residual"] <= (1e-11 if inf["status"] == "QCP_OK" else 1e-8), inf
    assert adjoint_gap(prob, d, jv, vv) < 1e-8
    plan.close()


@pytest.mark.parametrize("precond", ["none", "equilibrate"])
@pytest.mark.parametrize("name,mk", SMALL[:6], ids=[s[0] for s in SMALL[:6]])
def test_jvp_vjp_fp32_storage(q, name, mk, precond):
    prob = mk()
    r = g.round_to_fp32(prob)
    d = g.make_directions(prob, 12)
    d32 = g.Directions(*[np.asarray(a, np.float32).astype(np.float64) for a in
                         (d.dP, d.dA, d.dq, d.db, d.wx, d.wy, d.ws)])
    fac = D.DenseFactor(r)
    ref_j = D.jvp_dense(r, d32, fac)[:3]
    ref_v = D.vjp_dense(r, d32, fac)[:4]
    plan = _plan(q, prob, torch.float32)
    opts = q.options(rtol=1e-8, maxiter=100000, precond=precond)
    jv, ji = gpu_jvp(q, plan, d32, opts)
    vv, vi = gpu_vjp(q, plan, d32, opts)
    assert rel_err(jv, ref_j) < TOL32, (rel_err(jv, ref_j), ji)
    assert rel_err(vv, ref_v) < TOL32, (rel_err(vv, ref_v), vi)
    plan.close()


@pytest.fixture(scope="module")
def cfg2():
    prob = g.config2(0)
    dirs = g.make_directions_batch(prob, 5, 16)
    fac = D.DenseFactor(prob)
    ref_j = [D.jvp_dense(prob, d, fac)[:3] for d in dirs]
    ref_v = [D.vjp_dense(prob, d, fac)[:4] for d in dirs]
    return prob, dirs, ref_j, ref_v


def test_config2_sixteen_directions(q, cfg2):
    """Configuration 2 as stated: 16 JVP and 16 VJP directions, rtol 1e-10."""
    prob, dirs, ref_j, ref_v = cfg2
    k = len(dirs)
    plan = _plan(q, prob, max_rhs=k)
    opts = q.options(rtol=1e-10, maxiter=100000)
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs])
    dx, dy, ds, ji = q.qcp_derivative_jvp_multi(plan, k, cat("dP"), cat("dA"), cat("dq"), cat("db"), opts)
    dx, dy, ds = to_np(dx, dy, ds)
    n, m = prob.n, prob.m
    for i in range(k):
        got = (dx[i * n:(i + 1) * n], dy[i * m:(i + 1) * m], ds[i * m:(i + 1) * m])
        assert rel_err(got, ref_j[i]) < TOL64, (i, rel_err(got, ref_j[i]), ji[i])
        assert ji[i]["status"] == "QCP_OK"
    gP, gA, gq, gb, vi = q.qcp_derivative_vjp_multi(plan, k, cat("wx"), cat("wy"), cat("ws"), opts)
    gP, gA, gq, gb = to_np(gP, gA, gq, gb)
    nP, nA = prob.P.nnz, prob.A.nnz
    for i in range(k):
        got = (gP[i * nP:(i + 1) * nP], gA[i * nA:(i + 1) * nA], gq[i * n:(i + 1) * n], gb[i * m:(i + 1) * m])
        assert rel_err(got, ref_v[i]) < TOL64, (i, rel_err(got, ref_v[i]), vi[i])
    # with the engine and cluster size fixed, a single-direction solve
    # reproduces direction 0 of the multi solve bit for bit
    plan.set_cluster(4)
    for engine in ("passes", "cluster"):
        o = q.options(rtol=1e-10, maxiter=100000, engine=engine)
        mx, my, _, _ = q.qcp_derivative_jvp_multi(plan, 2, cat("dP")[:2 * nP], cat("dA")[:2 * nA], cat("dq")[:2 * n],
                                                  cat("db")[:2 * m], o)
        mx, my = to_np(mx, my)
        j0, _ = gpu_jvp(q, plan, dirs[0], o)
        assert np.array_equal(j0[0], mx[:n]) and np.array_equal(j0[1], my[:m]), engine
    plan.close()


@pytest.mark.parametrize("engine", ["passes", "persistent", "cluster", "cluster_fp64"])
def test_jvp_and_vjp_in_one_call(q, cfg2, engine):
    """qcp_derivative_jvp_vjp_multi (JVP systems first, VJP systems after
    them; side by side on the cluster engine) gives the oracle's results and,
    with the engine and cluster size fixed, exactly the separate calls'."""
    prob, dirs, ref_j, ref_v = cfg2
    kj, kv = 4, 3
    plan = _plan(q, prob, max_rhs=kj + kv)
    plan.set_cluster(4)
    opts = q.options(rtol=1e-10, maxiter=100000, engine=engine)
    cat = lambda name, ds: np.concatenate([getattr(d, name) for d in ds])
    J, V = dirs[:kj], dirs[5:5 + kv]
    (dx, dy, ds), (gP, gA, gq, gb), info = q.qcp_derivative_jvp_vjp_multi(
        plan, kj, cat("dP", J), cat("dA", J), cat("dq", J), cat("db", J), kv, cat("wx", V), cat("wy", V),
        cat("ws", V), opts)
    assert len(info) == kj + kv and all(i["status"] == "QCP_OK" for i in info), info
    dx, dy, ds, gP, gA, gq, gb = to_np(dx, dy, ds, gP, gA, gq, gb)
    n, m, nP, nA = prob.n, prob.m, prob.P.nnz, prob.A.nnz
    for i in range(kj):
        got = (dx[i * n:(i + 1) * n], dy[i * m:(i + 1) * m], ds[i * m:(i + 1) * m])
        assert rel_err(got, ref_j[i]) < TOL64, (i, rel_err(got, ref_j[i]))
    for i in range(kv):
        got = (gP[i * nP:(i + 1) * nP], gA[i * nA:(i + 1) * nA], gq[i * n:(i + 1) * n], gb[i * m:(i + 1) * m])
        assert rel_err(got, ref_v[5 + i]) < TOL64, (i, rel_err(got, ref_v[5 + i]))
    sx, sy, ss, sji = q.qcp_derivative_jvp_multi(plan, kj, cat("dP", J), cat("dA", J), cat("dq", J), cat("db", J),
                                                 opts)
    tP, tA, tq, tb, svi = q.qcp_derivative_vjp_multi(plan, kv, cat("wx", V), cat("wy", V), cat("ws", V), opts)
    for a, b in zip((dx, dy, ds, gP, gA, gq, gb), to_np(sx, sy, ss, tP, tA, tq, tb)):
        assert np.array_equal(a, b), engine
    assert [i["iters"] for i in info] == [i["iters"] for i in sji + svi]
    with pytest.raises(RuntimeError):
        q.qcp_derivative_jvp_vjp_multi(plan, kj, cat("dP", J), cat("dA", J), cat("dq", J), cat("db", J), kv + 1,
                                       cat("wx", dirs[:kv + 1]), cat("wy", dirs[:kv + 1]),
                                       cat("ws", dirs[:kv + 1]), opts)
    plan.close()


def test_config2_schedules_agree(q, cfg2):
    """Different tile sizes (multi-chunk tiles, CTA-per-row tiles) agree."""
    prob, dirs, ref_j, ref_v = cfg2
    plan = _plan(q, prob)
    outs = []
    # (16384, ...) stages several chunks per tile; long_row 8 / long_chunk 32
    # cuts most x-rows into several one-CTA pieces
    for tile_nnz, long_row, long_chunk in [(4096, 512, 4096), (16384, 4096, 4096), (256, 8, 32), (1024, 16, 64)]:
        plan.set_schedule(tile_nnz, long_row, long_chunk)
        for precond in ("none", "equilibrate"):
            opts = q.options(rtol=1e-10, precond=precond, engine="passes")
            jv, ji = gpu_jvp(q, plan, dirs[0], opts)
            assert rel_err(jv, ref_j[0]) < TOL64, (tile_nnz, long_row, precond, rel_err(jv, ref_j[0]))
            vv, vi = gpu_vjp(q, plan, dirs[0], opts)
            assert rel_err(vv, ref_v[0]) < TOL64, (tile_nnz, long_row, precond, rel_err(vv, ref_v[0]))
            outs.append(jv)
    plan.close()


@pytest.mark.parametrize("precond", ["none", "equilibrate"])
def test_persistent_matches_launch_per_pass(q, cfg2, precond):
    """One cooperative launch for the whole Krylov loop gives the same
    results as one launch per pass (same kernels, same reduction order)."""
    prob, dirs, ref_j, ref_v = cfg2
    k = 4
    plan = _plan(q, prob, max_rhs=k)
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs[:k]])
    res = {}
    for engine in ("passes", "persistent", "cluster", "cluster_fp64"):
        opts = q.options(rtol=1e-10, precond=precond, engine=engine)
        dx, dy, ds, ji = q.qcp_derivative_jvp_multi(plan, k, cat("dP"), cat("dA"), cat("dq"), cat("db"), opts)
        gP, gA, gq, gb, vi = q.qcp_derivative_vjp_multi(plan, k, cat("wx"), cat("wy"), cat("ws"), opts)
        res[engine] = (to_np(dx, dy, ds, gP, gA, gq, gb), ji, vi)
        assert all(i["status"] == "QCP_OK" for i in ji + vi), (engine, ji, vi)
    for x, y in zip(res["passes"][0], res["persistent"][0]):
        assert np.array_equal(x, y)
    n, m = prob.n, prob.m
    nP, nA = prob.P.nnz, prob.A.nnz
    for engine in ("persistent", "cluster", "cluster_fp64"):
        dx, dy, ds, gP, gA, gq, gb = res[engine][0]
        for i in range(k):
            got = (dx[i * n:(i + 1) * n], dy[i * m:(i + 1) * m], ds[i * m:(i + 1) * m])
            assert rel_err(got, ref_j[i]) < TOL64, (engine, i)
            got = (gP[i * nP:(i + 1) * nP], gA[i * nA:(i + 1) * nA], gq[i * n:(i + 1) * n], gb[i * m:(i + 1) * m])
            assert rel_err(got, ref_v[i]) < TOL64, (engine, i)
    plan.close()


@pytest.mark.parametrize("ctas", [1, 2, 3, 7, 8, 16])
def test_cluster_sizes_agree(q, ctas):
    """The cluster engine with 1 to 16 CTAs per system (row splits at SOC
    block boundaries, empty CTAs when a problem has few rows) matches the
    oracle on problems with SOC blocks, a large block and m = 0."""
    for prob in (g.small_qcp(61, 30, 3, 20, (3, 5, 9, 4)), g.small_qcp(25, 60, 3, 10, (40, 5), soc_mix=(0.5, 0.0)),
                 g.unconstrained_qp(2, 9), g.config3(2, scale=0.004)):
        d = g.make_directions(prob, 13)
        fac = D.DenseFactor(prob)
        ref_j = D.jvp_dense(prob, d, fac)[:3]
        ref_v = D.vjp_dense(prob, d, fac)[:4]
        plan = _plan(q, prob)
        plan.set_cluster(ctas)
        for precond in ("none", "equilibrate"):
            for engine in ("cluster", "cluster_fp64"):
                opts = q.options(rtol=1e-11, precond=precond, engine=engine)
                jv, ji = gpu_jvp(q, plan, d, opts)
                vv, vi = gpu_vjp(q, plan, d, opts)
                assert rel_err(jv, ref_j) < TOL64, (ctas, precond, engine, rel_err(jv, ref_j), ji)
                assert rel_err(vv, ref_v) < TOL64, (ctas, precond, engine, rel_err(vv, ref_v), vi)
                assert plan.last_launches() < 20  # the whole Krylov loop is one launch
        plan.close()


def test_cluster_engine_limits(q):
    """A system too large for 16 CTAs' shared memory: the cluster engine
    refuses it, the automatic choice runs the stream engine instead (the
    same bits as asking for it)."""
    from paper_2508_17522_gb300._native import QCPError
    prob = g.config3(3, scale=0.1)
    d = g.make_directions(prob, 4)
    plan = _plan(q, prob)
    with pytest.raises(QCPError, match="ERR_ARG"):
        gpu_jvp(q, plan, d, q.options(rtol=1e-8, engine="cluster"))
    a, ai = gpu_jvp(q, plan, d, q.options(rtol=1e-8, engine="auto", precond="equilibrate"))
    assert plan.last_engine() == "stream"
    b, bi = gpu_jvp(q, plan, d, q.options(rtol=1e-8, engine="stream", precond="equilibrate"))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for bad in (-1, 17):
        with pytest.raises(QCPError, match="ERR_ARG"):
            plan.set_cluster(bad)
    plan.close()


def test_determinism_and_graph(q):
    prob = g.small_qcp(30, 40, 5, 30, (3, 5, 9))
    d = g.make_directions(prob, 3)
    plan = _plan(q, prob)
    a, _ = gpu_jvp(q, plan, d, q.options(rtol=1e-12, engine="passes"))
    b, _ = gpu_jvp(q, plan, d, q.options(rtol=1e-12, engine="passes"))
    c, _ = gpu_jvp(q, plan, d, q.options(rtol=1e-12, engine="passes", use_graph=False))
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    a, _ = gpu_jvp(q, plan, d, q.options(rtol=1e-12, engine="cluster"))
    b, _ = gpu_jvp(q, plan, d, q.options(rtol=1e-12, engine="cluster"))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    plan.close()


def test_batched_uneven_problems(q):
    probs = [g.config1(0), g.small_qcp(41, 17, 2, 8, (3, 6)), g.unconstrained_qp(5, 4),
             g.small_qcp(42, 33, 0, 20, (4, 4, 12), soc_mix=(0.5, 0.2)), g.config3(1, scale=0.003)]
    dirs = [g.make_directions(p, 9) for p in probs]
    plan = q.qcp_batch_plan_create([q.problem_tensors(p, "cuda") for p in probs], torch.float64)
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs])
    opts = q.options(rtol=1e-13, engine="passes")
    dx, dy, ds, ji = q.qcp_derivative_jvp(plan, cat("dP"), cat("dA"), cat("dq"), cat("db"), opts)
    gP, gA, gq, gb, vi = q.qcp_derivative_vjp(plan, cat("wx"), cat("wy"), cat("ws"), opts)
    dx, dy, ds, gP, gA, gq, gb = to_np(dx, dy, ds, gP, gA, gq, gb)
    # the persistent form gives the same answers on uneven problems
    po = q.options(rtol=1e-13, engine="persistent")
    pdx, pdy, pds, pji = q.qcp_derivative_jvp(plan, cat("dP"), cat("dA"), cat("dq"), cat("db"), po)
    for x, y in zip(to_np(pdx, pdy, pds), (dx, dy, ds)):
        assert np.array_equal(x, y)
    _batched_check(probs, dirs, (dx, dy, ds, gP, gA, gq, gb), ji, vi)
    # the cluster engine: one cluster per problem, sizes chosen per problem
    co = q.options(rtol=1e-13, engine="cluster")
    cdx, cdy, cds, cji = q.qcp_derivative_jvp(plan, cat("dP"), cat("dA"), cat("dq"), cat("db"), co)
    cgP, cgA, cgq, cgb, cvi = q.qcp_derivative_vjp(plan, cat("wx"), cat("wy"), cat("ws"), co)
    _batched_check(probs, dirs, to_np(cdx, cdy, cds, cgP, cgA, cgq, cgb), cji, cvi)
    plan.close()


def test_autotuner_picks_the_fastest_and_auto_uses_it(q):
    """qcp_plan_autotune times every candidate on the plan, keeps the fastest
    per pass for engine="auto", and the tuned solves still match the oracle."""
    probs = [g.config1(0), g.small_qcp(41, 17, 2, 8, (3, 6)), g.config3(1, scale=0.003)]
    dirs = [g.make_directions(p, 9) for p in probs]
    plan = q.qcp_batch_plan_create([q.problem_tensors(p, "cuda") for p in probs], torch.float64)
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs])
    for mode in ("jvp", "vjp"):
        best, entries = plan.autotune(mode, iters=16, opts=q.options(precond="equilibrate"))
        kinds = {(e["engine"], e["cluster_ctas"], e["tile_nnz"]) for e in entries}
        assert len(kinds) == len(entries) >= 10, entries
        assert all(e["us_per_pass"] > 0 for e in entries), entries
        assert best["us_per_pass"] == min(e["us_per_pass"] for e in entries), (best, entries)
        opts = q.options(rtol=1e-13, precond="equilibrate", engine="auto")
        dx, dy, ds, ji = q.qcp_derivative_jvp(plan, cat("dP"), cat("dA"), cat("dq"), cat("db"), opts)
        used = plan.last_engine()
        assert used == best["engine"] or (best["engine"] == "cluster" and used == "cluster_fp64"), (used, best)
        gP, gA, gq, gb, vi = q.qcp_derivative_vjp(plan, cat("wx"), cat("wy"), cat("ws"), opts)
        _batched_check(probs, dirs, to_np(dx, dy, ds, gP, gA, gq, gb), ji, vi)
    # a single-problem plan with several directions
    prob = g.config1(0)
    plan2 = _plan(q, prob, max_rhs=4)
    best, entries = plan2.autotune("vjp", nsys=4, iters=16)
    assert best["us_per_pass"] == min(e["us_per_pass"] for e in entries)
    with pytest.raises(RuntimeError):
        plan2.autotune("vjp", nsys=5)
    plan2.close()
    plan.close()


def _batched_check(probs, dirs, outs, ji, vi):
    dx, dy, ds, gP, gA, gq, gb = outs
    on = om = op = oa = 0
    for p, d, a, b in zip(probs, dirs, ji, vi):
        fac = D.DenseFactor(p)
        rj = D.jvp_dense(p, d, fac)[:3]
        rv = D.vjp_dense(p, d, fac)[:4]
        got_j = (dx[on:on + p.n], dy[om:om + p.m], ds[om:om + p.m])
        got_v = (gP[op:op + p.P.nnz], gA[oa:oa + p.A.nnz], gq[on:on + p.n], gb[om:om + p.m])
        assert rel_err(got_j, rj) < TOL64, (rel_err(got_j, rj), a)
        assert rel_err(got_v, rv) < TOL64, (rel_err(got_v, rv), b)
        on, om, op, oa = on + p.n, om + p.m, op + p.P.nnz, oa + p.A.nnz


def test_zero_direction_and_maxiter(q):
    prob = g.config1(0)
    plan = _plan(q, prob)
    z = g.Directions(*[np.zeros_like(a) for a in g.make_directions(prob, 1).__dict__.values()])
    jv, ji = gpu_jvp(q, plan, z, q.options())
    assert all(np.all(x == 0) for x in jv) and ji[0]["iters"] == 0 and ji[0]["status"] == "QCP_OK"
    d = g.make_directions(prob, 1)
    jv, ji = gpu_jvp(q, plan, d, q.options(rtol=1e-14, maxiter=3))
    assert ji[0]["status"] == "QCP_NOT_CONVERGED" and ji[0]["iters"] == 3
    plan.close()


def test_invalid_inputs_rejected(q):
    from paper_2508_17522_gb300._native import QCPError
    prob = g.config1(0)
    bad = q.problem_tensors(prob, "cuda")
    bad.A_indices = bad.A_indices.flip(0).contiguous()           # unsorted and out of row order
    with pytest.raises(QCPError, match="ERR_ARG"):
        q.qcp_plan_create(bad, torch.float64)
    bad = q.problem_tensors(prob, "cuda")
    bad.AT_data = bad.AT_data * 1.5                              # A^T is not A's transpose
    with pytest.raises(QCPError, match="ERR_ARG"):
        q.qcp_plan_create(bad, torch.float64)
    bad = q.problem_tensors(prob, "cuda")
    bad.cone_dim = bad.cone_dim.copy()
    bad.cone_dim[-1] -= 1                                        # cones do not cover m rows
    with pytest.raises(QCPError, match="ERR_ARG"):
        q.qcp_plan_create(bad, torch.float64)
    # a lower-triangular entry in P
    import dataclasses
    Pl = dataclasses.replace(prob.P, indices=prob.P.indices.copy())
    Pl.indices[Pl.indptr[3]] = 0
    bad = q.problem_tensors(dataclasses.replace(prob, P=Pl), "cuda")
    with pytest.raises(QCPError, match="ERR_ARG"):
        q.qcp_plan_create(bad, torch.float64)


def test_at_perm_optional(q):
    prob = g.small_qcp(50, 20, 3, 12, (3, 4))
    d = g.make_directions(prob, 2)
    a = q.qcp_plan_create(q.problem_tensors(prob, "cuda", with_perm=False), torch.float64)
    b = _plan(q, prob)
    ja, _ = gpu_jvp(q, a, d, q.options(rtol=1e-12))
    jb, _ = gpu_jvp(q, b, d, q.options(rtol=1e-12))
    for x, y in zip(ja, jb):
        assert np.array_equal(x, y)
    a.close()
    b.close()


@pytest.mark.slow
def test_config3_full_size_properties(q):
    """The large sparse QCP at its stated size, in the benchmark's launch
    configuration: the JVP satisfies the differentiated optimality
    conditions, the reported true residual meets the tolerance, and JVP and
    VJP are adjoint."""
    prob = g.config3(0)
    d = g.make_directions(prob, 1)
    plan = _plan(q, prob)
    opts = q.options(rtol=1e-9, maxiter=400000, precond="equilibrate")
    jv, ji = gpu_jvp(q, plan, d, opts)
    vv, vi = gpu_vjp(q, plan, d, opts)
    assert ji[0]["status"] == "QCP_OK" and vi[0]["status"] == "QCP_OK", (ji, vi)
    assert ji[0]["rel_residual"] < 1e-9 and vi[0]["rel_residual"] < 1e-9, (ji, vi)
    assert KL.relative_residual(prob, d, *jv) < 1e-7
    assert adjoint_gap(prob, d, jv, vv) < 1e-7
    plan.close()


def test_warm_start_and_diag_preconditioner(q):
    """A warm start anywhere gives the same outputs; the exact dz (JVP) or r
    (VJP) as warm start needs at most one iteration; a caller-given diagonal
    right preconditioner (QCP_PRECOND_DIAG) gives the same outputs."""
    from oracle import embedding as E
    prob = g.small_qcp(81, 20, 2, 10, (3, 5, 4))
    d = g.make_directions(prob, 7)
    fac = D.DenseFactor(prob)
    ref_j = D.jvp_dense(prob, d, fac)[:3]
    ref_v = D.vjp_dense(prob, d, fac)[:4]
    z = fac.z
    dz, _ = fac.solve(-D.d_theta_N(prob, z, d.dP, d.dA, d.dq, d.db))
    r, _ = fac.solve(-(E.Dphi(prob, z).T @ np.concatenate([d.wx, d.wy, d.ws])), trans=1)
    plan = _plan(q, prob)
    N = prob.n + prob.m + 1
    rng = np.random.default_rng(3)
    cuda = lambda a: torch.tensor(np.asarray(a, np.float64), device="cuda")
    for engine in ("passes", "cluster", "persistent"):
        for precond in ("none", "equilibrate"):
            ws = cuda(rng.standard_normal(N))
            opts = q.options(rtol=1e-11, warm_start=ws, engine=engine, precond=precond)
            jv, ji = gpu_jvp(q, plan, d, opts)
            assert rel_err(jv, ref_j) < TOL64, (engine, precond, rel_err(jv, ref_j), ji)
            vv, vi = gpu_vjp(q, plan, d, opts)
            assert rel_err(vv, ref_v) < TOL64, (engine, precond, rel_err(vv, ref_v), vi)
            jv, ji = gpu_jvp(q, plan, d, q.options(rtol=1e-9, warm_start=cuda(dz), engine=engine, precond=precond))
            assert ji[0]["iters"] <= 1 and rel_err(jv, ref_j) < TOL64, (engine, precond, ji)
            vv, vi = gpu_vjp(q, plan, d, q.options(rtol=1e-9, warm_start=cuda(r), engine=engine, precond=precond))
            assert vi[0]["iters"] <= 1 and rel_err(vv, ref_v) < TOL64, (engine, precond, vi)
    # the caller's diagonal preconditioner, changing from call to call (the
    # cluster engine refills its copy of M diag(C) each time), with and
    # without a warm start
    for dd in (np.ones(N), np.exp(rng.uniform(-1.0, 1.0, N)), np.exp(rng.uniform(-2.0, 2.0, N))):
        for engine in ("passes", "persistent", "cluster", "cluster_fp64", "auto"):
            for ws in (None, cuda(rng.standard_normal(N))):
                opts = q.options(rtol=1e-11, precond="diag", precond_d=cuda(dd), engine=engine, warm_start=ws)
                jv, ji = gpu_jvp(q, plan, d, opts)
                assert rel_err(jv, ref_j) < TOL64, (engine, rel_err(jv, ref_j), ji)
                vv, vi = gpu_vjp(q, plan, d, opts)
                assert rel_err(vv, ref_v) < TOL64, (engine, rel_err(vv, ref_v), vi)
                if engine == "auto":
                    assert plan.last_engine() in ("cluster", "cluster_fp64"), plan.last_engine()
    from paper_2508_17522_gb300._native import QCPError
    with pytest.raises(QCPError, match="ERR_ARG"):
        gpu_jvp(q, plan, d, q.options(precond="diag", precond_d=cuda(np.ones(N)), engine="stream"))
    with pytest.raises(QCPError, match="ERR_ARG"):
        gpu_jvp(q, plan, d, q.options(precond="diag"))
    plan.close()


@pytest.mark.parametrize("precond", ["none", "equilibrate"])
@pytest.mark.parametrize("name,mk", SMALL[:6] + SMALL[8:], ids=[s[0] for s in SMALL[:6] + SMALL[8:]])
def test_lsmr_matches_oracle(q, name, mk, precond):
    """LSMR (solver 1) on the pass engine reaches the oracle's JVP and VJP;
    the persistent engine gives the same bits."""
    prob = mk()
    d = g.make_directions(prob, 7)
    fac = D.DenseFactor(prob)
    rj = D.jvp_dense(prob, d, fac)[:3]
    rv = D.vjp_dense(prob, d, fac)[:4]
    plan = _plan(q, prob)
    opts = q.options(rtol=1e-11, precond=precond, solver="lsmr", engine="passes")
    jv, ji = gpu_jvp(q, plan, d, opts)
    vv, vi = gpu_vjp(q, plan, d, opts)
    assert rel_err(jv, rj) < TOL64, (rel_err(jv, rj), ji)
    assert rel_err(vv, rv) < TOL64, (rel_err(vv, rv), vi)
    for inf in (ji[0], vi[0]):
        assert inf["status"] in ("QCP_OK", "QCP_NOT_CONVERGED"), inf
        assert inf["rel_residual"] <= (1e-11 if inf["status"] == "QCP_OK" else 1e-8), inf
    assert plan.last_engine() == "passes"
    po = q.options(rtol=1e-11, precond=precond, solver="lsmr", engine="persistent")
    pj, _ = gpu_jvp(q, plan, d, po)
    pv, _ = gpu_vjp(q, plan, d, po)
    for a, b in zip(pj + pv, jv + vv):
        assert np.array_equal(a, b)
    # the double-float cluster engine: the same recurrences, the oracle's results
    co = q.options(rtol=1e-11, precond=precond, solver="lsmr", engine="cluster")
    cj, cji = gpu_jvp(q, plan, d, co)
    cv, cvi = gpu_vjp(q, plan, d, co)
    assert plan.last_engine() == "cluster"
    assert rel_err(cj, rj) < TOL64, (rel_err(cj, rj), cji)
    assert rel_err(cv, rv) < TOL64, (rel_err(cv, rv), cvi)
    plan.close()


def test_lsmr_config2_and_engine_rules(q, cfg2):
    """Configuration 2 with LSMR: four directions each way at rtol 1e-10;
    auto runs LSMR on the (double-float) cluster engine; the FP64 cluster
    kernel refuses it."""
    prob, dirs, ref_j, ref_v = cfg2
    k = 4
    plan = _plan(q, prob, max_rhs=k)
    opts = q.options(rtol=1e-10, precond="equilibrate", solver="lsmr")
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs[:k]])
    dx, dy, ds, ji = q.qcp_derivative_jvp_multi(plan, k, cat("dP"), cat("dA"), cat("dq"), cat("db"), opts)
    assert plan.last_engine() == "cluster"
    dx, dy, ds = to_np(dx, dy, ds)
    n, m = prob.n, prob.m
    for i in range(k):
        got = (dx[i * n:(i + 1) * n], dy[i * m:(i + 1) * m], ds[i * m:(i + 1) * m])
        assert rel_err(got, ref_j[i]) < TOL64, (i, rel_err(got, ref_j[i]), ji[i])
    gP, gA, gq, gb, vi = q.qcp_derivative_vjp_multi(plan, k, cat("wx"), cat("wy"), cat("ws"), opts)
    gP, gA, gq, gb = to_np(gP, gA, gq, gb)
    nP, nA = prob.P.nnz, prob.A.nnz
    for i in range(k):
        got = (gP[i * nP:(i + 1) * nP], gA[i * nA:(i + 1) * nA], gq[i * n:(i + 1) * n], gb[i * m:(i + 1) * m])
        assert rel_err(got, ref_v[i]) < TOL64, (i, rel_err(got, ref_v[i]), vi[i])
    with pytest.raises(RuntimeError):
        q.qcp_derivative_jvp_multi(plan, 1, cat("dP")[:nP], cat("dA")[:nA], cat("dq")[:n], cat("db")[:m],
                                   q.options(solver="lsmr", engine="cluster_fp64"))
    plan.close()


@pytest.mark.parametrize("engine", ["auto", "passes"])
def test_paper_example_full_size(q, engine):
    """The paper's example shape at its size (Sec. 4: m = 2000, n = 1000; 3000
    variables, 3001 rows, C dense): 2 JVPs and 2 VJPs in one call against the
    dense oracle, rtol 1e-10."""
    prob = g.paper_example(0)
    dirs = g.make_directions_batch(prob, 13, 2)
    fac = D.DenseFactor(prob)
    plan = _plan(q, prob, max_rhs=4)
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs])
    (dx, dy, ds), (gP, gA, gq, gb), info = q.qcp_derivative_jvp_vjp_multi(
        plan, 2, cat("dP"), cat("dA"), cat("dq"), cat("db"), 2, cat("wx"), cat("wy"), cat("ws"),
        q.options(rtol=1e-10, precond="equilibrate", engine=engine))
    assert all(i["status"] == "QCP_OK" for i in info), info
    dx, dy, ds, gP, gA, gq, gb = to_np(dx, dy, ds, gP, gA, gq, gb)
    n, m, nP, nA = prob.n, prob.m, prob.P.nnz, prob.A.nnz
    for i, d in enumerate(dirs):
        rj = D.jvp_dense(prob, d, fac)[:3]
        rv = D.vjp_dense(prob, d, fac)[:4]
        got_j = (dx[i * n:(i + 1) * n], dy[i * m:(i + 1) * m], ds[i * m:(i + 1) * m])
        got_v = (gP[i * nP:(i + 1) * nP], gA[i * nA:(i + 1) * nA], gq[i * n:(i + 1) * n], gb[i * m:(i + 1) * m])
        assert rel_err(got_j, rj) < TOL64, (i, rel_err(got_j, rj))
        assert rel_err(got_v, rv) < TOL64, (i, rel_err(got_v, rv))
    plan.close()


@pytest.mark.parametrize("solver", ["lsqr", "lsmr"])
@pytest.mark.parametrize("name,mk", [SMALL[2], SMALL[5], SMALL[8]], ids=[SMALL[2][0], SMALL[5][0], SMALL[8][0]])
def test_jacobi_preconditioner(q, name, mk, solver):
    """The column-norm (Jacobi) preconditioner reaches the oracle's results
    with either solver."""
    prob = mk()
    d = g.make_directions(prob, 17)
    fac = D.DenseFactor(prob)
    plan = _plan(q, prob)
    opts = q.options(rtol=1e-11, precond="jacobi", solver=solver)
    jv, ji = gpu_jvp(q, plan, d, opts)
    vv, vi = gpu_vjp(q, plan, d, opts)
    assert rel_err(jv, D.jvp_dense(prob, d, fac)[:3]) < TOL64, ji
    assert rel_err(vv, D.vjp_dense(prob, d, fac)[:4]) < TOL64, vi
    # either solver with the Jacobi scaling runs on the cluster engine where it fits
    assert plan.last_engine() in ("cluster", "cluster_fp64"), plan.last_engine()
    plan.close()
