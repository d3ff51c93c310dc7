"""Paired stream iterations (qcp_plan_set_stream_pairing) against the oracle.

A call with K JVP and K VJP directions on the stream engine iterates JVP
system i and VJP system i in step, the VJP one pass behind, so that every
launch runs the same product (with G, then with G^T) for both and reads the
matrix once.  Each system still takes its own sequence of passes (Sec. 3.1
for the JVP, Sec. 3.2 for the VJP), so:
  * every output block matches the dense oracle (FP64 within 1e-6, FP32
    storage within 1e-4 of the oracle on the FP32-rounded data);
  * paired and one-after-the-other calls agree to rounding order (the CTA
    partial sums are grouped by the launch shape), also when both stop at an
    iteration cap, where the two schedules must have run the same passes;
  * a paired call reports shared passes, an unpaired one none, and a
    repeated paired call gives the same bits.
The problems reach every unit kind: packed cone blocks, blocks of 33 to 200
rows (run once per system inside a paired launch), rows of several 512-entry
chunks (split-row sums per system).
"""
import numpy as np
import pytest

from gpu_helpers import g, lib, rel_err, to_np, torch
from oracle import derivative as D

pytestmark = pytest.mark.gpu

TOL64 = 1e-6
TOL32 = 1e-4

PROBS = [
    ("soc_mix", lambda: g.small_qcp(21, 10, 2, 5, (3, 4, 5))),
    ("soc_200_block", lambda: g.small_qcp(26, 260, 10, 40, (200, 33, 31, 32, 9), soc_mix=(0.4, 0.3),
                                          nnz_per_row=3)),
    ("dense_P_long_rows", lambda: g.small_qcp(27, 1300, 100, 400, (10,) * 10, nnz_per_row=6)),
    ("equality", lambda: g.equality_qp(4, 12, 7)),
    ("config3_scaled", lambda: g.config3(0, scale=0.01)),
]


@pytest.fixture(scope="module")
def q():
    return lib()


def _check_blocks(got, ref, tol, what):
    assert rel_err(got, ref) < tol, (what, rel_err(got, ref))
    for i, (a, b) in enumerate(zip(got, ref)):
        nb = np.linalg.norm(b)
        err = np.linalg.norm(np.asarray(a) - b) / (nb if nb > 0 else 1.0)
        assert err < tol, (what, "block", i, err)


def _pair_call(q, plan, prob, dirs, opts):
    """One qcp_derivative_jvp_vjp_multi call; per direction the JVP blocks
    (dx, dy, ds) and the VJP blocks (dP, dA, dq, db), and the infos."""
    k = len(dirs)
    n, m, nP, nA = prob.n, prob.m, prob.P.nnz, prob.A.nnz
    cat = lambda name: np.concatenate([getattr(d, name) for d in dirs])
    (dx, dy, ds), (gP, gA, gq, gb), info = q.qcp_derivative_jvp_vjp_multi(
        plan, k, cat("dP"), cat("dA"), cat("dq"), cat("db"), k, cat("wx"), cat("wy"), cat("ws"), opts)
    dx, dy, ds, gP, gA, gq, gb = to_np(dx, dy, ds, gP, gA, gq, gb)
    jv = [(dx[i * n:(i + 1) * n], dy[i * m:(i + 1) * m], ds[i * m:(i + 1) * m]) for i in range(k)]
    vv = [(gP[i * nP:(i + 1) * nP], gA[i * nA:(i + 1) * nA], gq[i * n:(i + 1) * n], gb[i * m:(i + 1) * m])
          for i in range(k)]
    return jv, vv, info


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("precond", ["none", "equilibrate"])
@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_paired_matches_oracle_and_unpaired(q, name, mk, precond, k):
    prob = mk()
    dirs = g.make_directions_batch(prob, 61, k)
    fac = D.DenseFactor(prob)
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64, max_rhs=2 * k)
    opts = q.options(rtol=1e-11, maxiter=400000, precond=precond, engine="stream")
    jv, vv, info = _pair_call(q, plan, prob, dirs, opts)
    assert plan.last_engine() == "stream"
    shared = plan.last_shared_passes()
    assert shared > 0, shared
    for i, d in enumerate(dirs):
        _check_blocks(jv[i], D.jvp_dense(prob, d, fac)[:3], TOL64, (name, precond, "jvp", i, info[i]))
        _check_blocks(vv[i], D.vjp_dense(prob, d, fac)[:4], TOL64, (name, precond, "vjp", i, info[k + i]))
    for inf in info:
        assert inf["status"] in ("QCP_OK", "QCP_NOT_CONVERGED"), inf
        assert inf["rel_residual"] <= (1e-11 if inf["status"] == "QCP_OK" else 1e-8), inf
    # at most one shared read per launch of a pair, and none past the pair's
    # shorter solve (two passes an iteration)
    its = [inf["iters"] for inf in info]
    assert shared <= sum(2 * min(its[i], its[k + i]) + 2 for i in range(k)), (shared, its)
    # the same bits on a second paired call
    jv2, vv2, _ = _pair_call(q, plan, prob, dirs, opts)
    for i in range(k):
        for a, b in zip(jv[i] + vv[i], jv2[i] + vv2[i]):
            assert np.array_equal(a, b)
    # one range after the other: the same solutions to rounding order
    plan.set_stream_pairing(False)
    ju, vu, infu = _pair_call(q, plan, prob, dirs, opts)
    assert plan.last_shared_passes() == 0
    for i in range(k):
        assert rel_err(jv[i], ju[i]) < 1e-8, (i, rel_err(jv[i], ju[i]))
        assert rel_err(vv[i], vu[i]) < 1e-8, (i, rel_err(vv[i], vu[i]))
    plan.close()


@pytest.mark.parametrize("cap", [1, 2, 7, 40])
def test_paired_iteration_cap_same_passes(q, cap):
    """Stopped by maxiter, both schedules have run exactly the same passes of
    every system: the same iteration counts and the same iterates (to
    rounding order), whichever of the pair's systems stops first."""
    prob = g.small_qcp(26, 260, 10, 40, (200, 33, 31, 32, 9), soc_mix=(0.4, 0.3), nnz_per_row=3)
    dirs = g.make_directions_batch(prob, 62, 2)
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64, max_rhs=4)
    opts = q.options(rtol=1e-14, maxiter=cap, precond="equilibrate", engine="stream", compute_residual=False,
                     check_every=3)
    jv, vv, info = _pair_call(q, plan, prob, dirs, opts)
    # cap 1: the VJP systems stop after their lead-in pass, so no launch runs
    # a product for both systems of a pair
    assert (plan.last_shared_passes() > 0) == (cap > 1), plan.last_shared_passes()
    plan.set_stream_pairing(False)
    ju, vu, infu = _pair_call(q, plan, prob, dirs, opts)
    assert [i["iters"] for i in info] == [i["iters"] for i in infu] == [cap] * 4, (info, infu)
    assert [i["status"] for i in info] == [i["status"] for i in infu]
    for i in range(2):
        assert rel_err(jv[i], ju[i]) < 1e-9, (cap, i, rel_err(jv[i], ju[i]))
        assert rel_err(vv[i], vu[i]) < 1e-9, (cap, i, rel_err(vv[i], vu[i]))
    plan.close()


@pytest.mark.parametrize("name,mk", [PROBS[1], PROBS[2], PROBS[4]], ids=[PROBS[1][0], PROBS[2][0], PROBS[4][0]])
def test_paired_lsmr(q, name, mk):
    """LSMR in paired launches: the oracle, and the unpaired schedule."""
    prob = mk()
    dirs = g.make_directions_batch(prob, 65, 2)
    fac = D.DenseFactor(prob)
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64, max_rhs=4)
    opts = q.options(rtol=1e-11, maxiter=400000, precond="equilibrate", engine="stream", solver="lsmr")
    jv, vv, info = _pair_call(q, plan, prob, dirs, opts)
    assert plan.last_shared_passes() > 0
    for i, d in enumerate(dirs):
        _check_blocks(jv[i], D.jvp_dense(prob, d, fac)[:3], TOL64, (name, "jvp", i, info[i]))
        _check_blocks(vv[i], D.vjp_dense(prob, d, fac)[:4], TOL64, (name, "vjp", i, info[2 + i]))
    plan.set_stream_pairing(False)
    ju, vu, _ = _pair_call(q, plan, prob, dirs, opts)
    for i in range(2):
        assert rel_err(jv[i], ju[i]) < 1e-8 and rel_err(vv[i], vu[i]) < 1e-8
    plan.close()


def test_paired_fp32_storage(q):
    prob = g.small_qcp(27, 1300, 100, 400, (10,) * 10, nnz_per_row=6)
    r = g.round_to_fp32(prob)
    dirs = [g.Directions(*[np.asarray(a, np.float32).astype(np.float64) for a in
                           (d.dP, d.dA, d.dq, d.db, d.wx, d.wy, d.ws)]) for d in g.make_directions_batch(prob, 63, 2)]
    fac = D.DenseFactor(r)
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda", torch.float32), torch.float32, max_rhs=4)
    opts = q.options(rtol=1e-8, maxiter=400000, precond="equilibrate", engine="stream")
    jv, vv, _ = _pair_call(q, plan, prob, dirs, opts)
    assert plan.last_shared_passes() > 0
    for i, d in enumerate(dirs):
        _check_blocks(jv[i], D.jvp_dense(r, d, fac)[:3], TOL32, ("jvp", i))
        _check_blocks(vv[i], D.vjp_dense(r, d, fac)[:4], TOL32, ("vjp", i))
    plan.close()


def test_paired_zero_vjp_direction(q):
    """A VJP direction of zero stops its system before any pass (b = 0):
    the JVP system of the pair iterates alone inside the paired launches."""
    prob = g.small_qcp(21, 10, 2, 5, (3, 4, 5))
    d = g.make_directions(prob, 64)
    z = g.Directions(d.dP, d.dA, d.dq, d.db, 0 * d.wx, 0 * d.wy, 0 * d.ws)
    fac = D.DenseFactor(prob)
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64, max_rhs=2)
    opts = q.options(rtol=1e-11, maxiter=400000, precond="equilibrate", engine="stream")
    jv, vv, info = _pair_call(q, plan, prob, [z], opts)
    _check_blocks(jv[0], D.jvp_dense(prob, z, fac)[:3], TOL64, ("jvp", info))
    for a in vv[0]:
        assert np.all(a == 0.0), info
    assert info[0]["status"] == "QCP_OK" and info[1]["status"] == "QCP_OK", info
    plan.close()
