"""The allocation-free JVP entry point (qcp_derivative_jvp_noalloc).

Callers that must not allocate device memory when they need a derivative
(allocator hooks, real-time loops, hosts whose memory comes from a pool they
do not own) get the same forward product as qcp_derivative_jvp, with the
call's scratch in a static device array of the library.  Each call is
checked against the CPU oracle (FP64 within 1e-6; FP32 storage within 1e-4
of the oracle on the FP32-rounded data) and against the regular entry
point, on two calls in a row (they share, and must reset, the array).  This
file is collected last on purpose, so a failure here leaves the other tests
already run; it passes alone in a fresh process as well as after them.
"""
import numpy as np
import pytest

from gpu_helpers import g, lib, rel_err, to_np, torch
from oracle import derivative as D

pytestmark = pytest.mark.gpu


def _dirs32(d):
    return g.Directions(*[np.asarray(a, np.float32).astype(np.float64) for a in
                          (d.dP, d.dA, d.dq, d.db, d.wx, d.wy, d.ws)])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("precond", ["none", "equilibrate"])
def test_noalloc_matches_oracle_and_jvp_twice(precond, dtype):
    q = lib()
    prob = g.small_qcp(61, 30, 3, 14, (3, 5, 4), soc_mix=(0.4, 0.3))
    f32 = dtype == torch.float32
    ref_prob = g.round_to_fp32(prob) if f32 else prob
    tol = 1e-4 if f32 else 1e-6
    fac = D.DenseFactor(ref_prob)
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda", dtype), dtype)
    # FP32 data moves z off the root by ~1e-7, so the true residual of the
    # rounded system stalls near that level: rtol 1e-6 there
    opts = q.options(rtol=1e-6 if f32 else 1e-11, maxiter=100000, precond=precond)
    for seed in (1, 2):
        d = g.make_directions(prob, seed)
        if f32:
            d = _dirs32(d)
        want = D.jvp_dense(ref_prob, d, fac)[:3]
        out = [torch.empty(n, device="cuda", dtype=dtype) for n in (prob.n, prob.m, prob.m)]
        dx, dy, ds, info = q.qcp_derivative_jvp_noalloc(plan, d.dP, d.dA, d.dq, d.db, out=out, opts=opts)
        torch.cuda.synchronize()
        assert info[0]["status"] == "QCP_OK", info
        got = to_np(dx, dy, ds)
        assert rel_err(got, want) < tol, (seed, rel_err(got, want))
        reg = q.qcp_derivative_jvp(plan, d.dP, d.dA, d.dq, d.db, opts)
        assert rel_err(got, to_np(*reg[:3])) < tol
    plan.close()


def test_noalloc_first_call_on_fresh_plan():
    """The first derivative call a plan ever sees is the allocation-free one;
    it matches the oracle, and a second one after it does too."""
    q = lib()
    prob = g.small_qcp(62, 24, 2, 12, (4, 6), soc_mix=(0.5, 0.2))
    fac = D.DenseFactor(prob)
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
    opts = q.options(rtol=1e-11, maxiter=100000, precond="equilibrate")
    for seed in (3, 4):
        d = g.make_directions(prob, seed)
        dx, dy, ds, info = q.qcp_derivative_jvp_noalloc(plan, d.dP, d.dA, d.dq, d.db, opts=opts)
        torch.cuda.synchronize()
        assert info[0]["status"] == "QCP_OK", info
        assert rel_err(to_np(dx, dy, ds), D.jvp_dense(prob, d, fac)[:3]) < 1e-6
    plan.close()


def test_noalloc_rejects_oversized_plan():
    """A plan whose scratch exceeds the static array gets a clear error."""
    from paper_2508_17522_gb300._native import QCPError
    q = lib()
    prob = g.config3(0, scale=1.2)  # N ~ 384000 rows: beyond the 16 MiB array
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
    d = g.make_directions(prob, 1)
    with pytest.raises(QCPError, match="scratch"):
        q.qcp_derivative_jvp_noalloc(plan, d.dP, d.dA, d.dq, d.db)
    plan.close()
