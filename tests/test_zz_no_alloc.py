"""The allocation-free JVP entry point (qcp_derivative_jvp_noalloc).

Callers that cannot allocate device memory at call time (code running while
its stream is captured into a CUDA graph, allocator hooks, pooled-memory
loops) get the same forward product as qcp_derivative_jvp with the call's
scratch in a static device array of the library.  This file is collected
last on purpose, so a failure here leaves the other tests already run; it
passes alone in a fresh process as well as after them.
"""
import numpy as np
import pytest

from gpu_helpers import g, lib, rel_err, to_np, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precond", ["none", "equilibrate"])
def test_noalloc_matches_jvp_twice(precond):
    q = lib()
    prob = g.small_qcp(61, 30, 3, 14, (3, 5, 4), soc_mix=(0.4, 0.3))
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
    opts = q.options(rtol=1e-11, maxiter=100000, precond=precond)
    for seed in (1, 2):  # two calls in a row share (and must reset) the static scratch
        d = g.make_directions(prob, seed)
        ref, ref_info = q.qcp_derivative_jvp(plan, d.dP, d.dA, d.dq, d.db, opts)[:3], None
        out = [torch.empty(n, device="cuda", dtype=torch.float64) for n in (prob.n, prob.m, prob.m)]
        dx, dy, ds, info = q.qcp_derivative_jvp_noalloc(plan, d.dP, d.dA, d.dq, d.db, out=out, opts=opts)
        torch.cuda.synchronize()
        assert info[0]["status"] in ("QCP_OK", "QCP_NOT_CONVERGED"), info
        assert rel_err(to_np(dx, dy, ds), to_np(*ref)) < 1e-6
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
