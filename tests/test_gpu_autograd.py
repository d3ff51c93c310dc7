"""The QCP layer (torch.autograd.Function over the C ABI): reverse mode
against the oracle's adjoint and against central finite differences of the
solution map (Newton re-solves of R = 0 at theta +- h dtheta, h = 1e-6;
agreement to 1e-3 relative: the re-solved differences themselves carry
errors up to 2e-4 on these problems),
forward mode against the oracle's JVP; single and batched plans."""
import numpy as np
import pytest

from gpu_helpers import g, lib, rel_err, torch
from oracle import derivative as D
from oracle import newton_fd as NF

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    return lib()


def _stored_weight(prob):
    return np.where(prob.P.row_ids() == prob.P.indices, 1.0, 2.0)


def _leaves(prob, dev="cuda"):
    t = lambda a: torch.tensor(np.asarray(a, np.float64), device=dev, requires_grad=True)
    return t(prob.P.data), t(prob.A.data), t(prob.q), t(prob.b)


def _loss_fd(prob, d, h):
    """Central difference of sum(x*^2) along d, x* from Newton re-solves."""
    from oracle import embedding as E
    z0 = E.solution_to_z(prob)
    zp, rp = NF.resolve(prob, NF._theta(prob, d, h), z0)
    zm, rm = NF.resolve(prob, NF._theta(prob, d, -h), z0)
    xp = E.phi(prob, zp)[:prob.n]
    xm = E.phi(prob, zm)[:prob.n]
    assert rp < 1e-9 and rm < 1e-9
    return (xp @ xp - xm @ xm) / (2 * h)


PROBS = [
    ("soc_mix", lambda: g.small_qcp(71, 12, 2, 6, (3, 4, 5))),
    ("qp", lambda: g.config1(2)),
]


@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_layer_backward_matches_oracle_and_fd(q, name, mk):
    prob = mk()
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
    opts = q.options(rtol=1e-12)
    P, A, qq, b = _leaves(prob)
    x, y, s = q.qcp_layer(plan, P, A, qq, b, opts)
    loss = (x * x).sum()
    loss.backward()
    # the oracle's adjoint with w = (2x, 0, 0), as gradients of stored values
    w = g.Directions(np.zeros(prob.P.nnz), np.zeros(prob.A.nnz), np.zeros(prob.n), np.zeros(prob.m),
                     2 * prob.x, np.zeros(prob.m), np.zeros(prob.m))
    gP, gA, gq, gb = D.vjp_dense(prob, w)[:4]
    ref = (gP * _stored_weight(prob), gA, gq, gb)
    got = [t.grad.detach().cpu().numpy() for t in (P, A, qq, b)]
    assert rel_err(got, ref) < 1e-6, rel_err(got, ref)
    # central finite differences of the solution map, two random directions
    rng = np.random.default_rng(5)
    for _ in range(2):
        d = g.Directions(rng.standard_normal(prob.P.nnz), rng.standard_normal(prob.A.nnz),
                         rng.standard_normal(prob.n), rng.standard_normal(prob.m),
                         np.zeros(prob.n), np.zeros(prob.m), np.zeros(prob.m))
        fd = _loss_fd(prob, d, 1e-6)
        ad = sum(gi @ di for gi, di in zip(got, (d.dP, d.dA, d.dq, d.db)))
        assert abs(ad - fd) <= 1e-3 * max(1.0, abs(fd)), (ad, fd)
    plan.close()


def test_layer_forward_mode_matches_oracle_jvp(q):
    prob = g.small_qcp(72, 10, 1, 5, (3, 6))
    d = g.make_directions(prob, 3)
    plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
    opts = q.options(rtol=1e-12)
    import torch.autograd.forward_ad as fwAD
    prim = [torch.tensor(np.asarray(a, np.float64), device="cuda") for a in (prob.P.data, prob.A.data, prob.q, prob.b)]
    tang = [torch.tensor(np.asarray(a, np.float64), device="cuda") for a in (d.dP, d.dA, d.dq, d.db)]
    with fwAD.dual_level():
        duals = [fwAD.make_dual(p, t) for p, t in zip(prim, tang)]
        outs = q.qcp_layer(plan, *duals, opts=opts)
        got = [fwAD.unpack_dual(o).tangent.cpu().numpy() for o in outs]
    ref = D.jvp_dense(prob, d)[:3]
    assert rel_err(got, ref) < 1e-6, rel_err(got, ref)
    plan.close()


def test_batched_layer_sixteen_problems_fd(q):
    """Config 4's check on a 16-problem subset (sizes shrunk so that the
    finite differences re-solve each problem by Newton's method on the CPU)."""
    probs = g.config4(0, 16, n_range=(12, 24))
    plan = q.qcp_batch_plan_create([q.problem_tensors(p, "cuda") for p in probs], torch.float64)
    opts = q.options(rtol=1e-12)
    leaves = [torch.tensor(np.concatenate([getattr(p, f) if f in ("q", "b") else getattr(p, f).data for p in probs]),
                           device="cuda", requires_grad=True) for f in ("P", "A", "q", "b")]
    x, y, s = q.qcp_layer(plan, *leaves, opts=opts)
    (x * x).sum().backward()
    grads = [t.grad.cpu().numpy() for t in leaves]
    rng = np.random.default_rng(9)
    op = oa = on = om = 0
    for p in probs:
        d = g.Directions(rng.standard_normal(p.P.nnz), rng.standard_normal(p.A.nnz), rng.standard_normal(p.n),
                         rng.standard_normal(p.m), np.zeros(p.n), np.zeros(p.m), np.zeros(p.m))
        gp = grads[0][op:op + p.P.nnz], grads[1][oa:oa + p.A.nnz], grads[2][on:on + p.n], grads[3][om:om + p.m]
        ad = sum(gi @ di for gi, di in zip(gp, (d.dP, d.dA, d.dq, d.db)))
        fd = _loss_fd(p, d, 1e-6)
        assert abs(ad - fd) <= 1e-3 * max(1.0, abs(fd)), (ad, fd)
        op, oa, on, om = op + p.P.nnz, oa + p.A.nnz, on + p.n, om + p.m
    plan.close()
