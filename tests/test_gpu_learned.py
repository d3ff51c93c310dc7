"""The learned form on the GPU: features, the network's forward pass,
gradients and Adam step against the CPU reference (oracle/learned.py), and
what the trained network gains over the method without it on held-out
instances of the learned-preconditioner family (shrunk to n = 500)."""
import numpy as np
import pytest

from gpu_helpers import g, lib, rel_err, torch
from oracle import derivative as D
from oracle import learned as LO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    return lib()


@pytest.fixture(scope="module")
def L(q):
    from paper_2508_17522_gb300 import learned
    return learned


def test_features_match_reference(q, L):
    for prob in (g.small_qcp(92, 14, 2, 8, (3, 5, 6)), g.config5_family(1, scale=0.05).instance(3)):
        plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
        got = L.plan_features(plan).cpu().numpy().astype(np.float64)
        ref = LO.features(prob).astype(np.float32).astype(np.float64)
        assert np.allclose(got, ref, rtol=2e-6, atol=1e-7), np.abs(got - ref).max()
        plan.close()


def _case(seed, rows):
    rng = np.random.default_rng(seed)
    p = L_init(seed)
    x = rng.standard_normal((rows, LO.IN)) * rng.uniform(0.5, 3.0, LO.IN)
    mean = rng.standard_normal(LO.IN) * 0.1
    inv = rng.uniform(0.5, 2.0, LO.IN)
    t = rng.standard_normal((rows, LO.OUT))
    w = rng.uniform(0.0, 1.0, (rows, LO.OUT))
    return p, x, mean, inv, t, w


def L_init(seed):
    from paper_2508_17522_gb300.learned import init_params
    return init_params(seed).astype(np.float64)


def test_network_forward_gradient_adam_match_reference(q, L):
    rows = 700
    p, x, mean, inv, t, w = _case(7, rows)
    net = L.MLP(1024)
    net.set_params(p)
    net.set_input_norm(mean, inv)
    cu = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    y = net.forward(cu(x)).cpu().numpy()
    f = LO.forward(p.astype(np.float32).astype(np.float64), x.astype(np.float32), mean.astype(np.float32),
                   inv.astype(np.float32))
    assert rel_err([y], [f["y"]]) < 2e-3, rel_err([y], [f["y"]])
    lr = 1e-3
    loss, grad = net.train_step(cu(x), cu(t), cu(w), lr, want_grad=True)
    p32 = p.astype(np.float32).astype(np.float64)
    rloss, rgrad, _ = LO.loss_and_grad(p32, x.astype(np.float32), t.astype(np.float32), w.astype(np.float32),
                                       mean.astype(np.float32), inv.astype(np.float32))
    assert abs(loss - rloss) <= 1e-4 * abs(rloss)
    k = 0
    for name, shape in LO.SIZES:
        nn_ = int(np.prod(shape))
        assert rel_err([grad[k:k + nn_]], [rgrad[k:k + nn_]]) < 5e-3, (name, rel_err([grad[k:k + nn_]], [rgrad[k:k + nn_]]))
        k += nn_
    # Adam's first step: p - lr g / (|g| + eps) where the sign of g is clear
    p1 = net.get_params().astype(np.float64)
    ref, _, _ = LO.adam_step(p32, rgrad, np.zeros_like(p32), np.zeros_like(p32), 1, lr)
    clear = np.abs(rgrad) > 1e-2 * np.abs(rgrad).max()
    assert np.allclose(p1[clear], ref[clear], rtol=0, atol=1e-6)
    net.close()


def test_learned_solve_gains_over_plain(q, L):
    """Train on the method's own solves of 40 instances, then on 8 held-out
    instances compare adjoint solves of ||x*||^2 to rtol 1e-6: the plain
    method (no preconditioner, zero start; LSQR and LSMR), the classical
    equilibration (16 sweeps) and column-norm (Jacobi) scalings, the
    network's target scaling c^alpha alone (zero start, no network), and the
    learned warm start + preconditioner, all on the pass engine.  The
    learned solves must match the oracle and take at least 20% fewer
    iterations than the plain method, and fewer than c^alpha alone and the
    equilibration (the iterations are the solve time: all run the same
    kernels)."""
    fam = g.config5_family(2, scale=0.1)
    train = [fam.instance(j) for j in range(40)]
    held = [fam.instance(1000 + j) for j in range(8)]
    lp = L.LearnedPreconditioner(seed=3).fit(train, steps=800, lr=1e-3)
    assert np.mean(lp.losses[-50:]) < np.mean(lp.losses[:50])
    print("preconditioner exponent chosen on training instances:", lp.alpha, lp.alpha_cost)
    its = {"plain": [], "equilibrate": [], "jacobi": [], "plain_lsmr": [], "c_alpha": [], "learned": []}
    for prob in held:
        plan = q.qcp_plan_create(q.problem_tensors(prob, "cuda"), torch.float64)
        wx, wy, ws = L.adjoint_direction(prob)
        # the ablation: the preconditioner the network is trained toward
        # (c^alpha), with a zero start and no network
        calpha = (L.plan_scalings(plan)[1] ** lp.alpha).contiguous()
        for name, opts in (("plain", q.options(rtol=1e-6, engine="passes")),
                           ("equilibrate", q.options(rtol=1e-6, precond="equilibrate", engine="passes")),
                           ("jacobi", q.options(rtol=1e-6, precond="jacobi", engine="passes")),
                           ("plain_lsmr", q.options(rtol=1e-6, engine="passes", solver="lsmr")),
                           ("c_alpha", q.options(rtol=1e-6, precond="diag", precond_d=calpha, engine="passes"))):
            *_, info = q.qcp_derivative_vjp(plan, wx, wy, ws, opts)
            its[name].append(info[0]["iters"])
        gP, gA, gq, gb, info = lp.vjp(plan, prob, rtol=1e-6, engine="passes")
        assert info[0]["status"] == "QCP_OK" and info[0]["rel_residual"] <= 1e-6, info
        its["learned"].append(info[0]["iters"])
        d = g.Directions(np.zeros(prob.P.nnz), np.zeros(prob.A.nnz), np.zeros(prob.n), np.zeros(prob.m), wx, wy, ws)
        ref = D.vjp_dense(prob, d)[:4]
        got = [t.cpu().numpy() for t in (gP, gA, gq, gb)]
        assert rel_err(got, ref) < 1e-4, rel_err(got, ref)  # rtol 1e-6 on an ill-conditioned F
        plan.close()
    mean = {k: float(np.mean(v)) for k, v in its.items()}
    print("mean iterations to rtol 1e-6 on held-out instances:", mean)
    assert mean["learned"] < 0.8 * mean["plain"], mean
    # the network adds to the scaling it is trained toward, and beats the
    # 16-sweep equilibration in iterations (all on the same engine)
    assert mean["learned"] < 0.95 * mean["c_alpha"], mean
    assert mean["learned"] < 0.9 * mean["equilibrate"], mean
