"""Pins of the learned form's CPU reference (oracle/learned.py): BF16
rounding against torch's conversion, backpropagation against finite
differences, the affine case, Adam's first step in closed form, and the
feature layout on a problem built by hand."""
import numpy as np
import pytest
import torch

import qcpgen as g
from oracle import learned as LO


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-20, 20, 2000),
                        # exact ties between two bfloat16 neighbours round to even
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, -0.0])])
    x = x.astype(np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(LO.bf16(x), ref)


def _small_case(seed, rows=6, scale=0.3):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(LO.NPARAM) * scale
    x = rng.standard_normal((rows, LO.IN))
    t = rng.standard_normal((rows, LO.OUT))
    w = rng.uniform(0.5, 1.5, (rows, LO.OUT))
    return p, x, t, w


def test_backward_matches_finite_differences():
    p, x, t, w = _small_case(2)
    loss, grad, _ = LO.loss_and_grad(p, x, t, w, rounding=False)
    rng = np.random.default_rng(3)
    idx = rng.choice(LO.NPARAM, 80, replace=False)
    idx = np.concatenate([idx, [LO.NPARAM - 1, LO.NPARAM - 2]])  # the output biases
    h = 1e-6
    for i in idx:
        e = np.zeros(LO.NPARAM)
        e[i] = h
        fd = (LO.loss_and_grad(p + e, x, t, w, rounding=False)[0] - LO.loss_and_grad(p - e, x, t, w, rounding=False)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_affine_region():
    """With every pre-activation positive the network is the affine map
    W3 (W2 (W1 x + b1) + b2) + b3."""
    rng = np.random.default_rng(4)
    d = {"W1": rng.uniform(0.1, 1, (LO.HID, LO.IN)), "b1": rng.uniform(0, 1, LO.HID),
         "W2": rng.uniform(0.1, 1, (LO.HID, LO.HID)), "b2": rng.uniform(0, 1, LO.HID),
         "W3": rng.standard_normal((LO.OUT, LO.HID)), "b3": rng.standard_normal(LO.OUT)}
    x = rng.uniform(0, 1, (5, LO.IN))
    y = LO.forward(LO.pack(d), x, rounding=False)["y"]
    M = d["W3"] @ d["W2"] @ d["W1"]
    c = d["W3"] @ (d["W2"] @ d["b1"] + d["b2"]) + d["b3"]
    assert np.allclose(y, x @ M.T + c, rtol=1e-12, atol=1e-9)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    p0, gr = rng.standard_normal(50), rng.standard_normal(50)
    p1, m, v = LO.adam_step(p0, gr, np.zeros(50), np.zeros(50), 1, 1e-3)
    # at t = 1 the bias-corrected moments are g and g^2
    assert np.allclose(p1, p0 - 1e-3 * gr / (np.abs(gr) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * gr) and np.allclose(v, 0.001 * gr * gr)


def test_feature_layout_by_construction():
    prob = g.small_qcp(91, 6, 2, 4, (3, 4))
    f = LO.features(prob)
    n, m = prob.n, prob.m
    N = n + m + 1
    assert f.shape == (N, 16)
    assert np.all(f[:, 0] == 1)
    kinds = np.argmax(f[:, 1:6], axis=1)
    assert np.all(kinds[:n] == 0) and kinds[N - 1] == 4
    assert np.all(kinds[n:n + 2] == 1) and np.all(kinds[n + 2:n + 6] == 2) and np.all(kinds[n + 6:n + m] == 3)
    assert np.array_equal(f[:n, 6], prob.x) and np.array_equal(f[n:n + m, 6], prob.y)
    assert np.allclose(f[n:n + m, 7], prob.y - prob.s) and np.allclose(f[n:n + m, 9], prob.s)
    assert np.array_equal(f[:n, 8], prob.q) and np.array_equal(f[n:n + m, 8], prob.b)
    z = prob.y - prob.s
    assert np.array_equal(f[n + 2:n + 6, 10], (z[2:6] > 0).astype(float))   # R+ rows: 1{z > 0}
    assert np.all(f[n:n + 2, 10] == 1.0)                                      # zero cone: dual is R
    assert np.array_equal(f[n + 6:n + m, 13], np.array([3, 3, 3, 4, 4, 4, 4]) / 32.0)
    assert np.array_equal(f[n + 6:n + m, 14], np.array([0, 1, 1, 0, 1, 1, 1.0]))
    # row norms of M = [[P, A^T], [A, 0]] for a y-row: ||A row||
    A = prob.A.to_scipy().toarray()
    assert np.isclose(f[n + 1, 11], 0.125 * np.log(np.sum(A[1] ** 2)))
    assert np.isclose(f[n + 1, 12], 0.25 * np.log(np.count_nonzero(A[1]) + 1.0))
