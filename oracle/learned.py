"""CPU reference of the learned form's arithmetic: per-row features of a
problem and the 16-256-256-2 ReLU network's forward pass, loss, gradients
and Adam step.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/).  Numpy in FP64, with
the values rounded to BF16 (round to nearest even) exactly where the GPU
network rounds them: the normalised input, the weights, and the hidden
activations where they enter a product, and the hidden gradients where they
enter the weight-gradient and input-gradient products.  Everything else is
exact FP64, so the GPU's FP32 accumulation shows as differences of order
1e-6 relative.
"""
import numpy as np

from . import cones as C

IN, HID, OUT = 16, 256, 2
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[k:k + n], np.float64).reshape(shape)
        k += n
    return out


def pack(d):
    return np.concatenate([np.ravel(d[name]) for name, _ in SIZES])


def bf16(x):
    """Round binary32 values to the nearest bfloat16 (ties to even); the
    result is returned as float64 holding the rounded values."""
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x, mean=None, inv_std=None, rounding=True):
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    w = unpack(params)
    x = np.asarray(x, np.float64)
    if mean is not None:
        x = (x - mean) * inv_std
    xb = r(x)
    W1, W2, W3 = r(w["W1"]), r(w["W2"]), r(w["W3"])
    pre1 = xb @ W1.T + w["b1"]
    h1 = r(np.maximum(pre1, 0.0))
    pre2 = h1 @ W2.T + w["b2"]
    h2 = r(np.maximum(pre2, 0.0))
    y = h2 @ W3.T + w["b3"]
    return {"xb": xb, "W1": W1, "W2": W2, "W3": W3, "pre1": pre1, "h1": h1, "pre2": pre2, "h2": h2, "y": y}


def loss_and_grad(params, x, target, weight, mean=None, inv_std=None, rounding=True):
    """Weighted squared error sum w (y - t)^2 / max(sum w, 1) and its
    gradient with respect to the packed parameters (backpropagation)."""
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    f = forward(params, x, mean, inv_std, rounding)
    y = f["y"]
    sw = max(float(np.sum(weight)), 1.0)
    loss = float(np.sum(weight * (y - target) ** 2) / sw)
    dy = 2.0 * weight * (y - target) / sw
    g = {"W3": dy.T @ f["h2"], "b3": dy.sum(0)}
    dh2 = (dy @ f["W3"]) * (f["pre2"] > 0)
    g["W2"] = r(dh2).T @ f["h1"]
    g["b2"] = dh2.sum(0)
    dh1 = (r(dh2) @ f["W2"]) * (f["pre1"] > 0)
    g["W1"] = r(dh1).T @ f["xb"]
    g["b1"] = dh1.sum(0)
    return loss, pack(g), f


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One step of Adam (Kingma & Ba, 2015) at step count t >= 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v


def features(prob):
    """The per-row features of every embedding row (N x 16), as documented
    for qcp_plan_features."""
    n, m = prob.n, prob.m
    N = n + m + 1
    Pup = prob.P.to_scipy()
    Ps = (Pup + Pup.T - __import__("scipy").sparse.diags(Pup.diagonal())).tocsr()
    x, y, s = prob.x, prob.y, prob.s
    z = y - s
    g = 2 * (Ps @ x) + prob.q
    kappa = float(x @ (Ps @ x))
    f = np.zeros((N, IN))
    f[:, 0] = 1.0
    # row kinds and SOC positions from the cone list
    kind = np.zeros(N, int)
    kind[N - 1] = 4
    sdim = np.zeros(N)
    spos = np.zeros(N)
    row = n
    for t, d in zip(prob.cone_type, prob.cone_dim):
        kind[row:row + d] = {C.ZERO: 1, C.NONNEG: 2, C.SOC: 3}[int(t)]
        if int(t) == C.SOC:
            sdim[row:row + d] = d
            spos[row + 1:row + d] = 1.0
        row += d
    f[np.arange(N), 1 + kind] = 1.0
    f[:n, 6] = x
    f[n:n + m, 6] = y
    f[N - 1, 6] = 1.0
    f[n:n + m, 7] = z
    f[:n, 8] = prob.q
    f[n:n + m, 8] = prob.b
    f[:n, 9] = g
    f[n:n + m, 9] = s
    f[N - 1, 9] = kappa
    dd = np.ones(N)
    dd[n:n + m] = C.dproj_dual_sparse(list(zip(prob.cone_type, prob.cone_dim)), z).diagonal()
    f[:, 10] = dd
    # rows of M = [[P, A^T], [A, 0]]: norms and stored-entry counts
    Asp = prob.A.to_scipy()
    nrm2 = np.zeros(N)
    nnz = np.zeros(N)
    nrm2[:n] = np.asarray(Ps.multiply(Ps).sum(1)).ravel() + np.asarray(Asp.multiply(Asp).sum(0)).ravel()
    nnz[:n] = np.diff(Ps.tocsr().indptr) + np.diff(Asp.tocsc().indptr)
    nrm2[n:n + m] = np.asarray(Asp.multiply(Asp).sum(1)).ravel()
    nnz[n:n + m] = np.diff(Asp.tocsr().indptr)
    with np.errstate(divide="ignore"):
        f[:, 11] = np.where(nnz > 0, 0.125 * np.log(nrm2 + 1e-300), 0.0)
    f[:, 12] = 0.25 * np.log(nnz + 1.0)
    f[:, 13] = np.where(kind == 3, sdim / 32.0, 0.0)
    f[:, 14] = np.where(kind == 3, spos, 0.0)
    f[:, 15] = f[:, 6] * f[:, 10]
    return f
