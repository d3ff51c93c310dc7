"""The learned form: a network trained on the method's own solves predicts,
from per-row features of a problem, a warm start and a diagonal right
preconditioner for the Krylov solve (C ABI: qcp_plan_features, qcp_mlp_*,
qcp_plan_last_solution, qcp_plan_scalings, QCP_PRECOND_DIAG and
qcp_options.warm_start).

The features, the network's forward and backward passes (tensor cores),
Adam, the decoding and the solves run in the library's kernels; this module
orders the steps and prepares the training data (target scaling, input
mean and spread, minibatch indices) with torch tensor operations:

1. For each training instance of a family (fixed sparsity pattern, the
   rows line up across instances), solve the adjoint problem of ||x*||^2
   (equilibrated, on the fastest engine) and read back its solution r and
   the plan's column equilibration c.
2. Choose the preconditioner C = c^alpha: alpha in {0, 1/4, 1/2, 3/4, 1}
   with the fewest iterations on the first training instances (on this
   family full equilibration is slower than none, c^(1/2) faster).
3. Fit the network on all rows of all training instances with Adam: it
   predicts, per row, the deviation of (r / ||w||, alpha log c) from their
   mean over the training instances (inputs standardised with the training
   rows' mean and spread); the mean is kept as a per-row offset.
4. For a new instance: features -> network + offset -> (warm start
   ||w|| v0, preconditioner exp(v1)) -> QCP_PRECOND_DIAG solve with that warm
   start.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from . import api

IN, HID, OUT = 16, 256, 2


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def plan_features(plan: api.Plan) -> torch.Tensor:
    """(N_total x 16) float32 features of every embedding row of the plan."""
    nt = sum(pt.n + pt.m + 1 for pt in plan.problems)
    out = torch.empty((nt, IN), device=plan.device, dtype=torch.float32)
    api._check(N.lib().qcp_plan_features(plan.handle, _p(out)), "qcp_plan_features")
    return out


def plan_scalings(plan: api.Plan):
    """(w, c): the plan's row and column equilibration (N per problem)."""
    nt = sum(pt.n + pt.m + 1 for pt in plan.problems)
    w = torch.empty(nt, device=plan.device, dtype=torch.float64)
    c = torch.empty(nt, device=plan.device, dtype=torch.float64)
    api._check(N.lib().qcp_plan_scalings(plan.handle, _p(w), _p(c)), "qcp_plan_scalings")
    return w, c


def last_solution(plan: api.Plan, nsys: int = 1) -> torch.Tensor:
    """dz (after a JVP) or r (after a VJP) of the plan's last call, N per system."""
    per = sum(pt.n + pt.m + 1 for pt in plan.problems)
    nt = per if plan.batched else per * nsys
    out = torch.empty(nt, device=plan.device, dtype=torch.float64)
    api._check(N.lib().qcp_plan_last_solution(plan.handle, _p(out)), "qcp_plan_last_solution")
    return out


class MLP:
    """The 16-256-256-2 network of the C ABI (qcp_mlp_*)."""

    def __init__(self, max_rows: int, device="cuda", stream=None):
        self.device = torch.device(device)
        self.max_rows = int(max_rows)
        self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        api._check(N.lib().qcp_mlp_create(self.max_rows, ctypes.c_void_p(self._stream.cuda_stream or None),
                                          ctypes.byref(h)), "qcp_mlp_create")
        self._h = h
        self.nparam = int(N.lib().qcp_mlp_param_count())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().qcp_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        a = np.ascontiguousarray(params, np.float32)
        assert a.size == self.nparam
        api._check(N.lib().qcp_mlp_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p)), "qcp_mlp_set_params")

    def get_params(self) -> np.ndarray:
        a = np.empty(self.nparam, np.float32)
        api._check(N.lib().qcp_mlp_get_params(self._h, a.ctypes.data_as(ctypes.c_void_p)), "qcp_mlp_get_params")
        return a

    def set_input_norm(self, mean, inv_std):
        m = np.ascontiguousarray(mean, np.float32)
        s = np.ascontiguousarray(inv_std, np.float32)
        api._check(N.lib().qcp_mlp_set_input_norm(self._h, m.ctypes.data_as(ctypes.c_void_p),
                                                  s.ctypes.data_as(ctypes.c_void_p)), "qcp_mlp_set_input_norm")

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        x = x.to(device=self.device, dtype=torch.float32).contiguous()
        y = torch.empty((x.shape[0], OUT), device=self.device, dtype=torch.float32)
        for r0 in range(0, x.shape[0], self.max_rows):
            r1 = min(x.shape[0], r0 + self.max_rows)
            api._check(N.lib().qcp_mlp_forward(self._h, _p(x[r0:r1]), r1 - r0, _p(y[r0:r1])), "qcp_mlp_forward")
        return y

    def train_step(self, x, target, weight, lr, want_grad=False):
        x = x.to(device=self.device, dtype=torch.float32).contiguous()
        target = target.to(device=self.device, dtype=torch.float32).contiguous()
        weight = weight.to(device=self.device, dtype=torch.float32).contiguous()
        loss = ctypes.c_double()
        g = np.empty(self.nparam, np.float32) if want_grad else None
        api._check(N.lib().qcp_mlp_train_step(self._h, _p(x), _p(target), _p(weight), x.shape[0], float(lr),
                                              ctypes.byref(loss),
                                              g.ctypes.data_as(ctypes.c_void_p) if g is not None else None),
                   "qcp_mlp_train_step")
        return (loss.value, g) if want_grad else loss.value


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (seeded), zero biases, in the packed layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, shape in ((IN, (HID, IN)), (None, (HID,)), (HID, (HID, HID)), (None, (HID,)), (HID, (OUT, HID)),
                          (None, (OUT,))):
        if fan_in is None:
            parts.append(np.zeros(shape))
        else:
            b = np.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-b, b, shape))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def decode(y: torch.Tensor, scale: float, offset: torch.Tensor | None = None):
    """(warm start, preconditioner) float64 device tensors from network outputs."""
    rows = y.shape[0]
    warm = torch.empty(rows, device=y.device, dtype=torch.float64)
    d = torch.empty(rows, device=y.device, dtype=torch.float64)
    st = torch.cuda.current_stream(y.device)
    api._check(N.lib().qcp_mlp_decode(_p(y.contiguous()), _p(offset.contiguous()) if offset is not None else None,
                                      rows, float(scale), _p(warm), _p(d), ctypes.c_void_p(st.cuda_stream or None)),
               "qcp_mlp_decode")
    return warm, d


def adjoint_direction(prob):
    """w = (2 x*, 0, 0): the adjoint direction of the loss ||x*||^2."""
    return 2.0 * np.asarray(prob.x, np.float64), np.zeros(prob.m), np.zeros(prob.m)


def training_rows(prob, device="cuda", rtol=1e-10):
    """(features, r / ||w||, c, info) of one instance from the method's own
    adjoint solve (equilibrated, on the fastest engine: the solution r does
    not depend on how the solve is preconditioned)."""
    plan = api.qcp_plan_create(api.problem_tensors(prob, device), torch.float64)
    wx, wy, ws = adjoint_direction(prob)
    _, _, _, _, info = api.qcp_derivative_vjp(plan, wx, wy, ws,
                                              api.options(rtol=rtol, precond="equilibrate", engine="auto"))
    r = last_solution(plan)
    _, c = plan_scalings(plan)
    f = plan_features(plan)
    scale = float(np.linalg.norm(wx)) or 1.0
    plan.close()
    return f, (r / scale).float(), c, info[0]


def _iterations(prob, device, **opts):
    plan = api.qcp_plan_create(api.problem_tensors(prob, device), torch.float64)
    wx, wy, ws = adjoint_direction(prob)
    *_, info = api.qcp_derivative_vjp(plan, wx, wy, ws, api.options(rtol=1e-6, engine="auto", **opts))
    plan.close()
    return info[0]["iters"] if info[0]["status"] == "QCP_OK" else 10 ** 9


class LearnedPreconditioner:
    """Training and use of the learned warm start and preconditioner."""

    def __init__(self, seed=0, device="cuda", batch_rows=8192):
        self.device = torch.device(device)
        self.batch_rows = batch_rows
        self.net = MLP(batch_rows, device)
        self.net.set_params(init_params(seed))
        self.seed = seed
        self.losses = []
        self.alpha = None
        self.offset = None

    def fit(self, instances, steps=1500, lr=1e-3, alphas=(0.0, 0.25, 0.5, 0.75, 1.0), probe=2):
        rows = [training_rows(p, self.device) for p in instances]
        # the preconditioner exponent with the fewest iterations on the first instances
        cost = []
        for a in alphas:
            its = 0
            for p, rw in zip(instances[:probe], rows[:probe]):
                its += _iterations(p, self.device, precond="diag", precond_d=(rw[2] ** a).contiguous())
            cost.append(its)
        self.alpha = float(alphas[int(np.argmin(cost))])
        self.alpha_cost = dict(zip(alphas, cost))
        X = torch.cat([r[0] for r in rows])
        T = torch.stack([torch.stack([r[1], (self.alpha * torch.log(r[2])).float()], dim=1) for r in rows])
        self.offset = T.mean(0).contiguous()                 # per row (the family's rows line up)
        T = (T - self.offset).reshape(-1, 2)
        Wt = torch.ones_like(T)
        mean = X.mean(0)
        spread = X.std(0)
        inv = torch.where(spread > 1e-12, 1.0 / spread, torch.ones_like(spread))
        self.net.set_input_norm(mean.cpu().numpy(), inv.cpu().numpy())
        gen = torch.Generator(device="cpu").manual_seed(self.seed)
        for _ in range(steps):
            idx = torch.randint(0, X.shape[0], (min(self.batch_rows, X.shape[0]),), generator=gen).to(self.device)
            self.losses.append(self.net.train_step(X[idx], T[idx], Wt[idx], lr))
        return self

    def predict(self, plan: api.Plan, scale: float):
        """(warm start r0, preconditioner d) for the plan's single problem."""
        y = self.net.forward(plan_features(plan))
        return decode(y, scale, self.offset)

    def vjp(self, plan: api.Plan, prob, rtol=1e-6, engine="auto"):
        """The learned adjoint solve of ||x*||^2 on a new instance."""
        wx, wy, ws = adjoint_direction(prob)
        warm, d = self.predict(plan, float(np.linalg.norm(wx)) or 1.0)
        opts = api.options(rtol=rtol, precond="diag", precond_d=d, warm_start=warm, engine=engine)
        return api.qcp_derivative_vjp(plan, wx, wy, ws, opts)
