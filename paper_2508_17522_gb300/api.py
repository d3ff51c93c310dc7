"""Python binding of libqcpd: argument marshalling only.

Every step of the derivative runs in the library's CUDA kernels; this module
only turns torch tensors (device memory) and the current CUDA stream into
the C ABI's pointers, and allocates the output tensors.

Names follow the C ABI of include/qcpd.h:
    plan = qcp_plan_create(problem_tensors(...), dtype)
    dx, dy, ds, info = qcp_derivative_jvp(plan, dP, dA, dq, db)
    dP, dA, dq, db, info = qcp_derivative_vjp(plan, wx, wy, ws)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N

_DT = {torch.float64: N.QCP_F64, torch.float32: N.QCP_F32}


def _vp(t):
    if t is None or t.numel() == 0:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _check(code, where, ok=(N.QCP_OK,)):
    if code not in ok:
        raise N.QCPError(code, where)
    return code


def _t(a, device, dtype):
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a), device=device, dtype=dtype)


@dataclass
class ProblemTensors:
    """Device tensors of one problem and its solution (keeps them alive)."""
    n: int
    m: int
    P_indptr: torch.Tensor
    P_indices: torch.Tensor
    P_data: torch.Tensor
    A_indptr: torch.Tensor
    A_indices: torch.Tensor
    A_data: torch.Tensor
    AT_indptr: torch.Tensor
    AT_indices: torch.Tensor
    AT_data: torch.Tensor
    AT_perm: torch.Tensor | None
    q: torch.Tensor
    b: torch.Tensor
    cone_type: np.ndarray
    cone_dim: np.ndarray
    cone_param: np.ndarray
    x: torch.Tensor
    y: torch.Tensor
    s: torch.Tensor


def problem_tensors(prob, device="cuda", dtype=torch.float64, with_perm=True) -> ProblemTensors:
    """Copy a problem (any object with the fields n, m, P, A, AT, AT_perm, q,
    b, cone_type, cone_dim, x, y, s and optionally cone_param; P/A/AT having
    indptr, indices, data) to
    device tensors of the given floating-point dtype."""
    i64, i32 = torch.int64, torch.int32
    return ProblemTensors(
        int(prob.n), int(prob.m),
        _t(prob.P.indptr, device, i64), _t(prob.P.indices, device, i32), _t(prob.P.data, device, dtype),
        _t(prob.A.indptr, device, i64), _t(prob.A.indices, device, i32), _t(prob.A.data, device, dtype),
        _t(prob.AT.indptr, device, i64), _t(prob.AT.indices, device, i32), _t(prob.AT.data, device, dtype),
        _t(prob.AT_perm, device, i64) if (with_perm and prob.AT_perm is not None) else None,
        _t(prob.q, device, dtype), _t(prob.b, device, dtype),
        np.ascontiguousarray(prob.cone_type, dtype=np.int32), np.ascontiguousarray(prob.cone_dim, dtype=np.int32),
        np.ascontiguousarray(getattr(prob, "cone_param", None) if getattr(prob, "cone_param", None) is not None
                             else np.zeros(len(prob.cone_type)), dtype=np.float64),
        _t(prob.x, device, dtype), _t(prob.y, device, dtype), _t(prob.s, device, dtype))


def _c_problem(pt: ProblemTensors):
    def csr(nr, nc, ip, ix, v):
        return N.qcp_csr(nr, nc, int(ix.numel()), _vp(ip), _vp(ix), _vp(v))
    cone = N.qcp_cone(len(pt.cone_type), pt.cone_type.ctypes.data_as(ctypes.c_void_p),
                      pt.cone_dim.ctypes.data_as(ctypes.c_void_p), pt.cone_param.ctypes.data_as(ctypes.c_void_p))
    prob = N.qcp_problem(pt.n, pt.m, csr(pt.n, pt.n, pt.P_indptr, pt.P_indices, pt.P_data),
                         csr(pt.m, pt.n, pt.A_indptr, pt.A_indices, pt.A_data),
                         csr(pt.n, pt.m, pt.AT_indptr, pt.AT_indices, pt.AT_data),
                         _vp(pt.AT_perm), _vp(pt.q), _vp(pt.b), cone)
    sol = N.qcp_solution(_vp(pt.x), _vp(pt.y), _vp(pt.s))
    return prob, sol


_PRECOND = {"none": N.QCP_PRECOND_NONE, "equilibrate": N.QCP_PRECOND_EQUILIBRATE, "diag": N.QCP_PRECOND_DIAG,
            "jacobi": N.QCP_PRECOND_JACOBI}


_ENGINE = {"passes": N.QCP_ENGINE_PASSES, "persistent": N.QCP_ENGINE_PERSISTENT,
           "cluster": N.QCP_ENGINE_CLUSTER, "auto": N.QCP_ENGINE_AUTO, "cluster_fp64": N.QCP_ENGINE_CLUSTER_FP64,
           "stream": N.QCP_ENGINE_STREAM}


def options(rtol=1e-10, maxiter=100000, check_every=32, use_graph=True, compute_residual=True, precond="none",
            kink_tol=0.0, engine="auto", warm_start=None, precond_d=None, solver="lsqr"):
    """qcp_options; solver is "lsqr" or "lsmr" (LSMR runs on the pass and
    persistent engines); precond is "none" (the plain method), "equilibrate",
    "jacobi" (column norms of F) or
    "diag" (precond_d: a float64 device tensor, N per problem); warm_start:
    a float64 device tensor of N per system (dz for the JVP, r for the VJP).
    engine is "passes" (one launch per pass), "persistent" (one cooperative
    launch), "cluster" (one thread-block cluster per system, double-float
    vector arithmetic), "cluster_fp64" (the same in FP64), "stream" (one
    launch per pass, warp-sized units, double-float vector arithmetic) or
    "auto".  The returned object keeps the tensors alive."""
    o = N.qcp_options()
    N.lib().qcp_default_options(ctypes.byref(o))
    o.rtol, o.maxiter, o.check_every = float(rtol), int(maxiter), int(check_every)
    o.use_graph, o.compute_residual, o.kink_tol = int(bool(use_graph)), int(bool(compute_residual)), float(kink_tol)
    o.precond = _PRECOND[precond] if isinstance(precond, str) else int(precond)
    o.engine = _ENGINE[engine] if isinstance(engine, str) else int(engine)
    o.solver = {"lsqr": 0, "lsmr": 1}[solver] if isinstance(solver, str) else int(solver)
    keep = []
    for name, t in (("warm_start", warm_start), ("precond_d", precond_d)):
        if t is not None:
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
                raise ValueError(f"{name} must be a float64 CUDA tensor")
            t = t.contiguous()
            keep.append(t)
            setattr(o, name, t.data_ptr())
    o._keep = keep
    return o


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream or None)


class Plan:
    """A plan (include/qcpd.h: qcp_plan_create / qcp_batch_plan_create)."""

    def __init__(self, problems, dtype=torch.float64, max_rhs=1, batched=False, stream=None):
        if dtype not in _DT:
            raise ValueError("dtype must be torch.float64 or torch.float32")
        self.dtype = dtype
        self.problems = list(problems)
        self.batched = batched
        self.max_rhs = max_rhs
        self.device = self.problems[0].q.device
        L = N.lib()
        c = [_c_problem(p) for p in self.problems]
        handle = ctypes.c_void_p()
        sh = _stream_handle(stream)
        if batched:
            probs = (N.qcp_problem * len(c))(*[x[0] for x in c])
            sols = (N.qcp_solution * len(c))(*[x[1] for x in c])
            code = L.qcp_batch_plan_create(len(c), probs, sols, _DT[dtype], sh, ctypes.byref(handle))
        else:
            if len(c) != 1:
                raise ValueError("a single-problem plan takes one problem")
            code = L.qcp_plan_create(ctypes.byref(c[0][0]), ctypes.byref(c[0][1]), _DT[dtype], int(max_rhs), sh,
                                     ctypes.byref(handle))
        _check(code, "qcp_plan_create")
        self._h = handle
        sizes = [ctypes.c_int64() for _ in range(5)]
        _check(L.qcp_plan_sizes(self._h, *[ctypes.byref(s) for s in sizes]), "qcp_plan_sizes")
        self.nprob, self.n_total, self.m_total, self.nnzP_total, self.nnzA_total = [s.value for s in sizes]

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().qcp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def last_launches(self) -> int:
        return int(N.lib().qcp_plan_last_launches(self._h))

    def last_timing(self):
        """(device ms of the iteration chunks, pass launches in them) of the last call."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(N.lib().qcp_plan_last_timing(self._h, ctypes.byref(ms), ctypes.byref(n)), "qcp_plan_last_timing")
        return ms.value, n.value

    def last_shared_passes(self) -> int:
        """System passes of the last call that shared a launch's read of M
        (paired stream iterations; 0 otherwise)."""
        n = ctypes.c_int64()
        _check(N.lib().qcp_plan_last_shared_passes(self._h, ctypes.byref(n)), "qcp_plan_last_shared_passes")
        return n.value

    def last_engine(self) -> str:
        """Engine of the last call: passes, persistent, cluster, cluster_fp64 or stream."""
        e = N.lib().qcp_plan_last_engine(self._h)
        return {v: k for k, v in _ENGINE.items()}.get(e, str(e))

    def autotune(self, mode="jvp", nsys=None, iters=64, opts=None):
        """Time every engine / schedule candidate on this plan (qcp_plan_autotune)
        and keep the fastest for engine="auto".  Returns (best, all), dicts
        with engine, cluster_ctas, tile_nnz and us_per_pass."""
        cap = 32
        entries = (N.qcp_tune_entry * cap)()
        count = ctypes.c_int32()
        best = N.qcp_tune_entry()
        o = opts if opts is not None else options()
        nsys = self.nprob if self.batched else (nsys or 1)
        _check(N.lib().qcp_plan_autotune(self._h, ctypes.byref(o), 0 if mode == "jvp" else 1, int(nsys), int(iters),
                                         entries, cap, ctypes.byref(count), ctypes.byref(best)),
               "qcp_plan_autotune")
        names = {v: k for k, v in _ENGINE.items()}
        d = lambda e: {"engine": names.get(e.engine, str(e.engine)), "cluster_ctas": e.cluster_ctas,
                       "tile_nnz": e.tile_nnz, "us_per_pass": e.us_per_pass}
        return d(best), [d(entries[i]) for i in range(min(count.value, cap))]

    def set_cluster(self, max_ctas: int = 0):
        """CTAs per system of the cluster engine (0: chosen per call)."""
        _check(N.lib().qcp_plan_set_cluster(self._h, int(max_ctas)), "qcp_plan_set_cluster")

    def set_equilibration(self, sweeps: int = 1):
        """Sweeps of the row/column equilibration (1 to 64, before the first
        derivative or autotune call); more sweeps mean fewer Krylov
        iterations on badly scaled problems, with the same outputs."""
        _check(N.lib().qcp_plan_set_equilibration(self._h, int(sweeps)), "qcp_plan_set_equilibration")

    def set_barrier_wait(self, polls: int = 0, hold_ns: int = 0):
        """Bound of the persistent engine's barrier waits (0: the default) and
        a hold of CTA 0 before its first barrier (0: none; exercises the
        timeout path)."""
        _check(N.lib().qcp_plan_set_barrier_wait(self._h, int(polls), int(hold_ns)), "qcp_plan_set_barrier_wait")

    def set_stream_pairing(self, on: bool = True):
        """Stream engine: iterate a call's JVP and VJP ranges in step, one
        read of M per launch for both (True, the default), or one range
        after the other (False)."""
        _check(N.lib().qcp_plan_set_stream_pairing(self._h, 1 if on else 0), "qcp_plan_set_stream_pairing")

    def set_schedule(self, tile_nnz: int = 4096, long_row: int = 512, long_chunk: int = 1 << 20):
        _check(N.lib().qcp_plan_set_schedule(self._h, int(tile_nnz), int(long_row), int(long_chunk)),
               "qcp_plan_set_schedule")

    def _vec(self, a, n):
        t = _t(a, self.device, self.dtype)
        if t.numel() != n:
            raise ValueError(f"expected {n} values, got {t.numel()}")
        return t

    def _run(self, fn, k, ins, outs_sizes, opts, allow):
        nsys = self.nprob if self.batched else (k if k is not None else 1)
        infos = (N.qcp_info * nsys)()
        outs = [torch.empty(sz, device=self.device, dtype=self.dtype) for sz in outs_sizes]
        o = opts if opts is not None else options()
        args = [self._h, ctypes.byref(o)]
        if k is not None and not self.batched:
            args.append(int(k))
        args += [_vp(t) for t in ins] + [_vp(t) for t in outs] + [infos]
        code = fn(*args)
        _check(code, fn.__name__, ok=allow)
        return outs, [_info_dict(i) for i in infos], code


def _info_dict(i):
    return {"status": N.STATUS_NAMES.get(i.status, i.status), "iters": int(i.iters),
            "rel_residual": float(i.rel_residual), "rel_residual_est": float(i.rel_residual_est),
            "kink_margin": float(i.kink_margin)}


_ALLOW = (N.QCP_OK, N.QCP_NOT_CONVERGED, N.QCP_WARN_NEAR_KINK)


def qcp_plan_create(problem: ProblemTensors, dtype=torch.float64, max_rhs=1, stream=None) -> Plan:
    return Plan([problem], dtype=dtype, max_rhs=max_rhs, batched=False, stream=stream)


def qcp_batch_plan_create(problems, dtype=torch.float64, stream=None) -> Plan:
    return Plan(problems, dtype=dtype, batched=True, stream=stream)


def qcp_derivative_jvp(plan: Plan, dP, dA, dq, db, opts=None):
    """(dx, dy, ds, info) = D S(theta)[dP, dA, dq, db]  (Sec. 3.1)."""
    ins = [plan._vec(dP, plan.nnzP_total), plan._vec(dA, plan.nnzA_total), plan._vec(dq, plan.n_total),
           plan._vec(db, plan.m_total)]
    (dx, dy, ds), info, _ = plan._run(N.lib().qcp_derivative_jvp, None, ins,
                                      [plan.n_total, plan.m_total, plan.m_total], opts, _ALLOW)
    return dx, dy, ds, info


def qcp_derivative_jvp_noalloc(plan: Plan, dP, dA, dq, db, out=None, opts=None):
    """qcp_derivative_jvp with the call's scratch in the library's static
    device array (include/qcpd.h).  Pass preallocated outputs in `out`
    (dx, dy, ds) to keep the call itself free of device allocation."""
    ins = [plan._vec(dP, plan.nnzP_total), plan._vec(dA, plan.nnzA_total), plan._vec(dq, plan.n_total),
           plan._vec(db, plan.m_total)]
    if out is None:
        out = [torch.empty(sz, device=plan.device, dtype=plan.dtype)
               for sz in (plan.n_total, plan.m_total, plan.m_total)]
    info = (N.qcp_info * 1)()
    o = opts if opts is not None else options()
    code = N.lib().qcp_derivative_jvp_noalloc(plan.handle, ctypes.byref(o), *[_vp(t) for t in ins],
                                              *[_vp(t) for t in out], info)
    _check(code, "qcp_derivative_jvp_noalloc", ok=_ALLOW)
    return out[0], out[1], out[2], [_info_dict(info[0])]


def qcp_derivative_vjp(plan: Plan, wx, wy, ws, opts=None):
    """(dP, dA, dq, db, info) = D S(theta)^T [wx, wy, ws]  (Sec. 3.2)."""
    ins = [plan._vec(wx, plan.n_total), plan._vec(wy, plan.m_total), plan._vec(ws, plan.m_total)]
    (dP, dA, dq, db), info, _ = plan._run(N.lib().qcp_derivative_vjp, None, ins,
                                          [plan.nnzP_total, plan.nnzA_total, plan.n_total, plan.m_total],
                                          opts, _ALLOW)
    return dP, dA, dq, db, info


def qcp_derivative_jvp_multi(plan: Plan, k, dP, dA, dq, db, opts=None):
    """k directions at once; inputs/outputs hold the k directions back to back."""
    ins = [plan._vec(dP, k * plan.nnzP_total), plan._vec(dA, k * plan.nnzA_total),
           plan._vec(dq, k * plan.n_total), plan._vec(db, k * plan.m_total)]
    (dx, dy, ds), info, _ = plan._run(N.lib().qcp_derivative_jvp_multi, k, ins,
                                      [k * plan.n_total, k * plan.m_total, k * plan.m_total], opts, _ALLOW)
    return dx, dy, ds, info


def qcp_derivative_vjp_multi(plan: Plan, k, wx, wy, ws, opts=None):
    ins = [plan._vec(wx, k * plan.n_total), plan._vec(wy, k * plan.m_total), plan._vec(ws, k * plan.m_total)]
    (dP, dA, dq, db), info, _ = plan._run(N.lib().qcp_derivative_vjp_multi, k, ins,
                                          [k * plan.nnzP_total, k * plan.nnzA_total, k * plan.n_total,
                                           k * plan.m_total], opts, _ALLOW)
    return dP, dA, dq, db, info


def qcp_derivative_jvp_vjp_multi(plan: Plan, kj, dP, dA, dq, db, kv, wx, wy, ws, opts=None):
    """kj JVPs and kv VJPs of a single-problem plan in one call (the cluster
    engine runs the two kinds side by side).  Returns ((dx, dy, ds),
    (gP, gA, gq, gb), info) with info listing the JVPs first."""
    if plan.batched:
        raise ValueError("qcp_derivative_jvp_vjp_multi takes a single-problem plan")
    jin = [plan._vec(dP, kj * plan.nnzP_total), plan._vec(dA, kj * plan.nnzA_total),
           plan._vec(dq, kj * plan.n_total), plan._vec(db, kj * plan.m_total)]
    vin = [plan._vec(wx, kv * plan.n_total), plan._vec(wy, kv * plan.m_total), plan._vec(ws, kv * plan.m_total)]
    e = lambda n: torch.empty(n, device=plan.device, dtype=plan.dtype)
    jout = [e(kj * plan.n_total), e(kj * plan.m_total), e(kj * plan.m_total)]
    vout = [e(kv * plan.nnzP_total), e(kv * plan.nnzA_total), e(kv * plan.n_total), e(kv * plan.m_total)]
    infos = (N.qcp_info * (kj + kv))()
    o = opts if opts is not None else options()
    code = N.lib().qcp_derivative_jvp_vjp_multi(plan.handle, ctypes.byref(o), int(kj), *[_vp(t) for t in jin],
                                                *[_vp(t) for t in jout], int(kv), *[_vp(t) for t in vin],
                                                *[_vp(t) for t in vout], infos)
    _check(code, "qcp_derivative_jvp_vjp_multi", ok=_ALLOW)
    return tuple(jout), tuple(vout), [_info_dict(i) for i in infos]
