"""ctypes declarations of the C ABI in include/qcpd.h.

Loading fails loudly when libqcpd.so has not been built: there is no
fallback implementation of any step.
"""
import ctypes
import os

from .buildlib import LIB

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

QCP_OK, QCP_ERR_ARG, QCP_ERR_CUDA, QCP_ERR_ALLOC = 0, 1, 2, 3
QCP_NOT_CONVERGED, QCP_BREAKDOWN, QCP_ERR_TIMEOUT, QCP_WARN_NEAR_KINK = 4, 5, 6, 7
STATUS_NAMES = {0: "QCP_OK", 1: "QCP_ERR_ARG", 2: "QCP_ERR_CUDA", 3: "QCP_ERR_ALLOC",
                4: "QCP_NOT_CONVERGED", 5: "QCP_BREAKDOWN", 6: "QCP_ERR_TIMEOUT",
                7: "QCP_WARN_NEAR_KINK"}
QCP_F64, QCP_F32 = 0, 1
QCP_PRECOND_NONE, QCP_PRECOND_EQUILIBRATE, QCP_PRECOND_DIAG, QCP_PRECOND_JACOBI = 0, 1, 2, 3
QCP_ENGINE_PASSES, QCP_ENGINE_PERSISTENT, QCP_ENGINE_CLUSTER, QCP_ENGINE_AUTO, QCP_ENGINE_CLUSTER_FP64 = 0, 1, 2, 3, 4
QCP_ENGINE_STREAM = 5


class qcp_csr(ctypes.Structure):
    _fields_ = [("nrows", c_int64), ("ncols", c_int64), ("nnz", c_int64),
                ("indptr", c_void_p), ("indices", c_void_p), ("values", c_void_p)]


class qcp_cone(ctypes.Structure):
    _fields_ = [("nblocks", c_int32), ("type", c_void_p), ("dim", c_void_p), ("param", c_void_p)]


class qcp_problem(ctypes.Structure):
    _fields_ = [("n", c_int64), ("m", c_int64), ("P_upper", qcp_csr), ("A", qcp_csr), ("AT", qcp_csr),
                ("AT_perm", c_void_p), ("q", c_void_p), ("b", c_void_p), ("K", qcp_cone)]


class qcp_solution(ctypes.Structure):
    _fields_ = [("x", c_void_p), ("y", c_void_p), ("s", c_void_p)]


class qcp_options(ctypes.Structure):
    _fields_ = [("solver", c_int32), ("rtol", c_double), ("maxiter", c_int64), ("check_every", c_int32),
                ("use_graph", c_int32), ("compute_residual", c_int32), ("precond", c_int32),
                ("engine", c_int32), ("kink_tol", c_double),
                ("warm_start", c_void_p), ("precond_d", c_void_p)]


class qcp_info(ctypes.Structure):
    _fields_ = [("status", c_int32), ("iters", c_int64), ("rel_residual", c_double),
                ("rel_residual_est", c_double), ("kink_margin", c_double)]


class qcp_tune_entry(ctypes.Structure):
    _fields_ = [("engine", c_int32), ("cluster_ctas", c_int32), ("tile_nnz", c_int32), ("pad", c_int32),
                ("us_per_pass", c_double)]


_lib = None


def lib():
    """The loaded libqcpd.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"libqcpd.so not found at {LIB}: run paper_2508_17522_gb300.build.build() "
                          "(nvcc for sm_103a) first; the library has no CPU fallback")
    L = ctypes.CDLL(LIB)
    P = ctypes.POINTER
    L.qcp_last_error.restype = ctypes.c_char_p
    L.qcp_last_error.argtypes = []
    L.qcp_default_options.restype = None
    L.qcp_default_options.argtypes = [P(qcp_options)]
    L.qcp_version.restype = c_int32
    L.qcp_version.argtypes = []
    L.qcp_plan_create.restype = ctypes.c_int
    L.qcp_plan_create.argtypes = [P(qcp_problem), P(qcp_solution), ctypes.c_int, c_int32, c_void_p,
                                  P(c_void_p)]
    L.qcp_batch_plan_create.restype = ctypes.c_int
    L.qcp_batch_plan_create.argtypes = [c_int32, P(qcp_problem), P(qcp_solution), ctypes.c_int, c_void_p,
                                        P(c_void_p)]
    L.qcp_plan_destroy.restype = ctypes.c_int
    L.qcp_plan_destroy.argtypes = [c_void_p]
    L.qcp_plan_sizes.restype = ctypes.c_int
    L.qcp_plan_sizes.argtypes = [c_void_p] + [P(c_int64)] * 5
    for name in ("qcp_derivative_jvp", "qcp_derivative_vjp", "qcp_derivative_jvp_noalloc"):
        f = getattr(L, name)
        f.restype = ctypes.c_int
        f.argtypes = [c_void_p, P(qcp_options)] + [c_void_p] * 7 + [P(qcp_info)]
    for name in ("qcp_derivative_jvp_multi", "qcp_derivative_vjp_multi"):
        f = getattr(L, name)
        f.restype = ctypes.c_int
        f.argtypes = [c_void_p, P(qcp_options), c_int32] + [c_void_p] * 7 + [P(qcp_info)]
    L.qcp_derivative_jvp_vjp_multi.restype = ctypes.c_int
    L.qcp_derivative_jvp_vjp_multi.argtypes = ([c_void_p, P(qcp_options), c_int32] + [c_void_p] * 7 + [c_int32]
                                               + [c_void_p] * 7 + [P(qcp_info)])
    L.qcp_plan_autotune.restype = ctypes.c_int
    L.qcp_plan_autotune.argtypes = [c_void_p, P(qcp_options), c_int32, c_int32, c_int32, P(qcp_tune_entry), c_int32,
                                    P(c_int32), P(qcp_tune_entry)]
    L.qcp_plan_set_schedule.restype = ctypes.c_int
    L.qcp_plan_set_schedule.argtypes = [c_void_p, c_int32, c_int32, c_int32]
    for name, args in (("qcp_plan_last_solution", [c_void_p, c_void_p]),
                       ("qcp_plan_scalings", [c_void_p, c_void_p, c_void_p]),
                       ("qcp_plan_features", [c_void_p, c_void_p]),
                       ("qcp_mlp_create", [c_int32, c_void_p, P(c_void_p)]),
                       ("qcp_mlp_destroy", [c_void_p]),
                       ("qcp_mlp_set_params", [c_void_p, c_void_p]),
                       ("qcp_mlp_get_params", [c_void_p, c_void_p]),
                       ("qcp_mlp_set_input_norm", [c_void_p, c_void_p, c_void_p]),
                       ("qcp_mlp_forward", [c_void_p, c_void_p, c_int32, c_void_p]),
                       ("qcp_mlp_train_step", [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_float,
                                               P(c_double), c_void_p]),
                       ("qcp_mlp_decode", [c_void_p, c_void_p, c_int64, c_double, c_void_p, c_void_p, c_void_p])):
        f = getattr(L, name)
        f.restype = ctypes.c_int
        f.argtypes = args
    L.qcp_mlp_param_count.restype = c_int32
    L.qcp_mlp_param_count.argtypes = []
    L.qcp_plan_last_engine.restype = ctypes.c_int
    L.qcp_plan_last_engine.argtypes = [c_void_p]
    L.qcp_plan_set_cluster.restype = ctypes.c_int
    L.qcp_plan_set_cluster.argtypes = [c_void_p, c_int32]
    L.qcp_plan_set_equilibration.restype = ctypes.c_int
    L.qcp_plan_set_equilibration.argtypes = [c_void_p, c_int32]
    L.qcp_plan_set_barrier_wait.restype = ctypes.c_int
    L.qcp_plan_set_barrier_wait.argtypes = [c_void_p, c_int64, c_int64]
    L.qcp_plan_set_stream_pairing.restype = ctypes.c_int
    L.qcp_plan_set_stream_pairing.argtypes = [c_void_p, ctypes.c_int32]
    L.qcp_plan_last_shared_passes.restype = ctypes.c_int
    L.qcp_plan_last_shared_passes.argtypes = [c_void_p, ctypes.POINTER(c_int64)]
    L.qcp_plan_last_launches.restype = c_int64
    L.qcp_plan_last_launches.argtypes = [c_void_p]
    L.qcp_plan_last_timing.restype = ctypes.c_int
    L.qcp_plan_last_timing.argtypes = [c_void_p, P(c_double), P(c_int64)]
    _lib = L
    return L


def last_error() -> str:
    return lib().qcp_last_error().decode(errors="replace")


class QCPError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {last_error()}")
