"""GB300 (sm_103a) library for the derivative of a quadratic cone program's
solution map (arXiv 2508.17522): forward (JVP) and adjoint (VJP) products
through the implicit function theorem on the homogeneous embedding, behind
the C ABI of include/qcpd.h.  The CUDA library is loaded on first use and
there is no CPU fallback."""
from .api import (  # noqa: F401
    Plan, ProblemTensors, options, problem_tensors, qcp_batch_plan_create, qcp_derivative_jvp,
    qcp_derivative_jvp_multi, qcp_derivative_jvp_noalloc, qcp_derivative_jvp_vjp_multi, qcp_derivative_vjp,
    qcp_derivative_vjp_multi,
    qcp_plan_create,
)
from .autograd import QCPSolution, qcp_layer  # noqa: F401
from .buildlib import build  # noqa: F401
