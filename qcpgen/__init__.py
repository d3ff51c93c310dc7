"""Seeded synthetic inputs for the QCP solution-map derivative.

This package builds quadratic cone programs whose optimal primal-dual triple
(x*, y*, s*) is known by construction (the optimality conditions of the
conic pair, Sec. 2.1 "Optimality conditions", hold exactly up to rounding),
plus seeded perturbation directions.  It is shared by the CPU oracle, the GPU
tests and the benchmark, and it holds none of the derivative method's
arithmetic: no cone projection, no embedding, no residual map, no Krylov
solve.  It only draws random data and assembles problem data from the drawn
optimum (b = A x* + s*, q = -P x* - A^T y*).
"""
from .problems import (  # noqa: F401
    ZERO, NONNEG, SOC, PSD, EXP, POW, CSR, QCP, Directions,
    config1, config2, config3, config4, config5_family, paper_example, small_qcp,
    unconstrained_qp, equality_qp, make_directions, make_directions_batch,
    round_to_fp32, with_optimum, cone_dims_ok,
)
