"""CPU FP64 oracle for the derivative of a QCP's solution map.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the library itself never does,
and it shares no code with the library (only the seeded input generator
`qcpgen` serves both).

Contents, each following the paper's own definitions (arXiv 2508.17522):
  cones        projections onto K* and their derivatives (Appendix A)
  embedding    Q, the residual map R, its normalisation N, D_u Q, F = D_z N,
               D_theta Q and its adjoint, phi and D phi (Sec. 2.2-2.4)
  derivative   JVP and VJP of the solution map (Sec. 3.1, 3.2), by dense LU
               of a bordered F, and matrix-free by LSMR as the paper does
  qp_kkt       closed-form derivatives of strictly complementary QPs through
               their reduced KKT system (a pin, not part of the method)
  newton_fd    finite differences of the solution map by re-solving
               R(z, theta) = 0 with Newton (a pin, not part of the method)

Parity status of every function is "pinned" by the tests under
tests/test_oracle_*.py; no function here is parity-unpinned.
"""
