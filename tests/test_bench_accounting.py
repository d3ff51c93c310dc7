"""bench.py's byte model on CPU.

One product with F or F^T must move M's entries (FP64 value and int32
column: 12 B each; P's upper triangle once, the least a symmetric product
needs, and A twice, as A and A^T), the row pointers, and the LSQR vector
updates; a paired stream launch runs that product for two systems and reads
M once.  The roofline's algorithmic bytes must count M once per shared
launch, so a fully paired run moves M once per two system passes.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import qcpgen as g  # noqa: E402


def test_matrix_and_vector_bytes_of_config1():
    prob = g.config1(0)
    mat, vec = bench.algorithmic_bytes_split(prob)
    # P's upper triangle and A twice (A and A^T), 12 bytes an entry; 4-byte
    # row pointers of the three CSR arrays (P, A, A^T: n + 1, m + 1, n + 1)
    n, m = prob.n, prob.m
    entries = 2 * prob.A.nnz + prob.P.nnz
    assert mat == 12 * entries + 4 * ((n + 1) + (m + 1) + (n + 1))
    assert vec > 0
    assert bench.algorithmic_bytes_per_pass(prob) == pytest.approx(mat + vec)


@pytest.mark.parametrize("iters", [(10, 10), (7, 12)])
def test_paired_launches_count_the_matrix_once(iters):
    prob = g.config1(1)
    mat, vec = bench.algorithmic_bytes_split(prob)
    sys_passes = 2 * sum(iters)
    shared = 2 * min(iters)                 # launches that ran a product for both systems
    launches = sys_passes - shared          # paired launches count once
    alg = (mat + vec) * sys_passes - mat * shared
    # every launch reads M once; every system pass moves its own vectors
    assert alg == pytest.approx(mat * launches + vec * sys_passes)
