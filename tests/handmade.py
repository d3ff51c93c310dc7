"""Hand-written small QCPs for tests (built from dense data)."""
import numpy as np
import scipy.sparse as sp

from qcpgen.problems import CSR, QCP, _transpose_with_perm


def csr_dense(M, keep_zeros=False):
    M = np.atleast_2d(np.asarray(M, dtype=np.float64))
    if keep_zeros:
        r, c = np.nonzero(np.ones_like(M))
        S = sp.csr_matrix((M[r, c], (r, c)), shape=M.shape)
    else:
        S = sp.csr_matrix(M)
    S.sort_indices()
    return CSR(M.shape[0], M.shape[1], S.indptr.astype(np.int64), S.indices.astype(np.int32),
               S.data.astype(np.float64))


def qcp_from_dense(P, A, q, b, cones, x, y, s):
    P = np.atleast_2d(np.asarray(P, dtype=np.float64))
    A = np.asarray(A, dtype=np.float64).reshape(-1, P.shape[0])
    Pu = csr_dense(np.triu(P), keep_zeros=False)
    Ac = csr_dense(A)
    AT, perm = _transpose_with_perm(Ac)
    return QCP(P.shape[0], A.shape[0], Pu, Ac, AT, perm, np.asarray(q, float).ravel(),
               np.asarray(b, float).ravel(), np.array([c[0] for c in cones], np.int32),
               np.array([c[1] for c in cones], np.int32), np.asarray(x, float).ravel(),
               np.asarray(y, float).ravel(), np.asarray(s, float).ravel(), {})
