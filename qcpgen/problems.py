"""Seeded QCP instances with a known optimum, and seeded directions.

Every instance is built backwards from a drawn primal-dual triple
(x*, y*, s*) that satisfies the conic optimality conditions of Sec. 2.1
("Optimality conditions"): s* in K, y* in K*, s*^T y* = 0, and then
b = A x* + s*, q = -P x* - A^T y*.  The triple is strictly complementary and
the active constraints have full row rank, so the solution map is
single-valued and differentiable there (the regularity the implicit function
theorem of Sec. 2.4 needs).

Cone blocks are listed in row order as (type, dim) with type ZERO (the cone
{0}), NONNEG (the nonnegative orthant), SOC (the second-order cone, stored
(t, u) with t first, Appendix A) or PSD (the positive semidefinite cone of
order k, dim = k (k + 1) / 2, a symmetric matrix stored as its upper
triangle column by column with the off-diagonal entries times sqrt 2), EXP
(the exponential cone, dim 3) or POW (the power cone of exponent a, dim 3,
Appendix A; a in QCP.cone_param).

The five named workloads follow the problem descriptions of the benchmark
configurations; the readings of under-specified points are:
  * "half active" R+ rows and the SOC case mix are capped so that the number
    of active constraint directions stays at or below n (at or below 0.9 n
    for the larger workloads), else no derivative exists;
  * an SOC block on a boundary ray contributes one active direction, a block
    with s = 0 contributes all of its rows, a block with y = 0 none;
  * the 8000-row learned-preconditioner family has blocks
    1 + 5000 + 2001 + 998 = 8000 rows (the stated 999 would overshoot m);
  * "P low-rank(k=n/10)" is stored densely in the upper CSR;
  * "200k random symmetric nnz" are 200k stored upper entries, and P is made
    positive definite by diagonal dominance, P_ii = sum_j |P_ij| + 1e-3.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import structural_rank

ZERO, NONNEG, SOC, PSD, EXP, POW = 0, 1, 2, 3, 4, 5


# --------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------
@dataclass
class CSR:
    """Compressed sparse rows: int64 row pointers, int32 sorted columns."""
    nrows: int
    ncols: int
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def row_ids(self) -> np.ndarray:
        return np.repeat(np.arange(self.nrows, dtype=np.int64), np.diff(self.indptr))

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.data, self.indices, self.indptr),
                             shape=(self.nrows, self.ncols))

    def astype(self, dtype) -> "CSR":
        return CSR(self.nrows, self.ncols, self.indptr, self.indices,
                   self.data.astype(dtype))


@dataclass
class QCP:
    """One quadratic cone program with its constructed optimum.

    P holds the upper triangle (diagonal included) of a symmetric matrix.
    AT is A's transpose in CSR and AT_perm[k] is the position in A's value
    array of AT's k-th stored value.
    """
    n: int
    m: int
    P: CSR
    A: CSR
    AT: CSR
    AT_perm: np.ndarray
    q: np.ndarray
    b: np.ndarray
    cone_type: np.ndarray
    cone_dim: np.ndarray
    x: np.ndarray
    y: np.ndarray
    s: np.ndarray
    meta: dict = field(default_factory=dict)
    cone_param: np.ndarray = None   # per block: the power cone's exponent (0 elsewhere)

    @property
    def N(self) -> int:
        return self.n + self.m + 1

    @property
    def cones(self):
        return list(zip(self.cone_type.tolist(), self.cone_dim.tolist()))

    def with_values(self, **kw) -> "QCP":
        return dataclasses.replace(self, **kw)


@dataclass
class Directions:
    """A forward perturbation d(theta) and an adjoint vector w.

    dP holds values on P's stored upper pattern, dA on A's pattern.
    """
    dP: np.ndarray
    dA: np.ndarray
    dq: np.ndarray
    db: np.ndarray
    wx: np.ndarray
    wy: np.ndarray
    ws: np.ndarray


# --------------------------------------------------------------------------
# small helpers (data layout only)
# --------------------------------------------------------------------------
def _rng(*key) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


def _csr_from_scipy(M) -> CSR:
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    return CSR(M.shape[0], M.shape[1], M.indptr.astype(np.int64),
               M.indices.astype(np.int32), M.data.astype(np.float64))


def _transpose_with_perm(A: CSR):
    rows = A.row_ids()
    cols = A.indices.astype(np.int64)
    perm = np.lexsort((rows, cols)).astype(np.int64)
    counts = np.bincount(cols, minlength=A.ncols)
    indptr = np.zeros(A.ncols + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    AT = CSR(A.ncols, A.nrows, indptr, rows[perm].astype(np.int32), A.data[perm].copy())
    return AT, perm


def _rows_k_distinct(rng, nrows, ncols, k, weights=None):
    """Column indices: k distinct columns per row, uniform or weighted."""
    k = min(k, ncols)
    if weights is None:
        cols = rng.integers(0, ncols, size=(nrows, k))
    else:
        cdf = np.cumsum(weights / weights.sum())
        cdf[-1] = 1.0
        cols = np.searchsorted(cdf, rng.random((nrows, k)), side="right")
    cols = np.minimum(cols, ncols - 1)
    for _ in range(1000):
        srt = np.sort(cols, axis=1)
        bad = np.nonzero((np.diff(srt, axis=1) == 0).any(axis=1))[0] if k > 1 else np.array([], int)
        if bad.size == 0:
            return np.sort(cols, axis=1)
        if weights is None:
            cols[bad] = rng.integers(0, ncols, size=(bad.size, k))
        else:
            cols[bad] = np.minimum(np.searchsorted(cdf, rng.random((bad.size, k)), side="right"),
                                   ncols - 1)
    raise RuntimeError("could not draw distinct columns")


def _sparse_rows(rng, nrows, ncols, k, weights=None) -> CSR:
    if nrows == 0:
        return CSR(0, ncols, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    cols = _rows_k_distinct(rng, nrows, ncols, k, weights)
    kk = cols.shape[1]
    indptr = np.arange(0, nrows * kk + 1, kk, dtype=np.int64)
    return CSR(nrows, ncols, indptr, cols.reshape(-1).astype(np.int32),
               rng.standard_normal(nrows * kk))


def _bernoulli_sparse(rng, nrows, ncols, density) -> CSR:
    mask = rng.random((nrows, ncols)) < density
    vals = np.where(mask, rng.standard_normal((nrows, ncols)), 0.0)
    r, c = np.nonzero(mask)
    return _csr_from_scipy(sp.csr_matrix((vals[r, c], (r, c)), shape=(nrows, ncols)))


def _upper_csr_from_dense(Pd) -> CSR:
    n = Pd.shape[0]
    iu = np.triu_indices(n)
    counts = n - np.arange(n)
    indptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=indptr[1:])
    return CSR(n, n, indptr, iu[1].astype(np.int32), Pd[iu].astype(np.float64))


def _upper_csr_from_sym_sparse(S) -> CSR:
    return _csr_from_scipy(sp.triu(sp.csr_matrix(S)).tocsr())


def _sym_full(P: CSR) -> sp.csr_matrix:
    U = P.to_scipy()
    return (U + sp.triu(U, k=1).T).tocsr()


def _unit(rng, k):
    v = rng.standard_normal(k)
    nv = np.linalg.norm(v)
    while nv < 1e-3:
        v = rng.standard_normal(k)
        nv = np.linalg.norm(v)
    return v / nv


def _psd_order(d):
    k = int(round((np.sqrt(8 * d + 1) - 1) / 2))
    assert k * (k + 1) // 2 == d, d
    return k


def _sym_to_entries(X):
    """A symmetric matrix as a PSD block's entries (upper triangle column by
    column, off-diagonal entries times sqrt 2)."""
    k = X.shape[0]
    a, j = np.triu_indices(k)
    order = np.lexsort((a, j))                    # column-major over the upper triangle
    a, j = a[order], j[order]
    return np.where(a == j, 1.0, np.sqrt(2.0)) * X[a, j]


def _entries_to_sym(v):
    k = _psd_order(v.shape[0])
    a, j = np.triu_indices(k)
    order = np.lexsort((a, j))
    a, j = a[order], j[order]
    X = np.zeros((k, k))
    X[a, j] = np.where(a == j, 1.0, 1.0 / np.sqrt(2.0)) * v
    X[j, a] = X[a, j]
    return X


def _orthogonal(rng, k):
    Q, R = np.linalg.qr(rng.standard_normal((k, k)))
    return Q * np.sign(np.diag(R))


def cone_dims_ok(cone_type, cone_dim, m) -> bool:
    return int(np.sum(cone_dim)) == m and np.all(np.asarray(cone_dim) >= 1)


# --------------------------------------------------------------------------
# optimum construction
# --------------------------------------------------------------------------
def _optimum(rng, cones, nonneg_active, soc_kind, psd_rank=(), exp_kind=(), pow_spec=()):
    """Draw (y, s) block by block.

    nonneg_active: bool per row of the R+ blocks (concatenated in order).
    soc_kind: one of 'ray', 'yint', 'sint' per SOC block (in order).
    psd_rank: per PSD block (in order), the rank r of s; s = Q diag(sigma) Q^T
        on the first r columns of a random orthogonal Q and y on the other
        k - r columns (eigenvalues ~ U(0.5, 2)), so y s = 0 and y + s > 0.
    exp_kind: per exponential-cone block, 'ray' (s = b (r, 1, e^r) on the
        boundary of K_exp and y = a (-e^r, (r - 1) e^r, 1) on the boundary of
        K_exp*, orthogonal to it), 'sint' (s inside K_exp, y = 0) or 'yint'
        (y inside K_exp*, s = 0); r ~ U(-1, 1), a, b ~ U(0.5, 2).
    pow_spec: per power-cone block (kind, exponent a): 'ray' (s = (u, v,
        +-u^a v^(1-a)) on K_pow's boundary, y = c (a |s3| / u, (1 - a) |s3| / v,
        -sign s3) on K_pow*'s boundary, orthogonal to it), 'sint' or 'yint';
        u, v, c ~ U(0.5, 2).
    """
    m = int(sum(d for _, d in cones))
    y = np.zeros(m)
    s = np.zeros(m)
    r = 0
    ia = 0
    isoc = 0
    ipsd = 0
    iexp = 0
    ipow = 0
    for t, d in cones:
        if t == ZERO:
            y[r:r + d] = rng.standard_normal(d)
        elif t == NONNEG:
            act = nonneg_active[ia:ia + d]
            ia += d
            val = rng.uniform(0.5, 2.0, d)
            y[r:r + d] = np.where(act, val, 0.0)
            s[r:r + d] = np.where(act, 0.0, val)
        elif t == SOC:
            kind = soc_kind[isoc]
            isoc += 1
            if kind == "ray":
                if d < 2:
                    raise ValueError("a boundary ray needs an SOC of dim >= 2")
                ub = _unit(rng, d - 1)
                al, be = rng.uniform(0.5, 2.0, 2)
                y[r] = al
                y[r + 1:r + d] = al * ub
                s[r] = be
                s[r + 1:r + d] = -be * ub
            else:
                rho = rng.uniform(0.0, 1.0)
                u = _unit(rng, d - 1) * rho if d > 1 else np.zeros(0)
                tt = rho + rng.uniform(0.5, 2.0)
                tgt = y if kind == "yint" else s
                tgt[r] = tt
                tgt[r + 1:r + d] = u
        elif t == PSD:
            k = _psd_order(d)
            rk = psd_rank[ipsd]
            ipsd += 1
            Q = _orthogonal(rng, k)
            ev = rng.uniform(0.5, 2.0, k)
            s[r:r + d] = _sym_to_entries((Q[:, :rk] * ev[:rk]) @ Q[:, :rk].T)
            y[r:r + d] = _sym_to_entries((Q[:, rk:] * ev[rk:]) @ Q[:, rk:].T)
        elif t == EXP:
            kind = exp_kind[iexp]
            iexp += 1
            rr = rng.uniform(-1.0, 1.0)
            al, be = rng.uniform(0.5, 2.0, 2)
            er = np.exp(rr)
            if kind == "ray":
                s[r:r + 3] = be * np.array([rr, 1.0, er])
                y[r:r + 3] = al * np.array([-er, (rr - 1.0) * er, 1.0])
            elif kind == "sint":
                s[r:r + 3] = be * np.array([rr, 1.0, er * rng.uniform(1.5, 3.0)])
            else:
                v = rng.standard_normal()
                y[r:r + 3] = np.array([-al, v, al * np.exp(-v / al) / np.e * rng.uniform(1.5, 3.0)])
        elif t == POW:
            kind, a = pow_spec[ipow]
            ipow += 1
            u, v, c = rng.uniform(0.5, 2.0, 3)
            sg = 1.0 if rng.random() < 0.5 else -1.0
            top = u ** a * v ** (1 - a)
            if kind == "ray":
                s[r:r + 3] = [u, v, sg * top]
                y[r:r + 3] = c * np.array([a * top / u, (1 - a) * top / v, -sg])
            elif kind == "sint":
                s[r:r + 3] = [u, v, sg * top * rng.uniform(0.2, 0.8)]
            else:
                w = (u / a) ** a * (v / (1 - a)) ** (1 - a)
                y[r:r + 3] = [u, v, sg * w * rng.uniform(0.2, 0.8)]
        else:
            raise ValueError(f"unknown cone type {t}")
        r += d
    return y, s


def _constraint_rows(A: CSR, cones, y, s) -> sp.csr_matrix:
    """Rows (or row combinations) of A that the optimum holds active."""
    As = A.to_scipy()
    pieces = []
    r = 0
    for t, d in cones:
        if t == ZERO:
            pieces.append(As[r:r + d])
        elif t == NONNEG:
            idx = r + np.nonzero(s[r:r + d] == 0.0)[0]
            if idx.size:
                pieces.append(As[idx])
        elif t == PSD:
            # s = Q_S diag Q_S^T binds the directions svec(N M N^T), N an
            # orthonormal basis of s's null space and M any symmetric matrix
            k = _psd_order(d)
            lam, V = np.linalg.eigh(_entries_to_sym(s[r:r + d]))
            N = V[:, lam <= 1e-9 * max(1.0, float(np.abs(lam).max(initial=0.0)))]
            kn = N.shape[1]
            if kn:
                rows = []
                for j in range(kn):
                    for a in range(j + 1):
                        M = np.zeros((kn, kn))
                        M[a, j] = M[j, a] = 1.0
                        rows.append(_sym_to_entries(N @ M @ N.T))
                pieces.append(sp.csr_matrix(np.array(rows)) @ As[r:r + d])
        else:
            yb, sb = y[r:r + d], s[r:r + d]
            if np.all(sb == 0.0) and np.any(yb != 0.0):      # s = 0: all rows bind
                pieces.append(As[r:r + d])
            elif np.any(yb != 0.0) and np.any(sb != 0.0):    # boundary ray
                pieces.append(sp.csr_matrix(yb[None, :]) @ As[r:r + d])
        r += d
    if not pieces:
        return sp.csr_matrix((0, A.ncols))
    return sp.vstack(pieces).tocsr()


def _full_row_rank(C, mode) -> bool:
    if C.shape[0] == 0:
        return True
    if C.shape[0] > C.shape[1]:
        return False
    if mode == "dense":
        return int(np.linalg.matrix_rank(C.toarray())) == C.shape[0]
    return int(structural_rank(sp.csr_matrix(C))) == C.shape[0]


def _assemble(n, m, P, A, cones, x, y, s, meta, params=None) -> QCP:
    AT, perm = _transpose_with_perm(A)
    Pf = _sym_full(P)
    q = -(Pf @ x) - (A.to_scipy().T @ y)
    b = A.to_scipy() @ x + s
    ct = np.array([c[0] for c in cones], dtype=np.int32)
    cd = np.array([c[1] for c in cones], dtype=np.int32)
    cp = np.zeros(len(cones)) if params is None else np.asarray(params, np.float64)
    return QCP(n, m, P, A, AT, perm, np.asarray(q, np.float64), np.asarray(b, np.float64),
               ct, cd, x, y, s, meta, cp)


def _soc_kinds(rng, nblocks, frac_ray, frac_yint, dims=None):
    kinds = np.array(["sint"] * nblocks, dtype=object)
    perm = rng.permutation(nblocks)
    nray = int(round(frac_ray * nblocks))
    nyint = int(round(frac_yint * nblocks))
    kinds[perm[:nray]] = "ray"
    kinds[perm[nray:nray + nyint]] = "yint"
    if dims is not None:
        for i in range(nblocks):
            if kinds[i] == "ray" and dims[i] < 2:
                kinds[i] = "sint"
    return list(kinds)


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------
def config1(seed: int = 0, max_attempts: int = 200) -> QCP:
    """Tiny QP: n=50, m=80, cone {0}^20 x R+^60, A 80x50 density 0.1,
    P = B B^T/50 + 1e-3 I (B 50x10), half the R+ rows active.

    Active rows are picked greedily so that the 20 zero rows and 30 active R+
    rows are linearly independent; if no such choice exists A is redrawn.
    """
    n, mz, mp = 50, 20, 60
    m = mz + mp
    cones = [(ZERO, mz), (NONNEG, mp)]
    for attempt in range(max_attempts):
        rng = _rng(1001, seed, attempt)
        A = _bernoulli_sparse(rng, m, n, 0.1)
        Ad = A.to_scipy().toarray()
        if np.linalg.matrix_rank(Ad[:mz]) < mz:
            continue
        order = rng.permutation(mp)
        chosen = []
        cur = Ad[:mz]
        rank = mz
        for i in order:
            cand = np.vstack([cur, Ad[mz + i]])
            rk = np.linalg.matrix_rank(cand)
            if rk > rank:
                cur, rank = cand, rk
                chosen.append(i)
                if len(chosen) == mp // 2:
                    break
        if len(chosen) < mp // 2:
            continue
        active = np.zeros(mp, bool)
        active[chosen] = True
        B = rng.standard_normal((n, 10))
        P = _upper_csr_from_dense(B @ B.T / 50.0 + 1e-3 * np.eye(n))
        x = rng.standard_normal(n)
        y, s = _optimum(rng, cones, active, [])
        return _assemble(n, m, P, A, cones, x, y, s,
                         {"config": 1, "seed": seed, "attempts": attempt + 1})
    raise RuntimeError("config1: no differentiable draw")


def config2(seed: int = 0, max_attempts: int = 20, rank_mode: str = "dense") -> QCP:
    """Single SOC QCP: n=2000, m=5500, cone {0}^500 x R+^2000 x SOC(10)^300.

    A has 8 N(0,1) entries per row in random columns; P is the upper part of
    G^T G / n + 1e-4 I with G 400x2000 holding 5 entries per row.  The
    optimum has 1000 active R+ rows and SOC blocks split 150 on boundary rays,
    140 with y = 0 and 10 with s = 0 (1750 active directions <= 0.9 n).
    """
    n, m = 2000, 5500
    cones = [(ZERO, 500), (NONNEG, 2000)] + [(SOC, 10)] * 300
    for attempt in range(max_attempts):
        rng = _rng(1002, seed, attempt)
        A = _sparse_rows(rng, m, n, 8)
        G = _sparse_rows(rng, 400, n, 5).to_scipy()
        S = (G.T @ G) / n + 1e-4 * sp.identity(n)
        P = _upper_csr_from_sym_sparse(S)
        active = np.zeros(2000, bool)
        active[rng.permutation(2000)[:1000]] = True
        kinds = np.array(["sint"] * 300, dtype=object)
        pk = rng.permutation(300)
        kinds[pk[:150]] = "ray"
        kinds[pk[150:160]] = "yint"
        x = rng.standard_normal(n)
        y, s = _optimum(rng, cones, active, list(kinds))
        C = _constraint_rows(A, cones, y, s)
        if not _full_row_rank(C, rank_mode):
            continue
        return _assemble(n, m, P, A, cones, x, y, s,
                         {"config": 2, "seed": seed, "attempts": attempt + 1,
                          "active_dirs": int(C.shape[0])})
    raise RuntimeError("config2: no differentiable draw")


def _lognormal_blocks(rng, rows, mu, sigma, lo, hi):
    dims = []
    left = rows
    while left > 0:
        d = int(np.clip(np.round(rng.lognormal(mu, sigma)), lo, hi))
        d = min(d, left)
        if d < lo and dims:
            dims[-1] += d
        else:
            dims.append(d)
        left -= d
    return dims


def config3(seed: int = 0, max_attempts: int = 10, scale: float = 1.0) -> QCP:
    """Large sparse QCP: n=100000, m=220000, cone {0}^20000 x R+^150000 x
    SOC blocks with lognormal(2, 0.7) sizes clipped to [3, 200] over 50000
    rows.  A has 10 entries per row with power-law column degrees (exponent
    2.2: column weights (rank+1)^(-1/1.2) over a random ranking); P is banded
    (bandwidth 5) plus 200k random upper entries, diagonally dominant.  The
    optimum has 30% of R+ rows active and SOC blocks ~50% ray, ~45% y = 0,
    ~5% s = 0.  `scale` shrinks every size proportionally (tests only).
    """
    n = int(round(100000 * scale))
    mz = int(round(20000 * scale))
    mp = int(round(150000 * scale))
    msoc = int(round(50000 * scale))
    nrand = int(round(200000 * scale))
    for attempt in range(max_attempts):
        rng = _rng(1003, seed, attempt)
        dims = _lognormal_blocks(rng, msoc, 2.0, 0.7, 3, 200)
        cones = [(ZERO, mz), (NONNEG, mp)] + [(SOC, d) for d in dims]
        m = mz + mp + msoc
        rank = rng.permutation(n)
        w = (rank + 1.0) ** (-1.0 / 1.2)
        A = _sparse_rows(rng, m, n, 10, weights=w)
        # P: band of width 5 plus random upper entries, diagonal dominance
        rows, cols = [], []
        for d in range(1, 6):
            i = np.arange(n - d)
            rows.append(i)
            cols.append(i + d)
        ri = rng.integers(0, n, nrand)
        rj = rng.integers(0, n, nrand)
        keep = ri != rj
        ri, rj = np.minimum(ri[keep], rj[keep]), np.maximum(ri[keep], rj[keep])
        rows.append(ri)
        cols.append(rj)
        r_all = np.concatenate(rows)
        c_all = np.concatenate(cols)
        U = sp.coo_matrix((rng.standard_normal(r_all.size), (r_all, c_all)), shape=(n, n)).tocsr()
        U.sum_duplicates()
        absrow = np.asarray(abs(U).sum(axis=1)).ravel() + np.asarray(abs(U).sum(axis=0)).ravel()
        S = U + sp.diags(absrow + 1e-3)
        P = _csr_from_scipy(S)
        active = np.zeros(mp, bool)
        active[rng.permutation(mp)[:int(round(0.3 * mp))]] = True
        kinds = _soc_kinds(rng, len(dims), 0.50, 0.05, dims)
        x = rng.standard_normal(n)
        y, s = _optimum(rng, cones, active, kinds)
        C = _constraint_rows(A, cones, y, s)
        if not _full_row_rank(C, "structural"):
            continue
        return _assemble(n, m, P, A, cones, x, y, s,
                         {"config": 3, "seed": seed, "attempts": attempt + 1,
                          "active_dirs": int(C.shape[0])})
    raise RuntimeError("config3: no differentiable draw")


def _one_batched(rng, n, m, rank_mode):
    msoc = int(round(0.3 * m))
    dims = _lognormal_like_uniform(rng, msoc, 3, 20)
    mp = m - sum(dims)
    cones = ([(NONNEG, mp)] if mp > 0 else []) + [(SOC, d) for d in dims]
    A = _sparse_rows(rng, m, n, 6)
    k = max(1, int(round(n / 10)))
    G = rng.standard_normal((k, n)) / np.sqrt(k)
    P = _upper_csr_from_dense(G.T @ G + 1e-3 * np.eye(n))
    kinds = _soc_kinds(rng, len(dims), 0.50, 0.05, dims)
    ray = sum(1 for kk in kinds if kk == "ray")
    yint = sum(d for kk, d in zip(kinds, dims) if kk == "yint")
    nact = max(0, min(int(round(0.3 * n)), int(0.9 * n) - ray - yint, mp))
    active = np.zeros(mp, bool)
    active[rng.permutation(mp)[:nact]] = True
    x = rng.standard_normal(n)
    y, s = _optimum(rng, cones, active, kinds)
    C = _constraint_rows(A, cones, y, s)
    return (n, m, P, A, cones, x, y, s), _full_row_rank(C, rank_mode)


def _lognormal_like_uniform(rng, rows, lo, hi):
    dims = []
    left = rows
    while left > 0:
        d = int(rng.integers(lo, hi + 1))
        d = min(d, left)
        if d < lo and dims:
            dims[-1] += d
        else:
            dims.append(d)
        left -= d
    return dims


def config4(seed: int = 0, n_problems: int = 512, n_range=(50, 3000), first: int = 0,
            rank_mode: str = "structural"):
    """Batch of independent QCPs of uneven size: n ~ U[50, 3000],
    m = round(U[1.5, 3] n), R+ rows plus SOC blocks of dim U{3..20} on 30%
    of rows, A with 6 entries per row, P = G^T G + 1e-3 I with G (n/10) x n
    (stored densely).  Problem i is drawn from its own stream, so any subset
    [first, first + n_problems) can be drawn alone.
    """
    out = []
    for i in range(first, first + n_problems):
        for attempt in range(20):
            rng = _rng(1004, seed, i, attempt)
            n = int(rng.integers(n_range[0], n_range[1] + 1))
            m = int(round(rng.uniform(1.5, 3.0) * n))
            parts, ok = _one_batched(rng, n, m, rank_mode)
            if ok:
                out.append(_assemble(*parts, {"config": 4, "seed": seed, "index": i,
                                              "attempts": attempt + 1}))
                break
        else:
            raise RuntimeError(f"config4: no differentiable draw for problem {i}")
    return out


@dataclass
class Family:
    """A parametric family: fixed P, A and cones; per-instance optimum."""
    n: int
    m: int
    P: CSR
    A: CSR
    cones: list
    base: tuple
    active: np.ndarray
    kinds: list
    sigma: float
    seed: int

    def instance(self, j: int) -> QCP:
        rng = _rng(1005, self.seed, 7, j)
        x0, y0, s0 = self.base
        x = x0 + self.sigma * rng.standard_normal(self.n)
        y = y0.copy()
        s = s0.copy()
        r = 0
        for t, d in self.cones:
            if t == ZERO:
                y[r:r + d] += self.sigma * rng.standard_normal(d)
            elif t == NONNEG:
                f = np.exp(self.sigma * rng.standard_normal(d))
                y[r:r + d] *= f
                s[r:r + d] *= f
            else:
                al = np.exp(self.sigma * rng.standard_normal()) * y[r]
                be = np.exp(self.sigma * rng.standard_normal()) * s[r]
                ub = y[r + 1:r + d] / max(y[r], 1e-300)
                ub = ub + self.sigma * rng.standard_normal(d - 1) / np.sqrt(d)
                ub /= np.linalg.norm(ub)
                y[r], y[r + 1:r + d] = al, al * ub
                s[r], s[r + 1:r + d] = be, -be * ub
            r += d
        return _assemble(self.n, self.m, self.P, self.A, self.cones, x, y, s,
                         {"config": 5, "seed": self.seed, "instance": j})


def config5_family(seed: int = 0, scale: float = 1.0) -> Family:
    """Learned-preconditioner family: n=5000, m=8000, cone
    {0}^1 x R+^5000 x SOC(2001) x R+^998, A fixed with 6 entries per row,
    P = F^T F + diag(U(0.01, 0.1)) with F 50x5000 dense N(0, 1/50).
    Instances perturb the optimum inside its active pattern (35% of R+ rows
    active, the SOC block on a boundary ray) and rebuild q and b; the
    perturbation scale makes the spread of q and b about 0.1.
    `scale` shrinks n and the block sizes (tests only).
    """
    n = max(8, int(round(5000 * scale)))
    r1 = max(2, int(round(5000 * scale)))
    soc = max(3, int(round(2001 * scale)))
    r2 = max(2, int(round(998 * scale)))
    cones = [(ZERO, 1), (NONNEG, r1), (SOC, soc), (NONNEG, r2)]
    m = 1 + r1 + soc + r2
    for attempt in range(20):
        rng = _rng(1005, seed, attempt)
        A = _sparse_rows(rng, m, n, 6)
        kF = 50 if scale >= 1.0 else max(2, int(round(50 * scale)))
        Fm = rng.standard_normal((kF, n)) / np.sqrt(kF)
        P = _upper_csr_from_dense(Fm.T @ Fm + np.diag(rng.uniform(0.01, 0.1, n)))
        mp = r1 + r2
        active = np.zeros(mp, bool)
        active[rng.permutation(mp)[:int(round(0.35 * mp))]] = True
        kinds = ["ray"]
        x = rng.standard_normal(n)
        y, s = _optimum(rng, cones, active, kinds)
        C = _constraint_rows(A, cones, y, s)
        if not _full_row_rank(C, "structural"):
            continue
        # calibrate the perturbation so that q and b move by about 0.1
        fam = Family(n, m, P, A, cones, (x, y, s), active, kinds, 1.0, seed)
        base = _assemble(n, m, P, A, cones, x, y, s, {})
        probe = dataclasses.replace(fam, sigma=1e-3).instance(2**31)
        dev = np.concatenate([probe.q - base.q, probe.b - base.b])
        fam.sigma = 1e-3 * 0.1 / max(float(np.std(dev)), 1e-300)
        return fam
    raise RuntimeError("config5: no differentiable draw")


def paper_example(seed: int = 0, m: int = 2000, n: int = 1000, frac_active: float = 0.3,
                  max_attempts: int = 20) -> QCP:
    """The shape of the paper's worked example (Sec. 4, "Example"): variables
    (x, r) with x in R^n, r in R^m; constraints
        [C D; E 0; f^T 0] (x, r) + s = b,  s in {0}^m x R+^n x {0},
    C dense m x n, D and E diagonal, objective r^T P r + q^T (x, r) with P
    diagonal (no quadratic term on x).  The values and the optimum are
    drawn, not taken from a solve:
      * C ~ N(0, 1/n), D = -diag(U(0.5, 2)), E = -diag(U(0.5, 2)),
        f ~ U(0.5, 2), P = diag(U(0.5, 2)) on r (stored: m upper entries);
      * frac_active of the x entries are 0 with their R+ row active
        (y ~ U(0.5, 2), s = 0); the others have s = -E_ii x_i ~ U(0.5, 2)
        and y = 0, so b = 0 on the R+ rows as in the example's constraint
        x >= 0; r ~ N(0, 1); y ~ N(0, 1) on the zero rows;
      * b and q follow from the optimality conditions.
    The active rows (m + 1 zero rows and the active R+ rows) have full row
    rank, and the reduced Hessian is positive definite when C has full
    column rank, so the solution map is differentiable at the optimum.
    """
    nv = n + m
    cones = [(ZERO, m), (NONNEG, n), (ZERO, 1)]
    for attempt in range(max_attempts):
        rng = _rng(1006, seed, attempt)
        Cd = rng.standard_normal((m, n)) / np.sqrt(n)
        dD = -rng.uniform(0.5, 2.0, m)
        dE = -rng.uniform(0.5, 2.0, n)
        f = rng.uniform(0.5, 2.0, n)
        p = rng.uniform(0.5, 2.0, m)
        top = sp.hstack([sp.csr_matrix(Cd), sp.diags(dD)])
        mid = sp.hstack([sp.diags(dE), sp.csr_matrix((n, m))])
        bot = sp.hstack([sp.csr_matrix(f[None, :]), sp.csr_matrix((1, m))])
        A = _csr_from_scipy(sp.vstack([top, mid, bot]).tocsr())
        Pm = sp.diags(np.concatenate([np.zeros(n), p])).tocsr()
        Pm.eliminate_zeros()
        P = _upper_csr_from_sym_sparse(Pm)
        active = np.zeros(n, bool)
        active[rng.permutation(n)[:int(round(frac_active * n))]] = True
        y, s = _optimum(rng, cones, active, [])
        x = np.zeros(nv)
        x[:n] = np.where(active, 0.0, s[m:m + n] / -dE)
        x[n:] = rng.standard_normal(m)
        Cr = _constraint_rows(A, cones, y, s)
        if not _full_row_rank(Cr, "structural"):
            continue
        return _assemble(nv, m + n + 1, P, A, cones, x, y, s,
                         {"workload": "paper example", "seed": seed, "attempts": attempt + 1,
                          "active_dirs": int(Cr.shape[0])})
    raise RuntimeError("paper_example: no differentiable draw")


def small_qcp(seed: int, n: int, m_zero: int, m_nonneg: int, soc_dims=(), nnz_per_row: int = 4,
              p_rank: int | None = None, frac_active: float = 0.5, soc_mix=(0.4, 0.2),
              max_attempts: int = 200, psd_orders=(), psd_ranks=None, exp_kinds=(), pow_blocks=()) -> QCP:
    """A small QCP with any mix of blocks, for tests.

    The zero block comes first, then the R+ block, then the SOC blocks, then
    the PSD blocks (orders psd_orders; psd_ranks gives the rank of s in each,
    by default a draw from 0..k), then one exponential-cone block per entry
    of exp_kinds ('ray', 'sint' or 'yint'), then one power-cone block per
    (kind, exponent) of pow_blocks.
    soc_mix = (fraction on rays, fraction with s = 0); the rest have y = 0.
    """
    cones = []
    if m_zero:
        cones.append((ZERO, m_zero))
    if m_nonneg:
        cones.append((NONNEG, m_nonneg))
    cones += [(SOC, int(d)) for d in soc_dims]
    cones += [(PSD, int(k) * (int(k) + 1) // 2) for k in psd_orders]
    cones += [(EXP, 3) for _ in exp_kinds]
    cones += [(POW, 3) for _ in pow_blocks]
    params = [0.0] * (len(cones) - len(pow_blocks)) + [float(a) for _, a in pow_blocks]
    m = (m_zero + m_nonneg + int(sum(soc_dims)) + sum(int(k) * (int(k) + 1) // 2 for k in psd_orders)
         + 3 * len(exp_kinds) + 3 * len(pow_blocks))
    for attempt in range(max_attempts):
        rng = _rng(2000, seed, n, m, attempt)
        A = _sparse_rows(rng, m, n, min(nnz_per_row, n))
        k = p_rank if p_rank is not None else max(1, n // 2)
        B = rng.standard_normal((n, k))
        P = _upper_csr_from_dense(B @ B.T / k + 1e-2 * np.eye(n))
        active = np.zeros(m_nonneg, bool)
        active[rng.permutation(m_nonneg)[:int(round(frac_active * m_nonneg))]] = True
        kinds = _soc_kinds(rng, len(soc_dims), soc_mix[0], soc_mix[1], list(soc_dims))
        ranks = list(psd_ranks) if psd_ranks is not None else [int(rng.integers(0, k + 1)) for k in psd_orders]
        x = rng.standard_normal(n)
        y, s = _optimum(rng, cones, active, kinds, ranks, list(exp_kinds), list(pow_blocks))
        C = _constraint_rows(A, cones, y, s)
        if not _full_row_rank(C, "dense"):
            continue
        return _assemble(n, m, P, A, cones, x, y, s, {"seed": seed, "attempts": attempt + 1}, params)
    raise RuntimeError("small_qcp: no differentiable draw")


def unconstrained_qp(seed: int, n: int) -> QCP:
    """m = 0: minimize (1/2) x^T P x + q^T x with P positive definite."""
    rng = _rng(3000, seed, n)
    B = rng.standard_normal((n, n))
    P = _upper_csr_from_dense(B @ B.T / n + 0.5 * np.eye(n))
    A = CSR(0, n, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    x = rng.standard_normal(n)
    return _assemble(n, 0, P, A, [], x, np.zeros(0), np.zeros(0), {"seed": seed})


def equality_qp(seed: int, n: int, m: int) -> QCP:
    """Cone {0}^m: an equality-constrained QP (needs m <= n)."""
    return small_qcp(seed, n, m, 0, (), nnz_per_row=min(n, 4))


# --------------------------------------------------------------------------
# directions
# --------------------------------------------------------------------------
def make_directions(qcp: QCP, seed: int, index: int = 0) -> Directions:
    rng = _rng(4000, seed, index)
    return Directions(
        dP=rng.standard_normal(qcp.P.nnz), dA=rng.standard_normal(qcp.A.nnz),
        dq=rng.standard_normal(qcp.n), db=rng.standard_normal(qcp.m),
        wx=rng.standard_normal(qcp.n), wy=rng.standard_normal(qcp.m),
        ws=rng.standard_normal(qcp.m))


def make_directions_batch(qcp: QCP, seed: int, k: int):
    return [make_directions(qcp, seed, i) for i in range(k)]


def with_optimum(qcp: QCP, x, y, s) -> QCP:
    """The same P, A and cones with another constructed optimum (x, y, s):
    q = -P x - A^T y and b = A x + s are rebuilt so that (x, y, s) solves the
    pair.  The caller keeps y in K*, s in K and y^T s = 0 blockwise."""
    x, y, s = (np.asarray(a, np.float64).copy() for a in (x, y, s))
    q = -(_sym_full(qcp.P) @ x) - (qcp.A.to_scipy().T @ y)
    b = qcp.A.to_scipy() @ x + s
    return dataclasses.replace(qcp, x=x, y=y, s=s, q=np.asarray(q, np.float64), b=np.asarray(b, np.float64))


def round_to_fp32(qcp: QCP) -> QCP:
    """The same problem with every floating-point array rounded to binary32
    (round to nearest even) and held again in float64."""
    def r(a):
        return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)

    def rc(M: CSR):
        return CSR(M.nrows, M.ncols, M.indptr, M.indices, r(M.data))

    return dataclasses.replace(qcp, P=rc(qcp.P), A=rc(qcp.A), AT=rc(qcp.AT), q=r(qcp.q),
                               b=r(qcp.b), x=r(qcp.x), y=r(qcp.y), s=r(qcp.s))
