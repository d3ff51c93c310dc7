// Plan creation: validation, the combined matrix M = [[P, A^T], [A, 0]],
// the per-problem state of Sec. 3.1's first step (Pi z, g = 2 P x + q,
// kappa = x^T P x, D Pi_{K*}(y - s) per block, Appendix A) and the tile
// schedule.  Everything that touches problem data runs in kernels; the host
// only walks row lengths and cone sizes to cut the rows into tiles.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "qcpd_plan.h"

namespace qcpd {

static int grid_for(int64_t n, int threads) { return (int)std::max<int64_t>(1, (n + threads - 1) / threads); }

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

const char* last_error() { return g_err.c_str(); }

enum ErrBits : int {
    E_PTR = 1,        // bad row pointers
    E_COL = 2,        // column out of range or not strictly increasing
    E_UPPER = 4,      // P has an entry below the diagonal
    E_AT = 8,         // A^T inconsistent with A
    E_PERM = 16,      // AT_perm inconsistent
};

// ---------------------------------------------------------------- validation
__global__ void k_check_csr(const int64_t* ip, const int32_t* ix, int64_t nrows, int64_t ncols, int64_t nnz,
                            int upper, int* err) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r > nrows) return;
    if (r == 0 && ip[0] != 0) atomicOr(err, E_PTR);
    if (r == nrows) {
        if (ip[nrows] != nnz) atomicOr(err, E_PTR);
        return;
    }
    const int64_t a = ip[r], b = ip[r + 1];
    if (a < 0 || b < a || b > nnz) {
        atomicOr(err, E_PTR);
        return;
    }
    int64_t prev = -1;
    for (int64_t k = a; k < b; ++k) {
        const int64_t c = ix[k];
        if (c <= prev || c < 0 || c >= ncols) {
            atomicOr(err, E_COL);
            return;
        }
        if (upper && c < r) {
            atomicOr(err, E_UPPER);
            return;
        }
        prev = c;
    }
}

__global__ void k_rowids(const int64_t* ip, int64_t nrows, int32_t* rid) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    for (int64_t k = ip[r]; k < ip[r + 1]; ++k) rid[k] = (int32_t)r;
}

__device__ __forceinline__ bool same_bits(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_int(a) == __float_as_int(b); }

// For each stored entry of A^T (row c = column of A, index r = row of A)
// find the position of (r, c) in A by binary search; check or produce the
// permutation and that the values agree bit for bit.
template <typename T>
__global__ void k_at_perm(const int64_t* atip, const int32_t* atix, const T* atv, int64_t n, int64_t nnz,
                          const int64_t* aip, const int32_t* aix, const T* av, const int64_t* given,
                          int64_t* perm, int* err) {
    const int64_t kt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (kt >= nnz) return;
    // the A^T row (= A column) of entry kt: last c with atip[c] <= kt
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (atip[mid] <= kt) lo = mid;
        else hi = mid;
    }
    const int64_t c = lo;
    const int32_t r = atix[kt];
    lo = aip[r];
    hi = aip[r + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (aix[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= aip[r + 1] || aix[lo] != c) {
        atomicOr(err, E_AT);
        return;
    }
    if (given && given[kt] != lo) {
        atomicOr(err, E_PERM);
        return;
    }
    if (!same_bits(av[lo], atv[kt])) {
        atomicOr(err, E_AT);
        return;
    }
    perm[kt] = lo;
}

// ---------------------------------------------------------------- M assembly
__global__ void k_lower_keys(const int32_t* rid, const int32_t* pix, int64_t pnz, int32_t n, int32_t* key,
                             int32_t* val) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= pnz) return;
    const int32_t c = pix[k];
    key[k] = (rid[k] == c) ? n : c;  // diagonal entries sort last
    val[k] = (int32_t)k;
}

// lowptr[j] = first position of key >= j among the sorted keys (j = 0..n)
__global__ void k_lowptr(const int32_t* skey, int64_t pnz, int32_t n, int64_t* lowptr) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j > n) return;
    int64_t lo = 0, hi = pnz;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (skey[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    lowptr[j] = lo;
}

// Row lengths of M for one problem, written at global rows [mrow, mrow + N).
__global__ void k_mlen(const int64_t* lowptr, const int64_t* pip, const int64_t* atip, const int64_t* aip,
                       int32_t n, int32_t m, int64_t* len) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r > (int64_t)n + m) return;
    int64_t l = 0;
    if (r < n) l = (lowptr[r + 1] - lowptr[r]) + (pip[r + 1] - pip[r]) + (atip[r + 1] - atip[r]);
    else if (r < (int64_t)n + m) l = aip[r - n + 1] - aip[r - n];
    len[r] = l;
}

// Fill one problem's rows of M: for x-row i the strictly-lower part of P's
// row i (column i of the stored upper part), the stored upper part, then
// A^T's row i shifted by n; for y-row j, A's row j.  One warp per row.
__global__ void k_mfill(const int64_t* mrp, const int64_t* lowptr, const int32_t* sval, const int32_t* prid,
                        const int64_t* pip, const int32_t* pix, const int64_t* atip, const int32_t* atix,
                        const int64_t* perm, const int64_t* aip, const int32_t* aix, int32_t n, int32_t m,
                        int64_t pnz, int32_t* mcol, int32_t* mvmap) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= (int64_t)n + m) return;
    int64_t o = mrp[r];
    if (r < n) {
        const int64_t l0 = lowptr[r], l1 = lowptr[r + 1];
        for (int64_t q = l0 + lane; q < l1; q += 32) {
            const int32_t k = sval[q];
            mcol[o + (q - l0)] = prid[k];
            mvmap[o + (q - l0)] = k;
        }
        o += l1 - l0;
        const int64_t u0 = pip[r], u1 = pip[r + 1];
        for (int64_t k = u0 + lane; k < u1; k += 32) {
            mcol[o + (k - u0)] = pix[k];
            mvmap[o + (k - u0)] = (int32_t)k;
        }
        o += u1 - u0;
        const int64_t t0 = atip[r], t1 = atip[r + 1];
        for (int64_t k = t0 + lane; k < t1; k += 32) {
            mcol[o + (k - t0)] = n + atix[k];
            mvmap[o + (k - t0)] = (int32_t)(pnz + perm[k]);
        }
    } else {
        const int64_t j = r - n;
        const int64_t a0 = aip[j], a1 = aip[j + 1];
        for (int64_t k = a0 + lane; k < a1; k += 32) {
            mcol[o + (k - a0)] = aix[k];
            mvmap[o + (k - a0)] = (int32_t)(pnz + k);
        }
    }
}

template <typename T>
__global__ void k_mvals(const int32_t* mvmap, int64_t k0, int64_t k1, int64_t pnz, const T* pv, const T* av,
                        T* mval) {
    const int64_t k = k0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= k1) return;
    const int32_t v = mvmap[k];
    mval[k] = v < pnz ? pv[v] : av[v - pnz];
}

// ---------------------------------------------------------------- per-row state
// coefA = (q, b), pz = Pi z without tau = (x, y), zy = y - s, row flags of D.
template <typename T>
__global__ void k_rowdata(const T* q, const T* b, const T* x, const T* y, const T* s, const int8_t* ctype,
                          int32_t n, int32_t m, double* coefA, double* coefB, double* pz, double* zy,
                          int8_t* flag) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)n + m + 1;
    if (r >= N) return;
    if (r < n) {
        coefA[r] = (double)q[r];
        pz[r] = (double)x[r];
        zy[r] = 0.0;
        flag[r] = RF_ONE;
    } else if (r < (int64_t)n + m) {
        const int64_t j = r - n;
        coefA[r] = (double)b[j];
        coefB[r] = (double)b[j];
        pz[r] = (double)y[j];
        const double z = (double)y[j] - (double)s[j];
        zy[r] = z;
        const int8_t t = ctype[j];
        flag[r] = (t == QCP_CONE_ZERO) ? RF_ONE : (t == QCP_CONE_NONNEG ? (z > 0.0 ? RF_ONE : RF_ZERO) : RF_SOC);
    } else {
        coefA[r] = 0.0;
        coefB[r] = 0.0;
        pz[r] = 1.0;
        zy[r] = 0.0;
        flag[r] = RF_ONE;
    }
}

// Per SOC block: t, ||u|| of z_y and the case of Appendix A's derivative,
// tested in the projection's order with non-strict inequalities.
template <typename T>
__global__ void k_socprep(SocBlock* blk, int64_t nb, const double* zy) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    SocBlock B = blk[b];
    if (B.kase == kBlockPsd || B.kase == kBlockDense) return;
    double ss = 0.0;
    for (int k = 1 + lane; k < B.dim; k += 32) {
        const double u = (double)zy[B.start + k];
        ss += u * u;
    }
    ss = warp_sum(ss);
    if (lane == 0) {
        const double t = (double)zy[B.start];
        const double r = sqrt(ss);
        B.t = t;
        B.r = r;
        B.kase = (r <= -t) ? 0 : ((r <= t) ? 1 : 2);
        B.h = B.kase == 2 ? 0.5 / r : 0.0;
        B.tq = B.kase == 2 ? t / (r * r) : 0.0;
        blk[b] = B;
    }
}

// Distance to the nearest kink of D Pi: |z_i| on R+ rows, | ||u|| - |t| | on SOC blocks.
__device__ __forceinline__ void atomic_min_nonneg(unsigned long long* slot, double v) {
    atomicMin(slot, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__global__ void k_kink(const double* zy, const int8_t* ctype, int32_t n, int32_t m, const SocBlock* blk, int64_t nb,
                       unsigned long long* slot) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m && ctype[i] == QCP_CONE_NONNEG) atomic_min_nonneg(slot, fabs((double)zy[n + i]));
    if (i < nb && blk[i].kase != kBlockPsd && blk[i].kase != kBlockDense)
        atomic_min_nonneg(slot, fabs(blk[i].r - fabs(blk[i].t)));
}

// Per PSD block (one thread each): the eigendecomposition Z = V diag(lam) V^T
// of its z_y entries by the cyclic Jacobi method (rotations that zero one
// off-diagonal entry at a time, sweeps until the off-diagonal mass is below
// 1e-30 of the total or 60 sweeps), then the weights of D Pi (Appendix A):
// B_pq = 1 when lam_p, lam_q > 0, 0 when neither is, lam_p / (lam_p - lam_q)
// when only lam_p is.  V (column q = eigenvector q) and B go to the block's
// slot of the PSD array; the B half serves as the matrix during the sweeps.
// The kink margin is the smallest |lam|.
__global__ void k_psdprep(SocBlock* blk, int64_t nb, const double* zy, double* psd, unsigned long long* kink) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb || blk[b].kase != kBlockPsd) return;
    const SocBlock Bk = blk[b];
    const int k = Bk.order;
    double* V = psd + Bk.psd;
    double* A = V + k * k;
    const double* z = zy + Bk.start;
    for (int j = 0; j < k; ++j)
        for (int a = 0; a <= j; ++a) {
            const double v = z[j * (j + 1) / 2 + a] * (a == j ? 1.0 : 0.7071067811865476);
            A[a * k + j] = A[j * k + a] = v;
        }
    for (int i = 0; i < k * k; ++i) V[i] = 0.0;
    for (int i = 0; i < k; ++i) V[i * k + i] = 1.0;
    double total = 0.0;
    for (int i = 0; i < k * k; ++i) total += A[i] * A[i];
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) off += 2.0 * A[p * k + q] * A[p * k + q];
        if (!(off > 1e-30 * total)) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = A[p * k + q];
                if (apq == 0.0) continue;
                // the rotation (c, s) with tan(2 theta) = 2 a_pq / (a_qq - a_pp)
                const double th = (A[q * k + q] - A[p * k + p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int r = 0; r < k; ++r) {  // columns p, q
                    const double arp = A[r * k + p], arq = A[r * k + q];
                    A[r * k + p] = c * arp - sn * arq;
                    A[r * k + q] = sn * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {  // rows p, q
                    const double apr = A[p * k + r], aqr = A[q * k + r];
                    A[p * k + r] = c * apr - sn * aqr;
                    A[q * k + r] = sn * apr + c * aqr;
                }
                for (int r = 0; r < k; ++r) {
                    const double vrp = V[r * k + p], vrq = V[r * k + q];
                    V[r * k + p] = c * vrp - sn * vrq;
                    V[r * k + q] = sn * vrp + c * vrq;
                }
            }
    }
    double lam[kPsdMaxOrder];
    double margin = INFINITY;
    for (int i = 0; i < k; ++i) {
        lam[i] = A[i * k + i];
        margin = fmin(margin, fabs(lam[i]));
    }
    for (int p = 0; p < k; ++p)
        for (int q = 0; q < k; ++q) {
            const bool pp = lam[p] > 0.0, pq = lam[q] > 0.0;
            double w;
            if (pp && pq) w = 1.0;
            else if (!pp && !pq) w = 0.0;
            else if (pp) w = lam[p] / (lam[p] - lam[q]);
            else w = lam[q] / (lam[q] - lam[p]);
            A[p * k + q] = w;
        }
    atomic_min_nonneg(kink, margin);
}

// ---- exponential cone K_exp = cl{(x, y, z): y > 0, y e^(x/y) <= z} (Appendix A)
__device__ bool exp_in(double x, double y, double z) {
    if (y == 0.0 && x <= 0.0 && z >= 0.0) return true;
    return y > 0.0 && y * exp(x / y) <= z;
}

__device__ bool exp_dual_in(double u, double v, double w) {
    if (u == 0.0 && v >= 0.0 && w >= 0.0) return true;
    return u < 0.0 && -u * exp(v / u) <= 2.718281828459045 * w;
}

// Squared distance from p to the nearest point of the ray t (r, 1, e^r),
// t >= 0, and the stationarity function of r whose root is the best ray.
__device__ double exp_ray_dist2(double r, const double* p) {
    const double er = exp(r);
    const double aa = r * r + 1.0 + er * er, ap = r * p[0] + p[1] + er * p[2];
    const double t = ap > 0.0 ? ap / aa : 0.0;
    const double d0 = t * r - p[0], d1 = t - p[1], d2 = t * er - p[2];
    return d0 * d0 + d1 * d1 + d2 * d2;
}

__device__ double exp_ray_stat(double r, const double* p) {
    const double er = exp(r);
    const double aa = r * r + 1.0 + er * er, ap = r * p[0] + p[1] + er * p[2];
    return (p[0] + er * p[2]) * aa - ap * (r + er * er);
}

// D Pi of the projection onto K_exp at p (3 x 3, row-major), from the cases
// of Appendix A: I inside K, 0 inside the polar cone, diag(1, 0, 1{z > 0})
// for x < 0 and y < 0 (and when the nearest point lies on the face
// {(x, 0, z): x <= 0, z >= 0}); otherwise the nearest boundary point is
// found over the rays t (r, 1, e^r): a scan of r in [-700, 40] (and r = x/y)
// for the smallest distance, then bisection on the stationarity condition
// in the scan cell (120 halvings), and D Pi is the leading 3 x 3 block of
// J^-1 with J the Jacobian of the optimality conditions (multiplier
// mu = z* - z), inverted by Gauss-Jordan elimination with partial pivoting.
__device__ void exp_dproj(const double* p, double* Dm) {
    for (int i = 0; i < 9; ++i) Dm[i] = 0.0;
    const double x = p[0], y = p[1], z = p[2];
    if (exp_in(x, y, z)) {
        Dm[0] = Dm[4] = Dm[8] = 1.0;
        return;
    }
    if (exp_dual_in(-x, -y, -z)) return;
    if (x < 0.0 && y < 0.0) {
        Dm[0] = 1.0;
        Dm[8] = z > 0.0 ? 1.0 : 0.0;
        return;
    }
    double best = INFINITY, rb = 0.0, step = 0.0;
    for (int i = 0; i <= 6600; ++i) {  // [-700, -40] in steps of 0.1
        const double r = -700.0 + 0.1 * i;
        const double d2 = exp_ray_dist2(r, p);
        if (d2 < best) { best = d2; rb = r; step = 0.1; }
    }
    for (int i = 0; i <= 8000; ++i) {  // [-40, 40] in steps of 0.01
        const double r = -40.0 + 0.01 * i;
        const double d2 = exp_ray_dist2(r, p);
        if (d2 < best) { best = d2; rb = r; step = 0.01; }
    }
    if (y > 0.0 && x / y > -700.0 && x / y < 40.0 && exp_ray_dist2(x / y, p) < best) {
        rb = x / y;
        best = exp_ray_dist2(rb, p);
        step = 0.01;
    }
    double lo = rb - step, hi = rb + step;
    double flo = exp_ray_stat(lo, p), fhi = exp_ray_stat(hi, p);
    double rs = rb;
    if (flo * fhi < 0.0) {
        for (int it = 0; it < 120; ++it) {
            const double mid = 0.5 * (lo + hi);
            const double fm = exp_ray_stat(mid, p);
            if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
        }
        rs = 0.5 * (lo + hi);
    }
    const double er = exp(rs);
    const double aa = rs * rs + 1.0 + er * er, ap = rs * x + y + er * z;
    const double t = ap > 0.0 ? ap / aa : 0.0;
    const double xs = t * rs, ys = t, zs = t * er;
    const double fx = x < 0.0 ? x : 0.0, fz = z > 0.0 ? z : 0.0;  // the face candidate
    const double dray = (xs - x) * (xs - x) + (ys - y) * (ys - y) + (zs - z) * (zs - z);
    const double dface = (fx - x) * (fx - x) + y * y + (fz - z) * (fz - z);
    if (!(ys > 0.0) || dface < dray) {
        Dm[0] = x < 0.0 ? 1.0 : 0.0;
        Dm[8] = z > 0.0 ? 1.0 : 0.0;
        return;
    }
    const double mu = zs - z, e = exp(xs / ys), q = xs / ys;
    double J[4][8] = {
        {1.0 + mu * e / ys, -mu * q * e / ys, 0.0, e, 1, 0, 0, 0},
        {-mu * q * e / ys, 1.0 + mu * q * q * e / ys, 0.0, (1.0 - q) * e, 0, 1, 0, 0},
        {0.0, 0.0, 1.0, -1.0, 0, 0, 1, 0},
        {e, (1.0 - q) * e, -1.0, 0.0, 0, 0, 0, 1}};
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(J[r][c]) > fabs(J[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 8; ++k) {
                const double tmp = J[c][k];
                J[c][k] = J[piv][k];
                J[piv][k] = tmp;
            }
        const double inv = 1.0 / J[c][c];
        for (int k = 0; k < 8; ++k) J[c][k] *= inv;
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            const double f = J[r][c];
            for (int k = 0; k < 8; ++k) J[r][k] -= f * J[c][k];
        }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Dm[i * 3 + j] = J[i][4 + j];
}

// ---- power cone K_pow,a = {(x, y, z): x, y >= 0, x^a y^(1-a) >= |z|} (Appendix A)
__device__ bool pow_in(double x, double y, double z, double a) {
    return x >= 0.0 && y >= 0.0 && pow(x, a) * pow(y, 1.0 - a) >= fabs(z);
}

__device__ bool pow_dual_in(double u, double v, double w, double a) {
    return u >= 0.0 && v >= 0.0 && pow(u / a, a) * pow(v / (1.0 - a), 1.0 - a) >= fabs(w);
}

__device__ void pow_f(double x, double y, double az, double a, double r, double& fx, double& fy) {
    fx = 0.5 * (x + sqrt(x * x + 4.0 * a * r * (az - r)));
    fy = 0.5 * (y + sqrt(y * y + 4.0 * (1.0 - a) * r * (az - r)));
}

__device__ double pow_g(double x, double y, double az, double a, double r) {
    double fx, fy;
    pow_f(x, y, az, a, r, fx, fy);
    return pow(fx, a) * pow(fy, 1.0 - a) - r;
}

// D Pi of the projection onto K_pow,a at p (3 x 3, row-major), from the
// cases of Appendix A: I inside K, 0 inside the polar cone, the z = 0 case
// table, else the formula of its Theorem (Hien 2015, Theorem 3.1) at the
// root r in (0, |z|) of r = f_x(r)^a f_y(r)^(1-a).  r = 0 solves that
// equation as well when x <= 0 or y <= 0, so the bracket starts at the
// largest |z| 10^-k (k >= 1) with a positive residual; 200 bisections.
__device__ void pow_dproj(const double* p, double a, double* Dm) {
    for (int i = 0; i < 9; ++i) Dm[i] = 0.0;
    const double x = p[0], y = p[1], z = p[2];
    if (pow_in(x, y, z, a)) {
        Dm[0] = Dm[4] = Dm[8] = 1.0;
        return;
    }
    if (pow_dual_in(-x, -y, -z, a)) return;
    if (z == 0.0) {
        double d = 0.0;
        if (x > 0.0 && y < 0.0) d = a > 0.5 ? 1.0 : (a < 0.5 ? 0.0 : x / (2.0 * fabs(y) + x));
        else if (y > 0.0 && x < 0.0) d = a < 0.5 ? 1.0 : (a > 0.5 ? 0.0 : y / (2.0 * fabs(x) + y));
        Dm[0] = x > 0.0 ? 1.0 : 0.0;
        Dm[4] = y > 0.0 ? 1.0 : 0.0;
        Dm[8] = d;
        return;
    }
    const double az = fabs(z), sz = z > 0.0 ? 1.0 : -1.0;
    double lo = -1.0, hi = az;
    double scale = az;
    for (int k = 1; k < 300 && lo < 0.0; ++k) {
        scale *= 0.1;
        if (pow_g(x, y, az, a, scale) > 0.0) lo = scale;
    }
    double r = 0.0;
    if (lo > 0.0) {
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (pow_g(x, y, az, a, mid) > 0.0) lo = mid;
            else hi = mid;
        }
        r = 0.5 * (lo + hi);
    }
    double fx, fy;
    pow_f(x, y, az, a, r, fx, fy);
    const double gx = 2.0 * fx - x, gy = 2.0 * fy - y;
    const double cx = a * x / gx, cy = (1.0 - a) * y / gy;
    const double T = -(cx + cy);
    const double L = 2.0 * (az - r) / (az + (az - 2.0 * r) * (cx + cy));
    Dm[0] = 0.5 + x / (2.0 * gx) + a * a * (az - 2.0 * r) * r * L / (gx * gx);
    Dm[1] = Dm[3] = (a - a * a) * (az - 2.0 * r) * r * L / (gx * gy);
    Dm[2] = Dm[6] = sz * a * r * L / gx;
    Dm[4] = 0.5 + y / (2.0 * gy) + (1.0 - a) * (1.0 - a) * (az - 2.0 * r) * r * L / (gy * gy);
    Dm[5] = Dm[7] = sz * (1.0 - a) * r * L / gy;
    Dm[8] = r / az + r / az * T * L;
}

// Per exponential- or power-cone block (one thread each): D Pi onto the
// dual cone at z_y, by the Moreau decomposition D Pi_{K*}(z) = I - D Pi_K(-z).
__global__ void k_expprep(const SocBlock* blk, int64_t nb, const double* zy, double* dense) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb || blk[b].kase != kBlockDense) return;
    const SocBlock B = blk[b];
    const double p[3] = {-zy[B.start], -zy[B.start + 1], -zy[B.start + 2]};
    double Dk[9];
    if (B.cone == QCP_CONE_POW) pow_dproj(p, B.t, Dk);
    else exp_dproj(p, Dk);
    double* D = dense + B.psd;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[i * 3 + j] = (i == j ? 1.0 : 0.0) - Dk[i * 3 + j];
}

// g = 2 P x + q and kappa = x^T P x (Sec. 2.4: the last row of D_u Q at
// tau = 1 is (-(2 P x + q)^T, -b^T, x^T P x)).  P x comes from the columns
// < n of M's x-rows.  One warp per row; kappa through the tile reduction.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pre(const Tile* tiles, const Prob* probs_c, Prob* probs,
                                                  const Sys* psys, Reduce R, const int64_t* mrowptr,
                                                  const int32_t* mcol, const T* mval, const double* coefA,
                                                  double* coefB, const double* pz) {
    __shared__ Scratch scratch;
    const int ti = blockIdx.x;
    const Tile tl = tiles[ti];
    const Sys sy = psys[tl.sys];
    const Prob pr = probs_c[sy.prob];
    const int n = pr.n;
    const int64_t* rp = mrowptr + pr.mrow;
    const double* x = pz + pr.doff;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double kap = 0.0;
    const int rend = (tl.kind == TILE_LONG && tl.cb0 != 0) ? tl.r0 : tl.r1;  // one chunk per long row
    for (int r = tl.r0 + warp; r < rend; r += kWarps) {
        if (r >= n) continue;
        double h = 0.0;
        for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) {
            const int32_t c = mcol[k];
            if (c < n) h += (double)mval[k] * (double)x[c];
        }
        h = warp_sum(h);
        if (lane == 0) {
            coefB[pr.doff + r] = 2.0 * h + coefA[pr.doff + r];
            kap += (double)x[r] * h;
        }
    }
    const Part part = block_sum_part(Part{kap, 0.0, 0.0, 0.0}, &scratch);
    Part tot;
    if (!finish_tile(R, tl, sy.g0, sy.g1, ti, part, &tot, &scratch)) return;
    if (threadIdx.x == 0) probs[sy.prob].kappa = tot.a;
}

// ---------------------------------------------------------------- equilibration
// Diagonal of D = D Pi_{K*}(z_y) per y-row (Appendix A): 0/1 on R+ and zero-
// cone rows; on an SOC block in the formula case t-entry 1/2 and u-entries
// ((t + r) - (t / r^2) u_k^2) / (2 r).
template <typename T>
__global__ void k_dd_rows(const int8_t* flag, int32_t n, int32_t m, double* dd) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r > (int64_t)n + m) return;
    if (r < n || r == (int64_t)n + m) dd[r] = 1.0;
    else if (flag[r] != RF_SOC) dd[r] = flag[r] == RF_ONE ? 1.0 : 0.0;
}

template <typename T>
__global__ void k_dd_soc(const SocBlock* blk, int64_t nb, const double* zy, double* dd) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const SocBlock B = blk[b];
    if (B.kase == kBlockPsd || B.kase == kBlockDense) return;
    for (int k = lane; k < B.dim; k += 32) {
        double v;
        if (B.kase == 0) v = 0.0;
        else if (B.kase == 1) v = 1.0;
        else if (k == 0) v = 0.5;
        else {
            const double u = (double)zy[B.start + k];
            v = ((B.t + B.r) - (B.t / (B.r * B.r)) * u * u) / (2.0 * B.r);
        }
        dd[B.start + k] = v;
    }
}

// Diagonal of D Pi_psd per entry i of a PSD block: with E the symmetric
// matrix of unit entry i and T = V^T E V, D_ii = sum_pq B_pq T_pq^2.  One
// warp per block.
__global__ void k_dd_psd(const SocBlock* blk, int64_t nb, const double* psd, double* dd) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const SocBlock B = blk[b];
    if (B.kase == kBlockDense) {  // the stored matrix's diagonal
        for (int i = lane; i < B.dim; i += 32) dd[B.start + i] = psd[B.psd + i * B.dim + i];
        return;
    }
    if (B.kase != kBlockPsd) return;
    const int k = B.order;
    const double* V = psd + B.psd;
    const double* W = V + k * k;
    for (int i = lane; i < B.dim; i += 32) {
        int a, j;
        psd_pos(i, a, j);
        const double sc = a == j ? 1.0 : 0.7071067811865476;
        double acc = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = 0; q < k; ++q) {
                const double t = a == j ? V[a * k + p] * V[a * k + q]
                                        : sc * (V[a * k + p] * V[j * k + q] + V[j * k + p] * V[a * k + q]);
                acc += W[p * k + q] * t * t;
            }
        dd[B.start + i] = acc;
    }
}

// Row norms of F with D replaced by its diagonal:
//   x-row i: ||P_i||^2 + sum_j A_ji^2 D_jj^2 + q_i^2
//   y-row j: ||A_j||^2 + (1 - D_jj)^2 + b_j^2
//   tau row: ||g||^2 + sum_j (D_jj b_j)^2 + kappa^2
// w = 1 / norm.  One warp per row; tau through the tile reduction.
// With CW, the norms are those of F C: every entry in column j is weighted
// by cw_j (the current column scaling), for the repeated sweeps of the
// equilibration; without CW the arithmetic is that of the plain row norms.
template <typename T, bool CW>
__global__ void __launch_bounds__(kThreads) k_prec_rows(const Tile* tiles, const Prob* probs, const Sys* psys,
                                                        Reduce R, const int64_t* mrowptr, const int32_t* mcol,
                                                        const T* mval, const double* coefA, const double* coefB,
                                                        const double* dd, const double* cw, double* rw) {
    __shared__ Scratch scratch;
    const int ti = blockIdx.x;
    const Tile tl = tiles[ti];
    const Sys sy = psys[tl.sys];
    const Prob pr = probs[sy.prob];
    const int n = pr.n, N = pr.n + pr.m + 1;
    const int64_t* rp = mrowptr + pr.mrow;
    const double* d = dd + pr.doff;
    const double* cwp = CW ? cw + pr.doff : nullptr;
    const double cN2 = CW ? cwp[N - 1] * cwp[N - 1] : 1.0;  // the tau column's weight
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rend = (tl.kind == TILE_LONG && tl.cb0 != 0) ? tl.r0 : tl.r1;
    double ga = 0.0, gb = 0.0;
    for (int r = tl.r0 + warp; r < rend; r += kWarps) {
        double acc = 0.0;
        for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) {
            const int32_t c = mcol[k];
            const double v = (double)mval[k];
            const double f = c < n ? 1.0 : d[c];
            if (CW) {
                const double vc = v * f * cwp[c];
                acc += vc * vc;
            } else {
                acc += v * v * f * f;
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const double ca = (double)coefA[pr.doff + r];
            if (CW) {
                const double cr2 = cwp[r] * cwp[r];  // weight of the row's own column (diagonal and tau row)
                acc += ca * ca * cN2;
                if (r >= n) {
                    acc += (1.0 - d[r]) * (1.0 - d[r]) * cr2;
                    gb += (d[r] * ca) * (d[r] * ca) * cr2;
                } else {
                    const double g = (double)coefB[pr.doff + r];
                    ga += g * g * cr2;
                }
            } else {
                acc += ca * ca;
                if (r >= n) {
                    acc += (1.0 - d[r]) * (1.0 - d[r]);
                    gb += (d[r] * ca) * (d[r] * ca);
                } else {
                    const double g = (double)coefB[pr.doff + r];
                    ga += g * g;
                }
            }
            rw[pr.doff + r] = acc > 0.0 ? 1.0 / sqrt(acc) : 1.0;
        }
    }
    const Part part = block_sum_part(Part{ga, gb, 0.0, 0.0}, &scratch);
    Part tot;
    if (!finish_tile(R, tl, sy.g0, sy.g1, ti, part, &tot, &scratch)) return;
    if (threadIdx.x == 0) {
        const double t = CW ? tot.a + tot.b + pr.kappa * pr.kappa * cN2 : tot.a + tot.b + pr.kappa * pr.kappa;
        rw[pr.doff + N - 1] = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
    }
}

// Column norms^2 of W F (D by its diagonal), written to csq:
//   x-column j: sum_i w_i^2 P_ij^2 + sum_i w_{n+i}^2 A_ij^2 + w_N^2 g_j^2
//   y-column j: D_jj^2 sum_i w_i^2 A_ji^2 + w_{n+j}^2 (1 - D_jj)^2 + w_N^2 (D_jj b_j)^2
//   tau column: sum w_i^2 q_i^2 + sum w_{n+j}^2 b_j^2 + w_N^2 kappa^2
// (P is symmetric, so column j's P part is row j of M.)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_prec_cols(const Tile* tiles, const Prob* probs, const Sys* psys,
                                                        Reduce R, const int64_t* mrowptr, const int32_t* mcol,
                                                        const T* mval, const double* coefA, const double* coefB,
                                                        const double* dd, const double* rw, double* csq) {
    __shared__ Scratch scratch;
    const int ti = blockIdx.x;
    const Tile tl = tiles[ti];
    const Sys sy = psys[tl.sys];
    const Prob pr = probs[sy.prob];
    const int n = pr.n, N = pr.n + pr.m + 1;
    const int64_t* rp = mrowptr + pr.mrow;
    const double* d = dd + pr.doff;
    const double* w = rw + pr.doff;
    const double wN = w[N - 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rend = (tl.kind == TILE_LONG && tl.cb0 != 0) ? tl.r0 : tl.r1;
    double qa = 0.0, qb = 0.0;
    for (int r = tl.r0 + warp; r < rend; r += kWarps) {
        double acc = 0.0;
        for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) {
            const double v = (double)mval[k] * w[mcol[k]];
            acc += v * v;
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const double ca = (double)coefA[pr.doff + r];
            if (r < n) {
                const double g = (double)coefB[pr.doff + r];
                acc += wN * wN * g * g;
                qa += w[r] * w[r] * ca * ca;
            } else {
                acc = d[r] * d[r] * acc + w[r] * w[r] * (1.0 - d[r]) * (1.0 - d[r]) +
                      wN * wN * (d[r] * ca) * (d[r] * ca);
                qb += w[r] * w[r] * ca * ca;
            }
            csq[pr.doff + r] = acc;
        }
    }
    const Part part = block_sum_part(Part{qa, qb, 0.0, 0.0}, &scratch);
    Part tot;
    if (!finish_tile(R, tl, sy.g0, sy.g1, ti, part, &tot, &scratch)) return;
    if (threadIdx.x == 0) csq[pr.doff + N - 1] = tot.a + tot.b + wN * wN * pr.kappa * pr.kappa;
}

// c = 1 / column norm; on an SOC block one value, from the block's mean
// squared column norm, so that C commutes with D Pi.
__global__ void k_cd_rows(const double* csq, const int8_t* flag, int32_t n, int32_t m, double* cd) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r > (int64_t)n + m) return;
    if (r >= n && r < (int64_t)n + m && flag[r] == RF_SOC) return;
    cd[r] = csq[r] > 0.0 ? 1.0 / sqrt(csq[r]) : 1.0;
}

__global__ void k_cd_soc(const SocBlock* blk, int64_t nb, const double* csq, double* cd) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const SocBlock B = blk[b];
    double s = 0.0;
    for (int k = lane; k < B.dim; k += 32) s += csq[B.start + k];
    s = warp_sum(s) / B.dim;
    const double c = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    for (int k = lane; k < B.dim; k += 32) cd[B.start + k] = c;
}

// MG = M diag(c), MT = M diag(w) for one problem's nonzeros [k0, k1).
template <typename T>
__global__ void k_scale_vals(const T* mval, const int32_t* mcol, int64_t k0, int64_t k1, const double* cd,
                             const double* rw, T* mg, T* mt) {
    const int64_t k = k0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= k1) return;
    const int32_t c = mcol[k];
    const double v = (double)mval[k];
    mg[k] = (T)(v * cd[c]);
    mt[k] = (T)(v * rw[c]);
}

// ---------------------------------------------------------------- schedule
static void cut_tiles(const qcp_plan* p, int pi, std::vector<Tile>& out, int& rmax) {
    const Prob& pr = p->hprob[pi];
    const int n = pr.n, m = pr.m;
    const int64_t* rp = p->h_mrowptr.data() + pr.mrow;
    const int tile_nnz = p->tile_nnz, long_row = p->long_row;
    const int row_cap = 512;
    std::vector<std::vector<Tile>> longs;
    std::vector<Tile> streams;
    Tile cur{};
    bool open = false;
    int64_t cur_nnz = 0;
    auto flush = [&]() {
        if (open) streams.push_back(cur);
        open = false;
        cur_nnz = 0;
    };
    auto start = [&](int r) {
        cur = Tile{pi, TILE_STREAM, r, r, 0, 0, 0, 0};
        open = true;
        cur_nnz = 0;
    };
    auto add_rows = [&](int r0, int r1, int64_t nz) {
        if (!open) start(r0);
        cur.r1 = r1;
        cur_nnz += nz;
    };
    auto single_row = [&](int r) {
        const int64_t len = rp[r + 1] - rp[r];
        if (len > long_row) {
            flush();
            const int nc = (int)((len + p->long_chunk - 1) / p->long_chunk);
            std::vector<Tile> grp;
            for (int c = 0; c < nc; ++c) grp.push_back(Tile{pi, TILE_LONG, r, r + 1, c, nc, 0, 0});
            longs.push_back(grp);
            return;
        }
        if (open && (cur_nnz + len > tile_nnz || (cur.r1 - cur.r0) + 1 > row_cap)) flush();
        add_rows(r, r + 1, len);
    };
    for (int r = 0; r < n; ++r) single_row(r);
    int row = n;
    int sb = 0;
    for (size_t b = 0; b < p->cone_type[pi].size(); ++b) {
        const int t = p->cone_type[pi][b], d = p->cone_dim[pi][b];
        if (t != QCP_CONE_SOC && t != QCP_CONE_PSD && t != QCP_CONE_EXP && t != QCP_CONE_POW) {  // coupled blocks: one tile
            for (int r = row; r < row + d; ++r) single_row(r);
        } else {
            const int64_t nz = rp[row + d] - rp[row];
            if (open && (cur_nnz + nz > tile_nnz || (cur.r1 - cur.r0) + d > std::max(row_cap, d))) flush();
            if (!open) start(row);
            if (cur.cb1 == cur.cb0) {
                cur.cb0 = sb;
                cur.cb1 = sb;
            }
            cur.cb1 = sb + 1;
            add_rows(row, row + d, nz);
            ++sb;
        }
        row += d;
    }
    flush();
    (void)m;
    // long rows first (their chunks kept together and in order) so the
    // heaviest rows start earliest
    std::stable_sort(longs.begin(), longs.end(), [&](const std::vector<Tile>& a, const std::vector<Tile>& b) {
        return (rp[a[0].r0 + 1] - rp[a[0].r0]) > (rp[b[0].r0 + 1] - rp[b[0].r0]);
    });
    out.clear();
    for (const auto& grp : longs) out.insert(out.end(), grp.begin(), grp.end());
    out.insert(out.end(), streams.begin(), streams.end());
    for (const Tile& t : out) rmax = std::max(rmax, t.r1 - t.r0);
}

template <typename T>
static int run_pre(qcp_plan* p);

void drop_graphs(qcp_plan* p) {
    for (auto& kv : p->graphs) cudaGraphExecDestroy(kv.second);
    p->graphs.clear();
}

// Tiles of every system, reduction groups, and the Krylov workspace.
int build_schedule(qcp_plan* p) {
    drop_graphs(p);
    p->rmax = 1;
    p->ptiles.assign(p->nprob, {});
    for (int i = 0; i < p->nprob; ++i) cut_tiles(p, i, p->ptiles[i], p->rmax);
    if (sizeof(double) * (4 * (size_t)p->rmax + 1) > 200 * 1024) {
        set_error("a tile needs %d rows (a second-order-cone block that large does not fit in shared memory)",
                  p->rmax);
        return QCP_ERR_ARG;
    }

    // problem-level tiles/groups (precompute)
    {
        std::vector<Tile> all;
        std::vector<Group> groups;
        std::vector<Sys> psys(p->nprob);
        for (int i = 0; i < p->nprob; ++i) {
            psys[i] = Sys{};
            psys[i].prob = i;
            psys[i].g0 = (int)groups.size();
            const int t0 = (int)all.size();
            for (Tile t : p->ptiles[i]) {
                t.sys = i;
                all.push_back(t);
            }
            for (int g = t0; g < (int)all.size(); g += kGroup) {
                const int g1 = std::min((int)all.size(), g + kGroup);
                for (int k = g; k < g1; ++k) all[k].group = (int)groups.size();
                groups.push_back(Group{i, g, g1, 0});
            }
            psys[i].g1 = (int)groups.size();
        }
        QCP_TRY(p->d_ptiles.alloc(all.size() * sizeof(Tile)));
        QCP_TRY(p->d_pgroups.alloc(groups.size() * sizeof(Group)));
        QCP_TRY(p->d_psys.alloc(psys.size() * sizeof(Sys)));
        QCP_TRY(p->d_ppart.alloc(all.size() * sizeof(Part)));
        QCP_TRY(p->d_pgpart.alloc(groups.size() * sizeof(Part)));
        QCP_TRY(p->d_pgcnt.alloc(groups.size() * sizeof(int32_t)));
        QCP_TRY(p->d_pscnt.alloc(p->nprob * sizeof(int32_t)));
        QCP_CUDA(cudaMemcpyAsync(p->d_ptiles.p, all.data(), all.size() * sizeof(Tile), cudaMemcpyHostToDevice, p->stream));
        QCP_CUDA(cudaMemcpyAsync(p->d_pgroups.p, groups.data(), groups.size() * sizeof(Group), cudaMemcpyHostToDevice, p->stream));
        QCP_CUDA(cudaMemcpyAsync(p->d_psys.p, psys.data(), psys.size() * sizeof(Sys), cudaMemcpyHostToDevice, p->stream));
        QCP_CUDA(cudaMemsetAsync(p->d_pgcnt.p, 0, groups.size() * sizeof(int32_t), p->stream));
        QCP_CUDA(cudaMemsetAsync(p->d_pscnt.p, 0, p->nprob * sizeof(int32_t), p->stream));
        QCP_CUDA(cudaStreamSynchronize(p->stream));
    }

    // systems: batched plans have one per problem; single-problem plans max_rhs
    std::vector<Tile> all;
    std::vector<Group> groups;
    int nsplit = 0;
    p->hsys.clear();
    int64_t voff = 0;
    const int nsys = p->batched ? p->nprob : p->max_rhs;
    for (int s = 0; s < nsys; ++s) {
        const int pi = p->batched ? s : 0;
        const Prob& pr = p->hprob[pi];
        Sys sy{};
        sy.prob = pi;
        sy.voff = voff;
        voff += (int64_t)pr.n + pr.m + 1;
        if (p->batched) {
            sy.xo = 0;
            for (int k = 0; k < pi; ++k) sy.xo += p->hprob[k].n;
            sy.yo = 0;
            for (int k = 0; k < pi; ++k) sy.yo += p->hprob[k].m;
            sy.po = pr.poff;
            sy.ao = pr.aoff;
        } else {
            sy.xo = (int64_t)s * pr.n;
            sy.yo = (int64_t)s * pr.m;
            sy.po = (int64_t)s * pr.pnz;
            sy.ao = (int64_t)s * pr.anz;
        }
        sy.g0 = (int)groups.size();
        const int t0 = (int)all.size();
        for (Tile t : p->ptiles[pi]) {
            t.sys = s;
            t.split = 0;
            if (t.kind == TILE_LONG && t.cb1 > 1) {
                if (t.cb0 == 0) ++nsplit;
                t.split = nsplit - 1;
            }
            all.push_back(t);
        }
        for (int g = t0; g < (int)all.size(); g += kGroup) {
            const int g1 = std::min((int)all.size(), g + kGroup);
            for (int k = g; k < g1; ++k) all[k].group = (int)groups.size();
            groups.push_back(Group{s, g, g1, 0});
        }
        sy.g1 = (int)groups.size();
        p->hsys.push_back(sy);
    }
    p->nsys_cap = nsys;
    p->nsplit = nsplit;
    QCP_TRY(p->d_split_cnt.alloc(std::max(1, nsplit) * sizeof(int32_t)));
    QCP_TRY(p->d_pctl.alloc(4 * sizeof(int32_t)));
    QCP_TRY(p->d_row_part.alloc(std::max<size_t>(1, all.size()) * sizeof(double)));
    QCP_CUDA(cudaMemsetAsync(p->d_split_cnt.p, 0, std::max(1, nsplit) * sizeof(int32_t), p->stream));
    p->ntiles = (int)all.size();
    p->ngroups = (int)groups.size();
    p->tiles_per_sys = p->batched ? 0 : (int)p->ptiles[0].size();
    p->groups_per_sys = p->batched ? 0 : (p->tiles_per_sys + kGroup - 1) / kGroup;
    QCP_TRY(p->d_tiles.alloc(all.size() * sizeof(Tile)));
    QCP_TRY(p->d_groups.alloc(groups.size() * sizeof(Group)));
    QCP_TRY(p->d_sys.alloc(p->hsys.size() * sizeof(Sys)));
    QCP_TRY(p->d_tpart.alloc(all.size() * sizeof(Part)));
    QCP_TRY(p->d_gpart.alloc(groups.size() * sizeof(Part)));
    QCP_TRY(p->d_gcnt.alloc(groups.size() * sizeof(int32_t)));
    QCP_TRY(p->d_scnt.alloc(nsys * sizeof(int32_t)));
    QCP_TRY(p->d_state.alloc(nsys * sizeof(LsqrState)));
    QCP_TRY(p->d_active.alloc(kMaxSegments * sizeof(int)));  // one counter per system range of a call
    const size_t vb = (size_t)voff * sizeof(double);  // Krylov vectors are float64
    QCP_TRY(p->d_U.alloc(vb));
    QCP_TRY(p->d_V.alloc(vb));
    QCP_TRY(p->d_W.alloc(vb));
    QCP_TRY(p->d_X.alloc(vb));
    QCP_TRY(p->d_XI.alloc(vb));
    QCP_TRY(p->d_RHS.alloc(vb));
    QCP_TRY(p->d_HB.alloc(vb));
    QCP_CUDA(cudaMemcpyAsync(p->d_tiles.p, all.data(), all.size() * sizeof(Tile), cudaMemcpyHostToDevice, p->stream));
    QCP_CUDA(cudaMemcpyAsync(p->d_groups.p, groups.data(), groups.size() * sizeof(Group), cudaMemcpyHostToDevice, p->stream));
    QCP_CUDA(cudaMemcpyAsync(p->d_sys.p, p->hsys.data(), p->hsys.size() * sizeof(Sys), cudaMemcpyHostToDevice, p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_gcnt.p, 0, groups.size() * sizeof(int32_t), p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_scnt.p, 0, nsys * sizeof(int32_t), p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_state.p, 0, nsys * sizeof(LsqrState), p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_U.p, 0, vb, p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_V.p, 0, vb, p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_W.p, 0, vb, p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_X.p, 0, vb, p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_XI.p, 0, vb, p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_RHS.p, 0, vb, p->stream));
    QCP_CUDA(cudaMemsetAsync(p->d_HB.p, 0, vb, p->stream));
    QCP_CUDA(cudaStreamSynchronize(p->stream));
    return QCP_OK;
}

template <typename T>
static int run_pre(qcp_plan* p) {
    Reduce R{p->d_ppart.as<Part>(), p->d_pgpart.as<Part>(), p->d_pgcnt.as<int32_t>(), p->d_pscnt.as<int32_t>(),
             p->d_pgroups.as<Group>()};
    int nt = 0;
    for (auto& v : p->ptiles) nt += (int)v.size();
    if (nt == 0) return QCP_OK;
    k_pre<T><<<nt, kThreads, 0, p->stream>>>(p->d_ptiles.as<Tile>(), p->d_prob.as<Prob>(), p->d_prob.as<Prob>(),
                                             p->d_psys.as<Sys>(), R, p->d_mrowptr.as<int64_t>(),
                                             p->d_mcol.as<int32_t>(), p->d_mval.as<T>(), p->d_coefA.as<double>(),
                                             p->d_coefB.as<double>(), p->d_pz.as<double>());
    QCP_CUDA(cudaGetLastError());
    return QCP_OK;
}

// Row and column scalings of F (qcp_precond QCP_PRECOND_EQUILIBRATE) and the
// scaled copies of M's values.  Runs after k_pre (needs g and kappa).
// One sweep: w = 1 / row norms of F, then c = 1 / column norms of W F (D by
// its diagonal; c from the mean square over each coupled block).  Each
// further sweep recomputes w from the row norms of F C with the current c,
// then c from the new W F; the plan keeps the last w and c.  Everything is
// built in buffers of its own and swapped into the plan only once every
// kernel has run, so a failure (allocation or CUDA) leaves the plan's
// previous scaling in place.
template <typename T>
static int run_equilibrate(qcp_plan* p, int sweeps) {
    Reduce R{p->d_ppart.as<Part>(), p->d_pgpart.as<Part>(), p->d_pgcnt.as<int32_t>(), p->d_pscnt.as<int32_t>(),
             p->d_pgroups.as<Group>()};
    int nt = 0;
    for (auto& v : p->ptiles) nt += (int)v.size();
    cudaStream_t st = p->stream;
    DevBuf dd, csq, rwb, cdb, mvalG, mvalT;
    QCP_TRY(dd.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(csq.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(rwb.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(cdb.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(mvalG.alloc((p->mnnz + 16) * sizeof(T)));
    QCP_TRY(mvalT.alloc((p->mnnz + 16) * sizeof(T)));
    QCP_CUDA(cudaMemsetAsync(mvalG.p, 0, (p->mnnz + 16) * sizeof(T), st));
    QCP_CUDA(cudaMemsetAsync(mvalT.p, 0, (p->mnnz + 16) * sizeof(T), st));
    for (int i = 0; i < p->nprob; ++i) {
        const Prob& pr = p->hprob[i];
        k_dd_rows<T><<<grid_for((int64_t)pr.n + pr.m + 1, 256), 256, 0, st>>>(p->d_flag.as<int8_t>() + pr.doff, pr.n,
                                                                             pr.m, dd.as<double>() + pr.doff);
        if (pr.nsoc)
            k_dd_soc<T><<<grid_for((int64_t)pr.nsoc * 32, 256), 256, 0, st>>>(
                p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc, p->d_zy.as<double>() + pr.doff, dd.as<double>() + pr.doff);
        if (pr.nsoc && (p->kpsd || p->ndense))
            k_dd_psd<<<grid_for((int64_t)pr.nsoc * 32, 256), 256, 0, st>>>(
                p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc, p->d_psd.as<double>(), dd.as<double>() + pr.doff);
    }
    QCP_CUDA(cudaGetLastError());
    // c from the column norms in csq (one value per coupled block)
    auto columns_to_c = [&]() {
        for (int i = 0; i < p->nprob; ++i) {
            const Prob& pr = p->hprob[i];
            k_cd_rows<<<grid_for((int64_t)pr.n + pr.m + 1, 256), 256, 0, st>>>(
                csq.as<double>() + pr.doff, p->d_flag.as<int8_t>() + pr.doff, pr.n, pr.m,
                cdb.as<double>() + pr.doff);
            if (pr.nsoc)
                k_cd_soc<<<grid_for((int64_t)pr.nsoc * 32, 256), 256, 0, st>>>(
                    p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc, csq.as<double>() + pr.doff,
                    cdb.as<double>() + pr.doff);
        }
    };
    for (int sweep = 0; sweep < sweeps; ++sweep) {
        if (nt) {
            if (sweep == 0)
                k_prec_rows<T, false><<<nt, kThreads, 0, st>>>(
                    p->d_ptiles.as<Tile>(), p->d_prob.as<Prob>(), p->d_psys.as<Sys>(), R, p->d_mrowptr.as<int64_t>(),
                    p->d_mcol.as<int32_t>(), p->d_mval.as<T>(), p->d_coefA.as<double>(), p->d_coefB.as<double>(),
                    dd.as<double>(), nullptr, rwb.as<double>());
            else
                k_prec_rows<T, true><<<nt, kThreads, 0, st>>>(
                    p->d_ptiles.as<Tile>(), p->d_prob.as<Prob>(), p->d_psys.as<Sys>(), R, p->d_mrowptr.as<int64_t>(),
                    p->d_mcol.as<int32_t>(), p->d_mval.as<T>(), p->d_coefA.as<double>(), p->d_coefB.as<double>(),
                    dd.as<double>(), cdb.as<double>(), rwb.as<double>());
            k_prec_cols<T><<<nt, kThreads, 0, st>>>(p->d_ptiles.as<Tile>(), p->d_prob.as<Prob>(), p->d_psys.as<Sys>(),
                                                    R, p->d_mrowptr.as<int64_t>(), p->d_mcol.as<int32_t>(),
                                                    p->d_mval.as<T>(), p->d_coefA.as<double>(),
                                                    p->d_coefB.as<double>(), dd.as<double>(), rwb.as<double>(),
                                                    csq.as<double>());
            QCP_CUDA(cudaGetLastError());
        }
        columns_to_c();
        QCP_CUDA(cudaGetLastError());
    }
    for (int i = 0; i < p->nprob; ++i) {
        const Prob& pr = p->hprob[i];
        const int64_t k0 = p->h_mrowptr[pr.mrow], k1 = p->h_mrowptr[pr.mrow + pr.n + pr.m + 1];
        if (k1 > k0)
            k_scale_vals<T><<<grid_for(k1 - k0, 256), 256, 0, st>>>(
                p->d_mval.as<T>(), p->d_mcol.as<int32_t>(), k0, k1, cdb.as<double>() + pr.doff,
                rwb.as<double>() + pr.doff, mvalG.as<T>(), mvalT.as<T>());
    }
    QCP_CUDA(cudaGetLastError());
    QCP_CUDA(cudaStreamSynchronize(st));
    p->d_rw.swap(rwb);
    p->d_cd.swap(cdb);
    p->d_mvalG.swap(mvalG);
    p->d_mvalT.swap(mvalT);
    return QCP_OK;
}

int equilibrate_plan(qcp_plan* p, int sweeps) {
    return p->dtype == QCP_F64 ? run_equilibrate<double>(p, sweeps) : run_equilibrate<float>(p, sweeps);
}

// Column scaling of the Jacobi (column-norm) preconditioner: C = 1 / column
// norms of F itself (W = I), D Pi by its diagonal, averaged over each SOC
// block like the equilibration's C.
__global__ void k_fill(double* x, int64_t n, double v) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

template <typename T>
static int jacobi_cols_t(qcp_plan* p, double* out) {
    Reduce R{p->d_ppart.as<Part>(), p->d_pgpart.as<Part>(), p->d_pgcnt.as<int32_t>(), p->d_pscnt.as<int32_t>(),
             p->d_pgroups.as<Group>()};
    int nt = 0;
    for (auto& v : p->ptiles) nt += (int)v.size();
    cudaStream_t st = p->stream;
    DevBuf dd, csq, ones;
    QCP_TRY(dd.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(csq.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(ones.alloc(p->N_tot * sizeof(double)));
    k_fill<<<grid_for(p->N_tot, 256), 256, 0, st>>>(ones.as<double>(), p->N_tot, 1.0);
    for (int i = 0; i < p->nprob; ++i) {
        const Prob& pr = p->hprob[i];
        k_dd_rows<T><<<grid_for((int64_t)pr.n + pr.m + 1, 256), 256, 0, st>>>(p->d_flag.as<int8_t>() + pr.doff, pr.n,
                                                                             pr.m, dd.as<double>() + pr.doff);
        if (pr.nsoc)
            k_dd_soc<T><<<grid_for((int64_t)pr.nsoc * 32, 256), 256, 0, st>>>(
                p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc, p->d_zy.as<double>() + pr.doff, dd.as<double>() + pr.doff);
        if (pr.nsoc && (p->kpsd || p->ndense))
            k_dd_psd<<<grid_for((int64_t)pr.nsoc * 32, 256), 256, 0, st>>>(
                p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc, p->d_psd.as<double>(), dd.as<double>() + pr.doff);
    }
    if (nt)
        k_prec_cols<T><<<nt, kThreads, 0, st>>>(p->d_ptiles.as<Tile>(), p->d_prob.as<Prob>(), p->d_psys.as<Sys>(), R,
                                                p->d_mrowptr.as<int64_t>(), p->d_mcol.as<int32_t>(),
                                                p->d_mval.as<T>(), p->d_coefA.as<double>(), p->d_coefB.as<double>(),
                                                dd.as<double>(), ones.as<double>(), csq.as<double>());
    for (int i = 0; i < p->nprob; ++i) {
        const Prob& pr = p->hprob[i];
        k_cd_rows<<<grid_for((int64_t)pr.n + pr.m + 1, 256), 256, 0, st>>>(
            csq.as<double>() + pr.doff, p->d_flag.as<int8_t>() + pr.doff, pr.n, pr.m, out + pr.doff);
        if (pr.nsoc)
            k_cd_soc<<<grid_for((int64_t)pr.nsoc * 32, 256), 256, 0, st>>>(p->d_blocks.as<SocBlock>() + pr.soff,
                                                                          pr.nsoc, csq.as<double>() + pr.doff,
                                                                          out + pr.doff);
    }
    QCP_CUDA(cudaGetLastError());
    QCP_CUDA(cudaStreamSynchronize(st));
    return QCP_OK;
}

int jacobi_cols(qcp_plan* p, double* out) {
    return p->dtype == QCP_F64 ? jacobi_cols_t<double>(p, out) : jacobi_cols_t<float>(p, out);
}

// ---------------------------------------------------------------- plan build

template <typename T>
static int create_impl(qcp_plan* p, const qcp_problem* probs, const qcp_solution* sols) {
    const int np = p->nprob;
    cudaStream_t st = p->stream;
    // ---- host-side checks and layout
    p->hprob.resize(np);
    p->cone_type.resize(np);
    p->cone_dim.resize(np);
    int64_t mrow = 0, soff = 0, prow = 0, arow = 0, poff = 0, aoff = 0;
    int64_t max_pnz = 0, max_anz = 0, max_n = 0, psd_off = 0;
    std::vector<int8_t> hctype;
    std::vector<SocBlock> hblocks;
    for (int i = 0; i < np; ++i) {
        const qcp_problem& q = probs[i];
        const qcp_solution& s = sols[i];
        if (q.n < 1 || q.m < 0 || q.n > (1ll << 30) || q.m > (1ll << 30)) {
            set_error("problem %d: need n >= 1 and m >= 0 (n=%lld m=%lld)", i, (long long)q.n, (long long)q.m);
            return QCP_ERR_ARG;
        }
        if (q.P_upper.nrows != q.n || q.P_upper.ncols != q.n || q.A.nrows != q.m || q.A.ncols != q.n ||
            q.AT.nrows != q.n || q.AT.ncols != q.m || q.AT.nnz != q.A.nnz || q.P_upper.nnz < 0 || q.A.nnz < 0) {
            set_error("problem %d: matrix shapes do not match n=%lld, m=%lld", i, (long long)q.n, (long long)q.m);
            return QCP_ERR_ARG;
        }
        if (q.P_upper.nnz + q.A.nnz >= (1ll << 31)) {
            set_error("problem %d: nnz(P) + nnz(A) must stay below 2^31", i);
            return QCP_ERR_ARG;
        }
        if (!q.P_upper.indptr || (q.P_upper.nnz && (!q.P_upper.indices || !q.P_upper.values)) || !q.q ||
            !s.x || (q.m && (!q.A.indptr || !q.AT.indptr || !q.b || !s.y || !s.s)) ||
            (q.A.nnz && (!q.A.indices || !q.A.values || !q.AT.indices || !q.AT.values))) {
            set_error("problem %d: null pointer argument", i);
            return QCP_ERR_ARG;
        }
        if (q.K.nblocks < 0 || (q.K.nblocks && (!q.K.type || !q.K.dim))) {
            set_error("problem %d: bad cone description", i);
            return QCP_ERR_ARG;
        }
        int64_t msum = 0;
        int nsoc = 0;
        Prob pr{};
        pr.n = (int)q.n;
        pr.m = (int)q.m;
        for (int b = 0; b < q.K.nblocks; ++b) {
            const int t = q.K.type[b], d = q.K.dim[b];
            if ((t != QCP_CONE_ZERO && t != QCP_CONE_NONNEG && t != QCP_CONE_SOC && t != QCP_CONE_PSD &&
                 t != QCP_CONE_EXP && t != QCP_CONE_POW) ||
                d < 1 || ((t == QCP_CONE_EXP || t == QCP_CONE_POW) && d != 3)) {
                set_error("problem %d: cone block %d has type %d dim %d", i, b, t, d);
                return QCP_ERR_ARG;
            }
            if (msum + d > q.m) {  // before any per-row storage grows
                set_error("problem %d: cone dimensions exceed m = %lld at block %d", i, (long long)q.m, b);
                return QCP_ERR_ARG;
            }
            const double alpha = (t == QCP_CONE_POW && q.K.param) ? q.K.param[b] : 0.0;
            if (t == QCP_CONE_POW && !(alpha > 0.0 && alpha < 1.0)) {
                set_error("problem %d: power-cone block %d needs an exponent in (0, 1) in K.param", i, b);
                return QCP_ERR_ARG;
            }
            int order = 0;
            if (t == QCP_CONE_PSD) {
                // 64-bit and capped one past the largest order, so any dim terminates
                while (order <= kPsdMaxOrder && (int64_t)(order + 1) * (order + 2) / 2 <= d) ++order;
                if ((int64_t)order * (order + 1) / 2 != d || order > kPsdMaxOrder) {
                    set_error("problem %d: PSD block %d has %d entries: need k (k + 1) / 2 with k <= %d", i, b, d,
                              kPsdMaxOrder);
                    return QCP_ERR_ARG;
                }
            }
            if (t == QCP_CONE_SOC || t == QCP_CONE_PSD || t == QCP_CONE_EXP || t == QCP_CONE_POW) {
                SocBlock sb{};
                sb.start = (int)(q.n + msum);
                sb.dim = d;
                sb.cone = t;
                if (t == QCP_CONE_EXP || t == QCP_CONE_POW) {
                    sb.kase = kBlockDense;
                    sb.order = 3;
                    sb.t = alpha;
                    sb.psd = psd_off;
                    psd_off += 9;
                    ++p->ndense;
                }
                if (t == QCP_CONE_PSD) {
                    sb.kase = kBlockPsd;
                    sb.order = order;
                    sb.psd = psd_off;
                    psd_off += 2 * (int64_t)order * order;
                    p->kpsd = std::max(p->kpsd, order);
                }
                hblocks.push_back(sb);
                ++nsoc;
            }
            for (int k = 0; k < d; ++k) hctype.push_back((int8_t)t);
            p->cone_type[i].push_back(t);
            p->cone_dim[i].push_back(d);
            msum += d;
        }
        if (msum != q.m) {
            set_error("problem %d: cone dimensions sum to %lld, m = %lld", i, (long long)msum, (long long)q.m);
            return QCP_ERR_ARG;
        }
        pr.mrow = mrow;
        pr.doff = mrow;  // N-indexed data share the embedding row numbering
        pr.soff = soff;
        pr.nsoc = nsoc;
        pr.pnz = q.P_upper.nnz;
        pr.anz = q.A.nnz;
        pr.prow = prow;
        pr.arow = arow;
        pr.poff = poff;
        pr.aoff = aoff;
        p->hprob[i] = pr;
        mrow += q.n + q.m + 1;
        soff += nsoc;
        prow += q.n + 1;
        arow += q.m + 1;
        poff += q.P_upper.nnz;
        aoff += q.A.nnz;
        max_pnz = std::max<int64_t>(max_pnz, q.P_upper.nnz);
        max_anz = std::max<int64_t>(max_anz, q.A.nnz);
        max_n = std::max<int64_t>(max_n, q.n);
        p->n_tot += q.n;
        p->m_tot += q.m;
    }
    p->N_tot = mrow;
    p->pnz_tot = poff;
    p->anz_tot = aoff;
    p->nsoc_tot = soff;

    // ---- device buffers for the problem data
    QCP_TRY(p->d_prob.alloc(np * sizeof(Prob)));
    QCP_TRY(p->d_mrowptr.alloc((p->N_tot + 1) * sizeof(int64_t)));
    QCP_TRY(p->d_coefA.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(p->d_coefB.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(p->d_pz.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(p->d_zy.alloc(p->N_tot * sizeof(double)));
    QCP_TRY(p->d_flag.alloc(p->N_tot));
    QCP_TRY(p->d_blocks.alloc(std::max<int64_t>(1, soff) * sizeof(SocBlock)));
    QCP_TRY(p->d_psd.alloc(std::max<int64_t>(1, psd_off) * sizeof(double)));
    QCP_TRY(p->d_pip.alloc(prow * sizeof(int64_t)));
    QCP_TRY(p->d_pix.alloc(std::max<int64_t>(1, poff) * sizeof(int32_t)));
    QCP_TRY(p->d_aip.alloc(arow * sizeof(int64_t)));
    QCP_TRY(p->d_aix.alloc(std::max<int64_t>(1, aoff) * sizeof(int32_t)));
    DevBuf d_ctype, d_err, d_len, d_prid, d_keys, d_vals, d_skeys, d_svals, d_lowptr, d_perm, d_cub, d_kink, d_atip_zero;
    QCP_TRY(d_ctype.alloc(std::max<size_t>(1, hctype.size())));
    QCP_TRY(d_err.alloc(sizeof(int)));
    QCP_TRY(d_len.alloc((p->N_tot + 1) * sizeof(int64_t)));
    QCP_TRY(d_prid.alloc(std::max<int64_t>(1, max_pnz) * sizeof(int32_t)));
    QCP_TRY(d_keys.alloc(std::max<int64_t>(1, max_pnz) * sizeof(int32_t)));
    QCP_TRY(d_vals.alloc(std::max<int64_t>(1, max_pnz) * sizeof(int32_t)));
    QCP_TRY(d_skeys.alloc(std::max<int64_t>(1, max_pnz) * sizeof(int32_t)));
    QCP_TRY(d_svals.alloc(std::max<int64_t>(1, max_pnz) * sizeof(int32_t)));
    QCP_TRY(d_lowptr.alloc((max_n + 1) * sizeof(int64_t)));
    QCP_TRY(d_perm.alloc(std::max<int64_t>(1, max_anz) * sizeof(int64_t)));
    QCP_TRY(d_kink.alloc(np * sizeof(unsigned long long)));
    QCP_TRY(d_atip_zero.alloc((max_n + 1) * sizeof(int64_t)));
    QCP_CUDA(cudaMemsetAsync(d_atip_zero.p, 0, (max_n + 1) * sizeof(int64_t), st));
    QCP_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int), st));
    QCP_CUDA(cudaMemsetAsync(d_len.p, 0, (p->N_tot + 1) * sizeof(int64_t), st));
    {
        std::vector<unsigned long long> inf(np, 0x7ff0000000000000ull);
        QCP_CUDA(cudaMemcpyAsync(d_kink.p, inf.data(), np * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    }
    if (!hctype.empty())
        QCP_CUDA(cudaMemcpyAsync(d_ctype.p, hctype.data(), hctype.size(), cudaMemcpyHostToDevice, st));
    if (soff)
        QCP_CUDA(cudaMemcpyAsync(p->d_blocks.p, hblocks.data(), soff * sizeof(SocBlock), cudaMemcpyHostToDevice, st));
    int* err = d_err.as<int>();
    size_t cub_bytes = 0;
    {
        size_t b1 = 0, b2 = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, b1, (int32_t*)nullptr, (int32_t*)nullptr, (int32_t*)nullptr,
                                        (int32_t*)nullptr, (int)std::max<int64_t>(1, max_pnz), 0, 32, st);
        cub::DeviceScan::ExclusiveSum(nullptr, b2, (int64_t*)nullptr, (int64_t*)nullptr, (int)(p->N_tot + 1), st);
        cub_bytes = std::max(b1, b2);
        QCP_TRY(d_cub.alloc(cub_bytes));
    }

    // ---- pass 1: validation, structure copies, row data, M row lengths
    int64_t ctoff = 0;
    for (int i = 0; i < np; ++i) {
        const qcp_problem& q = probs[i];
        const qcp_solution& s = sols[i];
        const Prob& pr = p->hprob[i];
        const int n = pr.n, m = pr.m;
        k_check_csr<<<grid_for(n + 1, 256), 256, 0, st>>>(q.P_upper.indptr, q.P_upper.indices, n, n, pr.pnz, 1, err);
        if (m) {
            k_check_csr<<<grid_for(m + 1, 256), 256, 0, st>>>(q.A.indptr, q.A.indices, m, n, pr.anz, 0, err);
            k_check_csr<<<grid_for(n + 1, 256), 256, 0, st>>>(q.AT.indptr, q.AT.indices, n, m, pr.anz, 0, err);
        }
        QCP_CUDA(cudaGetLastError());
        QCP_CUDA(cudaMemcpyAsync(p->d_pip.as<int64_t>() + pr.prow, q.P_upper.indptr, (n + 1) * sizeof(int64_t),
                                 cudaMemcpyDeviceToDevice, st));
        if (pr.pnz)
            QCP_CUDA(cudaMemcpyAsync(p->d_pix.as<int32_t>() + pr.poff, q.P_upper.indices, pr.pnz * sizeof(int32_t),
                                     cudaMemcpyDeviceToDevice, st));
        if (m) {
            QCP_CUDA(cudaMemcpyAsync(p->d_aip.as<int64_t>() + pr.arow, q.A.indptr, (m + 1) * sizeof(int64_t),
                                     cudaMemcpyDeviceToDevice, st));
        } else {
            QCP_CUDA(cudaMemsetAsync(p->d_aip.as<int64_t>() + pr.arow, 0, sizeof(int64_t), st));
        }
        if (pr.anz)
            QCP_CUDA(cudaMemcpyAsync(p->d_aix.as<int32_t>() + pr.aoff, q.A.indices, pr.anz * sizeof(int32_t),
                                     cudaMemcpyDeviceToDevice, st));
        const T* dummy = static_cast<const T*>(q.q);
        k_rowdata<T><<<grid_for(n + m + 1, 256), 256, 0, st>>>(
            static_cast<const T*>(q.q), m ? static_cast<const T*>(q.b) : dummy, static_cast<const T*>(s.x),
            m ? static_cast<const T*>(s.y) : dummy, m ? static_cast<const T*>(s.s) : dummy,
            d_ctype.as<int8_t>() + ctoff, n, m, p->d_coefA.as<double>() + pr.doff, p->d_coefB.as<double>() + pr.doff,
            p->d_pz.as<double>() + pr.doff, p->d_zy.as<double>() + pr.doff, p->d_flag.as<int8_t>() + pr.doff);
        QCP_CUDA(cudaGetLastError());
        ctoff += m;
    }
    QCP_CUDA(cudaStreamSynchronize(st));
    int herr = 0;
    QCP_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        set_error("invalid CSR input (code %d: %s%s%s)", herr, (herr & E_PTR) ? "bad row pointers " : "",
                  (herr & E_COL) ? "columns out of range or not strictly increasing " : "",
                  (herr & E_UPPER) ? "P has entries below the diagonal" : "");
        return QCP_ERR_ARG;
    }
    // A^T consistency and M row lengths
    for (int i = 0; i < np; ++i) {
        const qcp_problem& q = probs[i];
        const Prob& pr = p->hprob[i];
        const int n = pr.n, m = pr.m;
        const int64_t* atip = m ? q.AT.indptr : d_atip_zero.as<int64_t>();
        if (m)
            k_at_perm<T><<<grid_for(pr.anz, 256), 256, 0, st>>>(
                q.AT.indptr, q.AT.indices, static_cast<const T*>(q.AT.values), n, pr.anz, q.A.indptr, q.A.indices,
                static_cast<const T*>(q.A.values), q.AT_perm, d_perm.as<int64_t>(), err);
        if (pr.pnz) {
            k_rowids<<<grid_for(n, 256), 256, 0, st>>>(q.P_upper.indptr, n, d_prid.as<int32_t>());
            k_lower_keys<<<grid_for(pr.pnz, 256), 256, 0, st>>>(d_prid.as<int32_t>(), q.P_upper.indices, pr.pnz, n,
                                                                d_keys.as<int32_t>(), d_vals.as<int32_t>());
            size_t bytes = cub_bytes;
            QCP_CUDA(cub::DeviceRadixSort::SortPairs(d_cub.p, bytes, d_keys.as<int32_t>(), d_skeys.as<int32_t>(),
                                                     d_vals.as<int32_t>(), d_svals.as<int32_t>(), (int)pr.pnz, 0, 32, st));
        }
        k_lowptr<<<grid_for(n + 1, 256), 256, 0, st>>>(d_skeys.as<int32_t>(), pr.pnz, n, d_lowptr.as<int64_t>());
        k_mlen<<<grid_for(n + m + 1, 256), 256, 0, st>>>(d_lowptr.as<int64_t>(), q.P_upper.indptr, atip,
                                                         m ? q.A.indptr : d_atip_zero.as<int64_t>(), n, m,
                                                         d_len.as<int64_t>() + pr.mrow);
        QCP_CUDA(cudaGetLastError());
    }
    QCP_CUDA(cudaStreamSynchronize(st));
    QCP_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        set_error("A^T is not the transpose of A%s (code %d)", (herr & E_PERM) ? " under AT_perm" : "", herr);
        return QCP_ERR_ARG;
    }
    {
        size_t bytes = cub_bytes;
        QCP_CUDA(cub::DeviceScan::ExclusiveSum(d_cub.p, bytes, d_len.as<int64_t>(), p->d_mrowptr.as<int64_t>(),
                                               (int)(p->N_tot + 1), st));
    }
    p->h_mrowptr.resize(p->N_tot + 1);
    QCP_CUDA(cudaMemcpyAsync(p->h_mrowptr.data(), p->d_mrowptr.p, (p->N_tot + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, st));
    QCP_CUDA(cudaStreamSynchronize(st));
    p->mnnz = p->h_mrowptr[p->N_tot];
    // M's arrays are padded by 16 zero entries: the pass kernels read
    // aligned groups of 8 entries that may run past the last one
    const int64_t mpad = p->mnnz + 16;
    QCP_TRY(p->d_mcol.alloc(mpad * sizeof(int32_t)));
    QCP_TRY(p->d_mvmap.alloc(mpad * sizeof(int32_t)));
    QCP_TRY(p->d_mval.alloc(mpad * sizeof(T)));
    QCP_CUDA(cudaMemsetAsync(p->d_mcol.p, 0, mpad * sizeof(int32_t), st));
    QCP_CUDA(cudaMemsetAsync(p->d_mvmap.p, 0, mpad * sizeof(int32_t), st));
    QCP_CUDA(cudaMemsetAsync(p->d_mval.p, 0, mpad * sizeof(T), st));

    // ---- pass 2: fill M and its values
    for (int i = 0; i < np; ++i) {
        const qcp_problem& q = probs[i];
        const Prob& pr = p->hprob[i];
        const int n = pr.n, m = pr.m;
        const int64_t* atip = m ? q.AT.indptr : d_atip_zero.as<int64_t>();
        if (m)
            k_at_perm<T><<<grid_for(pr.anz, 256), 256, 0, st>>>(
                q.AT.indptr, q.AT.indices, static_cast<const T*>(q.AT.values), n, pr.anz, q.A.indptr, q.A.indices,
                static_cast<const T*>(q.A.values), q.AT_perm, d_perm.as<int64_t>(), err);
        if (pr.pnz) {
            k_rowids<<<grid_for(n, 256), 256, 0, st>>>(q.P_upper.indptr, n, d_prid.as<int32_t>());
            k_lower_keys<<<grid_for(pr.pnz, 256), 256, 0, st>>>(d_prid.as<int32_t>(), q.P_upper.indices, pr.pnz, n,
                                                                d_keys.as<int32_t>(), d_vals.as<int32_t>());
            size_t bytes = cub_bytes;
            QCP_CUDA(cub::DeviceRadixSort::SortPairs(d_cub.p, bytes, d_keys.as<int32_t>(), d_skeys.as<int32_t>(),
                                                     d_vals.as<int32_t>(), d_svals.as<int32_t>(), (int)pr.pnz, 0, 32, st));
        }
        k_lowptr<<<grid_for(n + 1, 256), 256, 0, st>>>(d_skeys.as<int32_t>(), pr.pnz, n, d_lowptr.as<int64_t>());
        const int64_t rows = (int64_t)n + m;
        k_mfill<<<grid_for(rows * 32, 256), 256, 0, st>>>(
            p->d_mrowptr.as<int64_t>() + pr.mrow, d_lowptr.as<int64_t>(), d_svals.as<int32_t>(), d_prid.as<int32_t>(),
            q.P_upper.indptr, q.P_upper.indices, atip, m ? q.AT.indices : nullptr, d_perm.as<int64_t>(),
            m ? q.A.indptr : d_atip_zero.as<int64_t>(), m ? q.A.indices : nullptr, n, m, pr.pnz,
            p->d_mcol.as<int32_t>(), p->d_mvmap.as<int32_t>());
        const int64_t k0 = p->h_mrowptr[pr.mrow], k1 = p->h_mrowptr[pr.mrow + n + m + 1];
        if (k1 > k0)
            k_mvals<T><<<grid_for(k1 - k0, 256), 256, 0, st>>>(p->d_mvmap.as<int32_t>(), k0, k1, pr.pnz,
                                                               static_cast<const T*>(q.P_upper.values),
                                                               static_cast<const T*>(q.A.values), p->d_mval.as<T>());
        QCP_CUDA(cudaGetLastError());
        // the sort buffers are reused by the next problem
        QCP_CUDA(cudaStreamSynchronize(st));
    }
    // ---- D Pi state and kink margins
    for (int i = 0; i < np; ++i) {
        const Prob& pr = p->hprob[i];
        if (pr.nsoc)
            k_socprep<T><<<grid_for((int64_t)pr.nsoc * 32, 256), 256, 0, st>>>(
                p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc, p->d_zy.as<double>() + pr.doff);
        if (pr.nsoc && p->kpsd)
            k_psdprep<<<grid_for(pr.nsoc, 64), 64, 0, st>>>(p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc,
                                                           p->d_zy.as<double>() + pr.doff, p->d_psd.as<double>(),
                                                           d_kink.as<unsigned long long>() + i);
        if (pr.nsoc && p->ndense)
            k_expprep<<<grid_for(pr.nsoc, 64), 64, 0, st>>>(p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc,
                                                           p->d_zy.as<double>() + pr.doff, p->d_psd.as<double>());
    }
    QCP_CUDA(cudaGetLastError());
    ctoff = 0;
    for (int i = 0; i < np; ++i) {
        const Prob& pr = p->hprob[i];
        const int64_t cnt = std::max<int64_t>(pr.m, pr.nsoc);
        if (cnt)
            k_kink<T><<<grid_for(cnt, 256), 256, 0, st>>>(p->d_zy.as<double>() + pr.doff, d_ctype.as<int8_t>() + ctoff, pr.n,
                                                          pr.m, p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc,
                                                          d_kink.as<unsigned long long>() + i);
        ctoff += pr.m;
    }
    QCP_CUDA(cudaGetLastError());
    {
        std::vector<unsigned long long> hk(np);
        QCP_CUDA(cudaMemcpyAsync(hk.data(), d_kink.p, np * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        p->kink.resize(np);
        for (int i = 0; i < np; ++i) {
            double v;
            memcpy(&v, &hk[i], sizeof(double));
            p->kink[i] = v;
        }
    }
    QCP_CUDA(cudaMemcpyAsync(p->d_prob.p, p->hprob.data(), np * sizeof(Prob), cudaMemcpyHostToDevice, st));
    // ---- schedule, then g and kappa
    QCP_TRY(build_schedule(p));
    QCP_TRY(run_pre<T>(p));
    QCP_CUDA(cudaStreamSynchronize(st));
    // keep the host copy of kappa in step
    QCP_CUDA(cudaMemcpy(p->hprob.data(), p->d_prob.p, np * sizeof(Prob), cudaMemcpyDeviceToHost));
    QCP_TRY(run_equilibrate<T>(p, p->equil_sweeps));
    return QCP_OK;
}

int create_plan(qcp_plan* p, const qcp_problem* probs, const qcp_solution* sols) {
    if (p->dtype == QCP_F64) return create_impl<double>(p, probs, sols);
    return create_impl<float>(p, probs, sols);
}

}  // namespace qcpd

qcp_plan::~qcp_plan() {
    qcpd::drop_graphs(this);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (aux_stream) cudaStreamDestroy(aux_stream);
    if (h_active) cudaFreeHost(h_active);
}
