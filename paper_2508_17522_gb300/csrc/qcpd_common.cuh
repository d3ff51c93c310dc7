// Internal definitions shared by the translation units of libqcpd.
//
// Notation (arXiv 2508.17522, Sec. 2-3): a problem has n variables and m
// constraint rows; the embedding has N = n + m + 1 coordinates ordered
// (x-part, y-part, tau).  At a constructed root z = (x, y - s, 1) the
// derivative of the normalised residual map is
//     F = D_u Q(Pi z) D Pi(z) - D Pi(z) + I,  D Pi(z) = blkdiag(I_n, D, 1),
// D = D Pi_{K*}(y - s) (Appendix A), D_u Q as printed in Sec. 2.4 with tau = 1.
//
// Every product with F or F^T is evaluated through ONE combined sparse
// matrix M = [[P, A^T], [A, 0]] (P expanded to both triangles) and the sign
// matrix S = diag(I_n, -I_m, 1):  G := S F satisfies
//     G (a, c, t)   = (M_top xi + q t,  M_bot xi - b t - c + D c,
//                      -g^T a - b^T D c + kappa t),          xi = (a, D c)
//     G^T (r1,r2,r3) = (M_top rho - g r3,  D(M_bot rho - b r3 + r2) - r2,
//                      q^T r1 - b^T r2 + kappa r3),          rho = (r1, r2)
// with g = 2 P x + q and kappa = x^T P x.  Because S is orthogonal,
// min ||F dz + dN|| = min ||G dz + S dN|| and F^T r = G^T (S r): the JVP
// runs LSQR on G with right-hand side -S dN, the VJP runs LSQR on G^T with
// right-hand side -g_phi and returns r = S r'.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/qcpd.h"

namespace qcpd {

constexpr int kThreads = 256;   // threads per CTA of every tile kernel
constexpr int kWarps = kThreads / 32;
constexpr int kGroup = 64;      // tiles per first-level reduction group
constexpr int kE = 8;           // consecutive nonzeros each thread multiplies into one FMA chain
constexpr int kChunk = kThreads * kE;  // nonzeros one sweep of a CTA covers

enum TileKind : int32_t { TILE_STREAM = 0, TILE_LONG = 1 };

// Row flags of the y-part: which diagonal entry D has, or "SOC row".
enum RowFlag : int8_t { RF_ZERO = 0, RF_ONE = 1, RF_SOC = 2 };

// Krylov status of one system.
enum SysStatus : int32_t { S_ACTIVE = 0, S_FINAL = 1, S_DONE = 2 };
enum SysOutcome : int32_t { O_RUNNING = 0, O_CONVERGED = 1, O_MAXITER = 2, O_BREAKDOWN = 3 };

// A tile: a contiguous range of local rows of one system's embedding (rows of
// M), never splitting a second-order-cone block.  A row longer than the
// schedule's threshold is cut into chunks of long_chunk nonzeros, one LONG
// tile each (consecutive in the tile list); the last chunk to finish adds
// the chunk sums in order and runs the row's epilogue.
struct Tile {
    int32_t sys;       // system index
    int32_t kind;      // TileKind
    int32_t r0, r1;    // local rows [r0, r1), r1 <= n + m
    int32_t cb0, cb1;  // STREAM: SOC blocks [cb0, cb1) inside the tile; LONG: chunk index, chunk count
    int32_t group;     // first-level reduction group
    int32_t split;     // LONG: index of the split row's counter
};

struct Group {
    int32_t sys, t0, t1, pad;  // tiles [t0, t1)
};

// Per problem (device copy).  Offsets index the plan's concatenated arrays.
struct Prob {
    int64_t mrow;    // global row of local row 0 in M's row pointer array
    int64_t doff;    // offset of the N-indexed per-problem data (coefA, coefB, pz, zy, flags)
    int64_t soff;    // first SOC block
    int64_t pnz;     // nnz of P's upper pattern
    int64_t anz;     // nnz of A
    int64_t prow;    // offset of the problem's rows in the stored P-upper / A structure copies
    int64_t arow;
    int64_t poff;    // offset of the problem's values in concatenated P / A value arrays
    int64_t aoff;
    int32_t n, m, nsoc, pad;
    double kappa;    // x^T P x, filled at plan creation
};

// Per system: a (problem, direction) pair with its own Krylov vectors.
struct Sys {
    int32_t prob;
    int32_t g0, g1;  // reduction groups [g0, g1)
    int32_t pad;
    int64_t voff;    // offset of the system's N-vectors
    int64_t xo, yo;  // offsets into n-indexed / m-indexed user arrays
    int64_t po, ao;  // offsets into P-value / A-value user arrays
};

// A block of rows that D Pi couples: a second-order cone (kase 0..2) or a
// positive semidefinite cone (kase 3).
struct SocBlock {
    int32_t start;   // local embedding row of the block's first entry (n + first y row)
    int32_t dim;
    int32_t kase;    // SOC: 0 ||u|| <= -t (D = 0), 1 ||u|| <= t (D = I), 2 formula; 3: PSD; 4: dense D
    int32_t order;   // PSD: the matrix order k (dim = k (k + 1) / 2); SOC: 0
    double t, r;     // SOC: t and ||u|| of z_y on the block
    double h, tq;    // SOC: 1 / (2 r) and t / r^2 (kase 2), so no kernel divides
    int64_t psd;     // PSD: offset of its k x k eigenvectors V and weights B in the plan's block array;
                     // dense: offset of its dim x dim D Pi (row-major)
    int32_t cone;    // qcp_cone_type of the block (dense blocks: QCP_CONE_EXP or QCP_CONE_POW; t holds a pow's a)
    int32_t pad;
};

constexpr int kPsdMaxOrder = 64;  // largest PSD block order (its scratch is 2 k^2 doubles of shared memory)
constexpr int kBlockPsd = 3;      // SocBlock::kase of a PSD block
constexpr int kBlockDense = 4;    // SocBlock::kase of a block whose D Pi is a stored dense matrix (exp and power cones)

// LSQR scalars of one system (Paige & Saunders' recurrences).
struct LsqrState {
    double alpha, beta;     // current normalisers of v and u
    double rhobar, phibar;
    double inv_rho;         // 1 / rho of the last rotation
    double uc1, uc2;        // next u-update: 1/alpha, alpha/beta
    double vc1, vc2;        // next v-update: 1/beta, beta/alpha (0 at the first one)
    double wcoef;           // theta_{k+1} / rho_k  (w <- v - wcoef w)
    double xcoef;           // phi_k / rho_k        (x <- x + xcoef w)
    double c, s;
    double bnorm;           // ||b|| of the (scaled) least-squares problem
    double bnorm_true;      // ||b|| without the diagonal scaling (||dN|| or ||g||)
    double resid_true;      // unscaled ||F dz + dN|| / ||dN|| (or the adjoint's) when computed
    double rtol;
    int64_t iters, maxiter;
    int32_t status, outcome, first, upd;  // upd (LSMR): the next u-pass applies the deferred updates
    // LSMR (Fong & Saunders 2011) with damping 0: the two rotations' state
    // (alphabar_k, zetabar_k, rho_{k-1}, rhobar_{k-1}, cbar_{k-1},
    // sbar_{k-1}), the residual-norm estimate's state (betadd_k, betad_{k-1},
    // rhod_{k-1}, tautilde_{k-2}, thetatilde_{k-1}, zeta_{k-1}) and the
    // coefficient of hbar_k <- h_k - hcoef hbar_{k-1} (xcoef and wcoef are
    // then zeta_k / (rho_k rhobar_k) and theta_{k+1} / rho_k)
    double alphabar, zetabar, rho_old, rhobar_old, cbar, sbar;
    double betadd, betad, rhod_old, tautilde_old, thetatilde, zeta_old;
    double hcoef;
};

// Thread-block-cluster layout of one problem: CTA r of a system's cluster
// owns the local rows [split[r], split[r+1]) (never cutting a second-order-
// cone block) and keeps its slice of the gathered vector at poff[r] of the
// gather buffer (poff even, so every slice starts on a 16-byte boundary).
constexpr int kMaxCluster = 16;
struct ClusterProb {
    int32_t C;                        // CTAs per system
    int32_t FN;                       // gather-buffer length (poff[C])
    int32_t L;                        // most rows of one CTA
    int32_t nb;                       // most SOC blocks of one CTA
    int32_t split[kMaxCluster + 1];
    int32_t poff[kMaxCluster + 1];
    int32_t cb[kMaxCluster + 1];      // CTA r's SOC blocks [cb[r], cb[r+1]) (problem-relative)
    int32_t sl[kMaxCluster + 1];      // CTA r's row-sum slices [sl[r], sl[r+1]) (global indices)
    int32_t nlarge[kMaxCluster];      // CTA r's SOC blocks with more than kSocThread entries
};

// Four partial sums carried through the reductions.
struct __align__(16) Part {
    double a, b, c, d;
};

struct Reduce {
    Part* tile_part;
    Part* group_part;
    int32_t* group_cnt;
    int32_t* sys_cnt;
    const Group* groups;
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double ld(const T* p) { return static_cast<double>(*p); }

__device__ __forceinline__ Part pzero() { return Part{0.0, 0.0, 0.0, 0.0}; }

__device__ __forceinline__ Part padd(Part x, Part y) {
    return Part{x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d};
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ Part warp_sum_part(Part v) {
    return Part{warp_sum(v.a), warp_sum(v.b), warp_sum(v.c), warp_sum(v.d)};
}

// x is neither infinite nor NaN (integer test on the exponent field).
__device__ __forceinline__ bool finite64(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// 1 / sqrt(s).  A warp-wide FP64 instruction costs 1/64 of the FP32 rate on
// this GPU and the library's sqrt and division each take many, so for a
// positive normal s this scales s by an even power of two into [1, 4)
// (keeping it inside FP32's range), takes the FP32 estimate of 1/sqrt and
// refines it with two steps of Newton's iteration for 1/sqrt,
// y <- y + (y/2)(1 - m y^2), each of which squares the relative error
// (about 2^-22 -> 2^-43 -> FP64 rounding); the power of two goes back in
// through the exponent field.  Zero, subnormal, infinite and NaN inputs take
// the library's route.
__device__ __forceinline__ double rsqrt_fast(double s) {
    const long long b = __double_as_longlong(s);
    const int ef = (int)((b >> 52) & 0x7ff);
    if (b <= 0 || ef == 0 || ef == 0x7ff) return 1.0 / sqrt(s);
    const int k = (ef - 1023) >> 1;  // s = m 2^(2k), m in [1, 4)
    const double m = __longlong_as_double(b - ((long long)(2 * k) << 52));
    double y = (double)rsqrtf((float)m);
    y = fma(0.5 * y, fma(-(m * y), y, 1.0), y);
    y = fma(0.5 * y, fma(-(m * y), y, 1.0), y);
    return __longlong_as_double(__double_as_longlong(y) - ((long long)k << 52));
}

// sqrt(ss) and 1 / sqrt(ss) (0 for ss = 0; a non-finite norm for a
// non-finite ss) for a sum of squares ss.
__device__ __forceinline__ void norm_and_inverse(double ss, double& nrm, double& inv) {
    if (ss > 0.0) {
        const double y = rsqrt_fast(ss);
        nrm = ss * y;  // NaN for ss = inf (y = 0)
        inv = y;
    } else {
        nrm = ss;  // 0, or NaN
        inv = 0.0;
    }
}

// Block-wide sums of NV values per thread, in a fixed order (deterministic
// for a fixed block size); the sums are returned in every thread.  A
// warp-wide FP64 instruction costs the same on this GPU (1/64 of the FP32
// rate) however many lanes it has, so the sum is a halving tree in shared
// memory (NT/64 + NT/128 + ... + 1 warp-wide adds per value, spread over the
// warps) ending in one warp per value for the last 32 partial sums.
template <int NV, int NT = kThreads>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* red) {
    static_assert(NV <= NT / 32, "one warp per value in the last stage");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) red[j * NT + tid] = v[j];
    __syncthreads();
#pragma unroll
    for (int w = NT / 2; w >= 32; w >>= 1) {
        if (tid < w) {
#pragma unroll
            for (int j = 0; j < NV; ++j) red[j * NT + tid] += red[j * NT + tid + w];
        }
        __syncthreads();
    }
    if (warp < NV) {
        const double s = warp_sum(red[warp * NT + lane]);
        __syncwarp();
        if (lane == 0) red[warp * NT] = s;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = red[j * NT];
    __syncthreads();
}

// Shared scratch of the block reductions: up to 4 values per thread.
struct Scratch {
    double red[4 * kThreads];
};

// Block sums; valid in every thread.
__device__ __forceinline__ Part block_sum_part(Part p, Scratch* sc) {
    double v[4] = {p.a, p.b, p.c, p.d};
    block_reduce<4>(v, sc->red);
    return Part{v[0], v[1], v[2], v[3]};
}

__device__ __forceinline__ Part block_sum3(double a, double b, double c, Scratch* sc) {
    double v[3] = {a, b, c};
    block_reduce<3>(v, sc->red);
    return Part{v[0], v[1], v[2], 0.0};
}

__device__ __forceinline__ double block_sum(double a, Scratch* sc) {
    double v[1] = {a};
    block_reduce<1>(v, sc->red);
    return v[0];
}

// Load a Part written by another CTA in this launch (bypass L1).
__device__ __forceinline__ Part ld_part(const Part* p) {
    const double2 lo = __ldcg(reinterpret_cast<const double2*>(p));
    const double2 hi = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    return Part{lo.x, lo.y, hi.x, hi.y};
}

// Two-level last-CTA-done reduction of one Part per tile into one per
// system.  Called by every thread of the CTA with the tile's partial (valid
// in thread 0).  Returns true in warp 0 of the single CTA that completes the
// system, with the system total in *total; every other warp and CTA gets
// false.  After the arrival barrier only warp 0 works (shuffles, no block
// barriers): FP64 adds are scarce and every barrier and dependent add sits on
// the pass's critical path.  Sums run in a fixed order, so results do not
// depend on CTA scheduling (except for a row cut into several LONG tiles,
// whose terms arrive with whichever of its tiles finishes last).  No CTA ever waits on another: the last one to
// arrive does the work.
__device__ __forceinline__ bool finish_tile(const Reduce& R, const Tile& tl, int32_t g0, int32_t g1,
                                            int tile, Part part, Part* total, Scratch* scratch) {
    (void)scratch;
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        R.tile_part[tile] = part;
        __threadfence();
        const Group g = R.groups[tl.group];
        const int prev = atomicAdd(&R.group_cnt[tl.group], 1);
        s_last = (prev == g.t1 - g.t0 - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x >= 32) return false;
    const int lane = threadIdx.x;
    __threadfence();
    const Group g = R.groups[tl.group];
    Part acc = pzero();
    for (int i = g.t0 + lane; i < g.t1; i += 32) acc = padd(acc, ld_part(R.tile_part + i));
    acc = warp_sum_part(acc);
    if (g1 - g0 == 1) {  // the group is the whole system
        if (lane == 0) R.group_cnt[tl.group] = 0;
        *total = acc;
        return true;
    }
    int last = 0;
    if (lane == 0) {
        R.group_cnt[tl.group] = 0;
        R.group_part[tl.group] = acc;
        __threadfence();
        const int prev = atomicAdd(&R.sys_cnt[tl.sys], 1);
        last = (prev == g1 - g0 - 1);
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return false;
    __threadfence();
    acc = pzero();
    for (int i = g0 + lane; i < g1; i += 32) acc = padd(acc, ld_part(R.group_part + i));
    acc = warp_sum_part(acc);
    if (lane == 0) R.sys_cnt[tl.sys] = 0;
    *total = acc;
    return true;
}

// D Pi_{K*} applied to the tile's rows (Appendix A).  src/dst are shared
// arrays indexed by (row - r0); x-rows (row < n) pass through (D Pi = I on
// R^n).  y-rows: R+ rows use their 0/1 flag, zero-cone rows 1 (the dual of
// {0} is R), and a second-order-cone block (whole inside the range) with
// z_y = (t, u), r = ||u|| in the formula case maps (ct, cu) to
//   (1/(2r)) (r ct + u^T cu,  (ct - (t/r^2) u^T cu) u + (t + r) cu).
// Every warp-wide FP64 instruction costs the same on this GPU however many
// lanes it has, so blocks of up to kSocThread entries take one thread each
// (all lanes busy, two FP64 operations per entry) and only larger blocks
// take a warp.  zy[row - zoff] holds the block's z_y.  Caller synchronises
// before and after.
constexpr int kSocThread = 32;

// Row a <= column j of a PSD block's entry i (the upper triangle column by
// column: i = j (j + 1) / 2 + a).
__device__ __forceinline__ void psd_pos(int i, int& a, int& j) {
    j = (int)((sqrt(8.0 * i + 1.0) - 1.0) * 0.5);
    while ((j + 1) * (j + 2) / 2 <= i) ++j;
    while (j * (j + 1) / 2 > i) --j;
    a = i - j * (j + 1) / 2;
}

// D Pi_psd on every PSD block of [cb0, cb1) (Appendix A):
//   dZ -> V (B o (V^T dZ V)) V^T
// with Z's eigenvectors V (column q = eigenvector q) and the weights B made
// at plan time.  All threads of the CTA call it (it synchronises); the
// scratch holds 2 k^2 doubles.
static __device__ __noinline__ void apply_D_psd(const double* src, double* dst, int r0, const SocBlock* blocks, int cb0,
                                         int cb1, const double* psd, double* Y) {
    constexpr double kR2 = 1.4142135623730951, kIR2 = 0.7071067811865476;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int bi = cb0; bi < cb1; ++bi) {
        const SocBlock B = blocks[bi];
        if (B.kase != kBlockPsd) continue;
        const int k = B.order, kk = k * k, d = B.dim;
        const double* V = psd + B.psd;
        const double* W = V + kk;
        const double* sb = src + (B.start - r0);
        double* db = dst + (B.start - r0);
        double* T = Y + kk;
        for (int e = tid; e < kk; e += nt) {  // Y = dZ V
            const int a = e / k, q = e - a * k;
            double acc = 0.0;
            for (int c = 0; c < k; ++c) {
                const int lo = a < c ? a : c, hi = a < c ? c : a;
                const double z = sb[hi * (hi + 1) / 2 + lo] * (a == c ? 1.0 : kIR2);
                acc = fma(z, V[c * k + q], acc);
            }
            Y[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < kk; e += nt) {  // T = B o (V^T Y)
            const int p = e / k, q = e - p * k;
            double acc = 0.0;
            for (int a = 0; a < k; ++a) acc = fma(V[a * k + p], Y[a * k + q], acc);
            T[e] = W[e] * acc;
        }
        __syncthreads();
        for (int e = tid; e < kk; e += nt) {  // Y = V T
            const int a = e / k, q = e - a * k;
            double acc = 0.0;
            for (int p = 0; p < k; ++p) acc = fma(V[a * k + p], T[p * k + q], acc);
            Y[e] = acc;
        }
        __syncthreads();
        for (int i = tid; i < d; i += nt) {   // the upper triangle of Y V^T
            int a, j;
            psd_pos(i, a, j);
            double acc = 0.0;
            for (int q = 0; q < k; ++q) acc = fma(Y[a * k + q], V[j * k + q], acc);
            db[i] = a == j ? acc : kR2 * acc;
        }
        __syncthreads();
    }
}

template <typename T, int NW = kWarps>
__device__ __forceinline__ void apply_D_tile(const double* src, double* dst, int r0, int r1, int n,
                                             const int8_t* flag, const SocBlock* blocks, int cb0,
                                             int cb1, const T* zy, int zoff = 0, bool any_large = true,
                                             const double* psd = nullptr, double* pscr = nullptr) {
    for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
        if (i < n) {
            dst[i - r0] = src[i - r0];
        } else {
            const int8_t f = flag[i];
            if (f != RF_SOC) dst[i - r0] = (f == RF_ONE) ? src[i - r0] : 0.0;
        }
    }
    // small blocks: one thread each
    for (int bi = cb0 + (int)threadIdx.x; bi < cb1; bi += blockDim.x) {
        const SocBlock B = blocks[bi];
        if (B.dim > kSocThread || B.kase == kBlockPsd) continue;
        const double* sb = src + (B.start - r0);
        double* db = dst + (B.start - r0);
        if (B.kase == kBlockDense) {
            const double* Dm = psd + B.psd;
            for (int i = 0; i < B.dim; ++i) {
                double acc = 0.0;
                for (int j = 0; j < B.dim; ++j) acc = fma(Dm[i * B.dim + j], sb[j], acc);
                db[i] = acc;
            }
        } else if (B.kase == 0) {
            for (int k = 0; k < B.dim; ++k) db[k] = 0.0;
        } else if (B.kase == 1) {
            for (int k = 0; k < B.dim; ++k) db[k] = sb[k];
        } else {
            const T* u = zy + (B.start - zoff);
            double d0 = 0.0, d1 = 0.0;  // two chains: half the dependent latency
            int k = 1;
            for (; k + 1 < B.dim; k += 2) {
                d0 = fma(ld(u + k), sb[k], d0);
                d1 = fma(ld(u + k + 1), sb[k + 1], d1);
            }
            if (k < B.dim) d0 = fma(ld(u + k), sb[k], d0);
            const double dot = d0 + d1;
            const double ct = sb[0];
            db[0] = B.h * fma(B.r, ct, dot);
            const double a = B.h * fma(-B.tq, dot, ct), b = B.h * (B.t + B.r);
            for (int k = 1; k < B.dim; ++k) db[k] = fma(a, ld(u + k), b * sb[k]);
        }
    }
    // PSD blocks: the whole CTA, one block after the other
    if (psd) apply_D_psd(src, dst, r0, blocks, cb0, cb1, psd, pscr);
    // large blocks: one warp each
    if (!any_large) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int bi = cb0 + warp; bi < cb1; bi += NW) {
        const SocBlock B = blocks[bi];
        if (B.dim <= kSocThread || B.kase == kBlockPsd) continue;
        const double* sb = src + (B.start - r0);
        double* db = dst + (B.start - r0);
        if (B.kase == 0) {
            for (int k = lane; k < B.dim; k += 32) db[k] = 0.0;
        } else if (B.kase == 1) {
            for (int k = lane; k < B.dim; k += 32) db[k] = sb[k];
        } else {
            const T* u = zy + (B.start - zoff);
            double dot = 0.0;
            for (int k = 1 + lane; k < B.dim; k += 32) dot = fma(ld(u + k), sb[k], dot);
            dot = warp_sum(dot);
            const double ct = sb[0];
            if (lane == 0) db[0] = B.h * fma(B.r, ct, dot);
            const double a = B.h * fma(-B.tq, dot, ct), b = B.h * (B.t + B.r);
            for (int k = 1 + lane; k < B.dim; k += 32) db[k] = fma(a, ld(u + k), b * sb[k]);
        }
    }
}

}  // namespace qcpd
