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

struct SocBlock {
    int32_t start;   // local embedding row of the block's t entry (n + first y row)
    int32_t dim;
    int32_t kase;    // 0: ||u|| <= -t (D = 0), 1: ||u|| <= t (D = I), 2: formula
    int32_t pad;
    double t, r;     // t and ||u|| of z_y on the block
};

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
    int32_t status, outcome, first, pad;
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

// Block-wide sums of NV values per thread, in a fixed order (deterministic
// for a fixed block size).  The result is valid in warp 0.  FP64 issue is
// scarce on this GPU (1/64 of FP32), so the values go through shared memory
// and only warp 0 adds: NV * (kWarps + 5) warp-wide FP64 adds in total
// instead of NV * 5 per warp with shuffles alone.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) red[j * kThreads + threadIdx.x] = v[j];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < kWarps; ++q) s += red[j * kThreads + q * 32 + lane];
            v[j] = warp_sum(s);
        }
    }
    __syncthreads();
}

// Shared scratch of the block reductions: up to 4 values per thread.
struct Scratch {
    double red[4 * kThreads];
};

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
// depend on CTA scheduling.  No CTA ever waits on another: the last one to
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
// {0} is R), SOC blocks (whole inside the tile) use one warp each:
//   D(ct, cu) = (1/(2r)) (r ct + u^T cu,  u ct + (t + r) cu - (t/r^2)(u^T cu) u).
// Caller synchronises before and after.
template <typename T>
__device__ __forceinline__ void apply_D_tile(const double* src, double* dst, int r0, int r1, int n,
                                             const int8_t* flag, const SocBlock* blocks, int cb0,
                                             int cb1, const T* zy) {
    for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
        if (i < n) {
            dst[i - r0] = src[i - r0];
        } else {
            const int8_t f = flag[i];
            if (f != RF_SOC) dst[i - r0] = (f == RF_ONE) ? src[i - r0] : 0.0;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int bi = cb0 + warp; bi < cb1; bi += kWarps) {
        const SocBlock B = blocks[bi];
        const int s0 = B.start - r0;
        if (B.kase == 0) {
            for (int k = lane; k < B.dim; k += 32) dst[s0 + k] = 0.0;
        } else if (B.kase == 1) {
            for (int k = lane; k < B.dim; k += 32) dst[s0 + k] = src[s0 + k];
        } else {
            const double ct = src[s0];
            double dot = 0.0;
            for (int k = 1 + lane; k < B.dim; k += 32) dot += ld(zy + B.start + k) * src[s0 + k];
            dot = warp_sum(dot);
            const double inv2r = 0.5 / B.r;
            const double tr = B.t + B.r;
            const double tq = B.t / (B.r * B.r);
            if (lane == 0) dst[s0] = (B.r * ct + dot) * inv2r;
            for (int k = 1 + lane; k < B.dim; k += 32) {
                const double u = ld(zy + B.start + k);
                dst[s0 + k] = (u * ct + tr * src[s0 + k] - tq * dot * u) * inv2r;
            }
        }
    }
}

}  // namespace qcpd
