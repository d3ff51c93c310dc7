// Tile kernels of the Krylov hot loop and of the JVP/VJP right-hand sides
// and outputs (arXiv 2508.17522, Sec. 3.1-3.2).  See qcpd_common.cuh for the
// G = S F formulation that every kernel here follows.
//
// Diagonal scaling.  LSQR runs on Op = W G C, W = diag(w) (rows), C = diag(c)
// (columns, constant on each second-order-cone block so that C commutes with
// D Pi).  W = C = I is the plain method.  Because both linear systems are
// consistent, row scaling does not change their solutions; column scaling is
// undone on output (dz = C x, r' = W x).  The column scalings are folded into
// two copies of M's values, MG = M diag(c) for G-passes and MT = M diag(w)
// for G^T-passes, so a scaled pass moves the same bytes as a plain one.
//
// Precision.  M's values and the caller's arrays are T (float64 or float32);
// the per-row data derived at plan time (q, b, g, x, y, y - s), the Krylov
// vectors and every sum are float64, so FP32 storage only rounds the inputs.
#pragma once

#include "qcpd_common.cuh"

namespace qcpd {

enum PassKind { PASS_G = 0, PASS_GT = 1 };
enum RoleKind { ROLE_U = 0, ROLE_V = 1, ROLE_RES = 2, ROLE_WARM = 3 };

template <typename T>
struct PlanView {
    const Tile* tiles;
    const Sys* sys;
    const Prob* probs;
    LsqrState* state;
    Reduce R;
    int* active;             // number of systems still iterating
    int32_t* split_cnt;      // per split row: chunks finished in this launch
    double* row_part;        // per LONG tile: its chunk's partial row sum
    const int64_t* mrowptr;  // global row pointers of M
    const int32_t* mcol;     // local column indices of M
    const T* mval;           // values of M
    const T* mvalG;          // M diag(c)   (== mval when unscaled)
    const T* mvalT;          // M diag(w)   (== mval when unscaled)
    const int32_t* mvmap;    // position of each M value in the problem's [P values; A values]
    const double* coefA;     // N-indexed: q (x-rows), b (y-rows)
    const double* coefB;     // N-indexed: g = 2 P x + q (x-rows), b (y-rows)
    const double* pz;        // N-indexed: x (x-rows), y (y-rows)  -- Pi z without tau
    const double* zy;        // N-indexed: y - s on y-rows
    const int8_t* flag;      // N-indexed RowFlag on y-rows
    const SocBlock* blocks;
    const double* rw;        // N-indexed row scaling w
    const double* cd;        // N-indexed column scaling c
    int scaled;              // 0: plain method (w = c = 1)
    double* U;               // Krylov u (unnormalised: u * beta)
    double* V;               // Krylov v (unnormalised: v * alpha)
    double* W;               // LSQR direction w
    double* X;               // LSQR iterate
    double* XI;              // D Pi applied to the vector the G-pass gathers
    double* RHS;             // right-hand side b of min ||Op x - b||
    double* HB;              // LSMR hbar (W holds h)
    int lsmr;                // 0: LSQR, 1: LSMR (pass and persistent engines)
    const double* psd;       // PSD blocks' eigenvectors and weights (nullptr: the plan has none)
    int kpsd;                // largest PSD block order (0: none)
    int rmax;                // most rows in any tile (shared-memory sizing)
    int long_chunk;          // nonzeros per LONG tile
    int tile0;               // tile of blockIdx.x 0 in a tile launch (a range of the plan's systems)
};

// Dynamic shared memory of the tile kernels:
//   s0, s1, s2 rmax doubles each: per-row buffers (row sums, epilogue)
//   srp        rmax + 1 int64: the tile's row pointers
//   psd        2 kpsd^2 doubles: scratch of the PSD blocks' D Pi (kpsd = 0: none)
struct TileSmem {
    double *s0, *s1, *s2;
    int64_t* srp;
    double* psd;
};

__host__ __device__ inline size_t tile_smem_bytes(int rmax, int kpsd = 0) {
    return sizeof(double) * (size_t)(3 * rmax) + sizeof(int64_t) * (size_t)(rmax + 1) +
           sizeof(double) * 2 * (size_t)kpsd * (size_t)kpsd;
}

__device__ __forceinline__ TileSmem tile_smem(double* base, int rmax) {
    TileSmem t;
    t.s0 = base;
    t.s1 = t.s0 + rmax;
    t.s2 = t.s1 + rmax;
    t.srp = reinterpret_cast<int64_t*>(t.s2 + rmax);
    t.psd = reinterpret_cast<double*>(t.srp + rmax + 1);
    return t;
}

// Loads of vectors that other CTAs write during the same launch.  In a
// persistent launch they must bypass the (non-coherent) L1: L1 = false.
template <bool L1>
__device__ __forceinline__ double ldv(const double* p) {
    if (L1) return *p;
    return __ldcg(p);
}

// Eight consecutive stored entries starting at an index that is a multiple
// of 8 (the arrays are padded to a multiple of 8 entries): two 16-byte loads
// of column indices and 16-byte loads of values.
__device__ __forceinline__ void load8(const int32_t* col, const double* val, int64_t e, int32_t (&c)[kE],
                                      double (&v)[kE]) {
    const int4 c0 = __ldg(reinterpret_cast<const int4*>(col + e));
    const int4 c1 = __ldg(reinterpret_cast<const int4*>(col + e) + 1);
    c[0] = c0.x; c[1] = c0.y; c[2] = c0.z; c[3] = c0.w;
    c[4] = c1.x; c[5] = c1.y; c[6] = c1.z; c[7] = c1.w;
    const double2* vp = reinterpret_cast<const double2*>(val + e);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double2 t = __ldg(vp + j);
        v[2 * j] = t.x;
        v[2 * j + 1] = t.y;
    }
}

__device__ __forceinline__ void load8(const int32_t* col, const float* val, int64_t e, int32_t (&c)[kE],
                                      double (&v)[kE]) {
    const int4 c0 = __ldg(reinterpret_cast<const int4*>(col + e));
    const int4 c1 = __ldg(reinterpret_cast<const int4*>(col + e) + 1);
    c[0] = c0.x; c[1] = c0.y; c[2] = c0.z; c[3] = c0.w;
    c[4] = c1.x; c[5] = c1.y; c[6] = c1.z; c[7] = c1.w;
    const float4* vp = reinterpret_cast<const float4*>(val + e);
    const float4 t0 = __ldg(vp), t1 = __ldg(vp + 1);
    v[0] = t0.x; v[1] = t0.y; v[2] = t0.z; v[3] = t0.w;
    v[4] = t1.x; v[5] = t1.y; v[6] = t1.z; v[7] = t1.w;
}

// Row sums of rows [0, rows) whose row pointers (global nonzero indices)
// are srp[0..rows] in shared memory, into s0[] (zeroed by the caller, all
// threads synchronised).  The merge-style segmented SpMV described at
// tile_rowsums; gather(j) returns the vector entry of column j.  Ends with a
// block barrier.  NW: warps of the CTA.
template <int NW = kWarps, typename VT, typename GF>
__device__ __forceinline__ void stream_rowsums(const int64_t* srp, const int rows, const int32_t* mcol,
                                               const VT* vals, GF gather, double* s0) {
    const int tid = threadIdx.x;
    const int64_t K0 = srp[0], K1 = srp[rows];
    // Each warp owns the rows that start in its share (1/NW) of the tile's
    // nonzeros, so no partial sum crosses a warp and the sweeps below need
    // only warp-level synchronisation.
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t q = (K1 - K0 + NW - 1) / NW;
    auto lower = [&](int64_t key) {  // first row whose start is >= key
        int lo = 0, hi = rows;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (srp[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    const int w0 = (warp == 0) ? 0 : lower(K0 + warp * q);
    const int w1 = (warp == NW - 1) ? rows : lower(K0 + (warp + 1) * q);
    if (w1 > w0) {
        const int64_t WK0 = srp[w0], WK1 = srp[w1];
        for (int64_t c0 = WK0 & ~(int64_t)(kE - 1); c0 < WK1; c0 += 32 * kE) {
            const int64_t e0 = c0 + (int64_t)lane * kE;
            // head: the lane's first row segment; tail: its last (the same
            // segment when the lane's eight entries lie in one row)
            int hk = -1, tk = -1;
            double hv = 0.0, tv = 0.0;
            if (e0 < WK1 && e0 + kE > WK0) {
                int32_t c[kE];
                double v[kE], x[kE];
                load8(mcol, vals, e0, c, v);
#pragma unroll
                for (int j = 0; j < kE; ++j) {
                    const bool ok = (e0 + j >= WK0) && (e0 + j < WK1);
                    x[j] = ok ? gather(c[j]) : 0.0;
                }
                const int64_t kfirst = e0 > WK0 ? e0 : WK0;
                int lo = w0, hi = w1;  // last row whose start is <= kfirst
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (srp[mid] <= kfirst) lo = mid;
                    else hi = mid;
                }
                // row of each of the eight entries (-1: outside the warp's range)
                int rr[kE];
                int i = lo;
                int64_t rend = srp[i + 1];
#pragma unroll
                for (int j = 0; j < kE; ++j) {
                    const int64_t k = e0 + j;
                    if (k < kfirst || k >= WK1) {
                        rr[j] = -1;
                    } else {
                        while (k >= rend) {
                            ++i;
                            rend = srp[i + 1];
                        }
                        rr[j] = i;
                    }
                }
                // branch-free FMA chain: restart at every row change
                double acc = 0.0, part[kE];
#pragma unroll
                for (int j = 0; j < kE; ++j) {
                    const bool cont = (j > 0) && (rr[j] == rr[j - 1]);
                    acc = fma(v[j], x[j], cont ? acc : 0.0);
                    part[j] = acc;
                }
#pragma unroll
                for (int j = 0; j < kE; ++j) {
                    if (rr[j] >= 0) {
                        if (hk < 0) hk = rr[j];
                        tk = rr[j];
                    }
                }
#pragma unroll
                for (int j = 0; j < kE; ++j) {
                    const bool end = rr[j] >= 0 && (j == kE - 1 || rr[j + 1] != rr[j]);
                    if (end) {
                        if (rr[j] == hk) hv = part[j];
                        if (rr[j] == tk) tv = part[j];
                        // a row that starts and ends inside this lane's group
                        if (rr[j] != hk && rr[j] != tk) s0[rr[j]] = part[j];
                    }
                }
            }
            // Rows crossing lanes: a segmented inclusive scan of the tails
            // along the lanes.  A chain passes through lanes that hold one
            // segment of the same row and restarts at a lane with two or
            // more segments (or a new row); the lane whose head continues a
            // chain adds the chain's sum to its head.
            const unsigned full = 0xffffffffu;
            const bool single = (hk == tk);
            const int ptk = __shfl_up_sync(full, tk, 1);
            int f = (lane == 0) || !single || tk != ptk || tk < 0;
            double S = tv;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const double oS = __shfl_up_sync(full, S, d);
                const int of = __shfl_up_sync(full, f, d);
                if (lane >= d && !f) {
                    S = oS + S;
                    f = of;
                }
            }
            const double pS = __shfl_up_sync(full, S, 1);
            const int nhk = __shfl_down_sync(full, hk, 1);
            if (!single && hk >= 0) {
                const double h = (lane > 0 && hk == ptk) ? pS + hv : hv;
                s0[hk] += h;  // the head row closes here
            }
            if (tk >= 0 && (lane == 31 || nhk != tk)) s0[tk] += S;  // the tail row's chain ends here
            __syncwarp();
        }
    }
    __syncthreads();
}

// Row sums h_i = sum_k val_k * gv[col_k] of the tile's rows into sm.s0[].
//
// STREAM tiles (merge-style segmented SpMV): the tile's nonzeros are walked
// in aligned groups of kE = 8; thread t takes one group per sweep, loads its
// eight column indices and values with vector loads and issues the eight
// gathers at once (about 24 loads in flight per thread), then multiplies the
// eight entries in one FMA chain, cutting it at row ends.  Rows that start
// and end inside a thread's group are written directly; the first and last
// segment of each group go to boundary slots that one thread per row adds
// up in thread order.  Exactly one FP64 FMA per nonzero, and the result does
// not depend on scheduling.
//
// LONG tiles sum one chunk of one long row over the whole CTA (same aligned
// loads); the last chunk of the row to finish adds the chunk sums in order.
//
// Returns the number of rows whose sums are complete (0 for a LONG tile
// that is not the row's last chunk).
template <bool L1, typename VT>
__device__ __forceinline__ int tile_rowsums(const Tile& tl, int ti, const int64_t* rp, const int32_t* mcol,
                                            const VT* vals, const double* gv, const TileSmem& sm, Scratch* scratch,
                                            int32_t* split_cnt, double* row_part, int long_chunk) {
    const int tid = threadIdx.x;
    const int rows = tl.r1 - tl.r0;
    if (tl.kind == TILE_LONG) {
        const int64_t rs = rp[tl.r0], re = rp[tl.r0 + 1];
        const int64_t k0 = rs + (int64_t)tl.cb0 * long_chunk;
        const int64_t k1 = (k0 + long_chunk < re) ? k0 + long_chunk : re;
        double acc = 0.0;
        for (int64_t e = (k0 & ~(int64_t)(kE - 1)) + (int64_t)tid * kE; e < k1; e += (int64_t)kChunk) {
            int32_t c[kE];
            double v[kE];
            load8(mcol, vals, e, c, v);
            double x[kE];
#pragma unroll
            for (int j = 0; j < kE; ++j) {
                const bool ok = (e + j >= k0) && (e + j < k1);
                x[j] = ok ? ldv<L1>(gv + c[j]) : 0.0;
            }
#pragma unroll
            for (int j = 0; j < kE; ++j) acc = fma(v[j], x[j], acc);
        }
        const double s = block_sum(acc, scratch);
        __shared__ int s_last;
        if (tid == 0) {
            if (tl.cb1 == 1) {
                sm.s0[0] = s;
                s_last = 1;
            } else {
                row_part[ti] = s;
                __threadfence();
                const int prev = atomicAdd(split_cnt + tl.split, 1);
                s_last = (prev == tl.cb1 - 1);
                if (s_last) {
                    __threadfence();
                    double t = 0.0;
                    const int first = ti - tl.cb0;
                    for (int c = 0; c < tl.cb1; ++c) t += __ldcg(row_part + first + c);
                    sm.s0[0] = t;
                    split_cnt[tl.split] = 0;
                }
            }
        }
        __syncthreads();
        return s_last ? 1 : 0;
    }
    for (int i = tid; i < rows; i += kThreads) sm.s0[i] = 0.0;
    for (int i = tid; i <= rows; i += kThreads) sm.srp[i] = rp[tl.r0 + i];
    __syncthreads();
    stream_rowsums(sm.srp, rows, mcol, vals, [&](int32_t c) { return ldv<L1>(gv + c); }, sm.s0);
    return rows;
}

// The LSQR scalar recurrences (Paige & Saunders 1982) after a u-update with
// ||u_{k+1}|| = nrm (inv_nrm = 1/nrm, 0 when nrm = 0): the plane rotation
// eliminating beta_{k+1}, the coefficients of the next v-update and
// x-update, and the stopping tests.  S is LsqrState, volatile LsqrState or a
// register copy of the fields used here (the stream engine's LsqrHot).
// One thread runs this and every FP64 instruction here costs a full
// warp-wide issue, so the square root and the reciprocal of the rotation
// share one rsqrt_fast.
// nsq = nrm^2 (the sum of squares nrm came from), so the rotation's square
// root does not wait for nrm's.
template <typename S>
__device__ __forceinline__ void lsqr_step_u(S* st, double nrm, double inv_nrm, double nsq) {
    const double rhobar = st->rhobar;
    double rho, inv;
    norm_and_inverse(fma(rhobar, rhobar, nsq), rho, inv);
    const double c = rhobar * inv, s = nrm * inv;
    const double phibar = st->phibar;
    const double phi = c * phibar;
    st->phibar = s * phibar;
    st->inv_rho = inv;
    st->c = c;
    st->s = s;
    st->xcoef = phi * inv;
    st->beta = nrm;
    st->vc1 = inv_nrm;  // next v-update: 1/beta, beta/alpha
    st->vc2 = nrm * st->uc1;
    st->iters += 1;
    if (!finite64(rho) || !finite64(phi) || !(rho > 0.0)) {
        st->outcome = O_BREAKDOWN;
        st->xcoef = 0.0;
        st->status = S_FINAL;
    } else if (st->phibar <= st->rtol * st->bnorm || nrm == 0.0) {
        st->outcome = O_CONVERGED;
        st->status = S_FINAL;
    } else if (st->iters >= st->maxiter) {
        st->outcome = O_MAXITER;
        st->status = S_FINAL;
    }
}

// The same after a v-update with ||v_{k+1}|| = nrm.  Returns true when the
// system has just finished (v = 0: the current x solves the problem).
template <typename S>
__device__ __forceinline__ bool lsqr_step_v(S* st, double nrm, double inv_nrm) {
    if (st->first) {
        st->rhobar = nrm;
        st->phibar = st->beta;
        st->wcoef = 0.0;
        st->first = 0;
    } else {
        st->rhobar = -st->c * nrm;
        st->wcoef = (st->s * nrm) * st->inv_rho;
    }
    st->alpha = nrm;
    st->uc1 = inv_nrm;  // next u-update: 1/alpha, alpha/beta
    st->uc2 = nrm * st->vc1;
    if (!(nrm > 0.0) || !finite64(nrm)) {
        st->outcome = finite64(nrm) ? O_CONVERGED : O_BREAKDOWN;
        st->status = S_DONE;
        return true;
    }
    return false;
}

// LSMR (Fong & Saunders 2011, damping 0) on the same bidiagonalisation.
// The u-pass only stores beta_{k+1}; once the v-pass has alpha_{k+1}, the
// finisher runs both rotations of iteration k, the residual-norm estimate
// and the stopping test, and leaves the coefficients of the deferred vector
// updates for the next u-pass:
//   hbar_k = h_k - hcoef hbar_{k-1},  x_k = x_{k-1} + xcoef hbar_k,
//   h_{k+1} = v_{k+1} - wcoef h_k.
template <typename S>
__device__ __forceinline__ bool lsmr_step_u(S* st, double nrm, double inv_nrm) {
    st->beta = nrm;
    // beta = 0: the Krylov space is exhausted; the v-pass then yields
    // alpha = 0 and the finisher stops after the last update
    const bool live = nrm > 0.0 && finite64(nrm);
    st->vc1 = live ? inv_nrm : 0.0;
    st->vc2 = live ? nrm * st->uc1 : 0.0;
    if (!finite64(nrm)) {  // x keeps the last finite update
        st->outcome = O_BREAKDOWN;
        st->status = S_DONE;
        return true;
    }
    return false;
}

// Returns true when the system stops without a final update pass.
template <typename S>
__device__ __forceinline__ bool lsmr_step_v(S* st, double nrm, double inv_nrm) {
    const bool live = nrm > 0.0 && finite64(nrm);
    st->uc1 = live ? inv_nrm : 0.0;  // next u-update: 1/alpha, alpha/beta
    st->uc2 = nrm * st->vc1;
    st->alpha = nrm;
    st->upd = 1;
    if (st->first) {
        const double beta1 = st->beta;
        st->first = 0;
        st->alphabar = nrm;
        st->zetabar = nrm * beta1;
        st->rho_old = 1.0;
        st->rhobar_old = 1.0;
        st->cbar = 1.0;
        st->sbar = 0.0;
        st->betadd = beta1;
        st->betad = 0.0;
        st->rhod_old = 1.0;
        st->tautilde_old = 0.0;
        st->thetatilde = 0.0;
        st->zeta_old = 0.0;
        st->hcoef = st->xcoef = st->wcoef = 0.0;  // first u-pass: h_1 = v_1
        st->phibar = beta1;
        if (!live) {  // A^T b = 0: x = 0 is the least-squares solution
            st->outcome = finite64(nrm) ? O_CONVERGED : O_BREAKDOWN;
            st->status = S_DONE;
            return true;
        }
        return false;
    }
    const double beta = st->beta;  // beta_{k+1}
    // first rotation: (alphabar_k, beta_{k+1}) -> rho_k
    double rho, irho;
    norm_and_inverse(fma(st->alphabar, st->alphabar, beta * beta), rho, irho);
    const double c = st->alphabar * irho, s = beta * irho;
    const double theta_new = s * nrm;  // theta_{k+1}
    st->alphabar = c * nrm;
    // second rotation: (cbar_{k-1} rho_k, theta_{k+1}) -> rhobar_k
    const double thetabar = st->sbar * rho;
    const double t = st->cbar * rho;
    double rhobar, irhobar;
    norm_and_inverse(fma(t, t, theta_new * theta_new), rhobar, irhobar);
    const double cbar = t * irhobar, sbar = theta_new * irhobar;
    const double zeta = cbar * st->zetabar;
    st->zetabar = -sbar * st->zetabar;
    // deferred vector updates of iteration k
    st->hcoef = thetabar * rho / (st->rho_old * st->rhobar_old);
    st->xcoef = zeta * (irho * irhobar);
    st->wcoef = theta_new * irho;
    // estimate of ||r_k|| (the residual of the least-squares problem)
    const double betahat = c * st->betadd;
    st->betadd = -s * st->betadd;
    double rhotilde, irhotilde;
    norm_and_inverse(fma(st->rhod_old, st->rhod_old, thetabar * thetabar), rhotilde, irhotilde);
    const double ctilde = st->rhod_old * irhotilde, stilde = thetabar * irhotilde;
    const double thetatilde_old = st->thetatilde;
    st->thetatilde = stilde * rhobar;
    const double rhod = ctilde * rhobar;
    st->betad = -stilde * st->betad + ctilde * betahat;
    st->tautilde_old = (st->zeta_old - thetatilde_old * st->tautilde_old) * irhotilde;
    const double taud = (zeta - st->thetatilde * st->tautilde_old) / rhod;
    const double dr = st->betad - taud;
    const double normr = sqrt(fma(dr, dr, st->betadd * st->betadd));
    st->rhod_old = rhod;
    st->zeta_old = zeta;
    st->rho_old = rho;
    st->rhobar_old = rhobar;
    st->cbar = cbar;
    st->sbar = sbar;
    st->phibar = normr;
    st->iters += 1;
    if (!finite64(st->xcoef) || !finite64(st->hcoef) || !finite64(st->wcoef) || !(rho > 0.0) ||
        !(rhobar > 0.0)) {
        st->outcome = O_BREAKDOWN;
        st->status = S_DONE;
        return true;
    }
    if (normr <= st->rtol * st->bnorm || !live) {
        st->outcome = finite64(nrm) ? O_CONVERGED : O_BREAKDOWN;
        st->status = S_FINAL;
    } else if (st->iters >= st->maxiter) {
        st->outcome = O_MAXITER;
        st->status = S_FINAL;
    }
    return false;
}

// LSMR's deferred vector updates of row r (w holds h, hb holds hbar; iv is
// the row of the unnormalised v_{k+1}, c1 = 1 / alpha_{k+1}):
//   hbar <- h - hcoef hbar,  x <- x + xcoef hbar,  h <- v - wcoef h.
__device__ __forceinline__ void lsmr_update(double* X, double* W, double* HB, int r, double iv, double c1,
                                            double hcoef, double xcoef, double wcoef) {
    const double h = W[r];
    const double hb = fma(-hcoef, HB[r], h);
    HB[r] = hb;
    X[r] = fma(xcoef, hb, X[r]);
    W[r] = fma(iv, c1, -wcoef * h);
}

// One half-iteration of LSQR over all tiles of all systems.
//   PASS_G : out = W G C in     (gathers XI = D Pi in, values M diag(c))
//   PASS_GT: out = C G^T W in   (gathers in, values M diag(w); D Pi on the output side)
//   ROLE_U : u <- (Op v)/alpha - (alpha/beta) u,  w <- v/alpha - wcoef w   (in = V, out = U)
//   ROLE_V : v <- (Op^T u)/beta - (beta/alpha) v, x <- x + xcoef w         (in = U, out = V)
//   ROLE_RES: unscaled residual of the current iterate                    (in = X)
//   SC     : diagonal scaling on (compile-time, so the plain method pays no
//            multiplications by 1 on the scarce FP64 pipe)
// The CTA that completes a system also updates its tau entry and the LSQR
// scalars (Paige & Saunders 1982, algorithm LSQR).
// The work of one tile in one pass (and, in the CTA that completes its
// system, the system's finisher).  Every thread of the CTA calls it; it
// returns in a CTA-uniform way except for the finisher, which only thread 0
// runs, so callers synchronise before touching shared memory again.
template <int PASS, int ROLE, bool SC, bool L1, typename T>
__device__ __forceinline__ void run_tile(const PlanView<T>& a, const int ti, double* smem, Scratch& scratch) {
    const Tile tl = a.tiles[ti];
    const Sys sy = a.sys[tl.sys];
    volatile LsqrState* st = a.state + tl.sys;
    const int status = st->status;
    if (ROLE != ROLE_RES && status == S_DONE) return;
    const bool lsmr = a.lsmr != 0;
    // the last deferred update of a stopped system: LSQR's x-update in the
    // v-pass, LSMR's (hbar, x, h) updates in the u-pass
    const bool only_x = (ROLE == ROLE_V && status == S_FINAL && !lsmr);
    const bool only_upd = (ROLE == ROLE_U && status == S_FINAL && lsmr);
    const Prob pr = a.probs[sy.prob];
    const int n = pr.n;
    const int N = pr.n + pr.m + 1;
    const TileSmem sm = tile_smem(smem, a.rmax);
    double* s0 = sm.s0;
    double* s1 = sm.s1;
    double* s2 = sm.s2;

    const double* in = (ROLE == ROLE_U) ? a.V + sy.voff : (ROLE == ROLE_V ? a.U + sy.voff : a.X + sy.voff);
    double* outv = (ROLE == ROLE_U || ROLE == ROLE_WARM) ? a.U + sy.voff : (ROLE == ROLE_V ? a.V + sy.voff : nullptr);
    const double* cA = a.coefA + pr.doff;
    const double* cB = a.coefB + pr.doff;
    const double* rw = a.rw + pr.doff;
    const double* cd = a.cd + pr.doff;
    double* W = a.W + sy.voff;
    double* X = a.X + sy.voff;
    double* XI = a.XI + sy.voff;
    // the finisher of the previous pass stored this pass's coefficients, so
    // no tile divides (FP64 division is a long dependent chain here)
    double c1, c2;
    if (ROLE == ROLE_U) {
        c1 = st->uc1;
        c2 = st->uc2;
    } else if (ROLE == ROLE_V) {
        c1 = st->vc1;
        c2 = st->vc2;
    } else {
        c1 = 1.0;
        c2 = 0.0;
    }
    const double wcoef = st->wcoef, xcoef = st->xcoef;
    const double hcoef = lsmr ? st->hcoef : 0.0;
    const bool upd = lsmr && st->upd != 0;  // LSMR: this u-pass applies the deferred updates
    double* HB = lsmr ? a.HB + sy.voff : nullptr;
    const double tin = ldv<L1>(in + N - 1);  // tau entry of the input vector
    // the t-column term: (scaled) tau entry of the input
    const double tt = SC ? (PASS == PASS_G ? cd[N - 1] : rw[N - 1]) * tin : tin;

    Part part = pzero();
    int rows = tl.r1 - tl.r0;
    if (only_x || only_upd) {
        if (tl.kind == TILE_LONG && tl.cb0 != 0) rows = 0;  // one chunk updates the row
        for (int i = threadIdx.x; i < rows; i += kThreads) {
            const int r = tl.r0 + i;
            if (only_x) X[r] = fma(xcoef, ldv<L1>(W + r), ldv<L1>(X + r));
            else lsmr_update(X, W, HB, r, ldv<L1>(in + r), c1, hcoef, xcoef, wcoef);
        }
    } else {
        const int64_t* rp = a.mrowptr + pr.mrow;
        if (PASS == PASS_G)
            rows = tile_rowsums<L1>(tl, ti, rp, a.mcol, a.mvalG, XI, sm, &scratch, a.split_cnt, a.row_part,
                                    a.long_chunk);
        else
            rows = tile_rowsums<L1>(tl, ti, rp, a.mcol, a.mvalT, in, sm, &scratch, a.split_cnt, a.row_part,
                                    a.long_chunk);
        double ss = 0.0, dtop = 0.0, dbot = 0.0;
        if (PASS == PASS_G) {
            for (int i = threadIdx.x; i < rows; i += kThreads) {
                const int r = tl.r0 + i;
                const double iv = ldv<L1>(in + r);
                double o;
                if (r < n) {
                    o = fma(ld(cA + r), tt, s0[i]);
                    dtop = fma(ld(cB + r), SC ? cd[r] * iv : iv, dtop);
                } else {
                    const double xi = ldv<L1>(XI + r);
                    const double dxi = SC ? cd[r] * (xi - iv) : xi - iv;
                    o = fma(-ld(cA + r), tt, s0[i]) + dxi;
                    dbot = fma(ld(cB + r), SC ? cd[r] * xi : xi, dbot);
                }
                if (SC) o *= rw[r];
                if (ROLE == ROLE_RES) {
                    double e = o - ldv<L1>(a.RHS + sy.voff + r);
                    if (SC) e /= rw[r];
                    ss = fma(e, e, ss);
                } else if (ROLE == ROLE_WARM) {
                    const double u = ldv<L1>(a.RHS + sy.voff + r) - o;
                    outv[r] = u;
                    ss = fma(u, u, ss);
                } else {
                    const double nv = fma(c1, o, -c2 * ldv<L1>(outv + r));
                    outv[r] = nv;
                    ss = fma(nv, nv, ss);
                    if (ROLE == ROLE_U) {
                        if (!lsmr) W[r] = fma(iv, c1, -wcoef * ldv<L1>(W + r));
                        else if (upd) lsmr_update(X, W, HB, r, iv, c1, hcoef, xcoef, wcoef);
                    } else if (!lsmr) {
                        X[r] = fma(xcoef, ldv<L1>(W + r), ldv<L1>(X + r));
                    }
                }
            }
        } else {
            // G^T: top rows M rho - g r3; bottom rows D(M rho - b r3 + r2) - r2 (rho = W in)
            for (int i = threadIdx.x; i < rows; i += kThreads) {
                const int r = tl.r0 + i;
                const double iv = SC ? rw[r] * ldv<L1>(in + r) : ldv<L1>(in + r);
                const double h = fma(-ld(cB + r), tt, s0[i]);
                if (r < n) {
                    s1[i] = h;
                    dtop = fma(ld(cA + r), iv, dtop);
                } else {
                    s1[i] = h + iv;
                    dbot = fma(ld(cA + r), iv, dbot);
                }
            }
            __syncthreads();
            const int cb0 = tl.kind == TILE_STREAM ? tl.cb0 : 0, cb1 = tl.kind == TILE_STREAM ? tl.cb1 : 0;
            apply_D_tile<double>(s1, s2, tl.r0, tl.r0 + rows, n, a.flag + pr.doff, a.blocks + pr.soff, cb0, cb1,
                                 a.zy + pr.doff, 0, true, a.psd, sm.psd);
            __syncthreads();
            for (int i = threadIdx.x; i < rows; i += kThreads) {
                const int r = tl.r0 + i;
                const double iv = ldv<L1>(in + r);
                double o = (r < n) ? s2[i] : s2[i] - (SC ? rw[r] * iv : iv);
                if (SC) o *= cd[r];
                if (ROLE == ROLE_RES) {
                    double e = o - ldv<L1>(a.RHS + sy.voff + r);
                    if (SC) e /= cd[r];
                    ss = fma(e, e, ss);
                } else if (ROLE == ROLE_WARM) {
                    const double u = ldv<L1>(a.RHS + sy.voff + r) - o;
                    outv[r] = u;
                    s1[i] = u;
                    ss = fma(u, u, ss);
                } else {
                    const double nv = fma(c1, o, -c2 * ldv<L1>(outv + r));
                    outv[r] = nv;
                    s1[i] = nv;
                    ss = fma(nv, nv, ss);
                    if (ROLE == ROLE_U) {
                        if (!lsmr) W[r] = fma(iv, c1, -wcoef * ldv<L1>(W + r));
                        else if (upd) lsmr_update(X, W, HB, r, iv, c1, hcoef, xcoef, wcoef);
                    } else if (!lsmr) {
                        X[r] = fma(xcoef, ldv<L1>(W + r), ldv<L1>(X + r));
                    }
                }
            }
            if (ROLE != ROLE_RES) {
                __syncthreads();
                apply_D_tile<double>(s1, s2, tl.r0, tl.r0 + rows, n, a.flag + pr.doff, a.blocks + pr.soff, cb0, cb1,
                                     a.zy + pr.doff, 0, true, a.psd, sm.psd);
                __syncthreads();
                for (int i = threadIdx.x; i < rows; i += kThreads) XI[tl.r0 + i] = s2[i];
            }
        }
        part = block_sum3(ss, dtop, dbot, &scratch);
    }

    Part tot;
    if (!finish_tile(a.R, tl, sy.g0, sy.g1, ti, part, &tot, &scratch)) return;
    if (threadIdx.x != 0) return;

    // ---- the system's finisher: tau entry and LSQR scalars ----
    __threadfence();
    const int rN = N - 1;
    if (only_x || only_upd) {
        if (only_x) X[rN] = fma(xcoef, ldv<L1>(W + rN), ldv<L1>(X + rN));
        else lsmr_update(X, W, HB, rN, tin, c1, hcoef, xcoef, wcoef);
        st->upd = 0;  // applied: a continuation starts with a plain u-pass
        st->status = S_DONE;
        atomicSub(a.active, 1);
        return;
    }
    const double kappa = pr.kappa;
    double oN;
    if (PASS == PASS_G) {
        oN = -tot.b - tot.c + kappa * tt;
        if (SC) oN *= rw[rN];
    } else {
        oN = tot.b - tot.c + kappa * tt;
        if (SC) oN *= cd[rN];
    }
    // Gauge: dz_N = 0.  F z = 0 at a root, so F's last column is a
    // combination of the others and dropping it (the tau entry of every
    // x-space vector stays 0) keeps the solution set's image under D phi;
    // it also keeps the system well posed when rounding of the data has
    // moved z off the root.  G^T-passes therefore leave the tau entry of
    // their output at 0 and leave it out of norms and residuals.
    if (ROLE == ROLE_WARM) {
        // warm start: u = b - Op x0 is the new right-hand side of the
        // correction; ||b|| (bnorm) stays the reference of the stopping test
        double ss = tot.a;
        if (PASS == PASS_G) {
            const double uN = ldv<L1>(a.RHS + sy.voff + rN) - oN;
            outv[rN] = uN;
            ss = fma(uN, uN, ss);
        } else {
            outv[rN] = 0.0;
            XI[rN] = 0.0;
        }
        double nrm, inv;
        norm_and_inverse(ss, nrm, inv);
        st->beta = nrm;
        st->vc1 = inv;
        st->vc2 = 0.0;
        if (!(nrm > 0.0) || !finite64(nrm)) {
            st->outcome = finite64(nrm) ? O_CONVERGED : O_BREAKDOWN;
            st->status = S_DONE;
            atomicSub(a.active, 1);
        }
        return;
    }
    if (ROLE == ROLE_RES) {
        double ss = tot.a;
        if (PASS == PASS_G) {
            double e = oN - ldv<L1>(a.RHS + sy.voff + rN);
            if (SC) e /= rw[rN];
            ss += e * e;
        }
        st->resid_true = st->bnorm_true > 0.0 ? sqrt(ss) / st->bnorm_true : 0.0;
        return;
    }
    const double nvN = (PASS == PASS_GT) ? 0.0 : c1 * oN - c2 * ldv<L1>(outv + rN);
    outv[rN] = nvN;
    if (PASS == PASS_GT) XI[rN] = 0.0;
    const double nsq = fma(nvN, nvN, tot.a);
    double nrm, inv_nrm;
    norm_and_inverse(nsq, nrm, inv_nrm);
    if (lsmr) {
        if (ROLE == ROLE_U) {
            if (upd) lsmr_update(X, W, HB, rN, tin, c1, hcoef, xcoef, wcoef);
            if (lsmr_step_u(st, nrm, inv_nrm)) atomicSub(a.active, 1);
        } else {
            if (lsmr_step_v(st, nrm, inv_nrm)) atomicSub(a.active, 1);
        }
    } else if (ROLE == ROLE_U) {
        W[rN] = tin * c1 - wcoef * ldv<L1>(W + rN);
        lsqr_step_u(st, nrm, inv_nrm, nsq);
    } else {
        X[rN] = fma(xcoef, ldv<L1>(W + rN), ldv<L1>(X + rN));
        if (lsqr_step_v(st, nrm, inv_nrm)) atomicSub(a.active, 1);
    }
}

template <int PASS, int ROLE, bool SC, typename T>
__global__ void __launch_bounds__(kThreads, 3) k_pass(PlanView<T> a) {
    extern __shared__ double smem[];
    __shared__ Scratch scratch;
    run_tile<PASS, ROLE, SC, true, T>(a, a.tile0 + blockIdx.x, smem, scratch);
}

// ---------------------------------------------------------------------------
// Persistent form: all LSQR iterations of all systems in one cooperative
// launch.  Each CTA owns the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and runs them pass after pass; a grid barrier separates the passes (the
// CTA that completes a system still updates its scalars inside the pass).
// Every wait is bounded: after spin_limit polls (kSpinLimit unless the plan
// sets another bound) the waiting CTA records a timeout in *err and returns,
// and so do the others at their next barrier.  hold_ns > 0 makes CTA 0 wait
// that long, by the global timer, before its first barrier: a test of the
// timeout path that needs no fault and no unbounded wait.
struct PersistCtl {
    unsigned* bar_count;
    unsigned* bar_gen;
    int* stop;
    int* err;
    int64_t max_iters;
    unsigned long long spin_limit;
    long long hold_ns;
};

constexpr unsigned long long kSpinLimit = 1ull << 24;  // about 1 s with 64 ns naps

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool grid_sync(const PersistCtl& c, const int* active) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = c.bar_gen;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned prev = atomicAdd(c.bar_count, 1u);
        if (prev == gridDim.x - 1) {
            *c.bar_count = 0;  // nobody arrives again before the release below
            *(volatile int*)c.stop = (*(volatile const int*)active <= 0) ? 1 : 0;
            __threadfence();
            atomicAdd(c.bar_gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (*gen == g0) {
                if (++spins > c.spin_limit) {
                    atomicExch(c.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok && (*(volatile int*)c.err == 0) && (*(volatile int*)c.stop == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

template <int MODE, bool SC, typename T>
__global__ void __launch_bounds__(kThreads, 2) k_persist(PlanView<T> a, PersistCtl c, int ntiles) {
    extern __shared__ double smem[];
    __shared__ Scratch scratch;
    constexpr int PU = MODE == 0 ? PASS_G : PASS_GT;   // u-update pass
    constexpr int PV = MODE == 0 ? PASS_GT : PASS_G;   // v-update pass
    for (int64_t it = 0; it < c.max_iters; ++it) {
        for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
            run_tile<PU, ROLE_U, SC, false, T>(a, a.tile0 + ti, smem, scratch);
            __syncthreads();
        }
        if (c.hold_ns > 0 && it == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
            const unsigned long long t0 = global_ns();
            while (global_ns() - t0 < (unsigned long long)c.hold_ns) __nanosleep(1000);
        }
        if (!grid_sync(c, a.active)) return;
        for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
            run_tile<PV, ROLE_V, SC, false, T>(a, a.tile0 + ti, smem, scratch);
            __syncthreads();
        }
        if (!grid_sync(c, a.active)) return;
    }
}

// ---------------------------------------------------------------------------
// Warm start: the LSQR iterate of a caller-given initial dz (JVP:
// x0 = C^-1 dz0, tau entry 0 by the gauge dz_N = 0) or r (VJP:
// x0 = W^-1 S r0, every entry), one system per blockIdx.y.  z0 uses the
// systems' N-vector layout.
template <typename T>
__global__ void k_warm_init(PlanView<T> a, const double* z0, int mode, int s0) {
    const Sys sy = a.sys[s0 + blockIdx.y];
    const Prob pr = a.probs[sy.prob];
    const int n = pr.n, N = pr.n + pr.m + 1;
    const double* cd = a.cd + pr.doff;
    const double* rw = a.rw + pr.doff;
    double* X = a.X + sy.voff;
    const double* z = z0 + sy.voff;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
        double x = 0.0;
        if (mode == 0) {
            if (r < N - 1) x = a.scaled ? z[r] / cd[r] : z[r];
        } else {
            const double rp = (r >= n && r < N - 1) ? -z[r] : z[r];
            x = a.scaled ? rp / rw[r] : rp;
        }
        X[r] = x;
    }
}

// XI = D Pi(src) on the tile's rows (what a G-pass gathers): src = X for
// the warm start's first product, V when LSMR continues a JVP recurrence
// (the output pass has left D Pi(X) in XI).  src has the N-vector layout.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dpi(PlanView<T> a, const double* src) {
    extern __shared__ double smem[];
    const Tile tl = a.tiles[a.tile0 + blockIdx.x];
    if (tl.kind == TILE_LONG && tl.cb0 != 0) return;  // one chunk per long row
    const Sys sy = a.sys[tl.sys];
    const Prob pr = a.probs[sy.prob];
    const int rows = tl.r1 - tl.r0;
    const TileSmem sm = tile_smem(smem, a.rmax);
    const double* X = src + sy.voff;
    for (int i = threadIdx.x; i < rows; i += kThreads) sm.s1[i] = X[tl.r0 + i];
    __syncthreads();
    const int cb0 = tl.kind == TILE_STREAM ? tl.cb0 : 0, cb1 = tl.kind == TILE_STREAM ? tl.cb1 : 0;
    apply_D_tile<double>(sm.s1, sm.s2, tl.r0, tl.r0 + rows, pr.n, a.flag + pr.doff, a.blocks + pr.soff, cb0, cb1,
                         a.zy + pr.doff, 0, true, a.psd, sm.psd);
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += kThreads) a.XI[sy.voff + tl.r0 + i] = sm.s2[i];
}

// ---------------------------------------------------------------------------
// Solution export
// The embedding-space solution of the last solve: dz = C x (JVP) or
// r = S W x (VJP), N per system; systems below jvp_sys solved a JVP.
template <typename T>
__global__ void k_export(PlanView<T> a, int jvp_sys, double* out) {
    const Sys sy = a.sys[blockIdx.y];
    const int mode = (int)blockIdx.y < jvp_sys ? 0 : 1;
    const Prob pr = a.probs[sy.prob];
    const int n = pr.n, N = pr.n + pr.m + 1;
    const double* X = a.X + sy.voff;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
        double v;
        if (mode == 0) {
            v = a.scaled ? a.cd[pr.doff + r] * X[r] : X[r];
        } else {
            v = a.scaled ? a.rw[pr.doff + r] * X[r] : X[r];
            if (r >= n && r < N - 1) v = -v;
        }
        out[sy.voff + r] = v;
    }
}

// ---------------------------------------------------------------------------
template <typename T>
struct RhsArgs {
    const T* dP;
    const T* dA;
    const T* dq;
    const T* db;
    const T* wx;
    const T* wy;
    const T* ws;
    double rtol;
    int64_t maxiter;
    // user-array offsets of the call's first system (a call on a range of
    // a plan's systems indexes its arrays from that system)
    int64_t bx = 0, by = 0, bp = 0, ba = 0;
};

__device__ __forceinline__ void init_state(LsqrState* st, int* active, double bn, double bn_true, double rtol,
                                           int64_t maxiter) {
    LsqrState q{};
    q.beta = bn;
    q.bnorm = bn;
    q.bnorm_true = bn_true;
    q.rtol = rtol;
    q.maxiter = maxiter;
    q.first = 1;
    q.resid_true = -1.0;
    q.vc1 = bn > 0.0 ? 1.0 / bn : 0.0;  // the first v-update: v = G^T u / beta
    q.vc2 = 0.0;
    if (bn > 0.0 && isfinite(bn)) {
        q.status = S_ACTIVE;
        q.outcome = O_RUNNING;
        atomicAdd(active, 1);
    } else {
        q.status = S_DONE;
        q.outcome = isfinite(bn) ? O_CONVERGED : O_BREAKDOWN;
        q.resid_true = 0.0;
    }
    *st = q;
}

// JVP right-hand side (Sec. 3.1): dN = D_theta N(z)[d theta]
//   = (dP x + dA^T y + dq, -dA x + db, -x^T dP x - dq^T x - db^T y).
// LSQR solves min ||W G C x - b|| with b = -W S dN:
//   S dN negated = (-(dP x + dA^T y + dq), -dA x + db, x^T dP x + dq^T x + db^T y).
// The perturbation values are read through the M -> [P; A] value map, so
// the same pass yields dP x (both triangles) and dA^T y.  One warp per row.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_jvp_rhs(PlanView<T> a, RhsArgs<T> in) {
    __shared__ Scratch scratch;
    const int ti = a.tile0 + blockIdx.x;
    const Tile tl = a.tiles[ti];
    const Sys sy = a.sys[tl.sys];
    const Prob pr = a.probs[sy.prob];
    const int n = pr.n;
    const int N = pr.n + pr.m + 1;
    const int64_t* rp = a.mrowptr + pr.mrow;
    const double* pz = a.pz + pr.doff;
    const T* dP = in.dP + (sy.po - in.bp);
    const T* dA = in.dA + (sy.ao - in.ba);
    const double* rw = a.rw + pr.doff;
    const bool sc = a.scaled != 0;
    const int64_t pnz = pr.pnz;
    double* U = a.U + sy.voff;
    double* RHS = a.RHS + sy.voff;
    double* X = a.X + sy.voff;
    double* W = a.W + sy.voff;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // A LONG tile's chunks all cover the same row: chunk 0 does the whole row
    // with the CTA, the other chunks only join the reduction.
    const bool is_long = tl.kind == TILE_LONG;
    const bool skip = is_long && tl.cb0 != 0;
    double ss = 0.0, sst = 0.0, dtop = 0.0, dbot = 0.0;
    const int rstep = is_long ? 1 : kWarps;
    for (int r = tl.r0 + (is_long ? 0 : warp); r < tl.r1 && !skip; r += rstep) {
        double hp = 0.0, ha = 0.0;
        const int64_t kb = rp[r] + (is_long ? threadIdx.x : lane);
        const int stride = is_long ? kThreads : 32;
        for (int64_t k = kb; k < rp[r + 1]; k += stride) {
            const int32_t vm = a.mvmap[k];
            const double gx = ld(pz + a.mcol[k]);
            if (vm < pnz) hp += ld(dP + vm) * gx;
            else ha += ld(dA + (vm - pnz)) * gx;
        }
        if (is_long) {
            const Part h2 = block_sum_part(Part{hp, ha, 0.0, 0.0}, &scratch);
            hp = h2.a;
            ha = h2.b;
        } else {
            hp = warp_sum(hp);
            ha = warp_sum(ha);
        }
        if ((is_long ? threadIdx.x : lane) == 0) {
            double bval;
            if (r < n) {
                const double dq = ld(in.dq + (sy.xo - in.bx) + r), x = ld(pz + r);
                bval = -(hp + ha + dq);
                dtop += x * hp + dq * x;
            } else {
                const int j = r - n;
                const double db = ld(in.db + (sy.yo - in.by) + j);
                bval = -ha + db;
                dbot += db * ld(pz + r);
            }
            sst += bval * bval;
            if (sc) bval *= rw[r];
            U[r] = bval;
            RHS[r] = bval;
            X[r] = 0.0;
            W[r] = 0.0;
            if (a.HB) a.HB[sy.voff + r] = 0.0;
            ss += bval * bval;
        }
    }
    const Part part = block_sum_part(Part{ss, dtop, dbot, sst}, &scratch);
    Part tot;
    if (!finish_tile(a.R, tl, sy.g0, sy.g1, ti, part, &tot, &scratch)) return;
    if (threadIdx.x != 0) return;
    const double bNt = tot.b + tot.c;
    const double bN = sc ? rw[N - 1] * bNt : bNt;
    U[N - 1] = bN;
    RHS[N - 1] = bN;
    X[N - 1] = 0.0;
    W[N - 1] = 0.0;
    if (a.HB) a.HB[sy.voff + N - 1] = 0.0;
    init_state(a.state + tl.sys, a.active, sqrt(tot.a + bN * bN), sqrt(tot.d + bNt * bNt), in.rtol, in.maxiter);
}

// VJP right-hand side (Sec. 3.2): g = D phi(z)^T (wx, wy, ws)
//   = (wx, D (wy + ws) - ws, -x^T wx - y^T wy - s^T ws);
// LSQR solves min ||C G^T W r~ - b|| with b = -C g, and the G-pass of its
// first half-iteration gathers D Pi b, written here to XI.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_vjp_rhs(PlanView<T> a, RhsArgs<T> in) {
    extern __shared__ double smem[];
    __shared__ Scratch scratch;
    const int ti = a.tile0 + blockIdx.x;
    const Tile tl = a.tiles[ti];
    const Sys sy = a.sys[tl.sys];
    const Prob pr = a.probs[sy.prob];
    const int n = pr.n;
    const int N = pr.n + pr.m + 1;
    const bool skip = (tl.kind == TILE_LONG && tl.cb0 != 0);
    const int rows = skip ? 0 : tl.r1 - tl.r0;
    const int cb0 = tl.kind == TILE_STREAM ? tl.cb0 : 0, cb1 = tl.kind == TILE_STREAM ? tl.cb1 : 0;
    const double* pz = a.pz + pr.doff;
    const double* zy = a.zy + pr.doff;
    const double* cd = a.cd + pr.doff;
    const bool sc = a.scaled != 0;
    double* U = a.U + sy.voff;
    double* RHS = a.RHS + sy.voff;
    double* X = a.X + sy.voff;
    double* W = a.W + sy.voff;
    double* XI = a.XI + sy.voff;
    const TileSmem sm = tile_smem(smem, a.rmax);
    double* s0 = sm.s0;
    double* s1 = sm.s1;
    double* s2 = sm.s2;
    double dtop = 0.0, dbot = 0.0;
    for (int i = threadIdx.x; i < rows; i += kThreads) {
        const int r = tl.r0 + i;
        if (r < n) {
            const double w = ld(in.wx + (sy.xo - in.bx) + r);
            s0[i] = w;
            dtop += ld(pz + r) * w;
        } else {
            const int j = r - n;
            const double wy = ld(in.wy + (sy.yo - in.by) + j), ws = ld(in.ws + (sy.yo - in.by) + j);
            s0[i] = wy + ws;
            const double y = ld(pz + r);
            dbot += y * wy + (y - ld(zy + r)) * ws;
        }
    }
    __syncthreads();
    apply_D_tile<double>(s0, s1, tl.r0, tl.r0 + rows, n, a.flag + pr.doff, a.blocks + pr.soff, cb0, cb1, zy, 0,
                         true, a.psd, sm.psd);
    __syncthreads();
    double ss = 0.0, sst = 0.0;
    for (int i = threadIdx.x; i < rows; i += kThreads) {
        const int r = tl.r0 + i;
        double g = s1[i];
        if (r >= n) g -= ld(in.ws + (sy.yo - in.by) + (r - n));
        double bval = -g;
        sst += bval * bval;
        if (sc) bval *= cd[r];
        U[r] = bval;
        RHS[r] = bval;
        X[r] = 0.0;
        W[r] = 0.0;
        if (a.HB) a.HB[sy.voff + r] = 0.0;
        s0[i] = bval;
        ss += bval * bval;
    }
    __syncthreads();
    apply_D_tile<double>(s0, s2, tl.r0, tl.r0 + rows, n, a.flag + pr.doff, a.blocks + pr.soff, cb0, cb1, zy, 0,
                         true, a.psd, sm.psd);
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += kThreads) XI[tl.r0 + i] = s2[i];
    const Part part = block_sum_part(Part{ss, dtop, dbot, sst}, &scratch);
    Part tot;
    if (!finish_tile(a.R, tl, sy.g0, sy.g1, ti, part, &tot, &scratch)) return;
    if (threadIdx.x != 0) return;
    // The tau equation of F^T r = -g is dropped (gauge dz_N = 0, see k_pass):
    // the right-hand side lives in the x-space of the JVP, whose tau entry is 0.
    U[N - 1] = 0.0;
    RHS[N - 1] = 0.0;
    XI[N - 1] = 0.0;
    X[N - 1] = 0.0;
    W[N - 1] = 0.0;
    if (a.HB) a.HB[sy.voff + N - 1] = 0.0;
    init_state(a.state + tl.sys, a.active, sqrt(tot.a), sqrt(tot.d), in.rtol, in.maxiter);
}

// JVP output (Sec. 3.1): dz = C x, then (dx, dy, ds) = (dz_x - dz_N x,
// D dz_y - dz_N y, D dz_y - dz_y - dz_N s), s = y - z_y.  Also writes
// XI = D Pi x for the optional residual pass.
template <typename T>
struct OutArgs {
    T* o1;  // dx  | dP
    T* o2;  // dy  | dA
    T* o3;  // ds  | dq
    T* o4;  //     | db
    int64_t bx = 0, by = 0, bp = 0, ba = 0;  // user-array offsets of the first system (as RhsArgs)
    int32_t s0 = 0;                          // first system (k_vjp_out: system s0 + blockIdx.y)
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_jvp_out(PlanView<T> a, OutArgs<T> o) {
    extern __shared__ double smem[];
    const Tile tl = a.tiles[a.tile0 + blockIdx.x];
    const Sys sy = a.sys[tl.sys];
    const Prob pr = a.probs[sy.prob];
    const int n = pr.n;
    const int N = pr.n + pr.m + 1;
    const bool skip = (tl.kind == TILE_LONG && tl.cb0 != 0);
    const int rows = skip ? 0 : tl.r1 - tl.r0;
    const int cb0 = tl.kind == TILE_STREAM ? tl.cb0 : 0, cb1 = tl.kind == TILE_STREAM ? tl.cb1 : 0;
    const double* pz = a.pz + pr.doff;
    const double* zy = a.zy + pr.doff;
    const double* cd = a.cd + pr.doff;
    const bool sc = a.scaled != 0;
    const double* X = a.X + sy.voff;
    double* XI = a.XI + sy.voff;
    const TileSmem sm = tile_smem(smem, a.rmax);
    double* s0 = sm.s0;
    double* s1 = sm.s1;
    double* s2 = sm.s2;
    const double dzN = X[N - 1] * (sc ? cd[N - 1] : 1.0);
    for (int i = threadIdx.x; i < rows; i += kThreads) {
        const int r = tl.r0 + i;
        s0[i] = X[r];
        s2[i] = sc ? X[r] * cd[r] : X[r];  // dz = C x
    }
    __syncthreads();
    apply_D_tile<double>(s0, s1, tl.r0, tl.r0 + rows, n, a.flag + pr.doff, a.blocks + pr.soff, cb0, cb1, zy, 0,
                         true, a.psd, sm.psd);
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += kThreads) {
        const int r = tl.r0 + i;
        XI[r] = s1[i];
        const double cr = sc ? cd[r] : 1.0;  // D commutes with C (C is constant on SOC blocks)
        if (r < n) {
            o.o1[sy.xo - o.bx + r] = (T)(s2[i] - dzN * ld(pz + r));
        } else {
            const int j = r - n;
            const double y = ld(pz + r);
            const double s = y - ld(zy + r);
            const double Ddz = cr * s1[i];
            o.o2[sy.yo - o.by + j] = (T)(Ddz - dzN * y);
            o.o3[sy.yo - o.by + j] = (T)(Ddz - s2[i] - dzN * s);
        }
    }
}

// VJP output (Sec. 3.2, computed only on the stored patterns): with
// r = S W x = (r1, r2, r_N) = (w_x X_x, -w_y X_y, w_N X_N),
//   dP_ij = (r1_i x_j + x_i r1_j)/2 - r_N x_i x_j   on P's upper pattern
//   dA_ij = y_i r1_j - r2_i x_j                       on A's pattern
//   dq = r1 - r_N x,  db = r2 - r_N y.
// One warp per (system, row); blockIdx.y selects the system.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_vjp_out(PlanView<T> a, OutArgs<T> o, const int64_t* pip,
                                                     const int32_t* pix, const int64_t* aip,
                                                     const int32_t* aix) {
    const Sys sy = a.sys[o.s0 + blockIdx.y];
    const Prob pr = a.probs[sy.prob];
    const int n = pr.n, m = pr.m;
    const int N = n + m + 1;
    const double* pz = a.pz + pr.doff;
    const double* X = a.X + sy.voff;
    const double* rw = a.rw + pr.doff;
    const bool sc = a.scaled != 0;
    const double rN = X[N - 1] * (sc ? rw[N - 1] : 1.0);
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int nw = (gridDim.x * kThreads) >> 5;
    const int64_t* pp = pip + pr.prow;
    const int64_t* ap = aip + pr.arow;
    const int32_t* px = pix + pr.poff;
    const int32_t* ax = aix + pr.aoff;
    for (int row = gw; row < n + m; row += nw) {
        if (row < n) {
            const int i = row;
            const double xi = ld(pz + i), r1i = X[i] * (sc ? rw[i] : 1.0);
            for (int64_t k = pp[i] + lane; k < pp[i + 1]; k += 32) {
                const int j = px[k];
                const double xj = ld(pz + j), r1j = X[j] * (sc ? rw[j] : 1.0);
                o.o1[sy.po - o.bp + k] = (T)(0.5 * (r1i * xj + xi * r1j) - rN * xi * xj);
            }
            if (lane == 0) o.o3[sy.xo - o.bx + i] = (T)(r1i - rN * xi);
        } else {
            const int i = row - n;
            const double yi = ld(pz + n + i), r2i = -X[n + i] * (sc ? rw[n + i] : 1.0);
            for (int64_t k = ap[i] + lane; k < ap[i + 1]; k += 32) {
                const int j = ax[k];
                const double r1j = X[j] * (sc ? rw[j] : 1.0);
                o.o2[sy.ao - o.ba + k] = (T)(yi * r1j - r2i * ld(pz + j));
            }
            if (lane == 0) o.o4[sy.yo - o.by + i] = (T)(r2i - rN * yi);
        }
    }
}

}  // namespace qcpd
