// Double-float form of the cluster engine's kernel (see qcpd_cluster.cuh for
// the pass structure and qcpd_df64.cuh for the arithmetic).
//
// Every per-pass operation on vectors (row sums, epilogue, D Pi, block
// sums) runs in df64 on the FP32 pipes; the LSQR scalar recurrences (one
// lane per pass) stay in FP64.
//
// The vector a pass produces for the next one travels through L2, not
// shared memory: each CTA stores its slice in the system's broadcast buffer
// (gather-buffer layout, two buffers alternating by pass parity) and, after
// the cluster barrier, every CTA reads the whole buffer with coalesced
// loads.  The SM-to-SM network moves only about 10 bytes per cycle per SM,
// several times less than an SM reads from L2.  Warps 1.. do that copy and
// the row sums while warp 0 finishes the previous pass.
//
// The Krylov vectors live as df64 pairs: u, v, xi in shared memory, w and x
// in the plan's FP64 arrays reinterpreted as pairs for the kernel's lifetime
// (each CTA touches only its own rows).
// Matrix values, per-row data and second-order-cone constants come as df64
// copies made at plan time.
//
// Magnitudes: the right-hand side of each system is scaled by a power of two
// to norm in [1/2, 1) for the kernel's lifetime (exact; LSQR's iterates and
// scalars are homogeneous in it), so the vectors stay near unit scale; the
// plan falls back to the FP64 kernel when the data leave about 2^-90..2^90.
#pragma once

#include "qcpd_cluster.cuh"
#include "qcpd_df64.cuh"

namespace qcpd {

// df64 constants of one second-order-cone block in the formula case:
// r = ||u||, h = 1/(2r), tq = t/r^2, htr = h (t + r).
struct SocDf {
    df r, h, tq, htr;
};

struct ClusterDfArgs {
    df* bcast;        // per cluster of the launch (at cluster * 2 bhalf): two broadcast buffers
    int64_t bhalf;    // df entries per buffer (gather-buffer layout, even)
    const df* sval;   // SELL-32 values of M, M diag(c), M diag(w) per slot
    const df* svalG;
    const df* svalT;
    const df* cA;     // N-indexed (plan-wide offsets) per-row data: coefA, coefB, rw, cd, z_y
    const df* cB;
    const df* rw;
    const df* cd;
    const df* zy;
    const SocDf* soc;  // per SOC block (plan-wide indices)
    const df* dense;        // the exponential, power and PSD blocks' dense D Pi (row-major; null: none)
    const int64_t* doff;    // per coupled block (plan-wide): its offset in dense, -1 for SOC blocks
};

// This pass's scalars: FP64 for the finisher, df64 for the vector work.
struct PassScal {
    double c1, c2, tin, tout, tt, wcoef, xcoef, hcoef;
    df dc1, dnc2, dnw, dxc, dtt, dnhc;  // c1, -c2, -wcoef, xcoef, tt, -hcoef (LSMR)
    int upd;                            // LSMR: this u-pass applies the deferred (hbar, x, h) updates
};

struct CCtxDf {
    const ClusterProb* cp;
    LsqrState* st;
    PassScal* ps;
    double* tau;
    df* scr;
    df *F, *U, *V, *XI, *s0, *s1, *s2, *ZY, *red;
    const SellSlice* slices;
    const int32_t* perm;
    const int32_t* scol;
    const df* valG;
    const df* valT;
    const df *cA, *cB, *rw, *cd;  // problem-relative
    const double *rwd, *cdd;     // FP64 per-row scalings (tau entries)
    const int8_t* flag;
    const SocBlock* blocks;
    const SocDf* soc;
    const df* dense;  // the stored dense D Pi (offsets in bs[].w)
    df* W;  // the plan's w and x rows of this system, as df64 pairs
    df* X;
    df* HB;  // LSMR: hbar (W holds h), as df64 pairs
    df* B;  // the system's broadcast buffers (bhalf entries each)
    int64_t bhalf;
    bool any_large;
    int* active;
    double kappa;
    int n, N, R0, L, C, rank, cb0, cb1, sl0, sl1;
    // this CTA's SOC-block tables (shared memory): per local row its block
    // (RB_ONE / RB_ZERO off blocks), per block (local start, dim, kase) and
    // its derivative constants, and the dot products of one D Pi application
    int* rowblk;
    int4* bs;
    SocDf* bsdf;
    df* dotv;
};

constexpr int RB_ONE = -1;   // D Pi = 1 on the row (x-rows, zero-cone rows, R+ rows with z > 0)
constexpr int RB_ZERO = -2;  // D Pi = 0 on the row

// D Pi_{K*} in df64 on this CTA's rows, with the same arithmetic as the
// block-by-block form: first every SOC block's u^T c (one thread per block,
// one warp per block of more than kSocThread entries), then every row in
// parallel.  src and dst are indexed by local row; the CTA synchronises once.
__device__ __forceinline__ void apply_D_rows_df(const CCtxDf& c, const df* src, df* dst) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nb = c.cb1 - c.cb0;
    const df* zy = c.ZY;
    for (int j = tid; j < nb; j += nt) {
        const int4 B = c.bs[j];
        if (B.z != 2 || B.y > kSocThread) continue;
        DfAcc d = dfacc_zero();
        for (int k = 1; k < B.y; ++k) dfacc_fma(d, zy[B.x + k], src[B.x + k]);
        c.dotv[j] = dfacc_result(d);
    }
    if (c.any_large) {
        const int lane = tid & 31, warp = tid >> 5;
        for (int j = warp; j < nb; j += nt >> 5) {
            const int4 B = c.bs[j];
            if (B.z != 2 || B.y <= kSocThread) continue;
            DfAcc d = dfacc_zero();
            for (int k = 1 + lane; k < B.y; k += 32) dfacc_fma(d, zy[B.x + k], src[B.x + k]);
            const df dot = warp_sum_df(dfacc_result(d));
            if (lane == 0) c.dotv[j] = dot;
        }
    }
    __syncthreads();
    for (int i = tid; i < c.L; i += nt) {
        const int rb = c.rowblk[i];
        if (rb == RB_ONE) {
            dst[i] = src[i];
        } else if (rb == RB_ZERO) {
            dst[i] = df_zero();
        } else {
            const int4 B = c.bs[rb];
            if (B.w >= 0) {  // exponential, power or PSD block: its stored dense D Pi, in j order
                const df* D = c.dense + B.w + (int64_t)(i - B.x) * B.y;
                df acc = df_zero();
                for (int j = 0; j < B.y; ++j) acc = df_fma(__ldg(reinterpret_cast<const float2*>(D + j)), src[B.x + j], acc);
                dst[i] = acc;
            } else if (B.z == 0) {
                dst[i] = df_zero();
            } else if (B.z == 1) {
                dst[i] = src[i];
            } else {
                const SocDf S = c.bsdf[rb];
                const df dot = c.dotv[rb];
                const df ct = src[B.x];
                if (i == B.x) {
                    dst[i] = df_mul(S.h, df_fma(S.r, ct, dot));
                } else {
                    const df a = df_mul(S.h, df_fma(df_neg(S.tq), dot, ct));
                    dst[i] = df_fma(a, zy[i], df_mul(S.htr, src[i]));
                }
            }
        }
    }
}

// Block sums of three df64 values (fixed order), returned in every thread.
__device__ __forceinline__ void block_reduce_df3(df (&v)[3], df* red) {
    constexpr int NT = kCThreads;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 3; ++j) red[j * NT + tid] = v[j];
    __syncthreads();
#pragma unroll
    for (int w = NT / 2; w >= 32; w >>= 1) {
        if (tid < w) {
#pragma unroll
            for (int j = 0; j < 3; ++j) red[j * NT + tid] = df_add(red[j * NT + tid], red[j * NT + tid + w]);
        }
        __syncthreads();
    }
    if (warp < 3) {
        const df s = warp_sum_df(red[warp * NT + lane]);
        __syncwarp();
        if (lane == 0) red[warp * NT] = s;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 3; ++j) v[j] = red[j * NT];
    __syncthreads();
}

// Row sums by warps 1.. (the SELL-32 walk of sell_rowsums, one TwoProduct
// and one TwoSum per entry).
__device__ __forceinline__ void sell_rowsums_df(const CCtxDf& c, const df* sval, const df* F, df* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nw = kCWarps - 1;
    // Each step below waits one L2 round trip, so the loop keeps as many
    // loads in flight as it can: the next slice's header is fetched while
    // this slice runs, and the entries go eight at a time.
    int s = c.sl0 + warp - 1;
    SellSlice d{};
    if (s < c.sl1) d = c.slices[s];
    for (; s < c.sl1; s += nw) {
        SellSlice dn{};
        if (s + nw < c.sl1) dn = c.slices[s + nw];
        const int32_t* cp = c.scol + d.base + lane;
        const df* vp = sval + d.base + lane;
        DfAcc acc = dfacc_zero();
        int k = 0;
        for (; k + 8 <= d.width; k += 8) {
            int32_t j[8];
            df v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                j[u] = __ldg(cp + 32 * (k + u));
                v[u] = __ldg(vp + 32 * (k + u));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) dfacc_fma(acc, v[u], F[j[u]]);
        }
        if (k < d.width) {  // the last 1..7 entries in one round trip (a zero product leaves acc as it is)
            int32_t j[8];
            df v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool in = k + u < d.width;
                j[u] = in ? __ldg(cp + 32 * (k + u)) : 0;
                v[u] = in ? __ldg(vp + 32 * (k + u)) : df_zero();
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (k + u < d.width) dfacc_fma(acc, v[u], F[j[u]]);
        }
        df r = dfacc_result(acc);
        if (d.row >= 0) {
            r = warp_sum_df(r);
            if (lane == 0) out[d.row] = r;
        } else {
            const int row = c.perm[d.pidx + lane];
            if (row >= 0) out[row] = r;
        }
        d = dn;
    }
}

// Lane 0 of warp 0: this pass's scalars from the state and tau entries.
template <int PASS, int ROLE, bool SC, bool LS>
__device__ __forceinline__ void prep_scalars_df(const CCtxDf& c) {
    const LsqrState& st = *c.st;
    PassScal p;
    p.c1 = (ROLE == ROLE_U) ? st.uc1 : st.vc1;
    p.c2 = (ROLE == ROLE_U) ? st.uc2 : st.vc2;
    p.tin = c.tau[ROLE == ROLE_U ? TAU_V : TAU_U];
    p.tout = c.tau[ROLE == ROLE_U ? TAU_U : TAU_V];
    p.tt = SC ? (PASS == PASS_G ? c.cdd[c.N - 1] : c.rwd[c.N - 1]) * p.tin : p.tin;
    p.wcoef = st.wcoef;
    p.xcoef = st.xcoef;
    p.dc1 = df_from(p.c1);
    p.dnc2 = df_from(-p.c2);
    p.dnw = df_from(-p.wcoef);
    p.dxc = df_from(p.xcoef);
    p.dtt = df_from(p.tt);
    p.hcoef = LS ? st.hcoef : 0.0;
    p.dnhc = df_from(-p.hcoef);
    p.upd = LS && ROLE == ROLE_U ? st.upd : 0;
    *c.ps = p;
}

// LSMR's deferred updates of the tau entries (run_tile's lsmr_update):
// hbar <- h - hcoef hbar, x <- x + xcoef hbar, h <- v / alpha - wcoef h.
__device__ __forceinline__ void lsmr_tau_update(const CCtxDf& c, const PassScal& pd) {
    const double h = c.tau[TAU_W];
    const double hb = fma(-pd.hcoef, c.tau[TAU_HB], h);
    c.tau[TAU_HB] = hb;
    c.tau[TAU_X] = fma(pd.xcoef, hb, c.tau[TAU_X]);
    c.tau[TAU_W] = fma(pd.tin, pd.c1, -pd.wcoef * h);
}

// LSMR's deferred updates of row r (the df64 form of lsmr_update).
__device__ __forceinline__ void lsmr_row_update(const CCtxDf& c, int r, df iv, const PassScal& ps) {
    const df h = c.W[r];
    const df hb = df_fma(ps.dnhc, c.HB[r], h);
    c.HB[r] = hb;
    c.X[r] = df_fma(ps.dxc, hb, c.X[r]);
    c.W[r] = df_fma(iv, ps.dc1, df_mul(ps.dnw, h));
}

// The end of the previous pass (kind PASS, ROLE) by warp 0, as in
// cluster_finish, with the sums converted to FP64 once.
template <int PASS, int ROLE, bool SC, bool LS>
__device__ __forceinline__ void cluster_finish_df(const CCtxDf& c, const int par) {
    cg::cluster_group cl = cg::this_cluster();
    const int lane = threadIdx.x & 31;
    df ta = df_zero(), tb = df_zero(), tc = df_zero();
    if (lane < c.C) {
        const df* rr = cl.map_shared_rank(c.red + 4 * par, lane);
        ta = rr[0];
        tb = rr[1];
        tc = rr[2];
    }
    for (int o = 1; o < c.C; o <<= 1) {  // the same butterfly in every CTA
        df x;
        x.x = __shfl_xor_sync(0xffffffffu, ta.x, o);
        x.y = __shfl_xor_sync(0xffffffffu, ta.y, o);
        ta = df_add(ta, x);
        x.x = __shfl_xor_sync(0xffffffffu, tb.x, o);
        x.y = __shfl_xor_sync(0xffffffffu, tb.y, o);
        tb = df_add(tb, x);
        x.x = __shfl_xor_sync(0xffffffffu, tc.x, o);
        x.y = __shfl_xor_sync(0xffffffffu, tc.y, o);
        tc = df_add(tc, x);
    }
    if (lane != 0) return;
    const PassScal pd = *c.ps;
    LsqrState& st = *c.st;
    const int rN = c.N - 1;
    const double sa = df_to(ta), sb = df_to(tb), sc = df_to(tc);
    double oN;
    if (PASS == PASS_G) {
        oN = -sb - sc + c.kappa * pd.tt;
        if (SC) oN *= c.rwd[rN];
    } else {
        oN = sb - sc + c.kappa * pd.tt;
        if (SC) oN *= c.cdd[rN];
    }
    const double nvN = (PASS == PASS_GT) ? 0.0 : pd.c1 * oN - pd.c2 * pd.tout;
    c.tau[ROLE == ROLE_U ? TAU_U : TAU_V] = nvN;
    if (PASS == PASS_GT) c.tau[TAU_XI] = 0.0;
    const double nsq = fma(nvN, nvN, sa);
    double nrm, inv_nrm;
    norm_and_inverse(nsq, nrm, inv_nrm);
    if (LS) {  // LSMR (Fong & Saunders 2011): the pass engine's recurrences
        if (ROLE == ROLE_U) {
            if (pd.upd) lsmr_tau_update(c, pd);
            if (lsmr_step_u(&st, nrm, inv_nrm) && c.rank == 0) atomicSub(c.active, 1);
        } else {
            if (lsmr_step_v(&st, nrm, inv_nrm) && c.rank == 0) atomicSub(c.active, 1);
        }
    } else if (ROLE == ROLE_U) {
        c.tau[TAU_W] = pd.tin * pd.c1 - pd.wcoef * c.tau[TAU_W];
        lsqr_step_u(&st, nrm, inv_nrm, nsq);
    } else {
        c.tau[TAU_X] = fma(pd.xcoef, c.tau[TAU_W], c.tau[TAU_X]);
        if (lsqr_step_v(&st, nrm, inv_nrm) && c.rank == 0) atomicSub(c.active, 1);
    }
}

template <int PASS, int ROLE, bool SC, bool LS>
__device__ __forceinline__ bool cluster_pass_df(const CCtxDf& c, const int par, const bool pending) {
    constexpr int PPASS = (PASS == PASS_G) ? PASS_GT : PASS_G;
    constexpr int PROLE = (ROLE == ROLE_U) ? ROLE_V : ROLE_U;
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x;
    df* s0 = c.s0;
    if (tid < 32) {
        if (pending) cluster_finish_df<PPASS, PROLE, SC, LS>(c, par ^ 1);
        if (tid == 0) prep_scalars_df<PASS, ROLE, SC, LS>(c);
    } else {
        if (pending) {
            // the previous pass's vector, from its broadcast buffer (L2)
            const float4* src = reinterpret_cast<const float4*>(c.B + (par ^ 1) * c.bhalf);
            float4* dst = reinterpret_cast<float4*>(c.F);
            const int npairs = c.cp->FN >> 1;
            constexpr int kU = 4, nth = kCThreads - 32;
            for (int k0 = tid - 32; k0 < npairs; k0 += kU * nth) {
                float4 v[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int k = k0 + u * nth;
                    if (k < npairs) v[u] = __ldcg(src + k);
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int k = k0 + u * nth;
                    if (k < npairs) dst[k] = v[u];
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kCThreads - 32) : "memory");
        }
        sell_rowsums_df(c, PASS == PASS_G ? c.valG : c.valT, c.F, s0);
    }
    __syncthreads();

    LsqrState& st = *c.st;
    const int status = st.status;
    if (status == S_DONE) return true;
    const PassScal ps = *c.ps;
    // a stopped system's last deferred update: LSQR's x-update in its
    // v-pass, LSMR's (hbar, x, h) updates in its u-pass
    if (status == S_FINAL && (ROLE == ROLE_V) == !LS) {
        const df* vin = (ROLE == ROLE_U) ? c.V : c.U;
        for (int i = tid; i < c.L; i += kCThreads) {
            const int r = c.R0 + i;
            if (!LS) c.X[r] = df_fma(ps.dxc, c.W[r], c.X[r]);
            else lsmr_row_update(c, r, vin[i], ps);
        }
        __syncthreads();
        if (tid == 0) {
            if (!LS) {
                c.tau[TAU_X] = fma(ps.xcoef, c.tau[TAU_W], c.tau[TAU_X]);
            } else {
                lsmr_tau_update(c, ps);
                st.upd = 0;  // applied: a continuation starts with a plain u-pass
            }
            st.status = S_DONE;
            if (c.rank == 0) atomicSub(c.active, 1);
        }
        __syncthreads();
        return true;
    }
    const df c1 = ps.dc1, nc2 = ps.dnc2, nw = ps.dnw, xc = ps.dxc, tt = ps.dtt;
    df* in_s = (ROLE == ROLE_U) ? c.V : c.U;
    df* out_s = (ROLE == ROLE_U) ? c.U : c.V;
    const int L = c.L, R0 = c.R0, n = c.n;
    df* s1 = c.s1;
    df* s2 = c.s2;
    df* XIs = c.XI;
    df* bout = c.B + par * c.bhalf + c.cp->poff[c.rank];  // this CTA's slice of this pass's broadcast

    DfAcc ss = dfacc_zero(), dtop = dfacc_zero(), dbot = dfacc_zero();
    if (PASS == PASS_G) {
        // row i's per-row constants and w / x (from L2), then its update
        struct RowIn {
            df a, b, cd, rw, w, x;
        };
        auto load = [&](int i) {
            const int r = R0 + i;
            RowIn v;
            v.a = c.cA[r];
            v.b = c.cB[r];
            v.cd = SC ? c.cd[r] : df_zero();
            v.rw = SC ? c.rw[r] : df_zero();
            v.w = c.W[r];
            v.x = ROLE == ROLE_V && !LS ? c.X[r] : df_zero();
            return v;
        };
        auto row = [&](int i, const RowIn& v) {
            const int r = R0 + i;
            const df iv = in_s[i];
            df o;
            if (r < n) {
                o = df_fma(v.a, tt, s0[i]);
                dfacc_fma(dtop, v.b, SC ? df_mul(v.cd, iv) : iv);
            } else {
                const df xi = XIs[i];
                const df dxi = SC ? df_mul(v.cd, df_sub(xi, iv)) : df_sub(xi, iv);
                o = df_add(df_fma(df_neg(v.a), tt, s0[i]), dxi);
                dfacc_fma(dbot, v.b, SC ? df_mul(v.cd, xi) : xi);
            }
            if (SC) o = df_mul(o, v.rw);
            const df nv = df_fma(c1, o, df_mul(nc2, out_s[i]));
            out_s[i] = nv;
            bout[i] = nv;
            dfacc_fma(ss, nv, nv);
            if (ROLE == ROLE_U) {
                if (!LS) c.W[r] = df_fma(iv, c1, df_mul(nw, v.w));
                else if (ps.upd) lsmr_row_update(c, r, iv, ps);
            } else if (!LS) {
                c.X[r] = df_fma(xc, v.w, v.x);
            }
        };
        for (int i = tid; i < L; i += kCThreads) row(i, load(i));
    } else {
        for (int i = tid; i < L; i += kCThreads) {
            const int r = R0 + i;
            const df iv = SC ? df_mul(c.rw[r], in_s[i]) : in_s[i];
            const df h = df_fma(df_neg(c.cB[r]), tt, s0[i]);
            if (r < n) {
                s1[i] = h;
                dfacc_fma(dtop, c.cA[r], iv);
            } else {
                s1[i] = df_add(h, iv);
                dfacc_fma(dbot, c.cA[r], iv);
            }
        }
        __syncthreads();
        apply_D_rows_df(c, s1, s2);
        __syncthreads();
        for (int i = tid; i < L; i += kCThreads) {
            const int r = R0 + i;
            const df iv = in_s[i];
            df o = (r < n) ? s2[i] : df_sub(s2[i], SC ? df_mul(c.rw[r], iv) : iv);
            if (SC) o = df_mul(o, c.cd[r]);
            const df nv = df_fma(c1, o, df_mul(nc2, out_s[i]));
            out_s[i] = nv;
            s1[i] = nv;
            dfacc_fma(ss, nv, nv);
            if (ROLE == ROLE_U) {
                if (!LS) c.W[r] = df_fma(iv, c1, df_mul(nw, c.W[r]));
                else if (ps.upd) lsmr_row_update(c, r, iv, ps);
            } else if (!LS) {
                c.X[r] = df_fma(xc, c.W[r], c.X[r]);
            }
        }
        __syncthreads();
        apply_D_rows_df(c, s1, s2);
        __syncthreads();
        for (int i = tid; i < L; i += kCThreads) {
            XIs[i] = s2[i];
            bout[i] = s2[i];
        }
    }
    df v3[3] = {dfacc_result(ss), dfacc_result(dtop), dfacc_result(dbot)};
    block_reduce_df3(v3, c.scr);
    if (tid == 0) {
        c.red[4 * par + 0] = v3[0];
        c.red[4 * par + 1] = v3[1];
        c.red[4 * par + 2] = v3[2];
    }
    cl.sync();
    return false;
}

template <int MODE, bool SC, typename T, bool LS = false>
__global__ void __launch_bounds__(kCThreads, 1) k_cluster_df(PlanView<T> a, ClusterArgs ca, ClusterDfArgs da) {
    extern __shared__ __align__(16) double csm[];
    __shared__ df scr[3 * kCThreads];
    __shared__ LsqrState st;
    __shared__ PassScal ps;
    __shared__ double tau[6];
    __shared__ ClusterProb cp;
    __shared__ double s_scale;
    __shared__ int s_uscaled;
    constexpr int PU = MODE == 0 ? PASS_G : PASS_GT;
    constexpr int PV = MODE == 0 ? PASS_GT : PASS_G;
    cg::cluster_group cl = cg::this_cluster();
    const int C = ca.C;
    const int rank = (int)cl.block_rank();
    const int si = ca.sys_list[blockIdx.x / C];
    const Sys sy = a.sys[si];
    const Prob pr = a.probs[sy.prob];
    const int tid = threadIdx.x;
    const int N = pr.n + pr.m + 1, rN = N - 1;
    double* gU = a.U + sy.voff;
    double* gV = a.V + sy.voff;
    double* gXI = a.XI + sy.voff;
    double* gW = a.W + sy.voff;
    double* gX = a.X + sy.voff;
    if (tid == 0) {
        cp = ca.cprob[sy.prob];
        st = a.state[si];
        tau[TAU_U] = gU[rN];
        tau[TAU_V] = gV[rN];
        tau[TAU_W] = gW[rN];
        tau[TAU_X] = gX[rN];
        tau[TAU_XI] = gXI[rN];
        tau[TAU_HB] = LS ? a.HB[sy.voff + rN] : 0.0;
        // scale the right-hand side to norm in [1/2, 1) by a power of two:
        // x, phibar, xcoef and bnorm are proportional to it, and so are u,
        // beta and 1/uc2 before the first u-update (LSMR: no scaling, its
        // recurrences carry many quantities proportional to ||b||)
        double s = 1.0;
        if (!LS && st.bnorm > 0.0 && finite64(st.bnorm)) {
            int e = 0;
            frexp(st.bnorm, &e);
            s = ldexp(1.0, -e);
        }
        s_scale = s;
        s_uscaled = st.iters == 0;
        st.phibar *= s;
        st.xcoef *= s;
        st.bnorm *= s;
        tau[TAU_X] *= s;
        if (s_uscaled) {
            st.beta *= s;
            st.uc2 /= s;
            tau[TAU_U] *= s;
        }
    }
    __syncthreads();
    const double sc = s_scale;
    const double su = s_uscaled ? sc : 1.0;
    CCtxDf c;
    {
        const CSmem m = cluster_smem(csm, cp.FN, cp.L);  // the problem's own layout
        c.F = reinterpret_cast<df*>(m.F);
        c.U = reinterpret_cast<df*>(m.U);
        c.V = reinterpret_cast<df*>(m.V);
        c.XI = reinterpret_cast<df*>(m.XI);
        c.s0 = reinterpret_cast<df*>(m.s0);
        c.s1 = reinterpret_cast<df*>(m.s1);
        c.s2 = reinterpret_cast<df*>(m.s2);
        c.ZY = reinterpret_cast<df*>(m.ZY);
        c.red = reinterpret_cast<df*>(m.red);
    }
    c.cp = &cp;
    c.st = &st;
    c.ps = &ps;
    c.tau = tau;
    c.scr = scr;
    c.slices = ca.slices;
    c.perm = ca.perm;
    c.scol = ca.scol;
    c.valG = a.scaled ? da.svalG : da.sval;
    c.valT = a.scaled ? da.svalT : da.sval;
    c.cA = da.cA + pr.doff;
    c.cB = da.cB + pr.doff;
    c.rw = da.rw + pr.doff;
    c.cd = da.cd + pr.doff;
    c.rwd = a.rw + pr.doff;
    c.cdd = a.cd + pr.doff;
    c.flag = a.flag + pr.doff;
    c.blocks = a.blocks + pr.soff;
    c.soc = da.soc + pr.soff;
    c.dense = da.dense;
    c.W = reinterpret_cast<df*>(gW);
    c.X = reinterpret_cast<df*>(gX);
    c.HB = reinterpret_cast<df*>(a.HB + sy.voff);
    c.B = da.bcast + (int64_t)(blockIdx.x / C) * 2 * da.bhalf;
    c.bhalf = da.bhalf;
    c.any_large = cp.nlarge[rank] > 0;
    c.active = a.active;
    c.kappa = pr.kappa;
    c.n = pr.n;
    c.N = N;
    c.R0 = cp.split[rank];
    c.L = cp.split[rank + 1] - c.R0;
    c.C = C;
    c.rank = rank;
    c.cb0 = cp.cb[rank];
    c.cb1 = cp.cb[rank + 1];
    c.sl0 = cp.sl[rank];
    c.sl1 = cp.sl[rank + 1];
    {
        unsigned char* t = reinterpret_cast<unsigned char*>(csm) + cluster_smem_bytes(cp.FN, cp.L);
        const size_t rows = ((4 * (size_t)even_up(cp.L)) + 15) & ~(size_t)15;
        c.rowblk = reinterpret_cast<int*>(t);
        c.bs = reinterpret_cast<int4*>(t + rows);
        c.bsdf = reinterpret_cast<SocDf*>(t + rows + 16 * (size_t)cp.nb);
        c.dotv = reinterpret_cast<df*>(t + rows + 48 * (size_t)cp.nb);
    }

    const bool live = st.status != S_DONE;
    if (live) {
        const df* zyd = da.zy + pr.doff;
        for (int i = tid; i < c.L; i += kCThreads) {
            const int r = c.R0 + i;
            c.U[i] = df_from(gU[r] * su);
            c.V[i] = df_from(gV[r]);
            c.XI[i] = df_from(gXI[r]);
            c.ZY[i] = zyd[r];
            // w and x become df64 pairs in place (same 8 bytes per entry)
            const double w = gW[r], x = gX[r] * sc;
            c.W[r] = df_from(w);
            c.X[r] = df_from(x);
            if (LS) c.HB[r] = df_from(a.HB[sy.voff + r]);
            const int8_t f = c.flag[r];
            c.rowblk[i] = (r < c.n || f == RF_ONE) ? RB_ONE : (f == RF_SOC ? 0 : RB_ZERO);
        }
        for (int j = tid; j < c.cb1 - c.cb0; j += kCThreads) {
            const SocBlock B = c.blocks[c.cb0 + j];
            c.bs[j] = make_int4(B.start - c.R0, B.dim, B.kase, da.doff ? (int)da.doff[pr.soff + c.cb0 + j] : -1);
            c.bsdf[j] = c.soc[c.cb0 + j];
        }
        __syncthreads();
        for (int j = tid; j < c.cb1 - c.cb0; j += kCThreads) {  // the rows of each block (inside this CTA's rows)
            const int4 B = c.bs[j];
            for (int k = 0; k < B.y; ++k) c.rowblk[B.x + k] = j;
        }
        // the first u-update gathers xi (JVP) or v (VJP); slot FN stays 0 for padding
        const double* g0 = (MODE == 0) ? gXI : gV;
        for (int r = 0; r < C; ++r) {
            const int r0 = cp.split[r], len = cp.split[r + 1] - r0;
            df* dst = c.F + cp.poff[r];
            for (int i = tid; i < len; i += kCThreads) dst[i] = df_from(g0[r0 + i]);
        }
        if (tid == 0) c.F[cp.FN] = df_zero();
    }
    __syncthreads();
    cl.sync();  // every CTA of the cluster runs before any remote access
    if (live) {
        int par = 0;
        bool pending = false;
        for (int64_t pass = 0; pass < ca.max_passes; pass += 2) {
            if (cluster_pass_df<PU, ROLE_U, SC, LS>(c, par, pending)) break;
            pending = true;
            par ^= 1;
            if (cluster_pass_df<PV, ROLE_V, SC, LS>(c, par, true)) break;
            par ^= 1;
        }
        // undo the scaling; back to FP64
        const bool u_still = s_uscaled && st.iters == 0;
        const double iu = u_still ? 1.0 / sc : 1.0, ix = 1.0 / sc;
        for (int i = tid; i < c.L; i += kCThreads) {
            const int r = c.R0 + i;
            gU[r] = df_to(c.U[i]) * iu;
            gV[r] = df_to(c.V[i]);
            gXI[r] = df_to(c.XI[i]);
            const double w = df_to(c.W[r]), x = df_to(c.X[r]) * ix;
            gW[r] = w;
            gX[r] = x;
            if (LS) a.HB[sy.voff + r] = df_to(c.HB[r]);
        }
        if (tid == 0 && rank == 0) {
            st.phibar *= ix;
            st.xcoef *= ix;
            st.bnorm *= ix;
            if (u_still) {
                st.beta *= iu;
                st.uc2 /= iu;
            }
            gU[rN] = tau[TAU_U] * iu;
            gV[rN] = tau[TAU_V];
            gW[rN] = tau[TAU_W];
            gX[rN] = tau[TAU_X] * ix;
            gXI[rN] = tau[TAU_XI];
            if (LS) a.HB[sy.voff + rN] = tau[TAU_HB];
            a.state[si] = st;
        }
    }
    cl.sync();  // no CTA leaves while a peer may still read its shared memory
}

}  // namespace qcpd
