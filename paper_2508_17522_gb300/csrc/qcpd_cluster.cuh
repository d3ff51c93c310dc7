// Cluster form of the Krylov loop (QCP_ENGINE_CLUSTER).
//
// One thread-block cluster of C CTAs runs every LSQR iteration of one system
// (a problem and one direction) in a single launch.  CTA r owns a contiguous
// range of the embedding's rows (cut at second-order-cone block boundaries,
// balanced by stored entries) and keeps its slices of u, v and xi = D Pi(.)
// in shared memory; w and x stay in global memory, touched only by their
// owner.  A pass (one product with Op or Op^T, Sec. 3.1-3.2 through
// G = S F, see qcpd_common.cuh) is
//   1. row sums of the CTA's rows of M against the gather buffer F, a local
//      copy of the whole vector the pass multiplies, from a SELL-32 copy of
//      the rows (warps 1..), while warp 0 finishes the previous pass: it adds
//      the C partial sums that pass left in the CTAs' slots (rank order) and
//      runs the LSQR scalar recurrences, which nothing in the row sums needs;
//   2. the epilogue of the tile kernels on the CTA's own rows, with the new
//      scalars;
//   3. a block reduction of the pass's three sums into the CTA's slot;
//   4. one hardware cluster barrier (release/acquire);
//   5. every CTA copies the freshly written slices of the next pass's vector
//      from all CTAs' shared memory into its F.
// Every CTA of a cluster computes the same scalars from the same inputs in
// the same order, so all of them take the same decisions and arrive at the
// same barriers; no CTA waits on a flag, and clusters of different systems
// never wait on one another.
//
// FP64 cost model (this GPU issues FP64 at 1/64 of the FP32 rate and a
// warp-wide FP64 instruction costs the same however many lanes it has):
// SELL-32 gives one fully populated FMA instruction per 32 stored entries
// (plus padding) and no cross-lane reduction; rows longer than kSellLong get
// a warp each (lane-strided, one warp sum).
//
// Safety of the shared-memory copies: a slice read by peers in pass k is
// next rewritten in pass k + 2, after the barrier of pass k + 1, which every
// CTA reaches only once its copies of pass k are done; the partial-sum slots
// alternate between two buffers, and a slot of pass k is read (by the
// finishing warp during pass k + 1) before its owner can pass barrier k + 1.
#pragma once

#include <cooperative_groups.h>

#include "qcpd_kernels.cuh"

namespace qcpd {

namespace cg = cooperative_groups;

constexpr int kCThreads = 512;  // threads per CTA of the cluster kernel
constexpr int kCWarps = kCThreads / 32;
constexpr int kSellLong = 256;  // rows longer than this get a warp each

// One slice of the SELL-32 copy of M: entry k of lane l's row at
// base + 32 k + l, for k < width (zero-valued padding past a row's end).
// row >= 0: a single long row stored lane-strided (entry j at base + j);
// row < 0: 32 rows, lane l's local row at perm[pidx + l] (-1: none).
// A slice of the SELL-32 copy of M: 32 lanes x width slots from base (slot
// base + 32 k + lane).  row >= 0: one long row, lane-strided; row < 0: the
// 32 rows perm[pidx ..], one per lane.
struct SellSlice {
    int64_t base;
    int32_t width;
    int32_t row;
    int32_t pidx;
    int32_t pad;
};

struct ClusterArgs {
    const ClusterProb* cprob;  // per problem
    const SellSlice* slices;   // CTA r of a problem owns slices [sl[r], sl[r+1])
    const int32_t* perm;
    const int32_t* scol;       // gather-buffer index of every slot (cp.FN for padding)
    const void* sval;          // T values of M, M diag(c), M diag(w) per slot
    const void* svalG;
    const void* svalT;
    const int32_t* sys_list;   // the launch's systems, one cluster each
    int C;                     // CTAs per cluster
    int FN;                    // largest gather buffer of the launch's problems
    int L;                     // most rows of one CTA over the launch's problems
    int NB;                    // most SOC blocks of one CTA over the launch's problems
    int64_t max_passes;        // termination bound (the scalars stop it earlier)
};

__host__ __device__ inline int even_up(int x) { return (x + 1) & ~1; }

// Dynamic shared memory: F (FN entries and a zero slot), slices U V XI,
// row buffers s0 s1 s2 and the rows' z_y (L each), two partial-sum slots
// (2 x 4).
__host__ __device__ inline size_t cluster_smem_bytes(int FN, int L) {
    const size_t l2 = (size_t)even_up(L);
    return sizeof(double) * ((size_t)even_up(FN + 1) + 7 * l2 + 8);
}

// The double-float kernel's tables after the layout above: per row its
// SOC block (or a row kind), per SOC block its rows and kind, its derivative
// constants and the block's dot product of the current D Pi application.
__host__ __device__ inline size_t cluster_df_extra_bytes(int L, int NB) {
    const size_t rows = 4 * (size_t)even_up(L);
    return ((rows + 15) & ~(size_t)15) + (size_t)NB * (16 + 32 + 8);
}

struct CSmem {
    double *F, *U, *V, *XI, *s0, *s1, *s2, *ZY, *red;
};

__device__ __forceinline__ CSmem cluster_smem(double* base, int FN, int L) {
    const int l2 = even_up(L);
    CSmem s;
    s.F = base;
    s.U = s.F + even_up(FN + 1);
    s.V = s.U + l2;
    s.XI = s.V + l2;
    s.s0 = s.XI + l2;
    s.s1 = s.s0 + l2;
    s.s2 = s.s1 + l2;
    s.ZY = s.s2 + l2;
    s.red = s.ZY + l2;
    return s;
}

enum TauSlot { TAU_U = 0, TAU_V = 1, TAU_W = 2, TAU_X = 3, TAU_XI = 4, TAU_HB = 5 };  // TAU_HB: LSMR (df64 kernel)

// What a pass leaves for the warp that finishes it during the next pass.
struct Pending {
    double c1, c2, tin, tout, tt, wcoef, xcoef;
};

// Per-CTA constants of a cluster solve.
template <typename T>
struct CCtx {
    CSmem sm;
    const ClusterProb* cp;  // shared copy
    LsqrState* st;          // shared copy of the system's scalars
    Pending* pd;            // shared
    double* tau;            // shared: tau entries of U, V, W, X, XI (every CTA holds them)
    double* scr;            // shared: block-reduction scratch
    const SellSlice* slices;
    const int32_t* perm;
    const int32_t* scol;
    const T* valG;
    const T* valT;
    const double *cA, *cB, *rw, *cd, *zy;
    const int8_t* flag;
    const SocBlock* blocks;
    double* W;  // global, this system's w (own rows only)
    double* X;  // global, this system's x
    int* active;
    double kappa;
    int n, N, R0, L, C, rank, cb0, cb1, sl0, sl1;
};

// Row sums of the CTA's rows into out[] (local row index) by warps
// wfirst.., one slice at a time.  Every row is written exactly once.
template <typename T>
__device__ __forceinline__ void sell_rowsums(const CCtx<T>& c, const T* sval, const double* F, double* out,
                                             int wfirst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = kCWarps - wfirst;
    for (int s = c.sl0 + warp - wfirst; s < c.sl1; s += nw) {
        const SellSlice d = c.slices[s];
        const int32_t* cp = c.scol + d.base + lane;
        const T* vp = sval + d.base + lane;
        double acc = 0.0;
        int k = 0;
        for (; k + 4 <= d.width; k += 4) {
            int32_t j[4];
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                j[u] = __ldg(cp + 32 * (k + u));
                v[u] = ld(vp + 32 * (k + u));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc = fma(v[u], F[j[u]], acc);
        }
        for (; k < d.width; ++k) acc = fma(ld(vp + 32 * k), F[__ldg(cp + 32 * k)], acc);
        if (d.row >= 0) {
            acc = warp_sum(acc);
            if (lane == 0) out[d.row] = acc;
        } else {
            const int r = c.perm[d.pidx + lane];
            if (r >= 0) out[r] = acc;
        }
    }
}

// The end of a pass of kind (PASS, ROLE), run by warp 0 during the next
// pass: the pass's three sums over the cluster, its tau entries and the LSQR
// scalars (the same steps as the tile kernels' finisher).
template <int PASS, int ROLE, bool SC, typename T>
__device__ __forceinline__ void cluster_finish(const CCtx<T>& c, const int par) {
    cg::cluster_group cl = cg::this_cluster();
    const int lane = threadIdx.x & 31;
    double ta = 0.0, tb = 0.0, tc = 0.0;
    if (lane < c.C) {
        const double* rr = cl.map_shared_rank(c.sm.red + 4 * par, lane);
        ta = rr[0];
        tb = rr[1];
        tc = rr[2];
    }
    for (int o = 1; o < c.C; o <<= 1) {  // the same butterfly in every CTA
        ta += __shfl_xor_sync(0xffffffffu, ta, o);
        tb += __shfl_xor_sync(0xffffffffu, tb, o);
        tc += __shfl_xor_sync(0xffffffffu, tc, o);
    }
    if (lane != 0) return;
    const Pending pd = *c.pd;
    LsqrState& st = *c.st;
    const int rN = c.N - 1;
    double oN;
    if (PASS == PASS_G) {
        oN = -tb - tc + c.kappa * pd.tt;
        if (SC) oN *= c.rw[rN];
    } else {
        oN = tb - tc + c.kappa * pd.tt;
        if (SC) oN *= c.cd[rN];
    }
    // tau entries: G^T-passes keep them at 0 (the dz_N = 0 gauge of the tile kernels)
    const double nvN = (PASS == PASS_GT) ? 0.0 : pd.c1 * oN - pd.c2 * pd.tout;
    c.tau[ROLE == ROLE_U ? TAU_U : TAU_V] = nvN;
    if (PASS == PASS_GT) c.tau[TAU_XI] = 0.0;
    const double nsq = fma(nvN, nvN, ta);
    double nrm, inv_nrm;
    norm_and_inverse(nsq, nrm, inv_nrm);
    if (ROLE == ROLE_U) {
        c.tau[TAU_W] = pd.tin * pd.c1 - pd.wcoef * c.tau[TAU_W];
        lsqr_step_u(&st, nrm, inv_nrm, nsq);
    } else {
        c.tau[TAU_X] = fma(pd.xcoef, c.tau[TAU_W], c.tau[TAU_X]);
        if (lsqr_step_v(&st, nrm, inv_nrm) && c.rank == 0) atomicSub(c.active, 1);
    }
}

// One pass of the cluster loop.  `pending`: the previous pass (the other
// kind) still has to be finished.  Returns true once the system is finished.
template <int PASS, int ROLE, bool SC, typename T>
__device__ __forceinline__ bool cluster_pass(const CCtx<T>& c, const int par, const bool pending) {
    constexpr int PPASS = (PASS == PASS_G) ? PASS_GT : PASS_G;
    constexpr int PROLE = (ROLE == ROLE_U) ? ROLE_V : ROLE_U;
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x;
    double* s0 = c.sm.s0;
    if (tid < 32) {
        if (pending) cluster_finish<PPASS, PROLE, SC, T>(c, par ^ 1);
    } else {
        // speculative: discarded if the finisher ends the system
        sell_rowsums(c, PASS == PASS_G ? c.valG : c.valT, c.sm.F, s0, 1);
    }
    __syncthreads();

    LsqrState& st = *c.st;
    const int status = st.status;
    if (status == S_DONE) return true;
    const double wcoef = st.wcoef, xcoef = st.xcoef;
    if (ROLE == ROLE_V && status == S_FINAL) {
        // the u-update converged: finish x and stop
        for (int i = tid; i < c.L; i += kCThreads) {
            const int r = c.R0 + i;
            c.X[r] = fma(xcoef, c.W[r], c.X[r]);
        }
        __syncthreads();
        if (tid == 0) {
            c.tau[TAU_X] = fma(xcoef, c.tau[TAU_W], c.tau[TAU_X]);
            st.status = S_DONE;
            if (c.rank == 0) atomicSub(c.active, 1);
        }
        __syncthreads();
        return true;
    }
    const double c1 = (ROLE == ROLE_U) ? st.uc1 : st.vc1;
    const double c2 = (ROLE == ROLE_U) ? st.uc2 : st.vc2;
    double* in_s = (ROLE == ROLE_U) ? c.sm.V : c.sm.U;
    double* out_s = (ROLE == ROLE_U) ? c.sm.U : c.sm.V;
    const double tin = c.tau[ROLE == ROLE_U ? TAU_V : TAU_U];
    const double tout = c.tau[ROLE == ROLE_U ? TAU_U : TAU_V];
    const double tt = SC ? (PASS == PASS_G ? c.cd[c.N - 1] : c.rw[c.N - 1]) * tin : tin;
    const int L = c.L, R0 = c.R0, n = c.n;
    double* s1 = c.sm.s1;
    double* s2 = c.sm.s2;
    double* XIs = c.sm.XI;
    const double* cA = c.cA;
    const double* cB = c.cB;
    const double* rw = c.rw;
    const double* cd = c.cd;

    double ss = 0.0, dtop = 0.0, dbot = 0.0;
    if (PASS == PASS_G) {
        for (int i = tid; i < L; i += kCThreads) {
            const int r = R0 + i;
            const double iv = in_s[i];
            double o;
            if (r < n) {
                o = fma(cA[r], tt, s0[i]);
                dtop = fma(cB[r], SC ? cd[r] * iv : iv, dtop);
            } else {
                const double xi = XIs[i];
                const double dxi = SC ? cd[r] * (xi - iv) : xi - iv;
                o = fma(-cA[r], tt, s0[i]) + dxi;
                dbot = fma(cB[r], SC ? cd[r] * xi : xi, dbot);
            }
            if (SC) o *= rw[r];
            const double nv = fma(c1, o, -c2 * out_s[i]);
            out_s[i] = nv;
            ss = fma(nv, nv, ss);
            if (ROLE == ROLE_U) c.W[r] = fma(iv, c1, -wcoef * c.W[r]);
            else c.X[r] = fma(xcoef, c.W[r], c.X[r]);
        }
    } else {
        for (int i = tid; i < L; i += kCThreads) {
            const int r = R0 + i;
            const double iv = SC ? rw[r] * in_s[i] : in_s[i];
            const double h = fma(-cB[r], tt, s0[i]);
            if (r < n) {
                s1[i] = h;
                dtop = fma(cA[r], iv, dtop);
            } else {
                s1[i] = h + iv;
                dbot = fma(cA[r], iv, dbot);
            }
        }
        __syncthreads();
        apply_D_tile<double, kCWarps>(s1, s2, R0, R0 + L, n, c.flag, c.blocks, c.cb0, c.cb1, c.sm.ZY, R0,
                                      c.cp->nlarge[c.rank] > 0);
        __syncthreads();
        for (int i = tid; i < L; i += kCThreads) {
            const int r = R0 + i;
            const double iv = in_s[i];
            double o = (r < n) ? s2[i] : s2[i] - (SC ? rw[r] * iv : iv);
            if (SC) o *= cd[r];
            const double nv = fma(c1, o, -c2 * out_s[i]);
            out_s[i] = nv;
            s1[i] = nv;
            ss = fma(nv, nv, ss);
            if (ROLE == ROLE_U) c.W[r] = fma(iv, c1, -wcoef * c.W[r]);
            else c.X[r] = fma(xcoef, c.W[r], c.X[r]);
        }
        __syncthreads();
        apply_D_tile<double, kCWarps>(s1, s2, R0, R0 + L, n, c.flag, c.blocks, c.cb0, c.cb1, c.sm.ZY, R0,
                                      c.cp->nlarge[c.rank] > 0);
        __syncthreads();
        for (int i = tid; i < L; i += kCThreads) XIs[i] = s2[i];
    }
    double v3[3] = {ss, dtop, dbot};
    block_reduce<3, kCThreads>(v3, c.scr);
    if (tid == 0) {
        c.sm.red[4 * par + 0] = v3[0];
        c.sm.red[4 * par + 1] = v3[1];
        c.sm.red[4 * par + 2] = v3[2];
        *c.pd = Pending{c1, c2, tin, tout, tt, wcoef, xcoef};
    }
    cl.sync();

    // The vector the next pass gathers (xi after a G^T-pass, the new u or v
    // after a G-pass): pair k of F from the CTA whose range holds it, four
    // independent remote loads per thread issued before any store.
    {
        const double* bvec = (PASS == PASS_GT) ? XIs : out_s;
        double2* dst = reinterpret_cast<double2*>(c.sm.F);
        const int npairs = c.cp->FN >> 1;
        constexpr int kU = 4;
        for (int k0 = tid; k0 < npairs; k0 += kU * kCThreads) {
            double2 v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int k = k0 + u * kCThreads;
                if (k < npairs) {
                    int lo = 0, hi = c.C;  // the last CTA r with poff[r] <= 2k
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (c.cp->poff[mid] <= 2 * k) lo = mid;
                        else hi = mid;
                    }
                    const double2* src = reinterpret_cast<const double2*>(cl.map_shared_rank(bvec, lo));
                    v[u] = src[k - (c.cp->poff[lo] >> 1)];
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int k = k0 + u * kCThreads;
                if (k < npairs) dst[k] = v[u];
            }
        }
    }
    __syncthreads();
    return false;
}

// MODE 0: JVP (u-update = G-pass, v-update = G^T-pass); MODE 1: VJP.
template <int MODE, bool SC, typename T>
__global__ void __launch_bounds__(kCThreads, 1) k_cluster(PlanView<T> a, ClusterArgs ca) {
    extern __shared__ __align__(16) double csm[];
    __shared__ double scr[3 * kCThreads];
    __shared__ LsqrState st;
    __shared__ Pending pd;
    __shared__ double tau[5];
    __shared__ ClusterProb cp;
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
    if (tid == 0) {
        cp = ca.cprob[sy.prob];
        st = a.state[si];
        tau[TAU_U] = gU[rN];
        tau[TAU_V] = gV[rN];
        tau[TAU_W] = a.W[sy.voff + rN];
        tau[TAU_X] = a.X[sy.voff + rN];
        tau[TAU_XI] = gXI[rN];
    }
    __syncthreads();
    CCtx<T> c;
    c.sm = cluster_smem(csm, cp.FN, cp.L);  // the problem's own layout (a cluster holds one problem)
    c.cp = &cp;
    c.st = &st;
    c.pd = &pd;
    c.tau = tau;
    c.scr = scr;
    c.slices = ca.slices;
    c.perm = ca.perm;
    c.scol = ca.scol;
    c.valG = static_cast<const T*>(a.scaled ? ca.svalG : ca.sval);
    c.valT = static_cast<const T*>(a.scaled ? ca.svalT : ca.sval);
    c.cA = a.coefA + pr.doff;
    c.cB = a.coefB + pr.doff;
    c.rw = a.rw + pr.doff;
    c.cd = a.cd + pr.doff;
    c.zy = a.zy + pr.doff;
    c.flag = a.flag + pr.doff;
    c.blocks = a.blocks + pr.soff;
    c.W = a.W + sy.voff;
    c.X = a.X + sy.voff;
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

    const bool live = st.status != S_DONE;
    if (live) {
        for (int i = tid; i < c.L; i += kCThreads) {
            c.sm.U[i] = gU[c.R0 + i];
            c.sm.V[i] = gV[c.R0 + i];
            c.sm.XI[i] = gXI[c.R0 + i];
            c.sm.ZY[i] = c.zy[c.R0 + i];
        }
        // the first u-update gathers xi (JVP) or v (VJP); slot FN stays 0 for padding
        const double* g0 = (MODE == 0) ? gXI : gV;
        for (int r = 0; r < C; ++r) {
            const int r0 = cp.split[r], len = cp.split[r + 1] - r0;
            double* dst = c.sm.F + cp.poff[r];
            for (int i = tid; i < len; i += kCThreads) dst[i] = g0[r0 + i];
        }
        if (tid == 0) c.sm.F[cp.FN] = 0.0;
    }
    __syncthreads();
    cl.sync();  // every CTA of the cluster runs before any remote access
    if (live) {
        int par = 0;
        bool pending = false;
        for (int64_t pass = 0; pass < ca.max_passes; pass += 2) {
            if (cluster_pass<PU, ROLE_U, SC, T>(c, par, pending)) break;
            pending = true;
            par ^= 1;
            if (cluster_pass<PV, ROLE_V, SC, T>(c, par, true)) break;
            par ^= 1;
        }
        for (int i = tid; i < c.L; i += kCThreads) {
            gU[c.R0 + i] = c.sm.U[i];
            gV[c.R0 + i] = c.sm.V[i];
            gXI[c.R0 + i] = c.sm.XI[i];
        }
        if (tid == 0 && rank == 0) {
            gU[rN] = tau[TAU_U];
            gV[rN] = tau[TAU_V];
            a.W[sy.voff + rN] = tau[TAU_W];
            a.X[sy.voff + rN] = tau[TAU_X];
            gXI[rN] = tau[TAU_XI];
            a.state[si] = st;
        }
    }
    cl.sync();  // no CTA leaves while a peer may still read its shared memory
}

}  // namespace qcpd
