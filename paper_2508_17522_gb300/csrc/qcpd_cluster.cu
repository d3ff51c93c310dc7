// Host side of the cluster engine: per-problem row splits, the gather-buffer
// column map, and the launches (one per cluster size present in a call).
#include <algorithm>
#include <climits>
#include <cstring>

#include "qcpd_cluster.h"
#include "qcpd_stream.h"

namespace qcpd {

// Weight of one row against one stored entry when balancing CTAs: the
// epilogue spends about eight FP64 operations per row, the row sums one per
// stored entry.
constexpr double kRowWeight = 8.0;      // per row, next to its stored entries
constexpr double kSocRowWeight = 10.0;  // more per row of an SOC block (its D Pi rows cost more in the epilogue)

// Slot -> (gather-buffer column, values) of the SELL-32 copy: column j of M
// lives at poff[r] + j - split[r] of the gather buffer, r the CTA owning row
// j; padding slots point at the zero slot FN with value 0.
template <typename T>
__device__ __forceinline__ void sell_put(int64_t slot, int64_t src, const ClusterProb& cp, const int32_t* mcol,
                                         const T* mval, const T* mvalG, const T* mvalT, int32_t* scol, T* sval,
                                         T* svalG, T* svalT) {
    if (src < 0) {
        scol[slot] = cp.FN;
        sval[slot] = (T)0;
        svalG[slot] = (T)0;
        svalT[slot] = (T)0;
        return;
    }
    const int j = mcol[src];
    int lo = 0, hi = cp.C;  // the last r with split[r] <= j
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cp.split[mid] <= j) lo = mid;
        else hi = mid;
    }
    scol[slot] = cp.poff[lo] + (j - cp.split[lo]);
    sval[slot] = mval[src];
    svalG[slot] = mvalG[src];
    svalT[slot] = mvalT[src];
}

// One warp per slice.
template <typename T>
__global__ void k_sell_fill(const SellSlice* sl, int64_t nsl, const int32_t* perm, const int32_t* sl_prob,
                            const int32_t* sl_r0, const ClusterProb* cps, const Prob* probs, const int64_t* mrowptr,
                            const int32_t* mcol, const T* mval, const T* mvalG, const T* mvalT, int32_t* scol,
                            T* sval, T* svalG, T* svalT) {
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nsl) return;
    const SellSlice d = sl[s];
    const ClusterProb cp = cps[sl_prob[s]];
    const int64_t* rp = mrowptr + probs[sl_prob[s]].mrow;
    const int R0 = sl_r0[s];
    if (d.row >= 0) {
        const int64_t k0 = rp[R0 + d.row], len = rp[R0 + d.row + 1] - k0;
        for (int64_t j = lane; j < (int64_t)d.width * 32; j += 32)
            sell_put(d.base + j, j < len ? k0 + j : -1, cp, mcol, mval, mvalG, mvalT, scol, sval, svalG, svalT);
    } else {
        const int row = perm[d.pidx + lane];
        int64_t k0 = 0, len = 0;
        if (row >= 0) {
            k0 = rp[R0 + row];
            len = rp[R0 + row + 1] - k0;
        }
        for (int k = 0; k < d.width; ++k)
            sell_put(d.base + 32 * (int64_t)k + lane, k < len ? k0 + k : -1, cp, mcol, mval, mvalG, mvalT, scol,
                     sval, svalG, svalT);
    }
}

// Cut problem pi's n + m rows into C ranges of about equal weight, never
// inside a second-order-cone block and of at most lcap rows each.  Returns
// false when C such ranges cannot hold the rows.
static bool cluster_split(const qcp_plan* p, int pi, int C, int lcap, ClusterProb& cp) {
    const Prob& pr = p->hprob[pi];
    const int n = pr.n, Nx = pr.n + pr.m;
    const int64_t* rp = p->h_mrowptr.data() + pr.mrow;
    // cut candidates: the end of every row outside SOC blocks and of every SOC block
    std::vector<int> ends, socs, brows;  // brows: rows of coupled blocks up to each end
    ends.reserve(Nx);
    socs.reserve(Nx);
    brows.reserve(Nx);
    int row = 0, nsb = 0, nbr = 0;
    for (; row < n; ++row) {
        ends.push_back(row + 1);
        socs.push_back(0);
        brows.push_back(0);
    }
    for (size_t b = 0; b < p->cone_type[pi].size(); ++b) {
        const int t = p->cone_type[pi][b], d = p->cone_dim[pi][b];
        if (t == QCP_CONE_SOC || t == QCP_CONE_PSD || t == QCP_CONE_EXP || t == QCP_CONE_POW) {
            row += d;
            nbr += d;
            ++nsb;
            ends.push_back(row);
            socs.push_back(nsb);
            brows.push_back(nbr);
        } else {
            for (int k = 0; k < d; ++k) {
                ends.push_back(++row);
                socs.push_back(nsb);
                brows.push_back(nbr);
            }
        }
    }
    std::memset(&cp, 0, sizeof(cp));
    cp.C = C;
    const double total = (double)(rp[Nx] - rp[0]) + kRowWeight * Nx + kSocRowWeight * nbr;
    // a range closed by the row cap holds at least lcap - umax + 1 rows
    // (umax: the largest unit, an SOC block or one row)
    int umax = 1;
    for (size_t u = 0, prev = 0; u < ends.size(); prev = ends[u], ++u) umax = std::max(umax, ends[u] - (int)prev);
    const int64_t room = std::max(1, lcap - umax + 1);
    int k = 1, start = 0;
    for (size_t u = 0; u < ends.size() && k < C; ++u) {
        const int e = ends[u];
        // a range also closes before its next unit would take it past lcap
        // rows, and never closes at its weight target while the rows after
        // it would not fit in the remaining ranges (dense rows first, then
        // many light ones: the weight alone would give the light ones a
        // single range)
        const int next = (u + 1 < ends.size()) ? ends[u + 1] : e;
        const double acc = (double)(rp[e] - rp[0]) + kRowWeight * e + kSocRowWeight * brows[u];
        while (k < C && ((acc >= total * k / C && (int64_t)(Nx - e) <= (int64_t)(C - k) * room) ||
                         next - start > lcap)) {
            cp.split[k] = e;
            cp.cb[k] = socs[u];
            start = e;
            ++k;
        }
    }
    for (; k <= kMaxCluster; ++k) {
        cp.split[k] = Nx;
        cp.cb[k] = nsb;
    }
    cp.nb = 0;
    for (int r = 0; r < C; ++r) cp.nb = std::max(cp.nb, cp.cb[r + 1] - cp.cb[r]);
    for (int r = 0; r < C; ++r) {  // SOC blocks too large for one thread each
        int nl = 0, bi = 0;
        for (size_t b = 0; b < p->cone_type[pi].size(); ++b) {
            const int t = p->cone_type[pi][b], d = p->cone_dim[pi][b];
            if (t == QCP_CONE_SOC || t == QCP_CONE_PSD || t == QCP_CONE_EXP || t == QCP_CONE_POW) {
                if (bi >= cp.cb[r] && bi < cp.cb[r + 1] && d > kSocThread) ++nl;
                ++bi;
            }
        }
        cp.nlarge[r] = nl;
    }
    int L = 0;
    cp.poff[0] = 0;
    for (int r = 0; r < kMaxCluster; ++r) {
        const int len = (r < C) ? cp.split[r + 1] - cp.split[r] : 0;
        L = std::max(L, len);
        cp.poff[r + 1] = cp.poff[r] + even_up(len);
    }
    cp.FN = cp.poff[C];
    cp.L = L;
    return L <= lcap;
}

template <typename K>
static void max_static_smem(K k, size_t& s) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) == cudaSuccess) s = std::max(s, fa.sharedSizeBytes);
}

// Dynamic shared memory one CTA of the cluster kernels may use.
static int cluster_smem_limit(size_t* out) {
    int dev = 0, optin = 0;
    QCP_CUDA(cudaGetDevice(&dev));
    QCP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    size_t st = 0;
    max_static_smem(k_cluster<0, false, double>, st);
    max_static_smem(k_cluster<0, true, double>, st);
    max_static_smem(k_cluster<1, false, double>, st);
    max_static_smem(k_cluster<1, true, double>, st);
    max_static_smem(k_cluster<0, false, float>, st);
    max_static_smem(k_cluster<0, true, float>, st);
    max_static_smem(k_cluster<1, false, float>, st);
    max_static_smem(k_cluster<1, true, float>, st);
    max_static_smem(k_cluster_df<0, false, double>, st);
    max_static_smem(k_cluster_df<0, true, double>, st);
    max_static_smem(k_cluster_df<1, false, double>, st);
    max_static_smem(k_cluster_df<1, true, double>, st);
    max_static_smem(k_cluster_df<0, false, float>, st);
    max_static_smem(k_cluster_df<0, true, float>, st);
    max_static_smem(k_cluster_df<1, false, float>, st);
    max_static_smem(k_cluster_df<1, true, float>, st);
    max_static_smem(k_cluster_df<0, false, double, true>, st);
    max_static_smem(k_cluster_df<0, true, double, true>, st);
    max_static_smem(k_cluster_df<1, false, double, true>, st);
    max_static_smem(k_cluster_df<1, true, double, true>, st);
    max_static_smem(k_cluster_df<0, false, float, true>, st);
    max_static_smem(k_cluster_df<0, true, float, true>, st);
    max_static_smem(k_cluster_df<1, false, float, true>, st);
    max_static_smem(k_cluster_df<1, true, float, true>, st);
    *out = (size_t)optin > st ? (size_t)optin - st : 0;
    return QCP_OK;
}

// Clusters of C CTAs of the cluster kernel that can be resident at once.
static int max_active_clusters(int C) {
    static int cache[kMaxCluster + 1][64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cache[C][dev]) return cache[C][dev] - 1;
    auto fn = k_cluster<0, false, double>;
    const int smem = 64 * 1024;
    int n = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
        (C <= 8 || cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess)) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(kCThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    cache[C][dev] = n + 1;
    return n;
}

// The most CTAs per system, up to 8, with which every system's cluster is
// resident at once (clusters cannot straddle GPCs, so this is not simply
// SMs / systems); 1 when even single CTAs do not all fit.
static int auto_cap(int nsys) {
    for (int C = 8; C > 1; --C)
        if (max_active_clusters(C) >= nsys) return C;
    return 1;
}

// The SELL-32 copy of every problem's rows, CTA by CTA: rows longer than
// kSellLong get a lane-strided slice each; the others are sorted by length
// (longest first, so a slice's rows have similar lengths) and cut into
// slices of 32.
template <typename T>
static int fill_sell(qcp_plan* p, ClusterLayout* lay, const std::vector<SellSlice>& hs,
                     const std::vector<int32_t>& hsp, const std::vector<int32_t>& hsr, int64_t slots) {
    QCP_TRY(lay->d_scol.alloc(sizeof(int32_t) * (size_t)slots));
    QCP_TRY(lay->d_sval.alloc(sizeof(T) * (size_t)slots));
    QCP_TRY(lay->d_svalG.alloc(sizeof(T) * (size_t)slots));
    QCP_TRY(lay->d_svalT.alloc(sizeof(T) * (size_t)slots));
    DevBuf& d_sp = lay->d_sp;
    DevBuf& d_sr = lay->d_sr;
    QCP_TRY(d_sp.alloc(sizeof(int32_t) * hsp.size()));
    QCP_TRY(d_sr.alloc(sizeof(int32_t) * hsr.size()));
    QCP_CUDA(cudaMemcpyAsync(d_sp.p, hsp.data(), sizeof(int32_t) * hsp.size(), cudaMemcpyHostToDevice, p->stream));
    QCP_CUDA(cudaMemcpyAsync(d_sr.p, hsr.data(), sizeof(int32_t) * hsr.size(), cudaMemcpyHostToDevice, p->stream));
    const int64_t nsl = (int64_t)hs.size();
    lay->nslices = nsl;
    lay->slots = slots;
    if (nsl > 0) {
        const int64_t blocks = (nsl * 32 + 255) / 256;
        k_sell_fill<T><<<(unsigned)blocks, 256, 0, p->stream>>>(
            lay->d_slices.as<SellSlice>(), nsl, lay->d_perm.as<int32_t>(), d_sp.as<int32_t>(), d_sr.as<int32_t>(),
            lay->d_cprob.as<ClusterProb>(), p->d_prob.as<Prob>(), p->d_mrowptr.as<int64_t>(), p->d_mcol.as<int32_t>(),
            p->d_mval.as<T>(), p->d_mvalG.as<T>(), p->d_mvalT.as<T>(), lay->d_scol.as<int32_t>(), lay->d_sval.as<T>(),
            lay->d_svalG.as<T>(), lay->d_svalT.as<T>());
        QCP_CUDA(cudaGetLastError());
    }
    QCP_CUDA(cudaStreamSynchronize(p->stream));
    return QCP_OK;
}

// df64 copies: out[i] = (hi, lo) of in[i]; *bad set when a nonzero entry is
// outside [2^-90, 2^90] or not finite (the df64 kernel's safe range).
constexpr double kDfMin = 0x1p-90, kDfMax = 0x1p90;

__device__ __forceinline__ bool df_unsafe(double x) {
    const double a = fabs(x);
    return !(a == 0.0 || (a >= kDfMin && a <= kDfMax));
}

template <typename T>
__global__ void k_to_df(const T* in, int64_t n, df* out, int* bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)in[i];
        if (df_unsafe(x)) atomicExch(bad, 1);
        out[i] = df_from(x);
    }
}

__global__ void k_soc_df(const SocBlock* blk, int64_t nb, SocDf* out, int* bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
        const SocBlock B = blk[i];
        SocDf s;
        const double htr = B.h * (B.t + B.r);
        if (B.kase == 2 && (df_unsafe(B.r) || df_unsafe(B.h) || df_unsafe(B.tq) || df_unsafe(htr))) atomicExch(bad, 1);
        s.r = df_from(B.r);
        s.h = df_from(B.h);
        s.tq = df_from(B.tq);
        s.htr = df_from(htr);
        out[i] = s;
    }
}

template <typename T>
static int to_df(qcp_plan* p, const DevBuf& in, int64_t n, DevBuf& out, int* bad) {
    QCP_TRY(out.alloc(sizeof(df) * (size_t)std::max<int64_t>(n, 1)));
    if (n > 0) {
        const int grid = (int)std::min<int64_t>(4096, (n + 255) / 256);
        k_to_df<T><<<grid, 256, 0, p->stream>>>(in.as<T>(), n, out.as<df>(), bad);
    }
    return QCP_OK;
}

template <typename T>
static int build_df(qcp_plan* p, ClusterLayout* lay, int64_t slots) {
    DevBuf bad;
    QCP_TRY(bad.alloc(sizeof(int)));
    QCP_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), p->stream));
    int* b = bad.as<int>();
    QCP_TRY(to_df<T>(p, lay->d_sval, slots, lay->d_dsval, b));
    QCP_TRY(to_df<T>(p, lay->d_svalG, slots, lay->d_dsvalG, b));
    QCP_TRY(to_df<T>(p, lay->d_svalT, slots, lay->d_dsvalT, b));
    QCP_TRY(to_df<double>(p, p->d_coefA, p->N_tot, lay->d_dcA, b));
    QCP_TRY(to_df<double>(p, p->d_coefB, p->N_tot, lay->d_dcB, b));
    QCP_TRY(to_df<double>(p, p->d_rw, p->N_tot, lay->d_drw, b));
    QCP_TRY(to_df<double>(p, p->d_cd, p->N_tot, lay->d_dcd, b));
    QCP_TRY(to_df<double>(p, p->d_zy, p->N_tot, lay->d_dzy, b));
    QCP_TRY(lay->d_dsoc.alloc(sizeof(SocDf) * (size_t)std::max<int64_t>(p->nsoc_tot, 1)));
    if (p->nsoc_tot > 0) {
        const int grid = (int)std::min<int64_t>(4096, (p->nsoc_tot + 255) / 256);
        k_soc_df<<<grid, 256, 0, p->stream>>>(p->d_blocks.as<SocBlock>(), p->nsoc_tot, lay->d_dsoc.as<SocDf>(), b);
    }
    QCP_CUDA(cudaGetLastError());
    int hbad = 1;
    QCP_CUDA(cudaMemcpyAsync(&hbad, b, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    QCP_CUDA(cudaStreamSynchronize(p->stream));
    lay->df_ok = hbad == 0;
    return QCP_OK;
}

// QCP_PRECOND_DIAG on the cluster engine: the caller's C (block-averaged by
// prepare_diag into p->d_cdD, with M diag(C) in p->d_mvalD) changes from
// call to call, so every such call refills the layout's M diag(C) slots
// (the same slot map as the other value arrays; the plain values serve the
// G^T-passes, W = I) and the df64 copies of M diag(C), W = 1 and C.
template <typename T>
static int refresh_diag(qcp_plan* p, ClusterLayout* lay) {
    const int64_t slots = std::max<int64_t>(lay->slots, 1), nt = std::max<int64_t>(p->N_tot, 1);
    if (!lay->d_svalDG.p) {
        QCP_TRY(lay->d_svalDG.alloc(sizeof(T) * (size_t)slots));
        QCP_TRY(lay->d_dsvalDG.alloc(sizeof(df) * (size_t)slots));
        QCP_TRY(lay->d_drwD.alloc(sizeof(df) * (size_t)nt));
        QCP_TRY(lay->d_dcdD.alloc(sizeof(df) * (size_t)nt));
        QCP_TRY(lay->d_diag_bad.alloc(sizeof(int)));
    }
    cudaStream_t st = p->stream;
    int* b = lay->d_diag_bad.as<int>();
    QCP_CUDA(cudaMemsetAsync(b, 0, sizeof(int), st));
    if (lay->nslices > 0) {
        const int64_t blocks = (lay->nslices * 32 + 255) / 256;
        // scol and sval are rewritten with the values they already hold
        k_sell_fill<T><<<(unsigned)blocks, 256, 0, st>>>(
            lay->d_slices.as<SellSlice>(), lay->nslices, lay->d_perm.as<int32_t>(), lay->d_sp.as<int32_t>(),
            lay->d_sr.as<int32_t>(), lay->d_cprob.as<ClusterProb>(), p->d_prob.as<Prob>(), p->d_mrowptr.as<int64_t>(),
            p->d_mcol.as<int32_t>(), p->d_mval.as<T>(), p->d_mvalD.as<T>(), p->d_mval.as<T>(),
            lay->d_scol.as<int32_t>(), lay->d_sval.as<T>(), lay->d_svalDG.as<T>(), lay->d_sval.as<T>());
    }
    const int g1 = (int)std::min<int64_t>(4096, (slots + 255) / 256), g2 = (int)std::min<int64_t>(4096, (nt + 255) / 256);
    k_to_df<T><<<g1, 256, 0, st>>>(lay->d_svalDG.as<T>(), slots, lay->d_dsvalDG.as<df>(), b);
    k_to_df<double><<<g2, 256, 0, st>>>(p->d_onesD.as<double>(), p->N_tot, lay->d_drwD.as<df>(), b);
    k_to_df<double><<<g2, 256, 0, st>>>(p->d_cdD.as<double>(), p->N_tot, lay->d_dcdD.as<df>(), b);
    QCP_CUDA(cudaGetLastError());
    int hbad = 1;
    QCP_CUDA(cudaMemcpyAsync(&hbad, b, sizeof(int), cudaMemcpyDeviceToHost, st));
    QCP_CUDA(cudaStreamSynchronize(st));
    lay->diag_df_ok = hbad == 0;
    return QCP_OK;
}

static int build_sell(qcp_plan* p, ClusterLayout* lay) {
    std::vector<SellSlice> hs;
    std::vector<int32_t> hperm, hsp, hsr;
    int64_t slots = 0;
    std::vector<int> order;
    for (int pi = 0; pi < p->nprob; ++pi) {
        ClusterProb& cp = lay->hp[pi];
        const Prob& pr = p->hprob[pi];
        const int64_t* rp = p->h_mrowptr.data() + pr.mrow;
        for (int r = 0; r < cp.C; ++r) {
            cp.sl[r] = (int32_t)hs.size();
            const int R0 = cp.split[r], R1 = cp.split[r + 1];
            order.clear();
            for (int i = R0; i < R1; ++i) {
                const int64_t len = rp[i + 1] - rp[i];
                if (len > kSellLong) {
                    const int w = (int)((len + 31) / 32);
                    hs.push_back(SellSlice{slots, w, i - R0, 0, 0});
                    hsp.push_back(pi);
                    hsr.push_back(R0);
                    slots += 32 * (int64_t)w;
                } else {
                    order.push_back(i);
                }
            }
            std::stable_sort(order.begin(), order.end(),
                             [&](int x, int y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
            for (size_t q = 0; q < order.size(); q += 32) {
                const int w = (int)(rp[order[q] + 1] - rp[order[q]]);
                hs.push_back(SellSlice{slots, w, -1, (int32_t)hperm.size(), 0});
                hsp.push_back(pi);
                hsr.push_back(R0);
                for (size_t l = 0; l < 32; ++l) hperm.push_back(q + l < order.size() ? order[q + l] - R0 : -1);
                slots += 32 * (int64_t)w;
            }
        }
        for (int r = cp.C; r <= kMaxCluster; ++r) cp.sl[r] = (int32_t)hs.size();
    }
    if (hs.size() > (size_t)INT32_MAX || hperm.size() > (size_t)INT32_MAX) {
        set_error("cluster engine: too many row slices");
        return QCP_ERR_ARG;
    }
    QCP_TRY(lay->d_cprob.alloc(sizeof(ClusterProb) * p->nprob));
    QCP_CUDA(cudaMemcpyAsync(lay->d_cprob.p, lay->hp.data(), sizeof(ClusterProb) * p->nprob, cudaMemcpyHostToDevice,
                             p->stream));
    QCP_TRY(lay->d_slices.alloc(sizeof(SellSlice) * hs.size()));
    QCP_TRY(lay->d_perm.alloc(sizeof(int32_t) * hperm.size()));
    QCP_CUDA(cudaMemcpyAsync(lay->d_slices.p, hs.data(), sizeof(SellSlice) * hs.size(), cudaMemcpyHostToDevice,
                             p->stream));
    QCP_CUDA(cudaMemcpyAsync(lay->d_perm.p, hperm.data(), sizeof(int32_t) * hperm.size(), cudaMemcpyHostToDevice,
                             p->stream));
    if (p->dtype == QCP_F64) {
        QCP_TRY(fill_sell<double>(p, lay, hs, hsp, hsr, slots));
        return build_df<double>(p, lay, slots);
    }
    QCP_TRY(fill_sell<float>(p, lay, hs, hsp, hsr, slots));
    return build_df<float>(p, lay, slots);
}

static int get_layout(qcp_plan* p, int cap, ClusterLayout** out) {
    auto it = p->clusters.find(cap);
    if (it != p->clusters.end()) {
        *out = it->second.get();
        return QCP_OK;
    }
    size_t limit = 0;
    QCP_TRY(cluster_smem_limit(&limit));
    std::unique_ptr<ClusterLayout> lay(new ClusterLayout());
    lay->hp.resize(p->nprob);
    // exponential, power and PSD blocks: their dense D Pi (df64, the
    // double-float kernel only)
    lay->fits = true;
    if (p->kpsd || p->ndense) QCP_TRY(dense_dpi_ready(p, &lay->fits));
    for (int pi = 0; pi < p->nprob; ++pi) {
        bool ok = false;
        const Prob& pr = p->hprob[pi];
        for (int C = cap; C <= kMaxCluster && !ok; ++C) {
            // most rows per CTA next to a gather buffer of n + m + C entries
            int lcap = 0;
            const int FN = pr.n + pr.m + C;
            while (cluster_smem_bytes(FN, lcap + 2) + cluster_df_extra_bytes(lcap + 2, 0) <= limit) lcap += 2;
            if (lcap < 1) continue;
            // the SOC-block tables grow with the blocks a CTA gets: cap the
            // rows lower until the whole layout fits
            for (int t = 0; t < 5 && !ok && lcap >= 2; ++t, lcap = lcap * 17 / 20)
                ok = cluster_split(p, pi, C, lcap, lay->hp[pi]) &&
                     cluster_smem_bytes(lay->hp[pi].FN, lay->hp[pi].L) +
                             cluster_df_extra_bytes(lay->hp[pi].L, lay->hp[pi].nb) <= limit;
        }
        if (!ok) lay->fits = false;
    }
    if (lay->fits) QCP_TRY(build_sell(p, lay.get()));
    if (lay->fits && (p->kpsd || p->ndense) && !lay->df_ok) lay->fits = false;  // the FP64 kernel has no dense D Pi
    *out = lay.get();
    p->clusters.emplace(cap, std::move(lay));
    return QCP_OK;
}

static int cap_for(const qcp_plan* p, int nsys) { return p->cluster_cap > 0 ? p->cluster_cap : auto_cap(nsys); }

int cluster_ready(qcp_plan* p, int nsys, bool* ok, bool need_df) {
    ClusterLayout* lay = nullptr;
    QCP_TRY(get_layout(p, cap_for(p, nsys), &lay));
    *ok = lay->fits && (!need_df || lay->df_ok);
    return QCP_OK;
}

template <int MODE, typename T>
static auto cluster_kernel(bool scaled) -> void (*)(PlanView<T>, ClusterArgs) {
    return scaled ? k_cluster<MODE, true, T> : k_cluster<MODE, false, T>;
}

template <int MODE, typename T>
static auto cluster_kernel_df(bool scaled, bool lsmr) -> void (*)(PlanView<T>, ClusterArgs, ClusterDfArgs) {
    if (lsmr) return scaled ? k_cluster_df<MODE, true, T, true> : k_cluster_df<MODE, false, T, true>;
    return scaled ? k_cluster_df<MODE, true, T> : k_cluster_df<MODE, false, T>;
}

// Dynamic shared memory, non-portable size and occupancy of one cluster launch.
template <typename K>
static int prepare_launch(K fn, int C, size_t bytes, cudaLaunchConfig_t& cfg) {
    QCP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (C > 8) QCP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    int active = 0;
    QCP_CUDA(cudaOccupancyMaxActiveClusters(&active, fn, &cfg));
    if (active < 1) {
        set_error("cluster engine: a cluster of %d CTAs with %zu bytes of shared memory each cannot run", C, bytes);
        return QCP_ERR_ARG;
    }
    return QCP_OK;
}

template <typename T>
int iterate_cluster(qcp_plan* p, const ClusterSeg* segs, int nseg, int nsys_call, const PlanView<T>& v,
                    const qcp_options& opts) {
    ClusterLayout* lay = nullptr;
    QCP_TRY(get_layout(p, cap_for(p, nsys_call), &lay));
    if (!lay->fits) {
        set_error("cluster engine: a problem's vectors do not fit in the shared memory of 16 CTAs");
        return QCP_ERR_ARG;
    }
    cudaStream_t st = p->stream;
    // per range, its systems grouped by cluster size: one launch per group
    struct Launch {
        int seg, C, start, count, FN, L, NB;
        size_t bytes64, bytesdf;  // dynamic shared memory: the largest problem layout of the launch
        size_t boff;              // offset of the launch's broadcast buffers (df)
    };
    std::vector<Launch> launches;
    p->h_csys.clear();
    size_t bneed = 0;
    for (int k = 0; k < nseg; ++k) {
        for (int C = 1; C <= kMaxCluster; ++C) {
            Launch L{k, C, (int)p->h_csys.size(), 0, 0, 0, 0, 0, 0, 0};
            for (int s = segs[k].s0; s < segs[k].s0 + segs[k].ns; ++s) {
                const ClusterProb& cp = lay->hp[p->hsys[s].prob];
                if (cp.C != C) continue;
                p->h_csys.push_back(s);
                L.FN = std::max(L.FN, cp.FN);
                L.L = std::max(L.L, cp.L);
                L.NB = std::max(L.NB, cp.nb);
                // each CTA lays out shared memory for its own problem, so
                // the launch needs the largest single layout
                const size_t b64 = cluster_smem_bytes(cp.FN, cp.L);
                L.bytes64 = std::max(L.bytes64, b64);
                L.bytesdf = std::max(L.bytesdf, b64 + cluster_df_extra_bytes(cp.L, cp.nb));
            }
            L.count = (int)p->h_csys.size() - L.start;
            if (L.count == 0) continue;
            L.boff = bneed;
            bneed += sizeof(df) * 2 * (size_t)even_up(L.FN) * (size_t)L.count;
            launches.push_back(L);
        }
    }
    const size_t ncs = std::max<size_t>(1, p->h_csys.size());
    if (p->d_csys.bytes < sizeof(int32_t) * ncs) QCP_TRY(p->d_csys.alloc(sizeof(int32_t) * ncs));
    const bool diag = p->view_precond == QCP_PRECOND_DIAG;
    if (diag) QCP_TRY(refresh_diag<T>(p, lay));
    const bool use_df = lay->df_ok && (!diag || lay->diag_df_ok) && opts.engine != QCP_ENGINE_CLUSTER_FP64;
    if (!use_df && (p->kpsd || p->ndense)) {
        set_error("the FP64 cluster kernel applies D Pi to zero, R+ and SOC blocks only");
        return QCP_ERR_ARG;
    }
    if (!use_df && opts.solver == 1) {
        set_error("the FP64 cluster kernel runs LSQR only");
        return QCP_ERR_ARG;
    }
    if (use_df && p->d_bcast.bytes < bneed) QCP_TRY(p->d_bcast.alloc(bneed));
    QCP_CUDA(cudaMemcpyAsync(p->d_csys.p, p->h_csys.data(), sizeof(int32_t) * p->h_csys.size(),
                             cudaMemcpyHostToDevice, st));
    bool forked = false;
    for (const Launch& L : launches)
        if (L.seg > 0) forked = true;
    if (forked && !p->aux_stream) {
        QCP_CUDA(cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking));
        QCP_CUDA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
        QCP_CUDA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    }
    QCP_CUDA(cudaEventRecord(p->ev0, st));
    if (forked) {
        QCP_CUDA(cudaEventRecord(p->ev_fork, st));
        QCP_CUDA(cudaStreamWaitEvent(p->aux_stream, p->ev_fork, 0));
    }
    if (!use_df) p->last_engine = QCP_ENGINE_CLUSTER_FP64;
    for (const Launch& L : launches) {
        const int C = L.C;
        const size_t bytes = use_df ? L.bytesdf : L.bytes64;
        const int mode = segs[L.seg].mode;
        PlanView<T> vs = v;
        vs.active = p->d_active.as<int>() + segs[L.seg].seg;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(L.count * C));
        cfg.blockDim = dim3(kCThreads);
        cfg.dynamicSmemBytes = bytes;
        cfg.stream = L.seg == 0 ? st : p->aux_stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ClusterArgs ca;
        ca.cprob = lay->d_cprob.as<ClusterProb>();
        ca.slices = lay->d_slices.as<SellSlice>();
        ca.perm = lay->d_perm.as<int32_t>();
        ca.scol = lay->d_scol.as<int32_t>();
        ca.sval = lay->d_sval.p;
        ca.svalG = diag ? lay->d_svalDG.p : lay->d_svalG.p;
        ca.svalT = diag ? lay->d_sval.p : lay->d_svalT.p;
        ca.sys_list = p->d_csys.as<int32_t>() + L.start;
        ca.C = C;
        ca.FN = L.FN;
        ca.L = L.L;
        ca.NB = L.NB;
        ca.max_passes = 2 * (opts.maxiter + 2);
        if (use_df) {
            ClusterDfArgs da;
            da.bhalf = even_up(L.FN);
            da.bcast = reinterpret_cast<df*>(static_cast<unsigned char*>(p->d_bcast.p) + L.boff);
            da.sval = lay->d_dsval.as<df>();
            da.svalG = diag ? lay->d_dsvalDG.as<df>() : lay->d_dsvalG.as<df>();
            da.svalT = diag ? lay->d_dsval.as<df>() : lay->d_dsvalT.as<df>();
            da.cA = lay->d_dcA.as<df>();
            da.cB = lay->d_dcB.as<df>();
            da.rw = diag ? lay->d_drwD.as<df>() : lay->d_drw.as<df>();
            da.cd = diag ? lay->d_dcdD.as<df>() : lay->d_dcd.as<df>();
            da.zy = lay->d_dzy.as<df>();
            da.soc = lay->d_dsoc.as<SocDf>();
            const bool dense = p->kpsd || p->ndense;
            da.dense = dense ? p->d_dpi.as<df>() : nullptr;
            da.doff = dense ? p->d_dpi_off.as<int64_t>() : nullptr;
            const bool ls = opts.solver == 1;
            auto fn = mode == 0 ? cluster_kernel_df<0, T>(vs.scaled != 0, ls) : cluster_kernel_df<1, T>(vs.scaled != 0, ls);
            QCP_TRY(prepare_launch(fn, C, bytes, cfg));
            QCP_CUDA(cudaLaunchKernelEx(&cfg, fn, vs, ca, da));
        } else {
            auto fn = mode == 0 ? cluster_kernel<0, T>(vs.scaled != 0) : cluster_kernel<1, T>(vs.scaled != 0);
            QCP_TRY(prepare_launch(fn, C, bytes, cfg));
            QCP_CUDA(cudaLaunchKernelEx(&cfg, fn, vs, ca));
        }
        p->last_launches += 1;
    }
    if (forked) {
        QCP_CUDA(cudaEventRecord(p->ev_join, p->aux_stream));
        QCP_CUDA(cudaStreamWaitEvent(st, p->ev_join, 0));
    }
    QCP_CUDA(cudaEventRecord(p->ev1, st));
    QCP_CUDA(cudaEventSynchronize(p->ev1));
    float ms = 0.0f;
    QCP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    p->pass_ms += ms;
    return QCP_OK;
}
template int iterate_cluster<double>(qcp_plan*, const ClusterSeg*, int, int, const PlanView<double>&,
                                     const qcp_options&);
template int iterate_cluster<float>(qcp_plan*, const ClusterSeg*, int, int, const PlanView<float>&,
                                    const qcp_options&);

}  // namespace qcpd
