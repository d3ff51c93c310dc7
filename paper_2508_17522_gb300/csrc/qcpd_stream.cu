// Host side of the stream engine (see qcpd_stream.cuh): the plan's warp
// units, the df64 copies of M and of the per-row data, and the iteration
// loop (two launches per LSQR iteration, replayed from CUDA graphs in chunks
// of check_every iterations, as the pass engine does).
#include <algorithm>
#include <cstring>
#include <numeric>

#include "qcpd_stream.cuh"
#include "qcpd_stream.h"

namespace qcpd {

namespace {

constexpr double kSDfMin = 0x1p-90, kSDfMax = 0x1p90;

__device__ __forceinline__ bool s_df_unsafe(double x) {
    const double a = fabs(x);
    return !(a == 0.0 || (a >= kSDfMin && a <= kSDfMax));
}

template <typename T>
__device__ __forceinline__ void s_put(int64_t slot, int64_t src, const int32_t* mcol, const T* mval, const T* mvalG,
                                      const T* mvalT, int32_t* scol, df* val, df* valG, df* valT, int* bad) {
    const double v = (double)mval[src], g = (double)mvalG[src], t = (double)mvalT[src];
    if (s_df_unsafe(v) || s_df_unsafe(g) || s_df_unsafe(t)) atomicExch(bad, 1);
    scol[slot] = mcol[src];
    val[slot] = df_from(v);
    valG[slot] = df_from(g);
    valT[slot] = df_from(t);
}

__device__ __forceinline__ void s_pad(int64_t slot, int32_t col, int32_t* scol, df* val, df* valG, df* valT) {
    scol[slot] = col;
    val[slot] = df_zero();
    valG[slot] = df_zero();
    valT[slot] = df_zero();
}

// Slots of one SELL-32 sub-slice: this lane holds entries k G + sub
// (k < width) of `row`, then padding that repeats the row's last column.
template <typename T>
__device__ __forceinline__ void s_fill_slice(int64_t base, int width, int row, int G, int sub, const int64_t* rp,
                                             const int32_t* mcol, const T* mval, const T* mvalG, const T* mvalT,
                                             int32_t* scol, df* val, df* valG, df* valT, int* bad) {
    const int lane = threadIdx.x & 31;
    int64_t k0 = 0, len = 0;
    if (row >= 0) {
        k0 = rp[row];
        len = rp[row + 1] - k0;
    }
    const int32_t last = len > 0 ? mcol[k0 + len - 1] : 0;
    for (int k = 0; k < width; ++k) {
        const int64_t slot = base + 32 * (int64_t)k + lane;
        const int64_t e = (int64_t)k * G + sub;
        if (e < len) s_put(slot, k0 + e, mcol, mval, mvalG, mvalT, scol, val, valG, valT, bad);
        else s_pad(slot, last, scol, val, valG, valT);
    }
}

// One warp per unit.
template <typename T>
__global__ void k_stream_fill(const StreamUnit* units, int nunits, const int32_t* rows, const Prob* probs,
                              const int64_t* mrowptr, const int32_t* mcol, const T* mval, const T* mvalG,
                              const T* mvalT, int32_t* scol, df* val, df* valG, df* valT, int* bad) {
    const int lane = threadIdx.x & 31;
    const int64_t ui = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (ui >= nunits) return;
    const StreamUnit u = units[ui];
    const int64_t* rp = mrowptr + probs[u.prob].mrow;
    if (u.kind == SU_SLICE) {
        const int G = u.chunk;
        s_fill_slice(u.base, u.width, rows[u.aux + lane / G], G, lane & (G - 1), rp, mcol, mval, mvalG, mvalT, scol,
                     val, valG, valT, bad);
    } else if (u.kind == SU_SOCP) {
        s_fill_slice(u.base, u.width, rows[u.aux + lane], 1, 0, rp, mcol, mval, mvalG, mvalT, scol, val, valG, valT,
                     bad);
    } else if (u.kind == SU_SOCB) {
        int64_t base = u.base;
        for (int j = 0; j < u.width; ++j) {
            const int w = rows[u.aux + j];
            const int i = 32 * j + lane;
            s_fill_slice(base, w, i < u.nrows ? u.row0 + i : -1, 1, 0, rp, mcol, mval, mvalG, mvalT, scol, val, valG,
                         valT, bad);
            base += 32 * (int64_t)w;
        }
    } else {
        const int64_t k0 = rp[u.aux] + (int64_t)u.chunk * kSLongChunk;
        for (int k = lane; k < u.width; k += 32)
            s_put(u.base + k, k0 + k, mcol, mval, mvalG, mvalT, scol, val, valG, valT, bad);
    }
}

__global__ void k_stream_todf(const double* in, int64_t n, df* out, int* bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (s_df_unsafe(in[i])) atomicExch(bad, 1);
        out[i] = df_from(in[i]);
    }
}

// A stored D Pi entry as df64: entries below the double-float range are
// dropped (D Pi is nonexpansive, so they are far below the others), entries
// above it make the plan unusable for the engine.
__device__ __forceinline__ df s_dense_entry(double v, int* bad) {
    if (fabs(v) < kSDfMin) return df_zero();
    if (s_df_unsafe(v)) atomicExch(bad, 1);
    return df_from(v);
}

// The dense D Pi of every exponential, power and PSD block (doff[b] >= 0),
// row-major at out + doff[b] as df64 pairs: exponential and power blocks copy
// their stored 3 x 3; a PSD block (order <= 22) applies its
// V (B o (V^T dZ V)) V^T to each unit vector of its entries, one column at a
// time (apply_D_psd, the pass engine's map).  One CTA per block.
__global__ void k_stream_dense(const SocBlock* blk, int64_t nb, const int64_t* doff, const double* psd, df* out,
                               int* bad) {
    __shared__ double src[kSSocBig], dst[kSSocBig], scr[2 * 22 * 22];
    const int64_t b = blockIdx.x;
    if (b >= nb || doff[b] < 0) return;
    const SocBlock B = blk[b];
    const int d = B.dim;
    df* D = out + doff[b];
    if (B.kase == kBlockDense) {
        for (int e = threadIdx.x; e < d * d; e += blockDim.x) D[e] = s_dense_entry(psd[B.psd + e], bad);
        return;
    }
    if (B.kase != kBlockPsd || B.order > 22) {
        if (threadIdx.x == 0) atomicExch(bad, 1);
        return;
    }
    for (int c = 0; c < d; ++c) {
        for (int i = threadIdx.x; i < d; i += blockDim.x) src[i] = i == c ? 1.0 : 0.0;
        __syncthreads();
        apply_D_psd(src, dst, B.start, blk, (int)b, (int)b + 1, psd, scr);
        for (int i = threadIdx.x; i < d; i += blockDim.x) D[(int64_t)i * d + c] = s_dense_entry(dst[i], bad);
        __syncthreads();
    }
}

__global__ void k_stream_soc(const SocBlock* blk, int64_t nb, const int64_t* doff, StreamSoc* out, int* bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
        const SocBlock B = blk[i];
        StreamSoc s;
        if (doff[i] >= 0) {  // a stored dense D Pi
            s.r = s.h = s.tq = s.htr = df_zero();
            s.start = B.start;
            s.dim = B.dim;
            s.kase = kSDense;
            s.pad = (int32_t)doff[i];
            out[i] = s;
            continue;
        }
        const double htr = B.h * (B.t + B.r);
        if (B.kase == 2 && (s_df_unsafe(B.r) || s_df_unsafe(B.h) || s_df_unsafe(B.tq) || s_df_unsafe(htr)))
            atomicExch(bad, 1);
        s.r = df_from(B.r);
        s.h = df_from(B.h);
        s.tq = df_from(B.tq);
        s.htr = df_from(htr);
        s.start = B.start;
        s.dim = B.dim;
        s.kase = B.kase;
        s.pad = 0;
        out[i] = s;
    }
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(4096, (n + 255) / 256)); }

}  // namespace

// ---------------------------------------------------------------------------
// Layout.  Per problem: x-rows and zero-cone / R+ rows with at most
// kSLongChunk entries in SELL-32 slices of G lanes per row (x and y apart,
// each sorted by length, longest first, one G per slice); longer rows in
// chunks of kSLongChunk entries;
// second-order-cone blocks of at most 32 rows packed in order into units of
// at most 32 rows, larger ones (up to kSSocBig rows) one unit each.  Units
// are sorted by their per-lane chain of dependent loads (plus a share for
// the epilogue), longest first, for the kernel's snake order.
static bool build_units(const qcp_plan* p, StreamLayout* lay, std::vector<StreamUnit>& hu,
                        std::vector<int32_t>& hrows, std::vector<int32_t>& hlblk, int64_t& slots) {
    slots = 0;
    auto take = [&](int64_t n) {
        const int64_t b = (slots + 31) & ~(int64_t)31;  // every unit starts on a 32-slot boundary
        slots = b + n;
        return b;
    };
    lay->huoff.assign(1, 0);
    lay->hsoff.assign(1, 0);
    lay->nsplit = lay->nslot = 0;
    lay->max_units = 0;
    for (int pi = 0; pi < p->nprob; ++pi) {
        const Prob& pr = p->hprob[pi];
        const int64_t* rp = p->h_mrowptr.data() + pr.mrow;
        auto len = [&](int r) { return (int)(rp[r + 1] - rp[r]); };
        std::vector<int> xs, ys, longs;
        struct Blk { int start, dim, idx; };
        std::vector<Blk> socs;
        for (int r = 0; r < pr.n; ++r) (len(r) <= kSLongChunk ? xs : longs).push_back(r);
        int row = pr.n, bi = 0;
        for (size_t b = 0; b < p->cone_type[pi].size(); ++b) {
            const int t = p->cone_type[pi][b], d = p->cone_dim[pi][b];
            if (t == QCP_CONE_ZERO || t == QCP_CONE_NONNEG) {
                for (int k = 0; k < d; ++k) (len(row + k) <= kSLongChunk ? ys : longs).push_back(row + k);
            } else {  // a coupled block: second-order, PSD, exponential or power cone
                if (d > kSSocBig) {
                    lay->why = "a second-order-cone or PSD block has more than 256 rows";
                    return false;
                }
                socs.push_back({row, d, bi++});
            }
            row += d;
        }
        std::vector<StreamUnit> pu;
        std::vector<double> cost;
        // G lanes per row: the smallest power of two that leaves a lane at
        // most kSSteps entries; one slice holds 32 / G rows of one G
        auto lanes_for = [&](int L) {
            int G = 1;
            while (G < 32 && (L + G - 1) / G > kSSteps) G <<= 1;
            return G;
        };
        auto slice_units = [&](std::vector<int>& rows) {
            std::stable_sort(rows.begin(), rows.end(), [&](int a, int b) { return len(a) > len(b); });
            for (int G = 32; G >= 1; G >>= 1) {
                std::vector<int> cls;
                for (int r : rows)
                    if (lanes_for(len(r)) == G) cls.push_back(r);
                const int R = 32 / G;
                for (size_t i = 0; i < cls.size(); i += R) {
                    const int nr = (int)std::min<size_t>(R, cls.size() - i);
                    StreamUnit u{};
                    u.kind = SU_SLICE;
                    u.prob = pi;
                    u.nrows = nr;
                    u.chunk = G;
                    u.width = (len(cls[i]) + G - 1) / G;
                    u.aux = (int32_t)hrows.size();
                    for (int l = 0; l < 32; ++l) {
                        hrows.push_back(l < nr ? cls[i + l] : -1);
                        hlblk.push_back(-1);
                    }
                    u.base = take(32 * (int64_t)u.width);
                    pu.push_back(u);
                    cost.push_back(u.width + 3.0);
                }
            }
        };
        slice_units(xs);
        slice_units(ys);
        for (size_t i = 0; i < socs.size();) {
            StreamUnit u{};
            u.prob = pi;
            if (socs[i].dim > 32) {
                const Blk B = socs[i++];
                u.kind = SU_SOCB;
                u.nrows = B.dim;
                u.width = (B.dim + 31) / 32;
                u.blk = B.idx;
                u.row0 = B.start;
                u.aux = (int32_t)hrows.size();
                int64_t tot = 0;
                for (int j = 0; j < u.width; ++j) {
                    int w = 0;
                    for (int r = B.start + 32 * j; r < std::min(B.start + B.dim, B.start + 32 * j + 32); ++r)
                        w = std::max(w, len(r));
                    hrows.push_back(w);
                    hlblk.push_back(-1);
                    tot += w;
                }
                u.base = take(32 * tot);
                pu.push_back(u);
                cost.push_back(tot + 6.0);
                continue;
            }
            // consecutive blocks of at most 32 rows in all, one row per lane
            size_t j = i;
            int total = 0;
            while (j < socs.size() && socs[j].dim <= 32 && total + socs[j].dim <= 32) total += socs[j++].dim;
            u.kind = SU_SOCP;
            u.nrows = total;
            u.aux = (int32_t)hrows.size();
            int w = 0, lane = 0;
            for (size_t b = i; b < j; ++b)
                for (int k = 0; k < socs[b].dim; ++k, ++lane) {
                    hrows.push_back(socs[b].start + k);
                    hlblk.push_back(socs[b].idx);
                    w = std::max(w, len(socs[b].start + k));
                }
            for (; lane < 32; ++lane) {
                hrows.push_back(-1);
                hlblk.push_back(-1);
            }
            u.width = w;
            u.base = take(32 * (int64_t)w);
            pu.push_back(u);
            cost.push_back(w + 5.0);
            i = j;
        }
        for (int r : longs) {
            const int L = len(r);
            const int nch = (L + kSLongChunk - 1) / kSLongChunk;
            int split = -1, slot0 = 0;
            if (nch > 1) {
                split = lay->nsplit++;
                slot0 = lay->nslot;
                lay->nslot += nch;
            }
            for (int c = 0; c < nch; ++c) {
                StreamUnit u{};
                u.kind = SU_LONG;
                u.prob = pi;
                u.nrows = nch;
                u.width = std::min(kSLongChunk, L - c * kSLongChunk);
                u.aux = r;
                u.blk = split;
                u.chunk = c;
                u.row0 = slot0;
                u.base = take(u.width);
                pu.push_back(u);
                cost.push_back((u.width + 31) / 32 + 4.0);
            }
        }
        std::vector<int> ord(pu.size());
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        for (int o : ord) hu.push_back(pu[o]);
        lay->huoff.push_back((int32_t)hu.size());
        lay->hsoff.push_back(lay->nsplit);
        lay->max_units = std::max(lay->max_units, (int)pu.size());
    }
    return true;
}

int dense_dpi_ready(qcp_plan* p, bool* ok) {
    if (p->dpi_state == 0) {
        std::vector<int64_t> hoff((size_t)std::max<int64_t>(p->nsoc_tot, 1), -1);
        int64_t total = 0;
        bool fit = true;
        for (int pi = 0; pi < p->nprob; ++pi) {
            int64_t bi = p->hprob[pi].soff;
            for (size_t c = 0; c < p->cone_type[pi].size(); ++c) {
                const int t = p->cone_type[pi][c], d = p->cone_dim[pi][c];
                if (t == QCP_CONE_ZERO || t == QCP_CONE_NONNEG) continue;
                if (t != QCP_CONE_SOC) {
                    if (d > kSSocBig) fit = false;
                    hoff[bi] = total;
                    total += (int64_t)d * d;
                }
                ++bi;
            }
        }
        p->dpi_state = -1;
        if (!fit) {
            p->dpi_why = "a PSD block has more than 256 entries (order above 22)";
        } else if (total > (int64_t)1 << 28) {
            p->dpi_why = "the dense D Pi of the exponential, power and PSD blocks would exceed 2 GB";
        } else {
            cudaStream_t st = p->stream;
            QCP_TRY(p->d_dpi_off.alloc(sizeof(int64_t) * hoff.size()));
            QCP_CUDA(cudaMemcpyAsync(p->d_dpi_off.p, hoff.data(), sizeof(int64_t) * hoff.size(),
                                     cudaMemcpyHostToDevice, st));
            QCP_TRY(p->d_dpi.alloc(sizeof(df) * (size_t)std::max<int64_t>(total, 1)));
            DevBuf bad;
            QCP_TRY(bad.alloc(sizeof(int)));
            QCP_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
            if (total > 0)
                k_stream_dense<<<(unsigned)p->nsoc_tot, 128, 0, st>>>(p->d_blocks.as<SocBlock>(), p->nsoc_tot,
                                                                      p->d_dpi_off.as<int64_t>(),
                                                                      p->d_psd.as<double>(), p->d_dpi.as<df>(),
                                                                      bad.as<int>());
            QCP_CUDA(cudaGetLastError());
            int hbad = 1;
            QCP_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            QCP_CUDA(cudaStreamSynchronize(st));
            if (hbad == 0) p->dpi_state = 1;
            else p->dpi_why = "an entry of a stored D Pi lies above the double-float range";
        }
    }
    *ok = p->dpi_state > 0;
    return QCP_OK;
}

template <typename T>
static int build_stream(qcp_plan* p, StreamLayout* lay) {
    std::vector<StreamUnit> hu;
    std::vector<int32_t> hrows, hlblk;
    int64_t slots = 0;
    if (!build_units(p, lay, hu, hrows, hlblk, slots)) return QCP_OK;  // not usable: lay->ok stays false
    lay->nunits = (int)hu.size();
    cudaStream_t st = p->stream;
    auto up = [&](DevBuf& d, const void* h, size_t bytes) -> int {
        QCP_TRY(d.alloc(bytes));
        if (bytes) QCP_CUDA(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, st));
        return QCP_OK;
    };
    QCP_TRY(up(lay->d_units, hu.data(), sizeof(StreamUnit) * hu.size()));
    QCP_TRY(up(lay->d_uoff, lay->huoff.data(), sizeof(int32_t) * lay->huoff.size()));
    QCP_TRY(up(lay->d_soff, lay->hsoff.data(), sizeof(int32_t) * lay->hsoff.size()));
    QCP_TRY(up(lay->d_rows, hrows.data(), sizeof(int32_t) * hrows.size()));
    QCP_TRY(up(lay->d_lblk, hlblk.data(), sizeof(int32_t) * hlblk.size()));
    const int64_t ns = std::max<int64_t>(slots, 1);
    QCP_TRY(lay->d_scol.alloc(sizeof(int32_t) * ns));
    QCP_TRY(lay->d_val.alloc(sizeof(df) * ns));
    QCP_TRY(lay->d_valG.alloc(sizeof(df) * ns));
    QCP_TRY(lay->d_valT.alloc(sizeof(df) * ns));
    DevBuf bad;
    QCP_TRY(bad.alloc(sizeof(int)));
    QCP_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    int* b = bad.as<int>();
    if (!hu.empty())
        k_stream_fill<T><<<(unsigned)((hu.size() * 32 + 255) / 256), 256, 0, st>>>(
            lay->d_units.as<StreamUnit>(), (int)hu.size(), lay->d_rows.as<int32_t>(), p->d_prob.as<Prob>(),
            p->d_mrowptr.as<int64_t>(), p->d_mcol.as<int32_t>(), p->d_mval.as<T>(), p->d_mvalG.as<T>(),
            p->d_mvalT.as<T>(), lay->d_scol.as<int32_t>(), lay->d_val.as<df>(), lay->d_valG.as<df>(),
            lay->d_valT.as<df>(), b);
    auto todf = [&](const DevBuf& in, DevBuf& out) -> int {
        QCP_TRY(out.alloc(sizeof(df) * (size_t)std::max<int64_t>(p->N_tot, 1)));
        k_stream_todf<<<grid_of(p->N_tot), 256, 0, st>>>(in.as<double>(), p->N_tot, out.as<df>(), b);
        return QCP_OK;
    };
    QCP_TRY(todf(p->d_coefA, lay->d_cA));
    QCP_TRY(todf(p->d_coefB, lay->d_cB));
    QCP_TRY(todf(p->d_rw, lay->d_rw));
    QCP_TRY(todf(p->d_cd, lay->d_cd));
    QCP_TRY(todf(p->d_zy, lay->d_zy));
    // the coupled blocks' constants; exponential, power and PSD blocks get
    // their dense D Pi (plan-wide, shared with the cluster engine)
    bool dok = true;
    if (p->kpsd || p->ndense) QCP_TRY(dense_dpi_ready(p, &dok));
    if (!dok) {
        lay->why = p->dpi_why;
        return QCP_OK;
    }
    if (!p->d_dpi_off.p) {  // no such blocks: every offset -1
        std::vector<int64_t> none((size_t)std::max<int64_t>(p->nsoc_tot, 1), -1);
        QCP_TRY(up(p->d_dpi_off, none.data(), sizeof(int64_t) * none.size()));
    }
    QCP_TRY(lay->d_soc.alloc(sizeof(StreamSoc) * (size_t)std::max<int64_t>(p->nsoc_tot, 1)));
    if (p->nsoc_tot > 0)
        k_stream_soc<<<grid_of(p->nsoc_tot), 256, 0, st>>>(p->d_blocks.as<SocBlock>(), p->nsoc_tot,
                                                            p->d_dpi_off.as<int64_t>(), lay->d_soc.as<StreamSoc>(), b);
    QCP_CUDA(cudaGetLastError());
    // per-system workspace: CTAs per system up to the number resident at once
    int dev = 0, nsm = 0, occ = 0;
    QCP_CUDA(cudaGetDevice(&dev));
    QCP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    QCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_stream<PASS_GT, ROLE_V, true>, kSThreads, 0));
    lay->gmax = std::max(1, nsm * std::max(occ, 1));
    QCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_stream2<PASS_GT, true>, kSThreads, 0));
    lay->gmax2 = std::max(1, std::min(lay->gmax, nsm * std::max(occ, 1)));
    const int64_t nsys = std::max(1, p->nsys_cap);
    const int64_t per = p->batched ? 1 : nsys;  // split-row storage: per system unless each system is a problem
    QCP_TRY(lay->d_scal.alloc(sizeof(StreamScal) * nsys));
    QCP_TRY(lay->d_ssys.alloc(sizeof(StreamSys) * nsys));
    QCP_CUDA(cudaMemsetAsync(lay->d_ssys.p, 0, sizeof(StreamSys) * nsys, st));
    QCP_TRY(lay->d_cpart.alloc(2 * sizeof(float4) * nsys * lay->gmax));
    QCP_TRY(lay->d_ccnt.alloc(sizeof(int32_t) * nsys));
    QCP_CUDA(cudaMemsetAsync(lay->d_ccnt.p, 0, sizeof(int32_t) * nsys, st));
    QCP_TRY(lay->d_lchunk.alloc(sizeof(df) * per * std::max(1, lay->nslot)));
    QCP_TRY(lay->d_lcnt.alloc(sizeof(int32_t) * per * std::max(1, lay->nsplit)));
    QCP_CUDA(cudaMemsetAsync(lay->d_lcnt.p, 0, sizeof(int32_t) * per * std::max(1, lay->nsplit), st));
    QCP_TRY(lay->d_lrow.alloc(sizeof(df) * 3 * per * std::max(1, lay->nsplit)));
    QCP_TRY(lay->d_slist.alloc(sizeof(int32_t) * nsys));
    QCP_TRY(lay->d_scount.alloc(sizeof(int32_t)));
    QCP_TRY(lay->d_pshared.alloc(sizeof(unsigned long long)));
    int hbad = 1;
    QCP_CUDA(cudaMemcpyAsync(&hbad, b, sizeof(int), cudaMemcpyDeviceToHost, st));
    QCP_CUDA(cudaStreamSynchronize(st));
    lay->ok = hbad == 0;
    if (!lay->ok) lay->why = "a magnitude in the data lies outside the double-float range 2^-90..2^90";
    return QCP_OK;
}

int stream_ready(qcp_plan* p, bool* ok) {
    if (!p->stream_lay) {
        auto lay = std::make_unique<StreamLayout>();
        QCP_TRY(p->dtype == QCP_F64 ? build_stream<double>(p, lay.get()) : build_stream<float>(p, lay.get()));
        p->stream_lay = std::move(lay);
    }
    *ok = p->stream_lay->ok;
    if (!*ok) set_error("stream engine: %s", p->stream_lay->why.c_str());
    return QCP_OK;
}

// ---------------------------------------------------------------------------
// Iterations.
static StreamArgs stream_args(qcp_plan* p, const StreamLayout* lay, int scaled) {
    StreamArgs a{};
    a.units = lay->d_units.as<StreamUnit>();
    a.uoff = lay->d_uoff.as<int32_t>();
    a.soff = lay->d_soff.as<int32_t>();
    a.rows = lay->d_rows.as<int32_t>();
    a.lblk = lay->d_lblk.as<int32_t>();
    a.scol = lay->d_scol.as<int32_t>();
    a.valG = scaled ? lay->d_valG.as<df>() : lay->d_val.as<df>();
    a.valT = scaled ? lay->d_valT.as<df>() : lay->d_val.as<df>();
    a.cA = lay->d_cA.as<df>();
    a.cB = lay->d_cB.as<df>();
    a.rw = lay->d_rw.as<df>();
    a.cd = lay->d_cd.as<df>();
    a.zy = lay->d_zy.as<df>();
    a.flag = p->d_flag.as<int8_t>();
    a.soc = lay->d_soc.as<StreamSoc>();
    a.dense = p->d_dpi.as<df>();
    a.rwd = p->d_rw.as<double>();
    a.cdd = p->d_cd.as<double>();
    a.sys = p->d_sys.as<Sys>();
    a.probs = p->d_prob.as<Prob>();
    a.state = p->d_state.as<LsqrState>();
    a.scal = lay->d_scal.as<StreamScal>();
    a.ssys = lay->d_ssys.as<StreamSys>();
    a.U = reinterpret_cast<df*>(p->d_U.p);
    a.V = reinterpret_cast<df*>(p->d_V.p);
    a.W = reinterpret_cast<df*>(p->d_W.p);
    a.X = reinterpret_cast<df*>(p->d_X.p);
    a.XI = reinterpret_cast<df*>(p->d_XI.p);
    a.HB = reinterpret_cast<df*>(p->d_HB.p);
    a.cpart = lay->d_cpart.as<float4>();
    a.ccnt = lay->d_ccnt.as<int32_t>();
    a.lchunk = lay->d_lchunk.as<df>();
    a.lcnt = lay->d_lcnt.as<int32_t>();
    a.lrow = lay->d_lrow.as<df>();
    a.nsplit = lay->nsplit;
    a.nslot = lay->nslot;
    a.batched = p->batched ? 1 : 0;
    return a;
}

template <bool SC>
static void launch_stream_iter_sc(int mode, const StreamArgs& a, int ns, cudaStream_t st) {
    const dim3 grid((unsigned)a.gx, (unsigned)ns);
    if (mode == 0) {
        k_stream<PASS_G, ROLE_U, SC><<<grid, kSThreads, 0, st>>>(a);
        k_stream<PASS_GT, ROLE_V, SC><<<grid, kSThreads, 0, st>>>(a);
    } else {
        k_stream<PASS_GT, ROLE_U, SC><<<grid, kSThreads, 0, st>>>(a);
        k_stream<PASS_G, ROLE_V, SC><<<grid, kSThreads, 0, st>>>(a);
    }
}

static void launch_stream_iter(int mode, const StreamArgs& a, int ns, bool scaled, cudaStream_t st) {
    if (scaled) launch_stream_iter_sc<true>(mode, a, ns, st);
    else launch_stream_iter_sc<false>(mode, a, ns, st);
}

static int run_stream_chunk(qcp_plan* p, int mode, int s0, int ns, const StreamArgs& a, bool scaled, int chunk,
                            bool use_graph) {
    // ns: the systems in a.slist this chunk (graphs are kept per count: the
    // list's contents change between chunks, the launch shape does not)
    cudaStream_t st = p->stream;
    if (!use_graph || chunk < 2) {
        for (int c = 0; c < chunk; ++c) launch_stream_iter(mode, a, ns, scaled, st);
        QCP_CUDA(cudaGetLastError());
        p->last_launches += 2 * chunk;
        return QCP_OK;
    }
    GraphKey key{QCP_ENGINE_STREAM, mode, s0, ns, chunk, scaled ? 1 : 0, a.lsmr};
    auto it = p->graphs.find(key);
    if (it == p->graphs.end()) {
        cudaGraph_t g = nullptr;
        QCP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int c = 0; c < chunk; ++c) launch_stream_iter(mode, a, ns, scaled, st);
        const cudaError_t le = cudaGetLastError();
        const cudaError_t ee = cudaStreamEndCapture(st, &g);
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            set_error("graph capture failed: %s", cudaGetErrorString(le != cudaSuccess ? le : ee));
            return QCP_ERR_CUDA;
        }
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            set_error("graph instantiation failed: %s", cudaGetErrorString(ie));
            return QCP_ERR_CUDA;
        }
        it = p->graphs.emplace(key, ge).first;
    }
    QCP_CUDA(cudaGraphLaunch(it->second, st));
    p->last_launches += 2 * chunk;
    return QCP_OK;
}

int iterate_stream(qcp_plan* p, int mode, int s0, int ns, int* active, bool scaled, const qcp_options& opts) {
    const StreamLayout* lay = p->stream_lay.get();
    if (!lay || !lay->ok) {
        set_error("stream engine: the plan's layout is not usable");
        return QCP_ERR_ARG;
    }
    StreamArgs a = stream_args(p, lay, scaled ? 1 : 0);
    a.lsmr = opts.solver == 1 ? 1 : 0;
    a.s0 = s0;
    a.active = active;
    a.slist = lay->d_slist.as<int32_t>();
    a.gstride = lay->gmax;
    cudaStream_t st = p->stream;
    int maxN = 1;
    for (int s = s0; s < s0 + ns; ++s) {
        const Prob& pr = p->hprob[p->hsys[s].prob];
        maxN = std::max(maxN, pr.n + pr.m + 1);
    }
    const dim3 vgrid((unsigned)std::min(1024, (maxN + 255) / 256), (unsigned)ns);
    k_stream_enter_state<<<ns, 32, 0, st>>>(a, mode == 0 ? 1 : 0, scaled ? 1 : 0);
    k_stream_enter_vec<<<vgrid, 256, 0, st>>>(a);
    QCP_CUDA(cudaGetLastError());
    p->last_launches += 2;
    // The launches cover the range's systems still iterating (a device list,
    // rebuilt whenever the host's check sees fewer of them), and the GPU's
    // resident CTAs are shared among those: a system left alone gets them all.
    auto compact = [&](int* nact) -> int {
        k_stream_compact<<<1, 32, 0, st>>>(p->d_state.as<LsqrState>(), s0, ns, lay->d_slist.as<int32_t>(),
                                           lay->d_scount.as<int32_t>());
        QCP_CUDA(cudaGetLastError());
        QCP_CUDA(cudaMemcpyAsync(p->h_active, lay->d_scount.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        *nact = *p->h_active;
        p->last_launches += 1;
        return QCP_OK;
    };
    int nact = 0;
    QCP_TRY(compact(&nact));
    int64_t done = 0;
    const int64_t cap = opts.maxiter + 1;
    while (done < cap && nact > 0) {
        int gx = (lay->gmax + nact - 1) / nact;
        gx = std::min(gx, std::max(1, (lay->max_units + kSWarps - 1) / kSWarps));
        a.gx = std::max(1, gx);
        int64_t chunk = opts.check_every > 0 ? opts.check_every : cap;
        chunk = std::min<int64_t>(chunk, cap - done);
        const bool graph_ok = opts.use_graph && opts.check_every > 0 && chunk == opts.check_every;
        QCP_CUDA(cudaEventRecord(p->ev0, st));
        QCP_TRY(run_stream_chunk(p, mode, s0, nact, a, scaled, (int)chunk, graph_ok));
        QCP_CUDA(cudaEventRecord(p->ev1, st));
        done += chunk;
        p->pass_launches += 2 * chunk;
        if (opts.check_every > 0) {
            QCP_CUDA(cudaMemcpyAsync(p->h_active, active, sizeof(int), cudaMemcpyDeviceToHost, st));
            QCP_CUDA(cudaStreamSynchronize(st));
        } else {
            QCP_CUDA(cudaEventSynchronize(p->ev1));
        }
        float ms = 0.0f;
        QCP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->pass_ms += ms;
        if (opts.check_every > 0) {
            const int still = *p->h_active;
            if (still <= 0) break;
            if (still < nact) QCP_TRY(compact(&nact));
        }
    }
    k_stream_exit_vec<<<vgrid, 256, 0, st>>>(a);
    k_stream_exit_state<<<ns, 32, 0, st>>>(a);
    QCP_CUDA(cudaGetLastError());
    p->last_launches += 2;
    return QCP_OK;
}


// ---------------------------------------------------------------------------
// Paired iterations: a JVP range and a VJP range of equal size on one
// problem advance in step, the VJP systems one pass behind, so that every
// launch runs one product for both systems of each pair (k_stream2).
template <bool SC>
static void launch_stream_pair_iter_sc(const StreamArgs& a, int npairs, cudaStream_t st) {
    const dim3 grid((unsigned)a.gx, (unsigned)npairs);
    k_stream2<PASS_G, SC><<<grid, kSThreads, 0, st>>>(a);
    k_stream2<PASS_GT, SC><<<grid, kSThreads, 0, st>>>(a);
}

static void launch_stream_pair_iter(const StreamArgs& a, int npairs, bool scaled, cudaStream_t st) {
    if (scaled) launch_stream_pair_iter_sc<true>(a, npairs, st);
    else launch_stream_pair_iter_sc<false>(a, npairs, st);
}

static int run_stream_pair_chunk(qcp_plan* p, int sa0, int sb0, int npairs, const StreamArgs& a, bool scaled,
                                 int chunk, bool use_graph) {
    cudaStream_t st = p->stream;
    if (!use_graph || chunk < 2) {
        for (int c = 0; c < chunk; ++c) launch_stream_pair_iter(a, npairs, scaled, st);
        QCP_CUDA(cudaGetLastError());
        p->last_launches += 2 * chunk;
        return QCP_OK;
    }
    GraphKey key{QCP_ENGINE_STREAM, 2, sa0, npairs, chunk, scaled ? 1 : 0, a.lsmr, 1 + sb0};
    auto it = p->graphs.find(key);
    if (it == p->graphs.end()) {
        cudaGraph_t g = nullptr;
        QCP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int c = 0; c < chunk; ++c) launch_stream_pair_iter(a, npairs, scaled, st);
        const cudaError_t le = cudaGetLastError();
        const cudaError_t ee = cudaStreamEndCapture(st, &g);
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            set_error("graph capture failed: %s", cudaGetErrorString(le != cudaSuccess ? le : ee));
            return QCP_ERR_CUDA;
        }
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            set_error("graph instantiation failed: %s", cudaGetErrorString(ie));
            return QCP_ERR_CUDA;
        }
        it = p->graphs.emplace(key, ge).first;
    }
    QCP_CUDA(cudaGraphLaunch(it->second, st));
    p->last_launches += 2 * chunk;
    return QCP_OK;
}

bool stream_can_pair(const qcp_plan* p, int sa0, int sb0, int ns) {
    if (p->batched || ns <= 0) return false;
    for (int i = 0; i < ns; ++i)
        if (p->hsys[sa0 + i].prob != p->hsys[sb0 + i].prob) return false;
    return true;
}

int iterate_stream_pair(qcp_plan* p, int sa0, int sb0, int ns, int* active_a, int* active_b, bool scaled,
                        const qcp_options& opts) {
    const StreamLayout* lay = p->stream_lay.get();
    if (!lay || !lay->ok) {
        set_error("stream engine: the plan's layout is not usable");
        return QCP_ERR_ARG;
    }
    StreamArgs a = stream_args(p, lay, scaled ? 1 : 0);
    a.lsmr = opts.solver == 1 ? 1 : 0;
    a.active = active_a;
    a.active2 = active_b;
    a.pshared = lay->d_pshared.as<unsigned long long>();
    a.slist = lay->d_slist.as<int32_t>();
    a.gstride = lay->gmax;
    cudaStream_t st = p->stream;
    int maxN = 1;
    for (int i = 0; i < ns; ++i)
        for (int s : {sa0 + i, sb0 + i}) {
            const Prob& pr = p->hprob[p->hsys[s].prob];
            maxN = std::max(maxN, pr.n + pr.m + 1);
        }
    const dim3 vgrid((unsigned)std::min(1024, (maxN + 255) / 256), (unsigned)ns);
    a.s0 = sa0;
    k_stream_enter_state<<<ns, 32, 0, st>>>(a, 1, scaled ? 1 : 0);  // JVP: the first u-pass is a G-pass
    k_stream_enter_vec<<<vgrid, 256, 0, st>>>(a);
    a.s0 = sb0;
    k_stream_enter_state<<<ns, 32, 0, st>>>(a, 0, scaled ? 1 : 0);  // VJP: a G^T-pass
    k_stream_enter_vec<<<vgrid, 256, 0, st>>>(a);
    QCP_CUDA(cudaMemsetAsync(lay->d_pshared.p, 0, sizeof(unsigned long long), st));
    QCP_CUDA(cudaGetLastError());
    p->last_launches += 4;
    auto sync_read = [&](const void* src, int n) -> int {
        QCP_CUDA(cudaMemcpyAsync(p->h_active, src, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        return QCP_OK;
    };
    auto grid_x = [&](int nunits, int gmax) {
        int gx = (gmax + nunits - 1) / nunits;
        return std::max(1, std::min(gx, std::max(1, (lay->max_units + kSWarps - 1) / kSWarps)));
    };
    // the VJP systems' first u-pass, alone: afterwards both ranges need the
    // same product at every launch
    k_stream_compact<<<1, 32, 0, st>>>(p->d_state.as<LsqrState>(), sb0, ns, lay->d_slist.as<int32_t>(),
                                       lay->d_scount.as<int32_t>());
    QCP_CUDA(cudaGetLastError());
    QCP_TRY(sync_read(lay->d_scount.p, 1));
    p->last_launches += 1;
    const int nb = p->h_active[0];
    if (nb > 0) {
        StreamArgs b = a;
        b.active = active_b;
        b.gx = grid_x(nb, lay->gmax);
        QCP_CUDA(cudaEventRecord(p->ev0, st));
        const dim3 grid((unsigned)b.gx, (unsigned)nb);
        if (scaled) k_stream<PASS_GT, ROLE_U, true><<<grid, kSThreads, 0, st>>>(b);
        else k_stream<PASS_GT, ROLE_U, false><<<grid, kSThreads, 0, st>>>(b);
        QCP_CUDA(cudaGetLastError());
        QCP_CUDA(cudaEventRecord(p->ev1, st));
        QCP_CUDA(cudaEventSynchronize(p->ev1));
        float ms = 0.0f;
        QCP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->pass_ms += ms;
        p->pass_launches += 1;
        p->last_launches += 1;
    }
    auto compact = [&](int* npairs) -> int {
        k_stream_compact2<<<1, 32, 0, st>>>(p->d_state.as<LsqrState>(), sa0, sb0, ns, lay->d_slist.as<int32_t>(),
                                            lay->d_scount.as<int32_t>());
        QCP_CUDA(cudaGetLastError());
        QCP_TRY(sync_read(lay->d_scount.p, 1));
        *npairs = p->h_active[0];
        p->last_launches += 1;
        return QCP_OK;
    };
    int npairs = 0;
    QCP_TRY(compact(&npairs));
    // active_a and active_b are adjacent counters (one per range of the call)
    const bool adjacent = active_b == active_a + 1;
    int live_a = ns, live_b = ns;
    int64_t done = 0;
    const int64_t cap = opts.maxiter + 1;
    while (done < cap && npairs > 0) {
        a.gx = grid_x(npairs, lay->gmax2);
        int64_t chunk = opts.check_every > 0 ? opts.check_every : cap;
        chunk = std::min<int64_t>(chunk, cap - done);
        const bool graph_ok = opts.use_graph && opts.check_every > 0 && chunk == opts.check_every;
        QCP_CUDA(cudaEventRecord(p->ev0, st));
        QCP_TRY(run_stream_pair_chunk(p, sa0, sb0, npairs, a, scaled, (int)chunk, graph_ok));
        QCP_CUDA(cudaEventRecord(p->ev1, st));
        done += chunk;
        p->pass_launches += 2 * chunk;
        int still_a = 0, still_b = 0;
        if (opts.check_every > 0) {
            if (adjacent) {
                QCP_TRY(sync_read(active_a, 2));
                still_a = p->h_active[0];
                still_b = p->h_active[1];
            } else {
                QCP_TRY(sync_read(active_a, 1));
                still_a = p->h_active[0];
                QCP_TRY(sync_read(active_b, 1));
                still_b = p->h_active[0];
            }
        } else {
            QCP_CUDA(cudaEventSynchronize(p->ev1));
        }
        float ms = 0.0f;
        QCP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->pass_ms += ms;
        if (opts.check_every > 0) {
            if (still_a <= 0 && still_b <= 0) break;
            if (still_a < live_a || still_b < live_b) QCP_TRY(compact(&npairs));
            live_a = still_a;
            live_b = still_b;
        }
    }
    unsigned long long shared = 0;
    QCP_CUDA(cudaMemcpyAsync(&shared, lay->d_pshared.p, sizeof(shared), cudaMemcpyDeviceToHost, st));
    a.s0 = sa0;
    k_stream_exit_vec<<<vgrid, 256, 0, st>>>(a);
    k_stream_exit_state<<<ns, 32, 0, st>>>(a);
    a.s0 = sb0;
    k_stream_exit_vec<<<vgrid, 256, 0, st>>>(a);
    k_stream_exit_state<<<ns, 32, 0, st>>>(a);
    QCP_CUDA(cudaGetLastError());
    QCP_CUDA(cudaStreamSynchronize(st));
    p->shared_passes += (int64_t)shared;
    p->last_launches += 4;
    return QCP_OK;
}

}  // namespace qcpd
