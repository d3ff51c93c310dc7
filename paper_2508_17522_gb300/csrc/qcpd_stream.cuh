// The stream engine: one launch per pass for problems whose vectors do not
// fit in shared memory (arXiv 2508.17522, Sec. 3.1-3.3: every LSQR
// iteration is one product with F and one with F^T, here through
// G = S F and the combined matrix M; see qcpd_common.cuh).
//
// Work is cut into warp-sized units that need no CTA barrier:
//   SU_SLICE  32 / G rows with no coupling inside D Pi (x-rows, or zero-
//             cone and R+ rows), G lanes per row (G a power of two chosen so
//             that no lane holds more than kSSteps entries), stored SELL-32:
//             slot (k, lane) at base + 32 k + lane holds entry k G + (lane
//             mod G) of row lane / G (rows sorted by length, so a slice is
//             nearly dense); the G partial sums of a row are added in a fixed
//             butterfly;
//   SU_SOCP   consecutive coupled blocks (second-order, PSD, exponential,
//             power cone) of at most 32 rows in all, one row per lane; an SOC
//             block's D Pi dot products are segmented warp reductions (one
//             segment per block), the other cones' D Pi is a dense matrix
//             per block (made at plan time; Appendix A's maps are linear in
//             the direction) applied through shuffles inside the block;
//   SU_SOCB   one coupled block of 33 to kSSocBig rows, rows lane + 32 j, the
//             block's values through a per-warp shared-memory buffer;
//   SU_LONG   up to kSLongChunk stored entries of a row longer than that, read
//             lane-strided; the last chunk of a row to finish adds the
//             chunk sums in order and runs the row's epilogue.
// A launch has gridDim.y = systems; the warps of a system's CTAs take its
// units in snake order (units sorted by their per-lane chain of dependent
// loads, longest first: the passes are bound by latency, so that chain, not
// the slot count, is what to balance).  Per-lane sums
// of the pass (||out||^2 and the two tau-row dot products) are reduced per
// warp, per CTA and finally, by the system's last CTA, over CTAs in a
// fixed order, so results do not depend on scheduling.
//
// Arithmetic.  FP64 instructions issue at 1/64 of the FP32 rate on this
// GPU, so every per-row operation runs in double-float (df64, about 48
// significant bits; qcpd_df64.cuh) on df64 copies of M's values and of the
// per-row data; the Krylov vectors U, V, W, X, XI are the plan's FP64
// arrays reinterpreted as df64 pairs in place while the engine iterates
// (k_stream_enter / k_stream_exit convert them, the right-hand side scaled
// by a power of two to norm in [1/2, 1) as in the cluster engine).  Their
// tau entries and the LSQR scalar recurrences stay in FP64 (one thread per
// system and pass).
#pragma once

#include "qcpd_df64.cuh"
#include "qcpd_kernels.cuh"

namespace qcpd {

constexpr int kSThreads = 256;
constexpr int kS2Ctas = 4;  // resident CTAs per SM of the paired kernel (its register budget)
constexpr int kSWarps = kSThreads / 32;
constexpr int kSSteps = 16;        // most entries of one lane in a slice (its chain of dependent loads)
constexpr int kSLongChunk = 32 * kSSteps;  // rows with more entries are cut into SU_LONG units of this many
constexpr int kSSocBig = 256;      // largest coupled block (second-order, PSD) the engine takes
constexpr int kSDense = 4;         // StreamSoc::kase of a block whose D Pi is stored dense (exp, power, PSD)

enum StreamKind : int32_t { SU_SLICE = 0, SU_SOCP = 1, SU_SOCB = 2, SU_LONG = 3 };

struct StreamUnit {
    int32_t kind;
    int32_t prob;    // problem (batch plans: also the system)
    int32_t nrows;   // SLICE / SOCP: rows (<= 32); SOCB: the block's rows; LONG: chunks of the row
    int32_t width;   // SLICE / SOCP: SELL width; SOCB: sub-slices; LONG: entries of this chunk
    int64_t base;    // first slot of the unit's entries
    int32_t aux;     // SLICE / SOCP: offset of the lanes' rows in rows[] (SOCP: and block indices in
                     // lblk[]); SOCB: offset of the sub-slices' widths in rows[]; LONG: the row
    int32_t blk;     // SOCB: the block (problem-relative); LONG: split-row index (plan-wide, -1: one chunk)
    int32_t chunk;   // LONG: chunk index; SLICE: G, the lanes per row
    int32_t row0;    // SOCB: first row; LONG: first chunk slot (plan-wide) of the row's chunk sums
};

// df64 constants of a second-order-cone block in the formula case (Appendix A):
// r = ||u||, h = 1/(2r), tq = t/r^2, htr = h (t + r); and the block's layout.
struct StreamSoc {
    df r, h, tq, htr;
    int32_t start, dim, kase, pad;
};

// This pass's scalars for the vector work, written by the previous pass's
// finisher (or by k_stream_enter): c1, -c2, -wcoef, xcoef and the tau
// column's coefficient tt.
struct StreamScal {
    df c1, nc2, nw, xc, tt;
    df nhc;        // LSMR: -hcoef (hbar <- h - hcoef hbar)
    int32_t upd;   // LSMR: this u-pass applies the deferred (hbar, x, h) updates
    int32_t lsmr;  // 1: LSMR's vector updates, 0: LSQR's
};

// Per system while the engine iterates: the FP64 tau entries of U, V, W, X,
// XI (they never enter a gather) and the scale of the right-hand side.
enum { TS_U = 0, TS_V = 1, TS_W = 2, TS_X = 3, TS_XI = 4, TS_HB = 5 };
struct StreamSys {
    double tau[6];
    double scale;   // the right-hand side was multiplied by this power of two
    int32_t uscaled;  // U and beta carry the scale too (no u-update yet)
    int32_t pad;
};

struct StreamArgs {
    const StreamUnit* units;
    const int32_t* uoff;    // per problem: its units [uoff[p], uoff[p + 1])
    const int32_t* rows;    // per lane row ids (SLICE, SOCP) and SOCB sub-slice widths
    const int32_t* lblk;    // SOCP: the lane's block (problem-relative), -1 for padding lanes
    const int32_t* scol;    // slot -> local column of M
    const df* valG;         // slot values: M diag(c) for G-passes (M when unscaled)
    const df* valT;         // M diag(w) for G^T-passes (M when unscaled)
    const df* cA;           // N-indexed per-row data (plan-wide offsets): coefA, coefB, w, c, z_y
    const df* cB;
    const df* rw;
    const df* cd;
    const df* zy;
    const int8_t* flag;
    const StreamSoc* soc;   // per block (plan-wide)
    const df* dense;        // row-major dim x dim D Pi of each block of kase kSDense (offset StreamSoc::pad)
    const double* rwd;      // FP64 w and c (tau entries)
    const double* cdd;
    const Sys* sys;
    const Prob* probs;
    LsqrState* state;
    StreamScal* scal;       // per system
    StreamSys* ssys;        // per system
    df* U;                  // plan vectors as df64 pairs (system offsets voff)
    df* V;
    df* W;
    df* X;
    df* XI;
    df* HB;                 // LSMR's hbar (W holds h)
    int32_t lsmr;           // 1: LSMR (Fong & Saunders 2011), 0: LSQR
    float4* cpart;          // per (system, CTA): the three df64 partial sums as (a, b), (c, 0) pairs
    int32_t* ccnt;          // per system: CTAs done in this pass
    df* lchunk;             // per (system, chunk slot): chunk sums of split rows
    int32_t* lcnt;          // per (system, split row): chunks done
    df* lrow;               // per (system, split row): 3 sums of the row's epilogue
    int32_t nsplit;         // split rows per system stride
    int32_t nslot;          // chunk slots per system stride
    const int32_t* soff;    // per problem: its split rows [soff[p], soff[p + 1])
    int32_t gx;             // CTAs per system (gridDim.x)
    int32_t gstride;        // CTA partials per system in cpart (>= gx)
    int32_t s0;             // first system of the range (enter / exit kernels)
    const int32_t* slist;   // the pass kernels' systems: slist[blockIdx.y] (the range's systems still iterating)
    int32_t batched;
    int* active;            // running systems of the range (paired launches: of the JVP range)
    int* active2;           // paired launches: running systems of the VJP range
    unsigned long long* pshared;  // paired launches: system passes that shared their read of M
};

// ---------------------------------------------------------------------------
// Per-CTA constants of one pass of one system.
struct SCtx {
    StreamScal sc;
    int n, N;
    const df *cA, *cB, *rw, *cd, *zy;  // problem-relative
    const int8_t* flag;
    const StreamSoc* soc;              // the problem's blocks
    const df* dense;                   // dense D Pi of the blocks that store one (plan-wide offsets)
    const df* gin;                     // the gathered vector (XI for G-passes, the input for G^T-passes)
    df *IN, *OUT, *W, *X, *XI, *HB;    // system-relative
};

// Per-lane sums of the pass: ||out||^2 and the tau-row dot products.
struct SAcc {
    DfAcc ss, dtop, dbot;
};

__device__ __forceinline__ void sacc_zero(SAcc& a) {
    a.ss = dfacc_zero();
    a.dtop = dfacc_zero();
    a.dbot = dfacc_zero();
}

__device__ __forceinline__ df dfl(const df* p) { return __ldg(reinterpret_cast<const float2*>(p)); }

// M's slots are read once per pass: streaming loads (evict first), so L1 keeps
// the gathered vector's entries.
__device__ __forceinline__ df dfl_cs(const df* p) { return __ldcs(reinterpret_cast<const float2*>(p)); }

// The row sum of one lane's row in a SELL-32 slice: sum_k val[slot] g[col[slot]]
// over slots base + 32 k + lane, k < width.  A padding slot holds the value 0
// and repeats the row's last column (an L1 hit), so no slot needs a test.
// The sum is software-pipelined in batches of kSB slots: the next batch's
// columns and values are loaded while the current batch's gathers are in
// flight, so a lane has up to 3 kSB loads outstanding instead of waiting
// for the columns and then for the gathers of every batch.
constexpr int kSB = 4;

__device__ __forceinline__ void sell_load(const int32_t* scol, const df* val, int64_t base, int k, int width,
                                          int32_t (&c)[kSB], df (&v)[kSB]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < kSB; ++j) {
        const bool ok = k + j < width;
        const int64_t s = base + 32 * (int64_t)(k + j) + lane;
        c[j] = ok ? __ldcs(scol + s) : 0;
        v[j] = ok ? dfl_cs(val + s) : df_zero();
    }
}

__device__ __forceinline__ df sell_rowsum(const int32_t* scol, const df* val, const df* g, int64_t base,
                                          int width) {
    DfAcc acc = dfacc_zero();
    if (width <= 0) return dfacc_result(acc);
    int32_t c[kSB];
    df v[kSB];
    sell_load(scol, val, base, 0, width, c, v);
    for (int k = 0; k < width; k += kSB) {
        df x[kSB];
#pragma unroll
        for (int j = 0; j < kSB; ++j) x[j] = (k + j < width) ? dfl(g + c[j]) : df_zero();
        int32_t cn[kSB];
        df vn[kSB];
        sell_load(scol, val, base, k + kSB, width, cn, vn);
#pragma unroll
        for (int j = 0; j < kSB; ++j) dfacc_fma(acc, v[j], x[j]);
#pragma unroll
        for (int j = 0; j < kSB; ++j) {
            c[j] = cn[j];
            v[j] = vn[j];
        }
    }
    return dfacc_result(acc);
}

// One chunk of a long row read lane-strided (entries base .. base + cnt),
// pipelined as sell_rowsum, summed over the warp in a fixed order; every
// lane gets the sum.
__device__ __forceinline__ void long_load(const int32_t* scol, const df* val, int64_t base, int k, int cnt,
                                          int32_t (&c)[kSB], df (&v)[kSB]) {
#pragma unroll
    for (int j = 0; j < kSB; ++j) {
        const int e = k + 32 * j;
        const bool ok = e < cnt;
        c[j] = ok ? __ldcs(scol + base + e) : 0;
        v[j] = ok ? dfl_cs(val + base + e) : df_zero();
    }
}

__device__ __forceinline__ df long_rowsum(const int32_t* scol, const df* val, const df* g, int64_t base, int cnt) {
    const int lane = threadIdx.x & 31;
    DfAcc acc = dfacc_zero();
    int32_t c[kSB];
    df v[kSB];
    long_load(scol, val, base, lane, cnt, c, v);
    for (int k = lane; k < cnt; k += 32 * kSB) {
        df x[kSB];
#pragma unroll
        for (int j = 0; j < kSB; ++j) x[j] = (k + 32 * j < cnt) ? dfl(g + c[j]) : df_zero();
        int32_t cn[kSB];
        df vn[kSB];
        long_load(scol, val, base, k + 32 * kSB, cnt, cn, vn);
#pragma unroll
        for (int j = 0; j < kSB; ++j) dfacc_fma(acc, v[j], x[j]);
#pragma unroll
        for (int j = 0; j < kSB; ++j) {
            c[j] = cn[j];
            v[j] = vn[j];
        }
    }
    return warp_sum_df(dfacc_result(acc));
}

// Row sums of two systems over the same slots (a paired launch: the two
// systems' passes share one read of M's columns and values; g and g2 are
// their gathered vectors).  Each system's adds come in the order of
// sell_rowsum / long_rowsum, so either sum equals the one-system result.
__device__ __forceinline__ void sell_rowsum2(const int32_t* scol, const df* val, const df* g, const df* g2,
                                             int64_t base, int width, df& h, df& h2) {
    DfAcc acc = dfacc_zero(), acc2 = dfacc_zero();
    if (width > 0) {
        int32_t c[kSB];
        df v[kSB];
        sell_load(scol, val, base, 0, width, c, v);
        for (int k = 0; k < width; k += kSB) {
            df x[kSB], x2[kSB];
#pragma unroll
            for (int j = 0; j < kSB; ++j) {
                const bool ok = k + j < width;
                x[j] = ok ? dfl(g + c[j]) : df_zero();
                x2[j] = ok ? dfl(g2 + c[j]) : df_zero();
            }
            int32_t cn[kSB];
            df vn[kSB];
            sell_load(scol, val, base, k + kSB, width, cn, vn);
#pragma unroll
            for (int j = 0; j < kSB; ++j) {
                dfacc_fma(acc, v[j], x[j]);
                dfacc_fma(acc2, v[j], x2[j]);
            }
#pragma unroll
            for (int j = 0; j < kSB; ++j) {
                c[j] = cn[j];
                v[j] = vn[j];
            }
        }
    }
    h = dfacc_result(acc);
    h2 = dfacc_result(acc2);
}

__device__ __forceinline__ void long_rowsum2(const int32_t* scol, const df* val, const df* g, const df* g2,
                                             int64_t base, int cnt, df& h, df& h2) {
    const int lane = threadIdx.x & 31;
    DfAcc acc = dfacc_zero(), acc2 = dfacc_zero();
    int32_t c[kSB];
    df v[kSB];
    long_load(scol, val, base, lane, cnt, c, v);
    for (int k = lane; k < cnt; k += 32 * kSB) {
        df x[kSB], x2[kSB];
#pragma unroll
        for (int j = 0; j < kSB; ++j) {
            const bool ok = k + 32 * j < cnt;
            x[j] = ok ? dfl(g + c[j]) : df_zero();
            x2[j] = ok ? dfl(g2 + c[j]) : df_zero();
        }
        int32_t cn[kSB];
        df vn[kSB];
        long_load(scol, val, base, k + 32 * kSB, cnt, cn, vn);
#pragma unroll
        for (int j = 0; j < kSB; ++j) {
            dfacc_fma(acc, v[j], x[j]);
            dfacc_fma(acc2, v[j], x2[j]);
        }
#pragma unroll
        for (int j = 0; j < kSB; ++j) {
            c[j] = cn[j];
            v[j] = vn[j];
        }
    }
    h = warp_sum_df(dfacc_result(acc));
    h2 = warp_sum_df(dfacc_result(acc2));
}

// ---- row epilogues (the formulas of run_tile in qcpd_kernels.cuh, in df64)
// The vector entries of row r that a pass's update reads, loaded together
// before the row's first store (the arrays are distinct, but the compiler
// cannot know that and would reload them after each store).
struct SRowV {
    df in, out, w, x, hb;
};

template <int ROLE>
__device__ __forceinline__ SRowV row_vecs(const SCtx& c, int r) {
    SRowV v;
    v.in = c.IN[r];
    v.out = c.OUT[r];
    v.w = c.W[r];
    const bool upd = ROLE == ROLE_U && c.sc.upd;
    v.x = (ROLE == ROLE_V && !c.sc.lsmr) || upd ? c.X[r] : df_zero();
    v.hb = upd ? c.HB[r] : df_zero();
    return v;
}

// The u- or v-update of row r given its new product value o: out = c1 o -
// c2 out, then LSQR's w (u-update) or x (v-update), or in LSMR's u-update
// the deferred hbar <- h - hcoef hbar, x <- x + xcoef hbar, h <- v / alpha -
// wcoef h (run_tile's lsmr_update); returns the new out.
template <int ROLE>
__device__ __forceinline__ df row_update(const SCtx& c, int r, df o, const SRowV& v, SAcc& acc) {
    const df nv = df_fma(c.sc.c1, o, df_mul(c.sc.nc2, v.out));
    c.OUT[r] = nv;
    dfacc_fma(acc.ss, nv, nv);
    if (ROLE == ROLE_U) {
        if (c.sc.upd) {
            const df hb = df_fma(c.sc.nhc, v.hb, v.w);
            c.HB[r] = hb;
            c.X[r] = df_fma(c.sc.xc, hb, v.x);
        }
        if (!c.sc.lsmr || c.sc.upd) c.W[r] = df_fma(v.in, c.sc.c1, df_mul(c.sc.nw, v.w));
    } else if (!c.sc.lsmr) {
        c.X[r] = df_fma(c.sc.xc, v.w, v.x);
    }
    return nv;
}

// G-pass, row r with row sum h: out = W (M_top xi + q t | M_bot xi - b t - c + D c) C,
// then the u- or v-update of that row.
template <int ROLE, bool SC>
__device__ __forceinline__ void g_row(const SCtx& c, int r, df h, SAcc& acc) {
    const SRowV v = row_vecs<ROLE>(c, r);
    const df iv = v.in;
    df o;
    if (r < c.n) {
        o = df_fma(dfl(c.cA + r), c.sc.tt, h);
        dfacc_fma(acc.dtop, dfl(c.cB + r), SC ? df_mul(dfl(c.cd + r), iv) : iv);
    } else {
        const df xi = c.XI[r];
        const df dxi = SC ? df_mul(dfl(c.cd + r), df_sub(xi, iv)) : df_sub(xi, iv);
        o = df_add(df_fma(df_neg(dfl(c.cA + r)), c.sc.tt, h), dxi);
        dfacc_fma(acc.dbot, dfl(c.cB + r), SC ? df_mul(dfl(c.cd + r), xi) : xi);
    }
    if (SC) o = df_mul(o, dfl(c.rw + r));
    row_update<ROLE>(c, r, o, v, acc);
}

// G^T-pass, first half of row r (iv = in_r): s1 = (M rho - g r3)_r on
// x-rows, (M rho - b r3)_r + (w in)_r on y-rows; ivs = (w in)_r.
template <bool SC>
__device__ __forceinline__ df gt_pre(const SCtx& c, int r, df h, df iv, df& ivs, SAcc& acc) {
    ivs = SC ? df_mul(dfl(c.rw + r), iv) : iv;
    const df h1 = df_fma(df_neg(dfl(c.cB + r)), c.sc.tt, h);
    if (r < c.n) {
        dfacc_fma(acc.dtop, dfl(c.cA + r), ivs);
        return h1;
    }
    dfacc_fma(acc.dbot, dfl(c.cA + r), ivs);
    return df_add(h1, ivs);
}

// G^T-pass, second half of row r given s2 = (D s1)_r: the u- or v-update;
// returns the new out_r (whose D Pi the caller stores in XI).
template <int ROLE, bool SC>
__device__ __forceinline__ df gt_post(const SCtx& c, int r, df s2, df ivs, const SRowV& v, SAcc& acc) {
    df o = (r < c.n) ? s2 : df_sub(s2, ivs);
    if (SC) o = df_mul(o, dfl(c.cd + r));
    return row_update<ROLE>(c, r, o, v, acc);
}

// D on a row outside second-order-cone blocks: 1 on x-rows and zero-cone
// rows (the dual of {0} is R), the 0/1 flag on R+ rows.
__device__ __forceinline__ df d_diag(const SCtx& c, int r, df v) {
    if (r < c.n) return v;
    return c.flag[r] == RF_ONE ? v : df_zero();
}

// One non-coupled row of a G^T-pass (x-rows, zero-cone and R+ rows).
template <int ROLE, bool SC>
__device__ __forceinline__ void gt_row(const SCtx& c, int r, df h, SAcc& acc) {
    const SRowV v = row_vecs<ROLE>(c, r);
    df ivs;
    const df s1 = gt_pre<SC>(c, r, h, v.in, ivs, acc);
    const df nv = gt_post<ROLE, SC>(c, r, d_diag(c, r, s1), ivs, v, acc);
    c.XI[r] = d_diag(c, r, nv);
}

template <int PASS, int ROLE, bool SC>
__device__ __forceinline__ void plain_row(const SCtx& c, int r, df h, SAcc& acc) {
    if (PASS == PASS_G) g_row<ROLE, SC>(c, r, h, acc);
    else gt_row<ROLE, SC>(c, r, h, acc);
}

// ---- second-order-cone blocks (Appendix A): D Pi_{K*} at z_y = (t, u)
// maps (c_t, c_u) to h (r c_t + u^T c_u, ...) in the formula case (kase 2),
// to 0 inside the polar cone (kase 0) and to itself inside the cone (kase 1).
__device__ __forceinline__ df soc_d(df v, df u, int pos, df ct, df dot, int kase, const StreamSoc& B) {
    if (kase == 0) return df_zero();
    if (kase != 2) return v;
    if (pos == 0) return df_mul(B.h, df_fma(B.r, ct, dot));
    const df aa = df_mul(B.h, df_fma(df_neg(B.tq), dot, ct));
    return df_fma(aa, u, df_mul(B.htr, v));
}

__device__ __forceinline__ df shfl_xor_df(df v, int o) {
    df w;
    w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    return w;
}

__device__ __forceinline__ df shfl_df(df v, int src) {
    df o;
    o.x = __shfl_sync(0xffffffffu, v.x, src);
    o.y = __shfl_sync(0xffffffffu, v.y, src);
    return o;
}

// D on packed blocks, one row per lane: the lanes [head, end] hold one
// block; u^T c_u is a segmented sum (after the doubling steps the head lane
// holds its whole block's sum, each lane adding only from its own block).
// Every lane calls it.
__device__ __forceinline__ df socp_d(df v, df u, int pos, int head, int end, int kase, const StreamSoc& B,
                                     const df* dense) {
    const int lane = threadIdx.x & 31;
    // blocks with a stored D Pi (exponential and power cones, PSD blocks of
    // at most 32 entries): out_pos = sum_j D[pos][j] v_{head + j}, in j order
    const bool dn = kase == kSDense;
    if (__any_sync(0xffffffffu, dn)) {
        const int dim = end - head + 1;
        const int jmax = __reduce_max_sync(0xffffffffu, dn ? dim : 0);
        df acc = df_zero();
        for (int j = 0; j < jmax; ++j) {
            const df vj = shfl_df(v, dn && j < dim ? head + j : lane);
            if (dn && j < dim) acc = df_fma(dfl(dense + B.pad + pos * dim + j), vj, acc);
        }
        if (dn) v = acc;
    }
    df t = (kase == 2 && pos > 0) ? df_mul(u, v) : df_zero();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        df o;
        o.x = __shfl_down_sync(0xffffffffu, t.x, d);
        o.y = __shfl_down_sync(0xffffffffu, t.y, d);
        if (lane + d <= end) t = df_add(t, o);
    }
    const df dot = shfl_df(t, head);
    const df ct = shfl_df(v, head);
    return soc_d(v, u, pos, ct, dot, kase, B);
}

struct SUnitCtx {
    const int32_t* rows;
    const int32_t* lblk;
    const int32_t* scol;
    const df* val;
};

// SU_SLICE units (either pass) and SU_SOCP units of a G-pass, given each
// lane's row sum h: row i of the unit on lanes [G i, G i + G) (SU_SOCP:
// G = 1), no coupling.
template <int PASS, int ROLE, bool SC>
__device__ __forceinline__ void slice_rows(const SCtx& c, const SUnitCtx& k, const StreamUnit& u, df h, SAcc& acc) {
    const int lane = threadIdx.x & 31;
    const int G = u.kind == SU_SLICE ? u.chunk : 1;
    for (int o = G >> 1; o > 0; o >>= 1) h = df_add(h, shfl_xor_df(h, o));
    if ((lane & (G - 1)) != 0) return;
    const int r = k.rows[u.aux + lane / G];
    if (r >= 0) plain_row<PASS, ROLE, SC>(c, r, h, acc);
}

// SU_SOCB units of a G-pass: rows row0 + 32 j + lane, no coupling.
template <int ROLE, bool SC>
__device__ __forceinline__ void unit_socb_g(const SCtx& c, const SUnitCtx& k, const StreamUnit& u, SAcc& acc) {
    const int lane = threadIdx.x & 31;
    int64_t base = u.base;
    for (int j = 0; j < u.width; ++j) {
        const int w = k.rows[u.aux + j];
        const df h = sell_rowsum(k.scol, k.val, c.gin, base, w);
        base += 32 * (int64_t)w;
        const int i = 32 * j + lane;
        if (i < u.nrows) g_row<ROLE, SC>(c, u.row0 + i, h, acc);
    }
}

// SU_SOCP units of a G^T-pass, given each lane's row sum h.
template <int ROLE, bool SC>
__device__ __forceinline__ void socp_gt_rows(const SCtx& c, const SUnitCtx& k, const StreamUnit& u, df h,
                                             SAcc& acc) {
    const int lane = threadIdx.x & 31;
    const int r = k.rows[u.aux + lane];
    const int bi = k.lblk[u.aux + lane];
    int head = lane, end = lane, kase = 1, pos = 0;
    StreamSoc B{};
    if (bi >= 0) {
        B = c.soc[bi];
        pos = r - B.start;
        head = lane - pos;
        end = head + B.dim - 1;
        kase = B.kase;
    }
    SRowV v{};
    df ivs = df_zero(), s1 = df_zero(), uk = df_zero();
    if (r >= 0) {
        v = row_vecs<ROLE>(c, r);
        s1 = gt_pre<SC>(c, r, h, v.in, ivs, acc);
        uk = dfl(c.zy + r);
    }
    const df s2 = socp_d(s1, uk, pos, head, end, kase, B, c.dense);
    df nv = df_zero();
    if (r >= 0) nv = gt_post<ROLE, SC>(c, r, s2, ivs, v, acc);
    const df xi = socp_d(nv, uk, pos, head, end, kase, B, c.dense);
    if (r >= 0) c.XI[r] = xi;
}

// SU_SOCB units of a G^T-pass: the block's values go through the warp's
// shared-memory buffer sb (kSSocBig entries).
template <int ROLE, bool SC>
__device__ __forceinline__ void unit_socb_gt(const SCtx& c, const SUnitCtx& k, const StreamUnit& u, df* sb,
                                             SAcc& acc) {
    const int lane = threadIdx.x & 31;
    const StreamSoc B = c.soc[u.blk];
    const int dim = u.nrows, r0 = u.row0;
    int64_t base = u.base;
    df part = df_zero();
    for (int j = 0; j < u.width; ++j) {
        const int w = k.rows[u.aux + j];
        const df h = sell_rowsum(k.scol, k.val, c.gin, base, w);
        base += 32 * (int64_t)w;
        const int i = 32 * j + lane;
        if (i < dim) {
            df ivs;
            const df s1 = gt_pre<SC>(c, r0 + i, h, c.IN[r0 + i], ivs, acc);
            sb[i] = s1;
            if (i > 0 && B.kase == 2) part = df_fma(dfl(c.zy + r0 + i), s1, part);
        }
    }
    __syncwarp();
    if (B.kase == kSDense) {  // a stored D Pi: dense products in j order, the second on the new OUT entries
        const df* D = c.dense + B.pad;
        for (int i = lane; i < dim; i += 32) {
            df s2 = df_zero();
            for (int j = 0; j < dim; ++j) s2 = df_fma(dfl(D + (int64_t)i * dim + j), sb[j], s2);
            const int r = r0 + i;
            const SRowV v = row_vecs<ROLE>(c, r);
            const df ivs = SC ? df_mul(dfl(c.rw + r), v.in) : v.in;
            gt_post<ROLE, SC>(c, r, s2, ivs, v, acc);
        }
        __syncwarp();  // the lanes' new OUT entries are visible to the whole warp
        for (int i = lane; i < dim; i += 32) {
            df x = df_zero();
            for (int j = 0; j < dim; ++j) x = df_fma(dfl(D + (int64_t)i * dim + j), c.OUT[r0 + j], x);
            c.XI[r0 + i] = x;
        }
        __syncwarp();
        return;
    }
    df dot = warp_sum_df(part);
    df ct = sb[0];
    __syncwarp();
    part = df_zero();
    for (int i = lane; i < dim; i += 32) {
        const int r = r0 + i;
        const df uk = dfl(c.zy + r);
        const SRowV v = row_vecs<ROLE>(c, r);
        const df ivs = SC ? df_mul(dfl(c.rw + r), v.in) : v.in;
        const df nv = gt_post<ROLE, SC>(c, r, soc_d(sb[i], uk, i, ct, dot, B.kase, B), ivs, v, acc);
        sb[i] = nv;
        if (i > 0 && B.kase == 2) part = df_fma(uk, nv, part);
    }
    __syncwarp();
    dot = warp_sum_df(part);
    ct = sb[0];
    for (int i = lane; i < dim; i += 32) c.XI[r0 + i] = soc_d(sb[i], dfl(c.zy + r0 + i), i, ct, dot, B.kase, B);
    __syncwarp();
}

// Arrival at a counter (a CTA at the end of its pass, a chunk of a split
// row): add 1 with release semantics (the partial sums the arriving thread
// wrote before become visible with it) and acquire semantics (the last to
// arrive sees every earlier arrival's partials); returns the previous count.
__device__ __forceinline__ int arrive_acq_rel(int* cnt) {
    int prev;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(prev) : "l"(cnt) : "memory");
    return prev;
}

// SU_LONG units, given the chunk's sum h: a chunk of one long row (never
// inside a coupled block).  A row in one chunk is finished by lane 0; a split row's chunk sums go to
// its slots, and the chunk that completes the row adds them in order and
// runs the epilogue, whose contributions to the pass's sums go to the row's
// own slot (added by the finisher in row order, so the result does not
// depend on which chunk came last).
template <int PASS, int ROLE, bool SC>
__device__ __forceinline__ void long_rows(const SCtx& c, const StreamArgs& a, int si, const StreamUnit& u, df h,
                                          SAcc& acc) {
    const int lane = threadIdx.x & 31;
    const int r = u.aux;
    if (u.blk < 0) {
        if (lane == 0) plain_row<PASS, ROLE, SC>(c, r, h, acc);
        return;
    }
    const int64_t so = a.batched ? 0 : (int64_t)si * a.nslot;
    const int64_t sr = a.batched ? 0 : (int64_t)si * a.nsplit;
    int last = 0;
    if (lane == 0) {
        a.lchunk[so + u.row0 + u.chunk] = h;
        last = arrive_acq_rel(a.lcnt + sr + u.blk) == u.nrows - 1;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    __syncwarp();  // the lanes' reads below come after lane 0's acquire
    // the chunk sums: a fixed share per lane (independent loads), then a
    // fixed butterfly, so the sum does not depend on which chunk came last
    df t = df_zero();
    for (int q = lane; q < u.nrows; q += 32)
        t = df_add(t, __ldcg(reinterpret_cast<const float2*>(a.lchunk + so + u.row0 + q)));
    t = warp_sum_df(t);
    if (lane != 0) return;
    a.lcnt[sr + u.blk] = 0;
    SAcc racc;
    sacc_zero(racc);
    plain_row<PASS, ROLE, SC>(c, r, t, racc);
    df* o = a.lrow + 3 * (sr + u.blk);
    o[0] = dfacc_result(racc.ss);
    o[1] = dfacc_result(racc.dtop);
    o[2] = dfacc_result(racc.dbot);
    __threadfence();  // read by the system's last CTA within this launch
}

// ---------------------------------------------------------------------------
// The finisher of an LSMR system (one thread): the tau entries with the
// pass's vector updates, then lsmr_step_u / lsmr_step_v (Fong & Saunders
// 2011, the pass engine's finisher) on the state in global memory, then the
// next pass's scalars.  only: a stopped system's last deferred updates.
template <int PASS, int ROLE, bool SC>
__device__ __forceinline__ void stream_finish_lsmr(const StreamArgs& a, int si, const Prob& pr, Part tot, bool only,
                                                int* active) {
    LsqrState* st = a.state + si;
    double* tau = a.ssys[si].tau;
    const int rN = pr.n + pr.m;
    const double rwN = a.rwd[pr.doff + rN], cdN = a.cdd[pr.doff + rN];
    const double c1 = ROLE == ROLE_U ? st->uc1 : st->vc1;
    const double c2 = ROLE == ROLE_U ? st->uc2 : st->vc2;
    const double wcoef = st->wcoef, xcoef = st->xcoef, hcoef = st->hcoef;
    const int tin_i = ROLE == ROLE_U ? TS_V : TS_U, tout_i = ROLE == ROLE_U ? TS_U : TS_V;
    const double tin = tau[tin_i];
    auto tau_upd = [&]() {  // run_tile's lsmr_update on the tau entries
        const double h = tau[TS_W];
        const double hb = fma(-hcoef, tau[TS_HB], h);
        tau[TS_HB] = hb;
        tau[TS_X] = fma(xcoef, hb, tau[TS_X]);
        tau[TS_W] = fma(tin, c1, -wcoef * h);
    };
    if (only) {
        tau_upd();
        st->upd = 0;  // applied: a continuation starts with a plain u-pass
        st->status = S_DONE;
        atomicSub(active, 1);
        return;
    }
    const double tt = SC ? (PASS == PASS_G ? cdN : rwN) * tin : tin;
    double oN;
    if (PASS == PASS_G) {
        oN = -tot.b - tot.c + pr.kappa * tt;
        if (SC) oN *= rwN;
    } else {
        oN = tot.b - tot.c + pr.kappa * tt;
        if (SC) oN *= cdN;
    }
    // gauge dz_N = 0: G^T-passes leave the tau entry at 0 (see run_tile)
    const double nvN = (PASS == PASS_GT) ? 0.0 : c1 * oN - c2 * tau[tout_i];
    tau[tout_i] = nvN;
    if (PASS == PASS_GT) tau[TS_XI] = 0.0;
    const double nsq = fma(nvN, nvN, tot.a);
    double nrm, inv;
    norm_and_inverse(nsq, nrm, inv);
    bool stopped;
    if (ROLE == ROLE_U) {
        if (st->upd) tau_upd();
        stopped = lsmr_step_u(st, nrm, inv);
    } else {
        stopped = lsmr_step_v(st, nrm, inv);
    }
    constexpr int NPASS = PASS == PASS_G ? PASS_GT : PASS_G;
    const double nc1 = ROLE == ROLE_U ? st->vc1 : st->uc1;
    const double nc2 = ROLE == ROLE_U ? st->vc2 : st->uc2;
    const double ntt = SC ? (NPASS == PASS_G ? cdN : rwN) * nvN : nvN;
    StreamScal q;
    q.c1 = df_from(nc1);
    q.nc2 = df_from(-nc2);
    q.nw = df_from(-st->wcoef);
    q.xc = df_from(st->xcoef);
    q.tt = df_from(ntt);
    q.nhc = df_from(-st->hcoef);
    q.upd = st->upd;
    q.lsmr = 1;
    a.scal[si] = q;
    if (stopped) atomicSub(active, 1);
}

// The LSQR fields the finisher reads and writes, copied into registers with
// one batch of loads and written back at the end: on the state in global
// memory every read after a write would wait for its own round trip (the
// compiler cannot tell the fields and the tau entries apart).
struct LsqrHot {
    double alpha, beta, rhobar, phibar, inv_rho, uc1, uc2, vc1, vc2, wcoef, xcoef, c, s, bnorm, rtol;
    int64_t iters, maxiter;
    int32_t status, outcome, first;
};

__device__ __forceinline__ void hot_load(LsqrHot& h, const LsqrState* st) {
    h.alpha = st->alpha;
    h.beta = st->beta;
    h.rhobar = st->rhobar;
    h.phibar = st->phibar;
    h.inv_rho = st->inv_rho;
    h.uc1 = st->uc1;
    h.uc2 = st->uc2;
    h.vc1 = st->vc1;
    h.vc2 = st->vc2;
    h.wcoef = st->wcoef;
    h.xcoef = st->xcoef;
    h.c = st->c;
    h.s = st->s;
    h.bnorm = st->bnorm;
    h.rtol = st->rtol;
    h.iters = st->iters;
    h.maxiter = st->maxiter;
    h.status = st->status;
    h.outcome = st->outcome;
    h.first = st->first;
}

__device__ __forceinline__ void hot_store(LsqrState* st, const LsqrHot& h) {
    st->alpha = h.alpha;
    st->beta = h.beta;
    st->rhobar = h.rhobar;
    st->phibar = h.phibar;
    st->inv_rho = h.inv_rho;
    st->uc1 = h.uc1;
    st->uc2 = h.uc2;
    st->vc1 = h.vc1;
    st->vc2 = h.vc2;
    st->wcoef = h.wcoef;
    st->xcoef = h.xcoef;
    st->c = h.c;
    st->s = h.s;
    st->iters = h.iters;
    st->status = h.status;
    st->outcome = h.outcome;
    st->first = h.first;
}

// The system's finisher (one thread): the tau entry of the pass's output and
// the LSQR scalars, in FP64 as in run_tile, then the next pass's scalars.
template <int PASS, int ROLE, bool SC>
__device__ __forceinline__ void stream_finish(const StreamArgs& a, int si, const Prob& pr, Part tot, bool only_x,
                                              int* active) {
    if (a.lsmr) {
        stream_finish_lsmr<PASS, ROLE, SC>(a, si, pr, tot, only_x, active);
        return;
    }
    LsqrState* gst = a.state + si;
    double* gtau = a.ssys[si].tau;
    const int rN = pr.n + pr.m;
    const double rwN = a.rwd[pr.doff + rN], cdN = a.cdd[pr.doff + rN];
    double tau[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) tau[i] = gtau[i];
    LsqrHot h;
    hot_load(h, gst);
    LsqrHot* st = &h;
    if (only_x) {
        gtau[TS_X] = fma(st->xcoef, tau[TS_W], tau[TS_X]);
        gst->status = S_DONE;
        atomicSub(active, 1);
        return;
    }
    const double c1 = ROLE == ROLE_U ? st->uc1 : st->vc1;
    const double c2 = ROLE == ROLE_U ? st->uc2 : st->vc2;
    const double wcoef = st->wcoef, xcoef = st->xcoef;
    const int tin_i = ROLE == ROLE_U ? TS_V : TS_U, tout_i = ROLE == ROLE_U ? TS_U : TS_V;
    const double tin = tau[tin_i], tout = tau[tout_i], tw = tau[TS_W], tx = tau[TS_X];
    const double tt = SC ? (PASS == PASS_G ? cdN : rwN) * tin : tin;
    double oN;
    if (PASS == PASS_G) {
        oN = -tot.b - tot.c + pr.kappa * tt;
        if (SC) oN *= rwN;
    } else {
        oN = tot.b - tot.c + pr.kappa * tt;
        if (SC) oN *= cdN;
    }
    // gauge dz_N = 0: G^T-passes leave the tau entry at 0 (see run_tile)
    const double nvN = (PASS == PASS_GT) ? 0.0 : c1 * oN - c2 * tout;
    tau[tout_i] = nvN;
    if (PASS == PASS_GT) tau[TS_XI] = 0.0;
    const double nsq = fma(nvN, nvN, tot.a);
    double nrm, inv;
    norm_and_inverse(nsq, nrm, inv);
    bool stopped = false;
    if (ROLE == ROLE_U) {
        tau[TS_W] = tin * c1 - wcoef * tw;
        lsqr_step_u(st, nrm, inv, nsq);
    } else {
        tau[TS_X] = fma(xcoef, tw, tx);
        stopped = lsqr_step_v(st, nrm, inv);
    }
    // the next pass: the other product, the other update
    constexpr int NPASS = PASS == PASS_G ? PASS_GT : PASS_G;
    const double nc1 = ROLE == ROLE_U ? st->vc1 : st->uc1;
    const double nc2 = ROLE == ROLE_U ? st->vc2 : st->uc2;
    const double ntin = nvN;  // the next pass's input is this pass's output (U after a u-pass, V after a v-pass)
    const double ntt = SC ? (NPASS == PASS_G ? cdN : rwN) * ntin : ntin;
    StreamScal q;
    q.c1 = df_from(nc1);
    q.nc2 = df_from(-nc2);
    q.nw = df_from(-st->wcoef);
    q.xc = df_from(st->xcoef);
    q.tt = df_from(ntt);
    q.nhc = df_zero();
    q.upd = 0;
    q.lsmr = 0;
    a.scal[si] = q;
#pragma unroll
    for (int i = 0; i < 5; ++i) gtau[i] = tau[i];
    hot_store(gst, h);
    if (stopped) atomicSub(active, 1);
}


// ---------------------------------------------------------------------------
// The pieces of a pass.  The per-CTA constants live in shared memory, not in
// registers; thread 0 fills them.
template <int PASS, int ROLE>
__device__ __forceinline__ void stream_ctx(const StreamArgs& a, const Sys& sy, const Prob& pr, int si, SCtx& c) {
    c.sc = a.scal[si];
    c.n = pr.n;
    c.N = pr.n + pr.m + 1;
    c.cA = a.cA + pr.doff;
    c.cB = a.cB + pr.doff;
    c.rw = a.rw + pr.doff;
    c.cd = a.cd + pr.doff;
    c.zy = a.zy + pr.doff;
    c.flag = a.flag + pr.doff;
    c.soc = a.soc + pr.soff;
    c.dense = a.dense;
    c.IN = (ROLE == ROLE_U ? a.V : a.U) + sy.voff;
    c.OUT = (ROLE == ROLE_U ? a.U : a.V) + sy.voff;
    c.W = a.W + sy.voff;
    c.X = a.X + sy.voff;
    c.XI = a.XI + sy.voff;
    c.HB = a.HB + sy.voff;
    c.gin = PASS == PASS_G ? c.XI : c.IN;
}

// The units of one system in snake order (sorted by cost, largest first).
template <int PASS, int ROLE, bool SC>
__device__ __forceinline__ void stream_units(const StreamArgs& a, int si, int prob, const SCtx& c, df* sb,
                                             SAcc& acc) {
    const int warp = threadIdx.x >> 5;
    const SUnitCtx k{a.rows, a.lblk, a.scol, PASS == PASS_G ? a.valG : a.valT};
    const int wt = a.gx * kSWarps, wg = blockIdx.x * kSWarps + warp;
    const int u0 = a.uoff[prob], nu = a.uoff[prob + 1] - u0;
    for (int j = 0;; ++j) {
        const int idx = j * wt + ((j & 1) ? wt - 1 - wg : wg);
        if (idx >= nu) break;
        const StreamUnit u = a.units[u0 + idx];
        if (u.kind == SU_LONG) {
            long_rows<PASS, ROLE, SC>(c, a, si, u, long_rowsum(k.scol, k.val, c.gin, u.base, u.width), acc);
        } else if (u.kind == SU_SOCB) {
            if (PASS == PASS_G) unit_socb_g<ROLE, SC>(c, k, u, acc);
            else unit_socb_gt<ROLE, SC>(c, k, u, sb, acc);
        } else {
            const df h = sell_rowsum(k.scol, k.val, c.gin, u.base, u.width);
            if (PASS == PASS_G || u.kind == SU_SLICE) slice_rows<PASS, ROLE, SC>(c, k, u, h, acc);
            else socp_gt_rows<ROLE, SC>(c, k, u, h, acc);
        }
    }
}

// The units of two systems of one problem in one pass: A in role RA, B in
// role RB; slices, packed blocks and chunks of long rows read their slots
// once for both (SU_SOCB units, rare, run once per system).
template <int PASS, int RA, int RB, bool SC>
__device__ __forceinline__ void stream_units2(const StreamArgs& a, int sa, int sb2, int prob, const SCtx& ca,
                                              const SCtx& cb, df* sb, SAcc& acca, SAcc& accb) {
    const int warp = threadIdx.x >> 5;
    const SUnitCtx k{a.rows, a.lblk, a.scol, PASS == PASS_G ? a.valG : a.valT};
    const int wt = a.gx * kSWarps, wg = blockIdx.x * kSWarps + warp;
    const int u0 = a.uoff[prob], nu = a.uoff[prob + 1] - u0;
    for (int j = 0;; ++j) {
        const int idx = j * wt + ((j & 1) ? wt - 1 - wg : wg);
        if (idx >= nu) break;
        const StreamUnit u = a.units[u0 + idx];
        if (u.kind == SU_LONG) {
            df h, h2;
            long_rowsum2(k.scol, k.val, ca.gin, cb.gin, u.base, u.width, h, h2);
            long_rows<PASS, RA, SC>(ca, a, sa, u, h, acca);
            long_rows<PASS, RB, SC>(cb, a, sb2, u, h2, accb);
        } else if (u.kind == SU_SOCB) {
            if (PASS == PASS_G) {
                unit_socb_g<RA, SC>(ca, k, u, acca);
                unit_socb_g<RB, SC>(cb, k, u, accb);
            } else {
                unit_socb_gt<RA, SC>(ca, k, u, sb, acca);
                unit_socb_gt<RB, SC>(cb, k, u, sb, accb);
            }
        } else {
            df h, h2;
            sell_rowsum2(k.scol, k.val, ca.gin, cb.gin, u.base, u.width, h, h2);
            if (PASS == PASS_G || u.kind == SU_SLICE) {
                slice_rows<PASS, RA, SC>(ca, k, u, h, acca);
                slice_rows<PASS, RB, SC>(cb, k, u, h2, accb);
            } else {
                socp_gt_rows<RA, SC>(ca, k, u, h, acca);
                socp_gt_rows<RB, SC>(cb, k, u, h2, accb);
            }
        }
    }
}

// The end of a system's pass, in pieces.  cta_partial: the CTA's sums in a
// fixed order (lanes, then warps; df64 throughout) into the system's CTA
// slot, then its arrival; true in the system's last CTA (one thread).
__device__ __forceinline__ bool cta_partial(const StreamArgs& a, int si, df (*red)[3]) {
    df t0 = red[0][0], t1 = red[0][1], t2 = red[0][2];
    for (int w = 1; w < kSWarps; ++w) {
        t0 = df_add(t0, red[w][0]);
        t1 = df_add(t1, red[w][1]);
        t2 = df_add(t2, red[w][2]);
    }
    float4* o = a.cpart + 2 * ((int64_t)si * a.gstride + blockIdx.x);
    o[0] = make_float4(t0.x, t0.y, t1.x, t1.y);
    o[1] = make_float4(t2.x, t2.y, 0.f, 0.f);
    return arrive_acq_rel(a.ccnt + si) == a.gx - 1;
}

__device__ __forceinline__ void warp_sums_to(const SAcc& acc, df (*red)[3]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const df v0 = warp_sum_df(dfacc_result(acc.ss));
    const df v1 = warp_sum_df(dfacc_result(acc.dtop));
    const df v2 = warp_sum_df(dfacc_result(acc.dbot));
    if (lane == 0) {
        red[warp][0] = v0;
        red[warp][1] = v1;
        red[warp][2] = v2;
    }
}

// In the system's last CTA (every thread; thread 0 of some warp acquired
// every other CTA's partials and a barrier orders these reads after that):
// a fixed share of the CTA partials and of the split rows' sums per thread,
// then lanes, into red.
__device__ __forceinline__ void last_partials(const StreamArgs& a, int si, int prob, bool only_x, df (*red)[3]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    df v0 = df_zero(), v1 = df_zero(), v2 = df_zero();
    for (int i = threadIdx.x; i < a.gx; i += kSThreads) {
        const float4* o = a.cpart + 2 * ((int64_t)si * a.gstride + i);
        const float4 p0 = __ldcg(o), p1 = __ldcg(o + 1);
        v0 = df_add(v0, make_float2(p0.x, p0.y));
        v1 = df_add(v1, make_float2(p0.z, p0.w));
        v2 = df_add(v2, make_float2(p1.x, p1.y));
    }
    const int64_t sr = a.batched ? 0 : (int64_t)si * a.nsplit;
    if (!only_x) {
        for (int i = a.soff[prob] + threadIdx.x; i < a.soff[prob + 1]; i += kSThreads) {
            const float2* o = reinterpret_cast<const float2*>(a.lrow + 3 * (sr + i));
            v0 = df_add(v0, __ldcg(o));
            v1 = df_add(v1, __ldcg(o + 1));
            v2 = df_add(v2, __ldcg(o + 2));
        }
    }
    v0 = warp_sum_df(v0);
    v1 = warp_sum_df(v1);
    v2 = warp_sum_df(v2);
    if (lane == 0) {
        red[warp][0] = v0;
        red[warp][1] = v1;
        red[warp][2] = v2;
    }
}

// last_partials for the two systems of a paired launch (either or both
// last in this CTA), their loads issued together.
__device__ __forceinline__ void last_partials2(const StreamArgs& a, int sa, int sb, bool la, bool lb, int prob,
                                               df (*red)[kSWarps][3]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    df v[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) v[h][0] = v[h][1] = v[h][2] = df_zero();
    const int sys[2] = {sa, sb};
    const bool on[2] = {la, lb};
    for (int i = threadIdx.x; i < a.gx; i += kSThreads) {
        float4 p0[2], p1[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!on[h]) continue;
            const float4* o = a.cpart + 2 * ((int64_t)sys[h] * a.gstride + i);
            p0[h] = __ldcg(o);
            p1[h] = __ldcg(o + 1);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!on[h]) continue;
            v[h][0] = df_add(v[h][0], make_float2(p0[h].x, p0[h].y));
            v[h][1] = df_add(v[h][1], make_float2(p0[h].z, p0[h].w));
            v[h][2] = df_add(v[h][2], make_float2(p1[h].x, p1[h].y));
        }
    }
    for (int i = a.soff[prob] + threadIdx.x; i < a.soff[prob + 1]; i += kSThreads) {
        float2 q[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!on[h]) continue;
            const int64_t sr = a.batched ? 0 : (int64_t)sys[h] * a.nsplit;
            const float2* o = reinterpret_cast<const float2*>(a.lrow + 3 * (sr + i));
            q[h][0] = __ldcg(o);
            q[h][1] = __ldcg(o + 1);
            q[h][2] = __ldcg(o + 2);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!on[h]) continue;
            v[h][0] = df_add(v[h][0], q[h][0]);
            v[h][1] = df_add(v[h][1], q[h][1]);
            v[h][2] = df_add(v[h][2], q[h][2]);
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!on[h]) continue;
        const df w0 = warp_sum_df(v[h][0]), w1 = warp_sum_df(v[h][1]), w2 = warp_sum_df(v[h][2]);
        if (lane == 0) {
            red[h][warp][0] = w0;
            red[h][warp][1] = w1;
            red[h][warp][2] = w2;
        }
    }
}

// One thread of the system's last CTA: the warps' totals in order, then the
// finisher.
template <int PASS, int ROLE, bool SC>
__device__ __forceinline__ void last_finish(const StreamArgs& a, int si, const Prob& pr, bool only_x, int* active,
                                            df (*red)[3], unsigned long long* shared) {
    df t0 = red[0][0], t1 = red[0][1], t2 = red[0][2];
    for (int w = 1; w < kSWarps; ++w) {
        t0 = df_add(t0, red[w][0]);
        t1 = df_add(t1, red[w][1]);
        t2 = df_add(t2, red[w][2]);
    }
    a.ccnt[si] = 0;
    stream_finish<PASS, ROLE, SC>(a, si, pr, Part{df_to(t0), df_to(t1), df_to(t2), 0.0}, only_x, active);
    if (shared) atomicAdd(shared, 1ull);
}

// The end of a system's pass in every CTA: its partials and arrival; the
// system's last CTA adds every CTA's partials and the split rows' sums and
// finishes (FP64 only for the three totals, in the finisher's thread).
template <int PASS, int ROLE, bool SC>
__device__ __forceinline__ void stream_tail(const StreamArgs& a, int si, int prob, const Prob& pr, SAcc& acc,
                                            bool only_x, int* active, df (*red)[3], int* s_last) {
    __syncthreads();  // red and s_last may still be read by an earlier tail of this CTA
    warp_sums_to(acc, red);
    __syncthreads();
    if (threadIdx.x == 0) *s_last = cta_partial(a, si, red);
    __syncthreads();
    if (!*s_last) return;
    last_partials(a, si, prob, only_x, red);
    __syncthreads();
    if (threadIdx.x == 0) last_finish<PASS, ROLE, SC>(a, si, pr, only_x, active, red, nullptr);
}

// The same for the two systems of a paired launch: both arrivals first
// (threads 0 and 32), then in a CTA that is last for either system the
// partial sums of each such system, and the two finishers at once in two
// warps.
template <int PASS, int RA, int RB, bool SC>
__device__ __forceinline__ void stream_tail2(const StreamArgs& a, int sa, int sb, int prob, const Prob& pr,
                                             SAcc& acca, SAcc& accb, df (*red)[kSWarps][3], int* s_last) {
    __syncthreads();
    warp_sums_to(acca, red[0]);
    warp_sums_to(accb, red[1]);
    __syncthreads();
    if (threadIdx.x == 0) s_last[0] = cta_partial(a, sa, red[0]);
    if (threadIdx.x == 32) s_last[1] = cta_partial(a, sb, red[1]);
    __syncthreads();
    const bool la = s_last[0], lb = s_last[1];
    if (!la && !lb) return;
    last_partials2(a, sa, sb, la, lb, prob, red);
    __syncthreads();
    if (la && threadIdx.x == 0) last_finish<PASS, RA, SC>(a, sa, pr, false, a.active, red[0], a.pshared);
    if (lb && threadIdx.x == 32) last_finish<PASS, RB, SC>(a, sb, pr, false, a.active2, red[1], nullptr);
}

// One system's whole pass (status: its LSQR status, read at launch).
template <int PASS, int ROLE, bool SC>
__device__ __forceinline__ void stream_pass(const StreamArgs& a, int si, int status, int* active, SCtx& s_ctx,
                                            df* sb, df (*red)[3], int* s_last) {
    const Sys sy = a.sys[si];
    const Prob pr = a.probs[sy.prob];
    __syncthreads();  // s_ctx may still be read by an earlier pass of this CTA
    if (threadIdx.x == 0) stream_ctx<PASS, ROLE>(a, sy, pr, si, s_ctx);
    __syncthreads();
    const SCtx& c = s_ctx;
    // a stopped system's last deferred update: LSQR's x-update in its
    // v-pass, LSMR's (hbar, x, h) updates in its u-pass
    const bool only_x = status == S_FINAL && (ROLE == ROLE_V) == !a.lsmr;
    SAcc acc;
    sacc_zero(acc);
    if (only_x) {
        for (int r = blockIdx.x * kSThreads + threadIdx.x; r < c.N - 1; r += a.gx * kSThreads) {
            if (ROLE == ROLE_V) {
                c.X[r] = df_fma(c.sc.xc, c.W[r], c.X[r]);
            } else {
                const df h = c.W[r];
                const df hb = df_fma(c.sc.nhc, c.HB[r], h);
                c.HB[r] = hb;
                c.X[r] = df_fma(c.sc.xc, hb, c.X[r]);
                c.W[r] = df_fma(c.IN[r], c.sc.c1, df_mul(c.sc.nw, h));
            }
        }
    } else {
        stream_units<PASS, ROLE, SC>(a, si, sy.prob, c, sb, acc);
    }
    stream_tail<PASS, ROLE, SC>(a, si, sy.prob, pr, acc, only_x, active, red, s_last);
}

// One pass of the systems a.slist[blockIdx.y]: PASS_G or PASS_GT, ROLE_U or
// ROLE_V (the product and update of run_tile), SC = diagonal scaling.
template <int PASS, int ROLE, bool SC>
__global__ void __launch_bounds__(kSThreads, 4) k_stream(StreamArgs a) {
    __shared__ df sbuf[kSWarps][kSSocBig];
    __shared__ df red[kSWarps][3];
    __shared__ int s_last;
    __shared__ SCtx s_ctx;
    const int si = a.slist[blockIdx.y];
    const int status = a.state[si].status;
    if (status == S_DONE) return;
    stream_pass<PASS, ROLE, SC>(a, si, status, a.active, s_ctx, sbuf[threadIdx.x >> 5], red, &s_last);
}

// One pass of pairs of systems of one problem that iterate in step: a
// JVP system (mode 0) a.slist[2 y] and a VJP system (mode 1) a.slist[2 y + 1]
// whose own passes run one pass behind, so that both need the same product
// now (PASS_G: the JVP's u-update and the VJP's v-update; PASS_GT: the JVP's
// v-update and the VJP's next u-update) and read M once.  A pair with one
// system stopped (or in its last x-update) runs the one-system pass for
// each system still iterating.  The JVP systems count down a.active, the
// VJP systems a.active2.
template <int PASS, bool SC>
__global__ void __launch_bounds__(kSThreads, kS2Ctas) k_stream2(StreamArgs a) {
    constexpr int RA = PASS == PASS_G ? ROLE_U : ROLE_V;
    constexpr int RB = PASS == PASS_G ? ROLE_V : ROLE_U;
    __shared__ df sbuf[kSWarps][kSSocBig];
    __shared__ df red[2][kSWarps][3];
    __shared__ int s_last[2];
    __shared__ SCtx s_ctx[2];
    const int sa = a.slist[2 * blockIdx.y], sb = a.slist[2 * blockIdx.y + 1];
    const int ta = a.state[sa].status, tb = a.state[sb].status;
    const bool la = ta != S_DONE, lb = tb != S_DONE;
    // a stopped system's last update pass (LSQR: a v-pass, LSMR: a u-pass)
    const bool xa = ta == S_FINAL && (RA == ROLE_V) == !a.lsmr;
    const bool xb = tb == S_FINAL && (RB == ROLE_V) == !a.lsmr;
    df* sbw = sbuf[threadIdx.x >> 5];
    if (!(la && lb) || xa || xb) {
        if (la) stream_pass<PASS, RA, SC>(a, sa, ta, a.active, s_ctx[0], sbw, red[0], &s_last[0]);
        if (lb) stream_pass<PASS, RB, SC>(a, sb, tb, a.active2, s_ctx[1], sbw, red[0], &s_last[0]);
        return;
    }
    const Sys sya = a.sys[sa], syb = a.sys[sb];
    const Prob pr = a.probs[sya.prob];
    if (threadIdx.x == 0) {
        stream_ctx<PASS, RA>(a, sya, pr, sa, s_ctx[0]);
        stream_ctx<PASS, RB>(a, syb, pr, sb, s_ctx[1]);
    }
    __syncthreads();
    SAcc acca, accb;
    sacc_zero(acca);
    sacc_zero(accb);
    stream_units2<PASS, RA, RB, SC>(a, sa, sb, sya.prob, s_ctx[0], s_ctx[1], sbw, acca, accb);
    stream_tail2<PASS, RA, RB, SC>(a, sa, sb, sya.prob, pr, acca, accb, red, s_last);
}

// The systems of [s0, s0 + ns) still iterating (status other than
// S_DONE), in order, into slist; their number into *count.  One warp.
__global__ void k_stream_compact(const LsqrState* state, int s0, int ns, int32_t* slist, int32_t* count) {
    const int lane = threadIdx.x & 31;
    int base = 0;
    for (int i0 = 0; i0 < ns; i0 += 32) {
        const int i = i0 + lane;
        const bool live = i < ns && state[s0 + i].status != S_DONE;
        const unsigned m = __ballot_sync(0xffffffffu, live);
        if (live) slist[base + __popc(m & ((1u << lane) - 1u))] = s0 + i;
        base += __popc(m);
    }
    if (lane == 0) *count = base;
}

// The pairs (sa0 + i, sb0 + i), i < ns, with a system still iterating, in
// order, into slist (two entries a pair); their number into *count.  One warp.
__global__ void k_stream_compact2(const LsqrState* state, int sa0, int sb0, int ns, int32_t* slist,
                                  int32_t* count) {
    const int lane = threadIdx.x & 31;
    int base = 0;
    for (int i0 = 0; i0 < ns; i0 += 32) {
        const int i = i0 + lane;
        const bool live = i < ns && (state[sa0 + i].status != S_DONE || state[sb0 + i].status != S_DONE);
        const unsigned m = __ballot_sync(0xffffffffu, live);
        if (live) {
            const int o = 2 * (base + __popc(m & ((1u << lane) - 1u)));
            slist[o] = sa0 + i;
            slist[o + 1] = sb0 + i;
        }
        base += __popc(m);
    }
    if (lane == 0) *count = base;
}

// ---- entering and leaving the engine (per call and continuation round)
// State: the right-hand side's scale (a power of two putting ||b|| in
// [1/2, 1)), the tau entries into StreamSys, the scaled LSQR scalars
// (x, phibar, xcoef and bnorm are proportional to the right-hand side, and
// so are u, beta and 1/uc2 before the first u-update) and the first u-pass's
// df64 scalars.  One thread per system.
__global__ void k_stream_enter_state(StreamArgs a, int upass_g, int sc) {
    const int si = a.s0 + (int)blockIdx.x;
    if (threadIdx.x != 0) return;
    LsqrState* st = a.state + si;
    StreamSys* ss = a.ssys + si;
    ss->pad = st->status != S_DONE;
    if (!ss->pad) return;
    const Sys sy = a.sys[si];
    const Prob pr = a.probs[sy.prob];
    const int rN = pr.n + pr.m;
    const double* U = reinterpret_cast<const double*>(a.U + sy.voff);
    const double* V = reinterpret_cast<const double*>(a.V + sy.voff);
    const double* W = reinterpret_cast<const double*>(a.W + sy.voff);
    const double* X = reinterpret_cast<const double*>(a.X + sy.voff);
    const double* XI = reinterpret_cast<const double*>(a.XI + sy.voff);
    double s = 1.0;
    // LSMR keeps its scalars unscaled (its recurrences carry many quantities
    // proportional to ||b||); LSQR's right-hand side goes to norm [1/2, 1)
    if (!a.lsmr && st->bnorm > 0.0 && finite64(st->bnorm)) {
        int e = 0;
        frexp(st->bnorm, &e);
        s = ldexp(1.0, -e);
    }
    const int us = st->iters == 0;
    ss->scale = s;
    ss->uscaled = us;
    st->phibar *= s;
    st->xcoef *= s;
    st->bnorm *= s;
    if (us) {
        st->beta *= s;
        st->uc2 /= s;
    }
    ss->tau[TS_U] = U[rN] * (us ? s : 1.0);
    ss->tau[TS_V] = V[rN];
    ss->tau[TS_W] = W[rN];
    ss->tau[TS_X] = X[rN] * s;
    ss->tau[TS_XI] = XI[rN];
    ss->tau[TS_HB] = reinterpret_cast<const double*>(a.HB + sy.voff)[rN];
    const double tin = ss->tau[TS_V];
    const double tt = sc ? (upass_g ? a.cdd[pr.doff + rN] : a.rwd[pr.doff + rN]) * tin : tin;
    StreamScal q;
    q.c1 = df_from(st->uc1);
    q.nc2 = df_from(-st->uc2);
    q.nw = df_from(-st->wcoef);
    q.xc = df_from(st->xcoef);
    q.tt = df_from(tt);
    q.nhc = df_from(a.lsmr ? -st->hcoef : 0.0);
    q.upd = a.lsmr ? st->upd : 0;
    q.lsmr = a.lsmr;
    a.scal[si] = q;
}

// Vectors: FP64 -> df64 pairs in place (rows below the tau entry), with the
// scale.  blockIdx.y = system.
__global__ void k_stream_enter_vec(StreamArgs a) {
    const int si = a.s0 + (int)blockIdx.y;
    const StreamSys ss = a.ssys[si];
    if (!ss.pad) return;
    const Sys sy = a.sys[si];
    const Prob pr = a.probs[sy.prob];
    const int rN = pr.n + pr.m;
    const double su = ss.uscaled ? ss.scale : 1.0;
    double* U = reinterpret_cast<double*>(a.U + sy.voff);
    double* V = reinterpret_cast<double*>(a.V + sy.voff);
    double* W = reinterpret_cast<double*>(a.W + sy.voff);
    double* X = reinterpret_cast<double*>(a.X + sy.voff);
    double* XI = reinterpret_cast<double*>(a.XI + sy.voff);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rN; r += gridDim.x * blockDim.x) {
        a.U[sy.voff + r] = df_from(U[r] * su);
        a.V[sy.voff + r] = df_from(V[r]);
        a.W[sy.voff + r] = df_from(W[r]);
        a.X[sy.voff + r] = df_from(X[r] * ss.scale);
        a.XI[sy.voff + r] = df_from(XI[r]);
    }
    if (!a.lsmr) return;
    double* HB = reinterpret_cast<double*>(a.HB + sy.voff);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rN; r += gridDim.x * blockDim.x)
        a.HB[sy.voff + r] = df_from(HB[r]);
}

// df64 pairs -> FP64 in place, the scale undone (U only while no u-update
// has happened since entering).  Runs before k_stream_exit_state.
__global__ void k_stream_exit_vec(StreamArgs a) {
    const int si = a.s0 + (int)blockIdx.y;
    const StreamSys ss = a.ssys[si];
    if (!ss.pad) return;
    const Sys sy = a.sys[si];
    const Prob pr = a.probs[sy.prob];
    const int rN = pr.n + pr.m;
    const bool u_still = ss.uscaled && a.state[si].iters == 0;
    const double iu = u_still ? 1.0 / ss.scale : 1.0, ix = 1.0 / ss.scale;
    double* U = reinterpret_cast<double*>(a.U + sy.voff);
    double* V = reinterpret_cast<double*>(a.V + sy.voff);
    double* W = reinterpret_cast<double*>(a.W + sy.voff);
    double* X = reinterpret_cast<double*>(a.X + sy.voff);
    double* XI = reinterpret_cast<double*>(a.XI + sy.voff);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rN; r += gridDim.x * blockDim.x) {
        U[r] = df_to(a.U[sy.voff + r]) * iu;
        V[r] = df_to(a.V[sy.voff + r]);
        W[r] = df_to(a.W[sy.voff + r]);
        X[r] = df_to(a.X[sy.voff + r]) * ix;
        XI[r] = df_to(a.XI[sy.voff + r]);
    }
    if (!a.lsmr) return;
    double* HB = reinterpret_cast<double*>(a.HB + sy.voff);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rN; r += gridDim.x * blockDim.x)
        HB[r] = df_to(a.HB[sy.voff + r]);
}

__global__ void k_stream_exit_state(StreamArgs a) {
    const int si = a.s0 + (int)blockIdx.x;
    if (threadIdx.x != 0) return;
    StreamSys* ss = a.ssys + si;
    if (!ss->pad) return;
    LsqrState* st = a.state + si;
    const Sys sy = a.sys[si];
    const Prob pr = a.probs[sy.prob];
    const int rN = pr.n + pr.m;
    const bool u_still = ss->uscaled && st->iters == 0;
    const double iu = u_still ? 1.0 / ss->scale : 1.0, ix = 1.0 / ss->scale;
    st->phibar *= ix;
    st->xcoef *= ix;
    st->bnorm *= ix;
    if (u_still) {
        st->beta *= iu;
        st->uc2 /= iu;
    }
    reinterpret_cast<double*>(a.U + sy.voff)[rN] = ss->tau[TS_U] * iu;
    reinterpret_cast<double*>(a.V + sy.voff)[rN] = ss->tau[TS_V];
    reinterpret_cast<double*>(a.W + sy.voff)[rN] = ss->tau[TS_W];
    reinterpret_cast<double*>(a.X + sy.voff)[rN] = ss->tau[TS_X] * ix;
    reinterpret_cast<double*>(a.XI + sy.voff)[rN] = ss->tau[TS_XI];
    if (a.lsmr) reinterpret_cast<double*>(a.HB + sy.voff)[rN] = ss->tau[TS_HB];
    ss->pad = 0;
}

}  // namespace qcpd
