// Entry points of the C ABI (include/qcpd.h) and the LSQR driver.
//
// One JVP/VJP solve (Sec. 3.1 / 3.2) is, on the plan's stream:
//   right-hand side kernel (dN or D phi^T w, and ||b||)
//   one G^T- (JVP) or G-pass (VJP) starting the bidiagonalisation
//   repeated iterations: [G-pass, G^T-pass] (JVP) or [G^T-pass, G-pass]
//     (VJP), each a single launch over all tiles of all systems, replayed
//     from a captured CUDA graph in chunks of check_every iterations
//   output kernel (D phi dz, or the pattern-restricted D_theta N^T r)
//   optionally one more pass for the true residual.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "qcpd_cluster.h"
#include "qcpd_stream.h"
#include "qcpd_kernels.cuh"
#include "qcpd_plan.h"

namespace qcpd {
const char* last_error();
int create_plan(qcp_plan* p, const qcp_problem* probs, const qcp_solution* sols);

// precond: QCP_PRECOND_NONE, _EQUILIBRATE or _DIAG (caller's C, W = I)
template <typename T>
static PlanView<T> view(qcp_plan* p, int precond) {
    const bool scaled = precond != QCP_PRECOND_NONE;
    PlanView<T> v;
    v.tiles = p->d_tiles.as<Tile>();
    v.sys = p->d_sys.as<Sys>();
    v.probs = p->d_prob.as<Prob>();
    v.state = p->d_state.as<LsqrState>();
    v.R = Reduce{p->d_tpart.as<Part>(), p->d_gpart.as<Part>(), p->d_gcnt.as<int32_t>(), p->d_scnt.as<int32_t>(),
                 p->d_groups.as<Group>()};
    v.active = p->d_active.as<int>();
    v.split_cnt = p->d_split_cnt.as<int32_t>();
    v.row_part = p->d_row_part.as<double>();
    v.mrowptr = p->d_mrowptr.as<int64_t>();
    v.mcol = p->d_mcol.as<int32_t>();
    v.mval = p->d_mval.as<T>();
    v.mvalG = scaled ? p->d_mvalG.as<T>() : p->d_mval.as<T>();
    v.mvalT = scaled ? p->d_mvalT.as<T>() : p->d_mval.as<T>();
    v.rw = p->d_rw.as<double>();
    v.cd = p->d_cd.as<double>();
    v.scaled = scaled ? 1 : 0;
    if (precond == QCP_PRECOND_DIAG) {  // W = I, the caller's column scaling (block-averaged)
        v.rw = p->d_onesD.as<double>();
        v.cd = p->d_cdD.as<double>();
        v.mvalG = p->d_mvalD.as<T>();
        v.mvalT = p->d_mval.as<T>();
    }
    v.mvmap = p->d_mvmap.as<int32_t>();
    v.coefA = p->d_coefA.as<double>();
    v.coefB = p->d_coefB.as<double>();
    v.pz = p->d_pz.as<double>();
    v.zy = p->d_zy.as<double>();
    v.flag = p->d_flag.as<int8_t>();
    v.blocks = p->d_blocks.as<SocBlock>();
    v.U = p->d_U.as<double>();
    v.V = p->d_V.as<double>();
    v.W = p->d_W.as<double>();
    v.X = p->d_X.as<double>();
    v.XI = p->d_XI.as<double>();
    v.RHS = p->d_RHS.as<double>();
    v.HB = p->d_HB.as<double>();
    v.lsmr = 0;
    v.psd = (p->kpsd || p->ndense) ? p->d_psd.as<double>() : nullptr;
    v.kpsd = p->kpsd;
    v.rmax = p->rmax;
    v.long_chunk = p->long_chunk;
    v.tile0 = 0;
    return v;
}

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
    // static + dynamic shared memory above 48 KB needs the opt-in
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, bool SC>
static int set_smem_attrs_sc(size_t smem) {
    QCP_CUDA(allow_smem(k_pass<PASS_G, ROLE_U, SC, T>, smem));
    QCP_CUDA(allow_smem(k_pass<PASS_G, ROLE_V, SC, T>, smem));
    QCP_CUDA(allow_smem(k_pass<PASS_G, ROLE_RES, SC, T>, smem));
    QCP_CUDA(allow_smem(k_pass<PASS_GT, ROLE_U, SC, T>, smem));
    QCP_CUDA(allow_smem(k_pass<PASS_GT, ROLE_V, SC, T>, smem));
    QCP_CUDA(allow_smem(k_pass<PASS_GT, ROLE_RES, SC, T>, smem));
    QCP_CUDA(allow_smem(k_pass<PASS_G, ROLE_WARM, SC, T>, smem));
    QCP_CUDA(allow_smem(k_pass<PASS_GT, ROLE_WARM, SC, T>, smem));
    return QCP_OK;
}

template <typename T>
static int set_smem_attrs(size_t smem) {
    QCP_TRY((set_smem_attrs_sc<T, false>(smem)));
    QCP_TRY((set_smem_attrs_sc<T, true>(smem)));
    QCP_CUDA(allow_smem(k_vjp_rhs<T>, smem));
    QCP_CUDA(allow_smem(k_jvp_out<T>, smem));
    QCP_CUDA(allow_smem(k_dpi<T>, smem));
    return QCP_OK;
}

// Launch one pass kernel: PASS x ROLE, scaled or not.
template <int PASS, int ROLE, typename T>
static void launch_pass(const PlanView<T>& v, int ntiles, size_t smem, cudaStream_t st) {
    if (v.scaled) k_pass<PASS, ROLE, true, T><<<ntiles, kThreads, smem, st>>>(v);
    else k_pass<PASS, ROLE, false, T><<<ntiles, kThreads, smem, st>>>(v);
}

// Launch one LSQR iteration: u-update pass then v-update pass.
template <typename T>
static void launch_iter(int mode, const PlanView<T>& v, int ntiles, size_t smem, cudaStream_t st) {
    if (mode == 0) {
        launch_pass<PASS_G, ROLE_U, T>(v, ntiles, smem, st);
        launch_pass<PASS_GT, ROLE_V, T>(v, ntiles, smem, st);
    } else {
        launch_pass<PASS_GT, ROLE_U, T>(v, ntiles, smem, st);
        launch_pass<PASS_G, ROLE_V, T>(v, ntiles, smem, st);
    }
}

template <typename T>
static int run_chunk(qcp_plan* p, int mode, int nsys, const PlanView<T>& v, int ntiles, size_t smem, int chunk,
                     bool use_graph) {
    cudaStream_t st = p->stream;
    if (!use_graph || chunk < 2) {
        for (int c = 0; c < chunk; ++c) launch_iter<T>(mode, v, ntiles, smem, st);
        QCP_CUDA(cudaGetLastError());
        p->last_launches += 2 * chunk;
        return QCP_OK;
    }
    GraphKey key{QCP_ENGINE_PASSES, mode, v.tile0, nsys, chunk, p->view_precond, v.lsmr};
    auto it = p->graphs.find(key);
    if (it == p->graphs.end()) {
        cudaGraph_t g = nullptr;
        QCP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int c = 0; c < chunk; ++c) launch_iter<T>(mode, v, ntiles, smem, st);
        cudaError_t le = cudaGetLastError();
        cudaError_t ee = cudaStreamEndCapture(st, &g);
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            set_error("graph capture failed: %s", cudaGetErrorString(le != cudaSuccess ? le : ee));
            return QCP_ERR_CUDA;
        }
        cudaGraphExec_t ge = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
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

static int status_of(const LsqrState& s, double kink, double kink_tol) {
    if (s.outcome == O_BREAKDOWN) return QCP_BREAKDOWN;
    if (s.outcome == O_MAXITER) return QCP_NOT_CONVERGED;
    if (kink < kink_tol) return QCP_WARN_NEAR_KINK;
    return QCP_OK;
}

static int worse(int a, int b) {
    auto rank = [](int s) {
        switch (s) {
            case QCP_BREAKDOWN: return 3;
            case QCP_NOT_CONVERGED: return 2;
            case QCP_WARN_NEAR_KINK: return 1;
            default: return 0;
        }
    };
    return rank(b) > rank(a) ? b : a;
}

// Iterate until no system is active (host checks every check_every
// iterations) or the iteration budget of this round is spent.
template <typename T>
static int iterate(qcp_plan* p, int mode, int nsys, const PlanView<T>& v, int ntiles, size_t smem,
                   const qcp_options& opts) {
    int64_t done_iters = 0;
    const int64_t cap = opts.maxiter + 1;
    while (done_iters < cap) {
        int64_t chunk = opts.check_every > 0 ? opts.check_every : cap;
        chunk = std::min<int64_t>(chunk, cap - done_iters);
        const bool graph_ok = opts.use_graph && opts.check_every > 0 && chunk == opts.check_every;
        QCP_CUDA(cudaEventRecord(p->ev0, p->stream));
        QCP_TRY(run_chunk<T>(p, mode, nsys, v, ntiles, smem, (int)chunk, graph_ok));
        QCP_CUDA(cudaEventRecord(p->ev1, p->stream));
        done_iters += chunk;
        p->pass_launches += 2 * chunk;
        if (opts.check_every > 0) {
            QCP_CUDA(cudaMemcpyAsync(p->h_active, v.active, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
            QCP_CUDA(cudaStreamSynchronize(p->stream));
        } else {
            QCP_CUDA(cudaEventSynchronize(p->ev1));
        }
        float ms = 0.0f;
        QCP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->pass_ms += ms;
        if (opts.check_every > 0 && *p->h_active <= 0) break;
    }
    return QCP_OK;
}

// All remaining iterations in one cooperative launch (QCP_ENGINE_PERSISTENT).
template <typename T>
static int iterate_persistent(qcp_plan* p, int mode, const PlanView<T>& v, int ntiles, size_t smem,
                              const qcp_options& opts) {
    cudaStream_t st = p->stream;
    int dev = 0, nsm = 0, per_sm = 0;
    QCP_CUDA(cudaGetDevice(&dev));
    QCP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    void* fn = nullptr;
    if (mode == 0) fn = v.scaled ? (void*)k_persist<0, true, T> : (void*)k_persist<0, false, T>;
    else fn = v.scaled ? (void*)k_persist<1, true, T> : (void*)k_persist<1, false, T>;
    QCP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    QCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
    if (per_sm < 1) {
        set_error("persistent mode: a CTA of this plan does not fit on an SM");
        return QCP_ERR_ARG;
    }
    int grid = std::min(ntiles, per_sm * nsm);
    PersistCtl c;
    int32_t* ctl = p->d_pctl.as<int32_t>();
    c.bar_count = reinterpret_cast<unsigned*>(ctl);
    c.bar_gen = reinterpret_cast<unsigned*>(ctl + 1);
    c.stop = ctl + 2;
    c.err = ctl + 3;
    c.max_iters = opts.maxiter + 2;
    c.spin_limit = p->barrier_polls > 0 ? (unsigned long long)p->barrier_polls : kSpinLimit;
    c.hold_ns = p->barrier_hold_ns;
    QCP_CUDA(cudaMemsetAsync(ctl, 0, 4 * sizeof(int32_t), st));
    PlanView<T> va = v;
    void* args[] = {(void*)&va, (void*)&c, (void*)&ntiles};
    QCP_CUDA(cudaEventRecord(p->ev0, st));
    QCP_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, smem, st));
    QCP_CUDA(cudaEventRecord(p->ev1, st));
    QCP_CUDA(cudaEventSynchronize(p->ev1));
    float ms = 0.0f;
    QCP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    p->pass_ms += ms;
    p->last_launches += 1;
    int32_t hc[4];
    QCP_CUDA(cudaMemcpy(hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost));
    if (hc[3]) {
        set_error("persistent mode: a grid barrier gave up waiting (bounded spin)");
        return QCP_ERR_TIMEOUT;
    }
    return QCP_OK;
}

// The v-update pass of the operator: starts the bidiagonalisation and resumes it.
template <typename T>
static void launch_v_pass(int mode, const PlanView<T>& v, int ntiles, size_t smem, cudaStream_t st) {
    if (mode == 0) launch_pass<PASS_GT, ROLE_V, T>(v, ntiles, smem, st);
    else launch_pass<PASS_G, ROLE_V, T>(v, ntiles, smem, st);
}

template <typename T>
static void launch_output(qcp_plan* p, int mode, int nsys, const PlanView<T>& v, int ntiles, size_t smem,
                          const OutArgs<T>& out, bool residual) {
    cudaStream_t st = p->stream;
    if (mode == 0) {
        k_jvp_out<T><<<ntiles, kThreads, smem, st>>>(v, out);
        if (residual) launch_pass<PASS_G, ROLE_RES, T>(v, ntiles, smem, st);
    } else {
        int maxrows = 0;
        for (int s = out.s0; s < out.s0 + nsys; ++s) {
            const Prob& pr = p->hprob[p->hsys[s].prob];
            maxrows = std::max(maxrows, pr.n + pr.m);
        }
        dim3 grid((unsigned)std::max(1, std::min(4096, (maxrows + kWarps - 1) / kWarps)), (unsigned)nsys);
        k_vjp_out<T><<<grid, kThreads, 0, st>>>(v, out, p->d_pip.as<int64_t>(), p->d_pix.as<int32_t>(),
                                                p->d_aip.as<int64_t>(), p->d_aix.as<int32_t>());
        if (residual) launch_pass<PASS_GT, ROLE_RES, T>(v, ntiles, smem, st);
    }
    p->last_launches += 1 + (residual ? 1 : 0);
}

// QCP_PRECOND_DIAG: the caller's column scaling C, averaged over each
// second-order-cone block (the G-pass multiplies M diag(C) with D Pi x, which
// equals M D Pi C x only when C is constant on every block), unit W, and
// M diag(C).
template <typename T>
__global__ void k_scale_cols(const T* mval, const int32_t* mcol, int64_t k0, int64_t k1, const double* d, T* out) {
    const int64_t k = k0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < k1) out[k] = (T)((double)mval[k] * d[mcol[k]]);
}

__global__ void k_block_mean(const SocBlock* blocks, int64_t nb, double* d) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const SocBlock B = blocks[b];
    double s = 0.0;
    for (int k = 0; k < B.dim; ++k) s += d[B.start + k];
    s /= B.dim;
    for (int k = 0; k < B.dim; ++k) d[B.start + k] = s;
}

__global__ void k_set_ones(double* x, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = 1.0;
}


template <typename T>
static int prepare_diag(qcp_plan* p, const double* d) {
    cudaStream_t st = p->stream;
    if (!p->d_cdD.p) {
        QCP_TRY(p->d_cdD.alloc(sizeof(double) * (size_t)p->N_tot));
        QCP_TRY(p->d_onesD.alloc(sizeof(double) * (size_t)p->N_tot));
        QCP_TRY(p->d_mvalD.alloc(sizeof(T) * (size_t)(p->mnnz + 16)));
        QCP_CUDA(cudaMemsetAsync(p->d_mvalD.p, 0, sizeof(T) * (size_t)(p->mnnz + 16), st));
        k_set_ones<<<(unsigned)((p->N_tot + 255) / 256), 256, 0, st>>>(p->d_onesD.as<double>(), p->N_tot);
    }
    QCP_CUDA(cudaMemcpyAsync(p->d_cdD.p, d, sizeof(double) * (size_t)p->N_tot, cudaMemcpyDeviceToDevice, st));
    for (int pi = 0; pi < p->nprob; ++pi) {
        const Prob& pr = p->hprob[pi];
        if (pr.nsoc > 0)
            k_block_mean<<<(unsigned)((pr.nsoc + 255) / 256), 256, 0, st>>>(p->d_blocks.as<SocBlock>() + pr.soff,
                                                                             pr.nsoc, p->d_cdD.as<double>() + pr.doff);
    }
    for (int pi = 0; pi < p->nprob; ++pi) {
        const Prob& pr = p->hprob[pi];
        const int64_t k0 = p->h_mrowptr[pr.mrow], k1 = p->h_mrowptr[pr.mrow + pr.n + pr.m + 1];
        if (k1 > k0)
            k_scale_cols<T><<<(unsigned)((k1 - k0 + 255) / 256), 256, 0, st>>>(
                p->d_mval.as<T>(), p->d_mcol.as<int32_t>(), k0, k1, p->d_cdD.as<double>() + pr.doff,
                p->d_mvalD.as<T>());
    }
    QCP_CUDA(cudaGetLastError());
    return QCP_OK;
}

// A range of a plan's systems that a call solves in one mode: JVP (mode 0)
// or VJP (mode 1) on systems [s0, s0 + ns), with the user arrays of that
// range.
template <typename T>
struct Seg {
    int mode;
    int s0, ns;
    RhsArgs<T> ra;
    OutArgs<T> out;
};

// The view of a range: tile launches start at its first tile, and it has
// its own count of iterating systems.
template <typename T>
static PlanView<T> seg_view(const qcp_plan* p, PlanView<T> v, const Seg<T>& g, int gi) {
    v.tile0 = p->batched ? 0 : g.s0 * p->tiles_per_sys;
    v.active = p->d_active.as<int>() + gi;
    return v;
}

static int seg_tiles(const qcp_plan* p, int ns) { return p->batched ? p->ntiles : ns * p->tiles_per_sys; }

// Solve the systems of nseg ranges (the plan's systems [0, nsys) in all).
// Every range gets its right-hand side and first v-pass, then the engine
// iterates: the cluster engine runs the ranges side by side, the others one
// after another.  Outputs and the true-residual continuation are per range.
template <typename T>
static int solve(qcp_plan* p, const Seg<T>* segs, int nseg, const qcp_options* opts_in, qcp_info* info) {
    qcp_options opts;
    if (opts_in) opts = *opts_in;
    else qcp_default_options(&opts);
    if (!(opts.rtol >= 0.0) || opts.maxiter < 1 || opts.check_every < 0) {
        set_error("bad options: rtol >= 0, maxiter >= 1, check_every >= 0 required");
        return QCP_ERR_ARG;
    }
    if (opts.solver != 0 && opts.solver != 1) {
        set_error("solver must be 0 (LSQR) or 1 (LSMR)");
        return QCP_ERR_ARG;
    }
    if (opts.solver == 1 && opts.engine == QCP_ENGINE_CLUSTER_FP64) {
        set_error("LSMR runs on the pass, persistent, stream or (double-float) cluster engine");
        return QCP_ERR_ARG;
    }
    if (opts.precond != QCP_PRECOND_NONE && opts.precond != QCP_PRECOND_EQUILIBRATE &&
        opts.precond != QCP_PRECOND_DIAG && opts.precond != QCP_PRECOND_JACOBI) {
        set_error("precond must be QCP_PRECOND_NONE, _EQUILIBRATE, _DIAG or _JACOBI");
        return QCP_ERR_ARG;
    }
    // Jacobi is the diagonal right preconditioner with the plan's column norms
    if (opts.precond == QCP_PRECOND_JACOBI) {
        if (!p->d_cdJ.p) {
            QCP_TRY(p->d_cdJ.alloc(sizeof(double) * (size_t)p->N_tot));
            const int rc = jacobi_cols(p, p->d_cdJ.as<double>());
            if (rc != QCP_OK) {
                p->d_cdJ.release();
                return rc;
            }
        }
        opts.precond = QCP_PRECOND_DIAG;
        opts.precond_d = p->d_cdJ.as<double>();
    }
    if (opts.precond == QCP_PRECOND_DIAG && !opts.precond_d) {
        set_error("QCP_PRECOND_DIAG needs opts->precond_d");
        return QCP_ERR_ARG;
    }
    if (opts.engine < QCP_ENGINE_PASSES || opts.engine > QCP_ENGINE_STREAM) {
        set_error("engine must be one of QCP_ENGINE_PASSES, _PERSISTENT, _CLUSTER, _AUTO, _CLUSTER_FP64, _STREAM");
        return QCP_ERR_ARG;
    }
    if (nseg < 1 || nseg > kMaxSegments) {
        set_error("internal: %d system ranges in one call", nseg);
        return QCP_ERR_ARG;
    }
    if (nseg > 1 && opts.warm_start) {
        set_error("a warm start takes a call of one kind (JVP or VJP)");
        return QCP_ERR_ARG;
    }
    int nsys = 0;
    for (int gi = 0; gi < nseg; ++gi) nsys = std::max(nsys, segs[gi].s0 + segs[gi].ns);
    int engine = opts.engine;
    if (engine == QCP_ENGINE_AUTO && p->tuned_engine >= 0) engine = p->tuned_engine;
    // the stream engine takes no diagonal preconditioner: an autotuned choice of it becomes AUTO
    if (engine == QCP_ENGINE_STREAM && opts.engine == QCP_ENGINE_AUTO && opts.precond == QCP_PRECOND_DIAG)
        engine = QCP_ENGINE_AUTO;

    if (engine == QCP_ENGINE_CLUSTER || engine == QCP_ENGINE_AUTO || engine == QCP_ENGINE_CLUSTER_FP64) {
        bool fits = false;
        QCP_TRY(cluster_ready(p, nsys, &fits, opts.solver == 1));
        if (fits) {
            engine = QCP_ENGINE_CLUSTER;
        } else if (engine != QCP_ENGINE_AUTO) {
            set_error("cluster engine: a problem's vectors do not fit in the shared memory of 16 CTAs");
            return QCP_ERR_ARG;
        } else if (opts.precond == QCP_PRECOND_DIAG) {
            engine = QCP_ENGINE_PASSES;  // the stream engine takes no diagonal preconditioner
        } else {
            // too large for the cluster engine: the stream engine where it can run the plan
            bool sok = false;
            QCP_TRY(stream_ready(p, &sok));
            engine = sok ? QCP_ENGINE_STREAM : QCP_ENGINE_PASSES;
        }
    } else if (engine == QCP_ENGINE_STREAM) {
        if (opts.precond == QCP_PRECOND_DIAG) {
            set_error("the stream engine runs with precond NONE or EQUILIBRATE");
            return QCP_ERR_ARG;
        }
        bool sok = false;
        QCP_TRY(stream_ready(p, &sok));
        if (!sok) return QCP_ERR_ARG;  // stream_ready has set the reason
    }
    cudaStream_t st = p->stream;
    if (opts.precond == QCP_PRECOND_DIAG) QCP_TRY(prepare_diag<T>(p, opts.precond_d));
    p->view_precond = opts.precond;
    PlanView<T> v = view<T>(p, opts.precond);
    v.lsmr = opts.solver == 1 ? 1 : 0;
    const size_t smem = tile_smem_bytes(p->rmax, p->kpsd);
    QCP_TRY(set_smem_attrs<T>(smem));
    p->last_launches = 0;
    p->last_engine = engine;
    p->last_mode = nseg == 1 ? segs[0].mode : 2;
    p->last_nsys = nsys;
    p->last_jvp_sys = segs[0].mode == 0 ? segs[0].s0 + segs[0].ns : 0;
    p->pass_ms = 0.0;
    p->pass_launches = 0;
    p->shared_passes = 0;
    QCP_CUDA(cudaMemsetAsync(p->d_active.p, 0, kMaxSegments * sizeof(int), st));
    for (int gi = 0; gi < nseg; ++gi) {
        const Seg<T>& g = segs[gi];
        const PlanView<T> vs = seg_view(p, v, g, gi);
        const int nt = seg_tiles(p, g.ns);
        RhsArgs<T> ra = g.ra;
        ra.rtol = opts.rtol;
        ra.maxiter = opts.maxiter;
        if (g.mode == 0) k_jvp_rhs<T><<<nt, kThreads, 0, st>>>(vs, ra);
        else k_vjp_rhs<T><<<nt, kThreads, smem, st>>>(vs, ra);
        if (opts.warm_start) {
            // x0 from the caller's iterate; the right-hand side becomes b - Op x0
            int maxN = 1;
            for (int s = g.s0; s < g.s0 + g.ns; ++s) {
                const Prob& pr = p->hprob[p->hsys[s].prob];
                maxN = std::max(maxN, pr.n + pr.m + 1);
            }
            k_warm_init<T><<<dim3((unsigned)std::min(1024, (maxN + 255) / 256), (unsigned)g.ns), 256, 0, st>>>(
                vs, opts.warm_start, g.mode, g.s0);
            if (g.mode == 0) {
                k_dpi<T><<<nt, kThreads, smem, st>>>(vs, vs.X);
                launch_pass<PASS_G, ROLE_WARM, T>(vs, nt, smem, st);
            } else {
                launch_pass<PASS_GT, ROLE_WARM, T>(vs, nt, smem, st);
            }
            p->last_launches += g.mode == 0 ? 3 : 2;
        }
        launch_v_pass<T>(g.mode, vs, nt, smem, st);
        QCP_CUDA(cudaGetLastError());
        p->last_launches += 2;
    }
    // iterate the ranges whose flag is set
    auto run_iterations = [&](const std::vector<int>& todo) -> int {
        if (engine == QCP_ENGINE_CLUSTER) {
            ClusterSeg cs[kMaxSegments];
            int nc = 0;
            for (int gi = 0; gi < nseg; ++gi)
                if (todo[gi]) cs[nc++] = ClusterSeg{segs[gi].mode, segs[gi].s0, segs[gi].ns, gi};
            return iterate_cluster<T>(p, cs, nc, nsys, v, opts);
        }
        if (engine == QCP_ENGINE_STREAM) {
            // a JVP range and a VJP range of equal size on one problem: in step
            if (p->stream_pairing && nseg == 2 && todo[0] && todo[1] && segs[0].mode != segs[1].mode &&
                segs[0].ns == segs[1].ns) {
                const int ja = segs[0].mode == 0 ? 0 : 1, vb = 1 - ja;
                if (stream_can_pair(p, segs[ja].s0, segs[vb].s0, segs[ja].ns))
                    return iterate_stream_pair(p, segs[ja].s0, segs[vb].s0, segs[ja].ns,
                                               p->d_active.as<int>() + ja, p->d_active.as<int>() + vb,
                                               v.scaled != 0, opts);
            }
            for (int gi = 0; gi < nseg; ++gi)
                if (todo[gi])
                    QCP_TRY(iterate_stream(p, segs[gi].mode, segs[gi].s0, segs[gi].ns, p->d_active.as<int>() + gi,
                                           v.scaled != 0, opts));
            return QCP_OK;
        }
        for (int gi = 0; gi < nseg; ++gi) {
            if (!todo[gi]) continue;
            const Seg<T>& g = segs[gi];
            const PlanView<T> vs = seg_view(p, v, g, gi);
            const int nt = seg_tiles(p, g.ns);
            if (engine == QCP_ENGINE_PERSISTENT) QCP_TRY(iterate_persistent<T>(p, g.mode, vs, nt, smem, opts));
            else QCP_TRY(iterate<T>(p, g.mode, g.ns, vs, nt, smem, opts));
        }
        return QCP_OK;
    };
    QCP_TRY(run_iterations(std::vector<int>(nseg, 1)));
    std::vector<LsqrState> hs(nsys);
    std::vector<double> prev_res(nsys, INFINITY);
    const bool residual = opts.compute_residual != 0;
    for (int round = 0;; ++round) {
        for (int gi = 0; gi < nseg; ++gi) {
            const Seg<T>& g = segs[gi];
            launch_output<T>(p, g.mode, g.ns, seg_view(p, v, g, gi), seg_tiles(p, g.ns), smem, g.out, residual);
        }
        QCP_CUDA(cudaGetLastError());
        QCP_CUDA(cudaMemcpyAsync(hs.data(), p->d_state.p, nsys * sizeof(LsqrState), cudaMemcpyDeviceToHost, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        if (!residual || round == 4) break;
        // The Krylov estimate measures the scaled residual; where the true
        // one misses the target, continue the same recurrence with a tighter
        // internal tolerance.
        int resumed[kMaxSegments] = {0, 0};
        int total = 0;
        for (int gi = 0; gi < nseg; ++gi) {
            for (int s = segs[gi].s0; s < segs[gi].s0 + segs[gi].ns; ++s) {
                LsqrState& q = hs[s];
                const bool improving = q.resid_true < 0.5 * prev_res[s];  // else rounding has stalled it
                prev_res[s] = q.resid_true;
                if (q.outcome != O_CONVERGED || !(q.resid_true > opts.rtol) || !(q.alpha > 0.0) ||
                    !isfinite(q.resid_true) || q.iters >= q.maxiter || q.bnorm_true <= 0.0 || !improving)
                    continue;
                q.rtol *= std::max(0.01, 0.5 * opts.rtol / q.resid_true);
                q.status = S_ACTIVE;
                q.outcome = O_RUNNING;
                q.xcoef = 0.0;
                ++resumed[gi];
                ++total;
            }
        }
        if (!total) break;
        QCP_CUDA(cudaMemcpyAsync(p->d_state.p, hs.data(), nsys * sizeof(LsqrState), cudaMemcpyHostToDevice, st));
        QCP_CUDA(cudaMemcpyAsync(p->d_active.p, resumed, kMaxSegments * sizeof(int), cudaMemcpyHostToDevice, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        std::vector<int> todo(nseg, 0);
        for (int gi = 0; gi < nseg; ++gi) {
            if (!resumed[gi]) continue;
            todo[gi] = 1;
            const Seg<T>& g = segs[gi];
            const PlanView<T> vs = seg_view(p, v, g, gi);
            if (v.lsmr) {
                // LSMR's last update pass left u_{k+1}, v_{k+1}, h_{k+1} in
                // place; a JVP's u-pass gathers D Pi(v), which the output
                // pass overwrote
                if (g.mode == 0) {
                    k_dpi<T><<<seg_tiles(p, g.ns), kThreads, smem, st>>>(vs, vs.V);
                    p->last_launches += 1;
                }
            } else {
                launch_v_pass<T>(g.mode, vs, seg_tiles(p, g.ns), smem, st);
                p->last_launches += 1;
            }
        }
        QCP_TRY(run_iterations(todo));
    }
    if (engine != QCP_ENGINE_PASSES && engine != QCP_ENGINE_STREAM) {
        int64_t it = 0;
        for (int s = 0; s < nsys; ++s) it = std::max<int64_t>(it, hs[s].iters);
        p->pass_launches = 2 * it;  // passes the single-launch engines ran
    }
    int rc = QCP_OK;
    for (int s = 0; s < nsys; ++s) {
        const double kink = p->kink[p->hsys[s].prob];
        int ss = status_of(hs[s], kink, opts.kink_tol);
        if (residual && ss != QCP_BREAKDOWN && hs[s].resid_true > opts.rtol) ss = QCP_NOT_CONVERGED;
        rc = worse(rc, ss);
        if (info) {
            info[s].status = ss;
            info[s].iters = hs[s].iters;
            info[s].rel_residual = residual ? hs[s].resid_true : -1.0;
            info[s].rel_residual_est = hs[s].bnorm > 0 ? hs[s].phibar / hs[s].bnorm : 0.0;
            info[s].kink_margin = kink;
        }
    }
    return rc;
}

static bool ptr_ok(const void* p, int64_t count) { return count == 0 || p != nullptr; }

template <typename T>
static RhsArgs<T> jvp_in(const void* dP, const void* dA, const void* dq, const void* db) {
    RhsArgs<T> r{(const T*)dP, (const T*)dA, (const T*)dq, (const T*)db, nullptr, nullptr, nullptr, 0, 0};
    return r;
}
template <typename T>
static RhsArgs<T> vjp_in(const void* wx, const void* wy, const void* ws) {
    RhsArgs<T> r{nullptr, nullptr, nullptr, nullptr, (const T*)wx, (const T*)wy, (const T*)ws, 0, 0};
    return r;
}
template <typename T>
static OutArgs<T> jvp_out(void* dx, void* dy, void* ds) {
    OutArgs<T> o{(T*)dx, (T*)dy, (T*)ds, nullptr};
    return o;
}
template <typename T>
static OutArgs<T> vjp_out(void* dP, void* dA, void* dq, void* db) {
    OutArgs<T> o{(T*)dP, (T*)dA, (T*)dq, (T*)db};
    return o;
}

// JVPs of kj directions and VJPs of kv directions of a single-problem plan
// in one call: systems [0, kj) solve the JVPs, [kj, kj + kv) the VJPs.
static int pair_entry(qcp_plan* plan, const qcp_options* opts, int kj, const void* dP, const void* dA,
                      const void* dq, const void* db, void* dx, void* dy, void* ds, int kv, const void* wx,
                      const void* wy, const void* ws, void* gP, void* gA, void* gq, void* gb, qcp_info* info) {
    if (!plan || plan->batched) {
        set_error("qcp_derivative_jvp_vjp_multi takes a single-problem plan");
        return QCP_ERR_ARG;
    }
    if (kj < 1 || kv < 1 || kj + kv > plan->max_rhs) {
        set_error("kj = %d JVP and kv = %d VJP directions: each >= 1, together <= %d", kj, kv, plan->max_rhs);
        return QCP_ERR_ARG;
    }
    const Prob& pr = plan->hprob[0];
    const int64_t a = kj, b = kv;
    if (!ptr_ok(dP, pr.pnz * a) || !ptr_ok(dA, pr.anz * a) || !ptr_ok(dq, pr.n * a) || !ptr_ok(db, pr.m * a) ||
        !ptr_ok(dx, pr.n * a) || !ptr_ok(dy, pr.m * a) || !ptr_ok(ds, pr.m * a) || !ptr_ok(wx, pr.n * b) ||
        !ptr_ok(wy, pr.m * b) || !ptr_ok(ws, pr.m * b) || !ptr_ok(gP, pr.pnz * b) || !ptr_ok(gA, pr.anz * b) ||
        !ptr_ok(gq, pr.n * b) || !ptr_ok(gb, pr.m * b)) {
        set_error("null array argument");
        return QCP_ERR_ARG;
    }
    auto run = [&](auto tag) {
        using T = decltype(tag);
        Seg<T> g[2] = {{0, 0, kj, jvp_in<T>(dP, dA, dq, db), jvp_out<T>(dx, dy, ds)},
                       {1, kj, kv, vjp_in<T>(wx, wy, ws), vjp_out<T>(gP, gA, gq, gb)}};
        // the VJP range indexes its arrays from its first system
        g[1].ra.bx = g[1].out.bx = a * pr.n;
        g[1].ra.by = g[1].out.by = a * pr.m;
        g[1].ra.bp = g[1].out.bp = a * pr.pnz;
        g[1].ra.ba = g[1].out.ba = a * pr.anz;
        g[1].out.s0 = kj;
        return solve<T>(plan, g, 2, opts, info);
    };
    return plan->dtype == QCP_F64 ? run(double{}) : run(float{});
}

static int jvp_entry(qcp_plan* plan, const qcp_options* opts, int k, const void* dP, const void* dA,
                     const void* dq, const void* db, void* dx, void* dy, void* ds, qcp_info* info) {
    if (!plan) {
        set_error("null plan");
        return QCP_ERR_ARG;
    }
    const int nsys = plan->batched ? plan->nprob : k;
    if (!plan->batched && (k < 1 || k > plan->max_rhs)) {
        set_error("k = %d directions, plan built for 1..%d", k, plan->max_rhs);
        return QCP_ERR_ARG;
    }
    const int64_t kk = plan->batched ? 1 : k;
    if (!ptr_ok(dP, plan->pnz_tot * kk) || !ptr_ok(dA, plan->anz_tot * kk) || !ptr_ok(dq, plan->n_tot * kk) ||
        !ptr_ok(db, plan->m_tot * kk) || !ptr_ok(dx, plan->n_tot * kk) || !ptr_ok(dy, plan->m_tot * kk) ||
        !ptr_ok(ds, plan->m_tot * kk)) {
        set_error("null array argument");
        return QCP_ERR_ARG;
    }
    if (plan->dtype == QCP_F64) {
        using T = double;
        const Seg<T> g{0, 0, nsys, jvp_in<T>(dP, dA, dq, db), jvp_out<T>(dx, dy, ds)};
        return solve<T>(plan, &g, 1, opts, info);
    }
    using T = float;
    const Seg<T> g{0, 0, nsys, jvp_in<T>(dP, dA, dq, db), jvp_out<T>(dx, dy, ds)};
    return solve<T>(plan, &g, 1, opts, info);
}

static int vjp_entry(qcp_plan* plan, const qcp_options* opts, int k, const void* wx, const void* wy,
                     const void* ws, void* dP, void* dA, void* dq, void* db, qcp_info* info) {
    if (!plan) {
        set_error("null plan");
        return QCP_ERR_ARG;
    }
    const int nsys = plan->batched ? plan->nprob : k;
    if (!plan->batched && (k < 1 || k > plan->max_rhs)) {
        set_error("k = %d directions, plan built for 1..%d", k, plan->max_rhs);
        return QCP_ERR_ARG;
    }
    const int64_t kk = plan->batched ? 1 : k;
    if (!ptr_ok(wx, plan->n_tot * kk) || !ptr_ok(wy, plan->m_tot * kk) || !ptr_ok(ws, plan->m_tot * kk) ||
        !ptr_ok(dP, plan->pnz_tot * kk) || !ptr_ok(dA, plan->anz_tot * kk) || !ptr_ok(dq, plan->n_tot * kk) ||
        !ptr_ok(db, plan->m_tot * kk)) {
        set_error("null array argument");
        return QCP_ERR_ARG;
    }
    if (plan->dtype == QCP_F64) {
        using T = double;
        const Seg<T> g{1, 0, nsys, vjp_in<T>(wx, wy, ws), vjp_out<T>(dP, dA, dq, db)};
        return solve<T>(plan, &g, 1, opts, info);
    }
    using T = float;
    const Seg<T> g{1, 0, nsys, vjp_in<T>(wx, wy, ws), vjp_out<T>(dP, dA, dq, db)};
    return solve<T>(plan, &g, 1, opts, info);
}

// ---------------------------------------------------------------------------
// Autotuner: every candidate engine / schedule runs the same synthetic solve
// (fixed-hash directions, rtol 0, a fixed number of iterations) twice; the
// second run's device time per pass is the candidate's score.

// Uniform values in [-1, 1) from a SplitMix64 hash of (seed, index)
// (Steele, Lea and Flood, 2014).
template <typename T>
__global__ void k_hash_fill(T* x, int64_t n, uint64_t seed) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

template <typename T>
static int autotune(qcp_plan* p, const qcp_options& base, int mode, int nsys, int iters,
                    std::vector<qcp_tune_entry>& out, qcp_tune_entry* best_out) {
    const int64_t k = p->batched ? 1 : nsys;
    if (p->batched) nsys = p->nprob;
    const int64_t sz[7] = {mode == 0 ? p->pnz_tot : p->n_tot, mode == 0 ? p->anz_tot : p->m_tot,
                           mode == 0 ? p->n_tot : p->m_tot, mode == 0 ? p->m_tot : 0,
                           mode == 0 ? p->n_tot : p->pnz_tot, mode == 0 ? p->m_tot : p->anz_tot,
                           mode == 0 ? p->m_tot : p->n_tot};
    const int64_t sz_o4 = mode == 0 ? 0 : p->m_tot;
    DevBuf buf[8];
    cudaStream_t st = p->stream;
    for (int i = 0; i < 7; ++i) {
        QCP_TRY(buf[i].alloc(sizeof(T) * (size_t)(sz[i] * k)));
        if (i < 4 && sz[i] * k > 0)
            k_hash_fill<T><<<(unsigned)((sz[i] * k + 255) / 256), 256, 0, st>>>(buf[i].as<T>(), sz[i] * k,
                                                                                0x5eed0000ull + i);
    }
    QCP_TRY(buf[7].alloc(sizeof(T) * (size_t)(sz_o4 * k)));
    QCP_CUDA(cudaGetLastError());
    Seg<T> g{mode, 0, nsys, {}, {}};
    if (mode == 0) {
        g.ra = jvp_in<T>(buf[0].p, buf[1].p, buf[2].p, buf[3].p);
        g.out = jvp_out<T>(buf[4].p, buf[5].p, buf[6].p);
    } else {
        g.ra = vjp_in<T>(buf[0].p, buf[1].p, buf[2].p);
        g.out = vjp_out<T>(buf[4].p, buf[5].p, buf[6].p, buf[7].p);
    }
    qcp_options o = base;
    o.rtol = 0.0;
    o.maxiter = iters;
    o.compute_residual = 0;
    o.warm_start = nullptr;
    const int tiles[5] = {1024, 2048, 4096, 8192, 16384};
    const int ctas[5] = {1, 2, 4, 8, 16};
    const int tile0 = p->tile_nnz, lrow0 = p->long_row, lchunk0 = p->long_chunk, cap0 = p->cluster_cap;
    p->tuned_engine = -1;
    auto measure = [&](int engine, qcp_tune_entry& e) -> int {
        o.engine = engine;
        for (int rep = 0; rep < 2; ++rep) {
            const int rc = solve<T>(p, &g, 1, &o, nullptr);
            if (rc != QCP_OK && rc != QCP_NOT_CONVERGED && rc != QCP_WARN_NEAR_KINK) return rc;
        }
        e.us_per_pass = 1e3 * p->pass_ms / (double)std::max<int64_t>(1, p->pass_launches);
        return QCP_OK;
    };
    int best = -1;
    for (int engine : {(int)QCP_ENGINE_PASSES, (int)QCP_ENGINE_PERSISTENT}) {
        for (int t : tiles) {
            p->tile_nnz = t;
            p->long_row = std::max(1, t / 8);
            p->long_chunk = 1 << 20;
            QCP_TRY(build_schedule(p));
            qcp_tune_entry e{engine, 0, t, 0, 0.0};
            QCP_TRY(measure(engine, e));
            out.push_back(e);
            if (best < 0 || e.us_per_pass < out[best].us_per_pass) best = (int)out.size() - 1;
        }
    }
    // the cluster engine runs on the default tile schedule (its right-hand
    // side and output kernels use tiles)
    p->tile_nnz = tile0;
    p->long_row = lrow0;
    p->long_chunk = lchunk0;
    QCP_TRY(build_schedule(p));
    if (o.precond != QCP_PRECOND_DIAG) {
        for (int c : ctas) {
            p->cluster_cap = c;
            bool fits = false;
            QCP_TRY(cluster_ready(p, nsys, &fits));
            if (fits) {
                qcp_tune_entry e{QCP_ENGINE_CLUSTER, c, 0, 0, 0.0};
                QCP_TRY(measure(QCP_ENGINE_CLUSTER, e));
                out.push_back(e);
                if (e.us_per_pass < out[best].us_per_pass) best = (int)out.size() - 1;
            }
            // keep the device copies of the fastest cluster layout only
            if (!(best >= 0 && out[best].engine == QCP_ENGINE_CLUSTER && out[best].cluster_ctas == c))
                p->clusters.erase(c);
        }
    }
    if (o.precond != QCP_PRECOND_DIAG && o.solver == 0) {
        bool sok = false;
        QCP_TRY(stream_ready(p, &sok));
        if (sok) {
            qcp_tune_entry e{QCP_ENGINE_STREAM, 0, 0, 0, 0.0};
            QCP_TRY(measure(QCP_ENGINE_STREAM, e));
            out.push_back(e);
            if (e.us_per_pass < out[best].us_per_pass) best = (int)out.size() - 1;
        }
    }
    const qcp_tune_entry w = out[best];
    if (w.engine == QCP_ENGINE_CLUSTER) {
        p->cluster_cap = w.cluster_ctas;
    } else if (w.engine == QCP_ENGINE_STREAM) {
        p->cluster_cap = cap0;  // the stream engine uses the default tile schedule for its other kernels
    } else {
        p->cluster_cap = cap0;
        p->tile_nnz = w.tile_nnz;
        p->long_row = std::max(1, w.tile_nnz / 8);
        p->long_chunk = 1 << 20;
        QCP_TRY(build_schedule(p));
    }
    p->tuned_engine = w.engine;
    if (best_out) *best_out = w;
    return QCP_OK;
}

static int make_plan(int np, const qcp_problem* probs, const qcp_solution* sols, qcp_dtype dtype, int max_rhs,
                     bool batched, void* stream, qcp_plan** out) {
    if (!out || !probs || !sols || np < 1 || max_rhs < 1) {
        set_error("bad arguments to plan creation");
        return QCP_ERR_ARG;
    }
    *out = nullptr;
    if (dtype != QCP_F64 && dtype != QCP_F32) {
        set_error("dtype must be QCP_F64 or QCP_F32");
        return QCP_ERR_ARG;
    }
    qcp_plan* p = new qcp_plan();
    p->dtype = dtype;
    p->esz = dtype == QCP_F64 ? 8 : 4;
    p->nprob = np;
    p->max_rhs = max_rhs;
    p->batched = batched;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    if (user == nullptr) {
        // stream capture needs a stream other than the legacy default one;
        // a blocking stream keeps ordering with work on the default stream
        if (cudaStreamCreate(&p->stream) != cudaSuccess) {
            set_error("cudaStreamCreate failed");
            delete p;
            return QCP_ERR_CUDA;
        }
        p->owns_stream = true;
    } else {
        p->stream = user;
    }
    if (cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess) {
        set_error("cudaEventCreate failed");
        qcp_plan_destroy(p);
        return QCP_ERR_CUDA;
    }
    if (cudaMallocHost(&p->h_active, 2 * sizeof(int)) != cudaSuccess) {
        set_error("cudaMallocHost failed");
        qcp_plan_destroy(p);
        return QCP_ERR_ALLOC;
    }
    const int rc = create_plan(p, probs, sols);
    if (rc != QCP_OK) {
        qcp_plan_destroy(p);
        return rc;
    }
    *out = p;
    return QCP_OK;
}

// ---------------------------------------------------------------------------
// JVP without device allocation.
//
// Some callers cannot call cudaMalloc when they need a derivative:
// allocator hooks and callbacks that may not re-enter the allocator,
// real-time loops that forbid device allocation, or hosts whose memory is
// handed out by a pool they do not own.  For them the per-call
// scratch of the JVP (Krylov vectors, LSQR scalars, reduction partials and
// counters) lives in one file-scope device array of fixed size instead of
// plan memory.  Every GPU that loads the library holds the array until the
// process exits.
constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[256];  // device address of the array, per device ordinal

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
static int noalloc_scratch(void** out) {
    int dev = 0;
    QCP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("device ordinal %d out of range", dev);
        return QCP_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        QCP_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return QCP_OK;
}

// Bytes of scratch a one-direction JVP on this plan needs, and the view
// that points the kernels at it.
template <typename T>
static size_t noalloc_layout(qcp_plan* p, unsigned char* base, PlanView<T>* v, bool scaled) {
    const Prob& pr = p->hprob[0];
    const size_t N = (size_t)pr.n + pr.m + 1;
    const size_t nt = (size_t)p->tiles_per_sys, ng = (size_t)p->groups_per_sys;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        unsigned char* q = base ? base + off : nullptr;
        off += bytes;
        return q;
    };
    unsigned char* tpart = take(nt * sizeof(Part));
    unsigned char* gpart = take(ng * sizeof(Part));
    unsigned char* gcnt = take(ng * sizeof(int32_t));
    unsigned char* scnt = take(sizeof(int32_t));
    unsigned char* state = take(sizeof(LsqrState));
    unsigned char* active = take(sizeof(int));
    unsigned char* split = take(std::max(1, p->nsplit) * sizeof(int32_t));
    unsigned char* rowp = take(std::max<size_t>(1, nt) * sizeof(double));
    unsigned char* vec[6];
    for (int i = 0; i < 6; ++i) vec[i] = take(N * sizeof(double));
    if (v) {
        *v = view<T>(p, scaled ? QCP_PRECOND_EQUILIBRATE : QCP_PRECOND_NONE);
        v->state = reinterpret_cast<LsqrState*>(state);
        v->R = Reduce{reinterpret_cast<Part*>(tpart), reinterpret_cast<Part*>(gpart),
                      reinterpret_cast<int32_t*>(gcnt), reinterpret_cast<int32_t*>(scnt), p->d_groups.as<Group>()};
        v->active = reinterpret_cast<int*>(active);
        v->split_cnt = reinterpret_cast<int32_t*>(split);
        v->row_part = reinterpret_cast<double*>(rowp);
        v->U = reinterpret_cast<double*>(vec[0]);
        v->V = reinterpret_cast<double*>(vec[1]);
        v->W = reinterpret_cast<double*>(vec[2]);
        v->X = reinterpret_cast<double*>(vec[3]);
        v->XI = reinterpret_cast<double*>(vec[4]);
        v->RHS = reinterpret_cast<double*>(vec[5]);
        v->HB = nullptr;  // LSQR only
    }
    return off;
}

template <typename T>
static int jvp_noalloc(qcp_plan* p, const qcp_options* opts_in, const void* dP, const void* dA, const void* dq,
                       const void* db, void* dx, void* dy, void* ds, qcp_info* info) {
    qcp_options opts;
    if (opts_in) opts = *opts_in;
    else qcp_default_options(&opts);
    if (!(opts.rtol >= 0.0) || opts.maxiter < 1 || opts.check_every < 1 || opts.solver != 0 ||
        (opts.precond != QCP_PRECOND_NONE && opts.precond != QCP_PRECOND_EQUILIBRATE) || opts.warm_start) {
        set_error("bad options: rtol >= 0, maxiter >= 1, check_every >= 1, solver 0, precond NONE or EQUILIBRATE "
                  "and no warm start required");
        return QCP_ERR_ARG;
    }
    const size_t need = noalloc_layout<T>(p, nullptr, nullptr, false);
    if (need > kNoAllocScratchBytes) {
        set_error("qcp_derivative_jvp_noalloc: this plan needs %zu bytes of scratch, the static array holds %zu",
                  need, kNoAllocScratchBytes);
        return QCP_ERR_ARG;
    }
    void* base = nullptr;
    QCP_TRY(noalloc_scratch(&base));
    const bool scaled = opts.precond == QCP_PRECOND_EQUILIBRATE;
    PlanView<T> v;
    noalloc_layout<T>(p, static_cast<unsigned char*>(base), &v, scaled);
    cudaStream_t st = p->stream;
    const int ntiles = p->tiles_per_sys;
    const size_t smem = tile_smem_bytes(p->rmax, p->kpsd);
    QCP_TRY(set_smem_attrs<T>(smem));
    // the array keeps the previous call's contents: counters, partial sums,
    // the LSQR scalars and the Krylov vectors all start at zero
    QCP_CUDA(cudaMemsetAsync(base, 0, need, st));
    RhsArgs<T> ra{(const T*)dP, (const T*)dA, (const T*)dq, (const T*)db, nullptr, nullptr, nullptr,
                  opts.rtol, opts.maxiter};
    const OutArgs<T> out{(T*)dx, (T*)dy, (T*)ds, nullptr};
    k_jvp_rhs<T><<<ntiles, kThreads, 0, st>>>(v, ra);
    launch_pass<PASS_GT, ROLE_V, T>(v, ntiles, smem, st);
    QCP_CUDA(cudaGetLastError());
    LsqrState hs;
    double prev_res = INFINITY;
    for (int round = 0;; ++round) {
        for (int64_t done = 0; done <= opts.maxiter; done += opts.check_every) {
            for (int c = 0; c < opts.check_every; ++c) launch_iter<T>(0, v, ntiles, smem, st);
            QCP_CUDA(cudaGetLastError());
            int active = 0;
            QCP_CUDA(cudaMemcpyAsync(&active, v.active, sizeof(int), cudaMemcpyDeviceToHost, st));
            QCP_CUDA(cudaStreamSynchronize(st));
            if (active <= 0) break;
        }
        k_jvp_out<T><<<ntiles, kThreads, smem, st>>>(v, out);
        if (opts.compute_residual) launch_pass<PASS_G, ROLE_RES, T>(v, ntiles, smem, st);
        QCP_CUDA(cudaGetLastError());
        QCP_CUDA(cudaMemcpyAsync(&hs, v.state, sizeof(LsqrState), cudaMemcpyDeviceToHost, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        if (!opts.compute_residual || round == 4) break;
        // same continuation rule as qcp_derivative_jvp
        const bool improving = hs.resid_true < 0.5 * prev_res;
        prev_res = hs.resid_true;
        if (hs.outcome != O_CONVERGED || !(hs.resid_true > opts.rtol) || !(hs.alpha > 0.0) ||
            !isfinite(hs.resid_true) || hs.iters >= hs.maxiter || hs.bnorm_true <= 0.0 || !improving)
            break;
        hs.rtol *= std::max(0.01, 0.5 * opts.rtol / hs.resid_true);
        hs.status = S_ACTIVE;
        hs.outcome = O_RUNNING;
        hs.xcoef = 0.0;
        const int one = 1;
        QCP_CUDA(cudaMemcpyAsync(v.state, &hs, sizeof(LsqrState), cudaMemcpyHostToDevice, st));
        QCP_CUDA(cudaMemcpyAsync(v.active, &one, sizeof(int), cudaMemcpyHostToDevice, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        launch_pass<PASS_GT, ROLE_V, T>(v, ntiles, smem, st);
    }
    int rc = status_of(hs, p->kink[0], opts.kink_tol);
    if (opts.compute_residual && rc != QCP_BREAKDOWN && hs.resid_true > opts.rtol) rc = QCP_NOT_CONVERGED;
    if (info) {
        info->status = rc;
        info->iters = hs.iters;
        info->rel_residual = opts.compute_residual ? hs.resid_true : -1.0;
        info->rel_residual_est = hs.bnorm > 0 ? hs.phibar / hs.bnorm : 0.0;
        info->kink_margin = p->kink[0];
    }
    return rc;
}

}  // namespace qcpd

using namespace qcpd;

extern "C" {

const char* qcp_last_error(void) { return qcpd::last_error(); }

void qcp_default_options(qcp_options* o) {
    if (!o) return;
    o->solver = 0;
    o->rtol = 1e-10;
    o->maxiter = 100000;
    o->check_every = 32;
    o->use_graph = 1;
    o->compute_residual = 1;
    o->precond = QCP_PRECOND_NONE;
    o->engine = QCP_ENGINE_AUTO;
    o->warm_start = nullptr;
    o->precond_d = nullptr;
    o->kink_tol = 0.0;
}

int32_t qcp_version(void) { return 100; }

int qcp_plan_create(const qcp_problem* prob, const qcp_solution* sol, qcp_dtype dtype, int32_t max_rhs,
                    void* stream, qcp_plan** out) {
    return make_plan(1, prob, sol, dtype, max_rhs, false, stream, out);
}

int qcp_batch_plan_create(int32_t nprob, const qcp_problem* probs, const qcp_solution* sols, qcp_dtype dtype,
                          void* stream, qcp_plan** out) {
    return make_plan(nprob, probs, sols, dtype, 1, true, stream, out);
}

int qcp_plan_destroy(qcp_plan* plan) {
    if (!plan) return QCP_OK;
    if (plan->stream) cudaStreamSynchronize(plan->stream);
    const bool own = plan->owns_stream;
    cudaStream_t s = plan->stream;
    delete plan;
    if (own && s) cudaStreamDestroy(s);
    return QCP_OK;
}

int qcp_plan_sizes(const qcp_plan* p, int64_t* nprob, int64_t* n_total, int64_t* m_total, int64_t* nnzP_total,
                   int64_t* nnzA_total) {
    if (!p) {
        set_error("null plan");
        return QCP_ERR_ARG;
    }
    if (nprob) *nprob = p->nprob;
    if (n_total) *n_total = p->n_tot;
    if (m_total) *m_total = p->m_tot;
    if (nnzP_total) *nnzP_total = p->pnz_tot;
    if (nnzA_total) *nnzA_total = p->anz_tot;
    return QCP_OK;
}

int qcp_derivative_jvp(qcp_plan* plan, const qcp_options* opts, const void* dP, const void* dA, const void* dq,
                       const void* db, void* dx, void* dy, void* ds, qcp_info* info) {
    return jvp_entry(plan, opts, 1, dP, dA, dq, db, dx, dy, ds, info);
}

int qcp_derivative_vjp(qcp_plan* plan, const qcp_options* opts, const void* wx, const void* wy, const void* ws,
                       void* dP, void* dA, void* dq, void* db, qcp_info* info) {
    return vjp_entry(plan, opts, 1, wx, wy, ws, dP, dA, dq, db, info);
}

int qcp_derivative_jvp_multi(qcp_plan* plan, const qcp_options* opts, int32_t k, const void* dP, const void* dA,
                             const void* dq, const void* db, void* dx, void* dy, void* ds, qcp_info* info) {
    if (plan && plan->batched) {
        set_error("the _multi entry points take single-problem plans");
        return QCP_ERR_ARG;
    }
    return jvp_entry(plan, opts, k, dP, dA, dq, db, dx, dy, ds, info);
}

int qcp_derivative_vjp_multi(qcp_plan* plan, const qcp_options* opts, int32_t k, const void* wx, const void* wy,
                             const void* ws, void* dP, void* dA, void* dq, void* db, qcp_info* info) {
    if (plan && plan->batched) {
        set_error("the _multi entry points take single-problem plans");
        return QCP_ERR_ARG;
    }
    return vjp_entry(plan, opts, k, wx, wy, ws, dP, dA, dq, db, info);
}

int qcp_derivative_jvp_vjp_multi(qcp_plan* plan, const qcp_options* opts, int32_t kj, const void* dP,
                                 const void* dA, const void* dq, const void* db, void* dx, void* dy, void* ds,
                                 int32_t kv, const void* wx, const void* wy, const void* ws, void* gP, void* gA,
                                 void* gq, void* gb, qcp_info* info) {
    return pair_entry(plan, opts, kj, dP, dA, dq, db, dx, dy, ds, kv, wx, wy, ws, gP, gA, gq, gb, info);
}

int qcp_plan_autotune(qcp_plan* plan, const qcp_options* opts, int32_t mode, int32_t nsys, int32_t iters,
                      qcp_tune_entry* entries, int32_t cap, int32_t* count, qcp_tune_entry* best) {
    if (!plan || (mode != 0 && mode != 1) || iters < 4 || cap < 0 || (cap > 0 && !entries) ||
        (!plan->batched && (nsys < 1 || nsys > plan->max_rhs))) {
        set_error("autotune: plan, mode 0 or 1, 1 <= nsys <= max_rhs, iters >= 4 and room for the entries required");
        return QCP_ERR_ARG;
    }
    qcp_options o;
    if (opts) o = *opts;
    else qcp_default_options(&o);
    if (o.precond == QCP_PRECOND_DIAG) {
        set_error("autotune: tune with QCP_PRECOND_NONE or _EQUILIBRATE");
        return QCP_ERR_ARG;
    }
    std::vector<qcp_tune_entry> all;
    const int rc = plan->dtype == QCP_F64 ? autotune<double>(plan, o, mode, nsys, iters, all, best)
                                          : autotune<float>(plan, o, mode, nsys, iters, all, best);
    if (count) *count = (int32_t)all.size();
    for (int i = 0; i < (int)all.size() && i < cap; ++i) entries[i] = all[i];
    return rc;
}

int qcp_plan_set_schedule(qcp_plan* plan, int32_t tile_nnz, int32_t long_row, int32_t long_chunk) {
    if (!plan || tile_nnz < 64 || long_row < 1 || long_chunk < 32) {
        set_error("bad schedule: tile_nnz >= 64, long_row >= 1 and long_chunk >= 32 required");
        return QCP_ERR_ARG;
    }
    plan->tuned_engine = -1;
    plan->tile_nnz = tile_nnz;
    plan->long_row = long_row;
    plan->long_chunk = long_chunk;
    return build_schedule(plan);
}

int qcp_plan_set_cluster(qcp_plan* plan, int32_t max_ctas) {
    if (!plan || max_ctas < 0 || max_ctas > kMaxCluster) {
        set_error("cluster size must be 0 (automatic) or 1 to 16");
        return QCP_ERR_ARG;
    }
    plan->cluster_cap = max_ctas;
    plan->tuned_engine = -1;
    return QCP_OK;
}

int qcp_plan_set_equilibration(qcp_plan* plan, int32_t sweeps) {
    if (!plan || sweeps < 1 || sweeps > 64) {
        set_error("qcp_plan_set_equilibration: null plan or sweeps outside 1 to 64");
        return QCP_ERR_ARG;
    }
    // w and c are baked into captured graphs, cluster layouts and the
    // autotuner's timings, so they may change only before any of those exist
    if (plan->last_mode >= 0 || !plan->graphs.empty() || !plan->clusters.empty() || plan->stream_lay ||
        plan->tuned_engine >= 0) {
        set_error("qcp_plan_set_equilibration: call it before the plan's first derivative or autotune call");
        return QCP_ERR_ARG;
    }
    if (sweeps == plan->equil_sweeps) return QCP_OK;
    const int rc = equilibrate_plan(plan, sweeps);
    if (rc == QCP_OK) plan->equil_sweeps = sweeps;
    return rc;
}

int qcp_plan_set_barrier_wait(qcp_plan* plan, int64_t polls, int64_t hold_ns) {
    if (!plan || polls < 0 || hold_ns < 0 || hold_ns > 1000000000LL) {
        set_error("qcp_plan_set_barrier_wait: null plan, negative bound or hold above 1 s");
        return QCP_ERR_ARG;
    }
    plan->barrier_polls = polls;
    plan->barrier_hold_ns = hold_ns;
    return QCP_OK;
}

int qcp_plan_set_stream_pairing(qcp_plan* plan, int32_t on) {
    if (!plan || (on != 0 && on != 1)) {
        set_error("qcp_plan_set_stream_pairing: null plan or a value other than 0 and 1");
        return QCP_ERR_ARG;
    }
    plan->stream_pairing = on;
    return QCP_OK;
}

int qcp_plan_last_shared_passes(const qcp_plan* plan, int64_t* shared) {
    if (!plan || !shared) {
        set_error("qcp_plan_last_shared_passes: null plan or output");
        return QCP_ERR_ARG;
    }
    *shared = plan->shared_passes;
    return QCP_OK;
}

int64_t qcp_plan_last_launches(const qcp_plan* plan) { return plan ? plan->last_launches : 0; }

int qcp_plan_last_engine(const qcp_plan* plan) { return plan ? plan->last_engine : -1; }

int qcp_plan_last_solution(qcp_plan* plan, double* out) {
    if (!plan || !out || plan->last_mode < 0) {
        set_error("qcp_plan_last_solution: null argument or no solve yet");
        return QCP_ERR_ARG;
    }
    int maxN = 1;
    for (int s = 0; s < plan->last_nsys; ++s) {
        const Prob& pr = plan->hprob[plan->hsys[s].prob];
        maxN = std::max(maxN, pr.n + pr.m + 1);
    }
    const dim3 grid((unsigned)std::min(1024, (maxN + 255) / 256), (unsigned)plan->last_nsys);
    if (plan->dtype == QCP_F64)
        k_export<double><<<grid, 256, 0, plan->stream>>>(view<double>(plan, plan->view_precond), plan->last_jvp_sys,
                                                         out);
    else
        k_export<float><<<grid, 256, 0, plan->stream>>>(view<float>(plan, plan->view_precond), plan->last_jvp_sys,
                                                        out);
    QCP_CUDA(cudaGetLastError());
    QCP_CUDA(cudaStreamSynchronize(plan->stream));
    return QCP_OK;
}

int qcp_derivative_jvp_noalloc(qcp_plan* plan, const qcp_options* opts, const void* dP, const void* dA,
                               const void* dq, const void* db, void* dx, void* dy, void* ds, qcp_info* info) {
    if (!plan || plan->batched) {
        set_error("qcp_derivative_jvp_noalloc takes a single-problem plan");
        return QCP_ERR_ARG;
    }
    const qcpd::Prob& pr = plan->hprob[0];
    if ((pr.pnz && !dP) || (pr.anz && !dA) || !dq || (pr.m && !db) || !dx || (pr.m && (!dy || !ds))) {
        set_error("null array argument");
        return QCP_ERR_ARG;
    }
    if (plan->dtype == QCP_F64) return jvp_noalloc<double>(plan, opts, dP, dA, dq, db, dx, dy, ds, info);
    return jvp_noalloc<float>(plan, opts, dP, dA, dq, db, dx, dy, ds, info);
}

int qcp_plan_last_timing(const qcp_plan* plan, double* pass_ms, int64_t* passes) {
    if (!plan) {
        set_error("null plan");
        return QCP_ERR_ARG;
    }
    if (pass_ms) *pass_ms = plan->pass_ms;
    if (passes) *passes = plan->pass_launches;
    return QCP_OK;
}

}  // extern "C"
