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
    v.rmax = p->rmax;
    v.long_chunk = p->long_chunk;
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
    GraphKey key{mode, nsys, chunk, p->view_precond};
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
            QCP_CUDA(cudaMemcpyAsync(p->h_active, p->d_active.p, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
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
        for (int s = 0; s < nsys; ++s) {
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

// mode 0: JVP, 1: VJP.  nsys systems (the first nsys of the plan).
template <typename T>
static int solve(qcp_plan* p, int mode, int nsys, const qcp_options* opts_in, const RhsArgs<T>& rin,
                 const OutArgs<T>& out, qcp_info* info) {
    qcp_options opts;
    if (opts_in) opts = *opts_in;
    else qcp_default_options(&opts);
    if (!(opts.rtol >= 0.0) || opts.maxiter < 1 || opts.check_every < 0) {
        set_error("bad options: rtol >= 0, maxiter >= 1, check_every >= 0 required");
        return QCP_ERR_ARG;
    }
    if (opts.solver != 0) {
        set_error("only solver 0 (LSQR) is built");
        return QCP_ERR_ARG;
    }
    if (opts.precond != QCP_PRECOND_NONE && opts.precond != QCP_PRECOND_EQUILIBRATE &&
        opts.precond != QCP_PRECOND_DIAG) {
        set_error("precond must be QCP_PRECOND_NONE, _EQUILIBRATE or _DIAG");
        return QCP_ERR_ARG;
    }
    if (opts.precond == QCP_PRECOND_DIAG && !opts.precond_d) {
        set_error("QCP_PRECOND_DIAG needs opts->precond_d");
        return QCP_ERR_ARG;
    }
    if (opts.precond == QCP_PRECOND_DIAG &&
        (opts.engine == QCP_ENGINE_CLUSTER || opts.engine == QCP_ENGINE_CLUSTER_FP64)) {
        set_error("QCP_PRECOND_DIAG runs on the pass or persistent engine");
        return QCP_ERR_ARG;
    }
    if (opts.engine < QCP_ENGINE_PASSES || opts.engine > QCP_ENGINE_CLUSTER_FP64) {
        set_error("engine must be one of QCP_ENGINE_PASSES, _PERSISTENT, _CLUSTER, _AUTO, _CLUSTER_FP64");
        return QCP_ERR_ARG;
    }
    int engine = opts.engine;
    if (engine == QCP_ENGINE_AUTO && opts.precond == QCP_PRECOND_DIAG) engine = QCP_ENGINE_PASSES;
    if (engine == QCP_ENGINE_CLUSTER || engine == QCP_ENGINE_AUTO || engine == QCP_ENGINE_CLUSTER_FP64) {
        bool fits = false;
        QCP_TRY(cluster_ready(p, nsys, &fits));
        if (fits) {
            engine = QCP_ENGINE_CLUSTER;
        } else if (engine != QCP_ENGINE_AUTO) {
            set_error("cluster engine: a problem's vectors do not fit in the shared memory of 16 CTAs");
            return QCP_ERR_ARG;
        } else {
            engine = QCP_ENGINE_PASSES;
        }
    }
    cudaStream_t st = p->stream;
    if (opts.precond == QCP_PRECOND_DIAG) QCP_TRY(prepare_diag<T>(p, opts.precond_d));
    p->view_precond = opts.precond;
    const PlanView<T> v = view<T>(p, opts.precond);
    const int ntiles = p->batched ? p->ntiles : nsys * p->tiles_per_sys;
    const size_t smem = tile_smem_bytes(p->rmax);
    QCP_TRY(set_smem_attrs<T>(smem));
    p->last_launches = 0;
    p->last_engine = engine;
    p->last_mode = mode;
    p->last_nsys = nsys;
    p->pass_ms = 0.0;
    p->pass_launches = 0;
    QCP_CUDA(cudaMemsetAsync(p->d_active.p, 0, sizeof(int), st));
    RhsArgs<T> ra = rin;
    ra.rtol = opts.rtol;
    ra.maxiter = opts.maxiter;
    if (mode == 0) k_jvp_rhs<T><<<ntiles, kThreads, 0, st>>>(v, ra);
    else k_vjp_rhs<T><<<ntiles, kThreads, smem, st>>>(v, ra);
    if (opts.warm_start) {
        // x0 from the caller's iterate; the right-hand side becomes b - Op x0
        int maxN = 1;
        for (int s = 0; s < nsys; ++s) {
            const Prob& pr = p->hprob[p->hsys[s].prob];
            maxN = std::max(maxN, pr.n + pr.m + 1);
        }
        k_warm_init<T><<<dim3((unsigned)std::min(1024, (maxN + 255) / 256), (unsigned)nsys), 256, 0, st>>>(
            v, opts.warm_start, mode);
        if (mode == 0) {
            k_dpi<T><<<ntiles, kThreads, smem, st>>>(v);
            launch_pass<PASS_G, ROLE_WARM, T>(v, ntiles, smem, st);
        } else {
            launch_pass<PASS_GT, ROLE_WARM, T>(v, ntiles, smem, st);
        }
        p->last_launches += mode == 0 ? 3 : 2;
    }
    launch_v_pass<T>(mode, v, ntiles, smem, st);
    QCP_CUDA(cudaGetLastError());
    p->last_launches += 2;
    auto run_iterations = [&]() -> int {
        if (engine == QCP_ENGINE_PERSISTENT) return iterate_persistent<T>(p, mode, v, ntiles, smem, opts);
        if (engine == QCP_ENGINE_CLUSTER) return iterate_cluster<T>(p, mode, nsys, v, opts);
        return iterate<T>(p, mode, nsys, v, ntiles, smem, opts);
    };
    QCP_TRY(run_iterations());
    std::vector<LsqrState> hs(nsys);
    std::vector<double> prev_res(nsys, INFINITY);
    const bool residual = opts.compute_residual != 0;
    for (int round = 0;; ++round) {
        launch_output<T>(p, mode, nsys, v, ntiles, smem, out, residual);
        QCP_CUDA(cudaGetLastError());
        QCP_CUDA(cudaMemcpyAsync(hs.data(), p->d_state.p, nsys * sizeof(LsqrState), cudaMemcpyDeviceToHost, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        if (!residual || round == 4) break;
        // The Krylov estimate measures the scaled residual; where the true
        // one misses the target, continue the same recurrence with a tighter
        // internal tolerance.
        int resumed = 0;
        for (int s = 0; s < nsys; ++s) {
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
            ++resumed;
        }
        if (!resumed) break;
        QCP_CUDA(cudaMemcpyAsync(p->d_state.p, hs.data(), nsys * sizeof(LsqrState), cudaMemcpyHostToDevice, st));
        QCP_CUDA(cudaMemcpyAsync(p->d_active.p, &resumed, sizeof(int), cudaMemcpyHostToDevice, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        launch_v_pass<T>(mode, v, ntiles, smem, st);
        p->last_launches += 1;
        QCP_TRY(run_iterations());
    }
    if (engine != QCP_ENGINE_PASSES) {
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
        RhsArgs<T> r{(const T*)dP, (const T*)dA, (const T*)dq, (const T*)db, nullptr, nullptr, nullptr, 0, 0};
        OutArgs<T> o{(T*)dx, (T*)dy, (T*)ds, nullptr};
        return solve<T>(plan, 0, nsys, opts, r, o, info);
    }
    using T = float;
    RhsArgs<T> r{(const T*)dP, (const T*)dA, (const T*)dq, (const T*)db, nullptr, nullptr, nullptr, 0, 0};
    OutArgs<T> o{(T*)dx, (T*)dy, (T*)ds, nullptr};
    return solve<T>(plan, 0, nsys, opts, r, o, info);
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
        RhsArgs<T> r{nullptr, nullptr, nullptr, nullptr, (const T*)wx, (const T*)wy, (const T*)ws, 0, 0};
        OutArgs<T> o{(T*)dP, (T*)dA, (T*)dq, (T*)db};
        return solve<T>(plan, 1, nsys, opts, r, o, info);
    }
    using T = float;
    RhsArgs<T> r{nullptr, nullptr, nullptr, nullptr, (const T*)wx, (const T*)wy, (const T*)ws, 0, 0};
    OutArgs<T> o{(T*)dP, (T*)dA, (T*)dq, (T*)db};
    return solve<T>(plan, 1, nsys, opts, r, o, info);
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
    if (cudaMallocHost(&p->h_active, sizeof(int)) != cudaSuccess) {
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
// Some callers cannot call cudaMalloc when they need a derivative: code
// that runs while a stream is being captured into a CUDA graph, allocator
// hooks and real-time loops that forbid device allocation, or hosts whose
// memory is handed out by a pool they do not own.  For them the per-call
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
    const size_t smem = tile_smem_bytes(p->rmax);
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

int qcp_plan_set_schedule(qcp_plan* plan, int32_t tile_nnz, int32_t long_row, int32_t long_chunk) {
    if (!plan || tile_nnz < 64 || long_row < 1 || long_chunk < 32) {
        set_error("bad schedule: tile_nnz >= 64, long_row >= 1 and long_chunk >= 32 required");
        return QCP_ERR_ARG;
    }
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
        k_export<double><<<grid, 256, 0, plan->stream>>>(view<double>(plan, plan->view_precond), plan->last_mode, out);
    else
        k_export<float><<<grid, 256, 0, plan->stream>>>(view<float>(plan, plan->view_precond), plan->last_mode, out);
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
