// Host-side plan object and helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "qcpd_common.cuh"

namespace qcpd {

void set_error(const char* fmt, ...);

#define QCP_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            ::qcpd::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                              __LINE__);                                                     \
            return e_ == cudaErrorMemoryAllocation ? QCP_ERR_ALLOC : QCP_ERR_CUDA;           \
        }                                                                                    \
    } while (0)

#define QCP_TRY(expr)              \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != QCP_OK) return rc_; \
    } while (0)

// A device allocation freed on destruction.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t nbytes) {
        release();
        if (nbytes == 0) nbytes = 16;
        cudaError_t e = cudaMalloc(&p, nbytes);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMalloc(%zu) failed: %s", nbytes, cudaGetErrorString(e));
            return QCP_ERR_ALLOC;
        }
        bytes = nbytes;
        return QCP_OK;
    }
    // exchange the allocations of two buffers (no device work)
    void swap(DevBuf& o) {
        std::swap(p, o.p);
        std::swap(bytes, o.bytes);
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

// Sweeps of the row/column equilibration a plan starts with: on the
// configurations measured, 16 sweeps take 7 to 100 times fewer LSQR
// iterations than one, and more sweeps gain little.
constexpr int kDefaultEquilSweeps = 16;

constexpr int kMaxSegments = 2;  // system ranges of one call (JVP systems, VJP systems)

struct GraphKey {
    int engine;  // qcp_engine whose launches the graph holds
    int mode;    // 0 JVP, 1 VJP, 2 a JVP range and a VJP range in step (stream engine)
    int tile0;   // first tile of the system range
    int nsys;
    int chunk;
    int scaled;  // qcp_precond of the view (different kernels and value arrays)
    int solver;  // 0 LSQR, 1 LSMR (a kernel parameter of the captured launches)
    int pair = 0;  // paired stream launches: 1 + the first system of the VJP range (mode 2); else 0
    bool operator<(const GraphKey& o) const {
        if (pair != o.pair) return pair < o.pair;
        if (engine != o.engine) return engine < o.engine;
        if (mode != o.mode) return mode < o.mode;
        if (tile0 != o.tile0) return tile0 < o.tile0;
        if (nsys != o.nsys) return nsys < o.nsys;
        if (scaled != o.scaled) return scaled < o.scaled;
        if (solver != o.solver) return solver < o.solver;
        return chunk < o.chunk;
    }
};

// Thread-block-cluster layouts of every problem of a plan for one requested
// cluster size (QCP_ENGINE_CLUSTER).
struct ClusterLayout {
    bool fits = false;              // every problem has a layout within the shared-memory limit
    std::vector<ClusterProb> hp;    // per problem
    DevBuf d_cprob;                 // device copy of hp
    // SELL-32 copy of M by CTA: slices, row permutation, gather-buffer
    // columns and the plain / column-scaled / row-scaled values per slot
    DevBuf d_slices, d_perm, d_scol, d_sval, d_svalG, d_svalT;
    DevBuf d_sp, d_sr;          // per slice: its problem and the first row of its CTA
    int64_t nslices = 0, slots = 0;
    // double-float copies for the df64 kernel (df_ok: every magnitude in range)
    bool df_ok = false;
    DevBuf d_dsval, d_dsvalG, d_dsvalT, d_dcA, d_dcB, d_drw, d_dcd, d_dzy, d_dsoc;
    // QCP_PRECOND_DIAG (refilled on every such call, the caller's C changes):
    // M diag(C) per slot and its df64 copy, df64 copies of W = 1 and of C
    bool diag_df_ok = false;
    DevBuf d_svalDG, d_dsvalDG, d_drwD, d_dcdD, d_diag_bad;
};

// The stream engine's copy of a plan (QCP_ENGINE_STREAM, built on first
// use): warp units over every problem's rows, the slots of M they read as
// df64 values, df64 per-row data and per-block constants, and the engine's
// per-system workspace.
struct StreamLayout {
    bool ok = false;                 // usable: cones zero / R+ / SOC (blocks <= 256 rows), magnitudes in df64 range
    std::string why;                 // the reason when not
    int nunits = 0;                  // over all problems
    int max_units = 0;               // most units of one problem
    int nsplit = 0, nslot = 0;       // split rows and their chunk slots (plan-wide)
    int gmax = 0;                    // CTAs per system the workspace holds (all resident k_stream CTAs)
    int gmax2 = 0;                   // resident k_stream2 CTAs (<= gmax)
    std::vector<int32_t> huoff, hsoff;
    DevBuf d_units, d_uoff, d_soff, d_rows, d_lblk, d_scol, d_val, d_valG, d_valT;
    DevBuf d_cA, d_cB, d_rw, d_cd, d_zy, d_soc;
    DevBuf d_scal, d_ssys, d_cpart, d_ccnt, d_lchunk, d_lcnt, d_lrow;
    DevBuf d_slist, d_scount;        // the systems (or pairs) still iterating, their number
    DevBuf d_pshared;                // paired launches: system passes that shared their read of M
};

}  // namespace qcpd

struct qcp_plan {
    qcp_dtype dtype = QCP_F64;
    size_t esz = 8;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    int nprob = 0;
    int max_rhs = 1;
    bool batched = false;

    // host copies of the per-problem layout
    std::vector<qcpd::Prob> hprob;
    std::vector<std::vector<int32_t>> cone_type, cone_dim;
    std::vector<double> kink;  // per problem
    int64_t n_tot = 0, m_tot = 0, pnz_tot = 0, anz_tot = 0, N_tot = 0, nsoc_tot = 0, mnnz = 0;

    // problem data (device)
    qcpd::DevBuf d_prob, d_mrowptr, d_mcol, d_mvmap, d_mval;
    qcpd::DevBuf d_coefA, d_coefB, d_pz, d_zy, d_flag, d_blocks;
    qcpd::DevBuf d_psd;   // PSD blocks: eigenvectors V and D Pi weights B, 2 k^2 doubles each; exp blocks: D Pi
    int kpsd = 0;         // largest PSD block order (0: no PSD block)
    int ndense = 0;       // exponential-cone blocks (D Pi stored as a dense 3 x 3 in d_psd)
    // the exponential, power and PSD blocks' D Pi as dense df64 matrices for the
    // double-float engines (stream, cluster): offsets per coupled block (-1 for
    // SOC blocks) and the row-major matrices; dpi_state 0 not built, 1 built,
    // -1 unusable (dpi_why says why)
    qcpd::DevBuf d_dpi_off, d_dpi;
    int dpi_state = 0;
    std::string dpi_why;
    qcpd::DevBuf d_rw, d_cd, d_mvalG, d_mvalT;   // equilibration: row/column scalings, scaled values
    qcpd::DevBuf d_cdD, d_onesD, d_mvalD;        // QCP_PRECOND_DIAG: the caller's C, unit W, M diag(C)
    qcpd::DevBuf d_cdJ;                          // QCP_PRECOND_JACOBI: 1 / column norms of F (made on first use)
    qcpd::DevBuf d_pip, d_pix, d_aip, d_aix;

    // schedule
    int tile_nnz = 4096;
    int long_row = 512;
    int long_chunk = 1 << 20;
    int rmax = 1;
    std::vector<std::vector<qcpd::Tile>> ptiles;  // per problem, sys = problem
    std::vector<int64_t> h_mrowptr;               // host copy (schedule building)
    qcpd::DevBuf d_ptiles, d_pgroups, d_ppart, d_pgpart, d_pgcnt, d_pscnt, d_psys;

    // systems
    int nsys_cap = 0;
    int tiles_per_sys = 0;   // single-problem plans: tiles of one system
    int groups_per_sys = 0;
    std::vector<qcpd::Sys> hsys;
    int ntiles = 0, ngroups = 0;
    int nsplit = 0;          // rows cut into several LONG chunks (over all systems)
    qcpd::DevBuf d_sys, d_tiles, d_groups, d_state, d_tpart, d_gpart, d_gcnt, d_scnt, d_active;
    qcpd::DevBuf d_split_cnt, d_row_part;
    qcpd::DevBuf d_pctl;     // persistent mode: barrier count, generation, stop flag, error flag
    int64_t barrier_polls = 0;    // persistent mode: polls per barrier wait (0: the default bound)
    int64_t barrier_hold_ns = 0;  // persistent mode: CTA 0's wait before its first barrier (a test hook)
    qcpd::DevBuf d_U, d_V, d_W, d_X, d_XI, d_RHS, d_HB;  // Krylov vectors (HB: LSMR's hbar)
    int* h_active = nullptr;  // pinned, two counters (a paired stream iteration reads both of its ranges')

    // cluster engine
    int cluster_cap = 0;  // CTAs per system asked for (0: per call from the number of systems)
    int tuned_engine = -1; // the autotuner's choice for QCP_ENGINE_AUTO (-1: none)
    int equil_sweeps = qcpd::kDefaultEquilSweeps;  // sweeps of the row/column equilibration behind d_rw and d_cd
    std::map<int, std::unique_ptr<qcpd::ClusterLayout>> clusters;  // by CTAs asked for
    std::unique_ptr<qcpd::StreamLayout> stream_lay;  // QCP_ENGINE_STREAM (built on first use)
    qcpd::DevBuf d_csys;  // system lists of the cluster launches
    qcpd::DevBuf d_bcast; // broadcast buffers of the double-float cluster kernel
    std::vector<int32_t> h_csys;

    std::map<qcpd::GraphKey, cudaGraphExec_t> graphs;
    int64_t last_launches = 0;
    int last_engine = 0;   // qcp_engine the last call ran (CLUSTER_FP64 when the cluster kernel stayed in FP64)
    int view_precond = 0;  // qcp_precond of the current call's view (graph cache key)
    int last_mode = -1;    // 0 JVP, 1 VJP, 2 both (JVP systems first): the last call
    int last_nsys = 0;     // systems of the last call
    int last_jvp_sys = 0;  // of which the first last_jvp_sys solved a JVP
    // device time of the iteration chunks of the last call (CUDA events on
    // the plan's stream) and the number of pass launches they contain
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // a second stream for the cluster launches of a call's second system
    // range (JVP and VJP systems side by side), created on first use
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double pass_ms = 0.0;
    int64_t pass_launches = 0;
    int stream_pairing = 1;  // stream engine: iterate a JVP range and a VJP range in step
    int64_t shared_passes = 0;  // of the last call: system passes that shared a launch's read of M

    ~qcp_plan();
};

namespace qcpd {
// Build (or rebuild) the tile schedule, systems and workspace of a plan.
int build_schedule(qcp_plan* p);
// Free captured graphs.
void drop_graphs(qcp_plan* p);
// The Jacobi preconditioner's column scaling (N_tot doubles, device).
int jacobi_cols(qcp_plan* p, double* out);
// Recompute the equilibration's w and c with the given number of sweeps,
// and the scaled copies of M's values.
int equilibrate_plan(qcp_plan* p, int sweeps);
}  // namespace qcpd
