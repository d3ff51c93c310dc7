/*
 * qcpd.h -- C ABI of the GB300 library for derivatives of a quadratic cone
 * program's solution map (arXiv 2508.17522).
 *
 * The conic pair (Sec. 2.1, eq. conic-pair):
 *     minimize (1/2) x^T P x + q^T x  s.t.  A x + s = b,  s in K,
 * with dual variable y in K*.  Given a solution (x, y, s), the library
 * evaluates
 *   * the forward product (JVP, Sec. 3.1):
 *       (dx, dy, ds) = D S(theta)[dP, dA, dq, db]
 *   * the adjoint product (VJP, Sec. 3.2):
 *       (dP, dA, dq, db) = D S(theta)^T [dx, dy, ds], kept on the stored
 *       patterns of P and A (Sec. 3.2, last paragraph),
 * through the implicit function theorem on the homogeneous embedding
 * (Sec. 2.4): z = (x, y - s, 1), F = D_z N(z), dz solves F dz = -D_theta N,
 * and the outputs go through D phi(z).  The linear systems are solved
 * matrix-free by an LSQR Krylov iteration (Sec. 3.1 prescribes LSMR; both
 * need only products with F and F^T, which is what the kernels provide).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Memory     Every array argument is a DEVICE pointer owned by the caller
 *             (for example a torch tensor's data_ptr), except the cone
 *             description (qcp_cone), which lives in HOST memory, and the
 *             qcp_info outputs, which are host structs.  The library copies
 *             what it needs at plan creation; inputs may be freed after
 *             qcp_plan_create returns.  A plan owns its device workspace,
 *             allocated once at creation and freed by qcp_plan_destroy.
 *  Types      Floating-point arrays are all float64 (QCP_F64) or all
 *             float32 (QCP_F32, "FP32 storage": problem data, the combined
 *             matrix, perturbations and outputs in binary32; Krylov vectors
 *             and every dot product and norm in float64).
 *             Index arrays: row pointers int64, column indices int32,
 *             sorted and unique within each row.
 *  P          Symmetric; only its upper triangle (diagonal included) is
 *             stored, in CSR.  Explicit zeros are part of the pattern.
 *  dP         JVP input: values on P's stored upper pattern, read as the
 *             upper triangle of a symmetric perturbation.  VJP output: the
 *             entries of the symmetric matrix D_theta N^T[r]_P at the stored
 *             upper positions (so the gradient with respect to a stored
 *             off-diagonal value is twice the returned entry).
 *  A, AT      A is m x n CSR; AT is its transpose in CSR (n x m).  AT_perm
 *             (int64, nnz(A)) maps AT's k-th stored value to its position in
 *             A's value array; it may be NULL, in which case the plan derives
 *             it from A.
 *  Cones      K is a product of blocks listed in row order: QCP_CONE_ZERO
 *             (the cone {0}), QCP_CONE_NONNEG (R+^d), QCP_CONE_SOC
 *             (second-order cone, stored (t, u) with t first, Appendix A)
 *             and QCP_CONE_PSD (positive semidefinite k x k matrices,
 *             Appendix A: dim = k (k + 1) / 2 entries, the upper triangle
 *             column by column with the off-diagonal entries times sqrt 2,
 *             (X11, sqrt2 X12, X22, sqrt2 X13, sqrt2 X23, X33, ...), so the
 *             layout preserves inner products; k <= 64) and QCP_CONE_EXP
 *             (the exponential cone cl{(x, y, z): y > 0, y e^(x/y) <= z},
 *             dim 3) and QCP_CONE_POW (the power cone {(x, y, z): x, y >= 0,
 *             x^a y^(1-a) >= |z|}, dim 3, exponent a from K.param), both of
 *             Appendix A (the method projects onto their duals).  Plans with
 *             PSD, exponential or power blocks run on the pass and
 *             persistent engines, and on the stream and (double-float)
 *             cluster engines with each such block's D Pi stored dense
 *             (PSD orders up to 22).
 *  Streams    `stream` is a cudaStream_t (NULL = the legacy default stream).
 *             All work of a plan is enqueued on the stream given at creation.
 *             JVP/VJP calls return when the outputs are written: they
 *             synchronize the stream every opts->check_every iterations to
 *             test convergence (check_every = 0: run exactly opts->maxiter
 *             iterations without synchronizing; finished systems skip their
 *             work).
 *  Errors     Every entry point returns a qcp_status.  On an error the
 *             outputs are unspecified and qcp_last_error() describes it.
 *             QCP_NOT_CONVERGED still writes the outputs (the last iterate).
 *  Threads    A plan must not be used by two host threads at once.
 */
#ifndef QCPD_H
#define QCPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QCP_OK = 0,
    QCP_ERR_ARG = 1,          /* null pointer, bad size, unsorted CSR, P not upper, AT inconsistent, ... */
    QCP_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    QCP_ERR_ALLOC = 3,        /* device allocation failed */
    QCP_NOT_CONVERGED = 4,    /* rtol not reached (maxiter hit, or the true residual stalled above
                                 rtol at the attainable accuracy); outputs hold the last iterate */
    QCP_BREAKDOWN = 5,        /* a non-finite Krylov scalar appeared */
    QCP_ERR_TIMEOUT = 6,      /* a bounded device wait (persistent mode's grid barrier) gave up */
    QCP_WARN_NEAR_KINK = 7    /* solution within opts->kink_tol of a point where D Pi is undefined */
} qcp_status;

typedef enum { QCP_F64 = 0, QCP_F32 = 1 } qcp_dtype;

typedef enum {
    QCP_CONE_ZERO = 0,
    QCP_CONE_NONNEG = 1,
    QCP_CONE_SOC = 2,
    QCP_CONE_PSD = 3,
    QCP_CONE_EXP = 4,
    QCP_CONE_POW = 5
} qcp_cone_type;

/* CSR matrix; all pointers are device pointers. */
typedef struct {
    int64_t nrows, ncols, nnz;
    const int64_t* indptr;    /* nrows + 1 */
    const int32_t* indices;   /* nnz */
    const void* values;       /* nnz, float64 or float32 */
} qcp_csr;

/* Cone blocks in row order; HOST arrays of length nblocks. */
typedef struct {
    int32_t nblocks;
    const int32_t* type;      /* qcp_cone_type */
    const int32_t* dim;       /* block sizes, each >= 1, summing to m */
    const double* param;      /* per block: the exponent a in (0, 1) of a QCP_CONE_POW block (ignored
                                 elsewhere); may be NULL when there is none */
} qcp_cone;

typedef struct {
    int64_t n, m;             /* n >= 1 variables, m >= 0 constraint rows */
    qcp_csr P_upper;          /* n x n, upper triangle incl. diagonal */
    qcp_csr A;                /* m x n */
    qcp_csr AT;               /* n x m, the transpose of A */
    const int64_t* AT_perm;   /* nnz(A) or NULL */
    const void* q;            /* n */
    const void* b;            /* m */
    qcp_cone K;
} qcp_problem;

/* A solution of the conic pair: x (n), y (m) in K*, s (m) in K. */
typedef struct {
    const void* x;
    const void* y;
    const void* s;
} qcp_solution;

typedef enum {
    QCP_PRECOND_NONE = 0,     /* LSQR on F itself: the plain method of Sec. 3.1 */
    QCP_PRECOND_EQUILIBRATE = 1, /* LSQR on W F C: W = 1/(row norms of F), C = 1/(column norms of W F),
                                   C constant on each SOC block; D Pi's off-diagonal SOC terms are
                                   left out of the norms (any positive diagonal is a valid choice) */
    QCP_PRECOND_DIAG = 2,       /* LSQR on F C with C = diag(opts->precond_d), a caller-given positive
                                   right preconditioner (for instance the learned one), averaged
                                   over each SOC block (C must commute with D Pi); pass,
                                   persistent and cluster engines (the cluster engine refills its
                                   copy of M diag(C) on every such call) */
    QCP_PRECOND_JACOBI = 3      /* the classical column-norm (Jacobi) preconditioner: LSQR on F C with
                                   C = 1/(column norms of F), D Pi by its diagonal in the norms, C
                                   constant on each SOC block; computed on the plan's first such call;
                                   the engines of QCP_PRECOND_DIAG */
} qcp_precond;

/* How the Krylov iterations are run on the GPU (all give the same iterates up
   to rounding order; QCP_ENGINE_PASSES and QCP_ENGINE_PERSISTENT give
   bit-identical ones). */
typedef enum {
    QCP_ENGINE_PASSES = 0,      /* one launch per half-iteration over all tiles of all systems,
                                   replayed from CUDA graphs in chunks of check_every */
    QCP_ENGINE_PERSISTENT = 1,  /* every iteration of all systems in one cooperative launch,
                                   grid-wide barriers between passes, each wait bounded (a barrier
                                   that times out returns QCP_ERR_TIMEOUT) */
    QCP_ENGINE_CLUSTER = 2,     /* one thread-block cluster per system runs all of its iterations
                                   in one launch; the Krylov vectors live in the cluster's shared
                                   memory and only hardware cluster barriers separate passes.
                                   Needs every system to fit (about 8 N + 60 N / C bytes per CTA
                                   for C CTAs); zero, R+ and SOC blocks, and PSD (order <= 22),
                                   exponential and power blocks through their dense D Pi, and LSMR
                                   (the last two on the double-float kernel only; any qcp_precond);
                                   QCP_ERR_ARG otherwise */
    QCP_ENGINE_AUTO = 3,        /* the plan's autotuned engine when qcp_plan_autotune has run, else
                                   QCP_ENGINE_CLUSTER; a cluster choice becomes STREAM when a system
                                   does not fit the cluster engine (PASSES where STREAM cannot run
                                   the plan, and for QCP_PRECOND_DIAG / _JACOBI) */
    QCP_ENGINE_CLUSTER_FP64 = 4, /* QCP_ENGINE_CLUSTER with FP64 vector arithmetic.  The cluster engine
                                   otherwise computes its vector operations in double-float pairs of
                                   binary32 numbers (about 48 significant bits, on the FP32 pipes,
                                   which run 74 times faster than FP64 on this GPU), keeps the LSQR
                                   scalars in FP64, and itself uses FP64 when a magnitude in the
                                   data lies outside 2^-90..2^90 */
    QCP_ENGINE_STREAM = 5       /* one launch per half-iteration for problems of any size, the
                                   vector arithmetic in double-float pairs like the cluster engine
                                   (Krylov vectors in device memory, LSQR scalars and the tau
                                   entries in FP64): warp-sized work units (SELL-32 row slices,
                                   packed cone blocks, chunks of long rows) and no CTA-wide
                                   barrier inside a pass; replayed from CUDA graphs in chunks of
                                   check_every.  Zero, R+, SOC and PSD blocks of at most 256 rows,
                                   exponential and power blocks (the last three with D Pi stored
                                   as a dense matrix per block, made at plan time), precond
                                   NONE or EQUILIBRATE, LSQR or LSMR, magnitudes in the data within
                                   2^-90..2^90; QCP_ERR_ARG otherwise */
} qcp_engine;

typedef struct {
    int32_t solver;           /* 0 = LSQR (Paige & Saunders 1982), 1 = LSMR (Fong & Saunders 2011; the
                                 pass, persistent, stream and double-float cluster engines, AUTO
                                 choosing as for LSQR; CLUSTER_FP64 is an error).  Both minimise
                                 the same ||Op x - b|| and stop on the same estimate of
                                 ||r|| <= rtol ||b|| */
    double rtol;              /* target for ||F dz + dN|| / ||dN|| (JVP) or ||F^T r + g|| / ||g|| (VJP) */
    int64_t maxiter;          /* iteration cap per system (counted over all restarts) */
    int32_t check_every;      /* iterations between host convergence checks; 0 = none */
    int32_t use_graph;        /* 1 = replay the iteration chunk as a CUDA graph */
    int32_t compute_residual; /* 1 = recompute the true (unscaled) relative residual at exit and,
                                 if it is above rtol, continue iterating with a tighter internal
                                 tolerance (at most 4 times, while it keeps halving); 0 = trust the
                                 Krylov estimate */
    int32_t precond;          /* qcp_precond */
    int32_t engine;           /* qcp_engine */
    double kink_tol;          /* QCP_WARN_NEAR_KINK threshold on info.kink_margin */
    const double* warm_start; /* device, N = n + m + 1 entries per system (system-major), or NULL for
                                 the zero start: the initial iterate dz (JVP) or r (VJP) in the
                                 embedding's coordinates; its tau entry is ignored (gauge dz_N = 0).
                                 LSQR then solves for the correction, and rtol stays relative to the
                                 right-hand side itself */
    const double* precond_d;  /* device, N entries per problem (all directions of a problem share
                                 them): the positive column scaling C of QCP_PRECOND_DIAG */
} qcp_options;

typedef struct {
    int32_t status;           /* qcp_status of this system */
    int64_t iters;            /* Krylov iterations taken */
    double rel_residual;      /* true ||F dz + dN|| / ||dN|| at exit (if computed, else -1) */
    double rel_residual_est;  /* the Krylov recurrence's estimate of the same ratio */
    double kink_margin;       /* min over rows of the distance to a kink of D Pi (Appendix A) */
} qcp_info;

typedef struct qcp_plan qcp_plan;

/* Text of the last error on this host thread (never NULL). */
const char* qcp_last_error(void);

/* Fill *opts with defaults: LSQR, rtol 1e-10, maxiter 100000, check_every 32,
   use_graph 1, compute_residual 1, precond QCP_PRECOND_NONE,
   engine QCP_ENGINE_AUTO, kink_tol 0, warm_start NULL, precond_d NULL. */
void qcp_default_options(qcp_options* opts);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
int32_t qcp_version(void);

/*
 * Build a plan for one problem at one solution (Sec. 3.1, first step: form z
 * and Pi z; Sec. 2.4: the data of F).  Precomputes on the device P x,
 * g = 2 P x + q, kappa = x^T P x, z_y = y - s and the per-block state of
 * D Pi_{K*}(z_y) (Appendix A), lays out the combined matrix
 * [[P, A^T], [A, 0]] used by every product with F and F^T, and allocates
 * Krylov workspace for up to max_rhs simultaneous directions.
 * Errors: QCP_ERR_ARG (see qcp_status), QCP_ERR_ALLOC, QCP_ERR_CUDA.
 */
int qcp_plan_create(const qcp_problem* prob, const qcp_solution* sol, qcp_dtype dtype,
                    int32_t max_rhs, void* stream, qcp_plan** out);

/*
 * A plan over nprob independent problems of any sizes (probs[i], sols[i]),
 * run together in every launch (one direction per problem).  Vector and
 * value arguments of the batched calls are the per-problem arrays
 * concatenated in problem order.
 */
int qcp_batch_plan_create(int32_t nprob, const qcp_problem* probs, const qcp_solution* sols,
                          qcp_dtype dtype, void* stream, qcp_plan** out);

int qcp_plan_destroy(qcp_plan* plan);

/* Number of problems in the plan and total lengths of the concatenated
   arrays (n, m, nnz of P's upper pattern, nnz of A). */
int qcp_plan_sizes(const qcp_plan* plan, int64_t* nprob, int64_t* n_total, int64_t* m_total,
                   int64_t* nnzP_total, int64_t* nnzA_total);

/*
 * Forward product (Sec. 3.1): dN = D_theta N(z)[dP, dA, dq, db]
 * = (dP x + dA^T y + dq, -dA x + db, -x^T dP x - dq^T x - db^T y);
 * dz solves min ||F dz + dN||; (dx, dy, ds) = D phi(z) dz
 * = (dz_x - dz_N x, D dz_y - dz_N y, D dz_y - dz_y - dz_N s), D = D Pi_{K*}(z_y).
 * Inputs dP (nnz P), dA (nnz A), dq (n), db (m); outputs dx (n), dy (m), ds (m).
 * For a batched plan all arrays are concatenations over problems and info
 * points to nprob structs.  info may be NULL.
 */
int qcp_derivative_jvp(qcp_plan* plan, const qcp_options* opts, const void* dP, const void* dA,
                       const void* dq, const void* db, void* dx, void* dy, void* ds,
                       qcp_info* info);

/*
 * Adjoint product (Sec. 3.2): g = D phi(z)^T (wx, wy, ws)
 * = (wx, D (wy + ws) - ws, -x^T wx - y^T wy - s^T ws); r solves
 * min ||F^T r + g||; (dP, dA, dq, db) = D_theta N(z)^T [r] on the patterns:
 * dP_ij = (r1_i x_j + x_i r1_j)/2 - r_N x_i x_j, dA_ij = y_i r1_j - r2_i x_j,
 * dq = r1 - r_N x, db = r2 - r_N y.
 */
int qcp_derivative_vjp(qcp_plan* plan, const qcp_options* opts, const void* wx, const void* wy,
                       const void* ws, void* dP, void* dA, void* dq, void* db, qcp_info* info);

/*
 * k directions of a single-problem plan in one solve (k <= max_rhs): every
 * launch carries all k systems.  Arrays hold the k directions back to back
 * (direction i of dP at offset i * nnz(P), of dx at i * n, ...); info holds k
 * structs.
 */
int qcp_derivative_jvp_multi(qcp_plan* plan, const qcp_options* opts, int32_t k, const void* dP,
                             const void* dA, const void* dq, const void* db, void* dx, void* dy,
                             void* ds, qcp_info* info);
int qcp_derivative_vjp_multi(qcp_plan* plan, const qcp_options* opts, int32_t k, const void* wx,
                             const void* wy, const void* ws, void* dP, void* dA, void* dq, void* db,
                             qcp_info* info);

/*
 * JVPs of kj directions and VJPs of kv directions of a single-problem plan
 * in one call (kj, kv >= 1, kj + kv <= max_rhs): the two kinds of solve are
 * independent (Sec. 3.1 and 3.2 at the same point), so the cluster engine
 * runs them side by side, the JVP systems on the plan's stream and the VJP
 * systems on a second stream of the plan forked from it and joined back
 * before the call returns; the other engines run them one after the other.
 * The JVP arrays (dP .. ds) hold kj directions and the VJP arrays (wx .. gb)
 * kv directions, back to back as in the _multi calls; the results equal
 * those of qcp_derivative_jvp_multi and qcp_derivative_vjp_multi (bit for
 * bit on the same engine and cluster size).  info holds kj + kv structs, the
 * JVPs first.  opts->warm_start must be NULL.  Errors: QCP_ERR_ARG (batch
 * plan, bad counts, NULL arrays), the status codes of the single calls.
 */
int qcp_derivative_jvp_vjp_multi(qcp_plan* plan, const qcp_options* opts, int32_t kj, const void* dP,
                                 const void* dA, const void* dq, const void* db, void* dx, void* dy, void* ds,
                                 int32_t kv, const void* wx, const void* wy, const void* ws, void* gP, void* gA,
                                 void* gq, void* gb, qcp_info* info);

/*
 * Tile schedule of a plan (QCP_ENGINE_PASSES and _PERSISTENT): tile_nnz is
 * the target number of nonzeros of M per tile (rows are grouped into tiles,
 * never splitting an SOC block); a row with more than long_row nonzeros
 * leaves its tile and is cut into pieces of long_chunk nonzeros, one CTA
 * each.  Rebuilds the schedule and the Krylov workspace (and drops captured
 * graphs).  Defaults 4096, 512, 1 << 20.  Results are bit-reproducible from
 * run to run unless a row is cut into several pieces: the piece that
 * finishes last adds the row's terms to the pass's sums, so their position
 * in the summation (and the last bit of the result) depends on scheduling.
 * Used by the autotuner.  Errors: QCP_ERR_ARG (tile_nnz < 64, long_row < 1,
 * long_chunk < 32), QCP_ERR_ALLOC.
 */
int qcp_plan_set_schedule(qcp_plan* plan, int32_t tile_nnz, int32_t long_row, int32_t long_chunk);

/*
 * Autotuner.  Times every engine / schedule candidate on the plan itself
 * (synthetic directions from a fixed hash, rtol 0, `iters` LSQR iterations,
 * no true-residual pass) and keeps the fastest per pass as the plan's
 * choice for QCP_ENGINE_AUTO:
 *   - QCP_ENGINE_PASSES and _PERSISTENT with tile_nnz in {1024, 2048, 4096,
 *     8192, 16384} (long_row = tile_nnz / 8, long_chunk 1 << 20),
 *   - QCP_ENGINE_CLUSTER with 1, 2, 4, 8 and 16 CTAs per system, where every
 *     problem fits.
 * mode 0 tunes JVP solves, 1 VJP solves; nsys systems per call (ignored by
 * batch plans, which always solve all problems).  entries (host, capacity
 * cap, may be NULL) receives every candidate measured, *count their number
 * and *best (may be NULL) the chosen one, which stays in force until the
 * next qcp_plan_set_schedule, qcp_plan_set_cluster or autotune call (the
 * plan's schedule is left at the winner's tile size).  Errors: QCP_ERR_ARG
 * (bad mode, nsys, iters < 4), QCP_ERR_ALLOC, QCP_ERR_CUDA.
 */
typedef struct {
    int32_t engine;        /* qcp_engine */
    int32_t cluster_ctas;  /* CTAs per system (QCP_ENGINE_CLUSTER), else 0 */
    int32_t tile_nnz;      /* tile schedule (PASSES / PERSISTENT), else 0 */
    int32_t pad;
    double us_per_pass;    /* device time of one pass (one product with F or F^T of all systems) */
} qcp_tune_entry;

int qcp_plan_autotune(qcp_plan* plan, const qcp_options* opts, int32_t mode, int32_t nsys, int32_t iters,
                      qcp_tune_entry* entries, int32_t cap, int32_t* count, qcp_tune_entry* best);

/* CTAs per system under QCP_ENGINE_CLUSTER: 1 to 16 (above 8 is a
   non-portable cluster size), or 0 (the default) to choose per call: the
   most CTAs, up to 8, with which every system's cluster is resident at once
   (as the occupancy calculator reports it for this GPU).  A problem whose
   vectors need more CTAs' shared memory gets the smallest size that holds
   them.  Returns QCP_ERR_ARG for other values. */
int qcp_plan_set_cluster(qcp_plan* plan, int32_t max_ctas);

/* Sweeps of the QCP_PRECOND_EQUILIBRATE scaling (an addition to the
   paper's plain Krylov solve of Sec. 3.3): 1 to 64; a plan starts with 16.
   One sweep takes w = 1 / row norms of F and then c = 1 / column norms of
   W F, with D Pi by its diagonal and c constant on every coupled block;
   each further sweep recomputes w from the rows of F C and c from the new
   W F.  Both systems are consistent, so the outputs do not change, only
   the iteration count (on the 16-direction n = 2000 workload, 15 600 LSQR
   iterations per solve at 1 sweep, 1 140 at 16).  The plan recomputes w, c
   and its scaled copies of M on its stream before returning; if that fails
   the plan keeps its previous scaling.  Errors: QCP_ERR_ARG for a NULL
   plan, sweeps outside 1 to 64, or a plan that has already run a
   derivative or autotune call (w and c are then part of its captured
   graphs and cluster layouts); QCP_ERR_ALLOC, QCP_ERR_CUDA. */
int qcp_plan_set_equilibration(qcp_plan* plan, int32_t sweeps);

/* Bound of the waits at QCP_ENGINE_PERSISTENT's grid-wide barriers (an
   addition; the paper has no counterpart).  A CTA that waits at a barrier
   polls at most `polls` times, about 64 ns apart, then records a timeout;
   every CTA of the launch returns at its next barrier and the call returns
   QCP_ERR_TIMEOUT with the outputs unspecified.  polls = 0 restores the
   default bound (2^24 polls, about 1 s).  hold_ns > 0 (at most 1 s) makes
   CTA 0 of the next persistent launches wait that long by the GPU's global
   timer before its first barrier, so that the other CTAs' waits run out:
   a way to exercise the timeout path without any fault or unbounded wait.
   The plan stays usable after a timeout.  Errors: QCP_ERR_ARG (null plan,
   a negative value, hold_ns above 1e9). */
int qcp_plan_set_barrier_wait(qcp_plan* plan, int64_t polls, int64_t hold_ns);

/* Stream-engine scheduling of a call with one JVP range and one VJP range of
   equal size on one problem (qcp_derivative_jvp_vjp_multi on a plan that is
   not a batch plan); an addition, the paper solves the two systems
   separately.  on = 1 (the default): the two ranges iterate in step, the
   VJP systems one pass behind, so that every launch runs the same product
   (with G, then with G^T) for JVP system i and VJP system i and reads M's
   stored entries once for both.  on = 0: one range after the other.  Each
   system takes the same sequence of passes either way, so the outputs
   agree to rounding order (the CTA partial sums are grouped by the launch
   shape).  Errors: QCP_ERR_ARG (null plan, on not 0 or 1). */
int qcp_plan_set_stream_pairing(qcp_plan* plan, int32_t on);

/* The qcp_engine the most recent JVP/VJP call of the plan ran: PASSES,
   PERSISTENT, CLUSTER (double-float vector arithmetic) or CLUSTER_FP64; -1
   for a NULL plan. */
int qcp_plan_last_engine(const qcp_plan* plan);

/* Number of kernel launches made by the most recent JVP/VJP call of the plan
   (graph replays counted per kernel node). */
int64_t qcp_plan_last_launches(const qcp_plan* plan);

/*
 * The forward product of qcp_derivative_jvp for a single-problem plan and one
 * direction, for callers that must not allocate device memory when they ask
 * for a derivative: allocator hooks and callbacks that may not re-enter the
 * allocator, real-time loops where an allocation's latency or failure is not
 * acceptable, and hosts whose device memory is handed out by a pool they do
 * not own.  The paper has no counterpart; it is a deployment variant of the
 * same kernels (always the pass engine).
 *
 * All per-call scratch (Krylov vectors, LSQR scalars, reduction partials and
 * counters) lives in one 16 MiB file-scope device array of the library
 * instead of plan memory; about 48 bytes per embedding row N = n + m + 1
 * plus 40 bytes per tile, so problems up to roughly N = 340000 fit.  Larger
 * plans are rejected with QCP_ERR_ARG and a message giving the size needed.
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Every GPU that loads the library holds the array until the
 * process exits.
 *
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress, once per device).  Every call shares
 * the one array and clears it at entry, so calls whose work overlaps on the
 * GPU (two host threads, or two streams) race and must be serialised by the
 * caller.  Like qcp_derivative_jvp, the call reads convergence scalars back
 * to the host and synchronizes the plan's stream every check_every
 * iterations.  Arguments, options (check_every >= 1, LSQR, precond NONE or
 * EQUILIBRATE, no warm start) and outputs are those of qcp_derivative_jvp;
 * the plan must not be batched.  The plan's introspection queries
 * (qcp_plan_last_solution, _last_timing, _last_engine, _last_launches)
 * keep describing the plan's last regular call: a no-allocation call leaves
 * them as they were.
 */
int qcp_derivative_jvp_noalloc(qcp_plan* plan, const qcp_options* opts, const void* dP, const void* dA,
                               const void* dq, const void* db, void* dx, void* dy, void* ds,
                               qcp_info* info);

/* Device time (CUDA events on the plan's stream) of the Krylov iteration
   chunks of the most recent JVP/VJP call, and the number of pass launches
   (products with F or F^T over all systems) they contain; their ratio is
   the average duration of one pass.  Errors: QCP_ERR_ARG (null plan). */
int qcp_plan_last_timing(const qcp_plan* plan, double* pass_ms, int64_t* passes);

/* The system passes of the plan's most recent call that shared their read
   of M with another system's pass in the same launch (paired stream
   iterations, qcp_plan_set_stream_pairing; 0 otherwise): one per launch in
   which both systems of a pair ran a product.  Errors: QCP_ERR_ARG (null
   plan or output). */
int qcp_plan_last_shared_passes(const qcp_plan* plan, int64_t* shared);

/* The embedding-space solution of the plan's most recent call: dz (JVP) or
   r (VJP; F^T r = -g_phi), N = n + m + 1 doubles per system of that call
   (system-major; after qcp_derivative_jvp_vjp_multi the JVP systems come
   first), device pointer.  The training targets of the learned form
   come from here.  QCP_ERR_ARG before the first call. */
int qcp_plan_last_solution(qcp_plan* plan, double* out);

/* The plan's equilibration: row scaling w and column scaling c (N per
   problem, device, concatenated over the plan's problems). */
int qcp_plan_scalings(const qcp_plan* plan, double* w, double* c);

/* ---------------------------------------------------------------------------
 * Learned form: a network on per-row features predicts a warm start and a
 * diagonal right preconditioner for the Krylov solve (an addition: the
 * paper has no learned part).
 * ------------------------------------------------------------------------- */
#define QCP_MLP_IN 16
#define QCP_MLP_HIDDEN 256
#define QCP_MLP_OUT 2

/* Per-row features of every embedding row of the plan's problems (N per
   problem, concatenated), QCP_MLP_IN floats each, row-major, device:
   0 one; 1-5 one-hot row kind (x, zero cone, R+, SOC, tau); 6 x_i, y_i or 1;
   7 z_i = y_i - s_i; 8 q_i or b_i; 9 g_i = (2Px + q)_i, s_i or kappa; 10 the
   diagonal of D Pi; 11 log(||row of M||) / 4; 12 log(nnz(row of M) + 1) / 4;
   13 SOC block size / 32; 14 1 on an SOC block's entries after its first;
   15 feature 6 times feature 10 (0 where a feature does not apply).
   QCP_ERR_ARG for plans with PSD, exponential or power blocks (the
   features cover the zero, R+ and SOC blocks). */
int qcp_plan_features(qcp_plan* plan, float* out);

typedef struct qcp_mlp qcp_mlp;

/* Number of parameters, packed W1 [256 x 16], b1 [256], W2 [256 x 256],
   b2 [256], W3 [2 x 256], b3 [2] (FP32; W[j][i] maps input i to output j). */
int32_t qcp_mlp_param_count(void);

/* A 16-256-256-2 ReLU network for batches of up to max_rows rows on the given
   stream: BF16 weights and activations, FP32 accumulation (tensor cores),
   FP32 master weights and Adam state.  Parameters start at 0: set them with
   qcp_mlp_set_params. */
int qcp_mlp_create(int32_t max_rows, void* stream, qcp_mlp** out);
int qcp_mlp_destroy(qcp_mlp* mlp);
int qcp_mlp_set_params(qcp_mlp* mlp, const float* host_params);  /* also resets Adam */
/* Per-feature input normalisation x' = (x - mean) * inv_std (host arrays of
   QCP_MLP_IN; default 0 and 1), applied before x is rounded to BF16. */
int qcp_mlp_set_input_norm(qcp_mlp* mlp, const float* mean, const float* inv_std);
int qcp_mlp_get_params(const qcp_mlp* mlp, float* host_params);

/* y = W3 relu(W2 relu(W1 x' + b1) + b2) + b3 for rows x rows (device x:
   rows x 16, y: rows x 2; x' the normalised x), with x', the hidden
   activations and the weights rounded to BF16 (nearest even) where they
   enter a product. */
int qcp_mlp_forward(qcp_mlp* mlp, const float* x, int32_t rows, float* y);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the
   weighted squared error sum w (y - target)^2 / max(sum w, 1) (device
   rows x 2 arrays).  *loss_host gets the loss before the step; grad_host,
   if not NULL, the gradient in the packed layout (host). */
int qcp_mlp_train_step(qcp_mlp* mlp, const float* x, const float* target, const float* weight, int32_t rows,
                       float lr, double* loss_host, float* grad_host);

/* With v = y + offset (offset: rows x 2, or NULL for 0): warm_start[i] =
   scale * v[i][0] and precond_d[i] = exp(clamp(v[i][1], -8, 8)) (either
   output may be NULL); device arrays. */
int qcp_mlp_decode(const float* y, const float* offset, int64_t rows, double scale, double* warm_start,
                   double* precond_d, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QCPD_H */
