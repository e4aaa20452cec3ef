/*
 * ms.h -- C ABI of the GB300 multiscale fit library (libms.so).
 *
 * The library solves the monolithic multiscale system of Lot & Rieger
 * (arXiv 2503.04914): for a point hierarchy X_1..X_L with level supports
 * delta_l = nu * h_l (Assumption 2, eq. deltadef) and the scaled Wendland
 * kernel Phi_delta(x) = delta^-d phi(|x| / delta) (Assumption 1,
 * eq. kernelscaling), it finds coefficients alpha^(1..L) with
 *
 *     A_l alpha^(l) = f|_{X_l} - sum_{k<l} B_{lk} alpha^(k)           (eq. mas)
 *     A_l = Phi_{delta_l}(X_l, X_l),  B_{lk} = Phi_{delta_k}(X_l, X_k)  (Section 3)
 *
 * i.e. T_L alpha = f for the block lower-triangular T_L of eq. bigt.  It is
 * solved as eq. split: Jacobi sweeps on the normalised factor T'_L
 * (eq. jacobi, Theorem 9) whose inner steps are per-level conjugate
 * gradients on the block diagonal D_L (Theorem 8, eq. blockdiagonal_levelwise),
 * and the approximant f_L(x) = sum_l sum_n alpha_n^(l) Phi_{delta_l}(x - x_n^(l))
 * (eq. fapproximation) is evaluated at query points.
 *
 * Conventions (all entry points):
 *  - Every entry point returns an ms_status; MS_OK is 0.  On failure
 *    ms_last_error() gives a message (thread-local, valid until the next
 *    call on the same thread).  No C++ exception crosses this boundary.
 *  - Point arrays are float64, row-major [n][d], with the levels
 *    concatenated coarse to fine (level 1 first).  Coefficient and data
 *    arrays use the same level-concatenated order as the points the caller
 *    passed ("input order"); the library permutes internally and undoes it.
 *  - Multi-right-hand-side arrays are row-major [N][nrhs].
 *  - Plain entry points take HOST pointers; the caller owns them and the
 *    library copies what it needs before returning.  *_dev entry points take
 *    DEVICE pointers on the current CUDA device plus a cudaStream_t passed as
 *    void* (NULL = the legacy default stream); they enqueue work on that
 *    stream and may return before it completes, except where stated.
 *  - The hierarchy handle owns all device memory it allocates (cudaMalloc);
 *    ms_destroy frees it.  A handle is bound to the device that was current
 *    when it was built and must be used with that device current.
 *  - Device-side failures (CG breakdown, iteration caps, barrier time-outs)
 *    are recorded in device flags and reported by the call that waits for
 *    the result; the library never traps, asserts or spins unboundedly on
 *    the GPU.
 */
#ifndef MS_H
#define MS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MS_MAX_LEVELS 32
#define MS_ABI_VERSION 3

typedef struct ms_hierarchy ms_hierarchy;

typedef enum {
    MS_OK = 0,
    MS_ERR_ARG = 1,            /* invalid argument (sizes, d, L, delta, kernel, NULL) */
    MS_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    MS_ERR_OOM = 3,            /* device allocation failed */
    MS_ERR_NOT_SPD = 4,        /* CG breakdown: p^T A p <= 0 or non-finite on some level */
    MS_ERR_NOT_CONVERGED = 5,  /* a level hit its iteration cap before the tolerance */
    MS_ERR_TIMEOUT = 6,        /* a bounded device-side wait (grid barrier) ran out */
    MS_ERR_NUMERIC = 7,        /* non-finite input data */
    MS_ERR_STATE = 8           /* call not valid in the handle's current state */
} ms_status;

/* Operator used for a mat-vec family. */
enum { MS_OP_CSR = 0, MS_OP_MATRIX_FREE = 1, MS_OP_AUTO = 2 };
/* Arithmetic of the level CG solves. */
enum {
    MS_PREC_FP64 = 0,   /* FP64 mat-vecs, vectors and dots */
    MS_PREC_MIXED = 1   /* FP32 mat-vecs and inner vectors, FP64 dots, FP64 outer
                           true-residual refinement, FP64 level-finalising Jacobi updates */
};
/* Preconditioner of the level CG solves (MIXED precision only).  Both kinds are
 * factorised sparse approximate inverses M = G^T G (Kolotilina-Yeremin): row i of the
 * lower-triangular G lives on i and its (up to) 16 nearest same-level points within
 * delta_l that precede it in input order, and equals A_P^{-1} e_1 / sqrt((A_P^{-1})_11)
 * for the patch matrix A_P.  M is symmetric positive definite whenever G's diagonal is
 * positive, so the preconditioned CG cannot break down.  The paper has no
 * preconditioner; the locality it exploits is that of A_l^{-1} (Lemma 5). */
enum {
    MS_PRECOND_NONE = 0,
    MS_PRECOND_LEARNED = 1, /* rows predicted by the trained network (ms_train_precond) */
    MS_PRECOND_EXACT = 2    /* rows from exact FP64 patch solves (the network's teacher) */
};

/* Options of a hierarchy; fill with ms_default_opts() and override fields. */
typedef struct ms_opts {
    int wendland_d;      /* Wendland phi_{d,k}: space dimension index d (>= point dimension), 1..3 */
    int wendland_k;      /* smoothness index k, 0..3 (phi_{3,1} = (1-r)^4 (4r+1), Section 5) */
    double nu;           /* delta_l = nu * h_l (eq. deltadef); > 0 */
    int op;              /* operator for the level matrices A_l in the FP32 inner CG (MS_OP_*) */
    int precision;       /* MS_PREC_* */
    int precond;         /* MS_PRECOND_* */
    int max_iters;       /* cap on CG iterations per level and solve; 0 = 20000 */
    int jacobi_sweeps;   /* Jacobi sweeps on T'; 0 = L-1 (exact from beta_0 = f, Theorem 9);
                            -1 = none: the fit returns alpha = D_L^{-1} f, the block-diagonal
                            solve of eq. split alone (per-level CG on every level at once) */
    double inter_tol;    /* relative tolerance of the non-final (intermediate) level solves
                            inside the Jacobi sweeps.  0 = 1: a non-final level keeps its
                            previous iterate (no CG iterations until its beta is final; the
                            fastest schedule, same result).  inter_tol = rel_tol solves every
                            level in every sweep as Algorithm 2 does. */
    double inner_tol;    /* MIXED: relative tolerance of each FP32 inner CG; 0 = 1e-4 */
    int cell_split;      /* neighbour-grid cell size = delta_l / cell_split (1 or 2); 0 = 1, or
                            with autotune = 1 the faster of 1 and 2 (see autotune) */
    int threads_per_row; /* CSR sub-warp width for A (1..32, power of 2); 0 = automatic */
    int lower_fp32;      /* 1: also store FP32 values of the B blocks (for MS_APPLY_B32) */
    int solve_ctas_per_sm; /* CTAs of the persistent solve kernel per SM: 1 (up to 128
                              registers a thread) or 2 (up to 64); 0 = automatic (2, or with
                              autotune = 1 the tuned one) */
    int autotune;        /* 1: tune per hierarchy shape, each choice cached per process:
                            - at the build, if cell_split = 0: build with cells of delta and
                              delta / 2, keep the one whose build plus one application of the
                              fit's matrix-free operators is faster;
                            - at the first fit: time the CSR mat-vec of every level of at least
                              4096 rows with 1, 2, 4, 8, 16 and 32 lanes per row (the matrix-free
                              mat-vec: 1 to 8 lanes per point) and keep the fastest;
                            - at the first fit, if solve_ctas_per_sm = 0: fit with 1 and with 2
                              CTAs per SM and keep the faster (the call returns the second fit).
                            0 = rules (about 16 entries per lane, 2 CTAs per SM, cell = delta).
                            threads_per_row > 0 overrides the lane choice. */
    int lower_op;        /* operator of the strictly lower blocks B_kj in the fit's Jacobi updates:
                            MS_OP_CSR (default): B stored as CSR by the build (FP64 values);
                            MS_OP_MATRIX_FREE (MIXED only): the build stores no B and every
                            update recomputes B's entries in double-float arithmetic (the values a
                            MIXED build would store, about 1e-14 relative) and sums them in
                            double-float.  Under the default schedule each block is read once per
                            fit, so a hierarchy that is fitted once saves B's assembly and its
                            12 bytes per entry; one fitted many times is faster with CSR.  Needs
                            the default schedule (inter_tol 0 or >= 1); MS_APPLY_B64/B32 are then
                            unavailable. */
    int reserved[4];
} ms_opts;

/* Per-fit statistics (all levels 0-based, coarse to fine). */
typedef struct ms_fit_stats {
    int32_t L;
    int32_t sweeps;                      /* Jacobi sweeps run */
    int64_t cg_iterations[MS_MAX_LEVELS];/* CG iterations actually run, summed over all solves
                                            of the level (inner FP32 iterations in MIXED) */
    int32_t refinements[MS_MAX_LEVELS];  /* MIXED: FP64 outer residual evaluations per level */
    double rel_residual[MS_MAX_LEVELS];  /* final FP64 true relative residual
                                            |beta_l - A_l alpha_l| / |beta_l| per level */
    int32_t precond_fallbacks;           /* levels that fell back from the learned preconditioner */
    int32_t fp64_fallbacks;              /* MIXED: levels whose inner CG switched to FP64 because an
                                            outer refinement round did not halve the residual */
    int32_t device_status;               /* ms_status raised on the device (0 = none) */
    double fit_ms;                       /* device time of the solve (CUDA events) */
    double matvec_bytes;                 /* algorithmic bytes moved by the solve kernel
                                            (matrix + vector traffic of every phase) */
    int64_t kernel_launches;             /* library kernels launched by the call */
    double phase_ms[8];                  /* device timeline of the solve kernel as seen by its
                                            first CTA (%globaltimer): [0] FP64 true residuals,
                                            [1] CG mat-vec + dots, [2] CG vector updates,
                                            [3] grid-barrier waits (includes load imbalance),
                                            [4] lower-block (Jacobi) updates, [5] other vector
                                            phases, [6] scalar decisions, [7] unused */
    int32_t solve_launches;              /* cooperative solve launches of the call */
    int32_t rhs_per_launch;              /* most right-hand sides one solve launch carried: blocks
                                            of min(32, 256 / L) right-hand sides, up to 16 blocks in
                                            one launch (2 CTAs per SM; one partition of the grid
                                            per block) */
} ms_fit_stats;

/* Sizes of a built hierarchy. */
typedef struct ms_info {
    int32_t d, L;
    int64_t N;
    int64_t n_per_level[MS_MAX_LEVELS];
    double delta[MS_MAX_LEVELS];
    int64_t nnz_A;       /* stored entries of the block diagonal (all A_l) */
    int64_t nnz_B;       /* stored entries of the strictly lower blocks (all B_kj, k > j) */
    int64_t device_bytes;/* device memory held by the handle */
    double build_ms;     /* device time of the last build (CUDA events) */
    int32_t tpr_A[MS_MAX_LEVELS]; /* CSR lanes per row of A_l in the solve (as of the last fit) */
    int32_t pc_basis;    /* candidate rows per point of the handle's network (ms_train_opts.n_basis) */
    int32_t cell_split;  /* neighbour-grid cells per delta_l in use (opts.cell_split, or the tuned one) */
    int32_t solve_ctas_per_sm; /* solve-kernel CTAs per SM in use (opts, or the tuned one after a fit) */
} ms_info;

/* Fill *opts with defaults: phi_{3,1}, nu = 4, CSR, FP64, no preconditioner. */
void ms_default_opts(ms_opts* opts);

/*
 * Build a hierarchy: validate (Assumption 2 inputs), copy the points to the
 * device, bin every level into a uniform cell grid of cell size delta_l
 * (Morton order of cells, counting sort, ties by input index), and assemble
 * the block-diagonal A_l and strictly lower B_kj blocks in CSR
 * (int64 row offsets, int32 column indices, FP64 values and, for MIXED,
 * FP32 values).
 *   d            point dimension, 1..3
 *   L            number of levels, 1..MS_MAX_LEVELS
 *   n_per_level  host [L], N_l >= 1
 *   points       host [N][d] float64, level-concatenated (must be finite)
 *   h_per_level  host [L], h_l > 0; delta_l = opts->nu * h_l
 *   opts         host, NULL = defaults
 *   out          receives the handle (NULL on failure)
 * Errors: MS_ERR_ARG (d, L, N_l, h, nu, kernel, NULL pointers), MS_ERR_NUMERIC
 * (non-finite points), MS_ERR_OOM, MS_ERR_CUDA.  Synchronous.
 */
ms_status ms_build_hierarchy(int d, int L, const int64_t* n_per_level, const double* points,
                             const double* h_per_level, const ms_opts* opts, ms_hierarchy** out);

/* As ms_build_hierarchy with points_dev a DEVICE [N][d] float64 array; the build runs on
 * `stream` and the call returns once the handle is complete (it reads back the sizes). */
ms_status ms_build_hierarchy_dev(int d, int L, const int64_t* n_per_level, const double* points_dev,
                                 const double* h_per_level, const ms_opts* opts, void* stream,
                                 ms_hierarchy** out);

/*
 * Fit: solve T_L alpha = f (eq. bigt) by eq. split.  Jacobi sweeps m = 1..S on
 * T'_L beta = f starting from beta_0 = f (eq. jacobi); in sweep m the level
 * solves t_l = A_l^{-1} beta_l (l < L) run together, warm-started from the
 * previous sweep, and beta_k = f_k - sum_{j<k} B_kj t_j is recomputed.  Levels
 * whose beta is already final are not re-solved.  Finally alpha_l = A_l^{-1} beta_l
 * for every level.  Each level solve stops at |beta_l - A_l x| <= rel_tol |beta_l|
 * (FP64 true residual).  The whole fit is one persistent cooperative kernel per
 * batch of right-hand sides: up to min(32, 256 / L) right-hand sides share a
 * launch, each (right-hand side, level) pair with its own CG scalars and
 * stopping test (the batch reduces its dot products in another fixed order than
 * a single fit, so a column agrees with its single fit to the tolerance, not
 * bitwise; the result is deterministic).
 *   f          host [N] (nrhs == 1) or [N][nrhs], input order
 *   nrhs       >= 1
 *   rel_tol    in (0, 1)
 *   alpha_out  host, same shape as f, input order
 *   stats      nullable; over all right-hand sides: cg_iterations and
 *              refinements summed, rel_residual the largest, fit_ms and
 *              matvec_bytes summed over the launches
 * Errors: MS_ERR_ARG, MS_ERR_NUMERIC (non-finite f), MS_ERR_NOT_SPD,
 * MS_ERR_NOT_CONVERGED (alpha_out still holds the last iterate),
 * MS_ERR_TIMEOUT, MS_ERR_CUDA.  Synchronous.
 */
ms_status ms_fit(ms_hierarchy* h, const double* f, int nrhs, double rel_tol, double* alpha_out,
                 ms_fit_stats* stats);

/* As ms_fit with DEVICE f_dev / alpha_dev; synchronous with respect to `stream`
 * (it waits for the device status before returning). */
ms_status ms_fit_dev(ms_hierarchy* h, const double* f_dev, int nrhs, double rel_tol,
                     double* alpha_dev, ms_fit_stats* stats, void* stream);

/*
 * Allocation-free fit.  The paper has no counterpart: this is a service for
 * callers that cannot allocate device memory when they fit.  ms_fit_dev gives
 * the handle a work space with cudaMalloc on its first call; callers whose
 * device memory is already fully reserved by another allocator or pool, loops
 * that must not call the allocator (cudaMalloc/cudaFree can synchronise the
 * device), and processes with a device-memory budget fixed at start-up cannot
 * allow that.  This entry point computes the same fit as ms_fit_dev for ONE
 * right-hand side, but the call allocates nothing: its work space is a fixed
 * device array of about 5.6 MiB inside libms.so, held by every GPU that loads
 * the library until the process exits.
 *   h          a built hierarchy with at most 65536 points in total
 *              (larger ones are rejected with MS_ERR_ARG); its device must be current
 *   f_dev      DEVICE float64 [N], input order
 *   rel_tol    in (0, 1), as for ms_fit
 *   alpha_dev  DEVICE float64 [N], input order (written)
 *   stats      nullable
 *   stream     cudaStream_t as void*; the call waits for the stream before returning
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture.  Every call shares the one array per device, which keeps the
 * previous call's contents (the call clears what must start at zero): calls
 * whose work overlaps on the GPU (other threads, other streams, other
 * handles) race on it and must be serialised by the caller.
 * Errors: MS_ERR_ARG, MS_ERR_STATE (wrong device current, FP32 values missing
 * for MIXED), MS_ERR_NOT_SPD, MS_ERR_NOT_CONVERGED, MS_ERR_NUMERIC (non-finite
 * f), MS_ERR_TIMEOUT, MS_ERR_CUDA.
 */
ms_status ms_fit_static_dev(ms_hierarchy* h, const double* f_dev, double rel_tol, double* alpha_dev,
                            ms_fit_stats* stats, void* stream);

/*
 * Batched fit of nh independent hierarchies (one right-hand side each) in one
 * persistent cooperative launch: eq. split for every hierarchy, as ms_fit_dev
 * computes it.  The grid is split into partitions of CTAs, one per hierarchy, in
 * proportion to its work (A nonzeros + points); each partition has its own grid
 * barrier and reductions.  More hierarchies than the launch has CTAs (2 per SM)
 * run in successive launches.  The paper fits one hierarchy; this is the
 * throughput form for many small ones.
 *   hs         host [nh] built handles, all on the current device, all FP64 or all
 *              MIXED (each keeps its own kernel, op and preconditioner options)
 *   nh         >= 1
 *   f_dev      host [nh] of DEVICE float64 [N_i], input order
 *   rel_tol    in (0, 1), as for ms_fit
 *   alpha_dev  host [nh] of DEVICE float64 [N_i], input order (written)
 *   stats      nullable host [nh]; fit_ms and kernel_launches are those of the
 *              whole batch
 *   stream     cudaStream_t as void*; the call waits for the stream before returning
 * Errors: MS_ERR_ARG (NULL arrays, mixed precisions), MS_ERR_STATE (a handle of
 * another device, FP32 values missing), and the device statuses of ms_fit (the
 * first failing hierarchy is named in ms_last_error()).
 */
ms_status ms_fit_batch_dev(ms_hierarchy* const* hs, int nh, const double* const* f_dev, double rel_tol,
                           double* const* alpha_dev, ms_fit_stats* stats, void* stream);

/* As ms_fit_batch_dev with HOST f[i] / alpha_out[i] (float64 [N_i], input order). */
ms_status ms_fit_batch(ms_hierarchy* const* hs, int nh, const double* const* f, double rel_tol,
                       double* const* alpha_out, ms_fit_stats* stats);

/*
 * A prepared batched fit, for fitting the same hierarchies again and again (new
 * values in the same right-hand-side buffers).  ms_batch_plan_create does every
 * host-side step of ms_fit_batch_dev once: work space, preconditioner rows,
 * autotuning, the split of the grid among the hierarchies and the upload of the
 * kernel arguments; it binds the DEVICE buffers f_dev[i] and alpha_dev[i]
 * (float64 [N_i], input order), which must stay allocated while the plan lives.
 * Arguments and errors as for ms_fit_batch_dev, plus MS_ERR_ARG when a handle
 * appears twice.  Waits for `stream` before returning.
 *
 * While a plan lives, its hierarchies' work space cannot grow: an ms_fit with
 * more right-hand sides than the handle has fitted before returns MS_ERR_STATE.
 * Destroy every plan of a hierarchy before the hierarchy.
 */
typedef struct ms_batch_plan ms_batch_plan;
ms_status ms_batch_plan_create(ms_hierarchy* const* hs, int nh, const double* const* f_dev, double rel_tol,
                               double* const* alpha_dev, void* stream, ms_batch_plan** out);

/*
 * Enqueue one batched fit of the plan on `stream` (reads f_dev, writes alpha_dev).
 * Nothing here waits, allocates or copies from the host, so the call may be
 * captured into a CUDA graph by the caller.  use_graph = 1: the library captures
 * the launch sequence into a CUDA graph at the first such call (on a private
 * stream) and from then on replays it with one cudaGraphLaunch on `stream`.
 * Results: ms_batch_plan_stats after the stream has reached the launch.
 * Errors: MS_ERR_ARG (NULL plan), MS_ERR_STATE (another device is current),
 * MS_ERR_CUDA (a launch, a capture or an instantiation failed).
 */
ms_status ms_batch_plan_launch(ms_batch_plan* plan, void* stream, int use_graph);

/*
 * Waits for `stream`, then fills stats (nullable, host [nh]) from the plan's last
 * completed launch; fit_ms is 0 (time launches with events on the stream).
 * Returns the first non-zero device status of the batch (as ms_fit_batch_dev).
 */
ms_status ms_batch_plan_stats(ms_batch_plan* plan, void* stream, ms_fit_stats* stats);

/* Waits for the device, then frees the plan.  NULL is a no-op. */
void ms_batch_plan_destroy(ms_batch_plan* plan);

/*
 * Evaluate the approximant f_L(q) = sum_l sum_n alpha_n^(l) Phi_{delta_l}(q - x_n^(l))
 * (eq. fapproximation) at nq query points, FP64 throughout.
 *   alpha  host [N] or [N][nrhs], input order;  query host [nq][d];  out host [nq][nrhs].
 * Errors: MS_ERR_ARG, MS_ERR_CUDA.  Synchronous.  nq == 0 is valid (no work).
 */
ms_status ms_evaluate(ms_hierarchy* h, const double* alpha, int nrhs, const double* query,
                      int64_t nq, double* out);

/* As ms_evaluate with DEVICE pointers, enqueued on `stream`. */
ms_status ms_evaluate_dev(ms_hierarchy* h, const double* alpha_dev, int nrhs, const double* query_dev,
                          int64_t nq, double* out_dev, void* stream);

/* Building blocks of the solve, exposed for verification and benchmarking. */
enum {
    MS_APPLY_A64 = 0,   /* y = D_L x   (all A_l, FP64 CSR)                       Section 3 */
    MS_APPLY_A32 = 1,   /* y = D_L x   (FP32 CSR values, FP32 accumulation)      */
    MS_APPLY_AMF32 = 2, /* y = D_L x   (matrix-free FP32: entries recomputed)    */
    MS_APPLY_B64 = 3,   /* y = (T_L - D_L) x  (all B_kj, k > j, FP64 CSR)        eq. bigt */
    MS_APPLY_B32 = 4,   /* y = (T_L - D_L) x  (FP32 CSR)                          */
    MS_APPLY_BMF32 = 5, /* y = (T_L - D_L) x  (matrix-free FP32 entries and sums)  */
    MS_APPLY_BMFDF = 6  /* y = (T_L - D_L) x  (matrix-free double-float entries and
                           sums, the fit's lower_op = MS_OP_MATRIX_FREE; MIXED builds) */
};
/*
 * y = op x for one of the MS_APPLY_* operators.  x_dev, y_dev: DEVICE float64 [N].
 * sorted_order = 0: x and y are in input order (the library permutes);
 * sorted_order = 1: x and y are in the library's internal (cell-sorted) order,
 * see ms_get_permutation.  FP32 operators round x to FP32 and widen y to FP64;
 * MS_APPLY_BMFDF splits x into double-float parts.  The matrix-free lower operators
 * (the paper's McV, Section 5.3) give row y_s of level k the sum over the levels j < k
 * of the entries Phi_{delta_j}(x_s - x_p) x_p of the level-j points p within delta_j,
 * found through level j's cell grid.
 * Errors: MS_ERR_ARG (unknown op, an FP32 CSR op on a handle built without
 * FP32 values, a CSR lower op on a handle built with lower_op = MS_OP_MATRIX_FREE,
 * MS_APPLY_BMFDF on an FP64 build), MS_ERR_CUDA.  Enqueued on `stream`.
 */
ms_status ms_apply_dev(ms_hierarchy* h, int op, const double* x_dev, double* y_dev,
                       int sorted_order, void* stream);

/* perm_out (host int64 [N]): perm_out[s] = input index of the point at sorted position s. */
ms_status ms_get_permutation(const ms_hierarchy* h, int64_t* perm_out);

/* Sizes and timings of a built hierarchy. */
ms_status ms_hierarchy_info(const ms_hierarchy* h, ms_info* info);

/* ---------------------------------------------------------------- learned preconditioner
 * The network maps the delta-scaled offsets (x_j - x_i)/delta_l of a point's pattern
 * neighbours (16 d inputs, zero-padded, in the patch's canonical frame) through ReLU layers
 * of width 64 to 17 m outputs o_1..o_m: m candidate scale-free rows (self first, zero past
 * the patch), u_1 = mu + sigma o_1 (per-entry mean and deviation of the training targets)
 * and u_k = sigma o_k for k > 1.  The row is the factorised sparse approximate inverse
 * within their span: with U = [u_1..u_m] and K = phi(|z_a - z_b|) the scaled patch matrix,
 * ghat = U y / sqrt(q), y = (S + 1e-6 diag(S))^-1 U^T e_1, S = U^T K U, q = e_1^T U y -- the
 * minimiser of g^T K g with g_self = 1 in the span, normalised to g^T K g = 1 (the exact
 * row's value) with g_self = sqrt(q) > 0, and the exact row whenever the span holds it; a
 * patch of n <= m points takes the exact row.  Because A_P = delta^-d K(offsets / delta)
 * (eq. kernelscaling), ghat = delta_l^{-d/2} g does not depend on the level, so a network
 * trained on coarse levels serves every level.  Training minimises the mean gap
 * log q* - log q >= 0 to the exact row (q* = (K^-1)_11).  Inference uses BF16-valued
 * weights with FP32 accumulation and an FP32 combination; training is Adam on FP32 master
 * weights whose forward and backward passes use the BF16-rounded copies. */
typedef struct ms_train_opts {
    int epochs;          /* passes over the training patches (default 100) */
    int batch;           /* samples per Adam step, a multiple of 64 (default 512) */
    double lr;           /* initial learning rate (default 3e-3), cosine-decayed to lr_final */
    double lr_final;     /* default 1e-4 */
    uint64_t seed;       /* SplitMix64 seed of the initial weights and of the shuffles */
    int fp32_weights;    /* 1: train and infer with the FP32 master weights (no BF16 rounding) */
    float input_noise;   /* training inputs jittered by input_noise * U[-1, 1) per coordinate
                            (units of delta; default 0.005; 0 = off) */
    int augment;         /* extra training patches per point, 0..16 (default 4): draw r of point i
                            (level-local input index i of a level of n points) takes the 16
                            nearest points j != i within delta among the level's first p points,
                            p = i + 1 + min(floor(u (n - i)), n - i - 1), u = the SplitMix64
                            uniform draw (top 53 bits / 2^53) of seed ^ 0x6175676D656E74 with
                            counter r N + (global input index of i), N = the hierarchy's points */
    int n_basis;         /* candidate rows m the network predicts per point, 1..16 (0 = default 16) */
    int reserved[4];
} ms_train_opts;

typedef struct ms_train_stats {
    int64_t samples;     /* training patches: (1 + augment) x the points of the chosen levels */
    int64_t steps;       /* Adam steps taken */
    double loss_first;   /* mean gap log q* - log q of the first and of the last step's batch */
    double loss_last;
    double train_ms;     /* device time of the training loop */
    int32_t n_params;
} ms_train_stats;

void ms_default_train_opts(ms_train_opts* opts);

/* Train the network on the exact rows (FP64 patch Cholesky) of every point of the given
 * 0-based levels of h; the weights are kept in h and used by fits with
 * precond = MS_PRECOND_LEARNED.  opts NULL = defaults.  Errors: MS_ERR_ARG (levels,
 * options), MS_ERR_OOM, MS_ERR_CUDA.  Synchronous. */
ms_status ms_train_precond(ms_hierarchy* h, const int* levels, int n_levels, const ms_train_opts* opts,
                           ms_train_stats* stats);

/* Export (set = 0) or import (set = 1) the network: params is host float[n] with
 * n = n_weights + 34: the FP32 weights in the order W1 [64][16d], b1 [64], W2 [64][64],
 * b2 [64], W3 [17m][64], b3 [17m] (row-major; output 17 k + a is entry a of candidate k),
 * then the 17 per-entry means and 17 standard deviations.  n_weights = 1024 d + 4224 +
 * 1105 m; importing takes m from n (1..16) and marks the network trained; exporting needs
 * n for the handle's current m (ms_info.pc_basis).  Errors: MS_ERR_ARG (n), MS_ERR_STATE
 * (export without weights). */
ms_status ms_precond_params(ms_hierarchy* h, float* params, int64_t n, int set);

/* Inspection of the preconditioner's building blocks (host outputs, input order). */
enum {
    MS_INSPECT_PATTERN = 0, /* int32 [N][16]: pattern neighbours (input indices), -1 = none */
    MS_INSPECT_TARGETS = 1, /* double [N][17]: exact scale-free rows ghat (zeros past the pattern) */
    MS_INSPECT_PREDICT = 2, /* float [N][17]: the network's rows ghat */
    MS_INSPECT_GRAD = 3,    /* float [n_weights + 1]: full-batch gradient of the training loss on
                               the patterns of `levels` (no extra patches) with the FP32 master
                               weights, then the loss */
    MS_INSPECT_PATCHES = 4, /* int32 [S][18]: the training patches of `levels` with the options of
                               the last ms_train_precond (defaults before any): per patch its
                               centre, its prefix bound p (level-local; p = centre for the
                               pattern) and 16 neighbours (input indices, -1 = none); S =
                               (1 + augment) x the points of `levels`, patterns first, then
                               draw 0, 1, ... each in level order, points in input order */
    MS_INSPECT_CANDIDATES = 5 /* float [N][17 m]: the network's m candidate rows of every point,
                               entry a of candidate k at 17 k + a (u_1 = mu + sigma o_1,
                               u_k = sigma o_k, zero past the patch) */
};
ms_status ms_precond_inspect(ms_hierarchy* h, int what, const int* levels, int n_levels, void* out, int64_t n_out);

/* Instruction-rate probes of the current device, the denominators of the ALU-bound
 * rooflines: dependent chains of FP32 fused multiply-adds, of FP64 fused multiply-adds or of
 * FP32 reciprocal square roots (the special-function unit), eight independent chains per
 * thread on four 256-thread blocks per SM; the best of three timed launches.
 *   per_s  host, written: warp-lane instructions per second (an FMA is one instruction)
 * Errors: MS_ERR_ARG (kind, NULL), MS_ERR_CUDA.  Synchronous; runs about 10 ms. */
enum { MS_PROBE_FP32 = 0, MS_PROBE_FP64 = 1, MS_PROBE_XU = 2 };
ms_status ms_peak_probe(int kind, double* per_s);

/* Self-test of the solve kernel's bounded waits.  One CTA enters the grid barrier of the
 * persistent solve kernel (the same device code) as one of two CTAs of its partition; the
 * other never arrives, so the wait has to give up: after timeout_s it records MS_ERR_TIMEOUT
 * in the device status word and the kernel returns.  With peer_timed_out != 0 the status
 * word starts at MS_ERR_TIMEOUT, as if another CTA had timed out already, and the wait must
 * leave within a few hundred polls instead.  Nothing faults or hangs; the context stays
 * usable.
 *   timeout_s       the wait's limit in seconds, in (0, 10]
 *   device_status   host, written: the status word after the kernel (MS_ERR_TIMEOUT expected)
 *   waited_s        host, written (may be NULL): the kernel's duration (CUDA events)
 * Errors: MS_ERR_ARG (timeout_s out of range, device_status NULL), MS_ERR_CUDA.
 * Synchronous. */
ms_status ms_wait_selftest(double timeout_s, int peer_timed_out, int* device_status, double* waited_s);

/* Number of CUDA kernels this library has launched in the calling process so far
 * (all threads and handles; the count is taken at launch time, not completion). */
uint64_t ms_launch_count(void);

/* Message of the last failing call on this thread ("" if none). */
const char* ms_last_error(void);

/* Free the handle and all device memory it owns; NULL is a no-op.  Waits for the device
 * to finish pending work first.  The library draws device memory, the handles' and the
 * builds' scratch alike, from one memory pool per device that keeps freed memory mapped for
 * reuse by later handles and builds (released by ms_trim_memory or at process exit): the
 * pool's footprint is the largest amount in use at any one time.  A build's own scratch
 * (cell keys, per-row frames and pair counts, scan tiles) is freed when the build returns
 * but stays in the pool: about 0.8 GB for 1.4M points in 2-D (delta = 4 h) and a few GB for
 * 4.7M points in 3-D. */
void ms_destroy(ms_hierarchy* h);

/* Return the unused memory of the current device's library pool (memory no live handle,
 * plan or call holds) to the device, so that other allocators in the process can use it;
 * the library's next allocations map memory again.  The paper has no counterpart (memory
 * management).  Errors: MS_ERR_CUDA.  Synchronous with respect to the pool's own stream. */
ms_status ms_trim_memory(void);

#ifdef __cplusplus
}
#endif
#endif /* MS_H */
