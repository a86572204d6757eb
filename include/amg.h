/*
 * amg.h -- C ABI of the GB300 (sm_103a) smoothed-aggregation AMG solver.
 *
 * The library solves A x = f for a square sparse A with a Krylov method
 * preconditioned by one AMG V-cycle per iteration:
 *   - setup (Algorithm 1 of D. Demidov, "AMGCL: an Efficient, Flexible, and
 *     Extensible Algebraic Multigrid Implementation"): while A_i is too big to
 *     be solved directly, build the transfer operators P_i and R_i = P_i^T
 *     (Sec. 2) by smoothed aggregation (Sec. 3, "Coarsening strategies") and
 *     the Galerkin operator A_{i+1} = R_i A_i P_i; then a direct solver for
 *     the coarsest A_L.  Aggregation and prolongation smoothing run on the
 *     host; the Galerkin product runs on the GPU.
 *   - solve (Algorithm 2, one V-cycle as the preconditioning step, Sec. 2 last
 *     paragraph) inside CG or BiCGStab (Sec. 3, "Iterative solvers"), with
 *     damped Jacobi or SPAI-0 smoothing (Sec. 3, "Relaxation methods").  The
 *     whole iteration runs on the GPU; by default it is one CUDA-graph launch
 *     whose loop is a device-side conditional node.
 *
 * Conventions for every entry point:
 *   - Every call returns an amg_status; none aborts or exits.  On failure a
 *     message is available from amg_last_error() (thread-local).
 *   - Matrices are CSR: int32 row pointers (n + 1 entries, row_ptr[0] = 0),
 *     int32 column indices sorted ascending within each row without
 *     duplicates, float64 values.  nnz must be below 2^31.
 *   - "device" pointers are CUDA device (or managed) memory of the device that
 *     was current at amg_setup; "host" pointers are CPU memory.  Ownership of
 *     every buffer passed in stays with the caller; the library copies what it
 *     keeps.
 *   - Work is issued on the CUDA stream given at amg_setup (NULL = legacy
 *     default stream).  Calls that return results to the host synchronize
 *     that stream.
 */
#ifndef AMG_GB300_H
#define AMG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMG_OK = 0,
    AMG_ERR_INVALID_ARG = 1,        /* bad pointer, size, CSR structure or zero diagonal */
    AMG_ERR_OOM = 2,                /* device or host allocation failed */
    AMG_ERR_CUDA = 3,               /* a CUDA runtime call failed */
    AMG_ERR_NOT_CONVERGED = 4,      /* maxiter reached; x, iters, relres still valid */
    AMG_ERR_BREAKDOWN = 5,          /* Krylov breakdown; x, iters, relres still valid */
    AMG_ERR_COARSENING_STALLED = 6, /* aggregation stopped reducing a level too big to solve densely */
    AMG_ERR_TOO_LARGE = 7           /* a size exceeds a documented limit */
} amg_status;

typedef enum { AMG_SMOOTHER_JACOBI = 0, AMG_SMOOTHER_SPAI0 = 1 } amg_smoother;
typedef enum { AMG_SOLVER_CG = 0, AMG_SOLVER_BICGSTAB = 1 } amg_solver;
/* FP64: hierarchy and V-cycle in float64.  FP32: the V-cycle (level
 * matrices, smoother diagonals, level vectors) in float32 with float32
 * accumulation, the outer Krylov vectors, dot products, the fine-level
 * operator and the coarsest solve in float64.  BF16: as FP32, but the
 * V-cycle's matrix values (A_l, the smoother-scaled A_l of the first
 * pre-sweep, P_l and R_l) are stored in bfloat16 (each the float64 value
 * rounded once, to nearest) and widened to float32 as they are used; 6 bytes
 * per nonzero instead of 8.  FP32 and BF16 need npre = npost = 1; BF16 is
 * not available to the batched form and does not use the cooperative tail
 * (use_tail is ignored). */
typedef enum { AMG_PRECISION_FP64 = 0, AMG_PRECISION_FP32 = 1, AMG_PRECISION_BF16 = 2 } amg_precision;

#define AMG_MAX_LEVELS 32

/* Parameters (defaults from amg_params_default in brackets). */
typedef struct {
    double strength_eps;   /* [0.08] strength threshold on the finest level: j is a strong
                              neighbour of i iff a_ij^2 > eps^2 |a_ii a_jj| */
    int strength_halving;  /* [1] eps is halved on every coarser level */
    int smoother;          /* [AMG_SMOOTHER_JACOBI] */
    double jacobi_omega;   /* [0.72] damping of the Jacobi smoother */
    int npre, npost;       /* [1, 1] smoothing sweeps before / after the coarse correction */
    int coarse_enough;     /* [500] a level with at most this many rows is the coarsest */
    int max_levels;        /* [25] at most this many levels (<= AMG_MAX_LEVELS) */
    int max_coarse_dense;  /* [4096] largest coarsest level solved by a dense inverse */
    int solver;            /* [AMG_SOLVER_CG] */
    int precision;         /* [AMG_PRECISION_FP64] */
    int use_graph;         /* [1] run the Krylov loop as one CUDA graph with a device-side
                              while-node; 0 = host-driven launches (same kernels) */
    int use_stream;        /* [1] sparse products stream the matrix through shared memory with
                              bulk asynchronous copies (persistent kernels); 0 = row-chunk
                              kernels with plain loads.  Results agree to rounding. */
    int use_pdl;           /* [0] let consecutive sparse-product kernels overlap through
                              programmatic dependent launch (process-wide setting, applied
                              at each call that launches work).  Off by default: measured
                              slower in the solve's CUDA graph (150^3 FP64 8.72 against
                              8.62 ms, 200^3 variable coefficients 464 against 447 ms).
                              Products of matrices below 2^21 nonzeros (coarse levels)
                              use it either way. */
    int use_tail;          /* [0] run the small coarse levels (below about 4 million nonzeros,
                              finest level excluded) as one cooperative launch with grid-wide
                              barriers; applies when npre = npost = 1.  Off by default: inside
                              the solve's CUDA graph the separate launches were faster. */
    int device_setup;      /* [1] build the hierarchy on the GPU: strength of connection,
                              aggregation, smoothed prolongation, R = P^T and the Galerkin
                              product run as kernels and the level matrices stay on the
                              device; 0 = the graph steps on host threads (the Galerkin
                              product stays on the GPU).  Both give the same hierarchy, bit
                              for bit. */
    int fused_restriction; /* [1] form the fused restriction operator M = R - R A D on the
                              levels where one product with it moves fewer bytes than the
                              pre-sweep, residual and restriction (amg_fused_restriction_nnz);
                              it costs a sparse product per level at set-up and pays off over
                              a few solves, so callers that solve once per hierarchy may turn
                              it off.  Results agree to rounding either way. */
} amg_params;

/* A CSR matrix as passed in by the caller (see the conventions above). */
typedef struct {
    int64_t n;               /* rows = columns */
    int64_t nnz;             /* must equal row_ptr[n] */
    const int32_t *row_ptr;  /* n + 1 */
    const int32_t *col;      /* nnz */
    const double *val;       /* nnz */
    int on_device;           /* 0: the three arrays are host memory, 1: device memory */
} amg_csr;

typedef struct amg_handle amg_handle;

/* Fill *p with the defaults listed above.  Error: INVALID_ARG if p is NULL. */
amg_status amg_params_default(amg_params *p);

/* Build the hierarchy of A (Algorithm 1) and keep it resident on the device.
 * A is deep-copied; the caller may free it after the call.  prm may be NULL
 * (defaults).  stream is a cudaStream_t (may be NULL) used by every later call
 * on the handle.  Errors: INVALID_ARG (n < 1, broken CSR, zero or missing
 * diagonal), COARSENING_STALLED, TOO_LARGE (coarsest level above
 * max_coarse_dense, a Galerkin row wider than the GPU product supports),
 * OOM, CUDA.  On error *out is NULL. */
amg_status amg_setup(const amg_csr *A, const amg_params *prm, void *stream, amg_handle **out);

/* Solve A x = f (Krylov method of the parameters, one V-cycle per
 * preconditioner application).  f: device, n doubles.  x: device, n doubles,
 * initial guess on entry, solution on return.  Stops when the relative
 * recurrence residual ||r||/||f|| <= rtol or after maxiter iterations
 * (iteration = one product with A inside the loop for CG; one pass of the
 * loop body, including a final half step, for BiCGStab); then forms the true
 * residual and, if it misses rtol while iterations remain, restarts from it.
 * *iters (may be NULL): iterations done.  *relres (may be NULL): true relative
 * residual ||f - A x||_2 / ||f||_2 in float64.  If ||f|| = 0: x = 0,
 * iters = 0, relres = 0.  Returns NOT_CONVERGED or BREAKDOWN with valid x,
 * iters and relres; INVALID_ARG if f or the initial guess holds non-finite
 * values (nothing is iterated).  Synchronizes the handle's stream. */
amg_status amg_solve(amg_handle *h, const double *f, double *x, double rtol, int maxiter,
                     int *iters, double *relres);

/* amg_solve with host buffers: f_host (n doubles) is copied to the device,
 * x_host (n doubles) is the initial guess on entry and the solution on
 * return.  The copies are part of the call (pinned host memory makes them
 * faster).  Same results and errors as amg_solve. */
amg_status amg_solve_host(amg_handle *h, const double *f_host, double *x_host, double rtol,
                          int maxiter, int *iters, double *relres);

/* Release the handle and all its device memory.  NULL is accepted. */
amg_status amg_free(amg_handle *h);

/* Message of the last failing call on this thread ("" if none). */
const char *amg_last_error(void);

/* Hierarchy sizes.  levels: number of levels L.  rows, nnz_a: arrays of at
 * least AMG_MAX_LEVELS entries, rows and nnz of A_l; nnz_p: nnz of P_l (0 on
 * the coarsest level).  Any output may be NULL. */
amg_status amg_hierarchy_info(const amg_handle *h, int *levels, int64_t *rows, int64_t *nnz_a,
                              int64_t *nnz_p);

/* Algorithmic bytes of one Krylov iteration on this hierarchy, the roofline
 * numerator of the solve (Sec. 3: the solve phase is sparse products and
 * vector updates, bound by memory bandwidth).  Model: every array a kernel
 * reads or writes counts once per kernel and the gathered vector once;
 * 12 bytes per float64 nonzero (8 value + 4 column; 8 for float32 values,
 * 6 for bfloat16), 4 per row pointer, 8 (4) per float64 (float32) vector
 * entry.  Per V-cycle level: pre-sweep with residual, restriction,
 * prolongation with correction, post-sweep; the dense coarsest solve reads
 * its inverse.  CG adds q = A p with p.q (12 Z0 + 20 n0) and the x, r, p
 * updates (64 n0: r -= alpha q with r.r; x += alpha p with p = z + beta p);
 * BiCGStab two V-cycles, two products and 136 n0. */
amg_status amg_hierarchy_bytes(const amg_handle *h, double *bytes_per_iteration);

/* Copy level matrix `which` (0 = A_l, 1 = P_l, 2 = R_l, 3 = M_l) of level l
 * to host arrays sized from amg_hierarchy_info (amg_fused_restriction_nnz
 * for M_l): row_ptr (rows + 1), col and val (nnz).  P, R and M do not exist
 * on the coarsest level, M only where the level uses it (INVALID_ARG). */
amg_status amg_get_level_matrix(const amg_handle *h, int level, int which, int32_t *row_ptr,
                                int32_t *col, double *val);

/* Nonzeros of the fused restriction operator of level l, 0 if the level does
 * not use one (Algorithm 2's pre-smoothing from a zero guess, residual and
 * restriction, composed: with one pre-sweep x = d f, the restricted residual
 * is R (f - A D f) = M f, M = R - R A D, D = diag(d).  The set-up forms M
 * where one product with it moves fewer bytes than the three steps, and the
 * V-cycle then computes f_{l+1} = M f going down and x = d f + P x_{l+1}
 * coming up.  With npre = 1 and use_tail = 0; the float32 V-cycle uses it on
 * levels >= 1 only, the bfloat16-stored one not at all.) */
amg_status amg_fused_restriction_nnz(const amg_handle *h, int level, int64_t *nnz);

/* Aggregate id of every row of level l (host array of rows[l] entries);
 * INVALID_ARG on the coarsest level. */
amg_status amg_get_aggregates(const amg_handle *h, int level, int32_t *agg);

/* Smoother diagonal d_l of level l (host array of rows[l] doubles):
 * Jacobi d_i = omega / a_ii, SPAI-0 d_i = a_ii / sum_j a_ij^2. */
amg_status amg_get_smoother_diag(const amg_handle *h, int level, double *d);

/* One V-cycle (Algorithm 2 body, zero initial guess on every level):
 * z = M r.  r, z: device, n doubles, distinct buffers. */
amg_status amg_apply_precond(amg_handle *h, const double *r, double *z);

/* y = M x with the resident level matrix `which` (0 = A_l, 1 = P_l, 2 = R_l)
 * using the same SpMV kernel and schedule as the solve.  x: device, columns
 * of that matrix; y: device, its rows. */
amg_status amg_level_spmv(amg_handle *h, int level, int which, const double *x, double *y);

/* Outer Krylov product of step (a1): y = A x and dot = x . y for a CSR matrix
 * already on the device (A->on_device must be 1), on `stream`.  x, y: device,
 * n doubles each, distinct.  dot: device, one double.  Scratch (the row-block
 * schedule and per-block partial sums) is allocated with cudaMallocAsync on
 * the stream and freed before returning.  The dot is summed in a fixed order
 * (deterministic).  Errors: INVALID_ARG, OOM, CUDA. */
amg_status amg_spmv_dot(const amg_csr *A, const double *x, double *y, double *dot, void *stream);

/* ------------------------------------------------------------------
 * Batched form: many independent systems, each with its own hierarchy,
 * solved by one persistent launch.  A CTA takes the next system from a
 * device work queue and runs its whole preconditioned CG (the same
 * recurrences, stopping test and restart rule as amg_solve; Algorithm 2 as
 * the preconditioner) with block-level synchronisation.  The V-cycle runs in
 * the precision of the parameters (AMG_PRECISION_FP32: float32 V-cycle under
 * float64 CG).  Supports CG with npre = npost = 1. */
typedef struct amg_batch amg_batch;

/* Set up nsys systems (Algorithm 1 for each; the per-system host work runs on
 * a thread pool, and each level's Galerkin products of all systems run as one
 * GPU product over their block-diagonal concatenation, which gives every
 * system exactly its own hierarchy).  systems: nsys CSR matrices (host or
 * device, each deep-copied).  Errors as amg_setup, for any system. */
amg_status amg_batch_setup(int nsys, const amg_csr *systems, const amg_params *prm, void *stream,
                           amg_batch **out);

/* Solve all systems.  f, x: device, the systems' vectors concatenated in
 * order (offsets from amg_batch_info); x holds the initial guesses and
 * receives the solutions.  iters, relres, status: host arrays of nsys entries
 * (each may be NULL): per-system iterations, true relative residual and
 * status.  Returns the worst status over the systems (OK if all converged).
 * Synchronizes the batch's stream. */
amg_status amg_batch_solve(amg_batch *b, const double *f, double *x, double rtol, int maxiter,
                           int *iters, double *relres, int *status);

/* Autotune the schedule of amg_batch_solve: times candidate launch shapes
 * (threads per CTA x CTAs per SM) and queue orders (largest system first, or
 * input order) on these f and x, keeps the fastest for later solves and
 * reports it (threads, ctas_per_sm may be NULL).  x is left solved. */
amg_status amg_batch_tune(amg_batch *b, const double *f, double *x, double rtol, int maxiter,
                          int *threads, int *ctas_per_sm);

/* total_rows: sum of the systems' sizes; row_off: nsys + 1 offsets of the
 * systems in f and x; levels: nsys level counts.  Outputs may be NULL. */
amg_status amg_batch_info(const amg_batch *b, int64_t *total_rows, int64_t *row_off, int *levels);

/* Algorithmic bytes of one CG iteration of each system (nsys doubles), by
 * the model of amg_hierarchy_bytes, for the batch's precision, except that
 * the batched CG updates x together with r (72 n0 of Krylov updates). */
amg_status amg_batch_bytes(const amg_batch *b, double *bytes_per_iteration);

/* Release the batch and its device memory.  NULL is accepted. */
amg_status amg_batch_free(amg_batch *b);

/* amg_spmv_dot without allocating: the same product, dot and checks, for
 * callers that cannot allocate device memory while they run (a
 * latency-critical loop that cannot afford the allocator's locks and possible
 * device synchronisation, a process whose device memory is reserved up front
 * by another allocator, or rules that forbid dynamic allocation after
 * initialisation).  The paper has no counterpart; this is an interface
 * convenience.  Scratch lives in a static device array of the library, about
 * 1 MiB, that every GPU loading the library keeps until the process exits;
 * the call makes no cudaMalloc, cudaFree or other allocating call.  Limit:
 * the matrix may span at most 65,536 row blocks (n up to 16,777,216 rows when
 * rows average at most 8 nonzeros; fewer rows for longer rows); above that
 * the call returns AMG_ERR_TOO_LARGE.  The first call on a device looks up
 * the array's device address with cudaGetSymbolAddress; make that first call
 * before any stream capture, since the look-up is a runtime call outside any
 * stream.  Every call then waits on its stream twice, to read back the checks
 * of the row pointers and of the column indices.  All calls in the process
 * share the one array, and it keeps the
 * previous call's contents (the call clears what must start at zero): calls
 * that overlap on the GPU race and must be ordered by the caller.  Results
 * are identical to amg_spmv_dot's.  Errors: INVALID_ARG, TOO_LARGE, CUDA. */
amg_status amg_spmv_dot_noalloc(const amg_csr *A, const double *x, double *y, double *dot,
                                void *stream);

/* Solve server with continuous batching.  The set-up depends only on the
 * matrix, so one hierarchy serves any number of right-hand sides (Sec. 3,
 * design principles); the server keeps hierarchies resident on the device
 * under caller-chosen keys and serves a stream of requests.  Each request is
 * either a new matrix with a right-hand side (its hierarchy is built, used
 * and, for a key >= 0, kept) or the key of a resident hierarchy with a new
 * right-hand side.  Requests wait in a FIFO queue; each of `slots` worker
 * threads, with its own CUDA stream, admits the first queued request (looking
 * up to 16 entries ahead) that it can run: a resident key whose hierarchy is
 * idle, or a new matrix whose estimated device memory fits the HBM budget
 * after evicting idle resident hierarchies, least recently used first.  A new
 * matrix larger than the whole budget runs alone.  Admitted requests run
 * concurrently, so their kernels overlap on the GPU.  A set-up that runs out
 * of device memory is retried once after evicting every idle hierarchy.
 * Every solve is deterministic, so a request's result does not depend on
 * what else runs.
 * Thread-safe: any thread may submit and wait. */
typedef struct amg_server amg_server;

typedef struct {
    int slots;          /* concurrent requests (worker threads); <= 0: 4, capped at 64 */
    int reserved0;
    int64_t hbm_budget; /* device bytes for resident and in-flight hierarchies;
                           <= 0: 80% of the free device memory at creation.
                           A new matrix is charged 72 bytes per nonzero + 64
                           bytes per row + 8 MiB while its hierarchy is built
                           and solved, then the hierarchy's own device bytes
                           while it stays resident. */
    int64_t reserved[4];
} amg_server_params;

/* Start a server on the current device.  prm: the set-up and solver
 * parameters of requests that give none (NULL: amg_params_default).
 * Errors: INVALID_ARG, CUDA. */
amg_status amg_server_create(const amg_server_params *sp, const amg_params *prm, amg_server **out);

/* Queue a request and return at once with its id in *id.  key: >= 0 names a
 * hierarchy kept resident for later requests, < 0 builds a throw-away one.
 * A: the matrix in host memory (deep-copied), or NULL to reuse the resident
 * hierarchy of key (the request then fails with INVALID_ARG when it comes up
 * if the key is not resident).  A key names one matrix: a request that gives
 * a matrix for a key already resident, or being built, reuses that key's
 * hierarchy.  f_host: n doubles (copied).  prm: set-up and solver parameters
 * (copied; NULL: the server's) of a hierarchy this request builds; a reused
 * hierarchy keeps the parameters it was built with, solver included.  The
 * initial guess is zero.  Invalid parameters fail the request when it comes
 * up.  Errors: INVALID_ARG. */
amg_status amg_server_submit(amg_server *s, int64_t key, const amg_csr *A, const double *f_host, int64_t n,
                             const amg_params *prm, double rtol, int maxiter, int64_t *id);

/* Block until request id has finished; copy its solution to x_host (n
 * doubles, may be NULL) and report its iterations, true relative residual,
 * latency (submit to finish, seconds) and queueing time (submit to
 * admission); outputs may be NULL.  Returns the request's status (as
 * amg_setup / amg_solve).  The request is forgotten afterwards: wait once per
 * id.  An unknown id gives INVALID_ARG. */
amg_status amg_server_wait(amg_server *s, int64_t id, double *x_host, int *iters, double *relres,
                           double *latency_s, double *queue_s);

/* Counters: requests finished, resident hierarchies and their device bytes,
 * the peak of the bytes charged against the budget, and evictions.  Outputs
 * may be NULL. */
amg_status amg_server_stats(amg_server *s, int64_t *completed, int *resident_count, int64_t *resident_bytes,
                            int64_t *peak_bytes, int64_t *evictions);

/* Algorithmic bytes moved by the solves the server finished so far: for
 * each solve, amg_hierarchy_bytes of its hierarchy times its iterations. */
amg_status amg_server_solve_bytes(amg_server *s, double *bytes);

/* Finish every queued request, stop the workers and free the resident
 * hierarchies.  Results not yet collected are dropped.  NULL is accepted. */
amg_status amg_server_destroy(amg_server *s);

/* Kernel classes reported by amg_solve_profile. */
typedef enum {
    AMG_KC_SPMV_DOT = 0,      /* q = A p with p.q (a1) */
    AMG_KC_KRYLOV_UPDATE,     /* x, r updates with ||r||^2; p update (a2) */
    AMG_KC_PRESMOOTH_L0,      /* finest level: x = d f, t = f - A x (a3 + a4 residual) */
    AMG_KC_RESTRICT_L0,       /* finest level: f_1 = R t (a4 restriction) */
    AMG_KC_PROLONG_L0,        /* finest level: x += P x_1 (a6) */
    AMG_KC_POSTSMOOTH_L0,     /* finest level: z = x + d (f - A x) (a7) */
    AMG_KC_VCYCLE_COARSER,    /* the same four kernels on levels >= 1 */
    AMG_KC_COARSE_SOLVE,      /* dense coarsest solve (a5) */
    AMG_KC_OTHER,             /* residual, norms and remaining small kernels */
    AMG_KC_COUNT
} amg_kernel_class;

/* Same computation as amg_solve, but every kernel is launched from the host
 * (no graph) between two CUDA events on the handle's stream; *ms receives
 * the summed event time per kernel class (AMG_KC_COUNT doubles) and
 * *launches the number of launches per class (AMG_KC_COUNT ints).  Used to
 * attribute solve time to kernels; slower overall than amg_solve because of
 * the per-launch events. */
amg_status amg_solve_profile(amg_handle *h, const double *f, double *x, double rtol, int maxiter,
                             int *iters, double *relres, double *ms, int *launches);

/* Number of kernel launches the last amg_solve on this handle issued (all
 * loop iterations included). */
amg_status amg_last_launch_count(const amg_handle *h, int64_t *launches);

/* How the last amg_solve / amg_solve_host on this handle ran (Sec. 3: the
 * solve phase; no counterpart for the launch mode itself).  A solve is one or
 * more attempts: the first run of the Krylov loop, plus one per restart from
 * the true residual.  *graph_attempts (may be NULL) receives the number of
 * attempts launched as one CUDA graph with a device-side loop;
 * *host_attempts (may be NULL) the number whose kernels were launched one by
 * one from the host, because use_graph = 0 or because the graph could not be
 * built (the handle then keeps to host launches).  Both are 0 before the
 * first solve. */
amg_status amg_last_solve_mode(const amg_handle *h, int *graph_attempts, int *host_attempts);

/* Check of failure detection (no counterpart in the paper): on the current
 * device, one block of the streaming engine's pipeline waits on a barrier
 * that nothing completes, with the engine's bounded wait limited to 2^12 polls
 * (at most about 0.4 s).  The wait gives up, records the timeout in the
 * device error word and returns, as a streaming kernel whose copies never
 * arrived would.  The call reads and clears that word and returns
 * AMG_ERR_CUDA with the message a solve gives for it; *seconds (may be NULL)
 * receives the kernel's duration.  The device stays usable.  The error word
 * is shared by all handles of the process: do not run this while solves are
 * in flight. */
amg_status amg_check_wait_limit(double *seconds);

#ifdef __cplusplus
}
#endif
#endif /* AMG_GB300_H */
