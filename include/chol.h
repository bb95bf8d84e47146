/*
 * chol.h -- C ABI of the GB300 tiled Cholesky library (libchol.so).
 *
 * The library factors a symmetric positive-definite matrix A = L L^T with the
 * tiled right-looking algorithm of the paper (Section 3.1, Fig. 1): for each
 * block column J, POTRF on the diagonal tile A_JJ, TRSM on the tiles A_IJ
 * below it (A_IJ <- A_IJ A_JJ^{-T}), then SYRK (A_II <- A_II - A_IJ A_IJ^T)
 * and GEMM (A_IK <- A_IK - A_IJ A_KJ^T, J < K < I) on the trailing matrix.
 * Two GPU schedules answer the paper's fork-join versus asynchronous-task
 * question (Section 3.2): per-step kernel launches separated by stream order
 * (fork-join, collapsed or naive) and one persistent dataflow kernel driven by
 * per-task dependency counters (no barrier between steps).
 *
 * Conventions for every entry point unless stated otherwise:
 *   - matrices are COLUMN-major with a leading dimension (LAPACK, uplo='L');
 *     element (i, j) of A is A[j * lda + i];
 *   - matrix pointers are DEVICE pointers (cudaMalloc / torch CUDA memory),
 *     owned by the caller; no call frees or keeps caller memory past return
 *     except where a handle's documentation says so;
 *   - only the lower triangle including the diagonal is read or written; the
 *     strict upper triangle is never accessed (Section 3.1: only the diagonal
 *     and the strictly lower part are stored);
 *   - calls are ordered on opts->stream (NULL = the legacy default stream) and
 *     return after the work has completed: they synchronize on that stream to
 *     read back the status; the library allocates its workspace with the
 *     stream-ordered allocator and caches it between calls;
 *   - the return value is a chol_status (0 = success, < 0 = error); factor
 *     calls report a matrix that is not positive definite through *info, the
 *     LAPACK dpotrf way: info = k > 0 is the 1-based order of the first
 *     leading minor that is not positive definite (its pivot was <= 0 or
 *     NaN); the contents of A beyond column k-1 are then unspecified;
 *   - chol_last_error() returns a description of the last failure on the
 *     calling thread.
 * The library is not thread-safe except for the chol_server_* calls, which
 * may be called from any thread.
 */
#ifndef CHOL_H
#define CHOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum {
    CHOL_OK = 0,
    CHOL_ERR_ARG = -1,           /* an argument is out of range / NULL */
    CHOL_ERR_NOT_SPD = -2,       /* returned by chol_factor() when info > 0 */
    CHOL_ERR_NOMEM = -3,         /* device allocation failed or budget exceeded */
    CHOL_ERR_CUDA = -4,          /* a CUDA runtime call failed */
    CHOL_ERR_TIMEOUT = -5,       /* a bounded device-side wait expired */
    CHOL_ERR_NOT_CONVERGED = -6, /* iterative refinement missed its tolerance */
    CHOL_ERR_BUSY = -7,          /* server request still pending */
    CHOL_ERR_HANDLE = -8,        /* unknown or freed handle / ticket / factor id */
    CHOL_ERR_UNSUPPORTED = -9    /* option combination not supported */
} chol_status;

/* Precision of the trailing SYRK/GEMM update (Section 3.1 tile kernels).
 * CHOL_FP64: every tile kernel in binary64 (DFMA).  The others keep the tiles
 * in binary32, factor each diagonal tile in binary64 and run SYRK/GEMM on the
 * tcgen05 tensor cores with binary32 accumulation in tensor memory:
 *   CHOL_TF32: one TF32 product per update (operands rounded to 10 mantissa bits);
 *   CHOL_FP32: three TF32 products (hi*hi + hi*lo + lo*hi), about binary32 accuracy;
 *   CHOL_BF16, CHOL_FP16: operands rounded to bfloat16 / binary16 after a
 *   power-of-two scaling per tile (exact; keeps binary16 in range). */
typedef enum {
    CHOL_FP64 = 0,
    CHOL_FP32 = 1,
    CHOL_TF32 = 2,
    CHOL_BF16 = 3,
    CHOL_FP16 = 4
} chol_precision;

/* Task schedule (Section 3.2). */
typedef enum {
    CHOL_SCHED_AUTO = 0,            /* autotuner choice (or dataflow if untuned) */
    CHOL_SCHED_FORK_JOIN = 1,       /* per step J: POTRF, TRSM grid, collapsed SYRK+GEMM grid */
    CHOL_SCHED_FORK_JOIN_NAIVE = 2, /* as above, update grid over block rows only */
    CHOL_SCHED_DATAFLOW = 3,        /* one persistent kernel, dependency counters */
    CHOL_SCHED_LEFT_LOOKING = 4,    /* the left-looking variant (Section 3.1): per block column K, one
                                       CTA per tile (I, K) applies all its updates J < K, then POTRF,
                                       then the TRSM grid; same per-tile update order, same bits */
    CHOL_SCHED_TOP_LOOKING = 5      /* the top-looking variant (Section 3.1): block row I in one launch,
                                       one CTA per tile (I, K) applying its updates as the row's tiles
                                       to its left become final, then its TRSM (POTRF for K = I);
                                       same per-tile update order, same bits; its waits for the row's
                                       tiles are bounded by opts->timeout_s (CHOL_ERR_TIMEOUT) */
} chol_schedule;

/* opts->flags */
enum {
    CHOL_FLAG_NOOP = 1,          /* replace every tile kernel body by a no-op (Section 4.2 overhead runs) */
    CHOL_FLAG_PRIORITY = 2,      /* dataflow: POTRF, TRSM, SYRK and the GEMMs updating the next 16 panel columns
                                    before the other GEMMs (OpenMP 4.5 priorities analog) */
    CHOL_FLAG_GRAPH = 4,         /* launch-ordered schedules: capture the launches into a CUDA graph and
                                    launch it as one unit (the call then waits for it) */
    CHOL_FLAG_TEST_WITHHOLD = 8, /* test hook: never release the last POTRF (dataflow) or tile
                                    (M-1, 0) (top-looking), so the bounded waits must expire
                                    with CHOL_ERR_TIMEOUT */
    CHOL_FLAG_FP64_TC = 16,      /* FP64: run SYRK/GEMM (and TRSM, as a product with the inverted
                                    diagonal block when it is well conditioned) on the bf16 tensor
                                    cores with binary64 accuracy (exact 8 x 7-bit slicing of
                                    row-scaled values, 36 integer-exact products per 128 x 128
                                    block update); tile orders 128 r (r = 1 .. 16), each task
                                    running its r x r blocks of order 128 in the order the
                                    algorithm gives them at tile order 128, so every tile order
                                    gives the same bits.  This is the DEFAULT engine for n > 1024
                                    when nb is 0 (then 128) or a multiple of 128 up to 2048 */
    CHOL_FLAG_FP64_SIMT = 64,    /* FP64: run every tile kernel on the CUDA cores in binary64 (DFMA),
                                    the default for n <= 1024 or tile orders that are not multiples
                                    of 128 */
    CHOL_FLAG_GMRES_IR = 32      /* chol_mixed_solve: each refinement step solves the correction
                                    equation by GMRES(20) preconditioned with the low-precision
                                    factor (binary64 Krylov vectors) instead of one solve with it;
                                    iters then counts preconditioner applications */
};

/* One trace record per executed task (written when opts->trace != NULL). */
typedef struct {
    int32_t type;      /* 0 POTRF, 1 TRSM, 2 SYRK, 3 GEMM */
    int32_t I, K, J;   /* target tile (I, K) updated at step J */
    int32_t sm;        /* SM that ran it */
    int32_t matrix;    /* batched: matrix index, else 0 */
    uint64_t t_start;  /* %globaltimer, ns */
    uint64_t t_end;
} chol_trace_rec;

typedef struct {
    int32_t schedule;       /* chol_schedule */
    int32_t precision;      /* chol_precision */
    int64_t nb;             /* tile order; 0 = autotuner / default */
    int32_t flags;          /* CHOL_FLAG_* */
    int32_t max_iter;       /* refinement iterations (default 30) */
    double refine_tol;      /* refinement target backward error (default 1e-14) */
    double timeout_s;       /* bound on any device-side wait (default 60 s) */
    void *stream;           /* cudaStream_t; NULL = legacy default stream */
    int32_t num_ctas;       /* dataflow grid size; 0 = default (4 CTAs per SM for the CUDA-core
                               bodies, 1 per SM for the tensor-core body) */
    int32_t tc_min_order;   /* batched plans: matrices of order above this run on tensor-core bodies
                               (0 = 1024, the order above which a single FP64 factorization uses
                               them by default; 2048 keeps every matrix on the CUDA cores) */
    chol_trace_rec *trace;  /* device buffer of trace_capacity records, or NULL */
    int64_t trace_capacity;
} chol_opts;

/* Per-call statistics (optional output of the _ex calls). */
typedef struct {
    int64_t tasks[4];       /* POTRF, TRSM, SYRK, GEMM tasks executed on the device */
    int64_t nb;             /* tile order used */
    int32_t schedule;       /* schedule used */
    int32_t launches;       /* kernel launches issued for the factorization */
    int64_t trace_records;  /* records the device wanted to write (may exceed capacity) */
    double device_ms;       /* device time of the factorization kernels (CUDA events) */
} chol_stats;

/* Fill *opts with the defaults listed above. */
void chol_opts_init(chol_opts *opts);

/* Description of the last failure on this thread ("" if none). */
const char *chol_last_error(void);

/* Library version string. */
const char *chol_version(void);

/* ------------------------------------------------------------ factorization */

/* A = L L^T in place, FP64, tile order nb, dataflow schedule, default stream.
 * Section 3.1 / Fig. 1.  A: n x n device matrix, lda >= max(1, n); nb >= 1
 * (nb > n factors one padded tile).  Returns CHOL_OK, a negative chol_status,
 * or CHOL_ERR_NOT_SPD with the failing column recorded in chol_last_info(). */
int chol_factor(int64_t n, int64_t nb, double *A, int64_t lda);

/* info of the last chol_factor() call on this thread (0 if it succeeded). */
int64_t chol_last_info(void);

/* Full-control FP64 factorization.  opts may be NULL (defaults); info must
 * not be NULL; stats may be NULL.  opts->precision must be CHOL_FP64 (use
 * chol_mixed_factor for the others). */
int chol_factor_ex(int64_t n, double *A, int64_t lda, const chol_opts *opts,
                   int64_t *info, chol_stats *stats);

/* As chol_factor_ex, but A is a HOST buffer (end-to-end path; page-locked
 * memory copies fastest): the library copies the lower triangle to a device
 * buffer of n x n elements, factors it and copies the lower triangle back.
 * Each copy moves, per block of columns starting at column j0, rows j0 .. n-1
 * of those columns: the lower triangle plus the upper part of each block's
 * diagonal square, which is written back unchanged.  With the dataflow
 * schedule on the tensor-core engine the copy back overlaps the
 * factorization: the kernel writes each tile of the factor as soon as it is
 * final and flags each complete block column (of order nb) in page-locked
 * memory; the calling thread polls the flags and queues that column's copy on
 * a copy stream of its own, and copies whatever is left when the schedule has
 * ended.  The call returns after all copies. */
int chol_factor_host(int64_t n, double *A_host, int64_t lda, const chol_opts *opts,
                     int64_t *info, chol_stats *stats);

/* ------------------------------------------------------------------- solve */

/* B <- A^{-1} B given L from chol_factor (forward substitution L Y = B, then
 * backward L^T X = Y), FP64.  L: n x n lower, ldl = n; B: n x nrhs, ldb = n. */
int chol_solve(int64_t n, int64_t nrhs, const double *L, double *B);

int chol_solve_ex(int64_t n, int64_t nrhs, const double *L, int64_t ldl,
                  double *B, int64_t ldb, const chol_opts *opts);

/* The same FP64 solve as chol_solve_ex, for callers that cannot allocate
 * device memory: an application whose own memory manager has reserved the
 * GPU's memory, or a latency-critical loop that must not pay the
 * device-wide synchronization cudaMalloc / cudaFree can cause.  (The paper
 * has no counterpart; this is an interface of this library only.)
 *   - allocates nothing: its scratch is a fixed 4 MiB array in device memory
 *     that every GPU loading the library holds until the process exits;
 *   - the first call on a device looks up that array's device address (once
 *     per device, with that device current); make the first call before any
 *     stream capture;
 *   - sizes whose scratch exceeds 4 MiB (2 * ceil(n/64) * ceil(nrhs/16) flags
 *     of 4 bytes plus a 32 KiB control block) return CHOL_ERR_ARG with a
 *     message; use chol_solve_ex for those;
 *   - all calls share the one array and clear what they use at the start, so
 *     calls that overlap on the GPU (different streams, threads or devices'
 *     streams on the same device) race and must be serialized by the caller;
 *   - L: n x n lower factor (ldl >= n), B: n x nrhs (ldb >= n), device,
 *     column-major; B is overwritten with the solution; stream: cudaStream_t
 *     (NULL = legacy default stream); returns after the solve completed. */
int chol_solve_noalloc(int64_t n, int64_t nrhs, const double *L, int64_t ldl,
                       double *B, int64_t ldb, void *stream);

/* --------------------------------------------- mixed precision + refinement */

typedef struct chol_factor_s *chol_factor_h;

/* Factor A with the trailing update in opts->precision (FP32/TF32/BF16/FP16,
 * see chol_precision) and keep the factor in a handle.  A is READ ONLY and is
 * REFERENCED by the handle (for the FP64 residuals of refinement): the caller
 * keeps it alive and unchanged until chol_factor_free.  *info as for
 * chol_factor_ex.  opts->nb must be a multiple of 128 (0 = default 256). */
int chol_mixed_factor(int64_t n, const double *A, int64_t lda, const chol_opts *opts,
                      chol_factor_h *out, int64_t *info);

/* Solve A X = B with the handle's factor and FP64 iterative refinement: the
 * residual R = B - A X and the update X += D are FP64, the correction solve
 * L^ L^T D = R uses the low-precision factor.  Stops when the normwise
 * backward error max_j ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf)
 * is <= opts->refine_tol or after opts->max_iter iterations (options of the
 * factor call).  B: n x nrhs (read only), X: n x nrhs output, both device.
 * iters / berr (host, may be NULL) receive the iterations used and the final
 * backward error (NaN if an iterate was not finite).  Returns
 * CHOL_ERR_NOT_CONVERGED if the tolerance was missed (X then holds the last
 * iterate) and CHOL_ERR_NOT_SPD, without solving, if the handle's
 * factorization broke down (info > 0).
 * For n >= 1024 the residual runs on the tensor cores with binary64 accuracy
 * (exact bf16 slicing): the first solve on a handle builds the slices of A,
 * about 16 n^2 bytes of device memory (17 GB at n = 32768), which the handle
 * keeps until chol_factor_free; when that memory cannot be allocated the
 * residual runs on the FP64 pipe instead.  With CHOL_FLAG_GMRES_IR (a flag
 * of the factor call) each refinement step is a GMRES solve preconditioned
 * with the factor and *iters counts preconditioner applications. */
int chol_mixed_solve(chol_factor_h h, int64_t nrhs, const double *B, int64_t ldb,
                     double *X, int64_t ldx, int32_t *iters, double *berr);

/* Copy the handle's low-precision factor, widened to FP64, into the lower
 * triangle of L (device, column-major, ldl >= n). */
int chol_mixed_get_factor(chol_factor_h h, double *L, int64_t ldl);

void chol_factor_free(chol_factor_h h);

/* Statistics (tasks executed, tile order, schedule, device time of the
 * schedule kernels) of the last chol_mixed_factor call on this thread. */
int chol_mixed_last_stats(chol_stats *stats);

/* ----------------------------------------------------------------- batched */

typedef struct chol_batch_s *chol_batch_h;

/* Plan a batched factor + solve of `batch` independent SPD systems of orders
 * n[i] (host array, 1 <= n[i] <= 2048, batch <= 65535), 1 right-hand side
 * each, in one persistent kernel launch
 * that is captured once into a CUDA graph and replayed by chol_batch_run.
 * precision: CHOL_FP64 or CHOL_FP32 (binary32 tiles and results).  The tile
 * order of each matrix comes from the autotuner's table for its n (opts->nb
 * > 0 forces one nb for all).  The matrices of order above 1024 (or above
 * opts->tc_min_order) run on tensor-core bodies: tiles of order 128, all of
 * them in one persistent kernel of their own.  In FP64 plans that is the
 * exact-slice engine, each matrix with the bits of a single factorization of
 * it with CHOL_FLAG_FP64_TC and nb = 128 (the default single factorization
 * above order 1024); CHOL_FLAG_FP64_SIMT in opts->flags keeps every matrix on
 * the CUDA-core bodies.  In FP32 plans it is the mixed-precision engine's FP32
 * bodies with the diagonal tiles factored in binary32 (binary32 TRSM,
 * SYRK/GEMM as three TF32 products with binary32 accumulation), solved in
 * binary32; a matrix gets the same bits alone and in any batch.  The other
 * matrices run in true binary32 (FP32) or binary64 arithmetic on the CUDA
 * cores with opts->nb. */
int chol_batch_plan(int32_t batch, const int64_t *n, const chol_opts *opts, chol_batch_h *out);

/* Factor every A[i] in place (lower triangle <- L_i) and overwrite B[i] with
 * the solution of A_i x = b_i.  A, B: host arrays of `batch` device pointers
 * to FP64 column-major data (lda[i] >= n[i]; B[i] holds n[i] values).  For
 * CHOL_FP32 plans the data are still FP64 in memory and are converted on the
 * device.  info: host array of `batch` results (0 or the failing column). */
int chol_batch_run(chol_batch_h plan, double *const *A, const int64_t *lda,
                   double *const *B, int64_t *info);

/* Statistics of the last run: tasks executed (summed over both parts) and the
 * device time of the whole graph (repack, the persistent factor+solve
 * kernels, unpack). */
int chol_batch_stats(chol_batch_h plan, chol_stats *stats);

void chol_batch_free(chol_batch_h plan);

/* --------------------------------------------------------------- autotuner */

/* Measure candidate tile orders and schedules for order n at `precision` on
 * the current device and return the fastest in *opts_out (nb, schedule).
 * Results are cached per (device name, n bucket, precision) in memory and,
 * if cache_path is not NULL, in that JSON file (read first, written after).
 * budget_s bounds the measuring time (0 = default 5 s). */
int chol_autotune(int64_t n, int32_t precision, const char *cache_path, double budget_s,
                  chol_opts *opts_out);

/* The tile order the library picks for order n at `precision` without
 * measuring (deterministic table; used by the batched and served paths so a
 * matrix gets the same nb alone and in a mix). */
int64_t chol_default_nb(int64_t n, int32_t precision);

/* ----------------------------------------------------------------- serving */

typedef struct chol_server_s *chol_server_h;

typedef struct {
    int64_t n;               /* matrix order */
    const double *A;         /* device, column-major, lda; NULL = reuse factor_id */
    int64_t lda;
    uint64_t factor_id;      /* key of a resident factor (0 = do not keep the factor) */
    const double *B;         /* device, n x nrhs, ldb (read only) */
    int64_t ldb;
    double *X;               /* device, n x nrhs output, ldx */
    int64_t ldx;
    int64_t nrhs;
    int32_t precision;       /* CHOL_FP64, or a mixed precision (refined to opts refine_tol) */
    int32_t reserved;
} chol_request;

typedef struct {
    int32_t status;          /* chol_status of the request */
    int32_t iters;           /* refinement iterations (mixed) */
    int64_t info;            /* factor info */
    double berr;             /* final backward error (mixed) or -1 */
    double latency_ms;       /* submit -> completion */
    double queue_ms;         /* submit -> admission */
    int32_t reused_factor;   /* 1 if a resident factor served the request */
    int32_t slot;            /* device slot (stream) that ran it */
} chol_result;

typedef struct {
    int64_t completed, failed, rejected;
    int64_t resident_factors;
    size_t bytes_in_use, budget;
    double p50_ms, p99_ms, mean_ms;
    double solves_per_s;     /* completed requests / (last completion - first submit) */
    double elapsed_s;
} chol_server_stats_t;

/* Start a server with `slots` concurrent device streams (0 = 4) and a device
 * memory budget in bytes for workspaces plus resident factors.  Requests are
 * admitted in arrival order as slots and budget free up (continuous batching)
 * and their kernels overlap on the device.  The caller's A, B, X buffers must
 * stay valid until the request completes. */
int chol_server_create(size_t mem_budget_bytes, int32_t slots, const chol_opts *opts,
                       chol_server_h *out);
int chol_server_submit(chol_server_h s, const chol_request *req, uint64_t *ticket);
/* CHOL_ERR_BUSY while pending; the result is returned once and then forgotten. */
int chol_server_poll(chol_server_h s, uint64_t ticket, chol_result *res);
int chol_server_wait(chol_server_h s, uint64_t ticket, chol_result *res, double timeout_s);
int chol_server_release(chol_server_h s, uint64_t factor_id);
int chol_server_stats(chol_server_h s, chol_server_stats_t *st);
void chol_server_destroy(chol_server_h s);

#ifdef __cplusplus
}
#endif
#endif /* CHOL_H */
