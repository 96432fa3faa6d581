/*
 * rpcg.h -- C ABI of the reproducible Jacobi-preconditioned CG library for
 * one NVIDIA GB300 (sm_103a).
 *
 * The method is the reproducible PCG of Iakymchuk, Barreda, Graillat,
 * Aliaga and Quintana-Orti ("Reproducibility of Parallel Preconditioned
 * Conjugate Gradient in Hybrid Programming Environments"): the PCG loop of
 * Fig. 1 with S8 moved next to S6 (Fig. 2), a Jacobi preconditioner applied
 * as an elementwise multiply by the inverse diagonal (Sec. 3.1, Sec. 4.3),
 * SpMV rows and AXPY updates written with explicit fma (Sec. 4.3), and the
 * three dot products made reproducible either with an ExBLAS-style long
 * accumulator (Sec. 2.1, Sec. 4.1) or with floating-point expansions
 * (Sec. 4.2, Algs. 1-4).
 *
 * Conventions for every entry point:
 *   - All arithmetic is IEEE binary64, round to nearest even.
 *   - "device" pointers are CUDA device (or managed) memory on the current
 *     device; "host" pointers are ordinary host memory.  Vectors are dense,
 *     contiguous, unit stride.  CSR matrices use int32 row pointers
 *     (n + 1 entries, rowptr[0] = 0, non-decreasing) and int32 column
 *     indices, float64 values; columns may be in any order inside a row,
 *     and the SpMV sums each row in storage order.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it.  Entry points that return values
 *     into host memory synchronise that stream before returning.
 *   - Nothing aborts or throws across the ABI.  Every call returns an
 *     rpcg_status; rpcg_last_error() gives a human-readable message for the
 *     last failing call on the calling host thread.
 *   - A matrix handle may be used by one host thread at a time.
 */
#ifndef RPCG_H
#define RPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes.  Non-negative values are solver outcomes, negative values
 * are errors. */
typedef enum {
    RPCG_OK = 0,
    RPCG_NOT_CONVERGED = 1,  /* max_iter reached with relres >= tol */
    RPCG_FPE_INEXACT = 2,    /* fpe variant with fpe_strict = 1: an expansion lost bits (Sec. 4.3, warning) */
    RPCG_ERR_INVALID = -1,   /* bad argument */
    RPCG_ERR_NOT_SPD = -2,   /* missing or non-positive diagonal, <d,w> <= 0, or beta <= 0 with tau > 0 */
    RPCG_ERR_NONFINITE = -3, /* NaN or Inf met in a dot product or the diagonal */
    RPCG_ERR_OOM = -4,       /* device allocation failed, or a budget was exceeded */
    RPCG_ERR_CUDA = -5,      /* a CUDA runtime call failed */
    RPCG_ERR_TIMEOUT = -6    /* a bounded wait ran out (server wait) */
} rpcg_status;

/* Dot-product variants of the solver (Sec. 4). */
typedef enum {
    RPCG_PLAIN = 0,  /* ordinary FP64 dots with a fixed tree reduction (not reproducible across launch shapes) */
    RPCG_EXBLAS = 1, /* exact dot: long accumulator of 64-bit digits, one final rounding (Sec. 4.1) */
    RPCG_FPE = 2     /* floating-point-expansion dot with an exactness flag (Sec. 4.2) */
} rpcg_variant;

typedef struct rpcg_matrix_s *rpcg_matrix_t;
typedef struct rpcg_batch_s *rpcg_batch_t;
typedef struct rpcg_server_s *rpcg_server_t;

/* Solver options.  rpcg_opts_default() fills the defaults. */
typedef struct {
    double tol;         /* stop when RN(sqrt(tau) / ||b||) < tol (default 1e-8) */
    int32_t max_iter;   /* loop bodies at most (default 1000) */
    int32_t fpe_size;   /* terms per expansion p, 1..8 (default 8, Sec. 4.2); 0 = adaptive: start at 3 (Sec. 4.3's
                           size for Poisson) and add a term after every dot that lost bits, up to 8 */
    int32_t fpe_strict; /* fpe variant: 0 = recompute an inexact dot exactly (default), 1 = report RPCG_FPE_INEXACT */
    int32_t block;      /* threads per CTA of the streaming passes: 0 = auto, else 128, 256 or 512 */
    int32_t grid;       /* CTAs of the streaming passes: 0 = auto, else 1 .. 4096 */
    int32_t tile;       /* batched solves: rows per work unit, 0 = autotuned */
    double *history;    /* optional device array of max_iter + 1 doubles: relres at every loop test */
} rpcg_opts;

/* Outcome of a solve. */
typedef struct {
    int32_t iterations;        /* loop bodies executed */
    int32_t status;            /* rpcg_status of this solve */
    double relres;             /* RN(sqrt(tau) / ||b||) at the last loop test */
    double tau;                /* <r, r> at the last loop test */
    int32_t fpe_inexact_count; /* fpe variant: dots whose expansion lost bits */
    int32_t fpe_size_used;     /* fpe variant: expansion size at the end (grows when fpe_size = 0) */
} rpcg_result;

/* Fill `o` with the defaults listed in rpcg_opts. */
void rpcg_opts_default(rpcg_opts *o);

/* Text for a status code (static storage). */
const char *rpcg_status_string(int32_t status);

/* Message of the last failing call on this host thread ("" if none). */
const char *rpcg_last_error(void);

/*
 * rpcg_create -- build a matrix handle from CSR (Sec. 3.1: A is sparse SPD
 * with n rows and nnz nonzeros; the handle also computes the Jacobi
 * preconditioner's inverse diagonal on first use).
 *   A_out     receives the handle.
 *   n, nnz    rows and nonzeros, 0 <= n <= 2^31 - 2^25 (headroom for 32-bit
 *             row indices), 0 <= nnz < 2^31.
 *   rowptr, col, val   CSR arrays (n + 1, nnz, nnz entries).
 *   ptr_kind  0 = the three arrays are host pointers, 1 = device pointers.
 * The handle copies the arrays into device memory it owns (padded for
 * aligned bulk loads) and allocates the Krylov vectors; the caller's arrays
 * may be freed as soon as the call returns.  Row pointers are validated
 * (monotone, in range); column indices are checked to lie in [0, n).
 * Errors: RPCG_ERR_INVALID (bad sizes or CSR), RPCG_ERR_OOM, RPCG_ERR_CUDA.
 */
rpcg_status rpcg_create(rpcg_matrix_t *A_out, int32_t n, int32_t nnz, const int32_t *rowptr, const int32_t *col,
                        const double *val, int32_t ptr_kind, void *stream);

/* Release a handle and all device memory it owns (synchronises its work). */
rpcg_status rpcg_destroy(rpcg_matrix_t A);

/* Rows and nonzeros of a handle. */
rpcg_status rpcg_matrix_info(rpcg_matrix_t A, int32_t *n, int32_t *nnz);

/*
 * rpcg_spmv -- y = A x (S1 of Fig. 1), each row summed left to right in
 * storage order as acc = fma(val_k, x_col_k, acc) from acc = +0 (Sec. 4.3).
 * x, y: device arrays of n doubles (must not overlap).  Asynchronous.
 */
rpcg_status rpcg_spmv(rpcg_matrix_t A, const double *x, double *y, void *stream);

/*
 * rpcg_dot_exact -- out = RN(sum_i a_i * b_i) with the sum taken exactly
 * (Sec. 2.1 and Sec. 4.1: every product is kept exactly in a long
 * accumulator of 64-bit digits and rounded once, to nearest even).
 *   n       0 <= n <= 2^30.
 *   a, b    device arrays of n doubles.
 *   out     device pointer to one double.
 * An exactly zero sum gives +0; a non-zero sum that rounds to zero keeps
 * its sign; |sum| >= 2^1024 (1 - 2^-54) gives +-inf; any NaN or Inf input
 * gives NaN.  The result does not depend on the launch shape, the stream
 * or the order of the elements.  Scratch memory is taken from the
 * stream-ordered pool (cudaMallocAsync).  Asynchronous.
 */
rpcg_status rpcg_dot_exact(int64_t n, const double *a, const double *b, double *out, void *stream);

/*
 * rpcg_dot_exact_noalloc -- the same exact dot as rpcg_dot_exact (same
 * kernel, same result bits), for callers that cannot have the library
 * allocate device memory: e.g. a framework whose own allocator already
 * holds all of the GPU's memory, or a time-critical loop where an
 * allocation and the synchronisation it may cause are not acceptable.  The
 * paper has no counterpart.
 *   n         0 <= n <= 2^30 (larger n returns RPCG_ERR_INVALID).
 *   a, b      device arrays of n doubles; out: device pointer to one double.
 * It allocates nothing: its scratch is one fixed 64 KiB array inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.  The first call in each CUDA context (normally the device's primary
 * context; a context created later, e.g. after cudaDeviceReset, counts as a
 * new one) looks up that array's device address with the context current;
 * make that first call before any stream capture.  All calls on a device
 * share the one array, and each call clears the part that must start at
 * zero: calls that may overlap on the GPU (on different streams without
 * ordering between them) race and give wrong results; serialise them.
 * Asynchronous.
 */
rpcg_status rpcg_dot_exact_noalloc(int64_t n, const double *a, const double *b, double *out, void *stream);

/*
 * rpcg_dot_fpe -- FPE dot of Sec. 4.2: each thread keeps a result expansion
 * and an error expansion of p terms (Alg. 4 with the early exit, fed by
 * Alg. 2's product and error) and merges its two expansions with Alg. 3.
 * The threads' merged expansions are then added exactly: every term goes
 * into a long accumulator of 64-bit digits (the exact dot's), which is
 * rounded once to nearest even.  This replaces the paper's fpesum merge
 * across threads (Listing 2) and its NearSum; the merge itself loses nothing.
 *   p       terms per expansion, 1..8.
 *   out     device pointer to one double: the correctly rounded sum of the
 *           threads' terms (NaN if a term or an input is not finite).
 *   exact   device pointer to one int32: 1 if no thread's expansion lost
 *           bits (then *out equals rpcg_dot_exact's value), 0 if a thread's
 *           Accumulate carried a value out of its last term, a product of
 *           non-zero operands fell below 2^-969 (twoprod's error may not be
 *           representable), or a term or an input was not finite.  Only the
 *           threads' own losses count, so the flag and a lossy *out depend
 *           on how the elements are spread over threads; when one thread
 *           holds every product they equal the paper's algorithm exactly.
 * Asynchronous.
 */
rpcg_status rpcg_dot_fpe(int64_t n, const double *a, const double *b, int32_t p, double *out, int32_t *exact,
                         void *stream);

/*
 * rpcg_eft_twosum / rpcg_eft_twoprod -- the error-free transformations of
 * Alg. 1 (r = RN(a_i + b_i), s = a_i + b_i - r) and Alg. 2 (r = RN(a_i b_i),
 * s = fma(a_i, b_i, -r)) applied elementwise, with the FPE dot's
 * integer-pipe arithmetic: twosum of finite elements as one FP64 addition
 * with the error computed exactly on the integer pipe (the form of the FPE
 * dot's error expansion; its result expansion uses the FP64 Fast2Sum, whose
 * pairs are the same) (elements that are not finite,
 * or whose sum overflows, use the FP64 formulas); twoprod of normal
 * elements whose product lies in [2^-916, 2^1023) as exact integer
 * arithmetic, others with the FP64 formulas.  Every output equals the FP64
 * algorithm's bit for bit.
 *   a, b      device arrays of n doubles (inputs); r, s: device outputs.
 * Asynchronous.
 */
rpcg_status rpcg_eft_twosum(int64_t n, const double *a, const double *b, double *r, double *s, void *stream);
rpcg_status rpcg_eft_twoprod(int64_t n, const double *a, const double *b, double *r, double *s, void *stream);

/*
 * rpcg_dot_plain -- ordinary FP64 dot (fma per element per thread, fixed
 * shuffle/shared-memory tree, then a fixed tree over CTA partials).  The
 * non-reproducible baseline of the paper's "Regular" PCG (Sec. 5.2).
 * out: device pointer to one double.  Asynchronous.
 */
rpcg_status rpcg_dot_plain(int64_t n, const double *a, const double *b, double *out, void *stream);

/*
 * rpcg_solve -- Jacobi-PCG (Fig. 1, S8 next to S6 as in Fig. 2) on A.
 *   b        device array, n doubles (right-hand side).
 *   x        device array, n doubles: in = x0, out = the final iterate.
 *   v        dot variant (rpcg_variant).
 *   o        options (NULL = defaults).
 *   res      host pointer, receives the outcome (the stream is synchronised).
 * Steps per iteration: w = A d; rho = RN(beta / <d,w>); x = fma(rho, d, x);
 * r = fma(-rho, w, r); z = RN(inv .* r); beta' = beta; beta = <z,r>;
 * tau = <r,r>; d = fma(RN(beta / beta'), d, z).  Set-up: inv = RN(1/diag),
 * r0 = RN(b - A x0), z0 = inv .* r0, d0 = z0, beta0 = <z0,r0>,
 * tau0 = <r0,r0>, ||b|| = RN(sqrt(<b,b>)).  The loop runs on the device
 * while relres >= tol and iterations < max_iter: as a CUDA graph of
 * grid-wide passes with a conditional while node, or, for systems of up to
 * 16384 rows whose slabs fit shared memory (every variant, o->block
 * and o->grid 0), as one launch of a thread-block cluster of up to 16 CTAs
 * that keeps the matrix and vectors in shared memory (rpcg_solve_path).
 * With RPCG_EXBLAS, and RPCG_FPE with fpe_strict = 0, every iterate,
 * residual and the iteration count are bit-identical for every launch shape
 * and on both paths.  b = 0 gives x = 0, 0 iterations.
 * Returns res->status.
 */
rpcg_status rpcg_solve(rpcg_matrix_t A, const double *b, double *x, int32_t v, const rpcg_opts *o, rpcg_result *res,
                       void *stream);

/*
 * rpcg_solve_profiled -- rpcg_solve with the same kernels launched one by
 * one from the host instead of the graph, and CUDA events recorded on
 * `stream` around each pass.  Results are bit-identical to rpcg_solve.
 *   pass_ms   host array of 4 floats: total milliseconds spent in the
 *             set-up, pass A (S1 + S2), pass B (S3-S6, S8), pass C (S7).
 *   launches  optional host array of 4 int32: launches of each.
 * It synchronises the stream once per iteration: a measurement tool.
 */
rpcg_status rpcg_solve_profiled(rpcg_matrix_t A, const double *b, double *x, int32_t v, const rpcg_opts *o,
                                rpcg_result *res, float *pass_ms, int32_t *launches, void *stream);

/*
 * rpcg_solve_async -- rpcg_solve without synchronising the stream: the solve
 * and the writing of *res are enqueued on `stream` and the call returns.
 *   res   device memory or pinned (page-locked) host memory; valid once the
 *         stream reaches that point (e.g. after cudaStreamSynchronize).
 * Same steps, paths and result bits as rpcg_solve, including x = 0 for
 * b = 0 and the NOT_CONVERGED / FPE_INEXACT statuses (decided on the device).
 * The arguments are passed to the device by value at the call, so solves may
 * be enqueued back to back; a handle serves one solve at a time in stream
 * order (its vectors and state are shared), different handles may run on
 * different streams concurrently.  Returns RPCG_OK when enqueued; argument
 * errors (RPCG_ERR_INVALID) and launch failures are returned at once and
 * nothing is enqueued for them.
 */
rpcg_status rpcg_solve_async(rpcg_matrix_t A, const double *b, double *x, int32_t v, const rpcg_opts *o,
                             rpcg_result *res, void *stream);

/*
 * rpcg_solve_path -- which path rpcg_solve takes for (A, v, o): *path = 1
 * for the cluster-resident launch, 0 for the graph of grid-wide passes.
 * (If the cluster cannot be made resident on this GPU, the first solve
 * finds out and every later call answers 0.)  No GPU work.
 */
rpcg_status rpcg_solve_path(rpcg_matrix_t A, int32_t v, const rpcg_opts *o, int32_t *path);

/*
 * rpcg_solve_host -- rpcg_solve with b and x in host memory: b and x0 are
 * copied to device buffers the handle owns, the solve runs, and x is
 * copied back.  Same semantics and result as rpcg_solve.
 */
rpcg_status rpcg_solve_host(rpcg_matrix_t A, const double *b_host, double *x_host, int32_t v, const rpcg_opts *o,
                            rpcg_result *res, void *stream);

/*
 * Batched solves: many independent SPD systems, each with its own matrix
 * handle, solved together (the loop of rpcg_solve for all of them at once).
 *
 * rpcg_batch_create -- group `count` distinct handles (the array is copied;
 * the handles must outlive the batch and must not be used by other calls
 * while a batch solve runs: the batch iterates in their r, d, w, inv).
 * rpcg_batch_destroy -- release the batch (not the handles).
 *
 * rpcg_batch_solve -- Jacobi-PCG (the steps of rpcg_solve, Fig. 1/Fig. 2)
 * on every system of the batch in one launch sequence: each pass is one
 * persistent kernel whose CTAs take work units (o->tile rows of one system)
 * of the systems still iterating from a shared counter; each system has its
 * own exact accumulators, scalars and convergence test and leaves the work
 * when it stops.
 *   b, x      host arrays of `count` device pointers (b[i], x[i]: n_i doubles;
 *             x[i] in = x0, out = the iterate).
 *   v         RPCG_EXBLAS or RPCG_FPE with fpe_strict = 0 (bit-identical to
 *             rpcg_solve of each system alone; a system whose FPE dots lost
 *             bits recomputes them exactly, the others skip that pass),
 *             RPCG_FPE with fpe_strict = 1 (inexact dots counted, status
 *             RPCG_FPE_INEXACT), or RPCG_PLAIN.
 *   o         options; o->history, if set, is a device array of
 *             count x (max_iter + 1) doubles (row i for system i).
 *             o->block (0, 128, 256) and o->tile (0, or 1..2^24 rows per unit): a zero
 *             picks them with the autotuner on the first solve of the batch
 *             (block 128 or 256 x tile 1024, 4096 or 16384 rows;
 *             short timed runs of each candidate on internal buffers; the
 *             choice is kept for later solves).
 *   res       host array of `count` results.
 * Returns the worst status over the systems.  Synchronises the stream.
 */
rpcg_status rpcg_batch_create(rpcg_batch_t *B, int32_t count, const rpcg_matrix_t *A);
rpcg_status rpcg_batch_destroy(rpcg_batch_t B);
rpcg_status rpcg_batch_solve(rpcg_batch_t B, const double *const *b, double *const *x, int32_t v, const rpcg_opts *o,
                             rpcg_result *res, void *stream);
/*
 * rpcg_batch_solve_async -- rpcg_batch_solve without synchronising the
 * stream: the batch run and the writing of res[0..count-1] (device memory or
 * pinned host memory) are enqueued on `stream` and the call returns.  Same
 * results as rpcg_batch_solve (NOT_CONVERGED and x = 0 for b = 0 decided on
 * the device).  It does not autotune: a zero o->block / o->tile takes the
 * autotuned shape if an earlier rpcg_batch_solve chose one, else 128 and
 * 1024 rows.  A batch runs one solve at a time in stream order (its handles'
 * vectors are shared); the call waits only if its previous upload of the
 * system table has not yet executed.  Argument errors return at once.
 */
rpcg_status rpcg_batch_solve_async(rpcg_batch_t B, const double *const *b, double *const *x, int32_t v,
                                   const rpcg_opts *o, rpcg_result *res, void *stream);

/*
 * rpcg_batch_solve_profiled -- rpcg_batch_solve with the batch kernels
 * launched one by one from the host and CUDA events recorded on `stream`
 * around each kind of pass; bit-identical results.  A zero o->block or
 * o->tile takes the autotuned value if there is one (else 128 and 4096 rows);
 * the autotuner is not run.
 *   pass_ms   host array of 5 floats: total milliseconds of the set-up
 *             (state reset, inverse diagonal, set-up pass), pass A, pass B,
 *             pass C and the retire/list kernel.
 *   launches  optional host array of 5 int32: launches of each.
 * It synchronises the stream once per pass: a measurement tool.
 */
rpcg_status rpcg_batch_solve_profiled(rpcg_batch_t B, const double *const *b, double *const *x, int32_t v,
                                      const rpcg_opts *o, rpcg_result *res, float *pass_ms, int32_t *launches,
                                      void *stream);
/* Block size and tile the autotuner picked (0, 0 before the first autotuned solve). */
rpcg_status rpcg_batch_tuned(rpcg_batch_t B, int32_t *block, int32_t *tile);

/* One-shot form: rpcg_batch_create + rpcg_batch_solve + rpcg_batch_destroy. */
rpcg_status rpcg_solve_batched(int32_t count, const rpcg_matrix_t *A, const double *const *b, double *const *x,
                               int32_t v, const rpcg_opts *o, rpcg_result *res, void *stream);

/*
 * Serving: a request loop that batches solves of different sizes as they
 * arrive (continuous batching).  A scheduler thread admits queued requests
 * into a table of `max_slots` slots while the device bytes in use (cached
 * matrices plus the vectors of running systems) stay within the HBM budget;
 * matrices stay on the device in an LRU cache, so repeated requests on the
 * same matrix do not upload it again.  A cached copy is reused only when the
 * contents are known to be the same: for a matrix registered with
 * rpcg_server_register (the server holds its own host copy), or for host
 * arrays submitted while an earlier request on the same addresses is still
 * uncollected (those arrays must not change until then).  Once every
 * ticket on some arrays has been collected, their addresses name nothing:
 * the next submit with them uploads afresh, whatever they now hold.
 * Running systems advance together, 16 iterations per scheduling
 * step, through the batched passes of rpcg_batch_solve; systems that stop
 * leave and queued ones join between steps.  Every result is bit-identical
 * to rpcg_solve of the same system alone (exact dots).  The paper has no
 * serving layer; this is the deployment form of its solver (Sec. 4).
 *
 * rpcg_server_create -- start the loop on the current device.
 *   hbm_budget_bytes  >= 1 MiB; requests that can never fit fail with
 *                     RPCG_ERR_OOM.
 * rpcg_server_submit -- queue one solve (the exblas variant; tol and
 *   max_iter from o).  rowptr/col/val (n, nnz) and b, and x0 if not NULL
 *   (else x0 = 0), are host arrays that must stay valid and unchanged until
 *   rpcg_server_wait returns for this ticket.  Never blocks on the GPU.
 * rpcg_server_register -- copy a CSR matrix (host arrays, n and nnz as
 *   in rpcg_create) into the server and return its id in *matrix; the
 *   caller's arrays may be freed when the call returns.  The copy and the
 *   device copy made from it are kept until rpcg_server_unregister and the
 *   collection of every ticket on it (the device copy may be evicted under
 *   the budget and uploaded again from the server's copy).
 * rpcg_server_submit_registered -- queue one solve on a registered matrix;
 *   b, and x0 if not NULL, as in rpcg_server_submit.  RPCG_ERR_INVALID for
 *   an unknown or unregistered id.
 * rpcg_server_unregister -- release a registered matrix (requests already
 *   queued on it still run).
 * rpcg_server_wait -- wait up to timeout_us (< 0: forever) for a ticket;
 *   copies x into x_host (n doubles, may be NULL), fills res and, if not
 *   NULL, the time the request queued and the time it was served.  Returns
 *   res->status, or RPCG_ERR_TIMEOUT (the ticket stays valid) or
 *   RPCG_ERR_INVALID (unknown or already collected ticket).
 * rpcg_server_stats -- counters.
 * rpcg_server_destroy -- finish every queued request, stop the loop, free
 *   all device memory.  Results not collected are dropped.
 */
typedef struct {
    double queue_us;   /* submit -> admitted into a slot */
    double service_us; /* admitted -> result back in host memory */
} rpcg_server_timing;

typedef struct {
    uint64_t completed;       /* requests finished (including failures) */
    uint64_t failed;          /* requests finished with a negative status */
    uint64_t queued;          /* requests waiting for a slot */
    uint64_t chunks;          /* scheduling steps run */
    uint64_t bytes_in_use;    /* device bytes held by cached matrices and running systems */
    uint64_t matrices_cached; /* matrices resident on the device */
} rpcg_server_stats_t;

rpcg_status rpcg_server_create(rpcg_server_t *srv, size_t hbm_budget_bytes, int32_t max_slots);
rpcg_status rpcg_server_submit(rpcg_server_t srv, int32_t n, int32_t nnz, const int32_t *rowptr, const int32_t *col,
                               const double *val, const double *b, const double *x0, int32_t v, const rpcg_opts *o,
                               uint64_t *ticket);
rpcg_status rpcg_server_register(rpcg_server_t srv, int32_t n, int32_t nnz, const int32_t *rowptr, const int32_t *col,
                                 const double *val, uint64_t *matrix);
rpcg_status rpcg_server_submit_registered(rpcg_server_t srv, uint64_t matrix, const double *b, const double *x0,
                                          int32_t v, const rpcg_opts *o, uint64_t *ticket);
rpcg_status rpcg_server_unregister(rpcg_server_t srv, uint64_t matrix);
rpcg_status rpcg_server_wait(rpcg_server_t srv, uint64_t ticket, double *x_host, rpcg_result *res,
                             rpcg_server_timing *timing, int64_t timeout_us);
rpcg_status rpcg_server_stats(rpcg_server_t srv, rpcg_server_stats_t *st);
rpcg_status rpcg_server_destroy(rpcg_server_t srv);

#ifdef __cplusplus
}
#endif

#endif /* RPCG_H */
