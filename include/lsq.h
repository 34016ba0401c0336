/*
 * lsq.h -- C ABI of the GB300 (sm_103a) row-sampling SGS-preconditioned PCG solver for
 * overdetermined least squares, after Chen & Wu, "A Preconditioner based on Non-uniform
 * Row Sampling for Linear Least Squares Problems" (arXiv:1806.02968).
 *
 * Problem (Sec. 1, Eqs. AXB, OPT, NOR): A in R^{m x n}, m >> n, rank n, b in R^m;
 * find x_opt = argmin ||A x - b||_2, i.e. solve A^T A x = A^T b.
 *
 * Method (Alg. 2):
 *   1. normalise A <- A D^{-1}, D_jj = ||a^j||_2                 (lsq_sample_rows)
 *   2. draw s = ceil(4 n ln n) rows i.i.d. with p_i = ||â_i||^2 / n (Alg. 1, Eq. R2P)
 *                                                                (lsq_sample_rows)
 *   3. build A_s^T A_s = (1/s) sum_t â_{i_t}^T â_{i_t} / p_{i_t}  (Sec. 3.3) and the
 *      symmetric Gauss-Seidel preconditioner on it (Alg. 3)      (lsq_build_precond)
 *   4. PCG on A^T A x = A^T b until the relative residual < eps  (lsq_pcg_solve)
 * plus the adjoint solve used for gradients                       (lsq_pcg_adjoint).
 *
 * Conventions for every call:
 *   - Pointers named "device" must point to device memory of the current CUDA device;
 *     "host" pointers to host memory.  All array arguments are BORROWED: the caller owns
 *     them and they must stay valid until the call returns (or, for stream-ordered
 *     outputs, until the stream reaches that point).  The library never frees them.
 *   - The only library-owned object is lsq_precond (free it with lsq_precond_destroy).
 *     Per-call scratch is taken with cudaMallocAsync on the given stream and released on
 *     the same stream before the call returns.
 *   - Work is issued on the given stream (0 = legacy default stream).  Calls that report
 *     data-dependent status (every call below) synchronise that stream once at the end
 *     to read it.
 *   - Errors are returned, never raised or aborted on: invalid shapes, dtypes, NULL
 *     pointers or misaligned buffers give LSQ_ERR_INVALID; a failing CUDA call gives
 *     LSQ_ERR_CUDA (lsq_last_error_string() has the CUDA message).  Device-side waits
 *     (grid barriers) give up after a bounded number of polls and report LSQ_ERR_TIMEOUT.
 *   - Sampling indices are a deterministic function of (A's values, seed, s); for a
 *     given input the solver's floating-point results are deterministic as well (every
 *     reduction has a fixed order).
 */
#ifndef LSQ_H
#define LSQ_H

#include <stdint.h>

#if defined(__GNUC__)
#define LSQ_API __attribute__((visibility("default")))
#else
#define LSQ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSQ_OK = 0,
    LSQ_ERR_INVALID = 1,        /* bad argument: shape, dtype, NULL, alignment, range */
    LSQ_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    LSQ_ERR_NOMEM = 3,          /* device allocation failed */
    LSQ_ERR_NOT_CONVERGED = 4,  /* maxit reached; outputs hold the last iterate */
    LSQ_ERR_BREAKDOWN = 5,      /* PCG scalar rho <= 0, p^T w <= 0 or not finite */
    LSQ_ERR_TIMEOUT = 6,        /* a device-side wait gave up (bounded spin) */
    LSQ_ERR_UNSUPPORTED = 7     /* valid request this build does not implement */
} lsq_status;

/* Storage type of matrix values.  LSQ_F32X2 holds each value as an unevaluated sum of
 * two floats (hi, lo), interleaved: element e occupies floats [2e, 2e+1]. */
typedef enum { LSQ_F64 = 0, LSQ_F32 = 1, LSQ_BF16 = 2, LSQ_F32X2 = 3 } lsq_dtype;

/* A in R^{m x n} (Sec. 1).  Dense: row-major, element (i, j) at vals[i*ld + j], ld >= n.
 * CSR: row_ptr[m+1] (int64), col_idx[nnz] (int32, strictly increasing inside a row),
 * vals[nnz].  All arrays are device memory.  vals_f64 (optional, NULL if absent) is an
 * FP64 copy of the values in the same layout; when given with a lower-precision dtype,
 * the solver computes its true residuals (iterative-refinement steps) from it. */
typedef struct {
    int64_t m, n, nnz;
    int32_t dense;               /* 1 = dense row-major, 0 = CSR */
    int64_t ld;                  /* dense leading dimension in elements */
    const int64_t* row_ptr;      /* CSR, device, m+1 entries */
    const int32_t* col_idx;      /* CSR, device, nnz entries */
    const void* vals;            /* device, dtype as below */
    int32_t dtype;               /* lsq_dtype */
    const double* vals_f64;      /* optional device FP64 copy of vals (same layout) */
} lsq_matrix;

/* Options.  lsq_default_opts() fills the defaults shown. */
typedef struct {
    double tol;            /* relative residual tolerance eps (Alg. 2 step 4); 1e-10 */
    int32_t maxit;         /* cap on PCG iterations over all outer steps; 1000000 */
    int32_t max_outer;     /* cap on PCG (re)starts from the true residual; 20 */
    int32_t sweeps;        /* t of Alg. 3 (forward and backward sweeps each); 1.  0 selects
                              the paper's comparison method (Sec. 5): CG on the
                              column-normalised A, i.e. P = I */
    double sample_factor;  /* C in s = ceil(C n ln n) (Alg. 2 step 2); 4.0 */
    int32_t normalize;     /* Alg. 2 step 1 on (1) or off (0); 1 */
    int32_t precond_dtype; /* LSQ_F64 or LSQ_F32: storage/arithmetic of the SGS operator (CSR:
                              with LSQ_F32 the sweeps sum in double-float, ~48 bits) */
    uint64_t seed;         /* Philox key word for the draws of Alg. 1; 0 */
    double inner_tol;      /* refinement form only: relative tolerance of each inner
                              solve; 0 = tol (no separate inner tolerance) */
    int32_t grid_ctas;     /* 0 = one persistent CTA per SM (x occupancy); else a cap */
    int32_t sampling;      /* row sampling density of Alg. 1: 0 = p_i proportional to the squared
                              row norm (Eq. R2P, the method); 1 = uniform p_i = 1/m (the
                              comparison of Sec. 3.1, which coherent matrices defeat); 0 */
    int32_t device_loop;   /* CSR A, k >= 2 columns, FP64 or FP32 values: 1 = the whole solve in
                              one persistent launch, no host decision or synchronisation until
                              the results are read; 0 = stream-ordered kernels with the loop on
                              the host (their passes keep more warps resident).  Under stream
                              capture the persistent form is always used; 0 */
} lsq_opts;

/* Per-right-hand-side results, written to caller-owned HOST arrays of length k (any
 * pointer may be NULL).  relres_rec: recursive ||g||/||g0|| of the normalised normal
 * equation; relres_true: the same recomputed from D^{-1} A^T (b - A x); relres_raw:
 * ||A^T (b - A x)|| / ||A^T b|| without column scaling. */
typedef struct {
    int64_t k;
    int32_t* iters;
    int32_t* outer;
    double* relres_rec;
    double* relres_true;
    double* relres_raw;
    uint8_t* converged;
    /* filled for the whole call */
    int64_t s, nnz_M, n_fixed_diag, levels;
    double setup_ms, solve_ms;
} lsq_info;

typedef struct lsq_precond lsq_precond;

/* Defaults listed in lsq_opts. */
LSQ_API void lsq_default_opts(lsq_opts* o);

/* Alg. 2 step 2: s = ceil(C n ln n) (natural log, rounded up; Alg. 2 writes 4 n log n
 * and the paper's printed sample sizes pin the natural log and the ceiling). */
LSQ_API int64_t lsq_sample_size(int64_t n, double C);

/*
 * lsq_sample_rows -- Alg. 2 steps 1-2 and Alg. 1 with the density of Eq. (R2P).
 *
 * Computes the column scales d_j = ||a^j|| and draws s row indices i.i.d. with
 * probability p_i = ||a_i D^{-1}||^2 / ||A D^{-1}||_F^2 (or ||a_i||^2/||A||_F^2 when
 * o->normalize == 0).  The law is evaluated exactly in integers so that the indices
 * are reproducible bit for bit:
 *   t_ij = fl(a_ij^2) (FP64, one rounding), E1 = 52 - floor(log2 max t_ij),
 *   c_j = sum_i floor(t_ij 2^E1) (exact), d2_j = RNE(c_j) 2^-E1, d_j = sqrt(d2_j);
 *   w_i = sum_j floor(2^51 fl(t_ij fl(1/d2_j))) (exact), p_i = w_i / W, W = sum w_i;
 *   draw t: Philox4x64-10 with key (seed, 0x5A4D504C), counter (t,0,0,0) -> words
 *   (r0, r1, ...); U = r1 2^64 + r0; i_t = max{i : sum_{l<i} w_l <= floor(U W / 2^128)}.
 * A column with c_j = 0 keeps d_j = 1 and no sampling weight.  max a_ij^2 must lie in
 * [2^-900, 2^900] and every value must be finite (else LSQ_ERR_INVALID).  With
 * o->sampling == 1 every row has weight w_i = 1 (p_i = 1/m; the column scales are still
 * computed), so the same draws give i_t = floor(U m / 2^128).
 *
 *   A          matrix (device arrays), any dtype
 *   o          options (normalize, seed, sample_factor); host
 *   s          number of draws; 0 means lsq_sample_size(n, o->sample_factor)
 *   idx_out    device int32[s]: i_t in draw order (output)
 *   p_out      device double[s]: p_{i_t} = w_{i_t}/W rounded to FP64 (output, may be NULL)
 *   colscale_out device double[n]: d_j (output, may be NULL)
 *   s_out      host: the s actually used (may be NULL)
 *   stream     cudaStream_t as void*
 */
LSQ_API lsq_status lsq_sample_rows(const lsq_matrix* A, const lsq_opts* o, int64_t s,
                           int32_t* idx_out, double* p_out, double* colscale_out,
                           int64_t* s_out, void* stream);

/*
 * lsq_sample_rows_static -- lsq_sample_rows for callers that cannot allocate device memory.
 *
 * The paper has no counterpart; this is a deployment convenience.  Some callers must not
 * allocate: code that runs inside another framework's device-memory pool with no headroom
 * left, or a real-time loop where an allocator call could block on the device or fail at
 * run time.  This entry point computes exactly what lsq_sample_rows computes (same kernels,
 * same bits) but takes all of its scratch from one fixed array in device memory that the
 * library declares (8.6 MiB, held by every GPU that loads the library until the process
 * exits); it calls no allocation routine.
 *
 * Limits: A may have at most 262144 rows and 4096 columns (else LSQ_ERR_INVALID).  The
 * first call on a device looks up the array's device address (once per device, with that
 * device current), so make the first call on each device before any stream capture.  The
 * address is kept for the life of the process's primary context on that device: after
 * cudaDeviceReset the library must be reloaded before this entry point is used again.
 * Every call uses the same array and clears what it accumulates in it, so a call never
 * depends on the previous call's leftovers; but calls that overlap on the GPU (different
 * streams, or host threads) race, so serialise them.  colscale_out may be NULL (the scales
 * then stay in the array).  Arguments, outputs and status as lsq_sample_rows.
 */
LSQ_API lsq_status lsq_sample_rows_static(const lsq_matrix* A, const lsq_opts* o, int64_t s,
                                          int32_t* idx_out, double* p_out, double* colscale_out,
                                          int64_t* s_out, void* stream);

/*
 * lsq_build_precond -- Sec. 3.3 and Alg. 3.
 *
 * Assembles M = A_s^T A_s = (1/s) sum_t â_{i_t}^T â_{i_t} / p_{i_t} (â = a D^{-1},
 * duplicates of a row counted once per draw), replaces a zero diagonal entry by 1, and
 * prepares the SGS operator of Alg. 3 with t = o->sweeps: e = 0; t forward corrections
 * e <- e + B^{-1}(r - M e), B the lower triangle of M with its diagonal; then t backward
 * corrections with B^T.  For dense A (n <= 2048) the operator is materialised once as an
 * n x n matrix by running exactly those sweeps on the unit vectors, so that applying it
 * inside PCG is one parallel product.
 *
 *   A, idx, p, colscale  as produced by lsq_sample_rows (device)
 *   s          number of draws in idx/p
 *   o          options (sweeps, precond_dtype); host
 *   P_out      host: receives the new library-owned handle
 */
LSQ_API lsq_status lsq_build_precond(const lsq_matrix* A, const int32_t* idx, const double* p,
                             const double* colscale, int64_t s, const lsq_opts* o,
                             lsq_precond** P_out, void* stream);

/* Free a handle from lsq_build_precond (NULL is ignored).  Stream-ordered on the stream
 * the handle was built on. */
LSQ_API void lsq_precond_destroy(lsq_precond* P);

/* Copy the assembled M = A_s^T A_s of Sec. 3.3 out of a dense handle (row-major n x n into
 * M_out, device double[n*n]).  For checking and diagnostics.  LSQ_ERR_INVALID for a NULL
 * argument or a sparse handle. */
LSQ_API lsq_status lsq_precond_get_M(const lsq_precond* P, double* M_out, void* stream);

/* Sparse handles: number of stored entries of M = A_s^T A_s (Sec. 3.3) in *nnz_out, and
 * (when the pointers are not NULL) M in CSR with sorted columns and the diagonal always
 * stored: row_ptr device int64[n+1], col_idx device int32[nnz], vals device double[nnz]. */
LSQ_API lsq_status lsq_precond_get_M_csr(const lsq_precond* P, int64_t* nnz_out, int64_t* row_ptr,
                                         int32_t* col_idx, double* vals, void* stream);

/* Copy the materialised SGS operator P of Alg. 3 (dense handles only, row-major n x n,
 * device double[n*n], converted to FP64): column j is Alg. 3 applied to the unit vector e_j. */
LSQ_API lsq_status lsq_precond_get_op(const lsq_precond* P, double* op_out, void* stream);

/* Apply the preconditioner of Alg. 3: e = P r for k vectors (device, column c at
 * r + c*n, e + c*n).  Dense handles multiply by the materialised operator; sparse handles
 * run the t forward and t backward Gauss-Seidel sweeps on M. */
LSQ_API lsq_status lsq_precond_apply(const lsq_precond* P, const double* r, double* e, int64_t k,
                             void* stream);

/*
 * lsq_pcg_solve -- Alg. 2 step 4: PCG on A^T A x = A^T b with the preconditioner P.
 *
 * Works on the normalised system Â^T Â y = Â^T b, Â = A D^{-1}, x = D^{-1} y.  Textbook
 * PCG from y = 0: g = Â^T b, z = P g, p = z; each iteration w = Â^T(Â p) in one fused
 * pass over the rows of A, alpha = rho / ||Â p||^2, y += alpha p, g -= alpha w, stop when
 * ||g|| <= tol ||Â^T b||, z = P g, beta = rho'/rho, p = z + beta p.  On stop the true
 * residual Â^T (b - Â y) is recomputed (in FP64 from vals_f64 when given); if it misses
 * the tolerance PCG restarts from y (one outer step), up to o->max_outer times.
 *
 * Dense A (values F64, F32, BF16 or F32X2): the whole loop of each column runs inside one
 * persistent cooperative kernel.  FP32 and BF16 values are products and sums in FP32 (BF16
 * widened exactly on load), F32X2 in double-float, with FP64 restarts from vals_f64.
 * CSR A (values F64, F32, BF16 or F32X2; P built with sweeps <= 32): each iteration is a
 * row pass, a column pass and the level-ordered sweeps of Alg. 3; k >= 2 columns advance
 * together in blocks of up to 32, with one pass over A and one sweep per iteration for the
 * whole block.  With o->device_loop = 1, or when the stream is being captured, a block with
 * FP64 or FP32 values runs as ONE persistent cooperative launch.  Under stream capture the
 * call writes X from the graph, reports no per-column results (info is left untouched) and
 * returns LSQ_OK; other value types return LSQ_ERR_UNSUPPORTED there.
 *
 *   A      matrix (device)
 *   P      handle built for this A
 *   B      device double, k right-hand sides, column c at B + c*ldb (ldb >= m)
 *   X      device double, k solutions, column c at X + c*ldx (ldx >= n) (output)
 *   info   host (may be NULL); per-column arrays of length >= k
 * Returns LSQ_ERR_NOT_CONVERGED when some column misses the tolerance (X holds the last
 * iterate), LSQ_ERR_BREAKDOWN on a PCG breakdown.
 */
LSQ_API lsq_status lsq_pcg_solve(const lsq_matrix* A, const lsq_precond* P, const double* B,
                         int64_t k, int64_t ldb, double* X, int64_t ldx, const lsq_opts* o,
                         lsq_info* info, void* stream);

/*
 * lsq_pcg_adjoint -- gradients through x = argmin ||A x - b|| (not in the paper; it
 * reuses the paper's preconditioner for the adjoint normal equation).
 *
 * Given solutions X (n x k), right-hand sides B (m x k) and G = dL/dX (n x k): solves
 * A^T A Lambda = G with the same PCG and preconditioner, then
 *   grad_b    = A Lambda                                   (device double m x k, ldb)
 *   grad_vals = sum_c (r_c lambda_c^T - (A lambda_c) x_c^T) on A's pattern, r = b - A x
 *               (device double[nnz] for CSR, [m*ld] for dense)
 * Either output may be NULL.  Lambda (device double n x k, ldx) is returned when not NULL.
 */
LSQ_API lsq_status lsq_pcg_adjoint(const lsq_matrix* A, const lsq_precond* P, const double* X,
                           const double* B, const double* G, int64_t k, int64_t ldb,
                           int64_t ldx, double* grad_b, double* grad_vals, double* Lambda,
                           const lsq_opts* o, lsq_info* info, void* stream);

/*
 * Batches of small dense problems (the batching extension; not in the paper, which solves
 * one problem at a time).  Every problem is an independent instance of Alg. 2 step 4 with
 * its own preconditioner; lsq_batch_solve runs the PCG of all of them in ONE kernel launch.
 *
 * lsq_batch_problem: one problem.
 *   m, n, ld   A is m x n, row-major with leading dimension ld; 1 <= n <= 256, n <= ld,
 *              ld a multiple of 4, m >= 1
 *   A          device float, 16-byte aligned.  Entries A[i*ld + j] with n <= j < ld are
 *              never used.  FP32 is the storage and the arithmetic of the inner iteration;
 *              restarts use the FP64 residual of the same values.
 *   P          dense handle from lsq_build_precond for this A (any precond_dtype, sweeps)
 *   B, ldb     device double, k right-hand sides, column c at B + c*ldb (ldb >= m)
 *   X, ldx     device double, k solutions, column c at X + c*ldx (ldx >= n) (output)
 * Every pointer is borrowed and must stay valid for the life of the plan.
 *
 * lsq_batch_create   copies the problem table to the device with the problems ordered largest
 *                    first (thread-block clusters take them from a queue in that order),
 *                    allocates the workspace.  1 <= k <= 16.  o: tol, maxit, max_outer, inner_tol.
 *                    Synchronises the stream.  *out is library-owned.
 * lsq_batch_solve    a memset of the queue counter and one launch, stream-ordered, no host
 *                    synchronisation and no allocation: can be captured in a CUDA graph.  Results go to the plan's device
 *                    status table.
 * lsq_batch_autotune times lsq_batch_solve for each cluster size that fits (1, 2, 4, 8 and,
 *                    where the device allows it, 16 CTAs per problem) and keeps the fastest;
 *                    *cluster_out (may be NULL) receives it.  The solutions are those of a
 *                    final run with the chosen size.  Synchronises the stream.
 * lsq_batch_set_cluster  choose the cluster size by hand (1, 2, 4, 8, 16); LSQ_ERR_UNSUPPORTED
 *                    if the device cannot run it.
 * lsq_batch_info     copies the per-problem, per-column results of the last solve into
 *                    infos[p] (host, count entries; arrays of length >= k) and synchronises;
 *                    returns LSQ_ERR_NOT_CONVERGED if any column missed the tolerance.
 * lsq_batch_destroy  frees the plan (NULL is ignored) after synchronising its stream.
 */
typedef struct {
    int64_t m, n, ld;
    const float* A;
    const lsq_precond* P;
    const double* B;
    int64_t ldb;
    double* X;
    int64_t ldx;
} lsq_batch_problem;

typedef struct lsq_batch lsq_batch;

LSQ_API lsq_status lsq_batch_create(const lsq_batch_problem* probs, int64_t count, int64_t k,
                                    const lsq_opts* o, lsq_batch** out, void* stream);
LSQ_API lsq_status lsq_batch_solve(lsq_batch* b, void* stream);
LSQ_API lsq_status lsq_batch_autotune(lsq_batch* b, int32_t* cluster_out, void* stream);
LSQ_API lsq_status lsq_batch_set_cluster(lsq_batch* b, int32_t cluster);
LSQ_API lsq_status lsq_batch_info(const lsq_batch* b, lsq_info* infos, void* stream);
LSQ_API void lsq_batch_destroy(lsq_batch* b);

/*
 * Row-sharded sampling (the multi-GPU design of the sampling steps; not in the paper, which
 * runs on one machine).  Rank r holds the rows [row0, row0 + A->m) of the whole matrix as
 * its own lsq_matrix.  Because the sampling law of lsq_sample_rows is exact integer
 * arithmetic, the cross-rank steps are plain integer collectives done by the caller, and
 * the merged draws equal one process's lsq_sample_rows bit for bit:
 *   1. lsq_shard_colmax   colmax[j] = max_i |a_ij| (FP64 bit patterns)  -> all-reduce MAX
 *   2. lsq_shard_colsum   the exact column sums c_j of Alg. 2 step 1 as four 32-bit limbs,
 *                         limbs[4j + k] (int64)                           -> all-reduce SUM
 *   3. lsq_shard_weights  d_j (the same on every rank) and the rank's prefix of the row
 *                         weights of Eq. (R2P); W_local_limbs (host) = the rank's total
 *                                                                      -> all-gather
 *   4. lsq_shard_offsets  the rank's offset and the grand total from the gathered totals
 *                         (host only)
 *   5. lsq_shard_draw     every draw t of Alg. 1 against the grand total; idx_out[t] is the
 *                         global row when the draw falls in this rank's range, else -1,
 *                         and p_out[t] the row's probability, else 0    -> all-reduce MAX
 * Arrays named "device" are device memory; colmax has n entries, limbs 4n, prefix
 * (A->m + 1) x 16 bytes (16-byte aligned), idx_out and p_out s entries.  Status and errors as
 * lsq_sample_rows.  lsq_shard_draw_host is step 5 for a prefix held in host memory (two
 * 64-bit words per entry, low first), for draws t0 .. t0 + s - 1.
 */
LSQ_API lsq_status lsq_shard_colmax(const lsq_matrix* A, uint64_t* colmax, void* stream);
LSQ_API lsq_status lsq_shard_colsum(const lsq_matrix* A, const uint64_t* colmax, int64_t* limbs, void* stream);
LSQ_API lsq_status lsq_shard_weights(const lsq_matrix* A, const lsq_opts* o, const uint64_t* colmax,
                                     const int64_t* limbs, double* colscale_out, void* prefix,
                                     int64_t* W_local_limbs, void* stream);
LSQ_API lsq_status lsq_shard_offsets(const int64_t* W_all, int32_t world, int32_t rank, int64_t* W_offset,
                                     int64_t* W_total);
LSQ_API lsq_status lsq_shard_draw(const void* prefix, int64_t m_local, int64_t row0, const int64_t* W_offset,
                                  const int64_t* W_total, const lsq_opts* o, int64_t s, int32_t* idx_out,
                                  double* p_out, void* stream);
LSQ_API lsq_status lsq_shard_draw_host(const uint64_t* prefix, int64_t m_local, int64_t row0,
                                       const int64_t* W_offset, const int64_t* W_total, uint64_t seed,
                                       int64_t t0, int64_t s, int32_t* idx_out);

/* Convert FP64 values to the LSQ_F32X2 pair format (hi = RN(v), lo = RN(v - hi)),
 * count elements, device to device (a storage form of this library, not in the paper).
 * LSQ_ERR_INVALID for NULL pointers or count < 0; count = 0 launches nothing. */
LSQ_API lsq_status lsq_split_f64(const double* src, float* dst_pairs, int64_t count, void* stream);

/* Human-readable name of a status code. */
LSQ_API const char* lsq_status_string(lsq_status s);

/* Message of the last error in this thread (CUDA error text or argument check). */
LSQ_API const char* lsq_last_error_string(void);

/* Number of kernels this library launched since load (for launch accounting). */
LSQ_API int64_t lsq_kernel_launch_count(void);

/* Cap on every device-side wait of the library (a diagnostic and test setting; not in the
 * paper).  Each wait polls at most max_polls times: the grid barriers of the persistent PCG
 * kernel (default 2^26 polls), the dependency waits of the sparse Gauss-Seidel sweeps of
 * Alg. 3 and of the level schedule builder (default 2^22).  0 restores the defaults.  A wait
 * that runs out records a timeout in the call's device error word, every other wait of that
 * launch then gives up as well, the kernel returns, and the call reports LSQ_ERR_TIMEOUT;
 * the outputs of that call are then undefined, the context stays usable and nothing needs
 * resetting.  Process-wide, read at each kernel launch.  LSQ_ERR_INVALID unless
 * 0 <= max_polls <= 2^31. */
LSQ_API lsq_status lsq_set_wait_limit(int64_t max_polls);

/* Form of the one-column sparse Gauss-Seidel sweeps (Alg. 3 on a CSR A_s^T A_s), a tuning and
 * test setting; every form computes the same rows in the same level order with the same
 * per-row arithmetic:
 *   0  chosen from the level schedule's shape: one CTA or the grid (the default),
 *   1  the grid: every row waits (bounded) for the values of its own dependencies,
 *   2  one CTA: levels meet at block barriers,
 *   3  one thread-block cluster of 8 CTAs: the sweep vector in the cluster's shared memory
 *      and levels at cluster barriers; where it does not fit (n > 204,800 or no cluster slot
 *      on the device) the grid form runs instead.
 * Blocks of k >= 2 right-hand sides (stream-ordered solves) take form 3 as well, where their
 * n x k vector fits (n k <= 204,800); every other value leaves them on their grid forms.
 * Process-wide, read when a solve or preconditioner application starts.  LSQ_ERR_INVALID
 * unless 0 <= form <= 3. */
LSQ_API lsq_status lsq_set_sweep_form(int32_t form);

/* Latency figures of the current device, for the latency bound of the level-ordered sweeps of
 * Alg. 3 (a diagnostic, not in the paper).  out_ns (host, 5 doubles, caller-owned) receives,
 * in nanoseconds:
 *   [0] one dependent load from L2 (one thread chasing a scattered cycle through 64 MB),
 *   [1] the round trip of a value between two SMs through global memory (two CTAs of one
 *       cooperative launch hand a counter back and forth with volatile loads and stores, the
 *       value being the flag, as in the sweeps),
 *   [2] one barrier of an 8-CTA thread-block cluster,
 *   [3] one dependent load from another CTA's shared memory in a 2-CTA cluster,
 *   [4] the round trip of [1] with a fence before each store.
 * Allocates and frees its own 64 MB buffer and synchronises the stream.  LSQ_ERR_TIMEOUT if the
 * hand-off ran out of polls, LSQ_ERR_CUDA if a probe could not be launched. */
LSQ_API lsq_status lsq_measure_latency(double* out_ns, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LSQ_H */
