/*
 * rska.h -- C ABI of librska, a GB300 (sm_103a) implementation of randomized
 * sparse Kaczmarz with averaging (RSKA), Tondji & Lorenz, "Faster Randomized
 * Block Sparse Kaczmarz by Averaging" (arXiv 2203.10838).
 *
 * The method (eq. rska, Algorithm 1), with uniform weights w_i = t (variant
 * v2 of Sec. 5 with alpha = t; t = 1 is variant v1):
 *
 *     tau_k    = eta row indices drawn i.i.d. with replacement,
 *                P(i) = ||a_i||^2 / ||A||_F^2
 *     x_k      = S_lambda(z_k),     S_lambda(v) = max(|v| - lambda, 0) sign(v)
 *     z_{k+1}  = z_k - (t/eta) sum_{i in tau_k} (<a_i, x_k> - b_i)/||a_i||^2 a_i
 *
 * starting from z_0 = x_0 = 0 (z is the paper's x^*).  For consistent systems
 * the iterates approach the solution of min lambda||x||_1 + 1/2||x||^2 subject
 * to Ax = b (eq. RBPP).
 *
 * Conventions shared by every entry point
 *  - Pointers named A, b, x_out, z_out, z_in, xhat and the table pointers are
 *    DEVICE pointers (cudaMalloc'd or equivalent) unless a comment says HOST.
 *  - A is row-major m x n with leading dimension lda (elements): lda >= n,
 *    lda a multiple of 4 and A 16-byte aligned, so that every row starts on a
 *    16-byte boundary.  Columns n..lda-1 are never used in arithmetic.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work is ordered on it; calls that return host
 *    values synchronize it.
 *  - Return value: RSKA_OK (0) or one of the RSKA_E* codes below.  A device
 *    fault or watchdog timeout is sticky: every later call on the context
 *    returns the same code until rska_reset() clears it (a CUDA error that
 *    corrupted the CUDA context cannot be cleared).
 *  - A context is not thread-safe; distinct contexts are independent.
 *
 * Index contract (bit-exact; the paper only fixes the distribution):
 *  - nu_i = ||a_i||^2 in FP64, summed as 32 partial sums (partial L takes the
 *    columns j = L mod 32 in ascending j) folded pairwise p_L + p_{L xor o}
 *    for o = 16, 8, 4, 2, 1; the result is partial 0.
 *  - Alias table (Walker/Vose) for p_i = nu_i / sum nu, built sequentially in
 *    FP64: W = sum nu in ascending i; q_i = (nu_i m)/W; LIFO stacks "small"
 *    (q < 1) and "large" filled in ascending i; each step pops l (small) and
 *    g (large): thr[l] = trunc(q_l 2^32) (0 if q_l <= 0), alias[l] = g,
 *    q_g = (q_g + q_l) - 1, g is pushed back to small if q_g < 1 else to
 *    large; buckets left over get thr = 2^32-1 and alias = self.
 *  - Slot s of iteration k: Philox4x32-10 with key (lo32(seed), hi32(seed))
 *    and counter (lo32(k), hi32(k), s/2, problem); even s uses words 0 and 1,
 *    odd s words 2 and 3.  Bucket c = (word_a * m) >> 32; the draw is c if
 *    word_b < thr[c], else alias[c].  problem = 0 for a single system.
 */
#ifndef RSKA_H
#define RSKA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSKA_OK 0
#define RSKA_EINVAL 1        /* bad argument: size, pointer, alignment, parameter range */
#define RSKA_EZEROROW 2      /* some row a_i is zero (Algorithm 1 requires a_i != 0) */
#define RSKA_ENONFINITE 3    /* A or b holds Inf or NaN */
#define RSKA_ENOMEM 4        /* device allocation failed */
#define RSKA_ECUDA 5         /* a CUDA runtime call failed */
#define RSKA_ETIMEOUT 6      /* a device-side wait exceeded its limit; kernel returned early */
#define RSKA_EUNSUPPORTED 7  /* valid but outside the library's limits (e.g. n too large) */

typedef struct rska_ctx rska_ctx;

/*
 * rska_setup -- validate the problem, compute FP64 row norms ||a_i||^2
 * (Definition 1, matrix D), build the alias table for p_i (Sec. 5, v1/v2) and
 * set z = 0, k = 0 (Algorithm 1, "starting points x_0 = x^*_0 = 0").
 *   out     HOST pointer receiving the new context (set to NULL on failure).
 *   A, b    device, borrowed: they must stay valid and unmodified until
 *           rska_destroy.  A: m x n, leading dimension lda.  b: m floats.
 *   lambda  >= 0, the shrinkage threshold of S_lambda.
 *   eta     batch size |tau_k|, 1 <= eta <= 4096.
 *   t       > 0, the uniform weight w_i = t (relaxation alpha of Sec. 4).
 *   seed    Philox key of the index contract.
 * Synchronizes `stream`.  Errors: EINVAL, EZEROROW, ENONFINITE, ENOMEM, ECUDA,
 * EUNSUPPORTED (n above the kernel's column capacity).
 */
int rska_setup(rska_ctx **out, const float *A, int64_t m, int64_t n, int64_t lda,
               const float *b, float lambda, int32_t eta, float t, uint64_t seed,
               void *stream);

/*
 * rska_setup_host -- HOST: rska_setup for host buffers.  A_host (m x lda
 * floats, row-major) and b_host (m floats) are host memory, read during the
 * call and not kept; the library allocates the device copies (freed by
 * rska_destroy).  A is copied in row chunks on a second stream while the row
 * norms of each landed chunk and the ascending FP64 sum W = sum_i ||a_i||^2 of
 * the alias construction run on `cuda_stream`, so the copy, the norms and the
 * sum overlap (with pinned host memory; pageable memory is copied without
 * overlap).  Tables, indices and iterates are identical to rska_setup's for
 * the same values.  Same argument rules and errors as rska_setup (no
 * alignment rule on A_host); synchronous.
 */
int rska_setup_host(rska_ctx **out, const float *A_host, int64_t m, int64_t n, int64_t lda,
                    const float *b_host, float lambda, int32_t eta, float t, uint64_t seed,
                    void *cuda_stream);

/*
 * rska_load_host -- HOST: load a new problem of the same shape into a context
 * made by rska_setup_host, reusing its device memory (no allocation): A_host
 * (m x lda floats) and b_host (m floats) with the m, n, lda of that setup are
 * copied, row norms and alias table rebuilt exactly as rska_setup_host does
 * (same overlap of copy, norms and W), and z = 0, k = 0.  lambda, eta, t,
 * seed and the options are kept; row weights return to uniform.  For callers
 * that solve many systems of one shape (the allocation of the device copy of
 * A then happens once).  Synchronous.  Errors: EINVAL (null pointers, or a
 * context not made by rska_setup_host), EZEROROW, ENONFINITE, ECUDA; clears
 * a sticky ETIMEOUT.
 */
int rska_load_host(rska_ctx *ctx, const float *A_host, const float *b_host);

/*
 * rska_solve -- run K iterations of Algorithm 1 (k -> k + K) on the context's
 * stream: per chunk of up to 2^21/eta iterations, one pre-sampling kernel
 * (tau_k, b and 1/||a||^2 for the whole chunk) and one persistent kernel
 * launch.  Asynchronous; K = 0 is a no-op.  Errors: EINVAL (K < 0), a sticky
 * code.
 */
int rska_solve(rska_ctx *ctx, int64_t K);

/*
 * rska_solve_until -- the stopping rule of Algorithm 1 ("until a stopping
 * criterion is satisfied"): run chunks of `check_every` iterations; after each
 * chunk compute in FP64 either the relative error ||x - xhat|| / ||xhat|| (xhat
 * given, device, n floats) or the relative residual ||Ax - b|| / ||b|| (xhat
 * NULL), and stop once it is <= tol or max_iters iterations have run.  All
 * chunks are enqueued in growing waves; a device flag makes the chunks after
 * the stop return immediately (with the one-CTA small-system kernel and xhat
 * given, the kernel runs the test itself every check_every iterations and
 * ends its launch at the first test that passes; one launch then covers up
 * to 16 checks).  Synchronizes.
 * iters_out (HOST, nullable) receives the
 * iterations actually run by this call; metric_out (HOST, nullable) the last
 * measured value.
 */
int rska_solve_until(rska_ctx *ctx, int64_t max_iters, int64_t check_every, double tol,
                     const float *xhat, int64_t *iters_out, double *metric_out);

/*
 * rska_get_x -- copy x = S_lambda(z) (x_out) and/or z = x^* (z_out), n floats
 * each (device pointers, either may be NULL).  Synchronizes.
 */
int rska_get_x(rska_ctx *ctx, float *x_out, float *z_out);

/*
 * rska_set_state -- restore a checkpoint: z <- z_in (device, n floats) and the
 * iteration counter k <- k.  tau_k depends only on (seed, k), so a restored
 * run continues the same index sequence.  Synchronizes.
 */
int rska_set_state(rska_ctx *ctx, const float *z_in, int64_t k);

/* rska_iteration -- HOST: the iteration counter k (iterations applied so far). */
int rska_iteration(rska_ctx *ctx, int64_t *k_out);

/*
 * rska_get_indices -- write tau_{k0} .. tau_{k0+K-1} (eta*K int32, row-major
 * [k][slot]) to `out` (device) using the same device sampler as the solver.
 * Synchronizes.
 */
int rska_get_indices(rska_ctx *ctx, int64_t k0, int64_t K, int32_t *out);

/*
 * rska_get_tables -- copy the FP64 row norms (m doubles), alias thresholds (m
 * uint32) and aliases (m int32) to device buffers (each may be NULL).
 */
int rska_get_tables(rska_ctx *ctx, double *nu_out, uint32_t *thr_out, int32_t *alias_out);

/*
 * rska_metrics -- FP64 relative residual ||Ax - b|| / ||b|| and, when xhat
 * (device, n floats) is given, relative error ||x - xhat|| / ||xhat|| of the
 * current x = S_lambda(z) (Sec. 5 metrics).  HOST outputs; synchronizes.
 * A zero denominator is replaced by 1e-30.
 */
int rska_metrics(rska_ctx *ctx, const float *xhat, double *rel_res, double *rel_err);

/* rska_reset -- z = 0, k = 0 and clear a sticky error.  Synchronizes. */
int rska_reset(rska_ctx *ctx);

/* rska_destroy -- free the context's device memory (A and b are not touched). */
int rska_destroy(rska_ctx *ctx);

/*
 * rska_query -- HOST: launch facts of the solver for this context:
 *   what = 0: CTAs in the persistent grid of the kernel in use
 *          1: threads per CTA
 *          2: rows of tau_k kept on chip (shared memory + registers) per
 *             iteration by the widest CTA; the rest are fetched twice
 *          3: float4 columns owned by the widest CTA
 *          4: dynamic shared memory bytes per CTA of the kernel in use
 *          5: row steps per thread held in registers (0 when the shared
 *             memory tile holds all of tau_k)
 *          6: solver kernel in use: 1 column-split, 2 row-split, 3 one-CTA
 *             small-system kernel
 *          7: microseconds the last setup spent allocating device memory
 *             (host clock; 0 after rska_load_host)
 *          8: microseconds of the copy (host buffers only), FP64 row norms
 *             and the sum W of the last setup or load (device events)
 *          9: microseconds of the alias construction (device events)
 *         10: microseconds of the whole last setup or load call (host clock)
 * Items 2, 3 and 5 describe the column-split kernel.
 */
int rska_query(rska_ctx *ctx, int what, int64_t *value_out);

/*
 * rska_set_option -- tuning knobs, applied from the next solve:
 *   what = 0: CTAs in the persistent grid (0 = automatic)
 *          1: watchdog limit of each device-side wait, in microseconds
 *             (default 2,000,000; 0: a wait that is not satisfied at its first
 *             poll expires, which exercises the failure path)
 *          2: solver kernel: 0 automatic (row-split when n <= 11520, else
 *             column-split; the one-CTA small-system kernel where the
 *             row-split plan is a single CTA and it fits), 1 column-split,
 *             2 row-split, 3 one-CTA small-system kernel (n <= 1024,
 *             eta <= 256, one iteration of rows in shared memory; else
 *             EUNSUPPORTED)
 * The row-split kernel gives each CTA whole rows of tau_k (TMA bulk copies)
 * and exchanges one n-vector per iteration; the column-split kernel gives
 * each CTA a slice of every row and exchanges eta dots per iteration; the
 * small-system kernel runs on one CTA, gives each row of tau_k to one warp
 * and keeps D iterations of rows in flight.
 */
int rska_set_option(rska_ctx *ctx, int what, int64_t value);

/*
 * rska_set_weights -- HOST: a general diagonal weight matrix W = diag(w) in
 * eq. (rska) (Sec. 5, variants v3 and v4).  From the next solve, iteration k
 * applies
 *     z -= (t/eta) sum_{s} w_{i_s} (<a_{i_s}, x_k> - b_{i_s}) / ||a_{i_s}||^2 a_{i_s}
 * (t = 1 gives the paper's v3/v4; the product w_i/||a_i||^2 is formed in FP64
 * and rounded once to FP32).
 *   w:      device pointer to m floats (read during the call, not kept), each
 *           finite and > 0; NULL restores uniform weights (w_i = 1).
 *   couple: 0 keeps p_i = ||a_i||^2/||A||_F^2 (v3); 1 samples p_i proportional
 *           to ||a_i||^2/w_i (v4): the alias table is rebuilt over
 *           rho_i = nu_i / w_i (one FP64 division per row) by the same
 *           construction and Philox draws as the index contract above, so
 *           rska_get_tables and rska_get_indices return the coupled table and
 *           indices.  With w = NULL couple is ignored.
 * The iteration count k and the iterate are kept.  Synchronous on the
 * context's stream; allocates temporary device memory.  Returns RSKA_EINVAL
 * for a null context, couple not 0 or 1, or a weight that is not finite and
 * positive (then nothing is changed), RSKA_ENOMEM, RSKA_ECUDA, or the
 * context's sticky error.
 */
int rska_set_weights(rska_ctx *ctx, const float *w, int couple);

/*
 * rska_sigma_max2 -- HOST: an estimate of sigma_max(A)^2, which Corollary 1
 * needs for the step alpha^*(eta) and Theorem th:RSKA for the admissible range
 * of t.  `iters` power iterations on A^T A from a start vector drawn from
 * `seed` (splitmix64 per entry): u = A v, rq = ||u||^2 (FP64), w = A^T u,
 * v = w / ||w|| (FP64 norm); products in FP32, reduced in a fixed order.
 *   sigma2_out: the last Rayleigh quotient rq (a lower estimate that converges
 *               to sigma_max^2 as iters grows; the rate depends on the gap
 *               between the two largest singular values)
 *   fro2_out:   nullable; ||A||_F^2 = sum_i nu_i (FP64)
 *   alpha_out:  nullable; alpha^*(eta) = eta / (1 + (eta - 1) sigma2 / fro2)
 *               (Corollary 1, uniform weights), usable as t in rska_setup
 * Synchronous on the context's stream; allocates temporary device memory
 * (m + 19 n floats).  Returns RSKA_EINVAL for a null context or sigma2_out or
 * iters outside 1..100000, RSKA_ENOMEM, RSKA_ECUDA, or the sticky error.
 */
int rska_sigma_max2(rska_ctx *ctx, int32_t iters, uint64_t seed, double *sigma2_out,
                    double *fro2_out, double *alpha_out);

/*
 * rska_linearized_bregman -- HOST: K iterations of the linearized Bregman
 * method, the eta -> infinity limit of eq. (rska) (Sec. 4, the remark on the
 * linearized Bregman rate and the mini-batch versus full-batch remark):
 *     z -= step * A^T (A x - b),   x = S_lambda(z)
 * (the paper's step is 1/sigma_max(A)^2; rska_sigma_max2 estimates it).  Runs
 * as the row-split kernel over every row once per iteration (one pass over A)
 * from the context's current z, and leaves z, x there; the RSKA iteration
 * counter k and its index sequence are not touched.  Requires n <= 11520
 * (else RSKA_EUNSUPPORTED).  Synchronous; allocates temporary device memory
 * (3 m + 2 words).  Returns RSKA_EINVAL for a null context, K < 0 or a step
 * that is not finite and positive, RSKA_ETIMEOUT, RSKA_ECUDA, or the sticky
 * error.
 */
int rska_linearized_bregman(rska_ctx *ctx, int64_t K, double step);

/* ------------------------------------------------------------------------ */
/* Batched independent systems: eq. (rska) / Algorithm 1 run on P problems   */
/* (A_p, b_p) in one persistent launch, each with its own index stream       */
/* (counter word 3 of the index contract = the problem's stream id, p unless */
/* rska_batch_set_stream_ids says otherwise) and its own stopping test.      */
/* ------------------------------------------------------------------------ */
typedef struct rska_batch rska_batch;

/*
 * rska_batch_setup -- FP64 row norms and alias tables for every problem
 * (Definition 1; Sec. 5, v1/v2), W_p = sum ||a_i||^2 and ||b_p||^2.
 *   A       device, borrowed: all matrices, A_p at element offset a_off[p],
 *           row-major m[p] x n[p] with leading dimension lda[p] (a multiple
 *           of 4; a_off[p] a multiple of 4; A 16-byte aligned).
 *   b       device, borrowed: b_p at element offset b_off[p] (m[p] floats).
 *   a_off, m, n, lda, b_off   HOST arrays of P entries (copied).
 *   lambda, eta, t, seed      shared by all problems, as for rska_setup.
 * Limits: n[p] <= 2688, eta <= 448.  Synchronizes.  Errors: EINVAL, EUNSUPPORTED, ENOMEM,
 * ECUDA, and EZEROROW / ENONFINITE of the first failing problem.
 */
int rska_batch_setup(rska_batch **out, int32_t P, const float *A, const int64_t *a_off,
                     const int64_t *m, const int64_t *n, const int64_t *lda, const float *b,
                     const int64_t *b_off, float lambda, int32_t eta, float t, uint64_t seed,
                     void *stream);

/*
 * rska_batch_solve -- from z_p = 0, iterate every problem until its relative
 * residual ||A_p x - b_p|| / ||b_p|| <= tol (checked every check_every
 * iterations, 0 = ceil(m_p/eta)) or until max_iters.  The exact check (dot
 * products by compensated FP32 summation, accurate as if in twice the
 * working precision; sums of squares in FP64) runs only when a running
 * estimate from the sampled residuals is within 4 tol, and after an exact
 * check that does not stop the problem the next 1, 3, 7 or 15 passing check
 * points are skipped.  tol = 0 runs exactly max_iters iterations on every
 * problem (the reported residual is that of the last iterate).  One CTA per
 * problem at a time, problems taken largest first.  Asynchronous.
 */
int rska_batch_solve(rska_batch *bt, int64_t max_iters, double tol, int64_t check_every);

/*
 * rska_batch_set_stream_ids -- HOST: the index-stream id of each problem
 * (counter word 3 of the index contract), P entries read during the call;
 * by default problem p uses id p.  A caller that splits one problem set
 * across several batches (one per GPU) gives every problem its id in the
 * whole set, so each problem draws the same tau_k wherever it runs.  Applies
 * from the next rska_batch_solve.  Synchronizes.  Errors: EINVAL, ECUDA.
 */
int rska_batch_set_stream_ids(rska_batch *bt, const uint32_t *ids);

/* rska_batch_results -- HOST outputs (P entries each, nullable): iterations
 * run and the last exact relative residual per problem.  Synchronizes. */
int rska_batch_results(rska_batch *bt, int64_t *iters, double *rel_res);

/* rska_batch_offsets -- HOST: P+1 offsets of each problem's x / z in the
 * packed outputs (n rounded up to 4 per problem). */
int rska_batch_offsets(rska_batch *bt, int64_t *x_off);

/* rska_batch_get_x -- copy the packed x = S_lambda(z) and z (device, length
 * x_off[P] each, either may be NULL).  Synchronizes. */
int rska_batch_get_x(rska_batch *bt, float *x_out, float *z_out);

/* rska_batch_get_tables -- copy the packed FP64 row norms, thresholds and
 * aliases (device, sum of m[p] entries each, problem p's rows after those of
 * problems 0..p-1; either may be NULL).  Synchronizes. */
int rska_batch_get_tables(rska_batch *bt, double *nu_out, uint32_t *thr_out, int32_t *alias_out);

/* rska_batch_destroy -- free the batch's device memory. */
int rska_batch_destroy(rska_batch *bt);

/* ------------------------------------------------------------------------ */
/* Unrolled form: K iterations of eq. (rska) on P problems (each with its own */
/* lambda_p, t_p and index stream, counter word 3 = p) and the hand-written   */
/* adjoint of that computation.  The paper has no gradient; this             */
/* differentiates the iteration as written, with S_lambda's derivative taken */
/* as 1[|z| > lambda] in z and -sign(z) 1[|z| > lambda] in lambda.            */
/* ------------------------------------------------------------------------ */
typedef struct rska_unrolled rska_unrolled;

/*
 * rska_unrolled_setup -- FP64 row norms and alias tables of every A_p (laid
 * out as for rska_batch_setup; a_off, m, n, lda, b_off HOST arrays).  K must
 * be a multiple of ckpt_every (z is checkpointed every ckpt_every
 * iterations).  eta <= 1024, n[p] <= 4096.  A is borrowed.  Synchronizes.
 */
int rska_unrolled_setup(rska_unrolled **out, int32_t P, const float *A, const int64_t *a_off,
                        const int64_t *m, const int64_t *n, const int64_t *lda,
                        const int64_t *b_off, int32_t eta, uint64_t seed, int32_t K,
                        int32_t ckpt_every, void *stream);

/*
 * rska_unrolled_forward -- x_K of every problem from z_0 = 0 (x_out packed by
 * rska_unrolled_offsets, device).  b (device, packed by b_off), lambda and t
 * (device, P floats each) are borrowed until the matching backward.
 * Asynchronous.
 */
int rska_unrolled_forward(rska_unrolled *u, const float *b, const float *lambda, const float *t,
                          float *x_out);

/*
 * rska_unrolled_backward -- given dL/dx_K (gx, device, packed like x_out),
 * write dL/db (gb, device, packed by b_off; zeroed first), dL/dlambda and
 * dL/dt (device, P floats each) of the last forward.  Recomputes each
 * checkpoint segment and replays tau_k from the index contract.
 * Asynchronous.
 */
int rska_unrolled_backward(rska_unrolled *u, const float *gx, float *gb, float *glam, float *gt);

/* rska_unrolled_offsets -- HOST: P+1 offsets of each problem's x in the
 * packed x_out / gx (n rounded up to 4). */
int rska_unrolled_offsets(rska_unrolled *u, int64_t *x_off);

/* rska_unrolled_destroy -- free the context's device memory. */
int rska_unrolled_destroy(rska_unrolled *u);

/* ------------------------------------------------------------------------ */
/* Shared-A multi-right-hand-side form: R systems A x_j = b_j with one A and */
/* one index stream tau_k (problem = 0 of the index contract, so tau is the  */
/* single-system sequence of A).  Iteration k is eq. (rska) for every j at   */
/* once, i.e. with X = S_lambda(Z) the two products of the matrix form       */
/* A^T M_k (A x - b) (Sec. 3):                                               */
/*     Res = A_tau X - B_tau;   Z <- Z - (t/eta) A_tau^T D_tau^-2 Res         */
/* computed on the tensor cores with BF16 operands and FP32 accumulation.    */
/* ------------------------------------------------------------------------ */
typedef struct rska_mrhs rska_mrhs;

/*
 * rska_mrhs_setup -- FP64 row norms (from the BF16 values, same canonical
 * order as rska_setup), alias table, and the solver state Z = 0.
 *   A      device, m x n BF16 (raw 16-bit patterns), row-major, leading
 *          dimension lda: lda >= n, lda a multiple of 8, A 16-byte aligned.
 *          Borrowed until rska_mrhs_destroy; never written.
 *   B      device, R x m FP32, row j = b_j, leading dimension ldb >= m.
 *          Copied (transposed) during setup; not referenced afterwards.
 *   lambda, eta, t, seed as for rska_setup; eta <= 4096.
 * Synchronizes `stream`.  Errors: EINVAL (sizes, alignment, parameter
 * range), EZEROROW, ENONFINITE (A or B), ENOMEM, ECUDA (including a driver
 * without cuTensorMapEncodeTiled).
 */
int rska_mrhs_setup(rska_mrhs **out, const void *A, int64_t m, int64_t n, int64_t lda,
                    const float *B, int64_t R, int64_t ldb, float lambda, int32_t eta, float t,
                    uint64_t seed, void *stream);

/*
 * rska_mrhs_set_option -- what = 0: terms of the inexact operand (X in the
 * first product, the scaled residual in the second): 2 (default) = BF16 high
 * + BF16 low part (relative representation error 2^-17), 1 = one BF16 term
 * (2^-9).  what = 1: CTAs splitting the first product's contraction over n
 * (0 = automatic, one wave).  what = 2: device wait limit in microseconds (0: a wait not satisfied at
 * its first poll expires).
 * what = 3: 1 (default) replays 64-iteration chunks as a CUDA graph, 0
 * launches every kernel directly.  what = 4: 1 (default) launches each
 * kernel of an iteration as a programmatic dependent of the previous one
 * (its prologue overlaps the previous kernel's tail), 0 orders them fully.
 * what = 5: form of the iteration: 0 automatic, 1 staged kernels (gather,
 * residual product, scale, update product per iteration; options 1, 3, 4
 * apply), 2 one persistent kernel per launch of up to 512 iterations that
 * keeps Z^T in tensor memory (each CTA owns 128 right-hand sides x 256
 * columns; needs eta <= 256 and (n_p / 256) (R_p / 128) CTAs resident at
 * once, else EUNSUPPORTED).  what = 6: terms of the scaled residual in the
 * second product (1 or 2; 0 = the same as option 0).  what = 7: gather
 * schedule of the persistent form: 0 the helper warps copy the next
 * iteration's rows of A while the residual product runs, 1 as soon as the
 * grid barrier has passed, 2 + k (k = 0..3) once chunk k of the scaled
 * residual (64 rows of tau) is formed after the barrier (k is clamped to
 * the last chunk); 0..5, default 2.
 * Setting option 1, 4, 5 (non-zero) or 7 pins the schedule; otherwise the
 * first rska_mrhs_solve of at least 128 iterations picks it (rska_mrhs_tune).
 * EINVAL for an unknown `what` or value.
 */
int rska_mrhs_set_option(rska_mrhs *h, int what, int64_t value);

/*
 * rska_mrhs_query -- HOST *value: what = 0 iterations done, 1 CTAs of the
 * first product's split over n, 2 n padded (multiple of 256), 3 eta padded
 * (multiple of 128), 4 R padded (multiple of 256), 5 terms (option 0),
 * 6 form of the next solve (1 staged, 2 persistent), 7 terms of the scaled
 * residual, 8 gather schedule, 9 the autotuner's choice (a code as in
 * rska_mrhs_tune; 0 before tuning), 10 its time per iteration in
 * nanoseconds, 11 the split over n of the staged form (0 = one wave), 12
 * programmatic dependent launches on (1) or off.
 */
int rska_mrhs_query(rska_mrhs *h, int what, int64_t *value);

/*
 * rska_mrhs_tune -- pick the fastest schedule of the iteration on this device
 * (the matrix form of Sec. 3 has several valid ways to run): every candidate
 * of rska_tune_candidates runs `iters` iterations (1..100000) after a
 * warm-up, timed with CUDA events on the context's stream, starting each time
 * from a saved copy of the iterate; afterwards the iterate and the iteration
 * count are what they were, and the fastest candidate is used from the next
 * solve and cached under the problem's shape, precision options and device
 * (see rska_tune_cache).  HOST outputs (nullable): the chosen code and its
 * microseconds per iteration.  Synchronous; allocates a temporary copy of the
 * iterate.  Errors: EINVAL, ENOMEM, ECUDA, a sticky code.
 */
int rska_mrhs_tune(rska_mrhs *h, int32_t iters, int32_t *code_out, double *us_per_iter_out);

/*
 * rska_tune_candidates -- HOST, no device work: the candidate schedules of a
 * multi-right-hand-side problem with n columns, R right-hand sides and batch
 * size eta on a GPU with num_sms SMs.  Each is a code: bits 0-1 the form
 * (1 staged kernels, 2 persistent kernel); staged: bits 8-15 the split of the
 * first product over n (0 = one wave), bit 16 programmatic dependent
 * launches; persistent: bits 17-19 the gather schedule (as option 7 of
 * rska_mrhs_set_option; 0, 1 and one per 64-row chunk of eta).  Writes up to `max` codes
 * and the total count (count_out).  Errors: EINVAL.
 */
int rska_tune_candidates(int64_t n, int64_t R, int32_t eta, int32_t num_sms, int32_t *codes_out,
                         int32_t max, int32_t *count_out);

/*
 * rska_tune_cache -- HOST, no device work: the process-wide cache of tuned
 * choices.  op 0: look up `key` (code and us out; EUNSUPPORTED when absent);
 * 1: store code and us under `key` (no spaces, at most 500 characters);
 * 2: write every entry to the file `key_or_path`; 3: read entries from it;
 * 4: clear.  With the environment variable RSKA_TUNE_CACHE naming a file,
 * that file is read at the first lookup and each new entry is appended.
 * Errors: EINVAL.
 */
int rska_tune_cache(int32_t op, const char *key_or_path, int32_t *code, double *us);

/*
 * rska_mrhs_solve -- K more iterations (K >= 0) for every right-hand side,
 * continuing the index stream at the current k.  Asynchronous; a device
 * timeout is reported by the next rska_mrhs_get_x.  Errors: EINVAL, ECUDA,
 * or the sticky code of an earlier failure.
 */
int rska_mrhs_solve(rska_mrhs *h, int64_t K);

/*
 * rska_mrhs_get_x -- device, R x n FP32 each (row j = x_j = S_lambda(z_j),
 * resp. z_j); either may be NULL.  Synchronizes; returns ETIMEOUT if a
 * device wait of an earlier solve gave up.
 */
int rska_mrhs_get_x(rska_mrhs *h, float *x_out, float *z_out);

/* rska_mrhs_get_indices -- tau_k for k = k0 .. k0+K-1 into out (device,
 * K * eta int32, iteration-major).  Synchronizes. */
int rska_mrhs_get_indices(rska_mrhs *h, int64_t k0, int64_t K, int32_t *out);

/* rska_mrhs_get_tables -- copies of nu (FP64), thr and alias (device, m
 * each; any may be NULL).  Synchronizes. */
int rska_mrhs_get_tables(rska_mrhs *h, double *nu_out, uint32_t *thr_out, int32_t *alias_out);

/* rska_mrhs_reset -- Z = 0, k = 0, clears a sticky error.  Asynchronous. */
int rska_mrhs_reset(rska_mrhs *h);

/* rska_mrhs_destroy -- free the context's device memory.  Synchronizes. */
int rska_mrhs_destroy(rska_mrhs *h);

/*
 * rska_solve_noalloc -- one-shot solve that allocates no device memory.  The
 * paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc while they run (an external memory budget or custom allocator
 * that forbids it, or code that must not synchronize the device the way
 * cudaMalloc/cudaFree may).
 *   A, b, lambda, eta, t, seed  as for rska_setup (A, b device, read only).
 *   K       iterations of Algorithm 1 from z_0 = 0 (K >= 0).
 *   x_out   device, n floats: x_K = S_lambda(z_K) (may be NULL if z_out is set)
 *   z_out   device, n floats: z_K (may be NULL if x_out is set)
 * Results equal those of rska_setup + rska_solve(K) + rska_get_x within FP32
 * reduction-order rounding (same index sequence).  All working memory lives
 * in one 4 MiB file-scope device array that every GPU loading this library
 * reserves until the process exits.  Limits: m <= 65536, n <= 16384 and
 * eta <= 1024; larger problems return RSKA_EUNSUPPORTED.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress, once per device, under a lock), so make that first
 * call before any stream capture.  Every call shares the one array and
 * re-initializes it: calls whose work overlaps on the GPU (different streams
 * or threads without ordering) race and corrupt each other's results.
 * Synchronizes `stream`.  Errors: EINVAL, EUNSUPPORTED, EZEROROW, ENONFINITE,
 * ECUDA, ETIMEOUT.
 */
int rska_solve_noalloc(const float *A, int64_t m, int64_t n, int64_t lda, const float *b,
                       float lambda, int32_t eta, float t, uint64_t seed, int64_t K,
                       float *x_out, float *z_out, void *stream);

/* rska_strerror -- static English text for a return code. */
/*
 * rska_probe_l2_read -- HOST, asynchronous on `stream`: the measurement probe
 * of the L2 read bandwidth, the roof of a configuration whose matrix stays in
 * L2 (Sec. 5 runs the 1000 x 500 system, 2 MB of A).  Launches `ctas` CTAs of
 * 512 threads that each read the caller's device buffer `buf` (`bytes`, a
 * multiple of 16, 16-byte aligned, small enough to stay in L2) `reps` times
 * with L2-cached loads; the caller times the launch (after a warm-up launch)
 * and divides ctas * reps * bytes by the time.  `sink` (device, `ctas`
 * floats) is written only to keep the loads alive.  Returns RSKA_EINVAL for a
 * bad argument, RSKA_ECUDA when the launch fails.
 */
int rska_probe_l2_read(const void *buf, int64_t bytes, int32_t reps, int32_t ctas, float *sink,
                       void *stream);

const char *rska_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* RSKA_H */
