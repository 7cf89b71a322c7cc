/*
 * rska_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for randomized
 * sparse Kaczmarz with averaging (RSKA), Tondji & Lorenz, "Faster Randomized
 * Block Sparse Kaczmarz by Averaging" (arXiv 2203.10838).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header or table with the CUDA path in paper_2203_10838_gb300/csrc, and the
 * CUDA path never calls it.
 *
 * Everything is FP64 except the inputs A (FP32 values, widened exactly) and the
 * integer sampler.  Build with -O2 -ffp-contract=off so that no multiply-add is
 * contracted behind the reader's back.
 *
 * Parity status of each function (what pins it; the pins live in tests/):
 *   orc_philox4x32_10  pinned: an independent Philox4x32-10 (Triton's) and
 *                       uniformity statistics.
 *   orc_row_norms       pinned: exact on integer-valued rows; closed form.
 *   orc_alias_build     pinned: exact bucket-probability reconstruction,
 *                       uniform-norm special case, sampling frequencies.
 *   orc_sample          pinned: chi-square of frequencies against p_i.
 *   orc_rska_fixed      pinned: hand-worked 2x2 step (tests/golden), exact
 *                       first/second moments of the step over all index tuples
 *                       (Lemma 1 / Lemma 2), Lemma lm:bd decrease, eta=1 RSK,
 *                       lambda=0 minimum-norm limit (pseudo-inverse), range
 *                       invariant, brute-force RBPP limit.
 *   orc_rska_fixed_weighted  pinned: w = 1 and constant w reduce to
 *                       orc_rska_fixed bit for bit; the exact mean of the step
 *                       over all index tuples equals the closed forms of v3
 *                       (A^T W (A x - b)/||A||_F^2) and v4 (A^T (A x - b) /
 *                       sum_j ||a_j||^2/w_j).
 *   orc_unrolled_grad   pinned: central finite differences of orc_rska_fixed.
 *   orc_metrics         pinned: closed form on hand-made vectors.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): a 4-word counter, a 2-word key, ten rounds.     */
/* Each round multiplies words 0 and 2 by two fixed odd constants, keeps the */
/* 64-bit products' high and low halves, xors the high halves with the other */
/* two counter words and the round key, and permutes.  The key is advanced   */
/* by two Weyl constants (golden ratio and sqrt(3)-1 in 32-bit fixed point)   */
/* between rounds.                                                           */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Row norms nu_i = ||a_i||^2 (Definition 1: D = Diag(||a_i||); the sampling */
/* probabilities of variants v1/v2 in Sec. 5 are p_i = ||a_i||^2/||A||_F^2). */
/* The summation order is part of the index contract (the paper fixes only   */
/* the value): 32 partial sums, partial L taking columns j = L mod 32 in     */
/* ascending j, then five pairwise folds p_L <- p_L + p_{L xor o} for        */
/* o = 16, 8, 4, 2, 1, and the result is partial 0.  Squares of FP32 values  */
/* are exact in FP64, so only the additions round.                           */
/* ------------------------------------------------------------------------ */
void orc_row_norms(const float *A, int64_t m, int64_t n, int64_t lda, double *nu)
{
    for (int64_t i = 0; i < m; ++i) {
        double p[32];
        for (int L = 0; L < 32; ++L) p[L] = 0.0;
        const float *row = A + i * lda;
        for (int64_t j = 0; j < n; ++j) {
            double a = (double)row[j];
            double sq = a * a;
            p[j % 32] = p[j % 32] + sq;
        }
        for (int o = 16; o >= 1; o /= 2) {
            double q[32];
            for (int L = 0; L < 32; ++L) q[L] = p[L] + p[L ^ o];
            for (int L = 0; L < 32; ++L) p[L] = q[L];
        }
        nu[i] = p[0];
    }
}

/* ------------------------------------------------------------------------ */
/* Alias table (Walker's method in Vose's linear-time form) for the row      */
/* distribution p_i = nu_i / sum_j nu_j (Sec. 5, v1/v2).  Bucket c keeps row */
/* c with probability thr[c] / 2^32 and otherwise yields alias[c].           */
/* Canonical construction, all in FP64:                                      */
/*   W = nu_0 + nu_1 + ... (ascending i);  q_i = (nu_i * m) / W;             */
/*   two LIFO stacks filled in ascending i: small (q < 1) and large (q >= 1);*/
/*   while both are non-empty: pop l from small and g from large,            */
/*     thr[l] = trunc(q_l * 2^32) (0 if q_l <= 0), alias[l] = g,             */
/*     q_g = (q_g + q_l) - 1, and push g to small if q_g < 1, else to large; */
/*   every bucket left on either stack is full: thr = 2^32-1, alias = self.  */
/* Returns 0, or -1 if some nu_i is zero or not finite (Algorithm 1 needs   */
/* nonzero rows) or m < 1.                                                   */
/* ------------------------------------------------------------------------ */
int orc_alias_build(const double *nu, int64_t m, uint32_t *thr, int32_t *alias)
{
    if (m < 1) return -1;
    double W = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        if (!(nu[i] > 0.0) || !isfinite(nu[i])) return -1;
        W = W + nu[i];
    }
    if (!isfinite(W)) return -1;
    double *q = (double *)malloc(sizeof(double) * (size_t)m);
    int64_t *small = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    int64_t *large = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    if (!q || !small || !large) {
        free(q); free(small); free(large);
        return -2;
    }
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < m; ++i) {
        q[i] = (nu[i] * (double)m) / W;
        if (q[i] < 1.0) small[ns++] = i;
        else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        int64_t l = small[--ns];
        int64_t g = large[--nl];
        double scaled = q[l] * 4294967296.0;
        uint32_t t;
        if (q[l] <= 0.0) t = 0u;
        else if (scaled >= 4294967295.0) t = 4294967295u;
        else t = (uint32_t)scaled; /* truncation == floor for positives */
        thr[l] = t;
        alias[l] = (int32_t)g;
        q[g] = (q[g] + q[l]) - 1.0;
        if (q[g] < 1.0) small[ns++] = g;
        else large[nl++] = g;
    }
    while (ns > 0) {
        int64_t l = small[--ns];
        thr[l] = 4294967295u;
        alias[l] = (int32_t)l;
    }
    while (nl > 0) {
        int64_t g = large[--nl];
        thr[g] = 4294967295u;
        alias[g] = (int32_t)g;
    }
    free(q); free(small); free(large);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Draw tau_k (Algorithm 1, "tau_k <- eta indices sampled": i.i.d. with     */
/* replacement, P(i) = p_i).  Index contract: slot s of iteration k uses    */
/* Philox4x32-10 with key (lo32(seed), hi32(seed)) and counter             */
/* (lo32(k), hi32(k), s/2, problem); even slots use output words 0,1 and     */
/* odd slots words 2,3.  The first word picks bucket c = (u * m) >> 32, the */
/* second keeps c if it is below thr[c], else the draw is alias[c].         */
/* out has K*eta entries: out[(k-k0)*eta + s].                               */
/* ------------------------------------------------------------------------ */
static int32_t draw_from_words(uint32_t u_bucket, uint32_t u_accept, const uint32_t *thr,
                               const int32_t *alias, int64_t m)
{
    uint64_t c = ((uint64_t)u_bucket * (uint64_t)m) >> 32;
    return (u_accept < thr[c]) ? (int32_t)c : alias[c];
}

static void draw_iteration(const uint32_t *thr, const int32_t *alias, int64_t m, uint64_t seed,
                           uint32_t problem, int64_t k, int32_t eta, int32_t *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t s = 0; s < eta; s += 2) {
        uint32_t ctr[4] = {(uint32_t)(uint64_t)k, (uint32_t)((uint64_t)k >> 32), (uint32_t)(s / 2),
                           problem};
        uint32_t u[4];
        orc_philox4x32_10(ctr, key, u);
        out[s] = draw_from_words(u[0], u[1], thr, alias, m);
        if (s + 1 < eta) out[s + 1] = draw_from_words(u[2], u[3], thr, alias, m);
    }
}

void orc_sample(const uint32_t *thr, const int32_t *alias, int64_t m, uint64_t seed,
                uint32_t problem, int64_t k0, int64_t K, int32_t eta, int32_t *out)
{
    for (int64_t k = k0; k < k0 + K; ++k)
        draw_iteration(thr, alias, m, seed, problem, k, eta, out + (k - k0) * eta);
}

/* ------------------------------------------------------------------------ */
/* Soft shrinkage S_lambda(v) = max(|v| - lambda, 0) * sign(v) (Sec. 1.1,   */
/* after eq. rsk), sign(0) = 0.                                              */
/* ------------------------------------------------------------------------ */
static double soft_shrink(double v, double lambda)
{
    double mag = fabs(v) - lambda;
    if (mag <= 0.0) return 0.0;
    return v > 0.0 ? mag : -mag;
}

/* ------------------------------------------------------------------------ */
/* One RSKA iteration, eq. (rska) / Algorithm 1 with weights t w_i (w = NULL: */
/* uniform weights t, variant v2 of Sec. 5 with alpha = t, t = 1 is v1; a    */
/* general diagonal W = diag(w) with t = 1 is v3 or v4):                     */
/*   x_k      = S_lambda(z_k)                   (z = x^*, the dual iterate)  */
/*   delta_k  = (1/eta) sum_{s} t w_{i_s} (<a_{i_s}, x_k> - b_{i_s})         */
/*              / ||a_{i_s}||^2 * a_{i_s}  (the eta draws, duplicates count) */
/*   z_{k+1}  = z_k - delta_k ;   x_{k+1} = S_lambda(z_{k+1}).               */
/* Residuals are taken at the thresholded x_k, coefficient sums in draw     */
/* order.  x and delta are caller-provided work vectors of length n.         */
/* ------------------------------------------------------------------------ */
static void rska_iteration(const float *A, int64_t n, int64_t lda, const double *b,
                           const double *nu, const double *w, double lambda, double t,
                           int32_t eta, const int32_t *tau, double *z, double *x, double *delta)
{
    for (int64_t j = 0; j < n; ++j) {
        x[j] = soft_shrink(z[j], lambda);
        delta[j] = 0.0;
    }
    for (int32_t s = 0; s < eta; ++s) {
        int64_t i = tau[s];
        const float *row = A + i * lda;
        double dot = 0.0;
        for (int64_t j = 0; j < n; ++j) dot = dot + (double)row[j] * x[j];
        double weight = w ? t * w[i] : t;
        double coeff = weight * (dot - b[i]) / nu[i];
        for (int64_t j = 0; j < n; ++j) delta[j] = delta[j] + coeff * (double)row[j];
    }
    for (int64_t j = 0; j < n; ++j) z[j] = z[j] - delta[j] / (double)eta;
}

/* K iterations with a given index sequence tau (K*eta entries); z is the    */
/* dual iterate x^* on entry (x^*_0 = 0 for Algorithm 1) and on exit.        */
int orc_rska_fixed(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
                   const double *nu, double lambda, double t, int32_t eta, const int32_t *tau,
                   int64_t K, double *z)
{
    if (m < 1 || n < 1 || lda < n || eta < 1 || K < 0) return -1;
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *delta = (double *)malloc(sizeof(double) * (size_t)n);
    if (!x || !delta) {
        free(x); free(delta);
        return -2;
    }
    for (int64_t k = 0; k < K; ++k)
        rska_iteration(A, n, lda, b, nu, NULL, lambda, t, eta, tau + k * eta, z, x, delta);
    free(x); free(delta);
    return 0;
}

/* As orc_rska_fixed with row weights w (m entries, the diagonal of W in     */
/* eq. (rska)); the step of row i is scaled by t * w_i.                      */
int orc_rska_fixed_weighted(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
                            const double *nu, const double *w, double lambda, double t,
                            int32_t eta, const int32_t *tau, int64_t K, double *z)
{
    if (m < 1 || n < 1 || lda < n || eta < 1 || K < 0 || !w) return -1;
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *delta = (double *)malloc(sizeof(double) * (size_t)n);
    if (!x || !delta) {
        free(x); free(delta);
        return -2;
    }
    for (int64_t k = 0; k < K; ++k)
        rska_iteration(A, n, lda, b, nu, w, lambda, t, eta, tau + k * eta, z, x, delta);
    free(x); free(delta);
    return 0;
}

/* K iterations drawing tau_k for k = k0 .. k0+K-1 with the index contract. */
int orc_rska_sampled(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
                     const double *nu, const uint32_t *thr, const int32_t *alias,
                     double lambda, double t, int32_t eta, uint64_t seed, uint32_t problem,
                     int64_t k0, int64_t K, double *z)
{
    if (m < 1 || n < 1 || lda < n || eta < 1 || K < 0) return -1;
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *delta = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *tau = (int32_t *)malloc(sizeof(int32_t) * (size_t)eta);
    if (!x || !delta || !tau) {
        free(x); free(delta); free(tau);
        return -2;
    }
    for (int64_t k = k0; k < k0 + K; ++k) {
        draw_iteration(thr, alias, m, seed, problem, k, eta, tau);
        rska_iteration(A, n, lda, b, nu, NULL, lambda, t, eta, tau, z, x, delta);
    }
    free(x); free(delta); free(tau);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Metrics of Sec. 5: relative residual ||A x - b|| / ||b|| and relative     */
/* error ||x - xhat|| / ||xhat|| with x = S_lambda(z), all in FP64.  xhat    */
/* may be NULL (then *rel_err is left untouched).  A zero denominator is     */
/* replaced by 1e-30.                                                        */
/* ------------------------------------------------------------------------ */
void orc_metrics(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
                 const double *z, double lambda, const double *xhat, double *rel_res,
                 double *rel_err)
{
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) x[j] = soft_shrink(z[j], lambda);
    double rr = 0.0, bb = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        const float *row = A + i * lda;
        double dot = 0.0;
        for (int64_t j = 0; j < n; ++j) dot = dot + (double)row[j] * x[j];
        double r = dot - b[i];
        rr = rr + r * r;
        bb = bb + b[i] * b[i];
    }
    *rel_res = sqrt(rr) / (bb > 0.0 ? sqrt(bb) : 1e-30);
    if (xhat) {
        double ee = 0.0, hh = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double e = x[j] - xhat[j];
            ee = ee + e * e;
            hh = hh + xhat[j] * xhat[j];
        }
        *rel_err = sqrt(ee) / (hh > 0.0 ? sqrt(hh) : 1e-30);
    }
    free(x);
}

/* ------------------------------------------------------------------------ */
/* Reverse-mode gradient of K unrolled RSKA iterations (the paper has no     */
/* gradient; this differentiates eq. (rska) as written).  Loss              */
/*   L = 1/2 ||x_K - xhat||^2,  x_K = S_lambda(z_K),  z_0 = 0,              */
/* with tau fixed (K*eta entries).  S_lambda has derivative 1[|z| > lambda] */
/* in z and -sign(z) 1[|z| > lambda] in lambda (strict mask at |z| = lambda).*/
/* Every z_k is stored ((K+1)*n doubles).  Reverse sweep, g = dL/dz_{k+1}:   */
/*   u_s   = (t/eta) <a_{i_s}, g> / nu_{i_s}                                 */
/*   dL/db_{i_s} += u_s                 (duplicates add)                     */
/*   dL/dt += -(1/eta) sum_s r_s / nu_{i_s} <a_{i_s}, g>                     */
/*   xbar  = -sum_s u_s a_{i_s}                                              */
/*   dL/dlambda += sum_j xbar_j * (-sign(z_kj)) 1[|z_kj| > lambda]           */
/*   dL/dz_k = g + 1[|z_k| > lambda] * xbar                                  */
/* Outputs: *loss, gb[m] (overwritten), *glam, *gt.                          */
/* ------------------------------------------------------------------------ */
int orc_unrolled_grad(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
                      const double *nu, double lambda, double t, int32_t eta, const int32_t *tau,
                      int64_t K, const double *xhat, double *loss, double *gb, double *glam,
                      double *gt)
{
    if (m < 1 || n < 1 || lda < n || eta < 1 || K < 0) return -1;
    double *zs = (double *)calloc((size_t)(K + 1) * (size_t)n, sizeof(double));
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *delta = (double *)malloc(sizeof(double) * (size_t)n);
    double *g = (double *)malloc(sizeof(double) * (size_t)n);
    double *xbar = (double *)malloc(sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)eta);
    if (!zs || !x || !delta || !g || !xbar || !r) {
        free(zs); free(x); free(delta); free(g); free(xbar); free(r);
        return -2;
    }
    /* forward, keeping z_0 .. z_K */
    for (int64_t k = 0; k < K; ++k) {
        memcpy(zs + (k + 1) * n, zs + k * n, sizeof(double) * (size_t)n);
        rska_iteration(A, n, lda, b, nu, NULL, lambda, t, eta, tau + k * eta, zs + (k + 1) * n, x,
                       delta);
    }
    /* loss and its gradient at x_K */
    const double *zK = zs + K * n;
    double L = 0.0, gl = 0.0, gtt = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double xj = soft_shrink(zK[j], lambda);
        double e = xj - xhat[j];
        L = L + 0.5 * e * e;
        int active = fabs(zK[j]) > lambda;
        g[j] = active ? e : 0.0;
        if (active) gl = gl + e * (zK[j] > 0.0 ? -1.0 : 1.0);
    }
    for (int64_t i = 0; i < m; ++i) gb[i] = 0.0;
    /* reverse sweep */
    for (int64_t k = K - 1; k >= 0; --k) {
        const double *zk = zs + k * n;
        const int32_t *tk = tau + k * eta;
        for (int64_t j = 0; j < n; ++j) {
            x[j] = soft_shrink(zk[j], lambda);
            xbar[j] = 0.0;
        }
        for (int32_t s = 0; s < eta; ++s) {
            int64_t i = tk[s];
            const float *row = A + i * lda;
            double dx = 0.0, dg = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                dx = dx + (double)row[j] * x[j];
                dg = dg + (double)row[j] * g[j];
            }
            r[s] = dx - b[i];
            double u = (t / (double)eta) * dg / nu[i];
            gb[i] = gb[i] + u;
            gtt = gtt - (r[s] / nu[i]) * dg / (double)eta;
            for (int64_t j = 0; j < n; ++j) xbar[j] = xbar[j] - u * (double)row[j];
        }
        for (int64_t j = 0; j < n; ++j) {
            if (fabs(zk[j]) > lambda) {
                gl = gl + xbar[j] * (zk[j] > 0.0 ? -1.0 : 1.0);
                g[j] = g[j] + xbar[j];
            }
        }
    }
    *loss = L;
    *glam = gl;
    *gt = gtt;
    free(zs); free(x); free(delta); free(g); free(xbar); free(r);
    return 0;
}
