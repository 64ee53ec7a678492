/*
 * FP64 CPU oracle for GP reconstruction + level-crossing probability (LCP).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Plain, slow, obviously-correct definitions, in the paper's order:
 *   - kernel k(x1,x2): RBF sigma^2 exp(-|x1-x2|^2/(2 l^2)) (Sec. 3, Sec. 5.2);
 *     anisotropic lengths divide each axis; Matern-5/2 is the textbook
 *     (1+sqrt5 r+5r^2/3)exp(-sqrt5 r) (Rasmussen & Williams eq. 4.17).
 *   - posterior, Eq. (1): for plain GPR the stored inducing distribution is the
 *     latent posterior at the observations, and Eq. (1) reduces to
 *     mu(x) = k_x^T Kt^-1 y, Sigma(a,b) = k(a,b) - k_a^T Kt^-1 k_b,
 *     Kt = K(X,X) + sn2 I.  Both forms are implemented (or_posterior,
 *     or_posterior_sgpr) so a test can check the reduction.
 *   - cell LCP (Sec. 4): 1 - P(all 8 corners < theta) - P(all 8 > theta),
 *     estimated either by the Genz sequential-conditioning (SOV) rule over a
 *     shifted rank-1 lattice or by Monte Carlo (the paper's estimator, 1600
 *     samples, Sec. 6.4) with Philox-4x32-10 + Box-Muller normals.
 *   - regional bound, Eq. (upper_bound) with Slepian's inequality (Sec. 5.1):
 *     1 - B_l^d - B_u^d, B = min over the node of Phi(+-(theta-mu)/sigma).
 *   - octree adaptive query, Algorithm 1 (Sec. 5.3), one level per call.
 *
 * Readings where the paper is silent are fixed by the caller-visible options
 * (jitter tau, skip epsilon, minimiser steps T) and documented at each site.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_SE 0
#define OR_MATERN52 1

typedef struct {
    int64_t m;
    int kernel;
    double ell[3];
    double sf2, sn2;
    double *X;      /* m x 3 */
    double *y;      /* m */
    double *L;      /* m x m row-major, lower Cholesky factor of Kt */
    double *Linv;   /* m x m row-major, L^-1 (lower) */
    double *vy;     /* L^-1 y */
    double *alpha;  /* Kt^-1 y */
    double *mu_obs; /* latent posterior mean at the observations */
    double *var_obs;/* latent posterior variance at the observations */
    /* SGPR model (Eq. 1 with a stored inducing distribution N(mu_M, A_M)); 0 for plain GPR.
     * Then L is the Cholesky factor of K_MM (+ jitter I), alpha = K_MM^-1 mu_M, y = mu_M,
     * and mu_obs / var_obs are mu_M and diag(A_M). */
    int sgpr;
    double *A;      /* m x m A_M */
    double kmm_jitter; /* SGPR: jitter on the diagonal of K_MM */
} or_model;

/* ------------------------------------------------------------------ kernel */

double or_kernel_eval(int kernel, const double *ell, double sf2, const double *a, const double *b)
{
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double t = (a[d] - b[d]) / ell[d];
        r2 += t * t;
    }
    if (kernel == OR_SE) return sf2 * exp(-0.5 * r2);
    double r = sqrt(r2), s5r = sqrt(5.0) * r;
    return sf2 * (1.0 + s5r + 5.0 * r2 / 3.0) * exp(-s5r);
}

/* d k(x, b) / d x_d for the kernel above (gradient in the first argument). */
static void kernel_grad(int kernel, const double *ell, double sf2, const double *x, const double *b,
                        double *k_out, double g[3])
{
    double r2 = 0.0, dd[3];
    for (int d = 0; d < 3; ++d) {
        dd[d] = x[d] - b[d];
        double t = dd[d] / ell[d];
        r2 += t * t;
    }
    if (kernel == OR_SE) {
        double k = sf2 * exp(-0.5 * r2);
        *k_out = k;
        for (int d = 0; d < 3; ++d) g[d] = -k * dd[d] / (ell[d] * ell[d]);
    } else {
        double r = sqrt(r2), s5r = sqrt(5.0) * r, e = exp(-s5r);
        *k_out = sf2 * (1.0 + s5r + 5.0 * r2 / 3.0) * e;
        /* dk/dr = -(5/3) sf2 r (1 + sqrt5 r) e^{-sqrt5 r};  dr/dx_d = dd/(l^2 r) */
        double c = -(5.0 / 3.0) * sf2 * (1.0 + s5r) * e;
        for (int d = 0; d < 3; ++d) g[d] = c * dd[d] / (ell[d] * ell[d]);
    }
}

/* --------------------------------------------------------- dense algebra */

/* In-place Cholesky of an n x n row-major SPD matrix (lower). 0 on success. */
int or_cholesky(double *A, int64_t n)
{
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int64_t k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
        for (int64_t k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
    }
    return 0;
}

/* Solve L x = b (forward substitution), L lower n x n row-major. */
static void fwd_sub(const double *L, int64_t n, const double *b, double *x)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = b[i];
        const double *row = L + i * n;
        for (int64_t k = 0; k < i; ++k) s -= row[k] * x[k];
        x[i] = s / row[i];
    }
}

/* Solve L^T x = b (back substitution). */
static void back_sub_T(const double *L, int64_t n, const double *b, double *x)
{
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int64_t k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

static double dot(const double *a, const double *b, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------ model */

void or_model_destroy(or_model *M)
{
    if (!M) return;
    free(M->X); free(M->y); free(M->L); free(M->Linv); free(M->vy); free(M->alpha);
    free(M->mu_obs); free(M->var_obs); free(M->A);
    free(M);
}

/* Builds Kt = K(X,X) + sn2 I, its Cholesky factor, L^-1, L^-1 y, Kt^-1 y and the
 * latent posterior at the observations (Sec. 5.3's p1/p2 test needs it).  With
 * the observations as inducing set, mu_M = K Kt^-1 y = y - sn2 Kt^-1 y and
 * A_M = K - K Kt^-1 K = sn2 I - sn2^2 Kt^-1 (because K = Kt - sn2 I).
 * Variance floor: 1e-12 sf2 (reading; the paper is silent).
 * Returns NULL when Kt is not positive definite. */
or_model *or_model_create(const double *X, const double *y, int64_t m, int kernel,
                          const double *ell, double sf2, double sn2)
{
    or_model *M = (or_model *)calloc(1, sizeof(or_model));
    M->m = m; M->kernel = kernel; M->sf2 = sf2; M->sn2 = sn2;
    for (int d = 0; d < 3; ++d) M->ell[d] = ell[d];
    M->X = (double *)malloc(sizeof(double) * 3 * m);
    M->y = (double *)malloc(sizeof(double) * m);
    memcpy(M->X, X, sizeof(double) * 3 * m);
    memcpy(M->y, y, sizeof(double) * m);
    M->L = (double *)malloc(sizeof(double) * m * m);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j)
            M->L[i * m + j] = or_kernel_eval(kernel, ell, sf2, X + 3 * i, X + 3 * j) + (i == j ? sn2 : 0.0);
    if (or_cholesky(M->L, m) != 0) { or_model_destroy(M); return NULL; }
    /* L^-1 column by column: L x = e_j */
    M->Linv = (double *)calloc((size_t)(m * m), sizeof(double));
    double *e = (double *)calloc((size_t)m, sizeof(double));
    double *col = (double *)malloc(sizeof(double) * m);
    for (int64_t j = 0; j < m; ++j) {
        e[j] = 1.0;
        fwd_sub(M->L, m, e, col);
        e[j] = 0.0;
        for (int64_t i = 0; i < m; ++i) M->Linv[i * m + j] = col[i];
    }
    free(e); free(col);
    M->vy = (double *)malloc(sizeof(double) * m);
    M->alpha = (double *)malloc(sizeof(double) * m);
    fwd_sub(M->L, m, y, M->vy);
    back_sub_T(M->L, m, M->vy, M->alpha);
    M->mu_obs = (double *)malloc(sizeof(double) * m);
    M->var_obs = (double *)malloc(sizeof(double) * m);
    for (int64_t i = 0; i < m; ++i) {
        double qii = 0.0; /* [Kt^-1]_ii = sum_k (L^-1)_{ki}^2 */
        for (int64_t k = i; k < m; ++k) qii += M->Linv[k * m + i] * M->Linv[k * m + i];
        M->mu_obs[i] = y[i] - sn2 * M->alpha[i];
        double v = sn2 - sn2 * sn2 * qii;
        double fl = 1e-12 * sf2;
        M->var_obs[i] = v > fl ? v : fl;
    }
    return M;
}

/* SGPR model (Sec. 3): inducing sites X (m x 3) with the stored distribution N(mu_M, A_M) of
 * their values.  K_MM = K(X, X) + jitter I is factorised once; Eq. 1 is evaluated as printed by
 * the sgpr_* helpers below.  Algorithm 1's p-test reads the inducing distribution itself
 * (Sec. 5.3: mean vector mu_M and covariance A_M of the inducing points in the node), so
 * mu_obs = mu_M and var_obs = diag(A_M) (floor 1e-12 sf2).  NULL if K_MM is not PD. */
or_model *or_model_create_sgpr(const double *X, const double *muM, const double *AM, int64_t m, int kernel,
                               const double *ell, double sf2, double jitter)
{
    or_model *M = (or_model *)calloc(1, sizeof(or_model));
    M->m = m; M->kernel = kernel; M->sf2 = sf2; M->sn2 = 0.0; M->sgpr = 1; M->kmm_jitter = jitter;
    for (int d = 0; d < 3; ++d) M->ell[d] = ell[d];
    M->X = (double *)malloc(sizeof(double) * 3 * m);
    M->y = (double *)malloc(sizeof(double) * m);
    M->A = (double *)malloc(sizeof(double) * m * m);
    memcpy(M->X, X, sizeof(double) * 3 * m);
    memcpy(M->y, muM, sizeof(double) * m);
    memcpy(M->A, AM, sizeof(double) * m * m);
    M->L = (double *)malloc(sizeof(double) * m * m);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j)
            M->L[i * m + j] = or_kernel_eval(kernel, ell, sf2, X + 3 * i, X + 3 * j) + (i == j ? jitter : 0.0);
    if (or_cholesky(M->L, m) != 0) { or_model_destroy(M); return NULL; }
    M->vy = (double *)malloc(sizeof(double) * m);
    M->alpha = (double *)malloc(sizeof(double) * m);
    fwd_sub(M->L, m, muM, M->vy);
    back_sub_T(M->L, m, M->vy, M->alpha);
    M->mu_obs = (double *)malloc(sizeof(double) * m);
    M->var_obs = (double *)malloc(sizeof(double) * m);
    for (int64_t i = 0; i < m; ++i) {
        double fl = 1e-12 * sf2, v = AM[i * m + i];
        M->mu_obs[i] = muM[i];
        M->var_obs[i] = v > fl ? v : fl;
    }
    return M;
}

/* Eq. 1 pieces of one point x for an SGPR model: k = K_MI column of x, a = K_MM^-1 k,
 * c = A_M a.  Then mu(x) = a . mu_M, Sigma(x, z) = k(x, z) - k_x . a_z + a_x . c_z. */
static void sgpr_row(const or_model *M, const double *x, double *k, double *a, double *c, double *tmp)
{
    int64_t m = M->m;
    for (int64_t j = 0; j < m; ++j) k[j] = or_kernel_eval(M->kernel, M->ell, M->sf2, x, M->X + 3 * j);
    fwd_sub(M->L, m, k, tmp);
    back_sub_T(M->L, m, tmp, a);
    for (int64_t i = 0; i < m; ++i) c[i] = dot(M->A + i * m, a, m);
}

/* Sigma(x_a, x_b) of Eq. 1 from the pieces of sgpr_row: k(x_a, x_b) - K_aM K_MM^-1 K_Mb
 * + K_aM K_MM^-1 A_M K_MM^-1 K_Mb = k(a, b) - k_a . a_b + a_a . c_b. */
static double sgpr_cov(const or_model *M, const double *xa, const double *xb, const double *ka, const double *aa,
                       const double *ab, const double *cb)
{
    int64_t m = M->m;
    return or_kernel_eval(M->kernel, M->ell, M->sf2, xa, xb) - dot(ka, ab, m) + dot(aa, cb, m);
}

void or_model_get(const or_model *M, double *L, double *alpha, double *vy, double *mu_obs, double *var_obs)
{
    int64_t m = M->m;
    if (L) memcpy(L, M->L, sizeof(double) * m * m);
    if (alpha) memcpy(alpha, M->alpha, sizeof(double) * m);
    if (vy) memcpy(vy, M->vy, sizeof(double) * m);
    if (mu_obs) memcpy(mu_obs, M->mu_obs, sizeof(double) * m);
    if (var_obs) memcpy(var_obs, M->var_obs, sizeof(double) * m);
}

/* v = L^-1 k_x for one point (whitened kernel row). */
static void whiten_row(const or_model *M, const double *x, double *kbuf, double *v)
{
    for (int64_t j = 0; j < M->m; ++j) kbuf[j] = or_kernel_eval(M->kernel, M->ell, M->sf2, x, M->X + 3 * j);
    fwd_sub(M->L, M->m, kbuf, v);
}

/* Posterior of plain GPR at n points: mean (n) and, if cov != NULL, the full
 * n x n covariance; var (n) always.  Sigma(a,b) = k(a,b) - v_a . v_b. */
void or_posterior(const or_model *M, const double *P, int64_t n, double *mu, double *var, double *cov)
{
    int64_t m = M->m;
    if (M->sgpr) { /* Eq. 1 as printed */
        double *K = (double *)malloc(sizeof(double) * n * m), *A = (double *)malloc(sizeof(double) * n * m);
        double *Cr = (double *)malloc(sizeof(double) * n * m), *tmp = (double *)malloc(sizeof(double) * m);
        for (int64_t a = 0; a < n; ++a) {
            sgpr_row(M, P + 3 * a, K + a * m, A + a * m, Cr + a * m, tmp);
            mu[a] = dot(A + a * m, M->y, m);
            var[a] = sgpr_cov(M, P + 3 * a, P + 3 * a, K + a * m, A + a * m, A + a * m, Cr + a * m);
        }
        if (cov)
            for (int64_t a = 0; a < n; ++a)
                for (int64_t b = 0; b < n; ++b)
                    cov[a * n + b] = sgpr_cov(M, P + 3 * a, P + 3 * b, K + a * m, A + a * m, A + b * m, Cr + b * m);
        free(K); free(A); free(Cr); free(tmp);
        return;
    }
    double *V = (double *)malloc(sizeof(double) * n * m);
#pragma omp parallel
    {
        double *kb = (double *)malloc(sizeof(double) * m);
#pragma omp for schedule(static)
        for (int64_t a = 0; a < n; ++a) {
            whiten_row(M, P + 3 * a, kb, V + a * m);
            mu[a] = dot(V + a * m, M->vy, m);
            var[a] = or_kernel_eval(M->kernel, M->ell, M->sf2, P + 3 * a, P + 3 * a) - dot(V + a * m, V + a * m, m);
        }
        free(kb);
    }
    if (cov) {
#pragma omp parallel for schedule(static)
        for (int64_t a = 0; a < n; ++a)
            for (int64_t b = 0; b < n; ++b)
                cov[a * n + b] = or_kernel_eval(M->kernel, M->ell, M->sf2, P + 3 * a, P + 3 * b) - dot(V + a * m, V + b * m, m);
    }
    free(V);
}

/* Eq. (1) as printed (SGPR form): mu = K_IM K_MM^-1 mu_M,
 * Sigma = K_II - K_IM K_MM^-1 K_MI + K_IM K_MM^-1 A_M K_MM^-1 K_MI,
 * with K_MM = K(X,X) (no noise).  Returns 0, or -1 if K_MM is not PD. */
int or_posterior_sgpr(const or_model *M, const double *muM, const double *AM, const double *P, int64_t n,
                      double *mu, double *cov)
{
    int64_t m = M->m;
    double *Kmm = (double *)malloc(sizeof(double) * m * m);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j)
            Kmm[i * m + j] = or_kernel_eval(M->kernel, M->ell, M->sf2, M->X + 3 * i, M->X + 3 * j);
    if (or_cholesky(Kmm, m) != 0) { free(Kmm); return -1; }
    /* B = K_MM^-1 K_MI  (m x n), column a solves K_MM b = k_a */
    double *B = (double *)malloc(sizeof(double) * m * n);
    double *kb = (double *)malloc(sizeof(double) * m), *t = (double *)malloc(sizeof(double) * m);
    double *Kim = (double *)malloc(sizeof(double) * n * m);
    for (int64_t a = 0; a < n; ++a) {
        for (int64_t j = 0; j < m; ++j) {
            kb[j] = or_kernel_eval(M->kernel, M->ell, M->sf2, P + 3 * a, M->X + 3 * j);
            Kim[a * m + j] = kb[j];
        }
        fwd_sub(Kmm, m, kb, t);
        back_sub_T(Kmm, m, t, kb);
        for (int64_t j = 0; j < m; ++j) B[j * n + a] = kb[j];
    }
    for (int64_t a = 0; a < n; ++a) {
        double s = 0.0;
        for (int64_t j = 0; j < m; ++j) s += B[j * n + a] * muM[j];
        mu[a] = s;
    }
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = 0; b < n; ++b) {
            double kab = or_kernel_eval(M->kernel, M->ell, M->sf2, P + 3 * a, P + 3 * b);
            double s1 = 0.0, s2 = 0.0;
            for (int64_t j = 0; j < m; ++j) s1 += Kim[a * m + j] * B[j * n + b];
            for (int64_t i = 0; i < m; ++i) {
                double ai = 0.0;
                for (int64_t j = 0; j < m; ++j) ai += AM[i * m + j] * B[j * n + b];
                s2 += B[i * n + a] * ai;
            }
            cov[a * n + b] = kab - s1 + s2;
        }
    free(Kmm); free(B); free(kb); free(t); free(Kim);
    return 0;
}

/* ---------------------------------------------------- normal distribution */

double or_norm_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Inverse standard normal CDF.  Start from Abramowitz & Stegun 26.2.23
 * (|error| < 4.5e-4) and polish with three Halley steps on Phi(x) - p, which
 * converge cubically to full double precision for p >= 1e-300. */
double or_norm_ppf(double p)
{
    if (!(p > 0.0)) return -INFINITY;
    if (!(p < 1.0)) return INFINITY;
    int upper = p > 0.5;
    double q = upper ? 1.0 - p : p; /* exact for p in (0.5,1) */
    double t = sqrt(-2.0 * log(q));
    double x = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                     (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    for (int it = 0; it < 3; ++it) {
        double f = or_norm_cdf(x) - q;
        double phi = exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
        if (!(phi > 0.0)) break;
        double dx = f / phi;
        x = x - dx / (1.0 + 0.5 * x * dx);
    }
    return upper ? -x : x;
}

/* ln Phi(g), accurate in both tails. */
static double log_norm_cdf(double g)
{
    if (g >= 0.0) return log1p(-0.5 * erfc(g / sqrt(2.0)));
    double c = 0.5 * erfc(-g / sqrt(2.0));
    if (c > 0.0) return log(c);
    /* far lower tail: ln Phi(g) ~ -g^2/2 - ln(-g sqrt(2 pi)) */
    return -0.5 * g * g - log(-g * sqrt(2.0 * M_PI));
}

/* --------------------------------------------- counter-based generators */

/* SplitMix64 (Steele, Lea & Flood 2014): the k-th output (k >= 1) of the stream
 * started at state `seed` is mix(seed + k * 0x9E3779B97F4A7C15). */
uint64_t or_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from 32 random bits: odd multiples of 2^-24, exact in binary32. */
static double u01(uint32_t x) { return (double)(((x >> 9) << 1) | 1u) * (1.0 / 16777216.0); }

/* ------------------------------------------------------ orthant estimators */

/* Rank-1 lattice generators: frac(sqrt(p)) for the first primes, as 32-bit
 * fixed-point fractions (Richtmyer lattice, Genz 1992). */
static const int PRIMES[15] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47};
static uint32_t lattice_gen(int i)
{
    double s = sqrt((double)PRIMES[i]);
    double f = s - floor(s);
    return (uint32_t)floor(f * 4294967296.0);
}

/* P(X_i <= b_i for all i), X ~ N(0, L L^T), by Genz's sequential conditioning
 * over N points of the shifted lattice (point k, dimension i:
 * U = k*G_i + D_i mod 2^32, u = u01(U), w = |2u - 1|).  shift[] holds D_i. */
double or_sov_orthant(int d, const double *L, const double *b, int64_t N, const uint32_t *shift)
{
    uint32_t G[16];
    for (int i = 0; i < d - 1; ++i) G[i] = lattice_gen(i);
    double acc = 0.0;
    double z[16];
    for (int64_t k = 0; k < N; ++k) {
        double f = 1.0;
        for (int i = 0; i < d; ++i) {
            double s = 0.0;
            for (int j = 0; j < i; ++j) s += L[i * d + j] * z[j];
            double e = or_norm_cdf((b[i] - s) / L[i * d + i]);
            f *= e;
            if (!(f > 0.0)) { f = 0.0; break; } /* the sample contributes nothing further */
            if (i < d - 1) {
                uint32_t U = (uint32_t)((uint64_t)k * G[i]) + shift[i];
                double w = fabs(2.0 * u01(U) - 1.0);
                z[i] = or_norm_ppf(w * e);
            }
        }
        acc += f;
    }
    return acc / (double)N;
}

/* Cholesky of a d x d covariance with the pivot floor used by the cell rule:
 * a pivot below `floor_` is replaced by floor_ (reading; the paper is silent). */
static void chol_floor(const double *S, int d, double floor_, double *L)
{
    for (int i = 0; i < d * d; ++i) L[i] = 0.0;
    for (int j = 0; j < d; ++j) {
        double s = S[j * d + j];
        for (int k = 0; k < j; ++k) s -= L[j * d + k] * L[j * d + k];
        if (!(s > floor_)) s = floor_;
        double ljj = sqrt(s);
        L[j * d + j] = ljj;
        for (int i = j + 1; i < d; ++i) {
            double t = S[i * d + j];
            for (int k = 0; k < j; ++k) t -= L[i * d + k] * L[j * d + k];
            L[i * d + j] = t / ljj;
        }
    }
}

#define EST_SOV 0
#define EST_MC 1
#define EST_INDEP 2
#define EST_EDGE 3
#define EST_SOV_ORD 4

/* One orthant, P(s (theta - Y_c) > 0 for every corner c) with s = +1 (all below) or -1 (all
 * above), by the lattice rule of or_sov_orthant with the variables taken in ascending order of
 * their standardised thresholds s (theta - mu_c) / sigma_c (ties: lower index first), the
 * ordering Genz and Bretz recommend without its conditional updates.  The corner most likely to
 * leave the orthant comes first, so its factor, exact and independent of the sample, carries
 * most of the probability of strongly correlated corners and the lattice sees a flat integrand.
 * Sj: jittered covariance; floor_: the Cholesky pivot floor. */
static double sov_orthant_ordered(int d, const double *Sj, const double *mu, double theta, double s, double floor_,
                                  int64_t N, const uint32_t *sh)
{
    int perm[16];
    double key[16], Sp[256], Lp[256], bp[16];
    for (int i = 0; i < d; ++i) {
        key[i] = (s * (theta - mu[i])) / sqrt(Sj[i * d + i]);
        perm[i] = i;
    }
    for (int i = 1; i < d; ++i) { /* insertion sort, stable */
        int v = perm[i], j = i;
        while (j > 0 && key[v] < key[perm[j - 1]]) { perm[j] = perm[j - 1]; --j; }
        perm[j] = v;
    }
    for (int a = 0; a < d; ++a) {
        bp[a] = s * (theta - mu[perm[a]]);
        for (int b = 0; b < d; ++b) Sp[a * d + b] = Sj[perm[a] * d + perm[b]];
    }
    chol_floor(Sp, d, floor_, Lp);
    return or_sov_orthant(d, Lp, bp, N, sh);
}

/* P(X1 < a, X2 < b) for a standard bivariate normal with correlation r (|r| < 1): the
 * integral over x1 < a of phi(x1) P(X2 < b | X1 = x1) = phi(x1) Phi((b - r x1) / sqrt(1 - r^2)),
 * by adaptive Simpson on [-40, a] (the mass below -40 is under 1e-300). */
static double bvn_integrand(double t, double b, double r, double s)
{
    return exp(-0.5 * t * t) / sqrt(2.0 * M_PI) * or_norm_cdf((b - r * t) / s);
}

static double simpson_rec(double lo, double hi, double flo, double fmid, double fhi, double whole, double tol,
                          int depth, double b, double r, double s)
{
    double mid = 0.5 * (lo + hi), lm = 0.5 * (lo + mid), rm = 0.5 * (mid + hi);
    double flm = bvn_integrand(lm, b, r, s), frm = bvn_integrand(rm, b, r, s);
    double left = (mid - lo) / 6.0 * (flo + 4.0 * flm + fmid), right = (hi - mid) / 6.0 * (fmid + 4.0 * frm + fhi);
    double diff = left + right - whole;
    if (depth <= 0 || fabs(diff) <= 15.0 * tol) return left + right + diff / 15.0;
    return simpson_rec(lo, mid, flo, flm, fmid, left, 0.5 * tol, depth - 1, b, r, s) +
           simpson_rec(mid, hi, fmid, frm, fhi, right, 0.5 * tol, depth - 1, b, r, s);
}

double or_bvn_lower(double a, double b, double r)
{
    double s = sqrt(1.0 - r * r);
    double lo = -40.0, hi = a < 40.0 ? a : 40.0;
    if (!(hi > lo)) return 0.0;
    /* split at the kink of the conditional CDF (x1 = b / r) so each piece is smooth */
    double cuts[3] = {lo, hi, hi};
    int nc = 2;
    if (r != 0.0) {
        double k = b / r;
        if (k > lo && k < hi) { cuts[1] = k; cuts[2] = hi; nc = 3; }
    }
    double total = 0.0;
    for (int i = 0; i + 1 < nc; ++i) {
        double x0 = cuts[i], x1 = cuts[i + 1];
        double f0 = bvn_integrand(x0, b, r, s), f1 = bvn_integrand(x1, b, r, s), fm = bvn_integrand(0.5 * (x0 + x1), b, r, s);
        double whole = (x1 - x0) / 6.0 * (f0 + 4.0 * fm + f1);
        total += simpson_rec(x0, x1, f0, fm, f1, whole, 1e-15, 50, b, r, s);
    }
    return total;
}

/* Cell level-crossing probability for d corner variables (d = 8 for a cell):
 * LCP = 1 - P(all < theta) - P(all > theta)  (Sec. 4).
 * Readings (paper silent): Sigma += tau * max diag * I; pivot floor
 * 1e-3 * tau * max diag; if sum_c P(Y_c > theta) or sum_c P(Y_c < theta) is below
 * skip_eps, Boole's inequality bounds the LCP by it and the result is 0; a
 * cell whose largest variance is below 1e-30 is deterministic; a cell with a
 * variance that is not positive after the jitter is no Gaussian and gets NaN.
 * est = EST_SOV: shifts of cell `cell` are SplitMix64 outputs 8*cell+i+1, top
 * 32 bits.  est = EST_MC: Philox-4x32-10 with key (seed lo, seed hi) and counter
 * (sample, cell lo, cell hi, r), r = 0,1 giving 8 normals by Box-Muller.
 * est = EST_INDEP: the corners taken as independent (the closed forms of the
 * uncorrelated uncertainty models the paper reviews in Sec. 2.2):
 * 1 - prod_c P(Y_c < theta) - prod_c P(Y_c > theta).
 * est = EST_EDGE: Pothkow et al.'s approximation (Sec. 2.2, Sec. 9): the largest
 * crossing probability 1 - P(Y_i < theta, Y_j < theta) - P(Y_i > theta, Y_j > theta)
 * over the cell's edges (corner pairs i, j = i ^ 2^a; 12 for d = 8).
 * est = EST_SOV_ORD: EST_SOV with each orthant's variables reordered
 * (sov_orthant_ordered); the same lattice shifts. */
double or_cell_lcp(int d, const double *mu, const double *S, double theta, int est, int64_t N,
                   uint64_t seed, uint64_t cell, double tau, double skip_eps)
{
    double Sj[256], L[256];
    double maxdiag = 0.0;
    for (int i = 0; i < d; ++i) if (S[i * d + i] > maxdiag) maxdiag = S[i * d + i];
    if (!(maxdiag > 1e-30)) {
        int lo = 1, hi = 1;
        for (int i = 0; i < d; ++i) { if (!(mu[i] < theta)) lo = 0; if (!(mu[i] > theta)) hi = 0; }
        return (lo || hi) ? 0.0 : 1.0;
    }
    double jit = tau * maxdiag;
    for (int i = 0; i < d * d; ++i) Sj[i] = S[i];
    for (int i = 0; i < d; ++i) Sj[i * d + i] += jit;
    for (int i = 0; i < d; ++i)
        if (!(Sj[i * d + i] > 0.0)) return NAN;
    double s_above = 0.0, s_below = 0.0;
    for (int i = 0; i < d; ++i) {
        double sd = sqrt(Sj[i * d + i]);
        s_above += or_norm_cdf((mu[i] - theta) / sd);
        s_below += or_norm_cdf((theta - mu[i]) / sd);
    }
    if (s_above < skip_eps || s_below < skip_eps) return 0.0;
    if (est == EST_INDEP) {
        double plo = 1.0, phi = 1.0;
        for (int i = 0; i < d; ++i) {
            double sd = sqrt(Sj[i * d + i]);
            plo *= or_norm_cdf((theta - mu[i]) / sd);
            phi *= or_norm_cdf((mu[i] - theta) / sd);
        }
        return 1.0 - plo - phi;
    }
    if (est == EST_EDGE) {
        double best = 0.0;
        for (int i = 0; i < d; ++i)
            for (int a = 0; (1 << a) < d; ++a) {
                int j = i ^ (1 << a);
                if (j < i || j >= d) continue;
                double si = sqrt(Sj[i * d + i]), sj = sqrt(Sj[j * d + j]);
                double r = Sj[i * d + j] / (si * sj);
                double zi = (theta - mu[i]) / si, zj = (theta - mu[j]) / sj;
                double pe = 1.0 - or_bvn_lower(zi, zj, r) - or_bvn_lower(-zi, -zj, r);
                if (pe > best) best = pe;
            }
        return best;
    }
    if (est == EST_SOV_ORD) {
        uint32_t sh[16];
        for (int i = 0; i < d - 1; ++i) sh[i] = (uint32_t)(or_splitmix64(seed, (uint64_t)cell * 8 + i + 1) >> 32);
        double v = 1.0 - sov_orthant_ordered(d, Sj, mu, theta, 1.0, 1e-3 * jit, N, sh) -
                   sov_orthant_ordered(d, Sj, mu, theta, -1.0, 1e-3 * jit, N, sh);
        return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    }
    chol_floor(Sj, d, 1e-3 * jit, L);
    double p_lo, p_hi;
    if (est == EST_SOV) {
        uint32_t sh[16];
        for (int i = 0; i < d - 1; ++i) sh[i] = (uint32_t)(or_splitmix64(seed, (uint64_t)cell * 8 + i + 1) >> 32);
        double b[16];
        for (int i = 0; i < d; ++i) b[i] = theta - mu[i];
        p_lo = or_sov_orthant(d, L, b, N, sh);
        for (int i = 0; i < d; ++i) b[i] = mu[i] - theta;
        p_hi = or_sov_orthant(d, L, b, N, sh);
        double v = 1.0 - p_lo - p_hi;
        return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    }
    /* Monte Carlo: fraction of samples whose corners are not all on one side. */
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t crossed = 0;
    double z[16], yv[16];
    for (int64_t k = 0; k < N; ++k) {
        for (int r = 0; r < (d + 3) / 4; ++r) {
            uint32_t ctr[4] = {(uint32_t)k, (uint32_t)cell, (uint32_t)(cell >> 32), (uint32_t)r}, o[4];
            or_philox4x32_10(ctr, key, o);
            for (int p = 0; p < 2; ++p) {
                double u1 = u01(o[2 * p]), u2 = u01(o[2 * p + 1]);
                double rr = sqrt(-2.0 * log(u1));
                int i0 = 4 * r + 2 * p;
                if (i0 < 16) z[i0] = rr * cos(2.0 * M_PI * u2);
                if (i0 + 1 < 16) z[i0 + 1] = rr * sin(2.0 * M_PI * u2);
            }
        }
        int all_lo = 1, all_hi = 1;
        for (int i = 0; i < d; ++i) {
            double s = mu[i];
            for (int j = 0; j <= i; ++j) s += L[i * d + j] * z[j];
            yv[i] = s;
            if (!(s < theta)) all_lo = 0;
            if (!(s > theta)) all_hi = 0;
        }
        if (!(all_lo || all_hi)) ++crossed;
    }
    (void)p_lo; (void)p_hi;
    return (double)crossed / (double)N;
}

/* ------------------------------------------------------------------ grid */

typedef struct {
    double lo[3], hi[3];
    int64_t n[3];
} or_grid;

static double grid_h(const or_grid *g, int d) { return (g->hi[d] - g->lo[d]) / (double)(g->n[d] - 1); }
static double grid_x(const or_grid *g, int d, int64_t i) { return g->lo[d] + (double)i * grid_h(g, d); }

/* Forward neighbour offsets: the lexicographically positive half of
 * {-1,0,1}^3 \ 0, in this order; stats slot 2+e holds cov(p, p+off[e]). */
static const int OFF13[13][3] = {
    {1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1}, {1, 0, 0}, {1, 0, 1}, {1, 1, -1}, {1, 1, 0}, {1, 1, 1},
    {0, 1, -1}, {0, 1, 0}, {0, 1, 1}, {0, 0, 1}};

/* Posterior stats for the grid points in the index box [i0, i1):
 * out[p*15 + 0] = mu, [1] = var, [2+e] = cov(p, p+OFF13[e]) (NaN off-grid).
 * Points are ordered x-fastest inside the box.  Whitened rows are computed for
 * the box grown by one point on each side. */
static void sgpr_stats15_block(const or_model *M, const or_grid *g, const int64_t *i0, const int64_t *i1,
                               double *out);

void or_stats15_block(const or_model *M, const or_grid *g, const int64_t *i0, const int64_t *i1, double *out)
{
    if (M->sgpr) { sgpr_stats15_block(M, g, i0, i1, out); return; }
    int64_t m = M->m;
    int64_t e0[3], e1[3], en[3];
    for (int d = 0; d < 3; ++d) {
        e0[d] = i0[d] > 0 ? i0[d] - 1 : 0;
        e1[d] = i1[d] < g->n[d] ? i1[d] + 1 : g->n[d];
        en[d] = e1[d] - e0[d];
    }
    int64_t ne = en[0] * en[1] * en[2];
    double *V = (double *)malloc(sizeof(double) * ne * m);
#pragma omp parallel
    {
        double *kb = (double *)malloc(sizeof(double) * m);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < ne; ++q) {
            int64_t a = e0[0] + q % en[0], b = e0[1] + (q / en[0]) % en[1], c = e0[2] + q / (en[0] * en[1]);
            double x[3] = {grid_x(g, 0, a), grid_x(g, 1, b), grid_x(g, 2, c)};
            whiten_row(M, x, kb, V + q * m);
        }
        free(kb);
    }
    int64_t bn[3] = {i1[0] - i0[0], i1[1] - i0[1], i1[2] - i0[2]};
    int64_t nb = bn[0] * bn[1] * bn[2];
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < nb; ++p) {
        int64_t a = i0[0] + p % bn[0], b = i0[1] + (p / bn[0]) % bn[1], c = i0[2] + p / (bn[0] * bn[1]);
        int64_t q = (a - e0[0]) + en[0] * ((b - e0[1]) + en[1] * (c - e0[2]));
        double x[3] = {grid_x(g, 0, a), grid_x(g, 1, b), grid_x(g, 2, c)};
        double *o = out + p * 15;
        o[0] = dot(V + q * m, M->vy, m);
        o[1] = or_kernel_eval(M->kernel, M->ell, M->sf2, x, x) - dot(V + q * m, V + q * m, m);
        for (int e = 0; e < 13; ++e) {
            int64_t a2 = a + OFF13[e][0], b2 = b + OFF13[e][1], c2 = c + OFF13[e][2];
            if (a2 < 0 || b2 < 0 || c2 < 0 || a2 >= g->n[0] || b2 >= g->n[1] || c2 >= g->n[2]) { o[2 + e] = NAN; continue; }
            int64_t q2 = (a2 - e0[0]) + en[0] * ((b2 - e0[1]) + en[1] * (c2 - e0[2]));
            double x2[3] = {grid_x(g, 0, a2), grid_x(g, 1, b2), grid_x(g, 2, c2)};
            o[2 + e] = or_kernel_eval(M->kernel, M->ell, M->sf2, x, x2) - dot(V + q * m, V + q2 * m, m);
        }
    }
    free(V);
}

/* or_stats15_block for an SGPR model: Eq. 1 as printed, from the rows (k, K_MM^-1 k, A_M K_MM^-1 k)
 * of the box grown by one point on each side. */
static void sgpr_stats15_block(const or_model *M, const or_grid *g, const int64_t *i0, const int64_t *i1,
                               double *out)
{
    int64_t m = M->m;
    int64_t e0[3], e1[3], en[3];
    for (int d = 0; d < 3; ++d) {
        e0[d] = i0[d] > 0 ? i0[d] - 1 : 0;
        e1[d] = i1[d] < g->n[d] ? i1[d] + 1 : g->n[d];
        en[d] = e1[d] - e0[d];
    }
    int64_t ne = en[0] * en[1] * en[2];
    double *K = (double *)malloc(sizeof(double) * ne * m), *A = (double *)malloc(sizeof(double) * ne * m);
    double *Cr = (double *)malloc(sizeof(double) * ne * m);
#pragma omp parallel
    {
        double *tmp = (double *)malloc(sizeof(double) * m);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < ne; ++q) {
            int64_t a = e0[0] + q % en[0], b = e0[1] + (q / en[0]) % en[1], c = e0[2] + q / (en[0] * en[1]);
            double x[3] = {grid_x(g, 0, a), grid_x(g, 1, b), grid_x(g, 2, c)};
            sgpr_row(M, x, K + q * m, A + q * m, Cr + q * m, tmp);
        }
        free(tmp);
    }
    int64_t bn[3] = {i1[0] - i0[0], i1[1] - i0[1], i1[2] - i0[2]};
    int64_t nb = bn[0] * bn[1] * bn[2];
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < nb; ++p) {
        int64_t a = i0[0] + p % bn[0], b = i0[1] + (p / bn[0]) % bn[1], c = i0[2] + p / (bn[0] * bn[1]);
        int64_t q = (a - e0[0]) + en[0] * ((b - e0[1]) + en[1] * (c - e0[2]));
        double x[3] = {grid_x(g, 0, a), grid_x(g, 1, b), grid_x(g, 2, c)};
        double *o = out + p * 15;
        o[0] = dot(A + q * m, M->y, m);
        o[1] = sgpr_cov(M, x, x, K + q * m, A + q * m, A + q * m, Cr + q * m);
        for (int e = 0; e < 13; ++e) {
            int64_t a2 = a + OFF13[e][0], b2 = b + OFF13[e][1], c2 = c + OFF13[e][2];
            if (a2 < 0 || b2 < 0 || c2 < 0 || a2 >= g->n[0] || b2 >= g->n[1] || c2 >= g->n[2]) { o[2 + e] = NAN; continue; }
            int64_t q2 = (a2 - e0[0]) + en[0] * ((b2 - e0[1]) + en[1] * (c2 - e0[2]));
            double x2[3] = {grid_x(g, 0, a2), grid_x(g, 1, b2), grid_x(g, 2, c2)};
            o[2 + e] = sgpr_cov(M, x, x2, K + q * m, A + q * m, A + q2 * m, Cr + q2 * m);
        }
    }
    free(K); free(A); free(Cr);
}

/* or_lcp_block for an SGPR model: the corners' (mu_8, Sigma_8) from Eq. 1 as printed. */
static void sgpr_lcp_block(const or_model *M, const or_grid *g, double theta, int est, int64_t N, uint64_t seed,
                           double tau, double skip_eps, const int64_t *c0, const int64_t *c1, double *out);

/* LCP of the cells whose min-corner index lies in the box [c0, c1), written
 * x-fastest inside the box.  The 8x8 corner covariance of each cell is formed
 * directly as K_88 - V_8 V_8^T from the corners' whitened rows (Sec. 4, the
 * baseline dense method).  Corner c = bx + 2 by + 4 bz.  The cell index used
 * to key the estimator is the linear index of the cell in the whole grid. */
void or_lcp_block(const or_model *M, const or_grid *g, double theta, int est, int64_t N, uint64_t seed,
                  double tau, double skip_eps, const int64_t *c0, const int64_t *c1, double *out)
{
    if (M->sgpr) { sgpr_lcp_block(M, g, theta, est, N, seed, tau, skip_eps, c0, c1, out); return; }
    int64_t m = M->m;
    int64_t pn[3];
    for (int d = 0; d < 3; ++d) pn[d] = c1[d] - c0[d] + 1;
    int64_t np = pn[0] * pn[1] * pn[2];
    double *V = (double *)malloc(sizeof(double) * np * m);
#pragma omp parallel
    {
        double *kb = (double *)malloc(sizeof(double) * m);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < np; ++q) {
            int64_t a = c0[0] + q % pn[0], b = c0[1] + (q / pn[0]) % pn[1], c = c0[2] + q / (pn[0] * pn[1]);
            double x[3] = {grid_x(g, 0, a), grid_x(g, 1, b), grid_x(g, 2, c)};
            whiten_row(M, x, kb, V + q * m);
        }
        free(kb);
    }
    int64_t cn[3] = {c1[0] - c0[0], c1[1] - c0[1], c1[2] - c0[2]};
    int64_t nc = cn[0] * cn[1] * cn[2];
    int64_t gc[3] = {g->n[0] - 1, g->n[1] - 1, g->n[2] - 1};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < nc; ++p) {
        int64_t a = c0[0] + p % cn[0], b = c0[1] + (p / cn[0]) % cn[1], c = c0[2] + p / (cn[0] * cn[1]);
        int64_t q[8];
        double x[8][3], mu[8], S[64];
        for (int cc = 0; cc < 8; ++cc) {
            int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
            q[cc] = (a + bx - c0[0]) + pn[0] * ((b + by - c0[1]) + pn[1] * (c + bz - c0[2]));
            x[cc][0] = grid_x(g, 0, a + bx); x[cc][1] = grid_x(g, 1, b + by); x[cc][2] = grid_x(g, 2, c + bz);
            mu[cc] = dot(V + q[cc] * m, M->vy, m);
        }
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j <= i; ++j) {
                double s = or_kernel_eval(M->kernel, M->ell, M->sf2, x[i], x[j]) - dot(V + q[i] * m, V + q[j] * m, m);
                S[i * 8 + j] = s; S[j * 8 + i] = s;
            }
        uint64_t cell = (uint64_t)(a + gc[0] * (b + gc[1] * c));
        out[p] = or_cell_lcp(8, mu, S, theta, est, N, seed, cell, tau, skip_eps);
    }
    free(V);
}

static void sgpr_lcp_block(const or_model *M, const or_grid *g, double theta, int est, int64_t N, uint64_t seed,
                           double tau, double skip_eps, const int64_t *c0, const int64_t *c1, double *out)
{
    int64_t m = M->m;
    int64_t pn[3];
    for (int d = 0; d < 3; ++d) pn[d] = c1[d] - c0[d] + 1;
    int64_t np = pn[0] * pn[1] * pn[2];
    double *K = (double *)malloc(sizeof(double) * np * m), *A = (double *)malloc(sizeof(double) * np * m);
    double *Cr = (double *)malloc(sizeof(double) * np * m);
#pragma omp parallel
    {
        double *tmp = (double *)malloc(sizeof(double) * m);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < np; ++q) {
            int64_t a = c0[0] + q % pn[0], b = c0[1] + (q / pn[0]) % pn[1], c = c0[2] + q / (pn[0] * pn[1]);
            double x[3] = {grid_x(g, 0, a), grid_x(g, 1, b), grid_x(g, 2, c)};
            sgpr_row(M, x, K + q * m, A + q * m, Cr + q * m, tmp);
        }
        free(tmp);
    }
    int64_t cn[3] = {c1[0] - c0[0], c1[1] - c0[1], c1[2] - c0[2]};
    int64_t nc = cn[0] * cn[1] * cn[2];
    int64_t gc[3] = {g->n[0] - 1, g->n[1] - 1, g->n[2] - 1};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < nc; ++p) {
        int64_t a = c0[0] + p % cn[0], b = c0[1] + (p / cn[0]) % cn[1], c = c0[2] + p / (cn[0] * cn[1]);
        int64_t q[8];
        double x[8][3], mu[8], S[64];
        for (int cc = 0; cc < 8; ++cc) {
            int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
            q[cc] = (a + bx - c0[0]) + pn[0] * ((b + by - c0[1]) + pn[1] * (c + bz - c0[2]));
            x[cc][0] = grid_x(g, 0, a + bx); x[cc][1] = grid_x(g, 1, b + by); x[cc][2] = grid_x(g, 2, c + bz);
            mu[cc] = dot(A + q[cc] * m, M->y, m);
        }
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j <= i; ++j) {
                double s = sgpr_cov(M, x[i], x[j], K + q[i] * m, A + q[i] * m, A + q[j] * m, Cr + q[j] * m);
                S[i * 8 + j] = s; S[j * 8 + i] = s;
            }
        uint64_t cell = (uint64_t)(a + gc[0] * (b + gc[1] * c));
        out[p] = or_cell_lcp(8, mu, S, theta, est, N, seed, cell, tau, skip_eps);
    }
    free(K); free(A); free(Cr);
}

/* ---------------------------------------------------- regional bound, octree */

/* g(x) = side * (theta - mu(x)) / sigma(x) and its gradient; side = +1 gives
 * F = Phi(g) = P(Y < theta), side = -1 gives 1 - F = P(Y > theta) (Sec. 5.1). */
static double eval_g(const or_model *M, const double *x, double theta, int side, double grad[3],
                     double *kb, double *dk, double *v, double *P)
{
    int64_t m = M->m;
    for (int64_t j = 0; j < m; ++j) kernel_grad(M->kernel, M->ell, M->sf2, x, M->X + 3 * j, kb + j, dk + 3 * j);
    double mu, var;
    if (M->sgpr) {
        /* Eq. 1: mu = k^T K_MM^-1 mu_M; var = k(x,x) - k^T a + a^T A_M a with a = K_MM^-1 k;
         * d var / dx = -2 (dk)^T (a - K_MM^-1 A_M a), so P = a - K_MM^-1 A_M a plays the role of
         * Kt^-1 k below. */
        double *a = (double *)malloc(sizeof(double) * m), *c = (double *)malloc(sizeof(double) * m);
        fwd_sub(M->L, m, kb, v);
        back_sub_T(M->L, m, v, a);
        for (int64_t i = 0; i < m; ++i) c[i] = dot(M->A + i * m, a, m);
        mu = dot(a, M->y, m);
        var = or_kernel_eval(M->kernel, M->ell, M->sf2, x, x) - dot(kb, a, m) + dot(a, c, m);
        fwd_sub(M->L, m, c, v);
        back_sub_T(M->L, m, v, P);
        for (int64_t j = 0; j < m; ++j) P[j] = a[j] - P[j];
        free(a); free(c);
    } else {
        fwd_sub(M->L, m, kb, v);
        mu = dot(v, M->vy, m);
        var = or_kernel_eval(M->kernel, M->ell, M->sf2, x, x) - dot(v, v, m);
    }
    double fl = 1e-12 * M->sf2;
    if (!(var > fl)) var = fl;
    double sd = sqrt(var);
    if (!M->sgpr) back_sub_T(M->L, m, v, P); /* P = Kt^-1 k */
    double gmu[3] = {0, 0, 0}, gvar[3] = {0, 0, 0};
    for (int64_t j = 0; j < m; ++j)
        for (int d = 0; d < 3; ++d) {
            gmu[d] += dk[3 * j + d] * M->alpha[j];
            gvar[d] += -2.0 * dk[3 * j + d] * P[j];
        }
    double gl = (theta - mu) / sd;
    for (int d = 0; d < 3; ++d) {
        double gd = -gmu[d] / sd - gl * gvar[d] / (2.0 * var);
        grad[d] = side * gd;
    }
    return side * gl;
}

/* Node geometry at level l of a depth-D octree over the cell grid: node (i,j,k)
 * spans cells [i s, (i+1) s) per axis, s = 2^(D-l), i.e. grid points
 * [i s, min((i+1) s, n-1)]; its box is the span of those points.
 * kd != 0: the K-D tree of Sec. 9, which splits one axis per level in turn (x, y, z):
 * at level l (0 .. 3D) axis d has been halved floor((l + 2 - d) / 3) times, so its extent is
 * s_d = 2^(D - floor((l + 2 - d) / 3)). */
static int64_t axis_extent(int D, int l, int kd, int d)
{
    return (int64_t)1 << (D - (kd ? (l + 2 - d) / 3 : l));
}

static void node_geom(const or_grid *g, int D, int l, int kd, const int64_t ijk[3], int64_t p0[3], int64_t p1[3],
                      double blo[3], double bhi[3])
{
    for (int d = 0; d < 3; ++d) {
        int64_t s = axis_extent(D, l, kd, d);
        p0[d] = ijk[d] * s;
        p1[d] = (ijk[d] + 1) * s;
        if (p1[d] > g->n[d] - 1) p1[d] = g->n[d] - 1;
        blo[d] = grid_x(g, d, p0[d]);
        bhi[d] = grid_x(g, d, p1[d]);
    }
}

/* min over the node of g(x) for one side.  Reading of the paper's L-BFGS-B
 * step (the minimiser is not specified beyond "quasi-Newton"): when the node
 * has at most 3 grid points per axis, the minimum is taken exactly over its
 * grid points; otherwise over the continuous box, starting from the best of the
 * 3x3x3 lattice (corners, edge/face midpoints, centre; first in x-fastest order
 * on ties) and taking T projected steps x' = clamp(x + eta_t * w * u/|u|_inf),
 * u = -grad g * w (w = box widths), eta_t = 0.25 * 2^-t, each kept only if it
 * lowers g. */
static double node_min_g(const or_model *M, const or_grid *g, const int64_t p0[3], const int64_t p1[3],
                         const double blo[3], const double bhi[3], double theta, int side, int T,
                         double *kb, double *dk, double *v, double *P, double *xbest)
{
    double grad[3];
    int small = 1;
    for (int d = 0; d < 3; ++d) if (p1[d] - p0[d] + 1 > 3) small = 0;
    if (small) {
        double best = INFINITY;
        for (int64_t c = p0[2]; c <= p1[2]; ++c)
            for (int64_t b = p0[1]; b <= p1[1]; ++b)
                for (int64_t a = p0[0]; a <= p1[0]; ++a) {
                    double x[3] = {grid_x(g, 0, a), grid_x(g, 1, b), grid_x(g, 2, c)};
                    double val = eval_g(M, x, theta, side, grad, kb, dk, v, P);
                    if (val < best) {
                        best = val;
                        if (xbest) for (int d = 0; d < 3; ++d) xbest[d] = x[d];
                    }
                }
        return best;
    }
    double bx[3], bestg = INFINITY, bestgrad[3] = {0, 0, 0};
    for (int t = 0; t < 27; ++t) {
        int ia = t % 3, ib = (t / 3) % 3, ic = t / 9;
        int id[3] = {ia, ib, ic};
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = blo[d] + 0.5 * (double)id[d] * (bhi[d] - blo[d]);
        double val = eval_g(M, x, theta, side, grad, kb, dk, v, P);
        if (val < bestg) { bestg = val; for (int d = 0; d < 3; ++d) { bx[d] = x[d]; bestgrad[d] = grad[d]; } }
    }
    for (int t = 0; t < T; ++t) {
        double w[3], u[3], un = 0.0;
        for (int d = 0; d < 3; ++d) {
            w[d] = bhi[d] - blo[d];
            u[d] = -bestgrad[d] * w[d];
            if (fabs(u[d]) > un) un = fabs(u[d]);
        }
        if (!(un > 0.0)) break;
        double eta = 0.25 * ldexp(1.0, -t), xc[3];
        for (int d = 0; d < 3; ++d) {
            double xn = bx[d] + eta * w[d] * u[d] / un;
            xc[d] = xn < blo[d] ? blo[d] : (xn > bhi[d] ? bhi[d] : xn);
        }
        double val = eval_g(M, xc, theta, side, grad, kb, dk, v, P);
        if (val < bestg) { bestg = val; for (int d = 0; d < 3; ++d) { bx[d] = xc[d]; bestgrad[d] = grad[d]; } }
    }
    if (xbest) for (int d = 0; d < 3; ++d) xbest[d] = bx[d];
    return bestg;
}

/* The local model of Sec. 5.2 for a node box [blo, bhi]: the same model restricted to the
 * observations (inducing points) M' inside the box enlarged by beta * l_d on each side of axis d
 * (the local set Algorithm 1 passes down the tree; a child's enlarged box lies inside its
 * parent's, so filtering M by the child's box gives the same set).  Plain GPR: the GP conditioned
 * on y at M' only; SGPR: Eq. 1 with mu_M', A_M'M' and K_M'M'.  Returns NULL when M' = M (use the
 * full model); an empty M' gives the prior. */
static or_model *local_model(const or_model *M, const double blo[3], const double bhi[3], double beta)
{
    int64_t m = M->m, c = 0;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (m > 0 ? m : 1));
    for (int64_t i = 0; i < m; ++i) {
        const double *x = M->X + 3 * i;
        int in = 1;
        for (int d = 0; d < 3; ++d)
            if (x[d] < blo[d] - beta * M->ell[d] || x[d] > bhi[d] + beta * M->ell[d]) in = 0;
        if (in) idx[c++] = i;
    }
    if (c == m) { free(idx); return NULL; }
    double *X = (double *)malloc(sizeof(double) * 3 * (c > 0 ? c : 1));
    double *y = (double *)malloc(sizeof(double) * (c > 0 ? c : 1));
    for (int64_t a = 0; a < c; ++a) {
        for (int d = 0; d < 3; ++d) X[3 * a + d] = M->X[3 * idx[a] + d];
        y[a] = M->y[idx[a]];
    }
    or_model *L;
    if (M->sgpr) {
        double *A = (double *)malloc(sizeof(double) * (c > 0 ? c * c : 1));
        for (int64_t a = 0; a < c; ++a)
            for (int64_t b = 0; b < c; ++b) A[a * c + b] = M->A[idx[a] * m + idx[b]];
        L = or_model_create_sgpr(X, y, A, c, M->kernel, M->ell, M->sf2, M->kmm_jitter);
        free(A);
    } else {
        L = or_model_create(X, y, c, M->kernel, M->ell, M->sf2, M->sn2);
    }
    free(X); free(y); free(idx);
    return L;
}

/* One level of Algorithm 1 for `count` nodes (packed i | j<<21 | k<<42).
 * Per node: decision[q] = 0 (drop), 1 (subdivide: p1 > alpha and p2 > alpha),
 * 2 (subdivide: bound > alpha); bound[q] = the upper bound used (NaN for 1);
 * side[q] = 0 both sides, 1 lower only (p2 <= alpha), 2 upper only (p1 <= alpha).
 * The p-test uses the observations inside the closed node box with the latent
 * posterior at the observations.  d = number of grid points in the node.
 * beta >= 0: the bound is minimised on the node's local model (local_model above; beta in units
 * of the length scales); beta < 0: on the full model.  kd: the level of a K-D tree (node_geom). */
void or_octree_level(const or_model *M, const or_grid *g, int D, int l, int kd, double theta, double alpha, int T,
                     double beta, const int64_t *nodes, int64_t count, int8_t *decision, double *bound,
                     int8_t *side_out)
{
    int64_t m = M->m;
    int8_t *flo = (int8_t *)malloc((size_t)m), *fhi = (int8_t *)malloc((size_t)m);
    for (int64_t i = 0; i < m; ++i) {
        double sd = sqrt(M->var_obs[i]);
        flo[i] = or_norm_cdf((theta - M->mu_obs[i]) / sd) > alpha;
        fhi[i] = or_norm_cdf((M->mu_obs[i] - theta) / sd) > alpha;
    }
#pragma omp parallel
    {
        double *kb = (double *)malloc(sizeof(double) * m), *dk = (double *)malloc(sizeof(double) * 3 * m);
        double *v = (double *)malloc(sizeof(double) * m), *P = (double *)malloc(sizeof(double) * m);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < count; ++q) {
            int64_t ijk[3] = {nodes[q] & 0x1FFFFF, (nodes[q] >> 21) & 0x1FFFFF, (nodes[q] >> 42) & 0x1FFFFF};
            int64_t p0[3], p1[3];
            double blo[3], bhi[3];
            node_geom(g, D, l, kd, ijk, p0, p1, blo, bhi);
            int any = 0, anylo = 0, anyhi = 0;
            for (int64_t i = 0; i < m; ++i) {
                const double *x = M->X + 3 * i;
                if (x[0] >= blo[0] && x[0] <= bhi[0] && x[1] >= blo[1] && x[1] <= bhi[1] && x[2] >= blo[2] && x[2] <= bhi[2]) {
                    any = 1; anylo |= flo[i]; anyhi |= fhi[i];
                }
            }
            if (any && anylo && anyhi) { decision[q] = 1; bound[q] = NAN; side_out[q] = 0; continue; }
            int do_lo, do_hi;
            if (!any || (!anylo && !anyhi)) { do_lo = 1; do_hi = 1; }
            else if (!anyhi) { do_lo = 1; do_hi = 0; }
            else { do_lo = 0; do_hi = 1; }
            double dcount = (double)((p1[0] - p0[0] + 1) * (p1[1] - p0[1] + 1) * (p1[2] - p0[2] + 1));
            double lB_lo = -INFINITY, lB_hi = -INFINITY; /* ln B; B = 0 when the side is not used */
            or_model *Lm = beta >= 0.0 ? local_model(M, blo, bhi, beta) : NULL;
            const or_model *E = Lm ? Lm : M;
            if (do_lo) lB_lo = log_norm_cdf(node_min_g(E, g, p0, p1, blo, bhi, theta, +1, T, kb, dk, v, P, NULL));
            if (do_hi) lB_hi = log_norm_cdf(node_min_g(E, g, p0, p1, blo, bhi, theta, -1, T, kb, dk, v, P, NULL));
            if (Lm) or_model_destroy(Lm);
            double bnd;
            if (do_lo && do_hi) bnd = -expm1(dcount * lB_lo) - exp(dcount * lB_hi);
            else if (do_lo) bnd = -expm1(dcount * lB_lo);
            else bnd = -expm1(dcount * lB_hi);
            bound[q] = bnd;
            side_out[q] = (int8_t)((do_lo && do_hi) ? 0 : (do_lo ? 1 : 2));
            decision[q] = bnd > alpha ? 2 : 0;
        }
        free(kb); free(dk); free(v); free(P);
    }
    free(flo); free(fhi);
}

/* The box minimiser of one node on its own (test hook for the minimiser pins): node
 * (i | j<<21 | k<<42) at level l of a depth-D octree (kd: of the K-D tree), one side; returns min g and writes the
 * point where it was found to x_out, and the node box to box_lo / box_hi (all nullable). */
double or_node_min(const or_model *M, const or_grid *g, int D, int l, int kd, int64_t node, double theta, int side,
                   int T, double *x_out, double *box_lo, double *box_hi)
{
    int64_t m = M->m;
    int64_t ijk[3] = {node & 0x1FFFFF, (node >> 21) & 0x1FFFFF, (node >> 42) & 0x1FFFFF};
    int64_t p0[3], p1[3];
    double blo[3], bhi[3], xb[3];
    node_geom(g, D, l, kd, ijk, p0, p1, blo, bhi);
    double *kb = (double *)malloc(sizeof(double) * m), *dk = (double *)malloc(sizeof(double) * 3 * m);
    double *v = (double *)malloc(sizeof(double) * m), *P = (double *)malloc(sizeof(double) * m);
    double r = node_min_g(M, g, p0, p1, blo, bhi, theta, side, T, kb, dk, v, P, xb);
    free(kb); free(dk); free(v); free(P);
    for (int d = 0; d < 3; ++d) {
        if (x_out) x_out[d] = xb[d];
        if (box_lo) box_lo[d] = blo[d];
        if (box_hi) box_hi[d] = bhi[d];
    }
    return r;
}

/* g at arbitrary points (test hook for the minimiser pins). */
void or_eval_g(const or_model *M, const double *x, int64_t n, double theta, int side, double *g_out, double *grad_out)
{
    int64_t m = M->m;
    double *kb = (double *)malloc(sizeof(double) * m), *dk = (double *)malloc(sizeof(double) * 3 * m);
    double *v = (double *)malloc(sizeof(double) * m), *P = (double *)malloc(sizeof(double) * m);
    for (int64_t q = 0; q < n; ++q) g_out[q] = eval_g(M, x + 3 * q, theta, side, grad_out + 3 * q, kb, dk, v, P);
    free(kb); free(dk); free(v); free(P);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ----------------------------------------------------------------- adjoint
 * Gradient of loss = sum_c w_c LCP_c (SOV estimator) with respect to y and the
 * log length scales.  Parity unpinned against the paper (it has no gradient):
 * pinned by central finite differences of this oracle's own forward.
 *
 * Reverse sweep of the sequential-conditioning rule, per sample:
 *   u_i = (b_i - sum_{j<i} L_ij z_j) / L_ii, e_i = Phi(u_i), f = prod e_i,
 *   z_i = Phi^-1(w_i e_i)  =>  dz_i/de_i = w_i / phi(z_i). */
static double npdf(double x) { return exp(-0.5 * x * x) / sqrt(2.0 * M_PI); }

static void sov_orthant_adj(int d, const double *L, const double *b, int64_t N, const uint32_t *shift, double Pbar,
                            double *bbar, double *Lbar)
{
    uint32_t G[16];
    for (int i = 0; i < d - 1; ++i) G[i] = lattice_gen(i);
    double z[16], u[16], e[16], w[16], zbar[16];
    for (int64_t k = 0; k < N; ++k) {
        double f = 1.0;
        int ok = 1;
        for (int i = 0; i < d; ++i) {
            double s = 0.0;
            for (int j = 0; j < i; ++j) s += L[i * d + j] * z[j];
            u[i] = (b[i] - s) / L[i * d + i];
            e[i] = or_norm_cdf(u[i]);
            f *= e[i];
            if (!(f > 0.0)) { ok = 0; break; }
            if (i < d - 1) {
                uint32_t U = (uint32_t)((uint64_t)k * G[i]) + shift[i];
                w[i] = fabs(2.0 * u01(U) - 1.0);
                z[i] = or_norm_ppf(w[i] * e[i]);
            }
        }
        /* samples whose product is below 1e-200 carry a negligible share of the value and of
         * the gradient (both are proportional to f); skipping them keeps 1/phi(z) finite */
        if (!ok || !(f > 1e-200)) continue;
        double fbar = Pbar / (double)N;
        for (int i = 0; i < d; ++i) zbar[i] = 0.0;
        for (int i = d - 1; i >= 0; --i) {
            double ebar = fbar * (f / e[i]);
            if (i < d - 1) {
                double ph = npdf(z[i]);
                if (ph > 0.0) ebar += zbar[i] * w[i] / ph;
            }
            double ubar = ebar * npdf(u[i]);
            double lii = L[i * d + i];
            bbar[i] += ubar / lii;
            double sbar = -ubar / lii;
            Lbar[i * d + i] += -ubar * u[i] / lii;
            for (int j = 0; j < i; ++j) {
                Lbar[i * d + j] += sbar * z[j];
                zbar[j] += sbar * L[i * d + j];
            }
        }
    }
}

/* Sbar = L^-T sym(Phi(L^T Lbar)) L^-1, Phi = lower triangle with the diagonal halved:
 * the adjoint of Sigma = L L^T for a symmetric perturbation, dloss = sum_ij Sbar_ij dSigma_ij. */
static void chol_adj(int d, const double *L, const double *Lbar, double *Sbar)
{
    double Pm[256], T[256], Li[256];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += L[k * d + i] * Lbar[k * d + j]; /* (L^T Lbar)_ij */
            Pm[i * d + j] = s;
        }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double v = j < i ? Pm[i * d + j] : (j == i ? 0.5 * Pm[i * d + i] : 0.0);
            T[i * d + j] = v;
        }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Pm[i * d + j] = 0.5 * (T[i * d + j] + T[j * d + i]);
    /* Li = L^-1 (lower) */
    for (int i = 0; i < d * d; ++i) Li[i] = 0.0;
    for (int c = 0; c < d; ++c) {
        for (int i = 0; i < d; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * d + k] * Li[k * d + c];
            Li[i * d + c] = s / L[i * d + i];
        }
    }
    /* Sbar = Li^T Pm Li */
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += Pm[i * d + k] * Li[k * d + j];
            T[i * d + j] = s;
        }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += Li[k * d + i] * T[k * d + j];
            Sbar[i * d + j] = s;
        }
}

/* Adjoint of the SOV cell rule: given wbar = dloss/dLCP, fills mubar[d] and the
 * symmetric Sbar[d*d] with dloss = sum mubar_i dmu_i + sum_ij Sbar_ij dSigma_ij.
 * Returns the LCP.  Cells that the rule makes constant (Boole pre-skip, deterministic,
 * clamped) have zero gradient. */
double or_cell_lcp_adj(int d, const double *mu, const double *S, double theta, int64_t N, uint64_t seed, uint64_t cell,
                       double tau, double skip_eps, double wbar, double *mubar, double *Sbar)
{
    for (int i = 0; i < d; ++i) mubar[i] = 0.0;
    for (int i = 0; i < d * d; ++i) Sbar[i] = 0.0;
    double Sj[256], L[256], Lbar[256], b[16], bbar_lo[16], bbar_hi[16];
    double maxdiag = 0.0;
    int amax = 0;
    for (int i = 0; i < d; ++i) if (S[i * d + i] > maxdiag) { maxdiag = S[i * d + i]; amax = i; }
    if (!(maxdiag > 1e-30)) return or_cell_lcp(d, mu, S, theta, EST_SOV, N, seed, cell, tau, skip_eps);
    double jit = tau * maxdiag;
    for (int i = 0; i < d * d; ++i) Sj[i] = S[i];
    for (int i = 0; i < d; ++i) Sj[i * d + i] += jit;
    for (int i = 0; i < d; ++i)
        if (!(Sj[i * d + i] > 0.0)) return NAN;
    double s_above = 0.0, s_below = 0.0;
    for (int i = 0; i < d; ++i) {
        double sd = sqrt(Sj[i * d + i]);
        s_above += or_norm_cdf((mu[i] - theta) / sd);
        s_below += or_norm_cdf((theta - mu[i]) / sd);
    }
    if (s_above < skip_eps || s_below < skip_eps) return 0.0;
    chol_floor(Sj, d, 1e-3 * jit, L);
    uint32_t sh[16];
    for (int i = 0; i < d - 1; ++i) sh[i] = (uint32_t)(or_splitmix64(seed, (uint64_t)cell * 8 + i + 1) >> 32);
    for (int i = 0; i < d; ++i) b[i] = theta - mu[i];
    double p_lo = or_sov_orthant(d, L, b, N, sh);
    for (int i = 0; i < d; ++i) b[i] = mu[i] - theta;
    double p_hi = or_sov_orthant(d, L, b, N, sh);
    double v = 1.0 - p_lo - p_hi;
    if (v < 0.0 || v > 1.0) return v < 0.0 ? 0.0 : 1.0;
    for (int i = 0; i < d * d; ++i) Lbar[i] = 0.0;
    for (int i = 0; i < d; ++i) { bbar_lo[i] = 0.0; bbar_hi[i] = 0.0; }
    for (int i = 0; i < d; ++i) b[i] = theta - mu[i];
    sov_orthant_adj(d, L, b, N, sh, -wbar, bbar_lo, Lbar);
    for (int i = 0; i < d; ++i) b[i] = mu[i] - theta;
    sov_orthant_adj(d, L, b, N, sh, -wbar, bbar_hi, Lbar);
    for (int i = 0; i < d; ++i) mubar[i] = -bbar_lo[i] + bbar_hi[i];
    chol_adj(d, L, Lbar, Sbar);
    double tr = 0.0;
    for (int i = 0; i < d; ++i) tr += Sbar[i * d + i];
    Sbar[amax * d + amax] += tau * tr;
    return v;
}

/* Adjoint of the ordered rule (EST_SOV_ORD): each orthant's reverse sweep runs on its own
 * permuted factor, its Sigma adjoint is taken through that factor's Cholesky and permuted back;
 * the order itself is piecewise constant, so away from ties it contributes nothing.  Same
 * outputs and conventions as or_cell_lcp_adj. */
double or_cell_lcp_adj_ordered(int d, const double *mu, const double *S, double theta, int64_t N, uint64_t seed,
                               uint64_t cell, double tau, double skip_eps, double wbar, double *mubar, double *Sbar)
{
    for (int i = 0; i < d; ++i) mubar[i] = 0.0;
    for (int i = 0; i < d * d; ++i) Sbar[i] = 0.0;
    double Sj[256];
    double maxdiag = 0.0;
    int amax = 0;
    for (int i = 0; i < d; ++i) if (S[i * d + i] > maxdiag) { maxdiag = S[i * d + i]; amax = i; }
    if (!(maxdiag > 1e-30)) return or_cell_lcp(d, mu, S, theta, EST_SOV_ORD, N, seed, cell, tau, skip_eps);
    double jit = tau * maxdiag;
    for (int i = 0; i < d * d; ++i) Sj[i] = S[i];
    for (int i = 0; i < d; ++i) Sj[i * d + i] += jit;
    for (int i = 0; i < d; ++i)
        if (!(Sj[i * d + i] > 0.0)) return NAN;
    double v = or_cell_lcp(d, mu, S, theta, EST_SOV_ORD, N, seed, cell, tau, skip_eps);
    if (!(v > 0.0) || !(v < 1.0)) return v; /* skipped, clamped or deterministic: constant */
    uint32_t sh[16];
    for (int i = 0; i < d - 1; ++i) sh[i] = (uint32_t)(or_splitmix64(seed, (uint64_t)cell * 8 + i + 1) >> 32);
    for (int side = 0; side < 2; ++side) {
        const double s = side ? -1.0 : 1.0;
        int perm[16];
        double key[16], Sp[256], Lp[256], bp[16], bbar[16], Lbar[256], Sbp[256];
        for (int i = 0; i < d; ++i) {
            key[i] = (s * (theta - mu[i])) / sqrt(Sj[i * d + i]);
            perm[i] = i;
        }
        for (int i = 1; i < d; ++i) {
            int t = perm[i], j = i;
            while (j > 0 && key[t] < key[perm[j - 1]]) { perm[j] = perm[j - 1]; --j; }
            perm[j] = t;
        }
        for (int a = 0; a < d; ++a) {
            bp[a] = s * (theta - mu[perm[a]]);
            bbar[a] = 0.0;
            for (int b = 0; b < d; ++b) Sp[a * d + b] = Sj[perm[a] * d + perm[b]];
        }
        chol_floor(Sp, d, 1e-3 * jit, Lp);
        for (int i = 0; i < d * d; ++i) Lbar[i] = 0.0;
        sov_orthant_adj(d, Lp, bp, N, sh, -wbar, bbar, Lbar);
        chol_adj(d, Lp, Lbar, Sbp);
        for (int a = 0; a < d; ++a) {
            mubar[perm[a]] += -s * bbar[a]; /* b = s (theta - mu) */
            for (int b = 0; b < d; ++b) Sbar[perm[a] * d + perm[b]] += Sbp[a * d + b];
        }
    }
    double tr = 0.0;
    for (int i = 0; i < d; ++i) tr += Sbar[i * d + i];
    Sbar[amax * d + amax] += tau * tr;
    return v;
}

/* d k(a, b) / d log l_d for the kernel (a, b fixed). */
static double kernel_dlogl(int kernel, const double *ell, double sf2, const double *a, const double *b, int dd)
{
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double t = (a[d] - b[d]) / ell[d];
        r2 += t * t;
    }
    double t = (a[dd] - b[dd]) / ell[dd], t2 = t * t;
    if (kernel == OR_SE) return sf2 * exp(-0.5 * r2) * t2;
    double r = sqrt(r2), s5r = sqrt(5.0) * r;
    return (5.0 / 3.0) * sf2 * (1.0 + s5r) * exp(-s5r) * t2;
}

/* Gradient of loss = sum_c w[c] LCP_c over the cells with min corner in [c0, c1) (weights
 * indexed by the linear cell index of the whole grid).  dy[m], dlogl[3]; returns the loss.
 * Chain rule through Eq. (1) for plain GPR, per cell: with P_i = Kt^-1 k_i, alpha = Kt^-1 y,
 * Kd = dK(X,X)/dlog l_d, kd_i = dk(x_i, X)/dlog l_d:
 *   dmu_i/dy = P_i,   dmu_i/dlog l_d = kd_i . alpha - P_i^T Kd alpha,
 *   dSigma_ij/dlog l_d = dk(x_i,x_j) - kd_i . P_j - P_i . kd_j + P_i^T Kd P_j. */
double or_lcp_grad_block(const or_model *M, const or_grid *g, double theta, int64_t N, uint64_t seed, double tau,
                         double skip_eps, const double *weights, const int64_t *c0, const int64_t *c1, double *dy,
                         double *dlogl)
{
    if (M->sgpr) return NAN; /* the gradient is written for plain GPR only */
    int64_t m = M->m;
    int64_t pn[3];
    for (int d = 0; d < 3; ++d) pn[d] = c1[d] - c0[d] + 1;
    int64_t np = pn[0] * pn[1] * pn[2];
    double *V = (double *)malloc(sizeof(double) * np * m);
    double *Pr = (double *)malloc(sizeof(double) * np * m);
    double *Kd = (double *)malloc(sizeof(double) * np * m * 3);   /* kd rows */
    double *KdP = (double *)malloc(sizeof(double) * np * m * 3);  /* Kd_d P_p */
    double *Kda = (double *)malloc(sizeof(double) * m * 3);       /* Kd_d alpha */
    double *Kdm = (double *)malloc(sizeof(double) * m * m * 3);   /* Kd_d matrices */
    for (int d = 0; d < 3; ++d)
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < m; ++j)
                Kdm[(d * m + i) * m + j] = kernel_dlogl(M->kernel, M->ell, M->sf2, M->X + 3 * i, M->X + 3 * j, d);
    for (int d = 0; d < 3; ++d)
        for (int64_t i = 0; i < m; ++i) Kda[d * m + i] = dot(Kdm + (d * m + i) * m, M->alpha, m);
#pragma omp parallel
    {
        double *kb = (double *)malloc(sizeof(double) * m);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < np; ++q) {
            int64_t a = c0[0] + q % pn[0], b = c0[1] + (q / pn[0]) % pn[1], c = c0[2] + q / (pn[0] * pn[1]);
            double x[3] = {grid_x(g, 0, a), grid_x(g, 1, b), grid_x(g, 2, c)};
            whiten_row(M, x, kb, V + q * m);
            back_sub_T(M->L, m, V + q * m, Pr + q * m);
            for (int d = 0; d < 3; ++d) {
                for (int64_t j = 0; j < m; ++j)
                    Kd[(q * 3 + d) * m + j] = kernel_dlogl(M->kernel, M->ell, M->sf2, x, M->X + 3 * j, d);
                for (int64_t i = 0; i < m; ++i)
                    KdP[(q * 3 + d) * m + i] = dot(Kdm + (d * m + i) * m, Pr + q * m, m);
            }
        }
        free(kb);
    }
    int64_t cn[3] = {c1[0] - c0[0], c1[1] - c0[1], c1[2] - c0[2]};
    int64_t nc = cn[0] * cn[1] * cn[2];
    int64_t gc[3] = {g->n[0] - 1, g->n[1] - 1, g->n[2] - 1};
    double loss = 0.0, gl[3] = {0, 0, 0};
    for (int64_t i = 0; i < m; ++i) dy[i] = 0.0;
#pragma omp parallel
    {
        double *dyl = (double *)calloc((size_t)m, sizeof(double));
        double gll[3] = {0, 0, 0}, lossl = 0.0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < nc; ++p) {
            int64_t a = c0[0] + p % cn[0], b = c0[1] + (p / cn[0]) % cn[1], c = c0[2] + p / (cn[0] * cn[1]);
            uint64_t cell = (uint64_t)(a + gc[0] * (b + gc[1] * c));
            double wc = weights[cell];
            int64_t q[8];
            double x[8][3], mu[8], S[64], mubar[8], Sbar[64];
            for (int cc = 0; cc < 8; ++cc) {
                int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
                q[cc] = (a + bx - c0[0]) + pn[0] * ((b + by - c0[1]) + pn[1] * (c + bz - c0[2]));
                x[cc][0] = grid_x(g, 0, a + bx); x[cc][1] = grid_x(g, 1, b + by); x[cc][2] = grid_x(g, 2, c + bz);
                mu[cc] = dot(V + q[cc] * m, M->vy, m);
            }
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j <= i; ++j) {
                    double s = or_kernel_eval(M->kernel, M->ell, M->sf2, x[i], x[j]) - dot(V + q[i] * m, V + q[j] * m, m);
                    S[i * 8 + j] = s; S[j * 8 + i] = s;
                }
            lossl += wc * or_cell_lcp_adj(8, mu, S, theta, N, seed, cell, tau, skip_eps, wc, mubar, Sbar);
            for (int i = 0; i < 8; ++i) {
                if (mubar[i] != 0.0)
                    for (int64_t j = 0; j < m; ++j) dyl[j] += mubar[i] * Pr[q[i] * m + j];
                for (int d = 0; d < 3; ++d)
                    gll[d] += mubar[i] * (dot(Kd + (q[i] * 3 + d) * m, M->alpha, m) - dot(Pr + q[i] * m, Kda + d * m, m));
            }
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j < 8; ++j) {
                    double sb = Sbar[i * 8 + j];
                    if (sb == 0.0) continue;
                    for (int d = 0; d < 3; ++d) {
                        double dS = kernel_dlogl(M->kernel, M->ell, M->sf2, x[i], x[j], d) -
                                    dot(Kd + (q[i] * 3 + d) * m, Pr + q[j] * m, m) -
                                    dot(Pr + q[i] * m, Kd + (q[j] * 3 + d) * m, m) +
                                    dot(Pr + q[i] * m, KdP + (q[j] * 3 + d) * m, m);
                        gll[d] += sb * dS;
                    }
                }
        }
#pragma omp critical
        {
            for (int64_t j = 0; j < m; ++j) dy[j] += dyl[j];
            for (int d = 0; d < 3; ++d) gl[d] += gll[d];
            loss += lossl;
        }
        free(dyl);
    }
    for (int d = 0; d < 3; ++d) dlogl[d] = gl[d];
    free(V); free(Pr); free(Kd); free(KdP); free(Kda); free(Kdm);
    return loss;
}
