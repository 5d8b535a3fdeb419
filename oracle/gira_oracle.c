/*
 * gira_oracle.c -- plain, slow, obviously-correct FP64 CPU reference for GMM-EM.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code with the CUDA path.
 *
 * What it computes (GIRA, arXiv 2307.00071, Sec. V "Expectation Maximization"):
 *   E-step   responsibilities, Eq. (estep), evaluated in the log domain of
 *            Eq. (logestep), with the per-component log-density of
 *            Eq. (simplifiedGaussian):  Sigma = L L^T,  P = L^{-1},
 *            ln N(x|mu,Sigma) = -1/2 (D ln 2pi + ||P (x-mu)||^2) + sum_j ln P_jj.
 *   M-step   the paper names it but does not write it; the standard
 *            maximum-likelihood full-covariance update is used, with the
 *            conventions of the scikit-learn derivation the paper defers to:
 *            N_b = sum_n r_nb + 10 eps64,  pi_b = N_b / sum_a N_a,
 *            mu_b = sum_n r_nb x_n / N_b,
 *            Sigma_b = sum_n r_nb (x_n-mu_b)(x_n-mu_b)^T / N_b + reg I
 *            (two passes: exact centring about the new mean).
 *   KInit    Fig. "information flow": k-means initialisation produces the
 *            responsibility matrix the EM starts from.  Read as k-means++
 *            seeding (one candidate per step) followed by Lloyd iterations, then
 *            the M-step above applied to one-hot responsibilities.
 *
 * Precision: every floating-point quantity is binary64, except the k-means
 * point-to-centre squared distances, which are evaluated in binary32 in the
 * fixed order   d_i = x_i - c_i;  s = (d0*d0 + d1*d1) + d2*d2   (no fused
 * multiply-add; compiled with -ffp-contract=off) because they decide integers
 * (a sampled index, an argmin label) and the GPU takes the same decisions in
 * that same precision.  k-means centres are rounded to binary32 after each
 * update, as the GPU stores them.
 *
 * k-means++ draws are integer decisions taken in exact fixed point (see
 * oracle_fx48): no floating-point rounding enters the choice of a centre.
 *
 * Differentiable log-likelihood (oracle_loglik_grad): not in the paper, which
 * registers scans with its own distribution-to-distribution method; here the
 * plain definition  L = sum_n ln sum_b pi_b N(R x_n + t | mu_b, L_b L_b^T),
 * pi = softmax(alpha), and its gradient by ordinary calculus, term by term
 * per point and component (gamma = responsibility, y = L_b^{-1}(x'-mu_b)):
 *   dL/dx'_n   = -sum_b gamma_nb L_b^{-T} y_nb          (dL/dx_n = R^T dL/dx'_n)
 *   dL/dmu_b   =  sum_n gamma_nb L_b^{-T} y_nb
 *   dL/dL_b    =  sum_n gamma_nb (L_b^{-T} y y^T - diag(1/L_b,ii)), lower triangle
 *   dL/dalpha_b = sum_n gamma_nb - N pi_b
 *   twist xi = (omega, v), a left perturbation x' <- exp(xi^) x' (rotation
 *   first):  dL/domega = sum_n x'_n x dL/dx'_n,  dL/dv = sum_n dL/dx'_n.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
 * counter-based generator: draw j of seed s is the (j+1)-th output of the
 * SplitMix64 stream started at state s;  u_j = (r_j >> 11) * 2^-53.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>


/* binary32 expressions must be evaluated in binary32 (no excess precision) */
#if defined(__FLT_EVAL_METHOD__) && __FLT_EVAL_METHOD__ != 0
#error "the oracle needs FLT_EVAL_METHOD == 0"
#endif
#if defined(__FAST_MATH__)
#error "the oracle must not be built with -ffast-math"
#endif

/* status codes (same numbering as the library's, redefined here on purpose) */
enum { OR_OK = 0, OR_ERR_INVALID_ARG = 1, OR_ERR_NONFINITE = 2, OR_ERR_NOT_PD = 3, OR_ERR_OOM = 5 };

static int g_last_bad_component = -1;
int oracle_last_bad_component(void) { return g_last_bad_component; }
void oracle_note_bad_component(int b) { g_last_bad_component = b; }

/* ---------------------------------------------------------------- RNG -- */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t j) {
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double oracle_uniform(uint64_t seed, uint64_t j) {
    return (double)(oracle_splitmix64(seed, j) >> 11) * (1.0 / 9007199254740992.0);
}

/* ----------------------------------------------- d x d algebra (d <= 4) -- */
#define DMAX 4
/* Cholesky Sigma = L L^T (row-major d x d, L lower).  Returns 0, or -1 if a
 * pivot is not strictly positive (Sigma not positive definite). */
int oracle_cholesky_d(const double *S, double *L, int d) {
    memset(L, 0, (size_t)d * d * sizeof(double));
    for (int j = 0; j < d; ++j) {
        double s = S[j * d + j];
        for (int k = 0; k < j; ++k) s -= L[j * d + k] * L[j * d + k];
        if (!(s > 0.0)) return -1;
        L[j * d + j] = sqrt(s);
        for (int i = j + 1; i < d; ++i) {
            double t = S[i * d + j];
            for (int k = 0; k < j; ++k) t -= L[i * d + k] * L[j * d + k];
            L[i * d + j] = t / L[j * d + j];
        }
    }
    return 0;
}
int oracle_cholesky3(const double *S, double *L) { return oracle_cholesky_d(S, L, 3); }

/* P = L^{-1} for lower-triangular L (forward substitution on the identity). */
void oracle_tri_inverse_d(const double *L, double *P, int d) {
    memset(P, 0, (size_t)d * d * sizeof(double));
    for (int c = 0; c < d; ++c) {
        for (int i = c; i < d; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) t -= L[i * d + k] * P[k * d + c];
            P[i * d + c] = t / L[i * d + i];
        }
    }
}
void oracle_tri_inverse3(const double *L, double *P) { oracle_tri_inverse_d(L, P, 3); }

/* Eq. (simplifiedGaussian): ln N(x | mu, Sigma) with P = L^{-1}, dimension d. */
double oracle_log_gaussian_d(const double *x, const double *mu, const double *P, int d) {
    double q = 0.0, logdet = 0.0;
    for (int i = 0; i < d; ++i) {
        double y = 0.0;
        for (int j = 0; j <= i; ++j) y += P[i * d + j] * (x[j] - mu[j]);
        q += y * y;
        logdet += log(P[i * d + i]);
    }
    return -0.5 * (d * log(2.0 * M_PI) + q) + logdet;
}
double oracle_log_gaussian(const double *x, const double *mu, const double *P) {
    return oracle_log_gaussian_d(x, mu, P, 3);
}

static int all_finite_f(const float *a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(a[i])) return 0;
    return 1;
}
static int all_finite_d(const double *a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(a[i])) return 0;
    return 1;
}

/* Precision factors of every component: P_b = chol(Sigma_b)^{-1}. */
static int precision_factors(int K, const double *covs, double *P, int d) {
    const int dd = d * d;
    for (int b = 0; b < K; ++b) {
        double L[DMAX * DMAX];
        if (oracle_cholesky_d(covs + (size_t)dd * b, L, d) != 0) { g_last_bad_component = b; return OR_ERR_NOT_PD; }
        oracle_tri_inverse_d(L, P + (size_t)dd * b, d);
    }
    return OR_OK;
}

static int valid_dim(int d) { return d == 3 || d == 4; }

/* ------------------------------------------------------------ E-step -- */
/* Eq. (estep) in the form of Eq. (logestep), points of dimension d.  Writes
 * resp (N x K, row-major; may be NULL) and lse_n = ln sum_a pi_a N(x_n|a) (may
 * be NULL); returns the mean per-point log-likelihood (1/N) sum_n lse_n in
 * *mean_ll. */
int oracle_estep_d(const float *pts, int64_t N, int K, int d, const double *weights, const double *means,
                   const double *covs, double *resp, double *lse, double *mean_ll) {
    if (N < 1 || K < 1 || !valid_dim(d) || !pts || !weights || !means || !covs) return OR_ERR_INVALID_ARG;
    const int dd = d * d;
    if (!all_finite_f(pts, (int64_t)d * N)) return OR_ERR_NONFINITE;
    if (!all_finite_d(weights, K) || !all_finite_d(means, (int64_t)d * K) || !all_finite_d(covs, (int64_t)dd * K))
        return OR_ERR_NONFINITE;
    double *P = (double *)malloc(sizeof(double) * dd * K);
    double *a = (double *)malloc(sizeof(double) * K);
    if (!P || !a) { free(P); free(a); return OR_ERR_OOM; }
    int st = precision_factors(K, covs, P, d);
    if (st != OR_OK) { free(P); free(a); return st; }
    double total = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        double x[DMAX];
        for (int i = 0; i < d; ++i) x[i] = pts[(size_t)d * n + i];
        double m = -INFINITY;
        for (int b = 0; b < K; ++b) {
            a[b] = log(weights[b]) + oracle_log_gaussian_d(x, means + (size_t)d * b, P + (size_t)dd * b, d);
            if (a[b] > m) m = a[b];
        }
        double s = 0.0;
        for (int b = 0; b < K; ++b) s += exp(a[b] - m);
        double l = m + log(s);
        if (lse) lse[n] = l;
        if (resp)
            for (int b = 0; b < K; ++b) resp[n * K + b] = exp(a[b] - l);
        total += l;
    }
    *mean_ll = total / (double)N;
    free(P);
    free(a);
    return OR_OK;
}
int oracle_estep(const float *pts, int64_t N, int K, const double *weights, const double *means,
                 const double *covs, double *resp, double *lse, double *mean_ll) {
    return oracle_estep_d(pts, N, K, 3, weights, means, covs, resp, lse, mean_ll);
}

/* ------------------------------------------------------------ M-step -- */
int oracle_mstep_d(const float *pts, int64_t N, int K, int d, const double *resp, double reg, double *weights,
                   double *means, double *covs) {
    if (N < 1 || K < 1 || !valid_dim(d) || !pts || !resp || !weights || !means || !covs || !(reg >= 0.0))
        return OR_ERR_INVALID_ARG;
    const int dd = d * d;
    const double tiny = 10.0 * DBL_EPSILON;
    double nsum = 0.0;
    for (int b = 0; b < K; ++b) {
        double nb = 0.0, sx[DMAX] = {0, 0, 0, 0};
        for (int64_t n = 0; n < N; ++n) {
            double r = resp[n * K + b];
            nb += r;
            for (int i = 0; i < d; ++i) sx[i] += r * (double)pts[(size_t)d * n + i];
        }
        nb += tiny;
        double mu[DMAX];
        for (int i = 0; i < d; ++i) mu[i] = sx[i] / nb;
        double c[DMAX * DMAX] = {0};
        for (int64_t n = 0; n < N; ++n) {
            double r = resp[n * K + b];
            double dv[DMAX];
            for (int i = 0; i < d; ++i) dv[i] = (double)pts[(size_t)d * n + i] - mu[i];
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) c[i * d + j] += r * dv[i] * dv[j];
        }
        for (int i = 0; i < dd; ++i) c[i] /= nb;
        for (int i = 0; i < d; ++i) c[i * d + i] += reg;
        weights[b] = nb;
        nsum += nb;
        memcpy(means + (size_t)d * b, mu, sizeof(double) * d);
        memcpy(covs + (size_t)dd * b, c, sizeof(double) * dd);
    }
    for (int b = 0; b < K; ++b) weights[b] /= nsum;
    /* the new covariances must admit a Cholesky factor for the next E-step */
    for (int b = 0; b < K; ++b) {
        double L[DMAX * DMAX];
        if (oracle_cholesky_d(covs + (size_t)dd * b, L, d) != 0) { g_last_bad_component = b; return OR_ERR_NOT_PD; }
    }
    return OR_OK;
}
int oracle_mstep(const float *pts, int64_t N, int K, const double *resp, double reg, double *weights,
                 double *means, double *covs) {
    return oracle_mstep_d(pts, N, K, 3, resp, reg, weights, means, covs);
}

/* ------------------------------------------------------------ k-means -- */
/* squared distance in binary32, fixed order ((d0^2 + d1^2) + d2^2) + d3^2, no
 * FMA (see header) */
static float dist2_f32(const float *x, const float *c, int d) {
    float s = 0.0f;
    for (int i = 0; i < d; ++i) {
        const float di = x[i] - c[i];
        const float p = di * di;
        s = (i == 0) ? p : s + p;
    }
    return s;
}
float oracle_dist2_f32(const float *x, const float *c) { return dist2_f32(x, c, 3); }
float oracle_dist2_f32_d(const float *x, const float *c, int d) { return dist2_f32(x, c, d); }

/* The k-means++ weights D^2 are taken in exact fixed point so that the draw is
 * an integer decision with no rounding: fx(d) = floor(d * 2^48) for a binary32
 * d >= 0 (d >= 2^47 saturates to 2^95 - 1), summed exactly in 128 bits.  With
 * k_j = r_j >> 11 the 53-bit integer behind u_j and T the exact total, the
 * threshold is t = floor(k_j * T / 2^53) and the drawn point is the first n whose
 * running sum exceeds t.  (Points closer than 2^-24 m to a chosen centre get
 * weight 0; nothing else differs from real-valued D^2 sampling.) */
typedef unsigned __int128 u128;

u128 oracle_fx48(float d) {
    if (!(d > 0.0f)) return 0;
    if (d >= 140737488355328.0f) return (((u128)1) << 95) - 1; /* 2^47 */
    return (u128)floor(ldexp((double)d, 48)); /* exact: d has 24 bits, doubles 53 */
}

static u128 fx_threshold(uint64_t k53, u128 T) {
    uint64_t tl = (uint64_t)T, th = (uint64_t)(T >> 64);
    u128 a = (u128)k53 * tl, b = (u128)k53 * th; /* k*T = b*2^64 + a (192 bits) */
    uint64_t w0 = (uint64_t)a;
    uint64_t a_hi = (uint64_t)(a >> 64), b_lo = (uint64_t)b, b_hi = (uint64_t)(b >> 64);
    uint64_t w1 = a_hi + b_lo;
    uint64_t w2 = b_hi + (w1 < a_hi ? 1u : 0u);
    uint64_t t_lo = (w0 >> 53) | (w1 << 11), t_hi = (w1 >> 53) | (w2 << 11);
    return ((u128)t_hi << 64) | t_lo;
}

/* Exported for the pins: threshold t (as two 64-bit halves) for k53 and T. */
void oracle_fx_threshold(uint64_t k53, uint64_t T_lo, uint64_t T_hi, uint64_t *t_lo, uint64_t *t_hi) {
    u128 t = fx_threshold(k53, ((u128)T_hi << 64) | T_lo);
    *t_lo = (uint64_t)t;
    *t_hi = (uint64_t)(t >> 64);
}
void oracle_fx48_parts(float d, uint64_t *lo, uint64_t *hi) {
    u128 v = oracle_fx48(d);
    *lo = (uint64_t)v;
    *hi = (uint64_t)(v >> 64);
}

/* k-means++ seeding (Arthur & Vassilvitskii 2007, one candidate per step).
 * centers: K x d float (out); chosen: K indices into pts (out, may be NULL). */
int oracle_kmeanspp_d(const float *pts, int64_t N, int K, int d, uint64_t seed, float *centers, int64_t *chosen) {
    if (N < 1 || K < 1 || K > N || !valid_dim(d) || !pts || !centers) return OR_ERR_INVALID_ARG;
    if (!all_finite_f(pts, (int64_t)d * N)) return OR_ERR_NONFINITE;
    float *d2 = (float *)malloc(sizeof(float) * N);
    if (!d2) return OR_ERR_OOM;
    int64_t idx = (int64_t)floor(oracle_uniform(seed, 0) * (double)N);
    if (idx > N - 1) idx = N - 1;
    for (int j = 0; j < K; ++j) {
        if (j > 0) {
            /* D^2(x) = min over the centres chosen so far */
            u128 total = 0;
            for (int64_t n = 0; n < N; ++n) {
                float dn = dist2_f32(pts + (size_t)d * n, centers + (size_t)d * (j - 1), d);
                if (j == 1 || dn < d2[n]) d2[n] = dn;
                total += oracle_fx48(d2[n]);
            }
            if (total > 0) {
                const u128 t = fx_threshold(oracle_splitmix64(seed, (uint64_t)j) >> 11, total);
                u128 prefix = 0;
                idx = N - 1; /* unreachable: t < total */
                for (int64_t n = 0; n < N; ++n) {
                    prefix += oracle_fx48(d2[n]);
                    if (prefix > t) { idx = n; break; }
                }
            } else {
                idx = (int64_t)floor(oracle_uniform(seed, (uint64_t)j) * (double)N); /* all weights zero */
                if (idx > N - 1) idx = N - 1;
            }
        }
        for (int i = 0; i < d; ++i) centers[(size_t)d * j + i] = pts[(size_t)d * idx + i];
        if (chosen) chosen[j] = idx;
    }
    free(d2);
    return OR_OK;
}
int oracle_kmeanspp(const float *pts, int64_t N, int K, uint64_t seed, float *centers, int64_t *chosen) {
    return oracle_kmeanspp_d(pts, N, K, 3, seed, centers, chosen);
}

/* labels_n = argmin_b ||x_n - c_b||^2 in binary32, ties to the lowest b. */
static int64_t assign_labels(const float *pts, int64_t N, int K, int d, const float *centers, int32_t *labels) {
    int64_t changed = 0;
    for (int64_t n = 0; n < N; ++n) {
        int best = 0;
        float bd = dist2_f32(pts + (size_t)d * n, centers, d);
        for (int b = 1; b < K; ++b) {
            float dv = dist2_f32(pts + (size_t)d * n, centers + (size_t)d * b, d);
            if (dv < bd) { bd = dv; best = b; }
        }
        if (labels[n] != best) ++changed;
        labels[n] = best;
    }
    return changed;
}

/* Lloyd iterations from the given centres (in/out).  Each iteration: centres
 * = FP64 mean of their points (rounded to binary32; an empty cluster keeps its
 * centre), then re-assign; stop after lloyd_iters or when no label changed.
 * labels (out, N) hold the final assignment. */
int oracle_lloyd_d(const float *pts, int64_t N, int K, int d, float *centers, int lloyd_iters, int32_t *labels,
                   int *iters_done) {
    if (N < 1 || K < 1 || K > N || !valid_dim(d) || lloyd_iters < 0 || !pts || !centers || !labels)
        return OR_ERR_INVALID_ARG;
    if (!all_finite_f(pts, (int64_t)d * N) || !all_finite_f(centers, (int64_t)d * K)) return OR_ERR_NONFINITE;
    for (int64_t n = 0; n < N; ++n) labels[n] = -1;
    assign_labels(pts, N, K, d, centers, labels);
    const int w = d + 1;   /* coordinate sums, then the count */
    double *sum = (double *)malloc(sizeof(double) * w * K);
    if (!sum) return OR_ERR_OOM;
    int it = 0;
    while (it < lloyd_iters) {
        memset(sum, 0, sizeof(double) * w * K);
        for (int64_t n = 0; n < N; ++n) {
            int b = labels[n];
            for (int i = 0; i < d; ++i) sum[(size_t)w * b + i] += (double)pts[(size_t)d * n + i];
            sum[(size_t)w * b + d] += 1.0;
        }
        for (int b = 0; b < K; ++b)
            if (sum[(size_t)w * b + d] > 0.0)
                for (int i = 0; i < d; ++i)
                    centers[(size_t)d * b + i] = (float)(sum[(size_t)w * b + i] / sum[(size_t)w * b + d]);
        ++it;
        if (assign_labels(pts, N, K, d, centers, labels) == 0) break;
    }
    if (iters_done) *iters_done = it;
    free(sum);
    return OR_OK;
}
int oracle_lloyd(const float *pts, int64_t N, int K, float *centers, int lloyd_iters, int32_t *labels,
                 int *iters_done) {
    return oracle_lloyd_d(pts, N, K, 3, centers, lloyd_iters, labels, iters_done);
}

/* One-hot responsibilities from labels, then the M-step. */
int oracle_init_from_labels_d(const float *pts, int64_t N, int K, int d, const int32_t *labels, double reg,
                              double *weights, double *means, double *covs) {
    if (N < 1 || K < 1 || !labels) return OR_ERR_INVALID_ARG;
    double *resp = (double *)calloc((size_t)N * (size_t)K, sizeof(double));
    if (!resp) return OR_ERR_OOM;
    for (int64_t n = 0; n < N; ++n) {
        if (labels[n] < 0 || labels[n] >= K) { free(resp); return OR_ERR_INVALID_ARG; }
        resp[n * K + labels[n]] = 1.0;
    }
    int st = oracle_mstep_d(pts, N, K, d, resp, reg, weights, means, covs);
    free(resp);
    return st;
}
int oracle_init_from_labels(const float *pts, int64_t N, int K, const int32_t *labels, double reg,
                            double *weights, double *means, double *covs) {
    return oracle_init_from_labels_d(pts, N, K, 3, labels, reg, weights, means, covs);
}

/* ------------------------------------------------------------ EM fit -- */
/* EM from the given parameters (in/out).  Iteration t (1-based): E-step with
 * the current parameters gives ll_t (mean per-point log-likelihood, stored in
 * trace[t-1]), then the M-step.  Stops after `iters` iterations or when
 * t > 1 and |ll_t - ll_{t-1}| < tol.  final_ll (may be NULL) is the mean
 * log-likelihood of the returned parameters. */
int oracle_em_d(const float *pts, int64_t N, int K, int d, int iters, double tol, double reg, double *weights,
                double *means, double *covs, double *trace, int *iters_done, double *final_ll) {
    if (N < 1 || K < 1 || !valid_dim(d) || iters < 0 || !(tol >= 0.0) || !(reg >= 0.0)) return OR_ERR_INVALID_ARG;
    double *resp = (double *)malloc(sizeof(double) * (size_t)N * (size_t)K);
    if (!resp) return OR_ERR_OOM;
    double prev = -INFINITY;
    int t = 0, st = OR_OK;
    while (t < iters) {
        double ll;
        st = oracle_estep_d(pts, N, K, d, weights, means, covs, resp, NULL, &ll);
        if (st != OR_OK) break;
        st = oracle_mstep_d(pts, N, K, d, resp, reg, weights, means, covs);
        if (st != OR_OK) break;
        if (trace) trace[t] = ll;
        ++t;
        if (fabs(ll - prev) < tol) break;
        prev = ll;
    }
    if (iters_done) *iters_done = t;
    if (st == OR_OK && final_ll) st = oracle_estep_d(pts, N, K, d, weights, means, covs, NULL, NULL, final_ll);
    free(resp);
    return st;
}
int oracle_em(const float *pts, int64_t N, int K, int iters, double tol, double reg, double *weights,
              double *means, double *covs, double *trace, int *iters_done, double *final_ll) {
    return oracle_em_d(pts, N, K, 3, iters, tol, reg, weights, means, covs, trace, iters_done, final_ll);
}

/* Full fit: k-means++ (seed) + Lloyd (lloyd_iters) + init M-step, then EM. */
int oracle_gmm_fit_d(const float *pts, int64_t N, int K, int d, int iters, double tol, double reg, uint64_t seed,
                     int lloyd_iters, double *weights, double *means, double *covs, double *trace,
                     int *iters_done, double *final_ll) {
    if (N < 1 || K < 1 || K > N || !valid_dim(d)) return OR_ERR_INVALID_ARG;
    float *c = (float *)malloc(sizeof(float) * d * K);
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * N);
    if (!c || !lab) { free(c); free(lab); return OR_ERR_OOM; }
    int st = oracle_kmeanspp_d(pts, N, K, d, seed, c, NULL);
    if (st == OR_OK) st = oracle_lloyd_d(pts, N, K, d, c, lloyd_iters, lab, NULL);
    if (st == OR_OK) st = oracle_init_from_labels_d(pts, N, K, d, lab, reg, weights, means, covs);
    free(c);
    free(lab);
    if (st != OR_OK) return st;
    return oracle_em_d(pts, N, K, d, iters, tol, reg, weights, means, covs, trace, iters_done, final_ll);
}
int oracle_gmm_fit(const float *pts, int64_t N, int K, int iters, double tol, double reg, uint64_t seed,
                   int lloyd_iters, double *weights, double *means, double *covs, double *trace,
                   int *iters_done, double *final_ll) {
    return oracle_gmm_fit_d(pts, N, K, 3, iters, tol, reg, seed, lloyd_iters, weights, means, covs, trace,
                            iters_done, final_ll);
}

/* ------------------------------------------------ differentiable loglik -- */
/* L and its gradient (see the header).  pose12 = R (row-major 3x3) then t, or
 * NULL for the identity.  chol: K x 9 row-major, lower triangle read, diagonal
 * must be positive (else OR_ERR_NOT_PD).  Every gradient pointer may be NULL. */
int oracle_loglik_grad(const float *pts, int64_t N, int K, const double *pose12, const double *logits,
                       const double *means, const double *chol, double *loglik, double *grad_pts,
                       double *grad_twist, double *grad_logits, double *grad_means, double *grad_chol) {
    if (N < 1 || K < 1 || !pts || !logits || !means || !chol) return OR_ERR_INVALID_ARG;
    if (!all_finite_f(pts, 3 * N) || !all_finite_d(logits, K) || !all_finite_d(means, 3 * (int64_t)K) ||
        !all_finite_d(chol, 9 * (int64_t)K) || (pose12 && !all_finite_d(pose12, 12)))
        return OR_ERR_NONFINITE;
    const double I12[12] = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0};
    const double *R = pose12 ? pose12 : I12, *t = (pose12 ? pose12 : I12) + 9;
    double *logw = malloc(sizeof(double) * K), *gam = malloc(sizeof(double) * K);
    double *lgam = malloc(sizeof(double) * K);
    if (!logw || !gam || !lgam) {
        free(logw); free(gam); free(lgam);
        return OR_ERR_OOM;
    }
    /* log pi_b = alpha_b - ln sum_a exp(alpha_a) */
    double amax = logits[0];
    for (int b = 1; b < K; ++b) amax = logits[b] > amax ? logits[b] : amax;
    double z = 0.0;
    for (int b = 0; b < K; ++b) z += exp(logits[b] - amax);
    const double lz = amax + log(z);
    for (int b = 0; b < K; ++b) {
        const double *Lb = chol + 9 * (size_t)b;
        if (!(Lb[0] > 0.0 && Lb[4] > 0.0 && Lb[8] > 0.0)) {
            g_last_bad_component = b;
            free(logw); free(gam); free(lgam);
            return OR_ERR_NOT_PD;
        }
        /* ln pi_b - sum_j ln L_jj - (3/2) ln 2 pi */
        logw[b] = (logits[b] - lz) - (log(Lb[0]) + log(Lb[4]) + log(Lb[8])) - 1.5 * log(2.0 * M_PI);
    }
    if (grad_twist) memset(grad_twist, 0, sizeof(double) * 6);
    if (grad_logits) memset(grad_logits, 0, sizeof(double) * K);
    if (grad_means) memset(grad_means, 0, sizeof(double) * 3 * K);
    if (grad_chol) memset(grad_chol, 0, sizeof(double) * 9 * K);
    double total = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        const double x[3] = {pts[3 * n], pts[3 * n + 1], pts[3 * n + 2]};
        double xp[3];
        for (int i = 0; i < 3; ++i) xp[i] = R[3 * i] * x[0] + R[3 * i + 1] * x[1] + R[3 * i + 2] * x[2] + t[i];
        double lmax = -INFINITY;
        for (int b = 0; b < K; ++b) {
            const double *Lb = chol + 9 * (size_t)b, *mu = means + 3 * (size_t)b;
            const double d0 = xp[0] - mu[0], d1 = xp[1] - mu[1], d2 = xp[2] - mu[2];
            /* y = L^{-1} d (forward substitution) */
            const double y0 = d0 / Lb[0];
            const double y1 = (d1 - Lb[3] * y0) / Lb[4];
            const double y2 = (d2 - Lb[6] * y0 - Lb[7] * y1) / Lb[8];
            lgam[b] = logw[b] - 0.5 * (y0 * y0 + y1 * y1 + y2 * y2);
            lmax = lgam[b] > lmax ? lgam[b] : lmax;
        }
        double ssum = 0.0;
        for (int b = 0; b < K; ++b) ssum += exp(lgam[b] - lmax);
        const double lse = lmax + log(ssum);
        total += lse;
        for (int b = 0; b < K; ++b) gam[b] = exp(lgam[b] - lse);
        double g[3] = {0.0, 0.0, 0.0};
        for (int b = 0; b < K; ++b) {
            const double *Lb = chol + 9 * (size_t)b, *mu = means + 3 * (size_t)b;
            const double d0 = xp[0] - mu[0], d1 = xp[1] - mu[1], d2 = xp[2] - mu[2];
            const double y0 = d0 / Lb[0];
            const double y1 = (d1 - Lb[3] * y0) / Lb[4];
            const double y2 = (d2 - Lb[6] * y0 - Lb[7] * y1) / Lb[8];
            /* w = L^{-T} y (back substitution) = Sigma^{-1} d */
            const double w2 = y2 / Lb[8];
            const double w1 = (y1 - Lb[7] * w2) / Lb[4];
            const double w0 = (y0 - Lb[3] * w1 - Lb[6] * w2) / Lb[0];
            const double gb = gam[b];
            g[0] -= gb * w0;
            g[1] -= gb * w1;
            g[2] -= gb * w2;
            if (grad_means) {
                grad_means[3 * b] += gb * w0;
                grad_means[3 * b + 1] += gb * w1;
                grad_means[3 * b + 2] += gb * w2;
            }
            if (grad_chol) {
                const double w[3] = {w0, w1, w2}, y[3] = {y0, y1, y2};
                double *G = grad_chol + 9 * (size_t)b;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j <= i; ++j) G[3 * i + j] += gb * (w[i] * y[j] - (i == j ? 1.0 / Lb[4 * i] : 0.0));
            }
            if (grad_logits) grad_logits[b] += gb;
        }
        if (grad_pts)
            for (int i = 0; i < 3; ++i) grad_pts[3 * n + i] = R[i] * g[0] + R[3 + i] * g[1] + R[6 + i] * g[2];
        if (grad_twist) {
            grad_twist[0] += xp[1] * g[2] - xp[2] * g[1];
            grad_twist[1] += xp[2] * g[0] - xp[0] * g[2];
            grad_twist[2] += xp[0] * g[1] - xp[1] * g[0];
            for (int i = 0; i < 3; ++i) grad_twist[3 + i] += g[i];
        }
    }
    if (grad_logits)
        for (int b = 0; b < K; ++b) grad_logits[b] -= (double)N * exp(logits[b] - lz);
    if (loglik) *loglik = total;
    free(logw); free(gam); free(lgam);
    return OR_OK;
}

/* --------------------------------------- 4D mixtures: conditional, sampling -- */
/* Gaussian-mixture regression of the last coordinate on the first three for a
 * D = 4 mixture (xyz + intensity): with mu_b = (mu_x, mu_I) and Sigma_b split
 * as [[S_xx, S_xI], [S_Ix, S_II]], the conditional of I given x under component
 * b is normal with mean m_b = mu_I + S_Ix S_xx^{-1} (x - mu_x) and variance
 * v_b = S_II - S_Ix S_xx^{-1} S_xI; the mixture weight of b given x is
 * w_b ∝ pi_b N(x | mu_x, S_xx).  E[I|x] = sum_b w_b m_b,
 * V[I|x] = sum_b w_b (v_b + m_b^2) - E[I|x]^2.  locs: M x 3. */
int oracle_conditional4(const float *locs, int64_t M, int K, const double *weights, const double *means,
                        const double *covs, double *cmean, double *cvar) {
    if (M < 1 || K < 1 || !locs || !weights || !means || !covs || !cmean || !cvar) return OR_ERR_INVALID_ARG;
    double *P = (double *)malloc(sizeof(double) * 9 * K), *g = (double *)malloc(sizeof(double) * 3 * K);
    double *v = (double *)malloc(sizeof(double) * K), *a = (double *)malloc(sizeof(double) * K);
    if (!P || !g || !v || !a) { free(P); free(g); free(v); free(a); return OR_ERR_OOM; }
    for (int b = 0; b < K; ++b) {
        const double *S = covs + 16 * (size_t)b;
        const double Sxx[9] = {S[0], S[1], S[2], S[4], S[5], S[6], S[8], S[9], S[10]};
        const double SxI[3] = {S[3], S[7], S[11]};
        double L[9];
        if (oracle_cholesky_d(Sxx, L, 3) != 0) {
            g_last_bad_component = b;
            free(P); free(g); free(v); free(a);
            return OR_ERR_NOT_PD;
        }
        oracle_tri_inverse_d(L, P + 9 * (size_t)b, 3);
        /* g_b = S_xx^{-1} S_xI = P^T P S_xI */
        const double *Pb = P + 9 * (size_t)b;
        double u[3];
        for (int i = 0; i < 3; ++i) u[i] = Pb[3 * i] * SxI[0] + Pb[3 * i + 1] * SxI[1] + Pb[3 * i + 2] * SxI[2];
        for (int i = 0; i < 3; ++i) g[3 * b + i] = Pb[i] * u[0] + Pb[3 + i] * u[1] + Pb[6 + i] * u[2];
        v[b] = S[15] - (SxI[0] * g[3 * b] + SxI[1] * g[3 * b + 1] + SxI[2] * g[3 * b + 2]);
    }
    for (int64_t n = 0; n < M; ++n) {
        const double x[3] = {locs[3 * n], locs[3 * n + 1], locs[3 * n + 2]};
        double m = -INFINITY;
        for (int b = 0; b < K; ++b) {
            const double *mu = means + 4 * (size_t)b;
            a[b] = log(weights[b]) + oracle_log_gaussian_d(x, mu, P + 9 * (size_t)b, 3);
            if (a[b] > m) m = a[b];
        }
        double s = 0.0;
        for (int b = 0; b < K; ++b) s += exp(a[b] - m);
        double e1 = 0.0, e2 = 0.0;
        for (int b = 0; b < K; ++b) {
            const double *mu = means + 4 * (size_t)b;
            const double w = exp(a[b] - m) / s;
            const double mb = mu[3] + g[3 * b] * (x[0] - mu[0]) + g[3 * b + 1] * (x[1] - mu[1]) +
                              g[3 * b + 2] * (x[2] - mu[2]);
            e1 += w * mb;
            e2 += w * (v[b] + mb * mb);
        }
        cmean[n] = e1;
        cvar[n] = e2 - e1 * e1;
    }
    free(P); free(g); free(v); free(a);
    return OR_OK;
}

/* Draw M points from a d-dimensional mixture.  Sample i takes the uniforms of
 * draws 5i .. 5i+4 of `seed`: the first picks the component (the first b whose
 * running binary64 weight sum exceeds u * sum_a pi_a), the other four give four
 * standard normals by the Box-Muller transform, z = sqrt(-2 ln(1 - u1)) *
 * (cos, sin)(2 pi u2) for the pairs (u1, u2) = (5i+1, 5i+2) and (5i+3, 5i+4);
 * x = mu_b + L_b z (L_b = chol Sigma_b), rounded to binary32.  comp (may be
 * NULL) receives the component of each sample. */
int oracle_sample_d(int64_t M, int K, int d, const double *weights, const double *means, const double *covs,
                    uint64_t seed, float *out, int32_t *comp) {
    if (M < 1 || K < 1 || !valid_dim(d) || !weights || !means || !covs || !out) return OR_ERR_INVALID_ARG;
    const int dd = d * d;
    double *L = (double *)malloc(sizeof(double) * dd * K), *cum = (double *)malloc(sizeof(double) * K);
    if (!L || !cum) { free(L); free(cum); return OR_ERR_OOM; }
    double tot = 0.0;
    for (int b = 0; b < K; ++b) {
        if (oracle_cholesky_d(covs + (size_t)dd * b, L + (size_t)dd * b, d) != 0 || !(weights[b] >= 0.0)) {
            g_last_bad_component = b;
            free(L); free(cum);
            return OR_ERR_NOT_PD;
        }
        tot += weights[b];
        cum[b] = tot;
    }
    for (int64_t i = 0; i < M; ++i) {
        const double u0 = oracle_uniform(seed, 5 * (uint64_t)i) * tot;
        int b = K - 1;
        for (int a = 0; a < K; ++a)
            if (cum[a] > u0) { b = a; break; }
        double z[4];
        for (int p = 0; p < 2; ++p) {
            const double u1 = oracle_uniform(seed, 5 * (uint64_t)i + 1 + 2 * p);
            const double u2 = oracle_uniform(seed, 5 * (uint64_t)i + 2 + 2 * p);
            const double r = sqrt(-2.0 * log(1.0 - u1));
            z[2 * p] = r * cos(2.0 * M_PI * u2);
            z[2 * p + 1] = r * sin(2.0 * M_PI * u2);
        }
        const double *Lb = L + (size_t)dd * b, *mu = means + (size_t)d * b;
        for (int r = 0; r < d; ++r) {
            double x = mu[r];
            for (int c = 0; c <= r; ++c) x += Lb[r * d + c] * z[c];
            out[(size_t)d * i + r] = (float)x;
        }
        if (comp) comp[i] = b;
    }
    free(L); free(cum);
    return OR_OK;
}

/* ------------------------------------------------------------ GBMS -- */
/* Mode seeking that sets the number of components K (Sec. V, paragraph
 * "Gaussian Blurring Mean Shift", and Fig. "information flow"): seeds from a
 * binned estimator (Comaniciu & Meer 2002), each seed moved to the average of
 * the points within the bandwidth h of it until it stops moving or an iteration
 * limit is reached; the distinct end points are the modes.  Written out:
 *
 *   cells   c_i(x) = floor(x_i / h + 0.5)  (binary64);  one seed per occupied
 *           cell, at c h; seeds in ascending order of the cell key
 *           sum_i (c_i + 2^15) 2^(16 i)  (the last coordinate most significant).
 *   ball    x is within h of m when  s <= (float)(h*h),  s the binary32 squared
 *           distance between x and m rounded to binary32, in the order
 *           ((d0^2 + d1^2) + d2^2) [+ d3^2], each operation rounded (no FMA).
 *   mean    exact sums of q(x_i) = rint(x_i 2^24) in 64-bit integers;
 *           m_i = ((double)S_i / count) 2^-24.
 *   moves   m_0 = seed; m_t = mean of the ball of m_{t-1}; stop after the first
 *           t with ||m_t - m_{t-1}||^2 <= (1e-3 h)^2 (binary64) or t = max_iter;
 *           the mode is m_t with count = the size of that last ball.  A seed
 *           whose ball is empty is dropped.
 *   merge   modes ranked by count (descending), ties by seed order; in rank
 *           order a mode is kept unless a kept mode lies within h of it
 *           (binary64 squared distance <= h*h, coordinate order, no FMA).
 *
 * The fixed point makes the mean independent of the order of summation, so an
 * implementation that gathers the ball in another order reaches the same bits.
 * Requires |x_i| < 2^12 and |c_i| < 2^15 (else OR_ERR_INVALID_ARG).
 * Outputs: *K, modes (K x d binary64, rank order; capacity N x d), counts (K),
 * all may be NULL except K. */
static int cell_of(double v, double h, int32_t *c) {
    const double f = floor(v / h + 0.5);
    if (!(f > -32768.0 && f < 32768.0)) return 0;
    *c = (int32_t)f;
    return 1;
}
static uint64_t cell_key(const int32_t *c, int d) {
    uint64_t k = 0;
    for (int i = 0; i < d; ++i) k |= (uint64_t)(uint32_t)(c[i] + 32768) << (16 * i);
    return k;
}
static int cmp_u64(const void *a, const void *b) {
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}
typedef struct { int32_t count; int32_t seed; } ModeRank;
static int cmp_rank(const void *a, const void *b) {
    const ModeRank *x = (const ModeRank *)a, *y = (const ModeRank *)b;
    if (x->count != y->count) return x->count > y->count ? -1 : 1;
    return (x->seed > y->seed) - (x->seed < y->seed);
}

int oracle_gbms_d(const float *pts, int64_t N, int d, double h, int max_iter, int *K, double *modes_out,
                  int32_t *counts_out) {
    if (N < 1 || !valid_dim(d) || !pts || !K || !(h > 0.0) || !isfinite(h) || max_iter < 1) return OR_ERR_INVALID_ARG;
    if (!all_finite_f(pts, (int64_t)d * N)) return OR_ERR_NONFINITE;
    const float h2f = (float)(h * h);
    const double thr2 = (1e-3 * h) * (1e-3 * h);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * N);
    int64_t *q = (int64_t *)malloc(sizeof(int64_t) * d * N);
    if (!keys || !q) { free(keys); free(q); return OR_ERR_OOM; }
    for (int64_t n = 0; n < N; ++n) {
        int32_t c[DMAX];
        for (int i = 0; i < d; ++i) {
            const float x = pts[(size_t)d * n + i];
            if (!(fabsf(x) < 4096.0f) || !cell_of((double)x, h, &c[i])) { free(keys); free(q); return OR_ERR_INVALID_ARG; }
            q[(size_t)d * n + i] = llrint(ldexp((double)x, 24));
        }
        keys[n] = cell_key(c, d);
    }
    qsort(keys, (size_t)N, sizeof(uint64_t), cmp_u64);
    int64_t S = 0;   /* distinct cells, compacted in place */
    for (int64_t n = 0; n < N; ++n)
        if (n == 0 || keys[n] != keys[n - 1]) keys[S++] = keys[n];
    double *modes = (double *)malloc(sizeof(double) * d * S);
    ModeRank *rank = (ModeRank *)malloc(sizeof(ModeRank) * S);
    if (!modes || !rank) { free(keys); free(q); free(modes); free(rank); return OR_ERR_OOM; }
    int64_t live = 0;
    for (int64_t s = 0; s < S; ++s) {
        double m[DMAX];
        for (int i = 0; i < d; ++i) m[i] = (double)((int32_t)((keys[s] >> (16 * i)) & 0xFFFF) - 32768) * h;
        int32_t count = 0;
        for (int t = 1; t <= max_iter; ++t) {
            float mf[DMAX];
            for (int i = 0; i < d; ++i) mf[i] = (float)m[i];
            int64_t sum[DMAX] = {0, 0, 0, 0};
            count = 0;
            for (int64_t n = 0; n < N; ++n)
                if (dist2_f32(pts + (size_t)d * n, mf, d) <= h2f) {
                    ++count;
                    for (int i = 0; i < d; ++i) sum[i] += q[(size_t)d * n + i];
                }
            if (count == 0) break;
            double mv = 0.0;
            for (int i = 0; i < d; ++i) {
                const double v = ldexp((double)sum[i] / (double)count, -24);
                const double dv = v - m[i];
                mv = (i == 0) ? dv * dv : mv + dv * dv;
                m[i] = v;
            }
            if (mv <= thr2) break;
        }
        if (count == 0) continue;   /* dropped */
        memcpy(modes + (size_t)d * live, m, sizeof(double) * d);
        rank[live].count = count;
        rank[live].seed = (int32_t)live;   /* live modes keep the seed order */
        ++live;
    }
    qsort(rank, (size_t)live, sizeof(ModeRank), cmp_rank);
    int kept = 0;
    int32_t *keep_idx = (int32_t *)malloc(sizeof(int32_t) * (live > 0 ? live : 1));
    if (!keep_idx) { free(keys); free(q); free(modes); free(rank); return OR_ERR_OOM; }
    for (int64_t r = 0; r < live; ++r) {
        const double *a = modes + (size_t)d * rank[r].seed;
        int near = 0;
        for (int j = 0; j < kept && !near; ++j) {
            const double *b = modes + (size_t)d * keep_idx[j];
            double s2 = 0.0;
            for (int i = 0; i < d; ++i) {
                const double dv = a[i] - b[i];
                s2 = (i == 0) ? dv * dv : s2 + dv * dv;
            }
            near = s2 <= h * h;
        }
        if (near) continue;
        if (modes_out) memcpy(modes_out + (size_t)d * kept, a, sizeof(double) * d);
        if (counts_out) counts_out[kept] = rank[r].count;
        keep_idx[kept++] = rank[r].seed;
    }
    *K = kept;
    free(keys); free(q); free(modes); free(rank); free(keep_idx);
    return OR_OK;
}
