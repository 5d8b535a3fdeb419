/*
 * gira_oracle_par.c -- the oracle's EM iteration spread over the host's cores.
 *
 * TEST INFRASTRUCTURE ONLY, like gira_oracle.c (nothing in the product library
 * links, calls or includes it).  It computes exactly what oracle_em_d and
 * oracle_estep_d compute (GIRA, arXiv 2307.00071, Sec. V: the E-step of
 * Eq. (estep) in the log domain of Eq. (logestep) with the log-density of
 * Eq. (simplifiedGaussian); the standard full-covariance M-step with the
 * scikit-learn conventions: N_b = sum r + 10 eps64, pi = N_b / sum N,
 * mu = sum r x / N_b, Sigma = sum r (x - mu)(x - mu)^T / N_b + reg I, two passes
 * with exact centring).  Two things differ, neither in the arithmetic of a
 * single point:
 *
 *   - every sum over points is taken over fixed chunks of PAR_CHUNK points
 *     (each chunk in point order), and the chunk sums are added in chunk
 *     order.  The result is therefore the same whatever the number of threads,
 *     and differs from the single-threaded oracle only by the order of the
 *     binary64 additions (relative 1e-15 per sum);
 *   - the N x K responsibility matrix is not stored: the M-step's second pass
 *     (the centred second moments) recomputes each point's responsibilities
 *     with the same expressions, which gives the same values bit for bit.
 *     This is what lets it run at N = 4M, K = 8192.
 *
 * Per point it evaluates Eq. (simplifiedGaussian) with the expressions of the
 * single-threaded oracle_log_gaussian_d, in the same order, except that the
 * log-determinant sum_i ln P_ii (the same sum, in the same order) is taken once
 * per component instead of once per point; the values are the same bit for bit
 * (pinned against the single-threaded E-step).
 */
#include <float.h>
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DMAX 4
#define PAR_CHUNK 1024 /* points per chunk (the unit of every partial sum) */
#define PAR_GROUP 64   /* chunks summed in parallel before their ordered combine */

enum { OR_OK = 0, OR_ERR_INVALID_ARG = 1, OR_ERR_NONFINITE = 2, OR_ERR_NOT_PD = 3, OR_ERR_OOM = 5 };

/* from gira_oracle.c */
int oracle_cholesky_d(const double *S, double *L, int d);
void oracle_tri_inverse_d(const double *L, double *P, int d);
void oracle_note_bad_component(int b);

/* OpenMP's default team size (OMP_NUM_THREADS, else every core); never changed here */
int oracle_max_threads(void) { return omp_get_max_threads(); }
static int team(int threads) { return threads > 0 ? threads : omp_get_max_threads(); }

typedef struct {
    int K, d;
    const double *logw, *logdet, *means, *P;
} Model;

/* Eq. (simplifiedGaussian): ln N(x | mu, Sigma) with P = L^{-1} and
 * logdet = sum_i ln P_ii; the expressions of oracle_log_gaussian_d. */
static double log_gaussian(const double *x, const double *mu, const double *P, double logdet, int d) {
    double q = 0.0;
    for (int i = 0; i < d; ++i) {
        double y = 0.0;
        for (int j = 0; j <= i; ++j) y += P[i * d + j] * (x[j] - mu[j]);
        q += y * y;
    }
    return -0.5 * (d * log(2.0 * M_PI) + q) + logdet;
}

/* One point: a[b] <- r_nb (responsibilities); returns lse_n = ln sum_b pi_b N(x_n|b).
 * The same expressions, in the same order, as oracle_estep_d. */
static double point_resp(const Model *M, const float *xp, double *a) {
    const int K = M->K, d = M->d, dd = d * d;
    double x[DMAX];
    for (int i = 0; i < d; ++i) x[i] = xp[i];
    double m = -INFINITY;
    for (int b = 0; b < K; ++b) {
        a[b] = M->logw[b] + log_gaussian(x, M->means + (size_t)d * b, M->P + (size_t)dd * b, M->logdet[b], d);
        if (a[b] > m) m = a[b];
    }
    double s = 0.0;
    for (int b = 0; b < K; ++b) s += exp(a[b] - m);
    const double l = m + log(s);
    for (int b = 0; b < K; ++b) a[b] = exp(a[b] - l);
    return l;
}

static int finite_inputs(const float *pts, int64_t N, int K, int d, const double *w, const double *mu,
                         const double *cov) {
    for (int64_t i = 0; i < (int64_t)d * N; ++i)
        if (!isfinite(pts[i])) return 0;
    for (int64_t i = 0; i < K; ++i)
        if (!isfinite(w[i])) return 0;
    for (int64_t i = 0; i < (int64_t)d * K; ++i)
        if (!isfinite(mu[i])) return 0;
    for (int64_t i = 0; i < (int64_t)d * d * K; ++i)
        if (!isfinite(cov[i])) return 0;
    return 1;
}

/* logw and logdet: 2K doubles */
static int model_setup(int K, int d, const double *weights, const double *means, const double *covs, double *logw,
                       double *P, Model *M) {
    const int dd = d * d;
    double *logdet = logw + K;
    for (int b = 0; b < K; ++b) {
        double L[DMAX * DMAX];
        if (oracle_cholesky_d(covs + (size_t)dd * b, L, d) != 0) {
            oracle_note_bad_component(b);
            return OR_ERR_NOT_PD;
        }
        double *Pb = P + (size_t)dd * b;
        oracle_tri_inverse_d(L, Pb, d);
        logw[b] = log(weights[b]);
        double ld = 0.0;
        for (int i = 0; i < d; ++i) ld += log(Pb[i * d + i]);
        logdet[b] = ld;
    }
    M->K = K;
    M->d = d;
    M->logw = logw;
    M->logdet = logdet;
    M->means = means;
    M->P = P;
    return OR_OK;
}

/* Per-point log-likelihood (lse may be NULL) and its mean, over all cores. */
int oracle_estep_par_d(const float *pts, int64_t N, int K, int d, const double *weights, const double *means,
                       const double *covs, double *lse, double *mean_ll, int threads) {
    if (N < 1 || K < 1 || (d != 3 && d != 4) || !pts || !weights || !means || !covs || !mean_ll)
        return OR_ERR_INVALID_ARG;
    if (!finite_inputs(pts, N, K, d, weights, means, covs)) return OR_ERR_NONFINITE;
    const int nt = team(threads);
    double *logw = malloc(sizeof(double) * 2 * K), *P = malloc(sizeof(double) * d * d * K);
    const int64_t nch = (N + PAR_CHUNK - 1) / PAR_CHUNK;
    double *part = malloc(sizeof(double) * nch);
    if (!logw || !P || !part) { free(logw); free(P); free(part); return OR_ERR_OOM; }
    Model M;
    int st = model_setup(K, d, weights, means, covs, logw, P, &M);
    int oom = 0;
    if (st == OR_OK) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
        for (int64_t c = 0; c < nch; ++c) {
            double *a = malloc(sizeof(double) * K);
            if (!a) {
#pragma omp atomic write
                oom = 1;
                continue;
            }
            const int64_t n0 = c * PAR_CHUNK, n1 = (n0 + PAR_CHUNK < N) ? n0 + PAR_CHUNK : N;
            double s = 0.0;
            for (int64_t n = n0; n < n1; ++n) {
                const double l = point_resp(&M, pts + (size_t)d * n, a);
                if (lse) lse[n] = l;
                s += l;
            }
            part[c] = s;
            free(a);
        }
        if (oom) st = OR_ERR_OOM;
    }
    if (st == OR_OK) {
        double t = 0.0;
        for (int64_t c = 0; c < nch; ++c) t += part[c];
        *mean_ll = t / (double)N;
    }
    free(logw);
    free(P);
    free(part);
    return st;
}

/* One EM iteration (E-step, then the M-step's two passes) over all cores.
 * ll <- mean per-point log-likelihood under the parameters going in; the
 * parameters are replaced by the M-step's. */
static int em_iteration(const float *pts, int64_t N, int K, int d, double reg, double *weights, double *means,
                        double *covs, double *ll, int nt) {
    const int dd = d * d;
    const int64_t nch = (N + PAR_CHUNK - 1) / PAR_CHUNK;
    const size_t w1 = 1 + (size_t)K * (1 + d); /* pass 1 partial: ll, N_b, sum r x */
    const size_t w2 = (size_t)K * dd;          /* pass 2 partial: sum r (x-mu)(x-mu)^T */
    double *logw = malloc(sizeof(double) * 2 * K), *P = malloc(sizeof(double) * dd * K);
    double *tot1 = calloc(w1, sizeof(double)), *tot2 = calloc(w2, sizeof(double));
    double *grp = malloc(sizeof(double) * PAR_GROUP * (w1 > w2 ? w1 : w2));
    double *mu = malloc(sizeof(double) * d * K), *nb = malloc(sizeof(double) * K);
    if (!logw || !P || !tot1 || !tot2 || !grp || !mu || !nb) {
        free(logw); free(P); free(tot1); free(tot2); free(grp); free(mu); free(nb);
        return OR_ERR_OOM;
    }
    Model M;
    int st = model_setup(K, d, weights, means, covs, logw, P, &M);
    int oom = 0;
    for (int pass = 1; pass <= 2 && st == OR_OK; ++pass) {
        const size_t w = (pass == 1) ? w1 : w2;
        double *tot = (pass == 1) ? tot1 : tot2;
        for (int64_t g0 = 0; g0 < nch && !oom; g0 += PAR_GROUP) {
            const int ng = (int)((nch - g0 < PAR_GROUP) ? nch - g0 : PAR_GROUP);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
            for (int j = 0; j < ng; ++j) {
                double *acc = grp + (size_t)j * w;
                memset(acc, 0, sizeof(double) * w);
                double *a = malloc(sizeof(double) * K);
                if (!a) {
#pragma omp atomic write
                    oom = 1;
                    continue;
                }
                const int64_t n0 = (g0 + j) * PAR_CHUNK, n1 = (n0 + PAR_CHUNK < N) ? n0 + PAR_CHUNK : N;
                for (int64_t n = n0; n < n1; ++n) {
                    const float *xp = pts + (size_t)d * n;
                    const double l = point_resp(&M, xp, a);
                    if (pass == 1) {
                        acc[0] += l;
                        for (int b = 0; b < K; ++b) {
                            const double r = a[b];
                            acc[1 + b] += r;
                            double *sx = acc + 1 + K + (size_t)d * b;
                            for (int i = 0; i < d; ++i) sx[i] += r * (double)xp[i];
                        }
                    } else {
                        for (int b = 0; b < K; ++b) {
                            const double r = a[b];
                            double dv[DMAX];
                            for (int i = 0; i < d; ++i) dv[i] = (double)xp[i] - mu[(size_t)d * b + i];
                            double *c = acc + (size_t)dd * b;
                            for (int i = 0; i < d; ++i)
                                for (int k = 0; k < d; ++k) c[i * d + k] += r * dv[i] * dv[k];
                        }
                    }
                }
                free(a);
            }
            /* ordered combine: chunk g0, g0 + 1, ... */
            for (int j = 0; j < ng; ++j) {
                const double *acc = grp + (size_t)j * w;
                for (size_t i = 0; i < w; ++i) tot[i] += acc[i];
            }
        }
        if (oom) { st = OR_ERR_OOM; break; }
        if (pass == 1) {
            *ll = tot1[0] / (double)N;
            const double tiny = 10.0 * DBL_EPSILON;
            for (int b = 0; b < K; ++b) {
                nb[b] = tot1[1 + b] + tiny;
                for (int i = 0; i < d; ++i) mu[(size_t)d * b + i] = tot1[1 + K + (size_t)d * b + i] / nb[b];
            }
        }
    }
    if (st == OR_OK) {
        double nsum = 0.0;
        for (int b = 0; b < K; ++b) {
            double *c = covs + (size_t)dd * b;
            for (int i = 0; i < dd; ++i) c[i] = tot2[(size_t)dd * b + i] / nb[b];
            for (int i = 0; i < d; ++i) c[i * d + i] += reg;
            memcpy(means + (size_t)d * b, mu + (size_t)d * b, sizeof(double) * d);
            weights[b] = nb[b];
            nsum += nb[b];
        }
        for (int b = 0; b < K; ++b) weights[b] /= nsum;
        for (int b = 0; b < K; ++b) {
            double L[DMAX * DMAX];
            if (oracle_cholesky_d(covs + (size_t)dd * b, L, d) != 0) {
                oracle_note_bad_component(b);
                st = OR_ERR_NOT_PD;
                break;
            }
        }
    }
    free(logw); free(P); free(tot1); free(tot2); free(grp); free(mu); free(nb);
    return st;
}

/* EM from the given parameters (in/out), the same iteration and stopping rule
 * as oracle_em_d: iteration t stores ll_t (before its M-step) in trace[t-1];
 * stop after `iters` or when t > 1 and |ll_t - ll_{t-1}| < tol.  final_ll (may
 * be NULL) is the mean log-likelihood of the returned parameters.  threads <= 0:
 * OpenMP's default (every core). */
int oracle_em_par_d(const float *pts, int64_t N, int K, int d, int iters, double tol, double reg, double *weights,
                    double *means, double *covs, double *trace, int *iters_done, double *final_ll, int threads) {
    if (N < 1 || K < 1 || (d != 3 && d != 4) || iters < 0 || !(tol >= 0.0) || !(reg >= 0.0) || !pts || !weights ||
        !means || !covs)
        return OR_ERR_INVALID_ARG;
    if (!finite_inputs(pts, N, K, d, weights, means, covs)) return OR_ERR_NONFINITE;
    double prev = -INFINITY;
    int t = 0, st = OR_OK;
    while (t < iters) {
        double ll;
        st = em_iteration(pts, N, K, d, reg, weights, means, covs, &ll, team(threads));
        if (st != OR_OK) break;
        if (trace) trace[t] = ll;
        ++t;
        if (fabs(ll - prev) < tol) break;
        prev = ll;
    }
    if (iters_done) *iters_done = t;
    if (st == OR_OK && final_ll) st = oracle_estep_par_d(pts, N, K, d, weights, means, covs, NULL, final_ll, threads);
    return st;
}
