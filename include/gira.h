/*
 * gira.h -- C ABI of libgira: EM fitting of full-covariance Gaussian mixture
 * models to point clouds (xyz, or xyz + intensity) on one NVIDIA GB300 (sm_103a),
 * with the log-likelihood, its gradient, intensity regression, sampling and the
 * mode seeking that sets the number of components.
 *
 * The operations follow GIRA (Goel & Tabib, arXiv 2307.00071), Sec. V
 * "Implementation Details": KInit (Fig. "information flow": a k-means
 * initialisation yields the responsibilities EM starts from), the E-step
 * (Eq. estep, computed in the log form of Eq. logestep with the Cholesky
 * log-density of Eq. simplifiedGaussian) and the M-step.  The model layout is
 * the paper's (Sec. V: weights (1,K,1), means (1,K,D), covariances (1,K,D,D))
 * with D = 3 (the calls without a suffix) or D = 4 (the calls ending in 4).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Points are N x D binary32, row-major (x0,y0,z0,x1,... for D = 3), N >= 1.
 *  - Pointer arguments marked [host|device] may point to host memory or to
 *    device memory of the current CUDA device; the library detects which
 *    (cudaPointerGetAttributes).  Host buffers are staged through
 *    library-owned device memory; the copies are part of the call.
 *    Pointers marked [host] must be host memory.
 *  - The caller owns every buffer it passes.  The library owns a device
 *    workspace cached per device (grown on demand, freed by
 *    gira_release_workspace).  Calls on one device are serialised by a
 *    per-device lock.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All GPU
 *    work is issued on it; every call synchronises that stream before it
 *    returns, so outputs are ready when the call returns.
 *  - Errors are returned as gira_status; nothing aborts.  On error the
 *    outputs are unspecified; gira_last_error_message() (thread-local) says
 *    why and gira_last_error_component() names the offending component for
 *    GIRA_ERR_NOT_PD.
 */
#ifndef GIRA_H
#define GIRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GIRA_OK = 0,
    GIRA_ERR_INVALID_ARG = 1,      /* N < 1, K < 1, K > N, K > GIRA_MAX_K, iters < 0, tol < 0 or NaN,
                                      reg_covar < 0 or NaN, a required pointer NULL, weights <= 0 */
    GIRA_ERR_NONFINITE_INPUT = 2,  /* NaN or Inf in the points or in caller-supplied parameters */
    GIRA_ERR_NOT_PD = 3,           /* a covariance has no Cholesky factor (pivot <= 0 after reg_covar) */
    GIRA_ERR_CUDA = 4,             /* a CUDA runtime call failed; the message carries cudaGetErrorString */
    GIRA_ERR_OOM = 5,              /* the device workspace could not be allocated */
    GIRA_ERR_TIMEOUT = 6,          /* reserved for bounded device-side waits */
    GIRA_ERR_NUMERIC = 7,          /* a point's likelihood underflows binary32 under every component */
    GIRA_ERR_BOUNDS = 8            /* libraries built with GIRA_DEBUG only: a device-side index fell outside
                                      its buffer; the access was skipped */
} gira_status;

/* Largest number of mixture components one call accepts. */
#define GIRA_MAX_K 8192        /* gira_gmm_fit, gira_gmm_loglik, gira_kmeans_init */
#define GIRA_MAX_K_BATCHED 1024 /* per instance of gira_gmm_fit_batched; gira_gmm_loglik_grad;
                                   gira_gmm_loglik_noalloc */

typedef enum {
    GIRA_INIT_KMEANS = 0,  /* k-means++ (seed) + Lloyd (lloyd_iters) + one-hot M-step */
    GIRA_INIT_PARAMS = 1   /* start from the weights/means/covs passed in (they are read, then overwritten) */
} gira_init_mode;

typedef struct {
    int iters;          /* maximum EM iterations (>= 0) */
    double tol;         /* stop after iteration t > 1 when |l_t - l_{t-1}| < tol (mean per-point loglik); 0 = never */
    double reg_covar;   /* added to every covariance diagonal after each M-step (m^2), >= 0 */
    uint64_t seed;      /* k-means++ seed (SplitMix64 counter stream) */
    int lloyd_iters;    /* Lloyd iterations after k-means++ (>= 0; stops early when no label changes) */
    int init_mode;      /* gira_init_mode */
} gira_fit_opts;

/* Fill `opts` with the defaults: iters 100, tol 1e-3, reg_covar 1e-6, seed 0, lloyd_iters 10,
 * init_mode GIRA_INIT_KMEANS. */
void gira_fit_opts_default(gira_fit_opts *opts);

/*
 * gira_kmeans_init -- KInit seeding (Sec. V, Fig. "information flow").
 *
 * k-means++ (Arthur & Vassilvitskii 2007, one candidate per step): centre 0
 * is point floor(u_0 N); for centre j every point's weight is its binary32
 * squared distance D^2 to the nearest centre chosen so far (fixed order
 * (d0^2 + d1^2) + d2^2, no fused multiply-add), taken in exact fixed point as
 * the integer floor(D^2 2^48) (saturating at 2^95 - 1); with T the exact
 * integer total and k_j the top 53 bits of draw j of the SplitMix64 counter
 * stream of `seed` (u_j = k_j / 2^53), centre j is the first point n whose
 * exact running sum exceeds floor(k_j T / 2^53) (if T = 0: point
 * floor(u_j N)).  No rounding enters the choice, so the centres do not depend
 * on the order in which the GPU sums.  Then Lloyd iterations:
 * labels = argmin_b ||x - c_b||^2 (binary32, ties to the lowest b), centres
 * = binary64 mean of their points rounded to binary32 (empty clusters keep
 * their centre), until no label changes or `lloyd_iters` updates were made.
 *
 *   points       [host|device] N x 3 binary32 (read)
 *   n, k         1 <= k <= n, k <= GIRA_MAX_K
 *   centers      [host|device] K x 3 binary32 (written)
 *   labels       [host|device] N int32 final labels (written), or NULL
 *   iters_done   [host] number of Lloyd centre updates made, or NULL
 */
gira_status gira_kmeans_init(const float *points, int64_t n, int k, uint64_t seed, int lloyd_iters,
                             float *centers, int32_t *labels, int *iters_done, void *stream);

/*
 * gira_gmm_fit -- EM fit of a K-component full-covariance GMM (Sec. V).
 *
 * Initialisation per opts->init_mode.  Iteration t = 1, 2, ...: the E-step
 * with the current parameters gives the mean per-point log-likelihood l_t
 * (stored in loglik_trace[t-1]) and the sufficient statistics of the
 * responsibilities; the M-step then sets
 *   N_b = sum_n r_nb + 10 eps64,  pi_b = N_b / sum_a N_a,
 *   mu_b = sum_n r_nb x_n / N_b,
 *   Sigma_b = sum_n r_nb (x_n - mu_b)(x_n - mu_b)^T / N_b + reg_covar I.
 * The loop ends after opts->iters iterations, or after iteration t > 1 with
 * |l_t - l_{t-1}| < opts->tol.
 *
 *   points        [host|device] N x 3 binary32 (read)
 *   weights       [host|device] K binary32          (written; read first when GIRA_INIT_PARAMS)
 *   means         [host|device] K x 3 binary32      (same)
 *   covs          [host|device] K x 3 x 3 binary32  (same; symmetric positive definite when read)
 *   loglik_trace  [host] opts->iters binary64, or NULL
 *   iters_done    [host] iterations run, or NULL
 *   final_loglik  [host] mean per-point log-likelihood of the returned parameters, or NULL
 */
gira_status gira_gmm_fit(const float *points, int64_t n, int k, const gira_fit_opts *opts, float *weights,
                         float *means, float *covs, double *loglik_trace, int *iters_done,
                         double *final_loglik, void *stream);

/*
 * gira_gmm_fit_batched -- gira_gmm_fit for many independent point clouds of
 * uneven sizes and component counts in one call (an engineering extension:
 * the paper fits one cloud at a time).  Every instance follows exactly the
 * single fit's definition (KInit of Fig. "information flow", the E-step of
 * Eq. estep / logestep / simplifiedGaussian, the M-step and stopping rule of
 * gira_gmm_fit), with its own convergence: an instance that has converged
 * stops updating while the others go on.  The EM iterations of all instances
 * run as one CUDA graph: per iteration one E-step launch per block shape (the
 * instances with the same ceil(K / 128)) and one binary64 finalize launch.
 * Points per CTA are chosen by timing candidates on the first call for a
 * shape and size, and cached for the process.
 *
 *   points          [host|device] sum_i N_i x 3 binary32, instance i at rows
 *                   offsets[i] .. offsets[i+1]-1
 *   offsets         [host] batch + 1 int64, offsets[0] = 0, strictly increasing
 *   ks              [host] batch ints, 1 <= ks[i] <= min(N_i, GIRA_MAX_K_BATCHED)
 *   opts            as gira_gmm_fit (the same for every instance)
 *   weights, means, covs  [host|device] sum_i K_i, x 3, x 3 x 3 binary32:
 *                   instance i at components sum_{j<i} K_j ..; output (and
 *                   input with GIRA_INIT_PARAMS)
 *   loglik_traces   [host] batch x opts->iters binary64 (row i: instance i;
 *                   NaN after it stopped), or NULL
 *   iters_done      [host] batch ints, or NULL
 *   final_loglik    [host] batch binary64 mean log-likelihoods, or NULL
 *   statuses        [host] batch gira_status values of the instances, or NULL
 * Returns GIRA_OK when every instance succeeded, else the status of the first
 * failing instance (the others' results are still written).
 */
gira_status gira_gmm_fit_batched(const float *points, const int64_t *offsets, int batch, const int *ks,
                                 const gira_fit_opts *opts, float *weights, float *means, float *covs,
                                 double *loglik_traces, int *iters_done, double *final_loglik, int *statuses,
                                 void *stream);

/*
 * gira_gmm_loglik -- per-point log-likelihood under a GMM: the log-sum-exp of
 * Eq. logestep, ln sum_b pi_b N(x_n | mu_b, Sigma_b), with ln N from
 * Eq. simplifiedGaussian.
 *
 *   points       [host|device] N x 3 binary32
 *   weights      [host|device] K binary32, > 0 (used as given; not renormalised)
 *   means        [host|device] K x 3 binary32
 *   covs         [host|device] K x 3 x 3 binary32, symmetric positive definite
 *   mean_loglik  [host] (1/N) sum_n ln p(x_n) (written), or NULL
 *   per_point    [host|device] N binary32 ln p(x_n) (written), or NULL
 */
gira_status gira_gmm_loglik(const float *points, int64_t n, int k, const float *weights, const float *means,
                            const float *covs, double *mean_loglik, float *per_point, void *stream);

/*
 * gira_gmm_loglik_grad -- the log-likelihood of a rigidly moved scan and its
 * gradient (an extension beyond the paper, whose own registration is its
 * distribution-to-distribution method): with x'_n = R x_n + t,
 *   L = sum_n ln sum_b pi_b N(x'_n | mu_b, L_b L_b^T),  pi = softmax(logits),
 * the per-component log-density of Eq. simplifiedGaussian with P = L_b^{-1}
 * and the log-sum-exp of Eq. logestep.  Gradients (gamma = responsibility,
 * y = L_b^{-1}(x' - mu_b)), all in one pass that recomputes gamma and never
 * stores it:
 *   dL/dx_n      = R^T dL/dx'_n,   dL/dx'_n = -sum_b gamma_nb Sigma_b^{-1}(x'_n - mu_b)
 *   dL/dR, dL/dt = sum_n dL/dx'_n x_n^T,  sum_n dL/dx'_n
 *   dL/dtwist    = (sum_n x'_n x dL/dx'_n, sum_n dL/dx'_n): twist (omega, v) of a
 *                  left perturbation x' <- exp(twist^) x', rotation first
 *   dL/dlogits_b = sum_n gamma_nb - N pi_b
 *   dL/dmeans_b  = sum_n gamma_nb Sigma_b^{-1}(x'_n - mu_b)
 *   dL/dchol_b   = lower triangle of sum_n gamma_nb (L_b^{-T} y y^T - diag(1/L_b,ii))
 *
 *   points       [host|device] N x 3 binary32 (the scan before the move)
 *   pose12       [host|device] R row-major (9) then t (3), binary32, or NULL (identity)
 *   logits       [host|device] K binary32
 *   means        [host|device] K x 3 binary32
 *   chol         [host|device] K x 3 x 3 binary32 row-major; the lower triangle is
 *                read, the diagonal must be > 0 (else GIRA_ERR_NOT_PD)
 *   loglik       [host] L (a sum over points, binary64), or NULL
 *   grad_points  [host|device] N x 3 binary32, or NULL
 *   grad_pose    [host|device] 12 binary64: dL/dR (row-major 3x3) then dL/dt, or NULL
 *   grad_twist   [host|device] 6 binary64 (omega, v), or NULL
 *   grad_logits  [host|device] K binary32, or NULL
 *   grad_means   [host|device] K x 3 binary32, or NULL
 *   grad_chol    [host|device] K x 3 x 3 binary32 (zeros above the diagonal), or NULL
 * With every gradient pointer NULL only the log-likelihood pass runs.
 */
gira_status gira_gmm_loglik_grad(const float *points, int64_t n, int k, const float *pose12, const float *logits,
                                 const float *means, const float *chol, double *loglik, float *grad_points,
                                 double *grad_pose, double *grad_twist, float *grad_logits, float *grad_means,
                                 float *grad_chol, void *stream);

/*
 * gira_gmm_loglik_grad_batched -- gira_gmm_loglik_grad for a batch of scans,
 * each with its own model and pose (e.g. many registrations advanced together);
 * the whole evaluation (moving the scans, building the parameters, the adjoint
 * E-step per block shape, the binary64 gradients) runs as one CUDA graph,
 * cached per workspace and batch signature.
 *
 *   points, offsets, ks   as gira_gmm_fit_batched (ks[i] <= GIRA_MAX_K_BATCHED)
 *   poses                 [host|device] batch x 12 binary32 (R row-major, t), or NULL
 *   logits, means, chol   [host|device] stacked over instances (sum K, x 3, x 3 x 3)
 *   logliks               [host] batch binary64 L_i, or NULL
 *   grad_points           [host|device] sum N x 3 binary32, or NULL
 *   grad_pose, grad_twist [host|device] batch x 12, batch x 6 binary64, or NULL
 *   grad_logits, grad_means, grad_chol  [host|device] stacked, binary32, or NULL
 *   statuses              [host] batch gira_status values, or NULL
 * Every gradient is computed (NULL only skips its copy-out).  Returns the
 * status of the first failing instance, else GIRA_OK.
 */
gira_status gira_gmm_loglik_grad_batched(const float *points, const int64_t *offsets, int batch, const int *ks,
                                         const float *poses, const float *logits, const float *means,
                                         const float *chol, double *logliks, float *grad_points, double *grad_pose,
                                         double *grad_twist, float *grad_logits, float *grad_means,
                                         float *grad_chol, int *statuses, void *stream);

/*
 * Four dimensions: position and intensity (the paper's (1,K,D) / (1,K,D,D)
 * model layout with D = 4, as in its SOGMM intensity data).
 *
 * gira_gmm_fit4 -- gira_gmm_fit for N x 4 binary32 points (x, y, z, intensity),
 * rows contiguous.  The same KInit (k-means++ and Lloyd with squared distances
 * over all four coordinates, binary32 in the order ((d0^2 + d1^2) + d2^2) + d3^2),
 * the same E-step (Eq. estep / logestep with the log-density of
 * Eq. simplifiedGaussian for D = 4) and M-step, the same opts and stopping rule.
 * k <= GIRA_MAX_K4 (above 1024 the log-sum-exp runs in two levels, over chunks
 * of 512 components, with the exact per-point maximum for points whose total
 * underflows, as gira_gmm_fit does).
 *   weights [host|device] K binary32, means K x 4, covs K x 4 x 4 (row-major;
 *   the lower triangle is read when GIRA_INIT_PARAMS), written on return.
 */
#define GIRA_MAX_K4 8192   /* above 1024: the E-step runs over chunks of 512 components */
gira_status gira_gmm_fit4(const float *points, int64_t n, int k, const gira_fit_opts *opts, float *weights,
                          float *means, float *covs, double *loglik_trace, int *iters_done, double *final_loglik,
                          void *stream);

/* gira_gmm_loglik4 -- gira_gmm_loglik for N x 4 points and a D = 4 mixture (k <= GIRA_MAX_K4). */
gira_status gira_gmm_loglik4(const float *points, int64_t n, int k, const float *weights, const float *means,
                             const float *covs, double *mean_loglik, float *per_point, void *stream);

/*
 * gira_gmm_conditional4 -- Gaussian-mixture regression of the 4th coordinate
 * (intensity) on the first three at M query positions (Sec. IV: intensity
 * inferred from the joint model at any resolution).  With the blocks
 * Sigma_b = [[S_xx, S_xI], [S_Ix, S_II]]:
 *   w_b(x)  proportional to pi_b N(x | mu_b,xyz, S_xx)          (normalised over b)
 *   m_b(x)  = mu_b,I + S_Ix S_xx^{-1} (x - mu_b,xyz),  v_b = S_II - S_Ix S_xx^{-1} S_xI
 *   mean(x) = sum_b w_b m_b,  var(x) = sum_b w_b (v_b + m_b^2) - mean(x)^2.
 *
 *   locs         [host|device] M x 3 binary32
 *   weights      [host|device] K binary32 (> 0), means K x 4, covs K x 4 x 4 (lower triangle read)
 *   cond_mean    [host|device] M binary32 (written)
 *   cond_var     [host|device] M binary32 (written), or NULL
 */
gira_status gira_gmm_conditional4(const float *locs, int64_t m, int k, const float *weights, const float *means,
                                  const float *covs, float *cond_mean, float *cond_var, void *stream);

/*
 * gira_gmm_sample -- M draws from a d-dimensional mixture (d = 3 or 4; Sec. IV:
 * resampling a point cloud from the model).  Sample i takes draws 5i .. 5i+4 of
 * the SplitMix64 counter stream of `seed` (top 53 bits / 2^53): the first picks
 * the component, the first b whose running binary64 sum of weights exceeds
 * u * sum_a pi_a; the others give four standard normals by the Box-Muller
 * transform, z = sqrt(-2 ln(1 - u1)) (cos, sin)(2 pi u2) for (u1, u2) = draws
 * (5i+1, 5i+2) and (5i+3, 5i+4); x = mu_b + L_b z with L_b the binary64
 * Cholesky factor of Sigma_b, rounded to binary32.
 *
 *   weights      [host|device] K binary32 (>= 0, not all zero), means K x d, covs K x d x d
 *   out          [host|device] M x d binary32 (written)
 *   components   [host|device] M int32 (written), or NULL
 */
gira_status gira_gmm_sample(int64_t m, int k, int d, const float *weights, const float *means, const float *covs,
                            uint64_t seed, float *out, int32_t *components, void *stream);

/*
 * gira_gbms -- the number of components from a bandwidth (Sec. V, paragraph
 * "Gaussian Blurring Mean Shift", and Fig. "information flow": the step before
 * KInit).  Seeds from a binned estimator, each moved to the average of the
 * points within the bandwidth h of it until it stops; the distinct end points
 * (modes) give K.  Exactly:
 *   cells   c_i(x) = floor(x_i / h + 0.5) (binary64); one seed per occupied
 *           cell, at c h, in ascending order of sum_i (c_i + 2^15) 2^(16 i)
 *   ball    points whose binary32 squared distance to m (rounded to binary32),
 *           ((d0^2 + d1^2) + d2^2) [+ d3^2] without FMA, is <= (float)(h*h)
 *   mean    ((double)S_i / count) * 2^-24 with S_i the exact 64-bit sum of
 *           rint(x_i * 2^24) over the ball (independent of summation order)
 *   stop    after the first move with ||m_t - m_{t-1}||^2 <= (1e-3 h)^2
 *           (binary64) or after max_iter moves; a seed whose ball empties is
 *           dropped; count = the size of its last ball
 *   merge   modes ranked by count (descending), ties by seed order; a mode is
 *           kept unless a kept mode of lower rank is within h (binary64
 *           squared distance <= h*h)
 *
 *   points     [host|device] N x d binary32, d = 3 (xyz) or 4 (xyz + intensity);
 *              |x_i| < 4096 and |c_i| < 32768 (else GIRA_ERR_INVALID_ARG)
 *   bandwidth  h > 0
 *   max_iter   >= 1 (moves per seed)
 *   k          [host] number of modes K (written)
 *   modes      [host|device] capacity N x d binary64: the K modes in rank order, or NULL
 *   counts     [host|device] capacity N int32: each mode's count, or NULL
 */
gira_status gira_gbms(const float *points, int64_t n, int d, double bandwidth, int max_iter, int *k,
                      double *modes, int32_t *counts, void *stream);

/*
 * Profiling (off by default; process-wide).  When enabled, each call records
 * CUDA events on its stream around its phases and around every launch of the
 * fused E-step/statistics kernel, and accumulates the device times below when
 * it synchronises.  Times are device times in milliseconds.
 */
typedef struct {
    long long calls;            /* library calls accumulated */
    long long kernel_launches;  /* kernels those calls launched (early-exiting ones included) */
    long long estep_launches;   /* launches of the fused E-step/statistics kernel that did work */
    double estep_ms;            /* summed duration of those launches */
    long long em_iters;         /* EM iterations run */
    double init_ms;             /* pack + KInit (k-means++, Lloyd, one-hot M-step) or parameter upload */
    double em_ms;               /* the EM loop: E-step, reduction and FP64 finalize of every iteration */
    double total_ms;            /* whole calls, first upload to last download */
    char estep_kernel[128];     /* name of the last E-step kernel timed launch by launch ("" if none) */
    /* gira_gmm_fit's point-stationary E-step, over the launches timed launch by launch
       (warps x component pairs): the pairs a dense E-step would evaluate, those within
       reach of the warp's points (evaluated), and those with statistics */
    long long estep_pair_slots;
    long long estep_pairs_near;
    long long estep_pairs_live;
} gira_profile;

/*
 * Profiling: on = 0 off; on = 2 CUDA events at the phase boundaries of each call
 * (init_ms, em_ms, total_ms); any other nonzero value also brackets every
 * E-step launch with an event pair (estep_launches, estep_ms), for which the EM
 * loop launches its kernels plainly instead of as programmatic dependents of
 * one another (the results are the same).
 */
void gira_profile_enable(int on);

/* Copy the accumulated profile to *out (may be NULL); reset it when reset != 0. */
gira_status gira_profile_read(gira_profile *out, int reset);

/*
 * gira_gmm_loglik_noalloc -- gira_gmm_loglik for callers that cannot allocate
 * device memory.  (An engineering addition: the paper has no counterpart.)
 *
 * Who needs it: real-time control loops that forbid allocation after start-up
 * (cudaMalloc can block for an unbounded time, and can fail in the middle of a
 * run), and hosts whose device memory is owned by a pool they do not control
 * (memory the library took would be missing from the pool's budget).  It
 * computes the same mean and per-point log-likelihoods as
 * gira_gmm_loglik, with the same kernels, but never calls cudaMalloc,
 * cudaFree or any allocating routine: its scratch (packed points, component
 * parameters, per-CTA partial sums, status word) is one static device array of
 * 17 MiB inside the library, which every GPU that loads the library keeps until
 * the process exits.
 *
 *   points, weights, means, covs   device memory of the current device only
 *                                  (same layouts as gira_gmm_loglik)
 *   n                              1 <= n <= GIRA_NOALLOC_MAX_N, else GIRA_ERR_INVALID_ARG
 *   k                              1 <= k <= min(n, GIRA_MAX_K_BATCHED)
 *   mean_loglik                    [host] or NULL
 *   per_point                      [device] N binary32, or NULL
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * previous call's contents (the call re-initialises what it reads), so calls
 * that overlap on the GPU -- on different streams, or from processes sharing a
 * context -- race and must not be issued; calls from several host threads are
 * serialised by a lock.  The call synchronises `stream` before returning, so
 * it cannot be recorded into a CUDA graph: on a stream under capture it
 * returns GIRA_ERR_INVALID_ARG and leaves the capture untouched.
 */
#define GIRA_NOALLOC_MAX_N 524288
gira_status gira_gmm_loglik_noalloc(const float *points, int64_t n, int k, const float *weights,
                                    const float *means, const float *covs, double *mean_loglik,
                                    float *per_point, void *stream);

/*
 * Test hooks: failures made on purpose without faulting the GPU.
 *
 * gira_test_fail_next_allocations -- the next `count` workspace allocations
 * (made when a call needs more device workspace than is cached) fail with
 * GIRA_ERR_OOM before cudaMalloc is called; 0 clears.  Process-wide.
 *
 * gira_test_bounded_wait -- launches one wait that nothing will end and returns
 * the status the kernel recorded: mode 0 waits on an mbarrier phase that never
 * completes (the wait the E-step kernels use for their TMA copies) for `limit`
 * nanoseconds of wall time; mode 1 polls a global counter that nobody
 * increments (the wait of the persistent seeding kernel) `limit` times.  Both
 * return GIRA_ERR_TIMEOUT, and the context stays usable.  limit in [1, 2e9].
 */
void gira_test_fail_next_allocations(int count);
gira_status gira_test_bounded_wait(int mode, long long limit, void *stream);

/*
 * gira_test_point_order -- the spatial order the fits' E-steps visit points in:
 * order[j] = the index of the j-th point after a stable sort of each instance
 * (points[offsets[i] .. offsets[i+1]), or all n points when batch = 1 and
 * offsets = NULL) by the Morton code of the point in the instance's bounding
 * cube (6 bits per axis, cells of the largest extent / 64, clamped to [0, 63];
 * code bit 3 b + a = bit b of the cell index on axis a).  points: device,
 * n x 3 binary32; order: device, n ints; offsets: host, batch + 1 entries.
 */
gira_status gira_test_point_order(const float *points, int64_t n, int batch, const int64_t *offsets, int *order,
                                  void *stream);

/* Thread-local description of the last error on this thread ("" if none). */
const char *gira_last_error_message(void);

/* Component index behind the last GIRA_ERR_NOT_PD on this thread, else -1. */
int gira_last_error_component(void);

/* Free the device workspace of every device (the next call re-allocates it). */
gira_status gira_release_workspace(void);

/* Library version string, e.g. "gira-gb300 0.1.0 sm_103a". */
const char *gira_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GIRA_H */
