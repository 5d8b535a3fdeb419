// gira_internal.cuh -- shared definitions of the libgira CUDA kernels (sm_103a).
//
// Layout of the per-component E-step parameters ("pair-interleaved"):
// components 2p and 2p+1 form pair p; pair p owns PAIR_FLOATS floats at
// params[p * PAIR_FLOATS], stored as float2 slots {comp 2p, comp 2p+1}:
//   slot 0..5   P' = alpha * L^{-1}, lower triangle (p00, p10, p11, p20, p21, p22)
//   slot 6..8   b' = -P' mu
//   slot 9      c  = log2 pi + sum_j log2 (L^{-1})_jj - (3/2) log2(2 pi)
//   slot 10..12 -mu (binary32; mu is also the shift of the M-step statistics)
//   slot 13..15 padding
// alpha = sqrt(log2(e) / 2), so that c - ||P' x + b'||^2 = log2(pi N(x|mu,Sigma))
// (Eq. simplifiedGaussian scaled to base 2).  Padding components carry
// c = -inf, P' = b' = mu = 0, so they contribute exactly zero.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gira.h"

namespace gira {

constexpr int PAIR_FLOATS = 32;
constexpr int SLOT_P = 0, SLOT_B = 6, SLOT_C = 9, SLOT_NMU = 10;
constexpr int NSTAT = 10;   // S0, S1[3], S2[6] (00,01,02,11,12,22)
constexpr int MODEL = 10;   // pi, mu[3], Sigma[6] (00,01,02,11,12,22), binary64
constexpr int Q_BATCH = 8;  // points per E-step batch

// Device-side state of one library call (zeroed by the host at call start).
struct DeviceState {
    int error;             // first device-side gira_status (atomicCAS from 0)
    int bad_component;     // component behind GIRA_ERR_NOT_PD
    int stop_after;        // EM: last iteration to run (set on convergence); host sets it to iters
    int iters_done;        // EM iterations completed
    int lloyd_done;        // Lloyd centre updates made
    int pad0;
    double prev_ll;        // l_{t-1}
    double ll_sum;         // sum_n lse_n of the last E-step (natural log)
    int64_t chosen_last;   // k-means++: index chosen by the last select step
};

__device__ __forceinline__ void set_error(DeviceState* st, int code) { atomicCAS(&st->error, 0, code); }

// ---------------------------------------------------------------- packed FP32
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// binary32 squared distance in the fixed order d_i = x_i - c_i; (d0^2 + d1^2) + d2^2,
// every operation rounded separately (no contraction): k-means decisions are taken
// in exactly this arithmetic.
__device__ __forceinline__ float dist2_f32(float4 x, float4 c) {
    float d0 = __fsub_rn(x.x, c.x), d1 = __fsub_rn(x.y, c.y), d2 = __fsub_rn(x.z, c.z);
    float s = __fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1));
    return __fadd_rn(s, __fmul_rn(d2, d2));
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator:
// draw j of `seed` is output j+1 of the stream started at state `seed`.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t j) {
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double uniform53(uint64_t seed, uint64_t j) {
    return (double)(splitmix64(seed, j) >> 11) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------- kernel entry points
// (defined in em_kernels.cu / kmeans_kernels.cu, launched from gira_api.cu)
struct EStepLaunch {
    const float4* pts;
    int64_t n;
    int k;
    const float* params;     // pair-interleaved, npairs_pad * PAIR_FLOATS
    int64_t pts_per_cta;     // multiple of Q_BATCH
    float* partials;         // [grid][k][NSTAT] (stats kernels)
    double* ll_partials;     // [grid]
    float* per_point;        // [n] natural-log lse, or nullptr
    DeviceState* st;
    int iter;                // iteration index (1-based); kernels skip if iter > st->stop_after
};

// Chooses the template instance and block shape for K; returns the CTA count
// actually used in *grid_out (needed for the partials buffer size).
cudaError_t launch_estep(const EStepLaunch& a, bool stats, int grid, cudaStream_t s);
// Occupancy-derived grid size for (k, stats) with n points.
int estep_grid(int64_t n, int k, bool stats, int num_sms, int64_t* pts_per_cta);
// Pairs (padded) the parameter buffer must hold for k components.
int params_pairs_padded(int k);

cudaError_t launch_pack(const float* pts3, int64_t n, float4* pts4, DeviceState* st, cudaStream_t s);
cudaError_t launch_fill_padding(float* params, int k, int npairs_pad, cudaStream_t s);
cudaError_t launch_em_reduce(const float* partials, const double* ll_partials, int grid, int k, double* stats64,
                             DeviceState* st, int iter, cudaStream_t s);
cudaError_t launch_finalize(const double* stats64, float4* shift4, int k, int64_t n, double reg, double tol,
                            double* model64, float* params, double* trace, DeviceState* st, int iter, bool em,
                            cudaStream_t s);
cudaError_t launch_params_from_model(const float* w, const float* mu, const float* cov, int k, double* model64,
                                     float* params, float4* shift4, DeviceState* st, cudaStream_t s);
cudaError_t launch_model_out(const double* model64, int k, float* w, float* mu, float* cov, cudaStream_t s);

// k-means
cudaError_t launch_kpp(const float4* pts4, int64_t n, int k, uint64_t seed, float4* centers, float* d2,
                       double* blocksums, int64_t* chosen, DeviceState* st, cudaStream_t s);
int kpp_num_blocks(int64_t n);
cudaError_t launch_lloyd(const float4* pts4, int64_t n, int k, int lloyd_iters, float4* centers, int32_t* labels,
                         double* sums, unsigned long long* changed, DeviceState* st, cudaStream_t s);
cudaError_t launch_label_stats(const float4* pts4, int64_t n, int k, const int32_t* labels, const float4* shift4,
                               double* stats64, DeviceState* st, cudaStream_t s);
cudaError_t launch_centers_out(const float4* centers4, int k, float* centers3, cudaStream_t s);

// Set this thread's last-error message (msg may be nullptr to keep it) and
// component (what gira_last_error_message / gira_last_error_component return).
void record_error(const char* msg, int component);

}  // namespace gira
