// gira_internal.cuh -- shared definitions of the libgira CUDA kernels (sm_103a).
//
// Layout of the per-component E-step parameters ("pair-interleaved"):
// components 2p and 2p+1 form pair p; pair p owns PAIR_FLOATS floats at
// params[p * PAIR_FLOATS], stored as float2 slots {comp 2p, comp 2p+1}:
//   slot 0..5   P' = alpha * L^{-1}, lower triangle (p00, p10, p11, p20, p21, p22)
//   slot 6..8   b' = -P' mu
//   slot 9      c  = log2 pi + sum_j log2 (L^{-1})_jj - (3/2) log2(2 pi)
//   slot 10..12 -mu (binary32; mu is also the shift of the M-step statistics)
//   slot 13     the weight behind c: N_b after an M-step (c then uses log2 N_b and
//               the E-step subtracts log2 sum_a N_a), or the caller's weight
//   slot 14     a lower bound of sigma_min(P')^2 = alpha^2 / lambda_max(Sigma): the
//               point-stationary E-step's reach test (a pair whose q' is > 126 over a
//               warp's box of points gives exact zeros and is skipped)
//   slot 15..17 padding: a pair owns 36 floats (144 bytes), so lanes reading the
//               same slot of consecutive pairs in shared memory hit different banks
// alpha = sqrt(log2(e) / 2), so that c - ||P' x + b'||^2 = log2(pi N(x|mu,Sigma))
// (Eq. simplifiedGaussian scaled to base 2).  Padding components carry
// c = -inf, P' = b' = mu = 0, so they contribute exactly zero.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gira.h"

namespace gira {

constexpr int PAIR_FLOATS = 36;
constexpr int PAIR_F4 = PAIR_FLOATS / 4;   // float4 per pair block
constexpr int SLOT_P = 0, SLOT_B = 6, SLOT_C = 9, SLOT_NMU = 10, SLOT_W = 13, SLOT_S = 14;
constexpr int NSTAT = 10;   // S0, S1[3], S2[6] (00,01,02,11,12,22)
constexpr int MODEL = 10;   // w, mu[3], Sigma[6] (00,01,02,11,12,22), binary64; w = N_b or caller weight
constexpr int Q_BATCH = 8;  // points per E-step batch

// Device-side state of one library call (zeroed by the host at call start).
struct DeviceState {
    int error;             // first device-side gira_status (atomicCAS from 0)
    int bad_component;     // component behind GIRA_ERR_NOT_PD
    int stop_after;        // EM: last iteration to run (set on convergence); host sets it to iters
    int iters_done;        // EM iterations completed
    int lloyd_done;        // Lloyd centre updates made
    int w_raw;             // 1 once an M-step has run: weights are N_b, normalised by sum_a N_a on use
    double prev_ll;        // l_{t-1}
    double ll_sum;         // sum_n lse_n of the last E-step (natural log)
    int64_t chosen_last;   // k-means++: index chosen by the last select step
    // point-stationary E-step with statistics, summed over its launches: warp x pair
    // evaluations made (pairs within reach of the warp's box) and with statistics
    unsigned long long pairs_near, pairs_live;
};

__device__ __forceinline__ void set_error(DeviceState* st, int code) { atomicCAS(&st->error, 0, code); }

// Index checks of the debug build (-DGIRA_DEBUG): GIRA_IN(cond, st) is cond, and a
// false cond records GIRA_ERR_BOUNDS in st (the caller skips the access).  In
// release builds it is true and the condition is not evaluated.
#ifdef GIRA_DEBUG
__device__ __forceinline__ bool gira_in(bool ok, DeviceState* st) {
    if (!ok && st) set_error(st, GIRA_ERR_BOUNDS);
    return ok;
}
#define GIRA_IN(cond, st) ::gira::gira_in((cond), (st))
#else
#define GIRA_IN(cond, st) true
#endif

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

// ---------------------------------------------------------------- warp reductions
struct AddOp {
    __device__ __forceinline__ float operator()(float a, float b) const { return a + b; }
};
struct MaxOp {
    __device__ __forceinline__ float operator()(float a, float b) const { return fmaxf(a, b); }
};

// Per-lane batch index owned after the transpose-reduce: Q = 8 -> bits 4..2 of
// the lane, Q = 4 -> bits 4..3.  The owner of index q is lane q * (32 / Q).
template <int Q>
__device__ __forceinline__ int q_of_lane(int lane) {
    return Q == 8 ? (lane >> 2) & 7 : (lane >> 3) & 3;
}

// Combine Q per-lane values over the 32 lanes of a warp.  On return, lane l
// holds the combination for index q_of_lane<Q>(l); the order of combination is
// fixed, and the lanes sharing an index hold bit-identical results.
template <int Q, class Op>
__device__ __forceinline__ float warp_transpose_reduce(const float (&v)[Q], int lane, Op op) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float w[Q / 2];
#pragma unroll
    for (int i = 0; i < Q / 2; ++i) {
        const float send = b4 ? v[i] : v[i + Q / 2];
        const float keep = b4 ? v[i + Q / 2] : v[i];
        w[i] = op(keep, __shfl_xor_sync(0xffffffffu, send, 16));
    }
    float t;
    if (Q == 8) {
        float z[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float send = b3 ? w[i] : w[i + 2];
            const float keep = b3 ? w[i + 2] : w[i];
            z[i] = op(keep, __shfl_xor_sync(0xffffffffu, send, 8));
        }
        const float send = b2 ? z[0] : z[1];
        const float keep = b2 ? z[1] : z[0];
        t = op(keep, __shfl_xor_sync(0xffffffffu, send, 4));
    } else {
        const float send = b3 ? w[0] : w[1];
        const float keep = b3 ? w[1] : w[0];
        t = op(keep, __shfl_xor_sync(0xffffffffu, send, 8));
        t = op(t, __shfl_xor_sync(0xffffffffu, t, 4));
    }
    t = op(t, __shfl_xor_sync(0xffffffffu, t, 2));
    t = op(t, __shfl_xor_sync(0xffffffffu, t, 1));
    return t;
}


// ---------------------------------------------------------------- TMA bulk copy + mbarrier
// (PTX ISA: cp.async.bulk, mbarrier; a plain launch is a cluster of one CTA, so
// the CTA's own shared memory is addressed through the shared::cluster window.)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bytes: multiple of 16; src and dst 16-byte aligned.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Programmatic dependent launch (PTX griddepcontrol).  In a kernel launched with
// programmatic stream serialisation, pdl_wait() returns once the previous kernel
// of the stream has completed and its writes are visible, and pdl_allow_next()
// lets the next such kernel be scheduled before this one ends.  In a plain
// launch both have no effect.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase with the given parity: false once `limit_ns` of
// wall time has passed (try_wait itself may suspend between polls).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > (uint64_t)limit_ns) return false;
    }
}

// ---------------------------------------------------------------- bounded waits on global memory
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Wait until *counter >= target.  false when *abort is raised by another waiter,
// or after `limit` polls (each followed by a short sleep): then this waiter
// records GIRA_ERR_TIMEOUT and raises *abort so that the others leave too.
__device__ __forceinline__ bool wait_counter_bounded(const int* counter, int target, int* abort, long long limit,
                                                     DeviceState* st) {
    long long spins = 0;
    while (ld_acquire(counter) < target) {
        if (ld_acquire(abort)) return false;
        if (++spins > limit) {
            set_error(st, GIRA_ERR_TIMEOUT);
            st_release(abort, 1);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// binary32 squared distance in the fixed order d_i = x_i - c_i; (d0^2 + d1^2) + d2^2,
// every operation rounded separately (no contraction): k-means decisions are taken
// in exactly this arithmetic.
__device__ __forceinline__ float dist2_f32(float4 x, float4 c) {
    float d0 = __fsub_rn(x.x, c.x), d1 = __fsub_rn(x.y, c.y), d2 = __fsub_rn(x.z, c.z);
    float s = __fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1));
    return __fadd_rn(s, __fmul_rn(d2, d2));
}
// Four dimensions: ((d0^2 + d1^2) + d2^2) + d3^2, same rules.
__device__ __forceinline__ float dist2_f32_4(float4 x, float4 c) {
    const float d3 = __fsub_rn(x.w, c.w);
    return __fadd_rn(dist2_f32(x, c), __fmul_rn(d3, d3));
}

// ---------------------------------------------------------------- exact fixed-point weights
// k-means++ weights: fx(d) = floor(d * 2^48) for a binary32 d >= 0 (saturating
// at 2^95 - 1 for d >= 2^47), summed exactly in 128 bits; the draw threshold is
// floor(k * T / 2^53) for the 53-bit integer k behind u and the total T.
struct u128 {
    unsigned long long lo, hi;
};
__host__ __device__ __forceinline__ u128 u128_add(u128 a, u128 b) {
    u128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}
__host__ __device__ __forceinline__ u128 u128_sub(u128 a, u128 b) {
    u128 r;
    r.lo = a.lo - b.lo;
    r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
    return r;
}
__host__ __device__ __forceinline__ bool u128_gt(u128 a, u128 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__host__ __device__ __forceinline__ bool u128_zero(u128 a) { return (a.lo | a.hi) == 0ull; }
__device__ __forceinline__ u128 u128_shfl_up(u128 v, int o) {
    u128 r;
    r.lo = __shfl_up_sync(0xffffffffu, v.lo, o);
    r.hi = __shfl_up_sync(0xffffffffu, v.hi, o);
    return r;
}
__device__ __forceinline__ u128 u128_shfl(u128 v, int src) {
    u128 r;
    r.lo = __shfl_sync(0xffffffffu, v.lo, src);
    r.hi = __shfl_sync(0xffffffffu, v.hi, src);
    return r;
}
// Inclusive warp scan (exact, so the order of the additions does not matter).
__device__ __forceinline__ u128 u128_warp_incl_scan(u128 v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u128 u = u128_shfl_up(v, o);
        if (lane >= o) v = u128_add(v, u);
    }
    return v;
}
__device__ __forceinline__ u128 fx48(float d) {
    u128 r{0ull, 0ull};
    if (!(d > 0.f)) return r;
    if (d >= 140737488355328.0f) return u128{~0ull, (1ull << 31) - 1ull};   // 2^47 -> 2^95 - 1
    const unsigned bits = __float_as_uint(d);
    const int ex = (int)(bits >> 23);
    const unsigned long long mant = (bits & 0x7FFFFFu) | (ex ? 0x800000u : 0u);
    const int sh = (ex ? ex : 1) - 150 + 48;   // d = mant * 2^(sh - 48)
    if (sh >= 64) {
        r.hi = mant << (sh - 64);
    } else if (sh > 40) {
        r.lo = mant << sh;
        r.hi = mant >> (64 - sh);
    } else if (sh >= 0) {
        r.lo = mant << sh;
    } else if (sh > -24) {
        r.lo = mant >> (-sh);
    }
    return r;
}
__device__ __forceinline__ u128 fx_threshold(unsigned long long k53, u128 T) {
    const unsigned long long a_lo = k53 * T.lo, a_hi = __umul64hi(k53, T.lo);
    const unsigned long long b_lo = k53 * T.hi, b_hi = __umul64hi(k53, T.hi);
    const unsigned long long w0 = a_lo, w1 = a_hi + b_lo;
    const unsigned long long w2 = b_hi + (w1 < a_hi ? 1ull : 0ull);
    return u128{(w0 >> 53) | (w1 << 11), (w1 >> 53) | (w2 << 11)};
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

// K above this runs the chunked (two-level log-sum-exp) path; the batched and
// no-allocation entry points take K up to it only.
constexpr int MAX_K_DIRECT = 1024;

// ---------------------------------------------------------------- kernel entry points
// (defined in em_kernels.cu / kmeans_kernels.cu, launched from gira_api.cu)

// Batched fits: one entry per instance (device table).
struct BatchInst {
    int64_t pt_off;     // first point of the instance in the packed point arrays
    int64_t n;          // its points
    int64_t ppc;        // points per E-step CTA
    int64_t par_off;    // float offset of its E-step parameters (its class's padded pair count)
    int64_t part_off;   // float offset of its per-CTA statistic partials ([ctas][k][NSTAT])
    int64_t ll_off;     // double offset of its per-CTA log-likelihood partials
    int k;              // components
    int comp_off;       // first component in the per-component arrays
    int ctas;           // E-step CTAs of the instance
    int pad_;
    int64_t mask_off;   // word offset of its per-warp live masks (point-stationary E-step)
};
// One E-step CTA of a batched launch: instance and CTA index within it.
struct BatchUnit {
    int inst, cta;
};

struct EStepLaunch {
    const float4* pts8;      // 2 float4 per point: (x,x,y,y) (z,z,0,0)
    int64_t n;
    int k;
    const float* params;     // pair-interleaved, npairs_pad * PAIR_FLOATS
    int64_t pts_per_cta;     // multiple of Q_BATCH
    float* partials;         // [grid][k][NSTAT] (stats kernels)
    double* ll_partials;     // [grid]
    float* per_point;        // [n] natural-log lse, or nullptr
    DeviceState* st;
    int iter;                // iteration index (1-based); kernels skip if iter > st->stop_after
    // adjoint launches (log-likelihood gradient) only
    float* grad_pts = nullptr;           // [n][3] dL/dx (dL/dx' rotated back by R^T), or nullptr
    const float* rot = nullptr;          // R, row-major 3x3, of x' = R x + t; nullptr = identity
    double* pose_partials = nullptr;     // [grid][12]: per CTA sum dL/dx' x'^T (row-major), sum dL/dx'
    // batched launches: CTA b runs units[b]; pts8 / params / partials / ll_partials /
    // per_point are then bases offset by the instance's table entry, st = states + inst
    const BatchInst* insts = nullptr;
    const BatchUnit* units = nullptr;
    DeviceState* states = nullptr;
    // K split into chunks (one table entry per chunk, all over the same points):
    // pass A writes psum[chunk][n] = sum over the chunk of 2^(l - cmax); pass B
    // takes pref[n] = (shift, 1 / total) from the combine step
    const float* gref = nullptr;   // [0] cmax over all K, [1] log-likelihood reference (base 2)
    float* psum = nullptr;
    const float2* pref = nullptr;
    // point-stationary E-step (estep_pt_kernel): partial rows [rows][pairs][2 NSTAT],
    // row cta * PT_B + block written only where the block's live mask has the pair's
    // bit, and the live masks [npairs / 32][rows] (bit p: pair p reaches some point
    // of the block)
    uint32_t* masks = nullptr;
    int64_t pt_rows = 0;   // point blocks of the launch (the row count of partials and masks)
    int64_t n_buf = 0;     // points in pts8 (index checks of the debug build; 0: unchecked)
    // CTA order of a single fit's E-step: from iteration 3 on, CTA blockIdx.x takes the
    // point blocks of CTA cta_perm[(iter & 1) * grid + blockIdx.x] (longest expected
    // work first, written by the finalize two iterations earlier); cta_key[cta]
    // receives the CTA's work key for that order (nullptr: launch order, no keys)
    const int* cta_perm = nullptr;
    uint8_t* cta_key = nullptr;
};

// Chooses the template instance and block shape for K; returns the CTA count
// actually used in *grid_out (needed for the partials buffer size).
// grad: the differentiable path's kernels (d-form logits; with stats, the adjoint).
// A launch configuration, with programmatic stream serialisation when pdl (the
// kernel may start before the previous kernel in the stream has finished, and
// waits for it with pdl_wait()).
struct PdlConfig {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    PdlConfig(dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl) {
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = pdl ? 1 : 0;
    }
};
// pdl: launch as a programmatic dependent of the previous kernel in s (that kernel
// must not write the points).
cudaError_t launch_estep(const EStepLaunch& a, bool stats, int grid, cudaStream_t s, bool grad = false,
                         bool pdl = false);
// Occupancy-derived grid size for (k, stats) with n points.
int estep_grid(int64_t n, int k, bool stats, int num_sms, int64_t* pts_per_cta, bool grad = false);
// Pairs (padded) the parameter buffer must hold for k components.
int params_pairs_padded(int k);

// N x 3 -> pts4 (x,y,z,0) (nullable) and pts8 (x,x,y,y)(z,z,0,0); flags non-finite input.
cudaError_t launch_pack(const float* pts3, int64_t n, float4* pts4, float4* pts8, DeviceState* st, cudaStream_t s);
// Spatial order of packed points (order_kernels.cu): a stable radix sort by
// (instance, 18-bit Morton code in the instance's bounding cube).  offsets_d /
// units_d: the batch's point offsets and its (instance, chunk) bounding-box
// blocks (point_order_fill_units), or nullptr for one instance of n points.
// Writes the sorted points to p8_out (and, if p4_out, as (x, y, z, 0)) and, if
// order_out, the source index of every sorted point.  scratch: point_order_scratch_bytes(n, batch) bytes.
int64_t point_order_box_units(const int64_t* offsets, int batch);
void point_order_fill_units(const int64_t* offsets, int batch, int2* units);
size_t point_order_scratch_bytes(int64_t n, int batch);
int point_order_launches(int batch);   // kernels one launch_point_order makes
int64_t point_order_max_n();          // larger inputs keep the caller's order
cudaError_t launch_point_order(const float4* p8, int64_t n, const int64_t* offsets_d, const int2* units_d,
                               int nunits, int batch, void* scratch, float4* p8_out, float4* p4_out, int* order_out,
                               cudaStream_t s);
cudaError_t launch_fill_padding(float* params, int k, int npairs_pad, cudaStream_t s);
// Sum of the per-CTA log-likelihoods into st->ll_sum (fixed order).
cudaError_t launch_ll_reduce(const double* ll_partials, int grid, DeviceState* st, cudaStream_t s);
// M-step: reduce the per-CTA partials (or read binary64 stats64 when partials is
// nullptr), then binary64 finalize of every component; EM iterations (em) also
// reduce the log-likelihood, write the trace and decide convergence.
cudaError_t launch_reduce_finalize(const float* partials, int grid, const double* ll_partials,
                                   const double* stats64, float4* shift4, int k, int64_t n, double reg, double tol,
                                   double* model64, float* params, double* trace, DeviceState* st, int iter, bool em,
                                   cudaStream_t s, bool pdl = false, const int* perm = nullptr,
                                   const uint32_t* masks = nullptr, int nwords = 0, int ll_count = 0,
                                   const uint8_t* cta_key = nullptr, int* cta_perm = nullptr, int cta_grid = 0);
// Point-stationary E-step (3-D fits and log-likelihood, k <= 1024): CTAs for n
// points; partial rows (warps) of a grid; live-mask words per warp for k.
int estep_pt_grid(int64_t n);
int estep_pt_rows(int grid);
int estep_pt_row_floats(int k);   // floats of one partial row of the point-stationary E-step
int estep_pt_mask_words(int k);
// a.partials: [k * NSTAT][rows] (stats), a.masks: [mask words][rows], a.pt_rows = rows,
// a.ll_partials: [grid]
cudaError_t launch_estep_pt(const EStepLaunch& a, bool stats, int grid, cudaStream_t s, bool pdl = false);
// The same over a unit table (batched fits; a.insts / a.units / a.states; every
// instance's part_off, mask_off, ll_off and ctas for PT points per CTA).
cudaError_t launch_estep_pt_units(const EStepLaunch& a, bool stats, int nunits, int kmax, cudaStream_t s);
int estep_pt_points();   // points per CTA
int estep_pt_blocks();   // point blocks per CTA (partial and mask rows per CTA)
cudaError_t launch_params_from_model(const float* w, const float* mu, const float* cov, int k, double* model64,
                                     float* params, float4* shift4, DeviceState* st, cudaStream_t s);
// perm (nullable): slot s of model64 is the caller's component perm[s].
cudaError_t launch_model_out(const double* model64, int k, float* w, float* mu, float* cov, const DeviceState* st,
                             cudaStream_t s, const int* perm = nullptr);
// Reorder the k <= 8192 components of model64 along a space-filling curve of
// their means (Morton order) and rebuild params / shift4 / model64 in that order:
// slot s holds the caller's component perm[s].  scratch: k * MODEL doubles.
cudaError_t launch_order_components(double* model64, double* scratch, int k, int* perm, float* params,
                                    float4* shift4, DeviceState* st, cudaStream_t s);

// Batched EM (per-instance tables on the device).
// E-step block shape for k components (pairs per lane, warps, threads); the
// batch size Q of the kernels; the largest points-per-CTA; CTAs per SM.
void estep_shape(int k, int* np, int* g, int* threads);
int estep_batch_q();
int estep_ppc_max();
int estep_occupancy(int k, bool stats, int64_t ppc);
// One launch over nunits CTAs (a.units / a.insts / a.states set) of the class
// whose shape is that of k_class; every instance of the class has ppc_class.
cudaError_t launch_estep_units(const EStepLaunch& a, bool stats, int nunits, int k_class, int64_t ppc_class,
                               cudaStream_t s);
cudaError_t launch_pack_batched(const float* pts3, int64_t n, const int64_t* offsets, int batch, float4* pts4,
                                float4* pts8, DeviceState* states, cudaStream_t s);
// Finalize blocks: (instance, block index within the instance), FIN_CPB components each.
int fin_components_per_block();
cudaError_t launch_reduce_finalize_batched(const float* partials, const double* ll_partials, const double* stats64,
                                           float4* shift4, const BatchInst* insts, const int2* blocks, int nblocks,
                                           double reg, double tol, int iters, double* model64, float* params,
                                           double* trace, DeviceState* states, int iter, bool em, cudaStream_t s,
                                           const int* perm = nullptr, const uint32_t* masks = nullptr);
// Padding slots of every instance's parameter block (one block per instance).
cudaError_t launch_fill_padding_batched(float* params, const BatchInst* insts, int batch, int npairs_max,
                                        const int* npairs_of, cudaStream_t s);
// E-step parameters of every instance from (w, mu, Sigma) (comp_inst: instance of each component).
cudaError_t launch_params_from_model_batched(const float* w, const float* mu, const float* cov, int total_k,
                                             const int* comp_inst, const BatchInst* insts, double* model64,
                                             float* params, float4* shift4, DeviceState* states, cudaStream_t s);
// Normalised model of every instance (one block per instance).
cudaError_t launch_model_out_batched(const double* model64, const BatchInst* insts, int batch, float* w, float* mu,
                                     float* cov, const DeviceState* states, cudaStream_t s,
                                     const int* perm = nullptr);
// launch_order_components for every instance of a batch (one block each, k <= 8192).
cudaError_t launch_order_components_batched(double* model64, double* scratch, int total_k, int kmax,
                                            const BatchInst* insts, int batch, const int* comp_inst, int* perm,
                                            float* params, float4* shift4, DeviceState* states, cudaStream_t s);
// Per-instance sums of the log-likelihood partials into states[i].ll_sum.
cudaError_t launch_ll_reduce_batched(const double* ll_partials, const BatchInst* insts, int batch,
                                     DeviceState* states, cudaStream_t s);

// Large K: components in chunks of chunk_components() (one E-step shape),
// each chunk an entry of a BatchInst table over the same points.
int chunk_components();
// gref = (max_b c_b over all k components, log-likelihood reference) from the
// chunked parameter blocks (chunk c at c * chunk_param_floats()).
int64_t chunk_param_floats();
cudaError_t launch_chunk_ref(const float* params, int k, const DeviceState* st, float* gref, cudaStream_t s);
// Pass A / pass B over all chunks (units: chunk-major); see EStepLaunch.
cudaError_t launch_estep_chunks(const EStepLaunch& a, int pass, int nunits, int64_t ppc, cudaStream_t s);
// Per point: total over chunks -> pref, per-point log-likelihood llpt (natural);
// points whose total underflows (< 2^-100) are listed in flags for the exact step.
int chunk_combine_grid();
cudaError_t launch_chunk_combine(const float* psum, int chunks, int64_t n, const float* gref, float2* pref,
                                 double* llpt, int* flag_count, int* flags, DeviceState* st, cudaStream_t s);
// Listed points: exact per-point maximum over all k components (one warp each).
cudaError_t launch_chunk_exact(const float4* pts8, const float* params, int k, const float* gref, const int* flags,
                               const int* flag_count, float2* pref, double* llpt, DeviceState* st, cudaStream_t s);
cudaError_t launch_double_to_float(const double* x, int64_t n, float* y, cudaStream_t s);
// Fixed-order sums of llpt into chunk_combine_grid() partials, then (st != nullptr)
// into st->ll_sum.
cudaError_t launch_points_ll_reduce(const double* llpt, int64_t n, double* llp, DeviceState* st, cudaStream_t s);
// The chunks' finalize: like the batched one, but every chunk shares state st
// and trace; the log-likelihood / convergence step (em) runs once, from
// ll_partials[0 .. ll_count).
cudaError_t launch_reduce_finalize_chunks(const float* partials, const double* ll_partials, int ll_count,
                                          const double* stats64, float4* shift4, const BatchInst* insts,
                                          const int2* blocks, int nblocks, int64_t n, double reg, double tol,
                                          double* model64, float* params, double* trace, DeviceState* st, int iter,
                                          bool em, cudaStream_t s, const int* perm = nullptr);

// Batched differentiable log-likelihood (a batch table of scans, each with its
// own model and pose; poses: batch x 12, or nullptr for identities).
cudaError_t launch_pack_pose_batched(const float* pts3, int64_t n, const int64_t* offsets, int batch,
                                     const float* poses, float4* pts8, DeviceState* states, cudaStream_t s);
cudaError_t launch_params_from_chol_batched(const float* logits, const float* mu, const float* chol,
                                            const BatchInst* insts, int batch, double* model64, float* params,
                                            float4* shift4, DeviceState* states, cudaStream_t s);
cudaError_t launch_estep_grad_units(const EStepLaunch& a, int nunits, int k_class, int64_t ppc_class, cudaStream_t s);
int estep_grad_occupancy(int k, int64_t ppc);
cudaError_t launch_grad_finalize_batched(const float* partials, const double* ll_partials,
                                         const double* pose_partials, const float* poses, const float* chol,
                                         const double* model64, const BatchInst* insts, const int2* blocks,
                                         int nblocks, float* g_logits, float* g_means, float* g_chol, double* g_pose,
                                         double* g_twist, DeviceState* states, cudaStream_t s);

// Differentiable log-likelihood.  pose12 = R (row-major) then t, or nullptr.
// N x 3 -> pts8 of x' = R x + t (binary32, fixed order); flags non-finite input.
cudaError_t launch_pack_pose(const float* pts3, int64_t n, const float* pose12, float4* pts8, DeviceState* st,
                             cudaStream_t s);
// E-step parameters from (logits, means, Cholesky factors): pi = softmax in
// binary64, Sigma = L L^T, then the same binary64 build as the M-step.
cudaError_t launch_params_from_chol(const float* logits, const float* mu, const float* chol, int k, double* model64,
                                    float* params, float4* shift4, DeviceState* st, cudaStream_t s);
// Reduces the statistics, the log-likelihood and the pose partials of a
// gradient launch, then writes dL/dlogits (k), dL/dmeans (k x 3), dL/dchol
// (k x 3 x 3, lower) in binary32, and in binary64 dL/dpose (dL/dR row-major,
// dL/dt) and dL/dtwist (omega, v); loglik goes to st->ll_sum.  Outputs nullable.
cudaError_t launch_grad_finalize(const float* partials, int grid, const double* ll_partials,
                                 const double* pose_partials, const float* pose12, const float* chol,
                                 const double* model64, int k, int64_t n, float* g_logits, float* g_means,
                                 float* g_chol, double* g_pose, double* g_twist,
                                 DeviceState* st, cudaStream_t s);

// k-means
// dim: 3 (distances over x, y, z) or 4 (also the fourth coordinate)
cudaError_t launch_kpp(const float4* pts4, int64_t n, int k, uint64_t seed, float4* centers, float* d2,
                       u128* blocksums, int64_t* chosen, DeviceState* st, cudaStream_t s, int dim = 3);
int kpp_num_blocks(int64_t n);
// Persistent k-means++ (one cooperative launch for all K centres).  Grid size, or
// 0 when cooperative launch is unavailable (the per-centre launches are used).
int kpp_persistent_grid();
// sync_ints: k+1 zeroed ints (per-centre arrival counters, abort flag);
// sums: kpp_persistent_sum_words(grid, k) 128-bit words; d2: 2n floats.  Valid for
// n <= kpp_persistent_max_n(grid) (points held in registers).
size_t kpp_persistent_sum_words(int grid, int k);
int64_t kpp_persistent_max_n(int grid);
cudaError_t launch_kpp_persistent(const float4* pts4, int64_t n, int k, uint64_t seed, float4* centers, float* d2,
                                  int64_t* chosen, int* sync_ints, u128* sums, int grid, DeviceState* st,
                                  cudaStream_t s, int dim = 3);
// Batched KInit: one entry per instance.
struct KppInst {
    int64_t pt_off, n;
    int k, comp_off, inst, pad_;
};
// Batched seeding: cluster c of the launch (cs CTAs each) seeds instance
// table[c]; every instance needs n <= kpp_cluster_capacity(cs).
cudaError_t launch_kpp_cluster_batched(const float4* pts4, const KppInst* table, int clusters, uint64_t seed,
                                       float4* centers, int64_t* chosen, int cs, DeviceState* states,
                                       cudaStream_t s);
int kpp_cluster_capacity(int cs);
// Batched Lloyd: units (instance, tile of lloyd_tile() points); per-instance
// label / sum / changed slabs (changed: lloyd_iters + 1 counters per instance).
int lloyd_tile();
cudaError_t launch_lloyd_batched(const float4* pts4, const KppInst* table, const BatchUnit* units, int nunits,
                                 int total_k, const int* comp_inst, int lloyd_iters, float4* centers, int32_t* labels,
                                 double* sums, unsigned long long* changed, DeviceState* states, cudaStream_t s);
// One-hot statistics of every instance (instance of point i by binary search over offsets).
cudaError_t launch_label_stats_batched(const float4* pts4, int64_t n, const int64_t* offsets, int batch,
                                       const KppInst* table, const int32_t* labels, const float4* shift4,
                                       double* stats64, DeviceState* states, cudaStream_t s);
// One-cluster k-means++ (no global synchronisation): cluster size for n points,
// or 0 when the one-cluster path does not apply.
int kpp_cluster_size(int64_t n);
cudaError_t launch_kpp_cluster(const float4* pts4, int64_t n, int k, uint64_t seed, float4* centers, int64_t* chosen,
                               int cs, DeviceState* st, cudaStream_t s);
cudaError_t launch_lloyd(const float4* pts4, int64_t n, int k, int lloyd_iters, float4* centers, int32_t* labels,
                         double* sums, unsigned long long* changed, DeviceState* st, cudaStream_t s);
cudaError_t launch_label_stats(const float4* pts4, int64_t n, int k, const int32_t* labels, const float4* shift4,
                               double* stats64, DeviceState* st, cudaStream_t s);
cudaError_t launch_centers_out(const float4* centers4, int k, float* centers3, cudaStream_t s);

// ---------------------------------------------------------------- four dimensions (xyz + intensity)
// E-step parameters, pair-interleaved: components 2p, 2p+1 form pair p, which
// owns PAIR4_FLOATS floats at params[p * PAIR4_FLOATS] as float2 slots
// {comp 2p, comp 2p+1}:
//   slot 0..9   P' = alpha * L^{-1}, lower triangle (00,10,11,20,21,22,30,31,32,33)
//   slot 10     c = log2 w + sum_j log2 (L^{-1})_jj - (4/2) log2(2 pi)
//   slot 11..14 -mu (binary32; also the shift of the M-step statistics)
//   slot 15     w (N_b after an M-step, or the caller's weight)
// Statistics (NSTAT4): S0, S1[4], S2[10] in the order 00,01,02,03,11,12,13,22,23,33;
// binary64 model (MODEL4): w, mu[4], Sigma[10] in the same order.
constexpr int PAIR4_FLOATS = 32;
constexpr int SLOT4_P = 0, SLOT4_C = 10, SLOT4_NMU = 11, SLOT4_W = 15;
constexpr int NSTAT4 = 15;
constexpr int MODEL4 = 15;
// index of (i, j), i <= j, in the upper-triangle order 00,01,02,03,11,12,13,22,23,33
__host__ __device__ constexpr int sym4(int i, int j) { return i * (7 - i) / 2 + j; }

struct EStep4Launch {
    const float4* pts8;    // 2 float4 per point: (x,x,y,y) (z,z,I,I)
    int64_t n;
    int k;
    const float* params;   // estep4_threads(k) pairs * PAIR4_FLOATS (padding components: c = -inf)
    int64_t pts_per_cta;   // multiple of 8
    float* partials;       // [grid][k][NSTAT4] (stats launches)
    double* ll_partials;   // [grid]
    float* per_point;      // [n] natural-log lse, or nullptr
    DeviceState* st;
    int iter;              // 1-based EM iteration; skipped when iter > st->stop_after
    // K above MAX_K4_DIRECT: chunks of CHUNK4 components (blockIdx.y = chunk, all over
    // the same points, logits relative to gref[0] = max_b c_b).  Pass A writes
    // psum[chunk][n] = sum over the chunk of 2^(l - cmax); pass B takes
    // pref[n] = (shift, 1 / total) and writes the statistics, partials laid out
    // [chunk][grid][CHUNK4][NSTAT4].
    const float* gref = nullptr;
    float* psum = nullptr;
    const float2* pref = nullptr;
};

constexpr int MAX_K4_DIRECT = 1024;   // one CTA holds every component up to here
constexpr int CHUNK4 = 512;           // components per chunk above it

// Threads of the E-step block for k components (one pair per lane).
int estep4_threads(int k);
// Component pairs the parameter buffer holds for k (chunks padded to CHUNK4).
int params4_pairs(int k);
int estep4_grid(int64_t n, int k, int num_sms, int64_t* pts_per_cta);
// pdl: as for launch_estep.
cudaError_t launch_estep4(const EStep4Launch& a, bool stats, int grid, cudaStream_t s, bool pdl = false);
// N x 4 -> pts4 (x,y,z,I) (nullable) and pts8 (x,x,y,y)(z,z,I,I); flags non-finite input.
cudaError_t launch_pack4(const float* pts4in, int64_t n, float4* pts4, float4* pts8, DeviceState* st,
                         cudaStream_t s);
cudaError_t launch_fill_padding4(float* params, int k, cudaStream_t s);
// M-step from the per-CTA partials (or binary64 stats64 when partials is nullptr),
// about the shift shift4 (nullptr: the means held in params); em as in launch_reduce_finalize.
// kc: components per partial block (k for the direct E-step, CHUNK4 for chunks:
// component b's partials at ((b / kc) * grid + cta) * kc + b % kc); the
// log-likelihood is the sum of ll_partials[0 .. ll_count).
cudaError_t launch_reduce_finalize4(const float* partials, int grid, int kc, const double* ll_partials,
                                    int ll_count, const double* stats64, const float4* shift4, int k, int64_t n,
                                    double reg, double tol, double* model64, float* params, double* trace,
                                    DeviceState* st, int iter, bool em, cudaStream_t s, bool pdl = false);
// Chunked E-step (K > MAX_K4_DIRECT): gref from all k components; pass A / B over
// chunks x grid CTAs (pass 1 or 2); exact maximum for the points combine listed.
cudaError_t launch_chunk_ref4(const float* params, int k, const DeviceState* st, float* gref, cudaStream_t s);
cudaError_t launch_estep4_chunks(const EStep4Launch& a, int pass, int grid, cudaStream_t s);
cudaError_t launch_chunk_exact4(const float4* pts8, const float* params, int k, const float* gref, const int* flags,
                                const int* flag_count, float2* pref, double* llpt, DeviceState* st, cudaStream_t s);
cudaError_t launch_params_from_model4(const float* w, const float* mu, const float* cov, int k, double* model64,
                                      float* params, DeviceState* st, cudaStream_t s);
cudaError_t launch_model_out4(const double* model64, int k, float* w, float* mu, float* cov, const DeviceState* st,
                              cudaStream_t s);
// Lloyd in four dimensions and the one-hot statistics about the final centres.
cudaError_t launch_lloyd4(const float4* pts4, int64_t n, int k, int lloyd_iters, float4* centers, int32_t* labels,
                          double* sums, unsigned long long* changed, DeviceState* st, cudaStream_t s);
cudaError_t launch_label_stats4(const float4* pts4, int64_t n, int k, const int32_t* labels, const float4* shift4,
                                double* stats64, DeviceState* st, cudaStream_t s);
// Gaussian-mixture regression of the 4th coordinate on the first three.
int cond_floats();
cudaError_t launch_conditional4(const float* locs, int64_t m, int k, const float* w, const float* mu,
                                const float* cov, float* prep, float* cmean, float* cvar, DeviceState* st,
                                cudaStream_t s);
// m draws from a d-dimensional mixture (d = 3 or 4); cum: k doubles, chol: 16 k doubles.
cudaError_t launch_sample(int64_t m, int k, int d, const float* w, const float* mu, const float* cov, uint64_t seed,
                          double* cum, double* chol, float* out, int32_t* comp, DeviceState* st, cudaStream_t s);

// ---------------------------------------------------------------- mode seeking (K from a bandwidth)
// Temporary bytes the sorts / scans of one gira_gbms call need for n points.
size_t gbms_temp_bytes(int64_t n, int d);
// Points -> float4 copies, cell keys and identity indices; flags non-finite input
// (GIRA_ERR_NONFINITE_INPUT) and coordinates outside the cell range (GIRA_ERR_INVALID_ARG).
cudaError_t launch_gbms_keys(const float* pts, int64_t n, int d, double h, float4* pts4, uint64_t* keys, int* idx,
                             DeviceState* st, cudaStream_t s);
// Sort (key, index) pairs by key, then the distinct keys, their run lengths and
// starts; *ncells (device) receives the number of distinct keys.
cudaError_t gbms_sort_cells(void* temp, size_t temp_bytes, const uint64_t* keys_in, uint64_t* keys_out,
                            const int* idx_in, int* idx_out, int64_t n, int d, uint64_t* ukeys, int* ulen,
                            int* ustart, int* ncells, cudaStream_t s);
// Points in cell order, with their fixed-point coordinates (x, y) and (z, w).
cudaError_t launch_gbms_gather(const float4* pts4, const int* idx, int64_t n, float4* spts, longlong2* qxy,
                               longlong2* qzw, cudaStream_t s);
// One CTA per seed (cell): the seed's moves; modes[s] and counts[s] (0: dropped).
cudaError_t launch_gbms_shift(const float4* spts, const longlong2* qxy, const longlong2* qzw, const uint64_t* ukeys,
                              const int* ustart, const int* ulen, int ncells, int d, double h, int max_iter,
                              double4* modes, int* counts, const DeviceState* st, cudaStream_t s);
// Rank keys of the ns seeds and their sort; *nlive (device, zeroed by the caller)
// receives the number of live modes.
cudaError_t launch_gbms_rank(void* temp, size_t temp_bytes, const int* counts, int ns, uint64_t* rkeys,
                             uint64_t* rkeys_sorted, int* nlive, cudaStream_t s);
// Live modes in rank order (rmodes, rcount), their cell keys and rank indices for
// the merge grid, and the merge state (undecided).
cudaError_t launch_gbms_rank_modes(const uint64_t* rkeys_sorted, const int* nlive, int nmax, const double4* modes,
                                   const int* counts, int d, double h, double4* rmodes, int* rcount, uint64_t* mkeys,
                                   int* midx, int* state, DeviceState* st, cudaStream_t s);
// One merge round; *undecided (zeroed by the caller) counts ranks still open.
cudaError_t launch_gbms_merge_round(const double4* rmodes, const int* nlive, int nmax, const uint64_t* mukeys,
                                    const int* mustart, const int* mulen, const int* mncells, const int* midx_sorted,
                                    int d, double h, int* state, int* undecided, cudaStream_t s);
// Kept modes in rank order -> modes_out (k x d binary64) and counts_out (nullable);
// pos[r] is the output slot of rank r (exclusive sum of the kept flags).
cudaError_t launch_gbms_output(void* temp, size_t temp_bytes, const int* state, const int* nlive, int nmax,
                               const double4* rmodes, const int* rcount, int d, int* flags, int* pos,
                               double* modes_out, int* counts_out, cudaStream_t s);

// Test hook: one wait that nothing ends (mode 0: mbarrier, limit in ns; mode 1:
// global counter, limit in polls); counter and abort_flag: zeroed device ints.
cudaError_t launch_wait_probe(int mode, long long limit, int* counter, int* abort_flag, DeviceState* st,
                              cudaStream_t s);

// Set this thread's last-error message (msg may be nullptr to keep it) and
// component (what gira_last_error_message / gira_last_error_component return).
void record_error(const char* msg, int component);

// The status a call returns for the device status word it read back (GIRA_OK
// when no kernel recorded an error), with this thread's last-error message and,
// for GIRA_ERR_NOT_PD, the component.
gira_status device_status(const DeviceState& h);

// Name of the E-step kernel this host thread launched last (the runtime's name
// of the function, demangled; "" before the first launch).
const char* last_estep_kernel();
// Record fn (an E-step kernel about to be launched) as the last one.
void note_estep_kernel(const void* fn);

}  // namespace gira
