// em_kernels.cu -- fused E-step / M-step statistics, reduction and FP64 finalize.
//
// GIRA (arXiv 2307.00071) Sec. V: the E-step of Eq. (estep) is evaluated in the
// log domain (Eq. logestep) with the Cholesky form of the log-density
// (Eq. simplifiedGaussian); the M-step (standard full-covariance update, not
// written in the paper) is fed by per-component sufficient statistics.
//
// Mapping (component-stationary): one CTA holds ALL K components, spread over
// its G warps; lane (warp w, lane l) owns NP component pairs in registers.  All
// lanes walk the CTA's contiguous range of points together, Q_BATCH points at a
// time.  Pass 1 computes e_nb = 2^(l_nb - cmax) for the lane's components
// (kept in registers), the per-point sums are combined across lanes (shuffle
// transpose-reduce) and warps (shared memory), and pass 2 accumulates the
// per-component statistics S0 = sum r, S1 = sum r d, S2 = sum r d d^T with
// d = x - mu_old (binary32, per-CTA partials).  Component pairs are processed
// with packed FP32 (FFMA2/FADD2/FMUL2).  The responsibility matrix is never
// stored.
#include <float.h>
#include <math.h>

#include <algorithm>

#include "gira_internal.cuh"

namespace gira {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float LN2F = 0.693147180559945309f;
constexpr double LN2 = 0.693147180559945309417232121458;

struct AddOp {
    __device__ __forceinline__ float operator()(float a, float b) const { return a + b; }
};
struct MaxOp {
    __device__ __forceinline__ float operator()(float a, float b) const { return fmaxf(a, b); }
};

// Combine 8 per-lane values over the 32 lanes of a warp.  On return, lane l
// holds the combination for value index (l >> 2) & 7; the order of combination
// is fixed, and the 4 lanes sharing an index hold bit-identical results.
template <class Op>
__device__ __forceinline__ float warp_transpose_reduce8(const float (&v)[Q_BATCH], int lane, Op op) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float send = b4 ? v[i] : v[i + 4];
        float keep = b4 ? v[i + 4] : v[i];
        w[i] = op(keep, __shfl_xor_sync(FULL, send, 16));
    }
    float z[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float send = b3 ? w[i] : w[i + 2];
        float keep = b3 ? w[i + 2] : w[i];
        z[i] = op(keep, __shfl_xor_sync(FULL, send, 8));
    }
    float send = b2 ? z[0] : z[1];
    float keep = b2 ? z[1] : z[0];
    float t = op(keep, __shfl_xor_sync(FULL, send, 4));
    t = op(t, __shfl_xor_sync(FULL, t, 2));
    t = op(t, __shfl_xor_sync(FULL, t, 1));
    return t;
}

// Combine per-warp results across the CTA's G warps through shared memory, in
// warp order (identical result in every lane that shares a value index).
template <class Op>
__device__ __forceinline__ float cta_combine(float t, float (*buf)[Q_BATCH], int G, int warp, int lane, Op op) {
    if (G == 1) return t;
    const int q = (lane >> 2) & 7;
    if ((lane & 3) == 0) buf[warp][q] = t;
    __syncthreads();
    float r = buf[0][q];
    for (int w = 1; w < G; ++w) r = op(r, buf[w][q]);
    return r;
}

// Log-density in base 2 for a component pair and one point (pairs packed).
struct PairParams {
    float2 p[6], b[3], c, nmu[3];
};

__device__ __forceinline__ float2 logit2(const PairParams& P, float2 X0, float2 X1, float2 X2) {
    float2 y0 = fma2(P.p[0], X0, P.b[0]);
    float2 y1 = fma2(P.p[1], X0, fma2(P.p[2], X1, P.b[1]));
    float2 y2 = fma2(P.p[3], X0, fma2(P.p[4], X1, fma2(P.p[5], X2, P.b[2])));
    float2 l = fma2(neg2(y0), y0, P.c);
    l = fma2(neg2(y1), y1, l);
    return fma2(neg2(y2), y2, l);
}

template <int NP, int MAXT, int MINB, bool STATS>
__global__ void __launch_bounds__(MAXT, MINB) estep_kernel(const EStepLaunch a) {
    __shared__ float red_sum[2][32][Q_BATCH];
    __shared__ float red_aux[2][32][Q_BATCH];
    __shared__ float s_cmax[32];
    __shared__ int s_skip;

    const int G = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_skip = (a.iter > a.st->stop_after) || (a.st->error != 0);
    __syncthreads();
    if (s_skip) return;

    // ---- this lane's component pairs -> registers
    PairParams prm[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int pp = (j * G + warp) * 32 + lane;
        const float4* src = reinterpret_cast<const float4*>(a.params + (size_t)pp * PAIR_FLOATS);
        float4 v0 = src[0], v1 = src[1], v2 = src[2], v3 = src[3], v4 = src[4], v5 = src[5], v6 = src[6];
        prm[j].p[0] = f2(v0.x, v0.y); prm[j].p[1] = f2(v0.z, v0.w);
        prm[j].p[2] = f2(v1.x, v1.y); prm[j].p[3] = f2(v1.z, v1.w);
        prm[j].p[4] = f2(v2.x, v2.y); prm[j].p[5] = f2(v2.z, v2.w);
        prm[j].b[0] = f2(v3.x, v3.y); prm[j].b[1] = f2(v3.z, v3.w);
        prm[j].b[2] = f2(v4.x, v4.y); prm[j].c = f2(v4.z, v4.w);
        prm[j].nmu[0] = f2(v5.x, v5.y); prm[j].nmu[1] = f2(v5.z, v5.w);
        prm[j].nmu[2] = f2(v6.x, v6.y);
    }
    // ---- reference cmax = max_b c_b >= every logit, so every e <= 1
    float cm = -INFINITY;
#pragma unroll
    for (int j = 0; j < NP; ++j) cm = fmaxf(cm, fmaxf(prm[j].c.x, prm[j].c.y));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cm = fmaxf(cm, __shfl_xor_sync(FULL, cm, o));
    if (lane == 0) s_cmax[warp] = cm;
    __syncthreads();
    float cmax = s_cmax[0];
    for (int w = 1; w < G; ++w) cmax = fmaxf(cmax, s_cmax[w]);
#pragma unroll
    for (int j = 0; j < NP; ++j) prm[j].c = f2(prm[j].c.x - cmax, prm[j].c.y - cmax);

    float2 S[NP][NSTAT];
    if (STATS) {
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int s = 0; s < NSTAT; ++s) S[j][s] = f2(0.f, 0.f);
    }
    double ll_acc = 0.0;
    const int myq = (lane >> 2) & 7;
    const bool owner = (warp == 0) && ((lane & 3) == 0);

    const int64_t begin = (int64_t)blockIdx.x * a.pts_per_cta;
    const int64_t end = min(a.n, begin + a.pts_per_cta);
    int slot = 0;
    for (int64_t base = begin; base < end; base += Q_BATCH, slot ^= 1) {
        float4 x[Q_BATCH];
#pragma unroll
        for (int q = 0; q < Q_BATCH; ++q) x[q] = __ldg(a.pts + min(base + q, a.n - 1));

        // ---- pass 1: e = 2^(l - cmax) for every (point, own component); per-point sums
        float2 E[NP][Q_BATCH];
        float s[Q_BATCH];
#pragma unroll
        for (int q = 0; q < Q_BATCH; ++q) {
            const float2 X0 = dup(x[q].x), X1 = dup(x[q].y), X2 = dup(x[q].z);
            float2 acc = f2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                float2 l = logit2(prm[j], X0, X1, X2);
                float2 e = f2(ex2_approx(l.x), ex2_approx(l.y));
                E[j][q] = e;
                acc = add2(acc, e);
            }
            s[q] = acc.x + acc.y;
        }
        float tot = warp_transpose_reduce8(s, lane, AddOp());
        tot = cta_combine(tot, red_sum[slot], G, warp, lane, AddOp());
        const bool myvalid = base + myq < end;
        float ref = cmax;
        // Rare path: a point whose best component is > 100 binades below cmax.
        // Redo the batch with the exact per-point maximum (Eq. logestep's
        // max-subtraction) so that no responsibility is lost to underflow.
        if (__any_sync(FULL, myvalid && !(tot >= 0x1p-100f))) {
            float m[Q_BATCH];
#pragma unroll
            for (int q = 0; q < Q_BATCH; ++q) {
                const float2 X0 = dup(x[q].x), X1 = dup(x[q].y), X2 = dup(x[q].z);
                float mm = -INFINITY;
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    float2 l = logit2(prm[j], X0, X1, X2);
                    E[j][q] = l;
                    mm = fmaxf(mm, fmaxf(l.x, l.y));
                }
                m[q] = mm;
            }
            float mt = warp_transpose_reduce8(m, lane, MaxOp());
            mt = cta_combine(mt, red_aux[0], G, warp, lane, MaxOp());
#pragma unroll
            for (int q = 0; q < Q_BATCH; ++q) {
                float mq = __shfl_sync(FULL, mt, q * 4);
                mq = (mq > -INFINITY) ? mq : 0.f;
                float2 acc = f2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    float2 e = f2(ex2_approx(E[j][q].x - mq), ex2_approx(E[j][q].y - mq));
                    E[j][q] = e;
                    acc = add2(acc, e);
                }
                s[q] = acc.x + acc.y;
            }
            tot = warp_transpose_reduce8(s, lane, AddOp());
            tot = cta_combine(tot, red_aux[1], G, warp, lane, AddOp());
            if (myvalid && !(mt > -INFINITY)) set_error(a.st, GIRA_ERR_NUMERIC);
            ref = cmax + ((mt > -INFINITY) ? mt : 0.f);
        }
        const bool ok = myvalid && tot > 0.f;
        const float r = ok ? __frcp_rn(tot) : 0.f;
        const float lse2 = lg2_approx(tot) + ref;   // log2 sum_b pi_b N(x|b)
        if (owner && ok) {
            ll_acc += (double)lse2;
            if (!STATS && a.per_point) a.per_point[base + myq] = lse2 * LN2F;
        }

        // ---- pass 2: gamma = e / sum, statistics about the old means
        if (STATS) {
#pragma unroll
            for (int q = 0; q < Q_BATCH; ++q) {
                const float2 R = dup(__shfl_sync(FULL, r, q * 4));
                const float2 X0 = dup(x[q].x), X1 = dup(x[q].y), X2 = dup(x[q].z);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const float2 g = mul2(E[j][q], R);
                    const float2 d0 = add2(X0, prm[j].nmu[0]);
                    const float2 d1 = add2(X1, prm[j].nmu[1]);
                    const float2 d2 = add2(X2, prm[j].nmu[2]);
                    const float2 g0 = mul2(g, d0), g1 = mul2(g, d1), g2 = mul2(g, d2);
                    S[j][0] = add2(S[j][0], g);
                    S[j][1] = add2(S[j][1], g0);
                    S[j][2] = add2(S[j][2], g1);
                    S[j][3] = add2(S[j][3], g2);
                    S[j][4] = fma2(g0, d0, S[j][4]);
                    S[j][5] = fma2(g0, d1, S[j][5]);
                    S[j][6] = fma2(g0, d2, S[j][6]);
                    S[j][7] = fma2(g1, d1, S[j][7]);
                    S[j][8] = fma2(g1, d2, S[j][8]);
                    S[j][9] = fma2(g2, d2, S[j][9]);
                }
            }
        }
    }

    if (STATS) {
        float* dst = a.partials + (size_t)blockIdx.x * a.k * NSTAT;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const int b0 = 2 * ((j * G + warp) * 32 + lane);
            if (b0 < a.k)
#pragma unroll
                for (int s = 0; s < NSTAT; ++s) dst[(size_t)b0 * NSTAT + s] = S[j][s].x;
            if (b0 + 1 < a.k)
#pragma unroll
                for (int s = 0; s < NSTAT; ++s) dst[(size_t)(b0 + 1) * NSTAT + s] = S[j][s].y;
        }
    }
    if (warp == 0) {   // lanes 0,4,..,28 hold the per-point log-likelihood sums; fixed order
        double v = ll_acc;
        v += __shfl_xor_sync(FULL, v, 4);
        v += __shfl_xor_sync(FULL, v, 8);
        v += __shfl_xor_sync(FULL, v, 16);
        if (lane == 0) a.ll_partials[blockIdx.x] = v * LN2;
    }
}

// ------------------------------------------------------------------ launch policy
struct Shape {
    int np, g, threads;
};

Shape shape_for(int k) {
    if (k <= 64) return {1, 1, 32};
    int g = (k + 127) / 128;
    return {2, g, 32 * g};
}

template <bool STATS>
const void* kernel_for(const Shape& sh) {
    if (sh.np == 1) return (const void*)estep_kernel<1, 32, 16, STATS>;
    if (sh.g <= 4) return (const void*)estep_kernel<2, 128, 3, STATS>;
    return (const void*)estep_kernel<2, 256, 1, STATS>;
}

}  // namespace

int params_pairs_padded(int k) {
    Shape sh = shape_for(k);
    return sh.np * sh.g * 32;
}

int estep_grid(int64_t n, int k, bool stats, int num_sms, int64_t* pts_per_cta) {
    Shape sh = shape_for(k);
    const void* fn = stats ? kernel_for<true>(sh) : kernel_for<false>(sh);
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, sh.threads, 0) != cudaSuccess || occ < 1) occ = 1;
    int64_t batches = (n + Q_BATCH - 1) / Q_BATCH;
    int64_t grid = std::min<int64_t>(batches, (int64_t)num_sms * occ);
    int64_t ppc = ((n + grid - 1) / grid + Q_BATCH - 1) / Q_BATCH * Q_BATCH;
    grid = (n + ppc - 1) / ppc;
    *pts_per_cta = ppc;
    return (int)grid;
}

cudaError_t launch_estep(const EStepLaunch& a, bool stats, int grid, cudaStream_t s) {
    Shape sh = shape_for(a.k);
    void* args[] = {(void*)&a};
    const void* fn = stats ? kernel_for<true>(sh) : kernel_for<false>(sh);
    return cudaLaunchKernel(fn, dim3(grid), dim3(sh.threads), args, 0, s);
}

// ------------------------------------------------------------------ pack + padding
namespace {
__global__ void pack_kernel(const float* __restrict__ p3, int64_t n, float4* __restrict__ p4, DeviceState* st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = p3[3 * i], y = p3[3 * i + 1], z = p3[3 * i + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) set_error(st, GIRA_ERR_NONFINITE_INPUT);
    p4[i] = make_float4(x, y, z, 0.f);
}

__global__ void fill_padding_kernel(float* params, int k, int npairs_pad) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;   // component slot
    if (b >= 2 * npairs_pad || b < k) return;
    float* base = params + (size_t)(b >> 1) * PAIR_FLOATS + (b & 1);
    for (int s = 0; s < PAIR_FLOATS / 2; ++s) base[2 * s] = 0.f;
    base[2 * SLOT_C] = -INFINITY;
}
}  // namespace

cudaError_t launch_pack(const float* pts3, int64_t n, float4* pts4, DeviceState* st, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    pack_kernel<<<(unsigned)blocks, 256, 0, s>>>(pts3, n, pts4, st);
    return cudaGetLastError();
}

cudaError_t launch_fill_padding(float* params, int k, int npairs_pad, cudaStream_t s) {
    int slots = 2 * npairs_pad;
    fill_padding_kernel<<<(slots + 127) / 128, 128, 0, s>>>(params, k, npairs_pad);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ reduce
namespace {
// stats64[b][s] = sum over CTAs (fixed order: binary32 groups of 16, binary64 across groups);
// block 0 also sums the per-CTA log-likelihoods into st->ll_sum.
__global__ void em_reduce_kernel(const float* __restrict__ partials, const double* __restrict__ llp, int grid, int k,
                                 double* __restrict__ stats64, DeviceState* st, int iter) {
    if (iter > st->stop_after || st->error) return;
    const int total = k * NSTAT;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (partials && idx < total) {
        double acc = 0.0;
        for (int c0 = 0; c0 < grid; c0 += 16) {
            const int c1 = min(grid, c0 + 16);
            float f = 0.f;
            for (int c = c0; c < c1; ++c) f += partials[(size_t)c * total + idx];
            acc += (double)f;
        }
        stats64[idx] = acc;
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        double v = 0.0;
        for (int c = threadIdx.x; c < grid; c += 32) v += llp[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (threadIdx.x == 0) st->ll_sum = v;
    }
}
}  // namespace

cudaError_t launch_em_reduce(const float* partials, const double* ll_partials, int grid, int k, double* stats64,
                             DeviceState* st, int iter, cudaStream_t s) {
    int total = partials ? k * NSTAT : 1;
    em_reduce_kernel<<<(total + 255) / 256, 256, 0, s>>>(partials, ll_partials, grid, k, stats64, st, iter);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 finalize
namespace {

// From (pi, mu, Sigma) in binary64 to the E-step parameters of component b:
// Cholesky Sigma = L L^T (closed form 3x3), P = L^{-1}, scaled to base 2.
// Returns false (and flags GIRA_ERR_NOT_PD) if a pivot is not positive.
__device__ bool build_component(int b, double pi, const double mu[3], const double c[6], float* params,
                                float4* shift4, double* model64, DeviceState* st) {
    // c = (00, 01, 02, 11, 12, 22)
    const double a00 = c[0];
    bool pd = a00 > 0.0;
    const double L00 = pd ? sqrt(a00) : 1.0;
    const double L10 = c[1] / L00, L20 = c[2] / L00;
    const double a11 = c[3] - L10 * L10;
    pd = pd && a11 > 0.0;
    const double L11 = pd ? sqrt(a11) : 1.0;
    const double L21 = (c[4] - L20 * L10) / L11;
    const double a22 = c[5] - L20 * L20 - L21 * L21;
    pd = pd && a22 > 0.0;
    const double L22 = pd ? sqrt(a22) : 1.0;
    if (!pd) {
        atomicMin(&st->bad_component, b);
        set_error(st, GIRA_ERR_NOT_PD);
        return false;
    }
    const double P00 = 1.0 / L00, P11 = 1.0 / L11, P22 = 1.0 / L22;
    const double P10 = -L10 * P00 * P11;
    const double P21 = -L21 * P11 * P22;
    const double P20 = -(L20 * P00 + L21 * P10) * P22;
    const double alpha = 0.84932180028801904272;   // sqrt(log2(e) / 2)
    const double q[6] = {alpha * P00, alpha * P10, alpha * P11, alpha * P20, alpha * P21, alpha * P22};
    const double bb[3] = {-(q[0] * mu[0]), -(q[1] * mu[0] + q[2] * mu[1]), -(q[3] * mu[0] + q[4] * mu[1] + q[5] * mu[2])};
    const double LOG2_2PI = 2.6514961294723187980;     // log2(2 pi)
    const double cc = log2(pi) + log2(P00) + log2(P11) + log2(P22) - 1.5 * LOG2_2PI;
    float* base = params + (size_t)(b >> 1) * PAIR_FLOATS + (b & 1);
    for (int i = 0; i < 6; ++i) base[2 * (SLOT_P + i)] = (float)q[i];
    for (int i = 0; i < 3; ++i) base[2 * (SLOT_B + i)] = (float)bb[i];
    base[2 * SLOT_C] = (float)cc;
    float m32[3] = {(float)mu[0], (float)mu[1], (float)mu[2]};
    for (int i = 0; i < 3; ++i) base[2 * (SLOT_NMU + i)] = -m32[i];
    shift4[b] = make_float4(m32[0], m32[1], m32[2], 0.f);
    double* m = model64 + (size_t)b * MODEL;
    m[0] = pi;
    m[1] = mu[0]; m[2] = mu[1]; m[3] = mu[2];
    for (int i = 0; i < 6; ++i) m[4 + i] = c[i];
    return true;
}

// M-step from the shifted statistics (d = x - s_b):
//   N_b = S0 + 10 eps, mu = (S0 s + S1) / N_b, delta = mu - s,
//   sum r (x-mu)(x-mu)^T = S2 - delta S1^T - S1 delta^T + S0 delta delta^T,
//   Sigma = that / N_b + reg I,  pi = N_b / sum_a N_a.
__global__ void finalize_kernel(const double* __restrict__ stats64, float4* shift4, int k, int64_t n, double reg,
                                double tol, double* model64, float* params, double* trace, DeviceState* st, int iter,
                                int em) {
    __shared__ double s_part[32];
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (em && iter > st->stop_after) || st->error != 0;
    __syncthreads();
    if (s_skip) return;
    const double tiny = 10.0 * DBL_EPSILON;
    // sum_a N_a (every block computes it, same fixed order)
    double part = 0.0;
    for (int a = threadIdx.x; a < k; a += blockDim.x) part += stats64[(size_t)a * NSTAT] + tiny;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    double nsum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) nsum += s_part[w];

    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < k) {
        const double* S = stats64 + (size_t)b * NSTAT;
        const float4 sh = shift4[b];
        const double s[3] = {sh.x, sh.y, sh.z};
        const double s0 = S[0];
        const double nb = s0 + tiny;
        const double inv = 1.0 / nb;
        double mu[3], dl[3];
        for (int i = 0; i < 3; ++i) {
            mu[i] = (s0 * s[i] + S[1 + i]) * inv;
            dl[i] = mu[i] - s[i];
        }
        // S2 index: 00->4, 01->5, 02->6, 11->7, 12->8, 22->9
        const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        double c[6];
        for (int t = 0; t < 6; ++t) {
            const int i = ij[t][0], j = ij[t][1];
            double v = S[4 + t] - dl[i] * S[1 + j] - S[1 + i] * dl[j] + s0 * dl[i] * dl[j];
            c[t] = v * inv + ((i == j) ? reg : 0.0);
        }
        build_component(b, nb / nsum, mu, c, params, shift4, model64, st);
    }
    if (em && blockIdx.x == 0 && threadIdx.x == 0) {
        const double ll = st->ll_sum / (double)n;
        trace[iter - 1] = ll;
        if (iter > 1 && fabs(ll - st->prev_ll) < tol) st->stop_after = iter;
        st->prev_ll = ll;
        st->iters_done = iter;
    }
}

__global__ void params_from_model_kernel(const float* __restrict__ w, const float* __restrict__ mu,
                                         const float* __restrict__ cov, int k, double* model64, float* params,
                                         float4* shift4, DeviceState* st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= k) return;
    const double pi = w[b];
    const double m[3] = {mu[3 * b], mu[3 * b + 1], mu[3 * b + 2]};
    const float* S = cov + 9 * (size_t)b;
    const double c[6] = {S[0], S[3], S[6], S[4], S[7], S[8]};   // lower triangle, as the oracle reads it
    bool fin = isfinite(pi) && isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]);
    for (int i = 0; i < 9; ++i) fin = fin && isfinite(S[i]);
    if (!fin) { set_error(st, GIRA_ERR_NONFINITE_INPUT); return; }
    if (!(pi > 0.0)) { set_error(st, GIRA_ERR_INVALID_ARG); return; }
    build_component(b, pi, m, c, params, shift4, model64, st);
}

__global__ void model_out_kernel(const double* __restrict__ model64, int k, float* w, float* mu, float* cov) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= k) return;
    const double* m = model64 + (size_t)b * MODEL;
    w[b] = (float)m[0];
    for (int i = 0; i < 3; ++i) mu[3 * b + i] = (float)m[1 + i];
    const int idx[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    for (int i = 0; i < 9; ++i) cov[9 * (size_t)b + i] = (float)m[4 + idx[i]];
}
}  // namespace

cudaError_t launch_finalize(const double* stats64, float4* shift4, int k, int64_t n, double reg, double tol,
                            double* model64, float* params, double* trace, DeviceState* st, int iter, bool em,
                            cudaStream_t s) {
    finalize_kernel<<<(k + 31) / 32, 32, 0, s>>>(stats64, shift4, k, n, reg, tol, model64, params, trace, st, iter,
                                                 em ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_params_from_model(const float* w, const float* mu, const float* cov, int k, double* model64,
                                     float* params, float4* shift4, DeviceState* st, cudaStream_t s) {
    params_from_model_kernel<<<(k + 63) / 64, 64, 0, s>>>(w, mu, cov, k, model64, params, shift4, st);
    return cudaGetLastError();
}

cudaError_t launch_model_out(const double* model64, int k, float* w, float* mu, float* cov, cudaStream_t s) {
    model_out_kernel<<<(k + 63) / 64, 64, 0, s>>>(model64, k, w, mu, cov);
    return cudaGetLastError();
}

}  // namespace gira
