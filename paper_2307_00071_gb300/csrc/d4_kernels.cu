// d4_kernels.cu -- the fit in four dimensions (xyz + intensity, the paper's
// SOGMM data), Gaussian-mixture regression of intensity on xyz, and sampling
// from a mixture.
//
// GIRA (arXiv 2307.00071) Sec. V: the E-step of Eq. (estep) in the log domain
// of Eq. (logestep), the log-density of Eq. (simplifiedGaussian) with D = 4
// (the (1,K,4)/(1,K,4,4) layout of the paper's model), the standard M-step on
// the sufficient statistics; Sec. IV's use of the model: intensity inferred at
// given positions (conditional mean and variance) and points resampled from
// the joint distribution.
//
// The E-step here is the component-stationary design of the 3D kernel with one
// component per lane (scalar FP32): G = ceil(K / 32) warps hold all K <= 1024
// components, a CTA's points arrive by one TMA bulk copy (one float4 each),
// per batch of 8 points the sums over components are reduced across lanes
// (transpose-reduce) and warps (shared memory, one barrier), and pass 2
// accumulates S0, S1 (4), S2 (10) about mu_b.  Logits use d = x - mu_b
// (P'd, not P'x + b': intensity and metres-scale coordinates share a point).
#include <float.h>
#include <math.h>

#include <algorithm>

#include "gira_internal.cuh"

namespace gira {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int Q4 = 8;
constexpr int PPC4_MAX = 2048;                          // points staged per CTA (64 KB)
constexpr long long MBAR_LIMIT4 = 2000000000ll;         // bound on the TMA wait: 2 s of wall time
constexpr float LN2F4 = 0.693147180559945309f;
constexpr double LN2_4 = 0.693147180559945309417232121458;

// lower-triangular index of (i, j), j <= i: 00,10,11,20,21,22,30,31,32,33
__host__ __device__ constexpr int tri4(int i, int j) { return i * (i + 1) / 2 + j; }

// Slot s of component b in the pair-interleaved parameter buffer.
__host__ __device__ __forceinline__ size_t slot4(int b, int s) {
    return (size_t)(b >> 1) * PAIR4_FLOATS + 2 * s + (b & 1);
}

// CH = 0: the whole E-step of one CTA (every component); CH = 1: pass A of a
// chunk (per-point sums only); CH = 2: pass B of a chunk (statistics from pref).
template <bool STATS, int CH = 0>
__global__ void __launch_bounds__(512, 1) estep4_kernel(const EStep4Launch a) {
    extern __shared__ __align__(128) unsigned char dsm4[];
    __shared__ __align__(8) uint64_t bar_tma;
    __shared__ float red_sum[2][16][Q4];
    __shared__ float red_aux[2][16][Q4];
    __shared__ float s_cmax[16], s_wsum[16];
    __shared__ int s_skip, s_norm, s_dead;
    constexpr int LPQ = 32 / Q4;
    const int G = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int chunk = (CH != 0) ? (int)blockIdx.y : 0;
    const int pr = threadIdx.x;   // this lane's component pair: components 2 pr, 2 pr + 1 of the chunk
    const int k_here = (CH != 0) ? min(CHUNK4, a.k - chunk * CHUNK4) : a.k;
    const float* params = a.params + (size_t)chunk * (CHUNK4 / 2) * PAIR4_FLOATS;
    const int64_t begin = (int64_t)blockIdx.x * a.pts_per_cta;
    const int64_t end = min(a.n, begin + a.pts_per_cta);
    const int npts = (int)(end - begin);
    const int nb = (npts + Q4 - 1) / Q4;
    const float4* spts = reinterpret_cast<const float4*>(dsm4);   // (x,x,y,y)(z,z,w,w) per point
    if (threadIdx.x == 0) {
        // the points are never written by the kernel this one may overlap
        // (dependent launch), so their copy starts before the wait below
        mbar_init(&bar_tma, 1);
        mbar_fence_init();
        mbar_expect_tx(&bar_tma, (uint32_t)npts * 32u);
        tma_load_1d(reinterpret_cast<void*>(dsm4), a.pts8 + 2 * begin, (uint32_t)npts * 32u, &bar_tma);
    }
    pdl_wait();   // the parameters and the state written by the previous kernel
    if (threadIdx.x == 0) {
        s_skip = (a.iter > a.st->stop_after) || (a.st->error != 0);
        s_norm = a.st->w_raw;
        s_dead = 0;
    }
    __syncthreads();
    if (s_skip) {   // let the copy land before leaving
        if (threadIdx.x == 0) mbar_wait_bounded(&bar_tma, 0u, MBAR_LIMIT4);
        return;
    }
    pdl_allow_next();
    // ---- this lane's pair -> registers (padding components: c = -inf, never contribute)
    float2 P[10], nmu[4], c, w;
    {
        const float4* src = reinterpret_cast<const float4*>(params + (size_t)pr * PAIR4_FLOATS);
        float4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = src[i];
        const float2* f = reinterpret_cast<const float2*>(v);
#pragma unroll
        for (int i = 0; i < 10; ++i) P[i] = f[SLOT4_P + i];
        c = f[SLOT4_C];
#pragma unroll
        for (int i = 0; i < 4; ++i) nmu[i] = f[SLOT4_NMU + i];
        w = f[SLOT4_W];
    }
    float cm = fmaxf(c.x, c.y), ws = w.x + w.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cm = fmaxf(cm, __shfl_xor_sync(FULL, cm, o));
        ws += __shfl_xor_sync(FULL, ws, o);
    }
    if (lane == 0) {
        s_cmax[warp] = cm;
        s_wsum[warp] = ws;
    }
    if (!mbar_wait_bounded(&bar_tma, 0u, MBAR_LIMIT4)) s_dead = 1;
    __syncthreads();
    if (s_dead) {
        if (threadIdx.x == 0) {
            set_error(a.st, GIRA_ERR_TIMEOUT);
            mbar_wait_bounded(&bar_tma, 0u, MBAR_LIMIT4);
        }
        return;
    }
    float cmax = s_cmax[0], wsum = s_wsum[0];
    for (int i = 1; i < G; ++i) {
        cmax = fmaxf(cmax, s_cmax[i]);
        wsum += s_wsum[i];
    }
    if (CH != 0) cmax = a.gref[0];   // chunks: one reference for all K components
    const float2 cc = f2(cmax - c.x, cmax - c.y);   // >= 0; +inf for padding
    const float ref0 = s_norm ? cmax - __log2f(wsum) : cmax;
    float2 S[NSTAT4];   // statistics of the lane's two components, packed
    if (STATS)
#pragma unroll
        for (int i = 0; i < NSTAT4; ++i) S[i] = f2(0.f, 0.f);
    double ll_acc = 0.0;
    const int myq = q_of_lane<Q4>(lane);
    const bool owner = (warp == 0) && ((lane & (LPQ - 1)) == 0);

    // q' = |P'(x - mu)|^2 + (cmax - c) for both components: minus the base-2
    // logit relative to cmax (packed: one FFMA2 / FADD2 / FMUL2 per pair)
    auto qform = [&](int li) {
        const float4 xy = spts[2 * li], zw = spts[2 * li + 1];
        const float2 d0 = add2(f2(xy.x, xy.y), nmu[0]), d1 = add2(f2(xy.z, xy.w), nmu[1]);
        const float2 d2 = add2(f2(zw.x, zw.y), nmu[2]), d3 = add2(f2(zw.z, zw.w), nmu[3]);
        const float2 y0 = mul2(P[0], d0);
        const float2 y1 = fma2(P[2], d1, mul2(P[1], d0));
        const float2 y2 = fma2(P[5], d2, fma2(P[4], d1, mul2(P[3], d0)));
        const float2 y3 = fma2(P[9], d3, fma2(P[8], d2, fma2(P[7], d1, mul2(P[6], d0))));
        return fma2(y3, y3, fma2(y2, y2, fma2(y1, y1, fma2(y0, y0, cc))));
    };
    // pass 2: S0 = sum g, S1 = sum g d, S2 = sum g d d^T about mu_b for both
    // components at once (packed); g = e * R with R the owner lane's 1 / total
    // (r != nullptr) or already folded into e (pass B)
    auto accumulate = [&](int lb, int nvalid, const float2 (&Eq)[Q4], const float* r) {
#pragma unroll
        for (int q = 0; q < Q4; ++q) {
            const int li = (q < nvalid) ? lb + q : lb;
            const float4 xy = spts[2 * li], zw = spts[2 * li + 1];
            const float2 g = r ? mul2(Eq[q], dup(__shfl_sync(FULL, *r, q * LPQ))) : Eq[q];
            const float2 d[4] = {add2(f2(xy.x, xy.y), nmu[0]), add2(f2(xy.z, xy.w), nmu[1]),
                                 add2(f2(zw.x, zw.y), nmu[2]), add2(f2(zw.z, zw.w), nmu[3])};
            float2 gd[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) gd[i] = mul2(g, d[i]);
            S[0] = add2(S[0], g);
#pragma unroll
            for (int i = 0; i < 4; ++i) S[1 + i] = add2(S[1 + i], gd[i]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = i; j < 4; ++j) S[5 + sym4(i, j)] = fma2(gd[i], d[j], S[5 + sym4(i, j)]);
        }
    };
    float2 E[Q4];
    for (int t = 0; t < nb; ++t) {
        const int lb = t * Q4, nvalid = min(Q4, npts - lb);
        if (CH == 2) {
            // pass B: e relative to the point's reference, times 1 / total, into the statistics
#pragma unroll
            for (int q = 0; q < Q4; ++q) {
                const float2 prq = (q < nvalid) ? a.pref[begin + lb + q] : f2(0.f, 0.f);
                const float2 nq = qform((q < nvalid) ? lb + q : lb);
                E[q] = f2(ex2_approx(prq.x - nq.x) * prq.y, ex2_approx(prq.x - nq.y) * prq.y);
            }
            if (STATS) accumulate(lb, nvalid, E, nullptr);
            continue;
        }
        // pass 1: e for (point, own components), per-point sums over the CTA
        float part[Q4];
#pragma unroll
        for (int q = 0; q < Q4; ++q) {
            const float2 nq = qform((q < nvalid) ? lb + q : lb);
            E[q] = f2(ex2_approx(-nq.x), ex2_approx(-nq.y));
            part[q] = E[q].x + E[q].y;
        }
        const float wt = warp_transpose_reduce<Q4>(part, lane, AddOp());
        if ((lane & (LPQ - 1)) == 0) red_sum[t & 1][warp][myq] = wt;
        __syncthreads();
        float tot = red_sum[t & 1][0][myq];
        for (int i = 1; i < G; ++i) tot += red_sum[t & 1][i][myq];
        const bool myvalid = myq < nvalid;
        if (CH == 1) {   // pass A: the chunk's sum for each point
            if (owner && myvalid) a.psum[(size_t)chunk * a.n + begin + lb + myq] = tot;
            continue;
        }
        float ref = ref0;
        if (__any_sync(FULL, myvalid && !(tot >= 0x1p-100f))) {
            // rare: a point > 100 binades below cmax everywhere; exact per-point maximum
            float m[Q4];
#pragma unroll
            for (int q = 0; q < Q4; ++q) {
                const float2 nq = qform((q < nvalid) ? lb + q : lb);
                E[q] = f2(-nq.x, -nq.y);
                m[q] = fmaxf(E[q].x, E[q].y);
            }
            float mt = warp_transpose_reduce<Q4>(m, lane, MaxOp());
            if ((lane & (LPQ - 1)) == 0) red_aux[0][warp][myq] = mt;
            __syncthreads();
            mt = red_aux[0][0][myq];
            for (int i = 1; i < G; ++i) mt = fmaxf(mt, red_aux[0][i][myq]);
            float p2[Q4];
#pragma unroll
            for (int q = 0; q < Q4; ++q) {
                float mq = __shfl_sync(FULL, mt, q * LPQ);
                mq = (mq > -INFINITY) ? mq : 0.f;
                E[q] = f2(ex2_approx(E[q].x - mq), ex2_approx(E[q].y - mq));
                p2[q] = E[q].x + E[q].y;
            }
            const float w2 = warp_transpose_reduce<Q4>(p2, lane, AddOp());
            if ((lane & (LPQ - 1)) == 0) red_aux[1][warp][myq] = w2;
            __syncthreads();
            tot = red_aux[1][0][myq];
            for (int i = 1; i < G; ++i) tot += red_aux[1][i][myq];
            if (myvalid && !(mt > -INFINITY)) set_error(a.st, GIRA_ERR_NUMERIC);
            ref = ref0 + ((mt > -INFINITY) ? mt : 0.f);
        }
        const bool ok = myvalid && tot > 0.f;
        const float lse2 = lg2_approx(tot) + ref;
        if (owner && ok) {
            ll_acc += (double)lse2;
            if (!STATS && a.per_point) a.per_point[begin + lb + myq] = lse2 * LN2F4;
        }
        const float r = ok ? __frcp_rn(tot) : 0.f;
        if (STATS) accumulate(lb, nvalid, E, &r);
    }
    if (STATS) {
        const int kc = (CH != 0) ? CHUNK4 : a.k;   // components per partial block
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int b = 2 * pr + h;
            if (b < k_here) {
                float* dst = a.partials + (((size_t)chunk * gridDim.x + blockIdx.x) * kc + b) * NSTAT4;
#pragma unroll
                for (int i = 0; i < NSTAT4; ++i) dst[i] = h ? S[i].y : S[i].x;
            }
        }
    }
    if (CH != 0) return;
    if (warp == 0) {
        double v = ll_acc;
#pragma unroll
        for (int o = LPQ; o < 32; o <<= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0) a.ll_partials[blockIdx.x] = v * LN2_4;
    }
}

// From (w, mu, Sigma) in binary64: Cholesky, P = L^{-1}, the base-2 constants.
__device__ bool build_component4(int b, double w, const double mu[4], const double S[16], float* params,
                                 double* model64, DeviceState* st) {
    double L[16] = {0};
    bool pd = true;
    for (int j = 0; j < 4 && pd; ++j) {
        double s = S[4 * j + j];
        for (int k = 0; k < j; ++k) s -= L[4 * j + k] * L[4 * j + k];
        if (!(s > 0.0)) { pd = false; break; }
        L[4 * j + j] = sqrt(s);
        for (int i = j + 1; i < 4; ++i) {
            double t = S[4 * i + j];
            for (int k = 0; k < j; ++k) t -= L[4 * i + k] * L[4 * j + k];
            L[4 * i + j] = t / L[4 * j + j];
        }
    }
    if (!pd) {
        atomicMin(&st->bad_component, b);
        set_error(st, GIRA_ERR_NOT_PD);
        return false;
    }
    double P[16] = {0};
    for (int cidx = 0; cidx < 4; ++cidx)
        for (int i = cidx; i < 4; ++i) {
            double t = (i == cidx) ? 1.0 : 0.0;
            for (int k = cidx; k < i; ++k) t -= L[4 * i + k] * P[4 * k + cidx];
            P[4 * i + cidx] = t / L[4 * i + i];
        }
    const double alpha = 0.84932180028801904272;   // sqrt(log2(e) / 2)
    const double LOG2_2PI = 2.6514961294723187980;  // log2(2 pi)
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j <= i; ++j) params[slot4(b, SLOT4_P + tri4(i, j))] = (float)(alpha * P[4 * i + j]);
    // log2 w + sum_j log2 P_jj - (4/2) log2(2 pi)
    params[slot4(b, SLOT4_C)] = (float)(log2(w * (P[0] * P[5] * P[10] * P[15])) - 2.0 * LOG2_2PI);
    for (int i = 0; i < 4; ++i) params[slot4(b, SLOT4_NMU + i)] = -(float)mu[i];
    params[slot4(b, SLOT4_W)] = (float)w;
    double* m = model64 + (size_t)b * MODEL4;
    m[0] = w;
    for (int i = 0; i < 4; ++i) m[1 + i] = mu[i];
    for (int i = 0; i < 4; ++i)
        for (int j = i; j < 4; ++j) m[5 + sym4(i, j)] = S[4 * i + j];
    return true;
}

// One block per component: fixed-order binary64 sum of its per-CTA partials
// (32 slices, binary32 groups of 8 inside a slice), then the M-step and build.
// The E-step kept mu_b (as binary32) as the shift, so the statistics are about
// the previous mean, and the update un-shifts them exactly in binary64.
__global__ void __launch_bounds__(NSTAT4 * 32) reduce_finalize4_kernel(
    const float* __restrict__ partials, int grid, int kc, const double* __restrict__ llp, int ll_count,
    const double* __restrict__ stats64, const float4* __restrict__ shift4, int k, int64_t n, double reg, double tol,
    double* model64, float* params, double* trace, DeviceState* st, int iter, int em) {
    __shared__ double part[32][NSTAT4];
    __shared__ double Sb[NSTAT4];
    __shared__ int s_skip;
    pdl_wait();         // the E-step's partials (dependent launch)
    pdl_allow_next();   // the next E-step may stage its points meanwhile
    if (threadIdx.x == 0) s_skip = (em && iter > st->stop_after) || st->error != 0;
    __syncthreads();
    if (s_skip) return;
    const int b = blockIdx.x, t = threadIdx.x;
    if (partials) {
        const int o = t % NSTAT4, q = t / NSTAT4;
        const int c0 = q * grid / 32, c1 = (q + 1) * grid / 32;
        const float* src = partials + ((size_t)(b / kc) * grid * kc + b % kc) * NSTAT4 + o;
        double acc = 0.0;
        for (int cta = c0; cta < c1; cta += 8) {
            float f = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) f += (cta + u < c1) ? __ldcg(src + (size_t)(cta + u) * kc * NSTAT4) : 0.f;
            acc += (double)f;
        }
        part[q][o] = acc;
        __syncthreads();
        if (t < NSTAT4) {
            double v = 0.0;
            for (int q2 = 0; q2 < 32; ++q2) v += part[q2][t];
            Sb[t] = v;
        }
    } else if (t < NSTAT4) {
        Sb[t] = stats64[(size_t)b * NSTAT4 + t];
    }
    __syncthreads();
    if (t == 0) {
        double s[4];
        if (shift4) {
            const float4 v = shift4[b];
            s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
        } else {
            for (int i = 0; i < 4; ++i) s[i] = -(double)params[slot4(b, SLOT4_NMU + i)];
        }
        const double s0 = Sb[0];
        const double nbw = s0 + 10.0 * DBL_EPSILON;
        const double inv = 1.0 / nbw;
        double mu[4], dl[4];
        for (int i = 0; i < 4; ++i) {
            mu[i] = (s0 * s[i] + Sb[1 + i]) * inv;
            dl[i] = mu[i] - s[i];
        }
        double S[16];
        for (int i = 0; i < 4; ++i)
            for (int j = i; j < 4; ++j) {
                const double v = Sb[5 + sym4(i, j)] - dl[i] * Sb[1 + j] - Sb[1 + i] * dl[j] + s0 * dl[i] * dl[j];
                S[4 * i + j] = S[4 * j + i] = v * inv + ((i == j) ? reg : 0.0);
            }
        build_component4(b, nbw, mu, S, params, model64, st);
        if (b == 0) st->w_raw = 1;
    }
    if (em && b == 0 && t >= 32 && t < 64) {   // warp 1: log-likelihood, trace, convergence
        const int lane = t - 32;
        double v = 0.0;
        for (int cta = lane; cta < ll_count; cta += 32) v += llp[cta];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0) {
            st->ll_sum = v;
            const double ll = v / (double)n;
            trace[iter - 1] = ll;
            if (iter > 1 && fabs(ll - st->prev_ll) < tol) st->stop_after = iter;
            st->prev_ll = ll;
            st->iters_done = iter;
        }
    }
}

__global__ void params_from_model4_kernel(const float* __restrict__ w, const float* __restrict__ mu,
                                          const float* __restrict__ cov, int k, double* model64, float* params,
                                          DeviceState* st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= k) return;
    const double pi = w[b];
    double m[4], S[16];
    bool fin = isfinite(pi);
    for (int i = 0; i < 4; ++i) {
        m[i] = mu[4 * (size_t)b + i];
        fin = fin && isfinite(m[i]);
    }
    // the lower triangle is read, as the oracle's Cholesky reads it
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j <= i; ++j) {
            const double v = cov[16 * (size_t)b + 4 * i + j];
            fin = fin && isfinite(v);
            S[4 * i + j] = S[4 * j + i] = v;
        }
    if (!fin) { set_error(st, GIRA_ERR_NONFINITE_INPUT); return; }
    if (!(pi > 0.0)) { set_error(st, GIRA_ERR_INVALID_ARG); return; }
    build_component4(b, pi, m, S, params, model64, st);
}

__global__ void model_out4_kernel(const double* __restrict__ model64, int k, float* w, float* mu, float* cov,
                                  const DeviceState* st) {
    __shared__ double s_part[2];
    double part = 0.0;
    for (int a2 = threadIdx.x; a2 < k; a2 += blockDim.x) part += model64[(size_t)a2 * MODEL4];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    const double nsum = s_part[0] + s_part[1];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < k; b += gridDim.x * blockDim.x) {
        const double* m = model64 + (size_t)b * MODEL4;
        w[b] = (float)(st->w_raw ? m[0] / nsum : m[0]);
        for (int i = 0; i < 4; ++i) mu[4 * (size_t)b + i] = (float)m[1 + i];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) cov[16 * (size_t)b + 4 * i + j] = (float)m[5 + sym4(min(i, j), max(i, j))];
    }
}

// Padding components b in [k, kpad): zero parameters, c = -inf.
__global__ void fill_padding4_kernel(float* params, int k, int kpad) {
    const int b = k + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= kpad) return;
    for (int i = 0; i < PAIR4_FLOATS / 2; ++i) params[slot4(b, i)] = 0.f;
    params[slot4(b, SLOT4_C)] = -INFINITY;
}

// N x 4 -> p4 (x,y,z,I) (nullable) and p8 (x,x,y,y)(z,z,I,I); flags non-finite input.
__global__ void pack4_kernel(const float* __restrict__ p4in, int64_t n, float4* __restrict__ p4,
                             float4* __restrict__ p8, DeviceState* st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = make_float4(p4in[4 * i], p4in[4 * i + 1], p4in[4 * i + 2], p4in[4 * i + 3]);
    if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w))) set_error(st, GIRA_ERR_NONFINITE_INPUT);
    if (p4) p4[i] = v;
    p8[2 * i] = make_float4(v.x, v.x, v.y, v.y);
    p8[2 * i + 1] = make_float4(v.z, v.z, v.w, v.w);
}

// ------------------------------------------------------------------ regression of intensity on xyz
// Per component (binary64, then binary32): P_xx = chol(S_xx)^{-1} (6), g = S_xx^{-1} S_xI
// (3), v = S_II - S_Ix g, c = ln pi - sum ln L_ii - (3/2) ln 2 pi, mu (4): 17 floats.
constexpr int COND_FLOATS = 20;

__global__ void cond_prepare_kernel(const float* __restrict__ w, const float* __restrict__ mu,
                                    const float* __restrict__ cov, int k, float* prep, DeviceState* st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= k) return;
    bool fin = isfinite(w[b]);
    for (int i = 0; i < 4; ++i) fin = fin && isfinite(mu[4 * (size_t)b + i]);
    double S[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j <= i; ++j) {
            S[4 * i + j] = S[4 * j + i] = cov[16 * (size_t)b + 4 * i + j];
            fin = fin && isfinite(S[4 * i + j]);
        }
    if (!fin) {
        set_error(st, GIRA_ERR_NONFINITE_INPUT);
        return;
    }
    double L[9] = {0};
    for (int j = 0; j < 3; ++j) {
        double s = S[4 * j + j];
        for (int kk = 0; kk < j; ++kk) s -= L[3 * j + kk] * L[3 * j + kk];
        if (!(s > 0.0) || !isfinite(s)) {
            atomicMin(&st->bad_component, b);
            set_error(st, GIRA_ERR_NOT_PD);
            return;
        }
        L[3 * j + j] = sqrt(s);
        for (int i = j + 1; i < 3; ++i) {
            double t = S[4 * i + j];
            for (int kk = 0; kk < j; ++kk) t -= L[3 * i + kk] * L[3 * j + kk];
            L[3 * i + j] = t / L[3 * j + j];
        }
    }
    double P[9] = {0};
    for (int c = 0; c < 3; ++c)
        for (int i = c; i < 3; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int kk = c; kk < i; ++kk) t -= L[3 * i + kk] * P[3 * kk + c];
            P[3 * i + c] = t / L[3 * i + i];
        }
    const double sxi[3] = {S[3], S[7], S[11]};
    double u[3], g[3];
    for (int i = 0; i < 3; ++i) u[i] = P[3 * i] * sxi[0] + P[3 * i + 1] * sxi[1] + P[3 * i + 2] * sxi[2];
    for (int i = 0; i < 3; ++i) g[i] = P[i] * u[0] + P[3 + i] * u[1] + P[6 + i] * u[2];
    const double v = S[15] - (sxi[0] * g[0] + sxi[1] * g[1] + sxi[2] * g[2]);
    const double pi = w[b];
    if (!(pi > 0.0)) { set_error(st, GIRA_ERR_INVALID_ARG); return; }
    const double c = log(pi) - (log(L[0]) + log(L[4]) + log(L[8])) - 1.5 * log(2.0 * 3.14159265358979323846);
    float* o = prep + (size_t)b * COND_FLOATS;
    o[0] = (float)P[0]; o[1] = (float)P[3]; o[2] = (float)P[4]; o[3] = (float)P[6]; o[4] = (float)P[7];
    o[5] = (float)P[8];
    o[6] = (float)g[0]; o[7] = (float)g[1]; o[8] = (float)g[2];
    o[9] = (float)v;
    o[10] = (float)c;
    for (int i = 0; i < 4; ++i) o[11 + i] = mu[4 * (size_t)b + i];
}

// One thread per location, all K components in order, the prepared components
// staged through shared memory in tiles: pass 1 takes the maximum log-weight
// and, as a reference, the regression mean m_ref of that component; pass 2 sums
// w_b = exp(lw_b - max), w_b (m_b - m_ref) and w_b (v_b + (m_b - m_ref)^2) in
// binary32 (the shift keeps the variance free of cancellation).
constexpr int COND_THREADS = 256;
constexpr int COND_TILE = 256;

__global__ void __launch_bounds__(COND_THREADS) conditional4_kernel(const float* __restrict__ locs, int64_t m, int k,
                                                                    const float* __restrict__ prep, float* cmean,
                                                                    float* cvar, DeviceState* st) {
    __shared__ float sp[COND_TILE * COND_FLOATS];
    __shared__ int s_err;
    if (threadIdx.x == 0) s_err = st->error;
    __syncthreads();
    if (s_err) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < m;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (valid) {
        x0 = locs[3 * i];
        x1 = locs[3 * i + 1];
        x2 = locs[3 * i + 2];
        if (!(isfinite(x0) && isfinite(x1) && isfinite(x2))) set_error(st, GIRA_ERR_NONFINITE_INPUT);
    }
    // log-weight and regression mean of component o at this location
    auto eval = [&](const float* o, float& mb) {
        const float d0 = x0 - o[11], d1 = x1 - o[12], d2 = x2 - o[13];
        const float y0 = o[0] * d0;
        const float y1 = fmaf(o[2], d1, o[1] * d0);
        const float y2 = fmaf(o[5], d2, fmaf(o[4], d1, o[3] * d0));
        mb = fmaf(o[8], d2, fmaf(o[7], d1, fmaf(o[6], d0, o[14])));
        return fmaf(-0.5f, fmaf(y2, y2, fmaf(y1, y1, y0 * y0)), o[10]);
    };
    auto load_tile = [&](int b0, int nb) {
        __syncthreads();
        for (int t = threadIdx.x; t < nb * COND_FLOATS; t += blockDim.x) sp[t] = prep[(size_t)b0 * COND_FLOATS + t];
        __syncthreads();
    };
    float mx = -INFINITY, mref = 0.f;
    for (int b0 = 0; b0 < k; b0 += COND_TILE) {
        const int nb = min(COND_TILE, k - b0);
        load_tile(b0, nb);
        for (int b = 0; b < nb; ++b) {
            float mb;
            const float lw = eval(sp + b * COND_FLOATS, mb);
            if (lw > mx) {
                mx = lw;
                mref = mb;
            }
        }
    }
    float s = 0.f, e1 = 0.f, e2 = 0.f;
    for (int b0 = 0; b0 < k; b0 += COND_TILE) {
        const int nb = min(COND_TILE, k - b0);
        load_tile(b0, nb);
        for (int b = 0; b < nb; ++b) {
            const float* o = sp + b * COND_FLOATS;
            float mb;
            const float w = __expf(eval(o, mb) - mx);
            const float dm = mb - mref;
            s += w;
            e1 = fmaf(w, dm, e1);
            e2 = fmaf(w, fmaf(dm, dm, o[9]), e2);
        }
    }
    if (!valid) return;
    if (!(s > 0.f)) {
        set_error(st, GIRA_ERR_NUMERIC);
        return;
    }
    const float r = 1.f / s, a = e1 * r;
    cmean[i] = mref + a;
    if (cvar) cvar[i] = fmaf(-a, a, e2 * r);
}

// ------------------------------------------------------------------ sampling
// Cholesky factors (binary64, one thread per component) and the cumulative
// weights (binary64, in component order) for the sampler; one block.
__global__ void sample_prepare_kernel(const float* __restrict__ w, const float* __restrict__ mu,
                                      const float* __restrict__ cov, int k, int d, double* cum, double* chol,
                                      DeviceState* st) {
    for (int b = threadIdx.x; b < k; b += blockDim.x) {
        bool fin = isfinite(w[b]);
        for (int i = 0; i < d; ++i) fin = fin && isfinite(mu[(size_t)d * b + i]);
        for (int i = 0; i < d * d; ++i) fin = fin && isfinite(cov[(size_t)d * d * b + i]);
        if (!fin) {
            set_error(st, GIRA_ERR_NONFINITE_INPUT);
            continue;
        }
        if (!(w[b] >= 0.f)) set_error(st, GIRA_ERR_INVALID_ARG);
        double* L = chol + (size_t)16 * b;
        for (int i = 0; i < 16; ++i) L[i] = 0.0;
        for (int j = 0; j < d; ++j) {
            double s = cov[(size_t)d * d * b + d * j + j];
            for (int kk = 0; kk < j; ++kk) s -= L[4 * j + kk] * L[4 * j + kk];
            if (!(s > 0.0)) {
                atomicMin(&st->bad_component, b);
                set_error(st, GIRA_ERR_NOT_PD);
                break;
            }
            L[4 * j + j] = sqrt(s);
            for (int i = j + 1; i < d; ++i) {
                double t = cov[(size_t)d * d * b + d * i + j];
                for (int kk = 0; kk < j; ++kk) t -= L[4 * i + kk] * L[4 * j + kk];
                L[4 * i + j] = t / L[4 * j + j];
            }
        }
    }
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int b = 0; b < k; ++b) {
            tot += (double)w[b];
            cum[b] = tot;
        }
        if (!(tot > 0.0)) set_error(st, GIRA_ERR_INVALID_ARG);
    }
}

// Sample i: uniforms of draws 5i .. 5i+4 of seed (component, two Box-Muller
// pairs), x = mu_b + L_b z in binary64, rounded to binary32.
__global__ void sample_kernel(int64_t m, int k, int d, const float* __restrict__ mu, const double* __restrict__ cum,
                              const double* __restrict__ chol, uint64_t seed, float* out, int32_t* comp,
                              const DeviceState* st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || st->error) return;
    const double tot = cum[k - 1];
    const double u0 = uniform53(seed, 5 * (uint64_t)i) * tot;
    int lo = 0, hi = k - 1;   // first b with cum[b] > u0
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cum[mid] > u0) hi = mid; else lo = mid + 1;
    }
    const int b = lo;
    double z[4];
    for (int p = 0; p < 2; ++p) {
        const double u1 = uniform53(seed, 5 * (uint64_t)i + 1 + 2 * p);
        const double u2 = uniform53(seed, 5 * (uint64_t)i + 2 + 2 * p);
        const double r = sqrt(-2.0 * log(1.0 - u1));
        double sn, cs;
        sincos(2.0 * 3.14159265358979323846 * u2, &sn, &cs);
        z[2 * p] = r * cs;
        z[2 * p + 1] = r * sn;
    }
    const double* L = chol + (size_t)16 * b;
    for (int r = 0; r < d; ++r) {
        double x = mu[(size_t)d * b + r];
        for (int c = 0; c <= r; ++c) x += L[4 * r + c] * z[c];
        out[(size_t)d * i + r] = (float)x;
    }
    if (comp) comp[i] = b;
}

// ------------------------------------------------------------------ chunks (K above MAX_K4_DIRECT)
// gref[0] = max_b c_b over all k components; gref[1] = the log-likelihood
// reference (gref[0] - log2 sum_a w_a once the weights are raw N_b).
__global__ void chunk_ref4_kernel(const float* __restrict__ params, int k, const DeviceState* st, float* gref) {
    __shared__ float s_m[8];
    __shared__ double s_w[8];
    float m = -INFINITY;
    double w = 0.0;
    for (int b = threadIdx.x; b < k; b += blockDim.x) {
        m = fmaxf(m, params[slot4(b, SLOT4_C)]);
        w += (double)params[slot4(b, SLOT4_W)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
        w += __shfl_xor_sync(FULL, w, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_m[threadIdx.x >> 5] = m;
        s_w[threadIdx.x >> 5] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = s_m[0];
        double ww = s_w[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            mm = fmaxf(mm, s_m[i]);
            ww += s_w[i];
        }
        gref[0] = mm;
        gref[1] = st->w_raw ? (float)((double)mm - log2(ww)) : mm;
    }
}

// One warp per listed point (total over the chunks below 2^-100): the exact
// maximum of the logits over all k components, then (shift, 1 / sum) relative
// to it, with the E-step's arithmetic.
__global__ void chunk_exact4_kernel(const float4* __restrict__ pts8, const float* __restrict__ params, int k,
                                    const float* __restrict__ gref, const int* __restrict__ flags,
                                    const int* __restrict__ flag_count, float2* pref, double* llpt, DeviceState* st) {
    const int count = *flag_count;
    const float cmax = gref[0], ref0 = gref[1];
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int f = wg; f < count; f += nw) {
        const int64_t i = flags[f];
        const float4 xy = pts8[2 * i], zw = pts8[2 * i + 1];
        const float x[4] = {xy.x, xy.z, zw.x, zw.z};
        auto nlog = [&](int b) {   // q' = |P'(x - mu)|^2 + (cmax - c_b)
            float P[10], d[4];
            for (int j = 0; j < 10; ++j) P[j] = params[slot4(b, SLOT4_P + j)];
            for (int j = 0; j < 4; ++j) d[j] = x[j] + params[slot4(b, SLOT4_NMU + j)];
            const float y0 = P[0] * d[0];
            const float y1 = fmaf(P[2], d[1], P[1] * d[0]);
            const float y2 = fmaf(P[5], d[2], fmaf(P[4], d[1], P[3] * d[0]));
            const float y3 = fmaf(P[9], d[3], fmaf(P[8], d[2], fmaf(P[7], d[1], P[6] * d[0])));
            const float cc = cmax - params[slot4(b, SLOT4_C)];
            return fmaf(y3, y3, fmaf(y2, y2, fmaf(y1, y1, fmaf(y0, y0, cc))));
        };
        float mx = -INFINITY;
        for (int b = lane; b < k; b += 32) mx = fmaxf(mx, -nlog(b));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
        float sum = 0.f;
        if (mx > -INFINITY)
            for (int b = lane; b < k; b += 32) sum += ex2_approx(-nlog(b) - mx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
        if (lane == 0) {
            if (!(mx > -INFINITY) || !(sum > 0.f)) {
                set_error(st, GIRA_ERR_NUMERIC);
                pref[i] = make_float2(0.f, 0.f);
            } else {
                pref[i] = make_float2(-mx, __frcp_rn(sum));
                llpt[i] = (double)(lg2_approx(sum) + mx + ref0) * LN2_4;
            }
        }
    }
}

// ------------------------------------------------------------------ k-means in four dimensions
// labels = argmin_b ||x - c_b||^2 (binary32 in the order of dist2_f32_4, ties to
// the lowest b); binary64 sums of the coordinates and counts per label;
// changed[it] counts labels that moved (all of them for it == 0).
constexpr int LL4_THREADS = 256;

__global__ void __launch_bounds__(LL4_THREADS) lloyd4_assign_kernel(const float4* __restrict__ pts, int64_t n, int k,
                                                                    const float4* __restrict__ centers,
                                                                    int32_t* labels, double* sums,
                                                                    unsigned long long* changed, int it,
                                                                    DeviceState* st) {
    extern __shared__ float4 sc4[];
    if (st->error) return;
    if (it > 0 && changed[it - 1] == 0) return;
    for (int b = threadIdx.x; b < k; b += blockDim.x) sc4[b] = centers[b];
    __syncthreads();
    unsigned long long cnt = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 x = pts[i];
        int best = 0;
        float bd = dist2_f32_4(x, sc4[0]);
        for (int b = 1; b < k; ++b) {
            const float d = dist2_f32_4(x, sc4[b]);
            if (d < bd) {
                bd = d;
                best = b;
            }
        }
        if (it == 0 || labels[i] != best) ++cnt;
        labels[i] = best;
        double* S = sums + 5 * (size_t)best;
        atomicAdd(&S[0], (double)x.x);
        atomicAdd(&S[1], (double)x.y);
        atomicAdd(&S[2], (double)x.z);
        atomicAdd(&S[3], (double)x.w);
        atomicAdd(&S[4], 1.0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&changed[it], cnt);
}

__global__ void lloyd4_update_kernel(int k, double* sums, float4* centers, const unsigned long long* changed, int it,
                                     DeviceState* st) {
    if (st->error || changed[it - 1] == 0) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < k) {
        double* S = sums + 5 * (size_t)b;
        const double cnt = S[4];
        if (cnt > 0.0)
            centers[b] = make_float4((float)(S[0] / cnt), (float)(S[1] / cnt), (float)(S[2] / cnt), (float)(S[3] / cnt));
        for (int i = 0; i < 5; ++i) S[i] = 0.0;
    }
    if (b == 0) st->lloyd_done = it;
}

// One-hot statistics about the final centres: S0 = count, S1 = sum (x - s),
// S2 = sum (x - s)(x - s)^T, binary64.
// Each thread takes LS4_PPT consecutive points and sums each run of equal labels
// in registers (binary64) before its atomics, as in 3D.
constexpr int LS4_PPT = 8;

__global__ void label_stats4_kernel(const float4* __restrict__ pts, int64_t n, const int32_t* __restrict__ labels,
                                    const float4* __restrict__ shift4, double* stats64, DeviceState* st) {
    if (st->error) return;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * LS4_PPT;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * LS4_PPT; i0 < n; i0 += step) {
        int key = -1;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        double a[NSTAT4];
#pragma unroll
        for (int t = 0; t < NSTAT4; ++t) a[t] = 0.0;
        for (int r = 0; r < LS4_PPT; ++r) {
            const int64_t i = i0 + r;
            if (i >= n) break;
            const int b = labels[i];
            if (b != key) {
                if (key >= 0) {
                    double* S = stats64 + (size_t)key * NSTAT4;
#pragma unroll
                    for (int t = 0; t < NSTAT4; ++t) atomicAdd(&S[t], a[t]);
                }
#pragma unroll
                for (int t = 0; t < NSTAT4; ++t) a[t] = 0.0;
                key = b;
                s = shift4[b];
            }
            const float4 x = pts[i];
            const double d[4] = {(double)x.x - (double)s.x, (double)x.y - (double)s.y, (double)x.z - (double)s.z,
                                 (double)x.w - (double)s.w};
            a[0] += 1.0;
#pragma unroll
            for (int t = 0; t < 4; ++t) a[1 + t] += d[t];
#pragma unroll
            for (int i2 = 0; i2 < 4; ++i2)
#pragma unroll
                for (int j = i2; j < 4; ++j) a[5 + sym4(i2, j)] += d[i2] * d[j];
        }
        if (key >= 0) {
            double* S = stats64 + (size_t)key * NSTAT4;
#pragma unroll
            for (int t = 0; t < NSTAT4; ++t) atomicAdd(&S[t], a[t]);
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
static int num_sms_now() {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

cudaError_t launch_lloyd4(const float4* pts4, int64_t n, int k, int lloyd_iters, float4* centers, int32_t* labels,
                          double* sums, unsigned long long* changed, DeviceState* st, cudaStream_t s) {
    const size_t smem = sizeof(float4) * (size_t)k;
    const int64_t want = (n + LL4_THREADS - 1) / LL4_THREADS;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms_now() * 8));
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(lloyd4_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    lloyd4_assign_kernel<<<grid, LL4_THREADS, smem, s>>>(pts4, n, k, centers, labels, sums, changed, 0, st);
    for (int it = 1; it <= lloyd_iters; ++it) {
        lloyd4_update_kernel<<<(k + 127) / 128, 128, 0, s>>>(k, sums, centers, changed, it, st);
        lloyd4_assign_kernel<<<grid, LL4_THREADS, smem, s>>>(pts4, n, k, centers, labels, sums, changed, it, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_label_stats4(const float4* pts4, int64_t n, int k, const int32_t* labels, const float4* shift4,
                                double* stats64, DeviceState* st, cudaStream_t s) {
    (void)k;
    const int64_t want = (n + 256 * LS4_PPT - 1) / (256 * LS4_PPT);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms_now() * 8));
    label_stats4_kernel<<<grid, 256, 0, s>>>(pts4, n, labels, shift4, stats64, st);
    return cudaGetLastError();
}

int estep4_threads(int k) { return 32 * ((k + 63) / 64); }

// CTAs per SM of the statistics kernel for k components and ppc staged points.
static int estep4_occupancy(int k, int64_t ppc) {
    int occ = 0;
    const int smem = (int)(ppc * 32);
    cudaFuncSetAttribute(estep4_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, PPC4_MAX * 32);
    cudaFuncSetAttribute(estep4_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, PPC4_MAX * 32);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, estep4_kernel<true>, estep4_threads(k), smem) !=
            cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    return occ;
}

// One wave of CTAs (SMs x resident CTAs) over the points, at most PPC4_MAX
// points each (more waves beyond that).
int estep4_grid(int64_t n, int k, int num_sms, int64_t* ppc) {
    auto plan = [&](int occ) {
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((n + Q4 - 1) / Q4, (int64_t)num_sms * occ));
        return std::min<int64_t>(((n + grid - 1) / grid + Q4 - 1) / Q4 * Q4, PPC4_MAX);
    };
    int64_t p = plan(estep4_occupancy(k, 1024));
    if (p > 1024) p = plan(estep4_occupancy(k, p));
    *ppc = p;
    return (int)((n + p - 1) / p);
}

cudaError_t launch_estep4(const EStep4Launch& a, bool stats, int grid, cudaStream_t s, bool pdl) {
    const size_t smem = (size_t)a.pts_per_cta * 32;
    const void* fn = stats ? (const void*)estep4_kernel<true> : (const void*)estep4_kernel<false>;
    note_estep_kernel(fn);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    PdlConfig c(dim3(grid), dim3(estep4_threads(a.k)), smem, s, pdl);
    return cudaLaunchKernelExC(&c.cfg, fn, args);
}

cudaError_t launch_reduce_finalize4(const float* partials, int grid, int kc, const double* ll_partials,
                                    int ll_count, const double* stats64, const float4* shift4, int k, int64_t n,
                                    double reg, double tol, double* model64, float* params, double* trace,
                                    DeviceState* st, int iter, bool em, cudaStream_t s, bool pdl) {
    PdlConfig c(dim3(k), dim3(NSTAT4 * 32), 0, s, pdl);
    return cudaLaunchKernelEx(&c.cfg, reduce_finalize4_kernel, partials, grid, kc, ll_partials, ll_count, stats64,
                              shift4, k, n, reg, tol, model64, params, trace, st, iter, em ? 1 : 0);
}

cudaError_t launch_chunk_ref4(const float* params, int k, const DeviceState* st, float* gref, cudaStream_t s) {
    chunk_ref4_kernel<<<1, 256, 0, s>>>(params, k, st, gref);
    return cudaGetLastError();
}

cudaError_t launch_estep4_chunks(const EStep4Launch& a, int pass, int grid, cudaStream_t s) {
    const size_t smem = (size_t)a.pts_per_cta * 32;
    const void* fn = (pass == 1) ? (const void*)estep4_kernel<false, 1> : (const void*)estep4_kernel<true, 2>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int chunks = (a.k + CHUNK4 - 1) / CHUNK4;
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3(grid, chunks), dim3(CHUNK4 / 2), args, smem, s);
}

cudaError_t launch_chunk_exact4(const float4* pts8, const float* params, int k, const float* gref, const int* flags,
                                const int* flag_count, float2* pref, double* llpt, DeviceState* st, cudaStream_t s) {
    chunk_exact4_kernel<<<152, 256, 0, s>>>(pts8, params, k, gref, flags, flag_count, pref, llpt, st);
    return cudaGetLastError();
}

cudaError_t launch_params_from_model4(const float* w, const float* mu, const float* cov, int k, double* model64,
                                      float* params, DeviceState* st, cudaStream_t s) {
    params_from_model4_kernel<<<(k + 63) / 64, 64, 0, s>>>(w, mu, cov, k, model64, params, st);
    return cudaGetLastError();
}

cudaError_t launch_model_out4(const double* model64, int k, float* w, float* mu, float* cov, const DeviceState* st,
                              cudaStream_t s) {
    model_out4_kernel<<<1, 64, 0, s>>>(model64, k, w, mu, cov, st);
    return cudaGetLastError();
}

int params4_pairs(int k) {
    return k > MAX_K4_DIRECT ? ((k + CHUNK4 - 1) / CHUNK4) * (CHUNK4 / 2) : estep4_threads(k);
}

cudaError_t launch_fill_padding4(float* params, int k, cudaStream_t s) {
    const int kpad = 2 * params4_pairs(k);
    if (kpad > k) fill_padding4_kernel<<<(kpad - k + 63) / 64, 64, 0, s>>>(params, k, kpad);
    return cudaGetLastError();
}

cudaError_t launch_pack4(const float* pts4in, int64_t n, float4* pts4, float4* pts8, DeviceState* st,
                         cudaStream_t s) {
    pack4_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts4in, n, pts4, pts8, st);
    return cudaGetLastError();
}

int cond_floats() { return COND_FLOATS; }

cudaError_t launch_conditional4(const float* locs, int64_t m, int k, const float* w, const float* mu,
                                const float* cov, float* prep, float* cmean, float* cvar, DeviceState* st,
                                cudaStream_t s) {
    cond_prepare_kernel<<<(k + 63) / 64, 64, 0, s>>>(w, mu, cov, k, prep, st);
    conditional4_kernel<<<(unsigned)((m + COND_THREADS - 1) / COND_THREADS), COND_THREADS, 0, s>>>(locs, m, k, prep,
                                                                                                 cmean, cvar, st);
    return cudaGetLastError();
}

cudaError_t launch_sample(int64_t m, int k, int d, const float* w, const float* mu, const float* cov, uint64_t seed,
                          double* cum, double* chol, float* out, int32_t* comp, DeviceState* st, cudaStream_t s) {
    sample_prepare_kernel<<<1, 256, 0, s>>>(w, mu, cov, k, d, cum, chol, st);
    sample_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(m, k, d, mu, cum, chol, seed, out, comp, st);
    return cudaGetLastError();
}

}  // namespace gira
