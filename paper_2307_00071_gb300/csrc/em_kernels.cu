// em_kernels.cu -- fused E-step / M-step statistics, reduction and FP64 finalize.
//
// GIRA (arXiv 2307.00071) Sec. V: the E-step of Eq. (estep) is evaluated in the
// log domain (Eq. logestep) with the Cholesky form of the log-density
// (Eq. simplifiedGaussian); the M-step (standard full-covariance update, not
// written in the paper) is fed by per-component sufficient statistics.
//
// Mapping (component-stationary): one CTA holds ALL K components, spread over
// its G warps; lane (warp w, lane l) owns NP component pairs in registers, and
// warp w the contiguous block of pairs [w NP 32, (w + 1) NP 32).  All lanes walk
// the CTA's contiguous range of points together, Q_BATCH points at a time.
// Pass 1 computes e_nb = 2^(l_nb - cmax) for the lane's components (kept in
// registers), the per-point sums are combined across lanes (shuffle
// transpose-reduce) and warps (shared memory), and pass 2 accumulates the
// per-component statistics S0 = sum r, S1 = sum r d, S2 = sum r d d^T with
// d = x - mu_old (binary32, per-CTA partials).  Pass 1 processes component
// pairs with packed FP32 (FFMA2/FADD2); pass 2 uses scalar FP32.  The
// responsibility matrix is never stored.
//
// Pass 2 skips a (point, pair of lanes' components) wherever e is exactly 0
// for every lane of the warp (ex2.approx.ftz returns +0 below 2^-126, and a
// zero responsibility adds exactly nothing to any accumulator, so the skip
// changes no bit).  The fit orders the components along a space-filling curve
// of their means (order_components_kernel), so a warp's 128 components are
// close together and most of them are out of reach of any given point.
#include <cxxabi.h>
#include <float.h>
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <string>

#include "gira_internal.cuh"

namespace gira {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float LN2F = 0.693147180559945309f;
constexpr double LN2 = 0.693147180559945309417232121458;

// Log-density in base 2 for a component pair and one point (pairs packed).
struct PairParams {
    float2 p[6], c, nmu[3], w;
};

// P.c holds (cmax - c) >= 0: q' = |y|^2 + (cmax - c), y = P'(x - mu), and the
// logit relative to cmax is -q'.  The difference x - mu is taken first: it is
// exact or nearly so for the points a component reaches, so y carries only a
// few roundings relative to itself.  (The expanded form P'x + b' with
// b' = -P'mu would cancel two numbers of size |P'||x| -- a point metres from
// the origin against a millimetre-thin component: ~10^3 -- and carry the
// binary32 rounding of b' into every y; measured on the frame, one EM
// iteration in that form moves weights and covariances 10-20 times further from
// the binary64 result than this one.)
__device__ __forceinline__ float2 neg_logit2(const PairParams& P, float2 X0, float2 X1, float2 X2) {
    const float2 d0 = add2(X0, P.nmu[0]), d1 = add2(X1, P.nmu[1]), d2 = add2(X2, P.nmu[2]);
    const float2 y0 = mul2(P.p[0], d0);
    const float2 y1 = fma2(P.p[2], d1, mul2(P.p[1], d0));
    const float2 y2 = fma2(P.p[5], d2, fma2(P.p[4], d1, mul2(P.p[3], d0)));
    return fma2(y2, y2, fma2(y1, y1, fma2(y0, y0, P.c)));
}

// The same, also returning the whitened coordinates y = P'(x - mu) it formed
// (the same operations, so the same bits).
__device__ __forceinline__ float2 neg_logit2_y(const PairParams& P, float2 X0, float2 X1, float2 X2, float2& y0,
                                               float2& y1, float2& y2) {
    const float2 d0 = add2(X0, P.nmu[0]), d1 = add2(X1, P.nmu[1]), d2 = add2(X2, P.nmu[2]);
    y0 = mul2(P.p[0], d0);
    y1 = fma2(P.p[2], d1, mul2(P.p[1], d0));
    y2 = fma2(P.p[5], d2, fma2(P.p[4], d1, mul2(P.p[3], d0)));
    return fma2(y2, y2, fma2(y1, y1, fma2(y0, y0, P.c)));
}

constexpr long long MBAR_POLL_LIMIT = 2000000000ll;   // bound on any mbarrier wait: 2 s of wall time
constexpr int PPC_MAX = 2048;                         // points staged per CTA (64 KB)

// Fused E-step (+ statistics when STATS).  Component-stationary: one CTA holds
// all K components, G warps x 32 lanes x NP packed pairs.  The CTA's points
// arrive in one TMA bulk copy, laid out (x,x,y,y)(z,z,0,0) per point.  Per batch
// of Q points: pass 1 (logits, e, warp-level sums), one CTA barrier, the
// cross-warp total and 1/total, pass 2 (statistics).  The per-point sums are
// double-buffered by batch parity, so one barrier per batch suffices: a warp
// can only overwrite a buffer after the next barrier, which every warp reaches
// after reading it.
//
// GRAD (the adjoint of the log-likelihood, with STATS): pass 2 also forms each
// point's sum over components of gamma * Sigma_b^{-1} (x' - mu_b) (as
// P'^T P' d, in the base-2 scaling of P'), reduced across lanes and warps (a
// second barrier per batch) into dL/dx' = -(2 ln 2) * that sum; the owner lanes
// write dL/dx = R^T dL/dx' and accumulate the pose sums (dL/dx' x'^T, dL/dx').
// The statistics S0, S1, S2 give the parameter gradients (finalize).
//
// CH (K in chunks, each CTA one chunk of one tile; reference cmax over all K):
// CH = 1 (pass A): pass 1 and the per-point sums of the chunk into psum, no
// log-sum-exp; CH = 2 (pass B): e = 2^(shift_n - q') with (shift_n, 1 / total_n)
// from pref, pass 2 only -- no cross-lane reduction and no barrier per batch.
template <int NP, int Q, int MAXT, int MINB, bool STATS, bool GRAD = false, int CH = 0>
__global__ void __launch_bounds__(MAXT, MINB) estep_kernel(const EStepLaunch a_in) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar_tma;
    __shared__ float red_sum[2][32][Q];
    __shared__ float red_g[GRAD ? 2 : 1][GRAD ? 32 : 1][Q][3];
    __shared__ float red_aux[2][32][Q];
    __shared__ float s_cmax[32], s_wsum[32];
    __shared__ int s_skip, s_norm, s_dead;
    constexpr int LPQ = 32 / Q;   // lanes per batch index after the transpose-reduce

    // batched launches: this CTA's instance and CTA index within it
    int cta = blockIdx.x;
    EStepLaunch a = a_in;
    if (a_in.units) {
        const BatchUnit u = a_in.units[blockIdx.x];
        const BatchInst I = a_in.insts[u.inst];
        cta = u.cta;
        a.pts8 = a_in.pts8 + 2 * I.pt_off;
        a.n = I.n;
        a.k = I.k;
        a.params = a_in.params + I.par_off;
        a.pts_per_cta = I.ppc;
        a.partials = a_in.partials ? a_in.partials + I.part_off : nullptr;
        a.ll_partials = a_in.ll_partials + I.ll_off;
        a.per_point = a_in.per_point ? a_in.per_point + I.pt_off : nullptr;
        a.st = a_in.states + u.inst;
        if (CH != 0) {   // chunks share the points and the state; pass A's sums of this chunk
            a.st = a_in.states;
            if (a_in.psum) a.psum = a_in.psum + (size_t)u.inst * I.n;
        }
        if (GRAD) {   // per-instance scan gradient rows, pose and pose sums
            a.grad_pts = a_in.grad_pts ? a_in.grad_pts + 3 * I.pt_off : nullptr;
            a.rot = a_in.rot ? a_in.rot + 12 * (size_t)u.inst : nullptr;
            a.pose_partials = a_in.pose_partials + 12 * I.ll_off;
        }
    }
    const int G = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t begin = (int64_t)cta * a.pts_per_cta;
    const int64_t end = min(a.n, begin + a.pts_per_cta);
    const int npts = (int)(end - begin);
    const int nb = (npts + Q - 1) / Q;
    const float4* spts = reinterpret_cast<const float4*>(dsm);
    if (threadIdx.x == 0) {
        // the points are never written by the kernel this one may overlap
        // (dependent launch), so their copy starts before the wait below
        mbar_init(&bar_tma, 1);
        mbar_fence_init();
        mbar_expect_tx(&bar_tma, (uint32_t)npts * 32u);
        tma_load_1d(reinterpret_cast<void*>(dsm), a.pts8 + 2 * begin, (uint32_t)npts * 32u, &bar_tma);
    }
    pdl_wait();   // the parameters and the state written by the previous kernel
    if (threadIdx.x == 0) {
        s_skip = (a.iter > a.st->stop_after) || (a.st->error != 0);
        s_norm = a.st->w_raw;
        s_dead = 0;
    }
    __syncthreads();
    if (s_skip) {   // let the copy land before leaving
        if (threadIdx.x == 0) mbar_wait_bounded(&bar_tma, 0u, MBAR_POLL_LIMIT);
        return;
    }
    pdl_allow_next();

    // ---- this lane's component pairs -> registers (overlaps the TMA)
    PairParams prm[NP];
    float cm = -INFINITY, ws = 0.f;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int pp = (warp * NP + j) * 32 + lane;
        const float4* src = reinterpret_cast<const float4*>(a.params + (size_t)pp * PAIR_FLOATS);
        const float4 v0 = src[0], v1 = src[1], v2 = src[2], v4 = src[4], v5 = src[5], v6 = src[6];
        prm[j].p[0] = f2(v0.x, v0.y); prm[j].p[1] = f2(v0.z, v0.w);
        prm[j].p[2] = f2(v1.x, v1.y); prm[j].p[3] = f2(v1.z, v1.w);
        prm[j].p[4] = f2(v2.x, v2.y); prm[j].p[5] = f2(v2.z, v2.w);
        prm[j].c = f2(v4.z, v4.w);
        prm[j].nmu[0] = f2(v5.x, v5.y); prm[j].nmu[1] = f2(v5.z, v5.w);
        prm[j].nmu[2] = f2(v6.x, v6.y);
        cm = fmaxf(cm, fmaxf(prm[j].c.x, prm[j].c.y));
        ws += v6.z + v6.w;
    }
    // reference cmax = max_b c_b >= every logit (every e <= 1); after an M-step
    // also the weight normaliser sum_a N_a (shifts the log-likelihood only)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cm = fmaxf(cm, __shfl_xor_sync(FULL, cm, o));
        ws += __shfl_xor_sync(FULL, ws, o);
    }
    if (lane == 0) {
        s_cmax[warp] = cm;
        s_wsum[warp] = ws;
    }
    if (!mbar_wait_bounded(&bar_tma, 0u, MBAR_POLL_LIMIT)) s_dead = 1;
    __syncthreads();
    if (s_dead) {   // the points never arrived: report, let the copy land, leave
        if (threadIdx.x == 0) {
            set_error(a.st, GIRA_ERR_TIMEOUT);
            mbar_wait_bounded(&bar_tma, 0u, MBAR_POLL_LIMIT);
        }
        return;
    }
    float cmax = s_cmax[0], wsum = s_wsum[0];
    for (int w = 1; w < G; ++w) {
        cmax = fmaxf(cmax, s_cmax[w]);
        wsum += s_wsum[w];
    }
    float ref0 = s_norm ? cmax - __log2f(wsum) : cmax;
    if (CH != 0) {   // one reference for every chunk
        cmax = a.gref[0];
        ref0 = a.gref[1];
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) prm[j].c = f2(cmax - prm[j].c.x, cmax - prm[j].c.y);

    float Sx[NP][NSTAT], Sy[NP][NSTAT];   // statistics of components 2p and 2p+1
    if (STATS) {
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int s = 0; s < NSTAT; ++s) Sx[j][s] = Sy[j][s] = 0.f;
    }
    double ll_acc = 0.0;
    const int myq = q_of_lane<Q>(lane);
    const bool owner = (warp == 0) && ((lane & (LPQ - 1)) == 0);

    auto load_pt = [&](int li, float2& X0, float2& X1, float2& X2) {
        const float4 xy = spts[2 * li], zz = spts[2 * li + 1];
        X0 = f2(xy.x, xy.y);
        X1 = f2(xy.z, xy.w);
        X2 = f2(zz.x, zz.y);
    };
    // pass B: (shift, 1 / total) of the batch's points
    float2 pr[Q];
    // pass 1 of batch t: e for every (point, own component) into E, warp-level sums into red_sum[t & 1]
    auto pass1 = [&](int t, float2 (&E)[NP][Q]) {
        const int lb = t * Q, nvalid = min(Q, npts - lb);
        float part[Q];
        if (CH == 2) {
#pragma unroll
            for (int q = 0; q < Q; ++q) pr[q] = (q < nvalid) ? a.pref[begin + lb + q] : f2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float2 X0, X1, X2;
            load_pt((q < nvalid) ? lb + q : lb, X0, X1, X2);
            float2 acc = f2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const float2 nq = neg_logit2(prm[j], X0, X1, X2);
                const float sh = (CH == 2) ? pr[q].x : 0.f;
                const float2 e = f2(ex2_approx(sh - nq.x), ex2_approx(sh - nq.y));
                E[j][q] = e;
                acc = add2(acc, e);
            }
            part[q] = acc.x + acc.y;
        }
        if (CH != 2) {
            const float wt = warp_transpose_reduce<Q>(part, lane, AddOp());
            if ((lane & (LPQ - 1)) == 0) red_sum[t & 1][warp][myq] = wt;
        }
    };
    // statistics of batch t from E and the reciprocal sums r (owned by lane q * LPQ)
    auto pass2 = [&](int t, const float2 (&E)[NP][Q], float r) {
        const int lb = t * Q, nvalid = min(Q, npts - lb);
        float gq[Q][3];   // GRAD: this lane's share of sum_b gamma P'^T P' d, per point
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (GRAD) gq[q][0] = gq[q][1] = gq[q][2] = 0.f;
            // pairs with a nonzero e for this point on some lane of the warp (warp-uniform)
            bool live[NP], any = false;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                live[j] = __any_sync(FULL, (E[j][q].x != 0.f) || (E[j][q].y != 0.f));
                any = any || live[j];
            }
            if (!any) continue;
            float2 X0, X1, X2;
            load_pt((q < nvalid) ? lb + q : lb, X0, X1, X2);
            const float R = (CH == 2) ? pr[q].y : __shfl_sync(FULL, r, q * LPQ);
            // scalar FP32: measured faster than the packed form for this
            // accumulate-heavy pattern
            auto acc1 = [&](float e, float m0, float m1, float m2, float (&T)[NSTAT], const float2 (&pp)[6], int h) {
                const float g = e * R;
                float d0 = X0.x + m0, d1 = X1.x + m1, d2 = X2.x + m2;
                if (!GRAD) {   // the fit's statistics: whitened coordinates y = P'd, as the tile kernel
                    const float p0 = h ? pp[0].y : pp[0].x, p1 = h ? pp[1].y : pp[1].x, p2 = h ? pp[2].y : pp[2].x;
                    const float p3 = h ? pp[3].y : pp[3].x, p4 = h ? pp[4].y : pp[4].x, p5 = h ? pp[5].y : pp[5].x;
                    const float y0 = p0 * d0, y1 = fmaf(p2, d1, p1 * d0), y2 = fmaf(p5, d2, fmaf(p4, d1, p3 * d0));
                    d0 = y0;
                    d1 = y1;
                    d2 = y2;
                }
                if (GRAD) {
                    const float p0 = h ? pp[0].y : pp[0].x, p1 = h ? pp[1].y : pp[1].x, p2 = h ? pp[2].y : pp[2].x;
                    const float p3 = h ? pp[3].y : pp[3].x, p4 = h ? pp[4].y : pp[4].x, p5 = h ? pp[5].y : pp[5].x;
                    const float y0 = p0 * d0, y1 = fmaf(p2, d1, p1 * d0), y2 = fmaf(p5, d2, fmaf(p4, d1, p3 * d0));
                    const float z0 = fmaf(p3, y2, fmaf(p1, y1, p0 * y0)), z1 = fmaf(p4, y2, p2 * y1), z2 = p5 * y2;
                    gq[q][0] = fmaf(g, z0, gq[q][0]);
                    gq[q][1] = fmaf(g, z1, gq[q][1]);
                    gq[q][2] = fmaf(g, z2, gq[q][2]);
                }
                const float g0 = g * d0, g1 = g * d1, g2 = g * d2;
                T[0] += g;
                T[1] += g0;
                T[2] += g1;
                T[3] += g2;
                T[4] = fmaf(g0, d0, T[4]);
                T[5] = fmaf(g0, d1, T[5]);
                T[6] = fmaf(g0, d2, T[6]);
                T[7] = fmaf(g1, d1, T[7]);
                T[8] = fmaf(g1, d2, T[8]);
                T[9] = fmaf(g2, d2, T[9]);
            };
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                if (!live[j]) continue;
                acc1(E[j][q].x, prm[j].nmu[0].x, prm[j].nmu[1].x, prm[j].nmu[2].x, Sx[j], prm[j].p, 0);
                acc1(E[j][q].y, prm[j].nmu[0].y, prm[j].nmu[1].y, prm[j].nmu[2].y, Sy[j], prm[j].p, 1);
            }
        }
        if (GRAD) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float v[Q];
#pragma unroll
                for (int q = 0; q < Q; ++q) v[q] = gq[q][c];
                const float w = warp_transpose_reduce<Q>(v, lane, AddOp());
                if ((lane & (LPQ - 1)) == 0) red_g[t & 1][warp][myq][c] = w;
            }
        }
    };
    // batch t after its barrier: cross-warp total, rare exact-max path, 1/total
    auto finish = [&](int t, float2 (&E)[NP][Q]) -> float {
        const int lb = t * Q, nvalid = min(Q, npts - lb);
        float tot = red_sum[t & 1][0][myq];
        for (int w = 1; w < G; ++w) tot += red_sum[t & 1][w][myq];
        const bool myvalid = myq < nvalid;
        float ref = ref0;
        // Rare path: a point whose best component is > 100 binades below cmax.
        // Redo the batch with the exact per-point maximum (Eq. logestep's
        // max-subtraction) so that no responsibility is lost to underflow.
        if (__any_sync(FULL, myvalid && !(tot >= 0x1p-100f))) {
            float m[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                float2 X0, X1, X2;
                load_pt((q < nvalid) ? lb + q : lb, X0, X1, X2);
                float mm = -INFINITY;
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const float2 nq = neg_logit2(prm[j], X0, X1, X2);
                    const float2 l = f2(-nq.x, -nq.y);
                    E[j][q] = l;
                    mm = fmaxf(mm, fmaxf(l.x, l.y));
                }
                m[q] = mm;
            }
            float mt = warp_transpose_reduce<Q>(m, lane, MaxOp());
            if ((lane & (LPQ - 1)) == 0) red_aux[0][warp][myq] = mt;
            __syncthreads();
            mt = red_aux[0][0][myq];
            for (int w = 1; w < G; ++w) mt = fmaxf(mt, red_aux[0][w][myq]);
            float part[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                float mq = __shfl_sync(FULL, mt, q * LPQ);
                mq = (mq > -INFINITY) ? mq : 0.f;
                float2 acc = f2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const float2 e = f2(ex2_approx(E[j][q].x - mq), ex2_approx(E[j][q].y - mq));
                    E[j][q] = e;
                    acc = add2(acc, e);
                }
                part[q] = acc.x + acc.y;
            }
            const float wt = warp_transpose_reduce<Q>(part, lane, AddOp());
            if ((lane & (LPQ - 1)) == 0) red_aux[1][warp][myq] = wt;
            __syncthreads();
            tot = red_aux[1][0][myq];
            for (int w = 1; w < G; ++w) tot += red_aux[1][w][myq];
            if (myvalid && !(mt > -INFINITY)) set_error(a.st, GIRA_ERR_NUMERIC);
            ref = ref0 + ((mt > -INFINITY) ? mt : 0.f);
        }
        const bool ok = myvalid && tot > 0.f;
        const float lse2 = lg2_approx(tot) + ref;   // log2 sum_b pi_b N(x|b)
        if (owner && ok) {
            ll_acc += (double)lse2;
            if (!STATS && a.per_point) a.per_point[begin + lb + myq] = lse2 * LN2F;
        }
        return ok ? __frcp_rn(tot) : 0.f;
    };
    float2 E[NP][Q];
    float tw[12] = {};   // GRAD owner lanes: sum g x'^T (row-major), sum g
    for (int t = 0; t < nb; ++t) {
        if (CH == 2 && a.psum) {
            // pass B: a batch whose every point had an exactly zero sum over this
            // chunk in pass A (and takes the common reference, shift 0) has
            // e = 0 for every component of the chunk: nothing to accumulate
            const int lb = t * Q;
            bool live = false;
            if (lane < Q && lane < npts - lb) {
                const int64_t i = begin + lb + lane;
                live = (a.psum[i] != 0.f) || (a.pref[i].x != 0.f);
            }
            if (!__any_sync(FULL, live)) continue;
        }
        pass1(t, E);
        if (CH == 2) {
            pass2(t, E, 0.f);
            continue;
        }
        __syncthreads();   // every warp's sums of batch t are in red_sum[t & 1]
        if (CH == 1) {
            const int lb = t * Q;
            if (owner && myq < min(Q, npts - lb)) {
                float tot = red_sum[t & 1][0][myq];
                for (int w = 1; w < G; ++w) tot += red_sum[t & 1][w][myq];
                a.psum[begin + lb + myq] = tot;
            }
            continue;
        }
        const float r = finish(t, E);
        if (STATS) pass2(t, E, r);
        if (GRAD) {
            __syncthreads();   // every warp's gradient sums of batch t are in red_g[t & 1]
            const int lb = t * Q;
            if (owner && myq < min(Q, npts - lb)) {
                float g3[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float v = red_g[t & 1][0][myq][c];
                    for (int w = 1; w < G; ++w) v += red_g[t & 1][w][myq][c];
                    g3[c] = -1.38629436111989061883f * v;   // -(2 ln 2): P'^T P' = Sigma^{-1} log2(e) / 2
                }
                const float4 xy = spts[2 * (lb + myq)], zz = spts[2 * (lb + myq) + 1];
                const float x0 = xy.x, x1 = xy.z, x2 = zz.x;
                const float xq[3] = {x0, x1, x2};
#pragma unroll
                for (int i = 0; i < 3; ++i) {
#pragma unroll
                    for (int j = 0; j < 3; ++j) tw[3 * i + j] = fmaf(g3[i], xq[j], tw[3 * i + j]);
                    tw[9 + i] += g3[i];
                }
                if (a.grad_pts) {
                    float* gp = a.grad_pts + 3 * (begin + lb + myq);
                    if (a.rot) {
                        const float* Rm = a.rot;
                        gp[0] = fmaf(Rm[6], g3[2], fmaf(Rm[3], g3[1], Rm[0] * g3[0]));
                        gp[1] = fmaf(Rm[7], g3[2], fmaf(Rm[4], g3[1], Rm[1] * g3[0]));
                        gp[2] = fmaf(Rm[8], g3[2], fmaf(Rm[5], g3[1], Rm[2] * g3[0]));
                    } else {
                        gp[0] = g3[0];
                        gp[1] = g3[1];
                        gp[2] = g3[2];
                    }
                }
            }
        }
    }

    if (STATS) {
        float* dst = a.partials + (size_t)cta * a.k * NSTAT;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const int b0 = 2 * ((warp * NP + j) * 32 + lane);
            if (b0 < a.k)
#pragma unroll
                for (int s = 0; s < NSTAT; ++s) dst[(size_t)b0 * NSTAT + s] = Sx[j][s];
            if (b0 + 1 < a.k)
#pragma unroll
                for (int s = 0; s < NSTAT; ++s) dst[(size_t)(b0 + 1) * NSTAT + s] = Sy[j][s];
        }
    }
    if (warp == 0 && CH == 0) {   // owner lanes hold the per-point log-likelihood sums; fixed order
        double v = ll_acc;
#pragma unroll
        for (int o = LPQ; o < 32; o <<= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0) a.ll_partials[cta] = v * LN2;
        if (GRAD) {
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                double u = owner ? (double)tw[i] : 0.0;
#pragma unroll
                for (int o = LPQ; o < 32; o <<= 1) u += __shfl_xor_sync(FULL, u, o);
                if (lane == 0) a.pose_partials[(size_t)cta * 12 + i] = u;
            }
        }
    }
}

// ------------------------------------------------------------------ point-stationary E-step
// The E-step with the roles of the operands the other way round: each lane owns
// PT_P points in registers (a warp: 32 PT_P consecutive points), and every pair
// of components is read from shared memory as a broadcast (the CTA's copy of
// the parameters, staged once by one TMA bulk copy).  Per-point sums stay in
// their lane: no cross-lane or cross-warp reduction, no barrier.
//  phase 1  for every pair: both logits at the lane's points, e = 2^-q', the
//           per-point totals; one warp vote records whether the pair reaches any
//           point of the warp (some e nonzero: ex2.approx.ftz gives exact zeros);
//  totals   1 / total per point and the log-likelihood; a point whose total
//           falls below 2^-100 takes the exact per-point maximum (Eq. logestep's
//           max-subtraction) and makes every pair live for its warp;
//  phase 2  for the live pairs only: e again (the same instructions, so the same
//           bits), the statistics of both components over the warp's points in
//           whitened coordinates y = P'(x - mu_old) -- S0 = sum r, S1 = sum r y,
//           S2 = sum r y y^T -- reduced over the warp's lanes and written to the
//           warp's partials; the warp's live mask tells the finalize which ones.
// With the components in space-filling-curve order a warp's 128 neighbouring
// points reach about a sixth of the pairs (the depth frame at K = 512), and the
// other pairs cost only phase 1.  The statistics are sums of the same terms as
// the other kernels' in another order.
// Relative costs of a listed pair (phase 1) and a live pair (phase 2) per point,
// and the 8-bit logarithmic key of a CTA's work (16 steps per octave) by which
// the finalize orders the CTAs of a later iteration.
constexpr unsigned PT_COST_NEAR = 26, PT_COST_LIVE = 54;
__device__ __forceinline__ uint8_t work_key(unsigned w) {
    const int e = 31 - __clz(w | 1u);
    const unsigned m = (e >= 4 ? (w >> (e - 4)) : (w << (4 - e))) & 15u;
    return (uint8_t)min(255u, (unsigned)e * 16u + m);
}
constexpr int PT_P = 4;           // points per lane
constexpr int PT_W = 4;           // warps per CTA
constexpr int PT_H = 2;           // warps sharing a block of 32 * PT_P points (the pairs split between them)
constexpr int PT_B = PT_W / PT_H; // point blocks per CTA: partial rows and mask rows per CTA
constexpr int PT_PTS = 32 * PT_P * PT_B;   // points per CTA

// Pairs the kernel reads for k components: ceil(k / 2) rounded up to a multiple
// of 32 (never beyond the padded parameter block, whose extra slots are padding
// components with c = -inf).
__host__ __device__ constexpr int pt_pairs(int k) { return (((k + 1) / 2) + 31) & ~31; }
// floats of one partial row: [pairs][2 NSTAT], a pair's values 80 contiguous bytes
__host__ __device__ constexpr int pt_row_floats(int k) { return ((k + 1) / 2) * 2 * NSTAT; }
constexpr float PT_REACH = 128.f;  // q' above which a component is out of reach (e = 0 from q' > 126)
// parameters, then per warp the live-mask words and the list of reachable pairs
__host__ __device__ constexpr size_t pt_smem_bytes(int k) {
    return (size_t)pt_pairs(k) * PAIR_FLOATS * 4 + (size_t)PT_W * (pt_pairs(k) / 32) * 4 +
           (size_t)PT_W * pt_pairs(k) * 2;
}

// Sum of 20 values (10 float2: component 2p in .x, 2p+1 in .y) over the warp's
// lanes.  On return lane l with (l & 7) < 5 holds value 10 (l >> 4) + 5 ((l >> 3) & 1) + (l & 7):
// halving exchanges for the first two levels, butterflies for the last three.
__device__ __forceinline__ float pt_warp_reduce20(const float2 (&S)[NSTAT], int lane, int* vidx) {
    const bool b4 = lane & 16, b3 = lane & 8;
    float w[NSTAT];
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) {
        const float keep = b4 ? S[i].y : S[i].x, send = b4 ? S[i].x : S[i].y;
        w[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
    float z[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float keep = b3 ? w[5 + i] : w[i], send = b3 ? w[i] : w[5 + i];
        z[i] = keep + __shfl_xor_sync(FULL, send, 8);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 5; ++i) z[i] += __shfl_xor_sync(FULL, z[i], o);
    const int i = lane & 7;
    *vidx = 10 * (b4 ? 1 : 0) + 5 * (b3 ? 1 : 0) + i;
    return i == 0 ? z[0] : i == 1 ? z[1] : i == 2 ? z[2] : i == 3 ? z[3] : z[4];
}

// The barrier of point block blk's PT_H warps (barrier ids known at compile time,
// so the kernel holds PT_B + 1 of them).
__device__ __forceinline__ void pt_block_sync(int blk) {
    static_assert(PT_B == 2 && PT_H == 2, "one named barrier per point block");
    if (blk == 0) asm volatile("bar.sync 1, %0;" ::"n"(32 * PT_H) : "memory");
    else asm volatile("bar.sync 2, %0;" ::"n"(32 * PT_H) : "memory");
}

template <bool STATS>
__global__ void __launch_bounds__(32 * PT_W, 4) estep_pt_kernel(const EStepLaunch a_in) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar_tma;
    __shared__ int s_skip, s_norm, s_dead;
    __shared__ double s_ll[PT_W];
    __shared__ unsigned s_pairs[PT_W][2];
    __shared__ float2 s_tot[PT_W][PT_P][32];   // phase-1 sums of every warp, for its partner
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int blk = warp / PT_H, half = warp % PT_H;   // point block; which pairs (pp % PT_H == half)
    int cta = blockIdx.x;
    // the instance's first point (batched launches); the loads below index the
    // launch's own pointer by it (loads through the pointer advanced in the local
    // copy of the launch struct read the unadvanced one under nvcc 13.0 for sm_103a)
    int64_t pt0 = 0;
    EStepLaunch a = a_in;
    if (a_in.units) {
        const BatchUnit u = a_in.units[blockIdx.x];
        const BatchInst I = a_in.insts[u.inst];
        cta = u.cta;
        pt0 = I.pt_off;
        a.n = I.n;
        a.k = I.k;
        a.params = a_in.params + I.par_off;
        a.partials = a_in.partials ? a_in.partials + I.part_off : nullptr;
        a.masks = a_in.masks ? a_in.masks + I.mask_off : nullptr;
        a.pt_rows = (int64_t)I.ctas * PT_B;
        a.ll_partials = a_in.ll_partials ? a_in.ll_partials + I.ll_off : nullptr;
        a.per_point = a_in.per_point ? a_in.per_point + I.pt_off : nullptr;
        a.st = a_in.states + u.inst;
    }
    if (a_in.cta_perm && a_in.iter >= 3) {   // the order the finalize chose two iterations ago
        const int c = a_in.cta_perm[(size_t)(a_in.iter & 1) * gridDim.x + blockIdx.x];
        if (GIRA_IN(c >= 0 && c < (int)gridDim.x, a.st)) cta = c;
    }
    // pairs evaluated: ceil(k / 2) rounded up to even (within the padded block, whose
    // extra slots are padding components with c = -inf); mask words for pt_pairs(k)
    const int npairs = ((((a.k + 1) >> 1) + 1) & ~1);
    const int nwords = pt_pairs(a.k) / 32;
    const float4* spar = reinterpret_cast<const float4*>(dsm);   // [npairs][PAIR_F4]
    uint32_t* smask_all = reinterpret_cast<uint32_t*>(dsm + (size_t)pt_pairs(a.k) * PAIR_FLOATS * 4);
    uint32_t* smask = smask_all + warp * nwords;   // [nwords] live bits of the warp's pairs
    uint16_t* slist = reinterpret_cast<uint16_t*>(smask_all + PT_W * nwords) + warp * pt_pairs(a.k);
    // the lane's points (never written inside a fit: loaded before the wait); a slot
    // beyond n holds a point 1e18 m away, where every q' is +inf and e exactly 0
    const int64_t base = (int64_t)cta * PT_PTS + (int64_t)blk * 32 * PT_P + lane;
    float2 X[PT_P][3];
    bool valid[PT_P];
#pragma unroll
    for (int p = 0; p < PT_P; ++p) {
        const int64_t i = base + 32 * p;
        valid[p] = i < a.n && GIRA_IN(a_in.n_buf == 0 || pt0 + i < a_in.n_buf, a.st);
        if (valid[p]) {
            const float4 xy = a_in.pts8[2 * (pt0 + i)], zz = a_in.pts8[2 * (pt0 + i) + 1];
            X[p][0] = f2(xy.x, xy.y);
            X[p][1] = f2(xy.z, xy.w);
            X[p][2] = f2(zz.x, zz.y);
        } else {
            X[p][0] = X[p][1] = X[p][2] = dup(1e18f);
        }
    }
    pdl_wait();   // the parameters and the state written by the previous kernel
    if (threadIdx.x == 0) {
        s_skip = (a.iter > a.st->stop_after) || (a.st->error != 0);
        s_norm = a.st->w_raw;
        s_dead = 0;
        if (!s_skip) {
            mbar_init(&bar_tma, 1);
            mbar_fence_init();
            const uint32_t bytes = (uint32_t)npairs * PAIR_FLOATS * 4u;
            mbar_expect_tx(&bar_tma, bytes);
            tma_load_1d(reinterpret_cast<void*>(dsm), a.params, bytes, &bar_tma);
            if (!mbar_wait_bounded(&bar_tma, 0u, MBAR_POLL_LIMIT)) {
                s_dead = 1;
                set_error(a.st, GIRA_ERR_TIMEOUT);
                mbar_wait_bounded(&bar_tma, 0u, MBAR_POLL_LIMIT);   // let the copy land
            }
        }
    }
    __syncthreads();
    if (s_skip || s_dead) return;
    pdl_allow_next();

    // reference cmax = max_b c_b and the weight normaliser (every warp, same order)
    float cm = -INFINITY, wsv = 0.f;
    for (int pp = lane; pp < npairs; pp += 32) {
        const float4 v4 = spar[pp * PAIR_F4 + 4], v6 = spar[pp * PAIR_F4 + 6];
        cm = fmaxf(cm, fmaxf(v4.z, v4.w));
        wsv += v6.z + v6.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cm = fmaxf(cm, __shfl_xor_sync(FULL, cm, o));
        wsv += __shfl_xor_sync(FULL, wsv, o);
    }
    const float cmax = cm;
    const float ref0 = s_norm ? cmax - __log2f(wsv) : cmax;

    auto load_pair = [&](int pp, PairParams& P) {
        if (!GIRA_IN(pp >= 0 && pp < npairs, a.st)) pp = 0;
        const float4* q = spar + (size_t)pp * PAIR_F4;
        const float4 v0 = q[0], v1 = q[1], v2 = q[2], v4 = q[4], v5 = q[5], v6 = q[6];
        P.p[0] = f2(v0.x, v0.y); P.p[1] = f2(v0.z, v0.w);
        P.p[2] = f2(v1.x, v1.y); P.p[3] = f2(v1.z, v1.w);
        P.p[4] = f2(v2.x, v2.y); P.p[5] = f2(v2.z, v2.w);
        P.c = f2(cmax - v4.z, cmax - v4.w);
        P.nmu[0] = f2(v5.x, v5.y); P.nmu[1] = f2(v5.z, v5.w);
        P.nmu[2] = f2(v6.x, v6.y);
    };

    // ---- phase 0: the pairs that can reach a point of the warp.  Over the box of
    // the warp's points, two lower bounds of q' = |P'(x - mu)|^2 + (cmax - c):
    //   |P'(x - mu)| >= |P'(ctr - mu)| - sum_j h_j |column j of P'|  (h: half-extents)
    //   |P'(x - mu)|^2 >= sigma_min(P')^2 dist(mu, box)^2
    // A component whose bound exceeds PT_REACH (with relative slack for the binary32
    // rounding of the bound and of q' itself) has q' > 126 at every point of the warp,
    // where ex2.approx.ftz gives exact zeros: skipping it leaves every sum unchanged.
    int nlive = 0;
    {
        float lo[3], hi[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            lo[j] = INFINITY;
            hi[j] = -INFINITY;
        }
#pragma unroll
        for (int p = 0; p < PT_P; ++p)
            if (valid[p])
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    lo[j] = fminf(lo[j], X[p][j].x);
                    hi[j] = fmaxf(hi[j], X[p][j].x);
                }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                lo[j] = fminf(lo[j], __shfl_xor_sync(FULL, lo[j], o));
                hi[j] = fmaxf(hi[j], __shfl_xor_sync(FULL, hi[j], o));
            }
        const bool any_point = lo[0] <= hi[0];
        float ctr[3], h[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            ctr[j] = 0.5f * (lo[j] + hi[j]);
            h[j] = fmaxf(hi[j] - ctr[j], ctr[j] - lo[j]);
        }
        for (int j0 = 0; j0 < npairs; j0 += 32 * PT_H) {   // this warp's pairs: pp % PT_H == half
            const int pp = j0 + PT_H * lane + half;
            bool live = false;
            if (any_point && pp < npairs) {
                const float4* q = spar + (size_t)pp * PAIR_F4;
                const float4 v0 = q[0], v1 = q[1], v2 = q[2], v4 = q[4], v5 = q[5], v6 = q[6], v7 = q[7];
                const float pc[2][6] = {{v0.x, v0.z, v1.x, v1.z, v2.x, v2.z}, {v0.y, v0.w, v1.y, v1.w, v2.y, v2.w}};
                const float nm[2][3] = {{v5.x, v5.z, v6.x}, {v5.y, v5.w, v6.y}};
                const float cc[2] = {v4.z, v4.w}, s2[2] = {v7.x, v7.y};
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const float room = PT_REACH - (cmax - cc[m]);   // q' budget left for |y|^2
                    const float* P = pc[m];
                    const float d0 = ctr[0] + nm[m][0], d1 = ctr[1] + nm[m][1], d2 = ctr[2] + nm[m][2];
                    const float y0 = P[0] * d0, y1 = fmaf(P[2], d1, P[1] * d0);
                    const float y2 = fmaf(P[5], d2, fmaf(P[4], d1, P[3] * d0));
                    const float yy = fmaf(y2, y2, fmaf(y1, y1, y0 * y0));
                    const float r = fmaf(h[0], sqrtf(fmaf(P[0], P[0], fmaf(P[1], P[1], P[3] * P[3]))),
                                         fmaf(h[1], sqrtf(fmaf(P[2], P[2], P[4] * P[4])), h[2] * fabsf(P[5])));
                    const float reach = (r + sqrtf(fmaxf(room, 0.f))) * (1.f + 1.f / 256.f);
                    const float e0 = fmaxf(fabsf(d0) - h[0], 0.f), e1 = fmaxf(fabsf(d1) - h[1], 0.f),
                                e2 = fmaxf(fabsf(d2) - h[2], 0.f);
                    const float iso = s2[m] * fmaf(e2, e2, fmaf(e1, e1, e0 * e0)) * (1.f - 1.f / 128.f);
                    live = live || (room > 0.f && yy <= reach * reach && iso <= room);
                }
            }
            const uint32_t m = __ballot_sync(FULL, live);
            const int at = nlive + __popc(m & ((1u << lane) - 1u));
            if (live && GIRA_IN(at < pt_pairs(a.k), a.st)) slist[at] = (uint16_t)pp;
            nlive += __popc(m);
        }
    }
    __syncwarp();

    // ---- phase 1: the reachable pairs, the lane's points (two pairs per step)
    if (STATS && lane < nwords) smask[lane] = 0u;
    __syncwarp();
    float2 tot[PT_P];
#pragma unroll
    for (int p = 0; p < PT_P; ++p) tot[p] = f2(0.f, 0.f);
    for (int i = 0; i < nlive; i += 2) {
        const int pa = slist[i], pb = (i + 1 < nlive) ? (int)slist[i + 1] : -1;
        PairParams P0, P1;
        load_pair(pa, P0);
        load_pair(pb < 0 ? pa : pb, P1);
        if (pb < 0) P1.c = dup(INFINITY);   // no second pair: q' = inf, e = 0
        uint32_t nz0 = 0u, nz1 = 0u;   // OR of the bits of e: nonzero iff some e is
#pragma unroll
        for (int p = 0; p < PT_P; ++p) {
            const float2 nq0 = neg_logit2(P0, X[p][0], X[p][1], X[p][2]);
            const float2 nq1 = neg_logit2(P1, X[p][0], X[p][1], X[p][2]);
            const float2 e0 = f2(ex2_approx(-nq0.x), ex2_approx(-nq0.y));
            const float2 e1 = f2(ex2_approx(-nq1.x), ex2_approx(-nq1.y));
            tot[p] = add2(tot[p], add2(e0, e1));
            if (STATS) {
                nz0 |= __float_as_uint(e0.x) | __float_as_uint(e0.y);
                nz1 |= __float_as_uint(e1.x) | __float_as_uint(e1.y);
            }
        }
        if (STATS) {
            const bool v0 = __ballot_sync(FULL, nz0 != 0u) != 0u, v1 = __ballot_sync(FULL, nz1 != 0u) != 0u;
            if (lane == 0) {
                if (v0) smask[pa >> 5] |= 1u << (pa & 31);
                if (v1) smask[pb >> 5] |= 1u << (pb & 31);   // v1 implies pb >= 0
            }
        }
    }
    __syncwarp();

    // ---- totals (the block's warps add their sums in the same order), log-likelihood,
    // rare points
#pragma unroll
    for (int p = 0; p < PT_P; ++p) s_tot[warp][p][lane] = tot[p];
    pt_block_sync(blk);
    float2 pr[PT_P];   // (shift, 1 / total) per point
    double ll = 0.0;
    bool rare_any = false;
#pragma unroll
    for (int p = 0; p < PT_P; ++p) {
        pr[p] = f2(0.f, 0.f);
        if (!valid[p]) continue;
        float t = 0.f;
#pragma unroll
        for (int h = 0; h < PT_H; ++h) {
            const float2 u = s_tot[blk * PT_H + h][p][lane];
            t += u.x + u.y;
        }
        float sh = 0.f;
        if (!(t >= 0x1p-100f)) {
            // every component is > 100 binades below cmax at this point: the exact maximum
            rare_any = true;
            float mx = -INFINITY;
            for (int pp = 0; pp < npairs; ++pp) {
                PairParams P;
                load_pair(pp, P);
                const float2 nq = neg_logit2(P, X[p][0], X[p][1], X[p][2]);
                mx = fmaxf(mx, fmaxf(-nq.x, -nq.y));
            }
            if (!(mx > -INFINITY)) {
                set_error(a.st, GIRA_ERR_NUMERIC);
                continue;
            }
            float sm = 0.f;
            for (int pp = 0; pp < npairs; ++pp) {
                PairParams P;
                load_pair(pp, P);
                const float2 nq = neg_logit2(P, X[p][0], X[p][1], X[p][2]);
                sm += ex2_approx(-nq.x - mx) + ex2_approx(-nq.y - mx);
            }
            t = sm;
            sh = -mx;
        }
        pr[p] = f2(sh, __frcp_rn(t));
        const float lse2 = lg2_approx(t) + ref0 - sh;   // log2 sum_b pi_b N(x|b)
        if (half == 0) {   // (every warp of the block has the same totals)
            ll += (double)lse2;
            if (!STATS && a.per_point) a.per_point[base + 32 * p] = lse2 * LN2F;
        }
    }

    if (STATS) {
        __syncwarp();
        if (__any_sync(FULL, rare_any) && lane < nwords) {   // every evaluated pair of this warp
            const int lo = lane * 32;
            const uint32_t mine = PT_H == 1 ? 0xffffffffu : (half ? 0xaaaaaaaau : 0x55555555u);
            smask[lane] = mine & ((lo + 32 <= npairs) ? 0xffffffffu : (lo < npairs) ? ((1u << (npairs - lo)) - 1u) : 0u);
        }
        pt_block_sync(blk);   // the block's masks are final
        const int64_t gw = (int64_t)cta * PT_B + blk;
        const int64_t rows = a.pt_rows;
        if (half == 0 && lane < nwords) {
            uint32_t m = 0u;
#pragma unroll
            for (int h = 0; h < PT_H; ++h) m |= smask_all[(blk * PT_H + h) * nwords + lane];
            if (GIRA_IN(gw < rows, a.st)) a.masks[lane * rows + gw] = m;
        }
        if (lane == 0) {
            unsigned live = 0;
            for (int wd = 0; wd < nwords; ++wd) live += __popc(smask[wd]);
            s_pairs[warp][0] = (unsigned)nlive;
            s_pairs[warp][1] = live;
        }
        // ---- phase 2: this warp's live pairs; partials [rows][pairs][2 NSTAT], masks [nwords][rows]
        for (int wd = 0; wd < nwords; ++wd) {
            uint32_t m = smask[wd];
            while (m) {
                const int pp = wd * 32 + __ffs(m) - 1;
                m &= m - 1u;
                PairParams P;
                load_pair(pp, P);
                float2 S[NSTAT];
#pragma unroll
                for (int s2 = 0; s2 < NSTAT; ++s2) S[s2] = f2(0.f, 0.f);
#pragma unroll
                for (int p = 0; p < PT_P; ++p) {
                    float2 y0, y1, y2;
                    const float2 nq = neg_logit2_y(P, X[p][0], X[p][1], X[p][2], y0, y1, y2);
                    const float2 e = f2(ex2_approx(pr[p].x - nq.x), ex2_approx(pr[p].x - nq.y));
                    const float2 g = mul2(e, dup(pr[p].y));   // pr = 0 for invalid points: g = 0
                    const float2 g0 = mul2(g, y0), g1 = mul2(g, y1), g2 = mul2(g, y2);
                    S[0] = add2(S[0], g);
                    S[1] = add2(S[1], g0);
                    S[2] = add2(S[2], g1);
                    S[3] = add2(S[3], g2);
                    S[4] = fma2(g0, y0, S[4]);
                    S[5] = fma2(g0, y1, S[5]);
                    S[6] = fma2(g0, y2, S[6]);
                    S[7] = fma2(g1, y1, S[7]);
                    S[8] = fma2(g1, y2, S[8]);
                    S[9] = fma2(g2, y2, S[9]);
                }
                int v;
                const float r = pt_warp_reduce20(S, lane, &v);
                const int b = 2 * pp + (v >= NSTAT ? 1 : 0);
                if ((lane & 7) < 5 && b < a.k && GIRA_IN(gw < rows, a.st))
                    a.partials[(size_t)gw * pt_row_floats(a.k) + (size_t)pp * 2 * NSTAT + v] = r;
            }
        }
    }
    // the CTA's log-likelihood: lanes, then warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(FULL, ll, o);
    if (lane == 0) s_ll[warp] = ll;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = s_ll[0];
        for (int w = 1; w < PT_W; ++w) v += s_ll[w];
        if (GIRA_IN(cta < (a_in.units ? a.pt_rows / PT_B : (int64_t)gridDim.x), a.st)) a.ll_partials[cta] = v * LN2;
        if (STATS) {
            unsigned long long near = 0, live = 0;
            for (int w = 0; w < PT_W; ++w) {
                near += s_pairs[w][0];
                live += s_pairs[w][1];
            }
            atomicAdd(&a.st->pairs_near, near);
            atomicAdd(&a.st->pairs_live, live);
            if (a_in.cta_key) {   // the CTA's slowest warp, in units of a point's pair evaluations
                unsigned wmax = 0;
                for (int w = 0; w < PT_W; ++w)
                    wmax = max(wmax, PT_COST_NEAR * s_pairs[w][0] + PT_COST_LIVE * s_pairs[w][1]);
                if (GIRA_IN(cta < (int)gridDim.x, a.st)) a_in.cta_key[cta] = work_key(wmax);
            }
        }
    }
}

// ------------------------------------------------------------------ launch policy
// Shapes: K <= 64 -> one component pair per lane and one warp; otherwise two
// pairs per lane and G = ceil(K / 128) warps; batches of Q = 8 points, one CTA
// barrier per batch, statistics accumulated with scalar FP32 operations.
// Measured on GB300 for K = 512 (276,348 points): Q = 8 171 us, Q = 4 192 us,
// Q = 4 software-pipelined 203 us, scalar statistics 169 us; one pair per lane
// with 8 warps, other CTA-per-SM targets and a producer/consumer
// warp-specialised variant were slower.  Probes of the two passes alone show
// the FP32 pipe at ~60 % (pass 1) and ~74 % (pass 2) of its peak: the limit is
// register-file operand bandwidth (three distinct register operands per FFMA),
// not occupancy (3, 4 or 5 CTAs per SM run pass 1 at the same speed).
#ifndef GIRA_ESTEP_Q
#define GIRA_ESTEP_Q 8
#endif
constexpr int QB = GIRA_ESTEP_Q;

struct Shape {
    int np, g, threads;
};

Shape shape_for(int k) {
    if (k <= 64) return {1, 1, 32};
    const int g = (k + 127) / 128;
    return {2, g, 32 * g};
}

// A kernel of the launch policy (the batch-synchronous estep_kernel).
struct KSel {
    const void* fn;
};

template <bool STATS>
KSel kernel_for(const Shape& sh) {
    if (sh.np == 1) return {(const void*)estep_kernel<1, QB, 32, 16, STATS>};
    if (sh.g <= 4) return {(const void*)estep_kernel<2, QB, 128, 3, STATS>};
    return {(const void*)estep_kernel<2, QB, 256, 1, STATS>};
}
// Differentiable path: the adjoint kernel, or (forward only) the log-likelihood.
KSel grad_kernel_for(const Shape& sh, bool stats) {
    if (!stats) return kernel_for<false>(sh);
    if (sh.np == 1) return {(const void*)estep_kernel<1, QB, 32, 16, true, true>};
    if (sh.g <= 4) return {(const void*)estep_kernel<2, QB, 128, 2, true, true>};
    return {(const void*)estep_kernel<2, QB, 256, 1, true, true>};
}

size_t estep_smem(int64_t ppc) { return (size_t)ppc * 32; }
size_t smem_of(const KSel&, const Shape&, int64_t ppc) { return estep_smem(ppc); }

}  // namespace

int params_pairs_padded(int k) {
    Shape sh = shape_for(k);
    return sh.np * sh.g * 32;
}

// Points per CTA and grid: as many CTAs as fit on the SMs (points of a CTA
// staged in shared memory, at most PPC_MAX per CTA).
int estep_grid(int64_t n, int k, bool stats, int num_sms, int64_t* pts_per_cta, bool grad) {
    const Shape sh = shape_for(k);
    const KSel ks = grad ? grad_kernel_for(sh, stats) : stats ? kernel_for<true>(sh) : kernel_for<false>(sh);
    const void* fn = ks.fn;
    int occ = 1;
    // occupancy with the largest staging buffer the launch could use
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of(ks, sh, PPC_MAX));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, sh.threads, smem_of(ks, sh, PPC_MAX / 4)) !=
            cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    int64_t grid = std::max<int64_t>(1, std::min<int64_t>((n + QB - 1) / QB, (int64_t)num_sms * occ));
    int64_t ppc = ((n + grid - 1) / grid + QB - 1) / QB * QB;
    ppc = std::min<int64_t>(ppc, PPC_MAX);
    grid = (n + ppc - 1) / ppc;
    *pts_per_cta = ppc;
    return (int)grid;
}

void estep_shape(int k, int* np, int* g, int* threads) {
    const Shape sh = shape_for(k);
    *np = sh.np;
    *g = sh.g;
    *threads = sh.threads;
}

int estep_batch_q() { return QB; }

int estep_ppc_max() { return PPC_MAX; }

int estep_occupancy(int k, bool stats, int64_t ppc) {
    const Shape sh = shape_for(k);
    const KSel ks = stats ? kernel_for<true>(sh) : kernel_for<false>(sh);
    const void* fn = ks.fn;
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of(ks, sh, PPC_MAX));
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, sh.threads, smem_of(ks, sh, ppc)) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    return occ;
}

cudaError_t launch_estep_units(const EStepLaunch& a, bool stats, int nunits, int k_class, int64_t ppc_class,
                               cudaStream_t s) {
    const Shape sh = shape_for(k_class);
    void* args[] = {(void*)&a};
    const KSel ks = stats ? kernel_for<true>(sh) : kernel_for<false>(sh);
    const void* fn = ks.fn;
    const size_t smem = smem_of(ks, sh, ppc_class);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(fn, dim3(nunits), dim3(sh.threads), args, smem, s);
}

cudaError_t launch_estep_grad_units(const EStepLaunch& a, int nunits, int k_class, int64_t ppc_class, cudaStream_t s) {
    const Shape sh = shape_for(k_class);
    void* args[] = {(void*)&a};
    const KSel ks = grad_kernel_for(sh, true);
    const void* fn = ks.fn;
    const size_t smem = smem_of(ks, sh, ppc_class);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(fn, dim3(nunits), dim3(sh.threads), args, smem, s);
}

int estep_grad_occupancy(int k, int64_t ppc) {
    const Shape sh = shape_for(k);
    const KSel ks = grad_kernel_for(sh, true);
    const void* fn = ks.fn;
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of(ks, sh, PPC_MAX));
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, sh.threads, smem_of(ks, sh, ppc)) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    return occ;
}

constexpr int KCHUNK = 512;   // components per chunk: the 4-warp shape

int chunk_components() { return KCHUNK; }

int64_t chunk_param_floats() { return (int64_t)params_pairs_padded(KCHUNK) * PAIR_FLOATS; }

cudaError_t launch_estep_chunks(const EStepLaunch& a, int pass, int nunits, int64_t ppc, cudaStream_t s) {
    void* args[] = {(void*)&a};
    const void* fn = (pass == 1) ? (const void*)estep_kernel<2, QB, 128, 3, false, false, 1>
                                 : (const void*)estep_kernel<2, QB, 128, 3, true, false, 2>;
    const size_t smem = estep_smem(ppc);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(fn, dim3(nunits), dim3(128), args, smem, s);
}

namespace {
thread_local std::string t_estep_name;
thread_local const void* t_estep_fn = nullptr;
}  // namespace

// The launched function's name as the runtime reports it, demangled, without
// its namespaces and parameter list.
void note_estep_kernel(const void* fn) {
    if (fn == t_estep_fn) return;
    t_estep_fn = fn;
    const char* raw = nullptr;
    if (cudaFuncGetName(&raw, fn) != cudaSuccess || !raw) {
        cudaGetLastError();
        t_estep_name = "estep_kernel";
        return;
    }
    int ok = -1;
    char* dem = abi::__cxa_demangle(raw, nullptr, nullptr, &ok);
    std::string name = (ok == 0 && dem) ? dem : raw;
    std::free(dem);
    size_t at = name.find("estep_kernel<");
    if (at == std::string::npos) at = name.find("estep_pt_kernel<");
    if (at == std::string::npos) at = name.find("estep4_kernel<");
    if (at != std::string::npos) name = name.substr(at);
    const size_t par = name.rfind(">(");
    if (par != std::string::npos) name = name.substr(0, par + 1);
    t_estep_name = name;
}

const char* last_estep_kernel() { return t_estep_name.c_str(); }

int estep_pt_grid(int64_t n) { return (int)std::max<int64_t>(1, (n + PT_PTS - 1) / PT_PTS); }
int estep_pt_rows(int grid) { return grid * PT_B; }
int estep_pt_row_floats(int k) { return pt_row_floats(k); }
int estep_pt_mask_words(int k) { return pt_pairs(k) / 32; }

cudaError_t launch_estep_pt(const EStepLaunch& a, bool stats, int grid, cudaStream_t s, bool pdl) {
    void* args[] = {(void*)&a};
    const void* fn = stats ? (const void*)estep_pt_kernel<true> : (const void*)estep_pt_kernel<false>;
    note_estep_kernel(fn);
    const size_t smem = pt_smem_bytes(a.k);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    PdlConfig c(dim3(grid), dim3(32 * PT_W), smem, s, pdl);
    return cudaLaunchKernelExC(&c.cfg, fn, args);
}

cudaError_t launch_estep_pt_units(const EStepLaunch& a, bool stats, int nunits, int kmax, cudaStream_t s) {
    void* args[] = {(void*)&a};
    const void* fn = stats ? (const void*)estep_pt_kernel<true> : (const void*)estep_pt_kernel<false>;
    note_estep_kernel(fn);
    const size_t smem = pt_smem_bytes(kmax);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(fn, dim3(nunits), dim3(32 * PT_W), args, smem, s);
}

int estep_pt_points() { return PT_PTS; }
int estep_pt_blocks() { return PT_B; }

cudaError_t launch_estep(const EStepLaunch& a, bool stats, int grid, cudaStream_t s, bool grad, bool pdl) {
    const Shape sh = shape_for(a.k);
    void* args[] = {(void*)&a};
    const KSel ks = grad ? grad_kernel_for(sh, stats) : stats ? kernel_for<true>(sh) : kernel_for<false>(sh);
    const void* fn = ks.fn;
    note_estep_kernel(fn);
    const size_t smem = smem_of(ks, sh, a.pts_per_cta);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    PdlConfig c(dim3(grid), dim3(sh.threads), smem, s, pdl);
    return cudaLaunchKernelExC(&c.cfg, fn, args);
}

// ------------------------------------------------------------------ pack + padding
namespace {
__global__ void pack_kernel(const float* __restrict__ p3, int64_t n, float4* __restrict__ p4,
                            float4* __restrict__ p8, DeviceState* st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = p3[3 * i], y = p3[3 * i + 1], z = p3[3 * i + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) set_error(st, GIRA_ERR_NONFINITE_INPUT);
    if (p4) p4[i] = make_float4(x, y, z, 0.f);
    if (p8) {
        p8[2 * i] = make_float4(x, x, y, y);
        p8[2 * i + 1] = make_float4(z, z, 0.f, 0.f);
    }
}

// One block per instance: the padding component slots k .. 2 * npairs - 1 of its block.
__global__ void fill_padding_batched_kernel(float* params, const BatchInst* __restrict__ insts,
                                            const int* __restrict__ npairs_of) {
    const BatchInst I = insts[blockIdx.x];
    const int slots = 2 * npairs_of[blockIdx.x];
    for (int b = I.k + threadIdx.x; b < slots; b += blockDim.x) {
        float* base = params + I.par_off + (size_t)(b >> 1) * PAIR_FLOATS + (b & 1);
        for (int s = 0; s < PAIR_FLOATS / 2; ++s) base[2 * s] = 0.f;
        base[2 * SLOT_C] = -INFINITY;
    }
}

__global__ void fill_padding_kernel(float* params, int k, int npairs_pad) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;   // component slot
    if (b >= 2 * npairs_pad || b < k) return;
    float* base = params + (size_t)(b >> 1) * PAIR_FLOATS + (b & 1);
    for (int s = 0; s < PAIR_FLOATS / 2; ++s) base[2 * s] = 0.f;
    base[2 * SLOT_C] = -INFINITY;
}
}  // namespace

// Every point of a batch; the instance of point i (for the error flag) by binary
// search over the offsets (batch + 1 entries).
__global__ void pack_batched_kernel(const float* __restrict__ p3, int64_t n, const int64_t* __restrict__ offsets,
                                    int batch, float4* __restrict__ p4, float4* __restrict__ p8, DeviceState* states) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = p3[3 * i], y = p3[3 * i + 1], z = p3[3 * i + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
        int lo = 0, hi = batch;   // offsets[lo] <= i < offsets[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (offsets[mid] <= i) lo = mid; else hi = mid;
        }
        set_error(states + lo, GIRA_ERR_NONFINITE_INPUT);
    }
    if (p4) p4[i] = make_float4(x, y, z, 0.f);
    if (p8) {
        p8[2 * i] = make_float4(x, x, y, y);
        p8[2 * i + 1] = make_float4(z, z, 0.f, 0.f);
    }
}

cudaError_t launch_pack_batched(const float* pts3, int64_t n, const int64_t* offsets, int batch, float4* pts4,
                                float4* pts8, DeviceState* states, cudaStream_t s) {
    pack_batched_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts3, n, offsets, batch, pts4, pts8, states);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float* pts3, int64_t n, float4* pts4, float4* pts8, DeviceState* st, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    pack_kernel<<<(unsigned)blocks, 256, 0, s>>>(pts3, n, pts4, pts8, st);
    return cudaGetLastError();
}

cudaError_t launch_fill_padding(float* params, int k, int npairs_pad, cudaStream_t s) {
    int slots = 2 * npairs_pad;
    fill_padding_kernel<<<(slots + 127) / 128, 128, 0, s>>>(params, k, npairs_pad);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ log-likelihood reduce
namespace {
// ------------------------------------------------------------------ large K (chunks)
constexpr int CHUNK_K = 512;
constexpr int COMBINE_BLOCKS = 608;
constexpr int COMBINE_THREADS = 256;

// component b of a chunked parameter buffer
__device__ __forceinline__ const float* chunk_slot(const float* params, int b) {
    const int c = b / CHUNK_K, l = b - c * CHUNK_K;
    return params + (size_t)c * (CHUNK_K / 2) * PAIR_FLOATS + (size_t)(l >> 1) * PAIR_FLOATS + (l & 1);
}

// gref[0] = max_b c_b, gref[1] = the log-likelihood reference (cmax - log2 sum_a N_a
// after an M-step, else cmax): the per-CTA kernel's prologue over all k components.
__global__ void chunk_ref_kernel(const float* __restrict__ params, int k, const DeviceState* st, float* gref) {
    __shared__ float s_m[8];
    __shared__ double s_w[8];
    float m = -INFINITY;
    double w = 0.0;
    for (int b = threadIdx.x; b < k; b += blockDim.x) {
        const float* p = chunk_slot(params, b);
        m = fmaxf(m, p[2 * SLOT_C]);
        w += (double)p[2 * SLOT_W];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        w += __shfl_xor_sync(0xffffffffu, w, o);
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

// Per point: total over chunks (fixed order); (0, 1/total) and the natural-log
// log-likelihood, or, if the total is below 2^-100, listed for the exact step.
__global__ void __launch_bounds__(COMBINE_THREADS) chunk_combine_kernel(const float* __restrict__ psum, int chunks,
                                                                        int64_t n, const float* __restrict__ gref,
                                                                        float2* pref, double* llpt, int* flag_count,
                                                                        int* flags) {
    const float ref0 = gref[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float tot = 0.f;
        for (int c = 0; c < chunks; ++c) tot += psum[(size_t)c * n + i];
        if (tot >= 0x1p-100f) {
            pref[i] = make_float2(0.f, __frcp_rn(tot));
            llpt[i] = (double)(lg2_approx(tot) + ref0) * 0.693147180559945309417232121458;
        } else {
            pref[i] = make_float2(0.f, 0.f);
            llpt[i] = 0.0;
            flags[atomicAdd(flag_count, 1)] = (int)i;
        }
    }
}

// One warp per listed point: exact maximum of the logits over all k components,
// then (shift, 1/sum) relative to it (Eq. logestep's max-subtraction).
__global__ void chunk_exact_kernel(const float4* __restrict__ pts8, const float* __restrict__ params, int k,
                                   const float* __restrict__ gref, const int* __restrict__ flags,
                                   const int* __restrict__ flag_count, float2* pref, double* llpt, DeviceState* st) {
    const int count = *flag_count;
    const float cmax = gref[0], ref0 = gref[1];
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int f = wg; f < count; f += nw) {
        const int64_t i = flags[f];
        const float4 xy = pts8[2 * i], zz = pts8[2 * i + 1];
        const float x0 = xy.x, x1 = xy.z, x2 = zz.x;
        auto nlog = [&](int b) {   // q' = |P'(x - mu)|^2 + (cmax - c_b), as the E-step forms it
            const float* p = chunk_slot(params, b);
            const float d0 = x0 + p[2 * (SLOT_NMU + 0)], d1 = x1 + p[2 * (SLOT_NMU + 1)], d2 = x2 + p[2 * (SLOT_NMU + 2)];
            const float y0 = p[2 * (SLOT_P + 0)] * d0;
            const float y1 = fmaf(p[2 * (SLOT_P + 2)], d1, p[2 * (SLOT_P + 1)] * d0);
            const float y2 = fmaf(p[2 * (SLOT_P + 5)], d2, fmaf(p[2 * (SLOT_P + 4)], d1, p[2 * (SLOT_P + 3)] * d0));
            return fmaf(y2, y2, fmaf(y1, y1, fmaf(y0, y0, cmax - p[2 * SLOT_C])));
        };
        float mx = -INFINITY;
        for (int b = lane; b < k; b += 32) mx = fmaxf(mx, -nlog(b));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float sum = 0.f;
        if (mx > -INFINITY)
            for (int b = lane; b < k; b += 32) sum += ex2_approx(-nlog(b) - mx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) {
            if (!(mx > -INFINITY) || !(sum > 0.f)) {
                set_error(st, GIRA_ERR_NUMERIC);
                pref[i] = make_float2(0.f, 0.f);
            } else {
                pref[i] = make_float2(-mx, __frcp_rn(sum));
                llpt[i] = (double)(lg2_approx(sum) + mx + ref0) * 0.693147180559945309417232121458;
            }
        }
    }
}

// Fixed-order per-block sums of the per-point log-likelihoods.
__global__ void __launch_bounds__(COMBINE_THREADS) points_ll_reduce_kernel(const double* __restrict__ llpt, int64_t n,
                                                                           double* llp) {
    __shared__ double s_w[COMBINE_THREADS / 32];
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v += llpt[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < COMBINE_THREADS / 32; ++w) t += s_w[w];
        llp[blockIdx.x] = t;
    }
}

__global__ void ll_reduce_batched_kernel(const double* __restrict__ llp, const BatchInst* __restrict__ insts,
                                         DeviceState* states) {
    const BatchInst I = insts[blockIdx.x];
    double v = 0.0;
    for (int c = threadIdx.x; c < I.ctas; c += 32) v += llp[I.ll_off + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) states[blockIdx.x].ll_sum = v;
}

__global__ void ll_reduce_kernel(const double* __restrict__ llp, int grid, DeviceState* st) {
    if (st->error) return;
    double v = 0.0;
    for (int c = threadIdx.x; c < grid; c += 32) v += llp[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (threadIdx.x == 0) st->ll_sum = v;
}
}  // namespace

cudaError_t launch_ll_reduce(const double* ll_partials, int grid, DeviceState* st, cudaStream_t s) {
    ll_reduce_kernel<<<1, 32, 0, s>>>(ll_partials, grid, st);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 M-step
namespace {

constexpr int FIN_CPB = 2;          // components per block: spreads the binary64 work over SMs
constexpr int FIN_SPLIT_CTA = 16;   // per-CTA partials: one output summed in 16 fixed slices
constexpr int FIN_SPLIT = 64;       // per-warp rows: one float4 of outputs summed in 64 fixed slices
constexpr int FIN_THREADS = FIN_CPB * NSTAT * FIN_SPLIT_CTA;   // 320
constexpr int ORDER_THREADS = 1024;   // order_components_kernel: one block
constexpr int ORDER_MAX_K = 8192;     // keys in dynamic shared memory (64 KB)

// ---- the parameter build, shared by the scalar and the warp-parallel forms.
// Every helper fixes its binary64 operations (explicit rounding intrinsics, no
// contraction left to the compiler), so both forms give the same bits.

// Cholesky Sigma = L L^T of c = (00, 01, 02, 11, 12, 22) by Schur complements,
// in terms of the pivots' reciprocal square roots:
//   u = a00^-1/2, r0 = u^2, h0 = a01 r0,
//   s11 = a11 - h0 a01, s12 = a12 - h0 a02, s22 = a22 - (a02 r0) a02,
//   v = s11^-1/2, t = s12 v^2, a22' = s22 - t s12, z = a22'^-1/2, g = a02 - a01 t;
// then P = L^-1 has P00 = u, P11 = v, P22 = z, P10 = -h0 v, P21 = -t z,
// P20 = -(r0 g) z, and prod_j P_jj = u v z.  pd: every pivot positive.
struct CholInv {
    double u, v, z, r0, h0, t, g;
    bool pd;
};

__device__ __forceinline__ CholInv chol_inv(const double c[6]) {
    CholInv k;
    k.u = rsqrt(c[0]);
    k.r0 = __dmul_rn(k.u, k.u);
    k.h0 = __dmul_rn(c[1], k.r0);
    const double h1 = __dmul_rn(c[2], k.r0);
    const double s11 = __fma_rn(-k.h0, c[1], c[3]);
    const double s12 = __fma_rn(-k.h0, c[2], c[4]);
    const double s22 = __fma_rn(-h1, c[2], c[5]);
    k.v = rsqrt(s11);
    k.t = __dmul_rn(s12, __dmul_rn(k.v, k.v));
    const double a22 = __fma_rn(-k.t, s12, s22);
    k.z = rsqrt(a22);
    k.g = __fma_rn(-c[1], k.t, c[2]);
    k.pd = c[0] > 0.0 && s11 > 0.0 && a22 > 0.0;
    return k;
}

constexpr double ALPHA = 0.84932180028801904272;   // sqrt(log2(e) / 2)

// Entry e of P' = alpha L^-1 in the order (00, 10, 11, 20, 21, 22), as
// alpha ((A B) C) with (A, B, C) = (u, 1, 1), (h0, v, -1), (v, 1, 1), (r0, g, -z),
// (t, z, -1), (z, 1, 1): the same three products for every entry.
__device__ __forceinline__ double chol_q(const CholInv& k, int e) {
    const double A = e == 0 ? k.u : e == 1 ? k.h0 : e == 2 ? k.v : e == 3 ? k.r0 : e == 4 ? k.t : k.z;
    const double B = e == 1 ? k.v : e == 3 ? k.g : e == 4 ? k.z : 1.0;
    const double C = e == 1 || e == 4 ? -1.0 : e == 3 ? -k.z : 1.0;
    return __dmul_rn(ALPHA, __dmul_rn(__dmul_rn(A, B), C));
}

// b_i = -(P' mu)_i from the row (a0, a1, a2) of P' (zeros above the diagonal).
__device__ __forceinline__ double bias_row(double a0, double a1, double a2, const double mu[3]) {
    return -__fma_rn(a2, mu[2], __fma_rn(a1, mu[1], __dmul_rn(a0, mu[0])));
}

// c = log2(w prod_j P_jj) - (3/2) log2(2 pi) in binary32: the exponent of
// x = w u v z exactly, log2f of its significand rounded to 24 bits (error a
// few 1e-8), the constant 4 - (3/2) log2(2 pi) = 0.0227558057915218 folded in.
__device__ __forceinline__ float log2_norm(double w, const CholInv& k) {
    const double x = __dmul_rn(w, __dmul_rn(__dmul_rn(k.u, k.v), k.z));
    if (!(x >= DBL_MIN && x <= DBL_MAX)) return (float)(log2(x) - 3.9772441942084782);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ffu) - 1023;
    const unsigned int m24 = (unsigned int)(((bits & 0xfffffffffffffull) + (1ull << 28)) >> 29);   // 0 .. 2^23
    const float m = __int_as_float((127 << 23) + (int)m24);   // the significand in [1, 2]
    return __fadd_rn((float)(e - 4), __fadd_rn(log2f(m), 0.0227558057915218f));
}

// alpha^2 / lambda_max(Sigma), lowered by 1e-4 relative: a lower bound of
// sigma_min(P')^2 for the E-step's reach test.  lambda_max by the trigonometric
// solution of the characteristic cubic of a symmetric 3x3 matrix in binary32
// (error a few ulps), raised by 1e-4 relative; trace(Sigma) where the cubic is
// degenerate; never below the largest diagonal entry.
__device__ __forceinline__ float sigma_min_sq_bound(const float a[6]) {
    const float a00 = a[0], a01 = a[1], a02 = a[2], a11 = a[3], a12 = a[4], a22 = a[5];
    const float tr3 = (a00 + a11 + a22) * (1.f / 3.f);
    const float e0 = a00 - tr3, e1 = a11 - tr3, e2 = a22 - tr3;
    const float p2 = e0 * e0 + e1 * e1 + e2 * e2 + 2.f * (a01 * a01 + a02 * a02 + a12 * a12);
    float lmax = 3.f * tr3;
    if (p2 > 1e-30f) {
        const float pp = sqrtf(p2 * (1.f / 6.f)), ip = 1.f / pp;
        const float b00 = e0 * ip, b11 = e1 * ip, b22 = e2 * ip, b01 = a01 * ip, b02 = a02 * ip, b12 = a12 * ip;
        const float det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
        const float r = fminf(1.f, fmaxf(-1.f, 0.5f * det));
        const float trig = tr3 + 2.f * pp * cosf(acosf(r) * (1.f / 3.f));
        if (trig == trig) lmax = fminf(lmax, trig * (1.f + 1e-4f));
    }
    lmax = fmaxf(lmax, fmaxf(a00, fmaxf(a11, a22)) * (1.f + 1e-4f));
    return (float)(ALPHA * ALPHA) / lmax * (1.f - 1e-4f);
}

// From (w, mu, Sigma) in binary64 to the E-step parameters of component b
// (scalar form; the EM finalize runs the same helpers lane-parallel).
// Returns false (and flags GIRA_ERR_NOT_PD) if a pivot is not positive.
// report: the caller's index of the component (differs from b when the fit
// holds its components in another order).
__device__ bool build_component(int b, double w, const double mu[3], const double c[6], float* params,
                                float4* shift4, double* model64, DeviceState* st, int report) {
    const CholInv k = chol_inv(c);
    if (!k.pd) {
        atomicMin(&st->bad_component, report);
        set_error(st, GIRA_ERR_NOT_PD);
        return false;
    }
    double q[6];
    for (int e = 0; e < 6; ++e) q[e] = chol_q(k, e);
    float* base = params + (size_t)(b >> 1) * PAIR_FLOATS + (b & 1);
    for (int i = 0; i < 6; ++i) base[2 * (SLOT_P + i)] = (float)q[i];
    base[2 * (SLOT_B + 0)] = (float)bias_row(q[0], 0.0, 0.0, mu);
    base[2 * (SLOT_B + 1)] = (float)bias_row(q[1], q[2], 0.0, mu);
    base[2 * (SLOT_B + 2)] = (float)bias_row(q[3], q[4], q[5], mu);
    base[2 * SLOT_C] = log2_norm(w, k);
    const float m32[3] = {(float)mu[0], (float)mu[1], (float)mu[2]};
    for (int i = 0; i < 3; ++i) base[2 * (SLOT_NMU + i)] = -m32[i];
    base[2 * SLOT_W] = (float)w;
    const float c32[6] = {(float)c[0], (float)c[1], (float)c[2], (float)c[3], (float)c[4], (float)c[5]};
    base[2 * SLOT_S] = sigma_min_sq_bound(c32);
    shift4[b] = make_float4(m32[0], m32[1], m32[2], 0.f);
    double* m = model64 + (size_t)b * MODEL;
    m[0] = w;
    m[1] = mu[0]; m[2] = mu[1]; m[3] = mu[2];
    for (int i = 0; i < 6; ++i) m[4 + i] = c[i];
    return true;
}

// The statistics of components b0 .. b0 + nout / NSTAT - 1 summed over the
// per-CTA partials into S (binary64): FIN_SPLIT_CTA fixed slices of CTAs, binary32
// groups of 8 within a slice, binary64 across groups and slices.  Call with
// every thread of the block; ends with S valid after a barrier.
__device__ void reduce_partials(const float* __restrict__ partials, int grid, int k, int b0, int nout,
                                double (*part)[FIN_CPB * NSTAT], double* S) {
    const int t = threadIdx.x;
    const int o = t % (FIN_CPB * NSTAT), q = t / (FIN_CPB * NSTAT);
    if (o < nout) {
        const int c0 = q * grid / FIN_SPLIT_CTA, c1 = (q + 1) * grid / FIN_SPLIT_CTA;
        const float* src = partials + (size_t)b0 * NSTAT + o;
        const size_t stride = (size_t)k * NSTAT;
        double acc = 0.0;
        for (int c = c0; c < c1; c += 8) {   // eight independent loads in flight
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = (c + u < c1) ? __ldcg(src + (size_t)(c + u) * stride) : 0.f;
            float f = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) f += v[u];
            acc += (double)f;
        }
        part[q][o] = acc;
    }
    __syncthreads();
    if (t < nout) {
        double v = 0.0;
        for (int q2 = 0; q2 < FIN_SPLIT_CTA; ++q2) v += part[q2][t];
        S[t] = v;
    }
}

// Compensated binary32 accumulation (Knuth's TwoSum: the rounding error of each
// addition, exact under round-to-nearest, is carried in e).
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    e = __fadd_rn(e, err);
}

// Per-component binary64 work area of the finalize (shared memory), in doubles.
constexpr int FW = 64;
constexpr int W_S = 0;      // S0, S1[3], S2[6]
constexpr int W_QS = 10;    // P' (00,10,11,20,21,22) and the shift s[3]; later the new P' and b
constexpr int W_R = 19;     // 1/q00, 1/q11, 1/q22, 1/N_b
constexpr int W_T = 23;     // ybar[3], m10, m21
constexpr int W_M = 28;     // M = P'^-1 (3x3 row-major; the identity for one-hot statistics)
constexpr int W_CY = 37;    // C (3x3, both halves)
constexpr int W_MU = 46;    // the new mean
constexpr int W_MC = 49;    // M C (3x3)
constexpr int W_C = 58;     // the new Sigma (00,01,02,11,12,22)
constexpr int FF = 20;      // binary32 copies per component: P'[6], b[3], mu[3], w, Sigma[6]

// The statistics of the pair of components b0, b0 + 1 (b0 even) from the per-warp
// partial rows of the point-stationary E-step ([rows][pairs][2 NSTAT] binary32, a
// pair's 20 values 80 contiguous bytes): the rows whose live mask has the pair's bit
// are listed in row order (one block scan per segment of FIN_SEG rows, each thread
// ranking a contiguous run of rows).  Thread (c, q) = (t / 64, t % 64) sums float4 c
// of the pair's values (outputs 4c .. 4c + 3; output o is component o / NSTAT,
// statistic o % NSTAT) over the q-th of FIN_SPLIT fixed contiguous slices of the list
// in compensated binary32; a fixed butterfly of compensated additions joins the 32
// slices of a warp, then the two warps of c in order, and each (sum, error) becomes
// one binary64 value in W.  The list depends only on the masks, so the order of every
// addition is fixed.  Call with every thread of the block; s_skip (set by thread 0
// before the call) is read after the first barrier, and a skipped block returns false
// before touching W.
constexpr int FIN_SEG = 4096;
static_assert(FIN_THREADS == 5 * 64 && FIN_SPLIT == 64 && 2 * NSTAT == 20, "five float4 of a pair, 64 slices each");
__device__ bool reduce_partials_masked(const float* __restrict__ partials, int rows, int row_floats,
                                       const uint32_t* __restrict__ masks, int b0, int nout, double (*W)[FW],
                                       const int* s_skip, DeviceState* st) {
    __shared__ uint16_t s_list[FIN_SEG];
    __shared__ int s_wsum[FIN_THREADS / 32];
    __shared__ float s_hi[FIN_THREADS / 64][8];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int c = t >> 6, q = t & 63;
    const uint32_t* mrow = masks + (size_t)((b0 >> 1) >> 5) * rows;
    const uint32_t bit = 1u << ((b0 >> 1) & 31);
    const float4* src = reinterpret_cast<const float4*>(partials + (size_t)(b0 >> 1) * 2 * NSTAT) + c;
    const size_t stride4 = (size_t)row_floats / 4;
    float sum[4] = {0.f, 0.f, 0.f, 0.f}, err[4] = {0.f, 0.f, 0.f, 0.f};
    for (int seg0 = 0; seg0 < rows; seg0 += FIN_SEG) {
        const int seg1 = min(rows, seg0 + FIN_SEG);
        constexpr int RND = (FIN_SEG + FIN_THREADS - 1) / FIN_THREADS;
        const int per = (seg1 - seg0 + FIN_THREADS - 1) / FIN_THREADS;   // rows ranked by one thread
        const int r0 = seg0 + t * per;
        uint32_t live = 0u;   // bit u: row r0 + u is live
#pragma unroll
        for (int u = 0; u < RND; ++u) {
            const uint32_t mw = (u < per && r0 + u < seg1) ? __ldg(mrow + r0 + u) : 0u;
            if (mw & bit) live |= 1u << u;
        }
        const int cnt = __popc(live);
        int incl = cnt;   // inclusive scan of the counts over the warp
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (*s_skip) return false;
        int off = incl - cnt, nl = 0;
#pragma unroll
        for (int w = 0; w < FIN_THREADS / 32; ++w) {
            const int cw = s_wsum[w];
            off += (w < warp) ? cw : 0;
            nl += cw;
        }
        for (uint32_t m = live; m; m &= m - 1u) {
            const int r = r0 + __ffs(m) - 1;
            if (GIRA_IN(off < FIN_SEG, st)) s_list[off] = (uint16_t)(r - seg0);
            ++off;
        }
        __syncthreads();
        const int c0 = q * nl / FIN_SPLIT, c1 = (q + 1) * nl / FIN_SPLIT;
        const float4* sseg = src + (size_t)seg0 * stride4;
        for (int i = c0; i < c1; i += 8) {   // eight float4 loads in flight
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = (i + u < c1 && GIRA_IN(s_list[i + u] < seg1 - seg0, st))
                           ? __ldcg(sseg + (size_t)s_list[i + u] * stride4) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (i + u < c1) {
                    two_sum_acc(sum[0], err[0], v[u].x);
                    two_sum_acc(sum[1], err[1], v[u].y);
                    two_sum_acc(sum[2], err[2], v[u].z);
                    two_sum_acc(sum[3], err[3], v[u].w);
                }
            }
        }
        __syncthreads();   // the list is rebuilt for the next segment
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {   // butterfly over the warp: the same totals in every lane
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float s2 = __shfl_xor_sync(FULL, sum[j], d), e2 = __shfl_xor_sync(FULL, err[j], d);
            float e = __fadd_rn(err[j], e2);
            two_sum_acc(sum[j], e, s2);
            err[j] = e;
        }
    }
    if ((warp & 1) && lane == 0) {   // the second warp of c: slices 32 .. 63
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s_hi[c][j] = sum[j];
            s_hi[c][4 + j] = err[j];
        }
    }
    __syncthreads();
    if (!(warp & 1) && lane < 4) {
        const int j = lane;
        float sj = j == 0 ? sum[0] : j == 1 ? sum[1] : j == 2 ? sum[2] : sum[3];
        float ej = j == 0 ? err[0] : j == 1 ? err[1] : j == 2 ? err[2] : err[3];
        ej = __fadd_rn(ej, s_hi[c][4 + j]);
        two_sum_acc(sj, ej, s_hi[c][j]);
        const int o = 4 * c + j;
        if (o < nout) W[o / NSTAT][W_S + o % NSTAT] = __dadd_rn((double)sj, (double)ej);
    }
    return true;
}

// M-step (the standard full-covariance update) from shifted statistics:
//   N_b = S0 + 10 eps; with v = y = P'(x - s_b) (E-step partials, whitened) or
//   v = d = x - s_b (one-hot KInit statistics): vbar = S1 / N_b and the centred
//   second moment C = S2 / N_b - vbar vbar^T (S1 = N_b vbar); mu = s + M vbar and
//   Sigma = M C M^T + reg I with M = P'^-1 (whitened) or M = I (one-hot).  The
//   weight N_b is normalised by sum_a N_a where it is used (E-step reference,
//   model output).
struct FinArgs {
    const float* partials;     // [grid][k][NSTAT], or nullptr (then stats64)
    int grid;
    const double* llp;
    const double* stats64;
    float4* shift4;
    int k;
    int64_t n;
    double reg, tol;
    double* model64;
    float* params;
    double* trace;
    DeviceState* st;
    int iter, em;
    int ll_count;   // log-likelihood partials to sum (grid when 0)
    int do_ll;      // this launch's block 0 does the log-likelihood / convergence step
    const int* perm;   // slot b holds the caller's component perm[b] (nullptr: b)
    // point-stationary E-step: partial rows per block of points ([grid rows][pairs]
    // [2 NSTAT]), a pair's values valid only where the row's live mask ([nwords]
    // [grid rows]) has the pair's bit
    const uint32_t* masks;
    int nwords;
    // a single fit's CTA order: the launch's last block ranks the E-step's cta_grid
    // CTAs by cta_key into cta_perm[(iter & 1) * cta_grid ..] for iteration iter + 2
    const uint8_t* cta_key = nullptr;
    int* cta_perm = nullptr;
    int cta_grid = 0;
};

__device__ __forceinline__ int sym_i(int u) { return u < 3 ? 0 : (u < 5 ? 1 : 2); }   // (00,01,02,11,12,22)
__device__ __forceinline__ int sym_j(int u) { return u < 3 ? u : (u < 5 ? u - 2 : 2); }
__device__ __forceinline__ double dneg(double x) {   // sign flip on the integer pipe
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// The M-step and the parameter build of components b0 + h (h = 0, 1) by one
// warp: lanes 16 h .. 16 h + 15 take component b0 + h, and each stage computes
// its entries in parallel lanes, every entry by a fixed sequence of binary64
// operations (GB300 issues one binary64 warp instruction every 64 cycles per
// warp, whatever the number of active lanes, so a stage costs what one entry
// costs).  W[h][W_S ..] holds the statistics; pre is this lane's binary32 P'
// entry (l < 6) or shift coordinate (6 <= l < 9), loaded at the kernel's start.
__device__ void finalize_update_warp(const FinArgs& f, int b0, int nb, float pre, double (*W)[FW], float (*F)[FF]) {
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15;
    const int b = b0 + h;
    const bool on = h < nb;
    double* w = W[h];
    const bool white = f.partials != nullptr;
    if (on && l < 9) w[W_QS + l] = (double)pre;
    __syncwarp();
    const double nbw = __dadd_rn(w[W_S], 10.0 * DBL_EPSILON);
    // the reciprocals of q00, q11, q22 (the diagonal of M) and of N_b
    if (on && l < 4) {
        const double x = l == 3 ? nbw : (white ? w[W_QS + (l == 0 ? 0 : (l == 1 ? 2 : 5))] : 1.0);
        w[W_R + l] = __drcp_rn(x);
    }
    __syncwarp();
    const double inv = w[W_R + 3];
    // vbar = S1 / N_b (l < 3); m10 = -q10 m00 m11 (l == 3), m21 = -q21 m11 m22 (l == 4)
    if (on && l < 5) {
        double A, B, C;
        if (l < 3) {
            A = w[W_S + 1 + l]; B = inv; C = 1.0;
        } else {
            const int j = l - 3;
            A = dneg(w[W_QS + (j == 0 ? 1 : 4)]); B = w[W_R + j]; C = w[W_R + j + 1];
        }
        w[W_T + l] = __dmul_rn(__dmul_rn(A, B), C);
    }
    __syncwarp();
    // C = S2 / N_b - vbar vbar^T (l < 6), m20 = -(q20 m00 + q21 m10) m22 (l == 6);
    // lanes 7 .. 14 place the other entries of M
    if (on && l < 7) {
        const int i = sym_i(l < 6 ? l : 0), j = sym_j(l < 6 ? l : 0);
        double A0, B0, A1, B1, C;
        if (l < 6) {
            A0 = w[W_S + 4 + l]; B0 = inv; A1 = dneg(w[W_T + i]); B1 = w[W_T + j]; C = 1.0;
        } else {
            A0 = w[W_QS + 3]; B0 = w[W_R + 0]; A1 = w[W_QS + 4]; B1 = w[W_T + 3]; C = dneg(w[W_R + 2]);
        }
        const double v = __dmul_rn(__fma_rn(A1, B1, __dmul_rn(A0, B0)), C);
        if (l < 6) {
            w[W_CY + 3 * i + j] = v;
            w[W_CY + 3 * j + i] = v;
        } else {
            w[W_M + 6] = white ? v : 0.0;
        }
    } else if (on && l < 15) {
        const int e = l - 7 + (l >= 13 ? 1 : 0);   // 0 .. 5, 7, 8
        double v;
        if (!white) v = (e == 0 || e == 4 || e == 8) ? 1.0 : 0.0;
        else v = e == 0 ? w[W_R + 0] : e == 3 ? w[W_T + 3] : e == 4 ? w[W_R + 1] : e == 7 ? w[W_T + 4]
                                     : e == 8 ? w[W_R + 2] : 0.0;
        w[W_M + e] = v;
    }
    __syncwarp();
    // mu = s + M vbar (l < 3); M C (3 <= l < 12)
    if (on && l < 12) {
        const int i = l < 3 ? l : (l - 3) / 3, j = l < 3 ? 0 : (l - 3) % 3;
        const int bs = l < 3 ? 1 : 3;
        const double* Bv = l < 3 ? w + W_T : w + W_CY + j;
        const double* Mi = w + W_M + 3 * i;
        const double c0 = l < 3 ? w[W_QS + 6 + l] : 0.0;
        const double v = __fma_rn(Mi[2], Bv[2 * bs], __fma_rn(Mi[1], Bv[bs], __fma_rn(Mi[0], Bv[0], c0)));
        if (l < 3) w[W_MU + l] = v;
        else w[W_MC + l - 3] = v;
    }
    __syncwarp();
    // Sigma = M C M^T + reg I (l < 6)
    if (on && l < 6) {
        const int i = sym_i(l), j = sym_j(l);
        const double* a = w + W_MC + 3 * i;
        const double* m = w + W_M + 3 * j;
        w[W_C + l] = __fma_rn(a[2], m[2], __fma_rn(a[1], m[1], __fma_rn(a[0], m[0], i == j ? f.reg : 0.0)));
    }
    __syncwarp();
    // the parameters (the scalar build_component's helpers, entries in parallel lanes)
    double c[6], mu[3];
    for (int e = 0; e < 6; ++e) c[e] = w[W_C + e];
    for (int i = 0; i < 3; ++i) mu[i] = w[W_MU + i];
    const CholInv k = chol_inv(c);
    const bool ok = on && k.pd;
    if (on && !k.pd && l == 0) {
        atomicMin(&f.st->bad_component, f.perm ? f.perm[b] : b);
        set_error(f.st, GIRA_ERR_NOT_PD);
    }
    if (ok && l < MODEL) {
        double* m = f.model64 + (size_t)b * MODEL;
        m[l] = l == 0 ? nbw : (l < 4 ? w[W_MU + l - 1] : w[W_C + l - 4]);
    }
    if (ok && l < 6) w[W_QS + l] = chol_q(k, l);
    __syncwarp();
    if (ok && l < 3) {
        const double* qq = w + W_QS;
        const double a0 = l == 0 ? qq[0] : (l == 1 ? qq[1] : qq[3]);
        const double a1 = l == 0 ? 0.0 : (l == 1 ? qq[2] : qq[4]);
        const double a2 = l == 2 ? qq[5] : 0.0;
        w[W_QS + 6 + l] = bias_row(a0, a1, a2, mu);
    }
    const float cc = log2_norm(nbw, k);
    __syncwarp();
    // binary32 copies: P'[6] and b[3] (W_QS ..), mu[3], w, Sigma[6]
    float* fc = F[h];
    if (ok) {
        for (int e = l; e < FF - 1; e += 16)
            fc[e] = (float)(e < 9 ? w[W_QS + e] : (e < 12 ? w[W_MU + e - 9] : (e == 12 ? nbw : w[W_C + e - 13])));
    }
    __syncwarp();
    if (ok) {
        float* base = f.params + (size_t)(b >> 1) * PAIR_FLOATS + (b & 1);
        static_assert(SLOT_B == SLOT_P + 6, "P' and b are consecutive slots");
        if (l < 9) base[2 * (SLOT_P + l)] = fc[l];
        else if (l == 9) base[2 * SLOT_C] = cc;
        else if (l < 13) base[2 * (SLOT_NMU + l - 10)] = -fc[l - 1];
        else if (l == 13) base[2 * SLOT_W] = fc[12];
        else if (l == 14) base[2 * SLOT_S] = sigma_min_sq_bound(fc + 13);
        else f.shift4[b] = make_float4(fc[9], fc[10], fc[11], 0.f);
    }
}

// Components blk * FIN_CPB .. of one fit; block index blk == 0 also does the
// log-likelihood, trace and convergence of an EM iteration.
__device__ void reduce_finalize_body(const FinArgs& f, int blk) {
    __shared__ double W[FIN_CPB][FW];
    __shared__ float F[FIN_CPB][FF];
    __shared__ int s_skip;
    static_assert(FIN_CPB == 2, "one half-warp per component in the update");
    const int t = threadIdx.x;
    const int b0 = blk * FIN_CPB;
    const int nb = min(FIN_CPB, f.k - b0);
    const int nout = nb * NSTAT;
    float pre = 0.f;   // warp 0: this lane's binary32 P' entry or shift coordinate, loaded early
    if (t < 32) {
        const int h = t >> 4, l = t & 15, b = b0 + h;
        if (h < nb && l < 9) {
            if (l < 6) {
                pre = f.partials ? f.params[(size_t)(b >> 1) * PAIR_FLOATS + (b & 1) + 2 * (SLOT_P + l)] : 0.f;
            } else {
                const float4 sh = f.shift4[b];
                pre = l == 6 ? sh.x : (l == 7 ? sh.y : sh.z);
            }
        }
    }
    if (t == 0) s_skip = (f.em && f.iter > f.st->stop_after) || f.st->error != 0;
    if (f.partials && f.masks) {
        if (!reduce_partials_masked(f.partials, f.grid, pt_row_floats(f.k), f.masks, b0, nout, W, &s_skip, f.st))
            return;
    } else {
        __syncthreads();
        if (s_skip) return;
        if (f.partials) {
            __shared__ double part[FIN_SPLIT_CTA][FIN_CPB * NSTAT];
            __shared__ double S[FIN_CPB * NSTAT];
            reduce_partials(f.partials, f.grid, f.k, b0, nout, part, S);
            if (t < nout) W[t / NSTAT][W_S + t % NSTAT] = S[t];
        } else if (t < nout) {
            W[t / NSTAT][W_S + t % NSTAT] = f.stats64[(size_t)b0 * NSTAT + t];
        }
    }
    __syncthreads();
    if (t < 32) {
        finalize_update_warp(f, b0, nb, pre, W, F);
        if (t == 0 && b0 == 0) f.st->w_raw = 1;
    }
    if (f.em && f.do_ll && blk == 0 && t >= 32) {   // warps 1 ..: log-likelihood, trace, convergence
        __shared__ double s_llw[FIN_THREADS / 32];
        const int lane = t & 31, w = t >> 5;
        double v = 0.0;
        const int nll = f.ll_count ? f.ll_count : f.grid;
        for (int c = t - 32; c < nll; c += FIN_THREADS - 32) v += f.llp[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0) s_llw[w] = v;
        asm volatile("bar.sync 1, %0;" ::"n"(FIN_THREADS - 32) : "memory");   // warps 1 .. only
        if (t == 32) {
            v = 0.0;
            for (int u = 1; u < FIN_THREADS / 32; ++u) v += s_llw[u];
            DeviceState* st = f.st;
            st->ll_sum = v;
            const double ll = v / (double)f.n;
            f.trace[f.iter - 1] = ll;
            if (f.iter > 1 && fabs(ll - st->prev_ll) < f.tol) st->stop_after = f.iter;
            st->prev_ll = ll;
            st->iters_done = f.iter;
        }
    }
}

// The E-step's CTA order for iteration f.iter + 2: descending work key, ties in
// index order (a counting sort: position = keys above + equal keys before).  The
// order changes only which SM runs which point blocks when, never a result.
__device__ void order_ctas(const FinArgs& f) {
    __shared__ int s_above[256], s_run[256];
    __shared__ uint16_t s_wc[FIN_THREADS / 32][256];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int grid = f.cta_grid;
    int* out = f.cta_perm + (size_t)(f.iter & 1) * grid;
    for (int b = t; b < 256; b += FIN_THREADS) s_above[b] = s_run[b] = 0;
    __syncthreads();
    for (int i = t; i < grid; i += FIN_THREADS) atomicAdd(&s_above[f.cta_key[i]], 1);
    __syncthreads();
    if (warp == 0) {   // s_above[b] = number of keys above b (8 buckets per lane, from the top)
        int v[8], tot = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            v[u] = s_above[255 - (lane * 8 + u)];
            tot += v[u];
        }
        int incl = tot;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int x = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += x;
        }
        __syncwarp();
        int run = incl - tot;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            s_above[255 - (lane * 8 + u)] = run;
            run += v[u];
        }
    }
    __syncthreads();
    for (int c0 = 0; c0 < grid; c0 += FIN_THREADS) {
        const int i = c0 + t;
        const int key = i < grid ? (int)f.cta_key[i] : -1;
        const unsigned peers = __match_any_sync(FULL, key);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        for (int b = lane; b < 256; b += 32) s_wc[warp][b] = 0;
        __syncwarp();
        if (key >= 0 && rank == 0) s_wc[warp][key] = (uint16_t)__popc(peers);
        __syncthreads();
        if (key >= 0) {
            int pos = s_above[key] + s_run[key] + rank;
            for (int w = 0; w < warp; ++w) pos += s_wc[w][key];
            if (GIRA_IN(pos < grid, f.st)) out[pos] = i;
        }
        __syncthreads();
        for (int b = t; b < 256; b += FIN_THREADS) {
            int add = 0;
            for (int w = 0; w < FIN_THREADS / 32; ++w) add += s_wc[w][b];
            s_run[b] += add;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(FIN_THREADS) reduce_finalize_kernel(const FinArgs f) {
    pdl_wait();         // the E-step's partials (dependent launch)
    pdl_allow_next();   // the next E-step may stage its points meanwhile
    if (f.cta_key && blockIdx.x == gridDim.x - 1) {
        order_ctas(f);
        return;
    }
    reduce_finalize_body(f, blockIdx.x);
}

// Every instance of a batch: block (instance i, index j) finalizes components
// j * FIN_CPB .. of instance i from its own partials, into its own state.
// shared: the entries are chunks of one fit (state, trace and log-likelihood
// partials shared; the log-likelihood step runs in the block of (0, 0)).
__global__ void __launch_bounds__(FIN_THREADS) reduce_finalize_batched_kernel(const FinArgs base,
                                                                              const BatchInst* __restrict__ insts,
                                                                              const int2* __restrict__ blocks,
                                                                              DeviceState* states, int iters,
                                                                              int shared) {
    const int2 bi = blocks[blockIdx.x];
    const BatchInst I = insts[bi.x];
    FinArgs f = base;
    f.partials = base.partials ? base.partials + I.part_off : nullptr;
    f.grid = I.ctas;
    if (shared) {
        f.stats64 = base.stats64 ? base.stats64 + (size_t)I.comp_off * NSTAT : nullptr;
        f.shift4 = base.shift4 + I.comp_off;
        f.k = I.k;
        f.n = I.n;
        f.model64 = base.model64 + (size_t)I.comp_off * MODEL;
        f.params = base.params + I.par_off;
        f.perm = base.perm ? base.perm + I.comp_off : nullptr;
        f.st = states;
        f.do_ll = (bi.x == 0);
        reduce_finalize_body(f, bi.y);
        return;
    }
    f.llp = base.llp ? base.llp + I.ll_off : nullptr;
    f.perm = base.perm ? base.perm + I.comp_off : nullptr;
    if (base.masks) {   // point-stationary E-step: per-warp rows, live masks, one ll slot per CTA
        f.masks = base.masks + I.mask_off;
        f.grid = I.ctas * PT_B;
        f.ll_count = I.ctas;
    }
    f.stats64 = base.stats64 ? base.stats64 + (size_t)I.comp_off * NSTAT : nullptr;
    f.shift4 = base.shift4 + I.comp_off;
    f.k = I.k;
    f.n = I.n;
    f.model64 = base.model64 + (size_t)I.comp_off * MODEL;
    f.params = base.params + I.par_off;
    f.trace = base.trace + (size_t)bi.x * iters;
    f.st = states + bi.x;
    reduce_finalize_body(f, bi.y);
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
    build_component(b, pi, m, c, params, shift4, model64, st, b);
}

// ------------------------------------------------------------------ batched helpers
__global__ void params_from_model_batched_kernel(const float* __restrict__ w, const float* __restrict__ mu,
                                                 const float* __restrict__ cov, int total_k,
                                                 const int* __restrict__ comp_inst,
                                                 const BatchInst* __restrict__ insts, double* model64, float* params,
                                                 float4* shift4, DeviceState* states) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;   // global component
    if (g >= total_k) return;
    const int i = comp_inst[g];
    const BatchInst I = insts[i];
    const int b = g - I.comp_off;
    DeviceState* st = states + i;
    const double pi = w[g];
    const double m[3] = {mu[3 * (size_t)g], mu[3 * (size_t)g + 1], mu[3 * (size_t)g + 2]};
    const float* S = cov + 9 * (size_t)g;
    const double c[6] = {S[0], S[3], S[6], S[4], S[7], S[8]};
    bool fin = isfinite(pi) && isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]);
    for (int q = 0; q < 9; ++q) fin = fin && isfinite(S[q]);
    if (!fin) { set_error(st, GIRA_ERR_NONFINITE_INPUT); return; }
    if (!(pi > 0.0)) { set_error(st, GIRA_ERR_INVALID_ARG); return; }
    build_component(b, pi, m, c, params + I.par_off, shift4 + I.comp_off, model64 + (size_t)I.comp_off * MODEL, st,
                    b);
}

__global__ void model_out_batched_kernel(const double* __restrict__ model64, const BatchInst* __restrict__ insts,
                                         float* w, float* mu, float* cov, const DeviceState* states,
                                         const int* __restrict__ perm) {
    __shared__ double s_part[2];
    const BatchInst I = insts[blockIdx.x];
    const DeviceState* st = states + blockIdx.x;
    const double* M = model64 + (size_t)I.comp_off * MODEL;
    double part = 0.0;
    for (int a = threadIdx.x; a < I.k; a += blockDim.x) part += M[(size_t)a * MODEL];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    const double nsum = s_part[0] + s_part[1];
    if (st->error) return;
    for (int sl = threadIdx.x; sl < I.k; sl += blockDim.x) {   // slot; the caller's index is perm[slot]
        const double* m = M + (size_t)sl * MODEL;
        const size_t g = (size_t)I.comp_off + (perm ? perm[I.comp_off + sl] : sl);
        w[g] = (float)(st->w_raw ? m[0] / nsum : m[0]);
        for (int q = 0; q < 3; ++q) mu[3 * g + q] = (float)m[1 + q];
        const int idx[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
        for (int q = 0; q < 9; ++q) cov[9 * g + q] = (float)m[4 + idx[q]];
    }
}

__global__ void model_out_kernel(const double* __restrict__ model64, int k, float* w, float* mu, float* cov,
                                 const DeviceState* st, const int* __restrict__ perm) {
    __shared__ double s_part[2];
    // after an M-step the stored weights are N_b: pi_b = N_b / sum_a N_a (fixed order)
    double part = 0.0;
    for (int a = threadIdx.x; a < k; a += blockDim.x) part += model64[(size_t)a * MODEL];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    const double nsum = s_part[0] + s_part[1];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;   // slot; the caller's index is perm[s]
    if (s >= k) return;
    const int b = perm ? perm[s] : s;
    if (!GIRA_IN(b >= 0 && b < k, const_cast<DeviceState*>(st))) return;
    const double* m = model64 + (size_t)s * MODEL;
    w[b] = (float)(st->w_raw ? m[0] / nsum : m[0]);
    for (int i = 0; i < 3; ++i) mu[3 * (size_t)b + i] = (float)m[1 + i];
    const int idx[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    for (int i = 0; i < 9; ++i) cov[9 * (size_t)b + i] = (float)m[4 + idx[i]];
}

// Components in the order of a space-filling curve of their means: the Morton
// code (10 bits per axis over the means' bounding box, binary32) with the index
// as the low bits, sorted by one block (bitonic network in shared memory).
// Slot s then takes the component perm[s]: its row of `old` (a copy of model64)
// is rebuilt into slot s of model64, params and shift4.  Only the order of the
// components in the fit changes: the E-step's per-point sums see them in
// another order, and nothing else.
__device__ __forceinline__ unsigned spread10(unsigned v) {   // bit i -> bit 3 i
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// insts (batched fits): block i orders instance i (its own k, offsets and state).
__global__ void __launch_bounds__(ORDER_THREADS) order_components_kernel(const double* __restrict__ old, int k,
                                                                        int kp2, int* perm, double* model64,
                                                                        float* params, float4* shift4,
                                                                        DeviceState* st,
                                                                        const BatchInst* __restrict__ insts) {
    extern __shared__ unsigned long long keys[];   // kp2 = power of two >= k
    __shared__ float s_lo[3][32], s_hi[3][32];
    if (insts) {
        const BatchInst I = insts[blockIdx.x];
        k = I.k;
        old += (size_t)I.comp_off * MODEL;
        model64 += (size_t)I.comp_off * MODEL;
        perm += I.comp_off;
        params += I.par_off;
        shift4 += I.comp_off;
        st += blockIdx.x;
        kp2 = 1;
        while (kp2 < k) kp2 <<= 1;
    }
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // binary32 (the order only needs coarse cells; rounding to binary32 keeps min and max)
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = t; b < k; b += blockDim.x)
        for (int i = 0; i < 3; ++i) {
            const float v = (float)old[(size_t)b * MODEL + 1 + i];
            lo[i] = fminf(lo[i], v);
            hi[i] = fmaxf(hi[i], v);
        }
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[i] = fminf(lo[i], __shfl_xor_sync(FULL, lo[i], o));
            hi[i] = fmaxf(hi[i], __shfl_xor_sync(FULL, hi[i], o));
        }
        if (lane == 0) {
            s_lo[i][warp] = lo[i];
            s_hi[i][warp] = hi[i];
        }
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    float scale[3];
    for (int i = 0; i < 3; ++i) {
        lo[i] = s_lo[i][0];
        hi[i] = s_hi[i][0];
        for (int w = 1; w < nw; ++w) {
            lo[i] = fminf(lo[i], s_lo[i][w]);
            hi[i] = fmaxf(hi[i], s_hi[i][w]);
        }
        scale[i] = hi[i] > lo[i] ? 1024.f / (hi[i] - lo[i]) : 0.f;
    }
    for (int b = t; b < kp2; b += blockDim.x) {
        unsigned long long key = ~0ull;
        if (b < k) {
            unsigned code = 0;
            for (int i = 0; i < 3; ++i) {
                const float u = ((float)old[(size_t)b * MODEL + 1 + i] - lo[i]) * scale[i];
                const unsigned q = (unsigned)fminf(1023.f, fmaxf(0.f, floorf(u)));
                code |= spread10(q) << i;
            }
            key = ((unsigned long long)code << 32) | (unsigned)b;
        }
        keys[b] = key;
    }
    __syncthreads();
    for (int size = 2; size <= kp2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = t; i < kp2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const unsigned long long a = keys[i], c = keys[j];
                    const bool up = (i & size) == 0;
                    if ((a > c) == up) {
                        keys[i] = c;
                        keys[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int slot = t; slot < k; slot += blockDim.x) perm[slot] = (int)(keys[slot] & 0xffffffffu);
}

// Slot s of every fit takes component perm[s]: its row of `old` rebuilt into slot s
// of model64, params and shift4 (one thread per slot; insts / comp_inst: batched).
__global__ void rebuild_components_kernel(const double* __restrict__ old, const int* __restrict__ perm, int total_k,
                                          double* model64, float* params, float4* shift4, DeviceState* st,
                                          const BatchInst* __restrict__ insts, const int* __restrict__ comp_inst) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total_k) return;
    int slot = g;
    if (insts) {
        const int i = comp_inst[g];
        const BatchInst I = insts[i];
        slot = g - I.comp_off;
        old += (size_t)I.comp_off * MODEL;
        model64 += (size_t)I.comp_off * MODEL;
        params += I.par_off;
        shift4 += I.comp_off;
        st += i;
    }
    const int b = perm[g];
    if (!GIRA_IN(b >= 0 && b < (insts ? insts[comp_inst[g]].k : total_k), st)) return;
    const double* r = old + (size_t)b * MODEL;
    build_component(slot, r[0], r + 1, r + 4, params, shift4, model64, st, b);
}

// ------------------------------------------------------------------ differentiable log-likelihood
// x' = R x + t in binary32 (fixed order), stored as (x,x,y,y)(z,z,0,0).
__global__ void pack_pose_kernel(const float* __restrict__ p3, int64_t n, const float* __restrict__ pose,
                                 float4* __restrict__ p8, DeviceState* st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = p3[3 * i], y = p3[3 * i + 1], z = p3[3 * i + 2];
    float o[3] = {x, y, z};
    if (pose) {
#pragma unroll
        for (int r = 0; r < 3; ++r) o[r] = fmaf(pose[3 * r + 2], z, fmaf(pose[3 * r + 1], y, pose[3 * r] * x)) + pose[9 + r];
    }
    if (!(isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2]))) set_error(st, GIRA_ERR_NONFINITE_INPUT);
    p8[2 * i] = make_float4(o[0], o[0], o[1], o[1]);
    p8[2 * i + 1] = make_float4(o[2], o[2], 0.f, 0.f);
}

// Every point of a batch of scans: x' = R_i x + t_i with the pose of its scan
// (binary search over the offsets); flags non-finite input on its instance.
__global__ void pack_pose_batched_kernel(const float* __restrict__ p3, int64_t n, const int64_t* __restrict__ offsets,
                                         int batch, const float* __restrict__ poses, float4* __restrict__ p8,
                                         DeviceState* states) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = batch;   // offsets[lo] <= i < offsets[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offsets[mid] <= i) lo = mid; else hi = mid;
    }
    const float* pose = poses ? poses + 12 * (size_t)lo : nullptr;
    const float x = p3[3 * i], y = p3[3 * i + 1], z = p3[3 * i + 2];
    float o[3] = {x, y, z};
    if (pose) {
#pragma unroll
        for (int r = 0; r < 3; ++r) o[r] = fmaf(pose[3 * r + 2], z, fmaf(pose[3 * r + 1], y, pose[3 * r] * x)) + pose[9 + r];
    }
    if (!(isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2]))) set_error(states + lo, GIRA_ERR_NONFINITE_INPUT);
    p8[2 * i] = make_float4(o[0], o[0], o[1], o[1]);
    p8[2 * i + 1] = make_float4(o[2], o[2], 0.f, 0.f);
}

// One block: pi = softmax(logits) in binary64 (max, then fixed-order sums),
// Sigma_b = L_b L_b^T, then the M-step's binary64 build of the E-step
// parameters.  A non-positive diagonal entry of L_b is GIRA_ERR_NOT_PD.
constexpr int PFC_THREADS = 256;
__device__ void params_from_chol_body(const float* __restrict__ logits, const float* __restrict__ mu,
                                      const float* __restrict__ chol, int k, double* model64, float* params,
                                      float4* shift4, DeviceState* st);
__global__ void __launch_bounds__(PFC_THREADS) params_from_chol_kernel(const float* __restrict__ logits,
                                                                       const float* __restrict__ mu,
                                                                       const float* __restrict__ chol, int k,
                                                                       double* model64, float* params,
                                                                       float4* shift4, DeviceState* st) {
    params_from_chol_body(logits, mu, chol, k, model64, params, shift4, st);
}
// One block per instance of a batch.
__global__ void __launch_bounds__(PFC_THREADS) params_from_chol_batched_kernel(
    const float* __restrict__ logits, const float* __restrict__ mu, const float* __restrict__ chol,
    const BatchInst* __restrict__ insts, double* model64, float* params, float4* shift4, DeviceState* states) {
    const BatchInst I = insts[blockIdx.x];
    const size_t c = I.comp_off;
    params_from_chol_body(logits + c, mu + 3 * c, chol + 9 * c, I.k, model64 + c * MODEL, params + I.par_off,
                          shift4 + c, states + blockIdx.x);
}
__device__ void params_from_chol_body(const float* __restrict__ logits, const float* __restrict__ mu,
                                      const float* __restrict__ chol, int k, double* model64, float* params,
                                      float4* shift4, DeviceState* st) {
    __shared__ double s_red[PFC_THREADS / 32];
    __shared__ double s_max, s_lz;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    bool fin = true;
    double m = -INFINITY;
    for (int b = t; b < k; b += PFC_THREADS) {
        fin = fin && isfinite(logits[b]);
        m = fmax(m, (double)logits[b]);
    }
    if (!fin) set_error(st, GIRA_ERR_NONFINITE_INPUT);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(FULL, m, o));
    if (lane == 0) s_red[warp] = m;
    __syncthreads();
    if (t == 0) {
        double v = s_red[0];
        for (int w = 1; w < PFC_THREADS / 32; ++w) v = fmax(v, s_red[w]);
        s_max = v;
    }
    __syncthreads();
    const double amax = s_max;
    double z = 0.0;
    for (int b = t; b < k; b += PFC_THREADS) z += exp((double)logits[b] - amax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(FULL, z, o);
    __syncthreads();
    if (lane == 0) s_red[warp] = z;
    __syncthreads();
    if (t == 0) {
        double v = 0.0;
        for (int w = 0; w < PFC_THREADS / 32; ++w) v += s_red[w];
        s_lz = amax + log(v);
    }
    __syncthreads();
    const double lz = s_lz;
    for (int b = t; b < k; b += PFC_THREADS) {
        const float* L = chol + 9 * (size_t)b;
        const double m3[3] = {mu[3 * b], mu[3 * b + 1], mu[3 * b + 2]};
        bool ok = isfinite(m3[0]) && isfinite(m3[1]) && isfinite(m3[2]);
        const double L00 = L[0], L10 = L[3], L11 = L[4], L20 = L[6], L21 = L[7], L22 = L[8];
        ok = ok && isfinite(L00) && isfinite(L10) && isfinite(L11) && isfinite(L20) && isfinite(L21) && isfinite(L22);
        if (!ok) {
            set_error(st, GIRA_ERR_NONFINITE_INPUT);
            continue;
        }
        if (!(L00 > 0.0 && L11 > 0.0 && L22 > 0.0)) {
            atomicMin(&st->bad_component, b);
            set_error(st, GIRA_ERR_NOT_PD);
            continue;
        }
        const double c[6] = {L00 * L00, L00 * L10, L00 * L20, L10 * L10 + L11 * L11, L10 * L20 + L11 * L21,
                             L20 * L20 + L21 * L21 + L22 * L22};
        build_component(b, exp((double)logits[b] - lz), m3, c, params, shift4, model64, st, b);
    }
}

// Parameter gradients from the statistics about mu_b (d = x' - mu_b):
//   dL/dmu_b    = Sigma^{-1} S1 = P^T P S1
//   dL/dL_b     = lower(P^T (P S2 P^T) - S0 diag(1/L_ii))
//   dL/dalpha_b = S0 - N pi_b
// with P = L_b^{-1}; block 0 also sums the log-likelihood and the twist.
struct GradFinArgs {
    const float* partials;
    int grid;
    const double* llp;
    const double* pp;
    const float* pose;
    const float* chol;
    const double* model64;
    int k;
    int64_t n;
    float *g_logits, *g_means, *g_chol;
    double *g_pose, *g_twist;
    DeviceState* st;
};
__device__ void grad_finalize_body(const GradFinArgs& f, int blk);
__global__ void __launch_bounds__(FIN_THREADS) grad_finalize_kernel(const GradFinArgs f) {
    grad_finalize_body(f, blockIdx.x);
}
// Block (instance i, index j) of a batch: components j * FIN_CPB .. of instance i.
__global__ void __launch_bounds__(FIN_THREADS) grad_finalize_batched_kernel(const GradFinArgs base,
                                                                           const BatchInst* __restrict__ insts,
                                                                           const int2* __restrict__ blocks,
                                                                           DeviceState* states) {
    const int2 bi = blocks[blockIdx.x];
    const BatchInst I = insts[bi.x];
    const size_t c = I.comp_off;
    GradFinArgs f = base;
    f.partials = base.partials + I.part_off;
    f.grid = I.ctas;
    f.llp = base.llp + I.ll_off;
    f.pp = base.pp + 12 * I.ll_off;
    f.pose = base.pose ? base.pose + 12 * (size_t)bi.x : nullptr;
    f.chol = base.chol + 9 * c;
    f.model64 = base.model64 + c * MODEL;
    f.k = I.k;
    f.n = I.n;
    f.g_logits = base.g_logits ? base.g_logits + c : nullptr;
    f.g_means = base.g_means ? base.g_means + 3 * c : nullptr;
    f.g_chol = base.g_chol ? base.g_chol + 9 * c : nullptr;
    f.g_pose = base.g_pose ? base.g_pose + 12 * (size_t)bi.x : nullptr;
    f.g_twist = base.g_twist ? base.g_twist + 6 * (size_t)bi.x : nullptr;
    f.st = states + bi.x;
    grad_finalize_body(f, bi.y);
}
__device__ void grad_finalize_body(const GradFinArgs& f, int blk) {
    __shared__ double part[FIN_SPLIT_CTA][FIN_CPB * NSTAT];
    __shared__ double S[FIN_CPB * NSTAT];
    __shared__ int s_skip;
    const float* __restrict__ partials = f.partials;
    const int grid = f.grid;
    const double* __restrict__ llp = f.llp;
    const double* __restrict__ pp = f.pp;
    const float* __restrict__ pose = f.pose;
    const float* __restrict__ chol = f.chol;
    const double* __restrict__ model64 = f.model64;
    const int k = f.k;
    const int64_t n = f.n;
    float* g_logits = f.g_logits;
    float* g_means = f.g_means;
    float* g_chol = f.g_chol;
    double* g_pose = f.g_pose;
    double* g_twist = f.g_twist;
    DeviceState* st = f.st;
    if (threadIdx.x == 0) s_skip = st->error != 0;
    __syncthreads();
    if (s_skip) return;
    const int t = threadIdx.x;
    const int b0 = blk * FIN_CPB;
    const int nb = min(FIN_CPB, k - b0);
    reduce_partials(partials, grid, k, b0, nb * NSTAT, part, S);
    __syncthreads();
    if (t < nb) {
        const int b = b0 + t;
        const double* Sb = S + t * NSTAT;
        const float* L = chol + 9 * (size_t)b;
        const double L00 = L[0], L10 = L[3], L11 = L[4], L20 = L[6], L21 = L[7], L22 = L[8];
        const double P00 = 1.0 / L00, P11 = 1.0 / L11, P22 = 1.0 / L22;
        const double P10 = -L10 * P00 * P11, P21 = -L21 * P11 * P22, P20 = -(L20 * P00 + L21 * P10) * P22;
        const double P[3][3] = {{P00, 0.0, 0.0}, {P10, P11, 0.0}, {P20, P21, P22}};
        const double s0 = Sb[0];
        const double s1[3] = {Sb[1], Sb[2], Sb[3]};
        const double S2[3][3] = {{Sb[4], Sb[5], Sb[6]}, {Sb[5], Sb[7], Sb[8]}, {Sb[6], Sb[8], Sb[9]}};
        double u[3], gm[3];
        for (int i = 0; i < 3; ++i) u[i] = P[i][0] * s1[0] + P[i][1] * s1[1] + P[i][2] * s1[2];
        for (int i = 0; i < 3; ++i) gm[i] = P[0][i] * u[0] + P[1][i] * u[1] + P[2][i] * u[2];
        double A[3][3], M[3][3];   // A = P S2, M = A P^T
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) A[i][j] = P[i][0] * S2[0][j] + P[i][1] * S2[1][j] + P[i][2] * S2[2][j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = A[i][0] * P[j][0] + A[i][1] * P[j][1] + A[i][2] * P[j][2];
        const double Ld[3] = {L00, L11, L22};
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) {
                double v = 0.0;
                if (j <= i) {
                    v = P[0][i] * M[0][j] + P[1][i] * M[1][j] + P[2][i] * M[2][j];
                    if (i == j) v -= s0 / Ld[i];
                }
                if (g_chol) g_chol[9 * (size_t)b + 3 * i + j] = (float)v;
            }
            if (g_means) g_means[3 * (size_t)b + i] = (float)gm[i];
        }
        if (g_logits) g_logits[b] = (float)(s0 - (double)n * model64[(size_t)b * MODEL]);
    }
    if (blk == 0 && t >= 32 && t < 64) {   // warp 1: log-likelihood and pose sums, fixed order
        const int lane = t - 32;
        double v[13] = {};
        for (int c = lane; c < grid; c += 32) {
            v[0] += llp[c];
            for (int i = 0; i < 12; ++i) v[1 + i] += pp[(size_t)c * 12 + i];
        }
        for (int i = 0; i < 13; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(FULL, v[i], o);
        }
        if (lane == 0) {
            st->ll_sum = v[0];
            const double* M = v + 1;    // sum g x'^T
            const double* G = v + 10;   // sum g
            if (g_twist) {   // omega = sum x' x g, v = sum g
                g_twist[0] = M[3 * 2 + 1] - M[3 * 1 + 2];
                g_twist[1] = M[3 * 0 + 2] - M[3 * 2 + 0];
                g_twist[2] = M[3 * 1 + 0] - M[3 * 0 + 1];
                for (int i = 0; i < 3; ++i) g_twist[3 + i] = G[i];
            }
            if (g_pose) {    // x = R^T (x' - t): dL/dR = (sum g x'^T - G t^T) R, dL/dt = G
                const double tt[3] = {pose ? pose[9] : 0.0, pose ? pose[10] : 0.0, pose ? pose[11] : 0.0};
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double acc = 0.0;
                        for (int m = 0; m < 3; ++m) {
                            const double Rmj = pose ? (double)pose[3 * m + j] : (m == j ? 1.0 : 0.0);
                            acc += (M[3 * i + m] - G[i] * tt[m]) * Rmj;
                        }
                        g_pose[3 * i + j] = acc;
                    }
                for (int i = 0; i < 3; ++i) g_pose[9 + i] = G[i];
            }
        }
    }
}
}  // namespace

cudaError_t launch_reduce_finalize(const float* partials, int grid, const double* ll_partials,
                                   const double* stats64, float4* shift4, int k, int64_t n, double reg, double tol,
                                   double* model64, float* params, double* trace, DeviceState* st, int iter, bool em,
                                   cudaStream_t s, bool pdl, const int* perm, const uint32_t* masks, int nwords,
                                   int ll_count, const uint8_t* cta_key, int* cta_perm, int cta_grid) {
    FinArgs f{partials, grid, ll_partials, stats64, shift4, k, n, reg, tol, model64, params, trace, st, iter,
              em ? 1 : 0, ll_count, 1, perm, masks, nwords};
    const bool order = em && cta_key && cta_perm && cta_grid > 0;
    if (order) {
        f.cta_key = cta_key;
        f.cta_perm = cta_perm;
        f.cta_grid = cta_grid;
    }
    PdlConfig c(dim3((k + FIN_CPB - 1) / FIN_CPB + (order ? 1 : 0)), dim3(FIN_THREADS), 0, s, pdl);
    return cudaLaunchKernelEx(&c.cfg, reduce_finalize_kernel, f);
}

int fin_components_per_block() { return FIN_CPB; }

cudaError_t launch_reduce_finalize_batched(const float* partials, const double* ll_partials, const double* stats64,
                                           float4* shift4, const BatchInst* insts, const int2* blocks, int nblocks,
                                           double reg, double tol, int iters, double* model64, float* params,
                                           double* trace, DeviceState* states, int iter, bool em, cudaStream_t s,
                                           const int* perm, const uint32_t* masks) {
    const FinArgs f{partials, 0, ll_partials, stats64, shift4, 0, 0, reg, tol, model64, params, trace, nullptr,
                    iter, em ? 1 : 0, 0, 1, perm, masks, 0};
    reduce_finalize_batched_kernel<<<nblocks, FIN_THREADS, 0, s>>>(f, insts, blocks, states, std::max(iters, 1), 0);
    return cudaGetLastError();
}

cudaError_t launch_reduce_finalize_chunks(const float* partials, const double* ll_partials, int ll_count,
                                          const double* stats64, float4* shift4, const BatchInst* insts,
                                          const int2* blocks, int nblocks, int64_t n, double reg, double tol,
                                          double* model64, float* params, double* trace, DeviceState* st, int iter,
                                          bool em, cudaStream_t s, const int* perm) {
    const FinArgs f{partials, 0, ll_partials, stats64, shift4, 0, n, reg, tol, model64, params, trace, nullptr,
                    iter, em ? 1 : 0, ll_count, 1, perm};
    reduce_finalize_batched_kernel<<<nblocks, FIN_THREADS, 0, s>>>(f, insts, blocks, st, 1, 1);
    return cudaGetLastError();
}

cudaError_t launch_fill_padding_batched(float* params, const BatchInst* insts, int batch, int npairs_max,
                                        const int* npairs_of, cudaStream_t s) {
    fill_padding_batched_kernel<<<batch, 128, 0, s>>>(params, insts, npairs_of);
    return cudaGetLastError();
}

cudaError_t launch_params_from_model_batched(const float* w, const float* mu, const float* cov, int total_k,
                                             const int* comp_inst, const BatchInst* insts, double* model64,
                                             float* params, float4* shift4, DeviceState* states, cudaStream_t s) {
    params_from_model_batched_kernel<<<(total_k + 63) / 64, 64, 0, s>>>(w, mu, cov, total_k, comp_inst, insts, model64,
                                                                       params, shift4, states);
    return cudaGetLastError();
}

cudaError_t launch_model_out_batched(const double* model64, const BatchInst* insts, int batch, float* w, float* mu,
                                     float* cov, const DeviceState* states, cudaStream_t s, const int* perm) {
    model_out_batched_kernel<<<batch, 64, 0, s>>>(model64, insts, w, mu, cov, states, perm);
    return cudaGetLastError();
}

cudaError_t launch_ll_reduce_batched(const double* ll_partials, const BatchInst* insts, int batch,
                                     DeviceState* states, cudaStream_t s) {
    ll_reduce_batched_kernel<<<batch, 32, 0, s>>>(ll_partials, insts, states);
    return cudaGetLastError();
}

cudaError_t launch_params_from_model(const float* w, const float* mu, const float* cov, int k, double* model64,
                                     float* params, float4* shift4, DeviceState* st, cudaStream_t s) {
    params_from_model_kernel<<<(k + 63) / 64, 64, 0, s>>>(w, mu, cov, k, model64, params, shift4, st);
    return cudaGetLastError();
}

cudaError_t launch_model_out(const double* model64, int k, float* w, float* mu, float* cov, const DeviceState* st,
                             cudaStream_t s, const int* perm) {
    model_out_kernel<<<(k + 63) / 64, 64, 0, s>>>(model64, k, w, mu, cov, st, perm);
    return cudaGetLastError();
}

cudaError_t launch_order_components(double* model64, double* scratch, int k, int* perm, float* params,
                                    float4* shift4, DeviceState* st, cudaStream_t s) {
    if (k > ORDER_MAX_K) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(scratch, model64, sizeof(double) * (size_t)k * MODEL, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    int kp2 = 1;
    while (kp2 < k) kp2 <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)kp2;
    e = cudaFuncSetAttribute(order_components_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    order_components_kernel<<<1, ORDER_THREADS, smem, s>>>(scratch, k, kp2, perm, model64, params, shift4, st,
                                                           nullptr);
    rebuild_components_kernel<<<(k + 63) / 64, 64, 0, s>>>(scratch, perm, k, model64, params, shift4, st, nullptr,
                                                           nullptr);
    return cudaGetLastError();
}

cudaError_t launch_order_components_batched(double* model64, double* scratch, int total_k, int kmax,
                                            const BatchInst* insts, int batch, const int* comp_inst, int* perm,
                                            float* params, float4* shift4, DeviceState* states, cudaStream_t s) {
    if (kmax > ORDER_MAX_K) return cudaErrorInvalidValue;
    cudaError_t e =
        cudaMemcpyAsync(scratch, model64, sizeof(double) * (size_t)total_k * MODEL, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    int kp2 = 1;
    while (kp2 < kmax) kp2 <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)kp2;
    e = cudaFuncSetAttribute(order_components_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    order_components_kernel<<<batch, ORDER_THREADS, smem, s>>>(scratch, 0, 0, perm, model64, params, shift4, states,
                                                               insts);
    rebuild_components_kernel<<<(total_k + 63) / 64, 64, 0, s>>>(scratch, perm, total_k, model64, params, shift4,
                                                                 states, insts, comp_inst);
    return cudaGetLastError();
}

}  // namespace gira

namespace gira {
cudaError_t launch_pack_pose(const float* pts3, int64_t n, const float* pose12, float4* pts8, DeviceState* st,
                             cudaStream_t s) {
    pack_pose_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts3, n, pose12, pts8, st);
    return cudaGetLastError();
}

cudaError_t launch_params_from_chol(const float* logits, const float* mu, const float* chol, int k, double* model64,
                                    float* params, float4* shift4, DeviceState* st, cudaStream_t s) {
    params_from_chol_kernel<<<1, PFC_THREADS, 0, s>>>(logits, mu, chol, k, model64, params, shift4, st);
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize(const float* partials, int grid, const double* ll_partials,
                                 const double* pose_partials, const float* pose12, const float* chol,
                                 const double* model64, int k, int64_t n, float* g_logits, float* g_means,
                                 float* g_chol, double* g_pose, double* g_twist, DeviceState* st, cudaStream_t s) {
    const GradFinArgs f{partials, grid, ll_partials, pose_partials, pose12, chol, model64, k, n, g_logits, g_means,
                        g_chol, g_pose, g_twist, st};
    grad_finalize_kernel<<<(k + FIN_CPB - 1) / FIN_CPB, FIN_THREADS, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_pack_pose_batched(const float* pts3, int64_t n, const int64_t* offsets, int batch,
                                     const float* poses, float4* pts8, DeviceState* states, cudaStream_t s) {
    pack_pose_batched_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts3, n, offsets, batch, poses, pts8,
                                                                         states);
    return cudaGetLastError();
}

cudaError_t launch_params_from_chol_batched(const float* logits, const float* mu, const float* chol,
                                            const BatchInst* insts, int batch, double* model64, float* params,
                                            float4* shift4, DeviceState* states, cudaStream_t s) {
    params_from_chol_batched_kernel<<<batch, PFC_THREADS, 0, s>>>(logits, mu, chol, insts, model64, params, shift4,
                                                                  states);
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize_batched(const float* partials, const double* ll_partials,
                                         const double* pose_partials, const float* poses, const float* chol,
                                         const double* model64, const BatchInst* insts, const int2* blocks,
                                         int nblocks, float* g_logits, float* g_means, float* g_chol, double* g_pose,
                                         double* g_twist, DeviceState* states, cudaStream_t s) {
    const GradFinArgs f{partials, 0, ll_partials, pose_partials, poses, chol, model64, 0, 0, g_logits, g_means,
                        g_chol, g_pose, g_twist, nullptr};
    grad_finalize_batched_kernel<<<nblocks, FIN_THREADS, 0, s>>>(f, insts, blocks, states);
    return cudaGetLastError();
}
}  // namespace gira

namespace gira {
int chunk_combine_grid() { return COMBINE_BLOCKS; }

cudaError_t launch_chunk_ref(const float* params, int k, const DeviceState* st, float* gref, cudaStream_t s) {
    chunk_ref_kernel<<<1, 256, 0, s>>>(params, k, st, gref);
    return cudaGetLastError();
}

cudaError_t launch_chunk_combine(const float* psum, int chunks, int64_t n, const float* gref, float2* pref,
                                 double* llpt, int* flag_count, int* flags, DeviceState* st, cudaStream_t s) {
    (void)st;
    chunk_combine_kernel<<<COMBINE_BLOCKS, COMBINE_THREADS, 0, s>>>(psum, chunks, n, gref, pref, llpt, flag_count,
                                                                    flags);
    return cudaGetLastError();
}

cudaError_t launch_chunk_exact(const float4* pts8, const float* params, int k, const float* gref, const int* flags,
                               const int* flag_count, float2* pref, double* llpt, DeviceState* st, cudaStream_t s) {
    chunk_exact_kernel<<<152, 256, 0, s>>>(pts8, params, k, gref, flags, flag_count, pref, llpt, st);
    return cudaGetLastError();
}

cudaError_t launch_points_ll_reduce(const double* llpt, int64_t n, double* llp, DeviceState* st, cudaStream_t s) {
    points_ll_reduce_kernel<<<COMBINE_BLOCKS, COMBINE_THREADS, 0, s>>>(llpt, n, llp);
    if (!st) return cudaGetLastError();
    return launch_ll_reduce(llp, COMBINE_BLOCKS, st, s);
}
}  // namespace gira

namespace gira {
namespace {
__global__ void double_to_float_kernel(const double* __restrict__ x, int64_t n, float* y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}
}  // namespace

cudaError_t launch_double_to_float(const double* x, int64_t n, float* y, cudaStream_t s) {
    double_to_float_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, y);
    return cudaGetLastError();
}
}  // namespace gira
