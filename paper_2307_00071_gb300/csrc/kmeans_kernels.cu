// kmeans_kernels.cu -- KInit on the GPU: k-means++ seeding, Lloyd iterations
// and the one-hot sufficient statistics that start EM.
//
// GIRA (arXiv 2307.00071) Sec. V, Fig. "information flow": KInit turns the
// point cloud and the number of components into the responsibility matrix EM
// starts from.  Here: k-means++ (Arthur & Vassilvitskii 2007, one candidate
// per step) then Lloyd, then one-hot responsibilities.  Every decision that
// floating point takes (the sampled index, the argmin label) uses binary32
// squared distances in the fixed order of dist2_f32 and binary64 running sums,
// so that a CPU reference taking the same steps reaches the same integers.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <atomic>

#include <cooperative_groups.h>

#include "gira_internal.cuh"

namespace cg = cooperative_groups;

namespace gira {

namespace {
constexpr unsigned FULL = 0xffffffffu;
constexpr int KPP_THREADS = 256;
constexpr int KPP_ITEMS = 8;
constexpr int KPP_CHUNK = KPP_THREADS * KPP_ITEMS;   // points per update block
constexpr int SEL_THREADS = 1024;

// ---------------------------------------------------------------- k-means++
__global__ void kpp_first_kernel(const float4* __restrict__ pts, int64_t n, uint64_t seed, float4* centers,
                                 int64_t* chosen, DeviceState* st) {
    if (st->error) return;
    int64_t idx = (int64_t)floor(uniform53(seed, 0) * (double)n);
    if (idx > n - 1) idx = n - 1;
    centers[0] = pts[idx];
    chosen[0] = idx;
}

// D^2(x) = min(D^2(x), ||x - c_{j-1}||^2) and the exact fixed-point sum of each chunk
// (DIM 3: distances over x, y, z; DIM 4: also over the fourth coordinate).
template <int DIM>
__global__ void __launch_bounds__(KPP_THREADS) kpp_update_kernel(const float4* __restrict__ pts, int64_t n,
                                                                 const float4* __restrict__ centers, int j,
                                                                 float* __restrict__ d2, u128* blocksums,
                                                                 DeviceState* st) {
    __shared__ u128 sh[KPP_THREADS / 32];
    if (st->error) return;
    const float4 c = centers[j - 1];
    const int64_t base = (int64_t)blockIdx.x * KPP_CHUNK;
    u128 acc{0ull, 0ull};
#pragma unroll
    for (int it = 0; it < KPP_ITEMS; ++it) {
        const int64_t i = base + it * KPP_THREADS + threadIdx.x;
        if (i < n) {
            float d = (DIM == 4) ? dist2_f32_4(pts[i], c) : dist2_f32(pts[i], c);
            if (j > 1) d = fminf(d2[i], d);
            d2[i] = d;
            acc = u128_add(acc, fx48(d));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    acc = u128_warp_incl_scan(acc, lane);
    if (lane == 31) sh[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        u128 tot{0ull, 0ull};
        for (int w = 0; w < KPP_THREADS / 32; ++w) tot = u128_add(tot, sh[w]);
        blocksums[blockIdx.x] = tot;
    }
}

// Block-wide inclusive scan of one exact value per thread.
template <int THREADS>
__device__ u128 block_incl_scan128(u128 v, u128* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = u128_warp_incl_scan(v, lane);
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        u128 w = (lane < THREADS / 32) ? sh[lane] : u128{0ull, 0ull};
        w = u128_warp_incl_scan(w, lane);
        if (lane < THREADS / 32) sh[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v = u128_add(v, sh[warp - 1]);
    __syncthreads();
    return v;
}

// Draw centre j: the first point whose exact running sum of fx(D^2) exceeds
// t = floor(k_j * T / 2^53).
__global__ void __launch_bounds__(SEL_THREADS) kpp_select_kernel(const float4* __restrict__ pts, int64_t n,
                                                                 const float* __restrict__ d2,
                                                                 const u128* __restrict__ blocksums, int nblk,
                                                                 uint64_t seed, int j, float4* centers,
                                                                 int64_t* chosen, DeviceState* st) {
    __shared__ u128 sh[SEL_THREADS / 32];
    __shared__ u128 s_total, s_rel;
    __shared__ int s_blk;
    if (st->error) return;
    const int per = (nblk + SEL_THREADS - 1) / SEL_THREADS;   // consecutive chunks per thread
    const int b0 = threadIdx.x * per;
    u128 local{0ull, 0ull};
    for (int i = 0; i < per && b0 + i < nblk; ++i) local = u128_add(local, blocksums[b0 + i]);
    const u128 incl = block_incl_scan128<SEL_THREADS>(local, sh);
    if (threadIdx.x == SEL_THREADS - 1) s_total = incl;
    if (threadIdx.x == 0) s_blk = INT_MAX;
    __syncthreads();
    const u128 T = s_total;
    int64_t idx;
    if (!u128_zero(T)) {
        const u128 t = fx_threshold(splitmix64(seed, (uint64_t)j) >> 11, T);
        // the chunk with exclusive prefix <= t < inclusive prefix (exact and monotone:
        // exactly one thread finds it)
        u128 run = u128_sub(incl, local);
        for (int i = 0; i < per && b0 + i < nblk; ++i) {
            const u128 nxt = u128_add(run, blocksums[b0 + i]);
            if (!u128_gt(run, t) && u128_gt(nxt, t)) {
                s_blk = b0 + i;
                s_rel = u128_sub(t, run);
                break;
            }
            run = nxt;
        }
        __syncthreads();
        const int kb = s_blk;
        const u128 rel = s_rel;
        const int64_t p0 = (int64_t)kb * KPP_CHUNK + 2 * threadIdx.x;
        const u128 f0 = (p0 < n) ? fx48(d2[p0]) : u128{0ull, 0ull};
        const u128 f1 = (p0 + 1 < n) ? fx48(d2[p0 + 1]) : u128{0ull, 0ull};
        const u128 pin = block_incl_scan128<SEL_THREADS>(u128_add(f0, f1), sh);
        const u128 r0 = u128_add(u128_sub(pin, u128_add(f0, f1)), f0);
        if (threadIdx.x == 0) s_blk = INT_MAX;
        __syncthreads();
        int c2 = INT_MAX;
        if (p0 < n && u128_gt(r0, rel)) c2 = 2 * threadIdx.x;
        else if (p0 + 1 < n && u128_gt(pin, rel)) c2 = 2 * threadIdx.x + 1;
        if (c2 != INT_MAX) atomicMin(&s_blk, c2);
        __syncthreads();
        idx = (int64_t)kb * KPP_CHUNK + (s_blk == INT_MAX ? 0 : s_blk);   // s_blk is always set: rel < chunk sum
    } else {   // every weight is zero (duplicates of chosen centres): uniform index
        idx = (int64_t)floor(uniform53(seed, (uint64_t)j) * (double)n);
    }
    if (idx > n - 1) idx = n - 1;
    if (idx < 0) idx = 0;
    if (threadIdx.x == 0) {
        centers[j] = pts[idx];
        chosen[j] = idx;
        st->chosen_last = idx;
    }
}

// ---------------------------------------------------------------- k-means++, persistent
// One CTA per SM (cooperative launch, so every CTA is resident).  CTA c owns a
// contiguous range of points, split into one contiguous segment per warp; D^2
// stays with the warp that owns it.  Per centre j: every CTA updates D^2 and
// publishes its binary64 sum; after all have arrived (bounded wait), every CTA
// finds the winning CTA from the same fixed-order prefix; the winner locates the
// point and publishes centre j (bounded wait for the others).  The prefix used
// for the draw is exactly excl_c + (sequential warp sums), so the search always
// lands inside the winning CTA.
constexpr int KPPP_THREADS = 512;
constexpr int KPPP_WARPS = KPPP_THREADS / 32;
constexpr long long SPIN_LIMIT = 1ll << 22;   // polls of >= 100 ns: ~0.4 s or more


// Range of lane `lane` of warp `warp` of CTA `c` (contiguous sub-ranges, so the
// running sum in point order is: CTA prefix, warp prefix, lane prefix, then the
// lane's points in order).
constexpr int KPP_LANE_MAX = 8;    // points per lane kept in registers by the search
constexpr int KPP_SLICE_MAX = 8;   // CTA sums per lane in the search (grid <= 256)

struct LaneRange {
    int64_t lo, hi;
};
__device__ __forceinline__ LaneRange lane_range(int64_t n, int G, int c, int warp, int lane) {
    const int64_t per = (n + G - 1) / G;
    const int64_t clo = min(n, (int64_t)c * per), chi = min(n, clo + per);
    const int64_t pw = (chi - clo + KPPP_WARPS - 1) / KPPP_WARPS;
    const int64_t wlo = min(chi, clo + warp * pw), whi = min(chi, wlo + pw);
    const int64_t pl = (whi - wlo + 31) / 32;
    const int64_t llo = min(whi, wlo + lane * pl), lhi = min(whi, llo + pl);
    return {llo, lhi};
}


__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Per centre j (one grid-wide wait; all sums exact, so every CTA agrees bit for bit):
//  1. every lane updates D^2 of its <= KPP_LANE_MAX points (registers) and
//     publishes them; the CTA publishes its exact fixed-point sum to sums[j][c];
//  2. one thread per CTA arrives on the step's counter and waits (bounded) for
//     all CTAs (many pollers on shared lines are far slower on this GPU); warp 0
//     then loads the G sums in parallel and finds the CTA holding the threshold;
//  3. every CTA loads that CTA's D^2 with the owner's lane layout and locates the
//     point (no second wait: the arithmetic is exact, so all CTAs find the same one).
template <int DIM>
__global__ void __launch_bounds__(KPPP_THREADS, 1) kpp_persistent_kernel(
    const float4* __restrict__ pts, int64_t n, int k, uint64_t seed, float4* centers, float* d2pub, int64_t* chosen,
    u128* sums, int* arrive, int* abort_flag, DeviceState* st) {
    __shared__ u128 s_w[KPPP_WARPS];
    __shared__ u128 s_rel, s_wrel;
    __shared__ int s_ok, s_win, s_mode, s_ww;
    __shared__ long long s_idx;
    __shared__ float4 s_cen;
    if (st->error) return;
    const int G = gridDim.x, c = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const LaneRange mine = lane_range(n, G, c, warp, lane);
    const int mcnt = (int)(mine.hi - mine.lo);
    float4 P[KPP_LANE_MAX];
    float D[KPP_LANE_MAX];
#pragma unroll
    for (int q = 0; q < KPP_LANE_MAX; ++q) {
        P[q] = (q < mcnt) ? __ldg(pts + mine.lo + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        D[q] = 0.f;
    }
    int64_t idx = (int64_t)floor(uniform53(seed, 0) * (double)n);
    if (idx > n - 1) idx = n - 1;
    float4 cen = __ldg(pts + idx);
    if (c == 0 && threadIdx.x == 0) {
        centers[0] = cen;
        chosen[0] = idx;
    }
    for (int j = 1; j < k; ++j) {
        float* pub = d2pub + (size_t)(j & 1) * n;   // double-buffered: readers of step j-1 may lag
        // ---- 1. update, publish, exact sums
        u128 ls{0ull, 0ull};
#pragma unroll
        for (int q = 0; q < KPP_LANE_MAX; ++q) {
            if (q < mcnt) {
                float d = (DIM == 4) ? dist2_f32_4(P[q], cen) : dist2_f32(P[q], cen);
                if (j > 1) d = fminf(D[q], d);
                D[q] = d;
                pub[mine.lo + q] = d;
                ls = u128_add(ls, fx48(d));
            }
        }
        const u128 inc = u128_warp_incl_scan(ls, lane);
        if (lane == 31) s_w[warp] = inc;
        __threadfence();
        __syncthreads();
        if (warp == 0) {
            u128 wv = (lane < KPPP_WARPS) ? s_w[lane] : u128{0ull, 0ull};
            const u128 wi = u128_warp_incl_scan(wv, lane);
            const u128 csum_me = u128_shfl(wi, KPPP_WARPS - 1);
            // ---- 2. publish; one thread per CTA waits on the arrival counter
            bool ok = true;
            if (lane == 0) {
                sums[(size_t)j * G + c] = csum_me;
                red_release_add(&arrive[j], 1);
                ok = wait_counter_bounded(&arrive[j], G, abort_flag, SPIN_LIMIT, st);
            }
            ok = __shfl_sync(FULL, ok ? 1 : 0, 0) != 0;
            __syncwarp();
            if (lane == 0) s_ok = ok;
            if (ok) {
                const u128* js = sums + (size_t)j * G;
                const int sl = (G + 31) / 32;
                const int a0 = min(G, lane * sl), a1 = min(G, a0 + sl);
                u128 v[KPP_SLICE_MAX];
#pragma unroll
                for (int q = 0; q < KPP_SLICE_MAX; ++q) {
                    v[q] = u128{0ull, 0ull};
                    if (q < a1 - a0) {
                        v[q].lo = __ldcg(&js[a0 + q].lo);
                        v[q].hi = __ldcg(&js[a0 + q].hi);
                    }
                }
                u128 loc{0ull, 0ull};
#pragma unroll
                for (int q = 0; q < KPP_SLICE_MAX; ++q) loc = u128_add(loc, v[q]);
                const u128 cinc = u128_warp_incl_scan(loc, lane);
                const u128 T = u128_shfl(cinc, 31);
                if (!u128_zero(T)) {
                    const u128 t = fx_threshold(splitmix64(seed, (uint64_t)j) >> 11, T);
                    u128 run = u128_sub(cinc, loc);
                    int cand = -1;
                    u128 before{0ull, 0ull};
#pragma unroll
                    for (int q = 0; q < KPP_SLICE_MAX; ++q) {
                        const u128 nxt = u128_add(run, v[q]);
                        if (cand < 0 && q < a1 - a0 && u128_gt(nxt, t)) {
                            cand = a0 + q;
                            before = run;
                        }
                        run = nxt;
                    }
                    const unsigned hits = __ballot_sync(FULL, cand >= 0);   // exactly one lane (t < T)
                    const int src = hits ? __ffs(hits) - 1 : 0;
                    if (lane == src) {
                        s_win = hits ? cand : 0;
                        s_rel = u128_sub(t, before);
                        s_mode = 0;
                    }
                } else if (lane == 0) {   // every weight is zero: uniform index
                    long long id2 = (long long)floor(uniform53(seed, (uint64_t)j) * (double)n);
                    if (id2 > n - 1) id2 = n - 1;
                    s_idx = id2;
                    s_mode = 2;
                }
            }
        }
        __syncthreads();
        if (!s_ok) return;
        if (s_mode == 2) {
            if (threadIdx.x == 0) s_cen = __ldg(pts + s_idx);
        } else {
            // ---- 3. locate the point inside the winning CTA, from its published D^2
            const LaneRange lr = lane_range(n, G, s_win, warp, lane);
            const int cnt = (int)(lr.hi - lr.lo);
            float dv[KPP_LANE_MAX];
            u128 lsum{0ull, 0ull};
#pragma unroll
            for (int q = 0; q < KPP_LANE_MAX; ++q) {
                dv[q] = (q < cnt) ? __ldcg(pub + lr.lo + q) : 0.f;
                lsum = u128_add(lsum, fx48(dv[q]));
            }
            const u128 linc = u128_warp_incl_scan(lsum, lane);
            if (lane == 31) s_w[warp] = linc;
            __syncthreads();
            if (warp == 0) {
                const u128 rel = s_rel;
                const u128 wv = (lane < KPPP_WARPS) ? s_w[lane] : u128{0ull, 0ull};
                const u128 wi = u128_warp_incl_scan(wv, lane);
                const unsigned wh = __ballot_sync(FULL, lane < KPPP_WARPS && u128_gt(wi, rel));
                const int ww = wh ? __ffs(wh) - 1 : 0;
                const u128 wexcl = u128_sub(u128_shfl(wi, ww), u128_shfl(wv, ww));
                if (lane == 0) {
                    s_ww = ww;
                    s_wrel = u128_sub(rel, wexcl);
                }
            }
            __syncthreads();
            if (warp == s_ww) {
                const u128 wrel = s_wrel;
                const unsigned lh = __ballot_sync(FULL, cnt > 0 && u128_gt(linc, wrel));
                const int src = lh ? __ffs(lh) - 1 : 0;
                if (lane == src) {
                    u128 r = u128_sub(linc, lsum);
                    long long found = lr.lo;
                    bool got = false;
#pragma unroll
                    for (int q = 0; q < KPP_LANE_MAX; ++q) {
                        if (q < cnt && !got) {
                            r = u128_add(r, fx48(dv[q]));
                            if (u128_gt(r, wrel)) {
                                found = lr.lo + q;
                                got = true;
                            }
                        }
                    }
                    if (found > n - 1) found = n - 1;   // unreachable clamp (exact search)
                    s_idx = found;
                    s_cen = __ldg(pts + found);
                }
            }
        }
        __syncthreads();
        idx = s_idx;
        cen = s_cen;
        if (c == 0 && threadIdx.x == 0) {
            centers[j] = cen;
            chosen[j] = idx;
        }
    }
}

// ---------------------------------------------------------------- k-means++ in one cluster
// For N <= cs * 512 * KC_LMAX (cs = cluster size, 16 where the GPU allows it):
// one thread-block cluster seeds all K centres with no global-memory
// synchronisation at all.  Each of the cs CTAs (one per SM) keeps its points'
// coordinates in shared memory and their D^2 in registers; each lane keeps the
// exact fixed-point sum of its own D^2, recomputed only when a new centre
// lowers one of them.  The points are dealt to warps in blocks of KC_BLOCK
// consecutive points, round-robin over the CTAs, so the points a new centre
// reaches (a patch of consecutive image rows) are spread over the cluster.
// Per centre j:
//  1. lanes whose box is out of the new centre's reach skip it; the others
//     update D^2 and their lane sums; every warp scans its lane sums and stores
//     its block total into every CTA's shared memory (st.async, DSMEM),
//     completing bytes on the receiver's mbarrier;
//  2. once its mbarrier has every block total, warp 0 of every CTA evaluates the
//     same prefix over them and finds the block holding the threshold;
//  3. the warp holding that block locates the point (lane, then the lane's
//     points in order, their weights handed over through shared memory) and
//     stores it into every CTA's shared memory the same way; every CTA waits
//     for it on a second mbarrier.
// No cluster barrier per centre and one CTA barrier: each CTA waits only for
// the bytes it reads.
// Buffers and mbarriers alternate by the parity of j: a CTA can send centre
// j + 1's total while a slower peer still has centre j's in flight, but not
// centre j + 2's (that needs centre j + 1's point, which needs every total of
// j + 1, which each CTA sends only after reading centre j's).  Every wait is
// bounded (GIRA_ERR_TIMEOUT); a thread that timed out stops waiting and sending
// and the loop runs to its end, so every CTA reaches the final cluster barrier
// and none leaves while a live peer may still store to it.
// The arithmetic is the exact fixed point of the other seeding kernels, so the
// chosen indices are identical.
constexpr int KC_THREADS = 512;
constexpr int KC_WARPS = KC_THREADS / 32;
constexpr int KC_PMAX = 18;               // point pairs per lane
constexpr int KC_LMAX = 2 * KC_PMAX;      // points per lane
constexpr int KC_BLOCK = 32 * KC_LMAX;    // points per warp (one block of the running sum)
constexpr int KC_MAX_CS = 16;

constexpr long long KC_WAIT_NS = 2000000000ll;   // bound on any wait: 2 s of wall time

constexpr int KC_PER = KC_MAX_CS * KC_WARPS / 32;   // blocks per lane of the search, in order

struct KcShared {
    // by parity of j: every block's total, stored by its warp at slot (g % KC_PER) * 32 +
    // g / KC_PER (lane l's blocks l KC_PER .. in consecutive banks); once the total of
    // every weight is below 2^64 the first half holds 64-bit totals instead
    u128 csum[2][KC_MAX_CS * KC_WARPS];
    float4 cen[2];             // by parity of j: stored by the CTA holding the chosen point
    long long idx[2];
    uint64_t bar_sum[2], bar_cen[2];
    u128 rel;                  // the threshold within the chosen block
    int win, wwin, mode;       // the block's CTA and warp; 0 normal, 2 every weight zero
    int m64;                   // the total of every weight was below 2^64 (it never grows)
    float2 dsrc[KC_PMAX];      // the D^2 of the lane holding the chosen point
};

// Inclusive warp scan of 64-bit integers (exact).
__device__ __forceinline__ unsigned long long u64_warp_incl_scan(unsigned long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// st.async: a store into a peer CTA's shared memory that completes its byte
// count on the peer's mbarrier (release at cluster scope); addresses in the
// shared::cluster window (mapa).
__device__ __forceinline__ uint32_t kc_peer(const void* local, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ void kc_send_u128(uint32_t dst, u128 v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b64 [%0], {%1, %2}, [%3];" ::"r"(dst),
                 "l"(v.lo), "l"(v.hi), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void kc_send_f4(uint32_t dst, float4 v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     dst),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void kc_send_s64(uint32_t dst, long long v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(dst), "l"(v),
                 "r"(bar)
                 : "memory");
}
// The phase with the given parity has completed; acquire at cluster scope (the
// bytes were stored by peers).  False after KC_WAIT_NS of wall time.
__device__ __forceinline__ bool kc_wait(uint64_t* bar, uint32_t parity) {
    auto try_wait = [&]() {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        return ok != 0;
    };
    if (try_wait()) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (try_wait()) return true;
        if (globaltimer_ns() - t0 > (uint64_t)KC_WAIT_NS) return false;
    }
}

size_t kc_smem_bytes() { return (size_t)3 * KC_PMAX * KC_THREADS * sizeof(float2) + sizeof(KcShared) + 16; }

// fx48(d) = floor(d 2^48) for 0 <= d < 2^10, on the FMA pipe: d 2^48 = h 2^35 +
// m 2^12 + l with integers h, m < 2^23 and l < 2^12.  Each piece is taken exactly
// by a round-toward-zero fused multiply-add onto 2^23 (binary32's integer grid on
// [2^23, 2^24)), whose bit pattern is then 0x4B000000 + the piece; the remainders
// d - h 2^-13 and r1 - m 2^-36 are exact (they keep low bits of d's significand).
// The three bit patterns are summed in 32-bit integers (fx48_join removes the
// biases; 36 pieces stay below 2^32).
__device__ __forceinline__ void fx48_parts(float d, unsigned& ah, unsigned& am, unsigned& al) {
    const float y1 = __fmaf_rz(d, 0x1p13f, 0x1p23f);
    const float r1 = fmaf(-(y1 - 0x1p23f), 0x1p-13f, d);
    const float y2 = __fmaf_rz(r1, 0x1p36f, 0x1p23f);
    const float r2 = fmaf(-(y2 - 0x1p23f), 0x1p-36f, r1);
    const float y3 = __fmaf_rz(r2, 0x1p48f, 0x1p23f);
    ah += __float_as_uint(y1);
    am += __float_as_uint(y2);
    al += __float_as_uint(y3);
}
// the sum of `count` fx48_parts terms (below 2^64 for count <= 36)
__device__ __forceinline__ unsigned long long fx48_join(unsigned ah, unsigned am, unsigned al, unsigned count) {
    const unsigned bias = count * 0x4B000000u;
    return ((unsigned long long)(ah - bias) << 35) + ((unsigned long long)(am - bias) << 12) +
           (unsigned long long)(al - bias);
}

// table (batched seeding): cluster c of the launch seeds instance table[c]; the
// pointers are then bases offset by its entry.
__global__ void __launch_bounds__(KC_THREADS, 1) kpp_cluster_kernel(const float4* __restrict__ pts0, int64_t n0,
                                                                    int k0, uint64_t seed, float4* centers0,
                                                                    int64_t* chosen0, DeviceState* st0,
                                                                    const KppInst* __restrict__ table) {
    extern __shared__ __align__(16) unsigned char kc_dsm[];
    float2* xs = reinterpret_cast<float2*>(kc_dsm);   // [KC_PMAX][KC_THREADS] each: points 2p, 2p+1 of a lane
    float2* ys = xs + KC_PMAX * KC_THREADS;
    float2* zs = ys + KC_PMAX * KC_THREADS;
    KcShared& sh = *reinterpret_cast<KcShared*>(zs + KC_PMAX * KC_THREADS);
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks(), me = (int)cluster.block_rank();
    const float4* pts = pts0;
    int64_t n = n0;
    int k = k0;
    float4* centers = centers0;
    int64_t* chosen = chosen0;
    DeviceState* st = st0;
    if (table) {
        const KppInst e = table[blockIdx.x / cs];
        pts = pts0 + e.pt_off;
        n = e.n;
        k = e.k;
        centers = centers0 + e.comp_off;
        chosen = chosen0 + e.comp_off;
        st = st0 + e.inst;
    }
    if (st->error) return;   // set before the launch: every CTA of the cluster leaves
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // blocks of KC_BLOCK consecutive points, dealt round-robin: block g belongs to
    // warp g / cs of CTA g % cs, so a neighbourhood of consecutive points (a patch of
    // image rows) is spread over the cluster; within a block, lane l holds points
    // l KC_LMAX .. in order.  The running sum in point order is then: the prefix of
    // the blocks before g, the lane prefix in block g, the lane's points in order.
    const int g = warp * cs + me;
    const int64_t llo = min(n, (int64_t)g * KC_BLOCK + (int64_t)lane * KC_LMAX);
    const int mcnt = (int)min(n - llo, (int64_t)KC_LMAX);   // every point has a block by the host's size check
    float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};   // the lane's box
#pragma unroll
    for (int p = 0; p < KC_PMAX; ++p) {
        const float4 v0 = (2 * p < mcnt) ? __ldg(pts + llo + 2 * p) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 v1 = (2 * p + 1 < mcnt) ? __ldg(pts + llo + 2 * p + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        xs[p * KC_THREADS + tid] = f2(v0.x, v1.x);
        ys[p * KC_THREADS + tid] = f2(v0.y, v1.y);
        zs[p * KC_THREADS + tid] = f2(v0.z, v1.z);
        if (2 * p < mcnt) {
            blo[0] = fminf(blo[0], v0.x); blo[1] = fminf(blo[1], v0.y); blo[2] = fminf(blo[2], v0.z);
            bhi[0] = fmaxf(bhi[0], v0.x); bhi[1] = fmaxf(bhi[1], v0.y); bhi[2] = fmaxf(bhi[2], v0.z);
        }
        if (2 * p + 1 < mcnt) {
            blo[0] = fminf(blo[0], v1.x); blo[1] = fminf(blo[1], v1.y); blo[2] = fminf(blo[2], v1.z);
            bhi[0] = fmaxf(bhi[0], v1.x); bhi[1] = fmaxf(bhi[1], v1.y); bhi[2] = fmaxf(bhi[2], v1.z);
        }
    }
    float lmax = -INFINITY;   // the largest D^2 of the lane's points (an upper bound once set)
    float2 D[KC_PMAX];   // D^2 of points 2p, 2p+1 (padding lanes: +inf, never chosen, fx48 0 not used)
    u128 ls{0ull, 0ull}, linc{0ull, 0ull};   // the lane sum and its inclusive warp prefix
    int64_t idx = (int64_t)floor(uniform53(seed, 0) * (double)n);
    if (idx > n - 1) idx = n - 1;
    float4 cen = __ldg(pts + idx);
    if (me == 0 && tid == 0) {
        centers[0] = cen;
        chosen[0] = idx;
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh.bar_sum[b], 1);
            mbar_init(&sh.bar_cen[b], 1);
        }
        sh.m64 = 0;
        mbar_fence_init();
    }
    cluster.sync();   // every CTA has started and initialised its mbarriers before any DSMEM access
    unsigned ph_sum = 0u, ph_cen = 0u;   // per parity b: the parity of the phase to wait for next
    bool dead = false;                    // this thread gave up a wait: stop waiting, run to the end
    for (int j = 1; j < k; ++j) {
        const int b = j & 1;
        // 64-bit totals: set by this CTA's warp 0 at centre j - 1 or before, from the same
        // totals in every CTA; every warp reads it before warp 0 can change it again
        const bool m64 = sh.m64 != 0;
        // ---- 1. D^2 (packed: each lane of FADD2/FMUL2 rounds like dist2_f32) and,
        //         where any D^2 dropped, the lane's exact sum from scratch (raster-
        //         order lanes see their points' D^2 drop together, so one pass over
        //         the lane beats per-point differences)
        const float2 ncx = dup(-cen.x), ncy = dup(-cen.y), ncz = dup(-cen.z);
        bool changed = (j == 1);
        // a new centre farther from the lane's box than the lane's largest D^2 lowers none
        // of them (the slack covers the rounding of the box distance and of every D^2):
        // the lane skips the update
        const float gx = fmaxf(fmaxf(blo[0] - cen.x, cen.x - bhi[0]), 0.f);
        const float gy = fmaxf(fmaxf(blo[1] - cen.y, cen.y - bhi[1]), 0.f);
        const float gz = fmaxf(fmaxf(blo[2] - cen.z, cen.z - bhi[2]), 0.f);
        if (j == 1 || fmaf(gz, gz, fmaf(gy, gy, gx * gx)) * (1.f - 1e-5f) <= lmax) {
#pragma unroll
            for (int p = 0; p < KC_PMAX; ++p) {
                if (2 * p < mcnt) {
                    const float2 d0 = add2(xs[p * KC_THREADS + tid], ncx);
                    const float2 d1 = add2(ys[p * KC_THREADS + tid], ncy);
                    const float2 d2 = add2(zs[p * KC_THREADS + tid], ncz);
                    const float2 dd = add2(add2(mul2(d0, d0), mul2(d1, d1)), mul2(d2, d2));
                    if (j == 1) {
                        D[p] = dd;
                    } else {
                        changed |= (dd.x < D[p].x) || (dd.y < D[p].y);
                        D[p] = f2(fminf(D[p].x, dd.x), fminf(D[p].y, dd.y));
                    }
                }
            }
        }
        if (changed) {
            lmax = -INFINITY;
#pragma unroll
            for (int p = 0; p < KC_PMAX; ++p) {
                if (2 * p < mcnt) lmax = fmaxf(lmax, D[p].x);
                if (2 * p + 1 < mcnt) lmax = fmaxf(lmax, D[p].y);
            }
            bool big = false;   // a weight >= 2^10: sum in 128 bits
            unsigned ah = 0u, am = 0u, al = 0u;
#pragma unroll
            for (int p = 0; p < KC_PMAX; ++p) {   // padding points add fx48(0) = 0
                const float dx = (2 * p < mcnt) ? D[p].x : 0.f, dy = (2 * p + 1 < mcnt) ? D[p].y : 0.f;
                big |= !(dx < 1024.f) || !(dy < 1024.f);
                fx48_parts(dx, ah, am, al);
                fx48_parts(dy, ah, am, al);
            }
            ls = u128{fx48_join(ah, am, al, 2 * KC_PMAX), 0ull};
            if (big) {
                ls = u128{0ull, 0ull};
#pragma unroll
                for (int p = 0; p < KC_PMAX; ++p) {
                    if (2 * p < mcnt) ls = u128_add(ls, fx48(D[p].x));
                    if (2 * p + 1 < mcnt) ls = u128_add(ls, fx48(D[p].y));
                }
            }
        }
        // this phase of bar_sum[b] expects every block's total (the previous phase of it
        // completed before this CTA read centre j - 2's totals)
        const int nblk = cs * KC_WARPS;
        if (tid == 0 && !dead) mbar_expect_tx(&sh.bar_sum[b], (uint32_t)nblk * (m64 ? 8u : 16u));
        const unsigned long long k53 = splitmix64(seed, (uint64_t)j) >> 11;   // the draw: no data dependence
        if (__any_sync(FULL, changed)) {   // else unchanged since j - 1
            if (m64) linc = u128{u64_warp_incl_scan(ls.lo, lane), 0ull};   // the block's total < 2^64
            else linc = u128_warp_incl_scan(ls, lane);
        }
        {   // this warp's block total, to every CTA's slot of block g
            const u128 total = u128_shfl(linc, 31);
            const int slot = (g % KC_PER) * 32 + g / KC_PER;
            if (lane < cs && !dead) {
                const uint32_t bar = kc_peer(&sh.bar_sum[b], lane);
                if (m64) kc_send_s64(kc_peer(reinterpret_cast<unsigned long long*>(sh.csum[b]) + slot, lane),
                                     (long long)total.lo, bar);
                else kc_send_u128(kc_peer(&sh.csum[b][slot], lane), total, bar);
            }
        }
        if (warp == 0) {
            // ---- 2. every block's total has arrived: the block holding the threshold
            if (!dead && !kc_wait(&sh.bar_sum[b], (ph_sum >> b) & 1u)) {
                dead = true;
                set_error(st, GIRA_ERR_TIMEOUT);
            }
            constexpr int PER = KC_PER;   // blocks per lane, in order
            bool tz;   // every weight is zero
            if (m64) {
                // 64-bit totals: lane l's blocks in registers, their sum, the warp's prefix
                const unsigned long long* c64 = reinterpret_cast<const unsigned long long*>(sh.csum[b]);
                unsigned long long run = 0ull;
#pragma unroll
                for (int q = 0; q < PER; ++q) run += lane * PER + q < nblk ? c64[q * 32 + lane] : 0ull;
                const unsigned long long lincl = u64_warp_incl_scan(run, lane);
                const unsigned long long T = __shfl_sync(FULL, lincl, 31);
                tz = T == 0ull;
                if (!tz) {
                    const unsigned long long t = fx_threshold(k53, u128{T, 0ull}).lo;   // t < T
                    const unsigned hits = __ballot_sync(FULL, lincl > t);
                    const int hl = hits ? __ffs(hits) - 1 : 0;
                    if (lane == hl) {   // the first of this lane's blocks whose running sum exceeds r
                        const unsigned long long r = t - (lincl - run);
                        unsigned long long pre = 0ull, prev = 0ull;   // pre: the running sum through block u
                        int q = -1;
                        unsigned long long v[PER];   // the lane's blocks again (independent loads)
#pragma unroll
                        for (int u = 0; u < PER; ++u) v[u] = lane * PER + u < nblk ? c64[u * 32 + lane] : 0ull;
#pragma unroll
                        for (int u = 0; u < PER; ++u) {
                            const unsigned long long nx = pre + v[u];
                            if (q < 0 && nx > r) {
                                q = u;
                                prev = pre;
                            }
                            pre = nx;
                        }
                        if (q < 0) {   // never: r is below the lane's sum
                            q = PER - 1;
                            prev = pre - v[PER - 1];
                        }
                        const int gw = lane * PER + q;
                        sh.win = gw % cs;
                        sh.wwin = gw / cs;
                        sh.rel = u128{r - prev, 0ull};
                        sh.mode = 0;
                    }
                }
            } else {
                u128 run{0ull, 0ull};
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    const int gq = lane * PER + q;
                    run = u128_add(run, gq < nblk ? sh.csum[b][q * 32 + lane] : u128{0ull, 0ull});
                }
                const u128 lincl = u128_warp_incl_scan(run, lane);
                const u128 before = u128_sub(lincl, run);   // the blocks of lower lanes
                const u128 T = u128_shfl(lincl, 31);
                tz = u128_zero(T);
                if (lane == 0 && T.hi == 0ull) sh.m64 = 1;   // from the next centre on: 64-bit totals
                if (!tz) {
                    const u128 t = fx_threshold(k53, T);
                    const unsigned hits = __ballot_sync(FULL, u128_gt(lincl, t));   // t < T: not empty
                    const int hl = hits ? __ffs(hits) - 1 : 0;
                    if (lane == hl) {   // the first of this lane's blocks whose running sum exceeds r
                        const u128 r = u128_sub(t, before);
                        u128 acc{0ull, 0ull}, prev{0ull, 0ull};
                        int q = PER - 1;
                        for (int u = 0; u < PER; ++u) {
                            const int gq = lane * PER + u;
                            acc = u128_add(acc, gq < nblk ? sh.csum[b][u * 32 + lane] : u128{0ull, 0ull});
                            if (u128_gt(acc, r)) {
                                q = u;
                                break;
                            }
                            prev = acc;
                        }
                        const int gw = lane * PER + q;
                        sh.win = gw % cs;
                        sh.wwin = gw / cs;
                        sh.rel = u128_sub(r, prev);
                        sh.mode = 0;
                    }
                }
            }
            if (!tz) {
                // this phase of bar_cen[b] expects the chosen point and its index
                if (lane == 0 && !dead) mbar_expect_tx(&sh.bar_cen[b], (uint32_t)(sizeof(float4) + sizeof(long long)));
            } else if (lane == 0) {   // every weight is zero: uniform index, the same in every CTA
                long long id2 = (long long)floor(uniform53(seed, (uint64_t)j) * (double)n);
                if (id2 > n - 1) id2 = n - 1;
                sh.idx[b] = id2;
                sh.cen[b] = __ldg(pts + id2);
                sh.mode = 2;
                if (me == 0) {
                    centers[j] = sh.cen[b];
                    chosen[j] = id2;
                }
            }
        }
        ph_sum ^= 1u << b;
        __syncthreads();
        const int mode = sh.mode;
        if (mode == 0 && sh.win == me) {
            // ---- 3. this CTA holds the point: lane, then the lane's points
            if (warp == sh.wwin) {
                const u128 wrel = sh.rel;
                const unsigned lh = __ballot_sync(FULL, mcnt > 0 && u128_gt(linc, wrel));
                const int src = lh ? __ffs(lh) - 1 : 0;
                const u128 base = u128_sub(u128_shfl(linc, src), u128_shfl(ls, src));
                const u128 rel2 = u128_sub(wrel, base);
                const int cnt = __shfl_sync(FULL, mcnt, src);
                // the src lane's weights through shared memory: lane l takes points 2l, 2l + 1;
                // the hit is the first point whose running sum from the lane's start exceeds rel2
                if (lane == src) {
#pragma unroll
                    for (int p = 0; p < KC_PMAX; ++p) sh.dsrc[p] = D[p];
                }
                __syncwarp();
                const float2 dl = (lane < KC_PMAX) ? sh.dsrc[lane] : f2(0.f, 0.f);
                const float a0 = (2 * lane < cnt) ? dl.x : 0.f, a1 = (2 * lane + 1 < cnt) ? dl.y : 0.f;
                int qf;
                if (__all_sync(FULL, a0 < 1024.f && a1 < 1024.f)) {   // the lane's sum is below 2^64
                    unsigned h0 = 0u, m0 = 0u, l0 = 0u, h1 = 0u, m1 = 0u, l1 = 0u;
                    fx48_parts(a0, h0, m0, l0);
                    fx48_parts(a1, h1, m1, l1);
                    const unsigned long long f0 = fx48_join(h0, m0, l0, 1), f1 = fx48_join(h1, m1, l1, 1);
                    const unsigned long long inc2 = u64_warp_incl_scan(f0 + f1, lane);
                    const unsigned long long r = rel2.lo;   // rel2 < the lane's sum < 2^64
                    const unsigned hh = __ballot_sync(FULL, inc2 > r);   // rel2 < the sum: not empty
                    const int hl = hh ? __ffs(hh) - 1 : 0;
                    const bool second = inc2 - f1 <= r;   // point 2l reaches no further than rel2
                    qf = 2 * hl + (__shfl_sync(FULL, second ? 1 : 0, hl));
                } else {
                    const u128 u0 = fx48(a0), u1 = fx48(a1);
                    const u128 inc2 = u128_warp_incl_scan(u128_add(u0, u1), lane);
                    const unsigned hh = __ballot_sync(FULL, u128_gt(inc2, rel2));
                    const int hl = hh ? __ffs(hh) - 1 : 0;
                    const bool second = !u128_gt(u128_sub(inc2, u1), rel2);
                    qf = 2 * hl + (__shfl_sync(FULL, second ? 1 : 0, hl));
                }
                const int ft = warp * 32 + src;   // the src lane's column in xs / ys / zs
                const float2 px = xs[(qf >> 1) * KC_THREADS + ft], py = ys[(qf >> 1) * KC_THREADS + ft],
                             pz = zs[(qf >> 1) * KC_THREADS + ft];
                const float4 pf = (qf & 1) ? make_float4(px.y, py.y, pz.y, 0.f) : make_float4(px.x, py.x, pz.x, 0.f);
                const long long lo_src = __shfl_sync(FULL, (long long)llo, src);
                (void)GIRA_IN(lo_src + qf < n && qf < cnt, st);   // the point is one of the lane's
                const long long found = min((long long)n - 1, lo_src + qf);   // clamp never taken
                if (lane < cs && !dead) {
                    const uint32_t bar = kc_peer(&sh.bar_cen[b], lane);
                    kc_send_f4(kc_peer(&sh.cen[b], lane), pf, bar);
                    kc_send_s64(kc_peer(&sh.idx[b], lane), found, bar);
                }
                if (lane == 0) {
                    centers[j] = pf;
                    chosen[j] = found;
                }
            }
        }
        if (mode == 0) {   // uniform over the cluster: the same totals give the same mode
            if (!dead && !kc_wait(&sh.bar_cen[b], (ph_cen >> b) & 1u)) {
                dead = true;
                set_error(st, GIRA_ERR_TIMEOUT);
            }
            ph_cen ^= 1u << b;
        }
        cen = sh.cen[b];
        idx = sh.idx[b];
    }
    cluster.sync();   // no CTA leaves while a peer may still address its shared memory
}

// ---------------------------------------------------------------- Lloyd
// labels = argmin_b ||x - c_b||^2 (binary32, ties to the lowest b); binary64
// sums of the raw coordinates and counts per label; changed[it] counts labels
// that moved (every label for it == 0).  Centres are processed two at a time
// with packed FP32 (each lane of FADD2/FMUL2 rounds exactly like the scalar
// operation, so the distances are those of dist2_f32).  Each thread owns
// LL_PPT points; equal consecutive labels in a warp are summed before the
// atomics (runs of raster-order points share labels).
constexpr int LL_PPT = 4;
constexpr int LL_THREADS = 256;

struct CPair {
    float2 x, y, z;   // negated coordinates of centres 2p and 2p+1
};

// The points of groups g0 = first, first + stride, ... (LL_THREADS * LL_PPT points
// each) against the k centres in shared memory.
__device__ void lloyd_assign_groups(const float4* __restrict__ pts, int64_t n, int npair, const CPair* sc,
                                    int32_t* labels, double* sums, unsigned long long* changed, int it,
                                    int64_t first, int64_t stride, uint16_t* lists);

// Shared memory of an assignment block: the centre pairs, then (centre pairs up
// to LL_LIST_MAX) one list of candidate pairs per warp.
constexpr int LL_LIST_MAX = 1024;
__host__ __device__ inline size_t lloyd_smem_bytes(int npair) {
    return sizeof(CPair) * (size_t)npair + (npair <= LL_LIST_MAX ? (LL_THREADS / 32) * (size_t)npair * 2 : 0);
}

__global__ void __launch_bounds__(LL_THREADS) lloyd_assign_kernel(
    const float4* __restrict__ pts, int64_t n, int k, const float4* __restrict__ centers, int32_t* labels,
    double* sums, unsigned long long* changed, int it, DeviceState* st) {
    extern __shared__ CPair sc[];
    if (st->error) return;
    if (it > 0 && changed[it - 1] == 0) return;
    const int npair = (k + 1) / 2;
    for (int p = threadIdx.x; p < npair; p += blockDim.x) {
        const float4 a = centers[2 * p];
        const float4 b = (2 * p + 1 < k) ? centers[2 * p + 1] : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        sc[p] = CPair{f2(-a.x, -b.x), f2(-a.y, -b.y), f2(-a.z, -b.z)};
    }
    __syncthreads();
    const int64_t group = (int64_t)LL_THREADS * LL_PPT;
    uint16_t* lists = npair <= LL_LIST_MAX ? reinterpret_cast<uint16_t*>(sc + npair) : nullptr;
    lloyd_assign_groups(pts, n, npair, sc, labels, sums, changed, it, (int64_t)blockIdx.x * group,
                        (int64_t)gridDim.x * group, lists);
}

// Batched: CTA u assigns tile units[u].cta of instance units[u].inst.
__global__ void __launch_bounds__(LL_THREADS) lloyd_assign_batched_kernel(
    const float4* __restrict__ pts, const KppInst* __restrict__ table, const BatchUnit* __restrict__ units,
    const float4* __restrict__ centers, int32_t* labels, double* sums, unsigned long long* changed, int iters1,
    int it, DeviceState* states) {
    extern __shared__ CPair sc[];
    const BatchUnit u = units[blockIdx.x];
    const KppInst e = table[u.inst];
    if (states[e.inst].error) return;
    unsigned long long* chg = changed + (size_t)e.inst * iters1;
    if (it > 0 && chg[it - 1] == 0) return;
    const int k = e.k, npair = (k + 1) / 2;
    const float4* c = centers + e.comp_off;
    for (int p = threadIdx.x; p < npair; p += blockDim.x) {
        const float4 a = c[2 * p];
        const float4 b = (2 * p + 1 < k) ? c[2 * p + 1] : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        sc[p] = CPair{f2(-a.x, -b.x), f2(-a.y, -b.y), f2(-a.z, -b.z)};
    }
    __syncthreads();
    const int64_t group = (int64_t)LL_THREADS * LL_PPT;
    uint16_t* lists = npair <= LL_LIST_MAX ? reinterpret_cast<uint16_t*>(sc + npair) : nullptr;
    lloyd_assign_groups(pts + e.pt_off, e.n, npair, sc, labels + e.pt_off, sums + 4 * (size_t)e.comp_off, chg, it,
                        (int64_t)u.cta * group, INT64_MAX / 2, lists);
}

__device__ void lloyd_assign_groups(const float4* __restrict__ pts, int64_t n, int npair, const CPair* sc,
                                    int32_t* labels, double* sums, unsigned long long* changed, int it,
                                    int64_t first, int64_t stride, uint16_t* lists) {
    const int lane = threadIdx.x & 31;
    uint16_t* slist = lists ? lists + (threadIdx.x >> 5) * npair : nullptr;
    unsigned long long cnt = 0;
    for (int64_t g0 = first; g0 < n; g0 += stride) {
        // point r of this thread: g0 + warp_base + r * 32 + lane (coalesced per r)
        const int64_t wb = g0 + (int64_t)(threadIdx.x >> 5) * 32 * LL_PPT;
        float2 X[LL_PPT], Y[LL_PPT], Z[LL_PPT];
        float bd[LL_PPT];
        int best[LL_PPT];
#pragma unroll
        for (int r = 0; r < LL_PPT; ++r) {
            const int64_t i = min(wb + r * 32 + lane, n - 1);
            const float4 x = pts[i];
            X[r] = dup(x.x);
            Y[r] = dup(x.y);
            Z[r] = dup(x.z);
            bd[r] = INFINITY;
            best[r] = 0;
        }
        // After the first assignment: every point's previous centre bounds its nearest
        // distance from above (U, the warp's largest), and a centre whose distance to the
        // box of the warp's points exceeds U (with slack for the binary32 rounding of
        // both) is farther than that from every point: only the other pairs are scanned,
        // in increasing order, so the argmin and its ties are those of the full scan.
        int nl = npair;
        if (it > 0 && slist) {
            float U = 0.f, lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
            for (int r = 0; r < LL_PPT; ++r) {
                const int64_t i = min(wb + r * 32 + lane, n - 1);
                const int lp = labels[i];
                const CPair c = sc[lp >> 1];
                const float cx = (lp & 1) ? c.x.y : c.x.x, cy = (lp & 1) ? c.y.y : c.y.x, cz = (lp & 1) ? c.z.y : c.z.x;
                const float dx = __fadd_rn(X[r].x, cx), dy = __fadd_rn(Y[r].x, cy), dz = __fadd_rn(Z[r].x, cz);
                const float d = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                U = fmaxf(U, d);
                lo[0] = fminf(lo[0], X[r].x); lo[1] = fminf(lo[1], Y[r].x); lo[2] = fminf(lo[2], Z[r].x);
                hi[0] = fmaxf(hi[0], X[r].x); hi[1] = fmaxf(hi[1], Y[r].x); hi[2] = fmaxf(hi[2], Z[r].x);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                U = fmaxf(U, __shfl_xor_sync(FULL, U, o));
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    lo[j] = fminf(lo[j], __shfl_xor_sync(FULL, lo[j], o));
                    hi[j] = fmaxf(hi[j], __shfl_xor_sync(FULL, hi[j], o));
                }
            }
            nl = 0;
            for (int j0 = 0; j0 < npair; j0 += 32) {
                const int p = j0 + lane;
                bool live = false;
                if (p < npair) {
                    const CPair c = sc[p];
                    const float ncx[2] = {c.x.x, c.x.y}, ncy[2] = {c.y.x, c.y.y}, ncz[2] = {c.z.x, c.z.y};
#pragma unroll
                    for (int m = 0; m < 2; ++m) {   // the centre is (-ncx, -ncy, -ncz)
                        const float gx = fmaxf(fmaxf(lo[0] + ncx[m], -ncx[m] - hi[0]), 0.f);
                        const float gy = fmaxf(fmaxf(lo[1] + ncy[m], -ncy[m] - hi[1]), 0.f);
                        const float gz = fmaxf(fmaxf(lo[2] + ncz[m], -ncz[m] - hi[2]), 0.f);
                        live = live || !(fmaf(gz, gz, fmaf(gy, gy, gx * gx)) * (1.f - 1e-5f) > U);
                    }
                }
                const uint32_t mk = __ballot_sync(FULL, live);
                if (live) slist[nl + __popc(mk & ((1u << lane) - 1u))] = (uint16_t)p;
                nl += __popc(mk);
            }
            __syncwarp();
        }
        for (int q = 0; q < nl; ++q) {
            const int p = nl == npair ? q : slist[q];
            const CPair c = sc[p];
#pragma unroll
            for (int r = 0; r < LL_PPT; ++r) {
                const float2 dx = add2(X[r], c.x), dy = add2(Y[r], c.y), dz = add2(Z[r], c.z);
                const float2 d = add2(add2(mul2(dx, dx), mul2(dy, dy)), mul2(dz, dz));
                if (d.x < bd[r]) { bd[r] = d.x; best[r] = 2 * p; }
                if (d.y < bd[r]) { bd[r] = d.y; best[r] = 2 * p + 1; }
            }
        }
#pragma unroll
        for (int r = 0; r < LL_PPT; ++r) {
            const int64_t i = wb + r * 32 + lane;
            const bool valid = i < n;
            int key = -1;
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            if (valid) {
                if (it == 0 || labels[i] != best[r]) ++cnt;
                labels[i] = best[r];
                key = best[r];
                v[0] = (double)X[r].x;
                v[1] = (double)Y[r].x;
                v[2] = (double)Z[r].x;
                v[3] = 1.0;
            }
            // segmented inclusive scan over runs of equal keys (fixed order)
            const int prev = __shfl_up_sync(FULL, key, 1);
            const bool head = (lane == 0) || (prev != key);
            const unsigned heads = __ballot_sync(FULL, head);
            const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double u = __shfl_up_sync(FULL, v[q], o);
                    if (lane - o >= start) v[q] += u;
                }
            }
            const bool tail = (lane == 31) || ((heads >> (lane + 1)) & 1u);
            if (tail && key >= 0)
#pragma unroll
                for (int q = 0; q < 4; ++q) atomicAdd(&sums[4 * key + q], v[q]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
    if (lane == 0 && cnt) atomicAdd(&changed[it], cnt);
}

// centres = binary64 mean of their points, rounded to binary32; empty clusters
// keep their centre.  Runs only if the previous assignment moved a label.
__global__ void lloyd_update_kernel(int k, double* sums, float4* centers, const unsigned long long* changed, int it,
                                    DeviceState* st) {
    if (st->error || changed[it - 1] == 0) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < k) {
        const double cnt = sums[4 * b + 3];
        if (cnt > 0.0)
            centers[b] = make_float4((float)(sums[4 * b] / cnt), (float)(sums[4 * b + 1] / cnt),
                                     (float)(sums[4 * b + 2] / cnt), 0.f);
        for (int i = 0; i < 4; ++i) sums[4 * b + i] = 0.0;
    }
    if (b == 0) st->lloyd_done = it;
}

// Batched: global component g of instance comp_inst[g].
__global__ void lloyd_update_batched_kernel(int total_k, const int* __restrict__ comp_inst,
                                            const KppInst* __restrict__ table, double* sums, float4* centers,
                                            const unsigned long long* changed, int iters1, int it,
                                            DeviceState* states) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total_k) return;
    const KppInst e = table[comp_inst[g]];
    if (states[e.inst].error || changed[(size_t)e.inst * iters1 + it - 1] == 0) return;
    const double cnt = sums[4 * (size_t)g + 3];
    if (cnt > 0.0)
        centers[g] = make_float4((float)(sums[4 * (size_t)g] / cnt), (float)(sums[4 * (size_t)g + 1] / cnt),
                                 (float)(sums[4 * (size_t)g + 2] / cnt), 0.f);
    for (int i = 0; i < 4; ++i) sums[4 * (size_t)g + i] = 0.0;
    if (g == e.comp_off) states[e.inst].lloyd_done = it;
}

// One-hot statistics about the shift s_b (the final centre): S0 = count,
// S1 = sum (x - s), S2 = sum (x - s)(x - s)^T, binary64.  Each thread takes
// LS_PPT consecutive points and sums each run of equal labels in registers
// before its atomics (raster-order neighbours share labels, so most threads
// flush once).
constexpr int LS_PPT = 8;

__device__ __forceinline__ void label_stats_flush(double* stats64, int b, const double* a) {
    double* S = stats64 + (size_t)b * NSTAT;
#pragma unroll
    for (int t = 0; t < NSTAT; ++t) atomicAdd(&S[t], a[t]);
}

__global__ void label_stats_kernel(const float4* __restrict__ pts, int64_t n, int k, const int32_t* __restrict__ labels,
                                   const float4* __restrict__ shift4, double* stats64, DeviceState* st) {
    if (st->error) return;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * LS_PPT;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * LS_PPT; i0 < n; i0 += step) {
        int key = -1;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        double a[NSTAT];
#pragma unroll
        for (int t = 0; t < NSTAT; ++t) a[t] = 0.0;
#pragma unroll
        for (int r = 0; r < LS_PPT; ++r) {
            const int64_t i = i0 + r;
            if (i < n) {
                const int b = labels[i];
                if (!GIRA_IN(b >= 0 && b < k, st)) continue;
                if (b != key) {
                    if (key >= 0) label_stats_flush(stats64, key, a);
#pragma unroll
                    for (int t = 0; t < NSTAT; ++t) a[t] = 0.0;
                    key = b;
                    s = shift4[b];
                }
                const float4 x = pts[i];
                const double d0 = (double)x.x - (double)s.x, d1 = (double)x.y - (double)s.y,
                             d2 = (double)x.z - (double)s.z;
                a[0] += 1.0;
                a[1] += d0;
                a[2] += d1;
                a[3] += d2;
                a[4] += d0 * d0;
                a[5] += d0 * d1;
                a[6] += d0 * d2;
                a[7] += d1 * d1;
                a[8] += d1 * d2;
                a[9] += d2 * d2;
            }
        }
        if (key >= 0) label_stats_flush(stats64, key, a);
    }
}

// Batched: the instance of point i by binary search over the offsets.
__global__ void label_stats_batched_kernel(const float4* __restrict__ pts, int64_t n, const int64_t* __restrict__ offsets,
                                           int batch, const KppInst* __restrict__ table,
                                           const int32_t* __restrict__ labels, const float4* __restrict__ shift4,
                                           double* stats64, DeviceState* states) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = batch;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (offsets[mid] <= i) lo = mid; else hi = mid;
        }
        if (states[lo].error) continue;
        if (!GIRA_IN(labels[i] >= 0 && labels[i] < table[lo].k, states + lo)) continue;
        const int b = table[lo].comp_off + labels[i];
        const float4 x = pts[i], s = shift4[b];
        const double d[3] = {(double)x.x - (double)s.x, (double)x.y - (double)s.y, (double)x.z - (double)s.z};
        double* S = stats64 + (size_t)b * NSTAT;
        atomicAdd(&S[0], 1.0);
        for (int t = 0; t < 3; ++t) atomicAdd(&S[1 + t], d[t]);
        atomicAdd(&S[4], d[0] * d[0]);
        atomicAdd(&S[5], d[0] * d[1]);
        atomicAdd(&S[6], d[0] * d[2]);
        atomicAdd(&S[7], d[1] * d[1]);
        atomicAdd(&S[8], d[1] * d[2]);
        atomicAdd(&S[9], d[2] * d[2]);
    }
}

__global__ void centers_out_kernel(const float4* __restrict__ c4, int k, float* c3) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= k) return;
    const float4 c = c4[b];
    c3[3 * b] = c.x;
    c3[3 * b + 1] = c.y;
    c3[3 * b + 2] = c.z;
}
}  // namespace

int kpp_num_blocks(int64_t n) { return (int)((n + KPP_CHUNK - 1) / KPP_CHUNK); }

int kpp_persistent_grid() {
    int dev = 0, sms = 1, occ = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return 0;
    int occ4 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kpp_persistent_kernel<3>, KPPP_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ4, kpp_persistent_kernel<4>, KPPP_THREADS, 0) != cudaSuccess ||
        occ < 1 || occ4 < 1) {
        cudaGetLastError();
        return 0;
    }
    return std::min(sms, 256);   // the search keeps at most 8 CTA sums per lane
}

size_t kpp_persistent_sum_words(int grid, int k) { return (size_t)grid * (size_t)k; }

int64_t kpp_persistent_max_n(int grid) { return (int64_t)grid * KPPP_WARPS * 32 * KPP_LANE_MAX; }

cudaError_t launch_kpp_persistent(const float4* pts4, int64_t n, int k, uint64_t seed, float4* centers, float* d2,
                                  int64_t* chosen, int* sync_ints, u128* sums, int grid, DeviceState* st,
                                  cudaStream_t s, int dim) {
    int* arrive = sync_ints;
    int* abort_flag = sync_ints + k;
    void* args[] = {(void*)&pts4, (void*)&n, (void*)&k, (void*)&seed, (void*)&centers, (void*)&d2, (void*)&chosen,
                    (void*)&sums, (void*)&arrive, (void*)&abort_flag, (void*)&st};
    const void* fn = (dim == 4) ? (const void*)kpp_persistent_kernel<4> : (const void*)kpp_persistent_kernel<3>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(KPPP_THREADS), args, 0, s);
}

// Cluster size for the one-cluster seeding of n points, or 0 when it does not
// apply (too many points, or no cluster of that size fits on this GPU).
int kpp_cluster_size(int64_t n) {
    static std::atomic<int> cached_size{-1};   // largest usable cluster size (one GPU model per process)
    int cached = cached_size.load();
    if (cached < 0) {
        cached = 0;
        const size_t smem = kc_smem_bytes();
        if (cudaFuncSetAttribute(kpp_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                cudaSuccess &&
            cudaFuncSetAttribute(kpp_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess) {
            for (int cs : {KC_MAX_CS, 8}) {
                cudaLaunchConfig_t cfg{};
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = cs;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3(cs);
                cfg.blockDim = dim3(KC_THREADS);
                cfg.dynamicSmemBytes = smem;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int nclusters = 0;
                if (cudaOccupancyMaxActiveClusters(&nclusters, kpp_cluster_kernel, &cfg) == cudaSuccess &&
                    nclusters >= 1) {
                    cached = cs;
                    break;
                }
            }
        }
        cudaGetLastError();
        cached_size.store(cached);   // racing first calls compute the same value
    }
    if (cached == 0 || n > (int64_t)cached * KC_THREADS * KC_LMAX) return 0;
    return cached;
}

cudaError_t launch_kpp_cluster_batched(const float4* pts4, const KppInst* table, int clusters, uint64_t seed,
                                       float4* centers, int64_t* chosen, int cs, DeviceState* states,
                                       cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs * clusters);
    cfg.blockDim = dim3(KC_THREADS);
    cfg.dynamicSmemBytes = kc_smem_bytes();
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kpp_cluster_kernel, pts4, (int64_t)0, 0, seed, centers, chosen, states, table);
}

int kpp_cluster_capacity(int cs) { return cs * KC_THREADS * KC_LMAX; }

cudaError_t launch_kpp_cluster(const float4* pts4, int64_t n, int k, uint64_t seed, float4* centers, int64_t* chosen,
                               int cs, DeviceState* st, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(KC_THREADS);
    cfg.dynamicSmemBytes = kc_smem_bytes();
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kpp_cluster_kernel, pts4, n, k, seed, centers, chosen, st, (const KppInst*)nullptr);
}

cudaError_t launch_kpp(const float4* pts4, int64_t n, int k, uint64_t seed, float4* centers, float* d2,
                       u128* blocksums, int64_t* chosen, DeviceState* st, cudaStream_t s, int dim) {
    const int nblk = kpp_num_blocks(n);
    kpp_first_kernel<<<1, 1, 0, s>>>(pts4, n, seed, centers, chosen, st);
    for (int j = 1; j < k; ++j) {
        if (dim == 4)
            kpp_update_kernel<4><<<nblk, KPP_THREADS, 0, s>>>(pts4, n, centers, j, d2, blocksums, st);
        else
            kpp_update_kernel<3><<<nblk, KPP_THREADS, 0, s>>>(pts4, n, centers, j, d2, blocksums, st);
        kpp_select_kernel<<<1, SEL_THREADS, 0, s>>>(pts4, n, d2, blocksums, nblk, seed, j, centers, chosen, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_lloyd(const float4* pts4, int64_t n, int k, int lloyd_iters, float4* centers, int32_t* labels,
                         double* sums, unsigned long long* changed, DeviceState* st, cudaStream_t s) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = lloyd_smem_bytes((k + 1) / 2);
    const int threads = LL_THREADS;
    const int64_t want = (n + (int64_t)threads * LL_PPT - 1) / ((int64_t)threads * LL_PPT);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 4));
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024)
        e = cudaFuncSetAttribute(lloyd_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    lloyd_assign_kernel<<<grid, threads, smem, s>>>(pts4, n, k, centers, labels, sums, changed, 0, st);
    for (int it = 1; it <= lloyd_iters; ++it) {
        lloyd_update_kernel<<<(k + 127) / 128, 128, 0, s>>>(k, sums, centers, changed, it, st);
        lloyd_assign_kernel<<<grid, threads, smem, s>>>(pts4, n, k, centers, labels, sums, changed, it, st);
    }
    return cudaGetLastError();
}

int lloyd_tile() { return LL_THREADS * LL_PPT; }

cudaError_t launch_lloyd_batched(const float4* pts4, const KppInst* table, const BatchUnit* units, int nunits,
                                 int total_k, const int* comp_inst, int lloyd_iters, float4* centers, int32_t* labels,
                                 double* sums, unsigned long long* changed, DeviceState* states, cudaStream_t s) {
    const size_t smem = lloyd_smem_bytes((GIRA_MAX_K_BATCHED + 1) / 2);
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024)
        e = cudaFuncSetAttribute(lloyd_assign_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int iters1 = lloyd_iters + 1;
    lloyd_assign_batched_kernel<<<nunits, LL_THREADS, smem, s>>>(pts4, table, units, centers, labels, sums, changed,
                                                                 iters1, 0, states);
    for (int it = 1; it <= lloyd_iters; ++it) {
        lloyd_update_batched_kernel<<<(total_k + 127) / 128, 128, 0, s>>>(total_k, comp_inst, table, sums, centers,
                                                                          changed, iters1, it, states);
        lloyd_assign_batched_kernel<<<nunits, LL_THREADS, smem, s>>>(pts4, table, units, centers, labels, sums,
                                                                     changed, iters1, it, states);
    }
    return cudaGetLastError();
}

cudaError_t launch_label_stats_batched(const float4* pts4, int64_t n, const int64_t* offsets, int batch,
                                       const KppInst* table, const int32_t* labels, const float4* shift4,
                                       double* stats64, DeviceState* states, cudaStream_t s) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    label_stats_batched_kernel<<<grid, 256, 0, s>>>(pts4, n, offsets, batch, table, labels, shift4, stats64, states);
    return cudaGetLastError();
}

cudaError_t launch_label_stats(const float4* pts4, int64_t n, int k, const int32_t* labels, const float4* shift4,
                               double* stats64, DeviceState* st, cudaStream_t s) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 256 * LS_PPT - 1) / (256 * LS_PPT);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    label_stats_kernel<<<grid, 256, 0, s>>>(pts4, n, k, labels, shift4, stats64, st);
    return cudaGetLastError();
}

namespace {
// Test hook: waits that nothing will end, to exercise the bounded-wait exits.
// mode 0: an mbarrier phase that never completes (limit: wall time in ns);
// mode 1: a global counter that nobody increments (limit: polls), the wait of
// the persistent seeding kernel.
__global__ void wait_probe_kernel(int mode, long long limit, int* counter, int* abort_flag, DeviceState* st) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    if (mode == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        if (!mbar_wait_bounded(&bar, 0u, limit)) set_error(st, GIRA_ERR_TIMEOUT);
    } else {
        wait_counter_bounded(counter, 1, abort_flag, limit, st);
    }
}
}  // namespace

cudaError_t launch_wait_probe(int mode, long long limit, int* counter, int* abort_flag, DeviceState* st,
                              cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(mode, limit, counter, abort_flag, st);
    return cudaGetLastError();
}

cudaError_t launch_centers_out(const float4* centers4, int k, float* centers3, cudaStream_t s) {
    centers_out_kernel<<<(k + 127) / 128, 128, 0, s>>>(centers4, k, centers3);
    return cudaGetLastError();
}

}  // namespace gira
