// gbms_kernels.cu -- mode seeking that sets the number of components K.
//
// GIRA (arXiv 2307.00071) Sec. V, paragraph "Gaussian Blurring Mean Shift", and
// Fig. "information flow": seeds from a binned estimator, each seed moved to
// the average of the points within the bandwidth h of it until it stops moving
// (or an iteration limit), the distinct end points counted.  The paper queries
// neighbours with a kd-tree on the CPU; here the points are sorted by grid cell
// (cells of size h, the same cells that give the seeds) and a ball query visits
// the 3^D (at most 4^D) cells around the seed.
//
// Definitions taken by every step (both sides of the parity tests):
//   cell     c_i(x) = floor(x_i / h + 0.5) (binary64), |c_i| < 2^15;
//            key = sum_i (c_i + 2^15) 2^(16 i)
//   seeds    one per occupied cell, at c h, in ascending key order
//   ball     binary32 squared distance between x and (float)m in the order
//            ((d0^2 + d1^2) + d2^2) [+ d3^2], no FMA, <= (float)(h*h)
//   mean     exact 64-bit sums of rint(x_i 2^24) (|x_i| < 2^12), then
//            ((double)S / count) 2^-24: independent of the order of summation
//   stop     ||m_t - m_{t-1}||^2 <= (1e-3 h)^2 (binary64) or t = max_iter;
//            a seed whose ball is empty is dropped
//   merge    modes ranked by count (descending), ties by seed; in rank order a
//            mode is kept unless a kept mode lies within h (binary64 squared
//            distance, coordinate order, no FMA, <= h*h)
// The merge runs in rounds: a mode is kept once every earlier-ranked mode
// within h of it is known to be dropped, and dropped once one of them is kept;
// each round decides at least the lowest undecided rank, and the result is the
// sequential greedy one.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <cub/cub.cuh>

#include "gira_internal.cuh"

namespace gira {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int GB_WARPS = 8;          // warps (seeds or modes) per CTA
constexpr int GB_MAX_CELLS = 256;    // at most 4 cells per dimension, 4 dimensions
constexpr double Q_SCALE = 16777216.0;   // 2^24
constexpr float Q_SCALE_F = 16777216.0f;

__device__ __forceinline__ bool cell_of(double v, double h, int* c) {
    const double f = floor(__dadd_rn(__ddiv_rn(v, h), 0.5));
    if (!(f > -32768.0 && f < 32768.0)) return false;
    *c = (int)f;
    return true;
}

__device__ __forceinline__ uint64_t key_of(const int* c, int d) {
    uint64_t k = 0;
    for (int i = 0; i < d; ++i) k |= (uint64_t)(uint32_t)(c[i] + 32768) << (16 * i);
    return k;
}

__device__ __forceinline__ int cell_coord(uint64_t key, int i) { return (int)((key >> (16 * i)) & 0xFFFFu) - 32768; }

// first index in sorted[0, n) with sorted[i] >= key
__device__ __forceinline__ int lower_bound_u64(const uint64_t* sorted, int n, uint64_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sorted[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ float dist2_ball(float4 x, const float* mf, int d) {
    const float d0 = __fsub_rn(x.x, mf[0]), d1 = __fsub_rn(x.y, mf[1]), d2 = __fsub_rn(x.z, mf[2]);
    float s = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
    if (d == 4) {
        const float d3 = __fsub_rn(x.w, mf[3]);
        s = __fadd_rn(s, __fmul_rn(d3, d3));
    }
    return s;
}

__device__ __forceinline__ double dist2_modes(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        const double dv = __dsub_rn(a[i], b[i]);
        s = (i == 0) ? __dmul_rn(dv, dv) : __dadd_rn(s, __dmul_rn(dv, dv));
    }
    return s;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// The cells a ball of radius h around m can touch: per dimension [lo_i, lo_i + nr_i).
// Only a superset is needed (the ball test decides membership), so binary32
// with the radius inflated by 5 % suffices: the binary32 error of m_i / h is
// below 4e-3 cells for every |c_i| < 2^15, far inside the margin, and a point
// in the ball lies within h (1 + 2^-23) of m in every coordinate.
__device__ __forceinline__ int ball_cells(const float* m, int d, float h, float inv_h, int* lo, int* nr) {
    const float hin = 1.05f * h;
    int total = 1;
    for (int i = 0; i < d; ++i) {
        const float a = floorf(fmaf(m[i] - hin, inv_h, 0.5f));
        const float b = floorf(fmaf(m[i] + hin, inv_h, 0.5f));
        const int la = (int)fmaxf(a, -32767.f), lb = (int)fminf(b, 32767.f);
        lo[i] = la;
        nr[i] = lb >= la ? lb - la + 1 : 0;
        total *= nr[i];
    }
    return total;
}

// Lanes list the occupied cells of the candidate box (start, length) in the
// warp's shared arrays and fill pre[] with the exclusive prefix of the lengths
// (pre[count] = total points); returns the count.  The box is walked in rows
// along the first coordinate: the cells of a row have consecutive keys (the
// first coordinate is the key's lowest field), so one binary search per row
// finds the row's first occupied cell and the rest follow in order.
__device__ int gather_cells(const uint64_t* ukeys, const int* ustart, const int* ulen, int ncells, const int* lo,
                            const int* nr, int total, int d, int lane, int* cs, int* pre) {
    const int nrows = (nr[0] > 0) ? total / nr[0] : 0;
    int nfound = 0;
    for (int base = 0; base < nrows; base += 32) {
        const int row = base + lane;
        int st[4], ln[4], cnt = 0;
        if (row < nrows) {
            int c[4] = {lo[0], 0, 0, 0}, r = row;
            for (int i = 1; i < d; ++i) {
                c[i] = lo[i] + r % nr[i];
                r /= nr[i];
            }
            const uint64_t k0 = key_of(c, d);             // (lo_0, c_1, ...)
            const uint64_t k1 = k0 + (uint64_t)nr[0];      // one past the row's last candidate
            for (int pos = lower_bound_u64(ukeys, ncells, k0); pos < ncells && ukeys[pos] < k1 && cnt < 4; ++pos) {
                st[cnt] = ustart[pos];
                ln[cnt] = ulen[pos];
                ++cnt;
            }
        }
        // this lane's cells go after those of the lower lanes
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += u;
        }
        const int at = nfound + inc - cnt;
        for (int q = 0; q < cnt; ++q) {
            cs[at + q] = st[q];
            pre[at + q] = ln[q];   // lengths for now
        }
        nfound += __shfl_sync(FULL, inc, 31);
    }
    __syncwarp();
    // exclusive prefix of the lengths, 32 at a time
    int carry = 0;
    for (int base = 0; base < nfound; base += 32) {
        const int j = base + lane;
        const int v = (j < nfound) ? pre[j] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += u;
        }
        __syncwarp();
        if (j < nfound) pre[j] = carry + inc - v;
        carry += __shfl_sync(FULL, inc, 31);
    }
    if (lane == 0) pre[nfound] = carry;
    __syncwarp();
    return nfound;
}

// index j with pre[j] <= t < pre[j + 1]
__device__ __forceinline__ int cell_of_flat(const int* pre, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void gbms_keys_kernel(const float* __restrict__ pts, int64_t n, int d, double h, float4* pts4,
                                 uint64_t* keys, int* idx, DeviceState* st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    int c[4] = {0, 0, 0, 0};
    bool ok = true, fin = true;
    for (int j = 0; j < d; ++j) {
        v[j] = pts[(size_t)d * i + j];
        fin = fin && isfinite(v[j]);
        ok = ok && fabsf(v[j]) < 4096.0f && cell_of((double)v[j], h, &c[j]);
    }
    if (!fin) set_error(st, GIRA_ERR_NONFINITE_INPUT);
    else if (!ok) set_error(st, GIRA_ERR_INVALID_ARG);
    pts4[i] = make_float4(v[0], v[1], v[2], v[3]);
    keys[i] = key_of(c, d);
    idx[i] = (int)i;
}

// Points in cell order, with their fixed-point coordinates rint(x 2^24): x 2^24
// is exact in binary32 (|x| < 2^12), so one float -> int64 rounding gives it.
__global__ void gbms_gather_kernel(const float4* __restrict__ pts4, const int* __restrict__ idx, int64_t n,
                                   float4* spts, longlong2* qxy, longlong2* qzw) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 x = pts4[idx[i]];
    spts[i] = x;
    qxy[i] = make_longlong2(__float2ll_rn(x.x * Q_SCALE_F), __float2ll_rn(x.y * Q_SCALE_F));
    qzw[i] = make_longlong2(__float2ll_rn(x.z * Q_SCALE_F), __float2ll_rn(x.w * Q_SCALE_F));
}

// One CTA (GB_SHIFT_THREADS) per seed: the moves of the seed of cell ukeys[s]
// (see the header).  The occupied cells around the seed are listed by warp 0
// and kept while the seed stays in the same cells; the threads sweep the
// listed points (cell by cell, in flat order), the exact integer sums are
// reduced per warp and across warps, and thread 0 takes the move.
constexpr int GB_SHIFT_THREADS = 128;
constexpr int GB_UNROLL = 4;
constexpr int GB_SHIFT_WARPS = GB_SHIFT_THREADS / 32;

__global__ void __launch_bounds__(GB_SHIFT_THREADS) gbms_shift_kernel(
    const float4* __restrict__ spts, const longlong2* __restrict__ qxy, const longlong2* __restrict__ qzw,
    const uint64_t* __restrict__ ukeys, const int* __restrict__ ustart, const int* __restrict__ ulen, int ncells,
    int d, double h, int max_iter, double4* modes, int* counts, const DeviceState* st) {
    __shared__ int s_cs[GB_MAX_CELLS];
    __shared__ int s_pre[GB_MAX_CELLS + 1];
    __shared__ int s_nf;
    __shared__ long long s_red[GB_SHIFT_WARPS][5];
    __shared__ double s_m[4];
    __shared__ float s_mf[4];
    __shared__ int s_lo[4], s_nr[4], s_total, s_moved_cells;
    __shared__ int s_done, s_count;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s = blockIdx.x;
    if (st->error) return;   // set before the launch: uniform
    // binary64 work (the move, its stopping test, the cells around the seed) is
    // done by thread 0 alone: GB300 runs binary64 at a small fraction of binary32
    const float hf = (float)h, inv_hf = 1.0f / hf;
    auto place_cells = [&]() {   // thread 0: the cells of the ball around the binary32 seed s_mf
        int lo[4], nr[4];
        s_total = ball_cells(s_mf, d, hf, inv_hf, lo, nr);
        bool same = true;
        for (int i = 0; i < d; ++i) {
            same = same && lo[i] == s_lo[i] && nr[i] == s_nr[i];
            s_lo[i] = lo[i];
            s_nr[i] = nr[i];
        }
        s_moved_cells = same ? 0 : 1;
    };
    if (tid == 0) {
        const uint64_t key = ukeys[s];
        for (int i = 0; i < 4; ++i) {
            s_m[i] = (i < d) ? __dmul_rn((double)cell_coord(key, i), h) : 0.0;
            s_lo[i] = INT_MIN;
            s_nr[i] = 0;
        }
        for (int i = 0; i < 4; ++i) s_mf[i] = __double2float_rn(s_m[i]);
        s_done = 0;
        s_count = 0;
        place_cells();
    }
    const float h2f = __double2float_rn(__dmul_rn(h, h));
    const double thr = __dmul_rn(1e-3, h), thr2 = __dmul_rn(thr, thr);
    __syncthreads();
    for (int t = 1; t <= max_iter; ++t) {
        if (s_moved_cells) {   // uniform
            if (warp == 0) {
                int lo[4], nr[4];
                for (int i = 0; i < 4; ++i) {
                    lo[i] = s_lo[i];
                    nr[i] = s_nr[i];
                }
                const int nf = gather_cells(ukeys, ustart, ulen, ncells, lo, nr, s_total, d, lane, s_cs, s_pre);
                if (lane == 0) s_nf = nf;
            }
            __syncthreads();
        }
        const float mf[4] = {s_mf[0], s_mf[1], s_mf[2], s_mf[3]};
        const int nf = s_nf, npts = s_pre[nf];
        long long cnt = 0, s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        int j = 0;
        // GB_UNROLL points per thread per trip, all loads issued before any test
        // (a seed that keeps moving runs alone on its SM: latency, not bandwidth)
        for (int f0 = tid; f0 < npts; f0 += GB_UNROLL * GB_SHIFT_THREADS) {
            int pi[GB_UNROLL];
#pragma unroll
            for (int u = 0; u < GB_UNROLL; ++u) {
                const int f = f0 + u * GB_SHIFT_THREADS;
                pi[u] = -1;
                if (f < npts) {
                    while (s_pre[j + 1] <= f) ++j;   // f only grows: the cell index only moves forward
                    pi[u] = s_cs[j] + (f - s_pre[j]);
                }
            }
            float4 x[GB_UNROLL];
#pragma unroll
            for (int u = 0; u < GB_UNROLL; ++u) x[u] = spts[pi[u] >= 0 ? pi[u] : 0];
            bool in[GB_UNROLL];
#pragma unroll
            for (int u = 0; u < GB_UNROLL; ++u) in[u] = pi[u] >= 0 && dist2_ball(x[u], mf, d) <= h2f;
            // the fixed-point coordinates only for points in the ball (a few per cent
            // of the candidates), all loads issued before any use
            longlong2 qa[GB_UNROLL], qb[GB_UNROLL];
#pragma unroll
            for (int u = 0; u < GB_UNROLL; ++u) {
                qa[u] = in[u] ? qxy[pi[u]] : make_longlong2(0, 0);
                qb[u] = in[u] ? qzw[pi[u]] : make_longlong2(0, 0);
            }
#pragma unroll
            for (int u = 0; u < GB_UNROLL; ++u) {
                cnt += in[u] ? 1 : 0;
                s0 += qa[u].x;
                s1 += qa[u].y;
                s2 += qb[u].x;
                s3 += qb[u].y;
            }
        }
        cnt = warp_sum_ll(cnt);
        s0 = warp_sum_ll(s0);
        s1 = warp_sum_ll(s1);
        s2 = warp_sum_ll(s2);
        s3 = warp_sum_ll(s3);
        if (lane == 0) {
            s_red[warp][0] = cnt;
            s_red[warp][1] = s0;
            s_red[warp][2] = s1;
            s_red[warp][3] = s2;
            s_red[warp][4] = s3;
        }
        __syncthreads();
        if (warp == 0) {
            // the move: lane i < d takes coordinate i (one binary64 instruction serves
            // every coordinate), lane 0 sums the squared steps in coordinate order
            long long tot = 0;
            if (lane < 5)
                for (int w = 0; w < GB_SHIFT_WARPS; ++w) tot += s_red[w][lane];
            const long long count = __shfl_sync(FULL, tot, 0);
            const long long si = __shfl_down_sync(FULL, tot, 1);   // lane i: sum of coordinate i
            if (count == 0) {
                if (lane == 0) {
                    s_count = 0;
                    s_done = 1;
                }
            } else {
                double sq = 0.0, v = 0.0;
                if (lane < d) {
                    v = __dmul_rn(__ddiv_rn(__ll2double_rn(si), (double)count), 1.0 / Q_SCALE);
                    const double dv = __dsub_rn(v, s_m[lane]);
                    sq = __dmul_rn(dv, dv);
                }
                const double sq1 = __shfl_sync(FULL, sq, 1), sq2 = __shfl_sync(FULL, sq, 2),
                             sq3 = __shfl_sync(FULL, sq, 3);
                __syncwarp();
                if (lane < d) {
                    s_m[lane] = v;
                    s_mf[lane] = __double2float_rn(v);
                }
                __syncwarp();
                if (lane == 0) {
                    double mv = __dadd_rn(__dadd_rn(sq, sq1), sq2);
                    if (d == 4) mv = __dadd_rn(mv, sq3);
                    s_count = (int)count;
                    if (mv <= thr2 || t == max_iter) s_done = 1;
                    else place_cells();
                }
            }
        }
        __syncthreads();
        if (s_done) break;
    }
    if (tid == 0) {
        modes[s] = make_double4(s_m[0], s_m[1], s_m[2], s_m[3]);
        counts[s] = s_count;
    }
}

// Rank keys: (2^31 - 1 - count, seed) for live modes; dropped seeds sort last.
__global__ void gbms_rank_keys_kernel(const int* __restrict__ counts, int ns, uint64_t* rkeys, int* nlive) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int c = counts[s];
    rkeys[s] = c > 0 ? ((uint64_t)(0x7FFFFFFF - c) << 32) | (uint32_t)s : ~0ull;
    if (c > 0) atomicAdd(nlive, 1);
}

// Rank r: its mode, count and cell key (for the merge grid).
__global__ void gbms_rank_modes_kernel(const uint64_t* __restrict__ rkeys_sorted, const int* __restrict__ nlive,
                                       const double4* __restrict__ modes, const int* __restrict__ counts, int d,
                                       double h, double4* rmodes, int* rcount, uint64_t* mkeys, int* midx,
                                       int* state, DeviceState* st) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= *nlive) return;
    const int s = (int)(rkeys_sorted[r] & 0xFFFFFFFFull);
    const double4 m = modes[s];
    rmodes[r] = m;
    rcount[r] = counts[s];
    const double mv[4] = {m.x, m.y, m.z, m.w};
    int c[4] = {0, 0, 0, 0};
    bool ok = true;
    for (int i = 0; i < d; ++i) ok = ok && cell_of(mv[i], h, &c[i]);
    if (!ok) set_error(st, GIRA_ERR_INVALID_ARG);   // unreachable: a mean of points lies inside their cells
    mkeys[r] = key_of(c, d);
    midx[r] = r;
    state[r] = 0;
}

// One merge round over the undecided ranks (state 0 undecided, 1 kept, 2 dropped).
__global__ void __launch_bounds__(GB_WARPS * 32) gbms_merge_round_kernel(
    const double4* __restrict__ rmodes, const int* __restrict__ nlive, const uint64_t* __restrict__ mukeys,
    const int* __restrict__ mustart, const int* __restrict__ mulen, const int* __restrict__ mncells,
    const int* __restrict__ midx_sorted, int d, double h, int* state, int* undecided) {
    __shared__ int s_cs[GB_WARPS][GB_MAX_CELLS];
    __shared__ int s_pre[GB_WARPS][GB_MAX_CELLS + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * GB_WARPS + warp;
    if (r >= *nlive) return;
    volatile int* vstate = state;
    if (vstate[r] != 0) return;   // warp-uniform read of a decided rank
    const double4 mr = rmodes[r];
    const double a[4] = {mr.x, mr.y, mr.z, mr.w};
    const double h2 = __dmul_rn(h, h);
    const float af[4] = {(float)mr.x, (float)mr.y, (float)mr.z, (float)mr.w};
    int lo[4], nr[4];
    const int total = ball_cells(af, d, (float)h, 1.0f / (float)h, lo, nr);
    const int nf = gather_cells(mukeys, mustart, mulen, *mncells, lo, nr, total, d, lane, s_cs[warp], s_pre[warp]);
    const int nmodes = s_pre[warp][nf];
    bool kept_near = false, pending = false;
    for (int f = lane; f < nmodes; f += 32) {
        const int j = cell_of_flat(s_pre[warp], nf, f);
        const int o = midx_sorted[s_cs[warp][j] + (f - s_pre[warp][j])];
        if (o >= r) continue;
        const double4 mo = rmodes[o];
        const double b[4] = {mo.x, mo.y, mo.z, mo.w};
        if (dist2_modes(a, b, d) <= h2) {
            const int so = vstate[o];
            kept_near |= (so == 1);
            pending |= (so == 0);
        }
    }
    kept_near = __any_sync(FULL, kept_near);
    pending = __any_sync(FULL, pending);
    if (lane == 0) {
        if (kept_near) {
            vstate[r] = 2;
        } else if (!pending) {
            vstate[r] = 1;
        } else {
            atomicAdd(undecided, 1);
        }
    }
}

__global__ void gbms_kept_flags_kernel(const int* __restrict__ state, const int* __restrict__ nlive, int nmax,
                                       int* flags) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nmax) flags[r] = (r < *nlive && state[r] == 1) ? 1 : 0;
}

__global__ void gbms_output_kernel(const int* __restrict__ flags, const int* __restrict__ pos,
                                   const int* __restrict__ nlive, const double4* __restrict__ rmodes,
                                   const int* __restrict__ rcount, int d, double* modes_out, int* counts_out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= *nlive || !flags[r]) return;
    const int k = pos[r];
    const double4 m = rmodes[r];
    const double mv[4] = {m.x, m.y, m.z, m.w};
    if (modes_out)
        for (int i = 0; i < d; ++i) modes_out[(size_t)d * k + i] = mv[i];
    if (counts_out) counts_out[k] = rcount[r];
}

}  // namespace

// ------------------------------------------------------------------ host side
size_t gbms_temp_bytes(int64_t n, int d) {
    size_t a = 0, b = 0, c = 0, e = 0;
    const int nn = (int)n;
    cub::DeviceRadixSort::SortPairs(nullptr, a, (const uint64_t*)nullptr, (uint64_t*)nullptr, (const int*)nullptr,
                                    (int*)nullptr, nn, 0, 16 * d);
    cub::DeviceRunLengthEncode::Encode(nullptr, b, (const uint64_t*)nullptr, (uint64_t*)nullptr, (int*)nullptr,
                                       (int*)nullptr, nn);
    cub::DeviceScan::ExclusiveSum(nullptr, c, (const int*)nullptr, (int*)nullptr, nn);
    cub::DeviceRadixSort::SortKeys(nullptr, e, (const uint64_t*)nullptr, (uint64_t*)nullptr, nn);
    return std::max(std::max(a, b), std::max(c, e));
}

cudaError_t launch_gbms_keys(const float* pts, int64_t n, int d, double h, float4* pts4, uint64_t* keys, int* idx,
                             DeviceState* st, cudaStream_t s) {
    gbms_keys_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts, n, d, h, pts4, keys, idx, st);
    return cudaGetLastError();
}

cudaError_t gbms_sort_cells(void* temp, size_t temp_bytes, const uint64_t* keys_in, uint64_t* keys_out,
                            const int* idx_in, int* idx_out, int64_t n, int d, uint64_t* ukeys, int* ulen,
                            int* ustart, int* ncells, cudaStream_t s) {
    size_t tb = temp_bytes;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(temp, tb, keys_in, keys_out, idx_in, idx_out, (int)n, 0, 16 * d, s);
    if (e != cudaSuccess) return e;
    tb = temp_bytes;
    e = cub::DeviceRunLengthEncode::Encode(temp, tb, keys_out, ukeys, ulen, ncells, (int)n, s);
    if (e != cudaSuccess) return e;
    tb = temp_bytes;
    return cub::DeviceScan::ExclusiveSum(temp, tb, ulen, ustart, (int)n, s);
}

cudaError_t launch_gbms_gather(const float4* pts4, const int* idx, int64_t n, float4* spts, longlong2* qxy,
                               longlong2* qzw, cudaStream_t s) {
    gbms_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts4, idx, n, spts, qxy, qzw);
    return cudaGetLastError();
}

cudaError_t launch_gbms_shift(const float4* spts, const longlong2* qxy, const longlong2* qzw, const uint64_t* ukeys,
                              const int* ustart, const int* ulen, int ncells, int d, double h, int max_iter,
                              double4* modes, int* counts, const DeviceState* st, cudaStream_t s) {
    gbms_shift_kernel<<<ncells, GB_SHIFT_THREADS, 0, s>>>(spts, qxy, qzw, ukeys, ustart, ulen, ncells, d, h, max_iter,
                                                           modes, counts, st);
    return cudaGetLastError();
}

cudaError_t launch_gbms_rank(void* temp, size_t temp_bytes, const int* counts, int ns, uint64_t* rkeys,
                             uint64_t* rkeys_sorted, int* nlive, cudaStream_t s) {
    gbms_rank_keys_kernel<<<(ns + 255) / 256, 256, 0, s>>>(counts, ns, rkeys, nlive);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t tb = temp_bytes;
    return cub::DeviceRadixSort::SortKeys(temp, tb, rkeys, rkeys_sorted, ns, 0, 64, s);
}

cudaError_t launch_gbms_rank_modes(const uint64_t* rkeys_sorted, const int* nlive, int nmax, const double4* modes,
                                   const int* counts, int d, double h, double4* rmodes, int* rcount, uint64_t* mkeys,
                                   int* midx, int* state, DeviceState* st, cudaStream_t s) {
    gbms_rank_modes_kernel<<<(nmax + 255) / 256, 256, 0, s>>>(rkeys_sorted, nlive, modes, counts, d, h, rmodes,
                                                              rcount, mkeys, midx, state, st);
    return cudaGetLastError();
}

cudaError_t launch_gbms_merge_round(const double4* rmodes, const int* nlive, int nmax, const uint64_t* mukeys,
                                    const int* mustart, const int* mulen, const int* mncells, const int* midx_sorted,
                                    int d, double h, int* state, int* undecided, cudaStream_t s) {
    gbms_merge_round_kernel<<<(nmax + GB_WARPS - 1) / GB_WARPS, GB_WARPS * 32, 0, s>>>(
        rmodes, nlive, mukeys, mustart, mulen, mncells, midx_sorted, d, h, state, undecided);
    return cudaGetLastError();
}

cudaError_t launch_gbms_output(void* temp, size_t temp_bytes, const int* state, const int* nlive, int nmax,
                               const double4* rmodes, const int* rcount, int d, int* flags, int* pos,
                               double* modes_out, int* counts_out, cudaStream_t s) {
    gbms_kept_flags_kernel<<<(nmax + 255) / 256, 256, 0, s>>>(state, nlive, nmax, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t tb = temp_bytes;
    e = cub::DeviceScan::ExclusiveSum(temp, tb, flags, pos, nmax, s);
    if (e != cudaSuccess) return e;
    gbms_output_kernel<<<(nmax + 255) / 256, 256, 0, s>>>(flags, pos, nlive, rmodes, rcount, d, modes_out,
                                                          counts_out);
    return cudaGetLastError();
}

}  // namespace gira
