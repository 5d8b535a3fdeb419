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

#include "gira_internal.cuh"

namespace gira {

namespace {
constexpr unsigned FULL = 0xffffffffu;
constexpr int KPP_THREADS = 256;
constexpr int KPP_ITEMS = 8;
constexpr int KPP_CHUNK = KPP_THREADS * KPP_ITEMS;   // points per update block
constexpr int SEL_THREADS = 1024;

// Deterministic block-wide binary64 sum (fixed tree); result valid in thread 0.
template <int THREADS>
__device__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < THREADS / 32; ++w) r += sh[w];
    __syncthreads();
    return r;
}

// Block-wide inclusive scan of one binary64 value per thread (fixed order).
template <int THREADS>
__device__ double block_incl_scan(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = (lane < THREADS / 32) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double u = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += u;
        }
        if (lane < THREADS / 32) sh[lane] = w;   // inclusive warp prefix
    }
    __syncthreads();
    if (warp > 0) v += sh[warp - 1];
    __syncthreads();
    return v;
}

__device__ int block_min_int(int v, int* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    int r = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = min(r, sh[w]);
    __syncthreads();
    return r;
}

__device__ long long block_max_ll(long long v, long long* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, (long long)__shfl_xor_sync(FULL, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    long long r = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = max(r, sh[w]);
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- k-means++
__global__ void kpp_first_kernel(const float4* __restrict__ pts, int64_t n, uint64_t seed, float4* centers,
                                 int64_t* chosen, DeviceState* st) {
    if (st->error) return;
    int64_t idx = (int64_t)floor(uniform53(seed, 0) * (double)n);
    if (idx > n - 1) idx = n - 1;
    centers[0] = pts[idx];
    chosen[0] = idx;
}

// D^2(x) = min(D^2(x), ||x - c_{j-1}||^2) and the binary64 sum of each chunk.
__global__ void __launch_bounds__(KPP_THREADS) kpp_update_kernel(const float4* __restrict__ pts, int64_t n,
                                                                 const float4* __restrict__ centers, int j,
                                                                 float* __restrict__ d2, double* blocksums,
                                                                 DeviceState* st) {
    __shared__ double sh[KPP_THREADS / 32];
    if (st->error) return;
    const float4 c = centers[j - 1];
    const int64_t base = (int64_t)blockIdx.x * KPP_CHUNK;
    double acc = 0.0;
#pragma unroll
    for (int it = 0; it < KPP_ITEMS; ++it) {
        const int64_t i = base + it * KPP_THREADS + threadIdx.x;
        if (i < n) {
            float d = dist2_f32(pts[i], c);
            if (j > 1) d = fminf(d2[i], d);
            d2[i] = d;
            acc += (double)d;
        }
    }
    const double tot = block_sum<KPP_THREADS>(acc, sh);
    if (threadIdx.x == 0) blocksums[blockIdx.x] = tot;
}

// Draw centre j: the first point whose running binary64 sum of D^2 exceeds
// t = u_j * sum D^2 (u_j = draw j of the seed's SplitMix64 stream).  Every
// prefix used below comes from one chain of sequential additions per thread
// plus fixed-order scans, so the search is self-consistent.
__global__ void __launch_bounds__(SEL_THREADS) kpp_select_kernel(const float4* __restrict__ pts, int64_t n,
                                                                 const float* __restrict__ d2,
                                                                 const double* __restrict__ blocksums, int nblk,
                                                                 uint64_t seed, int j, float4* centers,
                                                                 int64_t* chosen, DeviceState* st) {
    __shared__ double sh[SEL_THREADS / 32];
    __shared__ double sh_incl[SEL_THREADS];
    __shared__ int shi[SEL_THREADS / 32];
    __shared__ long long shl[SEL_THREADS / 32];
    __shared__ double s_total, s_excl;
    if (st->error) return;
    const int per = (nblk + SEL_THREADS - 1) / SEL_THREADS;   // consecutive chunks per thread
    const int b0 = threadIdx.x * per;
    double local = 0.0;
    for (int i = 0; i < per && b0 + i < nblk; ++i) local += blocksums[b0 + i];
    sh_incl[threadIdx.x] = block_incl_scan<SEL_THREADS>(local, sh);
    __syncthreads();
    const double thread_excl = threadIdx.x ? sh_incl[threadIdx.x - 1] : 0.0;
    if (threadIdx.x == 0) s_total = sh_incl[SEL_THREADS - 1];
    __syncthreads();
    const double total = s_total;
    const double u = uniform53(seed, (uint64_t)j);
    int64_t idx = -1;
    if (total > 0.0) {
        const double t = u * total;
        // first chunk whose inclusive prefix exceeds t; remember its exclusive prefix
        double run = thread_excl, before = 0.0;
        int cand = INT_MAX;
        for (int i = 0; i < per && b0 + i < nblk; ++i) {
            before = run;
            run += blocksums[b0 + i];
            if (run > t) { cand = b0 + i; break; }
        }
        int kb = block_min_int(cand, shi);
        if (kb != INT_MAX && cand == kb) s_excl = before;
        __syncthreads();
        double excl = (kb != INT_MAX) ? s_excl : 0.0;
        while (kb < nblk) {
            const int64_t p0 = (int64_t)kb * KPP_CHUNK + 2 * threadIdx.x;
            const double v0 = (p0 < n) ? (double)d2[p0] : 0.0;
            const double v1 = (p0 + 1 < n) ? (double)d2[p0 + 1] : 0.0;
            sh_incl[threadIdx.x] = block_incl_scan<SEL_THREADS>(v0 + v1, sh);
            __syncthreads();
            const double in_excl = threadIdx.x ? sh_incl[threadIdx.x - 1] : 0.0;
            const double r0 = (excl + in_excl) + v0;
            const double r1 = r0 + v1;
            int c2 = INT_MAX;
            if (p0 < n && r0 > t) c2 = 2 * threadIdx.x;
            else if (p0 + 1 < n && r1 > t) c2 = 2 * threadIdx.x + 1;
            const int w = block_min_int(c2, shi);
            if (w != INT_MAX) { idx = (int64_t)kb * KPP_CHUNK + w; break; }
            excl += blocksums[kb];   // rounding put t past this chunk: continue with the next
            ++kb;
        }
        if (idx < 0) {   // t rounded up to the total: the last point with D^2 > 0
            long long last = -1;
            for (int64_t i = threadIdx.x; i < n; i += SEL_THREADS)
                if (d2[i] > 0.f) last = i;
            idx = block_max_ll(last, shl);
            if (idx < 0) idx = 0;   // unreachable for finite D^2 (total > 0 implies a positive term)
        }
    } else {   // every point coincides with a chosen centre: uniform index
        idx = (int64_t)floor(u * (double)n);
        if (idx > n - 1) idx = n - 1;
    }
    if (threadIdx.x == 0) {
        centers[j] = pts[idx];
        chosen[j] = idx;
        st->chosen_last = idx;
    }
}

// ---------------------------------------------------------------- Lloyd
// labels = argmin_b ||x - c_b||^2 (binary32, ties to the lowest b); binary64
// sums of the raw coordinates and counts per label; changed[it] counts labels
// that moved (every label for it == 0).
__global__ void lloyd_assign_kernel(const float4* __restrict__ pts, int64_t n, int k, const float4* __restrict__ centers,
                                    int32_t* labels, double* sums, unsigned long long* changed, int it,
                                    DeviceState* st) {
    extern __shared__ float4 sc[];
    if (st->error) return;
    if (it > 0 && changed[it - 1] == 0) return;
    for (int b = threadIdx.x; b < k; b += blockDim.x) sc[b] = centers[b];
    __syncthreads();
    unsigned long long cnt = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 x = pts[i];
        int best = 0;
        float bd = dist2_f32(x, sc[0]);
        for (int b = 1; b < k; ++b) {
            const float d = dist2_f32(x, sc[b]);
            if (d < bd) { bd = d; best = b; }
        }
        if (it == 0 || labels[i] != best) ++cnt;
        labels[i] = best;
        atomicAdd(&sums[4 * best + 0], (double)x.x);
        atomicAdd(&sums[4 * best + 1], (double)x.y);
        atomicAdd(&sums[4 * best + 2], (double)x.z);
        atomicAdd(&sums[4 * best + 3], 1.0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&changed[it], cnt);
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

// One-hot statistics about the shift s_b (the final centre): S0 = count,
// S1 = sum (x - s), S2 = sum (x - s)(x - s)^T, binary64.
__global__ void label_stats_kernel(const float4* __restrict__ pts, int64_t n, int k, const int32_t* __restrict__ labels,
                                   const float4* __restrict__ shift4, double* stats64, DeviceState* st) {
    if (st->error) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = labels[i];
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

cudaError_t launch_kpp(const float4* pts4, int64_t n, int k, uint64_t seed, float4* centers, float* d2,
                       double* blocksums, int64_t* chosen, DeviceState* st, cudaStream_t s) {
    const int nblk = kpp_num_blocks(n);
    kpp_first_kernel<<<1, 1, 0, s>>>(pts4, n, seed, centers, chosen, st);
    for (int j = 1; j < k; ++j) {
        kpp_update_kernel<<<nblk, KPP_THREADS, 0, s>>>(pts4, n, centers, j, d2, blocksums, st);
        kpp_select_kernel<<<1, SEL_THREADS, 0, s>>>(pts4, n, d2, blocksums, nblk, seed, j, centers, chosen, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_lloyd(const float4* pts4, int64_t n, int k, int lloyd_iters, float4* centers, int32_t* labels,
                         double* sums, unsigned long long* changed, DeviceState* st, cudaStream_t s) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = sizeof(float4) * (size_t)k;
    const int threads = 256;
    const int64_t want = (n + threads - 1) / threads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
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

cudaError_t launch_label_stats(const float4* pts4, int64_t n, int k, const int32_t* labels, const float4* shift4,
                               double* stats64, DeviceState* st, cudaStream_t s) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    label_stats_kernel<<<grid, 256, 0, s>>>(pts4, n, k, labels, shift4, stats64, st);
    return cudaGetLastError();
}

cudaError_t launch_centers_out(const float4* centers4, int k, float* centers3, cudaStream_t s) {
    centers_out_kernel<<<(k + 127) / 128, 128, 0, s>>>(centers4, k, centers3);
    return cudaGetLastError();
}

}  // namespace gira
