// order_kernels.cu -- spatial order of the points for the point-stationary E-step.
//
// The E-step skips, per warp of 128 points, every component that cannot reach
// the box of those points (Eq. logestep: such a component's terms are exact
// zeros in binary32).  How much it skips depends on how compact a warp's
// points are.  Scans arrive in sensor order (image rows), where 128
// consecutive points span up to a couple of metres; here they are put in the
// order of an 18-bit Morton code (6 bits per axis) of their position in the
// bounding cube of their cloud, so that a warp holds a few neighbouring cells.
//
// The sort is a stable least-significant-digit radix sort on 9-bit digits,
// deterministic (no order decided by atomics): per tile of 512 keys a
// histogram, one exclusive scan over (digit, tile), and a scatter in which
// one warp walks its tile in order and ranks equal digits with match_any.  A
// batch sorts by (instance, code), which keeps every instance in its own range.
// Only the order of the per-point terms in the E-step's sums changes; the
// fit's k-means++ and Lloyd steps run on the points in the caller's order.
#include <stdint.h>

#include <algorithm>

#include "gira_internal.cuh"

namespace gira {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RADIX_BITS = 9;
constexpr int RADIX = 1 << RADIX_BITS;   // 512 digits
constexpr int TILE = 512;                // keys per histogram / scatter tile (one warp)
constexpr int BOX_CHUNK = 4096;          // points per bounding-box block
constexpr int SCAN_PER_BLOCK = 8192;     // scan: 1024 threads x 8
constexpr int MORTON_BITS = 18;

// float -> int with the same order (min / max by integer atomics)
__device__ __forceinline__ int ord_of(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float float_of(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7fffffff); }

// the instance of a block of points: unit table (batched) or one instance
struct Span {
    int inst;
    int64_t begin, end;
};
__device__ __forceinline__ Span span_of(const int64_t* offs, const int2* units, int64_t n) {
    Span s;
    if (units) {
        const int2 u = units[blockIdx.x];
        s.inst = u.x;
        s.begin = offs[u.x] + (int64_t)u.y * BOX_CHUNK;
        s.end = min(offs[u.x + 1], s.begin + BOX_CHUNK);
    } else {
        s.inst = 0;
        s.begin = (int64_t)blockIdx.x * BOX_CHUNK;
        s.end = min(n, s.begin + BOX_CHUNK);
    }
    return s;
}

__device__ __forceinline__ float3 point_of(const float4* p8, int64_t i) {
    const float4 a = p8[2 * i], b = p8[2 * i + 1];
    return make_float3(a.x, a.z, b.x);
}

// Bounding box of every instance: block = one chunk of one instance; the box is
// kept as order-preserving ints, [inst][6] = min x, y, z, max x, y, z.
__global__ void __launch_bounds__(256) box_kernel(const float4* __restrict__ p8, int64_t n,
                                                  const int64_t* __restrict__ offs, const int2* __restrict__ units,
                                                  int* box) {
    const Span s = span_of(offs, units, n);
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = s.begin + threadIdx.x; i < s.end; i += blockDim.x) {
        const float3 p = point_of(p8, i);
        lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
        hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
    }
    __shared__ float red[6][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[j] = fminf(lo[j], __shfl_xor_sync(FULL, lo[j], o));
            hi[j] = fmaxf(hi[j], __shfl_xor_sync(FULL, hi[j], o));
        }
        if (lane == 0) {
            red[j][warp] = lo[j];
            red[3 + j][warp] = hi[j];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int j = threadIdx.x;
        float v = red[j][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = j < 3 ? fminf(v, red[j][w]) : fmaxf(v, red[j][w]);
        if (v == v) {   // a NaN coordinate is reported by the packing step; keep it out of the box
            if (j < 3) atomicMin(box + 6 * s.inst + j, ord_of(v));
            else atomicMax(box + 6 * s.inst + j, ord_of(v));
        }
    }
}

__global__ void box_init_kernel(int* box, int batch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 6 * batch) box[i] = (i % 6) < 3 ? ord_of(INFINITY) : ord_of(-INFINITY);
}

__device__ __forceinline__ uint32_t spread6(uint32_t v) {   // bit i -> bit 3 i
    v &= 0x3fu;
    v = (v | (v << 8)) & 0x0000f00fu;
    v = (v | (v << 4)) & 0x000c30c3u;
    v = (v | (v << 2)) & 0x00249249u;
    return v;
}

// key = (instance << 18) | Morton code of the point in its instance's bounding
// cube (cells of the largest extent / 64 on every axis); idx = the point
__global__ void __launch_bounds__(256) key_kernel(const float4* __restrict__ p8, int64_t n,
                                                  const int64_t* __restrict__ offs, const int2* __restrict__ units,
                                                  const int* __restrict__ box, uint32_t* keys, int* idx) {
    const Span s = span_of(offs, units, n);
    const int* bb = box + 6 * s.inst;
    const float lo[3] = {float_of(bb[0]), float_of(bb[1]), float_of(bb[2])};
    const float ext = fmaxf(fmaxf(float_of(bb[3]) - lo[0], float_of(bb[4]) - lo[1]), float_of(bb[5]) - lo[2]);
    const float scale = ext > 0.f ? 64.f / ext : 0.f;
    for (int64_t i = s.begin + threadIdx.x; i < s.end; i += blockDim.x) {
        const float3 p = point_of(p8, i);
        const float c[3] = {p.x, p.y, p.z};
        uint32_t code = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // fmaxf / fminf map a NaN to the bound: every key is a valid digit string
            const float q = fminf(63.f, fmaxf(0.f, floorf((c[j] - lo[j]) * scale)));
            code |= spread6((uint32_t)q) << j;
        }
        keys[i] = ((uint32_t)s.inst << MORTON_BITS) | code;
        idx[i] = (int)i;
    }
}

// Per tile (one warp, TILE keys): the count of every digit, stored digit-major
// ([digit][tile]) so that one exclusive scan gives every tile's output offsets.
__global__ void __launch_bounds__(256) radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                         int ntiles, int* counts) {
    __shared__ int hist[8][RADIX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * 8 + warp;
    int* h = hist[warp];
    for (int d = lane; d < RADIX; d += 32) h[d] = 0;
    __syncwarp();
    if (tile < ntiles) {
        const int64_t b = (int64_t)tile * TILE, e = min(n, b + TILE);
        for (int64_t i0 = b; i0 < e; i0 += 32) {   // equal digits of the 32 keys counted once
            const int64_t i = i0 + lane;
            const int d = i < e ? (int)((keys[i] >> shift) & (RADIX - 1)) : RADIX;
            const uint32_t peers = __match_any_sync(FULL, d);
            if (d < RADIX && (peers & ((1u << lane) - 1u)) == 0u) h[d] += __popc(peers);
            __syncwarp();
        }
        for (int d = lane; d < RADIX; d += 32) counts[(size_t)d * ntiles + tile] = h[d];
    }
}

// Exclusive scan of m ints in place: block sums, a scan of the block sums
// (one block), then every block's local scan plus its offset.
__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const int before = (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
    if (total) *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(1024) scan_sums_kernel(const int* __restrict__ a, int64_t m, int* bsum) {
    __shared__ int s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_PER_BLOCK + 8 * threadIdx.x;
    int v = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (base + j < m) v += a[base + j];
    int total;
    block_exclusive_scan(v, s_warp, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_bsum_kernel(int* bsum, int nb) {
    __shared__ int s_warp[32];
    int v[8], t = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = 8 * threadIdx.x + j;
        v[j] = i < nb ? bsum[i] : 0;
        t += v[j];
    }
    int run = block_exclusive_scan(t, s_warp, nullptr);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = 8 * threadIdx.x + j;
        if (i < nb) bsum[i] = run;
        run += v[j];
    }
}

// (writes the offsets tile-major too, [tile][digit], for the scatter's coalesced loads)
__global__ void __launch_bounds__(1024) scan_apply_kernel(const int* __restrict__ a, int64_t m,
                                                          const int* __restrict__ bsum, int ntiles, int* at) {
    __shared__ int s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_PER_BLOCK + 8 * threadIdx.x;
    int v[8], t = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        v[j] = base + j < m ? a[base + j] : 0;
        t += v[j];
    }
    int run = block_exclusive_scan(t, s_warp, nullptr) + bsum[blockIdx.x];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (base + j < m) {
            const int i = (int)(base + j);   // digit i / ntiles, tile i % ntiles (m < 2^31)
            at[(size_t)(i % ntiles) * RADIX + i / ntiles] = run;
        }
        run += v[j];
    }
}

// Stable scatter: one warp walks its tile 32 keys at a time, in order; lanes with
// equal digits rank among themselves (match_any) after the count of that digit so
// far in the tile, which starts at the tile's scanned offset.  The tile's keys and
// indices are loaded before the walk (all loads in flight at once).
constexpr int SC_ROUNDS = TILE / 32;
__global__ void __launch_bounds__(256) radix_scatter_kernel(const uint32_t* __restrict__ keys_in,
                                                            const int* __restrict__ idx_in, int64_t n, int shift,
                                                            int ntiles, const int* __restrict__ offs,
                                                            uint32_t* keys_out, int* idx_out) {
    __shared__ int cnt[8][RADIX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * 8 + warp;
    if (tile >= ntiles) return;
    const int64_t b = (int64_t)tile * TILE, e = min(n, b + TILE);
    uint32_t key[SC_ROUNDS];
    int src[SC_ROUNDS];
#pragma unroll
    for (int r = 0; r < SC_ROUNDS; ++r) {
        const int64_t i = b + r * 32 + lane;
        key[r] = i < e ? keys_in[i] : 0u;
        src[r] = i < e ? idx_in[i] : 0;
    }
    int* c = cnt[warp];
    for (int d = lane; d < RADIX; d += 32) c[d] = offs[(size_t)tile * RADIX + d];   // tile-major offsets
    __syncwarp();
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < SC_ROUNDS; ++r) {
        const bool valid = b + r * 32 + lane < e;
        const int d = valid ? (int)((key[r] >> shift) & (RADIX - 1)) : RADIX;   // RADIX: no slot
        const uint32_t peers = __match_any_sync(FULL, d);
        const int pos = valid ? c[d] + __popc(peers & lt) : 0;
        __syncwarp();
        if (valid && (peers & lt) == 0u) c[d] += __popc(peers);   // the lowest lane of each digit
        __syncwarp();
        if (valid && pos >= 0 && pos < n) {   // (the scanned counts place every key inside [0, n))
            keys_out[pos] = key[r];
            idx_out[pos] = src[r];
        }
    }
}

// The points in the sorted order: p8_out[j] = p8[order[j]] (and p4_out: (x, y, z, 0)).
__global__ void __launch_bounds__(256) gather_kernel(const int* __restrict__ order, int64_t n,
                                                     const float4* __restrict__ p8, float4* p8_out, float4* p4_out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t s = order[j];
    if (s < 0 || s >= n) return;
    const float4 a = p8[2 * s], b = p8[2 * s + 1];
    p8_out[2 * j] = a;
    p8_out[2 * j + 1] = b;
    if (p4_out) p4_out[j] = make_float4(a.x, a.z, b.x, 0.f);
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int radix_passes(int batch) {
    int bits = MORTON_BITS;
    while (batch > 1 && (1 << (bits - MORTON_BITS)) < batch) ++bits;
    return (int)ceil_div(bits, RADIX_BITS);
}

}  // namespace

int64_t point_order_box_units(const int64_t* offsets, int batch) {
    int64_t u = 0;
    for (int i = 0; i < batch; ++i) u += ceil_div(offsets[i + 1] - offsets[i], BOX_CHUNK);
    return u;
}

void point_order_fill_units(const int64_t* offsets, int batch, int2* units) {
    int64_t u = 0;
    for (int i = 0; i < batch; ++i)
        for (int64_t c = 0; c * BOX_CHUNK < offsets[i + 1] - offsets[i]; ++c) units[u++] = make_int2(i, (int)c);
}

int point_order_launches(int batch) { return 4 + 5 * radix_passes(batch); }   // with the gather

// the largest n the scan's two levels hold (every tile's 512 digit counts)
int64_t point_order_max_n() { return (int64_t)SCAN_PER_BLOCK * SCAN_PER_BLOCK / RADIX * TILE; }

size_t point_order_scratch_bytes(int64_t n, int batch) {
    const int64_t ntiles = ceil_div(n, TILE);
    const int64_t m = ntiles * RADIX;
    size_t bytes = 0;
    auto add = [&](size_t b) { bytes += (b + 255) & ~size_t(255); };
    add(sizeof(int) * 6 * (size_t)batch);   // boxes
    add(sizeof(uint32_t) * n);              // keys, two buffers
    add(sizeof(uint32_t) * n);
    add(sizeof(int) * n);                   // indices, two buffers
    add(sizeof(int) * n);
    add(sizeof(int) * m);                   // digit counts, digit-major
    add(sizeof(int) * m);                   // their offsets, tile-major
    add(sizeof(int) * ceil_div(m, SCAN_PER_BLOCK));
    return bytes;
}

cudaError_t launch_point_order(const float4* p8, int64_t n, const int64_t* offsets_d, const int2* units_d,
                               int nunits, int batch, void* scratch, float4* p8_out, float4* p4_out, int* order_out,
                               cudaStream_t s) {
    const int64_t ntiles = ceil_div(n, TILE);
    const int64_t m = ntiles * RADIX;
    const int64_t nb = ceil_div(m, SCAN_PER_BLOCK);
    if (nb > SCAN_PER_BLOCK || n > INT32_MAX) return cudaErrorInvalidValue;
    char* p = static_cast<char*>(scratch);
    auto take = [&](size_t b) {
        char* r = p;
        p += (b + 255) & ~size_t(255);
        return r;
    };
    int* box = reinterpret_cast<int*>(take(sizeof(int) * 6 * (size_t)batch));
    uint32_t* k0 = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    uint32_t* k1 = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    int* i0 = reinterpret_cast<int*>(take(sizeof(int) * n));
    int* i1 = reinterpret_cast<int*>(take(sizeof(int) * n));
    int* counts = reinterpret_cast<int*>(take(sizeof(int) * m));
    int* toffs = reinterpret_cast<int*>(take(sizeof(int) * m));
    int* bsum = reinterpret_cast<int*>(take(sizeof(int) * nb));

    box_init_kernel<<<(unsigned)ceil_div(6 * (int64_t)batch, 256), 256, 0, s>>>(box, batch);
    const int blocks = units_d ? nunits : (int)ceil_div(n, BOX_CHUNK);
    box_kernel<<<blocks, 256, 0, s>>>(p8, n, offsets_d, units_d, box);
    key_kernel<<<blocks, 256, 0, s>>>(p8, n, offsets_d, units_d, box, k0, i0);
    const int passes = radix_passes(batch);
    const unsigned tblocks = (unsigned)ceil_div(ntiles, 8);
    int *iin = i0, *iout = i1;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * RADIX_BITS;
        const bool last = pass == passes - 1;
        radix_hist_kernel<<<tblocks, 256, 0, s>>>(k0, n, shift, (int)ntiles, counts);
        scan_sums_kernel<<<(unsigned)nb, 1024, 0, s>>>(counts, m, bsum);
        scan_bsum_kernel<<<1, 1024, 0, s>>>(bsum, (int)nb);
        scan_apply_kernel<<<(unsigned)nb, 1024, 0, s>>>(counts, m, bsum, (int)ntiles, toffs);
        int* io = (last && order_out) ? order_out : iout;
        radix_scatter_kernel<<<tblocks, 256, 0, s>>>(k0, iin, n, shift, (int)ntiles, toffs, k1, io);
        std::swap(k0, k1);
        iout = iin;   // the input indices are free for the next pass's output
        iin = io;
    }
    if (p8_out) gather_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(iin, n, p8, p8_out, p4_out);
    return cudaGetLastError();
}

}  // namespace gira
