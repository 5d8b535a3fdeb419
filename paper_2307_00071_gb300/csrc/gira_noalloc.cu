// gira_noalloc.cu -- gira_gmm_loglik_noalloc: the log-likelihood entry point for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: real-time loops on a robot that forbid
// allocation after start-up (an allocation can block for an unbounded time and
// can fail in the middle of a mission), and hosts whose device memory is
// handed out by a pool they do not control (memory the library took would be
// missing from the pool's budget).  This entry point computes exactly what
// gira_gmm_loglik computes, with the same kernels, but its scratch memory
// (packed points, component parameters, per-CTA partial sums, the device
// status word) lives in one file-scope __device__ array of
// NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds that array
// until the process exits.
#include <cuda_runtime.h>

#include <climits>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

#include "gira_internal.cuh"

using namespace gira;

namespace {

constexpr int64_t NOALLOC_MAX_N = GIRA_NOALLOC_MAX_N;
constexpr int NOALLOC_MAX_CTAS = 4096;
constexpr size_t NOALLOC_SCRATCH_BYTES = 17u << 20;   // 17 MiB

// The scratch.  In host code this name is only a host-side stand-in: its
// device address comes from cudaGetSymbolAddress (see scratch_for_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

gira_status na_fail(gira_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    record_error(buf, -1);
    return s;
}

#define NA_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return na_fail(GIRA_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
        }                                                                                   \
    } while (0)

std::mutex g_na_mu;                 // serialises calls from host threads (not GPU-side overlap)
std::vector<void*> g_na_scratch;    // device address of g_noalloc_scratch, per device

// Once per device, with that device current: the device address of the array.
gira_status scratch_for_device(int dev, unsigned char** out) {
    if ((int)g_na_scratch.size() <= dev) g_na_scratch.resize(dev + 1, nullptr);
    if (!g_na_scratch[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return na_fail(GIRA_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) failed: %s",
                           cudaGetErrorString(e));
        }
        g_na_scratch[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_na_scratch[dev]);
    return GIRA_OK;
}

bool is_device_ptr(const void* p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" gira_status gira_gmm_loglik_noalloc(const float* points, int64_t n, int k, const float* weights,
                                               const float* means, const float* covs, double* mean_loglik,
                                               float* per_point, void* stream) {
    record_error("", -1);
    if (n < 1 || n > NOALLOC_MAX_N)
        return na_fail(GIRA_ERR_INVALID_ARG, "n = %lld outside [1, %lld] (the no-allocation limit)", (long long)n,
                       (long long)NOALLOC_MAX_N);
    if (k < 1 || k > GIRA_MAX_K_BATCHED || k > n) return na_fail(GIRA_ERR_INVALID_ARG, "k = %d outside [1, min(n, %d)]", k, GIRA_MAX_K_BATCHED);
    if (!points || !weights || !means || !covs) return na_fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    {   // the call reads its status back to the host and synchronises the stream, neither of
        // which a stream under capture allows: refuse before any other CUDA call
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        NA_CUDA(cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return na_fail(GIRA_ERR_INVALID_ARG, "the stream is being captured; this call synchronises it");
    }
    int dev = 0, sms = 1;
    NA_CUDA(cudaGetDevice(&dev));
    NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (!is_device_ptr(points, dev) || !is_device_ptr(weights, dev) || !is_device_ptr(means, dev) ||
        !is_device_ptr(covs, dev) || (per_point && !is_device_ptr(per_point, dev)))
        return na_fail(GIRA_ERR_INVALID_ARG, "every array must be device memory of the current device");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    std::lock_guard<std::mutex> lk(g_na_mu);
    unsigned char* base = nullptr;
    gira_status st0 = scratch_for_device(dev, &base);
    if (st0 != GIRA_OK) return st0;

    const int npairs = params_pairs_padded(k);
    const int grid = estep_pt_grid(n);
    if (grid > NOALLOC_MAX_CTAS) return na_fail(GIRA_ERR_INVALID_ARG, "launch needs %d CTAs > %d", grid, NOALLOC_MAX_CTAS);
    // carve the scratch
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = align256(off);
        unsigned char* p = base + off;
        off += bytes;
        return p;
    };
    DeviceState* st = reinterpret_cast<DeviceState*>(take(sizeof(DeviceState)));
    float4* p8 = reinterpret_cast<float4*>(take(2 * sizeof(float4) * (size_t)n));
    float* params = reinterpret_cast<float*>(take(sizeof(float) * (size_t)npairs * PAIR_FLOATS));
    float4* shift4 = reinterpret_cast<float4*>(take(sizeof(float4) * (size_t)k));
    double* model64 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)k * MODEL));
    double* llp = reinterpret_cast<double*>(take(sizeof(double) * (size_t)grid));
    if (off > NOALLOC_SCRATCH_BYTES)
        return na_fail(GIRA_ERR_INVALID_ARG, "call needs %zu bytes of scratch > %zu", off, NOALLOC_SCRATCH_BYTES);

    // The array keeps the previous call's contents: the status word is reset
    // here; every other region is fully rewritten below before it is read.
    DeviceState h{};
    h.stop_after = 0;
    h.bad_component = INT_MAX;
    NA_CUDA(cudaMemcpyAsync(st, &h, sizeof h, cudaMemcpyHostToDevice, s));
    NA_CUDA(launch_pack(points, n, nullptr, p8, st, s));
    NA_CUDA(launch_fill_padding(params, k, npairs, s));
    NA_CUDA(launch_params_from_model(weights, means, covs, k, model64, params, shift4, st, s));
    EStepLaunch a{p8, n, k, params, 0, nullptr, llp, per_point, st, 0};
    a.n_buf = n;
    NA_CUDA(launch_estep_pt(a, false, grid, s));
    NA_CUDA(launch_ll_reduce(llp, grid, st, s));
    NA_CUDA(cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    const gira_status dst = device_status(h);   // the allocating entry points' mapping and messages
    if (dst != GIRA_OK) return dst;
    if (mean_loglik) *mean_loglik = h.ll_sum / (double)n;
    return GIRA_OK;
}
