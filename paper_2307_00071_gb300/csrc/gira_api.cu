// gira_api.cu -- the extern "C" entry points declared in include/gira.h.
//
// Host-side orchestration only: argument validation, the per-device workspace,
// staging of host buffers, and the stream-ordered launch sequence
//   pack -> KInit (k-means++, Lloyd, one-hot M-step) or caller parameters
//        -> iters x [fused E-step/statistics -> reduce -> FP64 finalize]
//        -> final log-likelihood -> model out.
// Every arithmetic step of the method runs in the CUDA kernels; no loop waits
// on the host between EM iterations (convergence is decided on the device).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gira_internal.cuh"

using namespace gira;

namespace {

// One NVTX range per library call (visible in Nsight Systems; no cost without a tool attached).
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
};

thread_local std::string t_msg;
thread_local int t_bad = -1;

gira_status fail(gira_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_msg = buf;
    return s;
}

#define GIRA_CUDA(call)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError();                                                               \
            return fail(GIRA_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
        }                                                                                     \
    } while (0)

// ---------------------------------------------------------------- workspace
struct DeviceWs {
    std::mutex mu;
    void* ptr = nullptr;
    size_t bytes = 0;
    // the last batched-EM graph (valid for this workspace allocation only)
    std::string graph_key;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t capture_stream = nullptr;
};

void drop_graph(DeviceWs* ws) {
    if (ws->graph_exec) cudaGraphExecDestroy(ws->graph_exec);
    ws->graph_exec = nullptr;
    ws->graph_key.clear();
}
std::mutex g_table_mu;
std::vector<DeviceWs*> g_ws;

DeviceWs* ws_for(int dev) {
    std::lock_guard<std::mutex> lk(g_table_mu);
    if ((int)g_ws.size() <= dev) g_ws.resize(dev + 1, nullptr);
    if (!g_ws[dev]) g_ws[dev] = new DeviceWs();
    return g_ws[dev];
}

// Bump allocator: run once with base == nullptr to size, then for real.
struct Carver {
    char* base = nullptr;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += std::max<size_t>(count, 1) * sizeof(T);
        return p;
    }
};

std::atomic<int> g_fail_allocs{0};   // test hook: workspace allocations still to fail

gira_status ensure(DeviceWs* ws, size_t need, cudaStream_t s) {
    if (ws->bytes >= need) return GIRA_OK;
    if (g_fail_allocs.load() > 0 && g_fail_allocs.fetch_sub(1) > 0)
        return fail(GIRA_ERR_OOM, "workspace allocation of %zu bytes failed (injected by the test hook)", need);
    GIRA_CUDA(cudaStreamSynchronize(s));
    drop_graph(ws);
    if (ws->ptr) GIRA_CUDA(cudaFree(ws->ptr));
    ws->ptr = nullptr;
    ws->bytes = 0;
    size_t want = need + need / 4;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&p, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GIRA_ERR_OOM, "cannot allocate %zu bytes of device workspace: %s", need,
                        cudaGetErrorString(e));
        }
        want = need;
    }
    ws->ptr = p;
    ws->bytes = want;
    return GIRA_OK;
}

// ---------------------------------------------------------------- pointers
enum class Kind { Host, Device, Foreign };

Kind kind_of(const void* p, int dev) {
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return Kind::Host;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return a.device == dev ? Kind::Device : Kind::Foreign;
    return Kind::Host;
}

struct Ctx {
    int dev = 0, sms = 1;
    cudaStream_t s = nullptr;
};

void reset_error() {
    t_msg.clear();
    t_bad = -1;
}

gira_status begin(Ctx& c, void* stream) {
    GIRA_CUDA(cudaGetDevice(&c.dev));
    GIRA_CUDA(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, c.dev));
    c.s = reinterpret_cast<cudaStream_t>(stream);
    return GIRA_OK;
}

gira_status check_ptr(const void* p, const char* name, int dev, Kind* k) {
    *k = kind_of(p, dev);
    if (*k == Kind::Foreign) return fail(GIRA_ERR_INVALID_ARG, "%s is device memory of another device", name);
    return GIRA_OK;
}

gira_status check_nk(int64_t n, int k) {
    if (n < 1) return fail(GIRA_ERR_INVALID_ARG, "n = %lld < 1", (long long)n);
    if (k < 1 || k > GIRA_MAX_K) return fail(GIRA_ERR_INVALID_ARG, "k = %d outside [1, %d]", k, GIRA_MAX_K);
    if (k > n) return fail(GIRA_ERR_INVALID_ARG, "k = %d > n = %lld", k, (long long)n);
    return GIRA_OK;
}

gira_status check_opts(const gira_fit_opts& o) {
    if (o.iters < 0) return fail(GIRA_ERR_INVALID_ARG, "iters < 0");
    if (!(o.tol >= 0.0)) return fail(GIRA_ERR_INVALID_ARG, "tol must be >= 0");
    if (!(o.reg_covar >= 0.0) || !std::isfinite(o.reg_covar))
        return fail(GIRA_ERR_INVALID_ARG, "reg_covar must be finite and >= 0");
    if (o.lloyd_iters < 0) return fail(GIRA_ERR_INVALID_ARG, "lloyd_iters < 0");
    if (o.init_mode != GIRA_INIT_KMEANS && o.init_mode != GIRA_INIT_PARAMS)
        return fail(GIRA_ERR_INVALID_ARG, "unknown init_mode %d", o.init_mode);
    return GIRA_OK;
}

#define TRY(x)                          \
    do {                                \
        gira_status st_ = (x);          \
        if (st_ != GIRA_OK) return st_; \
    } while (0)

#define LAUNCH(x) GIRA_CUDA(x)
#define COUNTED(prof, n, x) \
    do {                      \
        LAUNCH(x);            \
        (prof).launches += (n); \
    } while (0)

// ---------------------------------------------------------------- profiling
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
gira_profile g_prof{};

// Events of one call: phase marks plus a pair per E-step launch.
struct CallProfile {
    bool on = false;
    bool per_launch = false;   // an event pair around every E-step launch (plain launches)
    cudaStream_t s = nullptr;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    cudaEvent_t t0 = nullptr, t_init = nullptr, t_em = nullptr, t_end = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> estep;
    std::string estep_name;   // the kernel those event pairs bracket
    long long launches = 0;
    long long pair_slots = 0, pairs_near = 0, pairs_live = 0;   // point-stationary E-step pair counts

    void timed(cudaEvent_t e0, cudaEvent_t e1) {
        estep.emplace_back(e0, e1);
        estep_name = last_estep_kernel();
    }

    cudaEvent_t mark_launch() { return per_launch ? mark() : nullptr; }
    cudaEvent_t mark() {
        if (!on) return nullptr;
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
            pool.push_back(e);
        }
        cudaEvent_t e = pool[used++];
        cudaEventRecord(e, s);
        return e;
    }
    ~CallProfile() {
        for (auto e : pool) cudaEventDestroy(e);
    }
    static double ms(cudaEvent_t a, cudaEvent_t b) {
        float v = 0.f;
        if (!a || !b || cudaEventElapsedTime(&v, a, b) != cudaSuccess) { cudaGetLastError(); return 0.0; }
        return v;
    }
    // after the stream has been synchronised
    void commit(int em_iters, int estep_done) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof.calls += 1;
        g_prof.kernel_launches += launches;
        if (!on) return;
        for (int i = 0; i < (int)estep.size() && i < estep_done; ++i) g_prof.estep_ms += ms(estep[i].first, estep[i].second);
        g_prof.estep_launches += std::min<long long>((long long)estep.size(), estep_done);
        if (per_launch) {
            g_prof.estep_pair_slots += pair_slots;
            g_prof.estep_pairs_near += pairs_near;
            g_prof.estep_pairs_live += pairs_live;
        }
        if (!estep_name.empty()) {
            std::strncpy(g_prof.estep_kernel, estep_name.c_str(), sizeof g_prof.estep_kernel - 1);
            g_prof.estep_kernel[sizeof g_prof.estep_kernel - 1] = 0;
        }
        g_prof.em_iters += em_iters;
        g_prof.init_ms += ms(t0, t_init);
        g_prof.em_ms += ms(t_init, t_em);
        g_prof.total_ms += ms(t0, t_end);
    }
};

}  // namespace

void gira::record_error(const char* msg, int component) {
    if (msg) t_msg = msg;
    t_bad = component;
}

gira_status gira::device_status(const DeviceState& h) {
    switch (h.error) {
        case 0: return GIRA_OK;
        case GIRA_ERR_NONFINITE_INPUT: return fail(GIRA_ERR_NONFINITE_INPUT, "NaN or Inf in the points or parameters");
        case GIRA_ERR_NOT_PD:
            t_bad = h.bad_component;
            return fail(GIRA_ERR_NOT_PD, "covariance of component %d is not positive definite", h.bad_component);
        case GIRA_ERR_INVALID_ARG: return fail(GIRA_ERR_INVALID_ARG, "a mixture weight is not positive");
        case GIRA_ERR_NUMERIC:
            return fail(GIRA_ERR_NUMERIC, "a point's likelihood underflows binary32 under every component");
        case GIRA_ERR_TIMEOUT: return fail(GIRA_ERR_TIMEOUT, "a bounded device-side wait ran out (k-means++ seeding)");
        case GIRA_ERR_BOUNDS: return fail(GIRA_ERR_BOUNDS, "a device-side index fell outside its buffer (debug build)");
        default: return fail((gira_status)h.error, "device error %d", h.error);
    }
}


// ---------------------------------------------------------------- batched EM helpers
namespace {

// Instances with the same E-step block shape run in one launch per iteration.
struct BatchClass {
    int np = 0, g = 0, threads = 0, kmax = 0;
    std::vector<int> insts;
    int64_t points = 0;
    int64_t ppc = 0;
    int unit_begin = 0, nunits = 0;
};

// Points per CTA chosen by measurement, per (device, shape, log2 of the class's points).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int64_t> g_tuned;

int ilog2(int64_t v) {
    int r = 0;
    while ((int64_t(1) << (r + 1)) <= v) ++r;
    return r;
}

// Per-instance offsets and the unit list for the classes' current ppc values.
// Returns the units, the partial floats and the log-likelihood slots used.
void build_tables(std::vector<BatchInst>& hi, std::vector<BatchClass>& cls, std::vector<BatchUnit>& units,
                  int64_t* part_floats, int64_t* ll_slots) {
    int64_t part = 0, ll = 0;
    units.clear();
    for (auto& c : cls) {
        c.unit_begin = (int)units.size();
        for (int i : c.insts) {
            BatchInst& I = hi[i];
            I.ppc = c.ppc;
            I.ctas = (int)((I.n + c.ppc - 1) / c.ppc);
            I.part_off = part;
            I.ll_off = ll;
            part += (int64_t)I.ctas * I.k * NSTAT;
            ll += I.ctas;
            for (int t = 0; t < I.ctas; ++t) units.push_back(BatchUnit{i, t});
        }
        c.nunits = (int)units.size() - c.unit_begin;
    }
    *part_floats = part;
    *ll_slots = ll;
}

}  // namespace


// ---------------------------------------------------------------- large K (chunked E-step)
namespace {

// The chunk table of one fit over n points with k components, and its unit list.
struct ChunkPlan {
    int chunks = 0;
    int64_t ppc = 0;
    std::vector<BatchInst> hi;
    std::vector<BatchUnit> units;
    std::vector<int2> blocks;
    std::vector<int> comp_inst, npairs;
    int64_t part_floats = 0;
};

ChunkPlan plan_chunks(int64_t n, int k, int sms) {
    ChunkPlan P;
    const int KC = chunk_components();
    P.chunks = (k + KC - 1) / KC;
    const int Q = estep_batch_q();
    const int occ = estep_occupancy(KC, true, 1024);
    int64_t ppc = (n * P.chunks + 2LL * sms * occ - 1) / (2LL * sms * occ);
    P.ppc = std::min<int64_t>(estep_ppc_max(), std::max<int64_t>(4 * Q, (ppc + Q - 1) / Q * Q));
    const int ctas = (int)((n + P.ppc - 1) / P.ppc);
    const int cpb = fin_components_per_block();
    for (int c = 0; c < P.chunks; ++c) {
        BatchInst I{};
        I.pt_off = 0;
        I.n = n;
        I.ppc = P.ppc;
        I.k = std::min(KC, k - c * KC);
        I.comp_off = c * KC;
        I.par_off = c * chunk_param_floats();
        I.ctas = ctas;
        I.part_off = P.part_floats;
        I.ll_off = 0;
        P.part_floats += (int64_t)ctas * I.k * NSTAT;
        P.hi.push_back(I);
        P.npairs.push_back((int)(chunk_param_floats() / PAIR_FLOATS));
        for (int t = 0; t < ctas; ++t) P.units.push_back(BatchUnit{c, t});
        for (int j = 0; j * cpb < I.k; ++j) P.blocks.push_back(make_int2(c, j));
        for (int b = 0; b < I.k; ++b) P.comp_inst.push_back(c);
    }
    return P;
}

struct ChunkBufs {
    float *params = nullptr, *partials = nullptr, *psum = nullptr, *gref = nullptr;
    float2* pref = nullptr;
    double *llpt = nullptr, *llp = nullptr;
    int *flags = nullptr, *flag_count = nullptr, *comp_inst = nullptr, *npairs = nullptr;
    BatchInst* insts = nullptr;
    BatchUnit* units = nullptr;
    int2* blocks = nullptr;
};

void carve_chunks(Carver& cv, const ChunkPlan& P, int64_t n, bool stats, ChunkBufs* b) {
    b->params = cv.take<float>((size_t)P.chunks * chunk_param_floats());
    b->partials = cv.take<float>(stats ? (size_t)P.part_floats : 0);
    b->psum = cv.take<float>((size_t)P.chunks * n);
    b->gref = cv.take<float>(2);
    b->pref = cv.take<float2>(n);
    b->llpt = cv.take<double>(n);
    b->llp = cv.take<double>(chunk_combine_grid());
    b->flags = cv.take<int>(n);
    b->flag_count = cv.take<int>(1);
    b->comp_inst = cv.take<int>(P.comp_inst.size());
    b->npairs = cv.take<int>(P.chunks);
    b->insts = cv.take<BatchInst>(P.chunks);
    b->units = cv.take<BatchUnit>(P.units.size());
    b->blocks = cv.take<int2>(P.blocks.size());
}

cudaError_t upload_chunks(const ChunkPlan& P, const ChunkBufs& b, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(b.insts, P.hi.data(), sizeof(BatchInst) * P.chunks, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.units, P.units.data(), sizeof(BatchUnit) * P.units.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.blocks, P.blocks.data(), sizeof(int2) * P.blocks.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.comp_inst, P.comp_inst.data(), sizeof(int) * P.comp_inst.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.npairs, P.npairs.data(), sizeof(int) * P.chunks, cudaMemcpyHostToDevice, s);
    return e;
}

// The two-level log-sum-exp: reference, pass A (chunk sums), combine, exact
// points, per-point log-likelihood partials (and into st when ll_to_state).
cudaError_t chunk_lse(const ChunkPlan& P, const ChunkBufs& b, const float4* p8, int64_t n, int k, DeviceState* st,
                      int iter, bool ll_to_state, long long* launches, cudaStream_t s) {
    cudaError_t e = launch_chunk_ref(b.params, k, st, b.gref, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.flag_count, 0, sizeof(int), s);
    EStepLaunch a{p8, n, k, b.params, P.ppc, nullptr, nullptr, nullptr, nullptr, iter};
    a.insts = b.insts;
    a.units = b.units;
    a.states = st;
    a.gref = b.gref;
    a.psum = b.psum;
    if (e == cudaSuccess) e = launch_estep_chunks(a, 1, (int)P.units.size(), P.ppc, s);
    if (e == cudaSuccess) e = launch_chunk_combine(b.psum, P.chunks, n, b.gref, b.pref, b.llpt, b.flag_count, b.flags, st, s);
    if (e == cudaSuccess) e = launch_chunk_exact(p8, b.params, k, b.gref, b.flags, b.flag_count, b.pref, b.llpt, st, s);
    if (e == cudaSuccess) e = launch_points_ll_reduce(b.llpt, n, b.llp, ll_to_state ? st : nullptr, s);
    *launches += 5 + (ll_to_state ? 1 : 0);
    return e;
}

cudaError_t chunk_em_iteration(const ChunkPlan& P, const ChunkBufs& b, const float4* p8, int64_t n, int k,
                               float4* shift4, double* model64, double* trace, const gira_fit_opts& o,
                               DeviceState* st, int iter, long long* launches, cudaStream_t s, const int* perm) {
    cudaError_t e = chunk_lse(P, b, p8, n, k, st, iter, false, launches, s);
    EStepLaunch a{p8, n, k, b.params, P.ppc, b.partials, nullptr, nullptr, nullptr, iter};
    a.insts = b.insts;
    a.units = b.units;
    a.states = st;
    a.gref = b.gref;
    a.pref = b.pref;
    a.psum = b.psum;   // pass B skips the batches pass A found out of this chunk's reach
    if (e == cudaSuccess) e = launch_estep_chunks(a, 2, (int)P.units.size(), P.ppc, s);
    if (e == cudaSuccess)
        e = launch_reduce_finalize_chunks(b.partials, b.llp, chunk_combine_grid(), nullptr, shift4, b.insts,
                                          b.blocks, (int)P.blocks.size(), n, o.reg_covar, o.tol, model64, b.params,
                                          trace, st, iter, true, s, perm);
    *launches += 2;
    return e;
}

}  // namespace

extern "C" {

void gira_fit_opts_default(gira_fit_opts* o) {
    if (!o) return;
    o->iters = 100;
    o->tol = 1e-3;
    o->reg_covar = 1e-6;
    o->seed = 0;
    o->lloyd_iters = 10;
    o->init_mode = GIRA_INIT_KMEANS;
}

void gira_profile_enable(int on) { g_prof_on.store(on == 2 ? 2 : on ? 1 : 0); }

gira_status gira_profile_read(gira_profile* out, int reset) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (out) *out = g_prof;
    if (reset) g_prof = gira_profile{};
    return GIRA_OK;
}

const char* gira_last_error_message(void) { return t_msg.c_str(); }
int gira_last_error_component(void) { return t_bad; }
const char* gira_version(void) { return "gira-gb300 0.1.0 sm_103a"; }

gira_status gira_release_workspace(void) {
    t_msg.clear();
    std::lock_guard<std::mutex> lk(g_table_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_ws.size(); ++d) {
        if (!g_ws[d]) continue;
        std::lock_guard<std::mutex> l2(g_ws[d]->mu);
        drop_graph(g_ws[d]);
        if (g_ws[d]->ptr) {
            cudaSetDevice((int)d);
            cudaError_t e = cudaFree(g_ws[d]->ptr);
            g_ws[d]->ptr = nullptr;
            g_ws[d]->bytes = 0;
            if (e != cudaSuccess) {
                cudaSetDevice(cur);
                return fail(GIRA_ERR_CUDA, "cudaFree failed: %s", cudaGetErrorString(e));
            }
        }
    }
    cudaSetDevice(cur);
    return GIRA_OK;
}

// ================================================================ kmeans_init
gira_status gira_kmeans_init(const float* points, int64_t n, int k, uint64_t seed, int lloyd_iters, float* centers,
                             int32_t* labels, int* iters_done, void* stream) {
    CallRange nvtx_range("gira_kmeans_init");
    reset_error();
    TRY(check_nk(n, k));
    if (lloyd_iters < 0) return fail(GIRA_ERR_INVALID_ARG, "lloyd_iters < 0");
    if (!points || !centers) return fail(GIRA_ERR_INVALID_ARG, "points and centers must not be NULL");
    Ctx c;
    TRY(begin(c, stream));
    Kind kp, kc, kl = Kind::Host;
    TRY(check_ptr(points, "points", c.dev, &kp));
    TRY(check_ptr(centers, "centers", c.dev, &kc));
    if (labels) TRY(check_ptr(labels, "labels", c.dev, &kl));
    const int nblk = kpp_num_blocks(n);
    int kgrid = kpp_persistent_grid();
    if (kgrid > 0 && n > kpp_persistent_max_n(kgrid)) kgrid = 0;
    int* ksync = nullptr;
    u128* ksums = nullptr;

    auto layout = [&](Carver& cv, DeviceState** st, float** pin, float4** p4, float4** c4, float** d2, u128** bs,
                      int64_t** ch, int32_t** lab, double** sums, unsigned long long** chg, float** cout) {
        ksync = cv.take<int>((size_t)k + 1);
        ksums = cv.take<u128>(kpp_persistent_sum_words(std::max(kgrid, 1), k));
        *st = cv.take<DeviceState>(1);
        *pin = cv.take<float>(kp == Kind::Host ? 3 * n : 0);
        *p4 = cv.take<float4>(n);
        *c4 = cv.take<float4>(k);
        *d2 = cv.take<float>(2 * (size_t)n);   // double-buffered by the persistent seeding
        *bs = cv.take<u128>(nblk);
        *ch = cv.take<int64_t>(k);
        *lab = cv.take<int32_t>((labels && kl == Kind::Device) ? 0 : n);
        *sums = cv.take<double>(4 * (size_t)k);
        *chg = cv.take<unsigned long long>(lloyd_iters + 1);
        *cout = cv.take<float>(kc == Kind::Host ? 3 * (size_t)k : 0);
    };
    DeviceState* st;
    float *pin, *d2, *cout;
    float4 *p4, *c4;
    u128* bs;
    double* sums;
    int64_t* ch;
    int32_t* lab;
    unsigned long long* chg;
    Carver sizer;
    layout(sizer, &st, &pin, &p4, &c4, &d2, &bs, &ch, &lab, &sums, &chg, &cout);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv, &st, &pin, &p4, &c4, &d2, &bs, &ch, &lab, &sums, &chg, &cout);
    if (labels && kl == Kind::Device) lab = labels;

    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    DeviceState h{};
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    const float* pts = points;
    if (kp == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(pin, points, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, c.s));
        pts = pin;
    }
    COUNTED(prof, 1, launch_pack(pts, n, p4, nullptr, st, c.s));
    const int kcs = kpp_cluster_size(n);
    if (kcs > 0) {
        COUNTED(prof, 1, launch_kpp_cluster(p4, n, k, seed, c4, ch, kcs, st, c.s));
    } else if (kgrid > 0) {
        GIRA_CUDA(cudaMemsetAsync(ksync, 0, sizeof(int) * (k + 1), c.s));
        COUNTED(prof, 1, launch_kpp_persistent(p4, n, k, seed, c4, d2, ch, ksync, ksums, kgrid, st, c.s));
    } else {
        COUNTED(prof, 2 * k - 1, launch_kpp(p4, n, k, seed, c4, d2, bs, ch, st, c.s));
    }
    GIRA_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * 4 * k, c.s));
    GIRA_CUDA(cudaMemsetAsync(chg, 0, sizeof(unsigned long long) * (lloyd_iters + 1), c.s));
    COUNTED(prof, 1 + 2 * lloyd_iters, launch_lloyd(p4, n, k, lloyd_iters, c4, lab, sums, chg, st, c.s));
    prof.t_init = prof.mark();
    prof.t_em = prof.t_init;
    float* cdst = (kc == Kind::Device) ? centers : cout;
    COUNTED(prof, 1, launch_centers_out(c4, k, cdst, c.s));
    if (kc == Kind::Host)
        GIRA_CUDA(cudaMemcpyAsync(centers, cout, sizeof(float) * 3 * k, cudaMemcpyDeviceToHost, c.s));
    if (labels && kl == Kind::Host)
        GIRA_CUDA(cudaMemcpyAsync(labels, lab, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    prof.commit(0, 0);
    TRY(device_status(h));
    if (iters_done) *iters_done = h.lloyd_done;
    return GIRA_OK;
}

// ================================================================ gmm_fit
gira_status gira_gmm_fit(const float* points, int64_t n, int k, const gira_fit_opts* opts, float* weights,
                         float* means, float* covs, double* loglik_trace, int* iters_done, double* final_loglik,
                         void* stream) {
    CallRange nvtx_range("gira_gmm_fit");
    reset_error();
    if (!opts) return fail(GIRA_ERR_INVALID_ARG, "opts is NULL");
    TRY(check_nk(n, k));
    const gira_fit_opts o = *opts;
    TRY(check_opts(o));
    if (!points || !weights || !means || !covs) return fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    Ctx c;
    TRY(begin(c, stream));
    Kind kp, kw, km, kc;
    TRY(check_ptr(points, "points", c.dev, &kp));
    TRY(check_ptr(weights, "weights", c.dev, &kw));
    TRY(check_ptr(means, "means", c.dev, &km));
    TRY(check_ptr(covs, "covs", c.dev, &kc));
    const bool model_host = kw == Kind::Host || km == Kind::Host || kc == Kind::Host;
    const bool kinit = o.init_mode == GIRA_INIT_KMEANS;
    const bool chunked = k > MAX_K_DIRECT;   // two-level log-sum-exp over chunks of components
    const ChunkPlan P = chunked ? plan_chunks(n, k, c.sms) : ChunkPlan{};
    ChunkBufs cb;
    const int npairs = chunked ? 0 : params_pairs_padded(k);
    // point-stationary E-step: one grid for the EM loop and the final log-likelihood;
    // per-warp partial rows and live masks
    const int grid = chunked ? 0 : estep_pt_grid(n);
    const int rows = chunked ? 0 : estep_pt_rows(grid);
    const int nwords = chunked ? 0 : estep_pt_mask_words(k);
    const int nblk = kpp_num_blocks(n);
    int kgrid = kinit ? kpp_persistent_grid() : 0;
    if (kgrid > 0 && n > kpp_persistent_max_n(kgrid)) kgrid = 0;

    struct Bufs {
        DeviceState* st;
        float *pin, *params, *partials, *d2, *mw, *mmu, *mcov;
        float4 *p4, *p8, *shift4, *c4;
        double *model64, *stats64, *llp, *trace, *sums;
        u128 *bs, *ksums;
        int64_t* ch;
        int32_t* lab;
        int *ksync, *perm;
        uint32_t* masks;
        unsigned long long* chg;
        float4 *p8s, *p4s;
        void* osc;
        uint8_t* cta_key;
        int* cta_perm;
    } b{};
    // the E-steps and Lloyd run on the points in a spatial order (a warp's points then
    // reach fewer components and centres); k-means++ on the caller's order, which
    // defines its draws
    const bool sorted = !chunked && n <= point_order_max_n();
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.perm = cv.take<int>(k);
        b.pin = cv.take<float>(kp == Kind::Host ? 3 * n : 0);
        b.p4 = cv.take<float4>(kinit ? n : 0);
        b.p8 = cv.take<float4>(2 * (size_t)n);
        b.p8s = cv.take<float4>(sorted ? 2 * (size_t)n : 0);
        b.p4s = cv.take<float4>(sorted && kinit ? (size_t)n : 0);
        b.osc = cv.take<char>(sorted ? point_order_scratch_bytes(n, 1) : 0);
        b.params = cv.take<float>((size_t)npairs * PAIR_FLOATS);
        b.shift4 = cv.take<float4>(k);
        b.model64 = cv.take<double>((size_t)k * MODEL);
        b.stats64 = cv.take<double>((size_t)k * NSTAT);
        b.partials = cv.take<float>((size_t)rows * estep_pt_row_floats(k));
        b.masks = cv.take<uint32_t>((size_t)rows * nwords);
        b.llp = cv.take<double>(grid);
        b.trace = cv.take<double>(std::max(o.iters, 1));
        b.cta_key = cv.take<uint8_t>(chunked ? 0 : grid);
        b.cta_perm = cv.take<int>(chunked ? 0 : 2 * (size_t)grid);
        if (chunked) carve_chunks(cv, P, n, true, &cb);
        b.mw = cv.take<float>(model_host ? k : 0);
        b.mmu = cv.take<float>(model_host ? 3 * (size_t)k : 0);
        b.mcov = cv.take<float>(model_host ? 9 * (size_t)k : 0);
        if (kinit) {
            b.c4 = cv.take<float4>(k);
            b.d2 = cv.take<float>(2 * (size_t)n);   // double-buffered by the persistent seeding
            b.bs = cv.take<u128>(nblk);
            b.ch = cv.take<int64_t>(k);
            b.lab = cv.take<int32_t>(n);
            b.sums = cv.take<double>(4 * (size_t)k);
            b.chg = cv.take<unsigned long long>(o.lloyd_iters + 1);
            b.ksync = cv.take<int>((size_t)k + 1);
            b.ksums = cv.take<u128>(kpp_persistent_sum_words(std::max(kgrid, 1), k));
        }
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);

    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    DeviceState h{};
    h.stop_after = o.iters;
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemsetAsync(b.trace, 0xff, sizeof(double) * std::max(o.iters, 1), c.s));   // NaN
    const float* pts = points;
    if (kp == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.pin, points, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, c.s));
        pts = b.pin;
    }
    COUNTED(prof, 1, launch_pack(pts, n, kinit ? b.p4 : nullptr, b.p8, b.st, c.s));
    if (sorted)
        COUNTED(prof, point_order_launches(1),
                launch_point_order(b.p8, n, nullptr, nullptr, 0, 1, b.osc, b.p8s, kinit ? b.p4s : nullptr, nullptr, c.s));
    if (chunked) {
        GIRA_CUDA(upload_chunks(P, cb, c.s));
        b.params = cb.params;
        COUNTED(prof, 1, launch_fill_padding_batched(cb.params, cb.insts, P.chunks, 0, cb.npairs, c.s));
    } else {
        COUNTED(prof, 1, launch_fill_padding(b.params, k, npairs, c.s));
    }

    float* w_d = (kw == Kind::Device) ? weights : b.mw;
    float* mu_d = (km == Kind::Device) ? means : b.mmu;
    float* cov_d = (kc == Kind::Device) ? covs : b.mcov;
    if (kinit) {
        const int kcs = kpp_cluster_size(n);
        if (kcs > 0) {
            COUNTED(prof, 1, launch_kpp_cluster(b.p4, n, k, o.seed, b.c4, b.ch, kcs, b.st, c.s));
        } else if (kgrid > 0) {
            GIRA_CUDA(cudaMemsetAsync(b.ksync, 0, sizeof(int) * (k + 1), c.s));
            COUNTED(prof, 1, launch_kpp_persistent(b.p4, n, k, o.seed, b.c4, b.d2, b.ch, b.ksync, b.ksums, kgrid, b.st,
                                                   c.s));
        } else {
            COUNTED(prof, 2 * k - 1, launch_kpp(b.p4, n, k, o.seed, b.c4, b.d2, b.bs, b.ch, b.st, c.s));
        }
        GIRA_CUDA(cudaMemsetAsync(b.sums, 0, sizeof(double) * 4 * k, c.s));
        GIRA_CUDA(cudaMemsetAsync(b.chg, 0, sizeof(unsigned long long) * (o.lloyd_iters + 1), c.s));
        COUNTED(prof, 1 + 2 * o.lloyd_iters,
                launch_lloyd(sorted ? b.p4s : b.p4, n, k, o.lloyd_iters, b.c4, b.lab, b.sums, b.chg, b.st, c.s));
        GIRA_CUDA(cudaMemsetAsync(b.stats64, 0, sizeof(double) * NSTAT * k, c.s));
        COUNTED(prof, 1, launch_label_stats(sorted ? b.p4s : b.p4, n, k, b.lab, b.c4, b.stats64, b.st, c.s));
        GIRA_CUDA(cudaMemcpyAsync(b.shift4, b.c4, sizeof(float4) * k, cudaMemcpyDeviceToDevice, c.s));
        if (chunked) {
            COUNTED(prof, 1, launch_reduce_finalize_chunks(nullptr, nullptr, 0, b.stats64, b.shift4, cb.insts,
                                                           cb.blocks, (int)P.blocks.size(), n, o.reg_covar, o.tol,
                                                           b.model64, cb.params, b.trace, b.st, 0, false, c.s));
        } else {
            COUNTED(prof, 1, launch_reduce_finalize(nullptr, 0, nullptr, b.stats64, b.shift4, k, n, o.reg_covar,
                                                    o.tol, b.model64, b.params, b.trace, b.st, 0, false, c.s));
        }
    } else {
        if (kw == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(b.mw, weights, sizeof(float) * k, cudaMemcpyHostToDevice, c.s));
        if (km == Kind::Host)
            GIRA_CUDA(cudaMemcpyAsync(b.mmu, means, sizeof(float) * 3 * k, cudaMemcpyHostToDevice, c.s));
        if (kc == Kind::Host)
            GIRA_CUDA(cudaMemcpyAsync(b.mcov, covs, sizeof(float) * 9 * k, cudaMemcpyHostToDevice, c.s));
        if (chunked) {
            COUNTED(prof, 1, launch_params_from_model_batched(w_d, mu_d, cov_d, k, cb.comp_inst, cb.insts, b.model64,
                                                              cb.params, b.shift4, b.st, c.s));
        } else {
            COUNTED(prof, 1, launch_params_from_model(w_d, mu_d, cov_d, k, b.model64, b.params, b.shift4, b.st, c.s));
        }
    }
    // the EM runs with the components along a space-filling curve of their means
    // (the E-step then skips the many point-component pairs out of reach);
    // model_out puts them back in the caller's order
    const int* perm = b.perm;
    COUNTED(prof, 2, launch_order_components(b.model64, b.stats64, k, b.perm, b.params, b.shift4, b.st, c.s));
    prof.t_init = prof.mark();

    if (chunked) {
        for (int t = 1; t <= o.iters; ++t)
            GIRA_CUDA(chunk_em_iteration(P, cb, b.p8, n, k, b.shift4, b.model64, b.trace, o, b.st, t, &prof.launches,
                                         c.s, perm));
        prof.t_em = prof.mark();
        if (final_loglik) GIRA_CUDA(chunk_lse(P, cb, b.p8, n, k, b.st, 0, true, &prof.launches, c.s));
    }
    EStepLaunch a{sorted ? b.p8s : b.p8, n, k, b.params, 0, b.partials, b.llp, nullptr, b.st, 0};
    a.n_buf = n;
    a.masks = b.masks;
    a.pt_rows = rows;
    a.cta_perm = b.cta_perm;   // from the third iteration on: the CTAs of most work first
    a.cta_key = b.cta_key;
    for (int t = 1; t <= o.iters && !chunked; ++t) {
        a.iter = t;
        // dependent launches unless an event pair brackets each E-step: each
        // kernel is resident before the previous one ends and waits on the
        // device for its results
        const bool pdl = !prof.per_launch;
        cudaEvent_t e0 = prof.mark_launch();
        COUNTED(prof, 1, launch_estep_pt(a, true, grid, c.s, pdl));
        cudaEvent_t e1 = prof.mark_launch();
        if (prof.per_launch) prof.timed(e0, e1);
        COUNTED(prof, 1, launch_reduce_finalize(b.partials, rows, b.llp, nullptr, b.shift4, k, n, o.reg_covar,
                                                o.tol, b.model64, b.params, b.trace, b.st, t, true, c.s, pdl, perm,
                                                b.masks, nwords, grid, b.cta_key, b.cta_perm, grid));
    }
    if (!chunked) prof.t_em = prof.mark();
    if (final_loglik && !chunked) {
        EStepLaunch f = a;
        f.iter = 0;
        f.partials = nullptr;
        f.masks = nullptr;
        COUNTED(prof, 1, launch_estep_pt(f, false, grid, c.s));
        COUNTED(prof, 1, launch_ll_reduce(b.llp, grid, b.st, c.s));
    }
    COUNTED(prof, 1, launch_model_out(b.model64, k, w_d, mu_d, cov_d, b.st, c.s, perm));
    if (kw == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(weights, b.mw, sizeof(float) * k, cudaMemcpyDeviceToHost, c.s));
    if (km == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(means, b.mmu, sizeof(float) * 3 * k, cudaMemcpyDeviceToHost, c.s));
    if (kc == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(covs, b.mcov, sizeof(float) * 9 * k, cudaMemcpyDeviceToHost, c.s));
    if (loglik_trace && o.iters > 0)
        GIRA_CUDA(cudaMemcpyAsync(loglik_trace, b.trace, sizeof(double) * o.iters, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    if (!chunked) {
        prof.pair_slots = (long long)h.iters_done * rows * ((((k + 1) >> 1) + 1) & ~1);
        prof.pairs_near = (long long)h.pairs_near;
        prof.pairs_live = (long long)h.pairs_live;
    }
    prof.commit(h.iters_done, h.iters_done);
    TRY(device_status(h));
    if (iters_done) *iters_done = h.iters_done;
    if (final_loglik) *final_loglik = h.ll_sum / (double)n;
    return GIRA_OK;
}

// ================================================================ gmm_loglik
gira_status gira_gmm_loglik(const float* points, int64_t n, int k, const float* weights, const float* means,
                            const float* covs, double* mean_loglik, float* per_point, void* stream) {
    CallRange nvtx_range("gira_gmm_loglik");
    reset_error();
    TRY(check_nk(n, k));
    if (!points || !weights || !means || !covs) return fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    Ctx c;
    TRY(begin(c, stream));
    Kind kp, kw, km, kc, kpp = Kind::Host;
    TRY(check_ptr(points, "points", c.dev, &kp));
    TRY(check_ptr(weights, "weights", c.dev, &kw));
    TRY(check_ptr(means, "means", c.dev, &km));
    TRY(check_ptr(covs, "covs", c.dev, &kc));
    if (per_point) TRY(check_ptr(per_point, "per_point", c.dev, &kpp));
    const bool chunked = k > MAX_K_DIRECT;   // two-level log-sum-exp over chunks of components
    const ChunkPlan P = chunked ? plan_chunks(n, k, c.sms) : ChunkPlan{};
    ChunkBufs cb;
    const int npairs = chunked ? 0 : params_pairs_padded(k);
    const int grid = chunked ? 0 : estep_pt_grid(n);
    struct Bufs {
        DeviceState* st;
        float *pin, *params, *mw, *mmu, *mcov, *pp;
        float4 *p8, *shift4;
        double *model64, *llp;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.pin = cv.take<float>(kp == Kind::Host ? 3 * n : 0);
        b.p8 = cv.take<float4>(2 * (size_t)n);
        b.params = cv.take<float>((size_t)npairs * PAIR_FLOATS);
        b.shift4 = cv.take<float4>(k);
        b.model64 = cv.take<double>((size_t)k * MODEL);
        b.llp = cv.take<double>(grid);
        b.mw = cv.take<float>(kw == Kind::Host ? k : 0);
        b.mmu = cv.take<float>(km == Kind::Host ? 3 * (size_t)k : 0);
        b.mcov = cv.take<float>(kc == Kind::Host ? 9 * (size_t)k : 0);
        b.pp = cv.take<float>((per_point && kpp == Kind::Host) ? n : 0);
        if (chunked) carve_chunks(cv, P, n, false, &cb);
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);

    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    DeviceState h{};
    h.stop_after = 0;
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    const float* pts = points;
    if (kp == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.pin, points, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, c.s));
        pts = b.pin;
    }
    const float* w_d = weights;
    const float* mu_d = means;
    const float* cov_d = covs;
    if (kw == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.mw, weights, sizeof(float) * k, cudaMemcpyHostToDevice, c.s));
        w_d = b.mw;
    }
    if (km == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.mmu, means, sizeof(float) * 3 * k, cudaMemcpyHostToDevice, c.s));
        mu_d = b.mmu;
    }
    if (kc == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.mcov, covs, sizeof(float) * 9 * k, cudaMemcpyHostToDevice, c.s));
        cov_d = b.mcov;
    }
    COUNTED(prof, 1, launch_pack(pts, n, nullptr, b.p8, b.st, c.s));
    float* ppd = per_point ? ((kpp == Kind::Device) ? per_point : b.pp) : nullptr;
    if (chunked) {
        GIRA_CUDA(upload_chunks(P, cb, c.s));
        COUNTED(prof, 1, launch_fill_padding_batched(cb.params, cb.insts, P.chunks, 0, cb.npairs, c.s));
        COUNTED(prof, 1, launch_params_from_model_batched(w_d, mu_d, cov_d, k, cb.comp_inst, cb.insts, b.model64,
                                                          cb.params, b.shift4, b.st, c.s));
        prof.t_init = prof.mark();
        prof.t_em = prof.t_init;
        GIRA_CUDA(chunk_lse(P, cb, b.p8, n, k, b.st, 0, true, &prof.launches, c.s));
        if (ppd) COUNTED(prof, 1, launch_double_to_float(cb.llpt, n, ppd, c.s));
    } else {
        COUNTED(prof, 1, launch_fill_padding(b.params, k, npairs, c.s));
        COUNTED(prof, 1, launch_params_from_model(w_d, mu_d, cov_d, k, b.model64, b.params, b.shift4, b.st, c.s));
        prof.t_init = prof.mark();
        prof.t_em = prof.t_init;
        EStepLaunch a{b.p8, n, k, b.params, 0, nullptr, b.llp, ppd, b.st, 0};
        a.n_buf = n;
        COUNTED(prof, 1, launch_estep_pt(a, false, grid, c.s));
        COUNTED(prof, 1, launch_ll_reduce(b.llp, grid, b.st, c.s));
    }
    if (per_point && kpp == Kind::Host)
        GIRA_CUDA(cudaMemcpyAsync(per_point, b.pp, sizeof(float) * n, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    prof.commit(0, 0);
    TRY(device_status(h));
    if (mean_loglik) *mean_loglik = h.ll_sum / (double)n;
    return GIRA_OK;
}

// ================================================================ gmm_loglik_grad
gira_status gira_gmm_loglik_grad(const float* points, int64_t n, int k, const float* pose12, const float* logits,
                                 const float* means, const float* chol, double* loglik, float* grad_points,
                                 double* grad_pose, double* grad_twist, float* grad_logits, float* grad_means,
                                 float* grad_chol, void* stream) {
    CallRange nvtx_range("gira_gmm_loglik_grad");
    reset_error();
    TRY(check_nk(n, k));
    if (k > GIRA_MAX_K_BATCHED) return fail(GIRA_ERR_INVALID_ARG, "k = %d > %d for the gradient", k, GIRA_MAX_K_BATCHED);
    if (!points || !logits || !means || !chol) return fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    Ctx c;
    TRY(begin(c, stream));
    Kind kp, kl, km, kc, kpose = Kind::Device, kgp = Kind::Device, kgo = Kind::Device, kgt = Kind::Device,
                         kgl = Kind::Device, kgm = Kind::Device, kgc = Kind::Device;
    TRY(check_ptr(points, "points", c.dev, &kp));
    TRY(check_ptr(logits, "logits", c.dev, &kl));
    TRY(check_ptr(means, "means", c.dev, &km));
    TRY(check_ptr(chol, "chol", c.dev, &kc));
    if (pose12) TRY(check_ptr(pose12, "pose12", c.dev, &kpose));
    if (grad_points) TRY(check_ptr(grad_points, "grad_points", c.dev, &kgp));
    if (grad_pose) TRY(check_ptr(grad_pose, "grad_pose", c.dev, &kgo));
    if (grad_twist) TRY(check_ptr(grad_twist, "grad_twist", c.dev, &kgt));
    if (grad_logits) TRY(check_ptr(grad_logits, "grad_logits", c.dev, &kgl));
    if (grad_means) TRY(check_ptr(grad_means, "grad_means", c.dev, &kgm));
    if (grad_chol) TRY(check_ptr(grad_chol, "grad_chol", c.dev, &kgc));
    const bool grad = grad_points || grad_pose || grad_twist || grad_logits || grad_means || grad_chol;
    const int npairs = params_pairs_padded(k);
    int64_t ppc = 0;
    const int grid = estep_grid(n, k, grad, c.sms, &ppc, true);
    auto host = [&](Kind kd, const void* ptr) { return ptr && kd == Kind::Host; };
    struct Bufs {
        DeviceState* st;
        float *pin, *pose, *lg, *mu, *ch, *params, *partials, *gp, *gl, *gm, *gc;
        float4 *p8, *shift4;
        double *model64, *llp, *ppart, *po64, *tw64;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.pin = cv.take<float>(host(kp, points) ? 3 * (size_t)n : 0);
        b.pose = cv.take<float>(host(kpose, pose12) ? 12 : 0);
        b.lg = cv.take<float>(host(kl, logits) ? k : 0);
        b.mu = cv.take<float>(host(km, means) ? 3 * (size_t)k : 0);
        b.ch = cv.take<float>(host(kc, chol) ? 9 * (size_t)k : 0);
        b.p8 = cv.take<float4>(2 * (size_t)n);
        b.params = cv.take<float>((size_t)npairs * PAIR_FLOATS);
        b.shift4 = cv.take<float4>(k);
        b.model64 = cv.take<double>((size_t)k * MODEL);
        b.llp = cv.take<double>(grid);
        b.partials = cv.take<float>(grad ? (size_t)grid * k * NSTAT : 0);
        b.ppart = cv.take<double>(grad ? (size_t)grid * 12 : 0);
        b.po64 = cv.take<double>(12);
        b.tw64 = cv.take<double>(6);
        b.gp = cv.take<float>(host(kgp, grad_points) ? 3 * (size_t)n : 0);
        b.gl = cv.take<float>(host(kgl, grad_logits) ? k : 0);
        b.gm = cv.take<float>(host(kgm, grad_means) ? 3 * (size_t)k : 0);
        b.gc = cv.take<float>(host(kgc, grad_chol) ? 9 * (size_t)k : 0);
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);

    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    DeviceState h{};
    h.stop_after = 0;
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    // inputs: device pointers as given, host arrays staged
    auto in = [&](const float* src, Kind kd, float* stage, size_t count) -> const float* {
        if (!src || kd != Kind::Host) return src;
        if (cudaMemcpyAsync(stage, src, sizeof(float) * count, cudaMemcpyHostToDevice, c.s) != cudaSuccess)
            return nullptr;
        return stage;
    };
    const float* pts_d = in(points, kp, b.pin, 3 * (size_t)n);
    const float* pose_d = in(pose12, kpose, b.pose, 12);
    const float* lg_d = in(logits, kl, b.lg, k);
    const float* mu_d = in(means, km, b.mu, 3 * (size_t)k);
    const float* ch_d = in(chol, kc, b.ch, 9 * (size_t)k);
    if (!pts_d || (pose12 && !pose_d) || !lg_d || !mu_d || !ch_d) {
        cudaGetLastError();
        return fail(GIRA_ERR_CUDA, "host-to-device copy of an input failed");
    }
    float* gp_d = grad_points ? (kgp == Kind::Host ? b.gp : grad_points) : nullptr;
    float* gl_d = grad_logits ? (kgl == Kind::Host ? b.gl : grad_logits) : nullptr;
    float* gm_d = grad_means ? (kgm == Kind::Host ? b.gm : grad_means) : nullptr;
    float* gc_d = grad_chol ? (kgc == Kind::Host ? b.gc : grad_chol) : nullptr;
    double* po_d = grad_pose ? (kgo == Kind::Host ? b.po64 : grad_pose) : nullptr;
    double* tw_d = grad_twist ? (kgt == Kind::Host ? b.tw64 : grad_twist) : nullptr;

    COUNTED(prof, 1, launch_pack_pose(pts_d, n, pose_d, b.p8, b.st, c.s));
    COUNTED(prof, 1, launch_fill_padding(b.params, k, npairs, c.s));
    COUNTED(prof, 1, launch_params_from_chol(lg_d, mu_d, ch_d, k, b.model64, b.params, b.shift4, b.st, c.s));
    prof.t_init = prof.mark();
    prof.t_em = prof.t_init;
    EStepLaunch a{b.p8, n, k, b.params, ppc, grad ? b.partials : nullptr, b.llp, nullptr, b.st, 0};
    if (grad) {
        a.grad_pts = gp_d;
        a.rot = pose_d;
        a.pose_partials = b.ppart;
        cudaEvent_t e0 = prof.mark_launch();
        COUNTED(prof, 1, launch_estep(a, true, grid, c.s, true));
        cudaEvent_t e1 = prof.mark_launch();
        if (prof.per_launch) prof.timed(e0, e1);
        COUNTED(prof, 1, launch_grad_finalize(b.partials, grid, b.llp, b.ppart, pose_d, ch_d, b.model64, k, n, gl_d,
                                              gm_d, gc_d, po_d, tw_d, b.st, c.s));
    } else {
        COUNTED(prof, 1, launch_estep(a, false, grid, c.s, true));
        COUNTED(prof, 1, launch_ll_reduce(b.llp, grid, b.st, c.s));
    }
    auto out = [&](void* dst, Kind kd, const void* stage, size_t bytes) -> gira_status {
        if (dst && kd == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyDeviceToHost, c.s));
        return GIRA_OK;
    };
    TRY(out(grad_points, kgp, b.gp, sizeof(float) * 3 * (size_t)n));
    TRY(out(grad_logits, kgl, b.gl, sizeof(float) * k));
    TRY(out(grad_means, kgm, b.gm, sizeof(float) * 3 * (size_t)k));
    TRY(out(grad_chol, kgc, b.gc, sizeof(float) * 9 * (size_t)k));
    TRY(out(grad_pose, kgo, b.po64, sizeof(double) * 12));
    TRY(out(grad_twist, kgt, b.tw64, sizeof(double) * 6));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    prof.commit(0, grad ? 1 : 0);
    TRY(device_status(h));
    if (loglik) *loglik = h.ll_sum;
    return GIRA_OK;
}

// ================================================================ gmm_fit_batched
gira_status gira_gmm_fit_batched(const float* points, const int64_t* offsets, int batch, const int* ks,
                                 const gira_fit_opts* opts, float* weights, float* means, float* covs,
                                 double* loglik_traces, int* iters_done, double* final_loglik, int* statuses,
                                 void* stream) {
    CallRange nvtx_range("gira_gmm_fit_batched");
    reset_error();
    if (!opts || !offsets || !ks) return fail(GIRA_ERR_INVALID_ARG, "opts, offsets and ks must not be NULL");
    if (batch < 1) return fail(GIRA_ERR_INVALID_ARG, "batch = %d < 1", batch);
    const gira_fit_opts o = *opts;
    TRY(check_opts(o));
    if (offsets[0] != 0) return fail(GIRA_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int i = 0; i < batch; ++i) {
        const int64_t n = offsets[i + 1] - offsets[i];
        if (n < 1) return fail(GIRA_ERR_INVALID_ARG, "instance %d has %lld points", i, (long long)n);
        if (ks[i] < 1 || ks[i] > GIRA_MAX_K_BATCHED || ks[i] > n)
            return fail(GIRA_ERR_INVALID_ARG, "instance %d: k = %d outside [1, min(n, %d)]", i, ks[i], GIRA_MAX_K_BATCHED);
    }
    if (!points || !weights || !means || !covs) return fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    const int64_t total_n = offsets[batch];
    Ctx c;
    TRY(begin(c, stream));
    Kind kp, kw, km, kc;
    TRY(check_ptr(points, "points", c.dev, &kp));
    TRY(check_ptr(weights, "weights", c.dev, &kw));
    TRY(check_ptr(means, "means", c.dev, &km));
    TRY(check_ptr(covs, "covs", c.dev, &kc));
    const bool model_host = kw == Kind::Host || km == Kind::Host || kc == Kind::Host;
    const bool kinit = o.init_mode == GIRA_INIT_KMEANS;
    const int iters = std::max(o.iters, 1);

    // ---- host tables: instances, finalize blocks
    std::vector<BatchInst> hi(batch);
    std::vector<int> npairs_of(batch);
    int total_k = 0;
    int64_t par_floats = 0;
    for (int i = 0; i < batch; ++i) {
        BatchInst& I = hi[i];
        I.pt_off = offsets[i];
        I.n = offsets[i + 1] - offsets[i];
        I.k = ks[i];
        I.comp_off = total_k;
        total_k += ks[i];
        npairs_of[i] = params_pairs_padded(ks[i]);
        I.par_off = par_floats;
        par_floats += (int64_t)npairs_of[i] * PAIR_FLOATS;
    }
    std::vector<int> comp_inst(total_k);
    std::vector<int2> fin_blocks;
    const int cpb = fin_components_per_block();
    for (int i = 0; i < batch; ++i) {
        for (int b = 0; b < ks[i]; ++b) comp_inst[hi[i].comp_off + b] = i;
        for (int j = 0; j * cpb < ks[i]; ++j) fin_blocks.push_back(make_int2(i, j));
    }
    // the point-stationary E-step: every instance in one launch, a fixed number of
    // points per CTA; per-warp partial rows and live masks per instance
    std::vector<BatchUnit> units;
    int64_t part_floats = 0, mask_words = 0, ll_slots = 0;
    int kmax_all = 0;
    {
        const int PTS = estep_pt_points(), W = estep_pt_blocks();
        for (int i = 0; i < batch; ++i) {
            BatchInst& I = hi[i];
            I.ppc = PTS;
            I.ctas = (int)((I.n + PTS - 1) / PTS);
            I.part_off = part_floats;
            I.mask_off = mask_words;
            I.ll_off = ll_slots;
            part_floats += (int64_t)I.ctas * W * estep_pt_row_floats(I.k);
            mask_words += (int64_t)I.ctas * W * estep_pt_mask_words(I.k);
            ll_slots += I.ctas;
            kmax_all = std::max(kmax_all, I.k);
            for (int t = 0; t < I.ctas; ++t) units.push_back(BatchUnit{i, t});
        }
    }
    const size_t max_units = units.size();

    // per-instance KInit scratch
    std::vector<int64_t> nblk_off(batch + 1, 0);
    for (int i = 0; i < batch; ++i) nblk_off[i + 1] = nblk_off[i] + (kinit ? kpp_num_blocks(hi[i].n) : 0);

    struct Bufs {
        DeviceState* st;
        float *pin, *params, *partials, *mw, *mmu, *mcov, *d2;
        float4 *p4, *p8, *shift4, *c4;
        double *model64, *stats64, *llp, *trace, *sums;
        BatchInst* insts;
        BatchUnit* units;
        int2* blocks;
        int *comp_inst, *npairs, *perm;
        uint32_t* masks;
        int64_t *offs, *ch;
        int32_t* lab;
        u128* bs;
        unsigned long long* chg;
        KppInst *ktab, *kseed;
        BatchUnit* lunits;
        float4 *p8s, *p4s;
        int2* ounits;
        void* osc;
    } b{};
    // the E-steps run on every instance's points in a spatial order
    const bool sorted = total_n <= point_order_max_n();
    const int64_t nounits = sorted ? point_order_box_units(offsets, batch) : 0;
    std::vector<int2> ounits((size_t)nounits);
    if (sorted) point_order_fill_units(offsets, batch, ounits.data());
    // KInit tables: every instance; the seeding clusters grouped by cluster size
    // (instances beyond one 16-CTA cluster are seeded alone); Lloyd tiles
    std::vector<KppInst> ktab(batch);
    std::vector<BatchUnit> lloyd_units;
    std::vector<KppInst> kseed;
    std::vector<std::pair<int, int>> seed_class;   // (cluster size, count), in kseed order
    std::vector<int> seed_alone;
    if (kinit) {
        const int cs_max = kpp_cluster_size(1);   // the largest cluster this GPU runs (0: none)
        std::map<int, std::vector<int>> by_cs;
        for (int i = 0; i < batch; ++i) {
            ktab[i] = KppInst{hi[i].pt_off, hi[i].n, hi[i].k, hi[i].comp_off, i, 0};
            for (int t = 0; (int64_t)t * lloyd_tile() < hi[i].n; ++t) lloyd_units.push_back(BatchUnit{i, t});
            int cs = 0;
            for (int c2 = 1; c2 <= cs_max; c2 *= 2)
                if (hi[i].n <= kpp_cluster_capacity(c2)) {
                    cs = c2;
                    break;
                }
            if (cs) by_cs[cs].push_back(i); else seed_alone.push_back(i);
        }
        for (auto& kv : by_cs) {
            seed_class.emplace_back(kv.first, (int)kv.second.size());
            for (int i : kv.second) kseed.push_back(ktab[i]);
        }
    }
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(batch);
        b.pin = cv.take<float>(kp == Kind::Host ? 3 * (size_t)total_n : 0);
        b.p4 = cv.take<float4>(kinit ? (size_t)total_n : 0);
        b.p8 = cv.take<float4>(2 * (size_t)total_n);
        b.p8s = cv.take<float4>(sorted ? 2 * (size_t)total_n : 0);
        b.p4s = cv.take<float4>(sorted && kinit ? (size_t)total_n : 0);
        b.ounits = cv.take<int2>((size_t)nounits);
        b.osc = cv.take<char>(sorted ? point_order_scratch_bytes(total_n, batch) : 0);
        b.params = cv.take<float>((size_t)par_floats);
        b.shift4 = cv.take<float4>(total_k);
        b.model64 = cv.take<double>((size_t)total_k * MODEL);
        b.stats64 = cv.take<double>((size_t)total_k * NSTAT);
        b.partials = cv.take<float>((size_t)part_floats);
        b.masks = cv.take<uint32_t>((size_t)mask_words);
        b.llp = cv.take<double>((size_t)ll_slots);
        b.trace = cv.take<double>((size_t)batch * iters);
        b.mw = cv.take<float>(model_host ? total_k : 0);
        b.mmu = cv.take<float>(model_host ? 3 * (size_t)total_k : 0);
        b.mcov = cv.take<float>(model_host ? 9 * (size_t)total_k : 0);
        b.insts = cv.take<BatchInst>(batch);
        b.units = cv.take<BatchUnit>(max_units);
        b.blocks = cv.take<int2>(fin_blocks.size());
        b.comp_inst = cv.take<int>(total_k);
        b.perm = cv.take<int>(total_k);
        b.npairs = cv.take<int>(batch);
        b.offs = cv.take<int64_t>(batch + 1);
        if (kinit) {
            b.c4 = cv.take<float4>(total_k);
            b.ch = cv.take<int64_t>(total_k);
            b.lab = cv.take<int32_t>(total_n);
            b.sums = cv.take<double>(4 * (size_t)total_k);
            b.chg = cv.take<unsigned long long>((size_t)batch * (o.lloyd_iters + 1));
            b.bs = cv.take<u128>((size_t)nblk_off[batch]);
            b.d2 = cv.take<float>((size_t)total_n);
            b.ktab = cv.take<KppInst>(batch);
            b.kseed = cv.take<KppInst>(batch);
            b.lunits = cv.take<BatchUnit>(lloyd_units.size());
        }
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);

    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    std::vector<DeviceState> hs(batch);
    for (auto& h : hs) {
        h = DeviceState{};
        h.stop_after = o.iters;
        h.bad_component = INT_MAX;
    }
    GIRA_CUDA(cudaMemcpyAsync(b.st, hs.data(), sizeof(DeviceState) * batch, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemsetAsync(b.trace, 0xff, sizeof(double) * batch * iters, c.s));   // NaN
    GIRA_CUDA(cudaMemcpyAsync(b.offs, offsets, sizeof(int64_t) * (batch + 1), cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.blocks, fin_blocks.data(), sizeof(int2) * fin_blocks.size(), cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.comp_inst, comp_inst.data(), sizeof(int) * total_k, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.npairs, npairs_of.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.insts, hi.data(), sizeof(BatchInst) * batch, cudaMemcpyHostToDevice, c.s));
    const float* pts = points;
    if (kp == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.pin, points, sizeof(float) * 3 * total_n, cudaMemcpyHostToDevice, c.s));
        pts = b.pin;
    }
    COUNTED(prof, 1, launch_pack_batched(pts, total_n, b.offs, batch, kinit ? b.p4 : nullptr, b.p8, b.st, c.s));
    if (sorted) {
        GIRA_CUDA(cudaMemcpyAsync(b.ounits, ounits.data(), sizeof(int2) * ounits.size(), cudaMemcpyHostToDevice, c.s));
        COUNTED(prof, point_order_launches(batch),
                launch_point_order(b.p8, total_n, b.offs, b.ounits, (int)nounits, batch, b.osc, b.p8s,
                                   kinit ? b.p4s : nullptr, nullptr, c.s));
    }
    COUNTED(prof, 1, launch_fill_padding_batched(b.params, b.insts, batch, 0, b.npairs, c.s));
    float* w_d = (kw == Kind::Device) ? weights : b.mw;
    float* mu_d = (km == Kind::Device) ? means : b.mmu;
    float* cov_d = (kc == Kind::Device) ? covs : b.mcov;
    if (kinit) {
        // KInit of every instance: batched seeding launches (one cluster per
        // instance, one launch per cluster size), batched Lloyd, batched one-hot
        // statistics
        GIRA_CUDA(cudaMemsetAsync(b.sums, 0, sizeof(double) * 4 * total_k, c.s));
        GIRA_CUDA(cudaMemsetAsync(b.chg, 0, sizeof(unsigned long long) * batch * (o.lloyd_iters + 1), c.s));
        GIRA_CUDA(cudaMemsetAsync(b.stats64, 0, sizeof(double) * NSTAT * total_k, c.s));
        GIRA_CUDA(cudaMemcpyAsync(b.ktab, ktab.data(), sizeof(KppInst) * batch, cudaMemcpyHostToDevice, c.s));
        if (!kseed.empty())
            GIRA_CUDA(cudaMemcpyAsync(b.kseed, kseed.data(), sizeof(KppInst) * kseed.size(), cudaMemcpyHostToDevice,
                                      c.s));
        GIRA_CUDA(cudaMemcpyAsync(b.lunits, lloyd_units.data(), sizeof(BatchUnit) * lloyd_units.size(),
                                  cudaMemcpyHostToDevice, c.s));
        int seed_off = 0;
        for (const auto& sc : seed_class) {
            COUNTED(prof, 1, launch_kpp_cluster_batched(b.p4, b.kseed + seed_off, sc.second, o.seed, b.c4, b.ch,
                                                        sc.first, b.st, c.s));
            seed_off += sc.second;
        }
        for (int i : seed_alone) {   // beyond one 16-CTA cluster: two launches per centre
            const BatchInst& I = hi[i];
            COUNTED(prof, 2 * I.k - 1, launch_kpp(b.p4 + I.pt_off, I.n, I.k, o.seed, b.c4 + I.comp_off,
                                                  b.d2 + I.pt_off, b.bs + nblk_off[i], b.ch + I.comp_off, b.st + i,
                                                  c.s));
        }
        const float4* p4l = sorted ? b.p4s : b.p4;   // Lloyd and the one-hot statistics: sorted points
        COUNTED(prof, 1 + 2 * o.lloyd_iters,
                launch_lloyd_batched(p4l, b.ktab, b.lunits, (int)lloyd_units.size(), total_k, b.comp_inst,
                                     o.lloyd_iters, b.c4, b.lab, b.sums, b.chg, b.st, c.s));
        COUNTED(prof, 1, launch_label_stats_batched(p4l, total_n, b.offs, batch, b.ktab, b.lab, b.c4, b.stats64,
                                                    b.st, c.s));
        GIRA_CUDA(cudaMemcpyAsync(b.shift4, b.c4, sizeof(float4) * total_k, cudaMemcpyDeviceToDevice, c.s));
        COUNTED(prof, 1, launch_reduce_finalize_batched(nullptr, nullptr, b.stats64, b.shift4, b.insts, b.blocks,
                                                        (int)fin_blocks.size(), o.reg_covar, o.tol, o.iters, b.model64,
                                                        b.params, b.trace, b.st, 0, false, c.s));
    } else {
        if (kw == Kind::Host)
            GIRA_CUDA(cudaMemcpyAsync(b.mw, weights, sizeof(float) * total_k, cudaMemcpyHostToDevice, c.s));
        if (km == Kind::Host)
            GIRA_CUDA(cudaMemcpyAsync(b.mmu, means, sizeof(float) * 3 * total_k, cudaMemcpyHostToDevice, c.s));
        if (kc == Kind::Host)
            GIRA_CUDA(cudaMemcpyAsync(b.mcov, covs, sizeof(float) * 9 * total_k, cudaMemcpyHostToDevice, c.s));
        COUNTED(prof, 1, launch_params_from_model_batched(w_d, mu_d, cov_d, total_k, b.comp_inst, b.insts, b.model64,
                                                          b.params, b.shift4, b.st, c.s));
    }
    // every instance's components along a space-filling curve of their means (as in the single fit)
    COUNTED(prof, 2, launch_order_components_batched(b.model64, b.stats64, total_k, kmax_all, b.insts, batch,
                                                     b.comp_inst, b.perm, b.params, b.shift4, b.st, c.s));
    prof.t_init = prof.mark();

    EStepLaunch base{sorted ? b.p8s : b.p8, 0, 0, b.params, 0, b.partials, b.llp, nullptr, nullptr, 0};
    base.n_buf = total_n;
    base.insts = b.insts;
    base.units = b.units;
    base.states = b.st;
    base.masks = b.masks;
    auto estep_all = [&](bool stats, int iter, cudaStream_t s) -> cudaError_t {
        EStepLaunch a = base;
        a.iter = iter;
        if (!stats) {
            a.partials = nullptr;
            a.masks = nullptr;
        }
        return launch_estep_pt_units(a, stats, (int)units.size(), kmax_all, s);
    };
    GIRA_CUDA(cudaMemcpyAsync(b.insts, hi.data(), sizeof(BatchInst) * batch, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.units, units.data(), sizeof(BatchUnit) * units.size(), cudaMemcpyHostToDevice, c.s));

    // ---- the EM loop: one captured graph (E-step launch per shape class + one finalize per iteration)
    std::string key = std::to_string((uintptr_t)ws->ptr) + "|" + std::to_string(sizer.off) + "|" +
                      std::to_string(batch) + "|" + std::to_string(o.iters) + "|" + std::to_string(o.reg_covar) +
                      "|" + std::to_string(o.tol) + "|" + std::to_string(o.lloyd_iters) + "|" +
                      std::to_string((int)kinit) + std::to_string((int)(kp == Kind::Host)) +
                      std::to_string((int)model_host);
    for (int i = 0; i < batch; ++i) key += "|" + std::to_string(hi[i].n) + ":" + std::to_string(hi[i].k);
    if (o.iters > 0) {
        if (ws->graph_key != key || !ws->graph_exec) {
            drop_graph(ws);
            if (!ws->capture_stream) GIRA_CUDA(cudaStreamCreateWithFlags(&ws->capture_stream, cudaStreamNonBlocking));
            cudaStream_t cs = ws->capture_stream;
            GIRA_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
            cudaError_t e = cudaSuccess;
            for (int t = 1; t <= o.iters && e == cudaSuccess; ++t) {
                e = estep_all(true, t, cs);
                if (e == cudaSuccess)
                    e = launch_reduce_finalize_batched(b.partials, b.llp, nullptr, b.shift4, b.insts, b.blocks,
                                                       (int)fin_blocks.size(), o.reg_covar, o.tol, o.iters,
                                                       b.model64, b.params, b.trace, b.st, t, true, cs, b.perm,
                                                       b.masks);
            }
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return fail(GIRA_ERR_CUDA, "capturing the batched EM graph failed: %s",
                            cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(GIRA_ERR_CUDA, "instantiating the batched EM graph failed: %s", cudaGetErrorString(e));
            }
            ws->graph_exec = exec;
            ws->graph_key = key;
        }
        prof.launches += (long long)o.iters * 2;
        GIRA_CUDA(cudaGraphLaunch(ws->graph_exec, c.s));
    }
    prof.t_em = prof.mark();
    if (final_loglik) {
        GIRA_CUDA(estep_all(false, 0, c.s));
        prof.launches += 1;
        COUNTED(prof, 1, launch_ll_reduce_batched(b.llp, b.insts, batch, b.st, c.s));
    }
    COUNTED(prof, 1, launch_model_out_batched(b.model64, b.insts, batch, w_d, mu_d, cov_d, b.st, c.s, b.perm));
    if (kw == Kind::Host)
        GIRA_CUDA(cudaMemcpyAsync(weights, b.mw, sizeof(float) * total_k, cudaMemcpyDeviceToHost, c.s));
    if (km == Kind::Host)
        GIRA_CUDA(cudaMemcpyAsync(means, b.mmu, sizeof(float) * 3 * total_k, cudaMemcpyDeviceToHost, c.s));
    if (kc == Kind::Host)
        GIRA_CUDA(cudaMemcpyAsync(covs, b.mcov, sizeof(float) * 9 * total_k, cudaMemcpyDeviceToHost, c.s));
    if (loglik_traces && o.iters > 0)
        GIRA_CUDA(cudaMemcpyAsync(loglik_traces, b.trace, sizeof(double) * batch * o.iters, cudaMemcpyDeviceToHost,
                                  c.s));
    GIRA_CUDA(cudaMemcpyAsync(hs.data(), b.st, sizeof(DeviceState) * batch, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    long long em_iters = 0;
    for (const auto& h : hs) em_iters += h.iters_done;
    prof.commit((int)std::min<long long>(em_iters, INT_MAX), 0);
    gira_status first = GIRA_OK;
    int first_i = -1;
    for (int i = 0; i < batch; ++i) {
        gira_status si = GIRA_OK;
        if (hs[i].error) {
            si = device_status(hs[i]);
            if (first == GIRA_OK) {
                first = si;
                first_i = i;
            }
        }
        if (statuses) statuses[i] = (int)si;
        if (iters_done) iters_done[i] = hs[i].iters_done;
        if (final_loglik) final_loglik[i] = hs[i].ll_sum / (double)hi[i].n;
    }
    if (first != GIRA_OK) {
        if (hs[first_i].error == GIRA_ERR_NOT_PD) t_bad = hs[first_i].bad_component;
        const std::string m = t_msg;
        return fail(first, "instance %d: %s", first_i, m.c_str());
    }
    return GIRA_OK;
}

// ================================================================ gmm_loglik_grad_batched
gira_status gira_gmm_loglik_grad_batched(const float* points, const int64_t* offsets, int batch, const int* ks,
                                         const float* poses, const float* logits, const float* means,
                                         const float* chol, double* logliks, float* grad_points, double* grad_pose,
                                         double* grad_twist, float* grad_logits, float* grad_means,
                                         float* grad_chol, int* statuses, void* stream) {
    CallRange nvtx_range("gira_gmm_loglik_grad_batched");
    reset_error();
    if (!offsets || !ks) return fail(GIRA_ERR_INVALID_ARG, "offsets and ks must not be NULL");
    if (batch < 1) return fail(GIRA_ERR_INVALID_ARG, "batch = %d < 1", batch);
    if (offsets[0] != 0) return fail(GIRA_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int i = 0; i < batch; ++i) {
        const int64_t n = offsets[i + 1] - offsets[i];
        if (n < 1) return fail(GIRA_ERR_INVALID_ARG, "instance %d has %lld points", i, (long long)n);
        if (ks[i] < 1 || ks[i] > GIRA_MAX_K_BATCHED || ks[i] > n)
            return fail(GIRA_ERR_INVALID_ARG, "instance %d: k = %d outside [1, min(n, %d)]", i, ks[i],
                        GIRA_MAX_K_BATCHED);
    }
    if (!points || !logits || !means || !chol) return fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    const int64_t total_n = offsets[batch];
    Ctx c;
    TRY(begin(c, stream));
    struct Arg {
        const void* p;
        const char* name;
        Kind k = Kind::Device;
    };
    Arg in[5] = {{points, "points"}, {poses, "poses"}, {logits, "logits"}, {means, "means"}, {chol, "chol"}};
    Arg out[7] = {{grad_points, "grad_points"}, {grad_pose, "grad_pose"}, {grad_twist, "grad_twist"},
                  {grad_logits, "grad_logits"}, {grad_means, "grad_means"}, {grad_chol, "grad_chol"},
                  {nullptr, ""}};
    for (auto& a : in)
        if (a.p) TRY(check_ptr(a.p, a.name, c.dev, &a.k));
    for (auto& a : out)
        if (a.p) TRY(check_ptr(a.p, a.name, c.dev, &a.k));
    const int Q = estep_batch_q();

    // ---- tables: instances, shape classes (points per CTA by a balance rule), finalize blocks
    std::vector<BatchInst> hi(batch);
    std::vector<int> npairs_of(batch);
    int total_k = 0;
    int64_t par_floats = 0;
    std::map<std::pair<int, int>, int> class_of_shape;
    std::vector<BatchClass> cls;
    for (int i = 0; i < batch; ++i) {
        BatchInst& I = hi[i];
        I.pt_off = offsets[i];
        I.n = offsets[i + 1] - offsets[i];
        I.k = ks[i];
        I.comp_off = total_k;
        total_k += ks[i];
        npairs_of[i] = params_pairs_padded(ks[i]);
        I.par_off = par_floats;
        par_floats += (int64_t)npairs_of[i] * PAIR_FLOATS;
        int np, g, th;
        estep_shape(ks[i], &np, &g, &th);
        auto key = std::make_pair(np, g);
        auto it = class_of_shape.find(key);
        if (it == class_of_shape.end()) {
            it = class_of_shape.emplace(key, (int)cls.size()).first;
            cls.emplace_back();
            cls.back().np = np;
            cls.back().g = g;
            cls.back().threads = th;
        }
        BatchClass& C = cls[it->second];
        C.insts.push_back(i);
        C.points += I.n;
        C.kmax = std::max(C.kmax, ks[i]);
    }
    for (auto& C : cls) {
        const int occ = estep_grad_occupancy(C.kmax, 1024);
        int64_t ppc = (C.points + 2LL * c.sms * occ - 1) / (2LL * c.sms * occ);
        C.ppc = std::min<int64_t>(estep_ppc_max(), std::max<int64_t>(4 * Q, (ppc + Q - 1) / Q * Q));
    }
    std::vector<BatchUnit> units;
    int64_t part_floats = 0, ll_slots = 0;
    build_tables(hi, cls, units, &part_floats, &ll_slots);
    std::vector<int2> fin_blocks;
    const int cpb = fin_components_per_block();
    for (int i = 0; i < batch; ++i)
        for (int j = 0; j * cpb < ks[i]; ++j) fin_blocks.push_back(make_int2(i, j));

    struct Bufs {
        DeviceState* st;
        float *pin, *poses, *lg, *mu, *ch, *params, *partials, *gp, *gl, *gm, *gc;
        float4 *p8, *shift4;
        double *model64, *llp, *ppart, *gpose, *gtwist;
        BatchInst* insts;
        BatchUnit* units;
        int2* blocks;
        int* npairs;
        int64_t* offs;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(batch);
        b.pin = cv.take<float>(3 * (size_t)total_n);
        b.poses = cv.take<float>(12 * (size_t)batch);
        b.lg = cv.take<float>(total_k);
        b.mu = cv.take<float>(3 * (size_t)total_k);
        b.ch = cv.take<float>(9 * (size_t)total_k);
        b.p8 = cv.take<float4>(2 * (size_t)total_n);
        b.params = cv.take<float>((size_t)par_floats);
        b.shift4 = cv.take<float4>(total_k);
        b.model64 = cv.take<double>((size_t)total_k * MODEL);
        b.partials = cv.take<float>((size_t)part_floats);
        b.llp = cv.take<double>((size_t)ll_slots);
        b.ppart = cv.take<double>(12 * (size_t)ll_slots);
        b.gp = cv.take<float>(3 * (size_t)total_n);
        b.gl = cv.take<float>(total_k);
        b.gm = cv.take<float>(3 * (size_t)total_k);
        b.gc = cv.take<float>(9 * (size_t)total_k);
        b.gpose = cv.take<double>(12 * (size_t)batch);
        b.gtwist = cv.take<double>(6 * (size_t)batch);
        b.insts = cv.take<BatchInst>(batch);
        b.units = cv.take<BatchUnit>(units.size());
        b.blocks = cv.take<int2>(fin_blocks.size());
        b.npairs = cv.take<int>(batch);
        b.offs = cv.take<int64_t>(batch + 1);
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);

    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    std::vector<DeviceState> hs(batch);
    for (auto& h : hs) {
        h = DeviceState{};
        h.bad_component = INT_MAX;
    }
    // every input staged into the workspace, so that the cached graph reads only workspace memory
    auto stage = [&](void* dst, const Arg& a, size_t bytes) -> gira_status {
        GIRA_CUDA(cudaMemcpyAsync(dst, a.p, bytes, a.k == Kind::Host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  c.s));
        return GIRA_OK;
    };
    GIRA_CUDA(cudaMemcpyAsync(b.st, hs.data(), sizeof(DeviceState) * batch, cudaMemcpyHostToDevice, c.s));
    TRY(stage(b.pin, in[0], sizeof(float) * 3 * total_n));
    if (poses) {
        TRY(stage(b.poses, in[1], sizeof(float) * 12 * batch));
    } else {
        std::vector<float> id(12 * (size_t)batch, 0.f);
        for (int i = 0; i < batch; ++i) id[12 * i] = id[12 * i + 4] = id[12 * i + 8] = 1.f;
        GIRA_CUDA(cudaMemcpyAsync(b.poses, id.data(), sizeof(float) * id.size(), cudaMemcpyHostToDevice, c.s));
        GIRA_CUDA(cudaStreamSynchronize(c.s));   // id is a host temporary
    }
    TRY(stage(b.lg, in[2], sizeof(float) * total_k));
    TRY(stage(b.mu, in[3], sizeof(float) * 3 * total_k));
    TRY(stage(b.ch, in[4], sizeof(float) * 9 * total_k));
    GIRA_CUDA(cudaMemcpyAsync(b.offs, offsets, sizeof(int64_t) * (batch + 1), cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.insts, hi.data(), sizeof(BatchInst) * batch, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.units, units.data(), sizeof(BatchUnit) * units.size(), cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.blocks, fin_blocks.data(), sizeof(int2) * fin_blocks.size(), cudaMemcpyHostToDevice,
                              c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.npairs, npairs_of.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, c.s));
    prof.t_init = prof.mark();

    // ---- one graph: move the scans, build the parameters, the adjoint E-step per shape class, finalize
    std::string key = "grad|" + std::to_string((uintptr_t)ws->ptr) + "|" + std::to_string(sizer.off) + "|" +
                      std::to_string(batch);
    for (int i = 0; i < batch; ++i) key += "|" + std::to_string(hi[i].n) + ":" + std::to_string(hi[i].k);
    if (ws->graph_key != key || !ws->graph_exec) {
        drop_graph(ws);
        if (!ws->capture_stream) GIRA_CUDA(cudaStreamCreateWithFlags(&ws->capture_stream, cudaStreamNonBlocking));
        cudaStream_t cs = ws->capture_stream;
        GIRA_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        cudaError_t e = launch_pack_pose_batched(b.pin, total_n, b.offs, batch, b.poses, b.p8, b.st, cs);
        if (e == cudaSuccess) e = launch_fill_padding_batched(b.params, b.insts, batch, 0, b.npairs, cs);
        if (e == cudaSuccess)
            e = launch_params_from_chol_batched(b.lg, b.mu, b.ch, b.insts, batch, b.model64, b.params, b.shift4, b.st,
                                                cs);
        EStepLaunch a{b.p8, 0, 0, b.params, 0, b.partials, b.llp, nullptr, nullptr, 0};
        a.insts = b.insts;
        a.states = b.st;
        a.grad_pts = b.gp;
        a.rot = b.poses;
        a.pose_partials = b.ppart;
        for (const BatchClass& C : cls) {
            if (e != cudaSuccess || !C.nunits) continue;
            a.units = b.units + C.unit_begin;
            e = launch_estep_grad_units(a, C.nunits, C.kmax, C.ppc, cs);
        }
        if (e == cudaSuccess)
            e = launch_grad_finalize_batched(b.partials, b.llp, b.ppart, b.poses, b.ch, b.model64, b.insts, b.blocks,
                                             (int)fin_blocks.size(), b.gl, b.gm, b.gc, b.gpose, b.gtwist, b.st, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail(GIRA_ERR_CUDA, "capturing the batched gradient graph failed: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GIRA_ERR_CUDA, "instantiating the batched gradient graph failed: %s", cudaGetErrorString(e));
        }
        ws->graph_exec = exec;
        ws->graph_key = key;
    }
    prof.launches += 4 + (long long)cls.size();
    GIRA_CUDA(cudaGraphLaunch(ws->graph_exec, c.s));
    prof.t_em = prof.mark();
    const void* src[6] = {b.gp, b.gpose, b.gtwist, b.gl, b.gm, b.gc};
    const size_t bytes[6] = {sizeof(float) * 3 * total_n, sizeof(double) * 12 * batch, sizeof(double) * 6 * batch,
                             sizeof(float) * total_k, sizeof(float) * 3 * total_k, sizeof(float) * 9 * total_k};
    for (int o = 0; o < 6; ++o)
        if (out[o].p)
            GIRA_CUDA(cudaMemcpyAsync(const_cast<void*>(out[o].p), src[o], bytes[o],
                                      out[o].k == Kind::Host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(hs.data(), b.st, sizeof(DeviceState) * batch, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    prof.commit(0, 0);
    gira_status first = GIRA_OK;
    int first_i = -1;
    for (int i = 0; i < batch; ++i) {
        gira_status si = GIRA_OK;
        if (hs[i].error) {
            si = device_status(hs[i]);
            if (first == GIRA_OK) {
                first = si;
                first_i = i;
            }
        }
        if (statuses) statuses[i] = (int)si;
        if (logliks) logliks[i] = hs[i].ll_sum;
    }
    if (first != GIRA_OK) {
        if (hs[first_i].error == GIRA_ERR_NOT_PD) t_bad = hs[first_i].bad_component;
        const std::string m = t_msg;
        return fail(first, "instance %d: %s", first_i, m.c_str());
    }
    return GIRA_OK;
}


// ================================================================ four dimensions
namespace {
gira_status check_nk4(int64_t n, int k) {
    if (n < 1) return fail(GIRA_ERR_INVALID_ARG, "n = %lld < 1", (long long)n);
    if (k < 1 || k > GIRA_MAX_K4) return fail(GIRA_ERR_INVALID_ARG, "k = %d outside [1, %d]", k, GIRA_MAX_K4);
    if (k > n) return fail(GIRA_ERR_INVALID_ARG, "k = %d > n = %lld", k, (long long)n);
    return GIRA_OK;
}

// K above MAX_K4_DIRECT: per-point state of the two-level log-sum-exp.
struct Chunk4Bufs {
    float* gref = nullptr;     // [2]: max_b c_b, log-likelihood reference
    float* psum = nullptr;     // [chunks][n]
    float2* pref = nullptr;    // [n] (shift, 1 / total)
    double* llpt = nullptr;    // [n] natural-log per-point log-likelihood
    int* flags = nullptr;      // [n] points for the exact step
    int* flag_count = nullptr;
};

void carve_chunk4(Carver& cv, int64_t n, int chunks, Chunk4Bufs* b) {
    b->gref = cv.take<float>(2);
    b->psum = cv.take<float>((size_t)chunks * n);
    b->pref = cv.take<float2>(n);
    b->llpt = cv.take<double>(n);
    b->flags = cv.take<int>(n);
    b->flag_count = cv.take<int>(1);
}

// Reference, pass A, per-point totals, exact step for underflowing points, and
// the fixed-order log-likelihood partials (into st->ll_sum when ll_to_state).
cudaError_t chunk4_lse(const Chunk4Bufs& b, EStep4Launch a, int grid, double* llp, bool ll_to_state,
                       long long* launches, cudaStream_t s) {
    const int chunks = (a.k + CHUNK4 - 1) / CHUNK4;
    a.partials = nullptr;
    a.gref = b.gref;
    a.psum = b.psum;
    cudaError_t e = launch_chunk_ref4(a.params, a.k, a.st, b.gref, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.flag_count, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_estep4_chunks(a, 1, grid, s);
    if (e == cudaSuccess)
        e = launch_chunk_combine(b.psum, chunks, a.n, b.gref, b.pref, b.llpt, b.flag_count, b.flags, a.st, s);
    if (e == cudaSuccess)
        e = launch_chunk_exact4(a.pts8, a.params, a.k, b.gref, b.flags, b.flag_count, b.pref, b.llpt, a.st, s);
    if (e == cudaSuccess) e = launch_points_ll_reduce(b.llpt, a.n, llp, ll_to_state ? a.st : nullptr, s);
    *launches += 5 + (ll_to_state ? 1 : 0);
    return e;
}
}  // namespace

gira_status gira_gmm_fit4(const float* points, int64_t n, int k, const gira_fit_opts* opts, float* weights,
                          float* means, float* covs, double* loglik_trace, int* iters_done, double* final_loglik,
                          void* stream) {
    CallRange nvtx_range("gira_gmm_fit4");
    reset_error();
    if (!opts) return fail(GIRA_ERR_INVALID_ARG, "opts is NULL");
    TRY(check_nk4(n, k));
    const gira_fit_opts o = *opts;
    TRY(check_opts(o));
    if (!points || !weights || !means || !covs) return fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    Ctx c;
    TRY(begin(c, stream));
    Kind kp, kw, km, kc;
    TRY(check_ptr(points, "points", c.dev, &kp));
    TRY(check_ptr(weights, "weights", c.dev, &kw));
    TRY(check_ptr(means, "means", c.dev, &km));
    TRY(check_ptr(covs, "covs", c.dev, &kc));
    const bool kinit = o.init_mode == GIRA_INIT_KMEANS;
    const bool chunked = k > MAX_K4_DIRECT;   // two-level log-sum-exp over chunks of CHUNK4 components
    const int chunks = chunked ? (k + CHUNK4 - 1) / CHUNK4 : 1;
    const int kpad = params4_pairs(k);
    int64_t ppc = 0;
    const int grid = estep4_grid(n, chunked ? CHUNK4 : k, c.sms, &ppc);   // CTAs per chunk when chunked
    const int kblk = chunked ? CHUNK4 : k;                                 // components per partial block
    const int nblk = kpp_num_blocks(n);
    int kgrid = kinit ? kpp_persistent_grid() : 0;
    if (kgrid > 0 && n > kpp_persistent_max_n(kgrid)) kgrid = 0;
    Chunk4Bufs cb;
    struct Bufs {
        DeviceState* st;
        float *pin, *params, *partials, *d2, *mw, *mmu, *mcov;
        float4 *p4, *p8, *c4;
        double *model64, *stats64, *llp, *trace, *sums;
        u128 *bs, *ksums;
        int64_t* ch;
        int32_t* lab;
        int *ksync, *perm;
        unsigned long long* chg;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.perm = cv.take<int>(k);
        b.pin = cv.take<float>(kp == Kind::Host ? 4 * n : 0);
        b.p4 = cv.take<float4>(n);
        b.p8 = cv.take<float4>(2 * (size_t)n);
        b.params = cv.take<float>((size_t)kpad * PAIR4_FLOATS);
        b.model64 = cv.take<double>((size_t)k * MODEL4);
        b.stats64 = cv.take<double>((size_t)k * NSTAT4);
        b.partials = cv.take<float>((size_t)chunks * grid * kblk * NSTAT4);
        b.llp = cv.take<double>(std::max(grid, chunk_combine_grid()));
        if (chunked) carve_chunk4(cv, n, chunks, &cb);
        b.trace = cv.take<double>(std::max(o.iters, 1));
        b.mw = cv.take<float>(kw == Kind::Host ? k : 0);
        b.mmu = cv.take<float>(km == Kind::Host ? 4 * (size_t)k : 0);
        b.mcov = cv.take<float>(kc == Kind::Host ? 16 * (size_t)k : 0);
        if (kinit) {
            b.c4 = cv.take<float4>(k);
            b.d2 = cv.take<float>(2 * (size_t)n);   // double-buffered by the persistent seeding
            b.bs = cv.take<u128>(nblk);
            b.ch = cv.take<int64_t>(k);
            b.lab = cv.take<int32_t>(n);
            b.sums = cv.take<double>(5 * (size_t)k);
            b.chg = cv.take<unsigned long long>(o.lloyd_iters + 1);
            b.ksync = cv.take<int>((size_t)k + 1);
            b.ksums = cv.take<u128>(kpp_persistent_sum_words(std::max(kgrid, 1), k));
        }
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);

    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    DeviceState h{};
    h.stop_after = o.iters;
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemsetAsync(b.trace, 0xff, sizeof(double) * std::max(o.iters, 1), c.s));   // NaN
    const float* pts = points;
    if (kp == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.pin, points, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, c.s));
        pts = b.pin;
    }
    COUNTED(prof, 1, launch_pack4(pts, n, b.p4, b.p8, b.st, c.s));
    COUNTED(prof, 1, launch_fill_padding4(b.params, k, c.s));
    float* w_d = (kw == Kind::Device) ? weights : b.mw;
    float* mu_d = (km == Kind::Device) ? means : b.mmu;
    float* cov_d = (kc == Kind::Device) ? covs : b.mcov;
    if (kinit) {
        if (kgrid > 0) {
            GIRA_CUDA(cudaMemsetAsync(b.ksync, 0, sizeof(int) * (k + 1), c.s));
            COUNTED(prof, 1, launch_kpp_persistent(b.p4, n, k, o.seed, b.c4, b.d2, b.ch, b.ksync, b.ksums, kgrid, b.st,
                                                   c.s, 4));
        } else {
            COUNTED(prof, 2 * k - 1, launch_kpp(b.p4, n, k, o.seed, b.c4, b.d2, b.bs, b.ch, b.st, c.s, 4));
        }
        GIRA_CUDA(cudaMemsetAsync(b.sums, 0, sizeof(double) * 5 * k, c.s));
        GIRA_CUDA(cudaMemsetAsync(b.chg, 0, sizeof(unsigned long long) * (o.lloyd_iters + 1), c.s));
        COUNTED(prof, 1 + 2 * o.lloyd_iters, launch_lloyd4(b.p4, n, k, o.lloyd_iters, b.c4, b.lab, b.sums, b.chg,
                                                          b.st, c.s));
        GIRA_CUDA(cudaMemsetAsync(b.stats64, 0, sizeof(double) * NSTAT4 * k, c.s));
        COUNTED(prof, 1, launch_label_stats4(b.p4, n, k, b.lab, b.c4, b.stats64, b.st, c.s));
        COUNTED(prof, 1, launch_reduce_finalize4(nullptr, 0, k, nullptr, 0, b.stats64, b.c4, k, n, o.reg_covar,
                                                 o.tol, b.model64, b.params, b.trace, b.st, 0, false, c.s));
    } else {
        if (kw == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(b.mw, weights, sizeof(float) * k, cudaMemcpyHostToDevice, c.s));
        if (km == Kind::Host)
            GIRA_CUDA(cudaMemcpyAsync(b.mmu, means, sizeof(float) * 4 * k, cudaMemcpyHostToDevice, c.s));
        if (kc == Kind::Host)
            GIRA_CUDA(cudaMemcpyAsync(b.mcov, covs, sizeof(float) * 16 * k, cudaMemcpyHostToDevice, c.s));
        COUNTED(prof, 1, launch_params_from_model4(w_d, mu_d, cov_d, k, b.model64, b.params, b.st, c.s));
    }
    prof.t_init = prof.mark();
    EStep4Launch a{b.p8, n, k, b.params, ppc, b.partials, b.llp, nullptr, b.st, 0};
    for (int t = 1; t <= o.iters; ++t) {
        a.iter = t;
        if (chunked) {
            GIRA_CUDA(chunk4_lse(cb, a, grid, b.llp, false, &prof.launches, c.s));
            EStep4Launch pb = a;
            pb.gref = cb.gref;
            pb.pref = cb.pref;
            COUNTED(prof, 1, launch_estep4_chunks(pb, 2, grid, c.s));
            COUNTED(prof, 1, launch_reduce_finalize4(b.partials, grid, kblk, b.llp, chunk_combine_grid(), nullptr,
                                                     nullptr, k, n, o.reg_covar, o.tol, b.model64, b.params, b.trace,
                                                     b.st, t, true, c.s));
            continue;
        }
        const bool pdl = !prof.per_launch;   // dependent launches, as in the 3-D loop
        cudaEvent_t e0 = prof.mark_launch();
        COUNTED(prof, 1, launch_estep4(a, true, grid, c.s, pdl));
        cudaEvent_t e1 = prof.mark_launch();
        if (prof.per_launch) prof.timed(e0, e1);
        COUNTED(prof, 1, launch_reduce_finalize4(b.partials, grid, kblk, b.llp, grid, nullptr, nullptr, k, n,
                                                 o.reg_covar, o.tol, b.model64, b.params, b.trace, b.st, t, true,
                                                 c.s, pdl));
    }
    prof.t_em = prof.mark();
    if (final_loglik) {
        EStep4Launch f = a;
        f.iter = 0;
        f.partials = nullptr;
        if (chunked) {
            GIRA_CUDA(chunk4_lse(cb, f, grid, b.llp, true, &prof.launches, c.s));
        } else {
            COUNTED(prof, 1, launch_estep4(f, false, grid, c.s));
            COUNTED(prof, 1, launch_ll_reduce(b.llp, grid, b.st, c.s));
        }
    }
    COUNTED(prof, 1, launch_model_out4(b.model64, k, w_d, mu_d, cov_d, b.st, c.s));
    if (kw == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(weights, b.mw, sizeof(float) * k, cudaMemcpyDeviceToHost, c.s));
    if (km == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(means, b.mmu, sizeof(float) * 4 * k, cudaMemcpyDeviceToHost, c.s));
    if (kc == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(covs, b.mcov, sizeof(float) * 16 * k, cudaMemcpyDeviceToHost, c.s));
    if (loglik_trace && o.iters > 0)
        GIRA_CUDA(cudaMemcpyAsync(loglik_trace, b.trace, sizeof(double) * o.iters, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    prof.commit(h.iters_done, h.iters_done);
    TRY(device_status(h));
    if (iters_done) *iters_done = h.iters_done;
    if (final_loglik) *final_loglik = h.ll_sum / (double)n;
    return GIRA_OK;
}

gira_status gira_gmm_loglik4(const float* points, int64_t n, int k, const float* weights, const float* means,
                             const float* covs, double* mean_loglik, float* per_point, void* stream) {
    CallRange nvtx_range("gira_gmm_loglik4");
    reset_error();
    TRY(check_nk4(n, k));
    if (!points || !weights || !means || !covs) return fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    Ctx c;
    TRY(begin(c, stream));
    Kind kp, kw, km, kc, kpp = Kind::Host;
    TRY(check_ptr(points, "points", c.dev, &kp));
    TRY(check_ptr(weights, "weights", c.dev, &kw));
    TRY(check_ptr(means, "means", c.dev, &km));
    TRY(check_ptr(covs, "covs", c.dev, &kc));
    if (per_point) TRY(check_ptr(per_point, "per_point", c.dev, &kpp));
    const bool chunked = k > MAX_K4_DIRECT;
    const int chunks = chunked ? (k + CHUNK4 - 1) / CHUNK4 : 1;
    const int kpad = params4_pairs(k);
    int64_t ppc = 0;
    const int grid = estep4_grid(n, chunked ? CHUNK4 : k, c.sms, &ppc);
    Chunk4Bufs cb;
    struct Bufs {
        DeviceState* st;
        float *pin, *params, *mw, *mmu, *mcov, *pp;
        float4* p8;
        double *model64, *llp;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.pin = cv.take<float>(kp == Kind::Host ? 4 * n : 0);
        b.p8 = cv.take<float4>(2 * (size_t)n);
        b.params = cv.take<float>((size_t)kpad * PAIR4_FLOATS);
        b.model64 = cv.take<double>((size_t)k * MODEL4);
        b.llp = cv.take<double>(std::max(grid, chunk_combine_grid()));
        if (chunked) carve_chunk4(cv, n, chunks, &cb);
        b.mw = cv.take<float>(kw == Kind::Host ? k : 0);
        b.mmu = cv.take<float>(km == Kind::Host ? 4 * (size_t)k : 0);
        b.mcov = cv.take<float>(kc == Kind::Host ? 16 * (size_t)k : 0);
        b.pp = cv.take<float>((per_point && kpp == Kind::Host) ? n : 0);
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);

    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    DeviceState h{};
    h.stop_after = 0;
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    const float* pts = points;
    if (kp == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.pin, points, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, c.s));
        pts = b.pin;
    }
    const float* w_d = weights;
    const float* mu_d = means;
    const float* cov_d = covs;
    if (kw == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.mw, weights, sizeof(float) * k, cudaMemcpyHostToDevice, c.s));
        w_d = b.mw;
    }
    if (km == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.mmu, means, sizeof(float) * 4 * k, cudaMemcpyHostToDevice, c.s));
        mu_d = b.mmu;
    }
    if (kc == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.mcov, covs, sizeof(float) * 16 * k, cudaMemcpyHostToDevice, c.s));
        cov_d = b.mcov;
    }
    COUNTED(prof, 1, launch_pack4(pts, n, nullptr, b.p8, b.st, c.s));
    COUNTED(prof, 1, launch_fill_padding4(b.params, k, c.s));
    COUNTED(prof, 1, launch_params_from_model4(w_d, mu_d, cov_d, k, b.model64, b.params, b.st, c.s));
    prof.t_init = prof.mark();
    prof.t_em = prof.t_init;
    float* ppd = per_point ? ((kpp == Kind::Device) ? per_point : b.pp) : nullptr;
    EStep4Launch a{b.p8, n, k, b.params, ppc, nullptr, b.llp, ppd, b.st, 0};
    if (chunked) {
        GIRA_CUDA(chunk4_lse(cb, a, grid, b.llp, true, &prof.launches, c.s));
        if (ppd) COUNTED(prof, 1, launch_double_to_float(cb.llpt, n, ppd, c.s));
    } else {
        COUNTED(prof, 1, launch_estep4(a, false, grid, c.s));
        COUNTED(prof, 1, launch_ll_reduce(b.llp, grid, b.st, c.s));
    }
    if (per_point && kpp == Kind::Host)
        GIRA_CUDA(cudaMemcpyAsync(per_point, b.pp, sizeof(float) * n, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    prof.commit(0, 0);
    TRY(device_status(h));
    if (mean_loglik) *mean_loglik = h.ll_sum / (double)n;
    return GIRA_OK;
}

gira_status gira_gmm_conditional4(const float* locs, int64_t m, int k, const float* weights, const float* means,
                                  const float* covs, float* cond_mean, float* cond_var, void* stream) {
    CallRange nvtx_range("gira_gmm_conditional4");
    reset_error();
    if (m < 1) return fail(GIRA_ERR_INVALID_ARG, "m = %lld < 1", (long long)m);
    if (k < 1 || k > GIRA_MAX_K4) return fail(GIRA_ERR_INVALID_ARG, "k = %d outside [1, %d]", k, GIRA_MAX_K4);
    if (!locs || !weights || !means || !covs || !cond_mean)
        return fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    Ctx c;
    TRY(begin(c, stream));
    Kind kl, kw, km, kc, ke, kv = Kind::Host;
    TRY(check_ptr(locs, "locs", c.dev, &kl));
    TRY(check_ptr(weights, "weights", c.dev, &kw));
    TRY(check_ptr(means, "means", c.dev, &km));
    TRY(check_ptr(covs, "covs", c.dev, &kc));
    TRY(check_ptr(cond_mean, "cond_mean", c.dev, &ke));
    if (cond_var) TRY(check_ptr(cond_var, "cond_var", c.dev, &kv));
    struct Bufs {
        DeviceState* st;
        float *lin, *mw, *mmu, *mcov, *prep, *e, *v;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.lin = cv.take<float>(kl == Kind::Host ? 3 * m : 0);
        b.mw = cv.take<float>(kw == Kind::Host ? k : 0);
        b.mmu = cv.take<float>(km == Kind::Host ? 4 * (size_t)k : 0);
        b.mcov = cv.take<float>(kc == Kind::Host ? 16 * (size_t)k : 0);
        b.prep = cv.take<float>((size_t)k * cond_floats());
        b.e = cv.take<float>(ke == Kind::Host ? m : 0);
        b.v = cv.take<float>((kv == Kind::Host || !cond_var) ? m : 0);
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);
    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    DeviceState h{};
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    auto stage = [&](const float* src, Kind kd, float* buf, size_t count) -> const float* {
        if (kd != Kind::Host) return src;
        if (cudaMemcpyAsync(buf, src, sizeof(float) * count, cudaMemcpyHostToDevice, c.s) != cudaSuccess) return nullptr;
        return buf;
    };
    const float* l_d = stage(locs, kl, b.lin, 3 * (size_t)m);
    const float* w_d = stage(weights, kw, b.mw, k);
    const float* mu_d = stage(means, km, b.mmu, 4 * (size_t)k);
    const float* cov_d = stage(covs, kc, b.mcov, 16 * (size_t)k);
    if (!l_d || !w_d || !mu_d || !cov_d) GIRA_CUDA(cudaGetLastError());
    float* e_d = (ke == Kind::Device) ? cond_mean : b.e;
    float* v_d = (cond_var && kv == Kind::Device) ? cond_var : b.v;
    prof.t_init = prof.mark();
    prof.t_em = prof.t_init;
    COUNTED(prof, 2, launch_conditional4(l_d, m, k, w_d, mu_d, cov_d, b.prep, e_d, v_d, b.st, c.s));
    if (ke == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(cond_mean, b.e, sizeof(float) * m, cudaMemcpyDeviceToHost, c.s));
    if (cond_var && kv == Kind::Host)
        GIRA_CUDA(cudaMemcpyAsync(cond_var, b.v, sizeof(float) * m, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    prof.commit(0, 0);
    return device_status(h);
}

gira_status gira_gmm_sample(int64_t m, int k, int d, const float* weights, const float* means, const float* covs,
                            uint64_t seed, float* out, int32_t* components, void* stream) {
    CallRange nvtx_range("gira_gmm_sample");
    reset_error();
    if (m < 1) return fail(GIRA_ERR_INVALID_ARG, "m = %lld < 1", (long long)m);
    if (d != 3 && d != 4) return fail(GIRA_ERR_INVALID_ARG, "d = %d is neither 3 nor 4", d);
    if (k < 1 || k > GIRA_MAX_K) return fail(GIRA_ERR_INVALID_ARG, "k = %d outside [1, %d]", k, GIRA_MAX_K);
    if (!weights || !means || !covs || !out) return fail(GIRA_ERR_INVALID_ARG, "a required pointer is NULL");
    Ctx c;
    TRY(begin(c, stream));
    Kind kw, km, kc, ko, kq = Kind::Host;
    TRY(check_ptr(weights, "weights", c.dev, &kw));
    TRY(check_ptr(means, "means", c.dev, &km));
    TRY(check_ptr(covs, "covs", c.dev, &kc));
    TRY(check_ptr(out, "out", c.dev, &ko));
    if (components) TRY(check_ptr(components, "components", c.dev, &kq));
    struct Bufs {
        DeviceState* st;
        float *mw, *mmu, *mcov, *o;
        double *cum, *chol;
        int32_t* q;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.mw = cv.take<float>(kw == Kind::Host ? k : 0);
        b.mmu = cv.take<float>(km == Kind::Host ? (size_t)d * k : 0);
        b.mcov = cv.take<float>(kc == Kind::Host ? (size_t)d * d * k : 0);
        b.cum = cv.take<double>(k);
        b.chol = cv.take<double>(16 * (size_t)k);
        b.o = cv.take<float>(ko == Kind::Host ? (size_t)d * m : 0);
        b.q = cv.take<int32_t>((components && kq == Kind::Host) ? m : 0);
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);
    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    DeviceState h{};
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    const float* w_d = weights;
    const float* mu_d = means;
    const float* cov_d = covs;
    if (kw == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.mw, weights, sizeof(float) * k, cudaMemcpyHostToDevice, c.s));
        w_d = b.mw;
    }
    if (km == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.mmu, means, sizeof(float) * d * k, cudaMemcpyHostToDevice, c.s));
        mu_d = b.mmu;
    }
    if (kc == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.mcov, covs, sizeof(float) * d * d * k, cudaMemcpyHostToDevice, c.s));
        cov_d = b.mcov;
    }
    float* o_d = (ko == Kind::Device) ? out : b.o;
    int32_t* q_d = components ? ((kq == Kind::Device) ? components : b.q) : nullptr;
    prof.t_init = prof.mark();
    prof.t_em = prof.t_init;
    COUNTED(prof, 2, launch_sample(m, k, d, w_d, mu_d, cov_d, seed, b.cum, b.chol, o_d, q_d, b.st, c.s));
    if (ko == Kind::Host) GIRA_CUDA(cudaMemcpyAsync(out, b.o, sizeof(float) * d * m, cudaMemcpyDeviceToHost, c.s));
    if (components && kq == Kind::Host)
        GIRA_CUDA(cudaMemcpyAsync(components, b.q, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    prof.t_end = prof.mark();
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    prof.commit(0, 0);
    return device_status(h);
}


// ================================================================ gbms (K from a bandwidth)
gira_status gira_gbms(const float* points, int64_t n, int d, double bandwidth, int max_iter, int* k_out,
                      double* modes, int32_t* counts, void* stream) {
    CallRange nvtx_range("gira_gbms");
    reset_error();
    if (n < 1 || n > (int64_t)INT_MAX / 2) return fail(GIRA_ERR_INVALID_ARG, "n = %lld outside [1, 2^30]", (long long)n);
    if (d != 3 && d != 4) return fail(GIRA_ERR_INVALID_ARG, "d = %d is neither 3 nor 4", d);
    if (!(bandwidth > 0.0) || !std::isfinite(bandwidth)) return fail(GIRA_ERR_INVALID_ARG, "bandwidth must be > 0");
    if (max_iter < 1) return fail(GIRA_ERR_INVALID_ARG, "max_iter < 1");
    if (!points || !k_out) return fail(GIRA_ERR_INVALID_ARG, "points and k must not be NULL");
    Ctx c;
    TRY(begin(c, stream));
    Kind kp, km = Kind::Host, kq = Kind::Host;
    TRY(check_ptr(points, "points", c.dev, &kp));
    if (modes) TRY(check_ptr(modes, "modes", c.dev, &km));
    if (counts) TRY(check_ptr(counts, "counts", c.dev, &kq));
    const size_t tb = gbms_temp_bytes(n, d);
    struct Bufs {
        DeviceState* st;
        float* pin;
        float4 *p4, *spts;
        uint64_t *keys, *keys2, *ukeys, *rkeys, *rkeys2, *mkeys, *mkeys2, *mukeys;
        int *idx, *idx2, *ulen, *ustart, *ints, *mcount, *rcount, *midx, *midx2, *mulen, *mustart, *state, *flags,
            *pos, *cout;
        double4 *modes64, *rmodes;
        longlong2 *qxy, *qzw;
        double* mout;
        void* temp;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.pin = cv.take<float>(kp == Kind::Host ? (size_t)d * n : 0);
        b.p4 = cv.take<float4>(n);
        b.spts = cv.take<float4>(n);
        for (uint64_t** p : {&b.keys, &b.keys2, &b.ukeys, &b.rkeys, &b.rkeys2, &b.mkeys, &b.mkeys2, &b.mukeys})
            *p = cv.take<uint64_t>(n);
        for (int** p : {&b.idx, &b.idx2, &b.ulen, &b.ustart, &b.mcount, &b.rcount, &b.midx, &b.midx2, &b.mulen,
                        &b.mustart, &b.state, &b.flags, &b.pos})
            *p = cv.take<int>(n);
        b.ints = cv.take<int>(4);   // cells, live modes, mode cells, undecided
        b.modes64 = cv.take<double4>(n);
        b.rmodes = cv.take<double4>(n);
        b.qxy = cv.take<longlong2>(n);
        b.qzw = cv.take<longlong2>(n);
        b.mout = cv.take<double>((modes && km == Kind::Host) ? (size_t)d * n : 0);
        b.cout = cv.take<int>((counts && kq == Kind::Host) ? n : 0);
        b.temp = cv.take<unsigned char>(tb);
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);
    int* ncells = b.ints;
    int* nlive = b.ints + 1;
    int* mncells = b.ints + 2;
    int* undecided = b.ints + 3;

    CallProfile prof;
    prof.on = g_prof_on.load() != 0;
    prof.per_launch = g_prof_on.load() == 1;
    prof.s = c.s;
    prof.t0 = prof.mark();
    DeviceState h{};
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemsetAsync(b.ints, 0, sizeof(int) * 4, c.s));
    const float* pts = points;
    if (kp == Kind::Host) {
        GIRA_CUDA(cudaMemcpyAsync(b.pin, points, sizeof(float) * d * n, cudaMemcpyHostToDevice, c.s));
        pts = b.pin;
    }
    COUNTED(prof, 1, launch_gbms_keys(pts, n, d, bandwidth, b.p4, b.keys, b.idx, b.st, c.s));
    COUNTED(prof, 3, gbms_sort_cells(b.temp, tb, b.keys, b.keys2, b.idx, b.idx2, n, d, b.ukeys, b.ulen, b.ustart,
                                     ncells, c.s));
    int hints[4];
    GIRA_CUDA(cudaMemcpyAsync(hints, b.ints, sizeof hints, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    TRY(device_status(h));
    const int S = hints[0];
    prof.t_init = prof.mark();
    COUNTED(prof, 1, launch_gbms_gather(b.p4, b.idx2, n, b.spts, b.qxy, b.qzw, c.s));
    COUNTED(prof, 1, launch_gbms_shift(b.spts, b.qxy, b.qzw, b.ukeys, b.ustart, b.ulen, S, d, bandwidth, max_iter,
                                       b.modes64, b.mcount, b.st, c.s));
    COUNTED(prof, 2, launch_gbms_rank(b.temp, tb, b.mcount, S, b.rkeys, b.rkeys2, nlive, c.s));
    GIRA_CUDA(cudaMemcpyAsync(hints, b.ints, sizeof hints, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    const int L = hints[1];
    int K = 0;
    if (L > 0) {
        COUNTED(prof, 1, launch_gbms_rank_modes(b.rkeys2, nlive, L, b.modes64, b.mcount, d, bandwidth, b.rmodes,
                                                b.rcount, b.mkeys, b.midx, b.state, b.st, c.s));
        COUNTED(prof, 3, gbms_sort_cells(b.temp, tb, b.mkeys, b.mkeys2, b.midx, b.midx2, L, d, b.mukeys, b.mulen,
                                         b.mustart, mncells, c.s));
        // every round decides at least the lowest undecided rank: at most L rounds
        for (int round = 0; round < L; round += 2) {
            GIRA_CUDA(cudaMemsetAsync(undecided, 0, sizeof(int), c.s));
            COUNTED(prof, 1, launch_gbms_merge_round(b.rmodes, nlive, L, b.mukeys, b.mustart, b.mulen, mncells,
                                                     b.midx2, d, bandwidth, b.state, undecided, c.s));
            GIRA_CUDA(cudaMemsetAsync(undecided, 0, sizeof(int), c.s));
            COUNTED(prof, 1, launch_gbms_merge_round(b.rmodes, nlive, L, b.mukeys, b.mustart, b.mulen, mncells,
                                                     b.midx2, d, bandwidth, b.state, undecided, c.s));
            int open = 0;
            GIRA_CUDA(cudaMemcpyAsync(&open, undecided, sizeof(int), cudaMemcpyDeviceToHost, c.s));
            GIRA_CUDA(cudaStreamSynchronize(c.s));
            if (open == 0) break;
        }
        double* m_d = modes ? ((km == Kind::Device) ? modes : b.mout) : nullptr;
        int* q_d = counts ? ((kq == Kind::Device) ? counts : b.cout) : nullptr;
        COUNTED(prof, 3, launch_gbms_output(b.temp, tb, b.state, nlive, L, b.rmodes, b.rcount, d, b.flags, b.pos,
                                            m_d, q_d, c.s));
        int last[2];
        GIRA_CUDA(cudaMemcpyAsync(&last[0], b.pos + (L - 1), sizeof(int), cudaMemcpyDeviceToHost, c.s));
        GIRA_CUDA(cudaMemcpyAsync(&last[1], b.flags + (L - 1), sizeof(int), cudaMemcpyDeviceToHost, c.s));
        GIRA_CUDA(cudaStreamSynchronize(c.s));
        K = last[0] + last[1];
        if (modes && km == Kind::Host && K > 0)
            GIRA_CUDA(cudaMemcpyAsync(modes, b.mout, sizeof(double) * d * K, cudaMemcpyDeviceToHost, c.s));
        if (counts && kq == Kind::Host && K > 0)
            GIRA_CUDA(cudaMemcpyAsync(counts, b.cout, sizeof(int) * K, cudaMemcpyDeviceToHost, c.s));
    }
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    prof.t_em = prof.mark();
    prof.t_end = prof.t_em;
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    prof.commit(0, 0);
    TRY(device_status(h));
    *k_out = K;
    return GIRA_OK;
}


// ================================================================ test hooks
void gira_test_fail_next_allocations(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

gira_status gira_test_bounded_wait(int mode, long long limit, void* stream) {
    reset_error();
    if (mode != 0 && mode != 1) return fail(GIRA_ERR_INVALID_ARG, "mode = %d is neither 0 nor 1", mode);
    if (limit < 1 || limit > 2000000000ll) return fail(GIRA_ERR_INVALID_ARG, "limit outside [1, 2e9]");
    Ctx c;
    TRY(begin(c, stream));
    struct Bufs {
        DeviceState* st;
        int* ints;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.ints = cv.take<int>(2);
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);
    DeviceState h{};
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemsetAsync(b.ints, 0, sizeof(int) * 2, c.s));
    GIRA_CUDA(launch_wait_probe(mode, limit, b.ints, b.ints + 1, b.st, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    return device_status(h);
}

gira_status gira_test_point_order(const float* points, int64_t n, int batch, const int64_t* offsets, int* order,
                                  void* stream) {
    reset_error();
    if (n < 1 || batch < 1 || !points || !order) return fail(GIRA_ERR_INVALID_ARG, "n, batch, points or order");
    if (batch > 1 && !offsets) return fail(GIRA_ERR_INVALID_ARG, "offsets is NULL with batch > 1");
    std::vector<int64_t> offs(batch + 1);
    if (offsets) offs.assign(offsets, offsets + batch + 1);
    else offs = {0, n};
    if (offs[0] != 0 || offs[batch] != n) return fail(GIRA_ERR_INVALID_ARG, "offsets must run from 0 to n");
    for (int i = 0; i < batch; ++i)
        if (offs[i + 1] <= offs[i]) return fail(GIRA_ERR_INVALID_ARG, "instance %d is empty", i);
    Ctx c;
    TRY(begin(c, stream));
    Kind kp, ko;
    TRY(check_ptr(points, "points", c.dev, &kp));
    TRY(check_ptr(order, "order", c.dev, &ko));
    if (kp != Kind::Device || ko != Kind::Device) return fail(GIRA_ERR_INVALID_ARG, "points and order: device");
    const int64_t nunits = point_order_box_units(offs.data(), batch);
    std::vector<int2> units((size_t)nunits);
    point_order_fill_units(offs.data(), batch, units.data());
    struct Bufs {
        DeviceState* st;
        float4* p8;
        int64_t* offs;
        int2* units;
        void* osc;
    } b{};
    auto layout = [&](Carver& cv) {
        b.st = cv.take<DeviceState>(1);
        b.p8 = cv.take<float4>(2 * (size_t)n);
        b.offs = cv.take<int64_t>(batch + 1);
        b.units = cv.take<int2>((size_t)nunits);
        b.osc = cv.take<char>(point_order_scratch_bytes(n, batch));
    };
    Carver sizer;
    layout(sizer);
    DeviceWs* ws = ws_for(c.dev);
    std::lock_guard<std::mutex> lk(ws->mu);
    TRY(ensure(ws, sizer.off, c.s));
    Carver cv;
    cv.base = static_cast<char*>(ws->ptr);
    layout(cv);
    DeviceState h{};
    h.bad_component = INT_MAX;
    GIRA_CUDA(cudaMemcpyAsync(b.st, &h, sizeof h, cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.offs, offs.data(), sizeof(int64_t) * (batch + 1), cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(cudaMemcpyAsync(b.units, units.data(), sizeof(int2) * units.size(), cudaMemcpyHostToDevice, c.s));
    GIRA_CUDA(launch_pack(points, n, nullptr, b.p8, b.st, c.s));
    GIRA_CUDA(launch_point_order(b.p8, n, b.offs, b.units, (int)nunits, batch, b.osc, nullptr, nullptr, order, c.s));
    GIRA_CUDA(cudaMemcpyAsync(&h, b.st, sizeof h, cudaMemcpyDeviceToHost, c.s));
    GIRA_CUDA(cudaStreamSynchronize(c.s));
    return device_status(h);
}

}  // extern "C"
