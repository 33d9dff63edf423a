// util.cu -- error reporting, allocation, bounded waits, grid save/load and
// the Philox entry point of libvdbc.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "vdbc_host.h"

namespace vdbc {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

vdbc_status set_error(vdbc_status s, const char* fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

// ---- releases held back by timeouts: a call whose bounded wait ran out
// returns VDBC_ERR_TIMEOUT with its GPU work still queued, so whatever that
// work reads or writes must outlive it.  Such a call hands the release of what
// it created to defer_release: an event is recorded on the stream behind the
// queued work, and the release runs at the entry of a later API call once the
// event has completed (never on the timeout path itself, which therefore
// never blocks in cudaFree either).
struct Deferred {
    cudaEvent_t done;
    std::function<void()> release;
};
static std::mutex g_deferred_mu;
static std::vector<Deferred> g_deferred;
static std::atomic<int> g_deferred_n{0};
static thread_local bool g_in_release = false;

void defer_release(cudaStream_t s, std::function<void()> release)
{
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(ev, s) != cudaSuccess) {
        // the stream cannot be tracked: keep the objects for the life of the
        // process rather than free memory that queued work may still use
        cudaGetLastError();
        if (ev) cudaEventDestroy(ev);
        return;
    }
    std::lock_guard<std::mutex> lock(g_deferred_mu);
    g_deferred.push_back(Deferred{ev, std::move(release)});
    g_deferred_n.store((int)g_deferred.size());
}

int run_ready_releases()
{
    if (g_deferred_n.load() == 0 || g_in_release) return 0;
    std::vector<Deferred> ready;
    {
        std::lock_guard<std::mutex> lock(g_deferred_mu);
        for (size_t i = 0; i < g_deferred.size();) {
            cudaError_t q = cudaEventQuery(g_deferred[i].done);
            if (q == cudaErrorNotReady) { ++i; continue; }
            cudaGetLastError();
            ready.push_back(std::move(g_deferred[i]));
            g_deferred.erase(g_deferred.begin() + (long)i);
        }
        g_deferred_n.store((int)g_deferred.size());
    }
    g_in_release = true;
    for (Deferred& d : ready) {
        d.release();
        cudaEventDestroy(d.done);
    }
    g_in_release = false;
    return (int)ready.size();
}

vdbc_status release_or_defer(vdbc_status st, cudaStream_t s, std::function<void()> release)
{
    if (st == VDBC_ERR_TIMEOUT) defer_release(s, std::move(release));
    else release();
    return st;
}

void clear_error()
{
    g_last_error.clear();
    run_ready_releases();
}

vdbc_status cuda_status(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation)
        return set_error(VDBC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(VDBC_ERR_CUDA, "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
}

bool fault_injected(const char* name)
{
    const char* f = std::getenv("VDBC_FAULT");
    return f && std::strstr(f, name) != nullptr;
}

// the default pool of the current device keeps freed memory for reuse
// (once per device; calls may come from several threads)
static void keep_pool_memory()
{
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    done.push_back(dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
}

vdbc_status dev_alloc(void** p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (fault_injected("oom")) return set_error(VDBC_ERR_OOM, "device allocation of %zu bytes refused (VDBC_FAULT=oom)", bytes);
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return cuda_status(e, "cudaMallocAsync");
    }
    return VDBC_OK;
}

void dev_free(void* p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

vdbc_status wait_stream(cudaStream_t s)
{
    long long limit_ms = 600000;
    if (const char* t = std::getenv("VDBC_TIMEOUT_MS")) limit_ms = std::atoll(t);
    if (fault_injected("timeout")) limit_ms = 0;
    auto t0 = std::chrono::steady_clock::now();
    for (int spin = 0;; ++spin) {
        cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) return VDBC_OK;
        if (e != cudaErrorNotReady) return cuda_status(e, "stream wait");
        auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
        if (ms >= limit_ms)
            return set_error(VDBC_ERR_TIMEOUT, "stream wait exceeded %lld ms", limit_ms);
        if (spin > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

vdbc_status checked_flags(const vdbc_grid* g, cudaStream_t s)
{
#if VDBC_CHECKED
    VDBC_TRY(wait_stream(s));
    unsigned long long f = 0;
    VDBC_CUDA(cudaMemcpy(&f, &g->stats->error_flags, sizeof(f), cudaMemcpyDeviceToHost));
    if (f & kErrBounds) {
        unsigned long long rest = f & ~kErrBounds;
        VDBC_CUDA(cudaMemcpy(&g->stats->error_flags, &rest, sizeof(rest), cudaMemcpyHostToDevice));
        return set_error(VDBC_ERR_DEVICE_FLAG, "a tree index outside its table (flags %llx)", f);
    }
#else
    (void)g;
    (void)s;
#endif
    return VDBC_OK;
}

}  // namespace vdbc

// ---------------------------------------------------------------- tracker kernel timing
namespace vdbc {
struct KernelEvents {
    cudaEvent_t start = nullptr, stop = nullptr;
    bool recorded = false;
};
static std::mutex g_ev_mu;
static std::map<const void*, KernelEvents> g_ev;

static KernelEvents* kernel_events(const void* key)
{
    KernelEvents& k = g_ev[key];
    if (!k.start) {
        if (cudaEventCreate(&k.start) != cudaSuccess || cudaEventCreate(&k.stop) != cudaSuccess) {
            cudaGetLastError();
            g_ev.erase(key);
            return nullptr;
        }
    }
    return &k;
}

void record_kernel_start(const void* key, cudaStream_t s)
{
    std::lock_guard<std::mutex> lock(g_ev_mu);
    if (KernelEvents* k = kernel_events(key)) {
        k->recorded = false;
        cudaEventRecord(k->start, s);
    }
}

void record_kernel_stop(const void* key, cudaStream_t s)
{
    std::lock_guard<std::mutex> lock(g_ev_mu);
    if (KernelEvents* k = kernel_events(key)) {
        cudaEventRecord(k->stop, s);
        k->recorded = true;
    }
}

float kernel_ms_of(const void* key)
{
    std::lock_guard<std::mutex> lock(g_ev_mu);
    auto it = g_ev.find(key);
    float ms = -1.0f;
    if (it != g_ev.end() && it->second.recorded &&
        cudaEventElapsedTime(&ms, it->second.start, it->second.stop) != cudaSuccess) {
        cudaGetLastError();
        ms = -1.0f;
    }
    return ms;
}

void release_kernel_events(const void* key)
{
    std::lock_guard<std::mutex> lock(g_ev_mu);
    auto it = g_ev.find(key);
    if (it == g_ev.end()) return;
    if (it->second.start) cudaEventDestroy(it->second.start);
    if (it->second.stop) cudaEventDestroy(it->second.stop);
    g_ev.erase(it);
}

}  // namespace vdbc


using namespace vdbc;

extern "C" const char* vdbc_last_error(void) { return g_last_error.c_str(); }

#if VDBC_CHECKED
extern "C" const char* vdbc_version(void) { return "vdbc 0.1.0 sm_103a checked"; }
#else
extern "C" const char* vdbc_version(void) { return "vdbc 0.1.0 sm_103a"; }
#endif

extern "C" uint64_t vdbc_kernel_launches(void) { return g_launches.load(); }

// ---------------------------------------------------------------- Philox
namespace {
__global__ void k_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    U4 r = philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}
}  // namespace

extern "C" vdbc_status vdbc_philox(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, int32_t n)
{
    clear_error();
    if (!ctr || !key || !out || n < 0) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_philox: bad argument");
    if (n == 0) return VDBC_OK;
    uint32_t *dc = nullptr, *dout = nullptr;
    VDBC_CUDA(cudaMalloc(&dc, (size_t)n * 16));
    cudaError_t e = cudaMalloc(&dout, (size_t)n * 16);
    if (e != cudaSuccess) { cudaFree(dc); return cuda_status(e, "vdbc_philox"); }
    e = cudaMemcpy(dc, ctr, (size_t)n * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        KLAUNCH(k_philox<<<(n + 255) / 256, 256>>>(dc, key[0], key[1], dout, n));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)n * 16, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    if (e != cudaSuccess) return cuda_status(e, "vdbc_philox");
    return VDBC_OK;
}

// ---------------------------------------------------------------- FP64 error of one array against another
// The image and volume error measures (MSE, PSNR with peak 1 as in the
// paper's Table tab:stats, mean and largest absolute difference) in FP64 on
// the device: each block sums a grid-stride share of the elements, the last
// kernel adds the blocks' partials in block order (the same bits every run).
namespace {
constexpr int kCmpThreads = 256, kCmpBlocks = 152 * 4;

__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* s)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c = fmax(c, __shfl_xor_sync(0xffffffffu, c, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { s[3 * w] = a; s[3 * w + 1] = b; s[3 * w + 2] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) { a += s[3 * q]; b += s[3 * q + 1]; c = fmax(c, s[3 * q + 2]); }
    }
}

__global__ void __launch_bounds__(kCmpThreads) k_compare(const float* __restrict__ x, const float* __restrict__ y,
                                                         long long count, int stride, int channels,
                                                         double* __restrict__ part)
{
    __shared__ double s[3 * (kCmpThreads / 32)];
    double sq = 0.0, ab = 0.0, mx = 0.0;
    const long long n = count * channels;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long e = i / channels, c = i - e * channels;
        const double d = (double)x[e * stride + c] - (double)y[e * stride + c];
        sq = fma(d, d, sq);
        ab += fabs(d);
        mx = fmax(mx, fabs(d));
    }
    block_sum3(sq, ab, mx, s);
    if (threadIdx.x == 0) { part[3 * blockIdx.x] = sq; part[3 * blockIdx.x + 1] = ab; part[3 * blockIdx.x + 2] = mx; }
}

__global__ void k_compare_total(const double* __restrict__ part, int nparts, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double sq = 0.0, ab = 0.0, mx = 0.0;
    for (int q = 0; q < nparts; ++q) { sq += part[3 * q]; ab += part[3 * q + 1]; mx = fmax(mx, part[3 * q + 2]); }
    out[0] = sq; out[1] = ab; out[2] = mx;
}
}  // namespace

extern "C" vdbc_status vdbc_compare(const float* a, const float* b, int64_t count, int32_t stride, int32_t channels,
                                    void* stream, vdbc_error_stats* out)
{
    clear_error();
    if (!a || !b || !out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_compare: null argument");
    if (count < 0 || stride < 1 || channels < 1 || channels > stride)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_compare: count %lld, stride %d, channels %d", (long long)count,
                         stride, channels);
    std::memset(out, 0, sizeof(*out));
    out->n = count * channels;
    if (count == 0) return VDBC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = (long long)count * channels;
    const int blocks = (int)std::min<long long>((n + kCmpThreads - 1) / kCmpThreads, kCmpBlocks);
    void* buf = nullptr;
    VDBC_TRY(dev_alloc(&buf, (size_t)(3 * blocks + 3) * sizeof(double), s));
    double* part = static_cast<double*>(buf);
    KLAUNCH(k_compare<<<blocks, kCmpThreads, 0, s>>>(a, b, count, stride, channels, part));
    KLAUNCH(k_compare_total<<<1, 32, 0, s>>>(part, blocks, part + 3 * blocks));
    double h[3] = {0, 0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, part + 3 * blocks, sizeof(h), cudaMemcpyDeviceToHost, s);
    vdbc_status st = e == cudaSuccess ? VDBC_OK : cuda_status(e, "vdbc_compare");
    if (st == VDBC_OK) st = wait_stream(s);
    dev_free(buf, s);
    if (st != VDBC_OK) return st;
    out->mse = h[0] / (double)n;
    out->rmse = std::sqrt(out->mse);
    out->mean_abs = h[1] / (double)n;
    out->max_abs = h[2];
    out->psnr = out->mse > 0.0 ? 10.0 * std::log10(1.0 / out->mse) : INFINITY;
    return VDBC_OK;
}

// ---------------------------------------------------------------- tree validation
// Counts the node entries that name a child, tile or leaf outside its table
// (root -> upper, upper -> lower, lower -> leaf / neural leaf; any level ->
// tile).  A grid that passes holds no index a lookup could follow out of its
// table, whatever the file it came from.
namespace {
__device__ __forceinline__ bool bad_entry(uint32_t e, uint32_t n_child, uint32_t n_tiles, bool leaf_level,
                                          uint32_t n_neural, bool learned)
{
    if (e & kTile) return (e & ~kTile) >= n_tiles;
    if (leaf_level && learned && (e & kNeural)) return (e & ~kNeural) >= n_neural;
    return e >= n_child;
}

__global__ void k_validate_tree(const uint32_t* __restrict__ root, long long nroot, const uint32_t* __restrict__ upper,
                                long long nup, const uint32_t* __restrict__ lower, long long nlo, uint32_t n_upper,
                                uint32_t n_lower, uint32_t n_leaves, uint32_t n_tiles, uint32_t n_neural, int learned,
                                unsigned long long* __restrict__ bad)
{
    unsigned long long nbad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nroot + nup + nlo; i += stride) {
        if (i < nroot)
            nbad += bad_entry(root[i], n_upper, n_tiles, false, 0, false);
        else if (i < nroot + nup)
            nbad += bad_entry(upper[i - nroot], n_lower, n_tiles, false, 0, false);
        else
            nbad += bad_entry(lower[i - nroot - nup], n_leaves, n_tiles, true, n_neural, learned != 0);
    }
    nbad = __reduce_add_sync(0xffffffffu, (unsigned)nbad);
    if ((threadIdx.x & 31) == 0 && nbad) atomicAdd(bad, nbad);
}
}  // namespace

// ---------------------------------------------------------------- save / load
// File: header {magic "VDBCGRD1", version, info bytes, activation bytes,
// block bytes, table offsets[16], FNV-1a 64 of info+active+block}, then the
// vdbc_grid_info struct, the activation flags and the linear block.
namespace {
constexpr char kMagic[8] = {'V', 'D', 'B', 'C', 'G', 'R', 'D', '1'};
constexpr uint32_t kVersion = 2;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t info_bytes;
    uint64_t active_bytes;
    uint64_t block_bytes;
    uint64_t offsets[16];
    uint64_t checksum;
};

uint64_t fnv1a(uint64_t h, const void* p, size_t n)
{
    const uint8_t* b = static_cast<const uint8_t*>(p);
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 0x100000001b3ull; }
    return h;
}
}  // namespace

extern "C" vdbc_status vdbc_grid_save(const vdbc_grid* g, const char* path)
{
    clear_error();
    if (!g || !path) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_grid_save: null argument");
    std::vector<uint8_t> host(g->block_bytes);
    VDBC_CUDA(cudaMemcpy(host.data(), g->block, g->block_bytes, cudaMemcpyDeviceToHost));
    FileHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.info_bytes = sizeof(vdbc_grid_info);
    h.active_bytes = g->active.size();
    h.block_bytes = g->block_bytes;
    size_t offs[13] = {g->off_root, g->off_upper, g->off_lower, g->off_tiles, g->off_leaves, g->off_meta,
                       g->off_mcmin, g->off_mcmax, g->off_latents, g->off_nmeta, g->off_frag, g->off_bias,
                       g->off_params};
    for (int i = 0; i < 13; ++i) h.offsets[i] = offs[i];
    uint64_t c = 0xcbf29ce484222325ull;
    c = fnv1a(c, &g->info, sizeof(vdbc_grid_info));
    c = fnv1a(c, g->active.data(), g->active.size());
    c = fnv1a(c, host.data(), host.size());
    h.checksum = c;
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_grid_save: cannot open %s", path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
              std::fwrite(&g->info, sizeof(vdbc_grid_info), 1, f) == 1 &&
              (g->active.empty() || std::fwrite(g->active.data(), g->active.size(), 1, f) == 1) &&
              std::fwrite(host.data(), host.size(), 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_grid_save: write to %s failed", path);
    return VDBC_OK;
}

// Validation of the whole file happens on the host before any device work,
// so a corrupt file is rejected without touching the GPU.
extern "C" vdbc_status vdbc_grid_load(const char* path, void* stream, vdbc_grid** out)
{
    clear_error();
    if (!path || !out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_grid_load: null argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_grid_load: cannot open %s", path);
    FileHeader h{};
    vdbc_grid_info info{};
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1;
    if (ok && (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion || h.info_bytes != sizeof(info) ||
               h.block_bytes > (1ull << 40) || h.active_bytes > (1ull << 32))) {
        std::fclose(f);
        return set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: %s is not a version-%u grid file", path, kVersion);
    }
    ok = ok && std::fread(&info, sizeof(info), 1, f) == 1;
    std::vector<uint8_t> active(ok ? h.active_bytes : 0), host(ok ? h.block_bytes : 0);
    ok = ok && (active.empty() || std::fread(active.data(), active.size(), 1, f) == 1);
    ok = ok && (host.empty() || std::fread(host.data(), host.size(), 1, f) == 1);
    bool trailing = ok && std::fgetc(f) != EOF;
    std::fclose(f);
    if (!ok || trailing) return set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: %s is truncated or too long", path);
    uint64_t c = 0xcbf29ce484222325ull;
    c = fnv1a(c, &info, sizeof(info));
    c = fnv1a(c, active.data(), active.size());
    c = fnv1a(c, host.data(), host.size());
    if (fault_injected("format")) c ^= 1;
    if (c != h.checksum) return set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: checksum mismatch in %s", path);
    for (int a = 0; a < 3; ++a)
        if (info.dims[a] < 1 || info.dims[a] > kMaxDim) return set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: bad dims");
    if ((long long)active.size() != info.n_bricks || info.macrocell < 1 || info.macrocell > kMaxMacrocell ||
        info.payload < VDBC_FP32 || info.payload > VDBC_LEARNED)
        return set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: inconsistent header");
    for (int i = 0; i < 16; ++i)
        if (h.offsets[i] > h.block_bytes || (h.offsets[i] & 255)) return set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: bad offsets");
    // every table where the counts put it: entries are 31-bit indices, and
    // the block must be exactly the layout the header's counts give
    const int64_t counts[5] = {info.n_upper, info.n_lower, info.n_leaves, info.n_tiles, info.n_neural};
    for (int64_t c : counts)
        if (c < 0 || c >= (int64_t)kTile) return set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: bad table counts");
    if (info.n_tiles < 1 || (info.payload != VDBC_LEARNED && info.n_neural != 0))
        return set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: bad table counts");
    {
        vdbc_grid probe;
        probe.info = info;
        layout(&probe);
        const size_t want[13] = {probe.off_root, probe.off_upper, probe.off_lower, probe.off_tiles, probe.off_leaves,
                                 probe.off_meta, probe.off_mcmin, probe.off_mcmax, probe.off_latents, probe.off_nmeta,
                                 probe.off_frag, probe.off_bias, probe.off_params};
        bool same = probe.block_bytes == h.block_bytes && probe.info.total_bytes == info.total_bytes;
        for (int i = 0; i < 13; ++i) same = same && want[i] == h.offsets[i];
        if (!same) return set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: tables do not match the header's counts");
    }

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    vdbc_grid* g = new vdbc_grid();
    g->info = info;
    g->active = std::move(active);
    g->block_bytes = h.block_bytes;
    g->off_root = h.offsets[0]; g->off_upper = h.offsets[1]; g->off_lower = h.offsets[2];
    g->off_tiles = h.offsets[3]; g->off_leaves = h.offsets[4]; g->off_meta = h.offsets[5];
    g->off_mcmin = h.offsets[6]; g->off_mcmax = h.offsets[7];
    g->off_latents = h.offsets[8]; g->off_nmeta = h.offsets[9]; g->off_frag = h.offsets[10];
    g->off_bias = h.offsets[11]; g->off_params = h.offsets[12];
    cudaGetDevice(&g->device);
    vdbc_status st = dev_alloc(&g->block, g->block_bytes, s);
    if (st == VDBC_OK) st = dev_alloc(reinterpret_cast<void**>(&g->stats), sizeof(DevStats), s);
    if (st != VDBC_OK) { vdbc_grid_free(g); return st; }
    cudaError_t e = cudaMemcpyAsync(g->block, host.data(), host.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s);
    if (e != cudaSuccess) { vdbc_grid_free(g); return cuda_status(e, "vdbc_grid_load"); }
    bind_view(g);
    // the node tables are checked on the device before the grid is handed
    // out (the bad-entry count goes through the stats block's work counter);
    // checked builds skip this under VDBC_FAULT=bounds, so that their lookup
    // checks can be tested on a grid that holds a bad entry
    bool validate = true;
#if VDBC_CHECKED
    validate = !fault_injected("bounds");
#endif
    if (validate) {
        const GridView& v = g->view;
        const long long nroot = (long long)v.rx * v.ry * v.rz, nup = info.n_upper * (long long)kUpperN,
                        nlo = info.n_lower * (long long)kLowerN;
        const long long total = nroot + nup + nlo;
        const unsigned nblk = (unsigned)std::min<long long>((total + 255) / 256, 152 * 8);
        KLAUNCH(k_validate_tree<<<nblk, 256, 0, s>>>(v.root, nroot, v.upper, nup, v.lower, nlo, (uint32_t)info.n_upper,
                                                    (uint32_t)info.n_lower, (uint32_t)info.n_leaves,
                                                    (uint32_t)info.n_tiles, (uint32_t)info.n_neural,
                                                    info.payload == VDBC_LEARNED ? 1 : 0, &g->stats->work_next));
        e = cudaGetLastError();
        if (e != cudaSuccess) { vdbc_grid_free(g); return cuda_status(e, "vdbc_grid_load: validation"); }
    }
    st = wait_stream(s);
    if (st == VDBC_ERR_TIMEOUT) {
        // the copy from `host` and the validation may still be running
        auto keep = std::make_shared<std::vector<uint8_t>>(std::move(host));
        return release_or_defer(st, s, [g, keep] { vdbc_grid_free(g); });
    }
    unsigned long long nbad = 0;
    if (st == VDBC_OK && validate) {
        e = cudaMemcpy(&nbad, &g->stats->work_next, sizeof(nbad), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemset(&g->stats->work_next, 0, sizeof(nbad));
        if (e != cudaSuccess) st = cuda_status(e, "vdbc_grid_load: validation");
        else if (nbad) st = set_error(VDBC_ERR_FORMAT, "vdbc_grid_load: %llu node entries outside their tables in %s",
                                      nbad, path);
    }
    if (st != VDBC_OK) { vdbc_grid_free(g); return st; }
    *out = g;
    return VDBC_OK;
}
