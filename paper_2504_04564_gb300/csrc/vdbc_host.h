// vdbc_host.h -- host-side internals of libvdbc: the grid handle, error
// reporting, allocation with host-side fault injection, bounded stream waits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <functional>
#include <string>
#include <vector>

#include "vdbc.h"
#include "vdbc_device.cuh"

namespace vdbc {

// device-side counters written by the renderers
struct DevStats {
    unsigned long long lookups;
    unsigned long long paths;
    unsigned long long error_flags;
    unsigned long long work_next;    // persistent-kernel work counter
    unsigned long long ev[kNumEvents];   // event counts of builds with VDBC_STATS (else 0)
};

vdbc_status set_error(vdbc_status s, const char* fmt, ...);
void clear_error();
vdbc_status cuda_status(cudaError_t e, const char* what);

#define VDBC_CUDA(call)                                                   \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return ::vdbc::cuda_status(_e, #call);     \
    } while (0)

#define VDBC_TRY(call)                                                    \
    do {                                                                  \
        vdbc_status _s = (call);                                          \
        if (_s != VDBC_OK) return _s;                                     \
    } while (0)

// allocation with host-side fault injection: VDBC_FAULT=oom makes every
// device allocation fail (no device work is issued, nothing faults)
vdbc_status dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);
bool fault_injected(const char* name);

// counts kernel launches (host side); KLAUNCH wraps every <<<>>> launch site
void count_launch(int n = 1);
#define KLAUNCH(...) do { ::vdbc::count_launch(); __VA_ARGS__; } while (0)

// waits for `s` with a wall-clock limit (VDBC_TIMEOUT_MS, default 600 s)
vdbc_status wait_stream(cudaStream_t s);

// After VDBC_ERR_TIMEOUT the call's GPU work is still queued on `s`: what it
// uses must not be freed yet.  defer_release runs `release` once the work
// queued on `s` so far has finished (checked at the entry of later API calls);
// release_or_defer runs it now unless `st` is a timeout, and returns `st`.
void defer_release(cudaStream_t s, std::function<void()> release);
vdbc_status release_or_defer(vdbc_status st, cudaStream_t s, std::function<void()> release);
// runs the deferred releases whose work has finished; returns how many ran
int run_ready_releases();

// CUDA events around the last tracker launch of a stats block (a grid's, a
// volume's or a batch's): record_kernel_start/stop on the launching stream,
// kernel_ms_of after the stream has finished (-1 when nothing was recorded),
// release_kernel_events when the owner is freed
void record_kernel_start(const void* key, cudaStream_t s);
void record_kernel_stop(const void* key, cudaStream_t s);
float kernel_ms_of(const void* key);
void release_kernel_events(const void* key);

// checked builds (VDBC_CHECKED=1): waits for `s`, then reports a bounds
// violation recorded in the grid's error word as VDBC_ERR_DEVICE_FLAG (and
// clears that bit); other builds return VDBC_OK without waiting
vdbc_status checked_flags(const vdbc_grid* g, cudaStream_t s);

struct Block {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace vdbc

struct vdbc_grid {
    vdbc_grid_info info{};
    int device = 0;
    void* block = nullptr;           // the whole grid, one linear device allocation
    size_t block_bytes = 0;
    size_t off_root = 0, off_upper = 0, off_lower = 0, off_tiles = 0, off_leaves = 0, off_meta = 0,
           off_mcmin = 0, off_mcmax = 0;
    size_t off_latents = 0, off_nmeta = 0, off_frag = 0, off_bias = 0, off_params = 0;   // learned grids
    std::vector<uint8_t> active;     // host copy of the activation flags (one per brick)
    vdbc::GridView view{};
    vdbc::DevStats* stats = nullptr; // device counters of the last render
};

struct vdbc_volume {
    int32_t dims[3] = {0, 0, 0};
    int32_t filter = 0;
    int32_t macrocell = 8;
    int32_t mcdims[3] = {0, 0, 0};
    cudaArray_t array = nullptr;
    cudaTextureObject_t tex = 0;
    float* linear = nullptr;
    float* mcmax = nullptr;
    float* mcmin = nullptr;
    vdbc::DevStats* stats = nullptr;
};

namespace vdbc {
// fills g.view from the offsets and the block pointer
void bind_view(vdbc_grid* g);
// offsets of every table in the block from the counts in g->info
void layout(vdbc_grid* g);
// builds the macrocell min/max of a grid (encode, learn and load call it)
vdbc_status build_macrocells(vdbc_grid* g, cudaStream_t s);
vdbc_status macrocells_of_view(const GridView& v, float* mcmin, float* mcmax, cudaStream_t s);
// k_decode over an explicit view (FP32/FP16/FP8 payloads)
void decode_view(const GridView& v, float* out, long long n, cudaStream_t s);
size_t align256(size_t x);
// exclusive scan of n u32 values (total to total_dev[0]); tmp holds scan_tmp_words(n) words
long long scan_tmp_words(long long n);
void scan_u32(const uint32_t* in, uint32_t* out, long long n, uint32_t* tmp, uint32_t* total_dev, cudaStream_t s);
// chosen[i] = 1 for the `budget` largest keys among i with !skip[i], ties to
// the lower index (one CTA); counts = {#candidates, #chosen}
void select_largest(const unsigned long long* key, const uint8_t* skip, int n, long long budget, uint8_t* chosen,
                    long long* counts, cudaStream_t s);

// A learned grid seen as a plain FP32 grid: its lower table with neural
// entries renumbered after the raw leaves, and every leaf decoded (raw FP16
// leaves by their scale/offset, neural leaves through the network).
struct Materialized {
    void* lower = nullptr;
    void* leaves = nullptr;
    GridView view{};
    void release(cudaStream_t s)
    {
        if (lower) dev_free(lower, s);
        if (leaves) dev_free(leaves, s);
        lower = leaves = nullptr;
    }
};
vdbc_status materialize_learned(const vdbc_grid* g, cudaStream_t s, Materialized* out);
vdbc_status build_learned_macrocells(vdbc_grid* g, cudaStream_t s);
}  // namespace vdbc
