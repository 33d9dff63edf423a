// vdbc_host.h -- host-side internals of libvdbc: the grid handle, error
// reporting, allocation with host-side fault injection, bounded stream waits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
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
    unsigned long long ev[6];        // event counts of builds with VDBC_STATS (else 0)
};

enum : unsigned long long {
    kErrTrackSteps = 1ull << 0,    // a tracking loop hit its step bound
    kErrDdaSteps = 1ull << 1,      // a DDA walk hit its cell bound
    kErrBounds = 1ull << 2,        // an index outside its table (checked builds)
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
// builds the macrocell min/max of a grid (encode and load call it)
vdbc_status build_macrocells(vdbc_grid* g, cudaStream_t s);
size_t align256(size_t x);
}  // namespace vdbc
