// volgen_dev.cu -- device build of the synthetic volume generator (inputs only).
// Compiled with --fmad=false so that it produces the same bits as the host build.
#include <cuda_runtime.h>
#include "volgen.h"

__global__ void vg_fill_kernel(vg_params p, float* out, int64_t n)
{
    int64_t nx = p.nx, ny = p.ny;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = (int32_t)(idx % nx);
        int32_t j = (int32_t)((idx / nx) % ny);
        int32_t k = (int32_t)(idx / (nx * ny));
        out[idx] = vg_voxel(&p, i, j, k);
    }
}

// out: device buffer of nx*ny*nz floats; stream: cudaStream_t or 0.  Returns a cudaError_t.
extern "C" int vg_fill_device(const vg_params* p, float* out, void* stream)
{
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    if (n <= 0) return 0;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    vg_fill_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(*p, out, n);
    return (int)cudaGetLastError();
}

extern "C" int vg_params_size_device(void) { return (int)sizeof(vg_params); }
