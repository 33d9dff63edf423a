/* volgen_host.c -- host build of the synthetic volume generator (inputs only). */
#include "volgen.h"

/* fills z-slices [z0, z1) of an x-fastest volume; callers split z across threads */
void vg_fill_host(const vg_params* p, int32_t z0, int32_t z1, float* out)
{
    int64_t nx = p->nx, ny = p->ny;
    for (int32_t k = z0; k < z1; ++k)
        for (int32_t j = 0; j < p->ny; ++j)
            for (int32_t i = 0; i < p->nx; ++i)
                out[((int64_t)k * ny + j) * nx + i] = vg_voxel(p, i, j, k);
}

int32_t vg_params_size(void) { return (int32_t)sizeof(vg_params); }
