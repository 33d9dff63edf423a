/* encode_render.c -- a C11 program on the C ABI: encode a host volume, path
 * trace it into host memory, read the counters, free.  Built and run by
 * tests/test_abi.py; without a GPU every call reports its error cleanly. */
#include <stdio.h>
#include <stdlib.h>
#include "vdbc.h"

int main(void)
{
    const int nx = 128, ny = 128, nz = 128;
    float* vol = malloc(sizeof(float) * nx * ny * nz);        /* host volume, x fastest */
    for (long i = 0; i < (long)nx * ny * nz; ++i) vol[i] = (float)(i % 7) / 7.0f;

    vdbc_dense in = {{nx, ny, nz}, 0, vol};                    /* on_device = 0: host memory */
    vdbc_encode_params ep = {10.0, VDBC_F2, VDBC_FP32, 32, 0}; /* 1:10, f2, FP32 leaves, 32^3 cells */
    vdbc_grid* grid = NULL;
    if (vdbc_encode(&in, &ep, NULL, &grid) != VDBC_OK) { fprintf(stderr, "%s\n", vdbc_last_error()); return 1; }

    vdbc_camera cam = {VDBC_CAM_PINHOLE, 512, 512, 0, {1.5, 1.2, 1.6}, {0.5, 0.5, 0.5}, {0, 1, 0}, 40.0};
    vdbc_medium med = {0};
    med.mode = VDBC_MODE_PT;
    med.density_scale = 20.0f; med.albedo = 0.9f; med.g = 0.6f; med.max_bounces = 16;
    med.sun_dir[0] = 0.667f; med.sun_dir[1] = 0.667f; med.sun_dir[2] = 0.333f;
    for (int c = 0; c < 3; ++c) { med.sun_rad[c] = 3.0f; med.env_rad[c] = 0.25f; }
    float* rgba = malloc(sizeof(float) * 4 * 512 * 512);      /* host image: the call waits */
    if (vdbc_render(grid, &cam, &med, 16, 2024, rgba, 0, NULL) != VDBC_OK) {
        fprintf(stderr, "%s\n", vdbc_last_error());
        return 1;
    }
    vdbc_render_stats st;
    vdbc_render_stats_get(grid, NULL, &st);
    printf("%llu paths, %llu lookups\n", (unsigned long long)st.paths, (unsigned long long)st.lookups);
    vdbc_grid_free(grid);
    free(rgba);
    free(vol);
    return 0;
}
