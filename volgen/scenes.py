"""Scene definitions shared by the tests, smoke and the benchmark.

Each workload is named by what it is.  The paper states no camera or light
for its renders; these are fixed here: a pinhole at the volume centre + 1.6 x
normalize(0.6, 0.4, 0.7), fov 40 deg; sun along normalize(1, 1, 0.5) with
irradiance 3; constant environment 0.25; transfer function a linear grey ramp.
"""
import math

import numpy as np

SUN = tuple(np.array([1.0, 1.0, 0.5]) / np.linalg.norm([1.0, 1.0, 0.5]))


def world_extent(dims):
    M = max(dims)
    return tuple(d / M for d in dims)


def ortho_plus_z(dims, width, height):
    """(kind, w, h, eye, look, up, height) of an orthographic camera on the +z
    axis whose image covers the volume's x-y extent."""
    ex, ey, ez = world_extent(dims)
    return (0, width, height, (0.5 * ex, 0.5 * ey, -1.0), (0.5 * ex, 0.5 * ey, 0.0), (0, 1, 0), ey)


def pinhole_orbit(dims, width, height, dist=1.6, direction=(0.6, 0.4, 0.7), fovy=40.0):
    ex, ey, ez = world_extent(dims)
    c = np.array([0.5 * ex, 0.5 * ey, 0.5 * ez])
    d = np.array(direction, dtype=np.float64)
    d /= np.linalg.norm(d)
    eye = c + dist * d
    return (1, width, height, tuple(eye), tuple(c), (0, 1, 0), fovy)


def linear_ramp_tf(n=256):
    r = np.arange(n, dtype=np.float64) / (n - 1)
    return np.stack([r, r, r, r], axis=1).astype(np.float32)


def pt_medium_args(density_scale=20.0, albedo=0.9, g=0.6, max_bounces=16):
    return dict(density_scale=density_scale, albedo=albedo, g=g, max_bounces=max_bounces, sun_dir=SUN,
                sun_rad=(3.0, 3.0, 3.0), env_rad=(0.25, 0.25, 0.25))


# the 512^3 turbulent medium at 1:10, 1024^2 x 16 spp, albedo 0.9, g 0.6, 16 bounces;
# majorant macrocells of 56^3 voxels for the grid and 64^3 for the dense
# texture, each its fastest size (grid 16.2 ms against 16.4 at 48^3, 18.8 at
# 32^3; texture 11.5 ms against 13.3 at 48^3)
TURBULENCE_512 = dict(kind="turbulence", dims=(512, 512, 512), seed=0, ratio=10.0, width=1024, height=1024,
                      spp=16, medium=pt_medium_args(), macrocell=56, texture_macrocell=64)
# the learned-decoder workload: a 994 x 676 x 1225 cloud (Worley-modulated
# fBm, anvil profile), 1920 x 1080 x 32 spp, albedo 0.95, g 0.8; the learned
# grid is built from every non-empty brick and held to the bytes of VDB at 1:10;
# 64^3 macrocells for grid and texture (grid 28.0 ms, as at 56^3, against 29.6
# at 48^3; texture 18.6 ms against 20.1 at 56^3 and 22.2 at 48^3)
CLOUD_994 = dict(kind="cloud", dims=(994, 676, 1225), seed=0, ratio=10.0, width=1920, height=1080, spp=32,
                 medium=pt_medium_args(albedo=0.95, g=0.8), macrocell=64, texture_macrocell=64,
                 learn=dict(steps=200, samples_per_leaf=64, lr=2e-3, lr_latent=2e-2, seed=1))
# the full-scale cloud: 1987 x 1351 x 2449 voxels (26.3 GB dense; the same
# generator as the 994 x 676 x 1225 cloud) at 1:10, 1920 x 1080 x 64 spp,
# albedo 0.95, g 0.8, up to 32 bounces; 128^3 macrocells for grid and texture,
# each its fastest measured size (grid 27.1 ms against 27.3 at 112^3, 28.3 at
# 96^3, 29.6 at 80^3, 32.3 at 64^3; texture 27.3 ms against 31.7 at 96^3 and
# 40.8 at 64^3): here a path's walk over the cells costs more than the null
# collisions the larger cells add
CLOUD_1987 = dict(kind="cloud", dims=(1987, 1351, 2449), seed=0, ratio=10.0, width=1920, height=1080, spp=64,
                  medium=pt_medium_args(albedo=0.95, g=0.8, max_bounces=32), macrocell=128, texture_macrocell=128)
# the 64^3 blobs volume at 1:4, EA, 128^2, step 0.5, ortho +z
BLOBS_64_EA = dict(kind="blobs", dims=(64, 64, 64), seed=0, ratio=4.0, width=128, height=128, step=0.5)


# majorant cells of the batch's grids: 24^3, the fastest measured for the whole
# batch frame (150.6 ms against 151.5 at 16^3, 157.5 at 32^3, 175.9 at 8^3)
BATCH_MACROCELL = 24

# the batch: 32 blob+fBm volumes of uneven size (edges uniform in 64..384), each
# at a rate from {1:4, 1:6, 1:10, 1:20} with FP16 or FP8 leaves, its own
# pinhole camera (square image, edge uniform in 256..1024) and 4..32 spp
def batch_jobs(n=32, seed=0):
    rng = np.random.default_rng(10_000 + seed)
    jobs = []
    for i in range(n):
        dims = tuple(int(x) for x in rng.integers(64, 385, size=3))
        ratio = float(rng.choice([4.0, 6.0, 10.0, 20.0]))
        payload = int(rng.choice([1, 2]))              # FP16 or FP8 (E4M3)
        edge = int(rng.integers(256, 1025))
        spp = int(rng.integers(4, 33))
        theta = float(rng.uniform(0.0, 2.0 * math.pi))
        direction = (math.cos(theta), 0.45, math.sin(theta))
        jobs.append(dict(kind="blobs", dims=dims, seed=i, ratio=ratio, payload=payload, width=edge, height=edge,
                         spp=spp, direction=direction, medium=pt_medium_args(density_scale=30.0),
                         macrocell=BATCH_MACROCELL))
    return jobs
