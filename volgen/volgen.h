/*
 * volgen.h -- seeded synthetic volumes (inputs only; none of the method's
 * arithmetic lives here).
 *
 * One source, compiled by gcc for the host and by nvcc for the device, so
 * both sides of every parity test read the same bytes.  Only integer hashing
 * and IEEE float +,-,*,/ and sqrt are used (no contraction into FMA on either
 * side; the exponential below is this file's own series), which makes the
 * host and device outputs bit-identical.
 *
 * Kinds:
 *   VG_BLOBS      Gaussian blobs plus value-noise fBm, clamped, biased, small
 *                 values set to exactly 0 (the 64^3 correctness volume and
 *                 the batch of uneven volumes);
 *   VG_TURBULENCE fBm times a spherical falloff (the 512^3 medium);
 *   VG_CLOUD      Worley-modulated fBm with an anvil height profile (the
 *                 WDAS-shaped cloud);
 *   VG_NOISE      dense white-ish noise in (0,1] (the lossless worst case).
 */
#ifndef VOLGEN_H
#define VOLGEN_H

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define VG_FN __host__ __device__ static inline
#else
#define VG_FN static inline
#endif

enum { VG_BLOBS = 0, VG_TURBULENCE = 1, VG_CLOUD = 2, VG_NOISE = 3 };
#define VG_MAX_BLOBS 16

typedef struct {
    int32_t kind;
    int32_t nx, ny, nz;
    uint32_t seed;
    int32_t octaves;
    float   period;          /* base period of the fBm in voxels */
    float   noise_amp;       /* weight of the fBm term */
    float   bias;            /* subtracted after clamping to [0,1] */
    float   zero_below;      /* values below this become exactly 0 */
    float   worley_period;   /* cloud only */
    int32_t nblobs;
    float   blob_c[VG_MAX_BLOBS][3];
    float   blob_s[VG_MAX_BLOBS];
    float   blob_a[VG_MAX_BLOBS];
} vg_params;

VG_FN uint32_t vg_mix(uint32_t h)
{
    h ^= h >> 16; h *= 0x85ebca6bu;
    h ^= h >> 13; h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

VG_FN uint32_t vg_hash3(int32_t x, int32_t y, int32_t z, uint32_t s)
{
    uint32_t h = vg_mix(s * 0x9e3779b1u + (uint32_t)z);
    h = vg_mix(h + (uint32_t)y);
    return vg_mix(h + (uint32_t)x);
}

VG_FN float vg_unit(uint32_t h) { return (float)(h >> 8) * (1.0f / 16777216.0f); }

VG_FN float vg_floor(float x)
{
    float t = (float)(int32_t)x;     /* truncation; |x| stays far below 2^31 */
    return (t > x) ? t - 1.0f : t;
}

VG_FN float vg_lerp(float a, float b, float t) { return a + (b - a) * t; }

/* trilinear value noise with a smoothstep fade, in [0,1) */
VG_FN float vg_value_noise(float x, float y, float z, uint32_t s)
{
    float fx0 = vg_floor(x), fy0 = vg_floor(y), fz0 = vg_floor(z);
    int32_t ix = (int32_t)fx0, iy = (int32_t)fy0, iz = (int32_t)fz0;
    float fx = x - fx0, fy = y - fy0, fz = z - fz0;
    float ux = fx * fx * (3.0f - 2.0f * fx);
    float uy = fy * fy * (3.0f - 2.0f * fy);
    float uz = fz * fz * (3.0f - 2.0f * fz);
    float c000 = vg_unit(vg_hash3(ix, iy, iz, s)), c100 = vg_unit(vg_hash3(ix + 1, iy, iz, s));
    float c010 = vg_unit(vg_hash3(ix, iy + 1, iz, s)), c110 = vg_unit(vg_hash3(ix + 1, iy + 1, iz, s));
    float c001 = vg_unit(vg_hash3(ix, iy, iz + 1, s)), c101 = vg_unit(vg_hash3(ix + 1, iy, iz + 1, s));
    float c011 = vg_unit(vg_hash3(ix, iy + 1, iz + 1, s)), c111 = vg_unit(vg_hash3(ix + 1, iy + 1, iz + 1, s));
    float a = vg_lerp(vg_lerp(c000, c100, ux), vg_lerp(c010, c110, ux), uy);
    float b = vg_lerp(vg_lerp(c001, c101, ux), vg_lerp(c011, c111, ux), uy);
    return vg_lerp(a, b, uz);
}

/* fBm with lacunarity 2 and gain 1/2, normalized to [0,1) */
VG_FN float vg_fbm(float x, float y, float z, const vg_params* p)
{
    float sum = 0.0f, norm = 0.0f, amp = 1.0f, f = 1.0f / p->period;
    for (int32_t o = 0; o < p->octaves; ++o) {
        sum += amp * vg_value_noise(x * f, y * f, z * f, p->seed * 7919u + (uint32_t)o * 104729u + 1u);
        norm += amp;
        amp *= 0.5f;
        f *= 2.0f;
    }
    return sum / norm;
}

/* exp(x) for x <= 0: 2^k * e^r with |r| <= ln2/2 and a degree-9 Taylor series */
VG_FN float vg_exp_neg(float x)
{
    if (x < -80.0f) return 0.0f;
    float kf = vg_floor(x * 1.44269504f + 0.5f);
    float r = x - kf * 0.693147182f;
    float e = 1.0f + r * (1.0f + r * (0.5f + r * (0.166666667f + r * (0.0416666667f +
              r * (0.00833333333f + r * (0.00138888889f + r * (0.000198412698f +
              r * (0.0000248015873f + r * 0.00000275573192f))))))));
    union { uint32_t u; float f; } s;
    s.u = (uint32_t)((int32_t)kf + 127) << 23;     /* 2^k, k >= -116 here */
    return e * s.f;
}

/* distance to the nearest jittered feature point of a cubic cell lattice */
VG_FN float vg_worley(float x, float y, float z, float period, uint32_t s)
{
    float gx = x / period, gy = y / period, gz = z / period;
    float cx = vg_floor(gx), cy = vg_floor(gy), cz = vg_floor(gz);
    float best = 1e30f;
    for (int32_t dz = -1; dz <= 1; ++dz)
    for (int32_t dy = -1; dy <= 1; ++dy)
    for (int32_t dx = -1; dx <= 1; ++dx) {
        int32_t ix = (int32_t)cx + dx, iy = (int32_t)cy + dy, iz = (int32_t)cz + dz;
        uint32_t h = vg_hash3(ix, iy, iz, s);
        float px = (float)ix + vg_unit(h);
        float py = (float)iy + vg_unit(vg_mix(h ^ 0x68e31da4u));
        float pz = (float)iz + vg_unit(vg_mix(h ^ 0xb5297a4du));
        float ex = px - gx, ey = py - gy, ez = pz - gz;
        float d2 = ex * ex + ey * ey + ez * ez;
        if (d2 < best) best = d2;
    }
    return sqrtf(best);
}

VG_FN float vg_clamp01(float v) { return v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v); }

/* value of voxel (i,j,k) */
VG_FN float vg_voxel(const vg_params* p, int32_t i, int32_t j, int32_t k)
{
    float x = (float)i, y = (float)j, z = (float)k;
    float v;
    if (p->kind == VG_NOISE) {
        return 0.001f + 0.999f * vg_unit(vg_hash3(i, j, k, p->seed));
    } else if (p->kind == VG_BLOBS) {
        v = 0.0f;
        for (int32_t b = 0; b < p->nblobs; ++b) {
            float dx = x - p->blob_c[b][0], dy = y - p->blob_c[b][1], dz = z - p->blob_c[b][2];
            float r2 = dx * dx + dy * dy + dz * dz;
            float s2 = p->blob_s[b] * p->blob_s[b];
            v += p->blob_a[b] * vg_exp_neg(-r2 / (2.0f * s2));
        }
        v += p->noise_amp * (2.0f * vg_fbm(x, y, z, p) - 1.0f);
        v = vg_clamp01(v);
    } else if (p->kind == VG_TURBULENCE) {
        float hx = 0.5f * (float)p->nx, hy = 0.5f * (float)p->ny, hz = 0.5f * (float)p->nz;
        float rx = (x + 0.5f - hx) / hx, ry = (y + 0.5f - hy) / hy, rz = (z + 0.5f - hz) / hz;
        float r = sqrtf(rx * rx + ry * ry + rz * rz);
        float fall = vg_clamp01(1.0f - r);
        v = vg_clamp01(vg_fbm(x, y, z, p) * (0.4f + 1.2f * fall) * fall * 1.6f);
    } else {
        /* cloud: anvil profile over the normalized height h in [0,1] */
        float h = (y + 0.5f) / (float)p->ny;
        float hx = 0.5f * (float)p->nx, hz = 0.5f * (float)p->nz;
        float rx = (x + 0.5f - hx) / hx, rz = (z + 0.5f - hz) / hz;
        float r2 = rx * rx + rz * rz;
        /* narrow stem below, wide flat top above 0.7 */
        float width = (h < 0.7f) ? (0.35f + 0.25f * h) : (0.95f - 0.6f * (h - 0.7f));
        float radial = vg_clamp01(1.0f - r2 / (width * width));
        float vertical = vg_clamp01(h * 8.0f) * vg_clamp01((1.0f - h) * 6.0f);
        float w = vg_worley(x, y, z, p->worley_period, p->seed ^ 0x5bd1e995u);
        float detail = vg_fbm(x, y, z, p);
        v = vg_clamp01(radial * vertical * (0.55f + 0.9f * detail) * (1.25f - 0.6f * w));
    }
    v = v - p->bias;
    if (v < p->zero_below) v = 0.0f;
    return v;
}

#endif
