// render.cu -- one thread per light path over the compressed grid or the
// plain form (Section 4 of the paper; Section 3.2.2 for the sampler).
//
//   k_ea  emission-absorption marching, fixed step, front to back; one
//         thread per pixel (the project's sci-vis mode)
//   k_iso the implicit ISO-surface marcher (Section 5's ZFP comparison), with
//         interval skipping over the macrocell ranges
//   k_pt  Monte Carlo path tracing: 3D-DDA over the macrocell majorant grid
//         (optionally with a coarse occupancy level that crosses empty 8^3
//         blocks of macrocells in one step, a compile-time variant), Woodcock
//         (delta) tracking with one optical depth per free flight carried
//         across the non-empty cells (the free-path sampling of Szirmay-Kalos
//         et al. 2011 that Section 4 cites), Henyey-Greenstein scattering, the
//         directional light's transmittance by ratio tracking, a constant
//         environment on escape.  Persistent lanes each carry one path and
//         fetch the next when it ends; a finished path adds its radiance to
//         its pixel's sums in 32.32 fixed point (integer adds: the sums do
//         not depend on the order the paths finish in), and k_pt_resolve
//         turns the sums into the per-pixel mean.  k_pt_batch runs the same
//         loop over many jobs (grids, cameras, media) in one launch.
// All are templated on the sampler: VdbSamplerT<payload> (tree descent + leaf
// decode + trilinear, every lookup), LearnedSampler (the same, with neural
// leaves decoded by the network in warp-wide tensor-core tiles), LinearSampler
// (dense array, the same software trilinear) and TexSampler (3D CUDA texture,
// hardware trilinear).
//
// Random numbers: Philox4x32-10, counter (pixel, sample, call, stream), key =
// seed; stream 0 for the camera and the walk, 1 for the light rays; one call
// per free flight: u0 = optical depth, u1 = accept, u2/u3 = phase function.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "learn.cuh"
#include "vdbc_host.h"

namespace vdbc {
namespace {

struct CamDev {
    int kind, w, h;
    float3 eye;           // index space
    float3 fwd, right, up;
    float sxs, sys;       // film-plane scale: pinhole tan(fov/2)*aspect, tan(fov/2); ortho in index units
};

struct MedDev {
    int mode;
    int tf_n;
    const float4* tf;
    float step;
    float sigma_scale;    // density_scale / max(dims): extinction per index unit at density 1
    float albedo, g;
    int max_bounces;
    float3 sun_dir, sun_rad, env_rad;
    float iso;
};

struct Majorants {
    const float* mcmax;
    int mc;
    int mx, my, mz;
    int nx, ny, nz;
    const float* mcmin;   // read by the ISO marcher's interval test only
};

// coarse occupancy level over kCoarse^3 macrocells: a ray crosses an empty
// coarse cell in one step instead of one step per macrocell
constexpr int kCoarse = 8;

constexpr int kMaxStepsPerCell = 1 << 20;

// Division in the tracker: with VDBC_PT_FASTDIV=1 (the default) the
// hardware's approximate reciprocal times the dividend (__fdividef, within
// 2 ulp for the magnitudes here), a few instructions instead of the correctly
// rounded sequence; 0 restores IEEE division.  The tracker is bound by
// instruction issue: 13.4 against 16.0 ms for the 1024^2 x 16 spp frame of
// the 512^3 medium, 61.4 against 69.4 ms for the 1920x1080 x 64 spp frame of
// the full-scale cloud, with the oracle parity tests unchanged.  Both forms
// are deterministic, so every sampler instantiation computes the same bits.
#ifndef VDBC_PT_FASTDIV
#define VDBC_PT_FASTDIV 1
#endif
__device__ __forceinline__ float fdiv(float a, float b)
{
#if VDBC_PT_FASTDIV
    return __fdividef(a, b);
#else
    return __fdiv_rn(a, b);
#endif
}

// Square root and logarithm in the tracker: with VDBC_PT_FASTMATH=1 (the
// default) the hardware approximations (sqrt.approx, __logf: a base-2
// logarithm instruction times ln 2) instead of the correctly rounded square
// root and the accurate logf (12.3 against 12.8 ms on the 512^3 frame, 59.7
// against 60.2 on the cloud; oracle parity unchanged); 0 keeps sqrtf and logf.
#ifndef VDBC_PT_FASTMATH
#define VDBC_PT_FASTMATH 1
#endif
__device__ __forceinline__ float fsqrt(float x)
{
#if VDBC_PT_FASTMATH
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return sqrtf(x);
#endif
}

__device__ __forceinline__ float flog(float x)
{
#if VDBC_PT_FASTMATH
    return __logf(x);
#else
    return logf(x);
#endif
}

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 norm3(float3 a)
{
    float l = fsqrt(dot3(a, a));
    return f3(fdiv(a.x, l), fdiv(a.y, l), fdiv(a.z, l));
}

// ray / box [-1/2, dim-1/2]^3, t >= 0
__device__ __forceinline__ bool clip_axis(float o, float d, float hi, float& t0, float& t1)
{
    if (d == 0.0f) return !(o < -0.5f || o > hi);
    float ta = fdiv(-0.5f - o, d), tb = fdiv(hi - o, d);
    if (ta > tb) { float s = ta; ta = tb; tb = s; }
    t0 = fmaxf(t0, ta);
    t1 = fminf(t1, tb);
    return true;
}

__device__ __forceinline__ bool clip_box(const Majorants& m, float3 o, float3 d, float& tin, float& tout)
{
    float t0 = 0.0f, t1 = INFINITY;
    if (!clip_axis(o.x, d.x, (float)m.nx - 0.5f, t0, t1)) return false;
    if (!clip_axis(o.y, d.y, (float)m.ny - 0.5f, t0, t1)) return false;
    if (!clip_axis(o.z, d.z, (float)m.nz - 0.5f, t0, t1)) return false;
    tin = t0;
    tout = t1;
    return t0 < t1;
}

// ray / box [lo, hi] (three lower then three upper bounds), t >= 0
__device__ __forceinline__ bool clip_span(const float* box, float3 o, float3 d, float& tin, float& tout)
{
    float t0 = 0.0f, t1 = INFINITY;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == 0.0f) {
            if (oo[a] < box[a] || oo[a] > box[3 + a]) return false;
        } else {
            float ta = fdiv(box[a] - oo[a], dd[a]), tb = fdiv(box[3 + a] - oo[a], dd[a]);
            if (ta > tb) { float s = ta; ta = tb; tb = s; }
            t0 = fmaxf(t0, ta);
            t1 = fminf(t1, tb);
        }
    }
    tin = t0;
    tout = t1;
    return t0 < t1;
}

// 3D-DDA over the macrocells (Amanatides-Woo stepping).  The next boundary of
// each axis is kept and only the stepped axis is recomputed, from its cell
// index (-1/2 + (c + [s > 0]) * cell - o) / d, so no error accumulates.
#ifndef VDBC_DDA_MAGIC
#define VDBC_DDA_MAGIC 1
#endif
struct Dda {
    int cx, cy, cz, sx, sy, sz;
    float ix, iy, iz;       // 1 / d per axis
    float nx, ny, nz;       // t of the next boundary per axis
    float t, tmax;
    __device__ __forceinline__ static float bnd(int c, int s, float mc, float o, float inv)
    {
        if (s == 0) return INFINITY;
#if VDBC_DDA_MAGIC
        // the boundary index as a float without a conversion instruction
        // (32.2 against 32.4 ms on the full-scale cloud frame, 7.70 against
        // 7.75 on the 512^3 frame, the same bits):
        // n + 1.5 * 2^23 read as a float, minus 1.5 * 2^23 (exact for
        // |n| < 2^22, which holds for every cell index)
        const float fn = __fsub_rn(__int_as_float(c + (s > 0 ? 1 : 0) + 0x4B400000), 12582912.0f);
#else
        const float fn = (float)(c + (s > 0 ? 1 : 0));
#endif
        float b = __fadd_rn(-0.5f, __fmul_rn(fn, mc));
        return __fmul_rn(__fsub_rn(b, o), inv);
    }
    __device__ __forceinline__ static int first_cell(float o, float d, float tmin, float mc, int n)
    {
        float p = __fmaf_rn(tmin, d, o);
        int ci = (int)floorf(fdiv(__fadd_rn(p, 0.5f), mc));
        return min(max(ci, 0), n - 1);
    }
    __device__ __forceinline__ void init(const Majorants& m, float3 o, float3 d, float tmin, float tmax_)
    {
        t = tmin;
        tmax = tmax_;
        float mc = (float)m.mc;
        sx = d.x > 0.0f ? 1 : (d.x < 0.0f ? -1 : 0);
        sy = d.y > 0.0f ? 1 : (d.y < 0.0f ? -1 : 0);
        sz = d.z > 0.0f ? 1 : (d.z < 0.0f ? -1 : 0);
        ix = fdiv(1.0f, d.x); iy = fdiv(1.0f, d.y); iz = fdiv(1.0f, d.z);
        cx = first_cell(o.x, d.x, tmin, mc, m.mx);
        cy = first_cell(o.y, d.y, tmin, mc, m.my);
        cz = first_cell(o.z, d.z, tmin, mc, m.mz);
        nx = bnd(cx, sx, mc, o.x, ix);
        ny = bnd(cy, sy, mc, o.y, iy);
        nz = bnd(cz, sz, mc, o.z, iz);
    }
    // current cell and its exit distance; false once the ray left the grid
    __device__ __forceinline__ bool cell(const Majorants& m, int& id, float& texit) const
    {
        if (t >= tmax) return false;
        if ((unsigned)cx >= (unsigned)m.mx || (unsigned)cy >= (unsigned)m.my || (unsigned)cz >= (unsigned)m.mz)
            return false;
        texit = fminf(fminf(tmax, nx), fminf(ny, nz));
        id = (cz * m.my + cy) * m.mx + cx;
        return true;
    }
    // Cross the whole kCoarse^3 block of macrocells around the current cell,
    // which holds no positive majorant.  The state becomes what cell-by-cell
    // stepping would reach: the block's exit time is the boundary formula of
    // the last macrocell on the exit face, and every other axis crosses the
    // boundaries whose times are <= that exit.  False if the ray ends first.
    __device__ __forceinline__ bool skip_block(const Majorants& m, float3 o)
    {
        float mc = (float)m.mc;
        int fx = sx > 0 ? min((cx / kCoarse) * kCoarse + kCoarse - 1, m.mx - 1) : (cx / kCoarse) * kCoarse;
        int fy = sy > 0 ? min((cy / kCoarse) * kCoarse + kCoarse - 1, m.my - 1) : (cy / kCoarse) * kCoarse;
        int fz = sz > 0 ? min((cz / kCoarse) * kCoarse + kCoarse - 1, m.mz - 1) : (cz / kCoarse) * kCoarse;
        float tx = bnd(fx, sx, mc, o.x, ix), ty = bnd(fy, sy, mc, o.y, iy), tz = bnd(fz, sz, mc, o.z, iz);
        float T = tx;
        int axis = 0;
        if (ty < T) { T = ty; axis = 1; }
        if (tz < T) { T = tz; axis = 2; }
        if (!(T < tmax)) { t = tmax; return false; }
        if (axis == 0) cx = fx + sx; else { for (int k = 0; k < kCoarse && bnd(cx, sx, mc, o.x, ix) <= T; ++k) cx += sx; }
        if (axis == 1) cy = fy + sy; else { for (int k = 0; k < kCoarse && bnd(cy, sy, mc, o.y, iy) <= T; ++k) cy += sy; }
        if (axis == 2) cz = fz + sz; else { for (int k = 0; k < kCoarse && bnd(cz, sz, mc, o.z, iz) <= T; ++k) cz += sz; }
        nx = bnd(cx, sx, mc, o.x, ix);
        ny = bnd(cy, sy, mc, o.y, iy);
        nz = bnd(cz, sz, mc, o.z, iz);
        if (T > t) t = T;
        return true;
    }
    // step the axis whose boundary is nearest (x, then y, then z on ties)
    __device__ __forceinline__ void advance(const Majorants& m, float3 o, float texit)
    {
        float mc = (float)m.mc;
        if (nx <= ny && nx <= nz) {
            if (!(nx < tmax)) { t = tmax; return; }
            cx += sx; nx = bnd(cx, sx, mc, o.x, ix);
        } else if (ny <= nz) {
            if (!(ny < tmax)) { t = tmax; return; }
            cy += sy; ny = bnd(cy, sy, mc, o.y, iy);
        } else {
            if (!(nz < tmax)) { t = tmax; return; }
            cz += sz; nz = bnd(cz, sz, mc, o.z, iz);
        }
        if (texit > t) t = texit;
    }
};

__device__ __forceinline__ float hg_eval(float mu, float g)
{
    float den = 1.0f + g * g - 2.0f * g * mu;
    return fdiv(1.0f - g * g, 4.0f * 3.14159265358979f * den * fsqrt(den));
}

__device__ __forceinline__ float hg_sample_mu(float g, float xi)
{
    float mu;
    if (fabsf(g) < 1e-3f) mu = 1.0f - 2.0f * xi;
    else {
        float s = fdiv(1.0f - g * g, 1.0f - g + 2.0f * g * xi);
        mu = fdiv(1.0f + g * g - s * s, 2.0f * g);
    }
    return fminf(fmaxf(mu, -1.0f), 1.0f);
}

// Duff et al., "Building an Orthonormal Basis, Revisited" (JCGT 2017)
__device__ __forceinline__ void onb(float3 n, float3& b1, float3& b2)
{
    float sign = n.z >= 0.0f ? 1.0f : -1.0f;
    float a = fdiv(-1.0f, sign + n.z);
    float b = n.x * n.y * a;
    b1 = f3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
    b2 = f3(b, sign + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ void camera_ray(const CamDev& cam, int px, int py, float jx, float jy, float3& o,
                                           float3& d)
{
    float sx = fdiv(2.0f * ((float)px + jx), (float)cam.w) - 1.0f;
    float sy = 1.0f - fdiv(2.0f * ((float)py + jy), (float)cam.h);
    if (cam.kind == VDBC_CAM_ORTHO) {
        float a = sx * cam.sxs, b = sy * cam.sys;
        o = f3(__fmaf_rn(b, cam.up.x, __fmaf_rn(a, cam.right.x, cam.eye.x)),
               __fmaf_rn(b, cam.up.y, __fmaf_rn(a, cam.right.y, cam.eye.y)),
               __fmaf_rn(b, cam.up.z, __fmaf_rn(a, cam.right.z, cam.eye.z)));
        d = cam.fwd;
    } else {
        float a = sx * cam.sxs, b = sy * cam.sys;
        o = cam.eye;
        d = norm3(f3(__fmaf_rn(b, cam.up.x, __fmaf_rn(a, cam.right.x, cam.fwd.x)),
                     __fmaf_rn(b, cam.up.y, __fmaf_rn(a, cam.right.y, cam.fwd.y)),
                     __fmaf_rn(b, cam.up.z, __fmaf_rn(a, cam.right.z, cam.fwd.z))));
    }
}

struct Rng {
    uint32_t pixel, sample, k0, k1;
    __device__ __forceinline__ U4 draw(uint32_t call, uint32_t stream) const
    {
        return philox4x32_10(pixel, sample, call, stream, k0, k1);
    }
};

struct Walk {
    unsigned long long lookups;
    unsigned long long flags;
#ifdef VDBC_STATS
    // loop iterations, DDA cells examined, coarse blocks crossed, free flights
    // drawn, rays started, paths fetched, accessor leaf queries, tree descents
    unsigned int ev[kNumEvents];
#endif
};

#ifdef VDBC_STATS
#define VDBC_EVENT(w, k) ((w).ev[k]++)
#else
#define VDBC_EVENT(w, k) ((void)0)
#endif

__device__ __forceinline__ void flush_stats(DevStats* st, const Walk& w, unsigned long long paths)
{
    unsigned long long a = w.lookups, p = paths;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        p += __shfl_xor_sync(0xffffffffu, p, o);
    }
    unsigned long long f = w.flags;
    for (int o = 16; o > 0; o >>= 1) f |= __shfl_xor_sync(0xffffffffu, f, o);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&st->lookups, a);
        atomicAdd(&st->paths, p);
        if (f) atomicOr(&st->error_flags, f);
    }
#ifdef VDBC_STATS
    for (int k = 0; k < kNumEvents; ++k) atomicAdd(&st->ev[k], (unsigned long long)w.ev[k]);
#endif
}

// ---------------------------------------------------------------- path tracer
// One lane carries one light path at a time and fetches the next path as soon
// as its own ends (persistent threads, warp-aggregated work counter), so the
// lanes of a warp stay busy until the work runs out.  Delta tracking and the
// light ray's ratio tracking are one loop: every iteration a lane either
// moves to its next non-empty macrocell or takes one tentative step with a
// density lookup, whichever its path needs; lanes therefore issue their
// lookups together.  Random-number use per path is the oracle's: the camera
// takes call 0 of stream 0, each tentative step of the walk the next call of
// stream 0, each tentative step of a light ray the next call of stream 1.
// A finished path adds its radiance to accum[3 * pixel + c] as a 32.32
// fixed-point integer (fix32 below): integer addition is associative, so the
// frame's sums are the same bits whatever order the paths finish in, and no
// per-path buffer is needed.

enum : int { kNeed = 0, kDone = 1, kDelta = 2, kRatio = 3 };

// radiance (>= 0) as a 32.32 fixed-point integer, rounded to nearest: exact
// for values of 2^-8 and above, within 2^-33 below; a frame's per-pixel sum
// stays far below 2^64 (radiance < 2^31 per path, clamped, times spp < 2^31)
__device__ __forceinline__ unsigned long long fix32(float x)
{
    x = fminf(fmaxf(x, 0.0f), 2147483648.0f);      // (a NaN becomes 0)
    return __float2ull_rn(__fmul_rn(x, 4294967296.0f));
}

struct Track {
    Dda dda;
    float tcur, texit, mj;
};

// next macrocell with a positive majorant at or after the current DDA cell;
// false when the ray leaves the grid.  Blocks of kCoarse^3 macrocells whose
// coarse bit is clear are crossed in one step; inside an occupied block,
// cells whose own bit is clear (majorant <= 0) are passed without loading
// their majorant.
// kUseCoarse: test the coarse level before the cell (compiled out where the
// coarse level is off, which also frees the registers skip_block needs)
// cells next_cell examines per call before it reports that the search goes
// on (0: no limit); the tracker resumes the search in its next iteration.
// Measured on the 512^3 medium with 48^3 cells: no limit 18.1 ms, 1: 30.0,
// 2: 28.4, 4: 35.8 (the walk loop in its present form, with the search state,
// compiles to a much faster tracker than the earlier loop with breaks: 30.1 ms)
#ifndef VDBC_PT_SEARCH
#define VDBC_PT_SEARCH 0
#endif
enum { kCellEnded = 0, kCellFound = 1, kCellSearching = 2 };

template <bool kUseCoarse>
__device__ __forceinline__ int next_cell(Track& tr, const Majorants& m, const MedDev& med, float3 o,
                                         const uint32_t* bits, const uint32_t* cbits, int cx_n, int cy_n,
                                         int& guard, Walk& w)
{
    int id;
    float texit;
    for (int n = 0; tr.dda.cell(m, id, texit); ++n) {
#if VDBC_PT_SEARCH > 0
        if (n == VDBC_PT_SEARCH) return kCellSearching;
#endif
        VDBC_EVENT(w, 1);
        if (--guard < 0) return kCellEnded;
        if constexpr (kUseCoarse) {
            int cid = ((tr.dda.cz / kCoarse) * cy_n + tr.dda.cy / kCoarse) * cx_n + tr.dda.cx / kCoarse;
            if (!((cbits[cid >> 5] >> (cid & 31)) & 1u)) {
                VDBC_EVENT(w, 2);
                if (!tr.dda.skip_block(m, o)) return kCellEnded;
                continue;
            }
        }
        if (((bits[id >> 5] >> (id & 31)) & 1u) && texit > tr.dda.t) {
            float mj = __fmul_rn(med.sigma_scale, __ldg(m.mcmax + id));
            if (mj > 0.0f) {
                tr.mj = mj;
                tr.texit = texit;
                tr.tcur = tr.dda.t;
                return kCellFound;
            }
        }
        tr.dda.advance(m, o, texit);
    }
    return kCellEnded;
}

// Division of a 32-bit n by an invariant d >= 1 with one high multiply, the
// round-up method of Granlund and Montgomery ("Division by Invariant Integers
// using Multiplication", PLDI 1994, Section 4): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n),
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), exact for every n.
struct DivU32 {
    uint32_t m;
    int s1, s2;
    __host__ void init(uint32_t d)
    {
        int l = 0;
        while ((1ull << l) < (unsigned long long)d) ++l;
        m = (uint32_t)(((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / d + 1ull);
        s1 = l > 0 ? 1 : 0;
        s2 = l > 0 ? l - 1 : 0;
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const
    {
        const uint32_t t = __umulhi(m, n);
        return (t + ((n - t) >> s1)) >> s2;
    }
};

// Constants of one render job as the tracker sees them.
struct JobView {
    Majorants m;
    CamDev cam;
    MedDev med;
    const uint32_t* bits;      // occupancy bit per macrocell (majorant > 0)
    const uint32_t* cbits;     // occupancy bit per kCoarse^3 block of macrocells
    int cx_n, cy_n;            // coarse grid size along x and y
    unsigned long long* accum; // 3 per pixel: the frame's radiance sums, 32.32 fixed point
    const int* occ_box;        // macrocell index box of the positive majorants (lo xyz, hi xyz), or null
    float clip[6];             // (batch jobs) the clip box in index space built from it, as k_pt builds it
    int npix, spp, tiles_x;
    uint32_t k0, k1;           // Philox key = the seed
    uint32_t sample_base;      // sample id of the frame's first sample (progressive frames)
    unsigned long long item_begin, items;   // this job's range of the work counter
    uint32_t per;              // work items per sample (8x4 tiles x 32)
    int items32;               // items < 2^32: item decode by the invariant divisions below
    DivU32 div_per, div_tiles_x;
    int tile_major;            // items ordered (tile, sample, pixel) instead of (sample, tile, pixel)
    uint32_t spp32;            // work items per tile over all samples (tile-major order)
    DivU32 div_spp32;
};

// one job: constants in kernel parameters, the grid's payload fixed at compile time
template <class S>
struct SingleSource {
    static constexpr bool kMulti = false;
    static constexpr bool kCollective = S::kCollective;
    const JobView& j;
    const S& smp;
    const uint32_t* b;
    const uint32_t* cb;
    const float* box;     // the clip box in index space (shared memory)
    const float* smaj;    // the macrocells' majorants in shared memory, or null
    __device__ __forceinline__ const float* maj(int) const { return smaj; }
    // rays are clipped to the box of the cells with a positive majorant: no
    // free flight starts outside it, so starting the walk at its boundary
    // changes no path
    __device__ __forceinline__ bool clip(int, const Majorants&, float3 o, float3 d, float& tin, float& tout) const
    {
        return clip_span(box, o, d, tin, tout);
    }
    __device__ __forceinline__ int find(unsigned long long, int) const { return 0; }
    __device__ __forceinline__ const JobView& job(int) const { return j; }
    __device__ __forceinline__ const uint32_t* bits(int) const { return b; }
    __device__ __forceinline__ const uint32_t* cbits(int) const { return cb; }
    __device__ __forceinline__ float sample(int, float x, float y, float z, Accessor& a) const { return smp(x, y, z, a); }
    __device__ __forceinline__ float collective(bool look, float x, float y, float z, Accessor& a) const
    {
        return smp.collective(look, x, y, z, a);
    }
};

// many jobs of one payload type P: their constants and grids staged in
// shared memory
template <int P, int D>
struct BatchSource {
    static constexpr bool kMulti = true;
    static constexpr bool kCollective = false;
    const JobView* jobs;
    const GridView* grids;
    int n;
    // a lane's items only grow, so the search starts at its current job
    __device__ __forceinline__ int find(unsigned long long item, int from) const
    {
        int j = from;
        while (j + 1 < n && item >= jobs[j + 1].item_begin) ++j;
        return j;
    }
    __device__ __forceinline__ const JobView& job(int i) const { return jobs[i]; }
    // each job's rays are clipped to the box of its occupied macrocells, as
    // single renders' (1:1 bit-identical images)
    __device__ __forceinline__ bool clip(int i, const Majorants&, float3 o, float3 d, float& tin, float& tout) const
    {
        return clip_span(jobs[i].clip, o, d, tin, tout);
    }
    __device__ __forceinline__ const uint32_t* bits(int i) const { return jobs[i].bits; }
    __device__ __forceinline__ const uint32_t* cbits(int i) const { return jobs[i].cbits; }
    __device__ __forceinline__ const float* maj(int) const { return nullptr; }
    __device__ __forceinline__ float sample(int i, float x, float y, float z, Accessor& a) const
    {
        // the payload is the group's, fixed at compile time (one kernel with a
        // run-time dispatch over the three samplers, and one trilinear switching
        // per voxel, both measured slower: 150.6 and 162.9 ms for the 32-job frame)
        return vdb_trilinear<P, D>(grids[i], x, y, z, a);
    }
};

// The tracker loop shared by the single-job and the batch kernels.
// stride > 1 renders every stride-th path only (the autotuner's sample of a frame)
//
// kPhased = false: in one iteration a lane goes through every block its path
// needs (ray start, free flight, lookup and collision, ray end), so the warp
// runs every block that any of its lanes needs.  kPhased = true: the warp
// runs one block per iteration, the one the most of its lanes wait for (ties:
// lookup, flight, start, end); a lane moves one block forward when its block
// runs.  Each lane's arithmetic is the same either way (equal images).
enum : int { kPhLook = 0, kPhFlight = 1, kPhStart = 2, kPhEnd = 3 };

// the walk of a free flight over the macrocells: 1 one flat loop of single
// cell steps shared by the warp's lanes, 0 a loop of crossings with an inner
// search (next_cell) per crossing
#ifndef VDBC_PT_FLAT
#define VDBC_PT_FLAT 1
#endif
// 1: a ray's search for its first occupied cell runs in the flat walk of the
// free flight, whose draw is then made before the cell is found (its call
// number counted once it is); 0: the search runs where the ray starts,
// before the draw
#ifndef VDBC_PT_SPECDRAW
#define VDBC_PT_SPECDRAW 1
#endif
// cells a lane's flat walk examines per loop iteration before it parks the
// free flight until the next iteration (0: no limit).  Parking measured
// slower at every limit: 55.7, 50.6 and 52.2 ms at 2, 4 and 8 cells against
// 37.9 unbounded on the full-scale cloud frame, 10.8, 10.1, 10.3 against 8.33
// on the 512^3 frame (the iterations it adds cost more than the lanes it
// keeps in step)
#ifndef VDBC_PT_WALK
#define VDBC_PT_WALK 0
#endif

template <bool kUseCoarse, class Src, bool kPhased = false>
__device__ __forceinline__ void pt_loop(const Src& src, unsigned long long nitems, DevStats* __restrict__ st,
                                        int chunk, unsigned stride)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    Walk w{};
    unsigned long long paths = 0;

    int mode = kNeed, jb = 0;
    uint32_t pixel = 0, sample = 0, call = 0, lcall = 0;
    int bounce = 0;
    float3 o = f3(0.f, 0.f, 0.f), d = f3(0.f, 0.f, 1.f), nd = d, L = f3(0.f, 0.f, 0.f);
    float beta = 1.0f, T = 1.0f, ph = 0.0f;
    float tau = -1.0f, ua = 0.0f, ub = 0.0f, uc = 0.0f;   // current free flight: optical depth left, u1..u3
    int steps_in_cell = 0, guard = 0;
    bool start = false;   // a ray to start before the next free flight
    bool searching = false;   // the ray's next occupied cell is still being searched for
    bool pend_look = false;   // (phased) a lookup waits at o + tcur d
    bool spec = false;        // the current free flight was drawn ahead of the ray's first occupied cell
    unsigned long long pool_next = 0, pool_end = 0;   // this warp's share of the work counter
    Track tr;
    Accessor acc;
    acc.reset();

    for (;;) {
        if (mode != kDone) VDBC_EVENT(w, 0);
        // ---- fetch work for lanes without a path: each warp takes `chunk`
        // items at a time from the global counter and hands them out to its
        // lanes in order, so the counter is touched once per chunk.  (Waiting
        // until 4, 8 or 16 lanes need a path, so that the ray starts run with
        // more lanes, measured equal or slower: 8.66, 8.87, 9.74 ms against
        // 8.57 on the 512^3 frame, 44.1, 44.4, 46.4 against 44.1 on the cloud.)
        const unsigned need = __ballot_sync(0xffffffffu, mode == kNeed);
        if (need) {
            const unsigned n = (unsigned)__popc(need);
            const unsigned long long avail = pool_end - pool_next;
            unsigned long long fresh = 0;
            if (avail < n) {
                if (lane == 0) fresh = atomicAdd(&st->work_next, (unsigned long long)chunk);
                fresh = __shfl_sync(0xffffffffu, fresh, 0);
            }
            if (mode == kNeed) {
                const unsigned long long r = (unsigned long long)__popc(need & lt_mask);
                unsigned long long item = (r < avail ? pool_next + r : fresh + (r - avail)) * stride;
                if (item >= nitems) {
                    mode = kDone;
                } else {
                    // item -> (job, 8x4 pixel tile, sample, pixel in tile), or (job,
                    // sample, tile, pixel) with the sample-first order: a warp's paths are neighbours
                    // (the divisions by invariants take one high multiply each;
                    // 64-bit division only for frames of 2^32 items or more)
                    jb = src.find(item, jb);
                    const JobView& F = src.job(jb);
                    const unsigned long long local = item - F.item_begin;
                    uint32_t q, ty, tx;
                    if (F.items32 && F.tile_major) {
                        // a tile's 32 pixels sample after sample: a warp's
                        // successive paths start from the same pixels
                        const uint32_t l32 = (uint32_t)local;
                        const uint32_t tile = F.div_spp32.div(l32);
                        const uint32_t r = l32 - tile * F.spp32;
                        sample = r >> 5;
                        q = (tile << 5) | (r & 31);
                        ty = F.div_tiles_x.div(tile);
                        tx = tile - ty * (uint32_t)F.tiles_x;
                    } else if (F.items32) {
                        const uint32_t l32 = (uint32_t)local;
                        sample = F.div_per.div(l32);
                        q = l32 - sample * F.per;
                        ty = F.div_tiles_x.div(q >> 5);
                        tx = (q >> 5) - ty * (uint32_t)F.tiles_x;
                    } else {
                        const unsigned long long per = F.per;
                        sample = (uint32_t)(local / per);
                        q = (uint32_t)(local - (unsigned long long)sample * per);
                        ty = (q >> 5) / (uint32_t)F.tiles_x;
                        tx = (q >> 5) - ty * (uint32_t)F.tiles_x;
                    }
                    const uint32_t in = q & 31;
                    int px = (int)tx * 8 + (int)(in & 7);
                    int py = (int)ty * 4 + (int)(in >> 3);
                    if (px < F.cam.w && py < F.cam.h) {
                        VDBC_EVENT(w, 5);
                        pixel = (uint32_t)(py * F.cam.w + px);
                        if (src.kMulti) acc.reset();   // another job may use another grid
                        Rng rng{pixel, F.sample_base + sample, F.k0, F.k1};
                        call = 0;
                        lcall = 0;
                        U4 r = rng.draw(call++, 0);
                        camera_ray(F.cam, px, py, u01(r.x), u01(r.y), o, d);
                        L = f3(0.f, 0.f, 0.f);
                        beta = 1.0f;
                        bounce = 0;
                        mode = kDelta;
                        start = true;
                    }
                }
            }
            if (avail < n) { pool_next = fresh + (n - avail); pool_end = fresh + (unsigned long long)chunk; }
            else pool_next += n;
        }
        if (__all_sync(0xffffffffu, mode == kDone)) break;
        const JobView& J = src.job(jb);
        // batch: copies in registers (the job table is in shared memory and the
        // DDA walk reads these per cell; references into it measured 162.6
        // against 150.6 ms for the 32-job frame despite fewer spills); one
        // job: references to kernel parameters
        typename std::conditional<Src::kMulti, const Majorants, const Majorants&>::type m = J.m;
        typename std::conditional<Src::kMulti, const MedDev, const MedDev&>::type med = J.med;
        const uint32_t* bits = src.bits(jb);
        const uint32_t* cbits = src.cbits(jb);
        const int cx_n = J.cx_n, cy_n = J.cy_n;

        int P = kPhLook;      // (phased) the block this iteration runs
        if constexpr (kPhased) {
            const bool live = mode == kDelta || mode == kRatio;
            const int cl = __popc(__ballot_sync(0xffffffffu, live && !start && pend_look));
            const int cf = __popc(__ballot_sync(0xffffffffu, live && !start && !pend_look));
            const int cs = __popc(__ballot_sync(0xffffffffu, start));
            const int ce = __popc(__ballot_sync(0xffffffffu, mode < 0));
            int best = cl;
            if (cf > best) { P = kPhFlight; best = cf; }
            if (cs > best) { P = kPhStart; best = cs; }
            if (ce > best) { P = kPhEnd; best = ce; }
        }

        // ---- the lane's pending ray (camera ray, light ray or next bounce):
        // box clip and first occupied cell, from one place in the code.
        // (Holding starts back until more lanes wait for one, and running the
        // block then for all of them, measured slower at every threshold:
        // 16.0 ms with no hold, 16.3 at 8 waiting lanes, 17.5 at 16.)
        if (start && (!kPhased || P == kPhStart)) {
            start = false;
            searching = false;
            float tin, tout;
            if (src.clip(jb, m, o, d, tin, tout)) {
                tr.dda.init(m, o, d, tin, tout);
                tau = -1.0f;   // every ray starts a new free flight
                VDBC_EVENT(w, 4);
                guard = m.mx + m.my + m.mz + 8;
                steps_in_cell = 0;
#if VDBC_PT_FLAT && VDBC_PT_SPECDRAW
                searching = true;   // the flight's walk finds the first occupied cell
#else
                const int st = next_cell<kUseCoarse>(tr, m, med, o, bits, cbits, cx_n, cy_n, guard, w);
                if (st == kCellEnded) mode = -mode;   // leaves at once
                searching = st == kCellSearching;
#endif
            } else {
                mode = -mode;
            }
        }

        // ---- one free flight per lane: draw tau, spend it over the cells, and
        // where it runs out evaluate the density (delta: accept or not;
        // ratio: attenuate)
        bool look = false;
        float3 x = f3(0.f, 0.f, 0.f);
        if ((mode == kDelta || mode == kRatio) && !start && (!kPhased || (P == kPhFlight && !pend_look))) {
            bool ended = false, parked = false;
            if (!VDBC_PT_FLAT && searching) {   // the search for the ray's next occupied cell goes on
                const int st = next_cell<kUseCoarse>(tr, m, med, o, bits, cbits, cx_n, cy_n, guard, w);
                if (st == kCellEnded) ended = true;
                else if (st == kCellSearching) parked = true;
                else searching = false;
            }
            if (!ended && !parked && tau < 0.0f) {
                Rng rng{pixel, J.sample_base + sample, J.k0, J.k1};
#if VDBC_PT_FLAT && VDBC_PT_SPECDRAW
                // a lane still looking for its ray's first occupied cell draws
                // ahead of finding it, and the draw's call number is taken
                // once the cell is found: a ray that meets no occupied cell
                // takes no call, as in the oracle
                spec = searching;
                U4 r = (mode == kDelta) ? rng.draw(call, 0) : rng.draw(lcall, 1);
                if (!spec) {
                    if (mode == kDelta) ++call;
                    else ++lcall;
                    VDBC_EVENT(w, 3);
                }
#else
                U4 r = (mode == kDelta) ? rng.draw(call++, 0) : rng.draw(lcall++, 1);
                VDBC_EVENT(w, 3);
#endif
                tau = -flog(1.0f - u01(r.x));
                ua = u01(r.y); ub = u01(r.z); uc = u01(r.w);
            }
            // spend tau over as many cells as it lasts, so that the draw and
            // the lookup below run once per iteration
#if VDBC_PT_FLAT
            // One DDA cell per trip for every lane: a lane standing in an
            // occupied cell spends tau over it (or stops at its collision
            // point), a lane between occupied cells examines the next cell as
            // next_cell does.  The lanes of a warp thus share one loop, whose
            // trips are the most cells any lane passes, instead of an inner
            // search loop per crossing; each lane's arithmetic is next_cell's.
            if (!ended && !parked) {
                // the lane stands in an occupied cell (tr.mj, tr.texit, tr.tcur)
                // unless it resumes a search it was parked in
                bool have = !searching;
                searching = false;
                for (int k = 0;; ++k) {
#if VDBC_PT_WALK > 0
                    if (k == VDBC_PT_WALK) {   // go on in the next iteration (tau kept)
                        parked = true;
                        searching = !have;
                        break;
                    }
#endif
                    float tadv = 0.0f;
                    if (!have) {
                        int id;
                        float tex;
                        if (!tr.dda.cell(m, id, tex)) { ended = true; break; }
                        VDBC_EVENT(w, 1);
                        if (--guard < 0) { ended = true; break; }
                        if constexpr (kUseCoarse) {
                            int cid = ((tr.dda.cz / kCoarse) * cy_n + tr.dda.cy / kCoarse) * cx_n + tr.dda.cx / kCoarse;
                            if (!((cbits[cid >> 5] >> (cid & 31)) & 1u)) {
                                VDBC_EVENT(w, 2);
                                if (!tr.dda.skip_block(m, o)) { ended = true; break; }
                                continue;
                            }
                        }
                        float mj = 0.0f;
                        const float* smaj = src.maj(jb);
                        if (smaj) {   // the same product, formed at launch (positive exactly where the bit is set)
                            if (tex > tr.dda.t) mj = smaj[id];
                        } else if (((bits[id >> 5] >> (id & 31)) & 1u) && tex > tr.dda.t) {
                            mj = __fmul_rn(med.sigma_scale, __ldg(m.mcmax + id));
                        }
                        if (mj > 0.0f) {
                            tr.mj = mj;
                            tr.texit = tex;
                            tr.tcur = tr.dda.t;
                            have = true;
#if VDBC_PT_SPECDRAW
                            if (spec) {   // the ray's first occupied cell: its draw counts
                                if (mode == kDelta) ++call;
                                else ++lcall;
                                VDBC_EVENT(w, 3);
                                spec = false;
                            }
#endif
                        }
                        tadv = tex;
                    }
                    if (have) {
                        const float reach = __fmul_rn(tr.mj, __fsub_rn(tr.texit, tr.tcur));
                        if (tau < reach) break;          // the collision point lies in this cell
                        tau = __fsub_rn(tau, reach);
                        tadv = tr.texit;
                        steps_in_cell = 0;
                        have = false;
                    }
                    tr.dda.advance(m, o, tadv);
                }
            }
#else
            // (nested form: each crossing searches the next occupied cell in
            // an inner loop)
            for (int k = 0; !ended && !parked; ++k) {
                float reach = __fmul_rn(tr.mj, __fsub_rn(tr.texit, tr.tcur));
                if (tau < reach) break;
                tau = __fsub_rn(tau, reach);
                tr.dda.advance(m, o, tr.texit);
                steps_in_cell = 0;
                const int st = next_cell<kUseCoarse>(tr, m, med, o, bits, cbits, cx_n, cy_n, guard, w);
                if (st == kCellEnded) {
                    ended = true;
                    break;
                }
                if (st == kCellSearching) {
                    searching = true;
                    parked = true;
                    break;
                }
            }
#endif
            if (ended && guard < 0) w.flags |= kErrDdaSteps;
            if (ended) {
                mode = -mode;            // ray ended
            } else if (parked) {
                // the free flight continues in the next iteration (tau kept)
            } else if (++steps_in_cell > kMaxStepsPerCell) {
                w.flags |= kErrTrackSteps;
                mode = -mode;            // give up on this ray (reported through the error word)
            } else {
                float t = __fadd_rn(tr.tcur, fdiv(tau, tr.mj));
                tr.tcur = t;
                tau = -1.0f;
                if constexpr (kPhased) {
                    pend_look = true;
                } else {
                    x = f3(__fmaf_rn(t, d.x, o.x), __fmaf_rn(t, d.y, o.y), __fmaf_rn(t, d.z, o.z));
                    look = true;
                }
            }
        }
        if constexpr (kPhased) {
            if (P == kPhLook && pend_look) {
                const float t = tr.tcur;
                x = f3(__fmaf_rn(t, d.x, o.x), __fmaf_rn(t, d.y, o.y), __fmaf_rn(t, d.z, o.z));
                look = true;
                pend_look = false;
            }
        }
        // ---- the density lookup: per lane, or for a learned grid by the whole
        // warp at once (its network runs on warp-wide tiles)
        float dens = 0.0f;
        if constexpr (Src::kCollective) {
            if (!kPhased || P == kPhLook) {      // P is the same in every lane
                __syncwarp();
                dens = src.collective(look, x.x, x.y, x.z, acc);
            }
        }
        if (look) {
            if constexpr (!Src::kCollective) dens = src.sample(jb, x.x, x.y, x.z, acc);
            float sigma = __fmul_rn(med.sigma_scale, dens);
            ++w.lookups;
            if (mode == kRatio) {
                T = __fmul_rn(T, __fsub_rn(1.0f, fdiv(sigma, tr.mj)));
            } else if (__fmul_rn(ua, tr.mj) < sigma) {
                // real collision: scatter, then trace the light ray from here (inline: the
                // same code out of line cost 17.0 against 16.1 ms on the benchmark frame)
                beta *= med.albedo;
                ph = hg_eval(dot3(d, med.sun_dir), med.g);
                float mu = hg_sample_mu(med.g, ub);
                float st_ = fsqrt(fmaxf(0.0f, 1.0f - mu * mu));
                float sphi, cphi;
                sincospif(2.0f * uc, &sphi, &cphi);
                float3 b1, b2;
                onb(d, b1, b2);
                nd = norm3(f3(st_ * cphi * b1.x + st_ * sphi * b2.x + mu * d.x,
                              st_ * cphi * b1.y + st_ * sphi * b2.y + mu * d.y,
                              st_ * cphi * b1.z + st_ * sphi * b2.z + mu * d.z));
                o = x;
                d = med.sun_dir;
                T = 1.0f;
                mode = kRatio;
                start = true;
            }
        }
        // ---- a ray ended (negative mode): escape, or the light ray's contribution
        if (mode < 0 && (!kPhased || P == kPhEnd)) {
            bool finished = false;
            if (mode == -kDelta) {
                L.x += beta * med.env_rad.x; L.y += beta * med.env_rad.y; L.z += beta * med.env_rad.z;
                finished = true;
            } else {
                float wgt = beta * ph * T;
                L.x += wgt * med.sun_rad.x; L.y += wgt * med.sun_rad.y; L.z += wgt * med.sun_rad.z;
                if (++bounce >= med.max_bounces) {
                    finished = true;
                } else {
                    d = nd;          // the next bounce starts at the top of the next iteration
                    mode = kDelta;
                    start = true;
                }
            }
            if (finished) {
                unsigned long long* a = J.accum + 3 * (size_t)pixel;
                atomicAdd(a + 0, fix32(L.x));
                atomicAdd(a + 1, fix32(L.y));
                atomicAdd(a + 2, fix32(L.z));
                ++paths;
                mode = kNeed;
            }
        }
    }
#ifdef VDBC_STATS
    w.ev[6] += acc.queries;
    w.ev[7] += acc.descents;
#endif
    flush_stats(st, w, paths);
}

// resident 256-thread blocks per SM the tracker is compiled for: 4 (64
// registers) measured fastest for the plain samplers without the coarse level
// (36.4 ms against 40.1 at 2, 44.0 at 3, 37.1 at 5 on the 512^3 medium with
// 48^3 cells; again with 32-item work chunks and 56^3 cells: 16.1 ms against
// 16.7 at 5 and 17.0 at 6; with the flat walk, the full-scale cloud frame
// 42.1 at 3 against 37.9 with 32-item chunks and 35.2 at 5 against 34.9 with
// adaptive chunks, the 512^3 frame 8.58 at 3 and 8.75 at 5 against 8.30); with
// the coarse level (8^3 cells) 2 is faster
// (130.9 against 153.6 ms), and the learned sampler keeps 2 (its tile code
// needs the registers)
#ifndef VDBC_PT_MIN_BLOCKS
#define VDBC_PT_MIN_BLOCKS 4
#endif
template <class S, bool kUseCoarse>
constexpr int pt_min_blocks()
{
    return (S::kCollective || kUseCoarse) ? 2 : VDBC_PT_MIN_BLOCKS;
}

// the ray clip box in index space (lo xyz, hi xyz): the volume's, or with
// `occ` (a macrocell index box) that of its cells, clamped to the volume
__device__ __forceinline__ void occupied_clip_box(const Majorants& m, const int* occ, float* box)
{
    const float dims[3] = {(float)m.nx, (float)m.ny, (float)m.nz};
    for (int a = 0; a < 3; ++a) { box[a] = -0.5f; box[3 + a] = dims[a] - 0.5f; }
    if (occ) {
        const float mc = (float)m.mc;
        for (int a = 0; a < 3; ++a) {
            const int lo = occ[a], hi = occ[3 + a];
            // (no positive majorant anywhere: an empty box, every ray misses)
            box[a] = lo <= hi ? __fsub_rn(__fmul_rn((float)lo, mc), 0.5f) : 1.0f;
            box[3 + a] = lo <= hi ? fminf(__fsub_rn(__fmul_rn((float)(hi + 1), mc), 0.5f), dims[a] - 0.5f) : 0.0f;
        }
    }
}

// gbits: nwords fine occupancy words followed by ncwords coarse words; the
// parts that fit in `smem_words` are staged in shared memory (coarse first);
// smaj_cells > 0: the majorant of every macrocell (sigma_scale x max, the
// product the walk forms) follows them in shared memory
template <class S, bool kUseCoarse, bool kPhased = false, int kBlocks = pt_min_blocks<S, kUseCoarse>()>
__global__ void __launch_bounds__(256, kBlocks)
    k_pt(S smp, JobView job, const uint32_t* __restrict__ gbits, int nwords, int ncwords, int smem_words,
         int smaj_cells, DevStats* __restrict__ st, int chunk)
{
    extern __shared__ uint32_t s_bits[];
    __shared__ float s_box[6];
    if (threadIdx.x == 0) occupied_clip_box(job.m, job.occ_box, s_box);
    const uint32_t* cbits = gbits + nwords;
    const uint32_t* bits = gbits;
    if (ncwords <= smem_words) {
        for (int i = threadIdx.x; i < ncwords; i += blockDim.x) s_bits[i] = gbits[nwords + i];
        cbits = s_bits;
        if (ncwords + nwords <= smem_words) {
            for (int i = threadIdx.x; i < nwords; i += blockDim.x) s_bits[ncwords + i] = gbits[i];
            bits = s_bits + ncwords;
        }
    }
    float* s_maj = nullptr;
    if (smaj_cells > 0) {
        s_maj = reinterpret_cast<float*>(s_bits + smem_words);
        for (int i = threadIdx.x; i < smaj_cells; i += blockDim.x)
            s_maj[i] = __fmul_rn(job.med.sigma_scale, __ldg(job.m.mcmax + i));
    }
    __syncthreads();
    SingleSource<S> src{job, smp, bits, cbits, s_box, s_maj};
    pt_loop<kUseCoarse, SingleSource<S>, kPhased>(src, job.items, st, chunk, 1u);
}

// the jobs of one payload type in one persistent launch; frame[0] numbers the
// progressive frame, so frame f renders sample ids [f*spp, (f+1)*spp)
template <int kThreads, bool kUseCoarse, int kPayload, int kDepth>
__global__ void __launch_bounds__(kThreads, (kUseCoarse ? 512 : 1024) / kThreads)
    k_pt_batch(const JobView* __restrict__ jobs, const GridView* __restrict__ grids, int n,
               unsigned long long nitems, const int* __restrict__ frame, DevStats* __restrict__ st, int chunk,
               unsigned stride)
{
    extern __shared__ unsigned char s_raw[];
    JobView* sj = reinterpret_cast<JobView*>(s_raw);
    GridView* sg = reinterpret_cast<GridView*>(s_raw + sizeof(JobView) * n);
    const int f = frame[0];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sj[i] = jobs[i];
        sj[i].sample_base = (uint32_t)f * (uint32_t)sj[i].spp;
        sg[i] = grids[i];
    }
    __syncthreads();
    BatchSource<kPayload, kDepth> src{sj, sg, n};
    pt_loop<kUseCoarse>(src, nitems, st, chunk, stride);
}

// a pixel's fixed-point sum as a float (2^-32 times the integer, rounded once)
__device__ __forceinline__ float unfix32(unsigned long long a)
{
    return __fmul_rn(__ull2float_rn(a), 2.3283064365386963e-10f);
}

// the per-pixel mean of the frame's spp path radiances
__global__ void k_pt_resolve(const unsigned long long* __restrict__ accum, int npix, int spp,
                             float4* __restrict__ out)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    // the batch's first frame computes the same expression (equal bits)
    const float inv = 1.0f / (float)spp;
    const unsigned long long* a = accum + 3 * (size_t)p;
    out[p] = make_float4(unfix32(a[0]) * inv, unfix32(a[1]) * inv, unfix32(a[2]) * inv, 1.0f);
}

// batch accumulation: per job (blockIdx.y) and pixel, add this frame's
// radiance sums to the running sum and write the mean
__global__ void k_batch_reduce(const JobView* __restrict__ jobs, float4* const* __restrict__ sums,
                               float* const* __restrict__ outs, const int* __restrict__ frame)
{
    const JobView& J = jobs[blockIdx.y];
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= J.npix) return;
    const unsigned long long* a = J.accum + 3 * (size_t)p;
    float r = unfix32(a[0]), g = unfix32(a[1]), b = unfix32(a[2]);
    float4 acc = sums[blockIdx.y][p];
    acc.x += r; acc.y += g; acc.z += b;
    sums[blockIdx.y][p] = acc;
    float inv = 1.0f / ((float)(frame[0] + 1) * (float)J.spp);
    reinterpret_cast<float4*>(outs[blockIdx.y])[p] = make_float4(acc.x * inv, acc.y * inv, acc.z * inv, 1.0f);
}

__global__ void k_batch_next_frame(int* frame)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) frame[0] += 1;
}

// coarse occupancy: a bit per kCoarse^3 block of macrocells, set if any
// macrocell inside has its occupancy bit
__global__ void k_coarse_occupancy(const uint32_t* __restrict__ bits, int mx, int my, int mz,
                                   uint32_t* __restrict__ cbits, int cxn, int cyn, int czn)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int n = cxn * cyn * czn;
    bool on = false;
    if (c < n) {
        int bx = c % cxn, by = (c / cxn) % cyn, bz = c / (cxn * cyn);
        for (int z = bz * kCoarse; z < min(bz * kCoarse + kCoarse, mz) && !on; ++z)
            for (int y = by * kCoarse; y < min(by * kCoarse + kCoarse, my) && !on; ++y)
                for (int x = bx * kCoarse; x < min(bx * kCoarse + kCoarse, mx); ++x) {
                    long long id = ((long long)z * my + y) * mx + x;
                    if ((bits[id >> 5] >> (id & 31)) & 1u) { on = true; break; }
                }
    }
    unsigned b = __ballot_sync(0xffffffffu, on);
    if ((threadIdx.x & 31) == 0 && c < n) cbits[c >> 5] = b;
}

// occupancy bit per macrocell: majorant > 0
__global__ void k_occupancy(const float* __restrict__ mcmax, long long ncell, float sigma_scale,
                            uint32_t* __restrict__ bits)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool on = i < ncell && sigma_scale * mcmax[i] > 0.0f;
    unsigned b = __ballot_sync(0xffffffffu, on);
    if ((threadIdx.x & 31) == 0 && i < ncell) bits[i >> 5] = b;
}

// a batch job's clip box (one thread)
__global__ void k_clip_box(Majorants m, const int* __restrict__ occ, float* __restrict__ box)
{
    occupied_clip_box(m, occ, box);
}

// index box (lo xyz, hi xyz) of the macrocells whose occupancy bit is set;
// box starts as (INT_MAX.., -1..)
__global__ void k_occupied_box(const uint32_t* __restrict__ bits, int mx, int my, long long ncell, int* __restrict__ box)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell || !((bits[i >> 5] >> (i & 31)) & 1u)) return;
    const int cx = (int)(i % mx), cy = (int)((i / mx) % my), cz = (int)(i / ((long long)mx * my));
    atomicMin(box + 0, cx); atomicMin(box + 1, cy); atomicMin(box + 2, cz);
    atomicMax(box + 3, cx); atomicMax(box + 4, cy); atomicMax(box + 5, cz);
}

template <class S>
__global__ void __launch_bounds__(128) k_ea(S smp, Majorants m, CamDev cam, MedDev med, float4* __restrict__ out,
                                            DevStats* __restrict__ st)
{
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < med.tf_n; i += blockDim.x) s_tf[i] = med.tf[i];
    __syncthreads();
    const int npix = cam.w * cam.h;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    Walk w{};
    unsigned long long paths = 0;
    if (pix < npix) {
        Accessor acc;
        acc.reset();
        float3 o, d;
        camera_ray(cam, pix % cam.w, pix / cam.w, 0.5f, 0.5f, o, d);
        float cr = 0.f, cg = 0.f, cb = 0.f, T = 1.0f, tin, tout;
        if (clip_box(m, o, d, tin, tout)) {
            const float dt = med.step;
            const float tfm = (float)(med.tf_n - 1);
            const long long kmax = (long long)((tout - tin) / dt) + 2;
            for (long long k = 0; k < kmax; ++k) {
                float t = tin + ((float)k + 0.5f) * dt;
                if (t >= tout) break;
                float s = smp(o.x + t * d.x, o.y + t * d.y, o.z + t * d.z, acc);
                ++w.lookups;
                s = fminf(fmaxf(s, 0.0f), 1.0f);
                float x = s * tfm;
                int i0 = min((int)floorf(x), med.tf_n - 2);
                float f = x - (float)i0;
                float4 a = s_tf[i0], b = s_tf[i0 + 1];
                float r = lerpf(a.x, b.x, f), gg = lerpf(a.y, b.y, f), bb = lerpf(a.z, b.z, f), al = lerpf(a.w, b.w, f);
                float alpha = 1.0f - expf(-al * dt);
                float ta = T * alpha;
                cr += ta * r; cg += ta * gg; cb += ta * bb;
                T *= 1.0f - alpha;
                if (T < 1e-6f) break;
            }
        }
        out[pix] = make_float4(cr, cg, cb, 1.0f - T);
        paths = 1;
    }
    flush_stats(st, w, paths);
}

// the same marcher for samplers whose lookups are warp-collective: every lane
// stays in the loop until the whole warp is done and calls the lookup each
// step (look = false once its own ray has ended)
template <class S>
__global__ void __launch_bounds__(128) k_ea_collective(S smp, Majorants m, CamDev cam, MedDev med,
                                                       float4* __restrict__ out, DevStats* __restrict__ st)
{
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < med.tf_n; i += blockDim.x) s_tf[i] = med.tf[i];
    __syncthreads();
    const int npix = cam.w * cam.h;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    Walk w{};
    unsigned long long paths = 0;
    Accessor acc;
    acc.reset();
    float3 o = f3(0.f, 0.f, 0.f), d = f3(0.f, 0.f, 1.f);
    float cr = 0.f, cg = 0.f, cb = 0.f, T = 1.0f, tin = 0.f, tout = 0.f;
    bool active = false;
    long long kmax = 0;
    const float dt = med.step;
    const float tfm = (float)(med.tf_n - 1);
    if (pix < npix) {
        camera_ray(cam, pix % cam.w, pix / cam.w, 0.5f, 0.5f, o, d);
        active = clip_box(m, o, d, tin, tout);
        if (active) kmax = (long long)((tout - tin) / dt) + 2;
    }
    for (long long k = 0;; ++k) {
        float t = tin + ((float)k + 0.5f) * dt;
        if (active && (k >= kmax || t >= tout)) active = false;
        if (!__any_sync(0xffffffffu, active)) break;
        float s = smp.collective(active, o.x + t * d.x, o.y + t * d.y, o.z + t * d.z, acc);
        if (active) {
            ++w.lookups;
            s = fminf(fmaxf(s, 0.0f), 1.0f);
            float x = s * tfm;
            int i0 = min((int)floorf(x), med.tf_n - 2);
            float f = x - (float)i0;
            float4 a = s_tf[i0], b = s_tf[i0 + 1];
            float r = lerpf(a.x, b.x, f), gg = lerpf(a.y, b.y, f), bb = lerpf(a.z, b.z, f), al = lerpf(a.w, b.w, f);
            float alpha = 1.0f - expf(-al * dt);
            float ta = T * alpha;
            cr += ta * r; cg += ta * gg; cb += ta * bb;
            T *= 1.0f - alpha;
            if (T < 1e-6f) active = false;
        }
    }
    if (pix < npix) {
        out[pix] = make_float4(cr, cg, cb, 1.0f - T);
        paths = 1;
    }
    flush_stats(st, w, paths);
}

// ---------------------------------------------------------------- ISO surface
// The implicit ISO-surface marcher the paper uses for its ZFP comparison
// (Section 5), which it names without details.  Samples t_k = t_in + (k + 1/2)
// step as the EA marcher, inside = (f >= iso); the first change of inside
// between consecutive samples is halved kIsoBisect times and shaded with its
// normal n = -grad f / |grad f| (central differences, 1/2 voxel) as
// rgb = (n + 1) / 2, alpha 1.  Interval skipping: in a macrocell whose dilated
// [min, max] (which bounds the trilinear field over the cell) excludes iso,
// every sample has a known inside, so the march crosses the cell without a
// lookup and lands on the sample before its exit; the result is the plain
// march's.  Each loop iteration makes at most one lookup per lane, at one
// program point, so a warp-collective sampler works unchanged.
constexpr int kIsoBisect = 12;
enum { kIsoMarch = 0, kIsoHalve = 1, kIsoNormal = 2, kIsoDone = 3 };

// inside of every point of macrocell `id`: 1, 0, or -1 when iso is inside its range
__device__ __forceinline__ int iso_known(const Majorants& m, int id, float iso)
{
    if (__ldg(m.mcmin + id) >= iso) return 1;
    if (__ldg(m.mcmax + id) < iso) return 0;
    return -1;
}

template <class S>
__global__ void __launch_bounds__(128) k_iso(S smp, Majorants m, CamDev cam, MedDev med, float4* __restrict__ out,
                                             DevStats* __restrict__ st)
{
    const int npix = cam.w * cam.h;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    Walk w{};
    Accessor acc;
    acc.reset();
    float3 o = f3(0.f, 0.f, 0.f), d = f3(0.f, 0.f, 1.f);
    float tin = 0.f, tout = 0.f;
    int phase = kIsoDone;
    if (pix < npix) {
        camera_ray(cam, pix % cam.w, pix / cam.w, 0.5f, 0.5f, o, d);
        if (clip_box(m, o, d, tin, tout)) phase = kIsoMarch;
    }
    const float dt = med.step, iso = med.iso;
    const long long kmax = phase == kIsoMarch ? (long long)((tout - tin) / dt) + 2 : 0;
    Dda dda;
    int cell_id = 0, known = -1;
    float texit = 0.f;
    bool have_cell = false;
    if (phase == kIsoMarch) {
        dda.init(m, o, d, tin, tout);
        have_cell = dda.cell(m, cell_id, texit);
        if (have_cell) known = iso_known(m, cell_id, iso);
    }
    int guard = m.mx + m.my + m.mz + 8;      // DDA cells a ray may cross
    long long k = 0;
    int prev = -1, halvings = 0, q = 0;
    float t = 0.f, t_prev = 0.f, a = 0.f, b = 0.f, th = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    float4 color = make_float4(0.f, 0.f, 0.f, 0.f);
    for (;;) {
        bool look = false;
        float3 p = o;
        if (phase == kIsoMarch) {
            for (;;) {
                if (k >= kmax) { phase = kIsoDone; break; }
                t = tin + ((float)k + 0.5f) * dt;
                if (t >= tout) { phase = kIsoDone; break; }
                while (have_cell && t >= texit) {
                    if (--guard < 0) { w.flags |= kErrDdaSteps; have_cell = false; break; }
                    dda.advance(m, o, texit);
                    have_cell = dda.cell(m, cell_id, texit);
                    if (have_cell) known = iso_known(m, cell_id, iso);
                }
                if (!have_cell) known = -1;      // past the cell grid by rounding: look the sample up
                if (known < 0) {
                    look = true;
                    p = f3(o.x + t * d.x, o.y + t * d.y, o.z + t * d.z);
                    break;
                }
                if (prev >= 0 && known != prev) { a = t_prev; b = t; halvings = 0; phase = kIsoHalve; break; }
                // the cell's later samples share this inside: go on from the last one before its exit
                prev = known;
                t_prev = t;
                long long kn = (long long)floorf((texit - tin) / dt - 0.5f);
                if (kn > k + 1) {
                    k = kn;
                    t_prev = tin + ((float)(kn - 1) + 0.5f) * dt;
                } else {
                    ++k;
                }
            }
        }
        if (phase == kIsoHalve) {
            const float mid = 0.5f * (a + b);
            p = f3(o.x + mid * d.x, o.y + mid * d.y, o.z + mid * d.z);
            look = true;
        } else if (phase == kIsoNormal) {
            p = f3(o.x + th * d.x, o.y + th * d.y, o.z + th * d.z);
            const float h = (q & 1) ? -0.5f : 0.5f;
            if (q < 2) p.x += h; else if (q < 4) p.y += h; else p.z += h;
            look = true;
        }
        float f = 0.0f;
        if constexpr (S::kCollective) {
            __syncwarp();
            f = smp.collective(look, p.x, p.y, p.z, acc);
        } else {
            if (look) f = smp(p.x, p.y, p.z, acc);
        }
        if (look) {
            ++w.lookups;
            const int in = f >= iso ? 1 : 0;
            if (phase == kIsoMarch) {
                if (prev >= 0 && in != prev) { a = t_prev; b = t; halvings = 0; phase = kIsoHalve; }
                else { prev = in; t_prev = t; ++k; }
            } else if (phase == kIsoHalve) {
                const float mid = 0.5f * (a + b);
                if (in == prev) a = mid; else b = mid;
                if (++halvings == kIsoBisect) { th = 0.5f * (a + b); q = 0; phase = kIsoNormal; }
            } else {
                const float sg = (q & 1) ? -f : f;
                if (q < 2) gx += sg; else if (q < 4) gy += sg; else gz += sg;
                if (++q == 6) {
                    const float gl = sqrtf(gx * gx + gy * gy + gz * gz);
                    float3 n = gl > 0.0f ? f3(-gx / gl, -gy / gl, -gz / gl) : f3(-d.x, -d.y, -d.z);
                    color = make_float4(0.5f * (n.x + 1.0f), 0.5f * (n.y + 1.0f), 0.5f * (n.z + 1.0f), 1.0f);
                    phase = kIsoDone;
                }
            }
        }
        if (__all_sync(0xffffffffu, phase == kIsoDone)) break;
    }
    if (pix < npix) out[pix] = color;
    flush_stats(st, w, pix < npix ? 1ull : 0ull);
}

unsigned blocks_for(long long n, int t) { return (unsigned)std::max<long long>(1, (n + t - 1) / t); }

}  // namespace
}  // namespace vdbc

namespace vdbc {
namespace {

vdbc_status check_camera(const vdbc_camera* c)
{
    if (!c) return set_error(VDBC_ERR_INVALID_ARG, "camera is null");
    if (c->kind != VDBC_CAM_ORTHO && c->kind != VDBC_CAM_PINHOLE)
        return set_error(VDBC_ERR_INVALID_ARG, "camera kind %d unknown", c->kind);
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
        return set_error(VDBC_ERR_INVALID_ARG, "image size %dx%d outside 1..16384", c->width, c->height);
    if (!(c->fovy_or_height > 0.0) || !std::isfinite(c->fovy_or_height) ||
        (c->kind == VDBC_CAM_PINHOLE && !(c->fovy_or_height < 180.0)))
        return set_error(VDBC_ERR_INVALID_ARG, "bad field of view / ortho height");
    // a basis must exist: finite vectors, look != eye, up not along the view
    double f[3], fl = 0.0, ul = 0.0, cl = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(c->eye[a]) || !std::isfinite(c->look[a]) || !std::isfinite(c->up[a]))
            return set_error(VDBC_ERR_INVALID_ARG, "camera vectors must be finite");
        f[a] = (double)c->look[a] - (double)c->eye[a];
        fl += f[a] * f[a];
        ul += (double)c->up[a] * c->up[a];
    }
    const double cr[3] = {f[1] * c->up[2] - f[2] * c->up[1], f[2] * c->up[0] - f[0] * c->up[2],
                          f[0] * c->up[1] - f[1] * c->up[0]};
    for (double x : cr) cl += x * x;
    if (!(fl > 0.0) || !(cl > 1e-24 * fl * ul))
        return set_error(VDBC_ERR_INVALID_ARG, "camera: look must differ from eye and up must not lie along the view");
    return VDBC_OK;
}

// camera basis in FP64 on the host, rounded once for the kernel
CamDev make_cam(const vdbc_camera* c, const int dims[3])
{
    double M = (double)std::max(dims[0], std::max(dims[1], dims[2]));
    double f[3] = {c->look[0] - c->eye[0], c->look[1] - c->eye[1], c->look[2] - c->eye[2]};
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (double& x : f) x /= fl;
    double r[3] = {f[1] * c->up[2] - f[2] * c->up[1], f[2] * c->up[0] - f[0] * c->up[2], f[0] * c->up[1] - f[1] * c->up[0]};
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (double& x : r) x /= rl;
    double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    double aspect = (double)c->width / (double)c->height;
    CamDev d;
    d.kind = c->kind;
    d.w = c->width;
    d.h = c->height;
    d.fwd = make_float3((float)f[0], (float)f[1], (float)f[2]);
    d.right = make_float3((float)r[0], (float)r[1], (float)r[2]);
    d.up = make_float3((float)u[0], (float)u[1], (float)u[2]);
    d.eye = make_float3((float)(c->eye[0] * M - 0.5), (float)(c->eye[1] * M - 0.5), (float)(c->eye[2] * M - 0.5));
    if (c->kind == VDBC_CAM_ORTHO) {
        double h = 0.5 * c->fovy_or_height;
        d.sxs = (float)(h * aspect * M);
        d.sys = (float)(h * M);
    } else {
        double th = std::tan(0.5 * c->fovy_or_height * 3.14159265358979323846 / 180.0);
        d.sxs = (float)(th * aspect);
        d.sys = (float)th;
    }
    return d;
}

struct MedHost {
    MedDev dev;
    float4* tf_dev = nullptr;
};

vdbc_status make_med(const vdbc_medium* m, const int dims[3], int spp, cudaStream_t s, MedHost& out)
{
    if (!m) return set_error(VDBC_ERR_INVALID_ARG, "medium is null");
    MedDev& d = out.dev;
    std::memset(&d, 0, sizeof(d));
    d.mode = m->mode;
    double M = (double)std::max(dims[0], std::max(dims[1], dims[2]));
    if (m->mode == VDBC_MODE_EA) {
        if (!m->tf_rgba || m->tf_n < 2 || m->tf_n > 2048)
            return set_error(VDBC_ERR_INVALID_ARG, "EA needs a transfer function of 2..2048 entries");
        if (!(m->step > 0.0f)) return set_error(VDBC_ERR_INVALID_ARG, "EA step must be > 0");
        if (spp != 1) return set_error(VDBC_ERR_INVALID_ARG, "EA renders 1 sample per pixel");
        d.tf_n = m->tf_n;
        d.step = m->step;
        VDBC_TRY(dev_alloc(reinterpret_cast<void**>(&out.tf_dev), (size_t)m->tf_n * 16, s));
        VDBC_CUDA(cudaMemcpyAsync(out.tf_dev, m->tf_rgba, (size_t)m->tf_n * 16, cudaMemcpyHostToDevice, s));
        d.tf = out.tf_dev;
    } else if (m->mode == VDBC_MODE_PT) {
        if (spp < 1 || spp > 65536) return set_error(VDBC_ERR_INVALID_ARG, "spp %d outside 1..65536", spp);
        if (m->max_bounces < 1 || m->max_bounces > 4096)
            return set_error(VDBC_ERR_INVALID_ARG, "max_bounces %d outside 1..4096", m->max_bounces);
        if (!(m->density_scale >= 0.0f) || !std::isfinite(m->density_scale) ||
            !(m->albedo >= 0.0f && m->albedo <= 1.0f) || !(m->g > -1.0f && m->g < 1.0f))
            return set_error(VDBC_ERR_INVALID_ARG, "medium parameters out of range");
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(m->sun_dir[a]) || !std::isfinite(m->sun_rad[a]) || !std::isfinite(m->env_rad[a]))
                return set_error(VDBC_ERR_INVALID_ARG, "sun and environment must be finite");
        double sl = std::sqrt((double)m->sun_dir[0] * m->sun_dir[0] + (double)m->sun_dir[1] * m->sun_dir[1] +
                              (double)m->sun_dir[2] * m->sun_dir[2]);
        if (!(sl > 0.0)) return set_error(VDBC_ERR_INVALID_ARG, "sun_dir must be nonzero");
        d.sigma_scale = (float)((double)m->density_scale / M);
        d.albedo = m->albedo;
        d.g = m->g;
        d.max_bounces = m->max_bounces;
        d.sun_dir = make_float3((float)(m->sun_dir[0] / sl), (float)(m->sun_dir[1] / sl), (float)(m->sun_dir[2] / sl));
        d.sun_rad = make_float3(m->sun_rad[0], m->sun_rad[1], m->sun_rad[2]);
        d.env_rad = make_float3(m->env_rad[0], m->env_rad[1], m->env_rad[2]);
    } else if (m->mode == VDBC_MODE_ISO) {
        if (!(m->step > 0.0f)) return set_error(VDBC_ERR_INVALID_ARG, "ISO step must be > 0");
        if (!std::isfinite(m->iso)) return set_error(VDBC_ERR_INVALID_ARG, "ISO value must be finite");
        if (spp != 1) return set_error(VDBC_ERR_INVALID_ARG, "ISO renders 1 sample per pixel");
        d.step = m->step;
        d.iso = m->iso;
    } else {
        return set_error(VDBC_ERR_INVALID_ARG, "medium mode %d unknown", m->mode);
    }
    return VDBC_OK;
}

// SMs of the current device (a host query, no device work)
int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

constexpr int kPtThreads = 256;

// The coarse level (empty kCoarse^3 blocks of macrocells crossed in one DDA
// step) is a compile-time variant of the tracker.  With the level compiled out
// the tracker fits 4 blocks per SM, and the uniform grid wins at every measured
// cell size on the 512^3 medium (8^3: 74.5 against 90.2 ms; 48^3: 30.1 against
// 47.9 ms), so it is off unless VDBC_PT_COARSE=1 (the batch tuner tries both).
bool coarse_skipping(int)
{
    const char* e = std::getenv("VDBC_PT_COARSE");
    return e && e[0] == '1';
}

// items a warp takes from the work counter at once.  A chunk is consecutive
// 8x4 pixel tiles of one sample, which the warp's lanes take in order: larger
// chunks keep a warp's successive paths next to each other in the image (and
// so in the volume), smaller ones leave each warp a shorter tail of paths when
// the counter runs out.  The chunk is the largest of 32, 64 and 128 items that
// still gives every resident warp 200 chunks, so that its last one is under
// half a percent of its share.  Measured (ms): the 1920x1080 x 64 spp frame of
// the full-scale cloud (27,000 items a warp) 37.65 at 32, 35.75 at 64, 34.79 at
// 128, 34.82 at 192, 35.14 at 256; the 1024^2 x 16 spp frame of the 512^3
// medium (3,400 items a warp) 8.32 at 32, 8.34 at 64, 8.61 at 128, 9.31 at 256.
// VDBC_PT_CHUNK overrides.
int work_chunk(unsigned long long items, long long resident_warps)
{
    if (const char* e = std::getenv("VDBC_PT_CHUNK")) {
        int c = std::atoi(e);
        return c < 32 ? 32 : c;
    }
    const unsigned long long w = (unsigned long long)std::max<long long>(resident_warps, 1);
    int c = 32;
    while (c < 128 && items >= 200ull * w * (unsigned long long)(2 * c)) c *= 2;
    return c;
}
constexpr size_t kSmemBitsMax = 96 * 1024;
// dynamic shared memory a tracker block may take for occupancy words and the
// majorant table together, leaving room for four blocks per SM
constexpr size_t kSmemMajMax = 40 * 1024;
// 1: stage the majorant table in shared memory when it fits (kSmemMajMax)
#ifndef VDBC_PT_SMEM_MAJ
#define VDBC_PT_SMEM_MAJ 1
#endif

// the job's constants for the tracker (bits are filled in by the caller)
JobView make_job(const Majorants& mj, const CamDev& cam, const MedDev& med, int spp, uint64_t seed,
                 unsigned long long* accum)
{
    JobView j;
    std::memset(&j, 0, sizeof(j));
    j.m = mj;
    j.cam = cam;
    j.med = med;
    j.cx_n = (mj.mx + kCoarse - 1) / kCoarse;
    j.cy_n = (mj.my + kCoarse - 1) / kCoarse;
    j.accum = accum;
    j.npix = cam.w * cam.h;
    j.spp = spp;
    j.tiles_x = (cam.w + 7) / 8;
    j.k0 = (uint32_t)seed;
    j.k1 = (uint32_t)(seed >> 32);
    j.sample_base = 0;
    j.item_begin = 0;
    j.items = (unsigned long long)spp * (unsigned long long)j.tiles_x * (unsigned long long)((cam.h + 3) / 4) * 32ull;
    j.per = (uint32_t)((unsigned long long)j.tiles_x * (unsigned long long)((cam.h + 3) / 4) * 32ull);
    j.items32 = j.items < (1ull << 32) ? 1 : 0;
    j.div_per.init(j.per);
    j.div_tiles_x.init((uint32_t)j.tiles_x);
    // Work items ordered by tile first: a tile's 32 pixels for every sample in
    // turn, so that the warps working at one time start their paths from few
    // pixels and read the same leaves (full-scale cloud frame 21.99 against
    // 23.97 ms ordered by sample first, 512^3 frame 6.55 against 6.99; the
    // per-pixel sums, and so the images, are the same).  VDBC_PT_ORDER=sample
    // restores the sample-first order.  Tiles visited in strips of 8 or 32
    // tile rows, each strip column by column, instead of row by row measured
    // 22.3 and 21.8 against 22.0 ms on the cloud, 6.65 and 6.60 against 6.55
    // on the 512^3 frame.
    const char* order = std::getenv("VDBC_PT_ORDER");
    j.tile_major = (order && std::strcmp(order, "sample") == 0) ? 0 : 1;
    j.spp32 = (uint32_t)((unsigned long long)spp * 32ull);
    if (j.items32) j.div_spp32.init(j.spp32);
    return j;
}

template <class S, bool kUseCoarse, bool kPhased = false, int kBlocks = pt_min_blocks<S, kUseCoarse>()>
vdbc_status launch_pt_t(const S& smp, const JobView& job, const uint32_t* bits, int nwords, int ncwords,
                        DevStats* stats, int chunk, cudaStream_t s)
{
    int smem_words = std::min<int>(nwords + ncwords, (int)(kSmemBitsMax / 4));
    if (smem_words < ncwords) smem_words = 0;
    // the majorants go to shared memory when the whole table fits beside the
    // occupancy words within kSmemMajMax: the walk then reads a found cell's
    // majorant there instead of from global memory
    const long long ncell = (long long)job.m.mx * job.m.my * job.m.mz;
    int smaj_cells = 0;
#if VDBC_PT_SMEM_MAJ
    if (smem_words == nwords + ncwords && (size_t)(smem_words + ncell) * 4 <= kSmemMajMax) smaj_cells = (int)ncell;
#endif
    size_t smem = (size_t)(smem_words + smaj_cells) * 4;
    auto kern = k_pt<S, kUseCoarse, kPhased, kBlocks>;
    if (smem > 48 * 1024) VDBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    VDBC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPtThreads, smem));
    if (per_sm < 1) per_sm = 1;
    long long want = (long long)((job.items + kPtThreads - 1) / kPtThreads);
    long long blocks = std::min<long long>((long long)sm_count() * per_sm, std::max<long long>(want, 1));
    if (chunk <= 0) chunk = work_chunk(job.items, blocks * (kPtThreads / 32));
    KLAUNCH(kern<<<(unsigned)blocks, kPtThreads, smem, s>>>(smp, job, bits, nwords, ncwords, smem_words, smaj_cells,
                                                            stats, chunk));
    VDBC_CUDA(cudaGetLastError());
    return VDBC_OK;
}

template <class S>
vdbc_status launch_pt(const S& smp, const JobView& job, const uint32_t* bits, int nwords, int ncwords,
                      DevStats* stats, int chunk, bool coarse, cudaStream_t s)
{
    if constexpr (!S::kCollective) {
        if (coarse) return launch_pt_t<S, true>(smp, job, bits, nwords, ncwords, stats, chunk, s);
    }
    if constexpr (std::is_same<S, VdbSamplerT<0>>::value) {
        // VDBC_PT_PHASED=1: the one-block-per-iteration loop, for measuring it
        // against the default.  Measured slower: 10.01 against 8.57 ms on the
        // 512^3 frame, 47.83 against 44.01 ms on the cloud (the warp then runs
        // more iterations per path than the lanes it regroups save)
        static const bool phased = [] { const char* e = std::getenv("VDBC_PT_PHASED"); return e && e[0] == '1'; }();
        if (phased) return launch_pt_t<S, false, true>(smp, job, bits, nwords, ncwords, stats, chunk, s);
    }
    if constexpr (S::kCollective) {
        // learned grids: VDBC_PT_LEARNED = p2 / p3 (one block per iteration at
        // 2 or 3 blocks per SM), f3 (fused at 3 blocks), for measuring them
        // against the default (fused, 2 blocks).  Measured on the 994x676x1225
        // cloud's learned grid at 1920x1080 x 32 spp: 74.5 ms (default) against
        // 82.6 (p2), 89.2 (p3) and 81.3 (f3: 80 registers with spills)
        static const int variant = [] {
            const char* e = std::getenv("VDBC_PT_LEARNED");
            if (!e || std::strlen(e) != 2) return 0;
            return (e[0] == 'p' ? 10 : 0) + (e[1] - '0');
        }();
        if (variant == 12) return launch_pt_t<S, false, true, 2>(smp, job, bits, nwords, ncwords, stats, chunk, s);
        if (variant == 13) return launch_pt_t<S, false, true, 3>(smp, job, bits, nwords, ncwords, stats, chunk, s);
        if (variant == 3) return launch_pt_t<S, false, false, 3>(smp, job, bits, nwords, ncwords, stats, chunk, s);
    }
    return launch_pt_t<S, false>(smp, job, bits, nwords, ncwords, stats, chunk, s);
}

// The grid's node tables (root, upper and lower nodes, tiles: the front of
// its block, before the leaves) as a persisting L2 window on the render's
// stream while the path tracer runs: every tree descent reads them.
// VDBC_L2_NODES=1 turns it on; the window is cleared after the launch.  Off
// by default: measured no faster (8.63 against 8.57 ms on the 512^3 frame,
// whose 54 MB grid L2 holds anyway; 44.45 against 44.01 ms on the cloud, whose
// node tables stay hot in L2 without the window).
template <class S>
struct NodeWindow {
    static void set(const S&, cudaStream_t) {}
    static void clear(cudaStream_t) {}
};

template <int P, int D, int T>
struct NodeWindow<VdbSamplerT<P, D, T>> {
    static bool enabled()
    {
        static const bool on = [] {
            const char* e = std::getenv("VDBC_L2_NODES");
            if (!(e && e[0] == '1')) return false;
            int dev = 0, maxp = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess || maxp <= 0) {
                cudaGetLastError();
                return false;
            }
            // a context limit: it ends with this process
            if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)maxp) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            return true;
        }();
        return on;
    }
    static void set(const VdbSamplerT<P, D, T>& smp, cudaStream_t s)
    {
        if (!enabled()) return;
        cudaStreamAttrValue a{};
        a.accessPolicyWindow.base_ptr = const_cast<uint32_t*>(smp.g.root);
        a.accessPolicyWindow.num_bytes = (size_t)(static_cast<const char*>(smp.g.leaves) -
                                                  reinterpret_cast<const char*>(smp.g.root));
        a.accessPolicyWindow.hitRatio = 1.0f;
        a.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        a.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        if (cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &a) != cudaSuccess) cudaGetLastError();
    }
    static void clear(cudaStream_t s)
    {
        if (!enabled()) return;
        cudaStreamAttrValue a{};
        a.accessPolicyWindow.num_bytes = 0;
        if (cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &a) != cudaSuccess) cudaGetLastError();
    }
};

template <class S>
vdbc_status launch(const S& smp, const Majorants& mj, const CamDev& cam, const MedDev& med, int spp, uint64_t seed,
                   float4* out, DevStats* stats, cudaStream_t s)
{
    long long npix = (long long)cam.w * cam.h;
    VDBC_CUDA(cudaMemsetAsync(stats, 0, sizeof(DevStats), s));
    if (med.mode == VDBC_MODE_ISO) {
        if (!mj.mcmin) return set_error(VDBC_ERR_INVALID_ARG, "ISO needs the macrocell minima");
        record_kernel_start(stats, s);
        KLAUNCH(k_iso<S><<<blocks_for(npix, 128), 128, 0, s>>>(smp, mj, cam, med, out, stats));
        record_kernel_stop(stats, s);
        VDBC_CUDA(cudaGetLastError());
        return VDBC_OK;
    }
    if (med.mode == VDBC_MODE_EA) {
        record_kernel_start(stats, s);
        if constexpr (S::kCollective)
            KLAUNCH(k_ea_collective<S><<<blocks_for(npix, 128), 128, (size_t)med.tf_n * 16, s>>>(smp, mj, cam, med, out,
                                                                                                stats));
        else
            KLAUNCH(k_ea<S><<<blocks_for(npix, 128), 128, (size_t)med.tf_n * 16, s>>>(smp, mj, cam, med, out, stats));
        record_kernel_stop(stats, s);
        VDBC_CUDA(cudaGetLastError());
        return VDBC_OK;
    }
    long long ncell = (long long)mj.mx * mj.my * mj.mz;
    int nwords = (int)((ncell + 31) / 32);
    int cxn = (mj.mx + kCoarse - 1) / kCoarse, cyn = (mj.my + kCoarse - 1) / kCoarse, czn = (mj.mz + kCoarse - 1) / kCoarse;
    int ncwords = (cxn * cyn * czn + 31) / 32;
    uint32_t* bits = nullptr;
    unsigned long long* accum = nullptr;
    VDBC_TRY(dev_alloc(reinterpret_cast<void**>(&bits), (size_t)(nwords + ncwords + 8) * 4, s));
    vdbc_status st = dev_alloc(reinterpret_cast<void**>(&accum), (size_t)npix * 3 * sizeof(unsigned long long), s);
    if (st != VDBC_OK) { dev_free(bits, s); return st; }
    VDBC_CUDA(cudaMemsetAsync(accum, 0, (size_t)npix * 3 * sizeof(unsigned long long), s));
    KLAUNCH(k_occupancy<<<blocks_for(ncell, 256), 256, 0, s>>>(mj.mcmax, ncell, med.sigma_scale, bits));
    const bool coarse = !S::kCollective && coarse_skipping(mj.mc);
    if (coarse) {
        KLAUNCH(k_coarse_occupancy<<<blocks_for((long long)cxn * cyn * czn, 256), 256, 0, s>>>(
            bits, mj.mx, mj.my, mj.mz, bits + nwords, cxn, cyn, czn));
    } else {
        VDBC_CUDA(cudaMemsetAsync(bits + nwords, 0xff, (size_t)ncwords * 4, s));   // every block "occupied"
    }
    JobView job = make_job(mj, cam, med, spp, seed, accum);
    // (rays walk only the box of the occupied macrocells: 12.08 -> 8.57 ms on the
    // 1024^2 x 16 spp frame of the 512^3 medium, whose occupied cells fill a
    // quarter of its grid; 58.89 -> 44.01 ms on the cloud; VDBC_PT_BOX=0 turns it off)
    static const bool use_box = [] { const char* e = std::getenv("VDBC_PT_BOX"); return !(e && e[0] == '0'); }();
    if (use_box) {
        // the clip box of the occupied macrocells, after the occupancy words
        int* box = reinterpret_cast<int*>(bits + nwords + ncwords);
        VDBC_CUDA(cudaMemsetAsync(box, 0x7f, 3 * sizeof(int), s));
        VDBC_CUDA(cudaMemsetAsync(box + 3, 0xff, 3 * sizeof(int), s));
        KLAUNCH(k_occupied_box<<<blocks_for(ncell, 256), 256, 0, s>>>(bits, mj.mx, mj.my, ncell, box));
        job.occ_box = box;
    }
    NodeWindow<S>::set(smp, s);
    record_kernel_start(stats, s);
    st = launch_pt<S>(smp, job, bits, nwords, ncwords, stats, 0, coarse, s);
    record_kernel_stop(stats, s);
    NodeWindow<S>::clear(s);
    if (st == VDBC_OK) {
        KLAUNCH(k_pt_resolve<<<blocks_for(npix, 256), 256, 0, s>>>(accum, (int)npix, spp, out));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_status(e, "k_pt_resolve");
    }
    dev_free(accum, s);
    dev_free(bits, s);
    return st;
}

template <class S>
vdbc_status render_common(const S& smp, const Majorants& mj, const int dims[3], DevStats* stats,
                          const vdbc_camera* camera, const vdbc_medium* medium, int32_t spp, uint64_t seed,
                          float* rgba_out, int32_t out_on_device, void* stream)
{
    if (!rgba_out) return set_error(VDBC_ERR_INVALID_ARG, "rgba_out is null");
    VDBC_TRY(check_camera(camera));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MedHost mh;
    vdbc_status st = make_med(medium, dims, spp, s, mh);
    if (st != VDBC_OK) { if (mh.tf_dev) dev_free(mh.tf_dev, s); return st; }
    CamDev cam = make_cam(camera, dims);
    size_t img = (size_t)camera->width * camera->height * 16;
    float4* dst = reinterpret_cast<float4*>(rgba_out);
    void* tmp = nullptr;
    if (!out_on_device) {
        st = dev_alloc(&tmp, img, s);
        if (st != VDBC_OK) { if (mh.tf_dev) dev_free(mh.tf_dev, s); return st; }
        dst = static_cast<float4*>(tmp);
    }
    st = launch(smp, mj, cam, mh.dev, spp, seed, dst, stats, s);
    if (mh.tf_dev) dev_free(mh.tf_dev, s);
    if (st == VDBC_OK && !out_on_device) {
        cudaError_t e = cudaMemcpyAsync(rgba_out, dst, img, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = cuda_status(e, "render D2H");
        if (st == VDBC_OK) st = wait_stream(s);
        if (st == VDBC_OK) {
            DevStats h;
            e = cudaMemcpy(&h, stats, sizeof(h), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = cuda_status(e, "render stats");
            else if (h.error_flags) st = set_error(VDBC_ERR_DEVICE_FLAG, "render hit a loop bound (flags %llx)", h.error_flags);
        }
    }
    if (tmp) dev_free(tmp, s);
    return st;
}

__global__ void k_dense_macrocells(const float* __restrict__ v, int nx, int ny, int nz, int mc, int mx, int my,
                                   float* __restrict__ mcmin, float* __restrict__ mcmax, long long ncell)
{
    long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= ncell) return;
    int cx = (int)(c % mx), cy = (int)((c / mx) % my), cz = (int)(c / ((long long)mx * my));
    int x0 = max(cx * mc - 1, 0), x1 = min(cx * mc + mc, nx - 1);
    int y0 = max(cy * mc - 1, 0), y1 = min(cy * mc + mc, ny - 1);
    int z0 = max(cz * mc - 1, 0), z1 = min(cz * mc + mc, nz - 1);
    int ex = x1 - x0 + 1, ey = y1 - y0 + 1, ez = z1 - z0 + 1;
    float vmin = INFINITY, vmax = -INFINITY;
    for (int q = lane; q < ex * ey * ez; q += 32) {
        int x = x0 + q % ex, y = y0 + (q / ex) % ey, z = z0 + q / (ex * ey);
        float val = __ldg(v + ((size_t)z * ny + y) * nx + x);
        vmin = fminf(vmin, val);
        vmax = fmaxf(vmax, val);
    }
    for (int o = 16; o > 0; o >>= 1) {
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if (lane == 0) { mcmin[c] = vmin; mcmax[c] = vmax; }
}

}  // namespace
}  // namespace vdbc

using namespace vdbc;

extern "C" vdbc_status vdbc_render(const vdbc_grid* grid, const vdbc_camera* camera, const vdbc_medium* medium,
                                   int32_t spp, uint64_t seed, float* rgba_out, int32_t out_on_device,
                                   void* stream)
{
    clear_error();
    if (!grid) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_render: grid is null");
    const GridView& g = grid->view;
    Majorants mj{g.mcmax, g.mc, g.mx, g.my, g.mz, g.nx, g.ny, g.nz, g.mcmin};
    if (g.payload == VDBC_LEARNED)
        return render_common(LearnedSampler{g}, mj, grid->info.dims, grid->stats, camera, medium, spp, seed, rgba_out,
                             out_on_device, stream);
    if (g.payload == VDBC_FP16)
        return render_common(VdbSamplerT<1>{g}, mj, grid->info.dims, grid->stats, camera, medium, spp, seed, rgba_out,
                             out_on_device, stream);
    if (g.payload == VDBC_FP8)
        return render_common(VdbSamplerT<2>{g}, mj, grid->info.dims, grid->stats, camera, medium, spp, seed, rgba_out,
                             out_on_device, stream);
    // VDBC_PT_LOOKUP = <depth><mode> picks another accessor depth (1, 2) and
    // stencil mode (11, 12, 22, 24; the default is depth 1, mode 5) for FP32
    // grids, for measuring them against each other
    const char* lk = std::getenv("VDBC_PT_LOOKUP");
    if (lk && std::strcmp(lk, "11") == 0)
        return render_common(VdbSamplerT<0, 1, 1>{g}, mj, grid->info.dims, grid->stats, camera, medium, spp, seed,
                             rgba_out, out_on_device, stream);
    if (lk && std::strcmp(lk, "12") == 0)
        return render_common(VdbSamplerT<0, 1, 2>{g}, mj, grid->info.dims, grid->stats, camera, medium, spp, seed,
                             rgba_out, out_on_device, stream);
    if (lk && std::strcmp(lk, "22") == 0)
        return render_common(VdbSamplerT<0, 2, 2>{g}, mj, grid->info.dims, grid->stats, camera, medium, spp, seed,
                             rgba_out, out_on_device, stream);
    if (lk && std::strcmp(lk, "24") == 0)
        return render_common(VdbSamplerT<0, 2, 4>{g}, mj, grid->info.dims, grid->stats, camera, medium, spp, seed,
                             rgba_out, out_on_device, stream);
    return render_common(VdbSamplerT<0>{g}, mj, grid->info.dims, grid->stats, camera, medium, spp, seed, rgba_out,
                         out_on_device, stream);
}

extern "C" vdbc_status vdbc_render_stats_get(const vdbc_grid* grid, void* stream, vdbc_render_stats* out)
{
    clear_error();
    if (!grid || !out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_render_stats_get: null argument");
    VDBC_TRY(wait_stream(static_cast<cudaStream_t>(stream)));
    DevStats h;
    VDBC_CUDA(cudaMemcpy(&h, grid->stats, sizeof(h), cudaMemcpyDeviceToHost));
    out->lookups = h.lookups;
    out->paths = h.paths;
    out->error_flags = h.error_flags;
    for (int k = 0; k < kNumEvents; ++k) out->events[k] = h.ev[k];
    out->kernel_ms = kernel_ms_of(grid->stats);
    out->reserved = 0;
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_volume_create(const vdbc_dense* in, int32_t filter, int32_t macrocell, void* stream,
                                          vdbc_volume** out)
{
    clear_error();
    if (!in || !in->data || !out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_volume_create: null argument");
    *out = nullptr;
    for (int a = 0; a < 3; ++a)
        if (in->dims[a] < 1 || in->dims[a] > kMaxDim)
            return set_error(VDBC_ERR_INVALID_ARG, "vdbc_volume_create: dims[%d] outside 1..%d", a, kMaxDim);
    if (filter != VDBC_FILTER_TEXTURE && filter != VDBC_FILTER_LINEAR)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_volume_create: unknown filter %d", filter);
    int mc = macrocell == 0 ? 8 : macrocell;
    if (mc < 1 || mc > kMaxMacrocell)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_volume_create: macrocell outside 1..%d", kMaxMacrocell);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    vdbc_volume* v = new vdbc_volume();
    for (int a = 0; a < 3; ++a) v->dims[a] = in->dims[a];
    v->filter = filter;
    v->macrocell = mc;
    for (int a = 0; a < 3; ++a) v->mcdims[a] = (in->dims[a] + mc - 1) / mc;
    size_t nvox = (size_t)in->dims[0] * in->dims[1] * in->dims[2];
    long long ncell = (long long)v->mcdims[0] * v->mcdims[1] * v->mcdims[2];
    auto fail = [&](vdbc_status st) { vdbc_volume_free(v); return st; };
    // a device copy is needed for the majorants and the linear form
    float* lin = nullptr;
    vdbc_status st = dev_alloc(reinterpret_cast<void**>(&lin), nvox * 4, s);
    if (st != VDBC_OK) return fail(st);
    cudaError_t e = cudaMemcpyAsync(lin, in->data, nvox * 4, in->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { dev_free(lin, s); return fail(cuda_status(e, "vdbc_volume_create copy")); }
    st = dev_alloc(reinterpret_cast<void**>(&v->mcmin), (size_t)ncell * 4, s);
    if (st == VDBC_OK) st = dev_alloc(reinterpret_cast<void**>(&v->mcmax), (size_t)ncell * 4, s);
    if (st == VDBC_OK) st = dev_alloc(reinterpret_cast<void**>(&v->stats), sizeof(DevStats), s);
    if (st != VDBC_OK) { dev_free(lin, s); return fail(st); }
    KLAUNCH(k_dense_macrocells<<<blocks_for(ncell * 32, 256), 256, 0, s>>>(lin, in->dims[0], in->dims[1], in->dims[2], mc,
                                                                   v->mcdims[0], v->mcdims[1], v->mcmin, v->mcmax,
                                                                   ncell));
    e = cudaGetLastError();
    if (e != cudaSuccess) { dev_free(lin, s); return fail(cuda_status(e, "vdbc_volume_create majorants")); }
    if (filter == VDBC_FILTER_LINEAR) {
        v->linear = lin;
    } else {
        cudaChannelFormatDesc ch = cudaCreateChannelDesc<float>();
        cudaExtent ext = make_cudaExtent(in->dims[0], in->dims[1], in->dims[2]);
        if (fault_injected("oom")) { dev_free(lin, s); return fail(set_error(VDBC_ERR_OOM, "3D array refused (VDBC_FAULT=oom)")); }
        e = cudaMalloc3DArray(&v->array, &ch, ext);
        if (e != cudaSuccess) { dev_free(lin, s); return fail(cuda_status(e, "cudaMalloc3DArray")); }
        cudaMemcpy3DParms p{};
        p.srcPtr = make_cudaPitchedPtr(lin, (size_t)in->dims[0] * 4, in->dims[0], in->dims[1]);
        p.dstArray = v->array;
        p.extent = ext;
        p.kind = cudaMemcpyDeviceToDevice;
        e = cudaMemcpy3DAsync(&p, s);
        if (e != cudaSuccess) { dev_free(lin, s); return fail(cuda_status(e, "cudaMemcpy3DAsync")); }
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = v->array;
        cudaTextureDesc td{};
        td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModeLinear;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&v->tex, &rd, &td, nullptr);
        dev_free(lin, s);
        if (e != cudaSuccess) return fail(cuda_status(e, "cudaCreateTextureObject"));
    }
    e = cudaMemsetAsync(v->stats, 0, sizeof(DevStats), s);
    if (e != cudaSuccess) return fail(cuda_status(e, "vdbc_volume_create stats"));
    *out = v;
    return VDBC_OK;
}

extern "C" void vdbc_volume_free(vdbc_volume* v)
{
    if (!v) return;
    if (v->tex) cudaDestroyTextureObject(v->tex);
    if (v->array) cudaFreeArray(v->array);
    if (v->linear) cudaFree(v->linear);
    if (v->mcmin) cudaFree(v->mcmin);
    if (v->mcmax) cudaFree(v->mcmax);
    if (v->stats) {
        release_kernel_events(v->stats);
        cudaFree(v->stats);
    }
    delete v;
}

extern "C" vdbc_status vdbc_render_dense(const vdbc_volume* vol, const vdbc_camera* camera, const vdbc_medium* medium,
                                         int32_t spp, uint64_t seed, float* rgba_out, int32_t out_on_device,
                                         void* stream)
{
    clear_error();
    if (!vol) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_render_dense: volume is null");
    Majorants mj{vol->mcmax, vol->macrocell, vol->mcdims[0], vol->mcdims[1], vol->mcdims[2],
                 vol->dims[0], vol->dims[1], vol->dims[2], vol->mcmin};
    if (vol->filter == VDBC_FILTER_LINEAR) {
        LinearSampler smp{vol->linear, vol->dims[0], vol->dims[1], vol->dims[2]};
        return render_common(smp, mj, vol->dims, vol->stats, camera, medium, spp, seed, rgba_out, out_on_device, stream);
    }
    TexSampler smp{vol->tex};
    return render_common(smp, mj, vol->dims, vol->stats, camera, medium, spp, seed, rgba_out, out_on_device, stream);
}

extern "C" vdbc_status vdbc_volume_render_stats_get(const vdbc_volume* vol, void* stream, vdbc_render_stats* out)
{
    clear_error();
    if (!vol || !out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_volume_render_stats_get: null argument");
    VDBC_TRY(wait_stream(static_cast<cudaStream_t>(stream)));
    DevStats h;
    VDBC_CUDA(cudaMemcpy(&h, vol->stats, sizeof(h), cudaMemcpyDeviceToHost));
    out->lookups = h.lookups;
    out->paths = h.paths;
    out->error_flags = h.error_flags;
    for (int k = 0; k < kNumEvents; ++k) out->events[k] = h.ev[k];
    out->kernel_ms = kernel_ms_of(vol->stats);
    out->reserved = 0;
    return VDBC_OK;
}

// ---------------------------------------------------------------- batches
namespace vdbc {
namespace {

struct TuneKey {
    std::string text;
};

std::mutex g_tune_mu;
std::map<std::string, vdbc_tuning> g_tune_cache;

std::string gpu_name()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    return p.name;
}

bool tune_file_lookup(const std::string& key, vdbc_tuning* t)
{
    const char* path = std::getenv("VDBC_TUNE_CACHE");
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        char k[900];
        vdbc_tuning v{};
        if (std::sscanf(line, "%899s %d %d %d %d %f", k, &v.threads, &v.chunk, &v.coarse, &v.depth, &v.frame_ms) == 6 &&
            key == k && (v.depth == 1 || v.depth == 2)) {
            *t = v;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void tune_file_store(const std::string& key, const vdbc_tuning& t)
{
    const char* path = std::getenv("VDBC_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %.4f\n", key.c_str(), t.threads, t.chunk, t.coarse, t.depth, t.frame_ms);
    std::fclose(f);
}

}  // namespace
}  // namespace vdbc

// the jobs of one payload type: one persistent launch per frame each
struct BatchGroup {
    int payload = 0;
    std::vector<int> members;                 // job indices, in the caller's order
    std::vector<vdbc::JobView> h_jobs;        // their job views, work items counted from 0
    vdbc::JobView* d_jobs = nullptr;
    vdbc::GridView* d_grids = nullptr;
    unsigned long long nitems = 0;
    vdbc::DevStats* stats = nullptr;
    unsigned blocks[2][2][2] = {};     // launch configuration per [256 threads][coarse level][accessor depth 2]
    size_t smem[2][2][2] = {};
};

struct vdbc_batch {
    int n = 0;
    std::vector<vdbc_job> jobs;
    vdbc::JobView* d_jobs = nullptr;        // device job table (bits point at the chosen variant)
    std::vector<BatchGroup> groups;         // by payload type
    std::vector<vdbc::JobView> h_jobs;
    std::vector<uint32_t*> bits_on, bits_off;   // per job: fine + coarse words, coarse skipping on / off
    std::vector<int> nwords;
    unsigned long long* accum = nullptr;    // the frame's fixed-point radiance sums, 3 per pixel of every job
    size_t accum_words = 0;
    float4* sums = nullptr;
    float4** d_sums = nullptr;
    float** d_outs = nullptr;
    int* d_frame = nullptr;
    size_t max_npix = 0;
    vdbc_tuning tuning{256, 256, 1, 1, 0.0f};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> allocs;
};

namespace vdbc {
namespace {

vdbc_status batch_alloc(vdbc_batch* b, void** p, size_t bytes)
{
    if (fault_injected("oom")) return set_error(VDBC_ERR_OOM, "device allocation of %zu bytes refused (VDBC_FAULT=oom)", bytes);
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) { *p = nullptr; cudaGetLastError(); return cuda_status(e, "vdbc_batch_create alloc"); }
    b->allocs.push_back(*p);
    return VDBC_OK;
}

// points every job's cbits at the coarse words with skipping on or off and uploads the table
vdbc_status batch_select_bits(vdbc_batch* b, bool coarse, cudaStream_t s)
{
    for (int i = 0; i < b->n; ++i) {
        uint32_t* base = coarse ? b->bits_on[i] : b->bits_off[i];
        b->h_jobs[i].bits = base;
        b->h_jobs[i].cbits = base + b->nwords[i];
    }
    VDBC_CUDA(cudaMemcpyAsync(b->d_jobs, b->h_jobs.data(), sizeof(JobView) * b->n, cudaMemcpyHostToDevice, s));
    for (BatchGroup& g : b->groups) {
        unsigned long long items = 0;
        for (size_t k = 0; k < g.members.size(); ++k) {
            JobView jv = b->h_jobs[g.members[k]];
            jv.item_begin = items;
            items += jv.items;
            g.h_jobs[k] = jv;
        }
        VDBC_CUDA(cudaMemcpyAsync(g.d_jobs, g.h_jobs.data(), sizeof(JobView) * g.h_jobs.size(),
                                  cudaMemcpyHostToDevice, s));
    }
    return VDBC_OK;
}

// grid size and shared memory of the batched tracker for a block size; called
// before any capture (it sets a function attribute and queries occupancy)
template <int kThreads, bool kUseCoarse, int P, int D>
vdbc_status group_config_t(BatchGroup& g)
{
    unsigned* blocks = &g.blocks[kThreads == 256][kUseCoarse][D == 2];
    size_t* smem = &g.smem[kThreads == 256][kUseCoarse][D == 2];
    *smem = (sizeof(JobView) + sizeof(GridView)) * g.members.size();
    auto kern = k_pt_batch<kThreads, kUseCoarse, P, D>;
    if (*smem > 48 * 1024)
        VDBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
    int per_sm = 0;
    VDBC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, *smem));
    if (per_sm < 1) per_sm = 1;
    long long want = (long long)((g.nitems + kThreads - 1) / kThreads);
    *blocks = (unsigned)std::min<long long>((long long)sm_count() * per_sm, std::max<long long>(want, 1));
    return VDBC_OK;
}

template <int kThreads, bool kUseCoarse, int P, int D>
vdbc_status group_launch_t(vdbc_batch* b, BatchGroup& g, int chunk, unsigned stride, cudaStream_t s)
{
    if (g.blocks[kThreads == 256][kUseCoarse][D == 2] == 0) VDBC_TRY((group_config_t<kThreads, kUseCoarse, P, D>(g)));
    const unsigned blocks = g.blocks[kThreads == 256][kUseCoarse][D == 2];
    const size_t smem = g.smem[kThreads == 256][kUseCoarse][D == 2];
    KLAUNCH((k_pt_batch<kThreads, kUseCoarse, P, D><<<blocks, kThreads, smem, s>>>(
        g.d_jobs, g.d_grids, (int)g.members.size(), g.nitems, b->d_frame, g.stats, chunk, stride)));
    VDBC_CUDA(cudaGetLastError());
    return VDBC_OK;
}

// the group's kernel for its payload type
template <int kThreads, bool kUseCoarse, int D>
vdbc_status group_launch(vdbc_batch* b, BatchGroup& g, int chunk, unsigned stride, cudaStream_t s)
{
    if (g.payload == VDBC_FP16) return group_launch_t<kThreads, kUseCoarse, 1, D>(b, g, chunk, stride, s);
    if (g.payload == VDBC_FP8) return group_launch_t<kThreads, kUseCoarse, 2, D>(b, g, chunk, stride, s);
    return group_launch_t<kThreads, kUseCoarse, 0, D>(b, g, chunk, stride, s);
}

template <int kThreads, bool kUseCoarse, int D>
vdbc_status group_config(BatchGroup& g)
{
    if (g.payload == VDBC_FP16) return group_config_t<kThreads, kUseCoarse, 1, D>(g);
    if (g.payload == VDBC_FP8) return group_config_t<kThreads, kUseCoarse, 2, D>(g);
    return group_config_t<kThreads, kUseCoarse, 0, D>(g);
}

template <int kThreads, bool kUseCoarse, int D>
vdbc_status batch_config(vdbc_batch* b)
{
    for (BatchGroup& g : b->groups) VDBC_TRY((group_config<kThreads, kUseCoarse, D>(g)));
    return VDBC_OK;
}

template <int kThreads, bool kUseCoarse, int D>
vdbc_status batch_launch_pt(vdbc_batch* b, int chunk, unsigned stride, cudaStream_t s)
{
    for (BatchGroup& g : b->groups) VDBC_TRY((group_launch<kThreads, kUseCoarse, D>(b, g, chunk, stride, s)));
    return VDBC_OK;
}

// the work of one frame: counters, one tracker launch per payload group,
// accumulation, next frame number
vdbc_status batch_frame(vdbc_batch* b, const vdbc_tuning& t, bool accumulate, cudaStream_t s, unsigned stride = 1)
{
    for (BatchGroup& g : b->groups) VDBC_CUDA(cudaMemsetAsync(g.stats, 0, sizeof(DevStats), s));
    VDBC_CUDA(cudaMemsetAsync(b->accum, 0, b->accum_words * sizeof(unsigned long long), s));
    if (t.threads == 128) {
        if (t.coarse) VDBC_TRY((batch_launch_pt<128, true, 1>(b, t.chunk, stride, s)));
        else VDBC_TRY((batch_launch_pt<128, false, 1>(b, t.chunk, stride, s)));
    } else if (t.depth == 2) {
        if (t.coarse) VDBC_TRY((batch_launch_pt<256, true, 2>(b, t.chunk, stride, s)));
        else VDBC_TRY((batch_launch_pt<256, false, 2>(b, t.chunk, stride, s)));
    } else {
        if (t.coarse) VDBC_TRY((batch_launch_pt<256, true, 1>(b, t.chunk, stride, s)));
        else VDBC_TRY((batch_launch_pt<256, false, 1>(b, t.chunk, stride, s)));
    }
    if (accumulate) {
        dim3 grid((unsigned)((b->max_npix + 255) / 256), (unsigned)b->n);
        KLAUNCH(k_batch_reduce<<<grid, 256, 0, s>>>(b->d_jobs, b->d_sums, b->d_outs, b->d_frame));
        KLAUNCH(k_batch_next_frame<<<1, 32, 0, s>>>(b->d_frame));
        VDBC_CUDA(cudaGetLastError());
    }
    return VDBC_OK;
}

std::string batch_key(const vdbc_batch* b)
{
    // GPU and the layout that decides the work: grid sizes, payloads, macrocells, images, spp
    unsigned long long h = 0xcbf29ce484222325ull;
    auto mix = [&](long long v) { h ^= (unsigned long long)v; h *= 0x100000001b3ull; };
    for (const vdbc_job& j : b->jobs) {
        for (int a = 0; a < 3; ++a) mix(j.grid->info.dims[a]);
        mix(j.grid->info.payload); mix(j.grid->info.macrocell); mix(j.grid->info.n_leaves);
        mix(j.camera.width); mix(j.camera.height); mix(j.spp); mix(j.medium.max_bounces);
    }
    char buf[64];
    std::snprintf(buf, sizeof(buf), "%016llx", h);
    std::string name = gpu_name();
    for (char& c : name) if (c == ' ') c = '_';
    return name + "|" + buf;
}

constexpr unsigned kTuneStride = 8;

// times (a sample of) one frame for each candidate shape and keeps the fastest
vdbc_status batch_autotune(vdbc_batch* b, cudaStream_t s)
{
    const std::string key = batch_key(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { b->tuning = it->second; return VDBC_OK; }
    }
    vdbc_tuning cached;
    if (tune_file_lookup(key, &cached)) {
        b->tuning = cached;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = cached;
        return VDBC_OK;
    }
    // launch shapes: (threads per block, accessor cache depth) pairs, work
    // items a warp takes per refill (32, 64, 128, 256: one, two, four or eight
    // paths per lane per refill), coarse DDA level on or off
    const int shapes[][2] = {{128, 1}, {256, 1}, {256, 2}};
    const int chunks[] = {32, 64, 128, 256};
    const int coarses[] = {1, 0};
    cudaEvent_t e0, e1;
    VDBC_CUDA(cudaEventCreate(&e0));
    VDBC_CUDA(cudaEventCreate(&e1));
    vdbc_tuning best{256, 256, 1, 1, 1e30f};
    vdbc_status st = VDBC_OK;
    for (int co : coarses) {
        st = batch_select_bits(b, co != 0, s);
        if (st != VDBC_OK) break;
        for (const auto& sh : shapes)
            for (int ch : chunks) {
                vdbc_tuning t{sh[0], ch, co, sh[1], 0.0f};
                // every kTuneStride-th path of a frame: a sample spread over all jobs
                st = batch_frame(b, t, false, s, kTuneStride);           // warm-up
                if (st == VDBC_OK && cudaEventRecord(e0, s) != cudaSuccess) st = set_error(VDBC_ERR_CUDA, "tune event");
                if (st == VDBC_OK) st = batch_frame(b, t, false, s, kTuneStride);
                if (st == VDBC_OK && cudaEventRecord(e1, s) != cudaSuccess) st = set_error(VDBC_ERR_CUDA, "tune event");
                if (st == VDBC_OK) st = wait_stream(s);
                if (st != VDBC_OK) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                t.frame_ms = ms;
                if (ms < best.frame_ms) best = t;
            }
        if (st != VDBC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != VDBC_OK) return st;
    b->tuning = best;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    tune_file_store(key, best);
    return VDBC_OK;
}

// captures one frame on a private stream (capture cannot use the legacy
// default stream); the graph is launched later into the caller's stream
vdbc_status batch_capture(vdbc_batch* b, cudaStream_t s)
{
    VDBC_TRY(batch_select_bits(b, b->tuning.coarse != 0, s));
    const bool c = b->tuning.coarse != 0;
    if (b->tuning.threads == 128) VDBC_TRY(c ? (batch_config<128, true, 1>(b)) : (batch_config<128, false, 1>(b)));
    else if (b->tuning.depth == 2) VDBC_TRY(c ? (batch_config<256, true, 2>(b)) : (batch_config<256, false, 2>(b)));
    else VDBC_TRY(c ? (batch_config<256, true, 1>(b)) : (batch_config<256, false, 1>(b)));
    VDBC_TRY(wait_stream(s));
    cudaStream_t cs = nullptr;
    VDBC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); return cuda_status(e, "cudaStreamBeginCapture"); }
    vdbc_status st = batch_frame(b, b->tuning, true, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st != VDBC_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    b->graph = g;
    VDBC_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    return VDBC_OK;
}

}  // namespace
}  // namespace vdbc

extern "C" vdbc_status vdbc_batch_create(const vdbc_job* jobs, int32_t n, int32_t autotune, void* stream,
                                         vdbc_batch** out)
{
    clear_error();
    if (!jobs || !out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_batch_create: null argument");
    *out = nullptr;
    if (n < 1 || n > 64) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_batch_create: %d jobs outside 1..64", n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    vdbc_batch* b = new vdbc_batch();
    auto fail = [&](vdbc_status st) { return release_or_defer(st, s, [b] { vdbc_batch_free(b); }); };
    b->n = n;
    b->jobs.assign(jobs, jobs + n);
    b->h_jobs.resize(n);
    b->bits_on.resize(n);
    b->bits_off.resize(n);
    b->nwords.resize(n);
    std::vector<GridView> grids(n);
    std::vector<float4*> sum_ptrs(n);
    std::vector<float*> outs(n);
    unsigned long long items = 0;
    size_t accum_pixels = 0, sum_floats4 = 0;
    for (int i = 0; i < n; ++i) {
        const vdbc_job& j = jobs[i];
        if (!j.grid || !j.rgba_out) return fail(set_error(VDBC_ERR_INVALID_ARG, "job %d: null grid or output", i));
        if (j.grid->info.payload == VDBC_LEARNED)
            return fail(set_error(VDBC_ERR_UNSUPPORTED, "job %d: learned grids render through vdbc_render", i));
        vdbc_status st = check_camera(&j.camera);
        if (st != VDBC_OK) return fail(st);
        if (j.medium.mode != VDBC_MODE_PT) return fail(set_error(VDBC_ERR_INVALID_ARG, "job %d: batches path trace", i));
        MedHost mh;
        st = make_med(&j.medium, j.grid->info.dims, j.spp, s, mh);
        if (st != VDBC_OK) return fail(st);
        const GridView& g = j.grid->view;
        Majorants mj{g.mcmax, g.mc, g.mx, g.my, g.mz, g.nx, g.ny, g.nz};
        CamDev cam = make_cam(&j.camera, j.grid->info.dims);
        JobView jv = make_job(mj, cam, mh.dev, j.spp, j.seed, nullptr);
        jv.item_begin = items;
        items += jv.items;
        accum_pixels += (size_t)jv.npix;
        sum_floats4 += (size_t)jv.npix;
        b->max_npix = std::max<size_t>(b->max_npix, (size_t)jv.npix);
        b->h_jobs[i] = jv;
        grids[i] = g;
        outs[i] = j.rgba_out;
    }
    (void)items;
    // payload groups, each with its own job and grid tables, work counter and stats
    for (int p = VDBC_FP32; p <= VDBC_FP8; ++p) {
        BatchGroup g;
        g.payload = p;
        for (int i = 0; i < n; ++i)
            if (jobs[i].grid->info.payload == p) {
                g.members.push_back(i);
                g.nitems += b->h_jobs[i].items;
            }
        if (!g.members.empty()) b->groups.push_back(std::move(g));
    }
    b->accum_words = accum_pixels * 3;
    vdbc_status st = batch_alloc(b, reinterpret_cast<void**>(&b->accum), b->accum_words * sizeof(unsigned long long));
    if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&b->sums), sum_floats4 * sizeof(float4));
    if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&b->d_jobs), sizeof(JobView) * n);
    if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&b->d_sums), sizeof(float4*) * n);
    if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&b->d_outs), sizeof(float*) * n);
    if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&b->d_frame), sizeof(int));
    for (BatchGroup& g : b->groups) {
        g.h_jobs.resize(g.members.size());
        if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&g.d_jobs), sizeof(JobView) * g.members.size());
        if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&g.d_grids), sizeof(GridView) * g.members.size());
        if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&g.stats), sizeof(DevStats));
    }
    if (st != VDBC_OK) return fail(st);
    std::vector<std::vector<GridView>> ggrids(b->groups.size());
    for (size_t k = 0; k < b->groups.size(); ++k)
        for (int m : b->groups[k].members) {
            GridView gv = grids[m];
#if VDBC_CHECKED
            gv.err = &b->groups[k].stats->error_flags;   // reported with the batch's flags
#endif
            ggrids[k].push_back(gv);
        }
    size_t po = 0, so = 0;
    for (int i = 0; i < n; ++i) {
        JobView& jv = b->h_jobs[i];
        jv.accum = b->accum + po;
        po += 3 * (size_t)jv.npix;
        sum_ptrs[i] = b->sums + so;
        so += (size_t)jv.npix;
        // occupancy bits, once with coarse skipping and once without
        const Majorants& mj = jv.m;
        long long ncell = (long long)mj.mx * mj.my * mj.mz;
        int nwords = (int)((ncell + 31) / 32);
        int czn = (mj.mz + kCoarse - 1) / kCoarse;
        int ncwords = (jv.cx_n * jv.cy_n * czn + 31) / 32;
        b->nwords[i] = nwords;
        st = batch_alloc(b, reinterpret_cast<void**>(&b->bits_on[i]), (size_t)(nwords + ncwords) * 4);
        if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&b->bits_off[i]), (size_t)(nwords + ncwords) * 4);
        if (st != VDBC_OK) return fail(st);
        KLAUNCH(k_occupancy<<<blocks_for(ncell, 256), 256, 0, s>>>(mj.mcmax, ncell, jv.med.sigma_scale, b->bits_on[i]));
        KLAUNCH(k_coarse_occupancy<<<blocks_for((long long)jv.cx_n * jv.cy_n * czn, 256), 256, 0, s>>>(
            b->bits_on[i], mj.mx, mj.my, mj.mz, b->bits_on[i] + nwords, jv.cx_n, jv.cy_n, czn));
        cudaError_t e = cudaMemcpyAsync(b->bits_off[i], b->bits_on[i], (size_t)nwords * 4, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->bits_off[i] + nwords, 0xff, (size_t)ncwords * 4, s);
        if (e != cudaSuccess) return fail(cuda_status(e, "vdbc_batch_create bits"));
    }
    {
        // each job's clip box: the box of its occupied macrocells, built on
        // the device as k_pt builds it, then held in the job table
        int* d_occ = nullptr;
        float* d_clip = nullptr;
        st = batch_alloc(b, reinterpret_cast<void**>(&d_occ), sizeof(int) * 6 * (size_t)n);
        if (st == VDBC_OK) st = batch_alloc(b, reinterpret_cast<void**>(&d_clip), sizeof(float) * 6 * (size_t)n);
        if (st != VDBC_OK) return fail(st);
        for (int i = 0; i < n; ++i) {
            const Majorants& mj = b->h_jobs[i].m;
            const long long ncell = (long long)mj.mx * mj.my * mj.mz;
            cudaError_t e = cudaMemsetAsync(d_occ + 6 * i, 0x7f, 3 * sizeof(int), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(d_occ + 6 * i + 3, 0xff, 3 * sizeof(int), s);
            if (e != cudaSuccess) return fail(cuda_status(e, "vdbc_batch_create box"));
            KLAUNCH(k_occupied_box<<<blocks_for(ncell, 256), 256, 0, s>>>(b->bits_on[i], mj.mx, mj.my, ncell,
                                                                          d_occ + 6 * i));
            KLAUNCH(k_clip_box<<<1, 1, 0, s>>>(mj, d_occ + 6 * i, d_clip + 6 * i));
        }
        std::vector<float> clip(6 * (size_t)n);
        cudaError_t e = cudaMemcpyAsync(clip.data(), d_clip, sizeof(float) * 6 * (size_t)n, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return fail(cuda_status(e, "vdbc_batch_create box"));
        st = wait_stream(s);
        if (st != VDBC_OK) return fail(st);
        for (int i = 0; i < n; ++i) std::memcpy(b->h_jobs[i].clip, clip.data() + 6 * i, sizeof(float) * 6);
    }
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < b->groups.size() && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(b->groups[k].d_grids, ggrids[k].data(), sizeof(GridView) * ggrids[k].size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_sums, sum_ptrs.data(), sizeof(float4*) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_outs, outs.data(), sizeof(float*) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_frame, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->sums, 0, sum_floats4 * sizeof(float4), s);
    if (e != cudaSuccess) return fail(cuda_status(e, "vdbc_batch_create upload"));
    st = batch_select_bits(b, true, s);
    if (st == VDBC_OK) st = wait_stream(s);      // (pageable host sources: the copies staged them already)
    if (st == VDBC_OK && autotune) st = batch_autotune(b, s);
    if (st == VDBC_OK) st = vdbc_batch_reset(b, stream);
    if (st == VDBC_OK) st = batch_capture(b, s);
    if (st != VDBC_OK) return fail(st);
    *out = b;
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_batch_render_frames(vdbc_batch* b, int32_t frames, void* stream)
{
    clear_error();
    if (!b || !b->exec || frames < 0) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_batch_render_frames: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int f = 0; f < frames; ++f) {
        count_launch((int)b->groups.size() + 2);      // a tracker per payload group, reduce, frame counter
        VDBC_CUDA(cudaGraphLaunch(b->exec, s));
    }
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_batch_reset(vdbc_batch* b, void* stream)
{
    clear_error();
    if (!b) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_batch_reset: null batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t npix = 0;
    for (const JobView& j : b->h_jobs) npix += (size_t)j.npix;
    VDBC_CUDA(cudaMemsetAsync(b->d_frame, 0, sizeof(int), s));
    VDBC_CUDA(cudaMemsetAsync(b->sums, 0, npix * sizeof(float4), s));
    return VDBC_OK;
}

// progressive accumulation state: the frame counter and the per-pixel sums
// of every job, one contiguous float4 array in job order
static size_t batch_state_pixels(const vdbc_batch* b)
{
    size_t npix = 0;
    for (const JobView& j : b->h_jobs) npix += (size_t)j.npix;
    return npix;
}

extern "C" vdbc_status vdbc_batch_state_size(const vdbc_batch* b, int64_t* floats)
{
    clear_error();
    if (!b || !floats) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_batch_state_size: null argument");
    *floats = (int64_t)batch_state_pixels(b) * 4;
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_batch_get_state(const vdbc_batch* b, int32_t* frame, float* host_sums, void* stream)
{
    clear_error();
    if (!b || !frame || !host_sums) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_batch_get_state: null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VDBC_CUDA(cudaMemcpyAsync(frame, b->d_frame, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    VDBC_CUDA(cudaMemcpyAsync(host_sums, b->sums, batch_state_pixels(b) * sizeof(float4), cudaMemcpyDeviceToHost, s));
    return wait_stream(s);
}

extern "C" vdbc_status vdbc_batch_set_state(vdbc_batch* b, int32_t frame, const float* host_sums, void* stream)
{
    clear_error();
    if (!b || !host_sums || frame < 0) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_batch_set_state: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VDBC_CUDA(cudaMemcpyAsync(b->d_frame, &frame, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    VDBC_CUDA(cudaMemcpyAsync(b->sums, host_sums, batch_state_pixels(b) * sizeof(float4), cudaMemcpyHostToDevice, s));
    return wait_stream(s);     // `frame` and `host_sums` must outlive the copies
}

extern "C" vdbc_status vdbc_batch_get_tuning(const vdbc_batch* b, vdbc_tuning* t)
{
    clear_error();
    if (!b || !t) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_batch_get_tuning: null argument");
    *t = b->tuning;
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_batch_stats_get(const vdbc_batch* b, void* stream, vdbc_render_stats* out)
{
    clear_error();
    if (!b || !out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_batch_stats_get: null argument");
    VDBC_TRY(wait_stream(static_cast<cudaStream_t>(stream)));
    out->lookups = out->paths = out->error_flags = 0;
    for (int k = 0; k < kNumEvents; ++k) out->events[k] = 0;
    for (const BatchGroup& g : b->groups) {          // the payload groups' counters, summed
        DevStats h;
        VDBC_CUDA(cudaMemcpy(&h, g.stats, sizeof(h), cudaMemcpyDeviceToHost));
        out->lookups += h.lookups;
        out->paths += h.paths;
        out->error_flags |= h.error_flags;
        for (int k = 0; k < kNumEvents; ++k) out->events[k] += h.ev[k];
    }
    out->kernel_ms = -1.0f;   // frames are replayed from a graph; time them around vdbc_batch_render_frames
    out->reserved = 0;
    return VDBC_OK;
}

extern "C" void vdbc_batch_free(vdbc_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void* p : b->allocs) cudaFree(p);
    delete b;
}
