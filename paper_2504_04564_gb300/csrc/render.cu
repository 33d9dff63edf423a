// render.cu -- one thread per light path over the compressed grid or the
// plain form (Section 4 of the paper; Section 3.2.2 for the sampler).
//
//   k_ea  emission-absorption marching, fixed step, front to back; one
//         thread per pixel (the project's sci-vis mode)
//   k_pt  Monte Carlo path tracing: 3D-DDA over the macrocell majorant grid,
//         Woodcock (delta) tracking inside every non-empty cell with a restart
//         at the next cell on overshoot, Henyey-Greenstein scattering, the
//         directional light's transmittance by ratio tracking, a constant
//         environment on escape.  One thread per pixel loops over its spp
//         paths so the per-pixel sum has a fixed order.
// Both are templated on the sampler: VdbSampler (tree descent + leaf decode +
// trilinear, every lookup), LinearSampler (dense array, the same software
// trilinear) and TexSampler (3D CUDA texture, hardware trilinear).
//
// Random numbers: Philox4x32-10, counter (pixel, sample, call, stream), key =
// seed; stream 0 for the camera and the walk, 1 for the light rays; one call
// per event, u0 = distance, u1 = accept, u2/u3 = phase function.
#include <algorithm>
#include <cmath>
#include <cstring>

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
};

struct Majorants {
    const float* mcmax;
    int mc;
    int mx, my, mz;
    int nx, ny, nz;
};

constexpr int kMaxStepsPerCell = 1 << 20;

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 norm3(float3 a)
{
    float l = sqrtf(dot3(a, a));
    return f3(a.x / l, a.y / l, a.z / l);
}

// ray / box [-1/2, dim-1/2]^3, t >= 0
__device__ __forceinline__ bool clip_axis(float o, float d, float hi, float& t0, float& t1)
{
    if (d == 0.0f) return !(o < -0.5f || o > hi);
    float ta = (-0.5f - o) / d, tb = (hi - o) / d;
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

// 3D-DDA over the macrocells (Amanatides-Woo stepping, boundaries recomputed
// from the cell index every step so no error accumulates)
struct Dda {
    int cx, cy, cz, sx, sy, sz;
    float t, tmax;
    __device__ __forceinline__ static float bnd(int c, int s, float mc, float o, float d)
    {
        if (s == 0) return INFINITY;
        float b = -0.5f + (float)(c + (s > 0 ? 1 : 0)) * mc;
        return (b - o) / d;
    }
    __device__ __forceinline__ static int first_cell(float o, float d, float tmin, float mc, int n)
    {
        float p = o + tmin * d;
        int ci = (int)floorf((p + 0.5f) / mc);
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
        cx = first_cell(o.x, d.x, tmin, mc, m.mx);
        cy = first_cell(o.y, d.y, tmin, mc, m.my);
        cz = first_cell(o.z, d.z, tmin, mc, m.mz);
    }
    // current cell and its exit distance; false once the ray left the grid
    __device__ __forceinline__ bool cell(const Majorants& m, float3 o, float3 d, int& id, float& texit) const
    {
        if (t >= tmax) return false;
        if (cx < 0 || cx >= m.mx || cy < 0 || cy >= m.my || cz < 0 || cz >= m.mz) return false;
        float mc = (float)m.mc;
        float te = fminf(tmax, bnd(cx, sx, mc, o.x, d.x));
        te = fminf(te, bnd(cy, sy, mc, o.y, d.y));
        te = fminf(te, bnd(cz, sz, mc, o.z, d.z));
        id = (cz * m.my + cy) * m.mx + cx;
        texit = te;
        return true;
    }
    // step the axis whose boundary is nearest (x, then y, then z on ties)
    __device__ __forceinline__ void advance(const Majorants& m, float3 o, float3 d, float texit)
    {
        float mc = (float)m.mc;
        float bx = bnd(cx, sx, mc, o.x, d.x), by = bnd(cy, sy, mc, o.y, d.y), bz = bnd(cz, sz, mc, o.z, d.z);
        float bt = bx;
        int best = 0;
        if (by < bt) { bt = by; best = 1; }
        if (bz < bt) { bt = bz; best = 2; }
        if (!(bt < tmax)) { t = tmax; return; }
        if (best == 0) cx += sx;
        else if (best == 1) cy += sy;
        else cz += sz;
        if (texit > t) t = texit;
    }
};

__device__ __forceinline__ float hg_eval(float mu, float g)
{
    float den = 1.0f + g * g - 2.0f * g * mu;
    return (1.0f - g * g) / (4.0f * 3.14159265358979f * den * sqrtf(den));
}

__device__ __forceinline__ float hg_sample_mu(float g, float xi)
{
    float mu;
    if (fabsf(g) < 1e-3f) mu = 1.0f - 2.0f * xi;
    else {
        float s = (1.0f - g * g) / (1.0f - g + 2.0f * g * xi);
        mu = (1.0f + g * g - s * s) / (2.0f * g);
    }
    return fminf(fmaxf(mu, -1.0f), 1.0f);
}

// Duff et al., "Building an Orthonormal Basis, Revisited" (JCGT 2017)
__device__ __forceinline__ void onb(float3 n, float3& b1, float3& b2)
{
    float sign = n.z >= 0.0f ? 1.0f : -1.0f;
    float a = -1.0f / (sign + n.z);
    float b = n.x * n.y * a;
    b1 = f3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
    b2 = f3(b, sign + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ void camera_ray(const CamDev& cam, int px, int py, float jx, float jy, float3& o,
                                           float3& d)
{
    float sx = 2.0f * ((float)px + jx) / (float)cam.w - 1.0f;
    float sy = 1.0f - 2.0f * ((float)py + jy) / (float)cam.h;
    if (cam.kind == VDBC_CAM_ORTHO) {
        float a = sx * cam.sxs, b = sy * cam.sys;
        o = f3(cam.eye.x + a * cam.right.x + b * cam.up.x, cam.eye.y + a * cam.right.y + b * cam.up.y,
               cam.eye.z + a * cam.right.z + b * cam.up.z);
        d = cam.fwd;
    } else {
        float a = sx * cam.sxs, b = sy * cam.sys;
        o = cam.eye;
        d = norm3(f3(cam.fwd.x + a * cam.right.x + b * cam.up.x, cam.fwd.y + a * cam.right.y + b * cam.up.y,
                     cam.fwd.z + a * cam.right.z + b * cam.up.z));
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
};

// Woodcock tracking through the macrocells; true on a real collision
template <class S>
__device__ __forceinline__ bool delta_track(const S& smp, Accessor& acc, const Majorants& m, const MedDev& med,
                                            const Rng& rng, float3 o, float3 d, float tmin, float tmax,
                                            uint32_t& call, float& thit, float& xi0, float& xi1, Walk& w)
{
    Dda dda;
    dda.init(m, o, d, tmin, tmax);
    int cell;
    float texit;
    int guard = m.mx + m.my + m.mz + 8;
    while (dda.cell(m, o, d, cell, texit)) {
        if (--guard < 0) { w.flags |= kErrDdaSteps; return false; }
        float mj = med.sigma_scale * __ldg(m.mcmax + cell);
        if (mj > 0.0f && texit > dda.t) {
            float t = dda.t;
            for (int it = 0;; ++it) {
                if (it >= kMaxStepsPerCell) { w.flags |= kErrTrackSteps; return false; }
                U4 r = rng.draw(call++, 0);
                t = t - logf(1.0f - u01(r.x)) / mj;
                if (t >= texit) break;
                float3 p = f3(o.x + t * d.x, o.y + t * d.y, o.z + t * d.z);
                float sigma = med.sigma_scale * smp(p.x, p.y, p.z, acc);
                ++w.lookups;
                if (u01(r.y) * mj < sigma) {
                    thit = t;
                    xi0 = u01(r.z);
                    xi1 = u01(r.w);
                    return true;
                }
            }
        }
        dda.advance(m, o, d, texit);
    }
    return false;
}

// ratio tracking: product of (1 - sigma / majorant) over the tentative collisions
template <class S>
__device__ __forceinline__ float ratio_track(const S& smp, Accessor& acc, const Majorants& m, const MedDev& med,
                                             const Rng& rng, float3 o, float3 d, float tmin, float tmax,
                                             uint32_t& call, Walk& w)
{
    Dda dda;
    dda.init(m, o, d, tmin, tmax);
    int cell;
    float texit, T = 1.0f;
    int guard = m.mx + m.my + m.mz + 8;
    while (dda.cell(m, o, d, cell, texit)) {
        if (--guard < 0) { w.flags |= kErrDdaSteps; return T; }
        float mj = med.sigma_scale * __ldg(m.mcmax + cell);
        if (mj > 0.0f && texit > dda.t) {
            float t = dda.t;
            for (int it = 0;; ++it) {
                if (it >= kMaxStepsPerCell) { w.flags |= kErrTrackSteps; return T; }
                U4 r = rng.draw(call++, 1);
                t = t - logf(1.0f - u01(r.x)) / mj;
                if (t >= texit) break;
                float3 p = f3(o.x + t * d.x, o.y + t * d.y, o.z + t * d.z);
                float sigma = med.sigma_scale * smp(p.x, p.y, p.z, acc);
                ++w.lookups;
                T *= 1.0f - sigma / mj;
            }
        }
        dda.advance(m, o, d, texit);
    }
    return T;
}

template <class S>
__device__ float3 trace_path(const S& smp, Accessor& acc, const Majorants& m, const CamDev& cam,
                             const MedDev& med, const Rng& rng, int px, int py, Walk& w)
{
    uint32_t call = 0, lcall = 0;
    U4 r = rng.draw(call++, 0);
    float3 o, d;
    camera_ray(cam, px, py, u01(r.x), u01(r.y), o, d);
    float3 L = f3(0.f, 0.f, 0.f);
    float beta = 1.0f;
    float tin, tout;
    if (!clip_box(m, o, d, tin, tout)) return med.env_rad;
    for (int bounce = 0; bounce < med.max_bounces; ++bounce) {
        float thit, xi0, xi1;
        if (!delta_track(smp, acc, m, med, rng, o, d, tin, tout, call, thit, xi0, xi1, w)) {
            L.x += beta * med.env_rad.x; L.y += beta * med.env_rad.y; L.z += beta * med.env_rad.z;
            return L;
        }
        float3 x = f3(o.x + thit * d.x, o.y + thit * d.y, o.z + thit * d.z);
        beta *= med.albedo;
        float ltin, ltout, T = 1.0f;
        if (clip_box(m, x, med.sun_dir, ltin, ltout))
            T = ratio_track(smp, acc, m, med, rng, x, med.sun_dir, ltin, ltout, lcall, w);
        float ph = hg_eval(dot3(d, med.sun_dir), med.g);
        float wgt = beta * ph * T;
        L.x += wgt * med.sun_rad.x; L.y += wgt * med.sun_rad.y; L.z += wgt * med.sun_rad.z;
        if (bounce + 1 == med.max_bounces) return L;
        float mu = hg_sample_mu(med.g, xi0);
        float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
        float sphi, cphi;
        sincospif(2.0f * xi1, &sphi, &cphi);   // phi = 2 pi xi1, reduction-free form
        float3 b1, b2;
        onb(d, b1, b2);
        float3 nd = f3(st * cphi * b1.x + st * sphi * b2.x + mu * d.x, st * cphi * b1.y + st * sphi * b2.y + mu * d.y,
                       st * cphi * b1.z + st * sphi * b2.z + mu * d.z);
        d = norm3(nd);
        o = x;
        if (!clip_box(m, o, d, tin, tout)) {
            L.x += beta * med.env_rad.x; L.y += beta * med.env_rad.y; L.z += beta * med.env_rad.z;
            return L;
        }
    }
    return L;
}

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
}

template <class S>
__global__ void __launch_bounds__(128, 4) k_pt(S smp, Majorants m, CamDev cam, MedDev med, int spp, uint32_t k0,
                                            uint32_t k1, float4* __restrict__ out, DevStats* __restrict__ st)
{
    const int npix = cam.w * cam.h;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    Walk w{0, 0};
    unsigned long long paths = 0;
    if (pix < npix) {
        Accessor acc;
        acc.reset();
        Rng rng{(uint32_t)pix, 0, k0, k1};
        const int px = pix % cam.w, py = pix / cam.w;
        float3 acc_l = f3(0.f, 0.f, 0.f);
        for (int s = 0; s < spp; ++s) {
            rng.sample = (uint32_t)s;
            float3 L = trace_path(smp, acc, m, cam, med, rng, px, py, w);
            acc_l.x += L.x; acc_l.y += L.y; acc_l.z += L.z;
        }
        float inv = 1.0f / (float)spp;
        out[pix] = make_float4(acc_l.x * inv, acc_l.y * inv, acc_l.z * inv, 1.0f);
        paths = (unsigned long long)spp;
    }
    flush_stats(st, w, paths);
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
    Walk w{0, 0};
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
    if (!(c->fovy_or_height > 0.0) || (c->kind == VDBC_CAM_PINHOLE && !(c->fovy_or_height < 180.0)))
        return set_error(VDBC_ERR_INVALID_ARG, "bad field of view / ortho height");
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
        if (!(m->density_scale >= 0.0f) || !(m->albedo >= 0.0f && m->albedo <= 1.0f) || !(m->g > -1.0f && m->g < 1.0f))
            return set_error(VDBC_ERR_INVALID_ARG, "medium parameters out of range");
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
    } else {
        return set_error(VDBC_ERR_INVALID_ARG, "medium mode %d unknown", m->mode);
    }
    return VDBC_OK;
}

template <class S>
vdbc_status launch(const S& smp, const Majorants& mj, const CamDev& cam, const MedDev& med, int spp, uint64_t seed,
                   float4* out, DevStats* stats, cudaStream_t s)
{
    long long npix = (long long)cam.w * cam.h;
    VDBC_CUDA(cudaMemsetAsync(stats, 0, sizeof(DevStats), s));
    if (med.mode == VDBC_MODE_EA) {
        KLAUNCH(k_ea<S><<<blocks_for(npix, 128), 128, (size_t)med.tf_n * 16, s>>>(smp, mj, cam, med, out, stats));
    } else {
        KLAUNCH(k_pt<S><<<blocks_for(npix, 128), 128, 0, s>>>(smp, mj, cam, med, spp, (uint32_t)seed,
                                                      (uint32_t)(seed >> 32), out, stats));
    }
    VDBC_CUDA(cudaGetLastError());
    return VDBC_OK;
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
    VdbSampler smp{g};
    Majorants mj{g.mcmax, g.mc, g.mx, g.my, g.mz, g.nx, g.ny, g.nz};
    return render_common(smp, mj, grid->info.dims, grid->stats, camera, medium, spp, seed, rgba_out, out_on_device,
                         stream);
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
    if (mc < 1 || mc > 64) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_volume_create: macrocell outside 1..64");
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
    if (v->stats) cudaFree(v->stats);
    delete v;
}

extern "C" vdbc_status vdbc_render_dense(const vdbc_volume* vol, const vdbc_camera* camera, const vdbc_medium* medium,
                                         int32_t spp, uint64_t seed, float* rgba_out, int32_t out_on_device,
                                         void* stream)
{
    clear_error();
    if (!vol) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_render_dense: volume is null");
    Majorants mj{vol->mcmax, vol->macrocell, vol->mcdims[0], vol->mcdims[1], vol->mcdims[2],
                 vol->dims[0], vol->dims[1], vol->dims[2]};
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
    return VDBC_OK;
}
