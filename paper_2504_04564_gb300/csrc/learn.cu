// learn.cu -- the learned leaf codec (a project extension: the paper's
// Section 2.3 cites NeuralVDB's network-decoded leaves only as related work,
// too slow there for real time).
//
// vdbc_learn turns an encoded grid into a learned grid:
//  1. per leaf: its position and the (scale, offset) of its values (range
//     and minimum, as the FP16 payload defines them);
//  2. auto-decoder training: the shared network and one latent per leaf are
//     fitted jointly to the leaves' normalised values (mean squared error,
//     Adam).  Each step draws S voxels of every leaf, one uniformly from each
//     stratum of 512 / S consecutive voxels; the forward and backward passes
//     run in FP32 on the CUDA cores (k_mlp_grad);
//  3. every leaf is decoded through the tensor-core network, the render's own
//     arithmetic, and its largest error against the source is measured;
//  4. leaves over the error bound keep a raw FP16 payload (the worst first,
//     as far as the byte budget allows); the others keep only a bf16 latent;
//  5. the learned grid is assembled (tree tables copied, leaf entries
//     renumbered: raw leaves by rank, neural leaves as kNeural | rank) and
//     its macrocell ranges are taken from the decoded values.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "learn.cuh"
#include "vdbc_host.h"

namespace vdbc {
namespace {

constexpr int kTrainThreads = 128;     // samples per tile = threads of k_mlp_grad
constexpr int kXs = 20;                // row stride of the inputs in shared memory
constexpr int kHs = 36;                // row stride of activations / their gradients (16-byte rows)
constexpr int kPart = 1792;            // one block's partial gradient (>= kMlpParams)
constexpr uint32_t kDrawTag = 0x4C454146u;   // fourth counter word of the voxel draws
constexpr uint32_t kInitTag = 0x494E4954u;   // fourth counter word of the weight initialisation
constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kEps = 1e-8f;
constexpr size_t kTrainSmem =
    (size_t)(32 * kXs + 32 + 1024 + 32 + 32 + 4 + kTrainThreads * kXs + 4 * kTrainThreads * kHs + kTrainThreads) * 4;

__device__ __forceinline__ uint32_t okey(uint32_t b) { return (b & 0x80000000u) ? ~b : (b | 0x80000000u); }
__device__ __forceinline__ uint32_t okey_inv(uint32_t k) { return (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k; }

// ---------------------------------------------------------------- leaf positions
// origin of every upper node (in units of 4096 voxels), of every lower node
// (units of 128) and the linear position (lk * nly + lj) * nlx + li of every leaf
__global__ void k_upper_origin(const uint32_t* __restrict__ root, int rx, int ry, int nroot, int3* __restrict__ uo)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nroot) return;
    uint32_t e = root[r];
    if (!(e & kTile)) uo[e] = make_int3(r % rx, (r / rx) % ry, r / (rx * ry));
}

__global__ void k_lower_origin(const uint32_t* __restrict__ upper, long long n, const int3* __restrict__ uo,
                               int3* __restrict__ lo)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t e = upper[i];
    if (e & kTile) return;
    int3 o = uo[i / kUpperN];
    int a = (int)(i % kUpperN);
    lo[e] = make_int3(o.x * 32 + (a & 31), o.y * 32 + ((a >> 5) & 31), o.z * 32 + (a >> 10));
}

__global__ void k_leaf_pos(const uint32_t* __restrict__ lower, long long n, const int3* __restrict__ lo, int nlx,
                           int nly, uint32_t* __restrict__ pos)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t e = lower[i];
    if (e & kTile) return;
    int3 o = lo[i / kLowerN];
    int b = (int)(i % kLowerN);
    int li = o.x * 16 + (b & 15), lj = o.y * 16 + ((b >> 4) & 15), lk = o.z * 16 + (b >> 8);
    pos[e & ~kNeural] = (uint32_t)(((long long)lk * nly + lj) * nlx + li);
}

// (scale, offset) of each source leaf: range and minimum of its decoded values
// in the total order of the bit patterns (-0 before +0), one warp per leaf
__global__ void k_leaf_range(GridView src, long long nleaves, float2* __restrict__ lmeta)
{
    long long leaf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (leaf >= nleaves) return;
    float2 sm = src.payload != 0 ? __ldg(src.meta + leaf) : make_float2(0.f, 0.f);
    uint32_t kmin = 0xffffffffu, kmax = 0;
    for (int n = lane; n < kLeafN; n += 32) {
        uint32_t k = okey(__float_as_uint(leaf_value_t<-1>(src, (uint32_t)leaf, n, sm)));
        kmin = min(kmin, k);
        kmax = max(kmax, k);
    }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    float off = __uint_as_float(okey_inv(kmin));
    float scale = __fsub_rn(__uint_as_float(okey_inv(kmax)), off);
    if (lane == 0) lmeta[leaf] = make_float2(scale, off);
}

// per-leaf flags from the per-position arrays: force (0 by error, 1 neural, 2 raw),
// initial latents; trains[] = 1 for leaves that take part in training
__global__ void k_gather_leaf(const uint32_t* __restrict__ pos, long long nleaves, const uint8_t* __restrict__ force_pos,
                              const float* __restrict__ lat_pos, uint8_t* __restrict__ force, float* __restrict__ lat,
                              uint32_t* __restrict__ trains)
{
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nleaves) return;
    uint32_t p = pos[l];
    uint8_t f = force_pos ? force_pos[p] : 0;
    if (f > 2) f = 0;
    force[l] = f;
    trains[l] = f != 2 ? 1u : 0u;
#pragma unroll
    for (int c = 0; c < kMlpLatent; ++c) lat[l * kMlpLatent + c] = lat_pos ? lat_pos[(size_t)p * kMlpLatent + c] : 0.0f;
}

__global__ void k_compact(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ rank, long long n,
                          uint32_t* __restrict__ list)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) list[rank[i]] = (uint32_t)i;
}

// seeded initialisation: weights uniform in +-sqrt(6 / fan_in) (He et al.,
// 2015), biases zero except b3 = 1/2, the middle of the normalised range
__global__ void k_init_params(float* __restrict__ p, uint32_t k0, uint32_t k1)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    float fan = 0.0f;
    if (i < kOffB1) fan = (float)kMlpIn;
    else if (i >= kOffW2 && i < kOffB2) fan = (float)kMlpHid;
    else if (i >= kOffW3 && i < kOffB3) fan = (float)kMlpHid;
    if (fan == 0.0f) { p[i] = i == kOffB3 ? 0.5f : 0.0f; return; }
    U4 r = philox4x32_10((uint32_t)i, 0u, 0u, kInitTag, k0, k1);
    p[i] = (2.0f * u01(r.x) - 1.0f) * sqrtf(6.0f / fan);
}

// ---------------------------------------------------------------- training
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// samples given explicitly: n rows of 19 inputs and their targets
struct ExplicitSamples {
    static constexpr bool kLeaf = false;
    const float* X;
    const float* T;
    __device__ __forceinline__ float get(long long q, float* row) const
    {
        const float* p = X + q * kMlpIn;
#pragma unroll
        for (int c = 0; c < 5; ++c)
            st4(row + 4 * c, __ldg(p + 4 * c), __ldg(p + 4 * c + 1), __ldg(p + 4 * c + 2),
                4 * c + 3 < kMlpIn ? __ldg(p + 4 * c + 3) : 0.0f);
        return __ldg(T + q);
    }
};

// samples drawn from the leaves: sample q = s-th voxel of training leaf q / S
struct LeafSamples {
    static constexpr bool kLeaf = true;
    GridView src;
    const uint32_t* list;      // training leaves
    const uint32_t* pos;       // leaf -> linear position
    const float2* lmeta;       // leaf -> (scale, offset)
    const float* lat;          // leaf -> FP32 latent (16)
    int lg_s;                  // log2 S
    uint32_t step, k0, k1;
    __device__ __forceinline__ float get(long long q, float* row) const
    {
        const uint32_t leaf = __ldg(list + (q >> lg_s));
        const int s = (int)(q & ((1 << lg_s) - 1));
        const int stratum = kLeafN >> lg_s;
        U4 r = philox4x32_10(__ldg(pos + leaf), step, (uint32_t)s, kDrawTag, k0, k1);
        const int n = s * stratum + (int)(r.x & (uint32_t)(stratum - 1));
        const float2 sm = src.payload != 0 ? __ldg(src.meta + leaf) : make_float2(0.f, 0.f);
        const float v = leaf_value_t<-1>(src, leaf, n, sm);
        const float2 lm = __ldg(lmeta + leaf);
        const float4* L = reinterpret_cast<const float4*>(lat + (size_t)leaf * kMlpLatent);
        const float4 z0 = __ldg(L), z1 = __ldg(L + 1), z2 = __ldg(L + 2), z3 = __ldg(L + 3);
        st4(row, __fdiv_rn((float)(n & 7), 7.0f), __fdiv_rn((float)((n >> 3) & 7), 7.0f),
            __fdiv_rn((float)(n >> 6), 7.0f), z0.x);
        st4(row + 4, z0.y, z0.z, z0.w, z1.x);
        st4(row + 8, z1.y, z1.z, z1.w, z2.x);
        st4(row + 12, z2.y, z2.z, z2.w, z3.x);
        st4(row + 16, z3.y, z3.z, z3.w, 0.0f);
        return lm.x != 0.0f ? __fdiv_rn(__fsub_rn(v, lm.y), lm.x) : 0.0f;
    }
};

// Forward and backward of kTrainThreads samples per tile, one sample per
// thread; the weight gradients are reduced over the tile in shared memory by
// thread-owned groups of four entries, in a fixed order, and each block
// writes one partial gradient (summed by k_sum_parts, again in fixed order),
// so a run is bit-reproducible on a given device.  Explicit samples write
// their input gradients to gx[q * 19 + k]; leaf samples sum the latent part
// over each leaf's S samples (S divides the tile) into gx[leaf * 16 + c].
template <class Src>
__global__ void __launch_bounds__(kTrainThreads) k_mlp_grad(Src src, long long n, float inv_n,
                                                            const float* __restrict__ params, float* __restrict__ part,
                                                            double* __restrict__ loss_part, float* __restrict__ gx)
{
    extern __shared__ float4 s_f4[];
    float* W1s = reinterpret_cast<float*>(s_f4);     // [32][20]
    float* b1s = W1s + 32 * kXs;
    float* W2s = b1s + 32;                           // [32][32]
    float* b2s = W2s + 1024;
    float* w3s = b2s + 32;
    float* b3s = w3s + 32;                           // [4]
    float* X = b3s + 4;                              // [128][20]
    float* H1 = X + kTrainThreads * kXs;             // [128][36] each
    float* H2 = H1 + kTrainThreads * kHs;
    float* DH1 = H2 + kTrainThreads * kHs;
    float* DH2 = DH1 + kTrainThreads * kHs;
    float* DY = DH2 + kTrainThreads * kHs;           // [128]
    const int tid = threadIdx.x;
    for (int e = tid; e < 32 * kXs; e += blockDim.x) {
        int i = e / kXs, k = e % kXs;
        W1s[e] = k < kMlpIn ? params[kOffW1 + i * kMlpIn + k] : 0.0f;
    }
    for (int e = tid; e < 1024; e += blockDim.x) W2s[e] = params[kOffW2 + e];
    for (int e = tid; e < 32; e += blockDim.x) {
        b1s[e] = params[kOffB1 + e];
        b2s[e] = params[kOffB2 + e];
        w3s[e] = params[kOffW3 + e];
    }
    if (tid < 4) b3s[tid] = tid == 0 ? params[kOffB3] : 0.0f;
    __syncthreads();

    // owned gradient groups: W1 groups tid, tid+128 (< 160: row g/5, columns
    // 4(g%5)..+3), W2 groups tid, tid+128 (row g/8, columns 4(g%8)..+3), and
    // vector group tid (< 25: b1, b2, w3 in fours, then b3)
    float4 aw1[2], aw2[2], av;
    aw1[0] = aw1[1] = aw2[0] = aw2[1] = av = make_float4(0.f, 0.f, 0.f, 0.f);
    double lacc = 0.0;
    const long long ntiles = (n + kTrainThreads - 1) / kTrainThreads;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long q = tile * kTrainThreads + tid;
        const bool valid = q < n;
        // forward, one layer's vector live at a time: each layer's output
        // goes to this thread's row in shared memory, four values at a time
        float* xr = X + tid * kXs;
        float* h1r = H1 + tid * kHs;
        float* h2r = H2 + tid * kHs;
        float tg = 0.0f;
        if (valid) {
            tg = src.get(q, xr);
        } else {
#pragma unroll
            for (int c = 0; c < 5; ++c) st4(xr + 4 * c, 0.f, 0.f, 0.f, 0.f);
        }
        float dx[kXs];
        {
            float x[kXs];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                float4 v = ld4(xr + 4 * c);
                x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
            }
#pragma unroll
            for (int i4 = 0; i4 < 8; ++i4) {
                float hv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = 4 * i4 + j;
                    float a = b1s[i];
#pragma unroll
                    for (int c = 0; c < 5; ++c) {
                        float4 ww = ld4(W1s + i * kXs + 4 * c);
                        a = fmaf(ww.x, x[4 * c], a); a = fmaf(ww.y, x[4 * c + 1], a);
                        a = fmaf(ww.z, x[4 * c + 2], a); a = fmaf(ww.w, x[4 * c + 3], a);
                    }
                    hv[j] = a > 0.0f ? a : 0.0f;
                }
                st4(h1r + 4 * i4, hv[0], hv[1], hv[2], hv[3]);
            }
        }
        float dy;
        asm volatile("" ::: "memory");
        {
            float h1[kMlpHid];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float4 v = ld4(h1r + 4 * c);
                h1[4 * c] = v.x; h1[4 * c + 1] = v.y; h1[4 * c + 2] = v.z; h1[4 * c + 3] = v.w;
            }
            float y = b3s[0];
#pragma unroll
            for (int i4 = 0; i4 < 8; ++i4) {
                float hv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = 4 * i4 + j;
                    float a = b2s[i];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float4 ww = ld4(W2s + i * 32 + 4 * c);
                        a = fmaf(ww.x, h1[4 * c], a); a = fmaf(ww.y, h1[4 * c + 1], a);
                        a = fmaf(ww.z, h1[4 * c + 2], a); a = fmaf(ww.w, h1[4 * c + 3], a);
                    }
                    hv[j] = a > 0.0f ? a : 0.0f;
                }
                y = fmaf(w3s[4 * i4], hv[0], y); y = fmaf(w3s[4 * i4 + 1], hv[1], y);
                y = fmaf(w3s[4 * i4 + 2], hv[2], y); y = fmaf(w3s[4 * i4 + 3], hv[3], y);
                st4(h2r + 4 * i4, hv[0], hv[1], hv[2], hv[3]);
            }
            const float e = valid ? y - tg : 0.0f;
            lacc += (double)e * (double)e;
            dy = 2.0f * e * inv_n;
        }
        // backward: dh2 = relu'(h2) dy w3, dh1 = relu'(h1) W2^T dh2, dx = W1^T dh1.
        // The compiler barrier makes the backward pass re-read the weights from
        // shared memory instead of keeping the forward pass's 1.6k values live.
        asm volatile("" ::: "memory");
        {
            float dh1[kMlpHid];
#pragma unroll
            for (int k = 0; k < kMlpHid; ++k) dh1[k] = 0.0f;
#pragma unroll
            for (int i4 = 0; i4 < 8; ++i4) {
                const float4 hv = ld4(h2r + 4 * i4);
                const float d[4] = {hv.x > 0.0f ? dy * w3s[4 * i4] : 0.0f, hv.y > 0.0f ? dy * w3s[4 * i4 + 1] : 0.0f,
                                    hv.z > 0.0f ? dy * w3s[4 * i4 + 2] : 0.0f, hv.w > 0.0f ? dy * w3s[4 * i4 + 3] : 0.0f};
                st4(DH2 + tid * kHs + 4 * i4, d[0], d[1], d[2], d[3]);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float4 ww = ld4(W2s + (4 * i4 + j) * 32 + 4 * c);
                        dh1[4 * c] = fmaf(ww.x, d[j], dh1[4 * c]); dh1[4 * c + 1] = fmaf(ww.y, d[j], dh1[4 * c + 1]);
                        dh1[4 * c + 2] = fmaf(ww.z, d[j], dh1[4 * c + 2]); dh1[4 * c + 3] = fmaf(ww.w, d[j], dh1[4 * c + 3]);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 hv = ld4(h1r + 4 * c);
                dh1[4 * c] = hv.x > 0.0f ? dh1[4 * c] : 0.0f; dh1[4 * c + 1] = hv.y > 0.0f ? dh1[4 * c + 1] : 0.0f;
                dh1[4 * c + 2] = hv.z > 0.0f ? dh1[4 * c + 2] : 0.0f; dh1[4 * c + 3] = hv.w > 0.0f ? dh1[4 * c + 3] : 0.0f;
                st4(DH1 + tid * kHs + 4 * c, dh1[4 * c], dh1[4 * c + 1], dh1[4 * c + 2], dh1[4 * c + 3]);
            }
#pragma unroll
            for (int k = 0; k < kXs; ++k) dx[k] = 0.0f;
            asm volatile("" ::: "memory");
#pragma unroll
            for (int i = 0; i < kMlpHid; ++i) {
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    float4 ww = ld4(W1s + i * kXs + 4 * c);
                    dx[4 * c] = fmaf(ww.x, dh1[i], dx[4 * c]); dx[4 * c + 1] = fmaf(ww.y, dh1[i], dx[4 * c + 1]);
                    dx[4 * c + 2] = fmaf(ww.z, dh1[i], dx[4 * c + 2]); dx[4 * c + 3] = fmaf(ww.w, dh1[i], dx[4 * c + 3]);
                }
            }
        }
        DY[tid] = dy;
        __syncthreads();
        // weight gradients of the tile, samples in order
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int g1 = tid + h * kTrainThreads;
            if (g1 < 160) {
                const int i = g1 / 5, c = g1 % 5;
                float4 a = aw1[h];
                for (int s = 0; s < kTrainThreads; ++s) {
                    const float d = DH1[s * kHs + i];
                    const float4 xv = *reinterpret_cast<const float4*>(X + s * kXs + 4 * c);
                    a.x = fmaf(d, xv.x, a.x); a.y = fmaf(d, xv.y, a.y); a.z = fmaf(d, xv.z, a.z); a.w = fmaf(d, xv.w, a.w);
                }
                aw1[h] = a;
            }
            const int g2 = tid + h * kTrainThreads;
            {
                const int i = g2 >> 3, c = g2 & 7;
                float4 a = aw2[h];
                for (int s = 0; s < kTrainThreads; ++s) {
                    const float d = DH2[s * kHs + i];
                    const float4 hv = *reinterpret_cast<const float4*>(H1 + s * kHs + 4 * c);
                    a.x = fmaf(d, hv.x, a.x); a.y = fmaf(d, hv.y, a.y); a.z = fmaf(d, hv.z, a.z); a.w = fmaf(d, hv.w, a.w);
                }
                aw2[h] = a;
            }
        }
        if (tid < 25) {
            float4 a = av;
            for (int s = 0; s < kTrainThreads; ++s) {
                float4 v;
                if (tid < 8) v = *reinterpret_cast<const float4*>(DH1 + s * kHs + 4 * tid);
                else if (tid < 16) v = *reinterpret_cast<const float4*>(DH2 + s * kHs + 4 * (tid - 8));
                else if (tid < 24) {
                    const float d = DY[s];
                    float4 hv = *reinterpret_cast<const float4*>(H2 + s * kHs + 4 * (tid - 16));
                    v = make_float4(d * hv.x, d * hv.y, d * hv.z, d * hv.w);
                } else {
                    v = make_float4(DY[s], 0.f, 0.f, 0.f);
                }
                a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w;
            }
            av = a;
        }
        __syncthreads();
        if constexpr (Src::kLeaf) {
            // latent gradient of each leaf of the tile: the sum over its S samples
            float* DX = H2;
#pragma unroll
            for (int c = 0; c < 4; ++c) st4(DX + tid * kHs + 4 * c, dx[3 + 4 * c], dx[4 + 4 * c], dx[5 + 4 * c], dx[6 + 4 * c]);
            __syncthreads();
            const int S = 1 << src.lg_s, per = kTrainThreads >> src.lg_s;
            if (tid < per * kMlpLatent) {
                const int a = tid >> 4, c = tid & 15;
                const long long first = tile * kTrainThreads + (long long)a * S;
                if (first < n) {
                    float sum = 0.0f;
                    for (int s = 0; s < S; ++s) sum += DX[(a * S + s) * kHs + c];
                    gx[(size_t)__ldg(src.list + (first >> src.lg_s)) * kMlpLatent + c] = sum;
                }
            }
            __syncthreads();
        } else {
            if (valid && gx) {
#pragma unroll
                for (int k = 0; k < kMlpIn; ++k) gx[q * kMlpIn + k] = dx[k];
            }
        }
    }
    // this block's partial gradient, in parameter order
    float* P = part + (size_t)blockIdx.x * kPart;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int g1 = tid + h * kTrainThreads;
        if (g1 < 160) {
            const int i = g1 / 5, c = g1 % 5;
            const float v[4] = {aw1[h].x, aw1[h].y, aw1[h].z, aw1[h].w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (4 * c + j < kMlpIn) P[kOffW1 + i * kMlpIn + 4 * c + j] = v[j];
        }
        const int g2 = tid + h * kTrainThreads;
        const int i = g2 >> 3, c = g2 & 7;
        st4(P + kOffW2 + i * 32 + 4 * c, aw2[h].x, aw2[h].y, aw2[h].z, aw2[h].w);
    }
    if (tid < 8) st4(P + kOffB1 + 4 * tid, av.x, av.y, av.z, av.w);
    else if (tid < 16) st4(P + kOffB2 + 4 * (tid - 8), av.x, av.y, av.z, av.w);
    else if (tid < 24) st4(P + kOffW3 + 4 * (tid - 16), av.x, av.y, av.z, av.w);
    else if (tid == 24) P[kOffB3] = av.x;
    // loss partial: warp sums, then the warps in order
    __shared__ double s_loss[kTrainThreads / 32];
    for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, o);
    if ((tid & 31) == 0) s_loss[tid >> 5] = lacc;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kTrainThreads / 32; ++w) t += s_loss[w];
        loss_part[blockIdx.x] = t;
    }
}

// grad = sum of the blocks' partials in block order; loss = their loss sum / n
__global__ void k_sum_parts(const float* __restrict__ part, int nb, float* __restrict__ grad,
                            const double* __restrict__ loss_part, double inv_n, double* __restrict__ loss)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kMlpParams) {
        float s = 0.0f;
        for (int b = 0; b < nb; ++b) s += part[(size_t)b * kPart + e];
        grad[e] = s;
    }
    if (e == 0 && loss) {
        double l = 0.0;
        for (int b = 0; b < nb; ++b) l += loss_part[b];
        loss[0] = l * inv_n;
    }
}

// one Adam step (Kingma and Ba, 2015) with bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float c1, float c2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = kBeta1 * m[i] + (1.0f - kBeta1) * gi;
        const float vi = kBeta2 * v[i] + (1.0f - kBeta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + kEps);
    }
}

// latents to their stored form: bf16 pairs, (z_2k, z_2k+1) in word k
__global__ void k_to_bf16(const float* __restrict__ a, uint32_t* __restrict__ b, long long nwords)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nwords) b[i] = pack_bf16(a[2 * i], a[2 * i + 1]);
}

// the network's B fragments and biases from the FP32 parameters
__global__ void k_pack_net(const float* __restrict__ params, uint2* __restrict__ frag, float* __restrict__ bias)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kMlpFrags * 32) frag[i] = mlp_frag(params, i >> 5, i & 31);
    if (i < kMlpHid) {
        bias[i] = params[kOffB1 + i];
        bias[kMlpHid + i] = params[kOffB2 + i];
    }
    if (i == 0) bias[2 * kMlpHid] = params[kOffB3];
}

// ---------------------------------------------------------------- decode through the network
// one warp per neural leaf, two 16-row tiles per pass: leaf id -> latent
// lat[id * 8] (bf16 pairs), (scale, offset) meta[id]; decoded = offset + scale * clamp(y, 0, 1).
// out (if given) receives the 512 decoded values at out[(out_base + id) * 512];
// err (if given) the largest |decoded - cmp| with cmp the source leaf `id`.
constexpr int kDecWarps = 8;
__global__ void __launch_bounds__(kDecWarps * 32) k_neural_decode(const uint32_t* __restrict__ lat,
                                                                 const float2* __restrict__ meta, long long count,
                                                                 const uint32_t* __restrict__ only,
                                                                 const uint2* __restrict__ frag,
                                                                 const float* __restrict__ bias, float* __restrict__ out,
                                                                 long long out_base, GridView cmp, float* __restrict__ err)
{
    __shared__ __align__(16) uint32_t s_rows[kDecWarps][2][256];
    __shared__ float s_out[kDecWarps][2][16];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long id = (long long)blockIdx.x * kDecWarps + wid;
    if (id >= count) return;                     // warp-uniform
    if (only && !only[id]) return;               // warp-uniform
    const uint32_t* z = lat + id * (kMlpLatent / 2);
    const float2 m = __ldg(meta + id);
    const float2 csm = (err && cmp.payload != 0) ? __ldg(cmp.meta + id) : make_float2(0.f, 0.f);
    const int r = lane & 15, half = lane >> 4;
    float e = 0.0f;
    for (int t = 0; t < 32; t += 2) {
        const int n = (t + half) * 16 + r;
        mlp_row(s_rows[wid][half], r, n, z);
        __syncwarp();
        mlp_tile(s_rows[wid][0], frag, bias, s_out[wid][0]);
        mlp_tile(s_rows[wid][1], frag, bias, s_out[wid][1]);
        __syncwarp();
        const float y = s_out[wid][half][r];
        const float dec = __fmaf_rn(m.x, fminf(fmaxf(y, 0.0f), 1.0f), m.y);
        if (out) out[(size_t)(out_base + id) * kLeafN + n] = dec;
        if (err) e = fmaxf(e, fabsf(__fsub_rn(dec, leaf_value_t<-1>(cmp, (uint32_t)id, n, csm))));
        __syncwarp();
    }
    if (err) {
        for (int o = 16; o > 0; o >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (lane == 0) err[id] = e;
    }
}

// ---------------------------------------------------------------- classification and assembly
// candidates for a raw payload: error over the bound (key = error bits), or forced
__global__ void k_classify(const float* __restrict__ err, const uint8_t* __restrict__ force, long long n,
                           float max_error, unsigned long long* __restrict__ key, uint8_t* __restrict__ skip,
                           unsigned long long* __restrict__ counts)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint8_t f = force[i];
    const float e = err[i];
    const bool cand = f == 0 && !(e <= max_error);     // NaN errors are candidates too
    key[i] = cand ? (unsigned long long)__float_as_uint(isnan(e) ? INFINITY : e) : 0ull;
    skip[i] = cand ? 0 : 1;
    if (f == 2) atomicAdd(&counts[0], 1ull);
    if (cand) atomicAdd(&counts[1], 1ull);
}

__global__ void k_raw_flags(const uint8_t* __restrict__ force, const uint8_t* __restrict__ chosen, long long n,
                            uint32_t* __restrict__ raw, uint32_t* __restrict__ neural)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool r = force[i] == 2 || (force[i] == 0 && chosen[i]);
    raw[i] = r ? 1u : 0u;
    neural[i] = r ? 0u : 1u;
}

__global__ void k_remap_lower(const uint32_t* __restrict__ in, long long n, const uint32_t* __restrict__ raw,
                              const uint32_t* __restrict__ raw_rank, const uint32_t* __restrict__ neural_rank,
                              uint32_t* __restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t e = in[i];
    if (e & kTile) { out[i] = e; return; }
    out[i] = raw[e] ? raw_rank[e] : (kNeural | neural_rank[e]);
}

// raw leaves: FP16 codes of (v - offset) / scale, as the FP16 payload of the encoder
__global__ void k_fill_raw(GridView src, const float2* __restrict__ lmeta, const uint32_t* __restrict__ raw,
                           const uint32_t* __restrict__ raw_rank, long long nleaves, __half* __restrict__ leaves,
                           float2* __restrict__ meta)
{
    long long leaf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (leaf >= nleaves || !raw[leaf]) return;
    const float2 sm = src.payload != 0 ? __ldg(src.meta + leaf) : make_float2(0.f, 0.f);
    const float2 lm = lmeta[leaf];
    const size_t r = raw_rank[leaf];
    if (lane == 0) meta[r] = lm;
    for (int n = lane; n < kLeafN; n += 32) {
        const float v = leaf_value_t<-1>(src, (uint32_t)leaf, n, sm);
        const float t = lm.x != 0.0f ? __fdiv_rn(__fsub_rn(v, lm.y), lm.x) : 0.0f;
        leaves[r * kLeafN + n] = __float2half_rn(t);
    }
}

__global__ void k_fill_neural(const uint32_t* __restrict__ lat, const float2* __restrict__ lmeta,
                              const uint32_t* __restrict__ neural, const uint32_t* __restrict__ neural_rank,
                              long long nleaves, uint32_t* __restrict__ latents, float2* __restrict__ nmeta)
{
    long long leaf = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= nleaves || !neural[leaf]) return;
    const size_t r = neural_rank[leaf];
    const uint4* a = reinterpret_cast<const uint4*>(lat + leaf * (kMlpLatent / 2));
    uint4* b = reinterpret_cast<uint4*>(latents + r * (kMlpLatent / 2));
    b[0] = a[0];
    b[1] = a[1];
    nmeta[r] = lmeta[leaf];
}

// materialised view: neural entries renumbered after the raw leaves
__global__ void k_remap_materialized(const uint32_t* __restrict__ in, long long n, uint32_t n_raw,
                                     uint32_t* __restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t e = in[i];
    out[i] = (!(e & kTile) && (e & kNeural)) ? n_raw + (e & ~kNeural) : e;
}

__global__ void k_raw_decode(GridView g, long long n_raw, float* __restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_raw * kLeafN) return;
    const long long leaf = i / kLeafN;
    out[i] = leaf_value_t<1>(g, (uint32_t)leaf, (int)(i % kLeafN), __ldg(g.meta + leaf));
}

unsigned blocks(long long n, int t) { return (unsigned)std::max<long long>(1, (n + t - 1) / t); }

int sm_count_dev()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// device allocations of one call, released on every exit path
struct Pool {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Pool(cudaStream_t st) : s(st) {}
    template <typename T>
    vdbc_status get(T** p, size_t count)
    {
        void* q = nullptr;
        vdbc_status st = dev_alloc(&q, std::max<size_t>(count * sizeof(T), 16), s);
        if (st != VDBC_OK) return st;
        ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return VDBC_OK;
    }
    ~Pool()
    {
        for (void* q : ptrs) dev_free(q, s);
    }
};

// gradient of the loss over n explicit or drawn samples into grad (and the
// loss, if asked); part / loss_part hold grid partials
template <class Src>
vdbc_status run_grad(const Src& src, long long n, const float* params, float* part, double* loss_part, int grid,
                     float* grad, double* loss, float* gx, cudaStream_t s)
{
    auto kern = k_mlp_grad<Src>;
    VDBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem));
    KLAUNCH(kern<<<grid, kTrainThreads, kTrainSmem, s>>>(src, n, (float)(1.0 / (double)n), params, part, loss_part, gx));
    KLAUNCH(k_sum_parts<<<blocks(kMlpParams, 256), 256, 0, s>>>(part, grid, grad, loss_part, 1.0 / (double)n, loss));
    VDBC_CUDA(cudaGetLastError());
    return VDBC_OK;
}

int grad_grid(long long n)
{
    static int per_sm = -1;
    if (per_sm < 0) {
        auto kern = k_mlp_grad<LeafSamples>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTrainThreads, kTrainSmem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    long long tiles = (n + kTrainThreads - 1) / kTrainThreads;
    return (int)std::max<long long>(1, std::min<long long>(tiles, (long long)sm_count_dev() * per_sm));
}

}  // namespace

vdbc_status materialize_learned(const vdbc_grid* g, cudaStream_t s, Materialized* m)
{
    const vdbc_grid_info& in = g->info;
    const long long n_raw = in.n_leaves, n_neu = in.n_neural, nlow = in.n_lower * (long long)kLowerN;
    VDBC_TRY(dev_alloc(&m->lower, (size_t)std::max<long long>(nlow, 1) * 4, s));
    VDBC_TRY(dev_alloc(&m->leaves, (size_t)std::max<long long>(n_raw + n_neu, 1) * kLeafN * 4, s));
    float* leaves = static_cast<float*>(m->leaves);
    if (nlow > 0)
        KLAUNCH(k_remap_materialized<<<blocks(nlow, 256), 256, 0, s>>>(g->view.lower, nlow, (uint32_t)n_raw,
                                                                       static_cast<uint32_t*>(m->lower)));
    if (n_raw > 0) KLAUNCH(k_raw_decode<<<blocks(n_raw * kLeafN, 256), 256, 0, s>>>(g->view, n_raw, leaves));
    if (n_neu > 0)
        KLAUNCH(k_neural_decode<<<blocks(n_neu, kDecWarps), kDecWarps * 32, 0, s>>>(
            g->view.latents, g->view.nmeta, n_neu, nullptr, g->view.mlp_frag, g->view.mlp_bias, leaves, n_raw,
            g->view, nullptr));
    VDBC_CUDA(cudaGetLastError());
    m->view = g->view;
    m->view.payload = VDBC_FP32;
    m->view.lower = static_cast<const uint32_t*>(m->lower);
    m->view.leaves = m->leaves;
    return VDBC_OK;
}

vdbc_status build_learned_macrocells(vdbc_grid* g, cudaStream_t s)
{
    Materialized m;
    vdbc_status st = materialize_learned(g, s, &m);
    if (st == VDBC_OK) {
        char* base = static_cast<char*>(g->block);
        st = macrocells_of_view(m.view, reinterpret_cast<float*>(base + g->off_mcmin),
                                reinterpret_cast<float*>(base + g->off_mcmax), s);
    }
    m.release(s);
    return st;
}

}  // namespace vdbc

using namespace vdbc;

namespace {
vdbc_status check_learn_params(const vdbc_learn_params* p)
{
    if (!p) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: params is null");
    if (p->steps < 0 || p->steps > 1000000) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: steps %d outside 0..1e6", p->steps);
    const int S = p->samples_per_leaf;
    if (S != 16 && S != 32 && S != 64 && S != 128)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: samples_per_leaf %d not one of 16, 32, 64, 128", S);
    if (p->steps > 0 && (!(p->lr > 0.0f) || !(p->lr_latent > 0.0f) || !std::isfinite(p->lr) || !std::isfinite(p->lr_latent)))
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: learning rates must be positive and finite");
    if (!(p->max_error >= 0.0f)) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: max_error must be >= 0");
    return VDBC_OK;
}
}  // namespace

extern "C" vdbc_status vdbc_learn(const vdbc_grid* src, const vdbc_learn_params* lp, void* stream, vdbc_grid** out,
                                  double* loss_out)
{
    clear_error();
    if (!src || !out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: null argument");
    *out = nullptr;
    VDBC_TRY(check_learn_params(lp));
    if (src->info.payload == VDBC_LEARNED) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: the source is already learned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const vdbc_grid_info& si = src->info;
    const long long nl = si.n_leaves;
    const int nlx = (si.dims[0] + 7) / 8, nly = (si.dims[1] + 7) / 8;
    const int lg_s = __builtin_ctz((unsigned)lp->samples_per_leaf);
    const uint32_t k0 = (uint32_t)lp->seed, k1 = (uint32_t)(lp->seed >> 32);
    Pool pool(s);

    // ---- 1. leaf positions, ranges, flags, initial latents
    int3 *uo = nullptr, *lo = nullptr;
    uint32_t *pos = nullptr, *trains = nullptr, *trank = nullptr, *list = nullptr, *total = nullptr, *scan_tmp = nullptr;
    float2* lmeta = nullptr;
    uint8_t* force = nullptr;
    float *lat = nullptr, *lat_m = nullptr, *lat_v = nullptr, *glat = nullptr;
    const long long nroot = (long long)src->view.rx * src->view.ry * src->view.rz;
    VDBC_TRY(pool.get(&uo, std::max<long long>(si.n_upper, 1)));
    VDBC_TRY(pool.get(&lo, std::max<long long>(si.n_lower, 1)));
    VDBC_TRY(pool.get(&pos, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&lmeta, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&force, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&trains, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&trank, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&list, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&total, 4));
    VDBC_TRY(pool.get(&scan_tmp, scan_tmp_words(std::max<long long>(nl, 1))));
    VDBC_TRY(pool.get(&lat, std::max<long long>(nl, 1) * kMlpLatent));
    VDBC_TRY(pool.get(&lat_m, std::max<long long>(nl, 1) * kMlpLatent));
    VDBC_TRY(pool.get(&lat_v, std::max<long long>(nl, 1) * kMlpLatent));
    VDBC_TRY(pool.get(&glat, std::max<long long>(nl, 1) * kMlpLatent));
    if (nroot > 0) KLAUNCH(k_upper_origin<<<blocks(nroot, 256), 256, 0, s>>>(src->view.root, src->view.rx, src->view.ry, (int)nroot, uo));
    const long long nup = si.n_upper * (long long)kUpperN, nlow = si.n_lower * (long long)kLowerN;
    if (nup > 0) KLAUNCH(k_lower_origin<<<blocks(nup, 256), 256, 0, s>>>(src->view.upper, nup, uo, lo));
    if (nlow > 0) KLAUNCH(k_leaf_pos<<<blocks(nlow, 256), 256, 0, s>>>(src->view.lower, nlow, lo, nlx, nly, pos));
    if (nl > 0) {
        KLAUNCH(k_leaf_range<<<blocks(nl * 32, 256), 256, 0, s>>>(src->view, nl, lmeta));
        KLAUNCH(k_gather_leaf<<<blocks(nl, 256), 256, 0, s>>>(pos, nl, lp->force, lp->init_latents, force, lat, trains));
    }
    scan_u32(trains, trank, nl, scan_tmp, total, s);
    if (nl > 0) KLAUNCH(k_compact<<<blocks(nl, 256), 256, 0, s>>>(trains, trank, nl, list));
    uint32_t n_train = 0;
    VDBC_CUDA(cudaMemcpyAsync(&n_train, total, 4, cudaMemcpyDeviceToHost, s));
    VDBC_TRY(wait_stream(s));

    // ---- 2. training
    float *params = nullptr, *pm = nullptr, *pv = nullptr, *grad = nullptr, *part = nullptr;
    double *loss_part = nullptr, *loss_hist = nullptr;
    VDBC_TRY(pool.get(&params, kMlpParams));
    VDBC_TRY(pool.get(&pm, kMlpParams));
    VDBC_TRY(pool.get(&pv, kMlpParams));
    VDBC_TRY(pool.get(&grad, kMlpParams));
    VDBC_CUDA(cudaMemsetAsync(pm, 0, kMlpParams * 4, s));
    VDBC_CUDA(cudaMemsetAsync(pv, 0, kMlpParams * 4, s));
    VDBC_CUDA(cudaMemsetAsync(lat_m, 0, (size_t)std::max<long long>(nl, 1) * kMlpLatent * 4, s));
    VDBC_CUDA(cudaMemsetAsync(lat_v, 0, (size_t)std::max<long long>(nl, 1) * kMlpLatent * 4, s));
    VDBC_CUDA(cudaMemsetAsync(glat, 0, (size_t)std::max<long long>(nl, 1) * kMlpLatent * 4, s));
    if (lp->init_params) {
        VDBC_CUDA(cudaMemcpyAsync(params, lp->init_params, kMlpParams * 4, cudaMemcpyDefault, s));
    } else {
        KLAUNCH(k_init_params<<<blocks(kMlpParams, 256), 256, 0, s>>>(params, k0, k1));
    }
    const long long nsamp = (long long)n_train << lg_s;
    if (lp->steps > 0 && nsamp > 0) {
        const int grid = grad_grid(nsamp);
        VDBC_TRY(pool.get(&part, (size_t)grid * kPart));
        VDBC_TRY(pool.get(&loss_part, grid));
        VDBC_TRY(pool.get(&loss_hist, lp->steps));
        LeafSamples ls{src->view, list, pos, lmeta, lat, lg_s, 0u, k0, k1};
        for (int t = 0; t < lp->steps; ++t) {
            ls.step = (uint32_t)t;
            VDBC_TRY(run_grad(ls, nsamp, params, part, loss_part, grid, grad, loss_hist + t, glat, s));
            const float c1 = (float)(1.0 - std::pow((double)kBeta1, (double)(t + 1)));
            const float c2 = (float)(1.0 - std::pow((double)kBeta2, (double)(t + 1)));
            KLAUNCH(k_adam<<<blocks(kMlpParams, 256), 256, 0, s>>>(params, grad, pm, pv, kMlpParams, lp->lr, c1, c2));
            const long long nz = nl * kMlpLatent;
            KLAUNCH(k_adam<<<(unsigned)std::min<long long>(blocks(nz, 256), 4096), 256, 0, s>>>(lat, glat, lat_m, lat_v, nz,
                                                                                              lp->lr_latent, c1, c2));
        }
        VDBC_CUDA(cudaGetLastError());
        if (loss_out) VDBC_CUDA(cudaMemcpyAsync(loss_out, loss_hist, (size_t)lp->steps * 8, cudaMemcpyDeviceToHost, s));
    } else if (loss_out && lp->steps > 0) {
        for (int t = 0; t < lp->steps; ++t) loss_out[t] = 0.0;
    }

    // ---- 3. bf16 latents, network tables, per-leaf error through the tensor cores
    uint32_t* lath = nullptr;
    uint2* frag = nullptr;
    float *bias = nullptr, *err = nullptr;
    VDBC_TRY(pool.get(&lath, std::max<long long>(nl, 1) * (kMlpLatent / 2)));
    VDBC_TRY(pool.get(&frag, kMlpFrags * 32));
    VDBC_TRY(pool.get(&bias, kMlpBias));
    VDBC_TRY(pool.get(&err, std::max<long long>(nl, 1)));
    if (nl > 0) KLAUNCH(k_to_bf16<<<blocks(nl * (kMlpLatent / 2), 256), 256, 0, s>>>(lat, lath, nl * (kMlpLatent / 2)));
    KLAUNCH(k_pack_net<<<blocks(kMlpFrags * 32, 256), 256, 0, s>>>(params, frag, bias));
    VDBC_CUDA(cudaMemsetAsync(err, 0, (size_t)std::max<long long>(nl, 1) * 4, s));
    if (nl > 0)
        KLAUNCH(k_neural_decode<<<blocks(nl, kDecWarps), kDecWarps * 32, 0, s>>>(lath, lmeta, nl, trains, frag, bias,
                                                                                nullptr, 0, src->view, err));

    // ---- 4. raw or neural
    unsigned long long *key = nullptr, *cnt = nullptr;
    uint8_t *skip = nullptr, *chosen = nullptr;
    long long* sel_counts = nullptr;
    uint32_t *raw = nullptr, *neural = nullptr, *raw_rank = nullptr, *neural_rank = nullptr;
    VDBC_TRY(pool.get(&key, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&cnt, 2));
    VDBC_TRY(pool.get(&skip, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&chosen, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&sel_counts, 2));
    VDBC_TRY(pool.get(&raw, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&neural, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&raw_rank, std::max<long long>(nl, 1)));
    VDBC_TRY(pool.get(&neural_rank, std::max<long long>(nl, 1)));
    VDBC_CUDA(cudaMemsetAsync(cnt, 0, 16, s));
    if (nl > 0) KLAUNCH(k_classify<<<blocks(nl, 256), 256, 0, s>>>(err, force, nl, lp->max_error, key, skip, cnt));
    unsigned long long hc[2] = {0, 0};
    VDBC_CUDA(cudaMemcpyAsync(hc, cnt, 16, cudaMemcpyDeviceToHost, s));
    VDBC_TRY(wait_stream(s));
    const long long n_forced_raw = (long long)hc[0], n_cand = (long long)hc[1];
    long long take = n_cand;
    if (lp->max_bytes > 0) {
        // bytes with only the forced leaves raw, then 992 more per extra raw
        // leaf (a 1024-byte FP16 payload + 8-byte meta instead of a 32-byte
        // latent + 8-byte meta), keeping 1 KB for the 256-byte alignments
        vdbc_grid probe;
        probe.info = si;
        probe.info.payload = VDBC_LEARNED;
        probe.info.n_leaves = n_forced_raw;
        probe.info.n_neural = nl - n_forced_raw;
        layout(&probe);
        const long long room = (long long)lp->max_bytes - (long long)probe.block_bytes - 1024;
        take = std::min<long long>(n_cand, std::max<long long>(0, room / 992));
    }
    if (nl > 0) {
        select_largest(key, skip, (int)nl, take, chosen, sel_counts, s);
        KLAUNCH(k_raw_flags<<<blocks(nl, 256), 256, 0, s>>>(force, chosen, nl, raw, neural));
    }
    uint32_t* totals = total;   // [0] raw, [1] neural
    scan_u32(raw, raw_rank, nl, scan_tmp, totals, s);
    scan_u32(neural, neural_rank, nl, scan_tmp, totals + 1, s);
    uint32_t ht[2] = {0, 0};
    VDBC_CUDA(cudaMemcpyAsync(ht, totals, 8, cudaMemcpyDeviceToHost, s));
    VDBC_TRY(wait_stream(s));

    // ---- 5. the learned grid
    vdbc_grid* g = new vdbc_grid();
    g->info = si;
    g->info.payload = VDBC_LEARNED;
    g->info.n_leaves = ht[0];
    g->info.n_neural = ht[1];
    g->device = src->device;
    g->active = src->active;
    layout(g);
    vdbc_status st = dev_alloc(&g->block, g->block_bytes, s);
    if (st != VDBC_OK) { delete g; return st; }
    bind_view(g);
    char* b = static_cast<char*>(g->block);
    const char* sb = static_cast<const char*>(src->block);
    cudaError_t e = cudaMemsetAsync(g->block, 0, g->block_bytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + g->off_root, sb + src->off_root, (size_t)nroot * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && nup > 0) e = cudaMemcpyAsync(b + g->off_upper, sb + src->off_upper, (size_t)nup * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + g->off_tiles, sb + src->off_tiles, (size_t)si.n_tiles * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + g->off_params, params, kMlpParams * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + g->off_frag, frag, kMlpFrags * 32 * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + g->off_bias, bias, kMlpBias * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) { vdbc_grid_free(g); return cuda_status(e, "vdbc_learn: copies"); }
    if (nlow > 0)
        KLAUNCH(k_remap_lower<<<blocks(nlow, 256), 256, 0, s>>>(src->view.lower, nlow, raw, raw_rank, neural_rank,
                                                               reinterpret_cast<uint32_t*>(b + g->off_lower)));
    if (nl > 0) {
        KLAUNCH(k_fill_raw<<<blocks(nl * 32, 256), 256, 0, s>>>(src->view, lmeta, raw, raw_rank, nl,
                                                               reinterpret_cast<__half*>(b + g->off_leaves),
                                                               reinterpret_cast<float2*>(b + g->off_meta)));
        KLAUNCH(k_fill_neural<<<blocks(nl, 256), 256, 0, s>>>(lath, lmeta, neural, neural_rank, nl,
                                                              reinterpret_cast<uint32_t*>(b + g->off_latents),
                                                              reinterpret_cast<float2*>(b + g->off_nmeta)));
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) { vdbc_grid_free(g); return cuda_status(e, "vdbc_learn: assembly"); }
    st = build_macrocells(g, s);
    if (st == VDBC_OK) st = dev_alloc(reinterpret_cast<void**>(&g->stats), sizeof(DevStats), s);
    if (st == VDBC_OK) {
        e = cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s);
        if (e != cudaSuccess) st = cuda_status(e, "vdbc_learn: stats");
    }
    if (st == VDBC_OK) st = wait_stream(s);
    if (st != VDBC_OK) { vdbc_grid_free(g); return st; }
    *out = g;
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_learn_loss_grad(const float* params, const float* inputs, const float* targets, int64_t n,
                                            double* loss, float* grad_params, float* grad_inputs, void* stream)
{
    clear_error();
    if (!params || !inputs || !targets || !grad_params) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn_loss_grad: null argument");
    if (n < 1 || n > ((int64_t)1 << 31)) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn_loss_grad: n %lld outside 1..2^31", (long long)n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Pool pool(s);
    const int grid = grad_grid(n);
    float* part = nullptr;
    double *loss_part = nullptr, *dloss = nullptr;
    VDBC_TRY(pool.get(&part, (size_t)grid * kPart));
    VDBC_TRY(pool.get(&loss_part, grid));
    VDBC_TRY(pool.get(&dloss, 1));
    ExplicitSamples es{inputs, targets};
    VDBC_TRY(run_grad(es, n, params, part, loss_part, grid, grad_params, dloss, grad_inputs, s));
    double h = 0.0;
    VDBC_CUDA(cudaMemcpyAsync(&h, dloss, 8, cudaMemcpyDeviceToHost, s));
    VDBC_TRY(wait_stream(s));
    if (loss) *loss = h;
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_learn_get_params(const vdbc_grid* g, float* host_params)
{
    clear_error();
    if (!g || !host_params) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn_get_params: null argument");
    if (g->info.payload != VDBC_LEARNED) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn_get_params: not a learned grid");
    VDBC_CUDA(cudaMemcpy(host_params, static_cast<const char*>(g->block) + g->off_params, kMlpParams * 4,
                         cudaMemcpyDeviceToHost));
    return VDBC_OK;
}
