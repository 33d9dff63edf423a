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
//     run on the tensor cores in the precision the network is evaluated in
//     (bf16 operands, FP32 accumulation; k_mlp_grad);
//  3. every leaf is decoded through the tensor-core network, the render's own
//     arithmetic, and its largest error against the source is measured;
//  4. leaves over the error bound keep a raw FP16 payload (the worst first,
//     as far as the byte budget allows); the others keep only a bf16 latent;
//  5. the learned grid is assembled (tree tables copied, leaf entries
//     renumbered: raw leaves by rank, neural leaves as kNeural | rank) and
//     its macrocell ranges are taken from the decoded values.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "learn.cuh"
#include "tcgen05.cuh"
#include "vdbc_host.h"

namespace vdbc {
namespace {

constexpr int kPart = 1792;            // one block's partial gradient (>= kMlpParams)
constexpr uint32_t kDrawTag = 0x4C454146u;   // fourth counter word of the voxel draws
constexpr uint32_t kInitTag = 0x494E4954u;   // fourth counter word of the weight initialisation
constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kEps = 1e-8f;

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

// 16-float rows between leaf order and leaf-position order (training states)
__global__ void k_gather_rows(const uint32_t* __restrict__ pos, long long nleaves, const float* __restrict__ by_pos,
                              float* __restrict__ by_leaf)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaves * kMlpLatent) return;
    const long long l = i / kMlpLatent;
    by_leaf[i] = by_pos[(size_t)pos[l] * kMlpLatent + (i - l * kMlpLatent)];
}

__global__ void k_scatter_rows(const uint32_t* __restrict__ pos, long long nleaves, const float* __restrict__ by_leaf,
                               float* __restrict__ by_pos)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaves * kMlpLatent) return;
    const long long l = i / kMlpLatent;
    by_pos[(size_t)pos[l] * kMlpLatent + (i - l * kMlpLatent)] = by_leaf[i];
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
// ---------------------------------------------------------------- training on the tensor cores
// One warp trains on tiles of 16 samples with mma.sync.m16n8k16 (bf16 in,
// FP32 accumulate), at the precision the network is evaluated in:
//   forward   a1 = W1 x + b1, h1 = relu(a1), a2 = W2 bf(h1) + b2, h2 = relu(a2),
//             y = b3 + bf(w3) . bf(h2)   (x, W1, W2 as bf16; FP32 sums)
//   backward  dy = 2 (y - t) / n, dh2 = relu'(a2) dy bf(w3),
//             dh1 = relu'(a1) (bf(W2)^T bf(dh2)), dx = bf(W1)^T bf(dh1)
//   weights   gW2 = sum_m bf(dh2) bf(h1)^T and gW1 = sum_m bf(dh1) bf(x)^T as MMAs
//             over the tile's samples (A and B read transposed from shared
//             memory by ldmatrix.trans); gb1, gb2, gw3, gb3 in FP32.
// Weight gradients accumulate in registers over all of a warp's tiles; the
// block adds its warps in order and writes one partial (k_sum_parts adds the
// blocks in order), so a run is bit-reproducible on a device.
constexpr int kTcWarps = 4;
constexpr int kTileWords = 256;                  // 16 rows x 16 words (bf16 pairs), swizzled
constexpr int kNetFrags = 30;                    // fwd W1 (8), fwd W2 (8), bwd W2 (8), bwd W1 (6)
constexpr size_t kTcSmem = (size_t)kNetFrags * 32 * 8 + 4 * (2 * kMlpHid + kMlpHid + 4) +
                           (size_t)kTcWarps * (4 * kTileWords * 4 + 16 * 4) + (size_t)kTcWarps * kPart * 4;

__device__ __forceinline__ void ldsm_x4_trans(uint32_t r[4], const uint32_t* p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// the 16-byte chunk c of row r of a swizzled tile
__device__ __forceinline__ const uint32_t* tile_chunk(const uint32_t* tile, int r, int c)
{
    return tile + r * 16 + (((c ^ (r >> 1)) & 3) << 2);
}

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// backward B fragments: bf(W2) as B[i][k] (f = s*4 + j: i = 16s.., k = 8j + g),
// bf(W1) as B[i][c] over the row columns c (f = s*3 + j: c = 8j + g, zero past 18)
__device__ __forceinline__ uint2 bwd_frag(const float* __restrict__ p, int f, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    float e[4];
    if (f < 8) {
        const int s = f >> 2, j = f & 3, k = 8 * j + g;
        const int is[4] = {16 * s + 2 * t, 16 * s + 2 * t + 1, 16 * s + 2 * t + 8, 16 * s + 2 * t + 9};
#pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = p[kOffW2 + is[q] * kMlpHid + k];
    } else {
        const int ff = f - 8, s = ff / 3, j = ff % 3, c = w1_column(8 * j + g);
        const int is[4] = {16 * s + 2 * t, 16 * s + 2 * t + 1, 16 * s + 2 * t + 8, 16 * s + 2 * t + 9};
#pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = c >= 0 ? p[kOffW1 + is[q] * kMlpIn + c] : 0.0f;
    }
    return make_uint2(pack_bf16(e[0], e[1]), pack_bf16(e[2], e[3]));
}

// samples given explicitly: n rows of 19 inputs (u, v, w, z) and their targets;
// a tile is 16 consecutive samples
struct ExplicitSamples {
    static constexpr bool kLeaf = false;
    const float* X;
    const float* T;
    long long n;
    // lane (r = lane >> 1, h = lane & 1) writes half of row r of the tile (the
    // latent columns for h = 0, the position columns for h = 1); returns the
    // row's target to the h = 1 lane
    __device__ __forceinline__ float row(long long tile, int r, int h, uint32_t* xt) const
    {
        const long long q = tile * 16 + r;
        uint4* rp = reinterpret_cast<uint4*>(xt) + r * 4;
        const int sw = (r >> 1) & 3;
        const bool ok = q < n;
        const float* x = X + q * kMlpIn;
        if (h == 0) {
            uint32_t w[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) w[k] = ok ? pack_bf16(__ldg(x + 3 + 2 * k), __ldg(x + 4 + 2 * k)) : 0u;
            rp[0 ^ sw] = make_uint4(w[0], w[1], w[2], w[3]);
            rp[1 ^ sw] = make_uint4(w[4], w[5], w[6], w[7]);
            return 0.0f;
        }
        rp[2 ^ sw] = make_uint4(ok ? pack_bf16(__ldg(x), __ldg(x + 1)) : 0u, ok ? pack_bf16(__ldg(x + 2), 0.0f) : 0u, 0u, 0u);
        rp[3 ^ sw] = make_uint4(0u, 0u, 0u, 0u);
        return ok ? __ldg(T + q) : 0.0f;
    }
    struct Next {};            // (rows are read when their tile starts)
    // one thread's whole row q (the tensor-memory kernel): the 32 bf16 row
    // columns as 16 words, the target, and whether the row exists
    __device__ __forceinline__ float row1(long long q, uint32_t (&w)[16], bool& ok) const
    {
        ok = q < n;
        const float* x = X + q * kMlpIn;
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = ok ? pack_bf16(__ldg(x + 3 + 2 * k), __ldg(x + 4 + 2 * k)) : 0u;
        w[8] = ok ? pack_bf16(__ldg(x), __ldg(x + 1)) : 0u;
        w[9] = ok ? pack_bf16(__ldg(x + 2), 0.0f) : 0u;
#pragma unroll
        for (int k = 10; k < 16; ++k) w[k] = 0u;
        return ok ? __ldg(T + q) : 0.0f;
    }
};

// samples drawn from the leaves: sample s of training leaf a is voxel
// s*(512/S) + (r mod 512/S) of it; a warp's task is one leaf (S/16 tiles)
struct LeafSamples {
    static constexpr bool kLeaf = true;
    GridView src;
    const uint32_t* list;      // training leaves
    const uint32_t* pos;       // leaf -> linear position
    const float2* lmeta;       // leaf -> (scale, offset)
    const float* lat;          // leaf -> FP32 latent (16)
    int lg_s;                  // log2 S
    uint32_t step, k0, k1;
    __device__ __forceinline__ float row(uint32_t leaf, int s, int r, int h, uint32_t* xt) const
    {
        uint4* rp = reinterpret_cast<uint4*>(xt) + r * 4;
        const int sw = (r >> 1) & 3;
        if (h == 0) {
            const float4* L = reinterpret_cast<const float4*>(lat + (size_t)leaf * kMlpLatent);
            const float4 z0 = __ldg(L), z1 = __ldg(L + 1), z2 = __ldg(L + 2), z3 = __ldg(L + 3);
            rp[0 ^ sw] = make_uint4(pack_bf16(z0.x, z0.y), pack_bf16(z0.z, z0.w), pack_bf16(z1.x, z1.y), pack_bf16(z1.z, z1.w));
            rp[1 ^ sw] = make_uint4(pack_bf16(z2.x, z2.y), pack_bf16(z2.z, z2.w), pack_bf16(z3.x, z3.y), pack_bf16(z3.z, z3.w));
            return 0.0f;
        }
        const int stratum = kLeafN >> lg_s;
        const U4 rr = philox4x32_10(__ldg(pos + leaf), step, (uint32_t)s, kDrawTag, k0, k1);
        const int nv = s * stratum + (int)(rr.x & (uint32_t)(stratum - 1));
        const float2 sm = src.payload != 0 ? __ldg(src.meta + leaf) : make_float2(0.f, 0.f);
        const float v = leaf_value_t<-1>(src, leaf, nv, sm);
        const float2 lm = __ldg(lmeta + leaf);
        const float u = __fdiv_rn((float)(nv & 7), 7.0f), vv = __fdiv_rn((float)((nv >> 3) & 7), 7.0f),
                    w = __fdiv_rn((float)(nv >> 6), 7.0f);
        rp[2 ^ sw] = make_uint4(pack_bf16(u, vv), pack_bf16(w, 0.0f), 0u, 0u);
        rp[3 ^ sw] = make_uint4(0u, 0u, 0u, 0u);
        return lm.x != 0.0f ? __fdiv_rn(__fsub_rn(v, lm.y), lm.x) : 0.0f;
    }
    // one thread's next row for the tensor-memory kernel, the same draw and
    // values as row(), fetched in three stages so that each dependent load
    // (leaf index; leaf position, latent and metadata; the drawn voxel) is in
    // flight during one contraction round of the current tile
    struct Next {
        bool ok;
        int s, nv;
        uint32_t leaf, p, raw;
        uint32_t zw[8];
        float2 sm, lm;
    };
    __device__ __forceinline__ void fetch1(Next& f, long long q, long long n) const
    {
        f.ok = q < n;
        f.s = (int)(q & ((1 << lg_s) - 1));
        f.leaf = f.ok ? __ldg(list + (q >> lg_s)) : 0u;
    }
    __device__ __forceinline__ void fetch2(Next& f) const
    {
        if (!f.ok) return;
        f.p = __ldg(pos + f.leaf);
        // (the latent is in L2; its wait overlaps the round's MMA)
        const float4* L = reinterpret_cast<const float4*>(lat + (size_t)f.leaf * kMlpLatent);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 z = __ldg(L + k);
            f.zw[2 * k] = pack_bf16(z.x, z.y);
            f.zw[2 * k + 1] = pack_bf16(z.z, z.w);
        }
    }
    __device__ __forceinline__ void fetch3(Next& f) const
    {
        if (!f.ok) return;
        const int stratum = kLeafN >> lg_s;
        const U4 rr = philox4x32_10(f.p, step, (uint32_t)f.s, kDrawTag, k0, k1);
        f.nv = f.s * stratum + (int)(rr.x & (uint32_t)(stratum - 1));
        f.sm = src.payload != 0 ? __ldg(src.meta + f.leaf) : make_float2(0.f, 0.f);
        f.lm = __ldg(lmeta + f.leaf);
        const size_t o = (size_t)f.leaf * kLeafN + f.nv;
        if (src.payload == 0) f.raw = __ldg(reinterpret_cast<const uint32_t*>(src.leaves) + o);
        else if (src.payload == 1) f.raw = __ldg(reinterpret_cast<const unsigned short*>(src.leaves) + o);
        else f.raw = __ldg(reinterpret_cast<const unsigned char*>(src.leaves) + o);
    }
    // the fetched row as 16 words (latent, position, zeros) and its target
    // (a voxel decoded as leaf_value_t does)
    __device__ __forceinline__ float finish(const Next& f, uint32_t (&w)[16]) const
    {
#pragma unroll
        for (int k = 0; k < 16; ++k) w[k] = 0u;
        if (!f.ok) return 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = f.zw[k];
        const float v = src.payload == 0 ? __uint_as_float(f.raw)
                        : src.payload == 1 ? __fmaf_rn(f.sm.x, __half2float(__ushort_as_half((unsigned short)f.raw)), f.sm.y)
                                           : __fmaf_rn(f.sm.x, e4m3_to_float((uint8_t)f.raw), f.sm.y);
        const float u = __fdiv_rn((float)(f.nv & 7), 7.0f), vv = __fdiv_rn((float)((f.nv >> 3) & 7), 7.0f),
                    ww = __fdiv_rn((float)(f.nv >> 6), 7.0f);
        w[8] = pack_bf16(u, vv);
        w[9] = pack_bf16(ww, 0.0f);
        return f.lm.x != 0.0f ? __fdiv_rn(__fsub_rn(v, f.lm.y), f.lm.x) : 0.0f;
    }
};

// a warp's gradient accumulators (per lane)
struct TcAcc {
    float gw2[2][4][4];    // gW2 [m-tile of i][n-tile of k][frag]
    float gw1[2][3][4];    // gW1 [m-tile of i][n-tile of row column][frag]
    float gb1[4][2], gb2[4][2], gw3[4][2];   // columns 8j + 2t (+1), summed over this lane's rows
    float gb3;
    double loss;
};

// one tile through the network and back: xt holds the 16 input rows, tg the
// targets of the lane's rows g and g + 8, val their validity; adds to acc,
// returns the latent-column input gradients of rows g and g + 8 in dz
// (columns 8j + 2t (+1), j = 0, 1) and, when `full`, the position columns in dx3
template <bool kFull>
__device__ __forceinline__ void tc_tile(const uint32_t* xt, uint32_t* h1t, uint32_t* dh2t, uint32_t* dh1t,
                                        const uint2* fr, const float* b1s, const float* b2s, const float* w3s,
                                        float b3, float tg0, float tg1, bool val0, bool val1, float inv_n, TcAcc& A,
                                        float dz[2][4], float dx3[4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t a[2][4];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        a[s][0] = xt[tile_word(g, s * 8 + t)];
        a[s][1] = xt[tile_word(g + 8, s * 8 + t)];
        a[s][2] = xt[tile_word(g, s * 8 + 4 + t)];
        a[s][3] = xt[tile_word(g + 8, s * 8 + 4 + t)];
    }
    // layer 1
    float c[4][4];
    unsigned m1 = 0, m2 = 0;           // relu' masks, bit j*4 + q
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0f;
#pragma unroll
        for (int s = 0; s < 2; ++s) mma_bf16_16816(c[j], a[s], fr[(s * 4 + j) * 32 + lane]);
        const float bb0 = b1s[8 * j + 2 * t], bb1 = b1s[8 * j + 2 * t + 1];
        c[j][0] = __fadd_rn(c[j][0], bb0); c[j][1] = __fadd_rn(c[j][1], bb1);
        c[j][2] = __fadd_rn(c[j][2], bb0); c[j][3] = __fadd_rn(c[j][3], bb1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (c[j][q] > 0.0f) m1 |= 1u << (j * 4 + q); else c[j][q] = 0.0f;
        }
        h1t[tile_word(g, 4 * j + t)] = pack_bf16(c[j][0], c[j][1]);
        h1t[tile_word(g + 8, 4 * j + t)] = pack_bf16(c[j][2], c[j][3]);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        a[s][0] = pack_bf16(c[2 * s][0], c[2 * s][1]);
        a[s][1] = pack_bf16(c[2 * s][2], c[2 * s][3]);
        a[s][2] = pack_bf16(c[2 * s + 1][0], c[2 * s + 1][1]);
        a[s][3] = pack_bf16(c[2 * s + 1][2], c[2 * s + 1][3]);
    }
    // layer 2 and the output
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0f;
#pragma unroll
        for (int s = 0; s < 2; ++s) mma_bf16_16816(c[j], a[s], fr[(8 + s * 4 + j) * 32 + lane]);
        const float bb0 = b2s[8 * j + 2 * t], bb1 = b2s[8 * j + 2 * t + 1];
        c[j][0] = __fadd_rn(c[j][0], bb0); c[j][1] = __fadd_rn(c[j][1], bb1);
        c[j][2] = __fadd_rn(c[j][2], bb0); c[j][3] = __fadd_rn(c[j][3], bb1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (c[j][q] > 0.0f) { m2 |= 1u << (j * 4 + q); c[j][q] = bfr(c[j][q]); } else c[j][q] = 0.0f;
        }
        const float w0 = w3s[8 * j + 2 * t], w1 = w3s[8 * j + 2 * t + 1];
        y0 = fmaf(w0, c[j][0], y0); y0 = fmaf(w1, c[j][1], y0);
        y1 = fmaf(w0, c[j][2], y1); y1 = fmaf(w1, c[j][3], y1);
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1); y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1); y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    const float e0 = val0 ? __fadd_rn(y0, b3) - tg0 : 0.0f, e1 = val1 ? __fadd_rn(y1, b3) - tg1 : 0.0f;
    if (t == 0) A.loss += (double)e0 * e0 + (double)e1 * e1;
    const float dy0 = 2.0f * e0 * inv_n, dy1 = 2.0f * e1 * inv_n;
    if (t == 0) A.gb3 += dy0 + dy1;
    // dh2 = relu'(a2) dy bf(w3); gw3 += dy bf(h2); gb2 += dh2
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float w0 = w3s[8 * j + 2 * t], w1 = w3s[8 * j + 2 * t + 1];
        A.gw3[j][0] += dy0 * c[j][0] + dy1 * c[j][2];
        A.gw3[j][1] += dy0 * c[j][1] + dy1 * c[j][3];
        c[j][0] = (m2 >> (j * 4 + 0)) & 1u ? dy0 * w0 : 0.0f;
        c[j][1] = (m2 >> (j * 4 + 1)) & 1u ? dy0 * w1 : 0.0f;
        c[j][2] = (m2 >> (j * 4 + 2)) & 1u ? dy1 * w0 : 0.0f;
        c[j][3] = (m2 >> (j * 4 + 3)) & 1u ? dy1 * w1 : 0.0f;
        A.gb2[j][0] += c[j][0] + c[j][2];
        A.gb2[j][1] += c[j][1] + c[j][3];
        dh2t[tile_word(g, 4 * j + t)] = pack_bf16(c[j][0], c[j][1]);
        dh2t[tile_word(g + 8, 4 * j + t)] = pack_bf16(c[j][2], c[j][3]);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        a[s][0] = pack_bf16(c[2 * s][0], c[2 * s][1]);
        a[s][1] = pack_bf16(c[2 * s][2], c[2 * s][3]);
        a[s][2] = pack_bf16(c[2 * s + 1][0], c[2 * s + 1][1]);
        a[s][3] = pack_bf16(c[2 * s + 1][2], c[2 * s + 1][3]);
    }
    // dh1 = relu'(a1) (bf(W2)^T bf(dh2)); gb1 += dh1
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0f;
#pragma unroll
        for (int s = 0; s < 2; ++s) mma_bf16_16816(c[j], a[s], fr[(16 + s * 4 + j) * 32 + lane]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (!((m1 >> (j * 4 + q)) & 1u)) c[j][q] = 0.0f;
        A.gb1[j][0] += c[j][0] + c[j][2];
        A.gb1[j][1] += c[j][1] + c[j][3];
        dh1t[tile_word(g, 4 * j + t)] = pack_bf16(c[j][0], c[j][1]);
        dh1t[tile_word(g + 8, 4 * j + t)] = pack_bf16(c[j][2], c[j][3]);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        a[s][0] = pack_bf16(c[2 * s][0], c[2 * s][1]);
        a[s][1] = pack_bf16(c[2 * s][2], c[2 * s][3]);
        a[s][2] = pack_bf16(c[2 * s + 1][0], c[2 * s + 1][1]);
        a[s][3] = pack_bf16(c[2 * s + 1][2], c[2 * s + 1][3]);
    }
    // dx = bf(W1)^T bf(dh1): latent columns (n-tiles 0, 1), position columns (n-tile 2)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        dz[j][0] = dz[j][1] = dz[j][2] = dz[j][3] = 0.0f;
#pragma unroll
        for (int s = 0; s < 2; ++s) mma_bf16_16816(dz[j], a[s], fr[(24 + s * 3 + j) * 32 + lane]);
    }
    if constexpr (kFull) {
        dx3[0] = dx3[1] = dx3[2] = dx3[3] = 0.0f;
#pragma unroll
        for (int s = 0; s < 2; ++s) mma_bf16_16816(dx3, a[s], fr[(24 + s * 3 + 2) * 32 + lane]);
    }
    __syncwarp();
    // weight gradients over the tile's samples
    const int q = lane >> 3, r = lane & 7;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        uint32_t at2[4], at1[4];
        ldsm_x4_trans(at2, tile_chunk(dh2t, ((q >> 1) << 3) + r, 2 * mi + (q & 1)));
        ldsm_x4_trans(at1, tile_chunk(dh1t, ((q >> 1) << 3) + r, 2 * mi + (q & 1)));
#pragma unroll
        for (int nj = 0; nj < 4; nj += 2) {
            uint32_t bh[4], bx[4];
            ldsm_x4_trans(bh, tile_chunk(h1t, ((q & 1) << 3) + r, nj + (q >> 1)));
            ldsm_x4_trans(bx, tile_chunk(xt, ((q & 1) << 3) + r, nj + (q >> 1)));
            mma_bf16_16816(A.gw2[mi][nj], at2, make_uint2(bh[0], bh[1]));
            mma_bf16_16816(A.gw2[mi][nj + 1], at2, make_uint2(bh[2], bh[3]));
            mma_bf16_16816(A.gw1[mi][nj], at1, make_uint2(bx[0], bx[1]));
            if (nj + 1 < 3) mma_bf16_16816(A.gw1[mi][nj + 1], at1, make_uint2(bx[2], bx[3]));
        }
    }
    __syncwarp();
}

template <class Src>
__global__ void __launch_bounds__(kTcWarps * 32) k_mlp_grad(Src src, long long ntasks, float inv_n,
                                                            const float* __restrict__ params, float* __restrict__ part,
                                                            double* __restrict__ loss_part, float* __restrict__ gx)
{
    extern __shared__ float4 s_f4[];
    uint2* fr = reinterpret_cast<uint2*>(s_f4);                       // [30][32]
    float* b1s = reinterpret_cast<float*>(fr + kNetFrags * 32);
    float* b2s = b1s + kMlpHid;
    float* w3s = b2s + kMlpHid;                                       // bf16-rounded w3
    float* b3s = w3s + kMlpHid;                                       // [4]
    uint32_t* tiles = reinterpret_cast<uint32_t*>(b3s + 4);           // [warps][4 tiles]
    float* tgs = reinterpret_cast<float*>(tiles + kTcWarps * 4 * kTileWords);   // [warps][16]
    float* red = tgs + kTcWarps * 16;                                 // [warps][kPart]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < kNetFrags * 32; i += blockDim.x) {
        const int f = i >> 5, l = i & 31;
        fr[i] = f < 16 ? mlp_frag(params, f, l) : bwd_frag(params, f - 16, l);
    }
    for (int i = tid; i < kMlpHid; i += blockDim.x) {
        b1s[i] = params[kOffB1 + i];
        b2s[i] = params[kOffB2 + i];
        w3s[i] = bfr(params[kOffW3 + i]);
    }
    if (tid == 0) b3s[0] = params[kOffB3];
    __syncthreads();
    const float b3 = b3s[0];
    uint32_t* xt = tiles + wid * 4 * kTileWords;
    uint32_t* h1t = xt + kTileWords;
    uint32_t* dh2t = h1t + kTileWords;
    uint32_t* dh1t = dh2t + kTileWords;
    float* tg = tgs + wid * 16;
    TcAcc A;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj)
#pragma unroll
            for (int k = 0; k < 4; ++k) { A.gw2[mi][nj][k] = 0.0f; if (nj < 3) A.gw1[mi][nj][k] = 0.0f; }
#pragma unroll
    for (int j = 0; j < 4; ++j) { A.gb1[j][0] = A.gb1[j][1] = A.gb2[j][0] = A.gb2[j][1] = A.gw3[j][0] = A.gw3[j][1] = 0.0f; }
    A.gb3 = 0.0f;
    A.loss = 0.0;
    const int g = lane >> 2, t = lane & 3, rr = lane >> 1, hh = lane & 1;
    const long long gw = (long long)blockIdx.x * kTcWarps + wid, nw = (long long)gridDim.x * kTcWarps;
    for (long long task = gw; task < ntasks; task += nw) {
        if constexpr (Src::kLeaf) {
            // a leaf: S / 16 tiles; its latent gradient sums over all of them
            const uint32_t leaf = __ldg(src.list + task);
            const int S = 1 << src.lg_s;
            float zs[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
            for (int s0 = 0; s0 < S; s0 += 16) {
                const float trow = src.row(leaf, s0 + rr, rr, hh, xt);
                if (hh) tg[rr] = trow;
                __syncwarp();
                float dz[2][4], dx3[4];
                tc_tile<false>(xt, h1t, dh2t, dh1t, fr, b1s, b2s, w3s, b3, tg[g], tg[g + 8], true, true, inv_n, A,
                               dz, dx3);
#pragma unroll
                for (int j = 0; j < 2; ++j) { zs[j][0] += dz[j][0] + dz[j][2]; zs[j][1] += dz[j][1] + dz[j][3]; }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) zs[j][k] += __shfl_xor_sync(0xffffffffu, zs[j][k], o);
            if (g == 0) {
                float* out = gx + (size_t)leaf * kMlpLatent;
                out[2 * t] = zs[0][0]; out[2 * t + 1] = zs[0][1];
                out[8 + 2 * t] = zs[1][0]; out[8 + 2 * t + 1] = zs[1][1];
            }
        } else {
            const float trow = src.row(task, rr, hh, xt);
            if (hh) tg[rr] = trow;
            __syncwarp();
            const long long q0 = task * 16 + g, q1 = q0 + 8;
            float dz[2][4], dx3[4];
            tc_tile<true>(xt, h1t, dh2t, dh1t, fr, b1s, b2s, w3s, b3, tg[g], tg[g + 8], q0 < src.n, q1 < src.n, inv_n, A,
                          dz, dx3);
            if (gx) {
                // row column c = 8j + 2t (+1): latent z_c (j < 2) or position c - 16 (j = 2)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float* v = j < 2 ? dz[j] : dx3;
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int col = w1_column(8 * j + 2 * t + k);
                        if (col < 0) continue;
                        if (q0 < src.n) gx[q0 * kMlpIn + col] = v[k];
                        if (q1 < src.n) gx[q1 * kMlpIn + col] = v[2 + k];
                    }
                }
            }
        }
    }
    // the warp's gradient to shared memory in parameter order, then the warps in order
    float* R = red + wid * kPart;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj) {
            const int i0 = 16 * mi + g, k0 = 8 * nj + 2 * t;
            R[kOffW2 + i0 * kMlpHid + k0] = A.gw2[mi][nj][0];
            R[kOffW2 + i0 * kMlpHid + k0 + 1] = A.gw2[mi][nj][1];
            R[kOffW2 + (i0 + 8) * kMlpHid + k0] = A.gw2[mi][nj][2];
            R[kOffW2 + (i0 + 8) * kMlpHid + k0 + 1] = A.gw2[mi][nj][3];
            if (nj < 3) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int col = w1_column(8 * nj + 2 * t + k);
                    if (col < 0) continue;
                    R[kOffW1 + i0 * kMlpIn + col] = A.gw1[mi][nj][k];
                    R[kOffW1 + (i0 + 8) * kMlpIn + col] = A.gw1[mi][nj][2 + k];
                }
            }
        }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float v1 = A.gb1[j][k], v2 = A.gb2[j][k], v3 = A.gw3[j][k];
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                v2 += __shfl_xor_sync(0xffffffffu, v2, o);
                v3 += __shfl_xor_sync(0xffffffffu, v3, o);
            }
            if (g == 0) {
                R[kOffB1 + 8 * j + 2 * t + k] = v1;
                R[kOffB2 + 8 * j + 2 * t + k] = v2;
                R[kOffW3 + 8 * j + 2 * t + k] = v3;
            }
        }
    float gb3 = A.gb3;
    double ls = A.loss;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
        ls += __shfl_xor_sync(0xffffffffu, ls, o);
    }
    if (lane == 0) R[kOffB3] = gb3;
    __shared__ double s_loss[kTcWarps];
    if (lane == 0) s_loss[wid] = ls;
    __syncthreads();
    float* P = part + (size_t)blockIdx.x * kPart;
    for (int e = tid; e < kMlpParams; e += blockDim.x) {
        float v = red[e];
#pragma unroll
        for (int w = 1; w < kTcWarps; ++w) v += red[w * kPart + e];
        P[e] = v;
    }
    if (tid == 0) {
        double l = 0.0;
        for (int w = 0; w < kTcWarps; ++w) l += s_loss[w];
        loss_part[blockIdx.x] = l;
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

// ---------------------------------------------------------------- training on tcgen05
// The gradient of k_mlp_grad (same bf16 roundings of the operands, FP32
// sums, FP32 bias and w3 gradients) on the fifth-generation tensor cores.  A
// CTA of 128 threads takes tiles of 128 samples, one row a thread; every
// contraction is one M = 128, N = 32 MMA (K = 32 as two K = 16 steps) issued
// by one thread into tensor memory, and read back a row a thread:
//   a1 = X W1^T, a2 = H W2^T (H = bf(relu(a1 + b1))), dh1 = (bf(dh2) W2)
//   masked, dx = bf(dh1) W1, and the weight gradients
//   [gW2; gW1] += G^T [H | X] over the tile's 128 samples, where G holds
//   bf(dh2) in columns 0-31 and bf(dh1) in 32-63: M = 128 rows of G's
//   columns, K = the 128 samples, accumulated in tensor memory over all of
//   the CTA's tiles.
// Accumulator lanes 64-127 of the weight gradients are never read, so G's
// columns 64-127 are free: each warp sums its 32 rows of the bias and w3
// gradient terms (and of the latent gradients) per column through them, in
// a fixed order, so a thread keeps three running sums instead of 96.  The
// next tile's samples are fetched in three dependent stages, one per
// contraction round, so their gathers overlap the current tile's MMAs.  With
// 56 KB of shared memory, 128 tensor-memory columns and at most 128
// registers a thread, four CTAs share an SM.
// The same shared-memory tile is the K-major A of one MMA and the MN-major
// A or B of another: core matrices are 8 rows by 8 bf16 along the row.
constexpr int kT5Rows = 128;
constexpr uint32_t kT5SrX = 384;       // row-block stride of X: column blocks 0-2 (row columns 0-23)
constexpr uint32_t kT5Sr = 512;        // row-block stride of a 32-column tile (4 column blocks)
constexpr uint32_t kT5SrG = 2048;      // row-block stride of the 128-column tile G
constexpr uint32_t kT5Sc = 128;        // column-block stride
constexpr uint32_t kT5Cols = 128;      // tensor-memory columns: scratch 0-31, gW2 32-63, gW1 64-95
// X's fourth column block (row columns 24-31) is not stored: the MMAs read
// the next row block's first block (or H's, after the last row block) in its
// place, finite values that meet zero weights in a1 and land in gW1 columns
// that are never read
constexpr size_t kT5OffX = 0, kT5OffH = 6144, kT5OffG = 14336, kT5OffW = 47104, kT5OffP = 55296,
                 kT5OffZ = kT5OffP + 3 * kMlpHid * 4, kT5OffL = kT5OffZ + 4 * kMlpLatent * 4,
                 kT5OffBar = kT5OffL + 4 * 8, kT5Smem = kT5OffBar + 16;
static_assert(kT5OffH == 16 * kT5SrX && kT5OffG == kT5OffH + 16 * kT5Sr && kT5OffW == kT5OffG + 16 * kT5SrG,
              "tile layout");
static_assert(kT5Smem <= 56 * 1024, "four CTAs an SM");
constexpr int kT5WaitPolls = 1 << 26;

__device__ __forceinline__ void t5_store_floats(uint8_t* tile, uint32_t sr, int r, int col0, const float* v)
{
#pragma unroll
    for (int k = 0; k < 4; ++k)
        *reinterpret_cast<uint4*>(tile + tc::tile_off(r, col0 + 8 * k, sr, kT5Sc)) =
            make_uint4(pack_bf16(v[8 * k], v[8 * k + 1]), pack_bf16(v[8 * k + 2], v[8 * k + 3]),
                       pack_bf16(v[8 * k + 4], v[8 * k + 5]), pack_bf16(v[8 * k + 6], v[8 * k + 7]));
}

// the warp's 4 KB of staging in G's columns 64-127 (one 1 KB piece in each of
// its four row blocks), column-major: value (row r of the warp, column c) at
// piece c >> 3, byte (c & 7) * 128 + 4 r.  A row's stores have fixed offsets
// and consecutive lanes hit consecutive banks; a column is 128 contiguous
// bytes, read as eight 16-byte groups, lane c starting at group c & 7 so that
// the eight lanes of a quarter-warp read eight different bank groups.
__device__ __forceinline__ uint8_t* t5_stage(uint8_t* G, int warp) { return G + (uint32_t)warp * 4u * kT5SrG + 1024u; }

template <int kCols>
__device__ __forceinline__ void t5_stage_store(uint8_t* G, int warp, int lane, const float (&v)[32])
{
    float* p = reinterpret_cast<float*>(t5_stage(G, warp)) + lane;
#pragma unroll
    for (int c = 0; c < kCols; ++c) p[(c >> 3) * (kT5SrG / 4) + (c & 7) * 32] = v[c];
}

// the warp's 32 rows of v summed per column: lane c returns column c (a
// fixed order of rows for each lane)
__device__ __forceinline__ float t5_colsum(uint8_t* G, int tid, const float (&v)[32])
{
    const int lane = tid & 31, warp = tid >> 5;
    t5_stage_store<32>(G, warp, lane, v);
    __syncwarp();
    const uint8_t* col = t5_stage(G, warp) + (lane >> 3) * kT5SrG + (lane & 7) * 128;
    float s[2] = {0.0f, 0.0f};
#pragma unroll 4
    for (int g = 0; g < 8; ++g) {
        const float4 q = *reinterpret_cast<const float4*>(col + (((g + lane) & 7) << 4));
        s[g & 1] += (q.x + q.y) + (q.z + q.w);
    }
    __syncwarp();
    return s[0] + s[1];
}

// latent columns 0-15 of the warp's rows: lane c + 16 h returns column c
// summed over rows 16 h .. 16 h + 15
__device__ __forceinline__ float t5_latsum(uint8_t* G, int tid, const float (&v)[32])
{
    const int lane = tid & 31, warp = tid >> 5, c = lane & 15, h = lane >> 4;
    t5_stage_store<kMlpLatent>(G, warp, lane, v);
    __syncwarp();
    const uint8_t* col = t5_stage(G, warp) + (c >> 3) * kT5SrG + (c & 7) * 128 + h * 64;
    float s = 0.0f;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const float4 q = *reinterpret_cast<const float4*>(col + (((g + c) & 3) << 4));
        s += (q.x + q.y) + (q.z + q.w);
    }
    __syncwarp();
    return s;
}

template <class Src>
__global__ void __launch_bounds__(kT5Rows, 4) k_mlp_grad_tc(Src src, long long nsamples, int lg_s, float inv_n,
                                                            const float* __restrict__ params, float* __restrict__ part,
                                                            double* __restrict__ loss_part, float* __restrict__ gx)
{
    extern __shared__ __align__(1024) uint8_t s5[];
    uint8_t* X = s5 + kT5OffX;
    uint8_t* H = s5 + kT5OffH;
    uint8_t* G = s5 + kT5OffG;
    uint8_t* W1B = s5 + kT5OffW;              // [n = i][k = row column c]: W1[i][w1_column(c)]
    uint8_t* W2B = W1B + 2048;                // [n = j][k = i]: W2[j][i]
    uint8_t* W2T = W2B + 2048;                // [n = i][k = j]: W2[j][i]
    uint8_t* W1T = W2T + 2048;                // [n = c][k = i]: W1[i][w1_column(c)]
    float* b1s = reinterpret_cast<float*>(s5 + kT5OffP);
    float* b2s = b1s + kMlpHid;
    float* w3s = b2s + kMlpHid;
    float* zpart = reinterpret_cast<float*>(s5 + kT5OffZ);   // [warp][16] latent column sums
    double* lsum = reinterpret_cast<double*>(s5 + kT5OffL);
    uint64_t* bar = reinterpret_cast<uint64_t*>(s5 + kT5OffBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(s5 + kT5OffBar + 8);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // the network's bf16 operand tiles, FP32 biases, bf(w3)
    for (int e = tid; e < 32 * 32; e += kT5Rows) {
        const int n = e >> 5, k = e & 31, c1 = w1_column(k), c2 = w1_column(n);
        const uint32_t o = tc::tile_off(n, k, kT5Sr, kT5Sc);
        *reinterpret_cast<__nv_bfloat16*>(W1B + o) = __float2bfloat16_rn(c1 >= 0 ? params[kOffW1 + n * kMlpIn + c1] : 0.0f);
        *reinterpret_cast<__nv_bfloat16*>(W2B + o) = __float2bfloat16_rn(params[kOffW2 + n * kMlpHid + k]);
        *reinterpret_cast<__nv_bfloat16*>(W2T + o) = __float2bfloat16_rn(params[kOffW2 + k * kMlpHid + n]);
        *reinterpret_cast<__nv_bfloat16*>(W1T + o) = __float2bfloat16_rn(c2 >= 0 ? params[kOffW1 + k * kMlpIn + c2] : 0.0f);
    }
    // H is read in place of X's missing column block before the first H is written
    for (int e = tid; e < (int)(16 * kT5Sr / 16); e += kT5Rows) reinterpret_cast<uint4*>(H)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid < kMlpHid) {
        b1s[tid] = params[kOffB1 + tid];
        b2s[tid] = params[kOffB2 + tid];
        w3s[tid] = bfr(params[kOffW3 + tid]);
    }
    if (tid == 0) tc::mbar_init(bar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, kT5Cols);
    tc::fence_smem_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
    const float b3 = params[kOffB3];
    constexpr uint32_t kIdK = tc::idesc_bf16(128, 32, 0, 0), kIdMN = tc::idesc_bf16(128, 32, 1, 1);
    const uint32_t aX = tc::smem_u32(X), aH = tc::smem_u32(H), aG = tc::smem_u32(G);
    const uint32_t aW1B = tc::smem_u32(W1B), aW2B = tc::smem_u32(W2B), aW2T = tc::smem_u32(W2T), aW1T = tc::smem_u32(W1T);

    // thread (warp w, lane c): column c of the bias and w3 gradients over warp w's rows
    float sb1 = 0.0f, sb2 = 0.0f, sw3 = 0.0f, gb3 = 0.0f;
    double loss = 0.0;
    uint32_t phase = 0;
    bool first = true, stalled = false;
    const int S = Src::kLeaf ? (1 << lg_s) : kT5Rows;     // 16 .. 128: whole leaves per tile
    const long long ntasks = (nsamples + kT5Rows - 1) / kT5Rows;
    long long pend = -1;       // a tile whose leaves span warps: latents combined after the next barrier
    // the pre-issue barrier of a round: the tile's shared-memory operands
    // visible to the tensor core, the tensor-memory reads of the last round
    // done, and a wait that ran out anywhere seen by every thread
    auto round_barrier = [&]() {
        tc::fence_smem_async();
        tc::fence_before_sync();
        stalled = __syncthreads_or(stalled) != 0;
    };
    // the round's MMAs complete; the warp reads its 32 lanes of scratch
    auto round_wait = [&](float (&a)[32]) {
        bool ok = tc::mbar_wait(bar, phase, kT5WaitPolls);
        phase ^= 1u;
        ok = __all_sync(0xffffffffu, ok);
        tc::fence_after_sync();
        if (ok) {
            tc::tmem_ld32(tlane, a);
        } else {
            stalled = true;
#pragma unroll
            for (int i = 0; i < 32; ++i) a[i] = 0.0f;
        }
    };
    // latent gradients of the pending tile's leaves (S = 64, 128): warp k sums leaf slot k's warps in order
    auto flush_pending = [&]() {
        if (pend < 0) return;
        const int per = S >> 5;
        if (warp < kT5Rows / S && lane < kMlpLatent) {
            float z = 0.0f;
            for (int w2 = warp * per; w2 < warp * per + per; ++w2) z += zpart[w2 * kMlpLatent + lane];
            const long long q0 = pend * kT5Rows + (long long)warp * S;
            if constexpr (Src::kLeaf)
                if (q0 < nsamples) gx[(size_t)__ldg(src.list + (q0 >> lg_s)) * kMlpLatent + lane] = z;
        }
        pend = -1;
    };

    typename Src::Next nx;
    if constexpr (Src::kLeaf) {
        src.fetch1(nx, (long long)blockIdx.x * kT5Rows + tid, nsamples);
        src.fetch2(nx);
        src.fetch3(nx);
    }
    for (long long task = blockIdx.x; task < ntasks; task += gridDim.x) {
        const long long q = task * kT5Rows + tid;
        const long long qn = q + (long long)gridDim.x * kT5Rows;
        uint32_t w[16];
        bool valid;
        float tgt;
        if constexpr (Src::kLeaf) {
            valid = nx.ok;
            tgt = src.finish(nx, w);
        } else {
            tgt = src.row1(q, w, valid);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
            *reinterpret_cast<uint4*>(X + tc::tile_off(tid, 8 * k, kT5SrX, kT5Sc)) =
                make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
        round_barrier();
        if (stalled) break;
        flush_pending();
        if (tid == 0) {
            tc::fence_after_sync();
            for (int k = 0; k < 2; ++k)
                tc::mma_bf16(tbase, tc::smem_desc(aX + 256 * k, kT5Sc, kT5SrX), tc::smem_desc(aW1B + 256 * k, kT5Sc, kT5Sr),
                             kIdK, k > 0);
            tc::mma_commit(bar);
        }
        if constexpr (Src::kLeaf) src.fetch1(nx, qn, nsamples);
        float a[kMlpHid];
        round_wait(a);
        uint32_t m1 = 0u, m2 = 0u;
#pragma unroll
        for (int i = 0; i < kMlpHid; ++i) {
            const float v = __fadd_rn(a[i], b1s[i]);
            if (v > 0.0f) { m1 |= 1u << i; a[i] = v; } else a[i] = 0.0f;
        }
        t5_store_floats(H, kT5Sr, tid, 0, a);
        round_barrier();
        if (stalled) break;
        if (tid == 0) {
            tc::fence_after_sync();
            for (int k = 0; k < 2; ++k)
                tc::mma_bf16(tbase, tc::smem_desc(aH + 256 * k, kT5Sc, kT5Sr), tc::smem_desc(aW2B + 256 * k, kT5Sc, kT5Sr),
                             kIdK, k > 0);
            tc::mma_commit(bar);
        }
        if constexpr (Src::kLeaf) src.fetch2(nx);
        round_wait(a);
        float y = 0.0f;
#pragma unroll
        for (int j = 0; j < kMlpHid; ++j) {
            const float v = __fadd_rn(a[j], b2s[j]);
            if (v > 0.0f) { m2 |= 1u << j; a[j] = bfr(v); } else a[j] = 0.0f;
            y = fmaf(w3s[j], a[j], y);
        }
        const float e = valid ? __fadd_rn(y, b3) - tgt : 0.0f;
        loss += (double)e * e;
        const float dy = 2.0f * e * inv_n;
        gb3 += dy;
#pragma unroll
        for (int j = 0; j < kMlpHid; ++j) a[j] = dy * a[j];
        sw3 += t5_colsum(G, tid, a);
#pragma unroll
        for (int j = 0; j < kMlpHid; ++j) a[j] = (m2 >> j) & 1u ? dy * w3s[j] : 0.0f;
        sb2 += t5_colsum(G, tid, a);
        t5_store_floats(G, kT5SrG, tid, 0, a);
        round_barrier();
        if (stalled) break;
        if (tid == 0) {
            tc::fence_after_sync();
            for (int k = 0; k < 2; ++k)
                tc::mma_bf16(tbase, tc::smem_desc(aG + 256 * k, kT5Sc, kT5SrG), tc::smem_desc(aW2T + 256 * k, kT5Sc, kT5Sr),
                             kIdK, k > 0);
            tc::mma_commit(bar);
        }
        if constexpr (Src::kLeaf) src.fetch3(nx);
        round_wait(a);
#pragma unroll
        for (int i = 0; i < kMlpHid; ++i)
            if (!((m1 >> i) & 1u)) a[i] = 0.0f;
        sb1 += t5_colsum(G, tid, a);
        t5_store_floats(G, kT5SrG, tid, 32, a);
        round_barrier();
        if (stalled) break;
        if (tid == 0) {
            tc::fence_after_sync();
            for (int k = 0; k < 2; ++k)
                tc::mma_bf16(tbase, tc::smem_desc(aG + 4 * kT5Sc + 256 * k, kT5Sc, kT5SrG),
                             tc::smem_desc(aW1T + 256 * k, kT5Sc, kT5Sr), kIdK, k > 0);
            // weight gradients: K = the 128 samples, 16 (two row blocks) a step
            for (int k = 0; k < 8; ++k) {
                const uint64_t ga = tc::smem_desc(aG + 2 * kT5SrG * k, kT5SrG, kT5Sc);
                tc::mma_bf16(tbase + 32, ga, tc::smem_desc(aH + 2 * kT5Sr * k, kT5Sr, kT5Sc), kIdMN, !(first && k == 0));
                tc::mma_bf16(tbase + 64, ga, tc::smem_desc(aX + 2 * kT5SrX * k, kT5SrX, kT5Sc), kIdMN, !(first && k == 0));
            }
            tc::mma_commit(bar);
        }
        first = false;
        round_wait(a);                          // dx: row columns 0-15 latent, 16-18 position
        if constexpr (Src::kLeaf) {
            float z = t5_latsum(G, tid, a);     // lane c + 16 h: column c over rows 16 h .. 16 h + 15
            if (S == 16) {
                const long long q0 = task * kT5Rows + warp * 32 + (lane >> 4) * 16;
                if (q0 < nsamples) gx[(size_t)__ldg(src.list + (q0 >> lg_s)) * kMlpLatent + (lane & 15)] = z;
            } else {
                z += __shfl_xor_sync(0xffffffffu, z, 16);
                if (S == 32) {
                    const long long q0 = task * kT5Rows + warp * 32;
                    if (lane < kMlpLatent && q0 < nsamples) gx[(size_t)__ldg(src.list + (q0 >> lg_s)) * kMlpLatent + lane] = z;
                } else {
                    if (lane < kMlpLatent) zpart[warp * kMlpLatent + lane] = z;
                    pend = task;
                }
            }
        } else {
            if (gx && valid) {
#pragma unroll
                for (int c = 0; c < kMlpIn; ++c) gx[q * kMlpIn + w1_column(c)] = a[c];
            }
        }
    }
    tc::fence_before_sync();
    stalled = __syncthreads_or(stalled) != 0;
    if (!stalled) flush_pending();
    // the CTA's partial gradient in parameter order: weight gradients from
    // tensor memory (warp 0: gW2 rows, warp 1: gW1 rows), the rest reduced
    // over the warps in a fixed order through G (no MMA reads it any more)
    float* P = part + (size_t)blockIdx.x * kPart;
    tc::fence_after_sync();
    if (warp < 2) {
        float v[32];
        if (!first && !stalled) tc::tmem_ld32(tlane + 32 + 32 * warp, v);
        else {
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] = 0.0f;
        }
        if (warp == 0) {
#pragma unroll
            for (int i = 0; i < kMlpHid; ++i) P[kOffW2 + lane * kMlpHid + i] = v[i];
        } else {
#pragma unroll
            for (int c = 0; c < kMlpIn; ++c) P[kOffW1 + lane * kMlpIn + w1_column(c)] = v[c];
        }
    }
    float* red = reinterpret_cast<float*>(G);     // [warp][100]
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
        loss += __shfl_xor_sync(0xffffffffu, loss, o);
    }
    red[warp * 100 + lane] = sb1;
    red[warp * 100 + 32 + lane] = sb2;
    red[warp * 100 + 64 + lane] = sw3;
    if (lane == 0) { red[warp * 100 + 96] = gb3; lsum[warp] = loss; }
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 97) {
        float v = red[tid];
        for (int w2 = 1; w2 < 4; ++w2) v += red[w2 * 100 + tid];
        const int dst = tid < 32 ? kOffB1 + tid : tid < 64 ? kOffB2 + tid - 32 : tid < 96 ? kOffW3 + tid - 64 : kOffB3;
        P[dst] = v;
    }
    if (tid == 0) {
        const double l = lsum[0] + lsum[1] + lsum[2] + lsum[3];
        loss_part[blockIdx.x] = stalled ? (double)NAN : l;
    }
    if (stalled) tc::mbar_wait(bar, phase ^ 1u, kT5WaitPolls);    // (a stalled MMA: wait once more before freeing)
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, kT5Cols);
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

// the training kernel: the tcgen05 one, or the mma.sync one with VDBC_MLP_TC=0
// (200 steps over the 994 x 676 x 1225 cloud's 455,433 leaves at 64 samples:
// 0.79 s with mma.sync)
bool mlp_tc()
{
    static const bool on = [] { const char* e = std::getenv("VDBC_MLP_TC"); return !(e && e[0] == '0'); }();
    return on;
}

// gradient of the loss over n samples (ntasks warp tasks of the mma.sync
// kernel) into grad, and the loss if asked; part / loss_part hold the
// grid's partials
template <class Src>
vdbc_status run_grad(const Src& src, long long ntasks, long long n, const float* params, float* part,
                     double* loss_part, int grid, float* grad, double* loss, float* gx, cudaStream_t s)
{
    if (mlp_tc()) {
        int lg_s = 0;
        if constexpr (Src::kLeaf) lg_s = src.lg_s;
        auto k5 = k_mlp_grad_tc<Src>;
        VDBC_CUDA(cudaFuncSetAttribute(k5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kT5Smem));
        VDBC_CUDA(cudaFuncSetAttribute(k5, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        KLAUNCH(k5<<<grid, kT5Rows, kT5Smem, s>>>(src, n, lg_s, (float)(1.0 / (double)n), params, part, loss_part, gx));
    } else {
        auto kern = k_mlp_grad<Src>;
        VDBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
        KLAUNCH(kern<<<grid, kTcWarps * 32, kTcSmem, s>>>(src, ntasks, (float)(1.0 / (double)n), params, part,
                                                          loss_part, gx));
    }
    KLAUNCH(k_sum_parts<<<blocks(kMlpParams, 256), 256, 0, s>>>(part, grid, grad, loss_part, 1.0 / (double)n, loss));
    VDBC_CUDA(cudaGetLastError());
    return VDBC_OK;
}

// blocks of the training kernel for ntasks warp tasks (mma.sync) or n
// samples (tcgen05: 128-sample tiles): at most one wave
int grad_grid(long long ntasks, long long n)
{
    static int per_sm = -1;
    if (mlp_tc()) {
        // four CTAs an SM by construction: 128 registers a thread (launch
        // bounds), at most 56 KB of shared memory, 128 of the SM's 512
        // tensor-memory columns.  (The occupancy query answers 1 for this
        // kernel; sized by it, the grid left three quarters of every SM idle:
        // 200 steps on the cloud took 1.73 s, against 0.59 s at four.)
        constexpr int per_sm5 = 512 / (int)kT5Cols;
        const long long need = (n + kT5Rows - 1) / kT5Rows;
        return (int)std::max<long long>(1, std::min<long long>(need, (long long)sm_count_dev() * per_sm5));
    }
    if (per_sm < 0) {
        auto kern = k_mlp_grad<LeafSamples>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTcWarps * 32, kTcSmem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    long long need = (ntasks + kTcWarps - 1) / kTcWarps;
    return (int)std::max<long long>(1, std::min<long long>(need, (long long)sm_count_dev() * per_sm));
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
#if VDBC_CHECKED
    m->view.n_leaves = (uint32_t)(n_raw + n_neu);
    m->view.n_neural = 0;
#endif
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
    for (const vdbc_learn_state* st : {static_cast<const vdbc_learn_state*>(p->resume),
                                       static_cast<const vdbc_learn_state*>(p->save)}) {
        if (!st) continue;
        if (!st->params || !st->params_m || !st->params_v || !st->latents || !st->latents_m || !st->latents_v)
            return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: a training state with a null array");
    }
    if (p->resume) {
        if (p->init_params || p->init_latents)
            return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: resume excludes init_params and init_latents");
        if (p->resume->step < 0 || p->resume->step > (int64_t)INT32_MAX - p->steps)
            return set_error(VDBC_ERR_INVALID_ARG, "vdbc_learn: resume step %lld outside 0..2^31-1-steps",
                             (long long)p->resume->step);
    }
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
        KLAUNCH(k_gather_leaf<<<blocks(nl, 256), 256, 0, s>>>(pos, nl, lp->force,
                                                              lp->resume ? lp->resume->latents : lp->init_latents,
                                                              force, lat, trains));
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
    const vdbc_learn_state* rs = lp->resume;
    if (rs) {
        VDBC_CUDA(cudaMemcpyAsync(params, rs->params, kMlpParams * 4, cudaMemcpyDefault, s));
        VDBC_CUDA(cudaMemcpyAsync(pm, rs->params_m, kMlpParams * 4, cudaMemcpyDefault, s));
        VDBC_CUDA(cudaMemcpyAsync(pv, rs->params_v, kMlpParams * 4, cudaMemcpyDefault, s));
        if (nl > 0) {
            KLAUNCH(k_gather_rows<<<blocks(nl * kMlpLatent, 256), 256, 0, s>>>(pos, nl, rs->latents_m, lat_m));
            KLAUNCH(k_gather_rows<<<blocks(nl * kMlpLatent, 256), 256, 0, s>>>(pos, nl, rs->latents_v, lat_v));
        }
    } else if (lp->init_params) {
        VDBC_CUDA(cudaMemcpyAsync(params, lp->init_params, kMlpParams * 4, cudaMemcpyDefault, s));
    } else {
        KLAUNCH(k_init_params<<<blocks(kMlpParams, 256), 256, 0, s>>>(params, k0, k1));
    }
    const long long t0 = rs ? rs->step : 0;     // Adam steps already taken
    const long long nsamp = (long long)n_train << lg_s;
    if (lp->steps > 0 && nsamp > 0) {
        const int grid = grad_grid((long long)n_train, nsamp);
        VDBC_TRY(pool.get(&part, (size_t)grid * kPart));
        VDBC_TRY(pool.get(&loss_part, grid));
        VDBC_TRY(pool.get(&loss_hist, lp->steps));
        LeafSamples ls{src->view, list, pos, lmeta, lat, lg_s, 0u, k0, k1};
        for (int t = 0; t < lp->steps; ++t) {
            const long long tg = t0 + t;
            ls.step = (uint32_t)tg;
            VDBC_TRY(run_grad(ls, (long long)n_train, nsamp, params, part, loss_part, grid, grad, loss_hist + t, glat, s));
            const float c1 = (float)(1.0 - std::pow((double)kBeta1, (double)(tg + 1)));
            const float c2 = (float)(1.0 - std::pow((double)kBeta2, (double)(tg + 1)));
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
    if (vdbc_learn_state* sv = lp->save) {
        const size_t npos = (size_t)nlx * nly * ((si.dims[2] + 7) / 8) * kMlpLatent;
        VDBC_CUDA(cudaMemcpyAsync(sv->params, params, kMlpParams * 4, cudaMemcpyDefault, s));
        VDBC_CUDA(cudaMemcpyAsync(sv->params_m, pm, kMlpParams * 4, cudaMemcpyDefault, s));
        VDBC_CUDA(cudaMemcpyAsync(sv->params_v, pv, kMlpParams * 4, cudaMemcpyDefault, s));
        float* rows[3][2] = {{lat, sv->latents}, {lat_m, sv->latents_m}, {lat_v, sv->latents_v}};
        for (auto& r : rows) {
            VDBC_CUDA(cudaMemsetAsync(r[1], 0, npos * 4, s));
            if (nl > 0) KLAUNCH(k_scatter_rows<<<blocks(nl * kMlpLatent, 256), 256, 0, s>>>(pos, nl, r[0], r[1]));
        }
        sv->step = t0 + lp->steps;
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
    st = dev_alloc(reinterpret_cast<void**>(&g->stats), sizeof(DevStats), s);
    if (st != VDBC_OK) { vdbc_grid_free(g); return st; }
    bind_view(g);
    char* b = static_cast<char*>(g->block);
    const char* sb = static_cast<const char*>(src->block);
    cudaError_t e = cudaMemsetAsync(g->block, 0, g->block_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s);
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
    if (st == VDBC_OK) st = checked_flags(g, s);
    if (st == VDBC_OK) st = wait_stream(s);
    if (st != VDBC_OK) return release_or_defer(st, s, [g] { vdbc_grid_free(g); });
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
    const long long ntiles = (n + 15) / 16;
    const int grid = grad_grid(ntiles, (long long)n);
    float* part = nullptr;
    double *loss_part = nullptr, *dloss = nullptr;
    VDBC_TRY(pool.get(&part, (size_t)grid * kPart));
    VDBC_TRY(pool.get(&loss_part, grid));
    VDBC_TRY(pool.get(&dloss, 1));
    ExplicitSamples es{inputs, targets, (long long)n};
    VDBC_TRY(run_grad(es, ntiles, (long long)n, params, part, loss_part, grid, grad_params, dloss, grad_inputs, s));
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
