// learn.cuh -- the learned leaf decoder's network on the tensor cores.
//
// Network (a project extension; the paper's Section 2.3 only mentions
// NeuralVDB as related work): x = (u, v, w, z_0..z_15) with (u, v, w) the
// voxel's position in its 8^3 leaf divided by 7 and z the leaf's latent;
// h1 = relu(W1 x + b1) (32), h2 = relu(W2 h1 + b2) (32), y = w3 . h2 + b3.
// A neural leaf decodes to offset + scale * clamp(y, 0, 1); its latent is
// stored in bf16, the precision the tensor cores read.
//
// Evaluation is warp-cooperative: 16 input rows (bf16, padded to 32
// columns; in a row the latent comes first, z_0..z_15, then u, v, w, so that
// the leaf's stored bf16 latent is copied into the row as it is) go through
// three layers of mma.sync.m16n8k16 (bf16 in, fp32
// accumulate): layer 1 = 2 k-steps x 4 n-tiles, layer 2 = 2 x 4, layer 3 =
// 2 x 1.  The accumulator fragments of two adjacent n-tiles are exactly the
// A fragment of the next layer's 16-wide k-step, so activations stay in
// registers (bias + relu + bf16 rounding on the way).  Weights are stored as
// per-lane B fragments (18 fragments x 32 lanes x 2 words).
//
// A row is 64 bytes = four 16-byte chunks; chunk c of row r sits at chunk
// slot c ^ ((r >> 1) & 3), which makes both the row stores and the fragment
// loads free of shared-memory bank conflicts.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "vdbc_device.cuh"

namespace vdbc {

constexpr int kMlpIn = 19, kMlpHid = 32, kMlpLatent = 16;
constexpr int kMlpParams = kMlpHid * kMlpIn + kMlpHid + kMlpHid * kMlpHid + kMlpHid + kMlpHid + 1;   // 1729
constexpr int kMlpFrags = 18;          // B fragments: layer 1 (0..7), layer 2 (8..15), layer 3 (16..17)
constexpr int kMlpBias = 2 * kMlpHid + 1;

// offsets of the parameter blocks in the FP32 parameter vector
constexpr int kOffW1 = 0, kOffB1 = kMlpHid * kMlpIn, kOffW2 = kOffB1 + kMlpHid, kOffB2 = kOffW2 + kMlpHid * kMlpHid,
              kOffW3 = kOffB2 + kMlpHid, kOffB3 = kOffW3 + kMlpHid;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);      // .x (low half) = lo
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], uint2 b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// word w of row r in a 16-row tile (16 words per row, swizzled chunks)
__device__ __forceinline__ int tile_word(int r, int w) { return r * 16 + ((((w >> 2) ^ (r >> 1)) & 3) << 2) + (w & 3); }

// y for the 16 rows of `rows` (16 x 16 words in shared memory, swizzled);
// all 32 lanes of the warp must call it together.  out[r] is written by the
// lanes with (lane & 3) == 0.
__device__ __forceinline__ void mlp_tile(const uint32_t* rows, const uint2* __restrict__ frag,
                                         const float* __restrict__ bias, float* out)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t a[2][4];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        a[s][0] = rows[tile_word(g, s * 8 + t)];
        a[s][1] = rows[tile_word(g + 8, s * 8 + t)];
        a[s][2] = rows[tile_word(g, s * 8 + 4 + t)];
        a[s][3] = rows[tile_word(g + 8, s * 8 + 4 + t)];
    }
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
        float c[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0f;
#pragma unroll
            for (int s = 0; s < 2; ++s) mma_bf16_16816(c[j], a[s], __ldg(frag + (layer * 8 + s * 4 + j) * 32 + lane));
        }
        const float* b = bias + layer * kMlpHid;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float b0 = __ldg(b + 8 * j + 2 * t), b1 = __ldg(b + 8 * j + 2 * t + 1);
            c[j][0] = fmaxf(__fadd_rn(c[j][0], b0), 0.0f);
            c[j][1] = fmaxf(__fadd_rn(c[j][1], b1), 0.0f);
            c[j][2] = fmaxf(__fadd_rn(c[j][2], b0), 0.0f);
            c[j][3] = fmaxf(__fadd_rn(c[j][3], b1), 0.0f);
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            a[s][0] = pack_bf16(c[2 * s][0], c[2 * s][1]);
            a[s][1] = pack_bf16(c[2 * s][2], c[2 * s][3]);
            a[s][2] = pack_bf16(c[2 * s + 1][0], c[2 * s + 1][1]);
            a[s][3] = pack_bf16(c[2 * s + 1][2], c[2 * s + 1][3]);
        }
    }
    float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int s = 0; s < 2; ++s) mma_bf16_16816(d, a[s], __ldg(frag + (16 + s) * 32 + lane));
    if (t == 0) {
        const float b3 = __ldg(bias + 2 * kMlpHid);
        out[g] = __fadd_rn(d[0], b3);
        out[g + 8] = __fadd_rn(d[2], b3);
    }
}

// row r of a tile: the leaf's latent (8 words of bf16 pairs, copied), then
// the voxel's position (i, j, k) / 7 rounded to bf16, zero padded to 32 columns
__device__ __forceinline__ void mlp_row_at(uint32_t* rows, int r, float u, float v, float w,
                                           const uint32_t* __restrict__ latent)
{
    const uint4* lp = reinterpret_cast<const uint4*>(latent);
    const uint4 q0 = __ldg(lp), q1 = __ldg(lp + 1);
    uint4* rp = reinterpret_cast<uint4*>(rows) + r * 4;
    const int sw = (r >> 1) & 3;
    rp[0 ^ sw] = q0;
    rp[1 ^ sw] = q1;
    rp[2 ^ sw] = make_uint4(pack_bf16(u, v), pack_bf16(w, 0.0f), 0u, 0u);
    rp[3 ^ sw] = make_uint4(0u, 0u, 0u, 0u);
}

__device__ __forceinline__ float seventh(int i) { return __fdiv_rn((float)i, 7.0f); }

// the same for voxel n = i + 8j + 64k of the leaf
__device__ __forceinline__ void mlp_row(uint32_t* rows, int r, int n, const uint32_t* __restrict__ latent)
{
    mlp_row_at(rows, r, seventh(n & 7), seventh((n >> 3) & 7), seventh(n >> 6), latent);
}

// the parameter column of W1 that row column k of a tile multiplies (-1: none)
__device__ __forceinline__ int w1_column(int k) { return k < kMlpLatent ? 3 + k : (k < kMlpIn ? k - kMlpLatent : -1); }

// B fragment f (0..17) of lane `lane` from the FP32 parameters, bf16-rounded:
// layer 1 (f = s*4 + j): W1[8j+g][c(16s+2t(+1))], W1[8j+g][c(16s+8+2t(+1))] with c the row
// column's parameter column (w1_column), zero where there is none;
// layer 2 (f = 8 + s*4 + j): W2[8j+g][16s+2t(+1)], ...; layer 3 (f = 16 + s): w3 in output column 0 only
__device__ __forceinline__ uint2 mlp_frag(const float* __restrict__ p, int f, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const int k0 = 16 * ((f < 8 ? f : (f < 16 ? f - 8 : f - 16)) >> (f < 16 ? 2 : 0)) + 2 * t;
    const int ks[4] = {k0, k0 + 1, k0 + 8, k0 + 9};
    float e[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (f < 8) {
            const int c = w1_column(ks[q]);
            e[q] = c >= 0 ? p[kOffW1 + (8 * (f & 3) + g) * kMlpIn + c] : 0.0f;
        } else if (f < 16) {
            e[q] = p[kOffW2 + (8 * ((f - 8) & 3) + g) * kMlpHid + ks[q]];
        } else {
            e[q] = g == 0 ? p[kOffW3 + ks[q]] : 0.0f;
        }
    }
    return make_uint2(pack_bf16(e[0], e[1]), pack_bf16(e[2], e[3]));
}

// Trilinear lookups in a learned grid.  Tiles and raw FP16 leaves decode as
// in a plain grid; a corner in a neural leaf becomes one row of a shared
// 16-row tile, and the warp pushes its tiles through the network together.
// collective() must be called by all 32 lanes of a warp at once (lanes
// without a lookup pass look = false); at most kMaxWarps warps per block.
struct LearnedSampler {
    static constexpr bool kCollective = true;
    static constexpr int kMaxWarps = 8;
    GridView g;

    // leaf-level entry through the accessor's cache; (scale, offset) of the
    // leaf from meta (raw) or nmeta (neural)
    __device__ __forceinline__ uint32_t leaf(Accessor& a, int li, int lj, int lk) const
    {
        if (a.find(g, li, lj, lk) && !(a.entry & kTile))
            a.sm = (a.entry & kNeural) ? __ldg(g.nmeta + (a.entry & ~kNeural)) : __ldg(g.meta + a.entry);
        return a.entry;
    }

    __device__ __forceinline__ float collective(bool look, float px, float py, float pz, Accessor& acc) const
    {
        __shared__ __align__(16) uint32_t s_rows[kMaxWarps][256];
        __shared__ float s_out[kMaxWarps][16];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        float v[8];
        uint32_t nmask = 0;
        float tx = 0.f, ty = 0.f, tz = 0.f;
        int xs[2] = {0, 0}, ys[2] = {0, 0}, zs[2] = {0, 0};
        if (look) {
            const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
            tx = px - fx; ty = py - fy; tz = pz - fz;
            const int i0 = (int)fx, j0 = (int)fy, k0 = (int)fz;
            xs[0] = min(max(i0, 0), g.nx - 1); xs[1] = min(max(i0 + 1, 0), g.nx - 1);
            ys[0] = min(max(j0, 0), g.ny - 1); ys[1] = min(max(j0 + 1, 0), g.ny - 1);
            zs[0] = min(max(k0, 0), g.nz - 1); zs[1] = min(max(k0 + 1, 0), g.nz - 1);
        }
        // As the plain sampler's default stencil mode: a stencil that
        // straddles at most two axes takes its up to four leaves at once (the
        // first corner's through the accessor, the others by descents that do
        // not wait on each other), for the whole warp unless one of its
        // lanes straddles all three axes; corner by corner otherwise.
        const int lx0 = xs[0] >> 3, ly0 = ys[0] >> 3, lz0 = zs[0] >> 3;
        const int S = (lx0 != (xs[1] >> 3) ? 1 : 0) | (ly0 != (ys[1] >> 3) ? 2 : 0) | (lz0 != (zs[1] >> 3) ? 4 : 0);
        if (__all_sync(0xffffffffu, !look || __popc(S) <= 2)) {
            if (look) {
                const int a1 = S & -S, a2 = S & ~a1;
                uint32_t e[4];
                float2 sm[4];
                e[0] = leaf(acc, lx0, ly0, lz0);
                sm[0] = acc.sm;
#pragma unroll
                for (int k = 1; k < 4; ++k) {
                    const int m = (k & 1 ? a1 : 0) | (k & 2 ? a2 : 0);
                    e[k] = e[0];
                    sm[k] = sm[0];
                    if (k == 1 ? a1 != 0 : a2 != 0) {   // a2 != 0 implies a1 != 0
                        e[k] = descend_to_leaf(g, m & 1 ? xs[1] >> 3 : lx0, m & 2 ? ys[1] >> 3 : ly0,
                                               m & 4 ? zs[1] >> 3 : lz0);
                        if (!(e[k] & kTile))
                            sm[k] = (e[k] & kNeural) ? __ldg(g.nmeta + (e[k] & ~kNeural)) : __ldg(g.meta + e[k]);
#ifdef VDBC_STATS
                        ++acc.queries;
                        ++acc.descents;
#endif
                    }
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int x = xs[c & 1], y = ys[(c >> 1) & 1], z = zs[c >> 2];
                    const int k = ((c & a1) ? 1 : 0) | ((c & a2) ? 2 : 0);
                    const uint32_t ek = k == 0 ? e[0] : k == 1 ? e[1] : k == 2 ? e[2] : e[3];
                    const float2 smk = k == 0 ? sm[0] : k == 1 ? sm[1] : k == 2 ? sm[2] : sm[3];
                    if (ek & kTile) {
                        v[c] = __ldg(g.tiles + (ek & ~kTile));
                    } else if (ek & kNeural) {
                        v[c] = __uint_as_float(ek & ~kNeural);      // the rank, until the network answers
                        nmask |= 1u << c;
                    } else {
                        v[c] = leaf_value_t<1>(g, ek, ((z & 7) << 6) | ((y & 7) << 3) | (x & 7), smk);
                    }
                }
            }
        } else if (look) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int x = xs[c & 1], y = ys[(c >> 1) & 1], z = zs[c >> 2];
                const uint32_t e = leaf(acc, x >> 3, y >> 3, z >> 3);
                if (e & kTile) {
                    v[c] = __ldg(g.tiles + (e & ~kTile));
                } else if (e & kNeural) {
                    v[c] = __uint_as_float(e & ~kNeural);      // the rank, until the network answers
                    nmask |= 1u << c;
                } else {
                    v[c] = leaf_value_t<1>(g, e, ((z & 7) << 6) | ((y & 7) << 3) | (x & 7), acc.sm);
                }
            }
        }
        // rows of the warp's neural corners: this lane's are [base, base + cnt)
        const int cnt = __popc(nmask);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int base = incl - cnt;
        uint32_t* rows = s_rows[wid];
        float* outs = s_out[wid];
        // the corners' in-leaf positions / 7: two values per axis, six divisions per lookup
        float pu[2] = {0.f, 0.f}, pv[2] = {0.f, 0.f}, pw[2] = {0.f, 0.f};
        if (nmask) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                pu[k] = seventh(xs[k] & 7);
                pv[k] = seventh(ys[k] & 7);
                pw[k] = seventh(zs[k] & 7);
            }
        }
        for (int t0 = 0; t0 < total; t0 += 16) {
            int q = base;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (nmask & (1u << c)) {
                    if (q >= t0 && q < t0 + 16)
                        mlp_row_at(rows, q - t0, pu[c & 1], pv[(c >> 1) & 1], pw[c >> 2],
                                   g.latents + (size_t)__float_as_uint(v[c]) * (kMlpLatent / 2));
                    ++q;
                }
            }
            __syncwarp();
            mlp_tile(rows, g.mlp_frag, g.mlp_bias, outs);   // rows past `total` are stale and unread
            __syncwarp();
            q = base;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (nmask & (1u << c)) {
                    if (q >= t0 && q < t0 + 16) {
                        const float2 m = __ldg(g.nmeta + __float_as_uint(v[c]));
                        v[c] = __fmaf_rn(m.x, fminf(fmaxf(outs[q - t0], 0.0f), 1.0f), m.y);
                    }
                    ++q;
                }
            }
            __syncwarp();
        }
        if (!look) return 0.0f;
        const float c00 = lerpf(v[0], v[1], tx), c10 = lerpf(v[2], v[3], tx);
        const float c01 = lerpf(v[4], v[5], tx), c11 = lerpf(v[6], v[7], tx);
        const float c0 = lerpf(c00, c10, ty), c1 = lerpf(c01, c11, ty);
        return lerpf(c0, c1, tz);
    }
};

}  // namespace vdbc
