// vdbc_device.cuh -- device-side data layout and lookup code of the grid.
//
// Layout (this library's own; the paper's NanoVDB is prior art, not copied):
//   one linear device block holds, at 256-byte aligned offsets,
//   root   u32[nroot]               dense table over the 4096^3 regions
//   upper  u32[n_upper * 32768]     32^3 children of 128^3 voxels each
//   lower  u32[n_lower * 4096]      16^3 children of 8^3 voxels each
//   tiles  f32[n_tiles]             tile values; tiles[0] is the background
//   leaves payload[n_leaves * 512]  8^3 values, x fastest (f32, f16 or e4m3)
//   meta   float2[n_leaves]         (scale, offset) of quantized leaves
//   mcmin, mcmax f32[n_macrocells]  min/max of the decoded grid per macrocell
//   learned grids add: latents bf16[n_neural * 16], nmeta float2[n_neural],
//   the network's B fragments u32x2[18 * 32], biases f32[65], params f32[1729]
// An entry of root/upper/lower is a child index (bit 31 clear) or a tile
// (bit 31 set, low bits index `tiles`).  This is the {5,4,3} tree of Section
// 2.3 with the root made a dense table because the input is a bounded
// structured-regular volume.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

// VDBC_CHECKED=1 builds (a separate library, libvdbc_checked.so) bounds-check
// every node, leaf and tile index against the grid's counts before the load;
// a violation sets kErrBounds in the grid's device error word and the lookup
// returns the background instead of reading outside the table.
#ifndef VDBC_CHECKED
#define VDBC_CHECKED 0
#endif

namespace vdbc {

// bits of the device error word (DevStats::error_flags)
enum : unsigned long long {
    kErrTrackSteps = 1ull << 0,    // a tracking loop hit its step bound
    kErrDdaSteps = 1ull << 1,      // a DDA walk hit its cell bound
    kErrBounds = 1ull << 2,        // an index outside its table (checked builds)
};

// tracker event counters of VDBC_STATS builds (vdbc_render_stats.events)
constexpr int kNumEvents = 8;

constexpr uint32_t kTile = 0x80000000u;
constexpr uint32_t kBackgroundEntry = 0x80000000u;   // tile 0
constexpr int kUpperN = 32768, kLowerN = 4096, kLeafN = 512;
constexpr int kMaxDim = 8192;
// largest macrocell edge in voxels (encode, dense volumes, grid files)
constexpr int kMaxMacrocell = 128;

struct GridView {
    int nx, ny, nz;
    int rx, ry, rz;           // root table size = ceil(dims / 4096)
    int payload;              // 0 f32, 1 f16, 2 e4m3
    int mc;                   // macrocell edge
    int mx, my, mz;           // macrocell grid
    float inv_m;              // 1 / max(dims)
    const uint32_t* root;
    const uint32_t* upper;
    const uint32_t* lower;
    const float* tiles;
    const void* leaves;
    const float2* meta;
    const float* mcmin;
    const float* mcmax;
    // learned grids (payload 3): latents (8 words per neural leaf: its 16
    // values as bf16 pairs) and (scale, offset) of neural leaves, network as B
    // fragments and biases; `leaves`/`meta` hold the FP16 fallbacks
    const uint32_t* latents;
    const float2* nmeta;
    const uint2* mlp_frag;
    const float* mlp_bias;
#if VDBC_CHECKED
    // checked builds: table sizes and the word a violation sets
    uint32_t n_upper, n_lower, n_tiles, n_leaves, n_neural;
    unsigned long long* err;
#endif
};

constexpr uint32_t kNeural = 0x40000000u;   // lower entry of a neural leaf (with bit 31 clear)
constexpr int kLearned = 3;

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: 10 rounds of two 32x32 multiplies, key bumped by the
// Weyl constants between rounds.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ float u01(uint32_t u) { return (float)(u >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------- leaf payload decode
__device__ __forceinline__ float e4m3_to_float(uint8_t b)
{
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
    return __half2float(__half(h));
}

// value `off` of leaf `leaf`; P is the payload (0 f32, 1 f16, 2 e4m3) or -1
// to read it from the grid at run time
template <int P>
__device__ __forceinline__ float leaf_value_t(const GridView& g, uint32_t leaf, int off, float2 sm)
{
    const int pay = P >= 0 ? P : g.payload;
    if (pay == 0) return __ldg(reinterpret_cast<const float*>(g.leaves) + (size_t)leaf * kLeafN + off);
    if (pay == 1) {
        __half h = reinterpret_cast<const __half*>(g.leaves)[(size_t)leaf * kLeafN + off];
        return __fmaf_rn(sm.x, __half2float(h), sm.y);
    }
    uint8_t b = reinterpret_cast<const uint8_t*>(g.leaves)[(size_t)leaf * kLeafN + off];
    return __fmaf_rn(sm.x, e4m3_to_float(b), sm.y);
}

__device__ __forceinline__ float leaf_value(const GridView& g, uint32_t leaf, int off, float2 sm)
{
    return leaf_value_t<-1>(g, leaf, off, sm);
}

// ---------------------------------------------------------------- descent
#if VDBC_CHECKED
static __device__ __noinline__ uint32_t bounds_violation(const GridView& g)
{
    atomicOr(g.err, kErrBounds);
    return kBackgroundEntry;
}

// a leaf-level entry names an existing tile, raw leaf or neural leaf
__device__ __forceinline__ bool entry_in_range(const GridView& g, uint32_t e)
{
    if (e & kTile) return (e & ~kTile) < g.n_tiles;
    if (g.payload == kLearned && (e & kNeural)) return (e & ~kNeural) < g.n_neural;
    return e < g.n_leaves;
}
#endif

// entry of the upper level that covers the lower node of voxel-leaf
// (li,lj,lk) = (i>>3, j>>3, k>>3): the lower node's index, or a tile entry
// (bit 31) when the node's whole 128^3 region is one value
__device__ __forceinline__ uint32_t descend_to_node(const GridView& g, int li, int lj, int lk)
{
    int i = li << 3, j = lj << 3, k = lk << 3;
#if VDBC_CHECKED
    if (li < 0 || lj < 0 || lk < 0 || i >= g.nx || j >= g.ny || k >= g.nz) return bounds_violation(g);
    uint32_t e = __ldg(g.root + ((k >> 12) * g.ry + (j >> 12)) * g.rx + (i >> 12));
    if (e & kTile) return entry_in_range(g, e) ? e : bounds_violation(g);
    if (e >= g.n_upper) return bounds_violation(g);
    e = __ldg(g.upper + (size_t)e * kUpperN + (((k >> 7) & 31) << 10) + (((j >> 7) & 31) << 5) + ((i >> 7) & 31));
    if (e & kTile) return entry_in_range(g, e) ? e : bounds_violation(g);
    return e < g.n_lower ? e : bounds_violation(g);
#else
    // (skipping the root load when the table is one entry naming upper node 0,
    // as it is for every volume up to 4096 voxels an edge, measured slower:
    // 8.97 against 8.59 ms on the 512^3 frame, 44.5 against 44.0 on the cloud)
    uint32_t e = __ldg(g.root + ((k >> 12) * g.ry + (j >> 12)) * g.rx + (i >> 12));
    if (e & kTile) return e;
    return __ldg(g.upper + (size_t)e * kUpperN + (((k >> 7) & 31) << 10) + (((j >> 7) & 31) << 5) + ((i >> 7) & 31));
#endif
}

// leaf-level entry of voxel-leaf (li,lj,lk) inside the lower node `node`
// (an entry from descend_to_node)
__device__ __forceinline__ uint32_t lower_entry(const GridView& g, uint32_t node, int li, int lj, int lk)
{
    if (node & kTile) return node;
    uint32_t e = __ldg(g.lower + (size_t)node * kLowerN + ((lk & 15) << 8) + ((lj & 15) << 4) + (li & 15));
#if VDBC_CHECKED
    return entry_in_range(g, e) ? e : bounds_violation(g);
#else
    return e;
#endif
}

// entry of the lower level that covers voxel-leaf (li,lj,lk): the whole
// descent root -> upper -> lower
__device__ __forceinline__ uint32_t descend_to_leaf(const GridView& g, int li, int lj, int lk)
{
    return lower_entry(g, descend_to_node(g, li, lj, lk), li, lj, lk);
}

// leaf coordinates (each below 1024, since no edge exceeds 8192 voxels)
// packed ten bits apiece; two keys with equal kNodeBits lie in one lower node
// (16^3 leaves).  Bit 30 never occurs in a key, so a reset accessor (key with
// every bit set) matches no leaf and no node.
__device__ __forceinline__ uint32_t leaf_key(int li, int lj, int lk)
{
    return (uint32_t)li | ((uint32_t)lj << 10) | ((uint32_t)lk << 20);
}
constexpr uint32_t kNodeBits = 0x3F0u | (0x3F0u << 10) | (0x3F0u << 20) | (1u << 30);

// Accessor cache depth (Section 3.2.2: NanoVDB's accessors cache the path of
// the last lookup).  1: the last leaf-level entry only, so another leaf costs
// the whole descent (three dependent loads); 2: also the lower node holding
// it, so another leaf of the same 128^3 region costs one load.  Depth 1 is
// the default: the tracker is bound by instruction issue, not by the load
// latency the deeper cache saves (1024^2 x 16 spp frame of the 512^3 medium:
// 8.57 ms at depth 1, 9.34 at depth 2; 1920x1080 x 64 spp of the
// 1987x1351x2449 cloud at 1:10: 44.01 against 45.53 ms).
#ifndef VDBC_ACC_DEPTH
#define VDBC_ACC_DEPTH 1
#endif
constexpr int kAccDepth = VDBC_ACC_DEPTH;

// per-thread cached accessor.  leaf() is for FP32/FP16/FP8 grids; learned
// grids resolve entries through LearnedSampler::leaf, which calls find() and
// knows the neural entries.
struct Accessor {
    uint32_t key;        // packed coordinates of the cached leaf (all ones: none)
    uint32_t entry;      // its leaf-level entry
    uint32_t node;       // depth 2: the lower node holding it (descend_to_node's answer)
    float2 sm;           // (scale, offset) of the cached leaf (quantized payloads)
#ifdef VDBC_STATS
    unsigned queries = 0, descents = 0;   // leaf queries, and those that changed the cached leaf
#endif
    __device__ __forceinline__ void reset()
    {
        key = 0xffffffffu;
        entry = kBackgroundEntry;
        node = kBackgroundEntry;
        sm = make_float2(0.f, 0.f);
    }
    // makes (a,b,c) the cached leaf; true when it was not already
    template <int D = kAccDepth>
    __device__ __forceinline__ bool find(const GridView& g, int a, int b, int c)
    {
        const uint32_t k = leaf_key(a, b, c);
#ifdef VDBC_STATS
        ++queries;
        if (k != key) ++descents;
#endif
        if (k == key) return false;
        if constexpr (D >= 2) {
            if ((k ^ key) & kNodeBits) node = descend_to_node(g, a, b, c);
            entry = lower_entry(g, node, a, b, c);
        } else {
            entry = descend_to_leaf(g, a, b, c);
        }
        key = k;
        return true;
    }
    template <int D = kAccDepth>
    __device__ __forceinline__ uint32_t leaf(const GridView& g, int a, int b, int c)
    {
        if (find<D>(g, a, b, c) && g.payload != 0 && !(entry & kTile)) sm = __ldg(g.meta + entry);
        return entry;
    }
};

template <int P, int D = kAccDepth>
__device__ __forceinline__ float voxel_t(const GridView& g, Accessor& acc, int i, int j, int k)
{
    uint32_t e = acc.leaf<D>(g, i >> 3, j >> 3, k >> 3);
    if (e & kTile) return __ldg(g.tiles + (e & ~kTile));
    return leaf_value_t<P>(g, e, ((k & 7) << 6) | ((j & 7) << 3) | (i & 7), acc.sm);
}

__device__ __forceinline__ float voxel(const GridView& g, Accessor& acc, int i, int j, int k)
{
    return voxel_t<-1>(g, acc, i, j, k);
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

// How the eight corners of a trilinear stencil are fetched.  A stencil inside
// one leaf can take the leaf once and its eight values from it (the one-leaf
// path); a stencil that straddles a leaf boundary (one in three at random
// positions) goes corner by corner through the accessor, where a corner in
// another leaf than the previous corner moves the cached leaf (a stencil
// across an x face alternates leaves corner by corner: up to eight descents,
// each waiting on the last).  The corner-by-corner path also serves one-leaf
// stencils, with the same values.
// 1: each lane takes the path its own stencil needs.  A warp whose lookups
//    include both kinds (nearly every warp) runs the two paths one after the
//    other.
// 4: the one-leaf path only when every active lane of the warp has a one-leaf
//    stencil, else corner by corner for all of them: one path per warp.
// 5: every stencil that straddles at most two axes (all but 0.2 % at random
//    positions) takes its up to four leaves at once: the first corner's
//    through the accessor, the others by descents that do not wait on each
//    other; corner by corner for the whole warp only when one of its lanes
//    straddles all three axes.
// 0: corner by corner always.
// 2: as 1, and stencils across one face (two leaves, the most frequent
//    straddle) take each leaf's entry once.
// 5 is the default: 24.5 ms against 27.1 (mode 4) on the full-scale cloud
// frame, 7.15 against 7.70 on the 512^3 frame; mode 4 had measured 33.99 ms
// against 34.98 (mode 1) and 34.26 (mode 0) on the cloud at 64^3 cells, 7.87
// against 8.31 and 7.83 on the 512^3 frame.  Images are bit-identical in
// every mode.  Mode 2's extra code cost more than the descents it saved (9.98
// against 8.57 ms on the 512^3 frame, 45.28 against 44.01 ms on the cloud,
// against mode 1 on an earlier tracker).  A form which found the lower node of
// the first corner's leaf once and took every other corner's leaf entry from
// it with independent loads measured 35.4 against 34.9 ms on the cloud and
// 8.28 against 8.30 on the 512^3 frame (against mode 1): the eight entries in
// flight cost spills (300 bytes a thread against 152).  Mode 5 with the lanes
// whose first corner shares a leaf taking its entry from one of them
// (__match_any_sync, one accessor lookup per leaf and warp, shuffles to the
// others) measured 25.5 against 23.9 ms on the cloud and 7.53 against 6.96 on
// the 512^3 frame: lanes that share a leaf already share its loads, which
// the memory system merges, and the match and shuffles cost every lookup.
// Mode 5 with the extra leaves taken from the first corner's lower node (one
// node descent, then one load per extra leaf) measured 24.4 against 23.9 ms
// on the cloud and 7.16 against 6.95 on the 512^3 frame.
#ifndef VDBC_TRI_STRADDLE
#define VDBC_TRI_STRADDLE 5
#endif
constexpr int kTriStraddle = VDBC_TRI_STRADDLE;

// trilinear reconstruction at index-space position p, clamp to edge; every
// call descends the tree (through the accessor's cached leaf) and decodes the
// eight voxels; P is the payload type of the grid (-1: read at run time), D
// the accessor's cache depth, T the straddle mode (kTriStraddle)
template <int P, int D = kAccDepth, int T = kTriStraddle>
__device__ __forceinline__ float vdb_trilinear(const GridView& g, float px, float py, float pz, Accessor& acc)
{
    float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
    float tx = px - fx, ty = py - fy, tz = pz - fz;
    int i0 = (int)fx, j0 = (int)fy, k0 = (int)fz;
    int x0 = min(max(i0, 0), g.nx - 1), x1 = min(max(i0 + 1, 0), g.nx - 1);
    int y0 = min(max(j0, 0), g.ny - 1), y1 = min(max(j0 + 1, 0), g.ny - 1);
    int z0 = min(max(k0, 0), g.nz - 1), z1 = min(max(k0 + 1, 0), g.nz - 1);
    float v000, v100, v010, v110, v001, v101, v011, v111;
    const int lx0 = x0 >> 3, ly0 = y0 >> 3, lz0 = z0 >> 3;
    const int S = (lx0 != (x1 >> 3) ? 1 : 0) | (ly0 != (y1 >> 3) ? 2 : 0) | (lz0 != (z1 >> 3) ? 4 : 0);
    bool fast = S == 0;
    if (T == 0 || T == 5) fast = false;
    if (T == 4) fast = __all_sync(__activemask(), S == 0);
    if (T == 5 && __all_sync(__activemask(), __popc(S) <= 2)) {
        // Up to four leaves: the stencil straddles at most two axes, a1 and
        // a2 (bit masks of x, y, z; zero when absent).  The first corner's
        // leaf comes through the accessor, the leaves across a1, a2 and both
        // from their own descents, which do not wait on each other; each
        // corner then takes the entry of the leaf its straddling bits name.
        const int a1 = S & -S, a2 = S & ~a1;
        const int lx1 = x1 >> 3, ly1 = y1 >> 3, lz1 = z1 >> 3;
        const int pay = P >= 0 ? P : g.payload;
        uint32_t e[4];
        float2 sm[4];
        e[0] = acc.leaf<D>(g, lx0, ly0, lz0);
        sm[0] = acc.sm;
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            const int m = (k & 1 ? a1 : 0) | (k & 2 ? a2 : 0);
            e[k] = e[0];
            sm[k] = sm[0];
            if (k == 1 ? a1 != 0 : a2 != 0) {   // a2 != 0 implies a1 != 0
                e[k] = descend_to_leaf(g, m & 1 ? lx1 : lx0, m & 2 ? ly1 : ly0, m & 4 ? lz1 : lz0);
                if (pay != 0 && !(e[k] & kTile)) sm[k] = __ldg(g.meta + e[k]);
#ifdef VDBC_STATS
                ++acc.queries;
                ++acc.descents;
#endif
            }
        }
        float v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int x = (c & 1) ? x1 : x0, y = (c & 2) ? y1 : y0, z = (c & 4) ? z1 : z0;
            const int k = ((c & a1) ? 1 : 0) | ((c & a2) ? 2 : 0);
            const uint32_t ek = k == 0 ? e[0] : k == 1 ? e[1] : k == 2 ? e[2] : e[3];
            const float2 smk = k == 0 ? sm[0] : k == 1 ? sm[1] : k == 2 ? sm[2] : sm[3];
            v[c] = (ek & kTile) ? __ldg(g.tiles + (ek & ~kTile))
                                : leaf_value_t<P>(g, ek, ((z & 7) << 6) | ((y & 7) << 3) | (x & 7), smk);
        }
        v000 = v[0]; v100 = v[1]; v010 = v[2]; v110 = v[3];
        v001 = v[4]; v101 = v[5]; v011 = v[6]; v111 = v[7];
    } else if (fast) {
        uint32_t e = acc.leaf<D>(g, lx0, ly0, lz0);
        if (e & kTile) return __ldg(g.tiles + (e & ~kTile));
        int ax = x0 & 7, bx = x1 & 7, ay = (y0 & 7) << 3, by = (y1 & 7) << 3;
        int az = (z0 & 7) << 6, bz = (z1 & 7) << 6;
        float2 sm = acc.sm;
        v000 = leaf_value_t<P>(g, e, az | ay | ax, sm); v100 = leaf_value_t<P>(g, e, az | ay | bx, sm);
        v010 = leaf_value_t<P>(g, e, az | by | ax, sm); v110 = leaf_value_t<P>(g, e, az | by | bx, sm);
        v001 = leaf_value_t<P>(g, e, bz | ay | ax, sm); v101 = leaf_value_t<P>(g, e, bz | ay | bx, sm);
        v011 = leaf_value_t<P>(g, e, bz | by | ax, sm); v111 = leaf_value_t<P>(g, e, bz | by | bx, sm);
    } else if (T == 2 && (S & (S - 1)) == 0) {
        // two leaves across one face: leaf A holds the corners whose bit S is
        // clear, leaf B the others
        const uint32_t eA = acc.leaf<D>(g, lx0, ly0, lz0);
        const float2 smA = acc.sm;
        const uint32_t eB = acc.leaf<D>(g, x1 >> 3, y1 >> 3, z1 >> 3);
        const float2 smB = acc.sm;
        float v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int x = (c & 1) ? x1 : x0, y = (c & 2) ? y1 : y0, z = (c & 4) ? z1 : z0;
            const bool b = (c & S) != 0;
            const uint32_t e = b ? eB : eA;
            v[c] = (e & kTile) ? __ldg(g.tiles + (e & ~kTile))
                               : leaf_value_t<P>(g, e, ((z & 7) << 6) | ((y & 7) << 3) | (x & 7), b ? smB : smA);
        }
        v000 = v[0]; v100 = v[1]; v010 = v[2]; v110 = v[3];
        v001 = v[4]; v101 = v[5]; v011 = v[6]; v111 = v[7];
    } else {
        v000 = voxel_t<P, D>(g, acc, x0, y0, z0); v100 = voxel_t<P, D>(g, acc, x1, y0, z0);
        v010 = voxel_t<P, D>(g, acc, x0, y1, z0); v110 = voxel_t<P, D>(g, acc, x1, y1, z0);
        v001 = voxel_t<P, D>(g, acc, x0, y0, z1); v101 = voxel_t<P, D>(g, acc, x1, y0, z1);
        v011 = voxel_t<P, D>(g, acc, x0, y1, z1); v111 = voxel_t<P, D>(g, acc, x1, y1, z1);
    }
    float c00 = lerpf(v000, v100, tx), c10 = lerpf(v010, v110, tx);
    float c01 = lerpf(v001, v101, tx), c11 = lerpf(v011, v111, tx);
    float c0 = lerpf(c00, c10, ty), c1 = lerpf(c01, c11, ty);
    return lerpf(c0, c1, tz);
}

template <int P, int D = kAccDepth, int T = kTriStraddle>
struct VdbSamplerT {
    static constexpr bool kCollective = false;
    GridView g;
    __device__ __forceinline__ float operator()(float px, float py, float pz, Accessor& acc) const
    {
        return vdb_trilinear<P, D, T>(g, px, py, pz, acc);
    }
};

// plain form, linear device array, the same software trilinear
struct LinearSampler {
    static constexpr bool kCollective = false;
    const float* d;
    int nx, ny, nz;
    __device__ __forceinline__ float at(int i, int j, int k) const
    {
        return __ldg(d + ((size_t)k * ny + j) * nx + i);
    }
    __device__ __forceinline__ float operator()(float px, float py, float pz, Accessor&) const
    {
        float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
        float tx = px - fx, ty = py - fy, tz = pz - fz;
        int i0 = (int)fx, j0 = (int)fy, k0 = (int)fz;
        int x0 = min(max(i0, 0), nx - 1), x1 = min(max(i0 + 1, 0), nx - 1);
        int y0 = min(max(j0, 0), ny - 1), y1 = min(max(j0 + 1, 0), ny - 1);
        int z0 = min(max(k0, 0), nz - 1), z1 = min(max(k0 + 1, 0), nz - 1);
        float c00 = lerpf(at(x0, y0, z0), at(x1, y0, z0), tx), c10 = lerpf(at(x0, y1, z0), at(x1, y1, z0), tx);
        float c01 = lerpf(at(x0, y0, z1), at(x1, y0, z1), tx), c11 = lerpf(at(x0, y1, z1), at(x1, y1, z1), tx);
        return lerpf(lerpf(c00, c10, ty), lerpf(c01, c11, ty), tz);
    }
};

// plain form, 3D CUDA texture with hardware trilinear and clamp addressing
// (unnormalized coordinates: texel centres sit at i + 1/2)
struct TexSampler {
    static constexpr bool kCollective = false;
    cudaTextureObject_t tex;
    __device__ __forceinline__ float operator()(float px, float py, float pz, Accessor&) const
    {
        return tex3D<float>(tex, px + 0.5f, py + 0.5f, pz + 0.5f);
    }
};

}  // namespace vdbc
