// encode.cu -- fixed-rate VDB encoding on the GPU.
//
// Section 3.1, Algorithm 1: histogram -> background B; 32^3 brick value
// ranges; sort by similarity f1/f2/f3 (Eq. f1-f3); activate the first bricks
// up to the rate.  Section 3.2.1: always keep the two extreme corner voxels,
// then prune (constant leaves become tiles).  Readings (shared with the
// CPU oracle, which is separate code): two-level bit-pattern histogram for B
// (ties to the smaller pattern), ceil brick grid, empty = range exactly
// [B,B], largest f first with ties to the lower brick index, exactly
// N = floor(numBricks * 131072 / (ratio * brick payload bytes)) bricks.
//
// Kernels, in order (every one is HBM- or latency-bound, none is a
// contraction):
//   k_candidate    one CTA: the most frequent of 1024 lattice voxels
//   k_pass1_maj    persistent: brick min/max and the exact count of that
//                  candidate; when it holds more than half of the voxels it
//                  is B, and the histogram kernels below return at once
//   k_pass1        persistent, one CTA per SM taking bricks in turn: min/max
//                  (total order) + upper-16-bit histogram (block histogram in
//                  shared memory, flushed per brick) + non-finite check
//   k_argmax       one CTA: most frequent bin, ties to the smaller index
//   k_pass2        one CTA per brick overlapping the winning bin: lower-16-bit
//                  histogram inside it (a brick of one bit pattern, known
//                  from its range, is counted without being read)
//   k_scores       one thread per brick: FP64 f with no contraction
//   k_select       one CTA: the N-th largest FP64 key, ties by brick index
//                  (bisection on keys in registers, up to 4096 bricks)
//   k_sel_*        the same above 4096 bricks over the whole GPU: radix
//                  passes by bytes, then ties ranked across CTAs
//   k_leaf_status  one warp per candidate leaf: constant? (prune) tile value?
//   scans (one CTA up to 64K entries), k_fill_* tree tables, k_fill_leaves
//                  payload copy / quantization
//   k_macrocells_input  FP32 grids: macrocell ranges from the input where a
//                  brick is active (else k_macrocells over the tree)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "vdbc_host.h"

namespace vdbc {
namespace {

__device__ __forceinline__ uint32_t okey(uint32_t b) { return (b & 0x80000000u) ? ~b : (b | 0x80000000u); }
__device__ __forceinline__ uint32_t okey_inv(uint32_t k) { return (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k; }

struct Dims {
    int nx, ny, nz;
    int bx, by, bz;     // brick grid
};

__device__ __forceinline__ void brick_coords(const Dims& d, int b, int& bx, int& by, int& bz)
{
    bx = b % d.bx;
    by = (b / d.bx) % d.by;
    bz = b / (d.bx * d.by);
}

// ---------------------------------------------------------------- pass 1
constexpr int kPassThreads = 256;

// Persistent blocks, one per SM, each taking bricks b = blockIdx.x, +grid,
// ...: a brick's min/max keys, and its counts of the upper 16 bits added to
// the global level-1 histogram.  The counts gather in a block-private
// histogram of 16-bit bins in shared memory, two to a word (a brick has 32768
// voxels, so no bin overflows into its neighbour); after each brick the block
// scans it, adds the non-zero bins to the global histogram and clears it.  A
// warp step whose values all share one key (empty space) adds to a per-warp
// run in registers; otherwise each lane adds its own values, equal keys
// merged first (the four of a float4, or a run down the lane's rows).
constexpr int kPass1Threads = 1024;
constexpr int kPass1Words = 32768;
constexpr size_t kPass1Smem = (size_t)kPass1Words * sizeof(uint32_t);

__device__ __forceinline__ void bin_add(uint32_t* h, uint32_t key, uint32_t n)
{
    atomicAdd(h + (key >> 1), n << ((key & 1u) * 16));
}

// adds the block histogram's non-zero bins to the global one and clears it
__device__ __forceinline__ void pass1_flush(uint32_t* h, unsigned long long* __restrict__ hist)
{
    uint4* h4 = reinterpret_cast<uint4*>(h);
    for (int i = threadIdx.x; i < kPass1Words / 4; i += kPass1Threads) {
        const uint4 c = h4[i];
        if ((c.x | c.y | c.z | c.w) == 0u) continue;
        h4[i] = make_uint4(0u, 0u, 0u, 0u);
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long bin = 2ll * (4 * i + j);
            if (w[j] & 0xffffu) atomicAdd(hist + bin, (unsigned long long)(w[j] & 0xffffu));
            if (w[j] >> 16) atomicAdd(hist + bin + 1, (unsigned long long)(w[j] >> 16));
        }
    }
}

// floor(r / d) for 0 <= r < 1024 and 1 <= d <= 32 by a multiply and a shift
// (m = ceil(2^21 / d); exact over that whole range, which an exhaustive check
// confirms, and r * m < 2^31): the row -> (y, z) split of a brick or part
__host__ __device__ __forceinline__ uint32_t div_magic(int d) { return ((1u << 21) + (uint32_t)d - 1u) / (uint32_t)d; }
__device__ __forceinline__ int div_small(int r, uint32_t m) { return (int)(((uint32_t)r * m) >> 21); }

// per-warp run of one key (warp-uniform): counts it in registers, and adds
// it to the global histogram when the key changes (runs are long: empty
// space, where a brick's every voxel may be one run; keeping them out of the
// block histogram lets a brick with no other counts skip the flush)
struct KeyRun {
    uint32_t key = 0xffffffffu, cnt = 0u;
    __device__ __forceinline__ void add(uint32_t k, uint32_t n, int lane, unsigned long long* g)
    {
        if (k == key) {
            cnt += n;
        } else {
            if (cnt && lane == 0) atomicAdd(g + key, (unsigned long long)cnt);
            key = k;
            cnt = n;
        }
    }
};

// ---------------------------------------------------------------- majority shortcut
// A bit pattern held by more than half of the voxels is the mode: its upper
// 16 bits win level 1 of the histogram and the pattern wins level 2, with no
// tie.  Sparse volumes are mostly one value (the cloud: 73 % zeros), so the
// encoder first samples a candidate, then counts it exactly while it takes
// the brick ranges (k_pass1_maj, no histogram); the histogram passes
// (k_pass1, k_pass2) and the argmax read the count and stand aside when the
// candidate holds the majority.  Otherwise they run in full and B comes from
// the histogram as before: the result is the same either way.
struct Majority {
    unsigned long long count;    // voxels holding `bits`
    uint32_t bits;               // the candidate pattern
    uint32_t pad;
};

__device__ __forceinline__ bool is_majority(const Majority* m, long long nvox)
{
    return m && 2ull * m->count > (unsigned long long)nvox;
}

// the candidate: the most frequent pattern among 1024 voxels on a 16 x 8 x 8
// lattice spanning the volume (ties to the smaller pattern); zeroes the count
__global__ void __launch_bounds__(1024) k_candidate(const float* __restrict__ v, Dims d, Majority* __restrict__ m)
{
    __shared__ uint32_t s_v[1024];
    __shared__ unsigned long long s_best[32];
    const int i = threadIdx.x;
    const int x = (int)((long long)(i & 15) * (d.nx - 1) / 15), y = (int)((long long)((i >> 4) & 7) * (d.ny - 1) / 7),
              z = (int)((long long)(i >> 7) * (d.nz - 1) / 7);
    s_v[i] = __float_as_uint(__ldg(v + ((size_t)z * d.ny + y) * d.nx + x));
    __syncthreads();
    const uint32_t mine = s_v[i];
    uint32_t n = 0;
    for (int j = 0; j < 1024; ++j) n += s_v[j] == mine ? 1u : 0u;
    unsigned long long best = ((unsigned long long)n << 32) | (uint32_t)~mine;
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
        best = t > best ? t : best;
    }
    if ((i & 31) == 0) s_best[i >> 5] = best;
    __syncthreads();
    if (i == 0) {
        for (int w = 1; w < 32; ++w) best = s_best[w] > best ? s_best[w] : best;
        m->bits = ~(uint32_t)best;
        m->count = 0ull;
    }
}

// pass 1 of the majority shortcut: every brick's min/max keys and the exact
// count of the candidate pattern c, with the loads of k_pass1 (kMode 1: float4
// rows; kMode 2: a warp steps one brick row through the z slices).  A step
// whose values all equal c only adds to the count; c joins the brick's range
// once at its end.  Non-finite input is found from the brick's keys.
template <int kMode>
__global__ void __launch_bounds__(kPass1Threads) k_pass1_maj(const float* __restrict__ v, Dims d, int nbricks,
                                                             uint32_t* __restrict__ lo_key, uint32_t* __restrict__ hi_key,
                                                             Majority* __restrict__ maj, int* __restrict__ nonfinite)
{
    constexpr int kWarps = kPass1Threads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t c = maj->bits;
    unsigned long long cnt = 0;          // (warp-uniform) voxels holding c
    bool bad = false;
    for (int b = blockIdx.x; b < nbricks; b += gridDim.x) {
        int bx, by, bz;
        brick_coords(d, b, bx, by, bz);
        const int x0 = bx * 32, y0 = by * 32, z0 = bz * 32;
        const int ex = min(32, d.nx - x0), ey = min(32, d.ny - y0), ez = min(32, d.nz - z0);
        uint32_t umax = 0u;
        int imin = 0x7fffffff, imax = (int)0x80000000;
        bool any = false, seen = false;
        if constexpr (kMode == 2) {
            constexpr int U = 32;          // a brick row's 32 slices in flight (16: 8.80 ms, 32: 8.06 on the
                                           // full-scale cloud encode; 24 splits the rows: 9.73).  Groups of
                                           // 2 or 4 bricks along x per warp row (256- or 512-byte runs, 8 to
                                           // 16 loads in flight within 64 registers) measured 9.5 against
                                           // 7.8 ms for the whole encode, and loads asking L2 for the
                                           // 256-byte block around them 7.80 against 7.81: the pass is
                                           // bound by the loads it keeps in flight, not by run length.
                                           // Four-byte cp.async copies into shared memory, one stage of
                                           // 16 slices in flight while the last is worked on, took 9.85
                                           // against 7.80 ms (the same grid): a four-byte asynchronous
                                           // copy costs more than the register it saves
            const bool valid = lane < ex;
            if (warp < ey) {
                const size_t slice = (size_t)d.nx * d.ny;
                const float* p = v + ((size_t)z0 * d.ny + (y0 + warp)) * d.nx + x0 + min(lane, ex - 1);
                for (int z = 0; z < ez; z += U) {
                    uint32_t u[U];
                    const float* a = p;
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        u[q] = 0u;
                        if (z + q < ez) u[q] = __float_as_uint(__ldg(a));
                        a += slice;
                    }
                    p = a;
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        if (z + q >= ez) break;                    // warp-uniform
                        const uint32_t w = u[q];
                        const bool eq = w == c;
                        if (__all_sync(0xffffffffu, eq)) {         // (lanes past the edge repeat a valid voxel)
                            cnt += (unsigned long long)ex;
                            seen = true;
                            continue;
                        }
                        any = true;
                        umax = max(umax, w);
                        imin = min(imin, (int)w);
                        imax = max(imax, (int)w);
                        cnt += (unsigned long long)__popc(__ballot_sync(0xffffffffu, eq && valid));
                    }
                }
            }
        } else {
            constexpr int U = 8;
            const int sub = lane & 7, rsub = lane >> 3;
            const bool xvalid = sub * 4 < ex;                      // ex is a multiple of 4 here
            const int rows = ey * ez;
            const uint32_t mey = div_magic(ey);
            const int quads = (rows + 3) >> 2;
            for (int g0 = warp; g0 < quads; g0 += kWarps * U) {
                uint4 u[U];
                bool ok[U];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int row = 4 * (g0 + q * kWarps) + rsub;
                    ok[q] = xvalid && row < rows;
                    u[q] = make_uint4(c, c, c, c);
                    if (ok[q]) {
                        const int z = div_small(row, mey), y = row - z * ey;
                        u[q] = __ldg(reinterpret_cast<const uint4*>(
                            v + ((size_t)(z0 + z) * d.ny + (y0 + y)) * d.nx + x0 + 4 * sub));
                    }
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    if (g0 + q * kWarps >= quads) break;                // warp-uniform
                    const uint32_t w[4] = {u[q].x, u[q].y, u[q].z, u[q].w};
                    const unsigned part = __ballot_sync(0xffffffffu, ok[q]);
                    const bool eq4 = w[0] == c && w[1] == c && w[2] == c && w[3] == c;   // (true where !ok)
                    if (__all_sync(0xffffffffu, eq4)) {
                        cnt += 4ull * (unsigned long long)__popc(part);
                        seen |= part != 0u;
                        continue;
                    }
                    unsigned n = 0u;
                    if (ok[q]) {
                        any = true;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            umax = max(umax, w[j]);
                            imin = min(imin, (int)w[j]);
                            imax = max(imax, (int)w[j]);
                            n += w[j] == c ? 1u : 0u;
                        }
                    }
                    cnt += (unsigned long long)__reduce_add_sync(0xffffffffu, n);
                }
            }
        }
        if (seen) {                                               // (warp-uniform)
            any = true;
            umax = max(umax, c);
            imin = min(imin, (int)c);
            imax = max(imax, (int)c);
        }
        // the warp's part of the brick folds into its keys (identity on
        // entry): no block barrier, warps move on to their next brick at once
        uint32_t kmin = 0xffffffffu, kmax = 0u;
        if (any) {
            kmin = okey((umax & 0x80000000u) ? umax : (uint32_t)imin);
            kmax = okey(imax >= 0 ? (uint32_t)imax : (uint32_t)imin);
        }
        kmin = __reduce_min_sync(0xffffffffu, kmin);
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        if (lane == 0 && kmin <= kmax) {
            atomicMin(lo_key + b, kmin);
            atomicMax(hi_key + b, kmax);
            if (kmax >= 0xff800000u || kmin <= 0x007fffffu) bad = true;   // a NaN or infinity in the part
        }
    }
    if (lane == 0 && cnt) atomicAdd(&maj->count, cnt);
    if (lane == 0 && bad) atomicOr(nonfinite, 1);
}

// kMode 1: the volume's rows start on 16-byte boundaries (nx % 4 == 0 and an
// aligned base), so a lane loads four voxels at once: lane = 8 * rsub + sub
// takes float4 `sub` of row 4g + rsub, and a warp covers four rows a load.
// kMode 2: scalar loads, one voxel a lane, for every other volume, each warp
// stepping one brick row through the z slices.  kMode 0: the scalar loads
// with the row index split per row (kept for comparison).  (Float4 loads of
// misaligned rows, masked to the brick row, measured slower than the scalar
// loads on both clouds, also as nine 16-byte blocks per row.)
template <int kMode, int kRowsInFlight = 8>
__global__ void __launch_bounds__(kPass1Threads) k_pass1(const float* __restrict__ v, Dims d, int nbricks,
                                                         uint32_t* __restrict__ lo_key,
                                                         uint32_t* __restrict__ hi_key,
                                                         unsigned long long* __restrict__ hist,
                                                         int* __restrict__ nonfinite,
                                                         const Majority* __restrict__ maj, long long nvox)
{
    if (is_majority(maj, nvox)) return;          // B is the counted candidate
    extern __shared__ __align__(16) uint32_t s_h[];
    __shared__ uint32_t s_min[2][kPass1Threads / 32], s_max[2][kPass1Threads / 32];
    __shared__ int s_bad;
    __shared__ int s_dirty[2];      // the block histogram holds counts of the brick (parity p)
    for (int i = threadIdx.x; i < kPass1Words; i += kPass1Threads) s_h[i] = 0u;
    if (threadIdx.x == 0) { s_bad = 0; s_dirty[0] = 0; s_dirty[1] = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int U = kRowsInFlight, kWarps = kPass1Threads / 32;
    bool bad = false;
    bool dirty = false;             // this thread added to the block histogram in this brick
    auto sadd = [&](uint32_t k, uint32_t n) {
        bin_add(s_h, k, n);
        dirty = true;
    };
    int p = 0;
    for (int b = blockIdx.x; b < nbricks; b += gridDim.x, p ^= 1) {
        int bx, by, bz;
        brick_coords(d, b, bx, by, bz);
        const int x0 = bx * 32, y0 = by * 32, z0 = bz * 32;
        const int ex = min(32, d.nx - x0), ey = min(32, d.ny - y0), ez = min(32, d.nz - z0);
        const int rows = ey * ez;
        const uint32_t mey = div_magic(ey);
        uint32_t kmin = 0xffffffffu, kmax = 0u;
        KeyRun run;
        if constexpr (kMode == 1) {
            const int sub = lane & 7, rsub = lane >> 3;
            const bool xvalid = sub * 4 < ex;             // ex is a multiple of 4 here
            const int quads = (rows + 3) >> 2;
            for (int g0 = warp; g0 < quads; g0 += kWarps * U) {
                uint4 u[U];
                bool ok[U];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int row = 4 * (g0 + q * kWarps) + rsub;
                    ok[q] = xvalid && row < rows;
                    u[q] = make_uint4(0u, 0u, 0u, 0u);
                    if (ok[q]) {
                        const int z = div_small(row, mey), y = row - z * ey;
                        u[q] = __ldg(reinterpret_cast<const uint4*>(
                            v + ((size_t)(z0 + z) * d.ny + (y0 + y)) * d.nx + x0 + 4 * sub));
                    }
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    if (g0 + q * kWarps >= quads) break;                // warp-uniform
                    const unsigned part = __ballot_sync(0xffffffffu, ok[q]);   // holds lane 0
                    const uint32_t w[4] = {u[q].x, u[q].y, u[q].z, u[q].w};
                    if (ok[q]) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            bad |= ((w[j] & 0x7f800000u) == 0x7f800000u);
                            const uint32_t k = okey(w[j]);
                            kmin = min(kmin, k);
                            kmax = max(kmax, k);
                        }
                    }
                    const uint32_t k0 = w[0] >> 16;
                    const uint32_t lead = __shfl_sync(0xffffffffu, k0, 0);
                    const bool same = !ok[q] || (k0 == lead && (w[1] >> 16) == lead && (w[2] >> 16) == lead &&
                                                 (w[3] >> 16) == lead);
                    if (__all_sync(0xffffffffu, same)) {
                        run.add(lead, 4u * (uint32_t)__popc(part), lane, hist);
                    } else {
                        // keys equal to the warp's run join it; the lane's other
                        // keys, equal ones merged, take one add per distinct key
                        const uint32_t k[4] = {w[0] >> 16, w[1] >> 16, w[2] >> 16, w[3] >> 16};
                        uint32_t n[4], c = 0u;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const bool in = ok[q] && k[j] == run.key;
                            c += in ? 1u : 0u;
                            n[j] = (ok[q] && !in) ? 1u : 0u;
                        }
                        run.cnt += __reduce_add_sync(0xffffffffu, c);
#pragma unroll
                        for (int j = 1; j < 4; ++j)
#pragma unroll
                            for (int i = 0; i < j; ++i)
                                if (n[j] && n[i] && k[i] == k[j]) { n[i] += n[j]; n[j] = 0u; }
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (n[j]) sadd(k[j], n[j]);
                    }
                }
            }
        } else if constexpr (kMode == 2) {
            // scalar loads with no index arithmetic per row: warp w takes brick
            // row y = w of every z slice, lane = x, and the row pointer
            // advances by one slice (the per-row index products of kMode 0
            // kept the integer multiply pipe busy).  Lanes past the brick's
            // edge load lane ex - 1's voxel again: a duplicate changes neither
            // the range nor whether a step is one key, so only the histogram
            // adds test `valid`.  The range is kept on the raw bits (unsigned
            // max, signed min and max) and mapped to the total-order keys once
            // per brick; non-finite values are found from the brick's keys.
            const bool valid = lane < ex;
            const uint32_t nvalid = (uint32_t)ex;
            if (warp < ey) {
                const size_t slice = (size_t)d.nx * d.ny;
                const float* p = v + ((size_t)z0 * d.ny + (y0 + warp)) * d.nx + x0 + min(lane, ex - 1);
                uint32_t umax = 0u;
                int imin = 0x7fffffff, imax = (int)0x80000000;
                // the value of the warp's run when a step of it was one value
                // (already in the range; its key is run.key): a step of only
                // that value adds nothing to the range and joins the run
                uint32_t rv = 0u;
                bool rvok = false;
                for (int z = 0; z < ez; z += U) {
                    uint32_t u[U];
                    const float* a = p;
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        u[q] = 0u;
                        if (z + q < ez) u[q] = __float_as_uint(__ldg(a));
                        a += slice;
                    }
                    p = a;
                    uint32_t lk = 0xffffffffu, ln = 0u;            // the lane's run of one key
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        if (z + q >= ez) break;                    // warp-uniform
                        const uint32_t w = u[q];
                        if (rvok && __all_sync(0xffffffffu, w == rv)) {
                            run.cnt += nvalid;
                            continue;
                        }
                        const uint32_t key = w >> 16;
                        umax = max(umax, w);
                        imin = min(imin, (int)w);
                        imax = max(imax, (int)w);
                        if (__all_sync(0xffffffffu, key == run.key)) {
                            run.cnt += nvalid;
                            if (!rvok) {                           // (warp-uniform)
                                rv = __shfl_sync(0xffffffffu, w, 0);
                                rvok = __all_sync(0xffffffffu, w == rv);
                            }
                            continue;
                        }
                        const uint32_t lw = __shfl_sync(0xffffffffu, w, 0), lead = lw >> 16;
                        if (__all_sync(0xffffffffu, key == lead)) {
                            run.add(lead, nvalid, lane, hist);
                            rv = lw;
                            rvok = __all_sync(0xffffffffu, w == lw);
                            continue;
                        }
                        const bool inrun = valid && key == run.key;
                        run.cnt += (uint32_t)__popc(__ballot_sync(0xffffffffu, inrun));
                        if (valid && !inrun) {
                            if (key == lk) {
                                ++ln;
                            } else {
                                if (ln) sadd(lk, ln);
                                lk = key;
                                ln = 1u;
                            }
                        }
                    }
                    if (ln) sadd(lk, ln);
                }
                // smallest in the total order: the largest negative pattern if
                // there is one, else the smallest non-negative; largest: the
                // largest non-negative if there is one, else the negative
                // pattern nearest -0
                kmin = okey((umax & 0x80000000u) ? umax : (uint32_t)imin);
                kmax = okey(imax >= 0 ? (uint32_t)imax : (uint32_t)imin);
            }
        } else {
            const bool valid = lane < ex;
            const unsigned vmask = __ballot_sync(0xffffffffu, valid);
            // U consecutive rows per warp, their loads in flight before any is
            // used; a lane's values are then vertical neighbours, and equal
            // keys in a row of them merge into one add
            for (int r0 = warp * U; r0 < rows; r0 += kWarps * U) {
                uint32_t u[U];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int row = r0 + q;
                    u[q] = 0u;
                    if (valid && row < rows) {
                        const int z = div_small(row, mey), y = row - z * ey;
                        u[q] = __float_as_uint(__ldg(v + ((size_t)(z0 + z) * d.ny + (y0 + y)) * d.nx + x0 + lane));
                    }
                }
                uint32_t lk = 0xffffffffu, ln = 0u;            // the lane's run of one key
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    if (r0 + q >= rows) break;                 // warp-uniform
                    const uint32_t w = u[q];
                    const uint32_t key = w >> 16;
                    if (valid) {
                        bad |= ((w & 0x7f800000u) == 0x7f800000u);
                        const uint32_t k = okey(w);
                        kmin = min(kmin, k);
                        kmax = max(kmax, k);
                    }
                    const uint32_t lead = __shfl_sync(0xffffffffu, key, 0);     // lane 0 is always valid
                    if (__all_sync(0xffffffffu, !valid || key == lead)) {
                        run.add(lead, (uint32_t)__popc(vmask), lane, hist);
                        continue;
                    }
                    // lanes holding the warp run's key join it; the others keep
                    // their own runs
                    const bool inrun = valid && key == run.key;
                    run.cnt += (uint32_t)__popc(__ballot_sync(0xffffffffu, inrun));
                    if (valid && !inrun) {
                        if (key == lk) {
                            ++ln;
                        } else {
                            if (ln) sadd(lk, ln);
                            lk = key;
                            ln = 1u;
                        }
                    }
                }
                if (ln) sadd(lk, ln);
            }
        }
        if (run.cnt && lane == 0) atomicAdd(hist + run.key, (unsigned long long)run.cnt);
        if (__any_sync(0xffffffffu, dirty) && lane == 0) s_dirty[p] = 1;
        dirty = false;
        kmin = __reduce_min_sync(0xffffffffu, kmin);
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        if (lane == 0) { s_min[p][warp] = kmin; s_max[p][warp] = kmax; }
        __syncthreads();                                   // the brick's counts and ranges are in
        if (threadIdx.x == 0) {
            uint32_t a = s_min[p][0], c = s_max[p][0];
            for (int w = 1; w < kWarps; ++w) { a = min(a, s_min[p][w]); c = max(c, s_max[p][w]); }
            lo_key[b] = a;
            hi_key[b] = c;
            // a NaN or infinity has a key beyond okey(+inf) or below okey(-inf)
            if (c >= 0xff800000u || a <= 0x007fffffu) bad = true;
        }
        if (s_dirty[p]) pass1_flush(s_h, hist);            // (a brick of runs alone left it empty)
        if (threadIdx.x == 0) s_dirty[p ^ 1] = 0;
        __syncthreads();                                   // histogram clear before the next brick
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&s_bad, 1);
    __syncthreads();
    if (threadIdx.x == 0 && s_bad) atomicOr(nonfinite, 1);
}

// most frequent of 65536 bins, ties to the smaller index; writes (out_base | idx)
__global__ void __launch_bounds__(1024) k_argmax(const unsigned long long* __restrict__ hist,
                                                 uint32_t* __restrict__ out, int stage,
                                                 const Majority* __restrict__ maj, long long nvox)
{
    if (is_majority(maj, nvox)) {                // the counted candidate is the mode
        if (threadIdx.x == 0) {
            if (stage == 0) out[0] = maj->bits >> 16;
            else out[1] = maj->bits;
        }
        return;
    }
    __shared__ unsigned long long s[32];
    unsigned long long best = 0;
    for (int i = threadIdx.x; i < 65536; i += 1024) {
        unsigned long long p = (hist[i] << 16) | (unsigned long long)(0xffffu - (uint32_t)i);
        best = p > best ? p : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
        best = t > best ? t : best;
    }
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 32; ++w) best = s[w] > best ? s[w] : best;
        s[0] = best > s[0] ? best : s[0];
        uint32_t idx = 0xffffu - (uint32_t)(s[0] & 0xffffu);
        // stage 0 -> upper 16 bits; stage 1 -> B = upper << 16 | lower
        if (stage == 0) out[0] = idx;
        else out[1] = (out[0] << 16) | idx;
    }
}

// ---------------------------------------------------------------- pass 2
// One block per brick whose range reaches the winning bin H: the lower 16 bits
// of its values inside the bin, counted into the level-2 histogram.  A warp
// step whose in-bin values all share one key (the background itself, inside
// empty space and at its edge) adds to a per-warp run in registers instead
// of an atomic on that one global bin.  kVec: float4 rows, as pass 1 in kMode 1.
template <bool kVec>
__device__ __forceinline__ void pass2_brick(const float* __restrict__ v, const Dims& d,
                                            const uint32_t* __restrict__ lo_key, const uint32_t* __restrict__ hi_key,
                                            const uint32_t* __restrict__ bsel, unsigned long long* __restrict__ hist,
                                            const int b)
{
    const uint32_t H = bsel[0];
    // key range of the bit patterns [H<<16, H<<16 | 0xffff]
    const uint32_t p0 = H << 16, p1 = (H << 16) | 0xffffu;
    const uint32_t ka = min(okey(p0), okey(p1)), kb = max(okey(p0), okey(p1));
    if (hi_key[b] < ka || lo_key[b] > kb) return;       // no value of this brick is in the bin
    int bx, by, bz;
    brick_coords(d, b, bx, by, bz);
    const int x0 = bx * 32, y0 = by * 32, z0 = bz * 32;
    const int ex = min(32, d.nx - x0), ey = min(32, d.ny - y0), ez = min(32, d.nz - z0);
    if (lo_key[b] == hi_key[b]) {
        // every voxel holds one bit pattern (the key order is a bijection on
        // patterns), and it lies in the bin: count the brick without reading it
        if (threadIdx.x == 0)
            atomicAdd(hist + (okey_inv(lo_key[b]) & 0xffffu), (unsigned long long)ex * ey * ez);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rows = ey * ez;
    const uint32_t mey = div_magic(ey);
    constexpr int kW = kPassThreads / 32;
    uint32_t run_key = 0xffffffffu;          // per-warp run of one key (warp-uniform)
    unsigned long long run_cnt = 0;
    auto run_add = [&](uint32_t k, unsigned long long n) {
        if (k == run_key) {
            run_cnt += n;
        } else {
            if (run_cnt && lane == 0) atomicAdd(hist + run_key, run_cnt);
            run_key = k;
            run_cnt = n;
        }
    };
    if constexpr (kVec) {
        constexpr int U = 4;
        const int sub = lane & 7, rsub = lane >> 3;
        const bool xvalid = sub * 4 < ex;
        const int quads = (rows + 3) >> 2;
        for (int g0 = warp; g0 < quads; g0 += kW * U) {
            uint4 u[U];
            bool ok[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int row = 4 * (g0 + q * kW) + rsub;
                ok[q] = xvalid && row < rows;
                u[q] = make_uint4(0u, 0u, 0u, 0u);
                if (ok[q]) {
                    const int z = div_small(row, mey), y = row - z * ey;
                    u[q] = __ldg(reinterpret_cast<const uint4*>(
                        v + ((size_t)(z0 + z) * d.ny + (y0 + y)) * d.nx + x0 + 4 * sub));
                }
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                if (g0 + q * kW >= quads) break;                      // warp-uniform
                const uint32_t w[4] = {u[q].x, u[q].y, u[q].z, u[q].w};
                unsigned in = 0u;                                     // this lane's values in the bin
#pragma unroll
                for (int j = 0; j < 4; ++j) in |= (ok[q] && (w[j] >> 16) == H) ? (1u << j) : 0u;
                const unsigned m = __ballot_sync(0xffffffffu, in != 0u);
                if (m == 0u) continue;
                const uint32_t first = (in & 1u) ? w[0] : (in & 2u) ? w[1] : (in & 4u) ? w[2] : w[3];
                const uint32_t mine = first & 0xffffu;          // only read from a lane with in != 0
                const uint32_t lead = __shfl_sync(0xffffffffu, mine, __ffs(m) - 1);
                bool same = true;
#pragma unroll
                for (int j = 0; j < 4; ++j) same &= !((in >> j) & 1u) || (w[j] & 0xffffu) == lead;
                if (__all_sync(0xffffffffu, same)) {
                    run_add(lead, (unsigned long long)__reduce_add_sync(0xffffffffu, (unsigned)__popc(in)));
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool inj = (in >> j) & 1u;
                        const unsigned mj = __ballot_sync(0xffffffffu, inj);
                        if (mj == 0u) continue;
                        const unsigned peers = inj ? __match_any_sync(mj, w[j] & 0xffffu) : 0u;
                        if (inj && lane == __ffs(peers) - 1)
                            atomicAdd(hist + (w[j] & 0xffffu), (unsigned long long)__popc(peers));
                    }
                }
            }
        }
    } else {
        constexpr int U = 8;
        const bool valid = lane < ex;
        for (int r0 = warp * U; r0 < rows; r0 += kW * U) {
            uint32_t u[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int row = r0 + q;
                u[q] = 0;
                if (valid && row < rows) {
                    const int z = div_small(row, mey), y = row - z * ey;
                    u[q] = __float_as_uint(__ldg(v + ((size_t)(z0 + z) * d.ny + (y0 + y)) * d.nx + x0 + lane));
                }
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                if (r0 + q >= rows) break;               // warp-uniform
                const uint32_t w = u[q];
                const bool in = valid && (w >> 16) == H;
                const unsigned m = __ballot_sync(0xffffffffu, in);       // warp-uniform
                if (m == 0u) continue;
                const unsigned peers = in ? __match_any_sync(m, w & 0xffffu) : 0u;   // only the lanes of m call it
                const int leader = __ffs(m) - 1;
                if (__shfl_sync(0xffffffffu, peers, leader) == m) {
                    run_add(__shfl_sync(0xffffffffu, w & 0xffffu, leader), (unsigned long long)__popc(m));
                } else if (in && lane == __ffs(peers) - 1) {
                    atomicAdd(hist + (w & 0xffffu), (unsigned long long)__popc(peers));
                }
            }
        }
    }
    if (run_cnt && lane == 0) atomicAdd(hist + run_key, run_cnt);
}

// blocks take bricks in turn (a few per SM): when the candidate holds the
// majority every block returns at once, and a block per brick cost 0.1 ms of
// launches on the full-scale cloud for nothing
template <bool kVec>
__global__ void __launch_bounds__(kPassThreads) k_pass2(const float* __restrict__ v, Dims d,
                                                        const uint32_t* __restrict__ lo_key,
                                                        const uint32_t* __restrict__ hi_key,
                                                        const uint32_t* __restrict__ bsel,
                                                        unsigned long long* __restrict__ hist,
                                                        const Majority* __restrict__ maj, long long nvox, int nbricks)
{
    if (is_majority(maj, nvox)) return;          // B is the counted candidate
    for (int b = blockIdx.x; b < nbricks; b += gridDim.x) pass2_brick<kVec>(v, d, lo_key, hi_key, bsel, hist, b);
}

// ---------------------------------------------------------------- scores (Eq. f1-f3)
__global__ void k_scores(const uint32_t* __restrict__ lo_key, const uint32_t* __restrict__ hi_key,
                         int nb, const uint32_t* __restrict__ bsel, int metric,
                         unsigned long long* __restrict__ fkey, uint8_t* __restrict__ empty)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    uint32_t bb = bsel[1];
    uint32_t lb = okey_inv(lo_key[i]), hb = okey_inv(hi_key[i]);
    double B = (double)__uint_as_float(bb);
    double lo = (double)__uint_as_float(lb), hi = (double)__uint_as_float(hb);
    double dl = fabs(__dsub_rn(lo, B)), dh = fabs(__dsub_rn(hi, B));
    double f;
    if (metric == VDBC_F1) f = dl < dh ? dl : dh;
    else if (metric == VDBC_F3) f = fabs(__dsub_rn(__ddiv_rn(__dadd_rn(lo, hi), 2.0), B));
    else f = dl > dh ? dl : dh;
    fkey[i] = (unsigned long long)__double_as_longlong(f);   // f >= 0: bits are monotone
    empty[i] = (uint8_t)(lb == bb && hb == bb);
}

// ---------------------------------------------------------------- selection
// sum over the block (1024 threads) of a per-thread count; every thread gets it
__device__ __forceinline__ unsigned block_count(unsigned x, unsigned* s, unsigned* s_tot)
{
    x = __reduce_add_sync(0xffffffffu, x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < (int)(blockDim.x >> 5) ? s[lane] : 0u;
        t = __reduce_add_sync(0xffffffffu, t);
        if (lane == 0) *s_tot = t;
    }
    __syncthreads();
    return *s_tot;
}

// the N largest keys among non-empty bricks, ties to the lower index; one CTA
// of 1024 threads.  A key is held as fkey + 1 (0 for an empty brick), in
// registers when there are at most 4096 bricks.
constexpr int kSelThreads = 1024, kSelCache = 4, kSelBatch = 8;

__global__ void __launch_bounds__(kSelThreads) k_select(const unsigned long long* __restrict__ fkey,
                                                        const uint8_t* __restrict__ empty, int nb,
                                                        long long budget, uint8_t* __restrict__ active,
                                                        long long* __restrict__ counts)
{
    __shared__ unsigned s[32];
    __shared__ unsigned s_tot;
    __shared__ long long s_run;
    const bool cached = nb <= kSelCache * kSelThreads;
    unsigned long long ck[kSelCache];
#pragma unroll
    for (int q = 0; q < kSelCache; ++q) {
        const int i = threadIdx.x + q * kSelThreads;
        ck[q] = (cached && i < nb && !empty[i]) ? fkey[i] + 1ull : 0ull;
    }
    auto key1 = [&](int i) -> unsigned long long { return empty[i] ? 0ull : fkey[i] + 1ull; };
    // number of keys (+1) >= c (c >= 1), and of keys (+1) > c
    auto count_ge = [&](unsigned long long c) -> unsigned {
        unsigned n = 0;
        if (cached) {
#pragma unroll
            for (int q = 0; q < kSelCache; ++q) n += ck[q] >= c ? 1u : 0u;
        } else {
            for (int i = threadIdx.x; i < nb; i += kSelThreads) n += key1(i) >= c ? 1u : 0u;
        }
        return block_count(n, s, &s_tot);
    };
    const long long m = count_ge(1ull);
    const long long take = budget < m ? budget : m;
    if (take == m || take == 0) {
        for (int i = threadIdx.x; i < nb; i += kSelThreads) active[i] = (take > 0 && !empty[i]) ? 1 : 0;
        if (threadIdx.x == 0) { counts[0] = m; counts[1] = take; }
        return;
    }
    // V = the take-th largest key (+1); gt = #{keys (+1) > V}
    unsigned long long V = 0;
    long long gt = 0;
    if (cached) {
        // bisection on the bits of the threshold T: the largest T with #{key >= T} >= take
        unsigned long long T = 0;
        for (int bit = 63; bit >= 0; --bit) {
            const unsigned long long cand = T | (1ull << bit);
            if (cand <= 0xFFFFFFFFFFFFFFFEull && (long long)count_ge(cand + 1ull) >= take) T = cand;
        }
        V = T + 1ull;
        gt = T == 0xFFFFFFFFFFFFFFFFull ? 0 : (long long)count_ge(T + 2ull);
    } else {
        // keys in global memory: radix selection from the top byte down, one
        // pass over the keys per byte (8 instead of 64 bisection passes); a
        // pass counts the byte of every key whose higher bytes equal the
        // prefix chosen so far, and keeps the byte at which the count from the
        // top reaches the rank still wanted
        // (per-warp digit counts, summed once per pass: the keys share their
        // top bytes, and one shared count per digit had every warp's adds
        // collide on a few bins)
        __shared__ unsigned s_hist[256];
        __shared__ unsigned s_whist[kSelThreads / 32][256];
        __shared__ unsigned long long s_prefix;
        __shared__ long long s_rank;
        unsigned long long prefix = 0, pmask = 0;
        long long rank = take;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int i = threadIdx.x; i < (kSelThreads / 32) * 256; i += kSelThreads) (&s_whist[0][0])[i] = 0u;
            __syncthreads();
            // kSelBatch keys a thread loaded before any is counted, so that
            // their L2 latencies overlap
            for (int base = 0; base < nb; base += kSelThreads * kSelBatch) {
                unsigned long long kk[kSelBatch];
#pragma unroll
                for (int j = 0; j < kSelBatch; ++j) {
                    const int i = base + j * kSelThreads + threadIdx.x;
                    kk[j] = i < nb ? key1(i) : 0ull;
                }
#pragma unroll
                for (int j = 0; j < kSelBatch; ++j) {
                    const unsigned long long k = kk[j];
                    const bool in = k != 0ull && (k & pmask) == prefix;
                    const unsigned digit = in ? (unsigned)(k >> shift) & 255u : 256u;
                    const unsigned peers = __match_any_sync(0xffffffffu, digit);
                    if (in && lane == __ffs(peers) - 1) s_whist[wid][digit] += (unsigned)__popc(peers);
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < 256; i += kSelThreads) {
                unsigned t = 0u;
                for (int w = 0; w < kSelThreads / 32; ++w) t += s_whist[w][i];
                s_hist[i] = t;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                long long above = 0;
                int d = 255;
                for (; d > 0; --d) {
                    if (above + (long long)s_hist[d] >= rank) break;
                    above += s_hist[d];
                }
                s_prefix = prefix | ((unsigned long long)d << shift);
                s_rank = rank - above;
            }
            __syncthreads();
            prefix = s_prefix;
            rank = s_rank;
            pmask |= 255ull << shift;
            __syncthreads();
        }
        V = prefix;
        gt = take - rank;
    }
    const unsigned long long T = V - 1ull;
    const long long need = take - gt;   // keys equal to T, lowest brick indices first
    // kSelBatch chunks of kSelThreads bricks a round: a tie's rank is the ties
    // of earlier rounds, of earlier chunks of this round, of earlier warps of
    // its chunk and of earlier lanes of its warp
    __shared__ unsigned s_ties[kSelBatch][kSelThreads / 32];
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += kSelThreads * kSelBatch) {
        unsigned long long kk[kSelBatch];
        unsigned bal[kSelBatch];
#pragma unroll
        for (int j = 0; j < kSelBatch; ++j) {
            const int i = base + j * kSelThreads + threadIdx.x;
            kk[j] = i < nb ? key1(i) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kSelBatch; ++j) {
            bal[j] = __ballot_sync(0xffffffffu, kk[j] != 0ull && kk[j] == T + 1ull);
            if (lane == 0) s_ties[j][w] = __popc(bal[j]);
        }
        __syncthreads();
        long long before = s_run;
#pragma unroll
        for (int j = 0; j < kSelBatch; ++j) {
            const int i = base + j * kSelThreads + threadIdx.x;
            long long mine = before + __popc(bal[j] & ((1u << lane) - 1u));
            for (int q = 0; q < w; ++q) mine += s_ties[j][q];
            const unsigned long long k = kk[j];
            const bool eq = k != 0ull && k == T + 1ull;
            if (i < nb) active[i] = (k != 0ull && (k > T + 1ull || (eq && mine < need))) ? 1 : 0;
            for (int q = 0; q < kSelThreads / 32; ++q) before += s_ties[j][q];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_run = before;
        __syncthreads();
    }
    if (threadIdx.x == 0) { counts[0] = m; counts[1] = take; }
}

// ---------------------------------------------------------------- selection above 4096 bricks, grid-wide
// The same selection as k_select's global-memory branch (the N-th largest
// key by bytes from the top, ties by brick index), over the whole GPU: one
// CTA on one SM spent most of its time in the warp matches of its eight
// passes (0.8 ms for the full-scale cloud's 208,593 bricks).  Per pass, the
// CTAs count the digit of every key under the prefix chosen so far (per-warp
// counts in shared memory, one global add per digit and CTA) and one thread
// picks the digit; then the CTAs count the keys equal to the threshold in
// their brick ranges, and rank them by brick index from those counts.
constexpr int kSelMaxCtas = 1024;
struct SelState {
    unsigned long long prefix, pmask;
    long long rank, m, take;
    int done;                     // take == m or take == 0: every non-empty brick, or none
    int pad;
    unsigned hist[256];
    unsigned ties[kSelMaxCtas];   // keys equal to the threshold in each CTA's brick range
};

__device__ __forceinline__ unsigned long long sel_key1(const unsigned long long* __restrict__ fkey,
                                                       const uint8_t* __restrict__ empty, int i)
{
    return empty[i] ? 0ull : fkey[i] + 1ull;
}

__global__ void k_sel_init(SelState* st)
{
    if (threadIdx.x == 0) {
        st->prefix = 0ull;
        st->pmask = 0ull;
        st->rank = st->m = st->take = 0;
        st->done = 0;
    }
    for (int i = threadIdx.x; i < 256; i += blockDim.x) st->hist[i] = 0u;
}

// one pass: the digit at `shift` of every non-empty key under the prefix
__global__ void __launch_bounds__(kSelThreads) k_sel_hist(const unsigned long long* __restrict__ fkey,
                                                          const uint8_t* __restrict__ empty, int nb,
                                                          SelState* __restrict__ st, int shift)
{
    __shared__ unsigned s_w[kSelThreads / 32][256];
    if (st->done) return;
    for (int i = threadIdx.x; i < (kSelThreads / 32) * 256; i += kSelThreads) (&s_w[0][0])[i] = 0u;
    __syncthreads();
    const unsigned long long prefix = st->prefix, pmask = st->pmask;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = blockIdx.x * kSelThreads * kSelBatch; base < nb; base += gridDim.x * kSelThreads * kSelBatch) {
        unsigned long long kk[kSelBatch];
#pragma unroll
        for (int j = 0; j < kSelBatch; ++j) {
            const int i = base + j * kSelThreads + threadIdx.x;
            kk[j] = i < nb ? sel_key1(fkey, empty, i) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kSelBatch; ++j) {
            const bool in = kk[j] != 0ull && (kk[j] & pmask) == prefix;
            const unsigned digit = in ? (unsigned)(kk[j] >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, digit);
            if (in && lane == __ffs(peers) - 1) s_w[wid][digit] += (unsigned)__popc(peers);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kSelThreads) {
        unsigned t = 0u;
        for (int w = 0; w < kSelThreads / 32; ++w) t += s_w[w][d];
        if (t) atomicAdd(&st->hist[d], t);
    }
}

// the digit at which the count from the top reaches the rank still wanted
// (the first pass also fixes m and take); clears the counts for the next pass
__global__ void k_sel_pick(SelState* st, int shift, long long budget, int first)
{
    __shared__ int s_skip;
    if (threadIdx.x == 0) {
        s_skip = st->done;
        if (first) {
            long long m = 0;
            for (int d = 0; d < 256; ++d) m += st->hist[d];
            const long long take = budget < m ? budget : m;
            st->m = m;
            st->take = take;
            st->rank = take;
            if (take == m || take == 0) st->done = s_skip = 1;
        }
        if (!s_skip) {
            const long long rank = st->rank;
            long long above = 0;
            int d = 255;
            for (; d > 0; --d) {
                if (above + (long long)st->hist[d] >= rank) break;
                above += st->hist[d];
            }
            st->prefix |= (unsigned long long)d << shift;
            st->pmask |= 255ull << shift;
            st->rank = rank - above;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) st->hist[i] = 0u;
}

// keys equal to the threshold V (= the chosen prefix) in each CTA's range
__global__ void __launch_bounds__(kSelThreads) k_sel_ties(const unsigned long long* __restrict__ fkey,
                                                          const uint8_t* __restrict__ empty, int nb,
                                                          SelState* __restrict__ st, int chunk)
{
    __shared__ unsigned s[32];
    __shared__ unsigned s_tot;
    if (st->done) return;
    const unsigned long long V = st->prefix;
    const int lo = blockIdx.x * chunk, hi = min(nb, lo + chunk);
    unsigned n = 0u;
    for (int i = lo + (int)threadIdx.x; i < hi; i += kSelThreads) n += sel_key1(fkey, empty, i) == V ? 1u : 0u;
    n = block_count(n, s, &s_tot);
    if (threadIdx.x == 0) st->ties[blockIdx.x] = n;
}

// the brick set: keys above V, and the first `need` keys equal to V in brick
// order (their rank: the ties of earlier CTAs, earlier rounds, warps, lanes)
__global__ void __launch_bounds__(kSelThreads) k_sel_assign(const unsigned long long* __restrict__ fkey,
                                                            const uint8_t* __restrict__ empty, int nb,
                                                            const SelState* __restrict__ st, int chunk,
                                                            uint8_t* __restrict__ active,
                                                            long long* __restrict__ counts)
{
    __shared__ unsigned s_w[32];
    __shared__ long long s_base;
    const int lo = blockIdx.x * chunk, hi = min(nb, lo + chunk);
    if (blockIdx.x == 0 && threadIdx.x == 0) { counts[0] = st->m; counts[1] = st->take; }
    if (st->done) {
        const bool all = st->take > 0;
        for (int i = lo + (int)threadIdx.x; i < hi; i += kSelThreads) active[i] = (all && !empty[i]) ? 1 : 0;
        return;
    }
    const unsigned long long V = st->prefix;
    const long long need = st->rank;
    if (threadIdx.x == 0) {
        long long b = 0;
        for (int c = 0; c < (int)blockIdx.x; ++c) b += st->ties[c];
        s_base = b;
    }
    __syncthreads();
    long long run = s_base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = lo; base < hi; base += kSelThreads) {
        const int i = base + (int)threadIdx.x;
        const unsigned long long k = i < hi ? sel_key1(fkey, empty, i) : 0ull;
        const bool eq = k != 0ull && k == V;
        const unsigned bal = __ballot_sync(0xffffffffu, eq);
        if (lane == 0) s_w[w] = (unsigned)__popc(bal);
        __syncthreads();
        long long mine = run + __popc(bal & ((1u << lane) - 1u));
        unsigned tot = 0u;
        for (int q = 0; q < kSelThreads / 32; ++q) {
            if (q < w) mine += s_w[q];
            tot += s_w[q];
        }
        if (i < hi) active[i] = (k != 0ull && (k > V || (eq && mine < need))) ? 1 : 0;
        run += tot;
        __syncthreads();
    }
}

// the brick selection: k_select up to 4096 bricks (keys in registers), the
// grid-wide passes above; st is scratch for the latter, sms the SM count
vdbc_status launch_select(const unsigned long long* fkey, const uint8_t* empty, int nb, long long budget,
                          uint8_t* active, long long* counts, SelState* st, int sms, cudaStream_t s)
{
    if (nb <= kSelCache * kSelThreads) {
        KLAUNCH(k_select<<<1, kSelThreads, 0, s>>>(fkey, empty, nb, budget, active, counts));
        return VDBC_OK;
    }
    const int ctas = std::min(kSelMaxCtas, std::min(2 * std::max(1, sms), (nb + kSelThreads - 1) / kSelThreads));
    const int chunk = (nb + ctas - 1) / ctas;
    KLAUNCH(k_sel_init<<<1, 256, 0, s>>>(st));
    for (int p = 0; p < 8; ++p) {
        const int shift = 56 - 8 * p;
        KLAUNCH(k_sel_hist<<<ctas, kSelThreads, 0, s>>>(fkey, empty, nb, st, shift));
        KLAUNCH(k_sel_pick<<<1, 256, 0, s>>>(st, shift, budget, p == 0));
    }
    KLAUNCH(k_sel_ties<<<ctas, kSelThreads, 0, s>>>(fkey, empty, nb, st, chunk));
    KLAUNCH(k_sel_assign<<<ctas, kSelThreads, 0, s>>>(fkey, empty, nb, st, chunk, active, counts));
    VDBC_CUDA(cudaGetLastError());
    return VDBC_OK;
}

// ---------------------------------------------------------------- exclusive scan (u32)
constexpr int kScanBlock = 1024, kScanItems = 4;

__global__ void __launch_bounds__(kScanBlock) k_scan_sums(const uint32_t* __restrict__ in, long long n,
                                                          uint32_t* __restrict__ sums)
{
    __shared__ uint32_t s[32];
    __shared__ uint32_t s_tot;
    long long base = (long long)blockIdx.x * kScanBlock * kScanItems;
    uint32_t t = 0;
    for (int q = 0; q < kScanItems; ++q) {
        long long i = base + (long long)q * kScanBlock + threadIdx.x;
        if (i < n) t += in[i];
    }
    t = block_count(t, s, &s_tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_top(uint32_t* __restrict__ sums, int nblocks,
                                                         uint32_t* __restrict__ total)
{
    __shared__ uint32_t s[32];
    __shared__ uint32_t run;
    if (threadIdx.x == 0) run = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += kScanBlock) {
        int i = base + threadIdx.x;
        uint32_t x = i < nblocks ? sums[i] : 0;
        uint32_t incl = x;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s[w] = incl;
        __syncthreads();
        uint32_t wbase = 0;
        for (int q = 0; q < w; ++q) wbase += s[q];
        uint32_t r0 = run;
        if (i < nblocks) sums[i] = r0 + wbase + incl - x;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) run = r0 + wbase + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) total[0] = run;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_apply(const uint32_t* __restrict__ in, long long n,
                                                           const uint32_t* __restrict__ sums,
                                                           uint32_t* __restrict__ out)
{
    __shared__ uint32_t s[32];
    __shared__ uint32_t run;
    if (threadIdx.x == 0) run = sums[blockIdx.x];
    __syncthreads();
    long long base = (long long)blockIdx.x * kScanBlock * kScanItems;
    for (int q = 0; q < kScanItems; ++q) {
        long long i = base + (long long)q * kScanBlock + threadIdx.x;
        uint32_t x = i < n ? in[i] : 0;
        uint32_t incl = x;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s[w] = incl;
        __syncthreads();
        uint32_t wbase = 0;
        for (int qq = 0; qq < w; ++qq) wbase += s[qq];
        uint32_t r0 = run;
        if (i < n) out[i] = r0 + wbase + incl - x;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) run = r0 + wbase + incl;
        __syncthreads();
    }
}

// the whole scan in one CTA, for small n: each pass takes 4096 values, four
// consecutive ones per thread, and carries the running total to the next
constexpr long long kScanSingleMax = 16ll * kScanBlock * kScanItems;

__global__ void __launch_bounds__(kScanBlock) k_scan_single(const uint32_t* __restrict__ in, long long n,
                                                            uint32_t* __restrict__ out, uint32_t* __restrict__ total)
{
    __shared__ uint32_t s[32];
    __shared__ uint32_t run;
    if (threadIdx.x == 0) run = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long base = 0; base < n; base += (long long)kScanBlock * kScanItems) {
        const long long i0 = base + (long long)threadIdx.x * kScanItems;
        uint32_t x[kScanItems], t = 0;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            x[q] = i0 + q < n ? in[i0 + q] : 0u;
            t += x[q];
        }
        uint32_t incl = t;                      // inclusive scan of the threads' sums in the warp
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s[w] = incl;
        __syncthreads();
        uint32_t wbase = 0;
        for (int q = 0; q < w; ++q) wbase += s[q];
        const uint32_t r0 = run;
        uint32_t acc = r0 + wbase + incl - t;   // exclusive prefix of this thread's first value
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            if (i0 + q < n) out[i0 + q] = acc;
            acc += x[q];
        }
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) run = acc;
        __syncthreads();
    }
    if (threadIdx.x == 0) total[0] = run;
}

// exclusive scan of n u32 values; total written to total_dev[0]; tmp holds >= scan_tmp_words(n)
long long scan_blocks(long long n) { return (n + kScanBlock * kScanItems - 1) / (kScanBlock * kScanItems); }

void scan_exclusive(const uint32_t* in, uint32_t* out, long long n, uint32_t* tmp, uint32_t* total_dev,
                    cudaStream_t s)
{
    long long nb = scan_blocks(n);
    if (nb == 0) {
        cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s);
        return;
    }
    if (n <= kScanSingleMax) {
        KLAUNCH(k_scan_single<<<1, kScanBlock, 0, s>>>(in, n, out, total_dev));
        return;
    }
    KLAUNCH(k_scan_sums<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, tmp));
    KLAUNCH(k_scan_top<<<1, kScanBlock, 0, s>>>(tmp, (int)nb, total_dev));
    KLAUNCH(k_scan_apply<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, tmp, out));
}

// ---------------------------------------------------------------- tree build
__global__ void k_active_list(const uint8_t* __restrict__ active, const uint32_t* __restrict__ rank, int nb,
                              int* __restrict__ list)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb && active[i]) list[rank[i]] = i;
}

__global__ void k_u8_to_u32(const uint8_t* __restrict__ a, uint32_t* __restrict__ b, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

struct Cand {
    int li, lj, lk;       // leaf slot (voxel >> 3)
    int corner;           // -1 for a leaf of an active brick, 0/1 for a corner leaf
};

__device__ __forceinline__ Cand candidate(const Dims& d, const int* __restrict__ list, long long nact, long long c)
{
    Cand r;
    if (c < nact * 64) {
        int b = list[c >> 6];
        int local = (int)(c & 63);
        int bx, by, bz;
        brick_coords(d, b, bx, by, bz);
        r.li = bx * 4 + (local & 3);
        r.lj = by * 4 + ((local >> 2) & 3);
        r.lk = bz * 4 + (local >> 4);
        r.corner = -1;
    } else {
        r.corner = (int)(c - nact * 64);
        if (r.corner == 0) { r.li = 0; r.lj = 0; r.lk = 0; }
        else { r.li = (d.nx - 1) >> 3; r.lj = (d.ny - 1) >> 3; r.lk = (d.nz - 1) >> 3; }
    }
    return r;
}

// value n (x fastest in the 8^3 leaf) of the decoded grid inside candidate leaf `c`
__device__ __forceinline__ float cand_value(const float* __restrict__ v, const Dims& d, const Cand& c, int n,
                                            float B)
{
    int x = c.li * 8 + (n & 7), y = c.lj * 8 + ((n >> 3) & 7), z = c.lk * 8 + (n >> 6);
    if (x >= d.nx || y >= d.ny || z >= d.nz) return B;
    if (c.corner < 0) return __ldg(v + ((size_t)z * d.ny + y) * d.nx + x);
    bool at = (c.corner == 0) ? (x == 0 && y == 0 && z == 0)
                              : (x == d.nx - 1 && y == d.ny - 1 && z == d.nz - 1);
    return at ? __ldg(v + ((size_t)z * d.ny + y) * d.nx + x) : B;
}

// status: 0 background (or inside an active brick's leaf that already holds the
// corner), 1 constant non-background (a tile after prune), 2 a leaf
__global__ void k_leaf_status(const float* __restrict__ v, Dims d, const int* __restrict__ list,
                              const long long* __restrict__ counts, long long ncand_cap,
                              const uint8_t* __restrict__ active, const uint32_t* __restrict__ bsel,
                              uint32_t* __restrict__ is_leaf, uint32_t* __restrict__ is_tile,
                              float* __restrict__ tval, int* __restrict__ lowslot, int lx, int ly)
{
    long long nact = counts[1];
    long long ncand = nact * 64 + 2;
    long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= ncand_cap) return;
    if (c >= ncand) {   // unused capacity
        if (lane == 0) { is_leaf[c] = 0; is_tile[c] = 0; lowslot[c] = -1; }
        return;
    }
    float B = __uint_as_float(bsel[1]);
    Cand cd = candidate(d, list, nact, c);
    if (cd.corner >= 0) {
        int x = cd.corner == 0 ? 0 : d.nx - 1, y = cd.corner == 0 ? 0 : d.ny - 1, z = cd.corner == 0 ? 0 : d.nz - 1;
        int b = ((z >> 5) * d.by + (y >> 5)) * d.bx + (x >> 5);
        bool dup = active[b] || (cd.corner == 1 && d.nx <= 8 && d.ny <= 8 && d.nz <= 8);
        if (dup) {   // covered by an active brick, or the same leaf as corner 0
            if (lane == 0) { is_leaf[c] = 0; is_tile[c] = 0; lowslot[c] = -1; }
            return;
        }
    }
    uint32_t first = 0;
    bool same = true;
    if (cd.corner < 0) {
        // a leaf of an active brick: lane = x + 8 (y & 3), step r covers
        // y + 4 (r & 1), z = r >> 1; the 16 loads are in flight before any
        // is compared
        const int x = cd.li * 8 + (lane & 7), yb = cd.lj * 8 + (lane >> 3), zb = cd.lk * 8;
        const bool xv = x < d.nx;
        const size_t slice = (size_t)d.nx * d.ny;
        const float* p = v + ((size_t)zb * d.ny + yb) * d.nx + x;
        uint32_t u[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const bool in = xv && yb + 4 * (r & 1) < d.ny && zb + (r >> 1) < d.nz;
            u[r] = in ? __float_as_uint(__ldg(p + (size_t)(r >> 1) * slice + (size_t)((r & 1) * 4) * d.nx)) : bsel[1];
        }
        first = __shfl_sync(0xffffffffu, u[0], 0);
#pragma unroll
        for (int r = 0; r < 16; ++r) same &= (u[r] == first);
    } else {
#pragma unroll 4
        for (int r = 0; r < 16; ++r) {
            int n = lane + 32 * r;
            float val;
            if (cd.corner == 0 && d.nx <= 8 && d.ny <= 8 && d.nz <= 8) {
                // a single leaf holds both corners
                int x = n & 7, y = (n >> 3) & 7, z = n >> 6;
                bool at = (x == 0 && y == 0 && z == 0) || (x == d.nx - 1 && y == d.ny - 1 && z == d.nz - 1);
                val = (x < d.nx && y < d.ny && z < d.nz && at) ? __ldg(v + ((size_t)z * d.ny + y) * d.nx + x) : B;
            } else {
                val = cand_value(v, d, cd, n, B);
            }
            uint32_t u = __float_as_uint(val);
            if (r == 0) first = __shfl_sync(0xffffffffu, u, 0);
            same &= (u == first);
        }
    }
    bool constant = __all_sync(0xffffffffu, same);
    if (lane == 0) {
        uint32_t st;
        if (!constant) st = 2;
        else st = (first == bsel[1]) ? 0 : 1;
        is_leaf[c] = st == 2;
        is_tile[c] = st == 1;
        tval[c] = __uint_as_float(first);
        lowslot[c] = st ? (((cd.lk >> 4) * ly + (cd.lj >> 4)) * lx + (cd.li >> 4)) : -1;
    }
}

__global__ void k_mark_lower(const int* __restrict__ lowslot, long long ncand, uint32_t* __restrict__ lflag)
{
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncand && lowslot[c] >= 0) lflag[lowslot[c]] = 1;
}

__global__ void k_mark_root(const uint32_t* __restrict__ lflag, int nlow, int lx, int ly, int rx, int ry,
                            uint32_t* __restrict__ rflag)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nlow || !lflag[s]) return;
    int li = s % lx, lj = (s / lx) % ly, lk = s / (lx * ly);
    rflag[((lk >> 5) * ry + (lj >> 5)) * rx + (li >> 5)] = 1;
}

__global__ void k_fill_u32(uint32_t* __restrict__ p, long long n, uint32_t value)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = value;
}

__global__ void k_fill_root(uint32_t* __restrict__ root, const uint32_t* __restrict__ rflag,
                            const uint32_t* __restrict__ rrank, int nroot)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nroot) root[s] = rflag[s] ? rrank[s] : kBackgroundEntry;
}

__global__ void k_fill_upper(uint32_t* __restrict__ upper, const uint32_t* __restrict__ lflag,
                             const uint32_t* __restrict__ lrank, const uint32_t* __restrict__ rrank, int nlow,
                             int lx, int ly, int rx, int ry)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nlow || !lflag[s]) return;
    int li = s % lx, lj = (s / lx) % ly, lk = s / (lx * ly);
    uint32_t u = rrank[((lk >> 5) * ry + (lj >> 5)) * rx + (li >> 5)];
    upper[(size_t)u * kUpperN + ((lk & 31) << 10) + ((lj & 31) << 5) + (li & 31)] = lrank[s];
}

__global__ void k_fill_lower(uint32_t* __restrict__ lower, float* __restrict__ tiles, Dims d,
                             const int* __restrict__ list, const long long* __restrict__ counts,
                             const int* __restrict__ lowslot, const uint32_t* __restrict__ is_leaf,
                             const uint32_t* __restrict__ leaf_rank, const uint32_t* __restrict__ tile_rank,
                             const float* __restrict__ tval, const uint32_t* __restrict__ lrank,
                             const uint32_t* __restrict__ bsel)
{
    long long nact = counts[1];
    long long ncand = nact * 64 + 2;
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) tiles[0] = __uint_as_float(bsel[1]);
    if (c >= ncand || lowslot[c] < 0) return;
    Cand cd = candidate(d, list, nact, c);
    uint32_t entry;
    if (is_leaf[c]) entry = leaf_rank[c];
    else {
        uint32_t t = 1 + tile_rank[c];
        tiles[t] = tval[c];
        entry = kTile | t;
    }
    lower[(size_t)lrank[lowslot[c]] * kLowerN + ((cd.lk & 15) << 8) + ((cd.lj & 15) << 4) + (cd.li & 15)] = entry;
}

// payload of every leaf: a copy (FP32) or the per-leaf quantized codes
__global__ void k_fill_leaves(const float* __restrict__ v, Dims d, const int* __restrict__ list,
                              const long long* __restrict__ counts, const uint32_t* __restrict__ is_leaf,
                              const uint32_t* __restrict__ leaf_rank, const uint32_t* __restrict__ bsel,
                              int payload, void* __restrict__ leaves, float2* __restrict__ meta)
{
    long long nact = counts[1];
    long long ncand = nact * 64 + 2;
    long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= ncand || !is_leaf[c]) return;
    float B = __uint_as_float(bsel[1]);
    Cand cd = candidate(d, list, nact, c);
    bool both = cd.corner == 0 && d.nx <= 8 && d.ny <= 8 && d.nz <= 8;
    float vals[16];
    uint32_t kmin = 0xffffffffu, kmax = 0;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        int n = lane + 32 * r;
        float val;
        if (both) {
            int x = n & 7, y = (n >> 3) & 7, z = n >> 6;
            bool at = (x == 0 && y == 0 && z == 0) || (x == d.nx - 1 && y == d.ny - 1 && z == d.nz - 1);
            val = (x < d.nx && y < d.ny && z < d.nz && at) ? __ldg(v + ((size_t)z * d.ny + y) * d.nx + x) : B;
        } else {
            val = cand_value(v, d, cd, n, B);
        }
        vals[r] = val;
        uint32_t k = okey(__float_as_uint(val));
        kmin = min(kmin, k);
        kmax = max(kmax, k);
    }
    size_t base = (size_t)leaf_rank[c] * kLeafN;
    if (payload == VDBC_FP32) {
        float* out = reinterpret_cast<float*>(leaves) + base;
#pragma unroll
        for (int r = 0; r < 16; ++r) out[lane + 32 * r] = vals[r];
        return;
    }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    float off = __uint_as_float(okey_inv(kmin));
    float scale = __fsub_rn(__uint_as_float(okey_inv(kmax)), off);
    if (lane == 0) meta[leaf_rank[c]] = make_float2(scale, off);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        float t = scale != 0.0f ? __fdiv_rn(__fsub_rn(vals[r], off), scale) : 0.0f;
        int n = lane + 32 * r;
        if (payload == VDBC_FP16) {
            reinterpret_cast<__half*>(leaves)[base + n] = __float2half_rn(t);
        } else {
            reinterpret_cast<uint8_t*>(leaves)[base + n] =
                (uint8_t)__nv_cvt_float_to_fp8(t, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// ---------------------------------------------------------------- macrocells
// min/max of the decoded grid over each macrocell's voxels dilated by one
// voxel (Section 4: the majorant ranges); kGroup threads per macrocell (a warp
// for small cells, a whole block for large ones)
template <int kGroup>
__device__ __forceinline__ bool group_all(bool p, int* s_flag)
{
    if constexpr (kGroup == 32) {
        return __all_sync(0xffffffffu, p);
    } else {
        __syncthreads();
        if (threadIdx.x == 0) *s_flag = 1;
        __syncthreads();
        if (!p) *s_flag = 0;
        __syncthreads();
        return *s_flag != 0;
    }
}

template <int kGroup>
__global__ void __launch_bounds__(kGroup == 32 ? 256 : kGroup)
    k_macrocells(GridView g, float* __restrict__ mcmin, float* __restrict__ mcmax, long long ncell)
{
    __shared__ int s_flag;
    __shared__ float s_lo[kGroup / 32], s_hi[kGroup / 32];
    long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kGroup;
    int lane = threadIdx.x % kGroup;
    if (kGroup == 32 && c >= ncell) return;     // a whole warp; block groups have one cell per block
    int cx = (int)(c % g.mx), cy = (int)((c / g.mx) % g.my), cz = (int)(c / ((long long)g.mx * g.my));
    int x0 = max(cx * g.mc - 1, 0), x1 = min(cx * g.mc + g.mc, g.nx - 1);
    int y0 = max(cy * g.mc - 1, 0), y1 = min(cy * g.mc + g.mc, g.ny - 1);
    int z0 = max(cz * g.mc - 1, 0), z1 = min(cz * g.mc + g.mc, g.nz - 1);
    // leaf slots under the box: if all are tiles, the answer is the min/max of their values
    int lx0 = x0 >> 3, lx1 = x1 >> 3, ly0 = y0 >> 3, ly1 = y1 >> 3, lz0 = z0 >> 3, lz1 = z1 >> 3;
    int nl = (lx1 - lx0 + 1) * (ly1 - ly0 + 1) * (lz1 - lz0 + 1);
    float vmin = INFINITY, vmax = -INFINITY;
    bool all_tiles = true;
    for (int q = lane; q < nl; q += kGroup) {
        int a = lx0 + q % (lx1 - lx0 + 1);
        int b = ly0 + (q / (lx1 - lx0 + 1)) % (ly1 - ly0 + 1);
        int e = lz0 + q / ((lx1 - lx0 + 1) * (ly1 - ly0 + 1));
        uint32_t en = descend_to_leaf(g, a, b, e);
        if (en & kTile) {
            float t = __ldg(g.tiles + (en & ~kTile));
            vmin = fminf(vmin, t);
            vmax = fmaxf(vmax, t);
        } else {
            all_tiles = false;
        }
    }
    if (!group_all<kGroup>(all_tiles, &s_flag)) {
        Accessor acc;
        acc.reset();
        int ex = x1 - x0 + 1, ey = y1 - y0 + 1, ez = z1 - z0 + 1;
        int n = ex * ey * ez;
        for (int q = lane; q < n; q += kGroup) {
            int x = x0 + q % ex, y = y0 + (q / ex) % ey, z = z0 + q / (ex * ey);
            float val = voxel(g, acc, x, y, z);
            vmin = fminf(vmin, val);
            vmax = fmaxf(vmax, val);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if constexpr (kGroup > 32) {
        if ((threadIdx.x & 31) == 0) { s_lo[threadIdx.x >> 5] = vmin; s_hi[threadIdx.x >> 5] = vmax; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kGroup / 32; ++w) { vmin = fminf(vmin, s_lo[w]); vmax = fmaxf(vmax, s_hi[w]); }
        }
    }
    if (lane == 0) { mcmin[c] = vmin; mcmax[c] = vmax; }
}

// Macrocell ranges of an FP32 grid straight from the input: the decoded grid
// is V in the activated bricks and at the two corner voxels and B elsewhere
// (its definition), so no tree descent is needed.  One block per macrocell:
// a thread per brick that the dilated box overlaps (at most 4 per axis) sorts
// it out, an inactive brick adding B (when its part of the box holds a voxel
// other than a corner) and an active one its part to a list; then the whole
// block reads the listed parts, eight rows in flight per warp, and a corner
// inside the box adds its own value.  Same values, same ranges as
// k_macrocells on the tree; the input is read only where a brick is active.
constexpr int kMcInThreads = 512;
__global__ void __launch_bounds__(kMcInThreads) k_macrocells_input(const float* __restrict__ v, Dims d,
                                                                   const uint8_t* __restrict__ active,
                                                                   const uint32_t* __restrict__ lo_key,
                                                                   const uint32_t* __restrict__ hi_key,
                                                                   const uint32_t* __restrict__ bsel, int mc, int mx,
                                                                   int my, float* __restrict__ mcmin,
                                                                   float* __restrict__ mcmax)
{
    // a cell of at most kMaxMacrocell voxels, dilated by one, overlaps at most
    // six bricks along an axis
    constexpr int kW = kMcInThreads / 32, kMaxParts = 216;
    static_assert(kMaxMacrocell <= 128 && kMaxParts <= kMcInThreads, "one thread per overlapped brick");
    __shared__ float s_lo[kW], s_hi[kW];
    __shared__ int s_part[kMaxParts][4];       // x0, width, y0 | z0 << 16, ey | ez << 16
    __shared__ int s_nparts, s_hasB;
    const long long c = blockIdx.x;
    const int cx = (int)(c % mx), cy = (int)((c / mx) % my), cz = (int)(c / ((long long)mx * my));
    const int x0 = max(cx * mc - 1, 0), x1 = min(cx * mc + mc, d.nx - 1);
    const int y0 = max(cy * mc - 1, 0), y1 = min(cy * mc + mc, d.ny - 1);
    const int z0 = max(cz * mc - 1, 0), z1 = min(cz * mc + mc, d.nz - 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) { s_nparts = 0; s_hasB = 0; }
    __syncthreads();
    const int nbx = (x1 >> 5) - (x0 >> 5) + 1, nby = (y1 >> 5) - (y0 >> 5) + 1, nbz = (z1 >> 5) - (z0 >> 5) + 1;
    float bmin = INFINITY, bmax = -INFINITY;   // ranges of the whole active bricks this thread lists
    if ((int)threadIdx.x < nbx * nby * nbz) {
        const int t = threadIdx.x;
        const int bx = (x0 >> 5) + t % nbx, by = (y0 >> 5) + (t / nbx) % nby, bz = (z0 >> 5) + t / (nbx * nby);
        const int ax0 = max(x0, bx * 32), ax1 = min(x1, bx * 32 + 31);
        const int ay0 = max(y0, by * 32), ay1 = min(y1, by * 32 + 31);
        const int az0 = max(z0, bz * 32), az1 = min(z1, bz * 32 + 31);
        const size_t bi = ((size_t)bz * d.by + by) * d.bx + bx;
        if (__ldg(active + bi) && ax0 == bx * 32 && ay0 == by * 32 && az0 == bz * 32 &&
            ax1 == min(bx * 32 + 31, d.nx - 1) && ay1 == min(by * 32 + 31, d.ny - 1) && az1 == min(bz * 32 + 31, d.nz - 1)) {
            // the whole brick: its range from pass 1 (the exact min and max of
            // its voxels in the total order), no voxel read
            bmin = __uint_as_float(okey_inv(__ldg(lo_key + bi)));
            bmax = __uint_as_float(okey_inv(__ldg(hi_key + bi)));
        } else if (__ldg(active + bi)) {
            const int i = atomicAdd(&s_nparts, 1);
            s_part[i][0] = ax0;
            s_part[i][1] = ax1 - ax0 + 1;
            s_part[i][2] = ay0 | (az0 << 16);
            s_part[i][3] = (ay1 - ay0 + 1) | ((az1 - az0 + 1) << 16);
        } else {
            const bool one_voxel = d.nx == 1 && d.ny == 1 && d.nz == 1;     // both corners are voxel 0
            const bool c0 = ax0 == 0 && ay0 == 0 && az0 == 0;
            const bool c1 = ax1 == d.nx - 1 && ay1 == d.ny - 1 && az1 == d.nz - 1;
            const long long corners = (long long)c0 + (long long)(c1 && !(c0 && one_voxel));
            if ((long long)(ax1 - ax0 + 1) * (ay1 - ay0 + 1) * (az1 - az0 + 1) > corners) s_hasB = 1;
        }
    }
    __syncthreads();
    float vmin = bmin, vmax = bmax;
    if (threadIdx.x == 0) {
        if (s_hasB) { const float B = __uint_as_float(bsel[1]); vmin = B; vmax = B; }
        if (x0 == 0 && y0 == 0 && z0 == 0) { vmin = fminf(vmin, __ldg(v)); vmax = fmaxf(vmax, __ldg(v)); }
        if (x1 == d.nx - 1 && y1 == d.ny - 1 && z1 == d.nz - 1) {
            const float t = __ldg(v + ((size_t)d.nz * d.ny * d.nx - 1));
            vmin = fminf(vmin, t);
            vmax = fmaxf(vmax, t);
        }
    }
    const int nparts = s_nparts;
    const size_t slice = (size_t)d.nx * d.ny;
    for (int i = 0; i < nparts; ++i) {
        const int ax0 = s_part[i][0], ex = s_part[i][1];
        const int ay0 = s_part[i][2] & 0xffff, az0 = s_part[i][2] >> 16;
        const int ey = s_part[i][3] & 0xffff, ez = s_part[i][3] >> 16;
        // a warp task: row y of the part over U consecutive z slices, the
        // row pointer stepping one slice a load (no index products per row);
        // lanes past the part's width read its last column again, which
        // changes neither extreme
        constexpr int U = 8;
        const int nzc = (ez + U - 1) / U;
        const uint32_t mey = div_magic(ey);
        for (int t = warp; t < ey * nzc; t += kW) {
            const int zc = div_small(t, mey), y = t - zc * ey;
            const int nz = min(U, ez - zc * U);
            const float* p = v + ((size_t)(az0 + zc * U) * d.ny + (ay0 + y)) * d.nx + ax0 + min(lane, ex - 1);
            float t8[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                t8[q] = q < nz ? __ldg(p) : t8[0];
                p += slice;
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                vmin = fminf(vmin, t8[q]);
                vmax = fmaxf(vmax, t8[q]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if (lane == 0) { s_lo[warp] = vmin; s_hi[warp] = vmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kW; ++w) { vmin = fminf(vmin, s_lo[w]); vmax = fmaxf(vmax, s_hi[w]); }
        mcmin[c] = vmin;
        mcmax[c] = vmax;
    }
}

// full decode, one thread per voxel (tests and the decode entry point)
__global__ void k_decode(GridView g, float* __restrict__ out, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((long long)g.nx * g.ny));
        Accessor acc;
        acc.reset();
        out[i] = voxel(g, acc, x, y, z);
    }
}

// k_pass1's 128 KB of shared memory needs an opt-in, once per device
// every row of the volume starts on a 16-byte boundary: the float4 passes apply
bool rows_aligned(const float* v, const Dims& d)
{
    return d.nx % 4 == 0 && (reinterpret_cast<uintptr_t>(v) & 15u) == 0;
}

// the background B (Algorithm 1's histogram, both levels) and the brick
// ranges, into bsel and lo_key / hi_key: the candidate and its exact count
// with the ranges, then the histogram passes, which stand aside when the
// candidate holds the majority.  hist and *nonfinite are zero on entry.
// (VDBC_MAJORITY=0 leaves the histogram to every volume, for measurement;
// VDBC_PASS1_MODE picks the row loads of the histogram pass for rows off a
// 16-byte boundary: 3 (the default) steps each warp's brick row through
// 16 z slices, 2 through 8, 0 splits the row index per row -- the full-scale
// cloud encoded in 19.6, 20.1 and 23.7 ms that way before the shortcut)
vdbc_status launch_background(const float* v, const Dims& d, int nb, unsigned grid, uint32_t* lo_key,
                              uint32_t* hi_key, unsigned long long* hist, uint32_t* bsel, int* nonfinite, Majority* maj,
                              cudaStream_t s)
{
    static const int mode = [] { const char* e = std::getenv("VDBC_PASS1_MODE"); return e ? std::atoi(e) : 3; }();
    static const bool shortcut = [] { const char* e = std::getenv("VDBC_MAJORITY"); return !(e && e[0] == '0'); }();
    const long long nvox = (long long)d.nx * d.ny * d.nz;
    const bool aligned = rows_aligned(v, d);
    const Majority* m = shortcut ? maj : nullptr;
    if (shortcut) {
        VDBC_CUDA(cudaMemsetAsync(lo_key, 0xff, (size_t)nb * 4, s));     // min / max identities
        VDBC_CUDA(cudaMemsetAsync(hi_key, 0, (size_t)nb * 4, s));
        KLAUNCH(k_candidate<<<1, 1024, 0, s>>>(v, d, maj));
        if (aligned)
            KLAUNCH(k_pass1_maj<1><<<grid, kPass1Threads, 0, s>>>(v, d, nb, lo_key, hi_key, maj, nonfinite));
        else
            KLAUNCH(k_pass1_maj<2><<<grid, kPass1Threads, 0, s>>>(v, d, nb, lo_key, hi_key, maj, nonfinite));
    }
    if (aligned)
        KLAUNCH(k_pass1<1><<<grid, kPass1Threads, kPass1Smem, s>>>(v, d, nb, lo_key, hi_key, hist, nonfinite, m, nvox));
    else if (mode == 2)
        KLAUNCH((k_pass1<2, 8><<<grid, kPass1Threads, kPass1Smem, s>>>(v, d, nb, lo_key, hi_key, hist, nonfinite, m,
                                                                       nvox)));
    else if (mode == 3)
        KLAUNCH((k_pass1<2, 16><<<grid, kPass1Threads, kPass1Smem, s>>>(v, d, nb, lo_key, hi_key, hist, nonfinite, m,
                                                                        nvox)));
    else
        KLAUNCH(k_pass1<0><<<grid, kPass1Threads, kPass1Smem, s>>>(v, d, nb, lo_key, hi_key, hist, nonfinite, m, nvox));
    KLAUNCH(k_argmax<<<1, 1024, 0, s>>>(hist, bsel, 0, m, nvox));
    VDBC_CUDA(cudaMemsetAsync(hist, 0, 65536 * sizeof(unsigned long long), s));
    const unsigned p2grid = (unsigned)std::min<long long>(nb, (long long)grid * 8);   // (grid: one block per SM)
    if (aligned)
        KLAUNCH(k_pass2<true><<<p2grid, kPassThreads, 0, s>>>(v, d, lo_key, hi_key, bsel, hist, m, nvox, nb));
    else
        KLAUNCH(k_pass2<false><<<p2grid, kPassThreads, 0, s>>>(v, d, lo_key, hi_key, bsel, hist, m, nvox, nb));
    KLAUNCH(k_argmax<<<1, 1024, 0, s>>>(hist, bsel, 1, m, nvox));
    return VDBC_OK;
}

// opts k_pass1 into its shared memory (once per device) and sizes its
// persistent grid: the resident blocks of the device, at most one per brick
vdbc_status pass1_setup(int nbricks, unsigned* grid)
{
    static std::mutex mu;
    static std::vector<std::pair<int, int>> done;     // (device, resident blocks)
    int dev = 0;
    VDBC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    int resident = 0;
    for (const auto& e : done)
        if (e.first == dev) resident = e.second;
    if (resident == 0) {
        VDBC_CUDA(cudaFuncSetAttribute(k_pass1<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPass1Smem));
        VDBC_CUDA(cudaFuncSetAttribute(k_pass1<2, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPass1Smem));
        VDBC_CUDA(cudaFuncSetAttribute(k_pass1<2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPass1Smem));
        VDBC_CUDA(cudaFuncSetAttribute(k_pass1<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPass1Smem));
        int per_sm = 0, sms = 0;
        VDBC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass1<0>, kPass1Threads, kPass1Smem));
        VDBC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        resident = std::max(1, per_sm) * std::max(1, sms);
        done.emplace_back(dev, resident);
    }
    *grid = (unsigned)std::max(1, std::min(nbricks, resident));
    return VDBC_OK;
}

unsigned grid1d(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int64_t brick_bytes(int payload)
{
    if (payload == VDBC_FP16) return 32768 * 2 + 64 * 8;
    if (payload == VDBC_FP8) return 32768 * 1 + 64 * 8;
    return 32768 * 4;
}

static int payload_elem(int payload)
{
    return payload == VDBC_FP32 ? 4 : (payload == VDBC_FP8 ? 1 : 2);   // learned fallbacks are FP16
}

void bind_view(vdbc_grid* g)
{
    GridView& v = g->view;
    const vdbc_grid_info& in = g->info;
    char* base = static_cast<char*>(g->block);
    v.nx = in.dims[0]; v.ny = in.dims[1]; v.nz = in.dims[2];
    v.rx = (v.nx + 4095) / 4096; v.ry = (v.ny + 4095) / 4096; v.rz = (v.nz + 4095) / 4096;
    v.payload = in.payload;
    v.mc = in.macrocell;
    v.mx = (v.nx + v.mc - 1) / v.mc; v.my = (v.ny + v.mc - 1) / v.mc; v.mz = (v.nz + v.mc - 1) / v.mc;
    int m = std::max(v.nx, std::max(v.ny, v.nz));
    v.inv_m = 1.0f / (float)m;
    v.root = reinterpret_cast<const uint32_t*>(base + g->off_root);
    v.upper = reinterpret_cast<const uint32_t*>(base + g->off_upper);
    v.lower = reinterpret_cast<const uint32_t*>(base + g->off_lower);
    v.tiles = reinterpret_cast<const float*>(base + g->off_tiles);
    v.leaves = base + g->off_leaves;
    v.meta = reinterpret_cast<const float2*>(base + g->off_meta);
    v.mcmin = reinterpret_cast<const float*>(base + g->off_mcmin);
    v.mcmax = reinterpret_cast<const float*>(base + g->off_mcmax);
    v.latents = reinterpret_cast<const uint32_t*>(base + g->off_latents);
    v.nmeta = reinterpret_cast<const float2*>(base + g->off_nmeta);
    v.mlp_frag = reinterpret_cast<const uint2*>(base + g->off_frag);
    v.mlp_bias = reinterpret_cast<const float*>(base + g->off_bias);
#if VDBC_CHECKED
    v.n_upper = (uint32_t)in.n_upper;
    v.n_lower = (uint32_t)in.n_lower;
    v.n_tiles = (uint32_t)in.n_tiles;
    v.n_leaves = (uint32_t)in.n_leaves;
    v.n_neural = (uint32_t)in.n_neural;
    v.err = &g->stats->error_flags;   // the grid's stats exist before its view is bound
#endif
}

// offsets of every table inside the one linear block, from the counts in g->info
void layout(vdbc_grid* g)
{
    vdbc_grid_info& in = g->info;
    long long rx = (in.dims[0] + 4095) / 4096, ry = (in.dims[1] + 4095) / 4096, rz = (in.dims[2] + 4095) / 4096;
    long long mc = in.macrocell;
    long long ncell = ((in.dims[0] + mc - 1) / mc) * ((in.dims[1] + mc - 1) / mc) * ((in.dims[2] + mc - 1) / mc);
    size_t off = 0;
    g->off_root = off;   off = align256(off + (size_t)(rx * ry * rz) * 4);
    g->off_upper = off;  off = align256(off + (size_t)in.n_upper * kUpperN * 4);
    g->off_lower = off;  off = align256(off + (size_t)in.n_lower * kLowerN * 4);
    g->off_tiles = off;  off = align256(off + (size_t)in.n_tiles * 4);
    g->off_leaves = off; off = align256(off + (size_t)in.n_leaves * kLeafN * payload_elem(in.payload));
    g->off_meta = off;   off = align256(off + (in.payload != VDBC_FP32 ? (size_t)in.n_leaves * 8 : 0));
    g->off_mcmin = off;  off = align256(off + (size_t)ncell * 4);
    g->off_mcmax = off;  off = align256(off + (size_t)ncell * 4);
    const bool learned = in.payload == VDBC_LEARNED;
    const size_t nn = learned ? (size_t)in.n_neural : 0;
    g->off_latents = off; off = align256(off + nn * 16 * 2);
    g->off_nmeta = off;   off = align256(off + nn * 8);
    g->off_frag = off;    off = align256(off + (learned ? (size_t)18 * 32 * 8 : 0));
    g->off_bias = off;    off = align256(off + (learned ? (size_t)65 * 4 : 0));
    g->off_params = off;  off = align256(off + (learned ? (size_t)1729 * 4 : 0));
    g->block_bytes = off;
    in.payload_bytes = (uint64_t)in.n_leaves * kLeafN * payload_elem(in.payload) +
                       (in.payload != VDBC_FP32 ? (uint64_t)in.n_leaves * 8 : 0) +
                       (learned ? (uint64_t)nn * (32 + 8) + 18 * 32 * 8 + 65 * 4 : 0);
    in.node_bytes = (uint64_t)(rx * ry * rz) * 4 + (uint64_t)in.n_upper * kUpperN * 4 +
                    (uint64_t)in.n_lower * kLowerN * 4 + (uint64_t)in.n_tiles * 4;
    in.total_bytes = off;
}

vdbc_status macrocells_of_view(const GridView& v, float* mcmin, float* mcmax, cudaStream_t s)
{
    long long ncell = (long long)v.mx * v.my * v.mz;
    const long long dil = (long long)(v.mc + 2) * (v.mc + 2) * (v.mc + 2);
    if (dil > 4096)
        KLAUNCH(k_macrocells<256><<<(unsigned)ncell, 256, 0, s>>>(v, mcmin, mcmax, ncell));
    else
        KLAUNCH(k_macrocells<32><<<grid1d(ncell * 32, 256), 256, 0, s>>>(v, mcmin, mcmax, ncell));
    VDBC_CUDA(cudaGetLastError());
    return VDBC_OK;
}

vdbc_status build_macrocells(vdbc_grid* g, cudaStream_t s)
{
    if (g->info.payload == VDBC_LEARNED) return build_learned_macrocells(g, s);
    char* base = static_cast<char*>(g->block);
    return macrocells_of_view(g->view, reinterpret_cast<float*>(base + g->off_mcmin),
                              reinterpret_cast<float*>(base + g->off_mcmax), s);
}

void decode_view(const GridView& v, float* out, long long n, cudaStream_t s)
{
    KLAUNCH(k_decode<<<grid1d(std::min<long long>(n, 152LL * 2048), 256), 256, 0, s>>>(v, out, n));
}

long long scan_tmp_words(long long n) { return scan_blocks(n) + 1; }

void scan_u32(const uint32_t* in, uint32_t* out, long long n, uint32_t* tmp, uint32_t* total_dev, cudaStream_t s)
{
    scan_exclusive(in, out, n, tmp, total_dev, s);
}

void select_largest(const unsigned long long* key, const uint8_t* skip, int n, long long budget, uint8_t* chosen,
                    long long* counts, cudaStream_t s)
{
    KLAUNCH(k_select<<<1, 1024, 0, s>>>(key, skip, n, budget, chosen, counts));
}

}  // namespace vdbc

using namespace vdbc;

namespace {
// scratch allocations of one encode call, released on every exit path
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
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
    ~Scratch()
    {
        for (void* q : ptrs) dev_free(q, s);
    }
};
}  // namespace

extern "C" vdbc_status vdbc_encode(const vdbc_dense* in, const vdbc_encode_params* params, void* stream,
                                   vdbc_grid** out)
{
    clear_error();
    if (!in || !params || !out || !in->data) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_encode: null argument");
    *out = nullptr;
    for (int a = 0; a < 3; ++a)
        if (in->dims[a] < 1 || in->dims[a] > kMaxDim)
            return set_error(VDBC_ERR_INVALID_ARG, "vdbc_encode: dims[%d]=%d outside 1..%d", a, in->dims[a], kMaxDim);
    double ratio = params->ratio;
    if (!(ratio >= 1.0) || !std::isfinite(ratio))
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_encode: ratio must be a finite value >= 1");
    int metric = params->metric == 0 ? VDBC_F2 : params->metric;
    if (metric < VDBC_F1 || metric > VDBC_F3) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_encode: unknown metric %d", metric);
    int payload = params->payload;
    if (payload < VDBC_FP32 || payload > VDBC_FP8)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_encode: unknown payload %d", payload);
    int mc = params->macrocell == 0 ? 8 : params->macrocell;
    if (mc < 1 || mc > kMaxMacrocell)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_encode: macrocell %d outside 1..%d", mc, kMaxMacrocell);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc(s);
    Dims d;
    d.nx = in->dims[0]; d.ny = in->dims[1]; d.nz = in->dims[2];
    d.bx = (d.nx + 31) / 32; d.by = (d.ny + 31) / 32; d.bz = (d.nz + 31) / 32;
    const long long nvox = (long long)d.nx * d.ny * d.nz;
    const int nb = d.bx * d.by * d.bz;

    const float* vol = in->data;
    if (!in->on_device) {
        float* dv = nullptr;
        VDBC_TRY(sc.get(&dv, (size_t)nvox));
        VDBC_CUDA(cudaMemcpyAsync(dv, in->data, (size_t)nvox * 4, cudaMemcpyHostToDevice, s));
        vol = dv;
    }
    uint32_t *lo_key, *hi_key, *bsel, *scan_tmp, *total;
    unsigned long long *hist, *fkey;
    uint8_t *empty, *active;
    int *nonfinite, *list;
    long long* counts;
    VDBC_TRY(sc.get(&lo_key, nb));
    VDBC_TRY(sc.get(&hi_key, nb));
    VDBC_TRY(sc.get(&bsel, 2));
    VDBC_TRY(sc.get(&hist, 65536));
    VDBC_TRY(sc.get(&fkey, nb));
    VDBC_TRY(sc.get(&empty, nb));
    VDBC_TRY(sc.get(&active, nb));
    VDBC_TRY(sc.get(&nonfinite, 1));
    VDBC_TRY(sc.get(&counts, 2));
    VDBC_TRY(sc.get(&total, 8));
    Majority* maj = nullptr;
    VDBC_TRY(sc.get(&maj, 1));
    SelState* selst = nullptr;
    VDBC_TRY(sc.get(&selst, 1));

    // phase 1: histogram -> B (two levels), brick ranges
    VDBC_CUDA(cudaMemsetAsync(hist, 0, 65536 * 8, s));
    VDBC_CUDA(cudaMemsetAsync(nonfinite, 0, 4, s));
    unsigned p1grid = 1;
    VDBC_TRY(pass1_setup(nb, &p1grid));
    VDBC_TRY(launch_background(vol, d, nb, p1grid, lo_key, hi_key, hist, bsel, nonfinite, maj, s));
    // phase 2: f per brick, selection of N bricks
    KLAUNCH(k_scores<<<grid1d(nb, 256), 256, 0, s>>>(lo_key, hi_key, nb, bsel, metric, fkey, empty));
    double nbud = std::floor((double)nb * 131072.0 / (ratio * (double)brick_bytes(payload)));
    const long long budget = nbud > (double)nb ? (long long)nb : (long long)nbud;
    VDBC_TRY(launch_select(fkey, empty, nb, budget, active, counts, selst, (int)p1grid, s));

    // compact list of active bricks (x-fastest brick order)
    uint32_t *act32, *brank;
    VDBC_TRY(sc.get(&act32, nb));
    VDBC_TRY(sc.get(&brank, nb));
    long long tmp_words = std::max<long long>(scan_blocks(std::max<long long>(nb, (long long)budget * 64 + 2)) + 1, 1024);
    VDBC_TRY(sc.get(&scan_tmp, (size_t)tmp_words + 4096));
    KLAUNCH(k_u8_to_u32<<<grid1d(nb, 256), 256, 0, s>>>(active, act32, nb));
    scan_exclusive(act32, brank, nb, scan_tmp, total, s);
    VDBC_TRY(sc.get(&list, (size_t)std::max<long long>(std::min<long long>(budget, nb), 1)));
    KLAUNCH(k_active_list<<<grid1d(nb, 256), 256, 0, s>>>(active, brank, nb, list));

    // candidate leaves: 64 per active brick + the two corner leaves
    const long long cap = std::min<long long>(budget, nb) * 64 + 2;
    const int lx = (d.nx + 127) / 128, ly = (d.ny + 127) / 128, lz = (d.nz + 127) / 128;
    const int nlow = lx * ly * lz;
    const int rx = (d.nx + 4095) / 4096, ry = (d.ny + 4095) / 4096, rz = (d.nz + 4095) / 4096;
    const int nroot = rx * ry * rz;
    uint32_t *is_leaf, *is_tile, *leaf_rank, *tile_rank, *lflag, *lrank, *rflag, *rrank;
    float* tval;
    int* lowslot;
    VDBC_TRY(sc.get(&is_leaf, cap));
    VDBC_TRY(sc.get(&is_tile, cap));
    VDBC_TRY(sc.get(&leaf_rank, cap));
    VDBC_TRY(sc.get(&tile_rank, cap));
    VDBC_TRY(sc.get(&tval, cap));
    VDBC_TRY(sc.get(&lowslot, cap));
    VDBC_TRY(sc.get(&lflag, nlow));
    VDBC_TRY(sc.get(&lrank, nlow));
    VDBC_TRY(sc.get(&rflag, nroot));
    VDBC_TRY(sc.get(&rrank, nroot));
    KLAUNCH(k_leaf_status<<<grid1d(cap * 32, 256), 256, 0, s>>>(vol, d, list, counts, cap, active, bsel, is_leaf, is_tile,
                                                         tval, lowslot, lx, ly));
    scan_exclusive(is_leaf, leaf_rank, cap, scan_tmp, total + 1, s);
    scan_exclusive(is_tile, tile_rank, cap, scan_tmp, total + 2, s);
    VDBC_CUDA(cudaMemsetAsync(lflag, 0, (size_t)nlow * 4, s));
    VDBC_CUDA(cudaMemsetAsync(rflag, 0, (size_t)nroot * 4, s));
    KLAUNCH(k_mark_lower<<<grid1d(cap, 256), 256, 0, s>>>(lowslot, cap, lflag));
    scan_exclusive(lflag, lrank, nlow, scan_tmp, total + 3, s);
    KLAUNCH(k_mark_root<<<grid1d(nlow, 256), 256, 0, s>>>(lflag, nlow, lx, ly, rx, ry, rflag));
    scan_exclusive(rflag, rrank, nroot, scan_tmp, total + 4, s);
    VDBC_CUDA(cudaGetLastError());

    // the one host wait of the encoder: table sizes
    uint32_t h_total[8] = {0};
    long long h_counts[2] = {0, 0};
    int h_bad = 0;
    uint32_t h_bsel[2] = {0, 0};
    VDBC_CUDA(cudaMemcpyAsync(h_total, total, sizeof(h_total), cudaMemcpyDeviceToHost, s));
    VDBC_CUDA(cudaMemcpyAsync(h_counts, counts, sizeof(h_counts), cudaMemcpyDeviceToHost, s));
    VDBC_CUDA(cudaMemcpyAsync(&h_bad, nonfinite, sizeof(int), cudaMemcpyDeviceToHost, s));
    VDBC_CUDA(cudaMemcpyAsync(h_bsel, bsel, sizeof(h_bsel), cudaMemcpyDeviceToHost, s));
    vdbc_grid* g = new vdbc_grid();
    g->active.resize(nb);
    VDBC_CUDA(cudaMemcpyAsync(g->active.data(), active, nb, cudaMemcpyDeviceToHost, s));
    vdbc_status ws = wait_stream(s);
    if (ws != VDBC_OK) return release_or_defer(ws, s, [g] { delete g; });   // g->active is a copy's target
    if (h_bad) {
        delete g;
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_encode: the volume holds non-finite values");
    }
    cudaGetDevice(&g->device);
    vdbc_grid_info& info = g->info;
    info.dims[0] = d.nx; info.dims[1] = d.ny; info.dims[2] = d.nz;
    info.payload = payload;
    info.macrocell = mc;
    info.metric = metric;
    info.background_bits = h_bsel[1];
    info.ratio = ratio;
    info.n_bricks = nb;
    info.n_nonempty = h_counts[0];
    info.budget = budget;
    info.n_active = h_counts[1];
    info.n_leaves = h_total[1];
    info.n_tiles = 1 + (int64_t)h_total[2];
    info.n_lower = h_total[3];
    info.n_upper = h_total[4];
    layout(g);
    vdbc_status st = dev_alloc(&g->block, g->block_bytes, s);
    if (st != VDBC_OK) { delete g; return st; }
    st = dev_alloc(reinterpret_cast<void**>(&g->stats), sizeof(DevStats), s);
    if (st != VDBC_OK) { vdbc_grid_free(g); return st; }
    cudaError_t e = cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s);
    if (e != cudaSuccess) { vdbc_grid_free(g); return cuda_status(e, "vdbc_encode: stats"); }
    bind_view(g);
    char* base = static_cast<char*>(g->block);
    uint32_t* root = reinterpret_cast<uint32_t*>(base + g->off_root);
    uint32_t* upper = reinterpret_cast<uint32_t*>(base + g->off_upper);
    uint32_t* lower = reinterpret_cast<uint32_t*>(base + g->off_lower);
    float* tiles = reinterpret_cast<float*>(base + g->off_tiles);
    long long nup = (long long)info.n_upper * kUpperN, nlo = (long long)info.n_lower * kLowerN;
    if (nup) KLAUNCH(k_fill_u32<<<grid1d(std::min<long long>(nup, 1 << 22), 256), 256, 0, s>>>(upper, nup, kBackgroundEntry));
    if (nlo) KLAUNCH(k_fill_u32<<<grid1d(std::min<long long>(nlo, 1 << 22), 256), 256, 0, s>>>(lower, nlo, kBackgroundEntry));
    KLAUNCH(k_fill_root<<<grid1d(nroot, 256), 256, 0, s>>>(root, rflag, rrank, nroot));
    KLAUNCH(k_fill_upper<<<grid1d(nlow, 256), 256, 0, s>>>(upper, lflag, lrank, rrank, nlow, lx, ly, rx, ry));
    KLAUNCH(k_fill_lower<<<grid1d(cap, 256), 256, 0, s>>>(lower, tiles, d, list, counts, lowslot, is_leaf, leaf_rank,
                                                  tile_rank, tval, lrank, bsel));
    KLAUNCH(k_fill_leaves<<<grid1d(cap * 32, 256), 256, 0, s>>>(vol, d, list, counts, is_leaf, leaf_rank, bsel, payload,
                                                        base + g->off_leaves,
                                                        reinterpret_cast<float2*>(base + g->off_meta)));
    e = cudaGetLastError();
    if (e != cudaSuccess) { vdbc_grid_free(g); return cuda_status(e, "vdbc_encode: tree kernels"); }
    if (payload == VDBC_FP32) {
        // FP32 leaves hold the input's values: the ranges come from the input itself
        const GridView& gv = g->view;
        const long long ncell = (long long)gv.mx * gv.my * gv.mz;
        KLAUNCH(k_macrocells_input<<<(unsigned)ncell, kMcInThreads, 0, s>>>(
            vol, d, active, lo_key, hi_key, bsel, gv.mc, gv.mx, gv.my, reinterpret_cast<float*>(base + g->off_mcmin),
            reinterpret_cast<float*>(base + g->off_mcmax)));
        e = cudaGetLastError();
        st = e == cudaSuccess ? VDBC_OK : cuda_status(e, "vdbc_encode: macrocells");
    } else {
        st = build_macrocells(g, s);
    }
    if (st == VDBC_OK) st = checked_flags(g, s);
    if (st != VDBC_OK) return release_or_defer(st, s, [g] { vdbc_grid_free(g); });
    *out = g;
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_grid_decode(const vdbc_grid* g, float* out, int32_t out_on_device, void* stream)
{
    clear_error();
    if (!g || !out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_grid_decode: null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long n = (long long)g->info.dims[0] * g->info.dims[1] * g->info.dims[2];
    float* dst = out;
    void* tmp = nullptr;
    if (!out_on_device) {
        VDBC_TRY(dev_alloc(&tmp, (size_t)n * 4, s));
        dst = static_cast<float*>(tmp);
    }
    cudaError_t e = cudaSuccess;
    if (g->info.payload == VDBC_LEARNED) {
        // neural leaves go through the network once, into a temporary FP32 view
        Materialized m;
        vdbc_status st = materialize_learned(g, s, &m);
        if (st == VDBC_OK) decode_view(m.view, dst, n, s);
        e = cudaGetLastError();
        m.release(s);
        if (st != VDBC_OK) { if (tmp) dev_free(tmp, s); return st; }
    } else {
        decode_view(g->view, dst, n, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !out_on_device) e = cudaMemcpyAsync(out, dst, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) { if (tmp) dev_free(tmp, s); return cuda_status(e, "vdbc_grid_decode"); }
    if (!out_on_device) {
        vdbc_status st = wait_stream(s);
        dev_free(tmp, s);
        if (st != VDBC_OK) return st;
    }
    return checked_flags(g, s);
}

extern "C" vdbc_status vdbc_grid_active_bricks(const vdbc_grid* g, uint8_t* host_out)
{
    clear_error();
    if (!g || !host_out) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_grid_active_bricks: null argument");
    std::memcpy(host_out, g->active.data(), g->active.size());
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_grid_macrocells(const vdbc_grid* g, float* host_min, float* host_max)
{
    clear_error();
    if (!g || !host_min || !host_max) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_grid_macrocells: null argument");
    long long n = (long long)g->view.mx * g->view.my * g->view.mz;
    const char* base = static_cast<const char*>(g->block);
    VDBC_CUDA(cudaMemcpy(host_min, base + g->off_mcmin, (size_t)n * 4, cudaMemcpyDeviceToHost));
    VDBC_CUDA(cudaMemcpy(host_max, base + g->off_mcmax, (size_t)n * 4, cudaMemcpyDeviceToHost));
    return VDBC_OK;
}

extern "C" vdbc_status vdbc_grid_get_info(const vdbc_grid* g, vdbc_grid_info* info)
{
    clear_error();
    if (!g || !info) return set_error(VDBC_ERR_INVALID_ARG, "vdbc_grid_get_info: null argument");
    *info = g->info;
    return VDBC_OK;
}

extern "C" void vdbc_grid_free(vdbc_grid* g)
{
    if (!g) return;
    if (g->block) cudaFree(g->block);
    if (g->stats) {
        release_kernel_events(g->stats);
        cudaFree(g->stats);
    }
    delete g;
}

// ---------------------------------------------------------------- brick selection without allocation
// Some callers cannot allocate device memory while they run: a renderer
// embedded in a host application that owns the whole device-memory budget
// and forbids allocation after start-up, or a frame loop where cudaMalloc /
// cudaFree would stall on their implicit device synchronization.  For them,
// vdbc_select_bricks_noalloc runs the selection phase of vdbc_encode (the
// histogram for B, brick ranges, scores, choice of the bricks to activate)
// with its scratch in the fixed array below, so the call allocates nothing.
// The array is part of this library's device image: every GPU that loads the
// library holds it (about 1.6 MiB) until the process exits.
namespace vdbc {
namespace {

constexpr long long kNoAllocMaxBricks = 65536;

struct NoAllocScratch {
    unsigned long long hist[65536];          // histogram of one level of B's bit pattern
    unsigned long long fkey[kNoAllocMaxBricks];
    uint32_t lo_key[kNoAllocMaxBricks];
    uint32_t hi_key[kNoAllocMaxBricks];
    uint8_t empty[kNoAllocMaxBricks];
    uint32_t bsel[2];
    int nonfinite;
    Majority maj;                            // the background's candidate pattern and its count
    SelState sel;                            // the grid-wide selection's state
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// device address of g_noalloc_scratch, looked up once per device (with that
// device current) and cached; host code must not use the symbol itself.  The
// cache is shared by every host thread, so the lookup runs under a lock.
vdbc_status noalloc_scratch(NoAllocScratch** out)
{
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static NoAllocScratch* cache[kMaxDevices] = {nullptr};
    int dev = 0;
    VDBC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(VDBC_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!cache[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(scratch)");
        cache[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = cache[dev];
    return VDBC_OK;
}

// a caller's pointer that kernels will read or write: device (or managed)
// memory of any device, aligned for its element type; anything else (a host
// pointer, an unregistered address) is refused before a kernel could touch it
vdbc_status check_device_pointer(const void* p, size_t align, const char* what)
{
    if (reinterpret_cast<uintptr_t>(p) % align != 0)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_select_bricks_noalloc: %s is not %zu-byte aligned", what, align);
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e, "cudaPointerGetAttributes");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_select_bricks_noalloc: %s is not device memory", what);
    return VDBC_OK;
}

__global__ void k_noalloc_finish(const uint32_t* __restrict__ bsel, const int* __restrict__ nonfinite,
                                 uint32_t* __restrict__ b_out, long long* __restrict__ counts_out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        b_out[0] = bsel[1];
        counts_out[2] = nonfinite[0];
    }
}

}  // namespace
}  // namespace vdbc

// Same results as the selection inside vdbc_encode, written to the caller's
// device buffers; enqueued on `stream`, nothing waits and nothing is
// allocated.  The first call on a device looks up the scratch address (make
// it before any stream capture).  All calls share one scratch array, so calls
// whose work overlaps on the GPU (different streams, or threads without an
// ordering) race: serialize them.
extern "C" vdbc_status vdbc_select_bricks_noalloc(const vdbc_dense* in, const vdbc_encode_params* params,
                                                  uint32_t* background_bits_out, uint8_t* active_out,
                                                  int64_t* counts_out, void* stream)
{
    clear_error();
    if (!in || !params || !in->data || !background_bits_out || !active_out || !counts_out)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_select_bricks_noalloc: null argument");
    if (!in->on_device)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_select_bricks_noalloc: the volume must be in device memory");
    for (int a = 0; a < 3; ++a)
        if (in->dims[a] < 1 || in->dims[a] > kMaxDim)
            return set_error(VDBC_ERR_INVALID_ARG, "vdbc_select_bricks_noalloc: dims[%d]=%d outside 1..%d", a,
                             in->dims[a], kMaxDim);
    const double ratio = params->ratio;
    if (!(ratio >= 1.0) || !std::isfinite(ratio))
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_select_bricks_noalloc: ratio must be a finite value >= 1");
    const int metric = params->metric == 0 ? VDBC_F2 : params->metric;
    if (metric < VDBC_F1 || metric > VDBC_F3)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_select_bricks_noalloc: unknown metric %d", metric);
    const int payload = params->payload;
    if (payload < VDBC_FP32 || payload > VDBC_FP8)
        return set_error(VDBC_ERR_INVALID_ARG, "vdbc_select_bricks_noalloc: unknown payload %d", payload);
    Dims d;
    d.nx = in->dims[0]; d.ny = in->dims[1]; d.nz = in->dims[2];
    d.bx = (d.nx + 31) / 32; d.by = (d.ny + 31) / 32; d.bz = (d.nz + 31) / 32;
    const long long nb = (long long)d.bx * d.by * d.bz;
    if (nb > kNoAllocMaxBricks)
        return set_error(VDBC_ERR_INVALID_ARG,
                         "vdbc_select_bricks_noalloc: %lld bricks of 32^3 exceed the fixed scratch limit of %lld",
                         nb, kNoAllocMaxBricks);
    // the outputs' lengths (1 word, nb bytes, 3 words) are the caller's to
    // guarantee; their kind and alignment are checked here
    VDBC_TRY(check_device_pointer(in->data, 4, "the volume"));
    VDBC_TRY(check_device_pointer(background_bits_out, 4, "background_bits_out"));
    VDBC_TRY(check_device_pointer(active_out, 1, "active_out"));
    VDBC_TRY(check_device_pointer(counts_out, 8, "counts_out"));
    NoAllocScratch* sc = nullptr;
    VDBC_TRY(noalloc_scratch(&sc));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double nbud = std::floor((double)nb * 131072.0 / (ratio * (double)brick_bytes(payload)));
    const long long budget = nbud > (double)nb ? nb : (long long)nbud;
    // the scratch keeps the previous call's contents: clear what accumulates
    VDBC_CUDA(cudaMemsetAsync(sc->hist, 0, sizeof(sc->hist), s));
    VDBC_CUDA(cudaMemsetAsync(&sc->nonfinite, 0, sizeof(int), s));
    unsigned p1grid = 1;
    VDBC_TRY(pass1_setup(nb, &p1grid));
    VDBC_TRY(launch_background(in->data, d, (int)nb, p1grid, sc->lo_key, sc->hi_key, sc->hist, sc->bsel,
                               &sc->nonfinite, &sc->maj, s));
    KLAUNCH(k_scores<<<grid1d(nb, 256), 256, 0, s>>>(sc->lo_key, sc->hi_key, (int)nb, sc->bsel, metric, sc->fkey,
                                                     sc->empty));
    VDBC_TRY(launch_select(sc->fkey, sc->empty, (int)nb, budget, active_out, reinterpret_cast<long long*>(counts_out),
                           &sc->sel, (int)p1grid, s));
    KLAUNCH(k_noalloc_finish<<<1, 32, 0, s>>>(sc->bsel, &sc->nonfinite, background_bits_out,
                                              reinterpret_cast<long long*>(counts_out)));
    VDBC_CUDA(cudaGetLastError());
    return VDBC_OK;
}
