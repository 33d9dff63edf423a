/*
 * encode.c -- the fixed-rate encoder of Section 3.1 (Algorithm 1, Eq. f1-f3)
 * and the tree of Section 3.2.1, written plainly.
 *
 * Readings of the paper taken here, where it is silent or ambiguous:
 *  - background value: the histogram of Algorithm 1 is a two-level histogram
 *    of the float bit patterns (upper 16 bits, then lower 16 bits inside the
 *    winning upper bin), ties to the smaller pattern;
 *  - bricks are 32^3 and the brick grid uses ceil division; edge bricks are
 *    clipped to the volume;
 *  - a brick is empty when its min and max are both bitwise the background;
 *    empty bricks are never activated;
 *  - bricks are activated in order of decreasing score f, ties to the lower
 *    brick index (x fastest), exactly N = floor(numBricks * 131072 /
 *    (ratio * brick_bytes)) of them (capped at the non-empty count);
 *  - the two extreme corner voxels are always set (Section 3.2.1);
 *  - the tree is root -> 32^3 upper -> 16^3 lower -> 8^3 leaf, prune collapses
 *    a leaf whose 512 values are bitwise equal into a tile, and a lower/upper
 *    node whose entries are all equal tiles into a tile of its parent;
 *  - FP16/FP8 payloads (a project extension: the paper stores FP32 leaves and
 *    prints no quantized value; the rounding is pinned to the IEEE 754 binary16
 *    and OCP E4M3 definitions instead): per leaf offset = min, scale = max -
 *    min, code = round to nearest even of (v - off) / scale in FP32, decode =
 *    fmaf(scale, code, off).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static uint32_t f2b(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float b2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

/* total order of IEEE binary32 bit patterns (-0 before +0) */
static uint32_t okey(uint32_t b) { return (b & 0x80000000u) ? ~b : (b | 0x80000000u); }
static uint32_t okey_inv(uint32_t k) { return (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k; }

/* ---- phase 1 of Algorithm 1: histogram, argmax, background value B ---- */
uint32_t or_background_bits(const float* v, int64_t n)
{
    uint64_t* h = (uint64_t*)calloc(65536, sizeof(uint64_t));
    for (int64_t i = 0; i < n; ++i) h[f2b(v[i]) >> 16] += 1;
    uint32_t hi = 0;
    for (uint32_t b = 1; b < 65536; ++b) if (h[b] > h[hi]) hi = b;
    memset(h, 0, 65536 * sizeof(uint64_t));
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u = f2b(v[i]);
        if ((u >> 16) == hi) h[u & 0xffffu] += 1;
    }
    uint32_t lo = 0;
    for (uint32_t b = 1; b < 65536; ++b) if (h[b] > h[lo]) lo = b;
    free(h);
    return (hi << 16) | lo;
}

/* ---- phase 2: 32^3 bricks (numBricks = ceil(dims / 32)) and their ranges */
void or_brick_grid(const int64_t dims[3], int64_t nb[3])
{
    for (int a = 0; a < 3; ++a) nb[a] = (dims[a] + 31) / 32;
}

void or_brick_ranges(const float* v, const int64_t dims[3], uint32_t* lo_bits, uint32_t* hi_bits)
{
    int64_t nb[3];
    or_brick_grid(dims, nb);
    for (int64_t bz = 0; bz < nb[2]; ++bz)
    for (int64_t by = 0; by < nb[1]; ++by)
    for (int64_t bx = 0; bx < nb[0]; ++bx) {
        uint32_t kmin = 0xffffffffu, kmax = 0u;
        for (int64_t z = bz * 32; z < bz * 32 + 32 && z < dims[2]; ++z)
        for (int64_t y = by * 32; y < by * 32 + 32 && y < dims[1]; ++y)
        for (int64_t x = bx * 32; x < bx * 32 + 32 && x < dims[0]; ++x) {
            uint32_t k = okey(f2b(v[(z * dims[1] + y) * dims[0] + x]));
            if (k < kmin) kmin = k;
            if (k > kmax) kmax = k;
        }
        int64_t b = (bz * nb[1] + by) * nb[0] + bx;
        lo_bits[b] = okey_inv(kmin);
        hi_bits[b] = okey_inv(kmax);
    }
}

/* ---- phase 3: similarity f1/f2/f3 of a brick range to B (Eq. f1-f3) ---- */
void or_brick_scores(const uint32_t* lo_bits, const uint32_t* hi_bits, int64_t nbricks,
                     uint32_t b_bits, int metric, double* f, uint8_t* empty)
{
    double B = (double)b2f(b_bits);
    for (int64_t i = 0; i < nbricks; ++i) {
        double lo = (double)b2f(lo_bits[i]);
        double hi = (double)b2f(hi_bits[i]);
        double dl = fabs(lo - B), dh = fabs(hi - B);
        double s;
        if (metric == OR_F1) s = (dl < dh) ? dl : dh;            /* closest  */
        else if (metric == OR_F3) s = fabs((lo + hi) / 2.0 - B); /* median   */
        else s = (dl > dh) ? dl : dh;                            /* farthest */
        f[i] = s;
        empty[i] = (uint8_t)(lo_bits[i] == b_bits && hi_bits[i] == b_bits);
    }
}

/* number of bricks to activate: the linear map of the rate onto the brick
 * count, in bytes so that FP16/FP8 payloads buy proportionally more bricks */
static int64_t brick_bytes(int payload)
{
    if (payload == OR_FP16) return 32768 * 2 + 64 * 8;
    if (payload == OR_FP8)  return 32768 * 1 + 64 * 8;
    return 32768 * 4;
}

int64_t or_brick_budget(int64_t nbricks, double ratio, int payload)
{
    double n = floor((double)nbricks * 131072.0 / (ratio * (double)brick_bytes(payload)));
    if (n < 0) n = 0;
    if (n > (double)nbricks) n = (double)nbricks;
    return (int64_t)n;
}

static const double* g_sort_f;
static int cmp_bricks(const void* a, const void* b)
{
    int64_t ia = *(const int64_t*)a, ib = *(const int64_t*)b;
    double fa = g_sort_f[ia], fb = g_sort_f[ib];
    if (fa > fb) return -1;
    if (fa < fb) return 1;
    return (ia < ib) ? -1 : (ia > ib);
}

/* SortBy + activation loop: exactly min(N, #non-empty) bricks, largest f first */
int64_t or_select(const double* f, const uint8_t* empty, int64_t nbricks, int64_t n_budget,
                  uint8_t* active)
{
    int64_t* refs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nbricks > 0 ? nbricks : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < nbricks; ++i) {
        active[i] = 0;
        if (!empty[i]) refs[m++] = i;
    }
    g_sort_f = f;
    qsort(refs, (size_t)m, sizeof(int64_t), cmp_bricks);
    int64_t take = n_budget < m ? n_budget : m;
    for (int64_t r = 0; r < take; ++r) active[refs[r]] = 1;
    free(refs);
    return take;
}

/* ---- minifloat rounding from the IEEE 754 / OCP FP8 definitions --------- */
/* Rounds x to the nearest value of a binary format with `ebits` exponent bits,
 * `mbits` fraction bits and exponent bias `bias` (ties to even).  Values past
 * the largest finite one become +-inf, or the largest finite one when
 * `saturate` (E4M3 has no infinity; its all-ones code is NaN). */
float or_round_minifloat(float x, int ebits, int mbits, int bias, int saturate)
{
    double a = fabs((double)x);
    if (a == 0.0 || isnan(a)) return x;
    int emin = 1 - bias;
    double maxfin;
    if (saturate)   /* E4M3: exponent field all ones is usable except mantissa all ones */
        maxfin = ldexp(2.0 - ldexp(2.0, -mbits), (1 << ebits) - 1 - bias);
    else
        maxfin = ldexp(2.0 - ldexp(1.0, -mbits), (1 << ebits) - 2 - bias);
    int e;
    frexp(a, &e);           /* a = m * 2^e, m in [0.5, 1) -> unbiased exponent e-1 */
    int ue = e - 1;
    if (ue < emin) ue = emin;                 /* subnormal spacing */
    double quantum = ldexp(1.0, ue - mbits);
    double n = nearbyint(a / quantum);        /* exact division, ties to even */
    double r = n * quantum;
    if (r > maxfin) {
        if (saturate) r = maxfin;
        else {
            /* IEEE: overflow to infinity once the value rounds past maxfin */
            r = INFINITY;
        }
    }
    return (float)(x < 0 ? -r : r);
}

float or_round_fp16(float x) { return or_round_minifloat(x, 5, 10, 15, 0); }
float or_round_e4m3(float x) { return or_round_minifloat(x, 4, 3, 7, 1); }

void or_quantize_leaf(const float in[512], int payload, float out[512], float* scale_out,
                      float* offset_out)
{
    uint32_t kmin = 0xffffffffu, kmax = 0u;
    for (int i = 0; i < 512; ++i) {
        uint32_t k = okey(f2b(in[i]));
        if (k < kmin) kmin = k;
        if (k > kmax) kmax = k;
    }
    float off = b2f(okey_inv(kmin));
    float mx = b2f(okey_inv(kmax));
    float scale = mx - off;                 /* FP32 subtraction */
    for (int i = 0; i < 512; ++i) {
        float t = 0.0f;
        if (scale != 0.0f) {
            float num = in[i] - off;        /* FP32 */
            t = num / scale;                /* FP32, correctly rounded */
        }
        float q = (payload == OR_FP16) ? or_round_fp16(t) : or_round_e4m3(t);
        out[i] = fmaf(scale, q, off);
    }
    *scale_out = scale;
    *offset_out = off;
}

/* ---- decoded grid D by definition (Sections 3.1, 3.2.1, 3.2.2) ---------
 * D(x) = V(x) where x lies in an activated brick or is one of the two extreme
 * corners, B elsewhere.  With FP16/FP8 payload every 8^3 leaf whose values of
 * D are not all bitwise equal is replaced by its quantized form (positions of
 * a leaf outside the volume hold B). */
void or_decode_dense(const float* v, const int64_t dims[3], const uint8_t* active,
                     uint32_t b_bits, int payload, float* out)
{
    int64_t nb[3];
    or_brick_grid(dims, nb);
    float B = b2f(b_bits);
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
    for (int64_t x = 0; x < nx; ++x) {
        int64_t b = ((z / 32) * nb[1] + (y / 32)) * nb[0] + (x / 32);
        int corner = (x == 0 && y == 0 && z == 0) || (x == nx - 1 && y == ny - 1 && z == nz - 1);
        int64_t idx = (z * ny + y) * nx + x;
        out[idx] = (active[b] || corner) ? v[idx] : B;
    }
    if (payload == OR_FP32) return;
    float leaf[512], q[512], s, o;
    for (int64_t lz = 0; lz < (nz + 7) / 8; ++lz)
    for (int64_t ly = 0; ly < (ny + 7) / 8; ++ly)
    for (int64_t lx = 0; lx < (nx + 7) / 8; ++lx) {
        int constant = 1;
        for (int n = 0; n < 512; ++n) {
            int64_t x = lx * 8 + (n & 7), y = ly * 8 + ((n >> 3) & 7), z = lz * 8 + (n >> 6);
            leaf[n] = (x < nx && y < ny && z < nz) ? out[(z * ny + y) * nx + x] : B;
            if (f2b(leaf[n]) != f2b(leaf[0])) constant = 0;
        }
        if (constant) continue;
        or_quantize_leaf(leaf, payload, q, &s, &o);
        for (int n = 0; n < 512; ++n) {
            int64_t x = lx * 8 + (n & 7), y = ly * 8 + ((n >> 3) & 7), z = lz * 8 + (n >> 6);
            if (x < nx && y < ny && z < nz) out[(z * ny + y) * nx + x] = q[n];
        }
    }
}

/* ---- the VDB tree (Section 2.3 layout {5,4,3}; Section 3.2.1 build) -----
 * Entries of internal nodes are either a child pointer or a tile value; the
 * root is a dense table over the 4096^3 regions an upper node covers. */
typedef struct { float v[512]; } or_leaf;
typedef struct { int is_child; float value; void* child; } or_entry;
typedef struct { or_entry e[4096]; } or_lower;     /* 16^3 */
typedef struct { or_entry e[32768]; } or_upper;    /* 32^3 */

struct or_tree {
    int64_t dims[3];
    int64_t nroot[3];
    or_entry* root;          /* children are or_upper* */
    float background;
    int payload;
};

static or_entry* root_slot(or_tree* t, int64_t i, int64_t j, int64_t k)
{
    return &t->root[((k >> 12) * t->nroot[1] + (j >> 12)) * t->nroot[0] + (i >> 12)];
}

/* Activate(voxel, value) of Algorithm 1: create nodes down to the leaf and set the value */
static void tree_set(or_tree* t, int64_t i, int64_t j, int64_t k, float value)
{
    or_entry* r = root_slot(t, i, j, k);
    if (!r->is_child) {
        or_upper* u = (or_upper*)malloc(sizeof(or_upper));
        for (int n = 0; n < 32768; ++n) { u->e[n].is_child = 0; u->e[n].value = r->value; u->e[n].child = NULL; }
        r->is_child = 1; r->child = u;
    }
    or_upper* u = (or_upper*)r->child;
    or_entry* ue = &u->e[(((k >> 7) & 31) * 32 + ((j >> 7) & 31)) * 32 + ((i >> 7) & 31)];
    if (!ue->is_child) {
        or_lower* l = (or_lower*)malloc(sizeof(or_lower));
        for (int n = 0; n < 4096; ++n) { l->e[n].is_child = 0; l->e[n].value = ue->value; l->e[n].child = NULL; }
        ue->is_child = 1; ue->child = l;
    }
    or_lower* l = (or_lower*)ue->child;
    or_entry* le = &l->e[(((k >> 3) & 15) * 16 + ((j >> 3) & 15)) * 16 + ((i >> 3) & 15)];
    if (!le->is_child) {
        or_leaf* f = (or_leaf*)malloc(sizeof(or_leaf));
        for (int n = 0; n < 512; ++n) f->v[n] = le->value;
        le->is_child = 1; le->child = f;
    }
    or_leaf* f = (or_leaf*)le->child;
    f->v[((k & 7) * 8 + (j & 7)) * 8 + (i & 7)] = value;
}

/* prune(): collapse children whose values are all bitwise equal into tiles */
static int entries_constant(const or_entry* e, int n, float* value)
{
    for (int a = 0; a < n; ++a) if (e[a].is_child) return 0;
    for (int a = 1; a < n; ++a) if (f2b(e[a].value) != f2b(e[0].value)) return 0;
    *value = e[0].value;
    return 1;
}

static void tree_prune(or_tree* t)
{
    int64_t nr = t->nroot[0] * t->nroot[1] * t->nroot[2];
    for (int64_t r = 0; r < nr; ++r) {
        if (!t->root[r].is_child) continue;
        or_upper* u = (or_upper*)t->root[r].child;
        for (int a = 0; a < 32768; ++a) {
            if (!u->e[a].is_child) continue;
            or_lower* l = (or_lower*)u->e[a].child;
            for (int b = 0; b < 4096; ++b) {
                if (!l->e[b].is_child) continue;
                or_leaf* f = (or_leaf*)l->e[b].child;
                int constant = 1;
                for (int n = 1; n < 512; ++n) if (f2b(f->v[n]) != f2b(f->v[0])) { constant = 0; break; }
                if (constant) {
                    l->e[b].is_child = 0; l->e[b].value = f->v[0]; l->e[b].child = NULL;
                    free(f);
                }
            }
            float value;
            if (entries_constant(l->e, 4096, &value)) {
                u->e[a].is_child = 0; u->e[a].value = value; u->e[a].child = NULL;
                free(l);
            }
        }
        float value;
        if (entries_constant(u->e, 32768, &value)) {
            t->root[r].is_child = 0; t->root[r].value = value; t->root[r].child = NULL;
            free(u);
        }
    }
}

static void tree_quantize(or_tree* t)
{
    int64_t nr = t->nroot[0] * t->nroot[1] * t->nroot[2];
    float q[512], s, o;
    for (int64_t r = 0; r < nr; ++r) {
        if (!t->root[r].is_child) continue;
        or_upper* u = (or_upper*)t->root[r].child;
        for (int a = 0; a < 32768; ++a) {
            if (!u->e[a].is_child) continue;
            or_lower* l = (or_lower*)u->e[a].child;
            for (int b = 0; b < 4096; ++b) {
                if (!l->e[b].is_child) continue;
                or_leaf* f = (or_leaf*)l->e[b].child;
                or_quantize_leaf(f->v, t->payload, q, &s, &o);
                memcpy(f->v, q, sizeof(q));
            }
        }
    }
}

or_tree* or_tree_build(const float* v, const int64_t dims[3], const uint8_t* active,
                       uint32_t b_bits, int payload)
{
    or_tree* t = (or_tree*)calloc(1, sizeof(or_tree));
    for (int a = 0; a < 3; ++a) { t->dims[a] = dims[a]; t->nroot[a] = (dims[a] + 4095) / 4096; }
    int64_t nr = t->nroot[0] * t->nroot[1] * t->nroot[2];
    t->background = b2f(b_bits);
    t->payload = payload;
    t->root = (or_entry*)malloc(sizeof(or_entry) * (size_t)nr);
    for (int64_t r = 0; r < nr; ++r) { t->root[r].is_child = 0; t->root[r].value = t->background; t->root[r].child = NULL; }

    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    /* the extreme corners are always set (Section 3.2.1) */
    tree_set(t, 0, 0, 0, v[0]);
    tree_set(t, nx - 1, ny - 1, nz - 1, v[(nz * ny) * nx - 1]);
    /* every voxel of every activated brick */
    int64_t nb[3];
    or_brick_grid(dims, nb);
    for (int64_t bz = 0; bz < nb[2]; ++bz)
    for (int64_t by = 0; by < nb[1]; ++by)
    for (int64_t bx = 0; bx < nb[0]; ++bx) {
        if (!active[(bz * nb[1] + by) * nb[0] + bx]) continue;
        for (int64_t z = bz * 32; z < bz * 32 + 32 && z < nz; ++z)
        for (int64_t y = by * 32; y < by * 32 + 32 && y < ny; ++y)
        for (int64_t x = bx * 32; x < bx * 32 + 32 && x < nx; ++x)
            tree_set(t, x, y, z, v[(z * ny + y) * nx + x]);
    }
    tree_prune(t);
    if (payload != OR_FP32) tree_quantize(t);
    return t;
}

/* descent root -> upper -> lower -> leaf; a tile answers for its whole region */
float or_tree_value(const or_tree* t, int64_t i, int64_t j, int64_t k)
{
    const or_entry* r = &t->root[((k >> 12) * t->nroot[1] + (j >> 12)) * t->nroot[0] + (i >> 12)];
    if (!r->is_child) return r->value;
    const or_upper* u = (const or_upper*)r->child;
    const or_entry* ue = &u->e[(((k >> 7) & 31) * 32 + ((j >> 7) & 31)) * 32 + ((i >> 7) & 31)];
    if (!ue->is_child) return ue->value;
    const or_lower* l = (const or_lower*)ue->child;
    const or_entry* le = &l->e[(((k >> 3) & 15) * 16 + ((j >> 3) & 15)) * 16 + ((i >> 3) & 15)];
    if (!le->is_child) return le->value;
    const or_leaf* f = (const or_leaf*)le->child;
    return f->v[((k & 7) * 8 + (j & 7)) * 8 + (i & 7)];
}

/* the 512 values of the leaf node at leaf position (li, lj, lk) (voxel
 * (8li + a, 8lj + b, 8lk + c) at a + 8b + 64c, including voxels past the
 * volume's edge); 0 (and out untouched) where that position is a tile */
int or_tree_leaf(const or_tree* t, int64_t li, int64_t lj, int64_t lk, float out[512])
{
    int64_t i = li * 8, j = lj * 8, k = lk * 8;
    const or_entry* r = &t->root[((k >> 12) * t->nroot[1] + (j >> 12)) * t->nroot[0] + (i >> 12)];
    if (!r->is_child) return 0;
    const or_upper* u = (const or_upper*)r->child;
    const or_entry* ue = &u->e[(((k >> 7) & 31) * 32 + ((j >> 7) & 31)) * 32 + ((i >> 7) & 31)];
    if (!ue->is_child) return 0;
    const or_lower* l = (const or_lower*)ue->child;
    const or_entry* le = &l->e[(((k >> 3) & 15) * 16 + ((j >> 3) & 15)) * 16 + ((i >> 3) & 15)];
    if (!le->is_child) return 0;
    memcpy(out, ((const or_leaf*)le->child)->v, sizeof(float) * 512);
    return 1;
}

/* out = {root entries, upper nodes, lower nodes, leaves, lower-level tiles
 *        that are not the background, upper-level tiles that are not the background} */
void or_tree_counts(const or_tree* t, int64_t out[6])
{
    int64_t nr = t->nroot[0] * t->nroot[1] * t->nroot[2];
    int64_t nu = 0, nl = 0, nf = 0, tl = 0, tu = 0;
    for (int64_t r = 0; r < nr; ++r) {
        if (!t->root[r].is_child) continue;
        ++nu;
        const or_upper* u = (const or_upper*)t->root[r].child;
        for (int a = 0; a < 32768; ++a) {
            if (!u->e[a].is_child) {
                if (f2b(u->e[a].value) != f2b(t->background)) ++tu;
                continue;
            }
            ++nl;
            const or_lower* l = (const or_lower*)u->e[a].child;
            for (int b = 0; b < 4096; ++b) {
                if (l->e[b].is_child) ++nf;
                else if (f2b(l->e[b].value) != f2b(t->background)) ++tl;
            }
        }
    }
    out[0] = nr; out[1] = nu; out[2] = nl; out[3] = nf; out[4] = tl; out[5] = tu;
}

void or_tree_free(or_tree* t)
{
    if (!t) return;
    int64_t nr = t->nroot[0] * t->nroot[1] * t->nroot[2];
    for (int64_t r = 0; r < nr; ++r) {
        if (!t->root[r].is_child) continue;
        or_upper* u = (or_upper*)t->root[r].child;
        for (int a = 0; a < 32768; ++a) {
            if (!u->e[a].is_child) continue;
            or_lower* l = (or_lower*)u->e[a].child;
            for (int b = 0; b < 4096; ++b) if (l->e[b].is_child) free(l->e[b].child);
            free(l);
        }
        free(u);
    }
    free(t->root);
    free(t);
}
