/*
 * render.c -- the renderer of Section 4, restated plainly in FP64.
 *
 * Conventions (readings of what the paper leaves open):
 *  - voxel (i,j,k) sits at index coordinate (i,j,k); the volume is the box
 *    [-1/2, dim-1/2]^3; world space is index space shifted by 1/2 and scaled
 *    so that the longest axis spans one unit: index = world * M - 1/2;
 *  - trilinear reconstruction from floor(p) and floor(p)+1, each clamped to
 *    [0, dim-1] (clamp to edge, as a texture does); the sampler of Section
 *    3.2.2 reads the decoded grid D;
 *  - macrocell grid (Section 4): cells of `cell` voxels starting at -1/2, the
 *    min/max of D over the cell's voxels dilated by one voxel on each side
 *    (the support of trilinear reconstruction inside the cell);
 *  - majorant of a cell = density_scale * max / M per index unit;
 *  - 3D-DDA over macrocells (Section 4, Amanatides-Woo stepping); Woodcock
 *    (delta) tracking with one optical depth per free flight carried across
 *    the non-empty cells (the majorant-grid free-path sampling of
 *    Szirmay-Kalos et al. 2011 that Section 4 cites for its DDA); cells of
 *    zero majorant or zero length consume nothing;
 *  - ratio tracking for the transmittance toward the directional light;
 *  - Philox counter = (pixel, sample, call, stream), key = seed; stream 0 is
 *    the camera and the scattering walk, stream 1 the light rays; each call
 *    gives u0 (optical depth of a free flight), u1 (accept test), u2/u3
 *    (phase function);
 *  - Henyey-Greenstein phase function; orthonormal basis of Duff et al.,
 *    "Building an Orthonormal Basis, Revisited" (JCGT 2017);
 *  - a path scatters at most max_bounces times; each scattering event adds
 *    the light's contribution; an escaping path adds the constant
 *    environment.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ---- sampler: trilinear over D, clamp to edge (Section 3.2.2) ---------- */
double or_trilinear(const float* d, const int64_t dims[3], const double p[3])
{
    int64_t i0[3], i1[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(p[a]);
        f[a] = p[a] - fl;
        i0[a] = clampi((int64_t)fl, 0, dims[a] - 1);
        i1[a] = clampi((int64_t)fl + 1, 0, dims[a] - 1);
    }
#define V(x, y, z) ((double)d[((z) * dims[1] + (y)) * dims[0] + (x)])
    double c00 = V(i0[0], i0[1], i0[2]) * (1.0 - f[0]) + V(i1[0], i0[1], i0[2]) * f[0];
    double c10 = V(i0[0], i1[1], i0[2]) * (1.0 - f[0]) + V(i1[0], i1[1], i0[2]) * f[0];
    double c01 = V(i0[0], i0[1], i1[2]) * (1.0 - f[0]) + V(i1[0], i0[1], i1[2]) * f[0];
    double c11 = V(i0[0], i1[1], i1[2]) * (1.0 - f[0]) + V(i1[0], i1[1], i1[2]) * f[0];
#undef V
    double c0 = c00 * (1.0 - f[1]) + c10 * f[1];
    double c1 = c01 * (1.0 - f[1]) + c11 * f[1];
    return c0 * (1.0 - f[2]) + c1 * f[2];
}

/* ---- macrocell min/max of D (Section 4) --------------------------------- */
void or_macrocell_minmax(const float* d, const int64_t dims[3], int32_t cell, float* mn, float* mx)
{
    int64_t nc[3];
    for (int a = 0; a < 3; ++a) nc[a] = (dims[a] + cell - 1) / cell;
    for (int64_t cz = 0; cz < nc[2]; ++cz)
    for (int64_t cy = 0; cy < nc[1]; ++cy)
    for (int64_t cx = 0; cx < nc[0]; ++cx) {
        int64_t lo[3] = {cx * cell - 1, cy * cell - 1, cz * cell - 1};
        int64_t hi[3] = {cx * cell + cell, cy * cell + cell, cz * cell + cell};
        for (int a = 0; a < 3; ++a) { lo[a] = clampi(lo[a], 0, dims[a] - 1); hi[a] = clampi(hi[a], 0, dims[a] - 1); }
        float vmin = INFINITY, vmax = -INFINITY;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
        for (int64_t y = lo[1]; y <= hi[1]; ++y)
        for (int64_t x = lo[0]; x <= hi[0]; ++x) {
            float v = d[(z * dims[1] + y) * dims[0] + x];
            if (v < vmin) vmin = v;
            if (v > vmax) vmax = v;
        }
        int64_t c = (cz * nc[1] + cy) * nc[0] + cx;
        mn[c] = vmin;
        mx[c] = vmax;
    }
}

/* ---- ray / box ---------------------------------------------------------- */
int or_clip_box(const int64_t dims[3], const double o[3], const double dir[3], double* tin, double* tout)
{
    double t0 = 0.0, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = -0.5, hi = (double)dims[a] - 0.5;
        if (dir[a] == 0.0) {
            if (o[a] < lo || o[a] > hi) return 0;
            continue;
        }
        double ta = (lo - o[a]) / dir[a], tb = (hi - o[a]) / dir[a];
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    *tin = t0;
    *tout = t1;
    return t0 < t1;
}

/* ---- 3D-DDA over the macrocell grid ------------------------------------- */
typedef struct {
    int64_t nc[3];
    int64_t c[3];
    int step[3];
    double o[3], d[3];
    double cell;
    double t, tmax;
} dda_t;

static double dda_boundary(const dda_t* s, int a)
{
    if (s->step[a] == 0) return INFINITY;
    double b = -0.5 + (double)(s->c[a] + (s->step[a] > 0 ? 1 : 0)) * s->cell;
    return (b - s->o[a]) / s->d[a];
}

static void dda_init(dda_t* s, const int64_t dims[3], int32_t cell, const double o[3],
                     const double dir[3], double tmin, double tmax)
{
    s->cell = (double)cell;
    s->t = tmin;
    s->tmax = tmax;
    for (int a = 0; a < 3; ++a) {
        s->nc[a] = (dims[a] + cell - 1) / cell;
        s->o[a] = o[a];
        s->d[a] = dir[a];
        s->step[a] = dir[a] > 0.0 ? 1 : (dir[a] < 0.0 ? -1 : 0);
        double p = o[a] + tmin * dir[a];
        s->c[a] = clampi((int64_t)floor((p + 0.5) / s->cell), 0, s->nc[a] - 1);
    }
}

/* current cell's [t, t_exit); returns 0 once the ray has left the grid */
static int dda_cell(const dda_t* s, int64_t* cell_id, double* texit)
{
    if (s->t >= s->tmax) return 0;
    for (int a = 0; a < 3; ++a) if (s->c[a] < 0 || s->c[a] >= s->nc[a]) return 0;
    double te = s->tmax;
    for (int a = 0; a < 3; ++a) { double b = dda_boundary(s, a); if (b < te) te = b; }
    *cell_id = (s->c[2] * s->nc[1] + s->c[1]) * s->nc[0] + s->c[0];
    *texit = te;
    return 1;
}

static void dda_advance(dda_t* s, double texit)
{
    /* step the axis whose boundary is nearest (x, then y, then z on ties) */
    int best = -1;
    double bt = INFINITY;
    for (int a = 0; a < 3; ++a) { double b = dda_boundary(s, a); if (b < bt) { bt = b; best = a; } }
    if (best < 0 || bt >= s->tmax) { s->t = s->tmax; return; }
    s->c[best] += s->step[best];
    if (texit > s->t) s->t = texit;
}

int64_t or_dda_cells(const int64_t dims[3], int32_t cell, const double o[3], const double dir[3],
                     double tmin, double tmax, int64_t* cells, double* t0, double* t1, int64_t cap)
{
    dda_t s;
    dda_init(&s, dims, cell, o, dir, tmin, tmax);
    int64_t n = 0, id;
    double te;
    while (n < cap && dda_cell(&s, &id, &te)) {
        cells[n] = id; t0[n] = s.t; t1[n] = te; ++n;
        dda_advance(&s, te);
    }
    return n;
}

/* ---- phase function ----------------------------------------------------- */
double or_hg_eval(double mu, double g)
{
    double den = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * M_PI * den * sqrt(den));
}

/* inverse CDF of the Henyey-Greenstein distribution of mu = cos(theta) */
double or_hg_sample_mu(double g, double xi)
{
    double mu;
    if (fabs(g) < 1e-3) mu = 1.0 - 2.0 * xi;
    else {
        double s = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
        mu = (1.0 + g * g - s * s) / (2.0 * g);
    }
    if (mu < -1.0) mu = -1.0;
    if (mu > 1.0) mu = 1.0;
    return mu;
}

void or_onb(const double n[3], double b1[3], double b2[3])
{
    double sign = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a; b1[1] = sign * b; b1[2] = -sign * n[0];
    b2[0] = b; b2[1] = sign + n[1] * n[1] * a; b2[2] = -n[1];
}

/* Direction after a scattering event (Section 4: the path goes on in a
 * direction drawn from the phase function around the incoming one): the
 * polar cosine mu is measured from the incoming direction `dir`, the azimuth
 * phi (radians) turns about it in the plane of the basis (b1, b2) of or_onb.
 * out = sin(theta) cos(phi) b1 + sin(theta) sin(phi) b2 + mu dir, normalized. */
void or_scatter_dir(const double dir[3], double mu, double phi, double out[3])
{
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double b1[3], b2[3];
    or_onb(dir, b1, b2);
    for (int a = 0; a < 3; ++a) out[a] = st * cos(phi) * b1[a] + st * sin(phi) * b2[a] + mu * dir[a];
    double l = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
    for (int a = 0; a < 3; ++a) out[a] /= l;
}

/* ---- camera ------------------------------------------------------------- */
static void normalize3(double v[3])
{
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= l; v[1] /= l; v[2] /= l;
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* primary ray in index space for pixel (px,py) with film offset (jx,jy) in [0,1) */
void or_camera_ray(const or_camera* cam, const int64_t dims[3], int64_t px, int64_t py,
                   double jx, double jy, double o[3], double dir[3])
{
    int64_t m = dims[0];
    if (dims[1] > m) m = dims[1];
    if (dims[2] > m) m = dims[2];
    double M = (double)m;
    double fwd[3] = {cam->look[0] - cam->eye[0], cam->look[1] - cam->eye[1], cam->look[2] - cam->eye[2]};
    normalize3(fwd);
    double right[3], upv[3];
    cross3(fwd, cam->up, right);
    normalize3(right);
    cross3(right, fwd, upv);
    double aspect = (double)cam->width / (double)cam->height;
    double sx = 2.0 * ((double)px + jx) / (double)cam->width - 1.0;
    double sy = 1.0 - 2.0 * ((double)py + jy) / (double)cam->height;
    double w[3], d[3];
    if (cam->kind == OR_CAM_ORTHO) {
        double h = 0.5 * cam->fovy_or_height;
        for (int a = 0; a < 3; ++a) {
            w[a] = cam->eye[a] + sx * h * aspect * right[a] + sy * h * upv[a];
            d[a] = fwd[a];
        }
    } else {
        double th = tan(0.5 * cam->fovy_or_height * M_PI / 180.0);
        for (int a = 0; a < 3; ++a) {
            w[a] = cam->eye[a];
            d[a] = fwd[a] + sx * th * aspect * right[a] + sy * th * upv[a];
        }
        normalize3(d);
    }
    for (int a = 0; a < 3; ++a) { o[a] = w[a] * M - 0.5; dir[a] = d[a]; }
}

/* ---- emission-absorption marching (front to back) ----------------------- */
static void ea_pixel(const float* d, const int64_t dims[3], const or_camera* cam,
                     const or_medium* m, int64_t px, int64_t py, double out[4])
{
    double o[3], dir[3], tin, tout;
    or_camera_ray(cam, dims, px, py, 0.5, 0.5, o, dir);
    double C[3] = {0, 0, 0}, T = 1.0;
    if (or_clip_box(dims, o, dir, &tin, &tout)) {
        double dt = m->step;
        for (int64_t k = 0;; ++k) {
            double t = tin + ((double)k + 0.5) * dt;
            if (t >= tout) break;
            double p[3] = {o[0] + t * dir[0], o[1] + t * dir[1], o[2] + t * dir[2]};
            double s = or_trilinear(d, dims, p);
            if (s < 0.0) s = 0.0;
            if (s > 1.0) s = 1.0;
            double x = s * (double)(m->tf_n - 1);
            int64_t i0 = (int64_t)floor(x);
            if (i0 > m->tf_n - 2) i0 = m->tf_n - 2;
            double f = x - (double)i0;
            double rgba[4];
            for (int c = 0; c < 4; ++c)
                rgba[c] = (double)m->tf_rgba[4 * i0 + c] * (1.0 - f) + (double)m->tf_rgba[4 * (i0 + 1) + c] * f;
            double alpha = 1.0 - exp(-rgba[3] * dt);
            for (int c = 0; c < 3; ++c) C[c] += T * alpha * rgba[c];
            T *= 1.0 - alpha;
            if (T < 1e-6) break;
        }
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
}

/* ---- implicit ISO surface (the ray marcher of Section 5's ZFP comparison,
 * Fig. fig:zfp-comparison-iso; the paper names it only) ---------------------
 * The samples are those of the EA marcher, t_k = t_in + (k + 1/2) step; the
 * surface is the first change of inside = (f >= iso) between consecutive
 * samples, located by OR_ISO_BISECT halvings of that step, and shaded with
 * its normal n = -grad f / |grad f| (central differences, h = 1/2 voxel) as
 * rgb = (n + 1) / 2, alpha 1.  A ray without a change gives (0, 0, 0, 0). */
static void iso_pixel(const float* d, const int64_t dims[3], const or_camera* cam,
                      const or_medium* m, int64_t px, int64_t py, double out[4])
{
    double o[3], dir[3], tin, tout;
    or_camera_ray(cam, dims, px, py, 0.5, 0.5, o, dir);
    out[0] = out[1] = out[2] = out[3] = 0.0;
    if (!or_clip_box(dims, o, dir, &tin, &tout)) return;
    double dt = m->step, t_prev = 0.0;
    int prev = -1;
    for (int64_t k = 0;; ++k) {
        double t = tin + ((double)k + 0.5) * dt;
        if (t >= tout) return;
        double p[3] = {o[0] + t * dir[0], o[1] + t * dir[1], o[2] + t * dir[2]};
        int in = or_trilinear(d, dims, p) >= m->iso;
        if (prev >= 0 && in != prev) {
            double a = t_prev, b = t;     /* inside(a) = prev, inside(b) = in */
            for (int j = 0; j < OR_ISO_BISECT; ++j) {
                double mid = 0.5 * (a + b);
                double q[3] = {o[0] + mid * dir[0], o[1] + mid * dir[1], o[2] + mid * dir[2]};
                if ((or_trilinear(d, dims, q) >= m->iso) == prev) a = mid; else b = mid;
            }
            double th = 0.5 * (a + b);
            double h[3] = {o[0] + th * dir[0], o[1] + th * dir[1], o[2] + th * dir[2]};
            double g[3];
            for (int ax = 0; ax < 3; ++ax) {
                double pp[3] = {h[0], h[1], h[2]}, pm[3] = {h[0], h[1], h[2]};
                pp[ax] += 0.5;
                pm[ax] -= 0.5;
                g[ax] = or_trilinear(d, dims, pp) - or_trilinear(d, dims, pm);
            }
            double gl = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            double n[3];
            for (int ax = 0; ax < 3; ++ax) n[ax] = gl > 0.0 ? -g[ax] / gl : -dir[ax];
            for (int c = 0; c < 3; ++c) out[c] = 0.5 * (n[c] + 1.0);
            out[3] = 1.0;
            return;
        }
        prev = in;
        t_prev = t;
    }
}

/* ---- tracking ----------------------------------------------------------- */
typedef struct {
    const float* d;
    const int64_t* dims;
    const float* cmax;
    const or_medium* m;
    double inv_m;       /* 1 / M: densities are per world unit, the walk is in index units */
    uint32_t key[2];
    uint32_t pixel, sample;
} walk_ctx;

static void rng(const walk_ctx* w, uint32_t call, uint32_t stream, double u[4])
{
    uint32_t ctr[4] = {w->pixel, w->sample, call, stream}, r[4];
    or_philox4x32_10(ctr, w->key, r);
    for (int i = 0; i < 4; ++i) u[i] = or_u01(r[i]);
}

static double sigma_at(const walk_ctx* w, const double o[3], const double dir[3], double t)
{
    double p[3] = {o[0] + t * dir[0], o[1] + t * dir[1], o[2] + t * dir[2]};
    return w->m->density_scale * or_trilinear(w->d, w->dims, p) * w->inv_m;
}

static double majorant(const walk_ctx* w, int64_t cell)
{
    return w->m->density_scale * (double)w->cmax[cell] * w->inv_m;
}

/* Woodcock tracking over the macrocell grid (Section 4, with the DDA of
 * Szirmay-Kalos et al. 2011 that it cites): one optical depth
 * tau = -ln(1 - u0) is drawn per tentative collision and spent along the
 * ray, majorant times length per non-empty cell; where it runs out inside a
 * cell, the density there decides (u1) between a real collision (phase
 * function numbers u2, u3) and a new draw from that point.  Cells of zero
 * majorant neither consume tau nor draw.  Returns 1 on a real collision. */
static int delta_track(const walk_ctx* w, const double o[3], const double dir[3], double tmin,
                       double tmax, uint32_t* call, double* thit, double xi[2])
{
    dda_t s;
    dda_init(&s, w->dims, w->m->macrocell, o, dir, tmin, tmax);
    int64_t cell;
    double texit, tau = -1.0, u[4] = {0, 0, 0, 0};
    while (dda_cell(&s, &cell, &texit)) {
        double mj = majorant(w, cell);
        if (mj > 0.0 && texit > s.t) {
            double t = s.t;
            for (;;) {
                if (tau < 0.0) {
                    rng(w, (*call)++, 0, u);
                    tau = -log(1.0 - u[0]);
                }
                double reach = mj * (texit - t);
                if (!(tau < reach)) { tau -= reach; break; }
                t = t + tau / mj;
                tau = -1.0;
                if (u[1] * mj < sigma_at(w, o, dir, t)) {
                    *thit = t; xi[0] = u[2]; xi[1] = u[3];
                    return 1;
                }
            }
        }
        dda_advance(&s, texit);
    }
    return 0;
}

/* ratio tracking: the same free flights; every tentative collision
 * multiplies the transmittance by (1 - sigma / majorant) */
static double ratio_track(const walk_ctx* w, const double o[3], const double dir[3],
                          double tmin, double tmax, uint32_t* call)
{
    dda_t s;
    dda_init(&s, w->dims, w->m->macrocell, o, dir, tmin, tmax);
    int64_t cell;
    double texit, T = 1.0, tau = -1.0, u[4] = {0, 0, 0, 0};
    while (dda_cell(&s, &cell, &texit)) {
        double mj = majorant(w, cell);
        if (mj > 0.0 && texit > s.t) {
            double t = s.t;
            for (;;) {
                if (tau < 0.0) {
                    rng(w, (*call)++, 1, u);
                    tau = -log(1.0 - u[0]);
                }
                double reach = mj * (texit - t);
                if (!(tau < reach)) { tau -= reach; break; }
                t = t + tau / mj;
                tau = -1.0;
                T *= 1.0 - sigma_at(w, o, dir, t) / mj;
            }
        }
        dda_advance(&s, texit);
    }
    return T;
}

static int64_t max_dim(const int64_t dims[3])
{
    int64_t m = dims[0];
    if (dims[1] > m) m = dims[1];
    if (dims[2] > m) m = dims[2];
    return m;
}

double or_ratio_transmittance(const float* d, const int64_t dims[3], const float* cell_max,
                              const or_medium* m, const double o[3], const double dir[3],
                              uint32_t pixel, uint32_t sample, uint32_t* call,
                              const uint32_t key[2])
{
    walk_ctx w = {d, dims, cell_max, m, 1.0 / (double)max_dim(dims), {key[0], key[1]}, pixel, sample};
    double tin, tout;
    if (!or_clip_box(dims, o, dir, &tin, &tout)) return 1.0;
    return ratio_track(&w, o, dir, tin, tout, call);
}

static void pt_path(const walk_ctx* w, const or_camera* cam, int64_t px, int64_t py, double L[3])
{
    const or_medium* m = w->m;
    uint32_t call = 0, lcall = 0;
    double u[4];
    rng(w, call++, 0, u);
    double o[3], dir[3];
    or_camera_ray(cam, w->dims, px, py, u[0], u[1], o, dir);
    L[0] = L[1] = L[2] = 0.0;
    double beta = 1.0;
    double tin, tout;
    if (!or_clip_box(w->dims, o, dir, &tin, &tout)) {
        for (int c = 0; c < 3; ++c) L[c] = m->env_rad[c];
        return;
    }
    for (int bounce = 0; bounce < m->max_bounces; ++bounce) {
        double thit, xi[2];
        if (!delta_track(w, o, dir, tin, tout, &call, &thit, xi)) {
            for (int c = 0; c < 3; ++c) L[c] += beta * m->env_rad[c];
            return;
        }
        double x[3] = {o[0] + thit * dir[0], o[1] + thit * dir[1], o[2] + thit * dir[2]};
        beta *= m->albedo;
        /* light sample toward the directional light, attenuated by ratio tracking */
        double ltin, ltout;
        double T = 1.0;
        if (or_clip_box(w->dims, x, m->sun_dir, &ltin, &ltout))
            T = ratio_track(w, x, m->sun_dir, ltin, ltout, &lcall);
        double mu_l = dir[0] * m->sun_dir[0] + dir[1] * m->sun_dir[1] + dir[2] * m->sun_dir[2];
        double ph = or_hg_eval(mu_l, m->g);
        for (int c = 0; c < 3; ++c) L[c] += beta * ph * m->sun_rad[c] * T;
        if (bounce + 1 == m->max_bounces) return;
        /* scatter: new direction from the phase function around dir */
        double mu = or_hg_sample_mu(m->g, xi[0]);
        double phi = 2.0 * M_PI * xi[1];
        double nd[3];
        or_scatter_dir(dir, mu, phi, nd);
        for (int a = 0; a < 3; ++a) { o[a] = x[a]; dir[a] = nd[a]; }
        if (!or_clip_box(w->dims, o, dir, &tin, &tout)) {
            for (int c = 0; c < 3; ++c) L[c] += beta * m->env_rad[c];
            return;
        }
    }
}

void or_render_pixels(const float* d, const int64_t dims[3], const float* cell_max,
                      const or_camera* cam, const or_medium* m, int32_t spp, uint64_t seed,
                      const int64_t* pixels, int64_t npix, double* out_rgba)
{
    walk_ctx w = {d, dims, cell_max, m, 1.0 / (double)max_dim(dims),
                  {(uint32_t)seed, (uint32_t)(seed >> 32)}, 0, 0};
    for (int64_t n = 0; n < npix; ++n) {
        int64_t pix = pixels[n];
        int64_t px = pix % cam->width, py = pix / cam->width;
        double* out = out_rgba + 4 * n;
        if (m->mode == OR_MODE_EA) {
            ea_pixel(d, dims, cam, m, px, py, out);
            continue;
        }
        if (m->mode == OR_MODE_ISO) {
            iso_pixel(d, dims, cam, m, px, py, out);
            continue;
        }
        double acc[3] = {0, 0, 0};
        w.pixel = (uint32_t)pix;
        for (int32_t s = 0; s < spp; ++s) {
            double L[3];
            w.sample = (uint32_t)s;
            pt_path(&w, cam, px, py, L);
            for (int c = 0; c < 3; ++c) acc[c] += L[c];
        }
        for (int c = 0; c < 3; ++c) out[c] = acc[c] / (double)spp;
        out[3] = 1.0;
    }
}
