/*
 * oracle.h -- declarations of the CPU oracle (test infrastructure only).
 *
 * The oracle is a plain, slow, single-threaded restatement of what the paper
 * "GPU Volume Rendering with Hierarchical Compression Using VDB" (arXiv
 * 2504.04564) computes: the fixed-rate brick encoder of Section 3.1
 * (Algorithm 1, Eq. f1-f3), the VDB tree with prune of Section 3.2.1, the
 * decoded-value definition of Section 3.2.2, and the renderer of Section 4
 * (macrocell majorants, 3D-DDA, Woodcock/delta tracking), plus the ratio
 * tracker, emission-absorption marcher and learned leaf decoder that the
 * project adds around it.  Floating point is FP64 unless a quantization
 * decision fixes FP32 (leaf codecs), in which case the FP32 steps are written
 * out explicitly.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py (cpu_baseline and the
 * reference arm) may load this library.  It shares no code with the CUDA
 * path: not a header, not a table, not a helper.
 */
#ifndef VDB_ORACLE_H
#define VDB_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- counter-based RNG (Salmon et al., SC'11) -------------- */
void   or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u01(uint32_t u);

/* ---------------- encoder: Algorithm 1 and Section 3.2.1 ---------------- */
enum { OR_F1 = 1, OR_F2 = 2, OR_F3 = 3 };
enum { OR_FP32 = 0, OR_FP16 = 1, OR_FP8 = 2 };

uint32_t or_background_bits(const float* v, int64_t n);
void     or_brick_grid(const int64_t dims[3], int64_t nb[3]);
void     or_brick_ranges(const float* v, const int64_t dims[3],
                         uint32_t* lo_bits, uint32_t* hi_bits);
void     or_brick_scores(const uint32_t* lo_bits, const uint32_t* hi_bits, int64_t nbricks,
                         uint32_t b_bits, int metric, double* f, uint8_t* empty);
int64_t  or_brick_budget(int64_t nbricks, double ratio, int payload);
int64_t  or_select(const double* f, const uint8_t* empty, int64_t nbricks, int64_t n_budget,
                   uint8_t* active);
void     or_decode_dense(const float* v, const int64_t dims[3], const uint8_t* active,
                         uint32_t b_bits, int payload, float* out);

float    or_round_minifloat(float x, int ebits, int mbits, int bias, int saturate);
float    or_round_fp16(float x);
float    or_round_e4m3(float x);
void     or_quantize_leaf(const float in[512], int payload, float out[512],
                          float* scale, float* offset);

/* the 4-level tree with 2^5 upper, 2^4 lower and 2^3 leaf nodes */
typedef struct or_tree or_tree;
or_tree* or_tree_build(const float* v, const int64_t dims[3], const uint8_t* active,
                       uint32_t b_bits, int payload);
float    or_tree_value(const or_tree* t, int64_t i, int64_t j, int64_t k);
void     or_tree_counts(const or_tree* t, int64_t out[6]);
int      or_tree_leaf(const or_tree* t, int64_t li, int64_t lj, int64_t lk, float out[512]);
void     or_tree_free(or_tree* t);

/* ---------------- renderer: Section 4 plus the project's extensions ----- */
enum { OR_CAM_ORTHO = 0, OR_CAM_PINHOLE = 1 };
enum { OR_MODE_EA = 0, OR_MODE_PT = 1, OR_MODE_ISO = 2 };
enum { OR_ISO_BISECT = 12 };

typedef struct {
    int32_t kind;
    int32_t width, height;
    double  eye[3], look[3], up[3];
    double  fovy_or_height;   /* degrees (pinhole) or world height (ortho) */
} or_camera;

typedef struct {
    int32_t mode;
    int32_t tf_n;
    const float* tf_rgba;     /* tf_n RGBA entries, used by EA */
    double  step;             /* EA step, index units */
    double  density_scale;    /* extinction per world unit per unit density (PT) */
    double  albedo, g;
    int32_t max_bounces;
    int32_t macrocell;        /* macrocell edge in voxels */
    double  sun_dir[3], sun_rad[3], env_rad[3];
    double  iso;              /* ISO: the surface value */
} or_medium;

double or_trilinear(const float* d, const int64_t dims[3], const double p[3]);
void   or_macrocell_minmax(const float* d, const int64_t dims[3], int32_t cell,
                           float* mn, float* mx);
int    or_clip_box(const int64_t dims[3], const double o[3], const double dir[3],
                   double* tin, double* tout);
int64_t or_dda_cells(const int64_t dims[3], int32_t cell, const double o[3], const double dir[3],
                     double tmin, double tmax, int64_t* cells, double* t0, double* t1,
                     int64_t cap);
double or_hg_eval(double mu, double g);
double or_hg_sample_mu(double g, double xi);
void   or_onb(const double n[3], double b1[3], double b2[3]);
void   or_scatter_dir(const double dir[3], double mu, double phi, double out[3]);
void   or_camera_ray(const or_camera* cam, const int64_t dims[3], int64_t px, int64_t py,
                     double jx, double jy, double o[3], double dir[3]);
double or_ratio_transmittance(const float* d, const int64_t dims[3], const float* cell_max,
                              const or_medium* m, const double o[3], const double dir[3],
                              uint32_t pixel, uint32_t sample, uint32_t* call,
                              const uint32_t key[2]);
void   or_render_pixels(const float* d, const int64_t dims[3], const float* cell_max,
                        const or_camera* cam, const or_medium* m, int32_t spp,
                        uint64_t seed, const int64_t* pixels, int64_t npix,
                        double* out_rgba);

/* ---------------- learned leaf decoder (a project extension) ------------ */
int    or_mlp_num_params(void);
void   or_mlp_forward(const double* params, const double* inputs, int64_t n, double* out);
double or_mlp_loss_grad(const double* params, const double* inputs, const double* targets, int64_t n,
                        double* grad_params, double* grad_inputs);
void   or_adam_step(double* params, const double* grads, double* m, double* v, int64_t n, int64_t step,
                    double lr, double beta1, double beta2, double eps);
float  or_round_bf16(float x);
void   or_mlp_forward_bf16(const double* params, const double* inputs, int64_t n, double* out);
void   or_learned_leaf(const double* params, const float latent[16], const float src[512], float out[512]);
double or_mlp_loss_grad_bf16(const double* params, const double* inputs, const double* targets, int64_t n,
                             double* grad_params, double* grad_inputs);

#ifdef __cplusplus
}
#endif
#endif
