/*
 * vdbc.h -- C ABI of the GB300 (sm_103a) compressed-VDB volume renderer.
 *
 * Method: Zellmann et al., "GPU Volume Rendering with Hierarchical
 * Compression Using VDB" (arXiv 2504.04564).  A dense float32 volume is
 * encoded at a fixed rate into a four-level VDB tree by activating whole
 * 32^3 bricks in order of their distance from the background value
 * (Section 3.1, Algorithm 1, Eq. f1-f3; Section 3.2.1); a renderer then
 * samples the tree at arbitrary positions, decoding every lookup on the fly
 * (Section 3.2.2), with a macrocell majorant grid, a 3D-DDA and Woodcock
 * tracking (Section 4).
 *
 * Conventions shared by every call:
 *  - Every call returns a vdbc_status; nothing throws across the ABI.  On an
 *    error, vdbc_last_error() gives a message for the calling thread.
 *  - Volumes are x-fastest float32 arrays of dims[0]*dims[1]*dims[2] values.
 *    Voxel (i,j,k) sits at index coordinate (i,j,k); the volume is the box
 *    [-1/2, dim-1/2]^3.  World space scales index space so that the longest
 *    axis spans one unit: index = world * max(dims) - 1/2.
 *  - Pointers passed in are borrowed for the duration of the call (or until
 *    the work enqueued on `stream` completes, for device pointers).  Grids
 *    and plain-form volumes are owned by the library and freed only by their
 *    *_free call.  Image buffers are owned by the caller.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    that return device results enqueue their work on it and return without
 *    waiting; calls that return host results wait for it, polling with a
 *    wall-clock limit (VDBC_TIMEOUT_MS, default 600000 ms) after which they
 *    return VDBC_ERR_TIMEOUT.
 *  - After VDBC_ERR_TIMEOUT the call's GPU work is still queued on `stream`
 *    and may still read the call's inputs and write its outputs.  The
 *    library frees nothing that work uses: a handle the call would have
 *    returned (a grid, a batch) is not returned, and its memory is released
 *    once the work has finished (at the entry of a later call of this
 *    library).  The caller must keep every buffer it passed (host or device)
 *    and every handle it passed valid, and must not free those handles,
 *    until `stream` has been synchronized (cudaStreamSynchronize, or
 *    cudaStreamQuery returning cudaSuccess).  Once it has, the handles are
 *    usable as before and an output buffer holds what the call would have
 *    given.
 *  - Device kernels bound every loop; a path or lookup that exceeds its bound
 *    sets a device error word, which the next host-synchronizing call of the
 *    same handle reports as VDBC_ERR_DEVICE_FLAG.
 *  - A handle may be used from several threads only if the calls are
 *    serialized by the caller.
 *  - The library is also built with VDBC_CHECKED=1 (and VDBC_STATS, see
 *    vdbc_render_stats.events) as libvdbc_checked.so (vdbc_version() ends in
 *    "checked"): there every tree lookup checks each
 *    node, leaf and tile index against the grid's counts before it loads, and
 *    an index outside its table is read as the background and reported as
 *    VDBC_ERR_DEVICE_FLAG (bit 2 of vdbc_render_stats.error_flags) by the
 *    call that made it (encode, learn, decode, or a render that waits).
 *  - Host-side fault injection, for tests: VDBC_FAULT=oom (every device
 *    allocation fails), =format (every checksum mismatches), =timeout (every
 *    host wait times out), =bounds (checked builds only: vdbc_grid_load skips
 *    the node-table validation, so the lookup checks meet the bad entry).
 */
#ifndef VDBC_H
#define VDBC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VDBC_OK = 0,
    VDBC_ERR_INVALID_ARG = 1,   /* a null pointer, a bad size or an out-of-range parameter */
    VDBC_ERR_OOM = 2,           /* a device or host allocation failed */
    VDBC_ERR_CUDA = 3,          /* a CUDA runtime call failed; see vdbc_last_error() */
    VDBC_ERR_FORMAT = 4,        /* a grid file is truncated, of another version or corrupt */
    VDBC_ERR_TIMEOUT = 5,       /* a host wait ran past its wall-clock limit */
    VDBC_ERR_DEVICE_FLAG = 6,   /* a kernel hit one of its loop bounds (or, checked builds, an index bound) */
    VDBC_ERR_UNSUPPORTED = 7    /* valid request the build does not implement */
} vdbc_status;

/* similarity of a brick's value range [lo,hi] to the background B (Eq. f1-f3) */
enum { VDBC_F1 = 1,  /* closest:  min(|lo-B|, |hi-B|)  */
       VDBC_F2 = 2,  /* farthest: max(|lo-B|, |hi-B|)  */
       VDBC_F3 = 3   /* median:   |(lo+hi)/2 - B|      */ };

/* leaf payload: FP32 as in the paper; FP16 / FP8 (E4M3) with a per-leaf
 * FP32 scale and offset are a project extension (not in the paper), as is
 * VDBC_LEARNED: leaves decoded by a small shared network from a per-leaf
 * bf16 latent, with FP16 leaves as the fallback (vdbc_learn) */
enum { VDBC_FP32 = 0, VDBC_FP16 = 1, VDBC_FP8 = 2, VDBC_LEARNED = 3 };

enum { VDBC_CAM_ORTHO = 0, VDBC_CAM_PINHOLE = 1 };
enum { VDBC_MODE_EA = 0,   /* emission-absorption ray marching (fixed step) */
       VDBC_MODE_PT = 1,   /* delta tracking, ratio-tracked light, scattering */
       VDBC_MODE_ISO = 2   /* implicit ISO surface, normals as colour (Section 5's ZFP comparison) */ };
enum { VDBC_FILTER_TEXTURE = 0,  /* plain form: 3D CUDA texture, hardware trilinear */
       VDBC_FILTER_LINEAR = 1    /* plain form: linear device array, software trilinear */ };

typedef struct vdbc_grid vdbc_grid;      /* compressed grid: opaque, library-owned */
typedef struct vdbc_volume vdbc_volume;  /* plain form of a dense volume: opaque, library-owned */

/* a dense input volume, x fastest; data is a device pointer if on_device != 0 */
typedef struct {
    int32_t dims[3];
    int32_t on_device;
    const float* data;
} vdbc_dense;

typedef struct {
    double  ratio;      /* R of the target rate 1:R, R >= 1; 1 keeps every non-empty brick */
    int32_t metric;     /* VDBC_F1, VDBC_F2 (default when 0) or VDBC_F3 */
    int32_t payload;    /* VDBC_FP32, VDBC_FP16 or VDBC_FP8 */
    int32_t macrocell;  /* edge of a majorant macrocell in voxels, 1..128; 0 means 8 */
    int32_t reserved;
} vdbc_encode_params;

typedef struct {
    int32_t  dims[3];
    int32_t  payload;
    int32_t  macrocell;
    int32_t  metric;
    uint32_t background_bits;  /* bit pattern of the background value B */
    int32_t  reserved;
    double   ratio;
    int64_t  n_bricks;         /* ceil(dims / 32) brick grid size */
    int64_t  n_nonempty;       /* bricks whose range is not exactly [B,B] */
    int64_t  budget;           /* N = floor(n_bricks * 131072 / (ratio * brick payload bytes)) */
    int64_t  n_active;         /* bricks activated = min(budget, n_nonempty) */
    int64_t  n_upper, n_lower, n_leaves, n_tiles;
    int64_t  n_neural;         /* learned grids: leaves decoded by the network (n_leaves = fallbacks) */
    uint64_t payload_bytes;    /* leaf values plus per-leaf scale/offset (and latents + network) */
    uint64_t node_bytes;       /* root, upper and lower tables plus tile values */
    uint64_t total_bytes;      /* everything the grid holds on the device, incl. majorants */
} vdbc_grid_info;

typedef struct {
    int32_t kind;              /* VDBC_CAM_ORTHO or VDBC_CAM_PINHOLE */
    int32_t width, height;     /* image size in pixels, 1..16384 each */
    int32_t reserved;
    double  eye[3];            /* world space */
    double  look[3];           /* a world point the camera looks at */
    double  up[3];
    double  fovy_or_height;    /* vertical field of view in degrees (pinhole) or
                                  world height of the image (ortho) */
} vdbc_camera;

typedef struct {
    int32_t mode;              /* VDBC_MODE_EA, VDBC_MODE_PT or VDBC_MODE_ISO */
    int32_t tf_n;              /* EA: number of RGBA entries of the transfer function, 2..2048 */
    const float* tf_rgba;      /* EA: host pointer to tf_n RGBA float entries; alpha is
                                  the extinction per voxel length */
    float   step;              /* EA, ISO: step in voxels (> 0) */
    float   density_scale;     /* PT: extinction per world unit at density 1 */
    float   albedo;            /* PT: single-scattering albedo in [0,1] */
    float   g;                 /* PT: Henyey-Greenstein asymmetry in (-1,1) */
    int32_t max_bounces;       /* PT: scattering events per path, 1..4096 */
    float   iso;               /* ISO: the surface value (finite) */
    float   sun_dir[3];        /* PT: unit direction toward the directional light */
    float   sun_rad[3];        /* PT: its irradiance (RGB) */
    float   env_rad[3];        /* PT: constant environment radiance (RGB) */
} vdbc_medium;

/* counters of the last render on a handle (read after the stream completes) */
typedef struct {
    uint64_t lookups;          /* density lookups (trilinear reconstructions) */
    uint64_t paths;
    uint64_t error_flags;      /* nonzero if a kernel hit one of its bounds */
    uint64_t events[8];        /* only in builds with VDBC_STATS defined (the checked build
                                  libvdbc_checked.so is one), else 0: tracker loop iterations,
                                  DDA cells examined, coarse blocks crossed, free flights
                                  drawn, rays started, paths fetched, leaf queries to the
                                  per-thread accessor, tree descents (the queries its cached
                                  leaf did not answer; queries - descents = descents saved) */
    float    kernel_ms;        /* duration of the last render's tracker kernel (k_pt, k_pt_batch,
                                  k_ea or k_iso), from CUDA events recorded around its launch on
                                  the render's stream; -1 if none was recorded */
    int32_t  reserved;
} vdbc_render_stats;

/*
 * vdbc_encode -- fixed-rate compression of a dense volume into a VDB grid.
 * Paper: Section 3.1, Algorithm 1 (histogram -> background B, 32^3 brick
 * ranges, sort by Eq. f1-f3, activate the first bricks up to the rate) and
 * Section 3.2.1 (always set the two extreme corner voxels; prune).
 *   in      dense volume (host or device pointer, x fastest); borrowed.
 *   params  rate, metric, payload, macrocell edge.
 *   stream  work is enqueued here; the call waits once for the tree sizes.
 *   out     receives a new grid handle; free with vdbc_grid_free.
 * Errors: INVALID_ARG for null pointers, dims < 1 or > 8192, ratio < 1 or not
 * finite, unknown metric/payload, or non-finite voxel values; OOM; CUDA.
 */
vdbc_status vdbc_encode(const vdbc_dense* in, const vdbc_encode_params* params, void* stream,
                        vdbc_grid** out);

/* vdbc_grid_get_info -- sizes and counts of a grid (host struct, no device work). */
vdbc_status vdbc_grid_get_info(const vdbc_grid* grid, vdbc_grid_info* info);

/*
 * vdbc_grid_decode -- the decoded grid D at every voxel (the value the
 * sampler of Section 3.2.2 reconstructs from: the voxel where the tree holds
 * it, a tile or the background elsewhere), x fastest.
 *   out        dims[0]*dims[1]*dims[2] floats, device pointer if out_on_device else host.
 * Errors: INVALID_ARG; CUDA; TIMEOUT (host output only).
 */
vdbc_status vdbc_grid_decode(const vdbc_grid* grid, float* out, int32_t out_on_device, void* stream);

/* vdbc_grid_active_bricks -- 1 byte per brick (x fastest): 1 if Algorithm 1
 * activated it.  host_out holds info.n_bricks bytes. */
vdbc_status vdbc_grid_active_bricks(const vdbc_grid* grid, uint8_t* host_out);

/* vdbc_grid_macrocells -- per macrocell min and max of D over the cell's voxels
 * dilated by one voxel (the majorant ranges of Section 4); host arrays of
 * prod(ceil(dims / macrocell)) floats each. */
vdbc_status vdbc_grid_macrocells(const vdbc_grid* grid, float* host_min, float* host_max);

/*
 * vdbc_grid_save / vdbc_grid_load -- the grid as one linear, pointer-free
 * block (the property Section 2.3 and Section 3.2.1 rely on for copying
 * NanoVDB grids with memcpy), behind a versioned header and a checksum.  No
 * entropy coding, so the file keeps random access (Section 5.5).
 * vdbc_grid_load checks the whole file on the host (magic, version, sizes,
 * checksum, table offsets against the layout the header's counts give), then
 * every root, upper and lower entry on the device against the table it
 * indexes, before it returns the grid.
 * Errors: INVALID_ARG; FORMAT (bad magic, version, size, checksum or table
 * layout, or a node entry outside its table); OOM; CUDA.
 */
vdbc_status vdbc_grid_save(const vdbc_grid* grid, const char* path);
vdbc_status vdbc_grid_load(const char* path, void* stream, vdbc_grid** out);
void        vdbc_grid_free(vdbc_grid* grid);

/*
 * vdbc_render -- render the compressed grid, one thread per light path,
 * every density lookup decoded on the fly (Section 3.2.2: tree descent with
 * a cached accessor, leaf decode, trilinear reconstruction; Section 4:
 * macrocell majorants, 3D-DDA, Woodcock tracking, volumetric scattering).
 *   mode EA: one ray per pixel through the pixel centre, front-to-back
 *            emission-absorption with a fixed step; spp must be 1.
 *   mode PT: spp paths per pixel, Philox counter (pixel, sample, call,
 *            stream) keyed by seed; light from a directional source by ratio
 *            tracking plus a constant environment.
 *   mode ISO: the implicit ISO-surface marcher the paper uses for its ZFP
 *            comparison (Section 5, fig:zfp-comparison-iso), which it names
 *            without details: one ray per pixel centre, samples t_k = t_in +
 *            (k + 1/2) step; the first change of (f >= iso) between
 *            consecutive samples is halved 12 times and shaded with its
 *            normal n = -grad f / |grad f| (central differences, 1/2 voxel)
 *            as rgb = (n + 1) / 2, alpha 1; rays without one give 0.
 *            Macrocells whose [min, max] excludes iso are crossed without
 *            lookups (the result is the plain march's); spp must be 1.
 *   rgba_out width*height*4 floats (RGBA per pixel, row 0 at the top),
 *            device pointer if out_on_device else host (the call then waits).
 * Errors: INVALID_ARG (null pointers; an image outside 1..16384 a side; a
 * camera without a basis: non-finite vectors, look == eye, up along the
 * view, a field of view outside (0, 180) degrees or a non-positive ortho
 * height; spp outside 1..65536 for PT or not 1 for EA/ISO; a PT medium with
 * a negative or non-finite density scale, albedo outside [0, 1], g outside
 * (-1, 1), max_bounces outside 1..4096, a zero or non-finite sun direction or
 * non-finite radiance; an EA transfer function of fewer than 2 or more than
 * 2048 entries; a non-positive step; a non-finite iso value); OOM; CUDA;
 * TIMEOUT; DEVICE_FLAG.
 */
vdbc_status vdbc_render(const vdbc_grid* grid, const vdbc_camera* camera, const vdbc_medium* medium,
                        int32_t spp, uint64_t seed, float* rgba_out, int32_t out_on_device,
                        void* stream);

/* vdbc_render_stats_get -- counters of the last vdbc_render on this grid;
 * waits for `stream`. */
vdbc_status vdbc_render_stats_get(const vdbc_grid* grid, void* stream, vdbc_render_stats* stats);

/*
 * vdbc_volume_create -- the plain form the paper compares against (Section
 * 5.3: the structured volume in a 3D CUDA texture) or, with
 * VDBC_FILTER_LINEAR, a linear device copy sampled by the same software
 * trilinear as the grid.  Builds the same macrocell majorant grid from the
 * dense values (macrocell edge 1..128 voxels, 0 means 8).
 */
vdbc_status vdbc_volume_create(const vdbc_dense* in, int32_t filter, int32_t macrocell,
                               void* stream, vdbc_volume** out);
void        vdbc_volume_free(vdbc_volume* vol);

/* vdbc_render_dense -- vdbc_render on the plain form; identical arguments and
 * tracking code, only the sampler differs. */
vdbc_status vdbc_render_dense(const vdbc_volume* vol, const vdbc_camera* camera,
                              const vdbc_medium* medium, int32_t spp, uint64_t seed,
                              float* rgba_out, int32_t out_on_device, void* stream);
vdbc_status vdbc_volume_render_stats_get(const vdbc_volume* vol, void* stream,
                                         vdbc_render_stats* stats);

/*
 * vdbc_select_bricks_noalloc -- for callers that cannot allocate device memory
 * while they run (a renderer inside a host application that owns the whole
 * device-memory budget and forbids allocation after start-up, or a frame loop
 * that cannot afford the implicit synchronization of cudaMalloc / cudaFree).
 * The paper has no counterpart: this is the brick-selection phase of
 * vdbc_encode (the histogram for the background B, the 32^3 brick ranges, the
 * f scores and the choice of the bricks to activate) with all its scratch in
 * one fixed array inside the library (about 1.6 MiB, held on every GPU that
 * loads the library until the process exits).  Nothing is allocated.
 *   in                    dense volume in DEVICE memory (on_device must be 1)
 *   params                ratio, metric and payload as for vdbc_encode
 *   background_bits_out   device pointer to one uint32: bit pattern of B
 *   active_out            device pointer to n_bricks bytes: 1 = activated
 *   counts_out            device pointer to three int64: number of non-empty
 *                         bricks, number activated, nonzero if the volume held
 *                         non-finite values (the other outputs are then invalid)
 * Results equal vdbc_encode's (vdbc_grid_get_info, vdbc_grid_active_bricks).
 * The work is enqueued on `stream`; the call does not wait.  The first call on
 * a device looks up the array's device address; make that call before any
 * stream capture.  Every call reuses the same array, so calls whose GPU work
 * overlaps (different streams, or unordered threads) race: serialize them.
 * The caller guarantees the outputs' lengths (active_out: one byte per 32^3
 * brick, ceil(nx/32) * ceil(ny/32) * ceil(nz/32)); the call checks that the
 * volume and every output are device (or managed) memory, aligned for their
 * element types.
 * Errors: INVALID_ARG for null pointers, a host volume, dims outside 1..8192,
 * bad ratio/metric/payload, more than 65,536 bricks (the array's limit:
 * 1024 x 1024 x 2048 voxels is exactly 65,536 and accepted, one more brick
 * along any axis is refused), or an input or output that is not device
 * memory or is misaligned; CUDA.
 */
vdbc_status vdbc_select_bricks_noalloc(const vdbc_dense* in, const vdbc_encode_params* params,
                                       uint32_t* background_bits_out, uint8_t* active_out,
                                       int64_t* counts_out, void* stream);

/* ---------------- many volumes in one launch (a project extension) ------ */
/* one render job of a batch: a grid, its own camera, medium (PT), spp per
 * frame and seed; rgba_out (device, width*height*4 floats) receives the
 * running mean over the frames rendered so far */
typedef struct {
    const vdbc_grid* grid;
    vdbc_camera camera;
    vdbc_medium medium;
    int32_t spp;
    int32_t reserved;
    uint64_t seed;
    float* rgba_out;
} vdbc_job;

/* launch shape of the batched path tracer, chosen by the autotuner */
typedef struct {
    int32_t threads;       /* threads per block: 128 or 256 */
    int32_t chunk;         /* paths a warp takes from the work counter at once (>= 32);
                              chunk / 32 is the paths each lane claims per refill */
    int32_t coarse;        /* 1: cross empty 8^3 blocks of macrocells in one DDA step */
    int32_t depth;         /* accessor cache depth: 1 the last leaf, 2 also its lower node */
    float   frame_ms;      /* the tuner's time for every 8th path of a frame with this shape */
} vdbc_tuning;

typedef struct vdbc_batch vdbc_batch;

/*
 * vdbc_batch_create -- prepare a batch of up to 64 path-tracing jobs on
 * grids of any size and payload, rendered together per frame by one
 * persistent launch for each payload type present (FP32, FP16, FP8), each
 * specialised on its sampler (Section 4's tracker; the paper renders one
 * volume at a time).  With autotune != 0 the launch shape is chosen by timing
 * every 8th path of a frame per candidate (cached per GPU and batch layout in
 * this process, and in the file named by VDBC_TUNE_CACHE when set).  The
 * per-frame work (work-counter resets, the persistent trackers, per-pixel
 * accumulation) is then captured in one CUDA graph on `stream`.  Grids must outlive the batch.  Errors: INVALID_ARG
 * (n outside 1..64, a null grid or output, EA media, bad spp/camera/medium);
 * OOM; CUDA.
 */
vdbc_status vdbc_batch_create(const vdbc_job* jobs, int32_t n, int32_t autotune, void* stream,
                              vdbc_batch** out);
/* renders `frames` more progressive frames of every job (frame f uses sample
 * ids [f*spp, (f+1)*spp), so F frames equal one render with F*spp samples)
 * by replaying the captured graph; does not wait */
vdbc_status vdbc_batch_render_frames(vdbc_batch* batch, int32_t frames, void* stream);
/* restarts the accumulation at frame 0 */
vdbc_status vdbc_batch_reset(vdbc_batch* batch, void* stream);
/* progressive accumulation state, for checkpoints: the frame counter and
 * every job's per-pixel radiance sums (4 floats a pixel: the r, g, b sums
 * and an unused one; jobs in order, pixels row-major), *floats in all.
 * get_state copies it to host memory and waits for `stream`; set_state
 * restores one taken from a batch of the same jobs (host memory, frame >= 0)
 * and waits, after which F more frames give the images of a batch that
 * rendered frame + F frames in one go. */
vdbc_status vdbc_batch_state_size(const vdbc_batch* batch, int64_t* floats);
vdbc_status vdbc_batch_get_state(const vdbc_batch* batch, int32_t* frame, float* host_sums, void* stream);
vdbc_status vdbc_batch_set_state(vdbc_batch* batch, int32_t frame, const float* host_sums, void* stream);
vdbc_status vdbc_batch_get_tuning(const vdbc_batch* batch, vdbc_tuning* tuning);
/* counters of the last frame; waits for `stream` */
vdbc_status vdbc_batch_stats_get(const vdbc_batch* batch, void* stream, vdbc_render_stats* stats);
void        vdbc_batch_free(vdbc_batch* batch);

/* ---------------- learned leaf codec (a project extension) -------------- */
/*
 * The paper's Section 2.3 mentions network-decoded leaves (NeuralVDB) only as
 * related work, too slow there for real-time rendering.  Here a leaf may be
 * "neural": it stores a 16-value bf16 latent z and its (scale, offset), and
 * voxel (i, j, k) of the leaf decodes to
 *     offset + scale * clamp(y, 0, 1),
 *     y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3,  x = (i/7, j/7, k/7, z),
 * one network (19 -> 32 -> 32 -> 1, 1729 FP32 parameters in the order W1
 * (32x19 row major), b1, W2 (32x32), b2, w3, b3) shared by all leaves.
 * Rendering evaluates it on the tensor cores with bf16 inputs, weights and
 * hidden activations and FP32 accumulation, at each of the 8 trilinear
 * corners that falls in a neural leaf; a leaf that the network cannot
 * represent within the error bound keeps a raw FP16 payload instead.
 */
/* training state of vdbc_learn, for checkpoints: device arrays the caller
 * owns.  Latent arrays are per leaf POSITION like init_latents (16 floats
 * each); in a saved state, positions without a leaf hold 0. */
typedef struct {
    float*  params;      /* 1729 network parameters */
    float*  params_m;    /* their Adam first moments */
    float*  params_v;    /* their Adam second moments */
    float*  latents;     /* 16 per leaf position */
    float*  latents_m;   /* the latents' Adam first moments */
    float*  latents_v;   /* the latents' Adam second moments */
    int64_t step;        /* Adam steps taken so far */
} vdbc_learn_state;

typedef struct {
    int32_t  steps;             /* Adam steps (0: keep the initial network and latents) */
    int32_t  samples_per_leaf;  /* S: voxels drawn per leaf per step, 16, 32, 64 or 128 */
    float    lr;                /* Adam step size of the network (beta1 0.9, beta2 0.999, eps 1e-8) */
    float    lr_latent;         /* Adam step size of the latents */
    float    max_error;         /* a leaf whose largest |decoded - source| exceeds this is a raw candidate */
    int32_t  reserved;
    uint64_t max_bytes;         /* size limit of the whole learned grid (0: none); raw candidates beyond
                                   it stay neural, the largest errors (then the lowest leaf numbers) kept raw */
    uint64_t seed;              /* Philox key of the initialisation and of the voxel draws */
    const float*   init_params;   /* device, 1729 floats, or NULL: weights uniform in +-sqrt(6/fan_in)
                                     (counter (i, 0, 0, 0x494E4954)), biases 0, b3 = 1/2 */
    const float*   init_latents;  /* device, 16 floats per leaf POSITION (lk*nly + lj)*nlx + li with
                                     nl = ceil(dims/8), or NULL: zeros */
    const uint8_t* force;         /* device, one byte per leaf position: 0 by error, 1 neural, 2 raw; or NULL */
    const vdbc_learn_state* resume; /* or NULL: continue from this state (then init_params and
                                       init_latents must be NULL); step t of the call counts as step
                                       resume->step + t in the voxel draws and Adam's bias corrections */
    vdbc_learn_state* save;       /* or NULL: receives the state after the last step */
} vdbc_learn_params;

/*
 * vdbc_learn -- fit the network and one latent per leaf of `src` (any
 * non-learned payload) to the leaves' values normalised by their
 * (scale, offset), and build the learned grid *out (free with
 * vdbc_grid_free; payload VDBC_LEARNED, n_leaves = raw leaves, n_neural =
 * neural leaves).  Training minimises the mean squared error of y against
 * (v - offset) / scale with Adam over `steps` steps (the gradient as in
 * vdbc_learn_loss_grad); step t (from 0) uses,
 * for every leaf not forced raw, voxel s*(512/S) + (r mod 512/S) for
 * s = 0..S-1, r the first word of Philox4x32-10 at counter
 * (leaf position, t, s, 0x4C454146) and key `seed`; the latents' gradient
 * is the sum over the leaf's samples.  Tree tables, tiles and the
 * background are those of `src`.  loss_out (host, `steps` doubles, or
 * NULL) receives the loss of each step.  Training state can be saved and
 * resumed: A steps with `save`, then B steps with `resume` from it, give the
 * same losses, final state and grid, bit for bit, as A + B steps in one call
 * (same src, S, learning rates and seed).  Waits for `stream`.
 * Errors: INVALID_ARG (null, a learned source, steps outside 0..1e6, S not
 * 16/32/64/128, non-positive learning rates, negative max_error, a state
 * with a null array or a step outside 0..2^31-1-steps, resume together with
 * init_params or init_latents); OOM; CUDA.
 */
vdbc_status vdbc_learn(const vdbc_grid* src, const vdbc_learn_params* params, void* stream, vdbc_grid** out,
                       double* loss_out);

/*
 * vdbc_learn_loss_grad -- the training kernels on explicit samples: loss =
 * mean over the n rows of (y - target)^2, grad_params (1729) its gradient,
 * grad_inputs (n x 19, or NULL) the gradient with respect to each input row.
 * params, inputs (n x 19 row major), targets, grad_* are device arrays; loss
 * a host double (or NULL).  Tensor-core arithmetic at the network's own
 * precision: y as the render evaluates it, the backward operands (dh2, dh1,
 * h1, x, weights) rounded to bf16, FP32 sums in a fixed order.  Waits for
 * `stream`.  Errors: INVALID_ARG (null arrays, n outside 1..2^31); CUDA.
 */
vdbc_status vdbc_learn_loss_grad(const float* params, const float* inputs, const float* targets, int64_t n,
                                 double* loss, float* grad_params, float* grad_inputs, void* stream);

/* the 1729 FP32 parameters of a learned grid's network (host array) */
vdbc_status vdbc_learn_get_params(const vdbc_grid* grid, float* host_params);

/* vdbc_philox -- n outputs of the device Philox4x32-10 (the generator every
 * render draws from), for checking it against its published definition.
 * ctr: 4*n counters, key: 2 words, out: 4*n words; all host arrays. */
vdbc_status vdbc_philox(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, int32_t n);

/* vdbc_compare -- error of one float array against another, summed in FP64
 * on the device: `count` elements of `stride` floats each, of which the first
 * `channels` are compared (an RGBA image: stride 4, channels 3; a volume:
 * stride 1, channels 1).  mse = mean squared difference over the count *
 * channels values, rmse its root, mean_abs / max_abs the mean and largest
 * absolute difference, psnr = 10 log10(1 / mse) (peak 1, the convention of
 * the paper's Table tab:stats; infinite when the arrays are equal), n the
 * number of values.  a and b are device arrays; the call waits for `stream`
 * (a fixed summation order: the same result every run).
 * Errors: INVALID_ARG (null pointers, count < 0, channels outside
 * 1..stride); OOM; CUDA; TIMEOUT. */
typedef struct {
    double mse, rmse, mean_abs, max_abs, psnr;
    int64_t n;
} vdbc_error_stats;
vdbc_status vdbc_compare(const float* a, const float* b, int64_t count, int32_t stride, int32_t channels,
                         void* stream, vdbc_error_stats* out);

/* number of kernels this library has launched in the process so far (every
 * launch increments it on the host); for counting device work per step */
uint64_t    vdbc_kernel_launches(void);

/* message of the last failed call on this thread ("" if none) */
const char* vdbc_last_error(void);
/* library version, e.g. "vdbc 0.1.0 sm_103a" */
const char* vdbc_version(void);

#ifdef __cplusplus
}
#endif
#endif
