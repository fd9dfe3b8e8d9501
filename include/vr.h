/*
 * vr.h -- C ABI of libvr, a direct volume ray caster for NVIDIA GB300 (sm_103a).
 *
 * The method is the one described in N. Kopal, "Volume Raycasting mit OpenCL" (2011,
 * arXiv:1609.01317), §3.10 "Gesamtaufbau eines Raycasters": for every pixel cast a ray,
 * intersect it with the bounding box (§3.3, §3.6), sample the volume at regular spacing
 * with trilinear interpolation (§3.4, Eq. 2), estimate a gradient with the central
 * difference, Sobel3D or Zucker-Hummel operator (§3.5, Eq. 3, Eq. 4), look up colour and
 * opacity in a transfer-function table (§3.7), shade with a point light (§3.8, Listing 3,
 * extended to Phong) and composite with the transparency formula (§3.9, Eq. 6) front to
 * back with early ray termination.  Empty space is skipped with per-brick min/max tables
 * (§5.3 "Empty-Space-Skipping", §5.4 "Octree").  A hand-written adjoint makes the image
 * differentiable with respect to voxel values and transfer-function entries.
 *
 * General conventions (apply to every entry point unless stated otherwise):
 *   - Every call returns a vr_status.  Argument errors are detected before any work is
 *     queued and leave the context unchanged (VR_ERR_INVALID_ARG, VR_ERR_UNSUPPORTED,
 *     VR_ERR_STATE).  CUDA errors, including asynchronous ones from earlier launches, are
 *     reported as VR_ERR_CUDA by the next call that checks.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work is queued
 *     on it and is asynchronous unless the call says it synchronises.
 *   - Caller buffers are never freed or retained past the call; buffers the library needs
 *     (padded volume, brick tables, transfer function, staging, adjoint scratch) come from
 *     the allocator given to vr_create and are released by vr_destroy.  Besides, each
 *     context holds 8 bytes of mapped pinned host memory (cudaHostAlloc) into which each
 *     render's march writes the visible-brick count it saw; the next render reads it to
 *     choose between two marches that give the same pixels.
 *   - Volumes are dense x-fastest arrays: voxel (x, y, z) is element x + nx*(y + ny*z)
 *     and sits at world point (x, y, z) (unit spacing, §2.1 Eq. 1).
 *   - Alignment: a voxel array must be aligned to its element size; device images, image
 *     gradients and a transfer function read in place (vr_render_noalloc) are accessed as
 *     16-byte RGBA vectors and must be 16-byte aligned; other device float arrays (volume
 *     and table gradients, depths, probe points) 4-byte aligned.  A misaligned pointer is
 *     rejected with VR_ERR_INVALID_ARG before any work is queued.
 *   - Images are H x W x 4 float32 RGBA, row-major, row 0 at the top; RGB is
 *     premultiplied over black and A = 1 - transmittance.
 *   - A context may be used from one host thread at a time, and its calls must be ordered
 *     on the device: issue them on one stream (or order the streams yourself).  Separate
 *     contexts on separate streams run concurrently (e.g. one frame's uploads overlapping
 *     the previous frame's rendering).
 *   - The first-hit surface renderer (vr_render_surface, §3.11 and §5.1) is the paper's own
 *     renderer; vr_render is the full method of §3.10 with the transparency formula.
 */
#ifndef VR_H
#define VR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vr_ctx vr_ctx;

typedef enum {
    VR_OK = 0,
    VR_ERR_INVALID_ARG = 1,   /* a pointer, size or parameter is out of its range      */
    VR_ERR_OUT_OF_MEMORY = 2, /* the allocator returned NULL                           */
    VR_ERR_CUDA = 3,          /* a CUDA call failed (text via vr_last_cuda_error)      */
    VR_ERR_UNSUPPORTED = 4,   /* valid request the library does not implement         */
    VR_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up                    */
    VR_ERR_STATE = 6          /* call order violated (no volume / no TF / no camera,   */
                              /* or checkpoints that do not match the current state)   */
} vr_status;

/* Voxel storage types (§3.2: CT data are 12-bit values in 16-bit shorts). */
typedef enum { VR_U8 = 0, VR_U16 = 1, VR_F16 = 2, VR_F32 = 3 } vr_dtype;

/* Gradient operators of §3.5. */
typedef enum {
    VR_GRAD_CENTRAL = 0,      /* Eq. 3, 6 taps                                          */
    VR_GRAD_SOBEL3D = 1,      /* Eq. 4, weights 1,3,6 per plane, 54 taps                */
    VR_GRAD_ZUCKER_HUMMEL = 2 /* 54 taps, weight of neighbour (+-1,b,c) = +-1/sqrt(1+b^2+c^2) */
} vr_grad;

/* Pinhole or orthographic camera (§3.3: one ray through every pixel).
 *   fwd = normalize(target - eye), right = normalize(fwd x up), up' = right x fwd.
 *   Pixel (px, py) has screen coordinates u = (2(px+1/2)/W - 1) * ax and
 *   v = (1 - 2(py+1/2)/H) * ay, with ay = tan(fov_y/2) (perspective) or ortho_height/2
 *   (orthographic) and ax = ay * W / H.
 *   Perspective: origin eye, direction normalize(fwd + u right + v up').
 *   Orthographic: origin eye + u right + v up', direction fwd.
 * The ray setup is evaluated in FP32 with every operation rounded separately, so the
 * integer sample count of each ray is reproducible on any IEEE-754 machine. */
typedef struct {
    float eye[3], target[3], up[3];
    int ortho;          /* 0 = perspective, 1 = orthographic                          */
    float fov_y_deg;    /* perspective vertical field of view, in (0, 180)            */
    float ortho_height; /* orthographic image height in world units, > 0              */
    int width, height;  /* image size in pixels, 1 .. 16384 each                      */
} vr_camera;

/* Per-render parameters. */
typedef struct {
    float step;          /* sample spacing along the unit ray direction, > 0 (§3.3)     */
    int grad;            /* vr_grad                                                     */
    float ka, kd, ks;    /* Phong ambient / diffuse / specular coefficients             */
    float shininess;     /* Phong exponent, >= 0                                        */
    float light[3];      /* point-light position (§3.8), used when headlight == 0       */
    int headlight;       /* 1: the light sits at the eye                                */
    float ert_threshold; /* stop a ray once 1 - T >= this, in (0, 1]; > 1 never stops   */
    int skip_empty;      /* 1: skip bricks whose opacity is zero for the current TF    */
    float clip_lo[3];    /* clip box (§3.6), intersected with [0, n-1]^3               */
    float clip_hi[3];
    int collect_stats;   /* 1: count rays and samples (read with vr_read_stats)         */
    /* Adaptive sampling (§5.2: coarser sampling in detail-poor regions), 0 = off.  With it
     * on, each 32^3-voxel region gets a multiplier m: 4 if the raw value range (max - min)
     * of its footprint [32r - 1, 32r + 33] is <= adapt_range4, else 2 if <= adapt_range2,
     * else 1 (a negative bound disables its level); sample k is taken iff
     * k mod m(region of sample k) == 0 and its opacity is corrected to 1 - (1 - a)^m (it
     * stands for m samples).  Only vr_render
     * supports it (VR_ERR_UNSUPPORTED elsewhere).  The sample counters still count every
     * sample of the regular grid up to termination (rays_hit, samples_plain) and the
     * samples taken (samples_visited). */
    int adaptive;
    float adapt_range2, adapt_range4;
    /* Which march a plain render (vr_render / vr_render_rows without adaptive sampling) runs;
     * every choice gives the same image bit for bit:
     *   VR_MARCH_AUTO (0)    as RECORDS (the faster of the two on every workload measured);
     *   VR_MARCH_RECORDS (1) the per-voxel gradient records of the visible bricks are
     *                        computed into device memory (kept until the volume, operator
     *                        or transfer function changes) and read by the tile march, or
     *                        for sparse data by the ray-list march;
     *   VR_MARCH_SLABS (2)   each 16 x 16 pixel tile walks the volume in slabs, staging the
     *                        raw voxels it crosses and their records in shared memory (no
     *                        record table in device memory), when the camera's rays lie
     *                        close enough together for a tile's region to fit; else as
     *                        RECORDS.  vr_read_stats reports which one ran.
     * Other values: INVALID_ARG. */
    int march;
} vr_render_params;

enum { VR_MARCH_AUTO = 0, VR_MARCH_RECORDS = 1, VR_MARCH_SLABS = 2 };

/* Sample counters of the most recent render with collect_stats = 1. */
typedef struct {
    unsigned long long rays_hit;        /* rays with at least one sample               */
    unsigned long long samples_plain;   /* samples the plain method marches: every     */
                                        /* t_k up to early termination, skipped or not */
    unsigned long long samples_visited; /* samples actually interpolated               */
    unsigned long long samples_shaded;  /* samples with opacity != 0 (gradient+Phong)  */
    unsigned long long march;           /* the march that rendered it: VR_MARCH_RECORDS */
                                        /* or VR_MARCH_SLABS                            */
} vr_stats;

/* Device allocator callback pair: alloc returns device memory aligned to 256 bytes or
 * NULL; free releases it.  Both may be NULL to use cudaMalloc / cudaFree. */
typedef void *(*vr_alloc_fn)(size_t bytes, void *user);
typedef void (*vr_free_fn)(void *ptr, void *user);

/* Create a context on CUDA device `device`.  *out receives the handle (NULL on error).
 * Errors: INVALID_ARG (out NULL, only one of alloc/free given), CUDA (no such device). */
vr_status vr_create(vr_ctx **out, int device, vr_alloc_fn alloc, vr_free_fn free_fn,
                    void *user);

/* Release every buffer of the context (after synchronising the device).  NULL is a no-op. */
void vr_destroy(vr_ctx *ctx);

/* Upload a volume (§3.1, §3.2: the host loads the slices and copies them to the GPU).
 * `voxels` is a dense nx*ny*nz array of `dtype` in host or device memory (detected);
 * it is only read during the call's stream work (host memory: before the call returns).
 * value_max maps raw values to [0, 1]: s = raw / value_max (255 for u8, 4095 for
 * 12-bit u16, 1 for f16/f32).  The library stores a copy with a clamp-to-edge border and
 * per-brick (8^3) min/max tables; if a transfer function is set, brick visibility is
 * recomputed.  Errors: INVALID_ARG (NULL, a size < 1, nx*ny*nz > 2^31, value_max <= 0),
 * UNSUPPORTED (dtype), OUT_OF_MEMORY, CUDA; after OUT_OF_MEMORY or CUDA the context holds no
 * volume until an upload succeeds. */
vr_status vr_upload_volume(vr_ctx *ctx, const void *voxels, vr_dtype dtype, int nx, int ny,
                           int nz, float value_max, void *stream);

/* Set the transfer function (§3.7 colour lookup table): n RGBA float32 entries in host or
 * device memory, entry i covering s = i / (n - 1), read with linear interpolation between
 * entries.  Values are used as given (no clamping of alpha).  Recomputes the per-brick
 * visibility flags when a volume is present.  A host table is copied into pinned memory the
 * context owns before the call returns, so the caller may reuse it at once; the call does
 * not wait for the stream's earlier work.  Errors: INVALID_ARG (NULL, n < 2,
 * n > 65536), OUT_OF_MEMORY, CUDA; after OUT_OF_MEMORY or CUDA the context holds no transfer
 * function until a set succeeds. */
vr_status vr_set_transfer_function(vr_ctx *ctx, const float *rgba, int n, void *stream);

/* Set the camera used by the following renders (host struct, copied).
 * Errors: INVALID_ARG (NULL, size out of range, fov out of (0,180), ortho_height <= 0,
 * eye == target, up parallel to the view direction, non-finite values). */
vr_status vr_set_camera(vr_ctx *ctx, const vr_camera *cam);

/* Render the current volume / transfer function / camera into out_rgba (H x W x 4 float32,
 * host or device memory, detected; host output is copied back on `stream` and is valid
 * once the stream is synchronised).  Errors: INVALID_ARG (NULL, step <= 0, ert_threshold
 * <= 0, shininess < 0, grad out of range, non-finite parameters), STATE (no volume, TF or
 * camera), OUT_OF_MEMORY, CUDA.  An empty clip box gives a black transparent image.
 * Every pixel is written: rays are marched only over the tiles of the sampling box's screen
 * rectangle (vr_screen_rect), and the pixels outside it, whose rays miss the box, are
 * cleared to (0, 0, 0, 0) first. */
vr_status vr_render(vr_ctx *ctx, const vr_render_params *params, float *out_rgba, void *stream);

/* vr_render's image with 8 bits per channel, for display and a read-back a quarter the size:
 * out_rgba8 (H x W x 4 bytes, row-major, host or device memory, detected; device memory
 * aligned to 4 bytes) receives for every pixel and channel round(255 * clamp(c, 0, 1)) of
 * the FP32 value c vr_render writes (the premultiplied colour and 1 - T of §3.9, Eq. 6;
 * product in FP32, round to nearest even) -- bit for bit the quantisation of vr_render's
 * image.  The FP32 image is rendered into the context's staging buffer and quantised there
 * by one more kernel.  Host output is copied back on `stream` and is valid once the stream
 * is synchronised.  Errors: as vr_render. */
vr_status vr_render_rgba8(vr_ctx *ctx, const vr_render_params *params, unsigned char *out_rgba8,
                          void *stream);

/* Rows [row0, row1) of the image vr_render would produce for the current volume, transfer
 * function and camera, written to out_rgba as a band of (row1 - row0) x W x 4 float32 (host
 * or device memory, detected), bit for bit equal to those rows of vr_render's image.
 * Rays are independent (§2.2, §6), so a frame can be split by rows over several GPUs that
 * hold the same volume (the image-space, sort-first partition): each renders its bands and
 * the bands are gathered.  With collect_stats = 1 the counters cover the band's rays.
 * Errors: as vr_render, plus INVALID_ARG unless 0 <= row0 < row1 <= H. */
vr_status vr_render_rows(vr_ctx *ctx, const vr_render_params *params, int row0, int row1,
                         float *out_rgba, void *stream);

/* The partial image of one z-slab of the volume (the object-space, sort-last partition):
 * the march of vr_render on the whole sampling box's grid of samples, compositing only the
 * samples whose position has z0 <= z < z1 (the others count as transparent), written to
 * out_rgba (H x W x 4 float32, host or device memory, detected) as premultiplied
 * (C, A = 1 - T).  Slabs [z_0, z_1), [z_1, z_2), ... that tile the volume composite, pixel by
 * pixel front to back along the pixel's ray ("over": C = C_f + (1 - A_f) C_b,
 * A = A_f + (1 - A_f) A_b, Eq. 6 is associative), to vr_render's image up to rounding when
 * early termination is off (ert_threshold > 1; with it each slab would stop on its own
 * transmittance).  The ray's direction in z gives the pixel's slab order.  The record march
 * always renders it.  Errors: as vr_render, plus INVALID_ARG unless z0 < z1 (either may be
 * infinite), UNSUPPORTED with adaptive sampling. */
vr_status vr_render_partial(vr_ctx *ctx, const vr_render_params *params, float z0, float z1,
                            float *out_rgba, void *stream);

/* Bytes of the checkpoint buffer vr_render_forward_train needs for the current camera,
 * volume and `params` (per-ray end index plus transmittance every 32 samples). */
vr_status vr_checkpoint_bytes(vr_ctx *ctx, const vr_render_params *params, size_t *bytes);

/* vr_render that also records, in the caller-owned device buffer `checkpoints` (at least
 * vr_checkpoint_bytes bytes, 256-byte aligned), what vr_render_backward needs: each ray's
 * end index and its transmittance before every 32nd sample.  The buffer begins with the
 * end indices: int32, one per pixel in image order (row-major), each the number of samples
 * the ray marched up to and including the one that terminated it (its sample count K when
 * it did not terminate).  out_rgba must be device memory.  Errors as vr_render, plus
 * INVALID_ARG for a short or unaligned buffer. */
vr_status vr_render_forward_train(vr_ctx *ctx, const vr_render_params *params,
                                  float *out_rgba, void *checkpoints, size_t checkpoint_bytes,
                                  void *stream);

/* Adjoint of vr_render_forward_train (reverse-mode differentiation of Eq. 6 through the
 * shading, normal, gradient operator, transfer function and trilinear interpolation).
 * grad_rgba: dL/dRGBA, H x W x 4 float32 device.  Accumulates (+=) dL/d(raw voxel) into
 * grad_volume (device float32, nx*ny*nz, x fastest) and dL/d(TF entry) into grad_tf
 * (device float32, n x 4); either may be NULL to skip it.  The rays are walked back to
 * front segment by segment, each segment recomputed from its stored transmittance.
 * Errors: INVALID_ARG, STATE (checkpoints not written by vr_render_forward_train for the
 * current volume, transfer function, camera and params), OUT_OF_MEMORY, CUDA. */
vr_status vr_render_backward(vr_ctx *ctx, const vr_render_params *params,
                             const void *checkpoints, const float *grad_rgba,
                             float *grad_volume, float *grad_tf, void *stream);

/* First-hit surface rendering -- the renderer the paper itself implements (§3.11): a
 * threshold window [iso_lo, iso_hi] of raw voxel values marks solid matter; each ray takes
 * coarse samples t_k = t_near + (k + 1/2) step (the sample grid of vr_render with this step)
 * until the first one whose trilinear value lies in the window, then refines the hit by
 * bisection between the previous sample (the entry point for k = 0) and that one, keeping
 * the outside end outside and the inside end inside, `refine` times (§5.1 hitpoint
 * refinement: 5-6 steps locate the surface 32-64 times more precisely, so the coarse step
 * can be 4-5 times the direct-rendering step); the hit is the middle of the final bracket,
 * or the entry point itself when that is already inside.  The inside tests run in FP32
 * exactly as: t = fma(k + 1/2, step, t_near), p = fma(t, d, o), cell and trilinear lerps
 * fma(f, b - a, a) along x, then y, then z; bisection midpoints (a + b) * 1/2.
 * At the hit, the operator gradient (§3.5) gives N = -g/|g|, turned to face the viewer, and
 * Phong (§3.8, as vr_render) with the surface colour gives the pixel (c, 1); rays without a
 * hit give (0, 0, 0, 0).  The output is H x W x 4 float32 (device or host memory);
 * out_depth (optional, NULL to skip; device or host) receives H x W float32 hit distances t
 * along the unit ray direction from the ray origin, +inf where nothing is hit.
 * skip_empty: coarse samples in 8^3 bricks (and 32^3 macro bricks) whose footprint value
 * range misses the window are skipped; this never changes a pixel.
 * Needs a volume and a camera (no transfer function).
 * Errors: INVALID_ARG (NULL params or output, step <= 0, iso_lo > iso_hi or NaN,
 * refine outside [0, 24], invalid shading parameters), STATE, OUT_OF_MEMORY, CUDA. */
typedef struct {
  float step;            /* coarse sample spacing (voxel units, > 0) */
  float iso_lo, iso_hi;  /* threshold window in raw voxel units, inclusive */
  int refine;            /* bisection steps after the first hit, 0..24 */
  vr_grad grad;
  float ka, kd, ks, shininess;
  float light[3];
  int headlight;
  float color[3];        /* surface colour */
  int skip_empty;
  float clip_lo[3], clip_hi[3];
} vr_surface_params;

vr_status vr_render_surface(vr_ctx *ctx, const vr_surface_params *params, float *out_rgba,
                            float *out_depth, void *stream);

/* Render without allocating any device memory.  (The paper has no counterpart: this entry
 * exists for callers that cannot allocate device memory when they render -- a plug-in
 * inside an application that owns the device's whole memory pool, a real-time loop that
 * must not allocate per frame, or a process whose device memory is already reserved by
 * another framework's caching allocator.)
 * No context is used: the caller passes, in device memory of the current CUDA device,
 * the dense volume `voxels` (nx*ny*nz of `dtype`, x fastest, read in place), the
 * transfer function `tf_rgba` (ntf x 4 float32) and the output `out_rgba` (H x W x 4
 * float32), plus the camera and the parameters as host structs; the result equals
 * vr_render's on the same inputs up to FP32 rounding (the operator gradient is evaluated
 * from each sample's neighbourhood instead of precomputed records).
 * The library's scratch (brick min/max and visibility tables, transfer-function prefix
 * counts, the work counter) is a fixed array in device memory that every GPU loading the
 * library holds until the process exits; its limits are at most 262144 bricks of 8^3
 * voxels (e.g. 512^3 voxels) and ntf <= 4096 -- larger requests return
 * VR_ERR_INVALID_ARG.  All calls on a device share that array and each call rewrites it
 * (the work counter is cleared on `stream` first), so calls whose work overlaps on the
 * GPU (different streams, or other host threads) race and must be serialised by the
 * caller.  The first call on a device looks up the array's device address (host code
 * cannot use the array's name as a device pointer); make that first call before any
 * stream capture.  collect_stats and adaptive (§5.2 adaptive sampling) must be 0: this
 * entry point counts no samples and marches only the regular grid (VR_ERR_UNSUPPORTED
 * otherwise).  `voxels` must be aligned to its element size, `tf_rgba` and `out_rgba` to
 * 16 bytes (they are read and written as float4).
 * Errors: INVALID_ARG (NULL, host or misaligned pointers, sizes out of range or beyond the
 * scratch limits, invalid camera or parameters), UNSUPPORTED, CUDA. */
vr_status vr_render_noalloc(const void *voxels, vr_dtype dtype, int nx, int ny, int nz,
                            float value_max, const float *tf_rgba, int ntf,
                            const vr_camera *cam, const vr_render_params *params,
                            float *out_rgba, void *stream);

/* vr_render_backward for `nviews` views (1 .. 256) of the current volume and transfer
 * function in one call: cams[v] is the camera view v was rendered with and checkpoints[v]
 * / grad_rgba[v] its checkpoint buffer and image gradient.  The gradients of all views
 * are summed into grad_volume / grad_tf (+=).  Equivalent to nviews vr_render_backward
 * calls, but the per-voxel accumulator is cleared once and the transposed operator
 * stencil applied once.  Errors as vr_render_backward; all views are validated before
 * any work is queued. */
vr_status vr_render_backward_views(vr_ctx *ctx, const vr_render_params *params, int nviews,
                                   const vr_camera *cams, const void *const *checkpoints,
                                   const float *const *grad_rgba, float *grad_volume,
                                   float *grad_tf, void *stream);

/* Copy the counters of the last render with collect_stats = 1 into *out.  Synchronises
 * `stream`.  Errors: INVALID_ARG, STATE (no such render), CUDA, TIMEOUT (an earlier pass that
 * computes the operator gradient records gave up waiting, after about a second, for a copy
 * of a brick's neighbourhood into shared memory: the records, and so images since, are
 * incomplete; upload the volume again). */
vr_status vr_read_stats(vr_ctx *ctx, vr_stats *out, void *stream);

/* ---- Batched rendering -------------------------------------------------------------
 * Many renders -- ncams cameras, camera i over the volume of ctxs[ctx_of_cam[i]] -- in one
 * persistent launch (rays are independent, §2.2), captured once into a CUDA graph and
 * replayed by vr_batch_run.  Every context must hold a volume and a transfer function;
 * volumes may differ in size and voxel type.  outs[i] is camera i's H x W x 4 float32
 * device image (caller-owned, must outlive the batch).  The batch records the contexts'
 * state at creation: vr_batch_run returns VR_ERR_STATE once any of them has a new volume
 * or transfer function (create a new batch then).  Device tables are allocated with
 * ctxs[0]'s allocator; destroy the batch before its contexts.  collect_stats must be 0.
 * Errors: INVALID_ARG, STATE, UNSUPPORTED (contexts on different devices, stats),
 * OUT_OF_MEMORY, CUDA. */
typedef struct vr_batch vr_batch;
vr_status vr_batch_create(vr_batch **out, vr_ctx *const *ctxs, int nctx, const vr_camera *cams,
                          const int *ctx_of_cam, int ncams, const vr_render_params *params,
                          float *const *outs, void *stream);

/* Replay the batch's graph on `stream` (asynchronous). */
vr_status vr_batch_run(vr_batch *batch, void *stream);

/* Time the batch with each block size (64, 128, 256 threads) and warp tile shape (4x2,
 * 2x4, 8x1 rays) on `stream` (synchronising), keep the fastest and rebuild the graph.
 * chosen (optional, 3 ints) receives {threads, tile width, tile height}. */
vr_status vr_batch_autotune(vr_batch *batch, void *stream, int *chosen);

/* Release the batch (synchronises the device).  NULL is a no-op. */
void vr_batch_destroy(vr_batch *batch);

/* One-shot batched render: camera i of n is rendered from vols[vol_of_cam[i]] into outs[i]
 * (H x W x 4 float32 device image, caller-owned) by one persistent launch over the
 * concatenated tiles of every render, without building a graph -- the same pixels as n
 * vr_render calls.  Rays are independent (§2.2), so renders of different volumes, sizes and
 * voxel types share the launch.  vols[k] for k <= max(vol_of_cam) must hold a volume and a
 * transfer function on one device; gradient records are brought up to date on `stream`.
 * The launch tables live in vols[0]'s context: calls that name the same vols[0] must be
 * issued on one stream (or ordered by the caller).  collect_stats must be 0.
 * Errors: INVALID_ARG, STATE, UNSUPPORTED (different devices, stats), OUT_OF_MEMORY, CUDA. */
vr_status vr_render_batch(vr_ctx *const *vols, const vr_camera *cams, const int *vol_of_cam,
                          int n, const vr_render_params *params, float *const *outs,
                          void *stream);

/* The pixel rectangle [rect[0], rect[2]) x [rect[1], rect[3]) outside which every ray of
 * `cam` misses the box [lo, hi] (world units; the renderers pass the sampling box, the clip
 * box intersected with [0, n-1]^3): the bounding rectangle of the eight box corners projected
 * through the camera (§3.3 ray set-up), widened by two pixels; the whole image when a corner
 * lies near or behind the eye plane of a perspective camera, an empty rectangle when the box
 * is empty.  vr_render, vr_render_batch and vr_render_surface march only the tiles of this
 * rectangle.  Host only (no device is used).  Errors: INVALID_ARG (NULL, NaN bounds, camera
 * as for vr_set_camera). */
vr_status vr_screen_rect(const vr_camera *cam, const float lo[3], const float hi[3], int rect[4]);

/* The march's per-sample stages at n caller-given points (a testing and inspection aid;
 * renders nothing).  pos: n x 3 float32 world points (device memory; a point outside the
 * volume box uses the nearest cell, as a sample on the box face does).  out: n x 12 float32
 * (device memory), per point:
 *   [0]     s = V(p) / value_max, V trilinear in the voxel values (§3.4, Eq. 2),
 *   [1..4]  the transfer function's RGBA at s (§3.7),
 *   [5..7]  the operator gradient at p (params->grad: Eq. 3, Eq. 4 or Zucker-Hummel, §3.5),
 *           scaled so that it estimates ds/dx per voxel,
 *   [8..10] the Phong colour (§3.8) for params' light and coefficients, viewed along the
 *           current camera's ray through p (the normal is -g/|g|),
 *   [11]    the gradient's length.
 * The same device functions as vr_render's march, on the context's volume, transfer function
 * and camera; gradient records of every brick are brought up to date on `stream`.
 * Errors: INVALID_ARG (NULL, n < 0, a host pointer, params), UNSUPPORTED (adaptive),
 * STATE (no volume, transfer function or camera), OUT_OF_MEMORY, CUDA. */
vr_status vr_probe_samples(vr_ctx *ctx, const vr_render_params *params, const float *pos, int n,
                           float *out, void *stream);

/* Measured ceilings of the march (measurement only; renders nothing).  The march is neither
 * a dense contraction nor HBM-bound, so its roofline is set by the FP32 pipes or by the rate
 * at which the SMs gather the 8 corner gradient records of a sample (§3.4 trilinear cell,
 * §3.5 operator gradient) and blend its value and gradient. */
typedef struct {
    double fma_tflops;            /* FP32 FMA throughput, TFLOP/s (an FMA counts 2)          */
    double gather_coherent_gsps;  /* gather + blend, Gsamples/s, the march's access pattern:
                                     quads of lanes on consecutive samples (step 0.5) of 4 x 2
                                     neighbouring rays 1.09 voxels apart, table in L2      */
    double gather_random_gsps;    /* the same at uniformly random cells of a 64 KiB table    */
    double gather_u16_random_gsps;   /* the method's own per-sample footprint: the 8 voxels of
                                        the sample's cell in 16-bit storage and their trilinear
                                        blend, Gsamples/s, random cells of a 64 KiB volume      */
    double gather_u16_coherent_gsps; /* the same in the march's pattern over a 32 MiB volume  */
} vr_peaks;

/* Time the five microbenchmarks of vr_peaks on `device` (synchronous; private stream and
 * buffers from cudaMalloc, about 65 MiB, released before returning), best of `repeats`
 * timed launches after one warm-up.  Errors: INVALID_ARG (out NULL, repeats outside
 * 1..1000, device < 0), OUT_OF_MEMORY, CUDA (no such device, a launch failed). */
vr_status vr_measure_peaks(int device, int repeats, vr_peaks *out);

/* Out-of-range gather and scatter indices met by this context's kernels since vr_create
 * (a testing aid).  Only a library built with -DVR_DEBUG_BOUNDS checks its indices: each
 * index outside its buffer is counted and clamped into the buffer, so the access stays in
 * bounds.  Synchronises `stream`.  Errors: INVALID_ARG (NULL), UNSUPPORTED (a regular build:
 * *count = 0), CUDA. */
vr_status vr_read_bounds_violations(vr_ctx *ctx, unsigned long long *count, void *stream);

/* Short English text of a status code (static storage). */
const char *vr_status_string(vr_status status);

/* Text of the last CUDA error seen by this thread (static storage, "" if none). */
const char *vr_last_cuda_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int vr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VR_H */
