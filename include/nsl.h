/* nsl.h -- C ABI of the GB300 neural six-way lightmap library (libnsl.so).
 *
 * The per-frame hot path of "Real-time Neural Six-way Lightmaps"
 * (arXiv 2604.03748):
 *   1. nsl_guiding_map        coarse camera-view ray march under three surrogate
 *                             lights -> guiding map (Sec. 4.2, Alg. 1, Eq. approx)
 *   2. nsl_predict_lightmaps  UNet + four NAFBlock channel adapters -> six
 *                             directional lightmaps + transparency + emissive
 *                             (Sec. 4.3, Fig. 3)
 *   3. nsl_shade              six-way directional interpolation for any set of
 *                             directional lights (Sec. 3, six-way interpolation)
 *
 * Conventions
 *   - World units are voxels.  A grid (nx, ny, nz) is stored [nz][ny][nx] with
 *     x fastest and occupies the box [0,nx] x [0,ny] x [0,nz]; voxel (i,j,k) is
 *     centred at (i+.5, j+.5, k+.5).
 *   - Camera frame: X = right, Y = up, Z = forward (into the screen).
 *   - Images are planar [C][H][W] float32, row 0 at the top.
 *   - Every *_dev pointer is a device pointer owned by the caller, 16-byte
 *     aligned, and borrowed until the work queued on `stream` completes.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     asynchronous on that stream unless stated otherwise.
 *   - Errors: argument errors are reported synchronously and nothing is queued.
 *     A CUDA error raised by a launch is returned as NSL_ERR_CUDA; an
 *     asynchronous fault surfaces on a later call or synchronisation.  No call
 *     aborts or prints.  nsl_last_error() gives a message for the calling thread.
 *   - Threading: one context may be used by one host thread at a time.
 */
#ifndef NSL_H
#define NSL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NSL_API __attribute__((visibility("default")))
#else
#define NSL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NSL_OK = 0,
  NSL_ERR_INVALID_ARG = 1,
  NSL_ERR_OOM = 2,
  NSL_ERR_CUDA = 3,
  NSL_ERR_UNSUPPORTED = 4,
  NSL_ERR_TIMEOUT = 5,
  NSL_ERR_BUDGET = 6
} nsl_status;

enum { NSL_F32 = 0, NSL_F16 = 1 };                           /* density storage */
/* network arithmetic: FP32 SIMT; or tensor cores with FP32 accumulation and
 * BF16, FP8 E4M3 or FP16 operands */
enum { NSL_PREC_F32 = 0, NSL_PREC_BF16 = 1, NSL_PREC_FP8 = 2, NSL_PREC_F16 = 3, NSL_PREC_BF16X3 = 4 };
enum { NSL_CAM_ORTHO = 0, NSL_CAM_PERSP = 1 };

typedef struct nsl_ctx nsl_ctx; /* opaque, library-owned */

typedef struct {
  int nx, ny, nz;     /* grid size in voxels, each in [1, 4096], with
                         (nx+1)(ny+1)(nz+2) < 2^32 (the staged cells the
                         march addresses with 32-bit indices); other sizes
                         are rejected with NSL_ERR_INVALID_ARG */
  int dtype;          /* NSL_F32 or NSL_F16 */
  float sigma_scale;  /* extinction = sigma_scale * density (albedo 1) */
} nsl_grid_desc;

typedef struct {
  int kind;                          /* NSL_CAM_ORTHO or NSL_CAM_PERSP */
  float eye[3], target[3], up[3];    /* world space */
  float fov_y_deg;                   /* perspective: vertical field of view */
  float ortho_height;                /* orthographic: view height in voxels */
  int width, height;                 /* billboard pixels, multiples of 8 */
} nsl_camera;

typedef struct {
  float dir[3];        /* world-space vector toward the light (normalised by the library) */
  float intensity[3];  /* RGB */
} nsl_light;

typedef struct {
  float tau_depth;       /* Alg. 1 depth threshold tau on the density (default 0.01) */
  float t_min;           /* early termination when transmittance < t_min (1e-4; 0 = off) */
  int jitter;            /* 1: per-pixel hash jitter of the first sample (Alg. 1 delta) */
  uint32_t seed, frame;  /* jitter hash inputs */
  float phase_g;         /* Henyey-Greenstein g of the surrogate lights (0 = isotropic) */
  float surrogate_I[3];  /* intensities of the front, top, bottom surrogate lights */
  int segment_exact;     /* 0: A_n = T_{n-1} sigma_n h;  1: A_n = T_{n-1}(1 - e^{-sigma_n h}) */
  int light_set;         /* surrogate lights (Sec. 5, ablation on the guiding light
                            directions): NSL_LIGHTS_FTB front/top/bottom (default),
                            NSL_LIGHTS_F front only (no shadow rays),
                            NSL_LIGHTS_FLR front/left/right (side pair along the
                            camera's right axis; surrogate_I[1] right, [2] left) */
  int shadow_volume;     /* 0: the side lights' shadow rays are marched from every
                            view sample (Alg. 1); 1: they are marched once from
                            every voxel centre into two transmittance volumes that
                            the view march reads trilinearly (an approximation of
                            Alg. 1, cheaper when view samples outnumber voxels;
                            single-plume entry points only) */
} nsl_march_opts;

enum { NSL_LIGHTS_FTB = 0, NSL_LIGHTS_F = 1, NSL_LIGHTS_FLR = 2 };

/* Default options: tau_depth 0.01, t_min 1e-4, jitter 1, seed 0, frame 0,
 * g 0, intensities 1, segment_exact 0, light_set NSL_LIGHTS_FTB,
 * shadow_volume 0. */
NSL_API void nsl_default_march_opts(nsl_march_opts* out);

/* Create a context.  Sec. 4.3 (one network for all scenes, Sec. 5).
 *   grid          grid shape and storage used by nsl_guiding_map and for the
 *                 network's depth normalisation (D / |grid diagonal|).
 *   weights_blob  NSLW blob: "NSLW", u32 version (1), u32 C0, u32 n_floats,
 *                 n_floats float32 parameters in the documented order, u32
 *                 checksum.  Copied; the caller keeps ownership.
 *   max_width, max_height  largest billboard any later call may use; the
 *                 network workspace is allocated for it (device memory).
 * C0 (the UNet base width, Sec. 4.3: widths C0, 2 C0, 4 C0, 8 C0, adapters of
 * C0 channels) is 16 or 32; a C0 = 32 context runs the FP32 network only (the
 * tensor-core precisions of nsl_predict_lightmaps return NSL_ERR_UNSUPPORTED).
 * Returns NSL_ERR_INVALID_ARG for a malformed blob or sizes, NSL_ERR_OOM when
 * device memory runs out, NSL_ERR_UNSUPPORTED for C0 other than 16 or 32. */
NSL_API nsl_status nsl_create(const nsl_grid_desc* grid, const void* weights_blob, size_t blob_bytes,
                      int max_width, int max_height, nsl_ctx** out);

/* Release the context and everything it owns (synchronises its work). */
NSL_API void nsl_destroy(nsl_ctx* ctx);

/* Stage a density grid into the context (Sec. 4.2: sigma_s in a 3D texture):
 * sigma' = sigma_scale * density * [mask == 0], kept in a context-owned device
 * buffer until the next staging.  A float32 grid is staged as float32 sigma':
 * as cells holding the 2x2x2 corner neighbourhood of each trilinear sample when
 * those, together with the same cells of the other live contexts on the device,
 * take at most 60% of its L2 (one grid of up to about 135^3 on a GB300; chosen
 * at nsl_create), else as cells holding the 2x2 x/y neighbourhood of one slice
 * (half the bytes); the two give bitwise equal guides.  A float16 grid is staged as float16 density *
 * [mask == 0] in the second form (its values
 * exactly) and the march applies sigma_scale after the trilinear blend, which
 * differs from blending sigma' by rounding only.  A later
 * nsl_guiding_map with density_dev == NULL marches this resident grid.
 *   density_dev   [nz][ny][nx] float32 or float16 (grid.dtype)
 *   mask_dev      [nz][ny][nx] uint8 obstacle mask (non-zero = obstacle) or NULL */
NSL_API nsl_status nsl_stage_grid(nsl_ctx* ctx, const void* density_dev, const uint8_t* mask_dev,
                                  void* stream);

/* Guiding map, Sec. 4.2 / Alg. 1 / Eq. approx.
 *   density_dev   [nz][ny][nx] float32 or float16 (grid.dtype), staged first
 *                 as by nsl_stage_grid; NULL = march the grid staged last
 *   mask_dev      [nz][ny][nx] uint8 obstacle mask, non-zero zeroes the voxel; may be NULL
 *   cam           camera; cam->width x cam->height <= the context maximum
 *   light         accepted and unused: the guide uses the fixed surrogate
 *                 lights of Eq. approx (front, top, bottom); may be NULL
 *   step_voxels   march step h in voxels (> 0)
 *   opts          march options (NULL = defaults)
 *   guide_dev     output [3][H][W] float32: (L_scattering, T, D in voxels)
 * Uses library-owned scratch (staged grid, tile counters). */
NSL_API nsl_status nsl_guiding_map(nsl_ctx* ctx, const void* density_dev, const uint8_t* mask_dev,
                           const nsl_camera* cam, const nsl_light* light, float step_voxels,
                           const nsl_march_opts* opts, float* guide_dev, void* stream);

/* Guide march without any device allocation by the library (the paper has no
 * counterpart of this entry point).  It is meant for callers that cannot call
 * cudaMalloc at all: a render thread whose frame budget cannot absorb the device
 * synchronisation an allocation may cause, an engine whose own allocator owns
 * every byte of device memory, or code that has no context to keep between
 * frames.  It stages the grid as x/y neighbourhood cells (float32 quads of
 * sigma' for a float32 grid, float16 quads for a float16 one) and then
 * runs the single-pass march kernel (the one nsl_guide_sample_count runs) rather
 * than nsl_guiding_map's three-pass segmented march, which would need per-pixel
 * segment scratch.  The two marches make the same samples and decisions; their
 * guides differ only by the rounding of the in-scattering sum's grouping (well
 * inside 1e-5 of the range), not bitwise.  The staged grid and the tile counter
 * live in one static device array of 40 MiB + 256 bytes inside libnsl, which
 * every GPU that loads the library holds until the process exits.
 *   grid          shape, storage and sigma_scale of density_dev
 *   density_dev, mask_dev, cam, step_voxels, opts, guide_dev, stream
 *                 as for nsl_guiding_map (no light argument); opts->shadow_volume
 *                 is refused with NSL_ERR_UNSUPPORTED (its volumes need a context)
 * Limits: the staged grid takes (nx+1)(ny+1)(nz+2) cells of 16 bytes (float32
 * grid) or 8 bytes (float16 grid) and must fit in 40 MiB: a float32 136^3 grid
 * fits and 137^3 does not; a float16 172^3 grid fits and 173^3 does not.  Larger
 * grids return NSL_ERR_INVALID_ARG with a message, and nothing is queued.  No
 * cudaMalloc, cudaFree or other allocating call is made.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and keeps it for the life of the process: make that first
 * call before any stream capture, and do not reset the device
 * (cudaDeviceReset) while the library is loaded, since the kept address
 * belongs to the device's primary context.  All calls share the one array and
 * it keeps the last call's contents (every call restages the grid and zeroes the
 * counter first); calls that overlap on the GPU (different streams, or devices
 * sharing nothing but this rule) race on it, so serialise them. */
NSL_API nsl_status nsl_guiding_map_noalloc(const nsl_grid_desc* grid, const void* density_dev,
                                           const uint8_t* mask_dev, const nsl_camera* cam,
                                           float step_voxels, const nsl_march_opts* opts,
                                           float* guide_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Training slice (Sec. 4.4, the MSE term only): Adam on the mean squared
 * error between the network's eight output planes and target planes, each
 * plane's term with its own weight (the paper trains on values encoded to
 * sRGB, which raises dark lightmap values; weights that equalise the planes'
 * ranges play that part here on linear values) (for
 * example nsl_reference_lightmaps with a zero emissive plane), for batches of
 * `batch` guides of width x height.  Forward and backward run in FP32 on the
 * SIMT cores with every activation kept (about 1.3 KB per pixel of the
 * batch); the trained weights leave as a weight blob for nsl_create.  The
 * paper's VGG and FlowNet loss terms need pretrained networks and are not
 * built.
 * ------------------------------------------------------------------------- */
typedef struct nsl_trainer nsl_trainer;
typedef struct {
  int batch;            /* images per step, 1..64 */
  int width, height;    /* image size, multiples of 8, at most 512^2 pixels */
  float lr, beta1, beta2, eps;   /* Adam */
  float plane_weight[8];         /* weight of each output plane's squared error */
} nsl_train_opts;
/* Defaults: batch 4, 64 x 64, lr 1e-3, beta1 0.9, beta2 0.999, eps 1e-8, every
 * plane weight 1 (the loss is then the plain mean squared error). */
NSL_API void nsl_default_train_opts(nsl_train_opts* o);
/* Starts from the weights of `weights_blob` (C0 = 16). */
NSL_API nsl_status nsl_trainer_create(const void* weights_blob, size_t blob_bytes, const nsl_train_opts* opts,
                                      nsl_trainer** out);
/* One step on device batches guides_dev [batch][3][H][W] (the guide, depth
 * channel in voxels, scaled by depth_scale as nsl_predict_lightmaps scales it:
 * 1 / |grid diagonal|) and targets_dev [batch][8][H][W]: forward, loss,
 * backward, and with update != 0 one Adam update.  Synchronises `stream` and
 * writes the loss (the mean over every plane and pixel of the batch of the
 * plane-weighted squared error) to *loss_out (nullable). */
NSL_API nsl_status nsl_trainer_step(nsl_trainer* t, const float* guides_dev, const float* targets_dev,
                                    float depth_scale, int update, float* loss_out, void* stream);
/* Learning rate of the following steps (a schedule is the caller's). */
NSL_API nsl_status nsl_trainer_set_lr(nsl_trainer* t, float lr);
/* The last step's gradient of the loss, in weight-blob order, into grad_dev
 * (count >= the number of parameters). */
NSL_API nsl_status nsl_trainer_gradients(nsl_trainer* t, float* grad_dev, size_t count, void* stream);
/* The current weights as a weight blob (host memory); *needed receives its
 * size, and blob_host = NULL only queries it. */
NSL_API nsl_status nsl_trainer_get_blob(nsl_trainer* t, void* blob_host, size_t bytes, size_t* needed);
NSL_API void nsl_trainer_destroy(nsl_trainer* t);

/* Roofline denominators measured on the current device (the paper has no
 * counterpart; used by the benchmark).  Runs three short kernels on `stream`,
 * each timed with CUDA events after a warm-up launch, and synchronises it;
 * allocates and frees about 65 MB of scratch.
 *   sms             multiprocessors of the device
 *   fp32_tflops     FP32 FMA rate (eight independent fmaf chains per thread)
 *   l1_gbps         L1 data path: warps reading 512 contiguous bytes (16 per
 *                   lane) from a 16 KB region held in L1
 *   l2_gather_gbps  16-byte loads at hashed positions of a 64 MiB buffer
 *                   resident in L2 (a warp's lanes touch unrelated lines) */
typedef struct {
  int sms;
  double fp32_tflops;
  double l1_gbps;
  double l2_gather_gbps;
} nsl_peaks;
NSL_API nsl_status nsl_measure_peaks(nsl_peaks* out, void* stream);

/* Number of density evaluations the guide march of nsl_guiding_map makes for
 * this camera, step and options on the staged grid: view samples plus the
 * shadow samples of every view sample with non-zero density (Alg. 1).  Runs a
 * counting variant of the march kernel and synchronises `stream`; the guide is
 * not written.  *samples_out receives the total. */
NSL_API nsl_status nsl_guide_sample_count(nsl_ctx* ctx, const nsl_camera* cam, float step_voxels,
                                          const nsl_march_opts* opts,
                                          unsigned long long* samples_out, void* stream);

/* Fine-step six-light reference lightmaps: single scattering of Sec. 3 (Eq. RE
 * with Eq. scatter) under six directional lights along the camera axes, the
 * physical quantity the lightmap network approximates and is trained toward
 * (Sec. 4.4; training data, not part of the per-frame path).  Per pixel, the
 * view ray's chord is split into ceil(chord / hf) equal steps sampled at their
 * midpoints; at every sample the transmittance toward each light is the
 * midpoint sum of its own ray to the box exit in steps of at most hf.
 *   density_dev, mask_dev  as for nsl_guiding_map (NULL density: the grid
 *                 staged last)
 *   cam           camera; cam->width x cam->height <= the context maximum
 *   hf            step in voxels, at least 1/64
 *   phase_g       Henyey-Greenstein parameter in (-1, 1) (0: isotropic)
 *   out_dev       output [7][H][W] float32: light from +X (right), -X, +Y (up),
 *                 -Y, +Z (back), -Z (front) in the camera frame, then the
 *                 view transmittance T
 * The cost grows as (extent / hf)^2 per pixel: meant for small images. */
NSL_API nsl_status nsl_reference_lightmaps(nsl_ctx* ctx, const void* density_dev, const uint8_t* mask_dev,
                                           const nsl_camera* cam, float hf, float phase_g, float* out_dev,
                                           void* stream);

/* Lightmap network, Sec. 4.3 / Fig. 3.
 *   guide_dev      [3][H][W] float32 guide
 *   width, height  multiples of 8, within the context maximum
 *   precision      NSL_PREC_F32 (SIMT FP32), NSL_PREC_BF16, NSL_PREC_F16,
 *                  NSL_PREC_FP8 or NSL_PREC_BF16X3 (tensor cores, FP32
 *                  accumulation; C0 = 16 contexts only, NSL_ERR_UNSUPPORTED at
 *                  C0 = 32).  NSL_PREC_BF16X3 is the split-BF16 form: every
 *                  convolution after the first takes the bfloat16 high part
 *                  hi = bf16(x) and low part lo = bf16(x - hi) of both
 *                  operands and adds hi*hi + hi*lo + lo*hi (three BF16
 *                  tensor-core products per multiply) on binary32 activations;
 *                  the adapters run as in the other tensor-core networks.  It is
 *                  the BF16 form within 2e-2 of the range of the FP64 network
 *                  (single-BF16 operands are several percent away on seeded
 *                  weights).  Its first call on a context may grow the context's
 *                  workspace (binary32 activations), which synchronises `stream`.
 *   lightmaps_dev  output [8][H][W] float32 planes
 *                  [+X right, -X left, +Y top, -Y bottom, +Z back, -Z front, T, E] */
NSL_API nsl_status nsl_predict_lightmaps(nsl_ctx* ctx, const float* guide_dev, int width, int height,
                                 int precision, float* lightmaps_dev, void* stream);

/* Diagnostic form of nsl_predict_lightmaps (the paper has no counterpart): the
 * same network run, which also copies every convolution's stored output into
 * trace_dev, so that each layer can be compared with an emulation of its
 * arithmetic on the same input.  Tensor-core precisions only (NSL_PREC_BF16,
 * NSL_PREC_F16, NSL_PREC_FP8, NSL_PREC_BF16X3; NSL_PREC_F32 returns
 * NSL_ERR_UNSUPPORTED).
 *   trace_dev     caller-owned device buffer, 16-byte aligned, of at least
 *                 nsl_lightmap_trace_bytes(width, height) bytes; it receives
 *                 the 17 stored tensors in network order (enc1a, enc1b,
 *                 enc2a, enc2b, enc3a, enc3b, enc4a, enc4b, up3, dec3a, dec3b,
 *                 up2, dec2a, dec2b, up1, dec1a, dec1b), back to back, each
 *                 NHWC [H/2^l][W/2^l][C] with l its level (0 at full size) and
 *                 C its channels, in the activation type: bfloat16 for
 *                 NSL_PREC_BF16, binary16 for NSL_PREC_F16 and NSL_PREC_FP8
 *                 (whose activations are binary16 between layers), binary32
 *                 for NSL_PREC_BF16X3
 *   other arguments as for nsl_predict_lightmaps
 * A smaller or unaligned trace buffer returns NSL_ERR_INVALID_ARG before any
 * work is queued.  The copies are ordered on `stream` after each layer. */
NSL_API nsl_status nsl_predict_lightmaps_trace(nsl_ctx* ctx, const float* guide_dev, int width,
                                               int height, int precision, float* lightmaps_dev,
                                               void* trace_dev, size_t trace_bytes, void* stream);
/* Bytes of the trace of a width x height image: 144 activation values per
 * pixel, four bytes each (the binary32 values of NSL_PREC_BF16X3; the 16-bit
 * forms fill the first half); 0 for a non-positive size. */
NSL_API size_t nsl_lightmap_trace_bytes(int width, int height);

/* Diagnostic of the failure detection (no paper counterpart).  Every wait of
 * the tensor-core kernels on an mbarrier is bounded (about 2 s); when one runs
 * out, the kernel records a code in the context's error word, releases its
 * tensor memory and returns, and the next nsl_predict_lightmaps returns
 * NSL_ERR_TIMEOUT.  This call launches, on the stream, one warp whose bounded
 * wait can never complete (nothing arrives at its mbarrier): after about 2 s
 * it records code 0x8000 and returns, so the caller can check that the timeout
 * is reported and that the context keeps working.  No GPU fault is involved. */
NSL_API nsl_status nsl_selftest_wait_timeout(nsl_ctx* ctx, void* stream);

/* Obstacle shadowing, Sec. 4.5 (a depth-based screen-space approximation).
 * Shadow map of the obstacle for one directional light: the obstacle mask is
 * rendered from the light as the depth of the first occupied voxel along each
 * light ray.  The light's frame is built in binary64 and rounded once: w =
 * -dir/|dir| (propagation), e1 = normalize(w x a) with a = +Y (+Z when
 * |w_y| > 0.9), e2 = e1 x w.  The map is the square of side S = |(nx, ny, nz)|
 * centred on the grid centre c in the plane through c spanned by (e1, e2):
 * texel (i, j) (column i, row j) holds the entry parameter t of the first
 * occupied voxel along c + a e1 + b e2 + t w, a = ((i + 0.5)/R - 0.5) S,
 * b = ((j + 0.5)/R - 0.5) S (signed distance from the map plane along w), or
 * +infinity when the line meets no occupied voxel.
 *   mask_dev        [nz][ny][nx] uint8, non-zero = obstacle (device)
 *   light_dir       world-space vector toward the light (host, 3 floats)
 *   resolution      R in [1, 8192]
 *   shadow_map_dev  output [R][R] float32 (device, 16-byte aligned)
 * Asynchronous on the stream; no context is needed.  NSL_ERR_INVALID_ARG for
 * bad arguments, NSL_ERR_CUDA for a launch failure. */
NSL_API nsl_status nsl_obstacle_shadow_map(const uint8_t* mask_dev, int nx, int ny, int nz,
                                           const float light_dir[3], int resolution, float* shadow_map_dev,
                                           void* stream);

/* Six-way shading with obstacle shadows (Sec. 4.5): nsl_shade with each light's
 * term multiplied by the visibility of the pixel's smoke shell.  The shell point
 * is x = o + (t_in + D) d on the pixel's camera ray (t_in its entry into the
 * context's grid box, D the guide's depth channel; the jitter offset below one
 * step is ignored).  In light l's frame it has map coordinates a = (x - c).e1,
 * b = (x - c).e2 and depth z = (x - c).w; it is shadowed when its texel
 * (floor((a/S + 1/2) R), floor((b/S + 1/2) R)) lies on the map and
 * z > t_hit + bias.  Pixels with D = 0 (no shell), rays that miss the box and
 * lights whose map pointer is NULL are lit.  These decisions are taken in
 * binary32 with one rounding per operation in a fixed order.
 *   guide_dev        [3][H][W] float32 guide of the same frame (D in plane 2)
 *   lights           n_lights in [0, 16]
 *   shadow_maps_dev  host array of n_lights device pointers to [R][R] maps from
 *                    nsl_obstacle_shadow_map (entries may be NULL), or NULL
 *   resolution       R of the maps;  bias  depth bias in voxels
 *   rgba_dev         output [4][H][W] float32
 * Buffers 16-byte aligned.  Asynchronous on the stream. */
NSL_API nsl_status nsl_shade_shadowed(nsl_ctx* ctx, const float* lightmaps_dev, const float* guide_dev,
                                      int width, int height, const nsl_camera* cam, const nsl_light* lights,
                                      int n_lights, const float* const* shadow_maps_dev, int resolution,
                                      float bias, float* rgba_dev, void* stream);

/* Texture formats of nsl_pack_lightmaps. */
enum { NSL_TEX_RGBA8 = 0, NSL_TEX_RGBA16F = 1, NSL_TEX_RGBA32F = 2 };

/* Pack the eight lightmap planes into the two RGBA textures of the six-way
 * layout (Sec. 3, Fig. 2), the form a game engine samples:
 *   tex1 = (R right +X, G top +Y, B back +Z, A transparency T)
 *   tex2 = (R left -X,  G bottom -Y, B front -Z, A emissive E)
 * each an interleaved [H][W][4] image, row 0 at the top, in the format:
 *   NSL_TEX_RGBA8    unsigned normalised bytes: the value clamped to [0, 1]
 *                    (NaN to 0), times 255 in float32, rounded to the nearest
 *                    integer, ties to even (4 bytes per texel)
 *   NSL_TEX_RGBA16F  binary16, round to nearest even (8 bytes per texel)
 *   NSL_TEX_RGBA32F  the float32 values (16 bytes per texel)
 *                    (in both float formats a NaN stays a NaN; its payload
 *                    is not specified)
 *   lightmaps_dev  [8][H][W] float32 planes as written by nsl_predict_lightmaps
 *   tex1_dev, tex2_dev  caller-owned device buffers of H*W texels each
 * All three buffers must be 16-byte aligned; width and height multiples of 8
 * in [8, 8192].  Asynchronous on the stream; no context is needed.  Returns
 * NSL_ERR_INVALID_ARG for bad arguments, NSL_ERR_CUDA for a launch failure. */
NSL_API nsl_status nsl_pack_lightmaps(const float* lightmaps_dev, int width, int height, int format,
                                      void* tex1_dev, void* tex2_dev, void* stream);

/* Six-way shading, Sec. 3 (directional interpolation, summed over lights):
 *   rgb = sum_l I_l * sum_{p in X,Y,Z} |w_p| L_p^{sign w_p} + E,  A = clamp(1 - T, 0, 1)
 * with w the unit toward-light vector of light l in the camera frame of cam.
 *   lights         n_lights in [0, 64]
 *   rgba_dev       output [4][H][W] float32 */
NSL_API nsl_status nsl_shade(nsl_ctx* ctx, const float* lightmaps_dev, int width, int height,
                     const nsl_camera* cam, const nsl_light* lights, int n_lights,
                     float* rgba_dev, void* stream);

/* One whole frame from HOST buffers: copies density (and mask) to the device,
 * runs the guide, the network and the shading, copies guide, lightmaps and
 * rgba back, and synchronises `stream`.  Host pointers may be NULL for outputs
 * that are not wanted.  Uses context-owned device staging buffers.  The copies
 * run on a copy stream owned by the context, overlapped with the kernels on
 * `stream` (the grid goes up in slabs of z slices, each staged on arrival; the
 * guide comes back while the network runs, the lightmaps while shading runs);
 * `stream` waits for that copy stream before the call returns, so the frame is
 * complete when `stream` is.  The outputs equal those of the device-buffer
 * calls bit for bit.
 *   density_host  grid.dtype elements; mask_host may be NULL */
NSL_API nsl_status nsl_render_frame_host(nsl_ctx* ctx, const void* density_host,
                                 const uint8_t* mask_host, const nsl_camera* cam,
                                 const nsl_light* lights, int n_lights, float step_voxels,
                                 const nsl_march_opts* opts, int precision, float* guide_host,
                                 float* lightmaps_host, float* rgba_host, void* stream);

/* nsl_render_frame_host without the final synchronisation: every copy and
 * kernel is enqueued (on `stream` and on the context's copy stream, which
 * `stream` then waits for) and the call returns.  With page-locked host
 * buffers the copies run asynchronously, so frames of two contexts on two
 * streams overlap one frame's copies with the other's kernels.  The caller
 * must not change the inputs nor read the outputs until the stream has
 * completed, and must not issue the next frame of the same context on another
 * stream before that (the context's device buffers are reused). */
NSL_API nsl_status nsl_render_frame_host_async(nsl_ctx* ctx, const void* density_host,
                                       const uint8_t* mask_host, const nsl_camera* cam,
                                       const nsl_light* lights, int n_lights, float step_voxels,
                                       const nsl_march_opts* opts, int precision,
                                       float* guide_host, float* lightmaps_host, float* rgba_host,
                                       void* stream);

/* ---------------------------------------------------------------------------
 * Batched frames: many plumes of different grid and billboard sizes per call.
 * Every stage runs as one launch over all plumes (staging, the guide march,
 * each network layer, shading), so the launch count does not grow with the
 * number of plumes.  The method is that of the single-plume calls. The
 * guide agrees with theirs to rounding, because the grouped march takes every
 * shadow sample at its exact position and stages float16 grids as float32.
 * The network and the shading are bit-identical given the same guide.
 * ------------------------------------------------------------------------- */
typedef struct {
  const void* density_dev;   /* [nz][ny][nx], grid.dtype */
  const uint8_t* mask_dev;   /* obstacle mask or NULL */
  nsl_grid_desc grid;
  nsl_camera camera;         /* billboard size = camera.width x camera.height */
  float step_voxels;         /* march step h */
  nsl_light light;           /* light for the shading of this plume */
  float* guide_dev;          /* out [3][H][W] */
  float* lightmaps_dev;      /* out [8][H][W] */
  float* rgba_dev;           /* out [4][H][W], or NULL to skip the shading */
} nsl_plume;

typedef struct nsl_batch nsl_batch;

/* Create a batch context for up to max_plumes (<= 64) plumes per call with
 * the network weights of an NSLW blob (see nsl_create; C0 = 16 only, other
 * widths return NSL_ERR_UNSUPPORTED).  Device buffers are
 * sized by the first call and grow when a later call needs more. */
NSL_API nsl_status nsl_batch_create(const void* weights_blob, size_t blob_bytes, int max_plumes,
                                    nsl_batch** out);
NSL_API void nsl_batch_destroy(nsl_batch* b);

/* Guide, lightmaps and (where rgba_dev is set) shading for n plumes, with one
 * set of march options for all; precision NSL_PREC_F16, NSL_PREC_BF16,
 * NSL_PREC_FP8 or NSL_PREC_BF16X3 (the split-BF16 form, see
 * nsl_predict_lightmaps; its per-plume network scratch is about twice that of
 * the 16-bit forms).
 * Asynchronous on `stream`; the caller owns every buffer of `plumes`. */
NSL_API nsl_status nsl_batch_render(nsl_batch* b, const nsl_plume* plumes, int n,
                                    const nsl_march_opts* opts, int precision, void* stream);

/* Capture one nsl_batch_render of exactly these plumes into a CUDA graph
 * (after one ordinary render, so that nothing is allocated while capturing);
 * `stream` must not be the legacy default stream.  nsl_batch_launch_graph
 * replays it; between replays nsl_batch_update_graph may change cameras,
 * lights, sigma scales and march options (buffers, grid and billboard sizes
 * and steps must stay those of the capture, else NSL_ERR_INVALID_ARG); call it
 * only once the previous replay has completed.  All calls on one batch must be
 * ordered on one stream (or synchronised): they share its scratch buffers. */
NSL_API nsl_status nsl_batch_capture_graph(nsl_batch* b, const nsl_plume* plumes, int n,
                                           const nsl_march_opts* opts, int precision,
                                           void* stream);
NSL_API nsl_status nsl_batch_update_graph(nsl_batch* b, const nsl_plume* plumes, int n,
                                          const nsl_march_opts* opts);
NSL_API nsl_status nsl_batch_launch_graph(nsl_batch* b, void* stream);

/* Tuning knobs of the batched path: view steps per segment of the march (1..64),
 * march CTAs per SM (0 = occupancy maximum), convolution CTAs per SM (1..4).
 * Changing them (nsl_batch_autotune does) drops a captured graph, as does a
 * render that has to grow a device buffer; capture again afterwards. */
NSL_API nsl_status nsl_batch_set_tuning(nsl_batch* b, int seg_len, int march_blocks_per_sm,
                                        int conv_ctas_per_sm);
NSL_API nsl_status nsl_batch_get_tuning(const nsl_batch* b, int* seg_len, int* march_blocks_per_sm,
                                        int* conv_ctas_per_sm);
/* Pixel tile of one warp of the batched march: tile_width x (32 / tile_width)
 * pixels, tile_width 2, 4, 8 (the default) or 16.  Every pixel's march is the
 * same whatever the tile, so results are bitwise unchanged; a change drops a
 * captured graph. */
NSL_API nsl_status nsl_batch_set_march_tile(nsl_batch* b, int tile_width);
NSL_API nsl_status nsl_batch_get_march_tile(const nsl_batch* b, int* tile_width);
/* Launch form of the batched march: persistent = 1 (the default) runs the view
 * pass, the segment pass and the finish pass in one cooperative launch of
 * resident CTAs separated by grid-wide barriers (each wait bounded at about
 * 2 s; a barrier that gives up records an error that the next render reports
 * as NSL_ERR_TIMEOUT); persistent = 0 runs them as three launches.  Results
 * are bitwise the same.  A cooperative launch needs every one of its CTAs
 * resident at once, so batches rendered concurrently on several streams (as a
 * server's slots are) use the three-launch form.  A change drops a captured
 * graph. */
NSL_API nsl_status nsl_batch_set_march_form(nsl_batch* b, int persistent);
NSL_API nsl_status nsl_batch_get_march_form(const nsl_batch* b, int* persistent);

/* Autotuner: renders the batch under each candidate setting of the march's
 * knobs (launch form persistent or three passes x tile width 8 or 4 x segment
 * length 4, 6 or 8 x march CTAs per SM), then of the convolutions' CTAs per SM
 * (1, 2, 4), times each with CUDA
 * events (median of 3) and keeps the fastest.  With
 * a cache path (JSON lines), a result stored for the same batch signature
 * (sizes, steps, precision) is applied without timing and new results are
 * appended.  Synchronises `stream`; *best_ms (may be NULL) gets the time. */
NSL_API nsl_status nsl_batch_autotune(nsl_batch* b, const nsl_plume* plumes, int n,
                                      const nsl_march_opts* opts, int precision,
                                      const char* cache_path, void* stream, float* best_ms);

/* ---------------------------------------------------------------------------
 * Serving: a frame-request loop over plumes kept resident on the device.
 *
 * Plumes are registered with their density on the host.  A plume is admitted
 * (its grid uploaded and staged, its guide / lightmap / RGBA state allocated)
 * when a request for it is scheduled and the device bytes it needs fit in the
 * HBM budget; otherwise the least recently used idle plumes are evicted first.
 * One scheduler thread batches queued requests of different grid and billboard
 * sizes as they arrive: whenever one of `streams` batch slots is free it takes
 * the oldest queued requests (at most one per plume, up to max_batch, within
 * the slot's scratch) and launches them as one batched render on that slot's
 * stream, so batches overlap on the device and later arrivals join the next
 * free slot (continuous batching).  Requests for one plume run in arrival order.
 * Each frame is the guide march, the network and shading of nsl_batch_render
 * with the server's march options; results are bitwise the same whichever
 * batch a request lands in.  The paper has no serving layer: this is a systems
 * form around its per-frame method.
 * ------------------------------------------------------------------------- */
typedef struct nsl_server nsl_server;

typedef struct {
  size_t hbm_budget_bytes;         /* device bytes for resident plumes + slot scratch */
  size_t scratch_bytes_per_stream; /* march + network scratch of one batch slot (0: budget/8) */
  int streams;                     /* batch slots in flight at once, 1..4 */
  int max_batch;                   /* requests per batch, 1..64 */
  int precision;                   /* NSL_PREC_F16, NSL_PREC_BF16, NSL_PREC_FP8 or NSL_PREC_BF16X3 */
  nsl_march_opts march;            /* march options of every frame */
  size_t max_batch_pixels;         /* billboard pixels a batch may hold (0: no cap); the
                                      oldest runnable request is always taken, later ones
                                      only while the batch stays under the cap, so a few
                                      large frames do not hold many small ones back */
  size_t small_first_pixels;       /* requests of at most this many pixels are taken
                                      into a forming batch before larger ones (0: plain
                                      arrival order); a plume's requests keep their order */
} nsl_server_opts;

typedef struct {
  uint64_t submitted, completed, failed, queued, running;
  uint64_t batches, admissions, evictions;
  double pixels_completed;         /* billboard pixels of completed requests */
  int resident_plumes;
  size_t resident_bytes;           /* staged grids + state of resident plumes */
  size_t used_bytes;               /* resident_bytes + slot scratch and upload buffers */
  size_t budget_bytes;
  double p50_ms, p99_ms, max_ms;   /* submit -> lightmaps ready, completed requests */
  double mean_batch;               /* requests per launched batch */
  double busy_s;                   /* first submit -> last completion */
} nsl_server_stats;

/* Defaults: 40 GiB budget, 2 streams, batches of up to 64 requests and
 * 1 Mi billboard pixels, requests of up to 256 x 256 pixels first, FP16
 * network. */
NSL_API void nsl_default_server_opts(nsl_server_opts* o);
NSL_API nsl_status nsl_server_create(const void* weights_blob, size_t blob_bytes,
                                     const nsl_server_opts* opts, nsl_server** out);
/* Waits for work in flight, then frees everything (host registrations too). */
NSL_API void nsl_server_destroy(nsl_server* s);

/* Register a plume.  density_host (grid->dtype elements, [nz][ny][nx]) and
 * mask_host (nullable) must stay valid until the plume is removed: they are
 * re-read whenever the plume is admitted again after an eviction; the server
 * page-locks them for fast uploads.  Requests may use billboards up to
 * max_width x max_height.  NSL_ERR_BUDGET if the plume alone cannot fit. */
NSL_API nsl_status nsl_server_add_plume(nsl_server* s, const nsl_grid_desc* grid,
                                        const void* density_host, const uint8_t* mask_host,
                                        float step_voxels, int max_width, int max_height,
                                        int* plume_id);
/* NSL_ERR_INVALID_ARG while the plume has queued or running requests. */
NSL_API nsl_status nsl_server_remove_plume(nsl_server* s, int plume_id);

/* Queue one frame of a plume (thread-safe).  lightmaps_dev ([8][H][W]) and
 * rgba_dev ([4][H][W]) are optional caller buffers for this request's output;
 * NULL writes the plume's resident state instead (see nsl_server_plume_state).
 * The server's streams do not wait on the caller's: output buffers must be
 * ready (no pending work on them) at submit and stay allocated until the
 * request completes.  The latency clock starts here. */
NSL_API nsl_status nsl_server_submit(nsl_server* s, int plume_id, const nsl_camera* cam,
                                     const nsl_light* light, float* lightmaps_dev, float* rgba_dev,
                                     uint64_t* request_id);
/* Block until the request completes (NSL_OK, latency in ms), fails (its error),
 * or timeout_ms passes (NSL_ERR_TIMEOUT; the request carries on). */
NSL_API nsl_status nsl_server_wait(nsl_server* s, uint64_t request_id, double timeout_ms,
                                   double* latency_ms);
/* Block until nothing is queued or running (NSL_ERR_TIMEOUT after timeout_ms). */
NSL_API nsl_status nsl_server_drain(nsl_server* s, double timeout_ms);
/* Device pointers of a plume's resident guide / lightmaps / RGBA state: the
 * last request's [3|8|4][H][W] planes (its width and height) at the start of
 * buffers sized for the plume's largest billboard; NULL and *resident = 0
 * when evicted.  Valid until the next request
 * for the plume is scheduled or the plume is evicted. */
NSL_API nsl_status nsl_server_plume_state(nsl_server* s, int plume_id, const float** guide_dev,
                                          const float** lightmaps_dev, const float** rgba_dev,
                                          int* resident);
NSL_API nsl_status nsl_server_get_stats(nsl_server* s, nsl_server_stats* out);
/* Clears the latency record and counters (not the resident set). */
NSL_API nsl_status nsl_server_reset_stats(nsl_server* s);

/* Description of the last error raised on the calling thread ("" if none). */
NSL_API const char* nsl_last_error(void);
NSL_API const char* nsl_status_str(nsl_status s);

#ifdef __cplusplus
}
#endif
#endif /* NSL_H */
