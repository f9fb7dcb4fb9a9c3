/* FP64 CPU oracle for the neural six-way lightmap hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: it is written from the paper (Sec. 3 six-way
 * interpolation, Sec. 4.2 guiding map / Alg. 1 / Eq. approx, Sec. 4.3
 * generator) and the readings listed in the design notes.
 *
 * Conventions: grids are [nz][ny][nx] (x fastest) in voxel units; images are
 * planar [C][H][W], row 0 at the top.
 */
#ifndef NSL_ORACLE_H
#define NSL_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int kind;               /* 0 orthographic, 1 perspective */
  float eye[3], target[3], up[3];
  float fov_y_deg, ortho_height;
  int width, height;
} nslo_camera;

typedef struct {
  float tau_depth;        /* depth threshold tau of Alg. 1 (per-voxel density) */
  float t_min;            /* early termination of view and shadow rays (0 = off) */
  int jitter;             /* 1: per-pixel hash jitter delta = u*h, 0: u = 0 */
  uint32_t seed, frame;
  float phase_g;          /* Henyey-Greenstein g (0 = isotropic 1/(4 pi)) */
  float surrogate_I[3];   /* intensities of the front, top, bottom lights */
  int segment_exact;      /* 0: A_n = T_{n-1} sigma_n h; 1: T_{n-1}(1-exp(-sigma_n h)) */
  float margin;           /* relative margin for threshold-decision flags */
  int light_set;          /* surrogate lights (Sec. 5, ablation on the guiding
                             light directions): 0 front/top/bottom, 1 front
                             only, 2 front/left/right */
  int shadow_volume;      /* 0: side-light shadows marched from every view
                             sample; 1: one shadow march per voxel centre into
                             two transmittance volumes, read trilinearly at the
                             view samples (an approximation) */
} nslo_march_opts;

typedef struct {
  float dir[3];           /* toward the light, world space */
  float intensity[3];
} nslo_light;

/* Guiding map (Alg. 1).  density: float32 [nz][ny][nx] (FP16 inputs are
 * widened exactly by the caller); mask: uint8 or NULL (non-zero = obstacle).
 * guide: double [3][H][W] = (L_scattering, T, D).  samples (nullable): int64
 * [H][W] density evaluations per pixel.  flags (nullable): uint8 [H][W], bit0 =
 * an early-termination decision lay within the margin, bit1 = a depth decision
 * lay within the margin.  Returns 0 on success. */
int nslo_guide(const float* density, const uint8_t* mask, int nx, int ny, int nz,
               double sigma_scale, const nslo_camera* cam, float h,
               const nslo_march_opts* opts, double* guide, int64_t* samples,
               uint8_t* flags);
/* Same as nslo_guide for image rows [row0, row1) only; other rows untouched. */
int nslo_guide_rows(const float* density, const uint8_t* mask, int nx, int ny, int nz,
                    double sigma_scale, const nslo_camera* cam, float h,
                    const nslo_march_opts* opts, int row0, int row1, double* guide,
                    int64_t* samples, uint8_t* flags);

/* Fine-step six-light single-scattering reference: 7 planes
 * [+X,-X,+Y,-Y,+Z,-Z,T] in the camera frame, midpoint rule with step hf. */
int nslo_reference_lightmaps(const float* density, const uint8_t* mask, int nx, int ny,
                             int nz, double sigma_scale, const nslo_camera* cam,
                             double hf, double phase_g, double* out);

/* Same for image rows [row0, row1) only; other rows untouched. */
int nslo_reference_lightmaps_rows(const float* density, const uint8_t* mask, int nx, int ny,
                                  int nz, double sigma_scale, const nslo_camera* cam, double hf,
                                  double phase_g, int row0, int row1, double* out);

/* Lightmap network forward (UNet + 4 NAFBlock adapters), all FP64.
 * guide: [3][H][W]; params: float64 values in the blob order; out: [8][H][W]. */
int nslo_net_forward(const double* guide, int H, int W, const double* params,
                     int64_t n_params, int c0, double depth_scale, double* out);

/* The same network with FP8 E4M3 convolutions (every 3x3 and transposed
 * convolution after the first): per-tensor power-of-two activation scales
 * (the smallest 2^k with amax <= 448 * 2^k) and per-output-channel weight
 * scales max|w|/448 in binary32, exact products summed, activations rounded
 * to binary16 between layers. */
int nslo_net_forward_q8(const double* guide, int H, int W, const double* params,
                        int64_t n_params, int c0, double depth_scale, double* out);
/* rounding primitives of that path */
double nslo_round_f16(double x);
double nslo_e4m3_rn(double x);
void nslo_q8_tensor(const double* x, size_t n, double* codes, float* deq);
void nslo_q8_weights(const double* w, int cout, int count, int64_t so, int64_t sj, double* codes,
                     float* s);

/* Per-layer precision forms of the network's 17 convolutions. */
enum {
  NSLO_PREC_F64 = 0,    /* exact */
  NSLO_PREC_F16 = 1,    /* binary16 weights and activations, exact sums */
  NSLO_PREC_BF16 = 2,   /* bfloat16 weights and activations, exact sums */
  NSLO_PREC_FP8 = 3,    /* the FP8 E4M3 scheme of nslo_net_forward_q8 */
  NSLO_PREC_BF16X3 = 4  /* bfloat16 hi/lo splits of weights and binary32
                           activations, hi*hi + hi*lo + lo*hi */
};
/* The network with convolution l (network order, 0 = enc1a .. 16 = dec1b) in
 * form prec[l]; the adapters in binary64 on the stored feature map.  trace
 * (nullable) receives the 17 stored layer outputs, planar, one after another. */
int nslo_net_forward_prec(const double* guide, int H, int W, const double* params,
                          int64_t n_params, int c0, double depth_scale, const int* prec,
                          double* out, double* trace);
int64_t nslo_net_trace_size(int c0, int H, int W, int l);
/* One convolution in form prec with explicit weights (k = 3: 3x3 + ReLU; k = 2:
 * 2x2 stride-2 transposed), and the storage rounding of a form. */
int nslo_conv_layer_prec(int prec, int k, const double* x, int cin, int H, int W, const double* w,
                         const double* b, int cout, double* out);
void nslo_store_as(int prec, const double* x, size_t n, double* out);
/* The adapters and heads alone on a feature map F [c0][H][W]. */
int nslo_net_adapters(const double* F, int c0, int H, int W, const double* params, int64_t n_params,
                      double* out);
double nslo_round_bf16(double x);

/* Six-way shading: rgba [4][H][W]. */
int nslo_shade(const double* lightmaps, int H, int W, const nslo_camera* cam,
               const nslo_light* lights, int n_lights, double* rgba);

/* primitives, exposed for pinning against closed forms and library routines */
double nslo_sample_sigma(const float* density, const uint8_t* mask, int nx, int ny,
                         int nz, double sigma_scale, const float p[3]);
double nslo_hg_phase(double g, double cos_theta);
uint32_t nslo_pcg_hash(uint32_t v);
void nslo_conv2d(const double* in, int cin, int H, int W, const double* w,
                 const double* b, int cout, int k, double* out);
void nslo_conv_transpose2x2(const double* in, int cin, int H, int W, const double* w,
                            const double* b, int cout, double* out);
void nslo_maxpool2(const double* in, int C, int H, int W, double* out);
void nslo_layernorm(const double* in, int C, int H, int W, const double* g,
                    const double* b, double eps, double* out);
void nslo_dwconv3(const double* in, int C, int H, int W, const double* w,
                  const double* b, double* out);
int nslo_nafblock(const double* in, int C, int H, int W, const double* params,
                  double* out);
int64_t nslo_nafblock_params(int C);

#ifdef __cplusplus
}
#endif

/* Obstacle shadowing (Sec. 4.5).  Shadow map of the obstacle mask for one
 * directional light (dir toward the light): R x R float32, texel (i, j) = the
 * entry parameter of the first occupied voxel along its light ray, +inf for
 * none.  Returns 0 on success. */
int nslo_shadow_map(const uint8_t* mask, int nx, int ny, int nz, const float dir[3], int R,
                    float* out);
/* nslo_shade with each light's term times the visibility of the pixel's smoke
 * shell (guide depth D) against that light's shadow map (maps[l] may be NULL). */
int nslo_shade_shadowed(const double* lm, const float* guide, int H, int W, const nslo_camera* cam,
                        const nslo_light* lights, int n_lights, int nx, int ny, int nz,
                        const float* const* maps, int R, float bias, double* rgba);
#endif
