// Internal declarations of libnsl (GB300 / sm_103a).  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/nsl.h"

#ifndef NSL_PDL
#define NSL_PDL 1   // network kernels use programmatic dependent launch
#endif

namespace nsl {
// Programmatic dependent launch (griddepcontrol).  A kernel started by
// launch_pdl may begin while its predecessor in the stream is finishing: it
// does its set-up (barriers, tensor memory, weights), then calls pdl_wait()
// before its first access to memory the predecessor writes or reads, and
// pdl_trigger() so that its own successor may start early.  Both are no-ops
// in a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#ifndef NSL_PDL_TRIGGER
#define NSL_PDL_TRIGGER 2   // 1: successor released once a kernel passed its wait, 2: at its end,
                            // 3: when each persistent CTA starts its last work item
#endif
__device__ __forceinline__ void pdl_trigger() { if (NSL_PDL_TRIGGER == 1) pdl_launch(); }
__device__ __forceinline__ void pdl_trigger_end() { if (NSL_PDL_TRIGGER == 2) pdl_launch(); }
__device__ __forceinline__ void pdl_trigger_last() { if (NSL_PDL_TRIGGER == 3) pdl_launch(); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = NSL_PDL;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
}  // namespace nsl

namespace nsl {

// Streaming multiprocessors of the current device
// (cudaDevAttrMultiProcessorCount; 152 on GB300), looked up once per device.
int num_sms();
constexpr int kMaxGroup = 64;   // images per grouped network launch / plumes per batch launch

// Error recording (thread-local message, see nsl_last_error).
void set_error(const char* fmt, ...);
nsl_status fail(nsl_status s, const char* fmt, ...);
nsl_status cuda_fail(cudaError_t e, const char* where);

#define NSL_CUDA_TRY(expr)                                     \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) return ::nsl::cuda_fail(_e, #expr); \
  } while (0)

// ---------------------------------------------------------------------------
// camera frame (binary32), computed on the host in binary64 and rounded once
// ---------------------------------------------------------------------------
struct CamFrame {
  float eye[3], r[3], u[3], f[3];
  float ax, ay;  // screen extents (ortho: height*W/H, height; persp: 2tan(fov/2)*W/H, 2tan(fov/2))
  int kind, W, H;
};
void cam_frame_from(const nsl_camera& c, CamFrame* out);

// Obstacle shadowing (Sec. 4.5): a directional light's frame and map square.
struct LightFrame {
  float w[3], e1[3], e2[3], c[3], S;
};
bool light_frame_from(const float dir[3], int nx, int ny, int nz, LightFrame* L);
constexpr int kMaxShadowLights = 16;
struct ShadowLight {
  float M[3][6];       // this light's six-way weights times its intensity
  LightFrame F;
  const float* map;    // [R][R] first-hit depths, or null (no obstacle shadow)
};
struct ShadowShadeArgs {
  const float* lm;     // [8][H][W]
  const float* guide;  // [3][H][W], depth D in plane 2
  float* rgba;         // [4][H][W]
  int W, H, R, n_lights;
  float bias, fx, fy, fz;
  CamFrame cam;
  ShadowLight light[kMaxShadowLights];
};
cudaError_t launch_shadow_map(const uint8_t* mask, int nx, int ny, int nz, const LightFrame& L, int R,
                              float* out, cudaStream_t s);
cudaError_t launch_shade_shadowed(const ShadowShadeArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// guide march
// ---------------------------------------------------------------------------
struct MarchPlume {
  const float* vol;   // staged extinction sigma' = scale*rho*[mask==0], padded quad layout, fp32
                      // (staged_half: FP16 quads of rho*[mask==0], sigma = scl * value)
  int staged_half;
  int staged_octo;    // vol holds float32 octo cells (single-plume contexts)
  float scl;
  int nx, ny, nz;
  CamFrame cam;
  float h;            // step in voxels
  float tau_depth;
  float t_min;        // view-ray early termination (0 = off)
  float tau_lim;      // shadow-ray termination threshold on the optical depth (-ln t_min)
  int jitter;
  uint32_t key;       // pcg(frame + pcg(seed))
  float g;            // HG parameter of the surrogate lights
  float I[3];         // front, top, bottom intensities
  int segment_exact;
  int light_set;      // NSL_LIGHTS_FTB / _F / _FLR
  int shadow_volume;  // side-light transmittances read from volT / volB
  const float* volT;  // staged transmittance volumes (top / bottom), padded quad layout
  const float* volB;
  float* guide;       // [3][H][W]
  int tiles_x;        // tiles per row
  int tx_log2;        // march tile: 2^tx_log2 x 2^(5 - tx_log2) pixels per warp (3: 8 x 4)
  int tile_start;     // first tile index of this plume in a batch
  unsigned long long* counter;  // density-evaluation counter (counting variant only)
  // segmented march scratch ([segment][pixel]) and the segment length S
  int seg_len;
  int* seg_nef;       // [pixel] processed view steps
  float* seg_tau;     // [segment][pixel] optical depth at the segment start
  float* seg_comp;    // [segment][pixel] its Kahan compensation
  float* seg_L;       // [segment][pixel] partial guide radiance
};

#ifndef NSL_MARCH_MIN_BLOCKS
#define NSL_MARCH_MIN_BLOCKS 7
#endif
#ifndef NSL_MARCH_SEG
#define NSL_MARCH_SEG 6
#endif
constexpr int kMarchSegLen = NSL_MARCH_SEG;  // view steps per segment of the segmented march
#ifndef NSL_MARCH_TX
#define NSL_MARCH_TX 8
#endif
constexpr int kMarchTX = NSL_MARCH_TX;  // default march tile: TX x (32/TX) pixels, one warp
constexpr int kMarchTY = 32 / kMarchTX;
constexpr int kMarchTXLog2 =
    kMarchTX == 16 ? 4 : (kMarchTX == 8 ? 3 : (kMarchTX == 4 ? 2 : (kMarchTX == 2 ? 1 : 0)));
static_assert((1 << kMarchTXLog2) == kMarchTX, "march tile width: 1, 2, 4, 8 or 16");
constexpr int kMarchThreads = 128;   // 4 independent warps per block
constexpr int kMarchMinBlocks = NSL_MARCH_MIN_BLOCKS;  // register cap for occupancy

// Order of the staged quad cells in memory: 0 = x fastest, then y, then z;
// 1 = y fastest, then x, then z.  Slices (z) are outermost in both, so the
// quad of slice z+1 is one plane (PX * PY cells) further on.
#ifndef NSL_MARCH_ORDER
#define NSL_MARCH_ORDER 0
#endif
constexpr int kMarchOrder = NSL_MARCH_ORDER;
static_assert(kMarchOrder == 0 || kMarchOrder == 1, "staged cell order: 0 (x fastest) or 1 (y fastest)");
// Staged grid layouts (grid_sample.cuh): quad cells, (nx+1)(ny+1)(nz+2) of 4
// values (float32 or float16), for every form; octo cells, (nx+1)(ny+1)(nz+1)
// of 8 float32 values, for single-plume float32 contexts whose octo grid fits
// the L2 share below (one 32-byte load per sample instead of two 16-byte ones).
__host__ __device__ inline size_t staged_cells(int nx, int ny, int nz) {
  return (size_t)(nx + 1) * (ny + 1) * (nz + 2);
}
__host__ __device__ inline size_t staged_cells_octo(int nx, int ny, int nz) {
  return (size_t)(nx + 1) * (ny + 1) * (nz + 1);
}
inline size_t staged_octo_bytes(int nx, int ny, int nz) { return staged_cells_octo(nx, ny, nz) * 8 * sizeof(float); }
// Grid sizes the march accepts: every axis in [1, 4096] and fewer than 2^32
// staged cells (the march addresses staged cells with 32-bit indices).
inline bool grid_dims_ok(int nx, int ny, int nz) {
  if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096) return false;
  return staged_cells(nx, ny, nz) < ((size_t)1 << 32);
}
inline size_t staged_floats(int nx, int ny, int nz) { return staged_cells(nx, ny, nz) * 4; }
cudaError_t launch_transmittance_volume(const MarchPlume& p, float* outT, float* outB, cudaStream_t s);
// Staging of the cell planes [c0, c1) of the padded quad layout (c1 < 0: to the
// last plane, nz + 1).  Cell plane cz reads density slice min(max(cz - 1, 0),
// nz - 1) only, so the planes of a slab of slices can be staged as soon as that
// slab has arrived.
cudaError_t launch_stage_volume(const void* density, int dtype, const uint8_t* mask, int nx,
                                int ny, int nz, float scale, float* staged, cudaStream_t s, int c0 = 0,
                                int c1 = -1);
cudaError_t launch_stage_volume_half(const __half* density, const uint8_t* mask, int nx, int ny, int nz,
                                     __half* staged, cudaStream_t s, int c0 = 0, int c1 = -1);
// Octo staging (float32 values sigma' as in the quad layout): cell plane cz in
// [0, nz] holds slices min(max(cz - 1, 0), nz - 1) and min(cz, nz - 1); planes
// [c0, c1) (c1 < 0: to the last plane, nz).
cudaError_t launch_stage_volume_octo(const void* density, int dtype, const uint8_t* mask, int nx, int ny, int nz,
                                     float scale, float* staged, cudaStream_t s, int c0 = 0, int c1 = -1);
int march_tiles(int W, int H, int tx_log2 = kMarchTXLog2);
cudaError_t launch_march(const MarchPlume& p, int* tile_counter, cudaStream_t s,
                         bool count = false);
int march_max_segments(int nx, int ny, int nz, float h, int seg_len);
cudaError_t launch_march_segmented(const MarchPlume& p, int max_segments, int* tile_counter,
                                   cudaStream_t s);
// fine-step six-light reference lightmaps [7][H][W] of the staged grid (reference.cu)
cudaError_t launch_reference_lightmaps(const MarchPlume& p, double hf, float g, float* out, cudaStream_t s);
// batched forms (device tables; see march.cu)
struct StageItem {
  const void* density;
  const uint8_t* mask;
  float* out;            // padded quad staging of this plume
  int nx, ny, nz, dtype;
  float scale;
  int half_out;          // a float16 grid staged as float16 quads of rho * [mask == 0]
                         // (sigma_scale applied by the march after the blend)
};
// Bytes of the staged grid of one plume: float16 quads for a float16 grid,
// float32 quads otherwise.
inline size_t staged_grid_bytes(const nsl_grid_desc& g) {
  return g.dtype == NSL_F16 ? staged_cells(g.nx, g.ny, g.nz) * 4 * sizeof(__half)
                            : staged_floats(g.nx, g.ny, g.nz) * sizeof(float);
}
int stage_batch_blocks(const StageItem& it);
cudaError_t launch_stage_batch(const StageItem* items_dev, const int* block_starts_dev, int n,
                               int total_blocks, cudaStream_t s);
cudaError_t launch_march_segmented_batch(const MarchPlume* table_dev, const int* tile_starts_dev,
                                         const int* item_starts_dev, const int* tile_counts_dev,
                                         int nplumes, int total_tiles, int total_items,
                                         int seg_blocks, int* counter, cudaStream_t s);
int march_segment_blocks_max();
// the batched march as one cooperative persistent launch (view pass, barrier,
// segment pass, barrier, finish pass); sync: three zero-initialised words
// (work queue, barrier arrivals, barrier generation); blocks <= 0 or above
// march_persistent_blocks_max(): every resident CTA
int march_persistent_blocks_max();
cudaError_t launch_march_persistent_batch(const MarchPlume* table_dev, const int* tile_starts_dev,
                                          const int* item_starts_dev, const int* tile_counts_dev, int nplumes,
                                          int total_tiles, int total_items, int blocks, unsigned* sync,
                                          unsigned* err, cudaStream_t s);
cudaError_t launch_march_batch(const MarchPlume* table_dev, int nplumes, int total_tiles,
                               int* tile_counter, cudaStream_t s);

// host helpers shared by the single-plume and batched entry points (api.cu)
nsl_status fill_march_plume(const nsl_grid_desc& grid, const nsl_camera& cam, float step,
                            const nsl_march_opts* opts, const char* fn, MarchPlume* p);
nsl_status check_camera_basic(const nsl_camera* cam, const char* fn);

// ---------------------------------------------------------------------------
// six-way shading
// ---------------------------------------------------------------------------
struct ShadeArgs {
  const float* lm;   // [8][H][W]
  float* rgba;       // [4][H][W]
  int W, H;
  float M[3][6];     // per colour channel: sum_l I_l,c * weight of plane q
};
cudaError_t launch_shade(const ShadeArgs& a, cudaStream_t s);
nsl_status shade_matrix(const nsl_camera& cam, const nsl_light* lights, int n_lights,
                        float M[3][6], const char* fn);
cudaError_t launch_shade_batch(const ShadeArgs* items_dev, const int* block_starts_dev, int n,
                               int total_blocks, cudaStream_t s);

// ---------------------------------------------------------------------------
// network
// ---------------------------------------------------------------------------
constexpr int kC0 = 16;        // base width of every network path
constexpr int kWideC0 = 32;    // the second base width, built in the FP32 path only
// floats of one adapter's parameters (LN1, pw1, dw, SCA, pw2, beta, LN2, ffn1,
// ffn2, gamma, head) at adapter width c
__host__ __device__ constexpr int adapter_param_count(int c) {
  return 2 * c + (2 * c * c + 2 * c) + (18 * c + 2 * c) + (c * c + c) + (c * c + c) + c + 2 * c +
         (2 * c * c + 2 * c) + (c * c + c) + c + 2 * c + 2;
}
constexpr int kAdapterParams = adapter_param_count(kC0);

// offsets (in floats) of every parameter tensor inside the flat NSLW payload
struct NetLayout {
  size_t conv_w[14], conv_b[14];   // enc1a..enc4b (8), dec3a,dec3b,dec2a,dec2b,dec1a,dec1b (6)
  int conv_cin[14], conv_cout[14];
  size_t up_w[3], up_b[3];         // up3, up2, up1
  int up_cin[3], up_cout[3];
  size_t adapter[4];               // start of each adapter's parameters (incl. head)
  size_t total;
  int c0;                          // base width
};
// Offsets of a blob of base width c0; false unless c0 is kC0 or kWideC0 (only
// the FP32 path runs kWideC0: callers of the other paths check c0 == kC0).
bool build_net_layout(int c0, NetLayout* L);

// device-side parameter sets of one adapter (offsets into a packed float array)
struct AdapterDev {
  const float* p;  // kAdapterParams floats in blob order
};

struct NetWorkspace;  // defined in net_*.cu

struct NetImage {     // one image of a (possibly batched) network call
  const float* guide; // [3][H][W]
  float* out;         // [8][H][W]
  int H, W;
  float depth_scale;
};

struct NetF32Weights;  // opaque
NetF32Weights* net_f32_create(const float* host_params, const NetLayout& L, cudaError_t* err);
void net_f32_destroy(NetF32Weights* w);
size_t net_f32_workspace_bytes(int max_w, int max_h, int c0 = kC0);
cudaError_t net_f32_forward(const NetF32Weights* w, const NetImage& img, void* workspace,
                            size_t ws_bytes, cudaStream_t s);
const float* net_f32_conv_w(const NetF32Weights* w, int l);  // SIMT-packed conv weights
const float* net_f32_conv_b(const NetF32Weights* w, int l);

// SIMT pieces shared with the tensor-core path
template <typename T>
cudaError_t simt_first_conv_half(const NetF32Weights* w, const NetImage& img, T* out,
                                 cudaStream_t s);

// NAFBlock adapters (adapters.cu): weights as kernel parameters, LayerNorm
// affines folded into the following 1x1 convolutions.
struct AdapterP1 {            // pass 1: pw1 (LN1 folded), depthwise 3x3
  float w1[4][2 * kC0][kC0];
  float b1[4][2 * kC0];
  float dww[4][2 * kC0][9];
  float dwb[4][2 * kC0];
};
struct AdapterSCA {           // simplified channel attention 1x1
  float w[4][kC0][kC0];
  float b[4][kC0];
};
struct AdapterP2 {            // pass 2: pw2, beta, ffn1 (LN2 folded), ffn2, gamma, head
  float w2[4][kC0][kC0];
  float b2[4][kC0];
  float beta[4][kC0];
  float f1[4][2 * kC0][kC0];
  float fb1[4][2 * kC0];
  float f2[4][kC0][kC0];
  float fb2[4][kC0];
  float gamma[4][kC0];
  float hw[4][2][kC0];
  float hb[4][2];
};
struct AdapterParamSet {
  AdapterP1 p1;
  AdapterSCA sca;
  AdapterP2 p2;
};
void adapter_params_from(const float* adapters_blob, AdapterP1* p1, AdapterSCA* sca,
                         AdapterP2* p2);
size_t adapter_partial_floats(int max_w, int max_h);
template <typename TA>
cudaError_t adapters_run(const AdapterParamSet& prm, const TA* F, TA* x1, float* partial,
                         float* att, float* out, int H, int W, cudaStream_t s);
// FP32 adapters at base width kWideC0 (weights in device memory, staged in
// shared memory per CTA); F, x1 [4][H][W][C], partial (adapter_wide_partial_floats)
struct AdapterWideWeights;
AdapterWideWeights* adapters_wide_create(const float* adapters_blob, cudaError_t* err);
void adapters_wide_destroy(AdapterWideWeights* w);
size_t adapter_wide_partial_floats(int max_w, int max_h);
cudaError_t adapters_wide_run(const AdapterWideWeights* w, const float* F, float* x1, float* partial,
                              float* mean, float* out, int H, int W, cudaStream_t s);
// one image of a grouped adapter launch (tensor-core passes and the reduction)
template <typename TA>
struct AdapterImg {
  const TA* F;
  __half* x1;       // the gated depthwise output: binary16 whatever F's type
                    // (it is LayerNorm-scaled, well inside the binary16 range),
                    // eight planes of 8 channels x H x W (16 bytes per pixel)
  float* partial;   // per-tile channel sums of this image
  float* att;       // 64 attention values of this image
  float* out;       // [8][H][W]
  int H, W;
};
// the SCA reduction alone (per image: partial tile sums -> att), two launches
template <typename TA>
cudaError_t adapters_reduce_only_group(const AdapterParamSet& prm, const AdapterImg<TA>* imgs, int n,
                                       cudaStream_t s);
// tensor-core adapters (adapters_tc.cu): pw1 with the depthwise 3x3 (as one
// 3x3 convolution), pw2, ffn1 and the heads folded through ffn2 on tcgen05
// with FP16 operands; same tiling and partial layout as the SIMT ones
struct AdapterTcWeights;
AdapterTcWeights* adapters_tc_create(const AdapterParamSet& prm, cudaError_t* err);
void adapters_tc_destroy(AdapterTcWeights* w);
template <typename TA>
cudaError_t adapters_tc_run_group(const AdapterTcWeights* w, const AdapterParamSet& prm,
                                  const AdapterImg<TA>* imgs, int n, unsigned int* err,
                                  cudaStream_t s);
// amax (nullable): per image, where the maximum of the stored outputs is
// accumulated (FP8 path)
template <typename T>
cudaError_t simt_first_conv_group(const NetF32Weights* w, const NetImage* imgs, T* const* outs,
                                  float* const* amax, int n, cudaStream_t s);
const AdapterParamSet& net_f32_adapter_params(const NetF32Weights* w);

// tensor-core (tcgen05) network: elem 0 = FP16 and 1 = BF16 operands
// (kind::f16), 2 = FP8 E4M3 operands (kind::f8f6f4) with per-tensor activation
// and per-output-channel weight scales; FP32 accumulation in TMEM, FP16
// activations between layers in the FP8 case
struct NetTcWeights;
NetTcWeights* net_tc_create(const float* host_params, const NetLayout& L, int elem,
                            cudaError_t* err);
void net_tc_destroy(NetTcWeights* w);
// workspace of a tensor-core network (elem 3, the split-BF16 form, keeps
// binary32 activations: about twice the bytes)
size_t net_tc_workspace_bytes(int max_w, int max_h, int elem = 0);
// tensor-core weight set of a precision: 0 FP16, 1 BF16, 2 FP8, 3 split BF16;
// -1 for a precision without one
inline int tc_elem_of(int precision) {
  switch (precision) {
    case NSL_PREC_F16: return 0;
    case NSL_PREC_BF16: return 1;
    case NSL_PREC_FP8: return 2;
    case NSL_PREC_BF16X3: return 3;
    default: return -1;
  }
}
constexpr int kTcElems = 4;
// trace (nullable): after each of the 17 convolutions a copy of its stored
// output (NHWC, 16-bit activation type) is appended; net_tc_trace_bytes bytes
cudaError_t net_tc_forward(const NetTcWeights* wt, const NetF32Weights* wf, const NetImage& img,
                           void* workspace, size_t ws_bytes, unsigned int* err_flag,
                           cudaStream_t s, uint8_t* trace = nullptr);
size_t net_tc_trace_bytes(int width, int height);
// grouped forward: n <= kMaxGroup images, image k uses workspace ws[k] of at
// least net_tc_workspace_bytes(W_k, H_k) bytes; every layer is one launch.
cudaError_t net_tc_forward_group(const NetTcWeights* wt, const NetF32Weights* wf,
                                 const NetImage* imgs, void* const* ws, int n,
                                 unsigned int* err_flag, cudaStream_t s);
// runtime tunable: CTAs per SM of the tensor-core convolutions (1..4)
void net_tc_set_ctas_per_sm(int v);

// CTAs of a tensor-memory kernel that fit on one SM (net_tc.cu)
cudaError_t launch_wait_timeout_probe(unsigned int* err, cudaStream_t s);
int tc_ctas_per_sm(const void* kernel, int threads, int dyn_smem, int tmem_cols);

// ---- batched frames (batch.cu), used by the server ----
void batch_plume_scratch(const nsl_plume& p, int seg_len, size_t* seg_bytes, size_t* net_bytes,
                         int precision = NSL_PREC_F16);
nsl_status batch_render_prestaged(nsl_batch* b, const nsl_plume* plumes, const float* const* staged,
                                  int n, const nsl_march_opts* opts, int precision, cudaStream_t s);
nsl_status batch_reserve(nsl_batch* b, size_t seg_bytes, size_t net_bytes, cudaStream_t s);
int batch_seg_len(const nsl_batch* b);
int net_tc_ctas_per_sm();

}  // namespace nsl
