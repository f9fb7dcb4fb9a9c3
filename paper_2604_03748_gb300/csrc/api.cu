// C ABI of libnsl: argument checking, contexts and orchestration of the
// kernels of the guide march (Sec. 4.2), the lightmap network (Sec. 4.3) and
// the six-way shading (Sec. 3).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "nsl_internal.cuh"

namespace nsl {

static thread_local char g_err[512] = "";

int num_sms() {
  constexpr int kMaxDev = 64;
  static int cached[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 152;
  int v = __atomic_load_n(&cached[dev], __ATOMIC_ACQUIRE);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
  __atomic_store_n(&cached[dev], v, __ATOMIC_RELEASE);
  return v;
}

// A single-plume float32 grid is staged as octo cells (one 32-byte load per
// trilinear sample instead of two 16-byte ones: 3-4% faster marches measured
// on the 128^3 workload) while the octo grids of all live contexts on the
// device take at most 60% of its L2 (81 MB of GB300's 135.5 MB; 68.7 MB at
// 128^3), so that a grid stays resident across its march like a quad grid
// even when several contexts' frames run at once: two 128^3 octo grids in
// flight together overflowed the L2 and halved the two-stream rate.  Larger
// grids, further contexts, float16 grids, batches and serving keep quad cells,
// which take half the bytes.  octo_reserve() books the grid's bytes,
// octo_release() returns them when the context is destroyed.
namespace {
std::mutex g_octo_mu;
size_t g_octo_bytes[64] = {};
}  // namespace

bool octo_reserve(int dev, size_t bytes) {
  int l2 = 0;
  if (dev < 0 || dev >= 64 || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lk(g_octo_mu);
  if ((double)(g_octo_bytes[dev] + bytes) > 0.6 * (double)l2) return false;
  g_octo_bytes[dev] += bytes;
  return true;
}

void octo_release(int dev, size_t bytes) {
  if (dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(g_octo_mu);
  g_octo_bytes[dev] = g_octo_bytes[dev] >= bytes ? g_octo_bytes[dev] - bytes : 0;
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

nsl_status fail(nsl_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}

nsl_status cuda_fail(cudaError_t e, const char* where) {
  set_error("%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? NSL_ERR_OOM : NSL_ERR_CUDA;
}

// Camera basis in binary64, rounded once to binary32 (same sequence as any
// other evaluation that must agree on integer decisions):
//   f = normalize(target - eye), r = normalize(f x up), u = r x f.
void cam_frame_from(const nsl_camera& c, CamFrame* fr) {
  double fx = (double)c.target[0] - (double)c.eye[0];
  double fy = (double)c.target[1] - (double)c.eye[1];
  double fz = (double)c.target[2] - (double)c.eye[2];
  double fl = std::sqrt(fx * fx + fy * fy + fz * fz);
  double Fx = fx / fl, Fy = fy / fl, Fz = fz / fl;
  double ux = c.up[0], uy = c.up[1], uz = c.up[2];
  double rx = Fy * uz - Fz * uy, ry = Fz * ux - Fx * uz, rz = Fx * uy - Fy * ux;
  double rl = std::sqrt(rx * rx + ry * ry + rz * rz);
  rx /= rl; ry /= rl; rz /= rl;
  double vx = ry * Fz - rz * Fy, vy = rz * Fx - rx * Fz, vz = rx * Fy - ry * Fx;
  for (int k = 0; k < 3; ++k) fr->eye[k] = c.eye[k];
  fr->f[0] = (float)Fx; fr->f[1] = (float)Fy; fr->f[2] = (float)Fz;
  fr->r[0] = (float)rx; fr->r[1] = (float)ry; fr->r[2] = (float)rz;
  fr->u[0] = (float)vx; fr->u[1] = (float)vy; fr->u[2] = (float)vz;
  fr->kind = c.kind; fr->W = c.width; fr->H = c.height;
  if (c.kind == NSL_CAM_ORTHO) {
    fr->ax = (float)(((double)c.ortho_height * (double)c.width) / (double)c.height);
    fr->ay = c.ortho_height;
  } else {
    double k = 2.0 * std::tan(((double)c.fov_y_deg * 3.14159265358979323846 / 180.0) * 0.5);
    fr->ax = (float)((k * (double)c.width) / (double)c.height);
    fr->ay = (float)k;
  }
}

bool build_net_layout(int c0, NetLayout* L) {
  size_t off = 0;
  const int c[4] = {c0, 2 * c0, 4 * c0, 8 * c0};
  auto conv = [&](int l, int cin, int cout) {
    L->conv_w[l] = off; off += (size_t)cout * cin * 9;
    L->conv_b[l] = off; off += cout;
    L->conv_cin[l] = cin; L->conv_cout[l] = cout;
  };
  auto up = [&](int l, int cin, int cout) {
    L->up_w[l] = off; off += (size_t)cin * cout * 4;
    L->up_b[l] = off; off += cout;
    L->up_cin[l] = cin; L->up_cout[l] = cout;
  };
  conv(0, 3, c[0]); conv(1, c[0], c[0]);
  conv(2, c[0], c[1]); conv(3, c[1], c[1]);
  conv(4, c[1], c[2]); conv(5, c[2], c[2]);
  conv(6, c[2], c[3]); conv(7, c[3], c[3]);
  up(0, c[3], c[2]); conv(8, c[3], c[2]); conv(9, c[2], c[2]);
  up(1, c[2], c[1]); conv(10, c[2], c[1]); conv(11, c[1], c[1]);
  up(2, c[1], c[0]); conv(12, c[1], c[0]); conv(13, c[0], c[0]);
  for (int a = 0; a < 4; ++a) {
    L->adapter[a] = off;
    off += adapter_param_count(c0);
  }
  L->total = off;
  L->c0 = c0;
  return c0 == kC0 || c0 == kWideC0;
}

}  // namespace nsl

using namespace nsl;

// nsl_render_frame_host uploads the density in this many slabs of z slices,
// staging each slab while the next one is copied.
constexpr int kUploadSlabs = 4;

struct nsl_ctx {
  nsl_grid_desc grid{};
  int max_w = 0, max_h = 0;
  int device = 0;
  std::vector<float> params;
  NetLayout layout{};
  float* staged = nullptr;          // staged extinction grid
  bool octo = false;                // float32 grid staged as octo cells (see octo_reserve)
  float* tvol = nullptr;            // transmittance volumes: raw top, raw bottom, staged top, staged bottom
  size_t tvol_bytes = 0;
  bool staged_valid = false;        // a staging has been queued
  unsigned long long* counter = nullptr;  // sample-count scratch
  int* tile_counter = nullptr;            // march tile queue (scratch)
  void* seg_scratch = nullptr;            // segmented-march scratch
  size_t seg_bytes = 0;
  NetF32Weights* wf32 = nullptr;
  NetTcWeights* wtc[kTcElems] = {}; // tensor-core weights: [0] FP16, [1] BF16, [2] FP8, [3] split BF16
                                    // (built on first use)
  void* ws = nullptr;               // network workspace (shared by both precisions)
  size_t ws_bytes = 0;
  unsigned int* err_host = nullptr; // device-written error word (mapped host memory)
  unsigned int* err_dev = nullptr;
  // device staging for nsl_render_frame_host
  void* h_density = nullptr;
  uint8_t* h_mask = nullptr;
  float* h_guide = nullptr;
  float* h_lm = nullptr;
  float* h_rgba = nullptr;
  // copy stream of nsl_render_frame_host and its events (created on first use)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev[kUploadSlabs + 4] = {};
};

static size_t grid_voxels(const nsl_grid_desc& g) { return (size_t)g.nx * g.ny * g.nz; }

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

extern "C" {

void nsl_default_march_opts(nsl_march_opts* o) {
  if (!o) return;
  o->tau_depth = 0.01f;
  o->t_min = 1e-4f;
  o->jitter = 1;
  o->seed = 0;
  o->frame = 0;
  o->phase_g = 0.f;
  o->surrogate_I[0] = o->surrogate_I[1] = o->surrogate_I[2] = 1.f;
  o->segment_exact = 0;
  o->light_set = NSL_LIGHTS_FTB;
  o->shadow_volume = 0;
}

const char* nsl_last_error(void) { return g_err; }

const char* nsl_status_str(nsl_status s) {
  switch (s) {
    case NSL_OK: return "ok";
    case NSL_ERR_INVALID_ARG: return "invalid argument";
    case NSL_ERR_OOM: return "out of device memory";
    case NSL_ERR_CUDA: return "CUDA error";
    case NSL_ERR_UNSUPPORTED: return "unsupported";
    case NSL_ERR_TIMEOUT: return "timeout";
    case NSL_ERR_BUDGET: return "over memory budget";
  }
  return "unknown status";
}

nsl_status nsl_create(const nsl_grid_desc* grid, const void* blob, size_t blob_bytes,
                      int max_width, int max_height, nsl_ctx** out) {
  if (!out) return fail(NSL_ERR_INVALID_ARG, "nsl_create: out is NULL");
  *out = nullptr;
  if (!grid || !blob) return fail(NSL_ERR_INVALID_ARG, "nsl_create: NULL grid or blob");
  if (!grid_dims_ok(grid->nx, grid->ny, grid->nz))
    return fail(NSL_ERR_INVALID_ARG, "nsl_create: grid dims out of range");
  if (grid->dtype != NSL_F32 && grid->dtype != NSL_F16)
    return fail(NSL_ERR_INVALID_ARG, "nsl_create: bad density dtype %d", grid->dtype);
  if (!(grid->sigma_scale >= 0.f) || !std::isfinite(grid->sigma_scale))
    return fail(NSL_ERR_INVALID_ARG, "nsl_create: bad sigma_scale");
  if (max_width < 8 || max_height < 8 || max_width % 8 || max_height % 8 || max_width > 8192 ||
      max_height > 8192)
    return fail(NSL_ERR_INVALID_ARG, "nsl_create: max size must be multiples of 8 in [8, 8192]");
  if (blob_bytes < 20) return fail(NSL_ERR_INVALID_ARG, "nsl_create: blob too small");
  const unsigned char* b = static_cast<const unsigned char*>(blob);
  if (std::memcmp(b, "NSLW", 4) != 0) return fail(NSL_ERR_INVALID_ARG, "nsl_create: bad magic");
  uint32_t ver, c0, nf;
  std::memcpy(&ver, b + 4, 4);
  std::memcpy(&c0, b + 8, 4);
  std::memcpy(&nf, b + 12, 4);
  if (ver != 1) return fail(NSL_ERR_INVALID_ARG, "nsl_create: blob version %u", ver);
  if ((size_t)nf * 4 + 20 != blob_bytes)
    return fail(NSL_ERR_INVALID_ARG, "nsl_create: blob size mismatch");
  NetLayout L{};
  if (!build_net_layout((int)c0, &L))
    return fail(NSL_ERR_UNSUPPORTED, "nsl_create: base width C0=%u (16 and 32 are built)", c0);
  if (L.total != nf) return fail(NSL_ERR_INVALID_ARG, "nsl_create: parameter count %u", nf);
  uint32_t chk = 0, stored;
  for (uint32_t i = 0; i < nf; ++i) {
    uint32_t w;
    std::memcpy(&w, b + 16 + 4 * (size_t)i, 4);
    chk += w;
  }
  std::memcpy(&stored, b + 16 + 4 * (size_t)nf, 4);
  if (chk != stored) return fail(NSL_ERR_INVALID_ARG, "nsl_create: blob checksum mismatch");

  nsl_ctx* c = new (std::nothrow) nsl_ctx();
  if (!c) return fail(NSL_ERR_OOM, "nsl_create: host allocation");
  c->grid = *grid;
  c->max_w = max_width;
  c->max_h = max_height;
  c->layout = L;
  c->params.resize(nf);
  std::memcpy(c->params.data(), b + 16, (size_t)nf * 4);
  cudaGetDevice(&c->device);
  c->octo = grid->dtype == NSL_F32 && octo_reserve(c->device, staged_octo_bytes(grid->nx, grid->ny, grid->nz));
  size_t sbytes = staged_floats(grid->nx, grid->ny, grid->nz) * sizeof(float);
  if (c->octo) sbytes = std::max(sbytes, staged_octo_bytes(grid->nx, grid->ny, grid->nz));
  cudaError_t e = cudaMalloc(&c->staged, sbytes);
  if (e != cudaSuccess) { nsl_destroy(c); return cuda_fail(e, "nsl_create: staged grid"); }
  e = cudaMalloc(&c->tile_counter, 256);
  if (e != cudaSuccess) { nsl_destroy(c); return cuda_fail(e, "nsl_create: tile counter"); }
  c->wf32 = net_f32_create(c->params.data(), L, &e);
  if (!c->wf32) { nsl_destroy(c); return cuda_fail(e, "nsl_create: FP32 weights"); }
  c->ws_bytes = net_f32_workspace_bytes(max_width, max_height, L.c0);
  if (L.c0 == kC0) {
    size_t tcb = net_tc_workspace_bytes(max_width, max_height);
    if (tcb > c->ws_bytes) c->ws_bytes = tcb;
  }
  e = cudaMalloc(&c->ws, c->ws_bytes);
  if (e != cudaSuccess) { nsl_destroy(c); return cuda_fail(e, "nsl_create: workspace"); }
  e = cudaHostAlloc(reinterpret_cast<void**>(&c->err_host), sizeof(unsigned int), cudaHostAllocMapped);
  if (e != cudaSuccess) { nsl_destroy(c); return cuda_fail(e, "nsl_create: error word"); }
  *c->err_host = 0;
  e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->err_dev), c->err_host, 0);
  if (e != cudaSuccess) { nsl_destroy(c); return cuda_fail(e, "nsl_create: error word"); }
  *out = c;
  return NSL_OK;
}

void nsl_destroy(nsl_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  if (c->octo) octo_release(c->device, staged_octo_bytes(c->grid.nx, c->grid.ny, c->grid.nz));
  cudaFree(c->staged);
  cudaFree(c->tvol);
  cudaFree(c->counter);
  cudaFree(c->tile_counter);
  cudaFree(c->seg_scratch);
  net_f32_destroy(c->wf32);
  for (NetTcWeights* w : c->wtc) net_tc_destroy(w);
  cudaFree(c->ws);
  if (c->err_host) cudaFreeHost(c->err_host);
  if (c->aux) cudaStreamDestroy(c->aux);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  cudaFree(c->h_density);
  cudaFree(c->h_mask);
  cudaFree(c->h_guide);
  cudaFree(c->h_lm);
  cudaFree(c->h_rgba);
  delete c;
}

static nsl_status check_camera(const nsl_ctx* c, const nsl_camera* cam, const char* fn) {
  if (!cam) return fail(NSL_ERR_INVALID_ARG, "%s: camera is NULL", fn);
  if (cam->kind != NSL_CAM_ORTHO && cam->kind != NSL_CAM_PERSP)
    return fail(NSL_ERR_INVALID_ARG, "%s: bad camera kind", fn);
  if (cam->width < 8 || cam->height < 8 || cam->width % 8 || cam->height % 8)
    return fail(NSL_ERR_INVALID_ARG, "%s: width/height must be positive multiples of 8", fn);
  if (cam->width > c->max_w || cam->height > c->max_h)
    return fail(NSL_ERR_INVALID_ARG, "%s: %dx%d exceeds the context maximum %dx%d", fn,
                cam->width, cam->height, c->max_w, c->max_h);
  double fx = (double)cam->target[0] - cam->eye[0], fy = (double)cam->target[1] - cam->eye[1],
         fz = (double)cam->target[2] - cam->eye[2];
  double fl = std::sqrt(fx * fx + fy * fy + fz * fz);
  if (!(fl > 0.0)) return fail(NSL_ERR_INVALID_ARG, "%s: eye == target", fn);
  double rx = fy * cam->up[2] - fz * cam->up[1], ry = fz * cam->up[0] - fx * cam->up[2],
         rz = fx * cam->up[1] - fy * cam->up[0];
  if (!(std::sqrt(rx * rx + ry * ry + rz * rz) > 1e-9 * fl))
    return fail(NSL_ERR_INVALID_ARG, "%s: up is parallel to the view direction", fn);
  if (cam->kind == NSL_CAM_PERSP && !(cam->fov_y_deg > 0.f && cam->fov_y_deg < 179.f))
    return fail(NSL_ERR_INVALID_ARG, "%s: fov_y_deg out of (0, 179)", fn);
  if (cam->kind == NSL_CAM_ORTHO && !(cam->ortho_height > 0.f))
    return fail(NSL_ERR_INVALID_ARG, "%s: ortho_height must be > 0", fn);
  return NSL_OK;
}

static uint32_t host_pcg(uint32_t v) {
  uint32_t state = v * 747796405u + 2891336453u;
  uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

// Stages cell planes [c0, c1) (c1 < 0: to the last) of the context's layout.
static cudaError_t stage_planes(nsl_ctx* c, const void* density, const uint8_t* mask, int c0, int c1,
                                cudaStream_t s) {
  const nsl_grid_desc& g = c->grid;
  if (g.dtype == NSL_F16)
    return launch_stage_volume_half(static_cast<const __half*>(density), mask, g.nx, g.ny, g.nz,
                                    reinterpret_cast<__half*>(c->staged), s, c0, c1);
  if (c->octo)
    return launch_stage_volume_octo(density, g.dtype, mask, g.nx, g.ny, g.nz, g.sigma_scale, c->staged, s, c0, c1);
  return launch_stage_volume(density, g.dtype, mask, g.nx, g.ny, g.nz, g.sigma_scale, c->staged, s, c0, c1);
}

nsl_status nsl_stage_grid(nsl_ctx* c, const void* density, const uint8_t* mask, void* stream) {
  if (!c) return fail(NSL_ERR_INVALID_ARG, "nsl_stage_grid: ctx is NULL");
  if (!density) return fail(NSL_ERR_INVALID_ARG, "nsl_stage_grid: density is NULL");
  if (!aligned16(density) || (mask && !aligned16(mask)))
    return fail(NSL_ERR_INVALID_ARG, "nsl_stage_grid: buffers must be 16-byte aligned");
  // an FP16 grid stays FP16 (half the march's gather bytes); sigma_scale is
  // applied after the trilinear blend
  cudaError_t e = stage_planes(c, density, mask, 0, -1, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "nsl_stage_grid");
  c->staged_valid = true;
  return NSL_OK;
}

}  // extern "C"

namespace nsl {
nsl_status fill_march_plume(const nsl_grid_desc& grid, const nsl_camera& cam, float step,
                            const nsl_march_opts* opts, const char* fn, MarchPlume* p) {
  if (!(step > 0.f) || !std::isfinite(step))
    return fail(NSL_ERR_INVALID_ARG, "%s: step must be > 0", fn);
  nsl_march_opts o;
  nsl_default_march_opts(&o);
  if (opts) o = *opts;
  if (!(o.t_min >= 0.f && o.t_min < 1.f))
    return fail(NSL_ERR_INVALID_ARG, "%s: t_min must be in [0, 1)", fn);
  if (!(o.phase_g > -1.f && o.phase_g < 1.f))
    return fail(NSL_ERR_INVALID_ARG, "%s: phase_g must be in (-1, 1)", fn);
  if (o.light_set < NSL_LIGHTS_FTB || o.light_set > NSL_LIGHTS_FLR)
    return fail(NSL_ERR_INVALID_ARG, "%s: bad light_set %d", fn, o.light_set);
  if (o.shadow_volume != 0 && o.shadow_volume != 1)
    return fail(NSL_ERR_INVALID_ARG, "%s: shadow_volume must be 0 or 1", fn);
  *p = MarchPlume{};
  p->nx = grid.nx; p->ny = grid.ny; p->nz = grid.nz;
  cam_frame_from(cam, &p->cam);
  p->h = step;
  p->tau_depth = o.tau_depth;
  p->t_min = o.t_min;
  p->tau_lim = o.t_min > 0.f ? (float)(-std::log((double)o.t_min)) : INFINITY;
  p->jitter = o.jitter ? 1 : 0;
  p->key = host_pcg(o.frame + host_pcg(o.seed));
  p->g = o.phase_g;
  for (int k = 0; k < 3; ++k) p->I[k] = o.surrogate_I[k];
  p->segment_exact = o.segment_exact ? 1 : 0;
  p->light_set = o.light_set;
  p->shadow_volume = o.shadow_volume && o.light_set != NSL_LIGHTS_F ? 1 : 0;
  p->tx_log2 = kMarchTXLog2;
  p->tiles_x = (cam.width + kMarchTX - 1) / kMarchTX;
  p->tile_start = 0;
  return NSL_OK;
}

nsl_status check_camera_basic(const nsl_camera* cam, const char* fn) {
  if (!cam) return fail(NSL_ERR_INVALID_ARG, "%s: camera is NULL", fn);
  if (cam->kind != NSL_CAM_ORTHO && cam->kind != NSL_CAM_PERSP)
    return fail(NSL_ERR_INVALID_ARG, "%s: bad camera kind", fn);
  if (cam->width < 8 || cam->height < 8 || cam->width % 8 || cam->height % 8 ||
      cam->width > 8192 || cam->height > 8192)
    return fail(NSL_ERR_INVALID_ARG, "%s: width/height must be multiples of 8 in [8, 8192]", fn);
  double fx = (double)cam->target[0] - cam->eye[0], fy = (double)cam->target[1] - cam->eye[1],
         fz = (double)cam->target[2] - cam->eye[2];
  double fl = std::sqrt(fx * fx + fy * fy + fz * fz);
  if (!(fl > 0.0)) return fail(NSL_ERR_INVALID_ARG, "%s: eye == target", fn);
  double rx = fy * cam->up[2] - fz * cam->up[1], ry = fz * cam->up[0] - fx * cam->up[2],
         rz = fx * cam->up[1] - fy * cam->up[0];
  if (!(std::sqrt(rx * rx + ry * ry + rz * rz) > 1e-9 * fl))
    return fail(NSL_ERR_INVALID_ARG, "%s: up is parallel to the view direction", fn);
  if (cam->kind == NSL_CAM_PERSP && !(cam->fov_y_deg > 0.f && cam->fov_y_deg < 179.f))
    return fail(NSL_ERR_INVALID_ARG, "%s: fov_y_deg out of (0, 179)", fn);
  if (cam->kind == NSL_CAM_ORTHO && !(cam->ortho_height > 0.f))
    return fail(NSL_ERR_INVALID_ARG, "%s: ortho_height must be > 0", fn);
  return NSL_OK;
}

// rgb_c = sum_q M[c][q] L_q + E: per colour channel the sum over lights of the
// light's intensity times the |w_p| weight of each of the six planes
nsl_status shade_matrix(const nsl_camera& cam, const nsl_light* lights, int n_lights,
                        float Mout[3][6], const char* fn) {
  CamFrame fr;
  cam_frame_from(cam, &fr);
  double M[3][6] = {};
  for (int l = 0; l < n_lights; ++l) {
    double v[3] = {lights[l].dir[0], lights[l].dir[1], lights[l].dir[2]};
    double nv = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(nv > 0.0) || !std::isfinite(nv))
      return fail(NSL_ERR_INVALID_ARG, "%s: light %d has a zero direction", fn, l);
    double w[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
      w[0] += v[k] / nv * fr.r[k];
      w[1] += v[k] / nv * fr.u[k];
      w[2] += v[k] / nv * fr.f[k];
    }
    for (int ch = 0; ch < 3; ++ch) {
      double I = lights[l].intensity[ch];
      for (int p = 0; p < 3; ++p) {
        if (w[p] >= 0.0) M[ch][2 * p] += I * w[p];
        else M[ch][2 * p + 1] += I * -w[p];
      }
    }
  }
  for (int ch = 0; ch < 3; ++ch)
    for (int q = 0; q < 6; ++q) Mout[ch][q] = (float)M[ch][q];
  return NSL_OK;
}
}  // namespace nsl

extern "C" {

static nsl_status march_setup(nsl_ctx* c, const nsl_camera* cam, float step,
                              const nsl_march_opts* opts, const char* fn, MarchPlume* p) {
  nsl_status st = check_camera(c, cam, fn);
  if (st != NSL_OK) return st;
  st = fill_march_plume(c->grid, *cam, step, opts, fn, p);
  if (st != NSL_OK) return st;
  p->vol = c->staged;
  p->staged_half = c->grid.dtype == NSL_F16;
  p->staged_octo = c->octo ? 1 : 0;
  if (c->octo) {   // 4 x 8 pixel tiles: measured 0.6% faster than 8 x 4 with octo cells
    p->tx_log2 = 2;
    p->tiles_x = (cam->width + 3) / 4;
  }
  p->scl = c->grid.sigma_scale;
  return NSL_OK;
}

nsl_status nsl_guiding_map(nsl_ctx* c, const void* density, const uint8_t* mask,
                           const nsl_camera* cam, const nsl_light* light, float step,
                           const nsl_march_opts* opts, float* guide, void* stream) {
  (void)light;  // the guide uses the surrogate lights of Eq. approx only
  if (!c) return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map: ctx is NULL");
  MarchPlume p;
  nsl_status st = march_setup(c, cam, step, opts, "nsl_guiding_map", &p);
  if (st != NSL_OK) return st;
  if (!guide) return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map: guide is NULL");
  if (!aligned16(guide))
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map: buffers must be 16-byte aligned");
  if (density) {
    st = nsl_stage_grid(c, density, mask, stream);
    if (st != NSL_OK) return st;
  } else if (!c->staged_valid) {
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map: density is NULL and no grid is staged");
  }
  p.guide = guide;
  if (p.shadow_volume) {
    // one shadow march per voxel centre into the two transmittance volumes,
    // staged like the density for the view march's trilinear reads
    const size_t nv = grid_voxels(c->grid), raw = (nv * sizeof(float) + 255) / 256 * 256;
    const size_t stg = (staged_floats(c->grid.nx, c->grid.ny, c->grid.nz) * sizeof(float) + 255) / 256 * 256;
    if (2 * raw + 2 * stg > c->tvol_bytes) {
      NSL_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
      cudaFree(c->tvol);
      c->tvol = nullptr;
      c->tvol_bytes = 0;
      NSL_CUDA_TRY(cudaMalloc(&c->tvol, 2 * raw + 2 * stg));
      c->tvol_bytes = 2 * raw + 2 * stg;
    }
    char* tb = reinterpret_cast<char*>(c->tvol);
    float* rawT = reinterpret_cast<float*>(tb);
    float* rawB = reinterpret_cast<float*>(tb + raw);
    float* stT = reinterpret_cast<float*>(tb + 2 * raw);
    float* stB = reinterpret_cast<float*>(tb + 2 * raw + stg);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_transmittance_volume(p, rawT, rawB, s);
    if (e == cudaSuccess)
      e = launch_stage_volume(rawT, NSL_F32, nullptr, c->grid.nx, c->grid.ny, c->grid.nz, 1.f, stT, s);
    if (e == cudaSuccess)
      e = launch_stage_volume(rawB, NSL_F32, nullptr, c->grid.nx, c->grid.ny, c->grid.nz, 1.f, stB, s);
    if (e != cudaSuccess) return cuda_fail(e, "nsl_guiding_map: transmittance volumes");
    p.volT = stT;
    p.volB = stB;
  }
  // segmented-march scratch, grown on demand: per pixel the step count, per
  // (segment, pixel) the optical depth, its compensation and the partial radiance
  const int maxseg = march_max_segments(c->grid.nx, c->grid.ny, c->grid.nz, step, kMarchSegLen);
  const size_t P = (size_t)cam->width * cam->height;
  const size_t need = P * sizeof(int) + 3 * (size_t)maxseg * P * sizeof(float) + 1024;
  if (need > c->seg_bytes) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NSL_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(c->seg_scratch);
    c->seg_scratch = nullptr;
    c->seg_bytes = 0;
    NSL_CUDA_TRY(cudaMalloc(&c->seg_scratch, need));
    c->seg_bytes = need;
  }
  char* base = static_cast<char*>(c->seg_scratch);
  p.seg_len = kMarchSegLen;
  p.seg_nef = reinterpret_cast<int*>(base);
  base += (P * sizeof(int) + 255) / 256 * 256;
  p.seg_tau = reinterpret_cast<float*>(base);
  p.seg_comp = p.seg_tau + (size_t)maxseg * P;
  p.seg_L = p.seg_comp + (size_t)maxseg * P;
  cudaError_t e = launch_march_segmented(p, maxseg, c->tile_counter, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "nsl_guiding_map: march");
  return NSL_OK;
}

nsl_status nsl_reference_lightmaps(nsl_ctx* c, const void* density, const uint8_t* mask, const nsl_camera* cam,
                                   float hf, float phase_g, float* out, void* stream) {
  static const char* fn = "nsl_reference_lightmaps";
  if (!c) return fail(NSL_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
  if (!(hf >= 1.f / 64.f) || !std::isfinite(hf))
    return fail(NSL_ERR_INVALID_ARG, "%s: hf must be a finite step of at least 1/64 voxel", fn);
  if (!(phase_g > -1.f && phase_g < 1.f)) return fail(NSL_ERR_INVALID_ARG, "%s: phase_g must be in (-1, 1)", fn);
  MarchPlume p;
  nsl_status st = march_setup(c, cam, 1.f, nullptr, fn, &p);
  if (st != NSL_OK) return st;
  if (!out || !aligned16(out)) return fail(NSL_ERR_INVALID_ARG, "%s: out NULL or not 16-byte aligned", fn);
  if (density) {
    st = nsl_stage_grid(c, density, mask, stream);
    if (st != NSL_OK) return st;
  } else if (!c->staged_valid) {
    return fail(NSL_ERR_INVALID_ARG, "%s: density is NULL and no grid is staged", fn);
  }
  cudaError_t e = launch_reference_lightmaps(p, (double)hf, phase_g, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return NSL_OK;
}

nsl_status nsl_guide_sample_count(nsl_ctx* c, const nsl_camera* cam, float step,
                                  const nsl_march_opts* opts, unsigned long long* out,
                                  void* stream) {
  if (!c || !out) return fail(NSL_ERR_INVALID_ARG, "nsl_guide_sample_count: NULL argument");
  MarchPlume p;
  nsl_status st = march_setup(c, cam, step, opts, "nsl_guide_sample_count", &p);
  if (st != NSL_OK) return st;
  if (!c->staged_valid) return fail(NSL_ERR_INVALID_ARG, "nsl_guide_sample_count: no grid staged");
  p.shadow_volume = 0;   // counts the density evaluations of Alg. 1's own shadow marches
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!c->counter) NSL_CUDA_TRY(cudaMalloc(&c->counter, sizeof(unsigned long long)));
  NSL_CUDA_TRY(cudaMemsetAsync(c->counter, 0, sizeof(unsigned long long), s));
  p.counter = c->counter;
  NSL_CUDA_TRY(launch_march(p, c->tile_counter, s, true));
  NSL_CUDA_TRY(cudaMemcpyAsync(out, c->counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  NSL_CUDA_TRY(cudaStreamSynchronize(s));
  return NSL_OK;
}

static nsl_status predict(nsl_ctx* c, const float* guide, int width, int height, int precision,
                          float* lm, uint8_t* trace, void* stream, const char* fn) {
  if (!c) return fail(NSL_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
  if (!guide || !lm) return fail(NSL_ERR_INVALID_ARG, "%s: NULL buffer", fn);
  if (!aligned16(guide) || !aligned16(lm))
    return fail(NSL_ERR_INVALID_ARG, "%s: buffers must be 16-byte aligned", fn);
  if (width < 8 || height < 8 || width % 8 || height % 8 || width > c->max_w || height > c->max_h)
    return fail(NSL_ERR_INVALID_ARG, "%s: bad size %dx%d", fn, width, height);
  NetImage img{guide, lm, height, width,
               (float)(1.0 / std::sqrt((double)c->grid.nx * c->grid.nx +
                                       (double)c->grid.ny * c->grid.ny +
                                       (double)c->grid.nz * c->grid.nz))};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // a bounded wait that gave up in an earlier tensor-core launch is reported here
  if (c->err_host && *reinterpret_cast<volatile unsigned int*>(c->err_host) != 0) {
    unsigned int code = *c->err_host;
    *c->err_host = 0;
    return fail(NSL_ERR_TIMEOUT, "%s: an earlier tensor-core launch timed out "
                "waiting on an mbarrier (code 0x%x)", fn, code);
  }
  switch (precision) {
    case NSL_PREC_F32:
      if (trace) return fail(NSL_ERR_UNSUPPORTED, "%s: no trace of the FP32 network", fn);
      e = net_f32_forward(c->wf32, img, c->ws, c->ws_bytes, s);
      break;
    case NSL_PREC_BF16:
    case NSL_PREC_F16:
    case NSL_PREC_FP8:
    case NSL_PREC_BF16X3: {
      if (c->layout.c0 != kC0)
        return fail(NSL_ERR_UNSUPPORTED, "%s: the tensor-core networks are built for C0=16 (this blob: C0=%d)",
                    fn, c->layout.c0);
      const int elem = tc_elem_of(precision);
      const size_t need = net_tc_workspace_bytes(c->max_w, c->max_h, elem);
      if (need > c->ws_bytes) {
        // the split-BF16 network keeps binary32 activations: grow the workspace
        // once (the old one stays if the allocation fails)
        NSL_CUDA_TRY(cudaStreamSynchronize(s));
        void* bigger = nullptr;
        NSL_CUDA_TRY(cudaMalloc(&bigger, need));
        cudaFree(c->ws);
        c->ws = bigger;
        c->ws_bytes = need;
      }
      if (!c->wtc[elem]) {
        c->wtc[elem] = net_tc_create(c->params.data(), c->layout, elem, &e);
        if (!c->wtc[elem]) return cuda_fail(e, "nsl_predict_lightmaps: tensor-core weights");
      }
      e = net_tc_forward(c->wtc[elem], c->wf32, img, c->ws, c->ws_bytes, c->err_dev, s, trace);
      break;
    }
    default:
      return fail(NSL_ERR_UNSUPPORTED, "%s: precision %d not built", fn, precision);
  }
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return NSL_OK;
}

nsl_status nsl_predict_lightmaps(nsl_ctx* c, const float* guide, int width, int height,
                                 int precision, float* lm, void* stream) {
  return predict(c, guide, width, height, precision, lm, nullptr, stream, "nsl_predict_lightmaps");
}

size_t nsl_lightmap_trace_bytes(int width, int height) {
  return width > 0 && height > 0 ? net_tc_trace_bytes(width, height) : 0;
}

nsl_status nsl_predict_lightmaps_trace(nsl_ctx* c, const float* guide, int width, int height,
                                       int precision, float* lm, void* trace, size_t trace_bytes,
                                       void* stream) {
  static const char* fn = "nsl_predict_lightmaps_trace";
  if (!trace || !aligned16(trace)) return fail(NSL_ERR_INVALID_ARG, "%s: trace buffer NULL or unaligned", fn);
  if (width > 0 && height > 0 && trace_bytes < net_tc_trace_bytes(width, height))
    return fail(NSL_ERR_INVALID_ARG, "%s: trace buffer of %zu bytes, needs %zu", fn, trace_bytes,
                net_tc_trace_bytes(width, height));
  return predict(c, guide, width, height, precision, lm, static_cast<uint8_t*>(trace), stream, fn);
}

nsl_status nsl_selftest_wait_timeout(nsl_ctx* c, void* stream) {
  if (!c) return fail(NSL_ERR_INVALID_ARG, "nsl_selftest_wait_timeout: ctx is NULL");
  if (!c->err_dev) return fail(NSL_ERR_UNSUPPORTED, "nsl_selftest_wait_timeout: no error word");
  cudaError_t e = launch_wait_timeout_probe(c->err_dev, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "nsl_selftest_wait_timeout");
  return NSL_OK;
}

nsl_status nsl_obstacle_shadow_map(const uint8_t* mask_dev, int nx, int ny, int nz, const float light_dir[3],
                                   int resolution, float* shadow_map_dev, void* stream) {
  const char* fn = "nsl_obstacle_shadow_map";
  if (!mask_dev || !light_dir || !shadow_map_dev) return fail(NSL_ERR_INVALID_ARG, "%s: NULL argument", fn);
  if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096)
    return fail(NSL_ERR_INVALID_ARG, "%s: grid dims out of range", fn);
  if (resolution < 1 || resolution > 8192)
    return fail(NSL_ERR_INVALID_ARG, "%s: resolution must be in [1, 8192]", fn);
  if (!aligned16(shadow_map_dev)) return fail(NSL_ERR_INVALID_ARG, "%s: map must be 16-byte aligned", fn);
  LightFrame L;
  if (!light_frame_from(light_dir, nx, ny, nz, &L))
    return fail(NSL_ERR_INVALID_ARG, "%s: zero or non-finite light direction", fn);
  cudaError_t e = launch_shadow_map(mask_dev, nx, ny, nz, L, resolution, shadow_map_dev,
                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return NSL_OK;
}

nsl_status nsl_shade_shadowed(nsl_ctx* c, const float* lm, const float* guide, int width, int height,
                              const nsl_camera* cam, const nsl_light* lights, int n_lights,
                              const float* const* shadow_maps_dev, int resolution, float bias, float* rgba,
                              void* stream) {
  const char* fn = "nsl_shade_shadowed";
  if (!c) return fail(NSL_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
  if (!lm || !guide || !rgba) return fail(NSL_ERR_INVALID_ARG, "%s: NULL buffer", fn);
  if (!aligned16(lm) || !aligned16(guide) || !aligned16(rgba))
    return fail(NSL_ERR_INVALID_ARG, "%s: buffers must be 16-byte aligned", fn);
  if (!cam) return fail(NSL_ERR_INVALID_ARG, "%s: camera is NULL", fn);
  if (width < 8 || height < 8 || width % 8 || height % 8 || width > 8192 || height > 8192)
    return fail(NSL_ERR_INVALID_ARG, "%s: bad size %dx%d", fn, width, height);
  if (n_lights < 0 || n_lights > kMaxShadowLights || (n_lights > 0 && !lights))
    return fail(NSL_ERR_INVALID_ARG, "%s: n_lights must be in [0, %d]", fn, kMaxShadowLights);
  if (resolution < 1 || resolution > 8192)
    return fail(NSL_ERR_INVALID_ARG, "%s: resolution must be in [1, 8192]", fn);
  if (!std::isfinite(bias)) return fail(NSL_ERR_INVALID_ARG, "%s: bias must be finite", fn);
  nsl_camera cc = *cam;
  cc.width = width;
  cc.height = height;
  nsl_status st = check_camera_basic(&cc, fn);
  if (st != NSL_OK) return st;
  ShadowShadeArgs a{};
  a.lm = lm;
  a.guide = guide;
  a.rgba = rgba;
  a.W = width;
  a.H = height;
  a.R = resolution;
  a.n_lights = n_lights;
  a.bias = bias;
  a.fx = (float)c->grid.nx;
  a.fy = (float)c->grid.ny;
  a.fz = (float)c->grid.nz;
  cam_frame_from(cc, &a.cam);
  for (int l = 0; l < n_lights; ++l) {
    if ((st = shade_matrix(cc, lights + l, 1, a.light[l].M, fn)) != NSL_OK) return st;
    if (!light_frame_from(lights[l].dir, c->grid.nx, c->grid.ny, c->grid.nz, &a.light[l].F))
      return fail(NSL_ERR_INVALID_ARG, "%s: light %d has a zero direction", fn, l);
    a.light[l].map = shadow_maps_dev ? shadow_maps_dev[l] : nullptr;
  }
  cudaError_t e = launch_shade_shadowed(a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return NSL_OK;
}

nsl_status nsl_shade(nsl_ctx* c, const float* lm, int width, int height, const nsl_camera* cam,
                     const nsl_light* lights, int n_lights, float* rgba, void* stream) {
  if (!c) return fail(NSL_ERR_INVALID_ARG, "nsl_shade: ctx is NULL");
  if (!lm || !rgba) return fail(NSL_ERR_INVALID_ARG, "nsl_shade: NULL buffer");
  if (!aligned16(lm) || !aligned16(rgba))
    return fail(NSL_ERR_INVALID_ARG, "nsl_shade: buffers must be 16-byte aligned");
  if (!cam) return fail(NSL_ERR_INVALID_ARG, "nsl_shade: camera is NULL");
  if (width < 8 || height < 8 || width % 8 || height % 8)
    return fail(NSL_ERR_INVALID_ARG, "nsl_shade: bad size %dx%d", width, height);
  if (n_lights < 0 || n_lights > 64 || (n_lights > 0 && !lights))
    return fail(NSL_ERR_INVALID_ARG, "nsl_shade: n_lights must be in [0, 64]");
  nsl_camera cc = *cam;
  cc.width = width;
  cc.height = height;
  ShadeArgs a{};
  a.lm = lm;
  a.rgba = rgba;
  a.W = width;
  a.H = height;
  nsl_status st = shade_matrix(cc, lights, n_lights, a.M, "nsl_shade");
  if (st != NSL_OK) return st;
  cudaError_t e = launch_shade(a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "nsl_shade");
  return NSL_OK;
}

static cudaError_t ensure(void** p, size_t bytes) {
  if (*p) return cudaSuccess;
  return cudaMalloc(p, bytes);
}

}  // extern "C"

// The host-buffer frame: uploads, the three stages, downloads, all on
// `stream`; `wait` synchronises the stream before returning.
static nsl_status render_frame_host(nsl_ctx* c, const void* density_host, const uint8_t* mask_host,
                                    const nsl_camera* cam, const nsl_light* lights, int n_lights,
                                    float step, const nsl_march_opts* opts, int precision,
                                    float* guide_host, float* lm_host, float* rgba_host,
                                    void* stream, bool wait) {
  if (!c) return fail(NSL_ERR_INVALID_ARG, "nsl_render_frame_host: ctx is NULL");
  if (!density_host) return fail(NSL_ERR_INVALID_ARG, "nsl_render_frame_host: NULL density");
  nsl_status st = check_camera(c, cam, "nsl_render_frame_host");
  if (st != NSL_OK) return st;
  const size_t nvox = grid_voxels(c->grid);
  const size_t dbytes = nvox * (c->grid.dtype == NSL_F16 ? 2 : 4);
  const size_t P = (size_t)c->max_w * c->max_h;
  NSL_CUDA_TRY(ensure(&c->h_density, dbytes));
  NSL_CUDA_TRY(ensure(reinterpret_cast<void**>(&c->h_mask), nvox));
  NSL_CUDA_TRY(ensure(reinterpret_cast<void**>(&c->h_guide), 3 * P * sizeof(float)));
  NSL_CUDA_TRY(ensure(reinterpret_cast<void**>(&c->h_lm), 8 * P * sizeof(float)));
  NSL_CUDA_TRY(ensure(reinterpret_cast<void**>(&c->h_rgba), 4 * P * sizeof(float)));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int W = cam->width, H = cam->height;
  const size_t px = (size_t)W * H;
  // The copies run on the context's copy stream `a`, overlapped with the
  // kernels on `s`: the density and mask go up in slabs of z slices, each
  // slab's cell planes staged on `s` as soon as it has arrived; the guide
  // comes back while the network runs and the lightmaps while shading runs.
  // `s` finally waits for `a`, so the frame is complete when `s` is.
  if (!c->aux) {
    NSL_CUDA_TRY(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
    for (cudaEvent_t& e : c->ev) NSL_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  cudaStream_t a = c->aux;
  cudaEvent_t* ev = c->ev;
  // the upload buffers are free once the work queued on s before this frame is done
  NSL_CUDA_TRY(cudaEventRecord(ev[0], s));
  NSL_CUDA_TRY(cudaStreamWaitEvent(a, ev[0], 0));
  const int nz = c->grid.nz, nslab = nz < kUploadSlabs ? nz : kUploadSlabs;
  const size_t slice = (size_t)c->grid.nx * c->grid.ny, esz = c->grid.dtype == NSL_F16 ? 2 : 4;
  const uint8_t* mdev = mask_host ? c->h_mask : nullptr;
  for (int k = 0; k < nslab; ++k) {
    const int z0 = nz * k / nslab, z1 = nz * (k + 1) / nslab;
    const size_t off = (size_t)z0 * slice, cnt = (size_t)(z1 - z0) * slice;
    NSL_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(c->h_density) + off * esz,
                                 static_cast<const char*>(density_host) + off * esz, cnt * esz,
                                 cudaMemcpyHostToDevice, a));
    if (mask_host)
      NSL_CUDA_TRY(cudaMemcpyAsync(c->h_mask + off, mask_host + off, cnt, cudaMemcpyHostToDevice, a));
    NSL_CUDA_TRY(cudaEventRecord(ev[1 + k], a));
    NSL_CUDA_TRY(cudaStreamWaitEvent(s, ev[1 + k], 0));
    // a quad cell plane cz holds slice cz - 1 (clamped): planes z0 + 1 .. z1,
    // plane 0 with the first slab, plane nz + 1 with the last; an octo plane
    // cz holds slices cz - 1 and cz: planes z0 .. z1 - 1, plane nz with the last
    const int c0 = k == 0 ? 0 : (c->octo ? z0 : z0 + 1);
    const int c1 = k == nslab - 1 ? -1 : (c->octo ? z1 : z1 + 1);
    const cudaError_t e = stage_planes(c, c->h_density, mdev, c0, c1, s);
    if (e != cudaSuccess) return cuda_fail(e, "nsl_render_frame_host: staging");
  }
  c->staged_valid = true;
  cudaEvent_t ev_g = ev[kUploadSlabs + 1], ev_l = ev[kUploadSlabs + 2], ev_a = ev[kUploadSlabs + 3];
  st = nsl_guiding_map(c, nullptr, nullptr, cam, nullptr, step, opts, c->h_guide, stream);
  if (st != NSL_OK) return st;
  if (guide_host) {
    NSL_CUDA_TRY(cudaEventRecord(ev_g, s));
    NSL_CUDA_TRY(cudaStreamWaitEvent(a, ev_g, 0));
    NSL_CUDA_TRY(cudaMemcpyAsync(guide_host, c->h_guide, 3 * px * sizeof(float), cudaMemcpyDeviceToHost, a));
  }
  st = nsl_predict_lightmaps(c, c->h_guide, W, H, precision, c->h_lm, stream);
  if (st != NSL_OK) return st;
  if (lm_host) {
    NSL_CUDA_TRY(cudaEventRecord(ev_l, s));
    NSL_CUDA_TRY(cudaStreamWaitEvent(a, ev_l, 0));
    NSL_CUDA_TRY(cudaMemcpyAsync(lm_host, c->h_lm, 8 * px * sizeof(float), cudaMemcpyDeviceToHost, a));
  }
  st = nsl_shade(c, c->h_lm, W, H, cam, lights, n_lights, c->h_rgba, stream);
  if (st != NSL_OK) return st;
  if (rgba_host)
    NSL_CUDA_TRY(cudaMemcpyAsync(rgba_host, c->h_rgba, 4 * px * sizeof(float), cudaMemcpyDeviceToHost, s));
  NSL_CUDA_TRY(cudaEventRecord(ev_a, a));
  NSL_CUDA_TRY(cudaStreamWaitEvent(s, ev_a, 0));
  if (wait) NSL_CUDA_TRY(cudaStreamSynchronize(s));
  return NSL_OK;
}

extern "C" {

nsl_status nsl_render_frame_host(nsl_ctx* c, const void* density_host, const uint8_t* mask_host,
                                 const nsl_camera* cam, const nsl_light* lights, int n_lights,
                                 float step, const nsl_march_opts* opts, int precision,
                                 float* guide_host, float* lm_host, float* rgba_host,
                                 void* stream) {
  return render_frame_host(c, density_host, mask_host, cam, lights, n_lights, step, opts, precision,
                           guide_host, lm_host, rgba_host, stream, true);
}

nsl_status nsl_render_frame_host_async(nsl_ctx* c, const void* density_host, const uint8_t* mask_host,
                                       const nsl_camera* cam, const nsl_light* lights, int n_lights,
                                       float step, const nsl_march_opts* opts, int precision,
                                       float* guide_host, float* lm_host, float* rgba_host,
                                       void* stream) {
  return render_frame_host(c, density_host, mask_host, cam, lights, n_lights, step, opts, precision,
                           guide_host, lm_host, rgba_host, stream, false);
}

}  // extern "C"
