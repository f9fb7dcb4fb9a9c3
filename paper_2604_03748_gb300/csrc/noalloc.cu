// nsl_guiding_map_noalloc: the guide march for callers that must not allocate
// device memory.  Its scratch (the staged grid and the march tile counter)
// lives in one file-scope __device__ array instead of context-owned cudaMalloc
// buffers; the kernels are the same staging and march kernels nsl_guiding_map
// launches.
#include <cmath>
#include <mutex>

#include "nsl_internal.cuh"

namespace nsl {

// Scratch bytes: 40 MiB for the staged grid (16 bytes per cell of the padded
// x/y-quad layout, (nx+1)(ny+1)(nz+2) cells: 128^3 takes 34.6 MB) plus 256 bytes
// for the tile counter.  Every GPU that loads the library holds this array until
// exit.
constexpr size_t kNoAllocGridBytes = size_t(40) << 20;
constexpr size_t kNoAllocBytes = kNoAllocGridBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

// Device address of the scratch array on the current device (host code must not
// pass the array's host-side name to a kernel).  Looked up once per device.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

uint32_t pcg_host(uint32_t v) {
  uint32_t state = v * 747796405u + 2891336453u;
  uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}
}  // namespace

}  // namespace nsl

using namespace nsl;

extern "C" nsl_status nsl_guiding_map_noalloc(const nsl_grid_desc* grid, const void* density,
                                              const uint8_t* mask, const nsl_camera* cam,
                                              float step, const nsl_march_opts* opts,
                                              float* guide, void* stream) {
  if (!grid || !density || !cam || !guide)
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map_noalloc: NULL argument");
  if (!grid_dims_ok(grid->nx, grid->ny, grid->nz) || (grid->dtype != NSL_F32 && grid->dtype != NSL_F16) ||
      !(grid->sigma_scale >= 0.f) || !std::isfinite(grid->sigma_scale))
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map_noalloc: bad grid description");
  const size_t need = staged_floats(grid->nx, grid->ny, grid->nz) * sizeof(float);
  if (need > kNoAllocGridBytes)
    return fail(NSL_ERR_INVALID_ARG,
                "nsl_guiding_map_noalloc: a %dx%dx%d grid needs %zu bytes of scratch; the "
                "built-in scratch holds %zu (use nsl_guiding_map with a context instead)",
                grid->nx, grid->ny, grid->nz, need, kNoAllocGridBytes);
  const uintptr_t align_bits = reinterpret_cast<uintptr_t>(density) |
                               reinterpret_cast<uintptr_t>(guide) |
                               reinterpret_cast<uintptr_t>(mask);
  if (align_bits & 15u)
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map_noalloc: buffers must be 16-byte aligned");
  if (cam->kind != NSL_CAM_ORTHO && cam->kind != NSL_CAM_PERSP)
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map_noalloc: bad camera kind");
  if (cam->width < 8 || cam->height < 8 || cam->width % 8 || cam->height % 8 ||
      cam->width > 8192 || cam->height > 8192)
    return fail(NSL_ERR_INVALID_ARG,
                "nsl_guiding_map_noalloc: width/height must be multiples of 8 in [8, 8192]");
  if (cam->kind == NSL_CAM_PERSP && !(cam->fov_y_deg > 0.f && cam->fov_y_deg < 179.f))
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map_noalloc: fov_y_deg out of (0, 179)");
  if (cam->kind == NSL_CAM_ORTHO && !(cam->ortho_height > 0.f))
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map_noalloc: ortho_height must be > 0");
  {
    const double fx = (double)cam->target[0] - cam->eye[0], fy = (double)cam->target[1] - cam->eye[1],
                 fz = (double)cam->target[2] - cam->eye[2];
    const double fl = std::sqrt(fx * fx + fy * fy + fz * fz);
    const double rx = fy * cam->up[2] - fz * cam->up[1], ry = fz * cam->up[0] - fx * cam->up[2],
                 rz = fx * cam->up[1] - fy * cam->up[0];
    if (!(fl > 0.0) || !(std::sqrt(rx * rx + ry * ry + rz * rz) > 1e-9 * fl))
      return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map_noalloc: degenerate camera basis");
  }
  if (!(step > 0.f) || !std::isfinite(step))
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map_noalloc: step must be > 0");
  nsl_march_opts o;
  nsl_default_march_opts(&o);
  if (opts) o = *opts;
  if (!(o.t_min >= 0.f && o.t_min < 1.f) || !(o.phase_g > -1.f && o.phase_g < 1.f) ||
      o.light_set < NSL_LIGHTS_FTB || o.light_set > NSL_LIGHTS_FLR)
    return fail(NSL_ERR_INVALID_ARG, "nsl_guiding_map_noalloc: t_min, phase_g or light_set out of range");
  if (o.shadow_volume)
    return fail(NSL_ERR_UNSUPPORTED, "nsl_guiding_map_noalloc: shadow_volume needs a context");

  unsigned char* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_guiding_map_noalloc: scratch address");
  float* staged = reinterpret_cast<float*>(scratch);
  int* tile_counter = reinterpret_cast<int*>(scratch + kNoAllocGridBytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  e = launch_stage_volume(density, grid->dtype, mask, grid->nx, grid->ny, grid->nz,
                          grid->sigma_scale, staged, s);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_guiding_map_noalloc: staging");
  MarchPlume p{};
  p.vol = staged;
  p.nx = grid->nx; p.ny = grid->ny; p.nz = grid->nz;
  cam_frame_from(*cam, &p.cam);
  p.h = step;
  p.tau_depth = o.tau_depth;
  p.t_min = o.t_min;
  p.tau_lim = o.t_min > 0.f ? (float)(-std::log((double)o.t_min)) : INFINITY;
  p.jitter = o.jitter ? 1 : 0;
  p.key = pcg_host(o.frame + pcg_host(o.seed));
  p.g = o.phase_g;
  for (int k = 0; k < 3; ++k) p.I[k] = o.surrogate_I[k];
  p.segment_exact = o.segment_exact ? 1 : 0;
  p.light_set = o.light_set;
  p.guide = guide;
  p.tiles_x = (cam->width + kMarchTX - 1) / kMarchTX;
  p.tile_start = 0;
  // launch_march zeroes the tile counter with cudaMemsetAsync before the march
  e = launch_march(p, tile_counter, s);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_guiding_map_noalloc: march");
  return NSL_OK;
}
