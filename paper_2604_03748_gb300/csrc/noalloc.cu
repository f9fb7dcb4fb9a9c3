// nsl_guiding_map_noalloc: the guide march for callers that must not allocate
// device memory.  Its scratch (the staged grid and the march tile counter)
// lives in one file-scope __device__ array instead of context-owned cudaMalloc
// buffers.  Staging is the kernel nsl_guiding_map uses (FP32 quads for a float32
// grid, FP16 quads for a float16 one); the march is the single-pass march kernel
// (the one nsl_guide_sample_count runs), which needs no per-segment scratch.  It
// equals nsl_guiding_map's three-pass segmented march up to the grouping of the
// in-scattering sum.
#include <cmath>
#include <mutex>

#include "nsl_internal.cuh"

namespace nsl {

// Scratch bytes: 40 MiB for the staged grid ((nx+1)(ny+1)(nz+2) cells of the
// padded x/y-quad layout, 16 bytes per cell for a float32 grid and 8 for a
// float16 one: a float32 128^3 grid takes 34.6 MB) plus 256 bytes for the tile
// counter.  Every GPU that loads the library holds this array until exit.
constexpr size_t kNoAllocGridBytes = size_t(40) << 20;
constexpr size_t kNoAllocBytes = kNoAllocGridBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

// Device address of the scratch array on the current device (host code must not
// pass the array's host-side name to a kernel).  Looked up once per device, in
// that device's primary context, and kept for the life of the process.
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
}  // namespace

}  // namespace nsl

using namespace nsl;

extern "C" nsl_status nsl_guiding_map_noalloc(const nsl_grid_desc* grid, const void* density,
                                              const uint8_t* mask, const nsl_camera* cam,
                                              float step, const nsl_march_opts* opts,
                                              float* guide, void* stream) {
  static const char* fn = "nsl_guiding_map_noalloc";
  if (!grid || !density || !cam || !guide)
    return fail(NSL_ERR_INVALID_ARG, "%s: NULL argument", fn);
  if (!grid_dims_ok(grid->nx, grid->ny, grid->nz) || (grid->dtype != NSL_F32 && grid->dtype != NSL_F16) ||
      !(grid->sigma_scale >= 0.f) || !std::isfinite(grid->sigma_scale))
    return fail(NSL_ERR_INVALID_ARG, "%s: bad grid description", fn);
  const bool half = grid->dtype == NSL_F16;
  const size_t need = staged_cells(grid->nx, grid->ny, grid->nz) * (half ? 4 * sizeof(__half) : 4 * sizeof(float));
  if (need > kNoAllocGridBytes)
    return fail(NSL_ERR_INVALID_ARG,
                "%s: a %dx%dx%d %s grid needs %zu bytes of scratch; the built-in scratch holds %zu "
                "(use nsl_guiding_map with a context instead)",
                fn, grid->nx, grid->ny, grid->nz, half ? "float16" : "float32", need, kNoAllocGridBytes);
  const uintptr_t align_bits = reinterpret_cast<uintptr_t>(density) |
                               reinterpret_cast<uintptr_t>(guide) |
                               reinterpret_cast<uintptr_t>(mask);
  if (align_bits & 15u)
    return fail(NSL_ERR_INVALID_ARG, "%s: buffers must be 16-byte aligned", fn);
  nsl_status st = check_camera_basic(cam, fn);
  if (st != NSL_OK) return st;
  MarchPlume p;
  st = fill_march_plume(*grid, *cam, step, opts, fn, &p);
  if (st != NSL_OK) return st;
  if (p.shadow_volume)
    return fail(NSL_ERR_UNSUPPORTED, "%s: shadow_volume needs a context", fn);

  unsigned char* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_guiding_map_noalloc: scratch address");
  int* tile_counter = reinterpret_cast<int*>(scratch + kNoAllocGridBytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  e = half ? launch_stage_volume_half(static_cast<const __half*>(density), mask, grid->nx, grid->ny, grid->nz,
                                      reinterpret_cast<__half*>(scratch), s)
           : launch_stage_volume(density, grid->dtype, mask, grid->nx, grid->ny, grid->nz, grid->sigma_scale,
                                 reinterpret_cast<float*>(scratch), s);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_guiding_map_noalloc: staging");
  p.vol = reinterpret_cast<const float*>(scratch);
  p.staged_half = half ? 1 : 0;
  p.scl = grid->sigma_scale;
  p.guide = guide;
  // launch_march zeroes the tile counter with cudaMemsetAsync before the march
  e = launch_march(p, tile_counter, s);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_guiding_map_noalloc: march");
  return NSL_OK;
}
