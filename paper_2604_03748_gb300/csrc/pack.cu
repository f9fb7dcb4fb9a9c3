// Packed two-texture export of the eight lightmap planes: the six-way layout
// of Sec. 3 / Fig. 2.  Texture 1 = (right +X, top +Y, back +Z, transparency
// T), texture 2 = (left -X, bottom -Y, front -Z, emissive E), each an
// interleaved [H][W][4] image.  One streaming pass: eight coalesced plane reads
// and two coalesced texel writes per pixel, HBM-bound.
#include "nsl_internal.cuh"

namespace nsl {
namespace {

// UNORM8 code of v: clamp to [0, 1] (NaN to 0), v * 255 in float32, nearest
// integer with ties to even.
__device__ __forceinline__ uint32_t unorm8(float v) { return __float2uint_rn(__fmul_rn(__saturatef(v), 255.f)); }

template <int FMT>
__device__ __forceinline__ void put(void* tex, size_t p, float r, float g, float b, float a) {
  if constexpr (FMT == NSL_TEX_RGBA8) {
    reinterpret_cast<uint32_t*>(tex)[p] = unorm8(r) | (unorm8(g) << 8) | (unorm8(b) << 16) | (unorm8(a) << 24);
  } else if constexpr (FMT == NSL_TEX_RGBA16F) {
    __half2 lo = __floats2half2_rn(r, g), hi = __floats2half2_rn(b, a);
    uint2 w;
    w.x = *reinterpret_cast<uint32_t*>(&lo);
    w.y = *reinterpret_cast<uint32_t*>(&hi);
    reinterpret_cast<uint2*>(tex)[p] = w;
  } else {
    reinterpret_cast<float4*>(tex)[p] = make_float4(r, g, b, a);
  }
}

template <int FMT>
__global__ void __launch_bounds__(256) pack_kernel(const float* __restrict__ lm, size_t P, void* tex1,
                                                    void* tex2) {
  pdl_wait();      // the lightmaps come from the network
  pdl_trigger();
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldcs(lm + q * P + p);
    put<FMT>(tex1, p, v[0], v[2], v[4], v[6]);
    put<FMT>(tex2, p, v[1], v[3], v[5], v[7]);
  }
}

}  // namespace
}  // namespace nsl

using namespace nsl;

extern "C" nsl_status nsl_pack_lightmaps(const float* lightmaps_dev, int width, int height, int format,
                                         void* tex1_dev, void* tex2_dev, void* stream) {
  const char* fn = "nsl_pack_lightmaps";
  if (!lightmaps_dev || !tex1_dev || !tex2_dev) return fail(NSL_ERR_INVALID_ARG, "%s: NULL buffer", fn);
  if (width < 8 || height < 8 || width % 8 || height % 8 || width > 8192 || height > 8192)
    return fail(NSL_ERR_INVALID_ARG, "%s: width/height must be multiples of 8 in [8, 8192]", fn);
  if (format < NSL_TEX_RGBA8 || format > NSL_TEX_RGBA32F)
    return fail(NSL_ERR_INVALID_ARG, "%s: bad format %d", fn, format);
  auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  if (!a16(lightmaps_dev) || !a16(tex1_dev) || !a16(tex2_dev))
    return fail(NSL_ERR_INVALID_ARG, "%s: buffers must be 16-byte aligned", fn);
  const size_t P = (size_t)width * height;
  int blocks = (int)((P + 255) / 256);
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (format == NSL_TEX_RGBA8)
    e = launch_pdl(pack_kernel<NSL_TEX_RGBA8>, dim3(blocks), dim3(256), 0, s, lightmaps_dev, P, tex1_dev, tex2_dev);
  else if (format == NSL_TEX_RGBA16F)
    e = launch_pdl(pack_kernel<NSL_TEX_RGBA16F>, dim3(blocks), dim3(256), 0, s, lightmaps_dev, P, tex1_dev,
                   tex2_dev);
  else
    e = launch_pdl(pack_kernel<NSL_TEX_RGBA32F>, dim3(blocks), dim3(256), 0, s, lightmaps_dev, P, tex1_dev,
                   tex2_dev);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return NSL_OK;
}
