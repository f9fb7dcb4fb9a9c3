// nsl_measure_peaks: the roofline denominators of the guide march, measured
// on the device the caller has current (the paper has no counterpart).
//
//  * FP32 FMA rate: every thread runs eight independent fmaf chains; 2 flop
//    per FMA.
//  * L1 data path: every warp reads 512 contiguous, aligned bytes (16 bytes
//    per lane) from a 16 KB region its CTA keeps in L1; bytes delivered to the
//    registers per second.  This is the best case of the path the march's
//    trilinear gathers use (four 128-byte wavefronts per warp-wide load).
//  * L2 random gathers: every lane reads 16 bytes at a hashed position of a
//    64 MiB buffer that stays in L2 (a warp's lanes touch unrelated lines).
// Each kernel is timed with CUDA events on the caller's stream after a
// warm-up launch; the buffers are allocated for the call and freed after it.
#include <cstdint>

#include "nsl_internal.cuh"

namespace nsl {
namespace {

constexpr int kThreads = 256;
constexpr int kL1Floats4 = 1024;             // 16 KB per CTA
constexpr size_t kL2Floats4 = size_t(1) << 22;  // 64 MiB

__global__ void __launch_bounds__(kThreads) fma_peak_kernel(float a, float b, int iters, float* sink) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = a + 1e-3f * (float)(threadIdx.x + k);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 32; ++r) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], b, a);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 1234.5678f) sink[blockIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) l1_peak_kernel(const float4* __restrict__ buf, int iters,
                                                           float* sink) {
  const float4* base = buf + (size_t)(blockIdx.x & 63) * kL1Floats4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc = 0.f;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int seg = (i * 7 + r * 3 + warp) & 31;     // one of 32 segments of 512 bytes
      const float4 v = __ldg(base + seg * 32 + lane);
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  if (acc == 1234.5678f) sink[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) l2_gather_kernel(const float4* __restrict__ buf, int iters,
                                                             float* sink) {
  uint32_t h = (blockIdx.x * kThreads + threadIdx.x) * 2654435761u + 12345u;
  float acc = 0.f;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      h = h * 1664525u + 1013904223u;
      const float4 v = __ldg(buf + ((h >> 6) & (uint32_t)(kL2Floats4 - 1)));
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  if (acc == 1234.5678f) sink[blockIdx.x] = acc;
}

__global__ void fill_kernel(float4* buf, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    buf[i] = make_float4(1e-3f, 2e-3f, 3e-3f, 4e-3f);
}

// milliseconds of `launch` on s, after one warm-up launch
template <typename F>
cudaError_t time_ms(F launch, cudaStream_t s, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e;
}

}  // namespace
}  // namespace nsl

using namespace nsl;

extern "C" nsl_status nsl_measure_peaks(nsl_peaks* out, void* stream) {
  if (!out) return fail(NSL_ERR_INVALID_ARG, "nsl_measure_peaks: out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int sms = num_sms();
  float4* l1 = nullptr;
  float4* l2 = nullptr;
  float* sink = nullptr;
  cudaError_t e = cudaMalloc(&l1, 64 * kL1Floats4 * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&l2, kL2Floats4 * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&sink, 64 * 1024 * sizeof(float));
  if (e == cudaSuccess) {
    fill_kernel<<<sms * 4, 256, 0, s>>>(l1, 64 * kL1Floats4);
    fill_kernel<<<sms * 4, 256, 0, s>>>(l2, kL2Floats4);
    e = cudaGetLastError();
  }
  const int blocks = sms * 8;   // 2048 threads per SM
  float ms_fma = 0.f, ms_l1 = 0.f, ms_l2 = 0.f;
  const int it_fma = 4096, it_l1 = 2048, it_l2 = 256;
  if (e == cudaSuccess)
    e = time_ms([&] {
      fma_peak_kernel<<<blocks, kThreads, 0, s>>>(1e-6f, 0.9999f, it_fma, sink);
      return cudaGetLastError();
    }, s, &ms_fma);
  if (e == cudaSuccess)
    e = time_ms([&] {
      l1_peak_kernel<<<blocks, kThreads, 0, s>>>(l1, it_l1, sink);
      return cudaGetLastError();
    }, s, &ms_l1);
  if (e == cudaSuccess)
    e = time_ms([&] {
      l2_gather_kernel<<<blocks, kThreads, 0, s>>>(l2, it_l2, sink);
      return cudaGetLastError();
    }, s, &ms_l2);
  cudaFree(l1);
  cudaFree(l2);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_measure_peaks");
  const double threads = (double)blocks * kThreads;
  out->sms = sms;
  out->fp32_tflops = threads * it_fma * 32.0 * 8.0 * 2.0 / (ms_fma * 1e-3) / 1e12;
  out->l1_gbps = threads * it_l1 * 16.0 * 16.0 / (ms_l1 * 1e-3) / 1e9;
  out->l2_gather_gbps = threads * it_l2 * 16.0 * 16.0 / (ms_l2 * 1e-3) / 1e9;
  return NSL_OK;
}
