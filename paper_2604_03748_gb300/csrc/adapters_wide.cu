// The four NAFBlock channel adapters (Sec. 4.3, Fig. 3) in FP32 on the SIMT
// cores at base width C0 = 32 (the FP32 path's second width).  The same
// computation as the C0 = 16 adapters:
//   x1 = SG(dw3x3(pw1(LN1(F)))),  att = W_sca mean_HW(x1) + b_sca,
//   y  = F + beta * pw2(x1 * att),  z = y + gamma * ffn2(SG(ffn1(LN2(y)))),
//   the adapter's two output planes = head(z),
// with the LayerNorm affines folded into pw1 and ffn1 on the host.  At 32
// channels the weights outgrow the kernel-parameter bank, so they live in
// device memory and each CTA stages the ones it needs in shared memory.
//   pass 1  one CTA per (16x8 tile, adapter): the 18x10 halo of F normalised,
//           pw1 on every halo pixel (zero outside the image: the depthwise
//           convolution pads its input with zeros), then per inner pixel the
//           depthwise 3x3 and the simple gate; x1 and the tile's channel sums out
//   mean    the tile sums of each (adapter, channel) in a fixed order
//   pass 2  persistent CTAs per adapter: att from the means, then per pixel
//           everything after x1
#include <cmath>
#include <vector>

#include "nsl_internal.cuh"

namespace nsl {

namespace {

constexpr int C = kWideC0;                 // channels per adapter
constexpr int kTW = 16, kTH = 8;           // pass-1 tile: 128 inner pixels
constexpr int kHW = kTW + 2, kHH = kTH + 2, kHalo = kHW * kHH;   // 18 x 10 = 180
constexpr int kHS = kHalo + 1;             // odd stride of one pw1 output plane
constexpr int kNS = C + 4;                 // padded row of the normalised halo

// Device layout of one adapter's folded parameters (floats).  Pass 1 reads
// [0, kP1), pass 2 reads [kP1, kP1 + kP2).
constexpr int kW1 = 0;                     // [2C][C] pw1 diag(ln1 w)
constexpr int kB1 = kW1 + 2 * C * C;       // [2C]    pw1 b + pw1 ln1 b
constexpr int kDww = kB1 + 2 * C;          // [2C][9] depthwise taps (ky, kx)
constexpr int kDwb = kDww + 18 * C;        // [2C]
constexpr int kP1 = kDwb + 2 * C;
constexpr int kScaW = 0;                   // [C][C]  (offsets inside the pass-2 block)
constexpr int kScaB = kScaW + C * C;       // [C]
constexpr int kW2 = kScaB + C;             // [C][C]
constexpr int kB2 = kW2 + C * C;
constexpr int kBeta = kB2 + C;
constexpr int kF1 = kBeta + C;             // [2C][C] ffn1 diag(ln2 w)
constexpr int kFb1 = kF1 + 2 * C * C;      // [2C]    ffn1 b + ffn1 ln2 b
constexpr int kF2 = kFb1 + 2 * C;          // [C][C]
constexpr int kFb2 = kF2 + C * C;
constexpr int kGamma = kFb2 + C;
constexpr int kHwt = kGamma + C;           // [2][C]
constexpr int kHb = kHwt + 2 * C;          // [2], padded to 4
constexpr int kP2 = kHb + 4;
constexpr int kAd = kP1 + kP2;             // floats per adapter (a multiple of 4)
static_assert(kP1 % 4 == 0 && kP2 % 4 == 0, "float4 staging");

constexpr int kP1Smem = (kHalo * kNS + 2 * C * kHS + kP1 + 4 * C) * 4 + kHalo;
constexpr int kP2Threads = 128;
constexpr int kP2Smem = (kP2 + C) * 4;

__device__ __forceinline__ void stage(float* dst, const float* src, int n) {
  for (int e = threadIdx.x; e < n / 4; e += blockDim.x)
    reinterpret_cast<float4*>(dst)[e] = __ldg(reinterpret_cast<const float4*>(src) + e);
}

// (x - mean) / sqrt(var + 1e-6) over the C channels
__device__ __forceinline__ void normalise(const float* x, float* y) {
  float mu = 0.f;
#pragma unroll
  for (int c = 0; c < C; ++c) mu += x[c];
  mu *= (1.f / C);
  float var = 0.f;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const float d = x[c] - mu;
    var = fmaf(d, d, var);
  }
  var *= (1.f / C);
  const float inv = 1.f / sqrtf(var + 1e-6f);
#pragma unroll
  for (int c = 0; c < C; ++c) y[c] = (x[c] - mu) * inv;
}

// s + row . v over C channels, the row read as float4 from shared memory
__device__ __forceinline__ float dot_row(const float* row, const float* v, float s) {
#pragma unroll
  for (int q = 0; q < C / 4; ++q) {
    const float4 w = reinterpret_cast<const float4*>(row)[q];
    s = fmaf(w.x, v[4 * q], s);
    s = fmaf(w.y, v[4 * q + 1], s);
    s = fmaf(w.z, v[4 * q + 2], s);
    s = fmaf(w.w, v[4 * q + 3], s);
  }
  return s;
}

}  // namespace

// Pass 1: grid (tiles, 4 adapters), 128 threads = the 16 x 8 inner pixels.
__global__ void __launch_bounds__(128) adapters_wide_pass1(const float* __restrict__ F,
                                                           const float* __restrict__ prm,
                                                           float* __restrict__ x1,
                                                           float* __restrict__ partial, int H, int W) {
  extern __shared__ __align__(16) float sm[];
  float* xh = sm;                                  // [180][kNS] normalised halo
  float* t = xh + kHalo * kNS;                     // [2C][kHS]  pw1 outputs
  float* wp = t + 2 * C * kHS;                     // pass-1 parameters of this adapter
  float* red = wp + kP1;                           // [4][C] per-warp channel sums
  unsigned char* inside = reinterpret_cast<unsigned char*>(red + 4 * C);
  const int tid = threadIdx.x, a = blockIdx.y;
  const int tiles_x = (W + kTW - 1) / kTW;
  const int x0 = (blockIdx.x % tiles_x) * kTW, y0 = (blockIdx.x / tiles_x) * kTH;
  const size_t P = (size_t)H * W;
  pdl_wait();      // F comes from the last convolution
  stage(wp, prm + (size_t)a * kAd, kP1);
  for (int hp = tid; hp < kHalo; hp += blockDim.x) {
    const int y = y0 + hp / kHW - 1, x = x0 + hp % kHW - 1;
    const bool in = y >= 0 && y < H && x >= 0 && x < W;
    inside[hp] = in ? 1 : 0;
    float v[C], n[C];
    const float4* src = reinterpret_cast<const float4*>(F + ((size_t)(in ? y : 0) * W + (in ? x : 0)) * C);
#pragma unroll
    for (int q = 0; q < C / 4; ++q) {
      const float4 u = __ldg(src + q);
      v[4 * q] = in ? u.x : 0.f;
      v[4 * q + 1] = in ? u.y : 0.f;
      v[4 * q + 2] = in ? u.z : 0.f;
      v[4 * q + 3] = in ? u.w : 0.f;
    }
    normalise(v, n);
#pragma unroll
    for (int q = 0; q < C / 4; ++q)
      reinterpret_cast<float4*>(xh + hp * kNS)[q] = make_float4(n[4 * q], n[4 * q + 1], n[4 * q + 2], n[4 * q + 3]);
  }
  __syncthreads();
  // pw1: work item e = (half, halo pixel), the half choosing outputs [0, C) or [C, 2C)
  for (int e = tid; e < 2 * kHalo; e += blockDim.x) {
    const int half = e / kHalo, hp = e % kHalo;
    float n[C];
#pragma unroll
    for (int q = 0; q < C / 4; ++q) {
      const float4 u = reinterpret_cast<const float4*>(xh + hp * kNS)[q];
      n[4 * q] = u.x; n[4 * q + 1] = u.y; n[4 * q + 2] = u.z; n[4 * q + 3] = u.w;
    }
    const bool in = inside[hp] != 0;
#pragma unroll 4
    for (int oo = 0; oo < C; ++oo) {
      const int o = half * C + oo;
      const float s = dot_row(wp + kW1 + o * C, n, wp[kB1 + o]);
      t[o * kHS + hp] = in ? s : 0.f;
    }
  }
  __syncthreads();
  // depthwise 3x3 + simple gate for this thread's inner pixel
  const int tx = tid % kTW, ty = tid / kTW;
  const int px = x0 + tx, py = y0 + ty;
  const bool valid = px < W && py < H;
  float g[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float d0 = wp[kDwb + c], d1 = wp[kDwb + c + C];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int hp = (ty + ky) * kHW + tx + kx;
        d0 = fmaf(wp[kDww + c * 9 + ky * 3 + kx], t[c * kHS + hp], d0);
        d1 = fmaf(wp[kDww + (c + C) * 9 + ky * 3 + kx], t[(c + C) * kHS + hp], d1);
      }
    g[c] = valid ? d0 * d1 : 0.f;
  }
  if (valid) {
    float4* dst = reinterpret_cast<float4*>(x1 + ((size_t)a * P + (size_t)py * W + px) * C);
#pragma unroll
    for (int q = 0; q < C / 4; ++q) dst[q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
  }
  // channel sums of the tile: butterfly in each warp, then the warps in order
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float v = g[c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    g[c] = v;
  }
  if ((tid & 31) == 0) {
#pragma unroll
    for (int c = 0; c < C; ++c) red[(tid >> 5) * C + c] = g[c];
  }
  __syncthreads();
  if (tid < C)
    partial[((size_t)blockIdx.x * 4 + a) * C + tid] =
        ((red[tid] + red[C + tid]) + red[2 * C + tid]) + red[3 * C + tid];
}

// Channel means: one CTA of 256 threads per (adapter, channel); thread k sums
// tiles k, k + 256, ... in order, then a fixed binary tree.
__global__ void __launch_bounds__(256) adapters_wide_mean(const float* __restrict__ partial, int ntiles,
                                                          float inv_count, float* __restrict__ mean) {
  __shared__ float r[256];
  pdl_wait();
  const int ac = blockIdx.x;  // a * C + c
  const int a = ac / C, c = ac % C;
  float s = 0.f;
  for (int k = threadIdx.x; k < ntiles; k += 256) s += partial[((size_t)k * 4 + a) * C + c];
  r[threadIdx.x] = s;
  __syncthreads();
  for (int half = 128; half > 0; half >>= 1) {
    if (threadIdx.x < half) r[threadIdx.x] += r[threadIdx.x + half];
    __syncthreads();
  }
  if (threadIdx.x == 0) mean[ac] = r[0] * inv_count;
}

// Pass 2: grid (CTAs, 4 adapters), pixels in a grid-stride loop; every
// product of the chain reads its weight row from shared memory.
__global__ void __launch_bounds__(kP2Threads) adapters_wide_pass2(const float* __restrict__ F,
                                                                  const float* __restrict__ x1,
                                                                  const float* __restrict__ prm,
                                                                  const float* __restrict__ mean,
                                                                  float* __restrict__ out, int npix) {
  extern __shared__ __align__(16) float sm[];
  float* wp = sm;            // pass-2 parameters of this adapter
  float* att = sm + kP2;     // [C]
  const int a = blockIdx.y;
  pdl_wait();      // x1 from pass 1, the means from the reduction
  stage(wp, prm + (size_t)a * kAd + kP1, kP2);
  __syncthreads();
  if (threadIdx.x < C) {
    float m[C];
#pragma unroll
    for (int c = 0; c < C; ++c) m[c] = mean[a * C + c];
    att[threadIdx.x] = dot_row(wp + kScaW + threadIdx.x * C, m, wp[kScaB + threadIdx.x]);
  }
  __syncthreads();
  constexpr int plane_of[4][2] = {{4, 5}, {0, 1}, {2, 3}, {6, 7}};   // F&B, L&R, U&D, A&E
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    float y[C], v[C];
    {
      const float4* fs = reinterpret_cast<const float4*>(F + (size_t)p * C);
      const float4* xs = reinterpret_cast<const float4*>(x1 + ((size_t)a * npix + p) * C);
      float f[C];
#pragma unroll
      for (int q = 0; q < C / 4; ++q) {
        const float4 u = __ldg(fs + q), w = __ldg(xs + q);
        f[4 * q] = u.x; f[4 * q + 1] = u.y; f[4 * q + 2] = u.z; f[4 * q + 3] = u.w;
        v[4 * q] = w.x * att[4 * q];
        v[4 * q + 1] = w.y * att[4 * q + 1];
        v[4 * q + 2] = w.z * att[4 * q + 2];
        v[4 * q + 3] = w.w * att[4 * q + 3];
      }
      // y = F + beta (pw2 (x1 att) + b2)
#pragma unroll
      for (int co = 0; co < C; ++co) y[co] = fmaf(wp[kBeta + co], dot_row(wp + kW2 + co * C, v, wp[kB2 + co]), f[co]);
    }
    // the gate of ffn1 on LN2(y) (its affine folded into ffn1)
    {
      float n[C];
      normalise(y, n);
#pragma unroll
      for (int co = 0; co < C; ++co)
        v[co] = dot_row(wp + kF1 + co * C, n, wp[kFb1 + co]) * dot_row(wp + kF1 + (co + C) * C, n, wp[kFb1 + co + C]);
    }
    // z = y + gamma (ffn2 g + b2'), then the head
    float h0 = wp[kHb], h1 = wp[kHb + 1];
#pragma unroll
    for (int co = 0; co < C; ++co) {
      const float z = fmaf(wp[kGamma + co], dot_row(wp + kF2 + co * C, v, wp[kFb2 + co]), y[co]);
      h0 = fmaf(wp[kHwt + co], z, h0);
      h1 = fmaf(wp[kHwt + C + co], z, h1);
    }
    out[(size_t)plane_of[a][0] * npix + p] = h0;
    out[(size_t)plane_of[a][1] * npix + p] = h1;
  }
}

struct AdapterWideWeights {
  float* prm = nullptr;   // 4 x kAd floats
};

// Fold and lay out the blob's four adapters (blob order per adapter: LN1 w, b;
// pw1 w [2C][C], b; dw w [2C][3][3], b; SCA w [C][C], b; pw2 w [C][C], b; beta;
// LN2 w, b; ffn1 w [2C][C], b; ffn2 w [C][C], b; gamma; head w [2][C], b).
AdapterWideWeights* adapters_wide_create(const float* ap4, cudaError_t* err) {
  const int ln1w = 0, ln1b = C, pw1w = 2 * C, pw1b = pw1w + 2 * C * C, dww = pw1b + 2 * C,
            dwb = dww + 18 * C, scaw = dwb + 2 * C, scab = scaw + C * C, pw2w = scab + C,
            pw2b = pw2w + C * C, beta = pw2b + C, ln2w = beta + C, ln2b = ln2w + C,
            f1w = ln2b + C, f1b = f1w + 2 * C * C, f2w = f1b + 2 * C, f2b = f2w + C * C,
            gamma = f2b + C, headw = gamma + C, headb = headw + 2 * C;
  static_assert(adapter_param_count(C) == 2 * C + 2 * C * C + 2 * C + 18 * C + 2 * C + C * C + C + C * C + C +
                                              C + 2 * C + 2 * C * C + 2 * C + C * C + C + C + 2 * C + 2,
                "adapter parameter count");
  std::vector<float> h((size_t)4 * kAd, 0.f);
  for (int a = 0; a < 4; ++a) {
    const float* q = ap4 + (size_t)a * adapter_param_count(C);
    float* d = h.data() + (size_t)a * kAd;
    float* d2 = d + kP1;
    for (int o = 0; o < 2 * C; ++o) {
      double b = q[pw1b + o];
      for (int c = 0; c < C; ++c) {
        d[kW1 + o * C + c] = (float)((double)q[pw1w + o * C + c] * q[ln1w + c]);
        b += (double)q[pw1w + o * C + c] * q[ln1b + c];
      }
      d[kB1 + o] = (float)b;
      for (int k = 0; k < 9; ++k) d[kDww + o * 9 + k] = q[dww + o * 9 + k];
      d[kDwb + o] = q[dwb + o];
      double b1 = q[f1b + o];
      for (int c = 0; c < C; ++c) {
        d2[kF1 + o * C + c] = (float)((double)q[f1w + o * C + c] * q[ln2w + c]);
        b1 += (double)q[f1w + o * C + c] * q[ln2b + c];
      }
      d2[kFb1 + o] = (float)b1;
    }
    for (int co = 0; co < C; ++co) {
      for (int ci = 0; ci < C; ++ci) {
        d2[kScaW + co * C + ci] = q[scaw + co * C + ci];
        d2[kW2 + co * C + ci] = q[pw2w + co * C + ci];
        d2[kF2 + co * C + ci] = q[f2w + co * C + ci];
      }
      d2[kScaB + co] = q[scab + co];
      d2[kB2 + co] = q[pw2b + co];
      d2[kBeta + co] = q[beta + co];
      d2[kFb2 + co] = q[f2b + co];
      d2[kGamma + co] = q[gamma + co];
      d2[kHwt + co] = q[headw + co];
      d2[kHwt + C + co] = q[headw + C + co];
    }
    d2[kHb] = q[headb];
    d2[kHb + 1] = q[headb + 1];
  }
  AdapterWideWeights* w = new AdapterWideWeights();
  *err = cudaMalloc(&w->prm, h.size() * sizeof(float));
  if (*err == cudaSuccess) *err = cudaMemcpy(w->prm, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (*err != cudaSuccess) {
    adapters_wide_destroy(w);
    return nullptr;
  }
  return w;
}

void adapters_wide_destroy(AdapterWideWeights* w) {
  if (!w) return;
  cudaFree(w->prm);
  delete w;
}

// tile sums [tiles][4][C] plus the 4C channel means
size_t adapter_wide_partial_floats(int max_w, int max_h) {
  return (size_t)((max_w + kTW - 1) / kTW) * ((max_h + kTH - 1) / kTH) * 4 * C + 4 * C;
}

cudaError_t adapters_wide_run(const AdapterWideWeights* w, const float* F, float* x1, float* partial,
                              float* mean, float* out, int H, int W, cudaStream_t s) {
  static const cudaError_t attr = [] {
    cudaError_t e = cudaFuncSetAttribute(adapters_wide_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kP1Smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(adapters_wide_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, kP2Smem);
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  const int tiles = ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH);
  const int npix = H * W;
  cudaError_t e = launch_pdl(adapters_wide_pass1, dim3(tiles, 4), dim3(128), (size_t)kP1Smem, s, F,
                             (const float*)w->prm, x1, partial, H, W);
  if (e != cudaSuccess) return e;
  e = launch_pdl(adapters_wide_mean, dim3(4 * C), dim3(256), 0, s, (const float*)partial, tiles,
                 1.f / (float)npix, mean);
  if (e != cudaSuccess) return e;
  int blocks = (npix + kP2Threads - 1) / kP2Threads;
  if (blocks > 2 * num_sms()) blocks = 2 * num_sms();
  return launch_pdl(adapters_wide_pass2, dim3(blocks, 4), dim3(kP2Threads), (size_t)kP2Smem, s, F,
                    (const float*)x1, (const float*)w->prm, (const float*)mean, out, npix);
}

}  // namespace nsl
