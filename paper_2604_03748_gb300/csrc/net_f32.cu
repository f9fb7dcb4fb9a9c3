// Lightmap network (Sec. 4.3, Fig. 3) in FP32 on the SIMT cores: the plain
// FP32 path.  Activations are NHWC float32.  Convolutions stage a halo tile of
// the input in shared memory and accumulate 16 output channels for two
// pixels per thread; max-pooling, channel concatenation and the guide's depth
// normalisation are fused into the input staging of the convolution that
// consumes them.  The four NAFBlock adapters run as two passes around the
// global average of their simplified channel attention.
#include <vector>

#include "nsl_internal.cuh"

namespace nsl {

enum InMode { IN_PLAIN = 0, IN_POOL = 1, IN_CONCAT = 2, IN_GUIDE = 3 };

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_float(__half v) { return __half2float(v); }
template <typename T> __device__ __forceinline__ T from_float(float v);
template <> __device__ __forceinline__ float from_float<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_float<__half>(float v) {
  return __float2half_rn(v);
}
// two floats rounded to a packed pair of 16-bit values
template <typename T> __device__ __forceinline__ uint32_t pack_pair(float a, float b);
template <> __device__ __forceinline__ uint32_t pack_pair<__nv_bfloat16>(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t pack_pair<__half>(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

constexpr int kTW = 16, kTH = 16;               // output tile (pixels)
constexpr int kHW = kTW + 2, kHH = kTH + 2;     // halo tile
constexpr int kHaloPix = kHW * kHH;             // 324
constexpr int kHaloStride = kHaloPix + 1;       // odd stride: conflict-free channel-major stores

struct ConvArgs {
  const float* inA;   // IN_PLAIN/IN_CONCAT/IN_POOL: NHWC; IN_GUIDE: planar [3][H][W]
  const float* inB;   // IN_CONCAT second operand (skip), NHWC
  const float* w;     // packed [cout/16][cin][9][16]
  const float* b;     // [cout]
  void* out;          // NHWC [H][W][cout], float or bf16
  int H, W;           // output (= conv) size
  float depth_scale;
  float* amax = nullptr;  // 16-bit output only: max of the stored values (FP8 path), or null
};

// Value of input channel c at conv-input pixel (y, x), already inside the image.
template <int MODE, int CIN>
__device__ __forceinline__ float load_in(const ConvArgs& a, int y, int x, int c) {
  if constexpr (MODE == IN_PLAIN) {
    return __ldg(a.inA + ((size_t)y * a.W + x) * CIN + c);
  } else if constexpr (MODE == IN_POOL) {
    const int W2 = 2 * a.W;
    const float* p = a.inA + ((size_t)(2 * y) * W2 + 2 * x) * CIN + c;
    float m = fmaxf(__ldg(p), __ldg(p + CIN));
    m = fmaxf(m, __ldg(p + (size_t)W2 * CIN));
    return fmaxf(m, __ldg(p + (size_t)W2 * CIN + CIN));
  } else if constexpr (MODE == IN_CONCAT) {
    constexpr int CH = CIN / 2;
    if (c < CH) return __ldg(a.inA + ((size_t)y * a.W + x) * CH + c);
    return __ldg(a.inB + ((size_t)y * a.W + x) * CH + (c - CH));
  } else {  // IN_GUIDE
    float v = __ldg(a.inA + ((size_t)c * a.H + y) * a.W + x);
    return c == 2 ? v * a.depth_scale : v;
  }
}

// Four consecutive channels c .. c+3 (c a multiple of 4) at conv-input pixel
// (y, x), already inside the image (not for IN_GUIDE).
template <int MODE, int CIN>
__device__ __forceinline__ float4 load_in4(const ConvArgs& a, int y, int x, int c) {
  auto ld4 = [](const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); };
  if constexpr (MODE == IN_PLAIN) {
    return ld4(a.inA + ((size_t)y * a.W + x) * CIN + c);
  } else if constexpr (MODE == IN_POOL) {
    const int W2 = 2 * a.W;
    const float* p = a.inA + ((size_t)(2 * y) * W2 + 2 * x) * CIN + c;
    const float4 u0 = ld4(p), u1 = ld4(p + CIN), u2 = ld4(p + (size_t)W2 * CIN), u3 = ld4(p + (size_t)W2 * CIN + CIN);
    return make_float4(fmaxf(fmaxf(fmaxf(u0.x, u1.x), u2.x), u3.x), fmaxf(fmaxf(fmaxf(u0.y, u1.y), u2.y), u3.y),
                       fmaxf(fmaxf(fmaxf(u0.z, u1.z), u2.z), u3.z), fmaxf(fmaxf(fmaxf(u0.w, u1.w), u2.w), u3.w));
  } else {  // IN_CONCAT: a group of four lies within one operand
    constexpr int CH = CIN / 2;
    return c < CH ? ld4(a.inA + ((size_t)y * a.W + x) * CH + c) : ld4(a.inB + ((size_t)y * a.W + x) * CH + (c - CH));
  }
}

template <int CIN, int MODE, typename TOut>
__device__ __forceinline__ void conv3x3_f32_tile(const ConvArgs& a, int cout, int bx, int by,
                                                 int cg, int ks = 0, int nks = 1, float* partial = nullptr);

// blockIdx.z = output-channel group x input-channel split: with nks > 1 each
// block sums CIN / nks input channels and writes its raw partial sums, which
// conv_split_finish adds in split order (a fixed order: deterministic)
template <int CIN, int MODE, typename TOut>
__global__ void __launch_bounds__(128) conv3x3_f32_kernel(ConvArgs a, int cout, int nks, float* partial) {
  conv3x3_f32_tile<CIN, MODE, TOut>(a, cout, blockIdx.x, blockIdx.y, blockIdx.z / nks, blockIdx.z % nks, nks,
                                    partial);
}

// out = ReLU(bias + sum over the nks partial sums, in split order), float4 of
// channels per thread; partial [nks][H*W][cout]
__global__ void __launch_bounds__(256) conv_split_finish(const float* __restrict__ partial, int nks,
                                                         const float* __restrict__ bias, float* __restrict__ out,
                                                         int P, int cout) {
  const int n4 = P * cout / 4;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += gridDim.x * blockDim.x) {
    float4 acc = reinterpret_cast<const float4*>(partial)[e];
    for (int k = 1; k < nks; ++k) {
      const float4 v = reinterpret_cast<const float4*>(partial)[(size_t)k * n4 + e];
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    const int c = (4 * e) % cout;
    acc.x = fmaxf(acc.x + __ldg(bias + c), 0.f);
    acc.y = fmaxf(acc.y + __ldg(bias + c + 1), 0.f);
    acc.z = fmaxf(acc.z + __ldg(bias + c + 2), 0.f);
    acc.w = fmaxf(acc.w + __ldg(bias + c + 3), 0.f);
    reinterpret_cast<float4*>(out)[e] = acc;
  }
}

// grouped first layer: 16x16 tiles numbered image after image
struct ConvGroupArgs {
  ConvArgs img[kMaxGroup];
  int tile_start[kMaxGroup + 1];
  int nimg;
};

template <typename TOut>
__global__ void __launch_bounds__(128) first_conv_group_kernel(const __grid_constant__ ConvGroupArgs G) {
  pdl_wait();      // the guide comes from the march
  pdl_trigger();
  int lo = 0, hi = G.nimg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (G.tile_start[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const ConvArgs& a = G.img[lo];
  const int t = blockIdx.x - G.tile_start[lo], tx = (a.W + kTW - 1) / kTW;
  conv3x3_f32_tile<3, IN_GUIDE, TOut>(a, 16, t % tx, t / tx, 0);
}

template <int CIN, int MODE, typename TOut>
__device__ __forceinline__ void conv3x3_f32_tile(const ConvArgs& a, int cout, int bx, int by,
                                                 int cg, int ks, int nks, float* partial) {
  constexpr int CT = CIN < 16 ? CIN : 16;  // input-channel chunk
  __shared__ float halo[CT * kHaloStride];
  __shared__ __align__(16) float ws[CT * 9 * 16];
  const int tid = threadIdx.x;
  const int x0 = bx * kTW, y0 = by * kTH;
  const int tx = tid % kTW, ty = (tid / kTW) * 2;
  // accumulators of output rows ty and ty + 1, as channel pairs: the packed
  // FP32 FMA updates two output channels per instruction, each lane rounded
  // once as fmaf
  float2 p0[8], p1[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) { p0[o] = make_float2(0.f, 0.f); p1[o] = make_float2(0.f, 0.f); }

  const int cbeg = CIN / nks * ks, cend = CIN / nks * (ks + 1);
  for (int c0 = cbeg; c0 < cend; c0 += CT) {
    __syncthreads();
    // Halo and weights of this channel chunk.  Each thread issues its loads in
    // batches before their first use (one round of memory latency per batch
    // instead of per element); out-of-image elements load from a clamped
    // in-image address and are replaced by zeros.
    if constexpr (CT % 4 == 0 && MODE != IN_GUIDE) {
      constexpr int NQ = CT / 4, NE = NQ * kHaloPix, NB = MODE == IN_POOL ? 4 : 8;
      for (int e0 = tid; e0 < NE; e0 += NB * 128) {
        float4 v[NB];
        bool in[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int e = min(e0 + b * 128, NE - 1);
          const int q = e % NQ, hp = e / NQ;
          const int y = y0 + hp / kHW - 1, x = x0 + hp % kHW - 1;
          in[b] = y >= 0 && y < a.H && x >= 0 && x < a.W;
          v[b] = load_in4<MODE, CIN>(a, min(max(y, 0), a.H - 1), min(max(x, 0), a.W - 1), c0 + 4 * q);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int e = e0 + b * 128;
          if (e < NE) {
            const int q = e % NQ, hp = e / NQ;
            float* h = halo + 4 * q * kHaloStride + hp;
            h[0] = in[b] ? v[b].x : 0.f;
            h[kHaloStride] = in[b] ? v[b].y : 0.f;
            h[2 * kHaloStride] = in[b] ? v[b].z : 0.f;
            h[3 * kHaloStride] = in[b] ? v[b].w : 0.f;
          }
        }
      }
    } else {
      constexpr int NE = CT * kHaloPix, NB = 8;
      for (int e0 = tid; e0 < NE; e0 += NB * 128) {
        float v[NB];
        bool in[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int e = min(e0 + b * 128, NE - 1);
          const int c = e % CT, hp = e / CT;
          const int y = y0 + hp / kHW - 1, x = x0 + hp % kHW - 1;
          in[b] = y >= 0 && y < a.H && x >= 0 && x < a.W;
          v[b] = load_in<MODE, CIN>(a, min(max(y, 0), a.H - 1), min(max(x, 0), a.W - 1), c0 + c);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int e = e0 + b * 128;
          if (e < NE) halo[(e % CT) * kHaloStride + e / CT] = in[b] ? v[b] : 0.f;
        }
      }
    }
    {
      constexpr int NW4 = CT * 9 * 4;  // float4 groups of this chunk's weights
      const float4* wsrc = reinterpret_cast<const float4*>(a.w + ((size_t)cg * CIN + c0) * 9 * 16);
#pragma unroll
      for (int k = 0; k < (NW4 + 127) / 128; ++k) {
        const int e = tid + k * 128;
        if (e < NW4) reinterpret_cast<float4*>(ws)[e] = __ldg(wsrc + e);
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < CT; ++c) {
      const float* hc = halo + c * kHaloStride;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          float v0 = hc[(ty + ky) * kHW + tx + kx];
          float v1 = hc[(ty + 1 + ky) * kHW + tx + kx];
          const float4* w4 = reinterpret_cast<const float4*>(ws + (c * 9 + ky * 3 + kx) * 16);
          const float2 vv0 = make_float2(v0, v0), vv1 = make_float2(v1, v1);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 w = w4[q];
            const float2 wa = make_float2(w.x, w.y), wb = make_float2(w.z, w.w);
            p0[2 * q] = __ffma2_rn(vv0, wa, p0[2 * q]);
            p0[2 * q + 1] = __ffma2_rn(vv0, wb, p0[2 * q + 1]);
            p1[2 * q] = __ffma2_rn(vv1, wa, p1[2 * q]);
            p1[2 * q + 1] = __ffma2_rn(vv1, wb, p1[2 * q + 1]);
          }
        }
    }
  }
  float acc0[16], acc1[16];
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    acc0[2 * o] = p0[o].x; acc0[2 * o + 1] = p0[o].y;
    acc1[2 * o] = p1[o].x; acc1[2 * o + 1] = p1[o].y;
  }
  const int x = x0 + tx;
  if constexpr (sizeof(TOut) == 2) {
    // maximum of this tile's stored outputs (every thread of the warp takes part)
    if (a.amax) {
      float mx = 0.f;
      const float* bias = a.b + cg * 16;
      for (int r = 0; r < 2; ++r) {
        if (x >= a.W || y0 + ty + r >= a.H) continue;
        const float* acc = r ? acc1 : acc0;
#pragma unroll
        for (int q = 0; q < 16; ++q) mx = fmaxf(mx, fmaxf(acc[q] + __ldg(bias + q), 0.f));
      }
      mx = __half2float(__float2half_rn(mx));
      const unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
      if ((threadIdx.x & 31) == 0 && bits) atomicMax(reinterpret_cast<unsigned int*>(a.amax), bits);
    }
  }
  if (x >= a.W) return;
  if (nks > 1) {   // raw partial sums of this split
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int y = y0 + ty + r;
      if (y >= a.H) continue;
      float* dst = partial + ((size_t)ks * a.H * a.W + (size_t)y * a.W + x) * cout + cg * 16;
      const float* acc = r ? acc1 : acc0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        reinterpret_cast<float4*>(dst)[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
    return;
  }
  const float* bias = a.b + cg * 16;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    int y = y0 + ty + r;
    if (y >= a.H) continue;
    TOut* dst = static_cast<TOut*>(a.out) + ((size_t)y * a.W + x) * cout + cg * 16;
    const float* acc = r ? acc1 : acc0;
    if constexpr (sizeof(TOut) == 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float4 v;
        v.x = fmaxf(acc[4 * q + 0] + __ldg(bias + 4 * q + 0), 0.f);
        v.y = fmaxf(acc[4 * q + 1] + __ldg(bias + 4 * q + 1), 0.f);
        v.z = fmaxf(acc[4 * q + 2] + __ldg(bias + 4 * q + 2), 0.f);
        v.w = fmaxf(acc[4 * q + 3] + __ldg(bias + 4 * q + 3), 0.f);
        reinterpret_cast<float4*>(dst)[q] = v;
      }
    } else {
      __align__(16) uint32_t h[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        h[q] = pack_pair<TOut>(fmaxf(acc[2 * q] + __ldg(bias + 2 * q), 0.f),
                               fmaxf(acc[2 * q + 1] + __ldg(bias + 2 * q + 1), 0.f));
      reinterpret_cast<uint4*>(dst)[0] = reinterpret_cast<const uint4*>(h)[0];
      reinterpret_cast<uint4*>(dst)[1] = reinterpret_cast<const uint4*>(h)[1];
    }
  }
}

// 2x2 stride-2 transposed convolution: one thread per input pixel, 16 output
// channels of all four output pixels it feeds.  Weights packed [cout/16][cin][4][16].
template <int CIN>
__global__ void __launch_bounds__(128) convT_f32_kernel(const float* __restrict__ in,
                                                        const float* __restrict__ w,
                                                        const float* __restrict__ b,
                                                        float* __restrict__ out, int H, int W,
                                                        int cout) {
  extern __shared__ __align__(16) float wsm[];  // CIN * 64
  const int cg = blockIdx.y;
  const float* wsrc = w + (size_t)cg * CIN * 64;
  for (int e = threadIdx.x; e < CIN * 64; e += 128) wsm[e] = __ldg(wsrc + e);
  __syncthreads();
  const int p = blockIdx.x * 128 + threadIdx.x;
  if (p >= H * W) return;
  const int y = p / W, x = p % W;
  float acc[4][16];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int o = 0; o < 16; ++o) acc[k][o] = 0.f;
  const float4* src = reinterpret_cast<const float4*>(in + (size_t)p * CIN);
#pragma unroll 1
  for (int c4 = 0; c4 < CIN / 4; ++c4) {
    float4 v4 = __ldg(src + c4);
    float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const float4* wr = reinterpret_cast<const float4*>(wsm + (c4 * 4 + cc) * 64);
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float4 ww = wr[k * 4 + q];
          acc[k][4 * q + 0] = fmaf(vv[cc], ww.x, acc[k][4 * q + 0]);
          acc[k][4 * q + 1] = fmaf(vv[cc], ww.y, acc[k][4 * q + 1]);
          acc[k][4 * q + 2] = fmaf(vv[cc], ww.z, acc[k][4 * q + 2]);
          acc[k][4 * q + 3] = fmaf(vv[cc], ww.w, acc[k][4 * q + 3]);
        }
    }
  }
  const int W2 = 2 * W;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int oy = 2 * y + (k >> 1), ox = 2 * x + (k & 1);
    float4* dst = reinterpret_cast<float4*>(out + ((size_t)oy * W2 + ox) * cout + cg * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float4 v;
      v.x = acc[k][4 * q + 0] + __ldg(b + cg * 16 + 4 * q + 0);
      v.y = acc[k][4 * q + 1] + __ldg(b + cg * 16 + 4 * q + 1);
      v.z = acc[k][4 * q + 2] + __ldg(b + cg * 16 + 4 * q + 2);
      v.w = acc[k][4 * q + 3] + __ldg(b + cg * 16 + 4 * q + 3);
      dst[q] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// weights and forward
// ---------------------------------------------------------------------------
struct NetF32Weights {
  float* conv_w[14];   // packed [cout/16][cin][9][16]
  float* conv_b[14];
  float* up_w[3];      // packed [cout/16][cin][4][16]
  float* up_b[3];
  AdapterParamSet adp; // folded adapter parameters (base width kC0)
  AdapterWideWeights* wide = nullptr;  // the adapters at base width kWideC0
  int c0 = kC0;
  int conv_cin[14], conv_cout[14], up_cin[3], up_cout[3];
  std::vector<void*> allocs;
};

static float* upload(NetF32Weights* w, const std::vector<float>& v, cudaError_t* err) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, v.size() * sizeof(float));
  if (e != cudaSuccess) { *err = e; return nullptr; }
  w->allocs.push_back(p);
  e = cudaMemcpy(p, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) *err = e;
  return static_cast<float*>(p);
}

NetF32Weights* net_f32_create(const float* hp, const NetLayout& L, cudaError_t* err) {
  *err = cudaSuccess;
  NetF32Weights* w = new NetF32Weights();
  for (int l = 0; l < 14; ++l) {
    int cin = L.conv_cin[l], cout = L.conv_cout[l];
    w->conv_cin[l] = cin; w->conv_cout[l] = cout;
    std::vector<float> pk((size_t)cout * cin * 9);
    const float* src = hp + L.conv_w[l];  // [cout][cin][3][3]
    for (int co = 0; co < cout; ++co)
      for (int ci = 0; ci < cin; ++ci)
        for (int k = 0; k < 9; ++k)
          pk[(((size_t)(co / 16) * cin + ci) * 9 + k) * 16 + co % 16] = src[((size_t)co * cin + ci) * 9 + k];
    w->conv_w[l] = upload(w, pk, err);
    w->conv_b[l] = upload(w, std::vector<float>(hp + L.conv_b[l], hp + L.conv_b[l] + cout), err);
  }
  for (int l = 0; l < 3; ++l) {
    int cin = L.up_cin[l], cout = L.up_cout[l];
    w->up_cin[l] = cin; w->up_cout[l] = cout;
    std::vector<float> pk((size_t)cout * cin * 4);
    const float* src = hp + L.up_w[l];  // [cin][cout][2][2]
    for (int ci = 0; ci < cin; ++ci)
      for (int co = 0; co < cout; ++co)
        for (int k = 0; k < 4; ++k)
          pk[(((size_t)(co / 16) * cin + ci) * 4 + k) * 16 + co % 16] = src[((size_t)ci * cout + co) * 4 + k];
    w->up_w[l] = upload(w, pk, err);
    w->up_b[l] = upload(w, std::vector<float>(hp + L.up_b[l], hp + L.up_b[l] + cout), err);
  }
  w->c0 = L.c0;
  if (L.c0 == kC0) {
    adapter_params_from(hp + L.adapter[0], &w->adp.p1, &w->adp.sca, &w->adp.p2);
  } else if (*err == cudaSuccess) {
    w->wide = adapters_wide_create(hp + L.adapter[0], err);
  }
  if (*err != cudaSuccess) { net_f32_destroy(w); return nullptr; }
  return w;
}

const float* net_f32_conv_w(const NetF32Weights* w, int l) { return w->conv_w[l]; }
const float* net_f32_conv_b(const NetF32Weights* w, int l) { return w->conv_b[l]; }
const AdapterParamSet& net_f32_adapter_params(const NetF32Weights* w) { return w->adp; }

void net_f32_destroy(NetF32Weights* w) {
  if (!w) return;
  for (void* p : w->allocs) cudaFree(p);
  adapters_wide_destroy(w->wide);
  delete w;
}

// workspace carve-up (floats), P = max pixels
struct F32Buffers {
  float *fa, *fb, *s1, *l1a, *l1b, *s2, *l2a, *l2b, *s3, *l3a, *l3b, *x1, *partial, *att;
  float* split;         // input-channel split partial sums of the low-resolution layers
  size_t split_floats;
};

// floats of the split partial sums (4 C0 bytes per pixel of the largest image
// plus 4 MiB): conv() splits a layer only as far as nks * pixels * cout fits
static size_t split_capacity(size_t P, int c0) { return P * c0 + ((size_t)1 << 20); }

// P = max pixels (a multiple of 64: both sides are multiples of 8), c0 = base width
static size_t carve(size_t P, int c0, F32Buffers* b, char* base) {
  size_t off = 0;
  auto take = [&](size_t nfloats) {
    float* p = base ? reinterpret_cast<float*>(base + off) : nullptr;
    off += ((nfloats * sizeof(float) + 255) / 256) * 256;
    return p;
  };
  const size_t c = (size_t)c0;
  b->fa = take(P * c); b->fb = take(P * c); b->s1 = take(P * c);
  b->l1a = take(P / 4 * 2 * c); b->l1b = take(P / 4 * 2 * c); b->s2 = take(P / 4 * 2 * c);
  b->l2a = take(P / 16 * 4 * c); b->l2b = take(P / 16 * 4 * c); b->s3 = take(P / 16 * 4 * c);
  b->l3a = take(P / 64 * 8 * c); b->l3b = take(P / 64 * 8 * c);
  b->x1 = take(P * 4 * c);
  b->partial = take(c0 == kC0 ? adapter_partial_floats((int)P, 1) + (P / 128 + 1024) * 64
                              : adapter_wide_partial_floats((int)P, 1));
  b->att = take(8 * c);
  b->split_floats = split_capacity(P, c0);
  b->split = take(b->split_floats);
  return off;
}

size_t net_f32_workspace_bytes(int max_w, int max_h, int c0) {
  F32Buffers b;
  return carve((size_t)max_w * max_h, c0, &b, nullptr);
}

// A layer whose tiles and output-channel groups give fewer than two blocks per
// SM splits its input channels over up to CIN / 16 blocks (powers of two),
// then conv_split_finish adds the partial sums: the low-resolution layers of a
// small image otherwise run a handful of blocks through long channel loops.
template <int CIN, int MODE, typename TOut = float>
static cudaError_t conv(const ConvArgs& a, int cout, cudaStream_t s, float* split = nullptr,
                        size_t split_floats = 0) {
  const int tiles = ((a.W + kTW - 1) / kTW) * ((a.H + kTH - 1) / kTH);
  const size_t P = (size_t)a.W * a.H;
  int nks = 1;
  if (sizeof(TOut) == 4 && CIN >= 32 && split)
    while (tiles * (cout / 16) * nks < 2 * num_sms() && 2 * nks <= CIN / 16 &&
           (size_t)(2 * nks) * P * cout <= split_floats)
      nks *= 2;
  dim3 grid((a.W + kTW - 1) / kTW, (a.H + kTH - 1) / kTH, cout / 16 * nks);
  conv3x3_f32_kernel<CIN, MODE, TOut><<<grid, 128, 0, s>>>(a, cout, nks, split);
  if (nks > 1) {
    int blocks = (int)((P * cout / 4 + 255) / 256);
    if (blocks > num_sms() * 8) blocks = num_sms() * 8;
    conv_split_finish<<<blocks, 256, 0, s>>>(split, nks, a.b, static_cast<float*>(a.out), (int)P, cout);
  }
  return cudaGetLastError();
}

// First layer (guide -> C0) on the SIMT cores with a 16-bit NHWC output: the
// tensor-core path starts at the second layer (K = 27 is too narrow a GEMM).
template <typename T>
cudaError_t simt_first_conv_half(const NetF32Weights* w, const NetImage& img, T* out,
                                 cudaStream_t s) {
  ConvArgs a{img.guide, nullptr, net_f32_conv_w(w, 0), net_f32_conv_b(w, 0), out, img.H, img.W,
             img.depth_scale};
  return conv<3, IN_GUIDE, T>(a, 16, s);
}
template <typename T>
cudaError_t simt_first_conv_group(const NetF32Weights* w, const NetImage* imgs, T* const* outs,
                                  float* const* amax, int n, cudaStream_t s) {
  if (n < 1 || n > kMaxGroup) return cudaErrorInvalidValue;
  ConvGroupArgs G{};
  G.nimg = n;
  int tiles = 0;
  for (int k = 0; k < n; ++k) {
    G.img[k] = ConvArgs{imgs[k].guide, nullptr, net_f32_conv_w(w, 0), net_f32_conv_b(w, 0), outs[k],
                        imgs[k].H, imgs[k].W, imgs[k].depth_scale, amax ? amax[k] : nullptr};
    G.tile_start[k] = tiles;
    tiles += ((imgs[k].W + kTW - 1) / kTW) * ((imgs[k].H + kTH - 1) / kTH);
  }
  G.tile_start[n] = tiles;
  return launch_pdl(first_conv_group_kernel<T>, dim3(tiles), dim3(128), 0, s, G);
}
template cudaError_t simt_first_conv_group<__nv_bfloat16>(const NetF32Weights*, const NetImage*,
                                                          __nv_bfloat16* const*, float* const*, int,
                                                          cudaStream_t);
template cudaError_t simt_first_conv_group<__half>(const NetF32Weights*, const NetImage*,
                                                   __half* const*, float* const*, int, cudaStream_t);
template cudaError_t simt_first_conv_group<float>(const NetF32Weights*, const NetImage*, float* const*,
                                                  float* const*, int, cudaStream_t);
template cudaError_t simt_first_conv_half<__nv_bfloat16>(const NetF32Weights*, const NetImage&,
                                                         __nv_bfloat16*, cudaStream_t);
template cudaError_t simt_first_conv_half<__half>(const NetF32Weights*, const NetImage&, __half*,
                                                  cudaStream_t);


template <int CIN>
static cudaError_t convT(const float* in, const float* w, const float* b, float* out, int H, int W,
                         int cout, cudaStream_t s) {
  dim3 grid((H * W + 127) / 128, cout / 16);
  size_t smem = (size_t)CIN * 64 * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(convT_f32_kernel<CIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  convT_f32_kernel<CIN><<<grid, 128, smem, s>>>(in, w, b, out, H, W, cout);
  return cudaGetLastError();
}

// The UNet of base width C0 (Fig. 3): encoder, decoder, then the adapters.
template <int C0>
static cudaError_t forward_f32(const NetF32Weights* w, const NetImage& img, const F32Buffers& B,
                               cudaStream_t s) {
  constexpr int C1 = 2 * C0, C2 = 4 * C0, C3 = 8 * C0;
  const int H = img.H, W = img.W;
  cudaError_t e;
#define TRY(x) if ((e = (x)) != cudaSuccess) return e
  auto A = [&](const float* inA, const float* inB, int l, float* out, int h, int ww) {
    ConvArgs a{inA, inB, w->conv_w[l], w->conv_b[l], out, h, ww, img.depth_scale};
    return a;
  };
  float* const sp = B.split;
  const size_t sf = B.split_floats;
  const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  // encoder
  TRY((conv<3, IN_GUIDE>(A(img.guide, nullptr, 0, B.fa, H, W), C0, s)));
  TRY((conv<C0, IN_PLAIN>(A(B.fa, nullptr, 1, B.s1, H, W), C0, s, sp, sf)));
  TRY((conv<C0, IN_POOL>(A(B.s1, nullptr, 2, B.l1a, H1, W1), C1, s, sp, sf)));
  TRY((conv<C1, IN_PLAIN>(A(B.l1a, nullptr, 3, B.s2, H1, W1), C1, s, sp, sf)));
  TRY((conv<C1, IN_POOL>(A(B.s2, nullptr, 4, B.l2a, H2, W2), C2, s, sp, sf)));
  TRY((conv<C2, IN_PLAIN>(A(B.l2a, nullptr, 5, B.s3, H2, W2), C2, s, sp, sf)));
  TRY((conv<C2, IN_POOL>(A(B.s3, nullptr, 6, B.l3a, H3, W3), C3, s, sp, sf)));
  TRY((conv<C3, IN_PLAIN>(A(B.l3a, nullptr, 7, B.l3b, H3, W3), C3, s, sp, sf)));
  // decoder
  TRY(convT<C3>(B.l3b, w->up_w[0], w->up_b[0], B.l2a, H3, W3, C2, s));
  TRY((conv<2 * C2, IN_CONCAT>(A(B.l2a, B.s3, 8, B.l2b, H2, W2), C2, s, sp, sf)));
  TRY((conv<C2, IN_PLAIN>(A(B.l2b, nullptr, 9, B.l2a, H2, W2), C2, s, sp, sf)));
  TRY(convT<C2>(B.l2a, w->up_w[1], w->up_b[1], B.l1a, H2, W2, C1, s));
  TRY((conv<2 * C1, IN_CONCAT>(A(B.l1a, B.s2, 10, B.l1b, H1, W1), C1, s, sp, sf)));
  TRY((conv<C1, IN_PLAIN>(A(B.l1b, nullptr, 11, B.l1a, H1, W1), C1, s, sp, sf)));
  TRY(convT<C1>(B.l1a, w->up_w[2], w->up_b[2], B.fa, H1, W1, C0, s));
  TRY((conv<2 * C0, IN_CONCAT>(A(B.fa, B.s1, 12, B.fb, H, W), C0, s, sp, sf)));
  TRY((conv<C0, IN_PLAIN>(A(B.fb, nullptr, 13, B.fa, H, W), C0, s, sp, sf)));
  // adapters
  if constexpr (C0 == kC0) {
    TRY(adapters_run<float>(w->adp, B.fa, B.x1, B.partial, B.att, img.out, H, W, s));
  } else {
    TRY(adapters_wide_run(w->wide, B.fa, B.x1, B.partial, B.att, img.out, H, W, s));
  }
#undef TRY
  return cudaSuccess;
}

cudaError_t net_f32_forward(const NetF32Weights* w, const NetImage& img, void* workspace,
                            size_t ws_bytes, cudaStream_t s) {
  const size_t P = (size_t)img.H * img.W;
  F32Buffers B;
  if (carve(P, w->c0, &B, nullptr) > ws_bytes) return cudaErrorInvalidValue;
  carve(P, w->c0, &B, static_cast<char*>(workspace));
  if (w->c0 == kWideC0) return forward_f32<kWideC0>(w, img, B, s);
  return forward_f32<kC0>(w, img, B, s);
}

}  // namespace nsl
