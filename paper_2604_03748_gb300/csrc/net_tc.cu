// Lightmap network convolutions on the 5th-generation tensor cores (sm_103a):
// implicit-GEMM 3x3 convolutions and 2x2 stride-2 transposed convolutions with
// BF16 operands and FP32 accumulation in tensor memory (Sec. 4.3 UNet).
//
// 3x3 convolution as a GEMM: M = 128 output pixels (a 16-row x 8-column patch),
// N = output channels, K = 9 taps x Cin.  The input patch plus its one-pixel
// halo (18 x 10 pixels) is staged once in shared memory as "core-matrix"
// planes: for each group of 8 channels, the 180 halo pixels lie 16 bytes apart.
// With that layout the A operand of tap (dy, dx) is the same planes read from a
// start address shifted by (dy*10 + dx) pixels: 8 consecutive halo pixels form
// one 8x16-byte core matrix, consecutive patch rows are 160 bytes apart (the
// stride-dimension offset), and the two 8-channel halves of a 16-channel K step
// are one plane apart (the leading-dimension offset).  No im2col copy exists.
//
// Weights (the B operand, K-major) are pre-packed on the host into the same
// core-matrix order, one 16-channel K slice per (tap, channel chunk), and
// copied into shared memory once per CTA with a bulk async copy.  A CTA is
// persistent over M tiles: while the tensor core works on tile i (accumulator
// buffer i%2 in TMEM), the CTA's 128 threads read tile i-1's accumulators out
// of TMEM (tcgen05.ld), add the bias, apply ReLU, convert to BF16 and store
// NHWC rows, and stage tile i+1's halo.
//
// Every wait on an mbarrier is bounded; on timeout the kernel records an error
// code in a host-visible word, frees its TMEM and returns.
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp8.h>
#include "nsl_internal.cuh"
#include "tc_ptx.cuh"

namespace nsl {

namespace {

enum TcMode { TC_PLAIN = 0, TC_POOL = 1, TC_CONCAT = 2 };

constexpr int kPatchW = 8, kPatchH = 16;                     // M tile = 128 pixels
constexpr int kHaloW = kPatchW + 2, kHaloH = kPatchH + 2;    // 10 x 18
constexpr int kHaloPix = kHaloW * kHaloH;                    // 180
constexpr int kPlane = kHaloPix * 16;                        // bytes per 8-channel plane
#ifndef NSL_CONV_CTAS_PER_SM
#define NSL_CONV_CTAS_PER_SM 4
#endif
#ifndef NSL_CONV_MIN_TILES
#define NSL_CONV_MIN_TILES 1
#endif
constexpr int kConvCtasPerSM = NSL_CONV_CTAS_PER_SM;

// 16-bit operand types of kind::f16: BF16 (format code 1) and FP16 (code 0).
template <typename T> struct Half;
template <> struct Half<__nv_bfloat16> {
  using T2 = __nv_bfloat162;
  static constexpr uint32_t kFmt = 1;
  static __device__ __forceinline__ T2 pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
  static __host__ __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
};
template <> struct Half<__half> {
  using T2 = __half2;
  static constexpr uint32_t kFmt = 0;
  static __device__ __forceinline__ T2 pack(float a, float b) { return __floats2half2_rn(a, b); }
  static __host__ __device__ __forceinline__ __half from(float v) { return __float2half_rn(v); }
};

template <typename T>
__device__ __forceinline__ uint4 half8_max(uint4 a, uint4 b) {
  using T2 = typename Half<T>::T2;
  uint4 r;
  const T2* pa = reinterpret_cast<const T2*>(&a);
  const T2* pb = reinterpret_cast<const T2*>(&b);
  T2* pr = reinterpret_cast<T2*>(&r);
#pragma unroll
  for (int i = 0; i < 4; ++i) pr[i] = __hmax2(pa[i], pb[i]);
  return r;
}

__device__ __forceinline__ uint4 ldg128(const void* p) {
  return __ldg(reinterpret_cast<const uint4*>(p));
}

// FP8 path: 16 FP16 activations (two 16-byte words, channel order) times the
// tensor's inverse scale (a power of two, so the product is exact), each
// converted to E4M3 by the hardware's paired conversion (round to nearest
// even, saturating at the largest finite magnitude 448); byte c of the result
// is channel c.
__device__ __forceinline__ uint4 q8_pack16(uint4 lo, uint4 hi, float inv) {
  const __half2* h0 = reinterpret_cast<const __half2*>(&lo);
  const __half2* h1 = reinterpret_cast<const __half2*>(&hi);
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __half2 pa = q < 2 ? h0[2 * q] : h1[2 * q - 4];
    const __half2 pb = q < 2 ? h0[2 * q + 1] : h1[2 * q - 3];
    const float2 fa = __half22float2(pa), fb = __half22float2(pb);
    const uint32_t c01 = __nv_cvt_float2_to_fp8x2(make_float2(__fmul_rn(fa.x, inv), __fmul_rn(fa.y, inv)),
                                                  __NV_SATFINITE, __NV_E4M3);
    const uint32_t c23 = __nv_cvt_float2_to_fp8x2(make_float2(__fmul_rn(fb.x, inv), __fmul_rn(fb.y, inv)),
                                                  __NV_SATFINITE, __NV_E4M3);
    w[q] = (c01 & 0xffffu) | (c23 << 16);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Per-tensor activation scale: the smallest power of two s = 2^k with
// amax <= 448 s (448 = 0.875 * 2^9, so with amax = f 2^e, f in [0.5, 1):
// k = e - 9 if f <= 0.875, else e - 8); s = 1 for an all-zero tensor.
// Quantising multiplies by 2^-k (exact), dequantising by 2^k.  A power of two
// leaves every quantisation decision unchanged under tiny changes of amax.
__device__ __forceinline__ int q8_exp(float amax) {
  if (!(amax > 0.f)) return 0;
  int e;
  const float f = frexpf(amax, &e);
  return e - 9 + (f > 0.875f ? 1 : 0);
}
__device__ __forceinline__ float q8_inv(float amax) { return ldexpf(1.f, -q8_exp(amax)); }
__device__ __forceinline__ float q8_deq(float amax) { return ldexpf(1.f, q8_exp(amax)); }

// Warp-wide max of non-negative values folded into a tensor's amax word.
__device__ __forceinline__ void amax_publish(float* slot, float v) {
  const unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
  if ((threadIdx.x & 31) == 0 && bits) atomicMax(reinterpret_cast<unsigned int*>(slot), bits);
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}


// One image of a (grouped) layer launch.  A launch covers up to kMaxGroup
// images of any sizes that share the layer's weights; tiles are numbered
// image after image (tile_start is the image's first global tile).
template <typename T>
struct ConvImg {
  const T* inA;              // NHWC input (POOL: at 2H x 2W; CONCAT: first CIN/2 channels)
  const T* inB;              // CONCAT: last CIN/2 channels (the skip tensor)
  T* out;                    // NHWC [H][W][COUT]
  int H, W;                  // convolution (output) size
  int tiles_x;               // M tiles per row
  int tile_start;
  // FP8 path: amax words of the input tensor (two for a concatenation) and of
  // the output tensor (accumulated here)
  const float* amax_a;
  const float* amax_b;
  float* amax_out;
};

template <typename T>
struct TcConvArgs {
  ConvImg<T> img[kMaxGroup];
  int nimg, total_tiles;
  const uint8_t* wpack;      // [n tiles][9 taps][K steps][NT rows x 32 bytes]
  const float* bias;         // [COUT]
  const float* wscale;       // FP8 path: per-output-channel weight scales [COUT]
  unsigned int* err;
};

// image of global tile t (uniform across the CTA) and the tile inside it
template <typename A>
__device__ __forceinline__ int image_of(const A& a, int t) {
  int lo = 0, hi = a.nimg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.img[mid].tile_start <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Stage the halo of M tile `tile` into `halo` (CIN/8 planes of 180 x 16 bytes).
template <typename T, int CIN, int MODE>
__device__ __forceinline__ void load_halo(const ConvImg<T>& a, int tile, uint8_t* halo);

// Stage the halo of M tile `tile` with asynchronous 16-byte copies (zero fill
// outside the image); the max-pool mode reduces 2x2 pixels in registers.
template <typename T, int CIN, int MODE>
__device__ __forceinline__ void load_halo_async(const ConvImg<T>& a, int tile, uint8_t* halo) {
  if constexpr (MODE == TC_POOL) {
    load_halo<T, CIN, MODE>(a, tile, halo);
  } else {
    constexpr int G = CIN / 8;
    const int ty = tile / a.tiles_x, tx = tile % a.tiles_x;
    const int y0 = ty * kPatchH - 1, x0 = tx * kPatchW - 1;
    for (int e = threadIdx.x; e < kHaloPix * G; e += blockDim.x) {
      const int hp = e / G, g = e % G;
      const int y = y0 + hp / kHaloW, x = x0 + hp % kHaloW;
      const bool in = y >= 0 && y < a.H && x >= 0 && x < a.W;
      const int yc = in ? y : 0, xc = in ? x : 0;
      const T* src;
      if constexpr (MODE == TC_PLAIN) {
        src = a.inA + ((size_t)yc * a.W + xc) * CIN + g * 8;
      } else {
        constexpr int CH = CIN / 2;
        src = g < G / 2 ? a.inA + ((size_t)yc * a.W + xc) * CH + g * 8
                        : a.inB + ((size_t)yc * a.W + xc) * CH + (g - G / 2) * 8;
      }
      cp_async16(halo + g * kPlane + hp * 16, src, in ? 16u : 0u);
    }
  }
}

// Synchronous halo loaders (max-pool mode, FP8 path): each thread takes its
// elements in batches of kLdBatch and issues every global load of a batch
// before the first use, so it waits for one round of memory latency per batch
// rather than per element (a low-resolution layer's CTA stages one tile, and
// those rounds were most of its time).  Out-of-image elements load from a
// clamped in-image address and are replaced by zeros afterwards, which keeps
// the loads free of branches.
constexpr int kLdBatch = 4;

// 8 channels (16 bytes) of halo pixel (y, x), clamped into the image, at
// channel group g (POOL: the 2x2 max of the finer level)
template <typename T, int CIN, int MODE>
__device__ __forceinline__ uint4 halo8(const ConvImg<T>& a, int y, int x, int g) {
  if constexpr (MODE == TC_PLAIN) {
    return ldg128(a.inA + ((size_t)y * a.W + x) * CIN + g * 8);
  } else if constexpr (MODE == TC_CONCAT) {
    constexpr int G = CIN / 8, CH = CIN / 2;
    return g < G / 2 ? ldg128(a.inA + ((size_t)y * a.W + x) * CH + g * 8)
                     : ldg128(a.inB + ((size_t)y * a.W + x) * CH + (g - G / 2) * 8);
  } else {
    const size_t W2 = 2 * (size_t)a.W;
    const T* p = a.inA + ((size_t)(2 * y) * W2 + 2 * x) * CIN + g * 8;
    return half8_max<T>(half8_max<T>(ldg128(p), ldg128(p + CIN)),
                        half8_max<T>(ldg128(p + W2 * CIN), ldg128(p + W2 * CIN + CIN)));
  }
}

template <typename T, int CIN, int MODE>
__device__ __forceinline__ void load_halo(const ConvImg<T>& a, int tile, uint8_t* halo) {
  constexpr int G = CIN / 8, NE = kHaloPix * G;
  const int ty = tile / a.tiles_x, tx = tile % a.tiles_x;
  const int y0 = ty * kPatchH - 1, x0 = tx * kPatchW - 1;
  for (int e0 = threadIdx.x; e0 < NE; e0 += kLdBatch * blockDim.x) {
    uint4 v[kLdBatch];
    bool in[kLdBatch];
#pragma unroll
    for (int b = 0; b < kLdBatch; ++b) {
      const int e = min(e0 + b * (int)blockDim.x, NE - 1);
      const int hp = e / G, g = e % G;
      const int y = y0 + hp / kHaloW, x = x0 + hp % kHaloW;
      in[b] = y >= 0 && y < a.H && x >= 0 && x < a.W;
      v[b] = halo8<T, CIN, MODE>(a, min(max(y, 0), a.H - 1), min(max(x, 0), a.W - 1), g);
    }
#pragma unroll
    for (int b = 0; b < kLdBatch; ++b) {
      const int e = e0 + b * (int)blockDim.x;
      if (e < NE)
        *reinterpret_cast<uint4*>(halo + (e % G) * kPlane + (e / G) * 16) = in[b] ? v[b] : make_uint4(0, 0, 0, 0);
    }
  }
}

// FP8 path: stage the halo as planes of 16 E4M3 channels (CIN/16 planes),
// quantising the FP16 activations with the input tensor's scale on the way.
template <int CIN, int MODE>
__device__ __forceinline__ void load_halo_q8(const ConvImg<__half>& a, int tile, uint8_t* halo) {
  constexpr int GR = CIN / 16, NE = kHaloPix * GR;
  const float am = a.amax_b ? fmaxf(__ldg(a.amax_a), __ldg(a.amax_b)) : __ldg(a.amax_a);
  const float inv = q8_inv(am);
  const int ty = tile / a.tiles_x, tx = tile % a.tiles_x;
  const int y0 = ty * kPatchH - 1, x0 = tx * kPatchW - 1;
  for (int e0 = threadIdx.x; e0 < NE; e0 += kLdBatch * blockDim.x) {
    uint4 lo[kLdBatch], hi[kLdBatch];
    bool in[kLdBatch];
#pragma unroll
    for (int b = 0; b < kLdBatch; ++b) {
      const int e = min(e0 + b * (int)blockDim.x, NE - 1);
      const int hp = e / GR, g = e % GR;
      const int y = y0 + hp / kHaloW, x = x0 + hp % kHaloW;
      in[b] = y >= 0 && y < a.H && x >= 0 && x < a.W;
      const int yc = min(max(y, 0), a.H - 1), xc = min(max(x, 0), a.W - 1);
      // channels 16g .. 16g+15 are the 8-channel groups 2g and 2g+1 (a
      // concatenation's halves hold whole 16-channel groups)
      lo[b] = halo8<__half, CIN, MODE>(a, yc, xc, 2 * g);
      hi[b] = halo8<__half, CIN, MODE>(a, yc, xc, 2 * g + 1);
    }
#pragma unroll
    for (int b = 0; b < kLdBatch; ++b) {
      const int e = e0 + b * (int)blockDim.x;
      if (e < NE)
        *reinterpret_cast<uint4*>(halo + (e % GR) * kPlane + (e / GR) * 16) =
            in[b] ? q8_pack16(lo[b], hi[b], inv) : make_uint4(0, 0, 0, 0);
    }
  }
}

template <typename T, int NT, bool Q8>
__device__ __forceinline__ float conv_epilogue(const ConvImg<T>& a, const float* __restrict__ bias,
                                              const float* __restrict__ wscale, int tile,
                                              uint32_t tacc, int n0, int cout) {
  const int warp = threadIdx.x >> 5;
  const int m = threadIdx.x;  // accumulator row = pixel of the patch
  const int ty = tile / a.tiles_x, tx = tile % a.tiles_x;
  const int y = ty * kPatchH + m / kPatchW, x = tx * kPatchW + m % kPatchW;
  const bool valid = y < a.H && x < a.W;
  T* dst = a.out + ((size_t)y * a.W + x) * cout + n0;
  float deq = 1.f, mx = 0.f;
  if constexpr (Q8)
    deq = q8_deq(a.amax_b ? fmaxf(__ldg(a.amax_a), __ldg(a.amax_b)) : __ldg(a.amax_a));
#pragma unroll
  for (int c = 0; c < NT; c += 16) {
    float v[16];
    tmem_ld16(tacc + ((uint32_t)(warp * 32) << 16) + c, v);
    __align__(16) typename Half<T>::T2 h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float r0, r1;
      if constexpr (Q8) {
        r0 = fmaxf(fmaf(v[2 * q], __fmul_rn(deq, __ldg(wscale + n0 + c + 2 * q)),
                        __ldg(bias + n0 + c + 2 * q)), 0.f);
        r1 = fmaxf(fmaf(v[2 * q + 1], __fmul_rn(deq, __ldg(wscale + n0 + c + 2 * q + 1)),
                        __ldg(bias + n0 + c + 2 * q + 1)), 0.f);
        mx = fmaxf(mx, fmaxf(r0, r1));
      } else {
        r0 = fmaxf(v[2 * q] + __ldg(bias + n0 + c + 2 * q), 0.f);
        r1 = fmaxf(v[2 * q + 1] + __ldg(bias + n0 + c + 2 * q + 1), 0.f);
      }
      h[q] = Half<T>::pack(r0, r1);
    }
    if (valid) {
      reinterpret_cast<uint4*>(dst + c)[0] = reinterpret_cast<const uint4*>(h)[0];
      reinterpret_cast<uint4*>(dst + c)[1] = reinterpret_cast<const uint4*>(h)[1];
    }
  }
  // FP8 path: this thread's largest stored (FP16-rounded) value, rounding
  // being monotonic; the kernel publishes the running maximum
  return Q8 && valid ? __half2float(__float2half_rn(mx)) : 0.f;
}


// N tile of a 3x3 layer: all output channels up to 64, and 32 when Cin = 128
// so that weights + two halo buffers fit in 227 KB of shared memory.
#ifndef NSL_CONV_NT_MAX
#define NSL_CONV_NT_MAX 64
#endif
__host__ __device__ constexpr int conv_nt(int cin, int cout) {
  return cin >= 128 ? (NSL_CONV_NT_MAX < 32 ? NSL_CONV_NT_MAX : 32)
                    : (cout > NSL_CONV_NT_MAX ? NSL_CONV_NT_MAX : cout);
}

template <int CIN, int COUT, int NT, bool Q8 = false>
struct ConvCfg {
  // a plane holds 16 bytes per halo pixel: 8 FP16/BF16 channels or 16 FP8 ones;
  // one MMA consumes two planes (K = 16 or 32).  FP8 with 16 channels stages
  // a zero second plane.
  static constexpr int GR = Q8 ? CIN / 16 : CIN / 8;     // planes holding channels
  static constexpr int G = GR < 2 ? 2 : GR;              // planes staged
  static constexpr int KS = G / 2;                       // K steps per tap
  static constexpr int WBYTES = 9 * KS * NT * 32;        // B operand of one N tile
  static constexpr int HBYTES = G * kPlane;              // one halo buffer
  // halo buffers in flight: as many as fit next to the weights (2..4)
  static constexpr int STAGES =
      (WBYTES + 4 * HBYTES + 64 <= 110 * 1024) ? 4 : ((WBYTES + 3 * HBYTES + 64 <= 227 * 1024) ? 3 : 2);
  static constexpr int TMEM_COLS = 2 * NT < 32 ? 32 : 2 * NT;
  static constexpr int SMEM = WBYTES + STAGES * HBYTES + 64;  // + barriers and TMEM slot
};

template <typename T, int CIN, int COUT, int NT, int MODE, bool Q8>
__global__ void __launch_bounds__(128) conv3x3_tc_kernel(TcConvArgs<T> a) {
  using Cfg = ConvCfg<CIN, COUT, NT, Q8>;
  constexpr int S = Cfg::STAGES;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* wsm = smem;
  uint8_t* halo = smem + Cfg::WBYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::WBYTES + S * Cfg::HBYTES);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 3);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nt = blockIdx.y;
  const int ntiles = a.total_tiles;
  // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int nmine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(slot, Cfg::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (tid == 0) {
    mbar_expect_tx(&bars[0], Cfg::WBYTES);
    const uint8_t* src = a.wpack + (size_t)nt * Cfg::WBYTES;
    for (int off = 0; off < Cfg::WBYTES; off += 32768) {
      const int n = Cfg::WBYTES - off < 32768 ? Cfg::WBYTES - off : 32768;
      bulk_g2s(wsm + off, src + off, (uint32_t)n, &bars[0]);
    }
  }
  if constexpr (Q8 && Cfg::GR < Cfg::G) {
    // FP8 with 16 input channels: the second plane of every halo buffer is zero
    for (int e = tid; e < S * kPlane / 16; e += blockDim.x)
      *reinterpret_cast<uint4*>(halo + (e / (kPlane / 16)) * Cfg::HBYTES + kPlane + (e % (kPlane / 16)) * 16) =
          make_uint4(0, 0, 0, 0);
  }
  pdl_wait();      // the input tiles come from the previous layer
  pdl_trigger();
  // prefetch the first S-1 halos while the weights arrive
  auto issue = [&](int k) {
    if (k < nmine) {
      const int t = blockIdx.x + k * gridDim.x, im = image_of(a, t);
      if constexpr (Q8)
        load_halo_q8<CIN, MODE>(a.img[im], t - a.img[im].tile_start, halo + (k % S) * Cfg::HBYTES);
      else
        load_halo_async<T, CIN, MODE>(a.img[im], t - a.img[im].tile_start, halo + (k % S) * Cfg::HBYTES);
    }
    cp_async_commit();  // one group per k, possibly empty, keeps the group count uniform
  };
#pragma unroll 1
  for (int k = 0; k < S - 1; ++k) issue(k);
  bool ok = mbar_wait(&bars[0], 0);
  if (!ok) record_error(a.err, 1u);

  // E4M3 has format code 0 in the f8f6f4 descriptor, like FP16 in the f16 one
  constexpr uint32_t idesc = idesc_f16kind(Q8 ? 0u : Half<T>::kFmt, 128, NT);
  uint32_t phase[2] = {0u, 0u};
  // FP8 path: running maximum of this CTA's outputs, published (one atomic per
  // warp) when its tiles move on to another image and once at the end, rather
  // than after every tile: per-tile atomics put thousands of updates per
  // layer on one word
  int run_im = -1;
  float run_mx = 0.f;
  auto amax_track = [&](int im, float v) {
    if (im != run_im) {
      if (run_im >= 0) amax_publish(a.img[run_im].amax_out, run_mx);
      run_im = im;
      run_mx = 0.f;
    }
    run_mx = fmaxf(run_mx, v);
  };
#pragma unroll 1
  for (int k = 0; ok && k < nmine; ++k) {
    const int buf = k % S, acc = k & 1;
    if (k == nmine - 1) pdl_trigger_last();
    cp_async_wait<S - 2>();  // this thread's copies of tile k have landed
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t hb = smem_u32(halo + buf * Cfg::HBYTES), wb = smem_u32(wsm);
      const uint32_t d = tmem + (uint32_t)(acc * NT);
      int kk = 0;
#pragma unroll 1
      for (int tap = 0; tap < 9; ++tap) {
        const uint32_t shift = (uint32_t)(((tap / 3) * kHaloW + tap % 3) * 16);
#pragma unroll
        for (int j = 0; j < Cfg::KS; ++j, ++kk) {
          const uint64_t ad = smem_desc(hb + (uint32_t)(2 * j * kPlane) + shift, kPlane, kHaloW * 16);
          const uint64_t bd = smem_desc(wb + (uint32_t)(kk * NT * 32), NT * 16, 128);
          if constexpr (Q8) mma_f8kind(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
          else mma_f16kind(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
        }
      }
      mma_commit(&bars[1 + acc]);
    }
    if (k > 0) {
      const int pacc = acc ^ 1;
      if (!mbar_wait(&bars[1 + pacc], phase[pacc])) {
        record_error(a.err, 2u);
        ok = false;
        break;
      }
      phase[pacc] ^= 1u;
      tc_fence_after();
      const int t = blockIdx.x + (k - 1) * gridDim.x, im = image_of(a, t);
      const float emx = conv_epilogue<T, NT, Q8>(a.img[im], a.bias, a.wscale, t - a.img[im].tile_start,
                                                 tmem + (uint32_t)(pacc * NT), nt * NT, COUT);
      if constexpr (Q8) amax_track(im, emx);
    }
    // the buffer of tile k-1 is free again (its MMAs completed): refill it
    issue(k + S - 1);
  }
  if (ok && nmine > 0) {
    const int pacc = (nmine - 1) & 1;
    if (!mbar_wait(&bars[1 + pacc], phase[pacc])) {
      record_error(a.err, 2u);
    } else {
      tc_fence_after();
      const int t = blockIdx.x + (nmine - 1) * gridDim.x, im = image_of(a, t);
      const float emx = conv_epilogue<T, NT, Q8>(a.img[im], a.bias, a.wscale, t - a.img[im].tile_start,
                                                 tmem + (uint32_t)(pacc * NT), nt * NT, COUT);
      if constexpr (Q8) amax_track(im, emx);
    }
  }
  if constexpr (Q8) {
    if (run_im >= 0) amax_publish(a.img[run_im].amax_out, run_mx);
  }
  cp_async_wait<0>();
  tc_fence_before();
  __syncthreads();
  pdl_trigger_end();
  if (warp == 0) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// 2x2 stride-2 transposed convolution: M = 128 input pixels (16 x 8 patch),
// N = 4 x COUT ordered [sub-position (a,b)][co], K = CIN.  Output pixel
// (2y+a, 2x+b) channel co = bias + sum_ci W[ci][co][a][b] in(y, x)[ci].
// ---------------------------------------------------------------------------
template <typename T>
struct ConvTImg {
  const T* in;               // NHWC [H][W][CIN]
  T* out;                    // NHWC [2H][2W][COUT]
  int H, W, tiles_x, tile_start;
  const float* amax_in;      // FP8 path: amax words of input and output
  float* amax_out;
};

template <typename T>
struct TcConvTArgs {
  ConvTImg<T> img[kMaxGroup];
  int nimg, total_tiles;
  const uint8_t* wpack;      // [K steps][N rows x 32 bytes]
  const float* bias;         // [COUT]
  const float* wscale;       // FP8 path: per-output-channel weight scales [COUT]
  unsigned int* err;
};

// CTAs that share one input tile of transposed convolution l (0: 128 -> 64
// channels, 1: 64 -> 32, 2: 32 -> 16), each taking N / split of the
// [sub-position][co] columns: the low-resolution layers have few tiles.
#ifndef NSL_UP_SPLIT0
#define NSL_UP_SPLIT0 4
#endif
#ifndef NSL_UP_SPLIT1
#define NSL_UP_SPLIT1 2
#endif
#ifndef NSL_UP_SPLIT2
#define NSL_UP_SPLIT2 1
#endif
constexpr int kUpSplit[3] = {NSL_UP_SPLIT0, NSL_UP_SPLIT1, NSL_UP_SPLIT2};

template <int CIN, int COUT, bool Q8 = false, int NS = 1>
struct ConvTCfg {
  static constexpr int N = 4 * COUT / NS;     // columns of one CTA
  static constexpr int G = Q8 ? CIN / 16 : CIN / 8;     // 16-byte planes (CIN >= 32)
  static constexpr int APLANE = 128 * 16;
  static constexpr int WBYTES = (G / 2) * N * 32;
  static constexpr int ABYTES = G * APLANE;
  static constexpr int TMEM_COLS = 2 * N > 512 ? 512 : (2 * N < 32 ? 32 : 2 * N);
  static constexpr int NBUF = 2 * N > 512 ? 1 : 2;
  static constexpr int SMEM = WBYTES + 2 * ABYTES + 64;
};

template <typename T, int CIN, int COUT, bool Q8, int NS>
__global__ void __launch_bounds__(128) convT_tc_kernel(TcConvTArgs<T> a) {
  using Cfg = ConvTCfg<CIN, COUT, Q8, NS>;
  static_assert((4 * COUT) % NS == 0 && Cfg::N % 16 == 0, "column split");
  static_assert(!Q8 || CIN >= 32, "FP8 transposed convolution needs K >= 32");
  constexpr int N = Cfg::N;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* wsm = smem;
  uint8_t* abuf = smem + Cfg::WBYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::WBYTES + 2 * Cfg::ABYTES);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 3);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ntiles = a.total_tiles;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(slot, Cfg::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    mbar_expect_tx(&bars[0], Cfg::WBYTES);
    // this CTA's column block: the weights are packed block-major
    const uint8_t* wsrc = a.wpack + (size_t)blockIdx.y * Cfg::WBYTES;
    for (int off = 0; off < Cfg::WBYTES; off += 32768) {
      const int n = Cfg::WBYTES - off < 32768 ? Cfg::WBYTES - off : 32768;
      bulk_g2s(wsm + off, wsrc + off, (uint32_t)n, &bars[0]);
    }
  }
  pdl_wait();
  pdl_trigger();
  bool ok = mbar_wait(&bars[0], 0);
  if (!ok) record_error(a.err, 4u);

  constexpr uint32_t idesc = idesc_f16kind(Q8 ? 0u : Half<T>::kFmt, 128, N);
  uint32_t phase[2] = {0u, 0u};
  int buf = 0, prev = -1, prevbuf = 0;
  int run_im = -1;
  float run_mx = 0.f;

  auto epilogue = [&](int gtile, int b) {
    const int imi = image_of(a, gtile);
    const ConvTImg<T>& im = a.img[imi];
    const int tile = gtile - im.tile_start;
    const int ty = tile / im.tiles_x, tx = tile % im.tiles_x;
    const int m = tid;
    const int y = ty * kPatchH + m / kPatchW, x = tx * kPatchW + m % kPatchW;
    const bool valid = y < im.H && x < im.W;
    const uint32_t tacc = tmem + (uint32_t)(b * N) + ((uint32_t)(warp * 32) << 16);
    float deq = 1.f, mx = 0.f;
    if constexpr (Q8) deq = q8_deq(__ldg(im.amax_in));
#pragma unroll 1
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tmem_ld16(tacc + c, v);
      const int n = (int)blockIdx.y * N + c, k = n / COUT, co = n % COUT;
      const int oy = 2 * y + (k >> 1), ox = 2 * x + (k & 1);
      __align__(16) typename Half<T>::T2 h[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float r0, r1;
        if constexpr (Q8) {
          r0 = fmaf(v[2 * q], __fmul_rn(deq, __ldg(a.wscale + co + 2 * q)), __ldg(a.bias + co + 2 * q));
          r1 = fmaf(v[2 * q + 1], __fmul_rn(deq, __ldg(a.wscale + co + 2 * q + 1)),
                    __ldg(a.bias + co + 2 * q + 1));
          mx = fmaxf(mx, fmaxf(fabsf(r0), fabsf(r1)));
        } else {
          r0 = v[2 * q] + __ldg(a.bias + co + 2 * q);
          r1 = v[2 * q + 1] + __ldg(a.bias + co + 2 * q + 1);
        }
        h[q] = Half<T>::pack(r0, r1);
      }
      if (valid) {
        T* dst = im.out + ((size_t)oy * (2 * im.W) + ox) * COUT + co;
        reinterpret_cast<uint4*>(dst)[0] = reinterpret_cast<const uint4*>(h)[0];
        reinterpret_cast<uint4*>(dst)[1] = reinterpret_cast<const uint4*>(h)[1];
      }
    }
    if constexpr (Q8) {
      // running maximum as in the 3x3 layers
      if (imi != run_im) {
        if (run_im >= 0) amax_publish(a.img[run_im].amax_out, run_mx);
        run_im = imi;
        run_mx = 0.f;
      }
      run_mx = fmaxf(run_mx, valid ? __half2float(__float2half_rn(mx)) : 0.f);
    }
  };

  for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
    if (tile + (int)gridDim.x >= ntiles) pdl_trigger_last();
    // stage the 128 input pixels of the patch: plane g holds channels 8g..8g+7
    {
      const int imi = image_of(a, tile);
      const ConvTImg<T>& im = a.img[imi];
      const int lt = tile - im.tile_start;
      const int ty = lt / im.tiles_x, tx = lt % im.tiles_x;
      uint8_t* dstb = abuf + buf * Cfg::ABYTES;
      constexpr int NE = 128 * Cfg::G;
      if constexpr (Q8) {
        // loads in batches issued before their first use (see load_halo)
        const float inv = q8_inv(__ldg(im.amax_in));
        for (int e0 = tid; e0 < NE; e0 += kLdBatch * blockDim.x) {
          uint4 lo[kLdBatch], hi[kLdBatch];
          bool in[kLdBatch];
#pragma unroll
          for (int b = 0; b < kLdBatch; ++b) {
            const int e = min(e0 + b * (int)blockDim.x, NE - 1);
            const int m = e / Cfg::G, g = e % Cfg::G;
            const int y = ty * kPatchH + m / kPatchW, x = tx * kPatchW + m % kPatchW;
            in[b] = y < im.H && x < im.W;
            const T* p = im.in + ((size_t)min(y, im.H - 1) * im.W + min(x, im.W - 1)) * CIN + g * 16;
            lo[b] = ldg128(p);
            hi[b] = ldg128(p + 8);
          }
#pragma unroll
          for (int b = 0; b < kLdBatch; ++b) {
            const int e = e0 + b * (int)blockDim.x;
            if (e < NE)
              *reinterpret_cast<uint4*>(dstb + (e % Cfg::G) * Cfg::APLANE + (e / Cfg::G) * 16) =
                  in[b] ? q8_pack16(lo[b], hi[b], inv) : make_uint4(0, 0, 0, 0);
          }
        }
      } else {
        // asynchronous 16-byte copies, zeros outside the image
        for (int e = tid; e < NE; e += blockDim.x) {
          const int m = e / Cfg::G, g = e % Cfg::G;
          const int y = ty * kPatchH + m / kPatchW, x = tx * kPatchW + m % kPatchW;
          const bool in = y < im.H && x < im.W;
          cp_async16(dstb + g * Cfg::APLANE + m * 16,
                     im.in + ((size_t)(in ? y : 0) * im.W + (in ? x : 0)) * CIN + g * 8, in ? 16u : 0u);
        }
        cp_async_commit();
        cp_async_wait<0>();
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (Cfg::NBUF == 1 && prev >= 0) {
      // single accumulator: drain the previous tile before the next MMAs
      if (!mbar_wait(&bars[1], phase[0])) { record_error(a.err, 8u); ok = false; break; }
      tc_fence_after();
      epilogue(prev, 0);
      phase[0] ^= 1u;
      prev = -1;
      tc_fence_before();
      __syncthreads();
    }
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ab = smem_u32(abuf + buf * Cfg::ABYTES), wb = smem_u32(wsm);
      const uint32_t d = tmem + (uint32_t)((Cfg::NBUF == 2 ? buf : 0) * N);
#pragma unroll
      for (int j = 0; j < Cfg::G / 2; ++j) {
        const uint64_t ad = smem_desc(ab + (uint32_t)(2 * j * Cfg::APLANE), Cfg::APLANE, 128);
        const uint64_t bd = smem_desc(wb + (uint32_t)(j * N * 32), N * 16, 128);
        if constexpr (Q8) mma_f8kind(d, ad, bd, idesc, j > 0 ? 1u : 0u);
        else mma_f16kind(d, ad, bd, idesc, j > 0 ? 1u : 0u);
      }
      mma_commit(&bars[1 + (Cfg::NBUF == 2 ? buf : 0)]);
    }
    if (Cfg::NBUF == 2 && prev >= 0) {
      if (!mbar_wait(&bars[1 + prevbuf], phase[prevbuf])) {
        record_error(a.err, 8u);
        ok = false;
      } else {
        tc_fence_after();
        epilogue(prev, prevbuf);
      }
      phase[prevbuf] ^= 1u;
    }
    prev = tile;
    prevbuf = Cfg::NBUF == 2 ? buf : 0;
    buf ^= 1;
  }
  if (ok && prev >= 0) {
    if (!mbar_wait(&bars[1 + prevbuf], phase[prevbuf])) {
      record_error(a.err, 8u);
    } else {
      tc_fence_after();
      epilogue(prev, prevbuf);
    }
  }
  if constexpr (Q8) {
    if (run_im >= 0) amax_publish(a.img[run_im].amax_out, run_mx);
  }
  tc_fence_before();
  __syncthreads();
  pdl_trigger_end();
  if (warp == 0) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Split-BF16 convolutions (NSL_PREC_BF16X3).  Activations are binary32 NHWC
// between layers; every operand x (activation or weight) is split into a
// bfloat16 high part hi = bf16(x) and the bfloat16 rounding of the remainder
// lo = bf16(x - hi) (x - hi is exact in binary32), and each product is taken
// as hi*hi + hi*lo + lo*hi: three kind::f16 MMAs with BF16 operands into the
// same FP32 accumulator (the lo*lo term, below 2^-16 of the product, is
// dropped).  The input channels are taken in chunks of up to 64 (16 planes:
// 8 of hi parts, 8 of lo parts, 46 KB of halo), so that the 128-channel
// layers fit in shared memory beside their hi + lo weights; a CTA stages a
// chunk, runs its MMAs, waits for them, and stages the next chunk into the
// same buffer.  The weights of all chunks stay in shared memory.
// ---------------------------------------------------------------------------

// 8 binary32 values -> 16 bytes of hi parts and 16 bytes of lo parts (BF16)
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  __align__(16) __nv_bfloat162 h[4], l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    const float2 hf = __bfloat1622float2(h[k]);
    l[k] = __floats2bfloat162_rn(__fsub_rn(v[2 * k], hf.x), __fsub_rn(v[2 * k + 1], hf.y));
  }
  hi = *reinterpret_cast<const uint4*>(h);
  lo = *reinterpret_cast<const uint4*>(l);
}

__device__ __forceinline__ void ldg8f(const float* p, float* v) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// 8 binary32 channels c .. c+7 of halo pixel (y, x) (clamped into the image by
// the caller): PLAIN, CONCAT (channels below CIN/2 from inA, the rest from
// inB) or POOL (the 2x2 maximum of the finer level)
template <int CIN, int MODE>
__device__ __forceinline__ void halo8f(const ConvImg<float>& a, int y, int x, int c, float* v) {
  if constexpr (MODE == TC_PLAIN) {
    ldg8f(a.inA + ((size_t)y * a.W + x) * CIN + c, v);
  } else if constexpr (MODE == TC_CONCAT) {
    constexpr int CH = CIN / 2;
    if (c < CH) ldg8f(a.inA + ((size_t)y * a.W + x) * CH + c, v);
    else ldg8f(a.inB + ((size_t)y * a.W + x) * CH + (c - CH), v);
  } else {
    const size_t W2 = 2 * (size_t)a.W;
    const float* p = a.inA + ((size_t)(2 * y) * W2 + 2 * x) * CIN + c;
    float q[8];
    ldg8f(p, v);
    ldg8f(p + CIN, q);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fmaxf(v[k], q[k]);
    ldg8f(p + W2 * CIN, q);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fmaxf(v[k], q[k]);
    ldg8f(p + W2 * CIN + CIN, q);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fmaxf(v[k], q[k]);
  }
}

// Stage channels [c0, c0 + 8 GC) of the halo of M tile `tile` as GC hi planes
// followed by GC lo planes (zeros outside the image); loads are issued in
// batches before their first use.
#ifndef NSL_SPLIT_LDB
#define NSL_SPLIT_LDB 4
#endif
constexpr int kLdBatchSplit = NSL_SPLIT_LDB;   // 8-channel groups loaded per thread before first use

template <int CIN, int MODE, int GC>
__device__ __forceinline__ void load_halo_split(const ConvImg<float>& a, int tile, int c0, uint8_t* halo) {
  constexpr int NE = kHaloPix * GC;
  constexpr int kLdBatch = kLdBatchSplit;
  const int ty = tile / a.tiles_x, tx = tile % a.tiles_x;
  const int y0 = ty * kPatchH - 1, x0 = tx * kPatchW - 1;
  for (int e0 = threadIdx.x; e0 < NE; e0 += kLdBatch * blockDim.x) {
    float v[kLdBatch][8];
    bool in[kLdBatch];
#pragma unroll
    for (int b = 0; b < kLdBatch; ++b) {
      const int e = min(e0 + b * (int)blockDim.x, NE - 1);
      const int hp = e / GC, g = e % GC;
      const int y = y0 + hp / kHaloW, x = x0 + hp % kHaloW;
      in[b] = y >= 0 && y < a.H && x >= 0 && x < a.W;
      halo8f<CIN, MODE>(a, min(max(y, 0), a.H - 1), min(max(x, 0), a.W - 1), c0 + 8 * g, v[b]);
    }
#pragma unroll
    for (int b = 0; b < kLdBatch; ++b) {
      const int e = e0 + b * (int)blockDim.x;
      if (e < NE) {
        uint4 hi = make_uint4(0, 0, 0, 0), lo = hi;
        if (in[b]) split8(v[b], hi, lo);
        const int hp = e / GC, g = e % GC;
        *reinterpret_cast<uint4*>(halo + g * kPlane + hp * 16) = hi;
        *reinterpret_cast<uint4*>(halo + (GC + g) * kPlane + hp * 16) = lo;
      }
    }
  }
}

// Shared-memory plan of a split 3x3 layer: N tile NT, chunks of CH input
// channels (GC hi planes + GC lo planes), hi and lo weights of every chunk.
template <int CIN, int COUT, int NT>
struct SplitCfg {
  static constexpr int CH = CIN < 64 ? CIN : 64;
  static constexpr int NCH = CIN / CH;
  static constexpr int GC = CH / 8;
  static constexpr int KSC = CH / 16;           // K steps per chunk
  static constexpr int KS = CIN / 16;           // K steps per tap
  static constexpr int WHALF = 9 * KS * NT * 32;
  static constexpr int WBYTES = 2 * WHALF;      // hi weights, then lo weights
  static constexpr int HBYTES = 2 * GC * kPlane;
  // layers of one chunk keep two halo buffers: the next tile is staged while
  // the tensor cores work on this one
  static constexpr int HBUF = NCH == 1 ? 2 : 1;
  // single-chunk layers keep two accumulators: the MMAs of tile t run during
  // the epilogue of tile t - 1 and the staging of tile t + 1
  static constexpr int TMEM_COLS = (NCH == 1 ? 2 * NT : NT) < 32 ? 32 : (NCH == 1 ? 2 * NT : NT);
  static constexpr int SMEM = WBYTES + HBUF * HBYTES + 64;
};
__host__ __device__ constexpr int split_nt(int cout) { return cout > 32 ? 32 : cout; }

// Bias, ReLU and the binary32 NHWC store of one split layer's M tile (thread
// = pixel of the patch, NT accumulator columns from column n0).
template <int NT>
__device__ __forceinline__ void split_epilogue(const ConvImg<float>& a, const float* __restrict__ bias, int tile,
                                               uint32_t tacc, int n0, int cout) {
  const int warp = threadIdx.x >> 5, m = threadIdx.x;
  const int ty = tile / a.tiles_x, tx = tile % a.tiles_x;
  const int y = ty * kPatchH + m / kPatchW, x = tx * kPatchW + m % kPatchW;
  const bool valid = y < a.H && x < a.W;
  float* dst = a.out + ((size_t)y * a.W + x) * cout + n0;
#pragma unroll
  for (int c = 0; c < NT; c += 16) {
    float v[16];
    tmem_ld16(tacc + ((uint32_t)(warp * 32) << 16) + c, v);
    if (valid) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        reinterpret_cast<float4*>(dst + c)[q] =
            make_float4(fmaxf(v[4 * q] + __ldg(bias + n0 + c + 4 * q), 0.f),
                        fmaxf(v[4 * q + 1] + __ldg(bias + n0 + c + 4 * q + 1), 0.f),
                        fmaxf(v[4 * q + 2] + __ldg(bias + n0 + c + 4 * q + 2), 0.f),
                        fmaxf(v[4 * q + 3] + __ldg(bias + n0 + c + 4 * q + 3), 0.f));
    }
  }
}

template <int CIN, int COUT, int NT, int MODE>
__global__ void __launch_bounds__(128) conv3x3_split_kernel(TcConvArgs<float> a) {
  using Cfg = SplitCfg<CIN, COUT, NT>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* wsm = smem;
  uint8_t* halo = smem + Cfg::WBYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::WBYTES + Cfg::HBUF * Cfg::HBYTES);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 3);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nt = blockIdx.y;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(slot, Cfg::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    mbar_expect_tx(&bars[0], Cfg::WBYTES);
    const uint8_t* src = a.wpack + (size_t)nt * Cfg::WBYTES;
    for (int off = 0; off < Cfg::WBYTES; off += 32768) {
      const int n = Cfg::WBYTES - off < 32768 ? Cfg::WBYTES - off : 32768;
      bulk_g2s(wsm + off, src + off, (uint32_t)n, &bars[0]);
    }
  }
  pdl_wait();      // the input tiles come from the previous layer
  pdl_trigger();
  bool ok = mbar_wait(&bars[0], 0);
  if (!ok) record_error(a.err, 0x10u);
  constexpr uint32_t idesc = idesc_f16kind(1u, 128, NT);   // BF16 operands, FP32 accumulation
  uint32_t phase = 0;
  // the MMAs of one chunk on halo buffer hb into the accumulator at column
  // acc, completion signalled on bars[bar]
  auto issue_chunk = [&](uint32_t hb, int kc, uint32_t acc = 0, int bar = 1) {
    const uint32_t wb = smem_u32(wsm);
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const uint32_t shift = (uint32_t)(((tap / 3) * kHaloW + tap % 3) * 16);
#pragma unroll
      for (int j = 0; j < Cfg::KSC; ++j) {
        const int kk = tap * Cfg::KS + kc * Cfg::KSC + j;
        const uint64_t ahi = smem_desc(hb + (uint32_t)(2 * j * kPlane) + shift, kPlane, kHaloW * 16);
        const uint64_t alo = smem_desc(hb + (uint32_t)((Cfg::GC + 2 * j) * kPlane) + shift, kPlane, kHaloW * 16);
        const uint64_t bhi = smem_desc(wb + (uint32_t)(kk * NT * 32), NT * 16, 128);
        const uint64_t blo = smem_desc(wb + (uint32_t)(Cfg::WHALF + kk * NT * 32), NT * 16, 128);
        mma_f16kind(tmem + acc, ahi, bhi, idesc, (kc | tap | j) ? 1u : 0u);
        mma_f16kind(tmem + acc, ahi, blo, idesc, 1u);
        mma_f16kind(tmem + acc, alo, bhi, idesc, 1u);
      }
    }
    mma_commit(&bars[bar]);
  };
  if constexpr (Cfg::NCH == 1) {
    // two halo buffers and two accumulators: while the MMAs of tile t run,
    // the CTA writes out tile t - 1 and stages tile t + grid
    uint32_t ph = 0u;   // bit b: the phase of accumulator b's barrier
    int k = 0, prev = -1;
    int t = blockIdx.x;
    if (ok && t < a.total_tiles) {
      const int im = image_of(a, t);
      load_halo_split<CIN, MODE, Cfg::GC>(a.img[im], t - a.img[im].tile_start, 0, halo);
    }
#pragma unroll 1
    for (; ok && t < a.total_tiles; t += gridDim.x, ++k) {
      if (t + (int)gridDim.x >= a.total_tiles) pdl_trigger_last();
      const int buf = k & 1;
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();   // halo[buf] staged; the epilogue of the tile before last read its accumulator
      if (tid == 0) {
        tc_fence_after();
        issue_chunk(smem_u32(halo + buf * Cfg::HBYTES), 0, (uint32_t)(buf * NT), 1 + buf);
      }
      if (prev >= 0) {
        // tile t - grid: its MMAs completed, so its accumulator can be read and
        // its halo buffer refilled
        if (!mbar_wait(&bars[1 + (buf ^ 1)], (ph >> (buf ^ 1)) & 1u)) {
          record_error(a.err, 0x20u);
          ok = false;
          break;
        }
        ph ^= 1u << (buf ^ 1);
        tc_fence_after();
        const int imp = image_of(a, prev);
        split_epilogue<NT>(a.img[imp], a.bias, prev - a.img[imp].tile_start, tmem + (uint32_t)((buf ^ 1) * NT),
                           nt * NT, COUT);
        tc_fence_before();
      }
      const int tn = t + (int)gridDim.x;
      if (tn < a.total_tiles) {
        const int imn = image_of(a, tn);
        load_halo_split<CIN, MODE, Cfg::GC>(a.img[imn], tn - a.img[imn].tile_start, 0,
                                            halo + (buf ^ 1) * Cfg::HBYTES);
      }
      prev = t;
    }
    if (ok && prev >= 0) {
      const int lb = (k - 1) & 1;
      if (!mbar_wait(&bars[1 + lb], (ph >> lb) & 1u)) {
        record_error(a.err, 0x20u);
      } else {
        tc_fence_after();
        const int imp = image_of(a, prev);
        split_epilogue<NT>(a.img[imp], a.bias, prev - a.img[imp].tile_start, tmem + (uint32_t)(lb * NT), nt * NT,
                           COUT);
      }
    }
  } else {
#pragma unroll 1
  for (int t = blockIdx.x; ok && t < a.total_tiles; t += gridDim.x) {
    if (t + (int)gridDim.x >= a.total_tiles) pdl_trigger_last();
    const int im = image_of(a, t);
    const int lt = t - a.img[im].tile_start;
#pragma unroll 1
    for (int kc = 0; kc < Cfg::NCH; ++kc) {
      __syncthreads();   // every read of the halo buffer by earlier MMAs has completed
      load_halo_split<CIN, MODE, Cfg::GC>(a.img[im], lt, kc * Cfg::CH, halo);
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        issue_chunk(smem_u32(halo), kc);
      }
      if (!mbar_wait(&bars[1], phase)) {
        record_error(a.err, 0x20u);
        ok = false;
        break;
      }
      phase ^= 1u;
      tc_fence_after();
    }
    if (!ok) break;
    split_epilogue<NT>(a.img[im], a.bias, lt, tmem, nt * NT, COUT);
    tc_fence_before();
  }
  }
  tc_fence_before();
  __syncthreads();
  pdl_trigger_end();
  if (warp == 0) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// Split transposed convolution: M = 128 input pixels, N = 4 COUT / NS columns
// [sub-position][co] per CTA, K = CIN in chunks of up to 64 channels.
template <int CIN, int COUT, int NS>
struct SplitTCfg {
  static constexpr int N = 4 * COUT / NS;
  static constexpr int CH = CIN < 64 ? CIN : 64;
  static constexpr int NCH = CIN / CH;
  static constexpr int GC = CH / 8;
  static constexpr int KSC = CH / 16;
  static constexpr int KS = CIN / 16;
  static constexpr int APLANE = 128 * 16;
  static constexpr int WHALF = KS * N * 32;
  static constexpr int WBYTES = 2 * WHALF;
  static constexpr int ABYTES = 2 * GC * APLANE;
  static constexpr int TMEM_COLS = N < 32 ? 32 : N;
  static constexpr int SMEM = WBYTES + ABYTES + 64;
};

template <int CIN, int COUT, int NS>
__global__ void __launch_bounds__(128) convT_split_kernel(TcConvTArgs<float> a) {
  using Cfg = SplitTCfg<CIN, COUT, NS>;
  constexpr int N = Cfg::N;
  static_assert(N % 16 == 0 && COUT % 16 == 0, "column blocks of one sub-position");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* wsm = smem;
  uint8_t* abuf = smem + Cfg::WBYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::WBYTES + Cfg::ABYTES);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(slot, Cfg::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    mbar_expect_tx(&bars[0], Cfg::WBYTES);
    const uint8_t* src = a.wpack + (size_t)blockIdx.y * Cfg::WBYTES;
    for (int off = 0; off < Cfg::WBYTES; off += 32768) {
      const int n = Cfg::WBYTES - off < 32768 ? Cfg::WBYTES - off : 32768;
      bulk_g2s(wsm + off, src + off, (uint32_t)n, &bars[0]);
    }
  }
  pdl_wait();
  pdl_trigger();
  bool ok = mbar_wait(&bars[0], 0);
  if (!ok) record_error(a.err, 0x40u);
  constexpr uint32_t idesc = idesc_f16kind(1u, 128, N);
  uint32_t phase = 0;
#pragma unroll 1
  for (int t = blockIdx.x; ok && t < a.total_tiles; t += gridDim.x) {
    if (t + (int)gridDim.x >= a.total_tiles) pdl_trigger_last();
    const int imi = image_of(a, t);
    const ConvTImg<float>& im = a.img[imi];
    const int lt = t - im.tile_start;
    const int ty = lt / im.tiles_x, tx = lt % im.tiles_x;
#pragma unroll 1
    for (int kc = 0; kc < Cfg::NCH; ++kc) {
      __syncthreads();   // every read of the A buffer by earlier MMAs has completed
      constexpr int NE = 128 * Cfg::GC;
      for (int e0 = tid; e0 < NE; e0 += kLdBatch * blockDim.x) {
        float v[kLdBatch][8];
        bool in[kLdBatch];
#pragma unroll
        for (int b = 0; b < kLdBatch; ++b) {
          const int e = min(e0 + b * (int)blockDim.x, NE - 1);
          const int m = e / Cfg::GC, g = e % Cfg::GC;
          const int y = ty * kPatchH + m / kPatchW, x = tx * kPatchW + m % kPatchW;
          in[b] = y < im.H && x < im.W;
          ldg8f(im.in + ((size_t)min(y, im.H - 1) * im.W + min(x, im.W - 1)) * CIN + kc * Cfg::CH + 8 * g, v[b]);
        }
#pragma unroll
        for (int b = 0; b < kLdBatch; ++b) {
          const int e = e0 + b * (int)blockDim.x;
          if (e < NE) {
            uint4 hi = make_uint4(0, 0, 0, 0), lo = hi;
            if (in[b]) split8(v[b], hi, lo);
            const int m = e / Cfg::GC, g = e % Cfg::GC;
            *reinterpret_cast<uint4*>(abuf + g * Cfg::APLANE + m * 16) = hi;
            *reinterpret_cast<uint4*>(abuf + (Cfg::GC + g) * Cfg::APLANE + m * 16) = lo;
          }
        }
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t ab = smem_u32(abuf), wb = smem_u32(wsm);
#pragma unroll
        for (int j = 0; j < Cfg::KSC; ++j) {
          const int kk = kc * Cfg::KSC + j;
          const uint64_t ahi = smem_desc(ab + (uint32_t)(2 * j * Cfg::APLANE), Cfg::APLANE, 128);
          const uint64_t alo = smem_desc(ab + (uint32_t)((Cfg::GC + 2 * j) * Cfg::APLANE), Cfg::APLANE, 128);
          const uint64_t bhi = smem_desc(wb + (uint32_t)(kk * N * 32), N * 16, 128);
          const uint64_t blo = smem_desc(wb + (uint32_t)(Cfg::WHALF + kk * N * 32), N * 16, 128);
          mma_f16kind(tmem, ahi, bhi, idesc, (kc | j) ? 1u : 0u);
          mma_f16kind(tmem, ahi, blo, idesc, 1u);
          mma_f16kind(tmem, alo, bhi, idesc, 1u);
        }
        mma_commit(&bars[1]);
      }
      if (!mbar_wait(&bars[1], phase)) {
        record_error(a.err, 0x80u);
        ok = false;
        break;
      }
      phase ^= 1u;
      tc_fence_after();
    }
    if (!ok) break;
    // bias and the binary32 store of the four output pixels each input pixel feeds
    const int m = tid;
    const int y = ty * kPatchH + m / kPatchW, x = tx * kPatchW + m % kPatchW;
    const bool valid = y < im.H && x < im.W;
#pragma unroll 1
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
      const int n = (int)blockIdx.y * N + c, k = n / COUT, co = n % COUT;
      const int oy = 2 * y + (k >> 1), ox = 2 * x + (k & 1);
      if (valid) {
        float* dst = im.out + ((size_t)oy * (2 * im.W) + ox) * COUT + co;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          reinterpret_cast<float4*>(dst)[q] =
              make_float4(v[4 * q] + __ldg(a.bias + co + 4 * q), v[4 * q + 1] + __ldg(a.bias + co + 4 * q + 1),
                          v[4 * q + 2] + __ldg(a.bias + co + 4 * q + 2), v[4 * q + 3] + __ldg(a.bias + co + 4 * q + 3));
      }
    }
    tc_fence_before();
  }
  tc_fence_before();
  __syncthreads();
  pdl_trigger_end();
  if (warp == 0) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// Failure-detection probe: one warp waits, with the same bounded wait as every
// tensor-core kernel, on an mbarrier that nothing arrives at; the wait gives up
// after its limit (about 2 s), records code 0x8000 in the error word and the
// kernel returns normally.
__global__ void __launch_bounds__(32) wait_timeout_probe(unsigned int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (!mbar_wait(&bar, 0) && threadIdx.x == 0) record_error(err, 0x8000u);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

}  // namespace

cudaError_t launch_wait_timeout_probe(unsigned int* err, cudaStream_t s) {
  wait_timeout_probe<<<1, 32, 0, s>>>(err);
  return cudaGetLastError();
}

// CTAs of a kernel that fit on one SM at once, from its shared memory,
// registers, threads and TMEM columns.  (The runtime's occupancy query reports
// one CTA per SM for every kernel that allocates tensor memory, whatever its
// resources, so it cannot size these grids.)
int tc_ctas_per_sm(const void* kernel, int threads, int dyn_smem, int tmem_cols) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 1;
  const int by_smem = 233472 / (dyn_smem + (int)fa.sharedSizeBytes + 1024);
  const int warps = (threads + 31) / 32;
  const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  const int by_regs = regs_per_warp > 0 ? 65536 / (regs_per_warp * warps) : 32;
  const int by_threads = 2048 / threads;
  const int by_tmem = tmem_cols > 0 ? 512 / tmem_cols : 32;
  int n = by_smem;
  if (by_regs < n) n = by_regs;
  if (by_threads < n) n = by_threads;
  if (by_tmem < n) n = by_tmem;
  if (n > 32) n = 32;
  return n < 1 ? 1 : n;
}

namespace {

// Kernel launch configuration: persistent grid of (CTAs per SM) x SMs, where
// the CTAs per SM are limited so that their TMEM allocations fit in 512 columns.
struct Launch {
  int smem = 0;
  int per_sm = 1;
};

template <typename K>
static cudaError_t configure(K kernel, int smem_needed, int tmem_cols, Launch* L) {
  const int tmem_fit = 512 / tmem_cols;
  int smem = smem_needed;
  // shared memory per SM is 228 KB (1 KB reserved per CTA): pad the request so
  // that no more CTAs than the TMEM can hold become resident at once
  const int cap = 233472 / (tmem_fit + 1) - 1024 + 128;
  if (tmem_fit < 16 && smem < cap) smem = cap;
  smem = (smem + 127) / 128 * 128;
  if (smem > 232448) smem = 232448;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  // prefer the largest shared-memory carveout, so that several CTAs fit per SM
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  L->smem = smem;
  L->per_sm = tc_ctas_per_sm(reinterpret_cast<const void*>(kernel), 128, smem, tmem_cols);
  return cudaSuccess;
}

// A kernel's launch configuration, computed once per process: held in a
// function-local static, whose initialisation is thread-safe (concurrent
// first calls wait for it).  A failed configuration is returned again on
// every call.
struct LaunchOnce {
  cudaError_t err = cudaSuccess;
  Launch L;
};
template <typename K>
static LaunchOnce configure_once(K kernel, int smem_needed, int tmem_cols) {
  LaunchOnce o;
  o.err = configure(kernel, smem_needed, tmem_cols, &o.L);
  return o;
}

// Pack a 3x3 conv weight [cout][cin][3][3] (float) into the B-operand tiles.
template <typename T>
static void pack_conv(const float* w, int cin, int cout, int NT, std::vector<uint8_t>& out) {
  const int KS = cin / 16;
  const size_t slice = (size_t)NT * 32;
  out.assign((size_t)(cout / NT) * 9 * KS * slice, 0);
  for (int nt = 0; nt < cout / NT; ++nt)
    for (int tap = 0; tap < 9; ++tap)
      for (int j = 0; j < KS; ++j) {
        uint8_t* s = out.data() + (((size_t)nt * 9 + tap) * KS + j) * slice;
        for (int n = 0; n < NT; ++n)
          for (int k = 0; k < 16; ++k) {
            const int co = nt * NT + n, ci = j * 16 + k;
            const float v = w[((size_t)co * cin + ci) * 9 + tap];
            T b = Half<T>::from(v);
            const size_t off = (size_t)(k / 8) * NT * 16 + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
            std::memcpy(s + off, &b, 2);
          }
      }
}

// Pack a transposed-conv weight [cin][cout][2][2] into B tiles with rows
// n = (2a+b)*cout + co and K = cin.
// The columns are cut into ns blocks of N / ns (one per CTA of a tile), each
// block stored whole: [block][K step][N/ns rows x 32 bytes].
template <typename T>
static void pack_convT(const float* w, int cin, int cout, int ns, std::vector<uint8_t>& out) {
  const int N = 4 * cout, Nb = N / ns, KS = cin / 16;
  const size_t slice = (size_t)Nb * 32;
  out.assign((size_t)ns * KS * slice, 0);
  for (int sb = 0; sb < ns; ++sb)
    for (int j = 0; j < KS; ++j) {
      uint8_t* s = out.data() + ((size_t)sb * KS + j) * slice;
      for (int r = 0; r < Nb; ++r)
        for (int k = 0; k < 16; ++k) {
          const int n = sb * Nb + r, kpos = n / cout, co = n % cout, ci = j * 16 + k;
          const float v = w[((size_t)ci * cout + co) * 4 + kpos];
          T b = Half<T>::from(v);
          const size_t off = (size_t)(k / 8) * Nb * 16 + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
          std::memcpy(s + off, &b, 2);
        }
    }
}

// Nearest-even E4M3 code of a float with saturation to the largest finite
// magnitude (448): exponent bias 7, 3 fraction bits, subnormal quantum 2^-9,
// S.1111.111 reserved for NaN.
static uint8_t e4m3_code(float v) {
  const uint8_t sign = std::signbit(v) ? 0x80 : 0x00;
  const double a = std::fabs((double)v);
  if (a == 0.0) return sign;
  int e;
  std::frexp(a, &e);
  int E = e - 1;                                  // a in [2^E, 2^(E+1))
  if (E < -6) E = -6;
  double r = std::nearbyint(a / std::ldexp(1.0, E - 3));  // in [0, 16]
  if (r >= 16.0) { r = 8.0; ++E; }
  int field, mant;
  if (r < 8.0) { field = 0; mant = (int)r; }      // subnormal (only when E = -6)
  else { field = E + 7; mant = (int)r - 8; }
  if (field > 15 || (field == 15 && mant == 7)) { field = 15; mant = 6; }  // saturate at 448
  return (uint8_t)(sign | (field << 3) | mant);
}

// Per-output-channel scale (max |w| / 448 in binary32; 1 for an all-zero
// channel) and the codes of w / scale.
static float channel_scale(const float* w, int count, long stride) {
  float amax = 0.f;
  for (int j = 0; j < count; ++j) amax = std::fmax(amax, std::fabs(w[(long)j * stride]));
  return amax > 0.f ? amax / 448.0f : 1.0f;
}

// FP8 packing of a 3x3 conv weight [cout][cin][3][3]: per (N tile, tap, K step
// of 32 channels) a slice of NT rows x 32 bytes, K core matrix k/16 at
// NT*16 bytes, rows grouped by 8 (128 bytes); channels >= cin are zero.
static void pack_conv_q8(const float* w, int cin, int cout, int NT, std::vector<uint8_t>& out,
                         std::vector<float>& scale) {
  const int KS = cin < 32 ? 1 : cin / 32;
  const size_t slice = (size_t)NT * 32;
  out.assign((size_t)(cout / NT) * 9 * KS * slice, 0);
  scale.resize(cout);
  for (int co = 0; co < cout; ++co) scale[co] = channel_scale(w + (size_t)co * cin * 9, cin * 9, 1);
  for (int nt = 0; nt < cout / NT; ++nt)
    for (int tap = 0; tap < 9; ++tap)
      for (int j = 0; j < KS; ++j) {
        uint8_t* s = out.data() + (((size_t)nt * 9 + tap) * KS + j) * slice;
        for (int n = 0; n < NT; ++n)
          for (int k = 0; k < 32; ++k) {
            const int co = nt * NT + n, ci = j * 32 + k;
            if (ci >= cin) continue;
            const float v = w[((size_t)co * cin + ci) * 9 + tap] / scale[co];
            s[(size_t)(k / 16) * NT * 16 + (n / 8) * 128 + (n % 8) * 16 + (k % 16)] = e4m3_code(v);
          }
      }
}

// FP8 packing of a transposed-conv weight [cin][cout][2][2]: rows
// n = (2a+b)*cout + co, K = cin in steps of 32; scale per output channel over
// ci and the four kernel positions.
static void pack_convT_q8(const float* w, int cin, int cout, int ns, std::vector<uint8_t>& out,
                          std::vector<float>& scale) {
  const int N = 4 * cout, Nb = N / ns, KS = cin / 32;
  const size_t slice = (size_t)Nb * 32;
  out.assign((size_t)ns * KS * slice, 0);
  scale.resize(cout);
  for (int co = 0; co < cout; ++co) {
    float amax = 0.f;
    for (int ci = 0; ci < cin; ++ci)
      for (int k = 0; k < 4; ++k) amax = std::fmax(amax, std::fabs(w[((size_t)ci * cout + co) * 4 + k]));
    scale[co] = amax > 0.f ? amax / 448.0f : 1.0f;
  }
  for (int sb = 0; sb < ns; ++sb)
    for (int j = 0; j < KS; ++j) {
      uint8_t* s = out.data() + ((size_t)sb * KS + j) * slice;
      for (int r = 0; r < Nb; ++r)
        for (int k = 0; k < 32; ++k) {
          const int n = sb * Nb + r, kpos = n / cout, co = n % cout, ci = j * 32 + k;
          const float v = w[((size_t)ci * cout + co) * 4 + kpos] / scale[co];
          s[(size_t)(k / 16) * Nb * 16 + (r / 8) * 128 + (r % 8) * 16 + (k % 16)] = e4m3_code(v);
        }
    }
}

}  // namespace

struct NetTcWeights {
  int elem = 0;              // 0 FP16 operands, 1 BF16 operands, 2 FP8 E4M3 operands,
                             // 3 split BF16 (hi and lo parts of both operands)
  uint8_t* conv_w[14] = {};  // layer 0 stays on the SIMT path
  float* conv_b[14] = {};
  float* conv_s[14] = {};    // FP8: per-output-channel weight scales
  int conv_nt[14] = {};
  uint8_t* up_w[3] = {};
  float* up_b[3] = {};
  float* up_s[3] = {};
  AdapterTcWeights* ad = nullptr;   // tensor-core adapters
  std::vector<void*> allocs;
};

template <typename V>
static V* dev_copy(NetTcWeights* w, const V* src, size_t n, cudaError_t* err) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, n * sizeof(V));
  if (e != cudaSuccess) { *err = e; return nullptr; }
  w->allocs.push_back(p);
  e = cudaMemcpy(p, src, n * sizeof(V), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) *err = e;
  return static_cast<V*>(p);
}

template <typename T>
static void fill_weights(NetTcWeights* w, const float* hp, const NetLayout& L, cudaError_t* err) {
  std::vector<uint8_t> pk;
  for (int l = 1; l < 14; ++l) {
    const int cin = L.conv_cin[l], cout = L.conv_cout[l];
    const int NT = conv_nt(cin, cout);
    w->conv_nt[l] = NT;
    pack_conv<T>(hp + L.conv_w[l], cin, cout, NT, pk);
    w->conv_w[l] = dev_copy(w, pk.data(), pk.size(), err);
    w->conv_b[l] = dev_copy(w, hp + L.conv_b[l], (size_t)cout, err);
  }
  for (int l = 0; l < 3; ++l) {
    pack_convT<T>(hp + L.up_w[l], L.up_cin[l], L.up_cout[l], kUpSplit[l], pk);
    w->up_w[l] = dev_copy(w, pk.data(), pk.size(), err);
    w->up_b[l] = dev_copy(w, hp + L.up_b[l], (size_t)L.up_cout[l], err);
  }
}

static void fill_weights_q8(NetTcWeights* w, const float* hp, const NetLayout& L, cudaError_t* err) {
  std::vector<uint8_t> pk;
  std::vector<float> sc;
  for (int l = 1; l < 14; ++l) {
    const int cin = L.conv_cin[l], cout = L.conv_cout[l];
    const int NT = conv_nt(cin, cout);
    w->conv_nt[l] = NT;
    pack_conv_q8(hp + L.conv_w[l], cin, cout, NT, pk, sc);
    w->conv_w[l] = dev_copy(w, pk.data(), pk.size(), err);
    w->conv_s[l] = dev_copy(w, sc.data(), sc.size(), err);
    w->conv_b[l] = dev_copy(w, hp + L.conv_b[l], (size_t)cout, err);
  }
  for (int l = 0; l < 3; ++l) {
    pack_convT_q8(hp + L.up_w[l], L.up_cin[l], L.up_cout[l], kUpSplit[l], pk, sc);
    w->up_w[l] = dev_copy(w, pk.data(), pk.size(), err);
    w->up_s[l] = dev_copy(w, sc.data(), sc.size(), err);
    w->up_b[l] = dev_copy(w, hp + L.up_b[l], (size_t)L.up_cout[l], err);
  }
}

// Split-BF16 weights: the high part bf16(w) and the low part bf16(w - hi) of
// every weight (w - hi is exact in binary32), each packed as pack_conv /
// pack_convT pack a 16-bit operand; per N tile (per column block of a
// transposed convolution) the hi block, then the lo block.
static void split_bf16(float v, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  *hi = __float2bfloat16_rn(v);
  *lo = __float2bfloat16_rn(v - __bfloat162float(*hi));
}

static void pack_conv_split(const float* w, int cin, int cout, int NT, std::vector<uint8_t>& out) {
  const int KS = cin / 16;
  const size_t slice = (size_t)NT * 32, half = 9 * (size_t)KS * slice;
  out.assign((size_t)(cout / NT) * 2 * half, 0);
  for (int nt = 0; nt < cout / NT; ++nt)
    for (int tap = 0; tap < 9; ++tap)
      for (int j = 0; j < KS; ++j) {
        uint8_t* s = out.data() + (size_t)nt * 2 * half + ((size_t)tap * KS + j) * slice;
        for (int n = 0; n < NT; ++n)
          for (int k = 0; k < 16; ++k) {
            const int co = nt * NT + n, ci = j * 16 + k;
            __nv_bfloat16 hi, lo;
            split_bf16(w[((size_t)co * cin + ci) * 9 + tap], &hi, &lo);
            const size_t off = (size_t)(k / 8) * NT * 16 + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
            std::memcpy(s + off, &hi, 2);
            std::memcpy(s + half + off, &lo, 2);
          }
      }
}

static void pack_convT_split(const float* w, int cin, int cout, int ns, std::vector<uint8_t>& out) {
  const int N = 4 * cout, Nb = N / ns, KS = cin / 16;
  const size_t slice = (size_t)Nb * 32, half = (size_t)KS * slice;
  out.assign((size_t)ns * 2 * half, 0);
  for (int sb = 0; sb < ns; ++sb)
    for (int j = 0; j < KS; ++j) {
      uint8_t* s = out.data() + (size_t)sb * 2 * half + (size_t)j * slice;
      for (int r = 0; r < Nb; ++r)
        for (int k = 0; k < 16; ++k) {
          const int n = sb * Nb + r, kpos = n / cout, co = n % cout, ci = j * 16 + k;
          __nv_bfloat16 hi, lo;
          split_bf16(w[((size_t)ci * cout + co) * 4 + kpos], &hi, &lo);
          const size_t off = (size_t)(k / 8) * Nb * 16 + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
          std::memcpy(s + off, &hi, 2);
          std::memcpy(s + half + off, &lo, 2);
        }
    }
}

static void fill_weights_split(NetTcWeights* w, const float* hp, const NetLayout& L, cudaError_t* err) {
  std::vector<uint8_t> pk;
  for (int l = 1; l < 14; ++l) {
    const int cin = L.conv_cin[l], cout = L.conv_cout[l];
    const int NT = split_nt(cout);
    w->conv_nt[l] = NT;
    pack_conv_split(hp + L.conv_w[l], cin, cout, NT, pk);
    w->conv_w[l] = dev_copy(w, pk.data(), pk.size(), err);
    w->conv_b[l] = dev_copy(w, hp + L.conv_b[l], (size_t)cout, err);
  }
  for (int l = 0; l < 3; ++l) {
    pack_convT_split(hp + L.up_w[l], L.up_cin[l], L.up_cout[l], kUpSplit[l], pk);
    w->up_w[l] = dev_copy(w, pk.data(), pk.size(), err);
    w->up_b[l] = dev_copy(w, hp + L.up_b[l], (size_t)L.up_cout[l], err);
  }
}

NetTcWeights* net_tc_create(const float* hp, const NetLayout& L, int elem, cudaError_t* err) {
  *err = cudaSuccess;
  NetTcWeights* w = new NetTcWeights();
  w->elem = elem;
  if (elem == 3) fill_weights_split(w, hp, L, err);
  else if (elem == 2) fill_weights_q8(w, hp, L, err);
  else if (elem == 1) fill_weights<__nv_bfloat16>(w, hp, L, err);
  else fill_weights<__half>(w, hp, L, err);
  if (*err == cudaSuccess) {
    AdapterParamSet* prm = new AdapterParamSet();
    adapter_params_from(hp + L.adapter[0], &prm->p1, &prm->sca, &prm->p2);
    w->ad = adapters_tc_create(*prm, err);
    delete prm;
  }
  if (*err != cudaSuccess) { net_tc_destroy(w); return nullptr; }
  return w;
}

void net_tc_destroy(NetTcWeights* w) {
  if (!w) return;
  for (void* p : w->allocs) cudaFree(p);
  adapters_tc_destroy(w->ad);
  delete w;
}

namespace {
template <typename T>
struct TcBuffers {
  T *fa, *fb, *s1, *l1a, *l1b, *s2, *l2a, *l2b, *s3, *l3a, *l3b, *x1;
  float *partial, *att;
  float* amax;               // FP8 path: [kMaxGroup][kAmaxSlots] tensor maxima (first image's region)
};
constexpr int kAmaxSlots = 32;

template <typename T>
size_t carve_tc(size_t P, size_t partial_floats, TcBuffers<T>* b, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return p;
  };
  auto hf = [&](size_t n) { return reinterpret_cast<T*>(take(n * sizeof(T))); };
  b->fa = hf(P * 16); b->fb = hf(P * 16); b->s1 = hf(P * 16);
  b->l1a = hf(P / 4 * 32); b->l1b = hf(P / 4 * 32); b->s2 = hf(P / 4 * 32);
  b->l2a = hf(P / 16 * 64); b->l2b = hf(P / 16 * 64); b->s3 = hf(P / 16 * 64);
  b->l3a = hf(P / 64 * 128); b->l3b = hf(P / 64 * 128);
  b->x1 = hf(P * 64);
  b->partial = reinterpret_cast<float*>(take(partial_floats * 4));
  b->att = reinterpret_cast<float*>(take(64 * 4));
  b->amax = reinterpret_cast<float*>(take((size_t)kMaxGroup * kAmaxSlots * 4));
  return off;
}

int g_conv_ctas_per_sm = kConvCtasPerSM;

// One grouped layer launch: `ins`, `skips`, `outs` hold each image's buffers,
// `H`, `W` each image's convolution size.
// FP8 tensor-maximum slots (per image): 0 = first conv output, l = conv l
// output (1..13), 14 + j = transposed conv j output.
struct AmaxSlots {
  float* base = nullptr;     // [n][kAmaxSlots], null outside the FP8 path
  int a = -1, b = -1, out = -1;
};

template <typename T, int CIN, int COUT, int MODE, bool Q8>
cudaError_t run_conv(const NetTcWeights* w, int l, int n, const T* const* ins, const T* const* skips,
                     T* const* outs, const int* H, const int* W, AmaxSlots am, unsigned int* err,
                     cudaStream_t s) {
  constexpr int NT = conv_nt(CIN, COUT);
  using Cfg = ConvCfg<CIN, COUT, NT, Q8>;
  static_assert(Cfg::SMEM <= 232448, "shared memory budget");
  static const LaunchOnce once =
      configure_once(conv3x3_tc_kernel<T, CIN, COUT, NT, MODE, Q8>, Cfg::SMEM, Cfg::TMEM_COLS);
  if (once.err != cudaSuccess) return once.err;
  const Launch& L = once.L;
  TcConvArgs<T> a{};
  a.nimg = n;
  int ntiles = 0;
  for (int k = 0; k < n; ++k) {
    const int tx = (W[k] + kPatchW - 1) / kPatchW, ty = (H[k] + kPatchH - 1) / kPatchH;
    float* ab = am.base ? am.base + (size_t)k * kAmaxSlots : nullptr;
    a.img[k] = ConvImg<T>{ins[k], skips ? skips[k] : nullptr, outs[k], H[k], W[k], tx, ntiles,
                          ab ? ab + am.a : nullptr, (ab && am.b >= 0) ? ab + am.b : nullptr,
                          ab ? ab + am.out : nullptr};
    ntiles += tx * ty;
  }
  a.total_tiles = ntiles;
  a.wpack = w->conv_w[l];
  a.bias = w->conv_b[l];
  a.wscale = w->conv_s[l];
  a.err = err;
  // enough CTAs to cover every SM, each pipelining >= NSL_CONV_MIN_TILES tiles
  // when there are that many; per-SM residency is capped by the tunable
  // CTAs-per-SM
  const int per_sm = L.per_sm < g_conv_ctas_per_sm ? L.per_sm : g_conv_ctas_per_sm;
  int grid = num_sms() * per_sm / (COUT / NT);
  if (grid > (ntiles + NSL_CONV_MIN_TILES - 1) / NSL_CONV_MIN_TILES)
    grid = (ntiles + NSL_CONV_MIN_TILES - 1) / NSL_CONV_MIN_TILES;
  if (grid < num_sms() / (COUT / NT)) grid = num_sms() / (COUT / NT);
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  return launch_pdl(conv3x3_tc_kernel<T, CIN, COUT, NT, MODE, Q8>, dim3(grid, COUT / NT), dim3(128),
                    (size_t)L.smem, s, a);
}

template <typename T, int CIN, int COUT, bool Q8, int LAYER>
cudaError_t run_convT(const NetTcWeights* w, int n, const T* const* ins, T* const* outs,
                      const int* H, const int* W, AmaxSlots am, unsigned int* err, cudaStream_t s) {
  constexpr int NS = kUpSplit[LAYER];
  using Cfg = ConvTCfg<CIN, COUT, Q8, NS>;
  static const LaunchOnce once = configure_once(convT_tc_kernel<T, CIN, COUT, Q8, NS>, Cfg::SMEM, Cfg::TMEM_COLS);
  if (once.err != cudaSuccess) return once.err;
  const Launch& L = once.L;
  TcConvTArgs<T> a{};
  a.nimg = n;
  int ntiles = 0;
  for (int k = 0; k < n; ++k) {
    const int tx = (W[k] + kPatchW - 1) / kPatchW, ty = (H[k] + kPatchH - 1) / kPatchH;
    float* ab = am.base ? am.base + (size_t)k * kAmaxSlots : nullptr;
    a.img[k] = ConvTImg<T>{ins[k], outs[k], H[k], W[k], tx, ntiles, ab ? ab + am.a : nullptr,
                           ab ? ab + am.out : nullptr};
    ntiles += tx * ty;
  }
  a.total_tiles = ntiles;
  a.wpack = w->up_w[LAYER];
  a.bias = w->up_b[LAYER];
  a.wscale = w->up_s[LAYER];
  a.err = err;
  int grid = (num_sms() * L.per_sm + NS - 1) / NS;
  if (grid > ntiles) grid = ntiles;
  return launch_pdl(convT_tc_kernel<T, CIN, COUT, Q8, NS>, dim3(grid, NS), dim3(128), (size_t)L.smem, s, a);
}

template <int CIN, int COUT, int MODE>
cudaError_t run_conv_split(const NetTcWeights* w, int l, int n, const float* const* ins, const float* const* skips,
                           float* const* outs, const int* H, const int* W, unsigned int* err, cudaStream_t s) {
  constexpr int NT = split_nt(COUT);
  using Cfg = SplitCfg<CIN, COUT, NT>;
  static_assert(Cfg::SMEM <= 232448, "shared memory budget");
  static const LaunchOnce once =
      configure_once(conv3x3_split_kernel<CIN, COUT, NT, MODE>, Cfg::SMEM, Cfg::TMEM_COLS);
  if (once.err != cudaSuccess) return once.err;
  const Launch& L = once.L;
  TcConvArgs<float> a{};
  a.nimg = n;
  int ntiles = 0;
  for (int k = 0; k < n; ++k) {
    const int tx = (W[k] + kPatchW - 1) / kPatchW, ty = (H[k] + kPatchH - 1) / kPatchH;
    a.img[k] = ConvImg<float>{ins[k], skips ? skips[k] : nullptr, outs[k], H[k], W[k], tx, ntiles,
                              nullptr, nullptr, nullptr};
    ntiles += tx * ty;
  }
  a.total_tiles = ntiles;
  a.wpack = w->conv_w[l];
  a.bias = w->conv_b[l];
  a.err = err;
#ifndef NSL_SPLIT_CTAS
#define NSL_SPLIT_CTAS 8   // CTAs per SM (4: 0.374 ms, 8: 0.368 ms for the 512^2 network)
#endif
  const int per_sm = L.per_sm < NSL_SPLIT_CTAS ? L.per_sm : NSL_SPLIT_CTAS;
  int grid = num_sms() * per_sm / (COUT / NT);
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  return launch_pdl(conv3x3_split_kernel<CIN, COUT, NT, MODE>, dim3(grid, COUT / NT), dim3(128), (size_t)L.smem, s,
                    a);
}

template <int CIN, int COUT, int LAYER>
cudaError_t run_convT_split(const NetTcWeights* w, int n, const float* const* ins, float* const* outs, const int* H,
                            const int* W, unsigned int* err, cudaStream_t s) {
  constexpr int NS = kUpSplit[LAYER];
  using Cfg = SplitTCfg<CIN, COUT, NS>;
  static_assert(Cfg::SMEM <= 232448, "shared memory budget");
  static const LaunchOnce once = configure_once(convT_split_kernel<CIN, COUT, NS>, Cfg::SMEM, Cfg::TMEM_COLS);
  if (once.err != cudaSuccess) return once.err;
  const Launch& L = once.L;
  TcConvTArgs<float> a{};
  a.nimg = n;
  int ntiles = 0;
  for (int k = 0; k < n; ++k) {
    const int tx = (W[k] + kPatchW - 1) / kPatchW, ty = (H[k] + kPatchH - 1) / kPatchH;
    a.img[k] = ConvTImg<float>{ins[k], outs[k], H[k], W[k], tx, ntiles, nullptr, nullptr};
    ntiles += tx * ty;
  }
  a.total_tiles = ntiles;
  a.wpack = w->up_w[LAYER];
  a.bias = w->up_b[LAYER];
  a.err = err;
  int grid = (num_sms() * L.per_sm + NS - 1) / NS;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  return launch_pdl(convT_split_kernel<CIN, COUT, NS>, dim3(grid, NS), dim3(128), (size_t)L.smem, s, a);
}

// The split-BF16 network: the first convolution on the SIMT cores (binary32
// output), the 16 tensor-core convolutions in the split form on binary32
// activations, then the tensor-core adapters (binary16 operands, as in the
// other tensor-core networks) on the binary32 feature map.
cudaError_t forward_split(const NetTcWeights* w, const NetF32Weights* wf, const NetImage* imgs, void* const* ws,
                          int n, unsigned int* err, cudaStream_t s, uint8_t* trace = nullptr) {
  if (n < 1 || n > kMaxGroup || (trace && n != 1)) return cudaErrorInvalidValue;
  TcBuffers<float> B[kMaxGroup];
  int Hs[4][kMaxGroup], Ws[4][kMaxGroup];
  for (int k = 0; k < n; ++k) {
    const size_t P = (size_t)imgs[k].H * imgs[k].W;
    carve_tc(P, adapter_partial_floats(imgs[k].W, imgs[k].H), &B[k], static_cast<char*>(ws[k]));
    for (int lv = 0; lv < 4; ++lv) {
      Hs[lv][k] = imgs[k].H >> lv;
      Ws[lv][k] = imgs[k].W >> lv;
    }
  }
  const float* in[kMaxGroup];
  const float* sk[kMaxGroup];
  float* out[kMaxGroup];
  cudaError_t e;
  // diagnostic trace (one image): after each layer, a copy of its binary32 output
  const size_t P0 = (size_t)imgs[0].H * imgs[0].W;
  size_t toff = 0;
  auto trace_copy = [&](const float* buf, int ch, int lv) -> cudaError_t {
    if (!trace) return cudaSuccess;
    const size_t bytes = (P0 >> (2 * lv)) * (size_t)ch * sizeof(float);
    cudaError_t ce = cudaMemcpyAsync(trace + toff, buf, bytes, cudaMemcpyDeviceToDevice, s);
    toff += bytes;
    return ce;
  };
#define TRY(x) if ((e = (x)) != cudaSuccess) return e
#define SET(IN, SKIP, OUT) for (int k = 0; k < n; ++k) { in[k] = B[k].IN; sk[k] = SKIP; out[k] = B[k].OUT; }
#define TRACE(BUF, CH, LV) TRY(trace_copy(B[0].BUF, CH, LV))
  for (int k = 0; k < n; ++k) out[k] = B[k].fa;
  TRY(simt_first_conv_group<float>(wf, imgs, out, nullptr, n, s));
  TRACE(fa, 16, 0);
  SET(fa, nullptr, s1);  TRY((run_conv_split<16, 16, TC_PLAIN>(w, 1, n, in, nullptr, out, Hs[0], Ws[0], err, s)));
  TRACE(s1, 16, 0);
  SET(s1, nullptr, l1a); TRY((run_conv_split<16, 32, TC_POOL>(w, 2, n, in, nullptr, out, Hs[1], Ws[1], err, s)));
  TRACE(l1a, 32, 1);
  SET(l1a, nullptr, s2); TRY((run_conv_split<32, 32, TC_PLAIN>(w, 3, n, in, nullptr, out, Hs[1], Ws[1], err, s)));
  TRACE(s2, 32, 1);
  SET(s2, nullptr, l2a); TRY((run_conv_split<32, 64, TC_POOL>(w, 4, n, in, nullptr, out, Hs[2], Ws[2], err, s)));
  TRACE(l2a, 64, 2);
  SET(l2a, nullptr, s3); TRY((run_conv_split<64, 64, TC_PLAIN>(w, 5, n, in, nullptr, out, Hs[2], Ws[2], err, s)));
  TRACE(s3, 64, 2);
  SET(s3, nullptr, l3a); TRY((run_conv_split<64, 128, TC_POOL>(w, 6, n, in, nullptr, out, Hs[3], Ws[3], err, s)));
  TRACE(l3a, 128, 3);
  SET(l3a, nullptr, l3b); TRY((run_conv_split<128, 128, TC_PLAIN>(w, 7, n, in, nullptr, out, Hs[3], Ws[3], err, s)));
  TRACE(l3b, 128, 3);
  SET(l3b, nullptr, l2a); TRY((run_convT_split<128, 64, 0>(w, n, in, out, Hs[3], Ws[3], err, s)));
  TRACE(l2a, 64, 2);
  SET(l2a, B[k].s3, l2b); TRY((run_conv_split<128, 64, TC_CONCAT>(w, 8, n, in, sk, out, Hs[2], Ws[2], err, s)));
  TRACE(l2b, 64, 2);
  SET(l2b, nullptr, l2a); TRY((run_conv_split<64, 64, TC_PLAIN>(w, 9, n, in, nullptr, out, Hs[2], Ws[2], err, s)));
  TRACE(l2a, 64, 2);
  SET(l2a, nullptr, l1a); TRY((run_convT_split<64, 32, 1>(w, n, in, out, Hs[2], Ws[2], err, s)));
  TRACE(l1a, 32, 1);
  SET(l1a, B[k].s2, l1b); TRY((run_conv_split<64, 32, TC_CONCAT>(w, 10, n, in, sk, out, Hs[1], Ws[1], err, s)));
  TRACE(l1b, 32, 1);
  SET(l1b, nullptr, l1a); TRY((run_conv_split<32, 32, TC_PLAIN>(w, 11, n, in, nullptr, out, Hs[1], Ws[1], err, s)));
  TRACE(l1a, 32, 1);
  SET(l1a, nullptr, fa); TRY((run_convT_split<32, 16, 2>(w, n, in, out, Hs[1], Ws[1], err, s)));
  TRACE(fa, 16, 0);
  SET(fa, B[k].s1, fb);  TRY((run_conv_split<32, 16, TC_CONCAT>(w, 12, n, in, sk, out, Hs[0], Ws[0], err, s)));
  TRACE(fb, 16, 0);
  SET(fb, nullptr, fa);  TRY((run_conv_split<16, 16, TC_PLAIN>(w, 13, n, in, nullptr, out, Hs[0], Ws[0], err, s)));
  TRACE(fa, 16, 0);
  AdapterImg<float> ai[kMaxGroup];
  for (int k = 0; k < n; ++k)
    ai[k] = AdapterImg<float>{B[k].fa, reinterpret_cast<__half*>(B[k].x1), B[k].partial, B[k].att, imgs[k].out,
                              imgs[k].H, imgs[k].W};
  TRY(adapters_tc_run_group<float>(w->ad, net_f32_adapter_params(wf), ai, n, err, s));
#undef TRACE
#undef SET
#undef TRY
  return cudaSuccess;
}

template <typename T, bool Q8>
cudaError_t forward(const NetTcWeights* w, const NetF32Weights* wf, const NetImage* imgs,
                    void* const* ws, int n, unsigned int* err, cudaStream_t s, uint8_t* trace) {
  if (n < 1 || n > kMaxGroup || (trace && n != 1)) return cudaErrorInvalidValue;
  TcBuffers<T> B[kMaxGroup];
  int Hs[4][kMaxGroup], Ws[4][kMaxGroup];
  for (int k = 0; k < n; ++k) {
    const size_t P = (size_t)imgs[k].H * imgs[k].W;
    carve_tc(P, adapter_partial_floats(imgs[k].W, imgs[k].H), &B[k], static_cast<char*>(ws[k]));
    for (int lv = 0; lv < 4; ++lv) {
      Hs[lv][k] = imgs[k].H >> lv;
      Ws[lv][k] = imgs[k].W >> lv;
    }
  }
  // per-layer pointer lists
  const T* in[kMaxGroup];
  const T* sk[kMaxGroup];
  T* out[kMaxGroup];
  cudaError_t e;
  // FP8: every image's tensor maxima live in the first image's workspace,
  // cleared once per forward
  float* amax = Q8 ? B[0].amax : nullptr;
  if (Q8 && (e = cudaMemsetAsync(amax, 0, (size_t)n * kAmaxSlots * sizeof(float), s)) != cudaSuccess)
    return e;
  auto slots = [&](int ia, int ib, int io) {
    AmaxSlots m;
    m.base = amax;
    m.a = ia;
    m.b = ib;
    m.out = io;
    return m;
  };
  // diagnostic trace (one image): after each layer, a copy of its stored
  // output (NHWC, the activation type) appended to `trace`
  const size_t P0 = (size_t)imgs[0].H * imgs[0].W;
  size_t toff = 0;
  auto trace_copy = [&](const T* buf, int ch, int lv) -> cudaError_t {
    if (!trace) return cudaSuccess;
    const size_t bytes = (P0 >> (2 * lv)) * (size_t)ch * sizeof(T);
    cudaError_t ce = cudaMemcpyAsync(trace + toff, buf, bytes, cudaMemcpyDeviceToDevice, s);
    toff += bytes;
    return ce;
  };
#define TRY(x) if ((e = (x)) != cudaSuccess) return e
#define SET(IN, SKIP, OUT) for (int k = 0; k < n; ++k) { in[k] = B[k].IN; sk[k] = SKIP; out[k] = B[k].OUT; }
#define TRACE(BUF, CH, LV) TRY(trace_copy(B[0].BUF, CH, LV))
  for (int k = 0; k < n; ++k) out[k] = B[k].fa;
  float* first_amax[kMaxGroup];
  for (int k = 0; k < n; ++k) first_amax[k] = Q8 ? amax + (size_t)k * kAmaxSlots : nullptr;
  TRY(simt_first_conv_group<T>(wf, imgs, out, Q8 ? first_amax : nullptr, n, s));
  TRACE(fa, 16, 0);
  SET(fa, nullptr, s1);  TRY((run_conv<T, 16, 16, TC_PLAIN, Q8>(w, 1, n, in, nullptr, out, Hs[0], Ws[0], slots(0, -1, 1), err, s)));
  TRACE(s1, 16, 0);
  SET(s1, nullptr, l1a); TRY((run_conv<T, 16, 32, TC_POOL, Q8>(w, 2, n, in, nullptr, out, Hs[1], Ws[1], slots(1, -1, 2), err, s)));
  TRACE(l1a, 32, 1);
  SET(l1a, nullptr, s2); TRY((run_conv<T, 32, 32, TC_PLAIN, Q8>(w, 3, n, in, nullptr, out, Hs[1], Ws[1], slots(2, -1, 3), err, s)));
  TRACE(s2, 32, 1);
  SET(s2, nullptr, l2a); TRY((run_conv<T, 32, 64, TC_POOL, Q8>(w, 4, n, in, nullptr, out, Hs[2], Ws[2], slots(3, -1, 4), err, s)));
  TRACE(l2a, 64, 2);
  SET(l2a, nullptr, s3); TRY((run_conv<T, 64, 64, TC_PLAIN, Q8>(w, 5, n, in, nullptr, out, Hs[2], Ws[2], slots(4, -1, 5), err, s)));
  TRACE(s3, 64, 2);
  SET(s3, nullptr, l3a); TRY((run_conv<T, 64, 128, TC_POOL, Q8>(w, 6, n, in, nullptr, out, Hs[3], Ws[3], slots(5, -1, 6), err, s)));
  TRACE(l3a, 128, 3);
  SET(l3a, nullptr, l3b); TRY((run_conv<T, 128, 128, TC_PLAIN, Q8>(w, 7, n, in, nullptr, out, Hs[3], Ws[3], slots(6, -1, 7), err, s)));
  TRACE(l3b, 128, 3);
  SET(l3b, nullptr, l2a); TRY((run_convT<T, 128, 64, Q8, 0>(w, n, in, out, Hs[3], Ws[3], slots(7, -1, 14), err, s)));
  TRACE(l2a, 64, 2);
  SET(l2a, B[k].s3, l2b); TRY((run_conv<T, 128, 64, TC_CONCAT, Q8>(w, 8, n, in, sk, out, Hs[2], Ws[2], slots(14, 5, 8), err, s)));
  TRACE(l2b, 64, 2);
  SET(l2b, nullptr, l2a); TRY((run_conv<T, 64, 64, TC_PLAIN, Q8>(w, 9, n, in, nullptr, out, Hs[2], Ws[2], slots(8, -1, 9), err, s)));
  TRACE(l2a, 64, 2);
  SET(l2a, nullptr, l1a); TRY((run_convT<T, 64, 32, Q8, 1>(w, n, in, out, Hs[2], Ws[2], slots(9, -1, 15), err, s)));
  TRACE(l1a, 32, 1);
  SET(l1a, B[k].s2, l1b); TRY((run_conv<T, 64, 32, TC_CONCAT, Q8>(w, 10, n, in, sk, out, Hs[1], Ws[1], slots(15, 3, 10), err, s)));
  TRACE(l1b, 32, 1);
  SET(l1b, nullptr, l1a); TRY((run_conv<T, 32, 32, TC_PLAIN, Q8>(w, 11, n, in, nullptr, out, Hs[1], Ws[1], slots(10, -1, 11), err, s)));
  TRACE(l1a, 32, 1);
  SET(l1a, nullptr, fa); TRY((run_convT<T, 32, 16, Q8, 2>(w, n, in, out, Hs[1], Ws[1], slots(11, -1, 16), err, s)));
  TRACE(fa, 16, 0);
  SET(fa, B[k].s1, fb);  TRY((run_conv<T, 32, 16, TC_CONCAT, Q8>(w, 12, n, in, sk, out, Hs[0], Ws[0], slots(16, 1, 12), err, s)));
  TRACE(fb, 16, 0);
  SET(fb, nullptr, fa);  TRY((run_conv<T, 16, 16, TC_PLAIN, Q8>(w, 13, n, in, nullptr, out, Hs[0], Ws[0], slots(12, -1, 13), err, s)));
  TRACE(fa, 16, 0);
  AdapterImg<T> ai[kMaxGroup];
  for (int k = 0; k < n; ++k)
    ai[k] = AdapterImg<T>{B[k].fa, reinterpret_cast<__half*>(B[k].x1), B[k].partial, B[k].att, imgs[k].out,
                          imgs[k].H, imgs[k].W};
  TRY(adapters_tc_run_group<T>(w->ad, net_f32_adapter_params(wf), ai, n, err, s));
#undef TRACE
#undef SET
#undef TRY
  return cudaSuccess;
}
}  // namespace

size_t net_tc_workspace_bytes(int max_w, int max_h, int elem) {
  if (elem == 3) {
    TcBuffers<float> b;
    return carve_tc((size_t)max_w * max_h, adapter_partial_floats(max_w, max_h), &b, nullptr);
  }
  TcBuffers<__half> b;
  return carve_tc((size_t)max_w * max_h, adapter_partial_floats(max_w, max_h), &b, nullptr);
}

cudaError_t net_tc_forward(const NetTcWeights* w, const NetF32Weights* wf, const NetImage& img,
                           void* workspace, size_t ws_bytes, unsigned int* err, cudaStream_t s,
                           uint8_t* trace) {
  if (net_tc_workspace_bytes(img.W, img.H, w->elem) > ws_bytes) return cudaErrorInvalidValue;
  void* ws[1] = {workspace};
  if (w->elem == 3) return forward_split(w, wf, &img, ws, 1, err, s, trace);
  if (w->elem == 2) return forward<__half, true>(w, wf, &img, ws, 1, err, s, trace);
  if (w->elem == 1) return forward<__nv_bfloat16, false>(w, wf, &img, ws, 1, err, s, trace);
  return forward<__half, false>(w, wf, &img, ws, 1, err, s, trace);
}

size_t net_tc_trace_bytes(int width, int height) {
  // 144 activation values per pixel of the full-resolution image (the 17
  // stored tensors), up to four bytes each (binary32 in the split-BF16 form)
  return (size_t)width * height * 144 * 4;
}

cudaError_t net_tc_forward_group(const NetTcWeights* w, const NetF32Weights* wf,
                                 const NetImage* imgs, void* const* ws, int n, unsigned int* err,
                                 cudaStream_t s) {
  if (w->elem == 3) return forward_split(w, wf, imgs, ws, n, err, s);
  if (w->elem == 2) return forward<__half, true>(w, wf, imgs, ws, n, err, s, nullptr);
  if (w->elem == 1) return forward<__nv_bfloat16, false>(w, wf, imgs, ws, n, err, s, nullptr);
  return forward<__half, false>(w, wf, imgs, ws, n, err, s, nullptr);
}

void net_tc_set_ctas_per_sm(int v) { g_conv_ctas_per_sm = v < 1 ? 1 : (v > 4 ? 4 : v); }
int net_tc_ctas_per_sm() { return g_conv_ctas_per_sm; }

}  // namespace nsl
