// The four NAFBlock channel adapters (Sec. 4.3, Fig. 3) with their 1x1
// convolutions on the tensor cores (tcgen05 kind::f16, FP16 operands, FP32
// accumulation in TMEM); used by the tensor-core network paths.
//
// Pass 1, per 16x8 tile (persistent CTAs of 256 threads): pw1 (a 1x1
// convolution) followed by the depthwise 3x3 is one linear map, a 3x3
// convolution from the 16 normalised channels to the 128 pw1 channels of the
// four adapters with weights dw[o, tap] * W1[o, c], plus the bias
// dw_b[o] + b1[o] * (sum of dw[o, tap] over the taps inside the image: the
// depthwise convolution pads its input, pw1's output, with zeros), read from a
// table of the 16 cases of a pixel's missing left, right, top and bottom
// neighbours.  The 18x10
// halo of F is normalised (LayerNorm without its affine, which is folded into
// pw1) into FP16 A planes stored column by column, so that each tap is the
// same planes shifted by whole rows; nine MMAs (M = 128 pixels, N = 128,
// K = 16) accumulate the convolution in TMEM, and the epilogue adds the bias,
// applies the simple gate, writes x1 and reduces the tile's per-channel sums
// with warp shuffles.
// Pass 2, per 128 pixels: three chained MMAs with block-diagonal weights (the
// four adapters side by side): pw2 on att * x1 (K = 64, N = 64), ffn1 on
// LN2(y) (N = 128), and on the gate g the heads folded through ffn2 (N = 16,
// eight used): z = y + gamma (W_f2 g + b_f2) only feeds the heads, so
// W_h z + b_h = W_h y + (W_h diag(gamma) W_f2) g + (W_h (gamma b_f2) + b_h),
// the first term on the SIMT cores.  Between the MMAs each thread handles its
// pixel's row.
// The SCA reduction between the passes is the deterministic SIMT one.
#include <cmath>
#include <cstring>
#include <vector>

#include "nsl_internal.cuh"
#include "tc_ptx.cuh"

namespace nsl {

namespace {

constexpr int C = kC0;                  // 16 channels per adapter
constexpr int kTW = 16, kTH = 8;        // pass-1 tile: same tiling as the SIMT pass 1
constexpr int kHW = kTW + 2, kHH = kTH + 2;
constexpr int kHalo = kHW * kHH;        // 180
// pass-1 halo, column by column: A row 10 hx + hy holds halo pixel (hx, hy), so
// M row m = 8 x + y (output pixel (x, y) of the tile) of tap (dx, dy) is A row
// m + 10 (x + dx) - 8 x + dy: eight-row groups (one output column each) 160
// bytes apart, the tap a shift of 10 dx + dy rows
constexpr int kP1Threads = 256;
constexpr int kP1Plane = kHalo * 16;                      // one 8-channel plane, 2880 B
constexpr int kP1A = 0;                                   // 2 planes
constexpr int kP1B = kP1A + 2 * kP1Plane;                 // 9 taps x (128 rows x 32 B)
constexpr int kP1Par = kP1B + 9 * 128 * 32;               // biases and depthwise weights (floats)
constexpr int kP1ParN = 16 * 128;                         // bias [edge case][128] (case 0: interior)
constexpr int kP1Red = kP1Par + kP1ParN * 4;              // warp sums [8 warps][32]
constexpr int kP1Bar = kP1Red + 8 * 32 * 4;               // mbarriers: MMAs, weights; TMEM slot
constexpr int kP1Smem = kP1Bar + 32;
constexpr int kP1WBytes = 9 * 128 * 32;
static_assert(kP1B % 128 == 0 && kP1Par % 16 == 0, "pass-1 shared-memory alignment");

// pass-2 shared memory (bytes)
constexpr int kP2W2 = 0;                  // 64 x 64 block-diagonal
constexpr int kP2F1 = kP2W2 + 64 * 64 * 2;
constexpr int kP2Hd = kP2F1 + 128 * 64 * 2;  // folded head on the gate, 16 x 64
constexpr int kP2A = kP2Hd + 16 * 64 * 2;  // 8 planes x 128 rows x 16 B
constexpr int kP2Par = kP2A + 8 * 128 * 16;
constexpr int kP2ParN = 64 + 64 + 128 + 16 + 128;   // b2, beta, fb1, head constant, head on y
constexpr int kP2Att = kP2Par + kP2ParN * 4;
constexpr int kP2Bar = kP2Att + 64 * 4;   // mbarriers: MMAs, weights; TMEM slot
constexpr int kP2Smem = kP2Bar + 32;
static_assert(kP2F1 % 16 == 0 && kP2Hd % 16 == 0 && kP2Par % 16 == 0 && (kP2ParN * 4) % 16 == 0,
              "pass-2 bulk copy alignment");

struct AdapterTcDev {
  const uint8_t* b9;   // pass-1 B operands of the nine taps (9 x 4096 B)
  const float* p1f;    // kP1ParN floats
  const uint8_t* w2;   // 8192 B
  const uint8_t* f1;   // 16384 B
  const uint8_t* hd;   // 2048 B: the heads folded through ffn2 and gamma
  const float* p2f;    // kP2ParN floats
};

template <typename T> __device__ __forceinline__ float tof(T v);
template <> __device__ __forceinline__ float tof<float>(float v) { return v; }
template <> __device__ __forceinline__ float tof<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T fromf(float v);
template <> __device__ __forceinline__ __half fromf<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 fromf<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// n (a multiple of 8) channels of a 16-bit or binary32 NHWC row into floats
template <typename T, int N>
__device__ __forceinline__ void load_row(const T* p, float* v) {
  constexpr int PER = 16 / (int)sizeof(T);   // values per 16-byte load
#pragma unroll
  for (int q = 0; q < N / PER; ++q) {
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(p) + q);
    const T* h = reinterpret_cast<const T*>(&t);
#pragma unroll
    for (int k = 0; k < PER; ++k) v[PER * q + k] = tof<T>(h[k]);
  }
}

// 8 floats -> one 16-byte row of an FP16 A plane
__device__ __forceinline__ uint4 pack8h(const float* v) {
  __align__(16) __half2 h[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
  return *reinterpret_cast<const uint4*>(h);
}

// (x - mean) / sqrt(var + 1e-6) over 16 channels
__device__ __forceinline__ void norm16(const float* x, float* y) {
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

// x1 (the gated depthwise output of the four adapters, 64 channels) is stored
// as eight planes of 16-byte chunks: plane q holds channels 8q .. 8q+7 of every
// pixel.  Pass 2's thread-per-pixel loads of one chunk are then 512
// contiguous bytes per warp, and pass 1's pixel-per-thread 16-byte stores
// cover 64 contiguous bytes in each of the 8 image rows of a warp's 4 x 8
// pixels (NHWC rows of 128 bytes would spread both over 32 lines per warp
// instruction).
__device__ __forceinline__ size_t x1_index(int npix, int pix, int ch) {
  return ((size_t)(ch >> 3) * npix + pix) * 8 + (ch & 7);
}

template <typename TA>
struct AdGroup {
  AdapterImg<TA> img[kMaxGroup];
  int tile_start[kMaxGroup + 1];
  int px_start[kMaxGroup + 1];
  int nimg;
};

__device__ __forceinline__ int find_group(const int* start, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename TA>
__global__ void __launch_bounds__(kP1Threads, 4) adapters_p1_tc(const __grid_constant__ AdGroup<TA> G,
                                                             const AdapterTcDev W, unsigned int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* A = smem + kP1A;
  const float* btab = reinterpret_cast<const float*>(smem + kP1Par);   // bias [edge case][128]
  float* red = reinterpret_cast<float*>(smem + kP1Red);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kP1Bar);       // [0] the MMAs, [1] the weights
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + kP1Bar + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(slot, 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    // the weights with bulk copies (pieces of at most 32 KB), while the
    // previous kernel may still run
    mbar_expect_tx(&bar[1], (uint32_t)(kP1WBytes + kP1ParN * 4));
    bulk_g2s(smem + kP1B, W.b9, 32768u, &bar[1]);
    bulk_g2s(smem + kP1B + 32768, W.b9 + 32768, (uint32_t)(kP1WBytes - 32768), &bar[1]);
    bulk_g2s(smem + kP1Par, W.p1f, (uint32_t)(kP1ParN * 4), &bar[1]);
  }
  pdl_wait();      // F comes from the last convolution
  pdl_trigger();
  constexpr uint32_t idesc = idesc_f16kind(0u, 128, 128);
  const int total = G.tile_start[G.nimg];
  uint32_t phase = 0;
  bool ok = __syncthreads_and(mbar_wait(&bar[1], 0u) ? 1 : 0) != 0;
  if (!ok) record_error(err, 0x100u);

  // halo staging: thread hp < 180 loads halo pixel (hp % 18, hp / 18) (row by
  // row, so a warp reads contiguous NHWC rows) and stores it column by column;
  // the next tile's loads are issued before the current tile's epilogue
  constexpr int RF = C * (int)sizeof(TA) / 16;   // 16-byte loads per F row
  const int hx = tid % kHW, hy = tid / kHW;
  uint4 raw[RF];
  bool rin = false;
  auto fetch = [&](int t) {
    rin = false;
    if (tid >= kHalo || t >= total) return;
    const int k = find_group(G.tile_start, G.nimg, t);
    const AdapterImg<TA>& im = G.img[k];
    const int lt = t - G.tile_start[k];
    const int ntx = (im.W + kTW - 1) / kTW;
    const int x = (lt % ntx) * kTW + hx - 1, y = (lt / ntx) * kTH + hy - 1;
    rin = x >= 0 && x < im.W && y >= 0 && y < im.H;
    if (rin) {
      const uint4* p = reinterpret_cast<const uint4*>(im.F + ((size_t)y * im.W + x) * C);
#pragma unroll
      for (int q = 0; q < RF; ++q) raw[q] = __ldg(p + q);
    }
  };

  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (M rows = pixels) and
  // the columns of adapters 2 (w / 4) and 2 (w / 4) + 1
  const int qt = warp & 3, hp2 = warp >> 2;
  const int m = qt * 32 + lane;                  // M row = 8 x + y

  fetch(blockIdx.x);
#pragma unroll 1
  for (int t = blockIdx.x; ok && t < total; t += gridDim.x) {
    if (t + (int)gridDim.x >= total) pdl_trigger_last();
    const int k = find_group(G.tile_start, G.nimg, t);
    const AdapterImg<TA>& im = G.img[k];
    const int lt = t - G.tile_start[k];
    const int ntx = (im.W + kTW - 1) / kTW;
    const int x0 = (lt % ntx) * kTW, y0 = (lt / ntx) * kTH;
    // this tile's halo into A (the previous tile's MMAs have completed)
    if (tid < kHalo) {
      float v[C], n[C];
      const TA* h = reinterpret_cast<const TA*>(raw);
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = rin ? tof<TA>(h[c]) : 0.f;
      norm16(v, n);
      const int r = hx * kHH + hy;
      *reinterpret_cast<uint4*>(A + r * 16) = pack8h(n);
      *reinterpret_cast<uint4*>(A + kP1Plane + r * 16) = pack8h(n + 8);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();  // A is staged; the previous tile's TMEM and warp-sum readers are done
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ab = smem_u32(A), bb = smem_u32(smem + kP1B);
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
        mma_f16kind(tmem, smem_desc(ab + (uint32_t)((dx * kHH + dy) * 16), kP1Plane, kHH * 16),
                    smem_desc(bb + (uint32_t)(tap * 128 * 32), 128 * 16, 128), idesc, tap > 0 ? 1u : 0u);
      }
      mma_commit(&bar[0]);
    }
    fetch(t + (int)gridDim.x);
    ok = __syncthreads_and(mbar_wait(&bar[0], phase) ? 1 : 0) != 0;
    if (!ok) {
      record_error(err, 0x100u);
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    {
      const int px = x0 + (m >> 3), py = y0 + (m & 7);
      const bool valid = px < im.W && py < im.H;
      // edge case: bit 0 no left neighbour, 1 no right, 2 no upper, 3 no lower
      const int ec = (px < 1 ? 1 : 0) | (px + 1 >= im.W ? 2 : 0) | (py < 1 ? 4 : 0) | (py + 1 >= im.H ? 8 : 0);
      const size_t npix = (size_t)im.H * im.W, pix = (size_t)py * im.W + px;
#pragma unroll 1
      for (int al = 0; al < 2; ++al) {
        const int a = 2 * hp2 + al;
        float d0[16], d1[16];
        const uint32_t ta = tmem + ((uint32_t)(qt * 32) << 16) + (uint32_t)(a * 32);
        tmem_ld16(ta, d0);
        tmem_ld16(ta + 16, d1);
        const float4* bt = reinterpret_cast<const float4*>(btab + ec * 128 + a * 32);
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) {
          const float4 c0 = bt[j4], c1 = bt[4 + j4];
          d0[4 * j4 + 0] = (d0[4 * j4 + 0] + c0.x) * (d1[4 * j4 + 0] + c1.x);   // the simple gate
          d0[4 * j4 + 1] = (d0[4 * j4 + 1] + c0.y) * (d1[4 * j4 + 1] + c1.y);
          d0[4 * j4 + 2] = (d0[4 * j4 + 2] + c0.z) * (d1[4 * j4 + 2] + c1.z);
          d0[4 * j4 + 3] = (d0[4 * j4 + 3] + c0.w) * (d1[4 * j4 + 3] + c1.w);
        }
        if (valid) {
          uint4* dst = reinterpret_cast<uint4*>(im.x1 + x1_index((int)npix, (int)pix, a * C));
          dst[0] = pack8h(d0);
          dst[npix] = pack8h(d0 + 8);              // the next 8-channel plane
        }
        // the tile's per-channel sums: halve the 16 values across lane bits
        // 4..1 (lane l ends with channel (l >> 1) & 15), then add the lane pair
#pragma unroll
        for (int j = 0; j < 16; ++j) d0[j] = valid ? d0[j] : 0.f;
#pragma unroll
        for (int w = 8, b = 16; w >= 1; w >>= 1, b >>= 1) {
          const bool up = (lane & b) != 0;
#pragma unroll
          for (int i = 0; i < w; ++i) {
            const float keep = up ? d0[i + w] : d0[i];
            const float give = up ? d0[i] : d0[i + w];
            d0[i] = keep + __shfl_xor_sync(0xffffffffu, give, b);
          }
        }
        d0[0] += __shfl_xor_sync(0xffffffffu, d0[0], 1);
        if ((lane & 1) == 0) red[warp * 32 + al * 16 + (lane >> 1)] = d0[0];
      }
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 4 * C) {
      // channel tid: adapter pair tid / 32, the four lane quarters in order
      const int h = tid >> 5, l = tid & 31;
      const float* r = red + h * 4 * 32 + l;
      im.partial[(size_t)lt * (4 * C) + tid] = ((r[0] + r[32]) + r[64]) + r[96];
    }
  }
  tc_fence_before();
  __syncthreads();
  pdl_trigger_end();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// one 16-channel row slice of an FP16 A plane pair at row `row`
__device__ __forceinline__ void put16(uint8_t* A, int plane, int row, const float* v) {
  *reinterpret_cast<uint4*>(A + plane * 2048 + row * 16) = pack8h(v);
  *reinterpret_cast<uint4*>(A + (plane + 1) * 2048 + row * 16) = pack8h(v + 8);
}

template <typename TA>
__global__ void __launch_bounds__(128) adapters_p2_tc(const __grid_constant__ AdGroup<TA> G,
                                                      const AdapterTcDev W, unsigned int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* A = smem + kP2A;
  const float* par = reinterpret_cast<const float*>(smem + kP2Par);
  const float* b2 = par;
  const float* beta = b2 + 64;
  const float* fb1 = beta + 64;
  const float* hc = fb1 + 128;     // folded head constant [8]
  const float* hy = hc + 16;       // head weights on y [8][16] (head j reads adapter j / 2)
  float* att = reinterpret_cast<float*>(smem + kP2Att);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kP2Bar);   // [0] the MMAs, [1] the weights
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + kP2Bar + 16);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(slot, 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    // the weights with bulk copies, while the previous kernel may still run
    mbar_expect_tx(&bar[1], (uint32_t)(64 * 64 * 2 + 128 * 64 * 2 + 16 * 64 * 2 + kP2ParN * 4));
    bulk_g2s(smem + kP2W2, W.w2, 64u * 64u * 2u, &bar[1]);
    bulk_g2s(smem + kP2F1, W.f1, 128u * 64u * 2u, &bar[1]);
    bulk_g2s(smem + kP2Hd, W.hd, 16u * 64u * 2u, &bar[1]);
    bulk_g2s(smem + kP2Par, W.p2f, (uint32_t)(kP2ParN * 4), &bar[1]);
  }
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t ab = smem_u32(A);
  const int total = G.px_start[G.nimg];
  constexpr int plane_of[8] = {4, 5, 0, 1, 2, 3, 6, 7};   // head column -> output plane
  uint32_t phase = 0;
  bool ok = __syncthreads_and(mbar_wait(&bar[1], 0u) ? 1 : 0) != 0;

  // one GEMM stage: D[0, n) = A(K = 64) x B(n rows), then wait
  auto stage = [&](const uint8_t* b, int n, uint32_t idesc) -> bool {
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t bb = smem_u32(b);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma_f16kind(tmem, smem_desc(ab + (uint32_t)(kk * 2 * 2048), 2048, 128),
                    smem_desc(bb + (uint32_t)(kk * n * 32), (uint32_t)(n * 16), 128), idesc,
                    kk > 0 ? 1u : 0u);
      mma_commit(&bar[0]);
    }
    const bool done = __syncthreads_and(mbar_wait(&bar[0], phase) ? 1 : 0) != 0;
    phase ^= 1u;
    tc_fence_after();
    return done;
  };

  // this thread's pixel of a block: raw x1 (64 channels) and F (16 channels);
  // the next block's are loaded while the current block's GEMMs run
  constexpr int RF = C * (int)sizeof(TA) / 16;   // 16-byte loads of a pixel's F row
  uint4 rx[8], rf[RF];
  auto fetch = [&](int blk) {
#pragma unroll
    for (int q = 0; q < 8; ++q) rx[q] = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int q = 0; q < RF; ++q) rf[q] = make_uint4(0, 0, 0, 0);
    if (blk >= total) return;
    const int kk = find_group(G.px_start, G.nimg, blk);
    const AdapterImg<TA>& m = G.img[kk];
    const int pp = (blk - G.px_start[kk]) * 128 + tid;
    if (pp >= m.H * m.W) return;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      rx[q] = __ldg(reinterpret_cast<const uint4*>(m.x1 + x1_index(m.H * m.W, pp, 8 * q)));
#pragma unroll
    for (int q = 0; q < RF; ++q) rf[q] = __ldg(reinterpret_cast<const uint4*>(m.F + (size_t)pp * C) + q);
  };
  pdl_wait();      // x1 and the attention weights come from pass 1 and the reduction
  pdl_trigger();
  fetch(blockIdx.x);

#pragma unroll 1
  for (int blk = blockIdx.x; ok && blk < total; blk += gridDim.x) {
    if (blk + (int)gridDim.x >= total) pdl_trigger_last();
    const int k = find_group(G.px_start, G.nimg, blk);
    const AdapterImg<TA>& im = G.img[k];
    const int npix = im.H * im.W;
    const int p = (blk - G.px_start[k]) * 128 + tid;
    const bool valid = p < npix;
    __syncthreads();  // the previous block is done with att and A
    if (tid < 64) att[tid] = im.att[tid];
    __syncthreads();
    float f[C], hs[8];
    // stage 1: A = att * x1
    {
      float xv[4 * C];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const __half* h = reinterpret_cast<const __half*>(&rx[q]);
#pragma unroll
        for (int e = 0; e < 8; ++e) xv[8 * q + e] = __half2float(h[e]) * att[8 * q + e];
      }
#pragma unroll
      for (int q = 0; q < RF; ++q) {
        const TA* h = reinterpret_cast<const TA*>(&rf[q]);
#pragma unroll
        for (int e = 0; e < C / RF; ++e) f[(C / RF) * q + e] = tof<TA>(h[e]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) put16(A, 2 * a, tid, xv + a * C);
    }
    fetch(blk + (int)gridDim.x);
    if (!(ok = stage(smem + kP2W2, 64, idesc_f16kind(0u, 128, 64)))) break;
    // stage 2: y = F + beta (pw2 + b2); the heads' part on y; A = LN2(y)
    // (affine folded into ffn1)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float d[16], y[16], n[16];
      tmem_ld16(lane_base + (uint32_t)(a * 16), d);
#pragma unroll
      for (int c = 0; c < C; ++c) y[c] = fmaf(beta[a * C + c], d[c] + b2[a * C + c], f[c]);
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        float h = hc[2 * a + jj];
#pragma unroll
        for (int c = 0; c < C; ++c) h = fmaf(hy[(2 * a + jj) * C + c], y[c], h);
        hs[2 * a + jj] = h;
      }
      norm16(y, n);
      put16(A, 2 * a, tid, n);
    }
    if (!(ok = stage(smem + kP2F1, 128, idesc_f16kind(0u, 128, 128)))) break;
    // the gate of ffn1 (channels o and o + 16 of each adapter)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float u[16], v[16], gt[16];
      tmem_ld16(lane_base + (uint32_t)(a * 32), u);
      tmem_ld16(lane_base + (uint32_t)(a * 32 + 16), v);
#pragma unroll
      for (int c = 0; c < C; ++c) gt[c] = (u[c] + fb1[a * 32 + c]) * (v[c] + fb1[a * 32 + 16 + c]);
      put16(A, 2 * a, tid, gt);
    }
    // stage 3: the folded heads on the gate, plus the part on y
    if (!(ok = stage(smem + kP2Hd, 16, idesc_f16kind(0u, 128, 16)))) break;
    {
      float d[16];
      tmem_ld16(lane_base, d);
      if (valid) {
#pragma unroll
        for (int j = 0; j < 8; ++j) im.out[(size_t)plane_of[j] * npix + p] = d[j] + hs[j];
      }
    }
  }
  if (!ok) record_error(err, 0x200u);
  tc_fence_before();
  __syncthreads();
  pdl_trigger_end();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// Pack a [N][K] row-major float matrix (K a multiple of 16) as the FP16
// K-major B operand: per 16-wide K slice, N rows x 32 bytes, the two 8-wide K
// core matrices N*16 bytes apart, rows grouped by 8 (128 bytes).
void pack_b(const std::vector<float>& w, int N, int K, std::vector<uint8_t>& out) {
  out.assign((size_t)N * K * 2, 0);
  for (int kk = 0; kk < K / 16; ++kk)
    for (int n = 0; n < N; ++n)
      for (int k = 0; k < 16; ++k) {
        const __half h = __float2half_rn(w[(size_t)n * K + kk * 16 + k]);
        std::memcpy(out.data() + (size_t)kk * N * 32 + (k / 8) * N * 16 + (n / 8) * 128 + (n % 8) * 16 +
                        (k % 8) * 2,
                    &h, 2);
      }
}

}  // namespace

struct AdapterTcWeights {
  AdapterTcDev dev{};
  std::vector<void*> allocs;
  int p1_grid = 0, p2_grid = 0;
};

AdapterTcWeights* adapters_tc_create(const AdapterParamSet& prm, cudaError_t* err) {
  *err = cudaSuccess;
  AdapterTcWeights* w = new AdapterTcWeights();
  auto up = [&](const void* src, size_t bytes) -> void* {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) { *err = e; return nullptr; }
    w->allocs.push_back(p);
    if ((e = cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice)) != cudaSuccess) *err = e;
    return p;
  };
  const AdapterP1& p1 = prm.p1;
  const AdapterP2& p2 = prm.p2;
  std::vector<float> m;
  std::vector<uint8_t> pk;
  // pw1 and the depthwise 3x3 as one 3x3 convolution: tap (dx, dy) (index
  // 3 dy + dx), row 32a + o (pw1 channel o of adapter a), K = the 16 normalised
  // channels, weight dw[o, tap] * W1[o, c] (the product in double, rounded once)
  std::vector<uint8_t> b9;
  for (int tap = 0; tap < 9; ++tap) {
    m.assign(128 * 16, 0.f);
    for (int a = 0; a < 4; ++a)
      for (int o = 0; o < 32; ++o)
        for (int c = 0; c < 16; ++c)
          m[(size_t)(a * 32 + o) * 16 + c] = (float)((double)p1.dww[a][o][tap] * (double)p1.w1[a][o][c]);
    pack_b(m, 128, 16, pk);
    b9.insert(b9.end(), pk.begin(), pk.end());
  }
  w->dev.b9 = static_cast<const uint8_t*>(up(b9.data(), b9.size()));
  // the bias of each edge case e (bit 0: no left neighbour, 1: no right,
  // 2: no upper, 3: no lower): dw_b + b1 * (sum of the taps inside)
  std::vector<float> f1s;
  for (int e = 0; e < 16; ++e)
    for (int a = 0; a < 4; ++a)
      for (int o = 0; o < 32; ++o) {
        double sw = 0.0;
        for (int dy = 0; dy < 3; ++dy)
          for (int dx = 0; dx < 3; ++dx) {
            const bool in = !((dx == 0 && (e & 1)) || (dx == 2 && (e & 2)) || (dy == 0 && (e & 4)) ||
                              (dy == 2 && (e & 8)));
            if (in) sw += p1.dww[a][o][dy * 3 + dx];
          }
        f1s.push_back((float)((double)p1.dwb[a][o] + (double)p1.b1[a][o] * sw));
      }
  w->dev.p1f = static_cast<const float*>(up(f1s.data(), f1s.size() * 4));
  // block-diagonal pass-2 weights: input channel a*16 + ci feeds only adapter a
  m.assign(64 * 64, 0.f);
  for (int a = 0; a < 4; ++a)
    for (int co = 0; co < 16; ++co)
      for (int ci = 0; ci < 16; ++ci) m[(size_t)(a * 16 + co) * 64 + a * 16 + ci] = p2.w2[a][co][ci];
  pack_b(m, 64, 64, pk);
  w->dev.w2 = static_cast<const uint8_t*>(up(pk.data(), pk.size()));
  m.assign(128 * 64, 0.f);
  for (int a = 0; a < 4; ++a)
    for (int o = 0; o < 32; ++o)
      for (int ci = 0; ci < 16; ++ci) m[(size_t)(a * 32 + o) * 64 + a * 16 + ci] = p2.f1[a][o][ci];
  pack_b(m, 128, 64, pk);
  w->dev.f1 = static_cast<const uint8_t*>(up(pk.data(), pk.size()));
  // heads folded through ffn2 and gamma: row 2a + j, input channel a*16 + ci,
  // W' = W_h diag(gamma) W_f2 (double accumulation); constant W_h (gamma b_f2) + b_h
  m.assign(16 * 64, 0.f);
  std::vector<float> hcst(16, 0.f), hyv(128, 0.f);
  for (int a = 0; a < 4; ++a)
    for (int j = 0; j < 2; ++j) {
      double cst = p2.hb[a][j];
      for (int co = 0; co < 16; ++co) cst += (double)p2.hw[a][j][co] * p2.gamma[a][co] * p2.fb2[a][co];
      hcst[2 * a + j] = (float)cst;
      for (int ci = 0; ci < 16; ++ci) {
        double v = 0.0;
        for (int co = 0; co < 16; ++co) v += (double)p2.hw[a][j][co] * p2.gamma[a][co] * p2.f2[a][co][ci];
        m[(size_t)(2 * a + j) * 64 + a * 16 + ci] = (float)v;
        hyv[(2 * a + j) * 16 + ci] = p2.hw[a][j][ci];
      }
    }
  pack_b(m, 16, 64, pk);
  w->dev.hd = static_cast<const uint8_t*>(up(pk.data(), pk.size()));
  std::vector<float> f2s;
  for (int a = 0; a < 4; ++a) for (int c = 0; c < 16; ++c) f2s.push_back(p2.b2[a][c]);
  for (int a = 0; a < 4; ++a) for (int c = 0; c < 16; ++c) f2s.push_back(p2.beta[a][c]);
  for (int a = 0; a < 4; ++a) for (int o = 0; o < 32; ++o) f2s.push_back(p2.fb1[a][o]);
  for (int k = 0; k < 16; ++k) f2s.push_back(hcst[k]);
  for (int k = 0; k < 128; ++k) f2s.push_back(hyv[k]);
  while (f2s.size() < (size_t)kP2ParN) f2s.push_back(0.f);
  w->dev.p2f = static_cast<const float*>(up(f2s.data(), f2s.size() * 4));
  if (*err != cudaSuccess) {
    adapters_tc_destroy(w);
    return nullptr;
  }
  return w;
}

void adapters_tc_destroy(AdapterTcWeights* w) {
  if (!w) return;
  for (void* p : w->allocs) cudaFree(p);
  delete w;
}

template <typename TA>
cudaError_t adapters_tc_run_group(const AdapterTcWeights* w, const AdapterParamSet& prm,
                                  const AdapterImg<TA>* imgs, int n, unsigned int* err,
                                  cudaStream_t s) {
  if (n < 1 || n > kMaxGroup) return cudaErrorInvalidValue;
  // kernel attributes and residency, set up once per process (a function-local
  // static is initialised thread-safely, so concurrent first calls wait for it)
  struct Setup {
    cudaError_t err;
    int occ1, occ2;
  };
  static const Setup setup = [] {
    Setup r{cudaSuccess, 0, 0};
    // the largest shared-memory carveout, so that several CTAs fit per SM
    cudaError_t e = cudaFuncSetAttribute(adapters_p1_tc<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, kP1Smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(adapters_p2_tc<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, kP2Smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(adapters_p1_tc<TA>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(adapters_p2_tc<TA>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) {
      r.err = e;
      return r;
    }
    r.occ1 = tc_ctas_per_sm(reinterpret_cast<const void*>(adapters_p1_tc<TA>), kP1Threads, kP1Smem, 128);
    r.occ2 = tc_ctas_per_sm(reinterpret_cast<const void*>(adapters_p2_tc<TA>), 128, kP2Smem, 128);
    return r;
  }();
  if (setup.err != cudaSuccess) return setup.err;
  const int occ1 = setup.occ1, occ2 = setup.occ2;
  AdGroup<TA> G{};
  G.nimg = n;
  int tiles = 0, blocks = 0;
  for (int k = 0; k < n; ++k) {
    G.img[k] = imgs[k];
    G.tile_start[k] = tiles;
    G.px_start[k] = blocks;
    tiles += ((imgs[k].W + kTW - 1) / kTW) * ((imgs[k].H + kTH - 1) / kTH);
    blocks += (imgs[k].W * imgs[k].H + 127) / 128;
  }
  G.tile_start[n] = tiles;
  G.px_start[n] = blocks;
  const int g1 = tiles < num_sms() * occ1 ? tiles : num_sms() * occ1;
  cudaError_t e = launch_pdl(adapters_p1_tc<TA>, dim3(g1), dim3(kP1Threads), (size_t)kP1Smem, s, G, w->dev, err);
  if (e != cudaSuccess) return e;
  if ((e = adapters_reduce_only_group<TA>(prm, imgs, n, s)) != cudaSuccess) return e;
  const int g2 = blocks < num_sms() * occ2 ? blocks : num_sms() * occ2;
  return launch_pdl(adapters_p2_tc<TA>, dim3(g2), dim3(128), (size_t)kP2Smem, s, G, w->dev, err);
}

template cudaError_t adapters_tc_run_group<__half>(const AdapterTcWeights*, const AdapterParamSet&,
                                                   const AdapterImg<__half>*, int, unsigned int*,
                                                   cudaStream_t);
template cudaError_t adapters_tc_run_group<__nv_bfloat16>(const AdapterTcWeights*, const AdapterParamSet&,
                                                          const AdapterImg<__nv_bfloat16>*, int,
                                                          unsigned int*, cudaStream_t);
template cudaError_t adapters_tc_run_group<float>(const AdapterTcWeights*, const AdapterParamSet&,
                                                  const AdapterImg<float>*, int, unsigned int*, cudaStream_t);

}  // namespace nsl
