// The four NAFBlock channel adapters of the lightmap generator (Sec. 4.3,
// Fig. 3: F&B, L&R, U&D, A&E), each followed by its 1x1 head, on the SIMT cores.
//
// Per adapter a and pixel:  x1 = SG(dw3x3(pw1(LN1(F))))
//                           y  = F + beta * pw2(x1 * att_a),  att_a = W_sca mean_HW(x1) + b_sca
//                           z  = y + gamma * ffn2(SG(ffn1(LN2(y))))
//                           out planes = head(z)
// The global mean of the simplified channel attention splits the work into
// pass 1 (x1 and per-tile channel sums), a deterministic reduction to att, and
// pass 2 (the rest, per pixel).  LayerNorm affines are folded into the 1x1
// convolution that follows them (W' = W diag(w_ln), b' = b + W b_ln), and all
// weights travel as kernel parameters: the loops are unrolled so every FMA reads
// its weight from the constant bank at a uniform address, with no shared-memory
// traffic for weights.
#include <cmath>
#include <type_traits>

#include "nsl_internal.cuh"

namespace nsl {

namespace {

constexpr int C = kC0;                  // 16 channels per adapter
constexpr int kTW = 16, kTH = 8;        // pass-1 tile (128 pixels)
constexpr int kHW = kTW + 2, kHH = kTH + 2;
constexpr int kHalo = kHW * kHH;        // 180
constexpr int kHaloS = kHalo + 1;
constexpr int kXS = C + 4;              // padded row of the normalised halo: 80 bytes,
                                        // conflict-free 16-byte accesses per quarter warp

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

// 16 consecutive channels (16-byte aligned) to / from float registers
__device__ __forceinline__ void load16(const float* p, float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p) + q);
    v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
  }
}
template <typename T>
__device__ __forceinline__ void load16(const T* p, float* v) {
  using T2 = typename std::conditional<std::is_same<T, __half>::value, __half2, __nv_bfloat162>::type;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(p) + q);
    const T2* h = reinterpret_cast<const T2*>(&t);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[8 * q + 2 * k] = to_f(h[k].x);
      v[8 * q + 2 * k + 1] = to_f(h[k].y);
    }
  }
}
__device__ __forceinline__ void store16(float* p, const float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
template <typename T>
__device__ __forceinline__ void store16(T* p, const float* v) {
  __align__(16) T h[C];
#pragma unroll
  for (int c = 0; c < C; ++c) h[c] = from_f<T>(v[c]);
  reinterpret_cast<uint4*>(p)[0] = reinterpret_cast<const uint4*>(h)[0];
  reinterpret_cast<uint4*>(p)[1] = reinterpret_cast<const uint4*>(h)[1];
}

// normalised (x - mean) / sqrt(var + eps) over 16 channels
__device__ __forceinline__ void normalise16(const float* x, float* y) {
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

}  // namespace

// Pass 1: one CTA per 16x8 tile; the 18x10 halo of F is normalised once and
// shared by the four adapters.
template <typename TA>
__device__ __forceinline__ void adapters_pass1_tile(const TA* __restrict__ F, const AdapterP1& P,
                                                    TA* __restrict__ x1,
                                                    float* __restrict__ partial, int H, int W,
                                                    int bx, int by, int tileid) {
  __shared__ __align__(16) float xh[kHalo * kXS];   // normalised halo
  __shared__ float t[2 * C * kHaloS];               // pw1 output of one adapter
  __shared__ float red[4][C];
  __shared__ bool inside[kHalo];
  const int tid = threadIdx.x;
  const int x0 = bx * kTW, y0 = by * kTH;
  for (int hp = tid; hp < kHalo; hp += 128) {
    const int y = y0 + hp / kHW - 1, x = x0 + hp % kHW - 1;
    const bool in = y >= 0 && y < H && x >= 0 && x < W;
    inside[hp] = in;
    float v[C], n[C];
    load16(F + ((size_t)(in ? y : 0) * W + (in ? x : 0)) * C, v);
    if (!in) {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = 0.f;
    }
    normalise16(v, n);
    float4* dst = reinterpret_cast<float4*>(xh + hp * kXS);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_float4(n[4 * q], n[4 * q + 1], n[4 * q + 2], n[4 * q + 3]);
  }
  const int tx = tid % kTW, ty = tid / kTW;
  const int px = x0 + tx, py = y0 + ty;
  const bool valid = px < W && py < H;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    __syncthreads();
    // pw1 (LN1 affine folded in) on every halo pixel; zero outside the image
    // (the depthwise convolution pads its input with zeros)
    for (int hp = tid; hp < kHalo; hp += 128) {
      float n[C];
      const float4* src = reinterpret_cast<const float4*>(xh + hp * kXS);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 v = src[q];
        n[4 * q] = v.x; n[4 * q + 1] = v.y; n[4 * q + 2] = v.z; n[4 * q + 3] = v.w;
      }
      const bool in = inside[hp];
#pragma unroll
      for (int o = 0; o < 2 * C; ++o) {
        float s = P.b1[a][o];
#pragma unroll
        for (int c = 0; c < C; ++c) s = fmaf(P.w1[a][o][c], n[c], s);
        t[o * kHaloS + hp] = in ? s : 0.f;
      }
    }
    __syncthreads();
    // depthwise 3x3 + simple gate for the inner pixel of this thread
    float g[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float d0 = P.dwb[a][c], d1 = P.dwb[a][c + C];
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const int hp = (ty + ky) * kHW + tx + kx;
          d0 = fmaf(P.dww[a][c][ky * 3 + kx], t[c * kHaloS + hp], d0);
          d1 = fmaf(P.dww[a][c + C][ky * 3 + kx], t[(c + C) * kHaloS + hp], d1);
        }
      g[c] = valid ? d0 * d1 : 0.f;
    }
    if (valid) store16(x1 + ((size_t)py * W + px) * (4 * C) + a * C, g);
    // per-channel sums of this tile: butterfly in each warp, then warps in order
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float v = g[c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      g[c] = v;
    }
    if ((tid & 31) == 0) {
#pragma unroll
      for (int c = 0; c < C; ++c) red[tid >> 5][c] = g[c];
    }
    __syncthreads();
    if (tid < C)
      partial[(size_t)tileid * (4 * C) + a * C + tid] =
          ((red[0][tid] + red[1][tid]) + red[2][tid]) + red[3][tid];
  }
}

template <typename TA>
__global__ void __launch_bounds__(128) adapters_pass1(const TA* __restrict__ F,
                                                      const __grid_constant__ AdapterP1 P,
                                                      TA* __restrict__ x1,
                                                      float* __restrict__ partial, int H, int W) {
  adapters_pass1_tile<TA>(F, P, x1, partial, H, W, blockIdx.x, blockIdx.y,
                          blockIdx.y * gridDim.x + blockIdx.x);
}

// grouped: tiles numbered image after image
template <typename TA>
struct AdapterGroupArgs {
  AdapterImg<TA> img[kMaxGroup];
  int tile_start[kMaxGroup + 1];
  int nimg;
};

// Deterministic reduction of the tile sums (fixed order: strided lane sums,
// then a fixed binary tree); att = W_sca mean + b_sca.
__device__ __forceinline__ void adapters_reduce_body(const float* __restrict__ partial, int ntiles,
                                                     float inv_count, const AdapterSCA& S,
                                                     float* __restrict__ att);

__global__ void __launch_bounds__(1024) adapters_reduce(const float* __restrict__ partial,
                                                        int ntiles, float inv_count,
                                                        const __grid_constant__ AdapterSCA S,
                                                        float* __restrict__ att) {
  adapters_reduce_body(partial, ntiles, inv_count, S, att);
}

// Sum of the pass-1 tile sums of tiles [t0, t1) in a fixed order: 1024 threads
// = 64 tile lanes x 16 channel quads, lane l sums tiles t0 + l, t0 + l + 64, ...
// of quad q (float4 loads, 16 consecutive threads read one 256-byte tile row),
// eight loads in flight; then a fixed binary tree over the 64 lanes.  The
// result is part[0][0..15].
__device__ __forceinline__ void tile_sums(const float* __restrict__ partial, int t0, int t1,
                                          float4 (&part)[64][16]) {
  const int q = threadIdx.x & 15, l = threadIdx.x >> 4;
  const float4* P = reinterpret_cast<const float4*>(partial);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  int t = t0 + l;
  for (; t + 7 * 64 < t1; t += 8 * 64) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = P[(size_t)(t + u * 64) * 16 + q];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s.x += v[u].x; s.y += v[u].y; s.z += v[u].z; s.w += v[u].w;
    }
  }
  for (; t < t1; t += 64) {
    const float4 v = P[(size_t)t * 16 + q];
    s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
  }
  part[l][q] = s;
  __syncthreads();
#pragma unroll
  for (int half = 32; half > 0; half >>= 1) {
    if (l < half) {
      const float4 o = part[l + half][q];
      float4 m = part[l][q];
      m.x += o.x; m.y += o.y; m.z += o.z; m.w += o.w;
      part[l][q] = m;
    }
    __syncthreads();
  }
}

// Channel attention of the four adapters from the channel means: att = W_sca
// mean + b_sca (threads 0 .. 4C-1).
__device__ __forceinline__ void sca_from_mean(const float* mean, const AdapterSCA& S, float* __restrict__ att) {
  if (threadIdx.x < 4 * C) {
    const int a = threadIdx.x / C, co = threadIdx.x % C;
    float v = S.b[a][co];
#pragma unroll
    for (int ci = 0; ci < C; ++ci) v = fmaf(S.w[a][co][ci], mean[a * C + ci], v);
    att[threadIdx.x] = v;
  }
}

__device__ __forceinline__ void adapters_reduce_body(const float* __restrict__ partial, int ntiles,
                                                     float inv_count, const AdapterSCA& S,
                                                     float* __restrict__ att) {
  __shared__ float4 part[64][16];
  __shared__ float mean[4 * C];
  tile_sums(partial, 0, ntiles, part);
  if (threadIdx.x < 16) {
    const float4 m = part[0][threadIdx.x];
    mean[4 * threadIdx.x + 0] = m.x * inv_count;
    mean[4 * threadIdx.x + 1] = m.y * inv_count;
    mean[4 * threadIdx.x + 2] = m.z * inv_count;
    mean[4 * threadIdx.x + 3] = m.w * inv_count;
  }
  __syncthreads();
  sca_from_mean(mean, S, att);
}

// The grouped reduction in two launches that keep the fixed order: kReduceSplit
// CTAs per image each sum a contiguous chunk of tiles (tile_sums) into the
// chunk's first tile slot, then one CTA per image adds the chunk slots in index
// order and applies the channel attention.  (One CTA per image summing every
// tile took 13.7 us on one SM for a 512 x 512 image.)
constexpr int kReduceSplit = 32;
__host__ __device__ __forceinline__ int reduce_chunk(int ntiles) { return (ntiles + kReduceSplit - 1) / kReduceSplit; }

template <typename TA>
__global__ void __launch_bounds__(1024) adapters_reduce_chunks(const __grid_constant__ AdapterGroupArgs<TA> G) {
  pdl_wait();      // the partial sums come from pass 1
  pdl_trigger();
  const int img = blockIdx.y;
  const int ntiles = G.tile_start[img + 1] - G.tile_start[img];
  const int chunk = reduce_chunk(ntiles), t0 = (int)blockIdx.x * chunk;
  if (t0 >= ntiles) return;
  __shared__ float4 part[64][16];
  float* partial = G.img[img].partial;
  tile_sums(partial, t0, min(t0 + chunk, ntiles), part);
  // every read of this chunk is done (tile_sums ends with a barrier)
  if (threadIdx.x < 16) reinterpret_cast<float4*>(partial)[(size_t)t0 * 16 + threadIdx.x] = part[0][threadIdx.x];
}

template <typename TA>
__global__ void __launch_bounds__(16 * kReduceSplit) adapters_reduce_finish(
    const __grid_constant__ AdapterGroupArgs<TA> G, const __grid_constant__ AdapterSCA S) {
  pdl_wait();      // the chunk sums
  pdl_trigger();
  const int img = blockIdx.x;
  const AdapterImg<TA>& im = G.img[img];
  const int ntiles = G.tile_start[img + 1] - G.tile_start[img];
  const int chunk = reduce_chunk(ntiles), nslots = (ntiles + chunk - 1) / chunk;
  __shared__ float4 slot[kReduceSplit][16];
  __shared__ float mean[4 * C];
  // every chunk sum loaded at once (thread = slot x quad), then added in slot order
  const float4* P = reinterpret_cast<const float4*>(im.partial);
  const int q = threadIdx.x & 15, k = threadIdx.x >> 4;
  if (k < nslots) slot[k][q] = P[(size_t)k * chunk * 16 + q];
  __syncthreads();
  if (threadIdx.x < 16) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k2 = 0; k2 < nslots; ++k2) {
      const float4 v = slot[k2][threadIdx.x];
      s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
    const float inv_count = 1.f / ((float)im.H * (float)im.W);
    mean[4 * threadIdx.x + 0] = s.x * inv_count;
    mean[4 * threadIdx.x + 1] = s.y * inv_count;
    mean[4 * threadIdx.x + 2] = s.z * inv_count;
    mean[4 * threadIdx.x + 3] = s.w * inv_count;
  }
  __syncthreads();
  sca_from_mean(mean, S, im.att);
}

// Pass 2: one thread per pixel, the four adapters in turn, output planes.
template <typename TA>
__device__ __forceinline__ void adapters_pass2_pixel(const TA* __restrict__ F,
                                                     const TA* __restrict__ x1, const float* at,
                                                     const AdapterP2& P, float* __restrict__ out,
                                                     int npix, int p);

template <typename TA>
__global__ void __launch_bounds__(128) adapters_pass2(const TA* __restrict__ F,
                                                      const TA* __restrict__ x1,
                                                      const float* __restrict__ att,
                                                      const __grid_constant__ AdapterP2 P,
                                                      float* __restrict__ out, int npix) {
  __shared__ float at[4 * C];
  if (threadIdx.x < 4 * C) at[threadIdx.x] = att[threadIdx.x];
  __syncthreads();
  const int p = blockIdx.x * 128 + threadIdx.x;
  if (p >= npix) return;
  adapters_pass2_pixel<TA>(F, x1, at, P, out, npix, p);
}

template <typename TA>
__device__ __forceinline__ void adapters_pass2_pixel(const TA* __restrict__ F,
                                                     const TA* __restrict__ x1, const float* at,
                                                     const AdapterP2& P, float* __restrict__ out,
                                                     int npix, int p) {
  float f[C];
  load16(F + (size_t)p * C, f);
  constexpr int plane_of[4][2] = {{4, 5}, {0, 1}, {2, 3}, {6, 7}};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float xa[C], y[C], n[C], gs[C];
    load16(x1 + (size_t)p * (4 * C) + a * C, xa);
#pragma unroll
    for (int c = 0; c < C; ++c) xa[c] *= at[a * C + c];
#pragma unroll
    for (int co = 0; co < C; ++co) {
      float s = P.b2[a][co];
#pragma unroll
      for (int ci = 0; ci < C; ++ci) s = fmaf(P.w2[a][co][ci], xa[ci], s);
      y[co] = fmaf(P.beta[a][co], s, f[co]);
    }
    normalise16(y, n);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float s0 = P.fb1[a][c], s1 = P.fb1[a][c + C];
#pragma unroll
      for (int ci = 0; ci < C; ++ci) {
        s0 = fmaf(P.f1[a][c][ci], n[ci], s0);
        s1 = fmaf(P.f1[a][c + C][ci], n[ci], s1);
      }
      gs[c] = s0 * s1;
    }
    float h0 = P.hb[a][0], h1 = P.hb[a][1];
#pragma unroll
    for (int co = 0; co < C; ++co) {
      float s = P.fb2[a][co];
#pragma unroll
      for (int ci = 0; ci < C; ++ci) s = fmaf(P.f2[a][co][ci], gs[ci], s);
      const float z = fmaf(P.gamma[a][co], s, y[co]);
      h0 = fmaf(P.hw[a][0][co], z, h0);
      h1 = fmaf(P.hw[a][1][co], z, h1);
    }
    out[(size_t)plane_of[a][0] * npix + p] = h0;
    out[(size_t)plane_of[a][1] * npix + p] = h1;
  }
}

// Fold the blob's adapter parameters into the kernel parameter blocks.
void adapter_params_from(const float* ap4, AdapterP1* p1, AdapterSCA* sca, AdapterP2* p2) {
  // offsets inside one adapter's parameters (blob order)
  const int ln1w = 0, ln1b = C, pw1w = 2 * C, pw1b = pw1w + 2 * C * C, dww = pw1b + 2 * C,
            dwb = dww + 18 * C, scaw = dwb + 2 * C, scab = scaw + C * C, pw2w = scab + C,
            pw2b = pw2w + C * C, beta = pw2b + C, ln2w = beta + C, ln2b = ln2w + C,
            f1w = ln2b + C, f1b = f1w + 2 * C * C, f2w = f1b + 2 * C, f2b = f2w + C * C,
            gamma = f2b + C, headw = gamma + C, headb = headw + 2 * C;
  for (int a = 0; a < 4; ++a) {
    const float* q = ap4 + (size_t)a * kAdapterParams;
    for (int o = 0; o < 2 * C; ++o) {
      double b = q[pw1b + o];
      for (int c = 0; c < C; ++c) {
        p1->w1[a][o][c] = (float)((double)q[pw1w + o * C + c] * q[ln1w + c]);
        b += (double)q[pw1w + o * C + c] * q[ln1b + c];
      }
      p1->b1[a][o] = (float)b;
      for (int k = 0; k < 9; ++k) p1->dww[a][o][k] = q[dww + o * 9 + k];
      p1->dwb[a][o] = q[dwb + o];
    }
    for (int co = 0; co < C; ++co) {
      sca->b[a][co] = q[scab + co];
      for (int ci = 0; ci < C; ++ci) sca->w[a][co][ci] = q[scaw + co * C + ci];
      p2->b2[a][co] = q[pw2b + co];
      for (int ci = 0; ci < C; ++ci) p2->w2[a][co][ci] = q[pw2w + co * C + ci];
      p2->beta[a][co] = q[beta + co];
      p2->gamma[a][co] = q[gamma + co];
      p2->fb2[a][co] = q[f2b + co];
      for (int ci = 0; ci < C; ++ci) p2->f2[a][co][ci] = q[f2w + co * C + ci];
    }
    for (int o = 0; o < 2 * C; ++o) {
      double b = q[f1b + o];
      for (int c = 0; c < C; ++c) {
        p2->f1[a][o][c] = (float)((double)q[f1w + o * C + c] * q[ln2w + c]);
        b += (double)q[f1w + o * C + c] * q[ln2b + c];
      }
      p2->fb1[a][o] = (float)b;
    }
    for (int k = 0; k < 2; ++k) {
      p2->hb[a][k] = q[headb + k];
      for (int c = 0; c < C; ++c) p2->hw[a][k][c] = q[headw + k * C + c];
    }
  }
}

size_t adapter_partial_floats(int max_w, int max_h) {
  return (size_t)((max_w + kTW - 1) / kTW) * ((max_h + kTH - 1) / kTH) * 4 * C;
}

template <typename TA>
cudaError_t adapters_run(const AdapterParamSet& prm, const TA* F, TA* x1, float* partial,
                         float* att, float* out, int H, int W, cudaStream_t s) {
  dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH);
  adapters_pass1<TA><<<grid, 128, 0, s>>>(F, prm.p1, x1, partial, H, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t P = (size_t)H * W;
  adapters_reduce<<<1, 1024, 0, s>>>(partial, (int)(grid.x * grid.y), 1.f / (float)P, prm.sca, att);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  adapters_pass2<TA><<<(unsigned)((P + 127) / 128), 128, 0, s>>>(F, x1, att, prm.p2, out, (int)P);
  return cudaGetLastError();
}

template <typename TA>
cudaError_t adapters_reduce_only_group(const AdapterParamSet& prm, const AdapterImg<TA>* imgs, int n,
                                       cudaStream_t s) {
  if (n < 1 || n > kMaxGroup) return cudaErrorInvalidValue;
  AdapterGroupArgs<TA> G{};
  G.nimg = n;
  int tiles = 0;
  for (int k = 0; k < n; ++k) {
    G.img[k] = imgs[k];
    G.tile_start[k] = tiles;
    tiles += ((imgs[k].W + kTW - 1) / kTW) * ((imgs[k].H + kTH - 1) / kTH);
  }
  G.tile_start[n] = tiles;
  cudaError_t e = launch_pdl(adapters_reduce_chunks<TA>, dim3(kReduceSplit, n), dim3(1024), 0, s, G);
  if (e != cudaSuccess) return e;
  return launch_pdl(adapters_reduce_finish<TA>, dim3(n), dim3(16 * kReduceSplit), 0, s, G, prm.sca);
}
template cudaError_t adapters_reduce_only_group<__half>(const AdapterParamSet&, const AdapterImg<__half>*,
                                                        int, cudaStream_t);
template cudaError_t adapters_reduce_only_group<__nv_bfloat16>(const AdapterParamSet&,
                                                               const AdapterImg<__nv_bfloat16>*, int,
                                                               cudaStream_t);
template cudaError_t adapters_reduce_only_group<float>(const AdapterParamSet&, const AdapterImg<float>*, int,
                                                       cudaStream_t);


template cudaError_t adapters_run<float>(const AdapterParamSet&, const float*, float*, float*,
                                         float*, float*, int, int, cudaStream_t);

}  // namespace nsl
