// Training slice of Sec. 4.4, restricted to its MSE term: the lightmap network
// (Sec. 4.3) is fitted to fine-step reference lightmaps of synthetic volumes by
// Adam on the mean squared error of its eight output planes.  The forward pass
// keeps every activation, the backward pass is the chain rule layer by layer,
// all in FP32 on the SIMT cores in NCHW layout (B images of one size): training
// is off the per-frame path, so these kernels are written for clarity and
// determinism (no atomics; every reduction in a fixed order), not speed.
#include <cmath>
#include <cstring>
#include <vector>

#include "nsl_internal.cuh"

namespace nsl {
namespace {

constexpr int kT = 256;   // threads per block of the element-wise kernels

inline int blocks_for(size_t n) {
  size_t b = (n + kT - 1) / kT;
  return (int)(b < 65535 * 16 ? b : 65535 * 16);
}

// ---------------------------------------------------------------------------
// convolution k x k (k = 1 or 3, zero padding k / 2), groups, optional ReLU;
// the input may be two tensors concatenated along channels (x1 then x2)
// ---------------------------------------------------------------------------
struct Conv {
  const float* x1;
  const float* x2;     // nullable
  int c1, c2;          // channels of x1 and x2
  const float* w;      // [cout][cin / groups][k][k]
  const float* b;      // [cout]
  int cout, k, groups, relu;
  int B, H, W;
};

__device__ __forceinline__ const float* in_plane(const Conv& p, int bi, int ci) {
  const size_t HW = (size_t)p.H * p.W;
  return ci < p.c1 ? p.x1 + ((size_t)bi * p.c1 + ci) * HW : p.x2 + ((size_t)bi * p.c2 + (ci - p.c1)) * HW;
}

__global__ void conv_fwd(Conv p, float* __restrict__ y) {
  const size_t HW = (size_t)p.H * p.W, n = (size_t)p.B * p.cout * HW;
  const int cin = p.c1 + p.c2, cig = cin / p.groups, cog = p.cout / p.groups, pad = p.k / 2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % p.W), yy = (int)((e / p.W) % p.H);
    const int co = (int)((e / HW) % p.cout), bi = (int)(e / (HW * p.cout));
    const int g = co / cog;
    float acc = p.b[co];
    for (int cl = 0; cl < cig; ++cl) {
      const float* xp = in_plane(p, bi, g * cig + cl);
      const float* wp = p.w + ((size_t)co * cig + cl) * p.k * p.k;
      for (int ky = 0; ky < p.k; ++ky) {
        const int sy = yy + ky - pad;
        if (sy < 0 || sy >= p.H) continue;
        for (int kx = 0; kx < p.k; ++kx) {
          const int sx = x + kx - pad;
          if (sx < 0 || sx >= p.W) continue;
          acc = fmaf(wp[ky * p.k + kx], xp[(size_t)sy * p.W + sx], acc);
        }
      }
    }
    y[e] = p.relu ? fmaxf(acc, 0.f) : acc;
  }
}

// dz = dy * relu'(y) in place (y > 0 exactly where the pre-activation was)
__global__ void relu_bwd(const float* __restrict__ y, float* __restrict__ dy, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    if (!(y[e] > 0.f)) dy[e] = 0.f;
}

// dx (of x1 into dx1, of x2 into dx2) = sum over the group's outputs and taps;
// accumulate: add to what dx holds (a tensor read by several layers)
__global__ void conv_bwd_data(Conv p, const float* __restrict__ dz, float* __restrict__ dx1,
                              float* __restrict__ dx2, int accumulate) {
  const size_t HW = (size_t)p.H * p.W;
  const int cin = p.c1 + p.c2, cig = cin / p.groups, cog = p.cout / p.groups, pad = p.k / 2;
  const size_t n = (size_t)p.B * cin * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % p.W), yy = (int)((e / p.W) % p.H);
    const int ci = (int)((e / HW) % cin), bi = (int)(e / (HW * cin));
    const int g = ci / cig, cl = ci % cig;
    float acc = 0.f;
    for (int oo = 0; oo < cog; ++oo) {
      const int co = g * cog + oo;
      const float* dzp = dz + ((size_t)bi * p.cout + co) * HW;
      const float* wp = p.w + ((size_t)co * cig + cl) * p.k * p.k;
      for (int ky = 0; ky < p.k; ++ky) {
        const int ty = yy - ky + pad;
        if (ty < 0 || ty >= p.H) continue;
        for (int kx = 0; kx < p.k; ++kx) {
          const int tx = x - kx + pad;
          if (tx < 0 || tx >= p.W) continue;
          acc = fmaf(wp[ky * p.k + kx], dzp[(size_t)ty * p.W + tx], acc);
        }
      }
    }
    float* dst = ci < p.c1 ? dx1 + ((size_t)bi * p.c1 + ci) * HW + (size_t)yy * p.W + x
                           : dx2 + ((size_t)bi * p.c2 + (ci - p.c1)) * HW + (size_t)yy * p.W + x;
    *dst = accumulate ? *dst + acc : acc;
  }
}

// Block-wide sum of NV values per thread, fixed order; result in r[] of thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float* sm) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) sm[q * kT + t] = v[q];
  __syncthreads();
  for (int s = kT / 2; s > 0; s >>= 1) {
    if (t < s)
#pragma unroll
      for (int q = 0; q < NV; ++q) sm[q * kT + t] += sm[q * kT + t + s];
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = sm[q * kT];
}

// dW of one (co, cl) pair per block (k*k sums over B x H x W), db with cl = 0
template <int K>
__global__ void __launch_bounds__(kT) conv_bwd_weight(Conv p, const float* __restrict__ dz,
                                                      float* __restrict__ dw, float* __restrict__ db) {
  __shared__ float sm[K * K * kT];
  const size_t HW = (size_t)p.H * p.W;
  const int cin = p.c1 + p.c2, cig = cin / p.groups, cog = p.cout / p.groups, pad = K / 2;
  const int co = blockIdx.x / cig, cl = blockIdx.x % cig, g = co / cog;
  float v[K * K];
#pragma unroll
  for (int q = 0; q < K * K; ++q) v[q] = 0.f;
  float bsum[1] = {0.f};
  for (int bi = 0; bi < p.B; ++bi) {
    const float* xp = in_plane(p, bi, g * cig + cl);
    const float* dzp = dz + ((size_t)bi * p.cout + co) * HW;
    for (size_t e = threadIdx.x; e < HW; e += kT) {
      const int x = (int)(e % p.W), yy = (int)(e / p.W);
      const float d = dzp[e];
      if (cl == 0) bsum[0] += d;
#pragma unroll
      for (int ky = 0; ky < K; ++ky) {
        const int sy = yy + ky - pad;
        if (sy < 0 || sy >= p.H) continue;
#pragma unroll
        for (int kx = 0; kx < K; ++kx) {
          const int sx = x + kx - pad;
          if (sx < 0 || sx >= p.W) continue;
          v[ky * K + kx] = fmaf(d, xp[(size_t)sy * p.W + sx], v[ky * K + kx]);
        }
      }
    }
  }
  block_sum<K * K>(v, sm);
  if (threadIdx.x == 0)
    for (int q = 0; q < K * K; ++q) dw[((size_t)co * cig + cl) * K * K + q] = v[q];
  __syncthreads();
  if (cl == 0) {
    block_sum<1>(bsum, sm);
    if (threadIdx.x == 0) db[co] = bsum[0];
  }
}

// ---------------------------------------------------------------------------
// 2x2 stride-2 transposed convolution, w [cin][cout][2][2]
// ---------------------------------------------------------------------------
struct ConvTr {
  const float* x;   // [B][cin][H][W]
  const float* w;
  const float* b;
  int cin, cout, B, H, W;   // input size; output 2H x 2W
};

__global__ void convt_fwd(ConvTr p, float* __restrict__ y) {
  const int H2 = 2 * p.H, W2 = 2 * p.W;
  const size_t HW = (size_t)p.H * p.W, HW2 = (size_t)H2 * W2, n = (size_t)p.B * p.cout * HW2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % W2), yy = (int)((e / W2) % H2);
    const int co = (int)((e / HW2) % p.cout), bi = (int)(e / (HW2 * p.cout));
    const int a = yy & 1, c = x & 1;
    float acc = p.b[co];
    for (int ci = 0; ci < p.cin; ++ci)
      acc = fmaf(p.w[(((size_t)ci * p.cout + co) * 2 + a) * 2 + c],
                 p.x[((size_t)bi * p.cin + ci) * HW + (size_t)(yy >> 1) * p.W + (x >> 1)], acc);
    y[e] = acc;
  }
}

__global__ void convt_bwd_data(ConvTr p, const float* __restrict__ dy, float* __restrict__ dx) {
  const int W2 = 2 * p.W;
  const size_t HW = (size_t)p.H * p.W, HW2 = 4 * HW, n = (size_t)p.B * p.cin * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % p.W), yy = (int)((e / p.W) % p.H);
    const int ci = (int)((e / HW) % p.cin), bi = (int)(e / (HW * p.cin));
    float acc = 0.f;
    for (int co = 0; co < p.cout; ++co) {
      const float* d = dy + ((size_t)bi * p.cout + co) * HW2;
      const float* w = p.w + ((size_t)ci * p.cout + co) * 4;
      acc = fmaf(w[0], d[(size_t)(2 * yy) * W2 + 2 * x], acc);
      acc = fmaf(w[1], d[(size_t)(2 * yy) * W2 + 2 * x + 1], acc);
      acc = fmaf(w[2], d[(size_t)(2 * yy + 1) * W2 + 2 * x], acc);
      acc = fmaf(w[3], d[(size_t)(2 * yy + 1) * W2 + 2 * x + 1], acc);
    }
    dx[e] = acc;
  }
}

// one (ci, co) pair per block: the four kernel taps; db with ci = 0
__global__ void __launch_bounds__(kT) convt_bwd_weight(ConvTr p, const float* __restrict__ dy,
                                                       float* __restrict__ dw, float* __restrict__ db) {
  __shared__ float sm[4 * kT];
  const int ci = blockIdx.x / p.cout, co = blockIdx.x % p.cout, W2 = 2 * p.W;
  const size_t HW = (size_t)p.H * p.W, HW2 = 4 * HW;
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  float bsum[1] = {0.f};
  for (int bi = 0; bi < p.B; ++bi) {
    const float* xp = p.x + ((size_t)bi * p.cin + ci) * HW;
    const float* d = dy + ((size_t)bi * p.cout + co) * HW2;
    for (size_t e = threadIdx.x; e < HW; e += kT) {
      const int x = (int)(e % p.W), yy = (int)(e / p.W);
      const float xv = xp[e];
      const float d00 = d[(size_t)(2 * yy) * W2 + 2 * x], d01 = d[(size_t)(2 * yy) * W2 + 2 * x + 1];
      const float d10 = d[(size_t)(2 * yy + 1) * W2 + 2 * x], d11 = d[(size_t)(2 * yy + 1) * W2 + 2 * x + 1];
      v[0] = fmaf(d00, xv, v[0]);
      v[1] = fmaf(d01, xv, v[1]);
      v[2] = fmaf(d10, xv, v[2]);
      v[3] = fmaf(d11, xv, v[3]);
      if (ci == 0) bsum[0] += (d00 + d01) + (d10 + d11);
    }
  }
  block_sum<4>(v, sm);
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) dw[((size_t)ci * p.cout + co) * 4 + q] = v[q];
  __syncthreads();
  if (ci == 0) {
    block_sum<1>(bsum, sm);
    if (threadIdx.x == 0) db[co] = bsum[0];
  }
}

// ---------------------------------------------------------------------------
// max-pool 2x2 (the gradient goes to the first maximum in the order (0,0),
// (0,1), (1,0), (1,1)), channel concatenation is handled by the convolutions
// ---------------------------------------------------------------------------
__global__ void pool_fwd(const float* __restrict__ x, float* __restrict__ y, int BC, int H, int W) {
  const int h = H / 2, w = W / 2;
  const size_t n = (size_t)BC * h * w;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int xx = (int)(e % w), yy = (int)((e / w) % h);
    const float* s = x + (e / ((size_t)h * w)) * H * W + (size_t)(2 * yy) * W + 2 * xx;
    y[e] = fmaxf(fmaxf(s[0], s[1]), fmaxf(s[W], s[W + 1]));
  }
}

__global__ void pool_bwd(const float* __restrict__ x, const float* __restrict__ dy, float* __restrict__ dx,
                         int BC, int H, int W, int accumulate) {
  const int h = H / 2, w = W / 2;
  const size_t n = (size_t)BC * h * w;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int xx = (int)(e % w), yy = (int)((e / w) % h);
    const size_t base = (e / ((size_t)h * w)) * H * W + (size_t)(2 * yy) * W + 2 * xx;
    const size_t off[4] = {0, 1, (size_t)W, (size_t)W + 1};
    int arg = 0;
    for (int q = 1; q < 4; ++q)
      if (x[base + off[q]] > x[base + off[arg]]) arg = q;
    for (int q = 0; q < 4; ++q) {
      const float g = q == arg ? dy[e] : 0.f;
      dx[base + off[q]] = accumulate ? dx[base + off[q]] + g : g;
    }
  }
}

// ---------------------------------------------------------------------------
// LayerNorm over the C channels of every pixel (eps 1e-6, affine w, b); the
// forward keeps xhat and 1/sigma for the backward
// ---------------------------------------------------------------------------
__global__ void ln_fwd(const float* __restrict__ x, const float* __restrict__ w, const float* __restrict__ b,
                       float* __restrict__ y, float* __restrict__ xhat, float* __restrict__ rstd, int B, int C,
                       int HW) {
  const size_t n = (size_t)B * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t bi = e / HW, p = e % HW;
    const float* xp = x + bi * C * HW + p;
    float mu = 0.f;
    for (int c = 0; c < C; ++c) mu += xp[(size_t)c * HW];
    mu /= (float)C;
    float var = 0.f;
    for (int c = 0; c < C; ++c) {
      const float d = xp[(size_t)c * HW] - mu;
      var = fmaf(d, d, var);
    }
    var /= (float)C;
    const float r = 1.f / sqrtf(var + 1e-6f);
    rstd[e] = r;
    for (int c = 0; c < C; ++c) {
      const size_t i = bi * C * HW + (size_t)c * HW + p;
      const float xh = (x[i] - mu) * r;
      xhat[i] = xh;
      y[i] = fmaf(w[c], xh, b[c]);
    }
  }
}

// dx = rstd (dxhat - mean_c dxhat - xhat mean_c(dxhat xhat)), dxhat = w dy
__global__ void ln_bwd_data(const float* __restrict__ dy, const float* __restrict__ w,
                            const float* __restrict__ xhat, const float* __restrict__ rstd,
                            float* __restrict__ dx, int B, int C, int HW, int accumulate) {
  const size_t n = (size_t)B * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t bi = e / HW, p = e % HW, base = bi * C * HW + p;
    float m1 = 0.f, m2 = 0.f;
    for (int c = 0; c < C; ++c) {
      const float g = w[c] * dy[base + (size_t)c * HW];
      m1 += g;
      m2 = fmaf(g, xhat[base + (size_t)c * HW], m2);
    }
    m1 /= (float)C;
    m2 /= (float)C;
    for (int c = 0; c < C; ++c) {
      const size_t i = base + (size_t)c * HW;
      const float g = rstd[e] * (w[c] * dy[i] - m1 - xhat[i] * m2);
      dx[i] = accumulate ? dx[i] + g : g;
    }
  }
}

// per channel c (one block each): out1[c] = sum dy a (a = null: sum dy),
// out2[c] (nullable) = sum dy; over every image and pixel
__global__ void __launch_bounds__(kT) chan_dot(const float* __restrict__ dy, const float* __restrict__ a,
                                               float* __restrict__ out1, float* __restrict__ out2, int B, int C,
                                               int HW) {
  __shared__ float sm[2 * kT];
  const int c = blockIdx.x;
  float v[2] = {0.f, 0.f};
  for (int bi = 0; bi < B; ++bi) {
    const size_t base = ((size_t)bi * C + c) * HW;
    for (int p = threadIdx.x; p < HW; p += kT) {
      const float d = dy[base + p];
      v[0] = a ? fmaf(d, a[base + p], v[0]) : v[0] + d;
      v[1] += d;
    }
  }
  block_sum<2>(v, sm);
  if (threadIdx.x == 0) {
    out1[c] = v[0];
    if (out2) out2[c] = v[1];
  }
}

// ---------------------------------------------------------------------------
// NAFBlock pieces: simple gate, channel mean, channel scaling, scaled residual
// ---------------------------------------------------------------------------
// g[b][c] = v[b][c] * v[b][c + C]   (v has 2C channels)
__global__ void gate_fwd(const float* __restrict__ v, float* __restrict__ g, int B, int C, int HW) {
  const size_t n = (size_t)B * C * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t bi = e / ((size_t)C * HW), r = e % ((size_t)C * HW);
    const float* vb = v + bi * 2 * C * HW;
    g[e] = vb[r] * vb[(size_t)C * HW + r];
  }
}

__global__ void gate_bwd(const float* __restrict__ v, const float* __restrict__ dg, float* __restrict__ dv, int B,
                         int C, int HW) {
  const size_t n = (size_t)B * C * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t bi = e / ((size_t)C * HW), r = e % ((size_t)C * HW);
    const float* vb = v + bi * 2 * C * HW;
    float* db = dv + bi * 2 * C * HW;
    db[r] = dg[e] * vb[(size_t)C * HW + r];
    db[(size_t)C * HW + r] = dg[e] * vb[r];
  }
}

// m[b][c] = mean over the pixels of x[b][c] (one block per (b, c))
__global__ void __launch_bounds__(kT) chan_mean(const float* __restrict__ x, float* __restrict__ m, int HW) {
  __shared__ float sm[kT];
  const float* xp = x + (size_t)blockIdx.x * HW;
  float v[1] = {0.f};
  for (int p = threadIdx.x; p < HW; p += kT) v[0] += xp[p];
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) m[blockIdx.x] = v[0] / (float)HW;
}

// y[b][c][p] = x[b][c][p] * s[b][c] (+ acc: y holds a sum to add to)
__global__ void chan_scale(const float* __restrict__ x, const float* __restrict__ s, float* __restrict__ y,
                           size_t BC, int HW, int accumulate) {
  const size_t n = BC * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float v = x[e] * s[e / HW];
    y[e] = accumulate ? y[e] + v : v;
  }
}

// d s[b][c] = sum over pixels of dy x (one block per (b, c)), plus, for the
// channel mean's backward, dx[b][c][p] += dm[b][c] / HW
__global__ void __launch_bounds__(kT) chan_scale_bwd(const float* __restrict__ dy, const float* __restrict__ x,
                                                     float* __restrict__ ds, int HW) {
  __shared__ float sm[kT];
  const size_t base = (size_t)blockIdx.x * HW;
  float v[1] = {0.f};
  for (int p = threadIdx.x; p < HW; p += kT) v[0] = fmaf(dy[base + p], x[base + p], v[0]);
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) ds[blockIdx.x] = v[0];
}

__global__ void add_mean_grad(const float* __restrict__ dm, float* __restrict__ dx, size_t BC, int HW) {
  const size_t n = BC * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dx[e] += dm[e / HW] / (float)HW;
}

// y = x + s[c] * k   (per-channel scale s shared by every image)
__global__ void scaled_residual(const float* __restrict__ x, const float* __restrict__ s,
                                const float* __restrict__ k, float* __restrict__ y, int C, int HW, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = fmaf(s[(e / HW) % C], k[e], x[e]);
}

// dk = s[c] dy
__global__ void chan_mul(const float* __restrict__ dy, const float* __restrict__ s, float* __restrict__ dk, int C,
                         int HW, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dk[e] = s[(e / HW) % C] * dy[e];
}

__global__ void axpy_kernel(const float* __restrict__ x, float* __restrict__ y, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] += x[e];
}

// ---------------------------------------------------------------------------
// input, loss, optimiser
// ---------------------------------------------------------------------------
// x0 = the guide with its depth channel scaled (every image of the batch)
__global__ void guide_input(const float* __restrict__ g, float* __restrict__ x0, float ds, int B, int HW) {
  const size_t n = (size_t)B * 3 * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    x0[e] = ((e / HW) % 3) == 2 ? g[e] * ds : g[e];
}

// planes [B][8][H][W] from the four heads' [B][2][H][W] outputs (F&B -> 4, 5;
// L&R -> 0, 1; U&D -> 2, 3; A&E -> 6, 7), and the planes' gradient back
__constant__ int c_plane_of[4][2] = {{4, 5}, {0, 1}, {2, 3}, {6, 7}};
__device__ __forceinline__ size_t plane_index(size_t e, int a, int HW) {
  const size_t bi = e / (2 * (size_t)HW), oc = (e / HW) % 2, p = e % HW;
  return (bi * 8 + c_plane_of[a][oc]) * HW + p;
}
__global__ void planes_from_head(const float* __restrict__ h, float* __restrict__ o, int a, int B, int HW) {
  const size_t n = (size_t)B * 2 * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    o[plane_index(e, a, HW)] = h[e];
}
__global__ void head_from_planes(const float* __restrict__ o, float* __restrict__ h, int a, int B, int HW) {
  const size_t n = (size_t)B * 2 * HW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    h[e] = o[plane_index(e, a, HW)];
}

// per-block partial sums of w_p (o - t)^2 and d o = 2 w_p (o - t) / n, with
// p = the plane of element e ([B][8][HW] layout)
struct PlaneWeights {
  float w[8];
};
__global__ void __launch_bounds__(kT) mse_loss(const float* __restrict__ o, const float* __restrict__ t,
                                               float* __restrict__ d, float* __restrict__ partial, size_t n,
                                               int HW, PlaneWeights pw) {
  __shared__ float sm[kT];
  float v[1] = {0.f};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float r = o[e] - t[e], w = pw.w[(e / HW) % 8];
    v[0] = fmaf(w * r, r, v[0]);
    d[e] = 2.f * w * r / (float)n;
  }
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = v[0];
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = fmaf(b1, m[e], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[e], (1.f - b2) * gi * gi);
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace
}  // namespace nsl

// ---------------------------------------------------------------------------
// host side: activations (value and gradient of every stored tensor), the
// forward with everything kept, the backward, Adam
// ---------------------------------------------------------------------------
namespace nsl {
namespace {

struct Act {           // one stored tensor and its gradient
  float* v = nullptr;
  float* g = nullptr;
  size_t n = 0;
};

struct AdapterActs {
  Act ln1, u, v, g, m, att, h, k, y, ln2, e, q, r, z, hd;
  float *ln1_xh = nullptr, *ln1_rs = nullptr, *ln2_xh = nullptr, *ln2_rs = nullptr;
};

}  // namespace
}  // namespace nsl

struct nsl_trainer {
  nsl_train_opts o{};
  int c0 = 16;
  nsl::NetLayout L{};
  size_t np = 0;
  float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // parameters and Adam state
  int t = 0;                                                         // Adam steps taken
  // activations
  nsl::Act x0, a0, s1, p1, a1, s2, p2, a2, s3, p3, a3, bt, u3, d3a, d3b, u2, d2a, d2b, u1, d1a, F, out;
  nsl::AdapterActs ad[4];
  float* partial = nullptr;     // loss partial sums [kLossBlocks]
  float* partial_host = nullptr;
  std::vector<void*> allocs;
};

namespace nsl {
namespace {

constexpr int kLossBlocks = 256;

cudaError_t alloc_f(nsl_trainer* T, float** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (n ? n : 1) * sizeof(float));
  if (e == cudaSuccess) T->allocs.push_back(q);
  *p = static_cast<float*>(q);
  return e;
}

cudaError_t alloc_act(nsl_trainer* T, Act* a, size_t n) {
  a->n = n;
  cudaError_t e = alloc_f(T, &a->v, n);
  if (e == cudaSuccess) e = alloc_f(T, &a->g, n);
  return e;
}

Conv conv_of(const float* x1, int c1, const float* x2, int c2, const float* w, const float* b, int cout, int k,
             int groups, int relu, int B, int H, int W) {
  return Conv{x1, x2, c1, c2, w, b, cout, k, groups, relu, B, H, W};
}

cudaError_t run_conv_fwd(const Conv& c, float* y, cudaStream_t s) {
  conv_fwd<<<blocks_for((size_t)c.B * c.cout * c.H * c.W), kT, 0, s>>>(c, y);
  return cudaGetLastError();
}

// backward of one convolution whose output (post-ReLU) is y and whose output
// gradient sits in dy (modified in place by the ReLU): weight and bias
// gradients into gw, gb; input gradients into dx1, dx2 (nullable: not needed)
cudaError_t run_conv_bwd(const Conv& c, const float* y, float* dy, float* gw, float* gb, float* dx1, float* dx2,
                         int accumulate, cudaStream_t s) {
  const size_t nout = (size_t)c.B * c.cout * c.H * c.W;
  if (c.relu) relu_bwd<<<blocks_for(nout), kT, 0, s>>>(y, dy, nout);
  const int cig = (c.c1 + c.c2) / c.groups;
  if (c.k == 3) conv_bwd_weight<3><<<c.cout * cig, kT, 0, s>>>(c, dy, gw, gb);
  else conv_bwd_weight<1><<<c.cout * cig, kT, 0, s>>>(c, dy, gw, gb);
  if (dx1) {
    const size_t nin = (size_t)c.B * (c.c1 + c.c2) * c.H * c.W;
    conv_bwd_data<<<blocks_for(nin), kT, 0, s>>>(c, dy, dx1, dx2, accumulate);
  }
  return cudaGetLastError();
}

// parameter offsets of adapter a (blob order of the NAFBlock, then its head)
struct AdOff {
  size_t ln1w, ln1b, pw1w, pw1b, dww, dwb, scaw, scab, pw2w, pw2b, beta, ln2w, ln2b, f1w, f1b, f2w, f2b, gamma,
      hw, hb;
};
AdOff adapter_offsets(const NetLayout& L, int a, int C) {
  AdOff o{};
  size_t q = L.adapter[a];
  auto take = [&](size_t n) { size_t r = q; q += n; return r; };
  o.ln1w = take(C); o.ln1b = take(C);
  o.pw1w = take(2 * C * C); o.pw1b = take(2 * C);
  o.dww = take(2 * C * 9); o.dwb = take(2 * C);
  o.scaw = take(C * C); o.scab = take(C);
  o.pw2w = take(C * C); o.pw2b = take(C);
  o.beta = take(C);
  o.ln2w = take(C); o.ln2b = take(C);
  o.f1w = take(2 * C * C); o.f1b = take(2 * C);
  o.f2w = take(C * C); o.f2b = take(C);
  o.gamma = take(C);
  o.hw = take(2 * C); o.hb = take(2);
  return o;
}

cudaError_t forward(nsl_trainer* T, const float* guides, float ds, cudaStream_t s) {
  const int B = T->o.batch, H = T->o.height, W = T->o.width, c = T->c0;
  const NetLayout& L = T->L;
  const float* P = T->p;
  const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  cudaError_t e;
#define TRY(x) if ((e = (x)) != cudaSuccess) return e
  guide_input<<<blocks_for((size_t)B * 3 * H * W), kT, 0, s>>>(guides, T->x0.v, ds, B, H * W);
  auto cv = [&](const Act& x1, int c1, const Act* x2, int c2, int l, int cout, int h, int w, Act& y) {
    return run_conv_fwd(conv_of(x1.v, c1, x2 ? x2->v : nullptr, c2, P + L.conv_w[l], P + L.conv_b[l], cout, 3, 1, 1,
                                B, h, w), y.v, s);
  };
  auto up = [&](const Act& x, int l, int h, int w, Act& y) {
    ConvTr t{x.v, P + L.up_w[l], P + L.up_b[l], L.up_cin[l], L.up_cout[l], B, h, w};
    convt_fwd<<<blocks_for((size_t)B * t.cout * 4 * h * w), kT, 0, s>>>(t, y.v);
    return cudaGetLastError();
  };
  auto pool = [&](const Act& x, int C, int h, int w, Act& y) {
    pool_fwd<<<blocks_for((size_t)B * C * h * w / 4), kT, 0, s>>>(x.v, y.v, B * C, h, w);
    return cudaGetLastError();
  };
  TRY(cv(T->x0, 3, nullptr, 0, 0, c, H, W, T->a0));
  TRY(cv(T->a0, c, nullptr, 0, 1, c, H, W, T->s1));
  TRY(pool(T->s1, c, H, W, T->p1));
  TRY(cv(T->p1, c, nullptr, 0, 2, 2 * c, H1, W1, T->a1));
  TRY(cv(T->a1, 2 * c, nullptr, 0, 3, 2 * c, H1, W1, T->s2));
  TRY(pool(T->s2, 2 * c, H1, W1, T->p2));
  TRY(cv(T->p2, 2 * c, nullptr, 0, 4, 4 * c, H2, W2, T->a2));
  TRY(cv(T->a2, 4 * c, nullptr, 0, 5, 4 * c, H2, W2, T->s3));
  TRY(pool(T->s3, 4 * c, H2, W2, T->p3));
  TRY(cv(T->p3, 4 * c, nullptr, 0, 6, 8 * c, H3, W3, T->a3));
  TRY(cv(T->a3, 8 * c, nullptr, 0, 7, 8 * c, H3, W3, T->bt));
  TRY(up(T->bt, 0, H3, W3, T->u3));
  TRY(cv(T->u3, 4 * c, &T->s3, 4 * c, 8, 4 * c, H2, W2, T->d3a));
  TRY(cv(T->d3a, 4 * c, nullptr, 0, 9, 4 * c, H2, W2, T->d3b));
  TRY(up(T->d3b, 1, H2, W2, T->u2));
  TRY(cv(T->u2, 2 * c, &T->s2, 2 * c, 10, 2 * c, H1, W1, T->d2a));
  TRY(cv(T->d2a, 2 * c, nullptr, 0, 11, 2 * c, H1, W1, T->d2b));
  TRY(up(T->d2b, 2, H1, W1, T->u1));
  TRY(cv(T->u1, c, &T->s1, c, 12, c, H, W, T->d1a));
  TRY(cv(T->d1a, c, nullptr, 0, 13, c, H, W, T->F));
  // the four adapters and their heads
  const int HW = H * W;
  const size_t nc = (size_t)B * c * HW;
  for (int a = 0; a < 4; ++a) {
    AdapterActs& A = T->ad[a];
    const AdOff q = adapter_offsets(L, a, c);
    auto c1x1 = [&](const Act& x, int cin, size_t w, size_t b, int cout, Act& y, int h = 0, int ww = 0) {
      return run_conv_fwd(conv_of(x.v, cin, nullptr, 0, P + w, P + b, cout, 1, 1, 0, B, h ? h : H, ww ? ww : W),
                          y.v, s);
    };
    ln_fwd<<<blocks_for((size_t)B * HW), kT, 0, s>>>(T->F.v, P + q.ln1w, P + q.ln1b, A.ln1.v, A.ln1_xh, A.ln1_rs,
                                                     B, c, HW);
    TRY(c1x1(A.ln1, c, q.pw1w, q.pw1b, 2 * c, A.u));
    TRY(run_conv_fwd(conv_of(A.u.v, 2 * c, nullptr, 0, P + q.dww, P + q.dwb, 2 * c, 3, 2 * c, 0, B, H, W), A.v.v, s));
    gate_fwd<<<blocks_for(nc), kT, 0, s>>>(A.v.v, A.g.v, B, c, HW);
    chan_mean<<<B * c, kT, 0, s>>>(A.g.v, A.m.v, HW);
    TRY(c1x1(A.m, c, q.scaw, q.scab, c, A.att, 1, 1));
    chan_scale<<<blocks_for(nc), kT, 0, s>>>(A.g.v, A.att.v, A.h.v, (size_t)B * c, HW, 0);
    TRY(c1x1(A.h, c, q.pw2w, q.pw2b, c, A.k));
    scaled_residual<<<blocks_for(nc), kT, 0, s>>>(T->F.v, P + q.beta, A.k.v, A.y.v, c, HW, nc);
    ln_fwd<<<blocks_for((size_t)B * HW), kT, 0, s>>>(A.y.v, P + q.ln2w, P + q.ln2b, A.ln2.v, A.ln2_xh, A.ln2_rs,
                                                     B, c, HW);
    TRY(c1x1(A.ln2, c, q.f1w, q.f1b, 2 * c, A.e));
    gate_fwd<<<blocks_for(nc), kT, 0, s>>>(A.e.v, A.q.v, B, c, HW);
    TRY(c1x1(A.q, c, q.f2w, q.f2b, c, A.r));
    scaled_residual<<<blocks_for(nc), kT, 0, s>>>(A.y.v, P + q.gamma, A.r.v, A.z.v, c, HW, nc);
    TRY(c1x1(A.z, c, q.hw, q.hb, 2, A.hd));
    planes_from_head<<<blocks_for((size_t)B * 2 * HW), kT, 0, s>>>(A.hd.v, T->out.v, a, B, HW);
  }
#undef TRY
  return cudaGetLastError();
}

// Backward from d out (in T->out.g) to every parameter gradient (T->grad).
cudaError_t backward(nsl_trainer* T, cudaStream_t s) {
  const int B = T->o.batch, H = T->o.height, W = T->o.width, c = T->c0, HW = H * W;
  const NetLayout& L = T->L;
  const float* P = T->p;
  float* G = T->grad;
  const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  const size_t nc = (size_t)B * c * HW;
  cudaError_t e;
#define TRY(x) if ((e = (x)) != cudaSuccess) return e
  // adapters: dF accumulates over the four adapters and their two paths
  for (int a = 0; a < 4; ++a) {
    AdapterActs& A = T->ad[a];
    const AdOff q = adapter_offsets(L, a, c);
    auto c1x1 = [&](const Act& x, int cin, size_t w, size_t b, int cout, int h = 0, int ww = 0) {
      return conv_of(x.v, cin, nullptr, 0, P + w, P + b, cout, 1, 1, 0, B, h ? h : H, ww ? ww : W);
    };
    head_from_planes<<<blocks_for((size_t)B * 2 * HW), kT, 0, s>>>(T->out.g, A.hd.g, a, B, HW);
    TRY(run_conv_bwd(c1x1(A.z, c, q.hw, q.hb, 2), A.hd.v, A.hd.g, G + q.hw, G + q.hb, A.z.g, nullptr, 0, s));
    // z = y + gamma r
    chan_dot<<<c, kT, 0, s>>>(A.z.g, A.r.v, G + q.gamma, nullptr, B, c, HW);
    chan_mul<<<blocks_for(nc), kT, 0, s>>>(A.z.g, P + q.gamma, A.r.g, c, HW, nc);
    TRY(cudaMemcpyAsync(A.y.g, A.z.g, nc * sizeof(float), cudaMemcpyDeviceToDevice, s));
    // r = ffn2(q), q = gate(e), e = ffn1(ln2)
    TRY(run_conv_bwd(c1x1(A.q, c, q.f2w, q.f2b, c), A.r.v, A.r.g, G + q.f2w, G + q.f2b, A.q.g, nullptr, 0, s));
    gate_bwd<<<blocks_for(nc), kT, 0, s>>>(A.e.v, A.q.g, A.e.g, B, c, HW);
    TRY(run_conv_bwd(c1x1(A.ln2, c, q.f1w, q.f1b, 2 * c), A.e.v, A.e.g, G + q.f1w, G + q.f1b, A.ln2.g, nullptr, 0,
                     s));
    chan_dot<<<c, kT, 0, s>>>(A.ln2.g, A.ln2_xh, G + q.ln2w, G + q.ln2b, B, c, HW);
    ln_bwd_data<<<blocks_for((size_t)B * HW), kT, 0, s>>>(A.ln2.g, P + q.ln2w, A.ln2_xh, A.ln2_rs, A.y.g, B, c, HW,
                                                          1);
    // y = F + beta k
    if (a == 0) {
      TRY(cudaMemcpyAsync(T->F.g, A.y.g, nc * sizeof(float), cudaMemcpyDeviceToDevice, s));
    } else {
      axpy_kernel<<<blocks_for(nc), kT, 0, s>>>(A.y.g, T->F.g, nc);
    }
    chan_dot<<<c, kT, 0, s>>>(A.y.g, A.k.v, G + q.beta, nullptr, B, c, HW);
    chan_mul<<<blocks_for(nc), kT, 0, s>>>(A.y.g, P + q.beta, A.k.g, c, HW, nc);
    // k = pw2(h), h = g * att, att = sca(mean g)
    TRY(run_conv_bwd(c1x1(A.h, c, q.pw2w, q.pw2b, c), A.k.v, A.k.g, G + q.pw2w, G + q.pw2b, A.h.g, nullptr, 0, s));
    chan_scale<<<blocks_for(nc), kT, 0, s>>>(A.h.g, A.att.v, A.g.g, (size_t)B * c, HW, 0);
    chan_scale_bwd<<<B * c, kT, 0, s>>>(A.h.g, A.g.v, A.att.g, HW);
    TRY(run_conv_bwd(c1x1(A.m, c, q.scaw, q.scab, c, 1, 1), A.att.v, A.att.g, G + q.scaw, G + q.scab, A.m.g,
                     nullptr, 0, s));
    add_mean_grad<<<blocks_for(nc), kT, 0, s>>>(A.m.g, A.g.g, (size_t)B * c, HW);
    // g = gate(v), v = dw3x3(u), u = pw1(ln1), ln1 = LN(F)
    gate_bwd<<<blocks_for(nc), kT, 0, s>>>(A.v.v, A.g.g, A.v.g, B, c, HW);
    TRY(run_conv_bwd(conv_of(A.u.v, 2 * c, nullptr, 0, P + q.dww, P + q.dwb, 2 * c, 3, 2 * c, 0, B, H, W), A.v.v,
                     A.v.g, G + q.dww, G + q.dwb, A.u.g, nullptr, 0, s));
    TRY(run_conv_bwd(c1x1(A.ln1, c, q.pw1w, q.pw1b, 2 * c), A.u.v, A.u.g, G + q.pw1w, G + q.pw1b, A.ln1.g, nullptr,
                     0, s));
    chan_dot<<<c, kT, 0, s>>>(A.ln1.g, A.ln1_xh, G + q.ln1w, G + q.ln1b, B, c, HW);
    ln_bwd_data<<<blocks_for((size_t)B * HW), kT, 0, s>>>(A.ln1.g, P + q.ln1w, A.ln1_xh, A.ln1_rs, T->F.g, B, c, HW,
                                                          1);
  }
  // UNet decoder and encoder
  auto cv = [&](const Act& x1, int c1, const Act* x2, int c2, int l, int cout, int h, int w) {
    return conv_of(x1.v, c1, x2 ? x2->v : nullptr, c2, P + L.conv_w[l], P + L.conv_b[l], cout, 3, 1, 1, B, h, w);
  };
  auto upb = [&](const Act& x, int l, int h, int w, Act& y, Act& dx) {
    ConvTr t{x.v, P + L.up_w[l], P + L.up_b[l], L.up_cin[l], L.up_cout[l], B, h, w};
    convt_bwd_weight<<<t.cin * t.cout, kT, 0, s>>>(t, y.g, G + L.up_w[l], G + L.up_b[l]);
    convt_bwd_data<<<blocks_for((size_t)B * t.cin * h * w), kT, 0, s>>>(t, y.g, dx.g);
    return cudaGetLastError();
  };
  auto poolb = [&](const Act& x, const Act& y, int C, int h, int w) {
    pool_bwd<<<blocks_for((size_t)B * C * h * w / 4), kT, 0, s>>>(x.v, y.g, x.g, B * C, h, w, 1);
    return cudaGetLastError();
  };
  auto wg = [&](int l) { return G + L.conv_w[l]; };
  auto bg = [&](int l) { return G + L.conv_b[l]; };
  TRY(run_conv_bwd(cv(T->d1a, c, nullptr, 0, 13, c, H, W), T->F.v, T->F.g, wg(13), bg(13), T->d1a.g, nullptr, 0, s));
  TRY(run_conv_bwd(cv(T->u1, c, &T->s1, c, 12, c, H, W), T->d1a.v, T->d1a.g, wg(12), bg(12), T->u1.g, T->s1.g, 0,
                   s));
  TRY(upb(T->d2b, 2, H1, W1, T->u1, T->d2b));
  TRY(run_conv_bwd(cv(T->d2a, 2 * c, nullptr, 0, 11, 2 * c, H1, W1), T->d2b.v, T->d2b.g, wg(11), bg(11), T->d2a.g,
                   nullptr, 0, s));
  TRY(run_conv_bwd(cv(T->u2, 2 * c, &T->s2, 2 * c, 10, 2 * c, H1, W1), T->d2a.v, T->d2a.g, wg(10), bg(10),
                   T->u2.g, T->s2.g, 0, s));
  TRY(upb(T->d3b, 1, H2, W2, T->u2, T->d3b));
  TRY(run_conv_bwd(cv(T->d3a, 4 * c, nullptr, 0, 9, 4 * c, H2, W2), T->d3b.v, T->d3b.g, wg(9), bg(9), T->d3a.g,
                   nullptr, 0, s));
  TRY(run_conv_bwd(cv(T->u3, 4 * c, &T->s3, 4 * c, 8, 4 * c, H2, W2), T->d3a.v, T->d3a.g, wg(8), bg(8), T->u3.g,
                   T->s3.g, 0, s));
  TRY(upb(T->bt, 0, H3, W3, T->u3, T->bt));
  TRY(run_conv_bwd(cv(T->a3, 8 * c, nullptr, 0, 7, 8 * c, H3, W3), T->bt.v, T->bt.g, wg(7), bg(7), T->a3.g, nullptr,
                   0, s));
  TRY(run_conv_bwd(cv(T->p3, 4 * c, nullptr, 0, 6, 8 * c, H3, W3), T->a3.v, T->a3.g, wg(6), bg(6), T->p3.g, nullptr,
                   0, s));
  TRY(poolb(T->s3, T->p3, 4 * c, H2, W2));
  TRY(run_conv_bwd(cv(T->a2, 4 * c, nullptr, 0, 5, 4 * c, H2, W2), T->s3.v, T->s3.g, wg(5), bg(5), T->a2.g, nullptr,
                   0, s));
  TRY(run_conv_bwd(cv(T->p2, 2 * c, nullptr, 0, 4, 4 * c, H2, W2), T->a2.v, T->a2.g, wg(4), bg(4), T->p2.g, nullptr,
                   0, s));
  TRY(poolb(T->s2, T->p2, 2 * c, H1, W1));
  TRY(run_conv_bwd(cv(T->a1, 2 * c, nullptr, 0, 3, 2 * c, H1, W1), T->s2.v, T->s2.g, wg(3), bg(3), T->a1.g, nullptr,
                   0, s));
  TRY(run_conv_bwd(cv(T->p1, c, nullptr, 0, 2, 2 * c, H1, W1), T->a1.v, T->a1.g, wg(2), bg(2), T->p1.g, nullptr, 0,
                   s));
  TRY(poolb(T->s1, T->p1, c, H, W));
  TRY(run_conv_bwd(cv(T->a0, c, nullptr, 0, 1, c, H, W), T->s1.v, T->s1.g, wg(1), bg(1), T->a0.g, nullptr, 0, s));
  TRY(run_conv_bwd(cv(T->x0, 3, nullptr, 0, 0, c, H, W), T->a0.v, T->a0.g, wg(0), bg(0), nullptr, nullptr, 0, s));
#undef TRY
  return cudaGetLastError();
}

}  // namespace
}  // namespace nsl

using namespace nsl;

extern "C" {

void nsl_default_train_opts(nsl_train_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->batch = 4;
  o->width = 64;
  o->height = 64;
  o->lr = 1e-3f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  for (int k = 0; k < 8; ++k) o->plane_weight[k] = 1.f;
}

void nsl_trainer_destroy(nsl_trainer* T) {
  if (!T) return;
  cudaDeviceSynchronize();
  for (void* p : T->allocs) cudaFree(p);
  if (T->partial_host) cudaFreeHost(T->partial_host);
  delete T;
}

nsl_status nsl_trainer_create(const void* blob, size_t blob_bytes, const nsl_train_opts* opts, nsl_trainer** out) {
  static const char* fn = "nsl_trainer_create";
  if (!out) return fail(NSL_ERR_INVALID_ARG, "%s: out is NULL", fn);
  *out = nullptr;
  nsl_train_opts o;
  nsl_default_train_opts(&o);
  if (opts) o = *opts;
  if (o.batch < 1 || o.batch > 64 || o.width < 8 || o.height < 8 || o.width % 8 || o.height % 8 ||
      (size_t)o.width * o.height > (size_t)512 * 512)
    return fail(NSL_ERR_INVALID_ARG, "%s: batch 1..64, width and height multiples of 8 with at most 512^2 pixels", fn);
  if (!(o.lr > 0.f) || !(o.beta1 >= 0.f && o.beta1 < 1.f) || !(o.beta2 >= 0.f && o.beta2 < 1.f) || !(o.eps > 0.f))
    return fail(NSL_ERR_INVALID_ARG, "%s: bad optimiser settings", fn);
  for (int k = 0; k < 8; ++k)
    if (!(o.plane_weight[k] >= 0.f) || !std::isfinite(o.plane_weight[k]))
      return fail(NSL_ERR_INVALID_ARG, "%s: plane weights must be finite and >= 0", fn);
  if (!blob || blob_bytes < 20) return fail(NSL_ERR_INVALID_ARG, "%s: bad blob", fn);
  const unsigned char* bb = static_cast<const unsigned char*>(blob);
  uint32_t ver, c0, nf;
  if (std::memcmp(bb, "NSLW", 4) != 0) return fail(NSL_ERR_INVALID_ARG, "%s: bad magic", fn);
  std::memcpy(&ver, bb + 4, 4);
  std::memcpy(&c0, bb + 8, 4);
  std::memcpy(&nf, bb + 12, 4);
  if (ver != 1 || (size_t)nf * 4 + 20 != blob_bytes)
    return fail(NSL_ERR_INVALID_ARG, "%s: blob version or size mismatch", fn);
  NetLayout L{};
  if (!build_net_layout((int)c0, &L) || L.c0 != kC0)
    return fail(NSL_ERR_UNSUPPORTED, "%s: C0=%u (the trainer runs C0=16)", fn, c0);
  if (L.total != nf) return fail(NSL_ERR_INVALID_ARG, "%s: parameter count", fn);
  nsl_trainer* T = new nsl_trainer();
  T->o = o;
  T->c0 = (int)c0;
  T->L = L;
  T->np = nf;
  const int B = o.batch, c = T->c0;
  const size_t P0 = (size_t)o.width * o.height, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  cudaError_t e = cudaSuccess;
  auto A = [&](Act* a, size_t n) { if (e == cudaSuccess) e = alloc_act(T, a, n); };
  auto F_ = [&](float** p, size_t n) { if (e == cudaSuccess) e = alloc_f(T, p, n); };
  F_(&T->p, nf); F_(&T->grad, nf); F_(&T->m, nf); F_(&T->v, nf);
  A(&T->x0, B * 3 * P0);
  A(&T->a0, B * c * P0); A(&T->s1, B * c * P0); A(&T->p1, B * c * P1);
  A(&T->a1, B * 2 * c * P1); A(&T->s2, B * 2 * c * P1); A(&T->p2, B * 2 * c * P2);
  A(&T->a2, B * 4 * c * P2); A(&T->s3, B * 4 * c * P2); A(&T->p3, B * 4 * c * P3);
  A(&T->a3, B * 8 * c * P3); A(&T->bt, B * 8 * c * P3);
  A(&T->u3, B * 4 * c * P2); A(&T->d3a, B * 4 * c * P2); A(&T->d3b, B * 4 * c * P2);
  A(&T->u2, B * 2 * c * P1); A(&T->d2a, B * 2 * c * P1); A(&T->d2b, B * 2 * c * P1);
  A(&T->u1, B * c * P0); A(&T->d1a, B * c * P0); A(&T->F, B * c * P0);
  A(&T->out, B * 8 * P0);
  for (int a = 0; a < 4; ++a) {
    AdapterActs& D = T->ad[a];
    const size_t nc = B * c * P0;
    A(&D.ln1, nc); A(&D.u, 2 * nc); A(&D.v, 2 * nc); A(&D.g, nc); A(&D.m, (size_t)B * c); A(&D.att, (size_t)B * c);
    A(&D.h, nc); A(&D.k, nc); A(&D.y, nc); A(&D.ln2, nc); A(&D.e, 2 * nc); A(&D.q, nc); A(&D.r, nc);
    A(&D.z, nc); A(&D.hd, B * 2 * P0);
    F_(&D.ln1_xh, nc); F_(&D.ln1_rs, B * P0); F_(&D.ln2_xh, nc); F_(&D.ln2_rs, B * P0);
  }
  F_(&T->partial, kLossBlocks);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&T->partial_host), kLossBlocks * sizeof(float),
                                          cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMemcpy(T->p, bb + 16, (size_t)nf * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(T->m, 0, (size_t)nf * 4);
  if (e == cudaSuccess) e = cudaMemset(T->v, 0, (size_t)nf * 4);
  if (e != cudaSuccess) {
    nsl_trainer_destroy(T);
    return e == cudaErrorMemoryAllocation ? fail(NSL_ERR_OOM, "%s: out of device memory", fn) : cuda_fail(e, fn);
  }
  *out = T;
  return NSL_OK;
}

nsl_status nsl_trainer_step(nsl_trainer* T, const float* guides, const float* targets, float depth_scale,
                            int update, float* loss_out, void* stream) {
  static const char* fn = "nsl_trainer_step";
  if (!T || !guides || !targets) return fail(NSL_ERR_INVALID_ARG, "%s: NULL argument", fn);
  if (!(depth_scale > 0.f) || !std::isfinite(depth_scale))
    return fail(NSL_ERR_INVALID_ARG, "%s: depth_scale must be > 0", fn);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = forward(T, guides, depth_scale, s);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  const size_t n = T->out.n;
  PlaneWeights pw;
  for (int k = 0; k < 8; ++k) pw.w[k] = T->o.plane_weight[k];
  mse_loss<<<kLossBlocks, kT, 0, s>>>(T->out.v, targets, T->out.g, T->partial, n, T->o.width * T->o.height, pw);
  if ((e = backward(T, s)) != cudaSuccess) return cuda_fail(e, fn);
  if (update) {
    ++T->t;
    const float c1 = 1.f - std::pow(T->o.beta1, (float)T->t), c2 = 1.f - std::pow(T->o.beta2, (float)T->t);
    adam_kernel<<<blocks_for(T->np), kT, 0, s>>>(T->p, T->grad, T->m, T->v, T->np, T->o.lr, T->o.beta1,
                                                 T->o.beta2, T->o.eps, c1, c2);
  }
  if ((e = cudaMemcpyAsync(T->partial_host, T->partial, kLossBlocks * sizeof(float), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, fn);
  double sum = 0.0;
  for (int k = 0; k < kLossBlocks; ++k) sum += T->partial_host[k];
  if (loss_out) *loss_out = (float)(sum / (double)n);
  return NSL_OK;
}

nsl_status nsl_trainer_set_lr(nsl_trainer* T, float lr) {
  if (!T || !(lr > 0.f) || !std::isfinite(lr))
    return fail(NSL_ERR_INVALID_ARG, "nsl_trainer_set_lr: trainer NULL or lr not > 0");
  T->o.lr = lr;
  return NSL_OK;
}

nsl_status nsl_trainer_gradients(nsl_trainer* T, float* grad_dev, size_t count, void* stream) {
  if (!T || !grad_dev) return fail(NSL_ERR_INVALID_ARG, "nsl_trainer_gradients: NULL argument");
  if (count < T->np) return fail(NSL_ERR_INVALID_ARG, "nsl_trainer_gradients: needs %zu floats", T->np);
  NSL_CUDA_TRY(cudaMemcpyAsync(grad_dev, T->grad, T->np * sizeof(float), cudaMemcpyDeviceToDevice,
                               static_cast<cudaStream_t>(stream)));
  return NSL_OK;
}

nsl_status nsl_trainer_get_blob(nsl_trainer* T, void* blob_host, size_t bytes, size_t* needed) {
  if (!T) return fail(NSL_ERR_INVALID_ARG, "nsl_trainer_get_blob: trainer is NULL");
  const size_t need = 20 + 4 * T->np;
  if (needed) *needed = need;
  if (!blob_host) return NSL_OK;
  if (bytes < need) return fail(NSL_ERR_INVALID_ARG, "nsl_trainer_get_blob: needs %zu bytes", need);
  unsigned char* b = static_cast<unsigned char*>(blob_host);
  const uint32_t hdr[4] = {0, 1u, (uint32_t)T->c0, (uint32_t)T->np};
  std::memcpy(b, "NSLW", 4);
  std::memcpy(b + 4, hdr + 1, 12);
  NSL_CUDA_TRY(cudaDeviceSynchronize());
  NSL_CUDA_TRY(cudaMemcpy(b + 16, T->p, T->np * 4, cudaMemcpyDeviceToHost));
  uint32_t chk = 0;
  for (size_t i = 0; i < T->np; ++i) {
    uint32_t w;
    std::memcpy(&w, b + 16 + 4 * i, 4);
    chk += w;
  }
  std::memcpy(b + 16 + 4 * T->np, &chk, 4);
  return NSL_OK;
}

}  // extern "C"
