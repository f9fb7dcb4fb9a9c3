// Obstacle shadowing (Sec. 4.5): a depth-based screen-space approximation.
// shadow_map_kernel renders, for one directional light, the depth of the first
// obstacle voxel along each light ray (a voxel traversal of the obstacle mask);
// shade_shadowed_kernel moves each pixel's smoke shell (the guide's depth D
// along the camera ray) into every light's frame, compares it with that light's
// map and weights the light's six-way term by the resulting visibility.  Every
// decision (texel choice, the depth comparison) is made in binary32 with one
// rounding per operation in a fixed order.
#include <cmath>

#include "nsl_internal.cuh"

namespace nsl {
namespace {

// Slab test of the unit voxel (i, j, k) against the line o + t w (t unbounded):
// true and the entry parameter when the line meets it (touching counts).
__device__ __forceinline__ bool voxel_entry(const float o[3], const float w[3], int i, int j, int k,
                                            float* t_enter) {
  const float lo[3] = {(float)i, (float)j, (float)k};
  float tn = -INFINITY, tf = INFINITY;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float hi = __fadd_rn(lo[q], 1.f);
    if (w[q] != 0.f) {
      const float ta = __fdiv_rn(__fsub_rn(lo[q], o[q]), w[q]);
      const float tb = __fdiv_rn(__fsub_rn(hi, o[q]), w[q]);
      const float nr = ta < tb ? ta : tb, fr = ta < tb ? tb : ta;
      if (nr > tn) tn = nr;
      if (fr < tf) tf = fr;
    } else if (o[q] < lo[q] || o[q] > hi) {
      return false;
    }
  }
  if (!(tn <= tf)) return false;
  *t_enter = tn;
  return true;
}

// One thread per texel: the depth is the smallest slab-test entry parameter
// over every occupied voxel the line through the texel centre (along w) meets,
// the same minimum a brute force over all occupied voxels takes.  The line is
// walked voxel by voxel (each boundary crossing recomputed from o, no
// accumulated steps), and at every visited voxel the 27 voxels of its 3x3x3
// neighbourhood are tested: a voxel that the binary32 slab test reports as met
// lies within rounding of the line, so it shares at least a corner with a
// voxel the walk visits.  The walk is clipped to the box grown by half a voxel
// (a line grazing the box still visits the voxels beside it) and may visit the
// layer of voxels just outside the grid, whose neighbours inside are tested.
// It stops once the entry parameter of the visited voxel exceeds the best
// depth by 4: any voxel met later is entered at least 2*sqrt(3) after the
// entry of a visited voxel it touches.  +infinity when no occupied voxel is met.
__global__ void __launch_bounds__(256) shadow_map_kernel(const uint8_t* __restrict__ mask, int nx, int ny,
                                                         int nz, LightFrame L, int R, float* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  const int n3[3] = {nx, ny, nz};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < R * R; t += gridDim.x * blockDim.x) {
    const int i = t % R, j = t / R;
    const float ua = __fdiv_rn(__fadd_rn((float)i, 0.5f), (float)R);
    const float ub = __fdiv_rn(__fadd_rn((float)j, 0.5f), (float)R);
    const float a = __fmul_rn(__fsub_rn(ua, 0.5f), L.S), b = __fmul_rn(__fsub_rn(ub, 0.5f), L.S);
    float o[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = __fadd_rn(__fadd_rn(L.c[k], __fmul_rn(a, L.e1[k])), __fmul_rn(b, L.e2[k]));
    float best = INFINITY;
    // clip the line to the box [-1/2, n + 1/2]
    float t0 = -INFINITY, t1 = INFINITY;
    bool hit = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float lo = -0.5f, hi = __fadd_rn((float)n3[k], 0.5f);
      if (L.w[k] != 0.f) {
        const float ta = __fdiv_rn(__fsub_rn(lo, o[k]), L.w[k]);
        const float tb = __fdiv_rn(__fsub_rn(hi, o[k]), L.w[k]);
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
      } else if (o[k] < lo || o[k] > hi) {
        hit = false;
      }
    }
    if (hit && t0 <= t1) {
      // voxel index in [-1, n], step and next boundary parameter per axis, in
      // scalars (no dynamically indexed arrays)
      auto start = [&](int k, int& v, int& st, float& tm) {
        const float pk = __fadd_rn(o[k], __fmul_rn(t0, L.w[k]));
        v = min(max((int)floorf(pk), -1), n3[k]);
        st = L.w[k] > 0.f ? 1 : (L.w[k] < 0.f ? -1 : 0);
        tm = st == 0 ? INFINITY : __fdiv_rn(__fsub_rn((float)(v + (st > 0 ? 1 : 0)), o[k]), L.w[k]);
      };
      int vx, vy, vz, sx, sy, sz;
      float tx, ty, tz;
      start(0, vx, sx, tx);
      start(1, vy, sy, ty);
      start(2, vz, sz, tz);
      float tcur = t0;
      for (int guard = nx + ny + nz + 9; guard > 0; --guard) {
        if (tcur > __fadd_rn(best, 4.f)) break;
        for (int dz = -1; dz <= 1; ++dz) {
          const int kz = vz + dz;
          if (kz < 0 || kz >= nz) continue;
          for (int dy = -1; dy <= 1; ++dy) {
            const int ky = vy + dy;
            if (ky < 0 || ky >= ny) continue;
            const uint8_t* row = mask + ((size_t)kz * ny + ky) * nx;
            for (int dx = -1; dx <= 1; ++dx) {
              const int kx = vx + dx;
              float te;
              if (kx >= 0 && kx < nx && __ldg(row + kx) && voxel_entry(o, L.w, kx, ky, kz, &te) && te < best)
                best = te;
            }
          }
        }
        if (tx <= ty && tx <= tz) {
          if (!(tx <= t1)) break;
          tcur = tx;
          vx += sx;
          if (vx < -1 || vx > nx) break;
          tx = __fdiv_rn(__fsub_rn((float)(vx + (sx > 0 ? 1 : 0)), o[0]), L.w[0]);
        } else if (ty <= tz) {
          if (!(ty <= t1)) break;
          tcur = ty;
          vy += sy;
          if (vy < -1 || vy > ny) break;
          ty = __fdiv_rn(__fsub_rn((float)(vy + (sy > 0 ? 1 : 0)), o[1]), L.w[1]);
        } else {
          if (!(tz <= t1)) break;
          tcur = tz;
          vz += sz;
          if (vz < -1 || vz > nz) break;
          tz = __fdiv_rn(__fsub_rn((float)(vz + (sz > 0 ? 1 : 0)), o[2]), L.w[2]);
        }
      }
    }
    out[t] = best;
  }
}

// The pixel's camera ray and box entry, with the march's arithmetic.
__device__ __forceinline__ bool shell_point(const CamFrame& c, float fx, float fy, float fz, int i, int j,
                                            float D, float x[3]) {
  const float sxs = __fsub_rn(__fdiv_rn(__fadd_rn((float)i, 0.5f), (float)c.W), 0.5f);
  const float sys = __fsub_rn(0.5f, __fdiv_rn(__fadd_rn((float)j, 0.5f), (float)c.H));
  const float a = __fmul_rn(sxs, c.ax), b = __fmul_rn(sys, c.ay);
  float o[3], d[3];
  if (c.kind == NSL_CAM_ORTHO) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[k] = __fadd_rn(__fadd_rn(c.eye[k], __fmul_rn(a, c.r[k])), __fmul_rn(b, c.u[k]));
      d[k] = c.f[k];
    }
  } else {
    float v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v[k] = __fadd_rn(__fadd_rn(c.f[k], __fmul_rn(a, c.r[k])), __fmul_rn(b, c.u[k]));
      o[k] = c.eye[k];
    }
    const float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(v[0], v[0]), __fmul_rn(v[1], v[1])),
                                           __fmul_rn(v[2], v[2])));
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = __fdiv_rn(v[k], len);
  }
  const float n3[3] = {fx, fy, fz};
  float tn = -INFINITY, tf = INFINITY;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (d[k] != 0.f) {
      const float ta = __fdiv_rn(__fsub_rn(0.f, o[k]), d[k]);
      const float tb = __fdiv_rn(__fsub_rn(n3[k], o[k]), d[k]);
      const float lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
      if (lo > tn) tn = lo;
      if (hi < tf) tf = hi;
    } else if (o[k] < 0.f || o[k] > n3[k]) {
      return false;
    }
  }
  if (tn < 0.f) tn = 0.f;
  if (!(tf > tn)) return false;
  const float t = __fadd_rn(tn, D);
#pragma unroll
  for (int k = 0; k < 3; ++k) x[k] = __fadd_rn(o[k], __fmul_rn(t, d[k]));
  return true;
}

__global__ void __launch_bounds__(256) shade_shadowed_kernel(ShadowShadeArgs A) {
  pdl_wait();      // the lightmaps come from the network
  pdl_trigger();
  const size_t P = (size_t)A.W * A.H;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
    float Lq[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) Lq[q] = __ldcs(A.lm + q * P + p);
    const float D = __ldg(A.guide + 2 * P + p);
    const int i = (int)(p % A.W), j = (int)(p / A.W);
    float x[3];
    const bool shell = D > 0.f && shell_point(A.cam, A.fx, A.fy, A.fz, i, j, D, x);
    float rgb[3] = {Lq[7], Lq[7], Lq[7]};
    for (int l = 0; l < A.n_lights; ++l) {
      const ShadowLight& S = A.light[l];
      bool lit = true;
      if (shell && S.map) {
        float rel[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) rel[k] = __fsub_rn(x[k], S.F.c[k]);
        const float pa = __fadd_rn(__fadd_rn(__fmul_rn(rel[0], S.F.e1[0]), __fmul_rn(rel[1], S.F.e1[1])),
                                   __fmul_rn(rel[2], S.F.e1[2]));
        const float pb = __fadd_rn(__fadd_rn(__fmul_rn(rel[0], S.F.e2[0]), __fmul_rn(rel[1], S.F.e2[1])),
                                   __fmul_rn(rel[2], S.F.e2[2]));
        const float pz = __fadd_rn(__fadd_rn(__fmul_rn(rel[0], S.F.w[0]), __fmul_rn(rel[1], S.F.w[1])),
                                   __fmul_rn(rel[2], S.F.w[2]));
        const float fa = floorf(__fmul_rn(__fadd_rn(__fdiv_rn(pa, S.F.S), 0.5f), (float)A.R));
        const float fb = floorf(__fmul_rn(__fadd_rn(__fdiv_rn(pb, S.F.S), 0.5f), (float)A.R));
        if (fa >= 0.f && fa < (float)A.R && fb >= 0.f && fb < (float)A.R) {
          const float th = __ldg(S.map + (size_t)(int)fb * A.R + (int)fa);
          lit = !(pz > __fadd_rn(th, A.bias));
        }
      }
      if (lit) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float s = 0.f;
#pragma unroll
          for (int q = 0; q < 6; ++q) s = fmaf(S.M[c][q], Lq[q], s);
          rgb[c] += s;
        }
      }
    }
    float* out = A.rgba;
#pragma unroll
    for (int c = 0; c < 3; ++c) __stcs(out + c * P + p, rgb[c]);
    __stcs(out + 3 * P + p, fminf(fmaxf(1.f - Lq[6], 0.f), 1.f));
  }
}

}  // namespace

// Light frame (binary64, rounded once): w = -dir/|dir|, e1 = normalize(w x a)
// with a = +Y, or +Z when |w_y| > 0.9, e2 = e1 x w; the map square of side
// |grid diagonal| centred on the grid centre.
bool light_frame_from(const float dir[3], int nx, int ny, int nz, LightFrame* L) {
  const double v[3] = {dir[0], dir[1], dir[2]};
  const double nv = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  if (!(nv > 0.0) || !std::isfinite(nv)) return false;
  const double w[3] = {-v[0] / nv, -v[1] / nv, -v[2] / nv};
  double a[3] = {0.0, 1.0, 0.0};
  if (std::fabs(w[1]) > 0.9) { a[1] = 0.0; a[2] = 1.0; }
  double e1[3] = {w[1] * a[2] - w[2] * a[1], w[2] * a[0] - w[0] * a[2], w[0] * a[1] - w[1] * a[0]};
  const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (double& e : e1) e /= l1;
  const double e2[3] = {e1[1] * w[2] - e1[2] * w[1], e1[2] * w[0] - e1[0] * w[2], e1[0] * w[1] - e1[1] * w[0]};
  for (int k = 0; k < 3; ++k) {
    L->w[k] = (float)w[k];
    L->e1[k] = (float)e1[k];
    L->e2[k] = (float)e2[k];
  }
  L->c[0] = (float)nx * 0.5f;
  L->c[1] = (float)ny * 0.5f;
  L->c[2] = (float)nz * 0.5f;
  L->S = (float)std::sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
  return true;
}

cudaError_t launch_shadow_map(const uint8_t* mask, int nx, int ny, int nz, const LightFrame& L, int R,
                              float* out, cudaStream_t s) {
  int blocks = (R * R + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  return launch_pdl(shadow_map_kernel, dim3(blocks), dim3(256), 0, s, mask, nx, ny, nz, L, R, out);
}

cudaError_t launch_shade_shadowed(const ShadowShadeArgs& a, cudaStream_t s) {
  const size_t P = (size_t)a.W * a.H;
  int blocks = (int)((P + 255) / 256);
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  return launch_pdl(shade_shadowed_kernel, dim3(blocks), dim3(256), 0, s, a);
}

}  // namespace nsl
