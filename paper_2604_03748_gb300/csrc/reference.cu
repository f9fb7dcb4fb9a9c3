// Fine-step six-light reference lightmaps (single scattering, Sec. 3 Eq. RE and
// Eq. scatter, the physical target the lightmap network of Sec. 4.3 is trained
// toward; Sec. 4.4 trains against path-traced renders of the same quantity).
//
// Per pixel the view ray (the guide march's pixel ray and closed-box clip) is
// split into M = ceil(chord / hf) equal steps and sampled at their midpoints;
// at every sample with non-zero extinction the transmittance toward each of
// the six camera-frame light directions (+r, -r, +u, -u, +f, -f) is the
// midpoint sum of its own ray to the box exit, in steps of at most hf.  The
// contribution of a sample is T (1 - exp(-sigma hs)) P(cos) exp(-tau_light),
// with T the view transmittance before it.  Output: 7 planes [+X, -X, +Y, -Y,
// +Z, -Z, T].
//
// The integer decisions (step counts), the sample parameters and positions and
// the sums are evaluated in binary64, with each position rounded once to
// binary32; the density itself is the march's binary32 trilinear sample.  This
// is a training-data generator, not part of the per-frame path: one thread per
// pixel, warps over 8 x 4 tiles.
#include <cmath>

#include "grid_sample.cuh"
#include "nsl_internal.cuh"

namespace nsl {
namespace {

struct RefArgs {
  CamFrame cam;
  float fx, fy, fz;     // box extents
  double hf;
  float g;              // Henyey-Greenstein parameter
  float* out;           // [7][H][W]
};

// Optical depth from p toward the unit direction s to the box exit: M = ceil(te
// / hf) midpoint samples of step te / M.
template <class G>
__device__ double light_tau(const G& grid, const RefArgs& a, const float p[3], const double s[3]) {
  const double n3[3] = {a.fx, a.fy, a.fz};
  double te = INFINITY;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (s[k] > 0.0) te = fmin(te, (n3[k] - (double)p[k]) / s[k]);
    else if (s[k] < 0.0) te = fmin(te, (0.0 - (double)p[k]) / s[k]);
  }
  if (!(te > 0.0)) return 0.0;
  const int M = (int)ceil(te / a.hf);
  const double hs = te / M;
  double tau = 0.0;
  for (int m = 1; m <= M; ++m) {
    const double t = ((double)m - 0.5) * hs;
    const float q0 = (float)__dadd_rn((double)p[0], __dmul_rn(t, s[0]));
    const float q1 = (float)__dadd_rn((double)p[1], __dmul_rn(t, s[1]));
    const float q2 = (float)__dadd_rn((double)p[2], __dmul_rn(t, s[2]));
    tau = __dadd_rn(tau, __dmul_rn((double)sigma_at(grid, q0, q1, q2), hs));
  }
  return tau;
}

__device__ __forceinline__ double hg(double g, double c) {
  const double den = 1.0 + g * g - 2.0 * g * c;
  return (1.0 - g * g) / (12.566370614359172 * den * sqrt(den));
}

template <class G>
__global__ void __launch_bounds__(128) reference_kernel(G grid, RefArgs a) {
  const CamFrame& c = a.cam;
  const int lane = threadIdx.x & 31;
  const int tiles_x = (c.W + 7) / 8;
  const int tile = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int i = (tile % tiles_x) * 8 + lane % 8, j = (tile / tiles_x) * 4 + lane / 8;
  if (j >= c.H || i >= c.W) return;
  // the pixel ray and its clip, as the guide march computes them
  const float sxs = __fsub_rn(__fdiv_rn(__fadd_rn((float)i, 0.5f), (float)c.W), 0.5f);
  const float sys = __fsub_rn(0.5f, __fdiv_rn(__fadd_rn((float)j, 0.5f), (float)c.H));
  const float aa = __fmul_rn(sxs, c.ax), bb = __fmul_rn(sys, c.ay);
  float o[3], d[3];
  if (c.kind == NSL_CAM_ORTHO) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[k] = __fadd_rn(__fadd_rn(c.eye[k], __fmul_rn(aa, c.r[k])), __fmul_rn(bb, c.u[k]));
      d[k] = c.f[k];
    }
  } else {
    float v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v[k] = __fadd_rn(__fadd_rn(c.f[k], __fmul_rn(aa, c.r[k])), __fmul_rn(bb, c.u[k]));
      o[k] = c.eye[k];
    }
    const float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(v[0], v[0]), __fmul_rn(v[1], v[1])),
                                           __fmul_rn(v[2], v[2])));
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = __fdiv_rn(v[k], len);
  }
  const float n3[3] = {a.fx, a.fy, a.fz};
  float tn = -INFINITY, tf = INFINITY;
  bool hit = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (d[k] != 0.f) {
      const float ta = __fdiv_rn(__fsub_rn(0.f, o[k]), d[k]);
      const float tb = __fdiv_rn(__fsub_rn(n3[k], o[k]), d[k]);
      const float lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
      if (lo > tn) tn = lo;
      if (hi < tf) tf = hi;
    } else if (o[k] < 0.f || o[k] > n3[k]) {
      hit = false;
    }
  }
  if (tn < 0.f) tn = 0.f;
  if (!(tf > tn)) hit = false;
  // toward-light directions: +r, -r, +u, -u, +f, -f
  double dirs[6][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dirs[0][k] = c.r[k]; dirs[1][k] = -(double)c.r[k];
    dirs[2][k] = c.u[k]; dirs[3][k] = -(double)c.u[k];
    dirs[4][k] = c.f[k]; dirs[5][k] = -(double)c.f[k];
  }
  double Lp[6] = {0, 0, 0, 0, 0, 0}, T = 1.0;
  if (hit) {
    const double chord = (double)tf - (double)tn;
    const int M = (int)ceil(chord / a.hf);
    const double hs = chord / M;
    double tau = 0.0;
    for (int m = 1; m <= M; ++m) {
      const double t = __dadd_rn((double)tn, __dmul_rn((double)m - 0.5, hs));
      const float p[3] = {(float)__dadd_rn((double)o[0], __dmul_rn(t, (double)d[0])),
                          (float)__dadd_rn((double)o[1], __dmul_rn(t, (double)d[1])),
                          (float)__dadd_rn((double)o[2], __dmul_rn(t, (double)d[2]))};
      const double sg = sigma_at(grid, p[0], p[1], p[2]);
      if (sg > 0.0) {
        const double w = T * (1.0 - exp(-sg * hs));
#pragma unroll 1
        for (int l = 0; l < 6; ++l) {
          const double cth = dirs[l][0] * d[0] + dirs[l][1] * d[1] + dirs[l][2] * d[2];
          Lp[l] += w * hg((double)a.g, cth) * exp(-light_tau(grid, a, p, dirs[l]));
        }
      }
      tau = __dadd_rn(tau, __dmul_rn(sg, hs));
      T = exp(-tau);
    }
  }
  const size_t plane = (size_t)c.W * c.H, pix = (size_t)j * c.W + i;
#pragma unroll
  for (int l = 0; l < 6; ++l) a.out[l * plane + pix] = (float)Lp[l];
  a.out[6 * plane + pix] = (float)T;
}

}  // namespace

cudaError_t launch_reference_lightmaps(const MarchPlume& p, double hf, float g, float* out, cudaStream_t s) {
  RefArgs a{};
  a.cam = p.cam;
  a.fx = (float)p.nx;
  a.fy = (float)p.ny;
  a.fz = (float)p.nz;
  a.hf = hf;
  a.g = g;
  a.out = out;
  const int tiles = ((p.cam.W + 7) / 8) * ((p.cam.H + 3) / 4);
  const int blocks = (tiles + 3) / 4;
  if (p.staged_half) {
    const GridH gh{reinterpret_cast<const __half*>(p.vol), p.nx, p.ny, p.nz, a.fx, a.fy, a.fz, p.scl};
    reference_kernel<GridH><<<blocks, 128, 0, s>>>(gh, a);
  } else if (p.staged_octo) {
    const GridO go{p.vol, p.nx, p.ny, p.nz, a.fx, a.fy, a.fz};
    reference_kernel<GridO><<<blocks, 128, 0, s>>>(go, a);
  } else {
    const Grid gf{p.vol, p.nx, p.ny, p.nz, a.fx, a.fy, a.fz};
    reference_kernel<Grid><<<blocks, 128, 0, s>>>(gf, a);
  }
  return cudaGetLastError();
}

}  // namespace nsl
