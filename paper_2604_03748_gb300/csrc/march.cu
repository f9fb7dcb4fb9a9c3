// Guiding-map ray march (Sec. 4.2, Alg. 1, Eq. approx) and grid staging for sm_103a.
//
// One thread marches one pixel's view ray.  Along it, every sample p_n with a
// non-zero density shoots two shadow rays toward the top and bottom surrogate
// lights (camera up / down) to the box exit; the front light's transmittance
// is the view ray's own T_{n-1} (a front-light march from p_n toward the camera
// visits exactly the earlier samples).  A staged grid that fits the 129 MB L2
// (34.6 MB at 128^3) stays resident after its first touch, so the kernel is
// bound by L1/L2 gather throughput and FP32 issue, not by HBM; a larger one
// (256^3: 136 MB as FP16 quads) is partly re-read from DRAM.
//
// Geometry that decides integers (sample counts, positions) is evaluated with
// one IEEE rounding per operation in a fixed order (__fadd_rn & co. are never
// contracted into FMAs), so that the counts agree bit for bit with any other
// binary32 evaluation of the same sequence.
#include <cmath>

#include "grid_sample.cuh"
#include "nsl_internal.cuh"

namespace nsl {

__device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
  // Jarzynski & Olano 2020, "Hash Functions for GPU Rendering": PCG output permutation
  uint32_t state = v * 747796405u + 2891336453u;
  uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

// Two-stage form of sigma_at for software pipelining (quad layout): fetch()
// computes the cell and issues its two 16-byte loads with every index clamped
// into the grid, so it is always safe to issue ahead; interp() finishes the
// trilinear blend and applies the box test.  The value equals sigma_at's.
struct Fetch {
  float4 a, b;
  float tx, ty, tz;
  bool in;
};

template <class G>
__device__ __forceinline__ Fetch fetch(const G& g, float px, float py, float pz) {
  Fetch f;
  f.in = px >= 0.f && px <= g.fx && py >= 0.f && py <= g.fy && pz >= 0.f && pz <= g.fz;
  float qx = __fsub_rn(px, 0.5f), qy = __fsub_rn(py, 0.5f), qz = __fsub_rn(pz, 0.5f);
  float flx = floorf(qx), fly = floorf(qy), flz = floorf(qz);
  f.tx = __fsub_rn(qx, flx);
  f.ty = __fsub_rn(qy, fly);
  f.tz = __fsub_rn(qz, flz);
  // clamp into the padded array so that a speculative fetch is always in range
  const int ix = min(max((int)flx, -1), g.nx - 1), iy = min(max((int)fly, -1), g.ny - 1);
  const int iz = min(max((int)flz, -1), g.nz - 1);
  const unsigned pl = ((unsigned)g.nx + 1u) * ((unsigned)g.ny + 1u);
  load_cell(g, cell_index(g.nx, g.ny, (unsigned)(ix + 1), (unsigned)(iy + 1), (unsigned)(iz + 1)), pl, f.a, f.b);
  return f;
}

// fetch() without the index clamps, for points within rounding of the closed
// box (every shadow sample k <= K is): floor(p - 0.5) then lies in [-1, n-1]
// on every axis, inside the padded array.
template <class G>
__device__ __forceinline__ Fetch fetch_in(const G& g, float px, float py, float pz) {
  Fetch f;
  f.in = px >= 0.f && px <= g.fx && py >= 0.f && py <= g.fy && pz >= 0.f && pz <= g.fz;
  float qx = __fsub_rn(px, 0.5f), qy = __fsub_rn(py, 0.5f), qz = __fsub_rn(pz, 0.5f);
  float flx = floorf(qx), fly = floorf(qy), flz = floorf(qz);
  f.tx = __fsub_rn(qx, flx);
  f.ty = __fsub_rn(qy, fly);
  f.tz = __fsub_rn(qz, flz);
  const unsigned pl = ((unsigned)g.nx + 1u) * ((unsigned)g.ny + 1u);
  load_cell(g, cell_index(g.nx, g.ny, (unsigned)((int)flx + 1), (unsigned)((int)fly + 1), (unsigned)((int)flz + 1)),
            pl, f.a, f.b);
  return f;
}

// Cell fetch at q = p - 0.5 of a point strictly inside the closed box (no box
// test, no clamps): floor(q) lies in [-1, n-1] on every axis.
template <class G>
__device__ __forceinline__ Fetch fetch_q(const G& g, float qx, float qy, float qz) {
  Fetch f;
  f.in = true;
  const float flx = floorf(qx), fly = floorf(qy), flz = floorf(qz);
  f.tx = __fsub_rn(qx, flx);
  f.ty = __fsub_rn(qy, fly);
  f.tz = __fsub_rn(qz, flz);
  const unsigned pl = ((unsigned)g.nx + 1u) * ((unsigned)g.ny + 1u);
  load_cell(g, cell_index(g.nx, g.ny, (unsigned)((int)flx + 1), (unsigned)((int)fly + 1), (unsigned)((int)flz + 1)),
            pl, f.a, f.b);
  return f;
}

__device__ __forceinline__ float interp(const Fetch& f) {
  const float c00 = fmaf(f.tx, f.a.y - f.a.x, f.a.x);
  const float c10 = fmaf(f.tx, f.a.w - f.a.z, f.a.z);
  const float c01 = fmaf(f.tx, f.b.y - f.b.x, f.b.x);
  const float c11 = fmaf(f.tx, f.b.w - f.b.z, f.b.z);
  const float c0 = fmaf(f.ty, c10 - c00, c00);
  const float c1 = fmaf(f.ty, c11 - c01, c01);
  const float v = fmaf(f.tz, c1 - c0, c0);
  return f.in ? v : 0.f;
}

__device__ __forceinline__ float hg_phase(float g, float c) {
  float den = 1.f + g * g - 2.f * g * c;
  return (1.f - g * g) / (12.566370614359172f * den * sqrtf(den));
}

// Number of shadow steps K = floor(t_exit / h) from p along the unit direction
// s to the exit of the closed box.
template <class G>
__device__ __forceinline__ int shadow_steps(const G& g, float px, float py, float pz, float sx,
                                            float sy, float sz, float h) {
  float te = INFINITY;
  if (sx > 0.f) te = fminf(te, __fdiv_rn(__fsub_rn(g.fx, px), sx));
  else if (sx < 0.f) te = fminf(te, __fdiv_rn(__fsub_rn(0.f, px), sx));
  if (sy > 0.f) te = fminf(te, __fdiv_rn(__fsub_rn(g.fy, py), sy));
  else if (sy < 0.f) te = fminf(te, __fdiv_rn(__fsub_rn(0.f, py), sy));
  if (sz > 0.f) te = fminf(te, __fdiv_rn(__fsub_rn(g.fz, pz), sz));
  else if (sz < 0.f) te = fminf(te, __fdiv_rn(__fsub_rn(0.f, pz), sz));
  return te > 0.f ? (int)floorf(__fdiv_rn(te, h)) : 0;
}

// Transmittances toward the top (+u) and bottom (-u) surrogate lights from p:
// each ray is marched at step h to the box exit, T = exp(-h sum_k sigma(p +- k h u)),
// and stops once its optical depth exceeds tau_lim (transmittance below t_min).
// The two rays run back to back as one sequence of K_t + K_b samples, two per
// loop step (two gathers in flight): that length is nearly the same on every
// lane of a warp (the box's extent along u), where max(K_t, K_b) is not.  Each
// ray's samples and sums keep their order.
//
// kExactLast = true (single-plume kernels): samples 1..K-1 of a ray lie strictly
// inside the closed box (K h <= t_exit up to one rounding, so (K-1) h falls
// short of every face crossing by h, far more than the rounding of p + k h s for
// any step above 1e-3 voxel); they need no box test and their cell coordinates
// come from q = fma(k h, s, p - 0.5) (the trilinear value is continuous in q).
// The last sample of each ray, which can lie on or just past the exit face, is
// taken after the others at its exact position with the box test.
// kExactLast = false (grouped kernels): every sample at its exact position with
// the box test, the rays' last samples inside the two-per-step sequence; in the
// grouped march the separate last-sample step cost more latency than the box
// tests it saved (measured: 16.4 against 17.5 ms per 64-plume batch).
template <bool kCount, bool kExactLast, class G>
__device__ __forceinline__ void shadow_pair(const G& g, float px, float py, float pz,
                                            const float u_in[3], float h, float tau_lim, float& Tt,
                                            float& Tb, unsigned long long& nsamp) {
  // the direction in registers: u_in may point into a plume table in global memory
  const float u[3] = {u_in[0], u_in[1], u_in[2]};
  const int Kt = shadow_steps(g, px, py, pz, u[0], u[1], u[2], h);
  const int Kb = shadow_steps(g, px, py, pz, -u[0], -u[1], -u[2], h);
  float taut = 0.f, taub = 0.f;
  bool at = Kt > 0, ab = Kb > 0;
  if constexpr (kExactLast) {
    const int Mt = Kt > 0 ? Kt - 1 : 0, Mb = Kb > 0 ? Kb - 1 : 0;
    const int Mall = Mt + Mb;
    const float qx0 = __fsub_rn(px, 0.5f), qy0 = __fsub_rn(py, 0.5f), qz0 = __fsub_rn(pz, 0.5f);
    int j = 1;
    while (j <= Mall) {
      const bool hasB = j + 1 <= Mall;
      const int j2 = hasB ? j + 1 : j;  // a lone last sample is fetched twice
      const bool tA = j <= Mt, tB = j2 <= Mt;
      // signed step count: negative along the bottom ray (direction -u)
      const float khA = __fmul_rn((float)(tA ? j : Mt - j), h);
      const float khB = __fmul_rn((float)(tB ? j2 : Mt - j2), h);
      const Fetch fA = fetch_q(g, fmaf(khA, u[0], qx0), fmaf(khA, u[1], qy0), fmaf(khA, u[2], qz0));
      const Fetch fB = fetch_q(g, fmaf(khB, u[0], qx0), fmaf(khB, u[1], qy0), fmaf(khB, u[2], qz0));
      const float vA = scaled(g, interp(fA)), vB = scaled(g, interp(fB));
      int jn = j + 2;
      if (tA) {
        taut = fmaf(vA, h, taut);
        if (kCount) ++nsamp;
        if (taut > tau_lim) {
          at = false;
          jn = Mt + 1;             // top ray done; sample B (if bottom) is taken next
        } else if (hasB) {
          if (tB) {
            taut = fmaf(vB, h, taut);
            if (kCount) ++nsamp;
            if (taut > tau_lim) { at = false; jn = Mt + 1; }
          } else {
            taub = fmaf(vB, h, taub);
            if (kCount) ++nsamp;
            if (taub > tau_lim) { ab = false; break; }
          }
        }
      } else {
        taub = fmaf(vA, h, taub);
        if (kCount) ++nsamp;
        if (taub > tau_lim) { ab = false; break; }
        if (hasB) {
          taub = fmaf(vB, h, taub);
          if (kCount) ++nsamp;
          if (taub > tau_lim) { ab = false; break; }
        }
      }
      j = jn;
    }
    if (at || ab) {
      const float kt = __fmul_rn((float)Kt, h), kb = __fmul_rn((float)Kb, h);
      const Fetch ft = fetch(g, __fadd_rn(px, __fmul_rn(kt, u[0])), __fadd_rn(py, __fmul_rn(kt, u[1])),
                             __fadd_rn(pz, __fmul_rn(kt, u[2])));
      const Fetch fb = fetch(g, __fsub_rn(px, __fmul_rn(kb, u[0])), __fsub_rn(py, __fmul_rn(kb, u[1])),
                             __fsub_rn(pz, __fmul_rn(kb, u[2])));
      if (at) {
        taut = fmaf(scaled(g, interp(ft)), h, taut);
        if (kCount) ++nsamp;
      }
      if (ab) {
        taub = fmaf(scaled(g, interp(fb)), h, taub);
        if (kCount) ++nsamp;
      }
    }
  } else {
    // every sample k <= K lies within rounding of the closed box, so
    // floor(p - 0.5) is within [-1, n-1] on every axis: fetch_in needs no clamps
    const int Kall = Kt + (ab ? Kb : 0);
    int j = at ? 1 : Kt + 1;
    while (j <= Kall) {
      const bool hasB = j + 1 <= Kall;
      const int j2 = hasB ? j + 1 : j;  // a lone last sample is fetched twice, never past the ray's end
      const bool tA = j <= Kt, tB = j2 <= Kt;
      const float khA = __fmul_rn((float)(tA ? j : j - Kt), h);
      const float khB = __fmul_rn((float)(tB ? j2 : j2 - Kt), h);
      const float dAx = __fmul_rn(khA, u[0]), dAy = __fmul_rn(khA, u[1]), dAz = __fmul_rn(khA, u[2]);
      const float dBx = __fmul_rn(khB, u[0]), dBy = __fmul_rn(khB, u[1]), dBz = __fmul_rn(khB, u[2]);
      const Fetch fA = fetch_in(g, tA ? __fadd_rn(px, dAx) : __fsub_rn(px, dAx),
                                tA ? __fadd_rn(py, dAy) : __fsub_rn(py, dAy),
                                tA ? __fadd_rn(pz, dAz) : __fsub_rn(pz, dAz));
      const Fetch fB = fetch_in(g, tB ? __fadd_rn(px, dBx) : __fsub_rn(px, dBx),
                                tB ? __fadd_rn(py, dBy) : __fsub_rn(py, dBy),
                                tB ? __fadd_rn(pz, dBz) : __fsub_rn(pz, dBz));
      const float vA = scaled(g, interp(fA)), vB = scaled(g, interp(fB));
      int jn = j + 2;
      if (tA) {
        taut = fmaf(vA, h, taut);
        if (kCount) ++nsamp;
        if (taut > tau_lim) {
          jn = Kt + 1;               // top ray done; sample B (if bottom) is taken next
        } else if (hasB) {
          if (tB) {
            taut = fmaf(vB, h, taut);
            if (kCount) ++nsamp;
            if (taut > tau_lim) jn = Kt + 1;
          } else {
            taub = fmaf(vB, h, taub);
            if (kCount) ++nsamp;
            if (taub > tau_lim) break;
          }
        }
      } else {
        taub = fmaf(vA, h, taub);
        if (kCount) ++nsamp;
        if (taub > tau_lim) break;
        if (hasB) {
          taub = fmaf(vB, h, taub);
          if (kCount) ++nsamp;
          if (taub > tau_lim) break;
        }
      }
      j = jn;
    }
  }
  Tt = expf(-taut);
  Tb = expf(-taub);
}

// One pixel's view ray: origin, direction, the clipped interval, the jitter u,
// the sample count N and the surrogate-light weights (phase x intensity).
struct Ray {
  float o[3], d[3];
  float tn, tf, u;
  int N;
  bool hit;
  float wf, wt, wb;
};

template <class G>
__device__ __forceinline__ Ray ray_setup(const MarchPlume& P, const G& g, int i, int j) {
  const CamFrame& c = P.cam;
  Ray r;
  // ray through the pixel centre
  const float sxs = __fsub_rn(__fdiv_rn(__fadd_rn((float)i, 0.5f), (float)c.W), 0.5f);
  const float sys = __fsub_rn(0.5f, __fdiv_rn(__fadd_rn((float)j, 0.5f), (float)c.H));
  const float a = __fmul_rn(sxs, c.ax), b = __fmul_rn(sys, c.ay);
  if (c.kind == NSL_CAM_ORTHO) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      r.o[k] = __fadd_rn(__fadd_rn(c.eye[k], __fmul_rn(a, c.r[k])), __fmul_rn(b, c.u[k]));
      r.d[k] = c.f[k];
    }
  } else {
    float v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v[k] = __fadd_rn(__fadd_rn(c.f[k], __fmul_rn(a, c.r[k])), __fmul_rn(b, c.u[k]));
      r.o[k] = c.eye[k];
    }
    const float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(v[0], v[0]), __fmul_rn(v[1], v[1])),
                                           __fmul_rn(v[2], v[2])));
#pragma unroll
    for (int k = 0; k < 3; ++k) r.d[k] = __fdiv_rn(v[k], len);
  }
  // slab clip against the closed box
  const float n3[3] = {g.fx, g.fy, g.fz};
  float tn = -INFINITY, tf = INFINITY;
  r.hit = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (r.d[k] != 0.f) {
      const float ta = __fdiv_rn(__fsub_rn(0.f, r.o[k]), r.d[k]);
      const float tb = __fdiv_rn(__fsub_rn(n3[k], r.o[k]), r.d[k]);
      const float lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
      if (lo > tn) tn = lo;
      if (hi < tf) tf = hi;
    } else if (r.o[k] < 0.f || r.o[k] > n3[k]) {
      r.hit = false;
    }
  }
  if (tn < 0.f) tn = 0.f;
  if (!(tf > tn)) r.hit = false;
  r.tn = tn;
  r.tf = tf;
  r.u = 0.f;
  r.N = 0;
  if (r.hit) {
    if (P.jitter) {
      const uint32_t hv = pcg_hash((uint32_t)(j * c.W + i) + P.key);
      r.u = __fmul_rn((float)(hv >> 8), 1.0f / 16777216.0f);
    }
    r.N = (int)floorf(__fadd_rn(__fdiv_rn(__fsub_rn(tf, tn), P.h), r.u));
  }
  // surrogate lights: front (toward the camera), top (+up), bottom (-up); the
  // front/left/right set takes the side pair along +-right
  float Pf = 0.07957747154594767f, Pt = Pf, Pb = Pf;
  if (P.g != 0.f) {
    const float* sd = P.light_set == NSL_LIGHTS_FLR ? c.r : c.u;
    const float cu = r.d[0] * sd[0] + r.d[1] * sd[1] + r.d[2] * sd[2];
    Pf = hg_phase(P.g, -1.f);
    Pt = hg_phase(P.g, cu);
    Pb = hg_phase(P.g, -cu);
  }
  r.wf = Pf * P.I[0];
  r.wt = Pt * P.I[1];
  r.wb = Pb * P.I[2];
  return r;
}

// position of view sample n: t_n = t_in + (n - u) h
__device__ __forceinline__ void view_point(const Ray& r, int n, float h, float& px, float& py,
                                           float& pz) {
  const float t = __fadd_rn(r.tn, __fmul_rn(__fsub_rn((float)n, r.u), h));
  px = __fadd_rn(r.o[0], __fmul_rn(t, r.d[0]));
  py = __fadd_rn(r.o[1], __fmul_rn(t, r.d[1]));
  pz = __fadd_rn(r.o[2], __fmul_rn(t, r.d[2]));
}

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
  const float y = __fsub_rn(v, comp);
  const float t = __fadd_rn(sum, y);
  comp = __fsub_rn(__fsub_rn(t, sum), y);
  sum = t;
}

// One view step n with sigma = s > 0: A_n, the three surrogate lights, L_n;
// accumulates A_n L_n into (L, Lc) and the optical depth into (tau, tc).
template <bool kCount, bool kExactLast, bool kVolume = false, class G = Grid>
__device__ __forceinline__ void view_step(const MarchPlume& P, const G& g, const Ray& r,
                                          float px, float py, float pz, float s, float& T,
                                          float& tau, float& tc, float& L, float& Lc,
                                          unsigned long long& nsamp) {
  const float h = P.h;
  const float A = P.segment_exact ? T * (1.f - expf(-s * h)) : T * s * h;
  float Ln;
  if (P.light_set == NSL_LIGHTS_F) {
    Ln = r.wf * T;                 // front only: no shadow rays
  } else {
    float Tt, Tb;
    if constexpr (kVolume) {
      // the shadow_volume option: the side lights' transmittances interpolated
      // from the voxel-centre volumes
      const Grid gT{P.volT, P.nx, P.ny, P.nz, g.fx, g.fy, g.fz}, gB{P.volB, P.nx, P.ny, P.nz, g.fx, g.fy, g.fz};
      Tt = interp(fetch(gT, px, py, pz));
      Tb = interp(fetch(gB, px, py, pz));
    } else {
      shadow_pair<kCount, kExactLast>(g, px, py, pz, P.light_set == NSL_LIGHTS_FLR ? P.cam.r : P.cam.u, h,
                                      P.tau_lim, Tt, Tb, nsamp);
    }
    Ln = fmaf(r.wf, T, fmaf(r.wt, Tt, r.wb * Tb));
  }
  kahan_add(L, Lc, A * Ln);
  kahan_add(tau, tc, s * h);
  T = expf(-tau);
}

// The staged density of a plume as the sampling functions see it.
template <class G>
__device__ __forceinline__ G plume_grid(const MarchPlume& P);
template <>
__device__ __forceinline__ Grid plume_grid<Grid>(const MarchPlume& P) {
  return Grid{P.vol, P.nx, P.ny, P.nz, (float)P.nx, (float)P.ny, (float)P.nz};
}
template <>
__device__ __forceinline__ GridO plume_grid<GridO>(const MarchPlume& P) {
  return GridO{P.vol, P.nx, P.ny, P.nz, (float)P.nx, (float)P.ny, (float)P.nz};
}
template <>
__device__ __forceinline__ GridH plume_grid<GridH>(const MarchPlume& P) {
  return GridH{reinterpret_cast<const __half*>(P.vol), P.nx, P.ny, P.nz, (float)P.nx, (float)P.ny, (float)P.nz,
               P.scl};
}

// Single-pass march of one pixel (Alg. 1): used by the sample-count variant and
// the allocation-free entry point.
template <bool kCount, bool kExactLast, class G = Grid>
__device__ __forceinline__ void march_pixel(const MarchPlume& P, int i, int j) {
  unsigned long long nsamp = 0;
  const CamFrame& c = P.cam;
  const G g = plume_grid<G>(P);
  const size_t plane = (size_t)c.W * c.H;
  const size_t pix = (size_t)j * c.W + i;
  const Ray r = ray_setup(P, g, i, j);
  float L = 0.f, Lc = 0.f;             // Kahan-compensated guide radiance
  float T = 1.f, tau = 0.f, tc = 0.f;  // Kahan-compensated view optical depth
  float D = 0.f;
  for (int n = 1; n <= r.N; ++n) {
    float px, py, pz;
    view_point(r, n, P.h, px, py, pz);
    const float s = sigma_at(g, px, py, pz);
    if (kCount) ++nsamp;
    if (D == 0.f && s > P.tau_depth) D = __fmul_rn((float)n, P.h);
    if (s > 0.f) {
      view_step<kCount, kExactLast, false, G>(P, g, r, px, py, pz, s, T, tau, tc, L, Lc, nsamp);
      if (T < P.t_min) break;
    }
  }
  if (kCount) {
    atomicAdd(P.counter, nsamp);  // counting variant: density evaluations only
    return;
  }
  P.guide[pix] = L;
  P.guide[plane + pix] = T;
  P.guide[2 * plane + pix] = D;
}

// ---------------------------------------------------------------------------
// Segmented march.  The serial chain of one pixel (every view step with its two
// shadow marches) is split into segments of S view steps handled by different
// threads.  Pass 1 marches the view ray alone and records the compensated
// optical depth (tau, tc) at every segment start, the number of processed
// steps, T and D; pass 2 marches each (pixel, segment) with its shadow rays
// from the recorded state, which reproduces the single-pass T_{n-1} bit for
// bit; pass 3 adds the segment partials of each pixel in order.
// ---------------------------------------------------------------------------
template <class G = Grid>
__device__ __forceinline__ void march_view_pixel(const MarchPlume& P, int i, int j) {
  const CamFrame& c = P.cam;
  const G g = plume_grid<G>(P);
  const size_t plane = (size_t)c.W * c.H;
  const size_t pix = (size_t)j * c.W + i;
  const Ray r = ray_setup(P, g, i, j);
  const int S = P.seg_len;
  float T = 1.f, tau = 0.f, tc = 0.f, D = 0.f;
  int nef = 0;
  for (int n = 1; n <= r.N; ++n) {
    if ((n - 1) % S == 0) {
      const size_t k = (size_t)((n - 1) / S) * plane + pix;
      P.seg_tau[k] = tau;
      P.seg_comp[k] = tc;
    }
    float px, py, pz;
    view_point(r, n, P.h, px, py, pz);
    const float s = sigma_at(g, px, py, pz);
    if (D == 0.f && s > P.tau_depth) D = __fmul_rn((float)n, P.h);
    nef = n;
    if (s > 0.f) {
      kahan_add(tau, tc, s * P.h);
      T = expf(-tau);
      if (T < P.t_min) break;
    }
  }
  P.guide[plane + pix] = T;
  P.guide[2 * plane + pix] = D;
  P.seg_nef[pix] = nef;
}

template <bool kExactLast, bool kVolume = false, class G = Grid>
__device__ __forceinline__ void march_segment(const MarchPlume& P, int i, int j, int seg) {
  const CamFrame& c = P.cam;
  const size_t plane = (size_t)c.W * c.H;
  const size_t pix = (size_t)j * c.W + i;
  const int S = P.seg_len;
  const int nef = __ldcg(P.seg_nef + pix);
  const int first = seg * S + 1;
  if (first > nef) return;
  const int last = min(first + S - 1, nef);
  const G g = plume_grid<G>(P);
  const Ray r = ray_setup(P, g, i, j);
  const size_t k = (size_t)seg * plane + pix;
  float tau = __ldcg(P.seg_tau + k), tc = __ldcg(P.seg_comp + k);
  float T = expf(-tau);
  float L = 0.f, Lc = 0.f;
  unsigned long long nsamp = 0;
  for (int n = first; n <= last; ++n) {
    float px, py, pz;
    view_point(r, n, P.h, px, py, pz);
    const float s = sigma_at(g, px, py, pz);
    if (s > 0.f) view_step<false, kExactLast, kVolume, G>(P, g, r, px, py, pz, s, T, tau, tc, L, Lc, nsamp);
  }
  P.seg_L[k] = L;
}

__device__ __forceinline__ void march_finish_pixel(const MarchPlume& P, int i, int j) {
  const CamFrame& c = P.cam;
  const size_t plane = (size_t)c.W * c.H;
  const size_t pix = (size_t)j * c.W + i;
  const int nseg = (__ldcg(P.seg_nef + pix) + P.seg_len - 1) / P.seg_len;
  float L = 0.f, Lc = 0.f;
  for (int s = 0; s < nseg; ++s) kahan_add(L, Lc, __ldcg(P.seg_L + (size_t)s * plane + pix));
  P.guide[pix] = L;
}

__device__ __forceinline__ int find_plume(const MarchPlume* __restrict__ t, int n, int tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (t[mid].tile_start <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Persistent march: every warp repeatedly takes the next 8x4-pixel tile from a
// global counter (dynamic balancing of very uneven per-pixel costs).  The
// counter lives in library scratch and is zeroed before each launch.
template <bool kBatch, bool kCount, class G = Grid>
__global__ void __launch_bounds__(kMarchThreads, kMarchMinBlocks)
march_kernel(MarchPlume single, const MarchPlume* __restrict__ table, int nplumes, int total_tiles,
             int* __restrict__ tile_counter) {
  const int lane = threadIdx.x & 31;
  while (true) {
    int tile = 0;
    if (lane == 0) tile = atomicAdd(tile_counter, 1);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= total_tiles) break;
    const MarchPlume* P = &single;
    if (kBatch) {
      P = table + find_plume(table, nplumes, tile);
      tile -= P->tile_start;
    }
    const int tx = tile % P->tiles_x, ty = tile / P->tiles_x;
    const int i = (tx << P->tx_log2) + (lane & ((1 << P->tx_log2) - 1));
    const int j = (ty << (5 - P->tx_log2)) + (lane >> P->tx_log2);
    if (i < P->cam.W && j < P->cam.H) march_pixel<kCount, !kBatch, G>(*P, i, j);
  }
}

// Resident blocks of a march kernel over the whole GPU, computed once per
// process (function-local statics are initialised thread-safely).
template <class K>
static int resident_blocks(K kernel) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kMarchThreads, 0) != cudaSuccess || occ < 1)
    occ = 1;
  return occ * num_sms();
}

template <bool kBatch, bool kCount>
static int march_grid() {
  static const int blocks = resident_blocks(march_kernel<kBatch, kCount>);
  return blocks;
}

int march_tiles(int W, int H, int tx_log2) {
  const int tx = 1 << tx_log2, ty = 32 / tx;
  return ((W + tx - 1) / tx) * ((H + ty - 1) / ty);
}

template <class G>
static cudaError_t launch_march_g(const MarchPlume& p, int ntiles, int* tile_counter, cudaStream_t s, bool count) {
  if (count) {
    static const int grid = resident_blocks(march_kernel<false, true, G>);
    march_kernel<false, true, G><<<grid, kMarchThreads, 0, s>>>(p, nullptr, 1, ntiles, tile_counter);
  } else {
    static const int grid = resident_blocks(march_kernel<false, false, G>);
    march_kernel<false, false, G><<<grid, kMarchThreads, 0, s>>>(p, nullptr, 1, ntiles, tile_counter);
  }
  return cudaGetLastError();
}

cudaError_t launch_march(const MarchPlume& p, int* tile_counter, cudaStream_t s, bool count) {
  const int ntiles = march_tiles(p.cam.W, p.cam.H, p.tx_log2);
  if (ntiles == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(tile_counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (p.staged_half) return launch_march_g<GridH>(p, ntiles, tile_counter, s, count);
  if (p.staged_octo) return launch_march_g<GridO>(p, ntiles, tile_counter, s, count);
  return launch_march_g<Grid>(p, ntiles, tile_counter, s, count);
}

cudaError_t launch_march_batch(const MarchPlume* table_dev, int nplumes, int total_tiles,
                               int* tile_counter, cudaStream_t s) {
  if (total_tiles == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(tile_counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  MarchPlume dummy{};
  march_kernel<true, false><<<march_grid<true, false>(), kMarchThreads, 0, s>>>(
      dummy, table_dev, nplumes, total_tiles, tile_counter);
  return cudaGetLastError();
}

// pass 1 and pass 3: one thread per pixel, warps over 8x4 tiles
template <int kPass, class G = Grid>
__global__ void __launch_bounds__(kMarchThreads) march_pixel_pass_kernel(MarchPlume P, int ntiles,
                                                                        int* __restrict__ counter) {
  pdl_wait();      // the staged grid (pass 1) or the segment partials (pass 3)
  pdl_trigger();
  // pass 1 clears the work queue of pass 2 (pass 2 starts after pass 1 ends)
  if (kPass == 1 && blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x * (kMarchThreads / 32) + (threadIdx.x >> 5);
  if (tile >= ntiles) return;
  const int i = ((tile % P.tiles_x) << P.tx_log2) + (lane & ((1 << P.tx_log2) - 1));
  const int j = ((tile / P.tiles_x) << (5 - P.tx_log2)) + (lane >> P.tx_log2);
  if (i >= P.cam.W || j >= P.cam.H) return;
  if (kPass == 1) march_view_pixel<G>(P, i, j);
  else march_finish_pixel(P, i, j);
}

// pass 2: warps take (tile, segment) items from a queue, segment-major
// (kVolume: the side lights' transmittances from the shadow_volume volumes)
template <bool kVolume, class G = Grid>
__global__ void __launch_bounds__(kMarchThreads, kMarchMinBlocks)
march_segment_kernel(MarchPlume P, int ntiles, int nitems, int* __restrict__ counter) {
  pdl_wait();      // the view pass's segment starts and the cleared queue
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    const int seg = item / ntiles, tile = item % ntiles;
    const int i = ((tile % P.tiles_x) << P.tx_log2) + (lane & ((1 << P.tx_log2) - 1));
    const int j = ((tile / P.tiles_x) << (5 - P.tx_log2)) + (lane >> P.tx_log2);
    if (i < P.cam.W && j < P.cam.H) march_segment<true, kVolume, G>(P, i, j, seg);
  }
}

int march_max_segments(int nx, int ny, int nz, float h, int seg_len) {
  const double diag = std::sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
  const double nmax = std::floor(diag / h + 1.0) + 1.0;
  return (int)std::ceil(nmax / seg_len) + 1;
}

template <class G>
static cudaError_t launch_march_segmented_g(const MarchPlume& p, int ntiles, int max_segments, int* tile_counter,
                                           cudaStream_t s) {
  const int warps_per_block = kMarchThreads / 32;
  const int blocks = (ntiles + warps_per_block - 1) / warps_per_block;
  cudaError_t e = launch_pdl(march_pixel_pass_kernel<1, G>, dim3(blocks), dim3(kMarchThreads), 0, s, p, ntiles,
                             tile_counter);
  if (e != cudaSuccess) return e;
  const int nitems = ntiles * max_segments;
  if (p.shadow_volume) {
    static const int grid = resident_blocks(march_segment_kernel<true, G>);
    e = launch_pdl(march_segment_kernel<true, G>, dim3(grid), dim3(kMarchThreads), 0, s, p, ntiles, nitems,
                   tile_counter);
  } else {
    static const int grid = resident_blocks(march_segment_kernel<false, G>);
    e = launch_pdl(march_segment_kernel<false, G>, dim3(grid), dim3(kMarchThreads), 0, s, p, ntiles, nitems,
                   tile_counter);
  }
  if (e != cudaSuccess) return e;
  return launch_pdl(march_pixel_pass_kernel<3>, dim3(blocks), dim3(kMarchThreads), 0, s, p, ntiles, tile_counter);
}

cudaError_t launch_march_segmented(const MarchPlume& p, int max_segments, int* tile_counter,
                                   cudaStream_t s) {
  const int ntiles = march_tiles(p.cam.W, p.cam.H, p.tx_log2);
  if (ntiles == 0) return cudaSuccess;
  if (p.staged_half) return launch_march_segmented_g<GridH>(p, ntiles, max_segments, tile_counter, s);
  if (p.staged_octo) return launch_march_segmented_g<GridO>(p, ntiles, max_segments, tile_counter, s);
  return launch_march_segmented_g<Grid>(p, ntiles, max_segments, tile_counter, s);
}

// ---------------------------------------------------------------------------
// batched forms: many plumes of different sizes per launch (device tables)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_start(const int* __restrict__ starts, int n, int v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(starts + mid) <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// pass 1 / pass 3 over the tiles of all plumes (tile_starts[p] = first tile of plume p)
template <int kPass>
__global__ void __launch_bounds__(kMarchThreads) march_pass_batch_kernel(
    const MarchPlume* __restrict__ table, const int* __restrict__ tile_starts, int nplumes,
    int total_tiles, int* __restrict__ counter) {
  pdl_wait();
  pdl_trigger();
  if (kPass == 1 && blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
  const int lane = threadIdx.x & 31;
  const int gt = blockIdx.x * (kMarchThreads / 32) + (threadIdx.x >> 5);
  if (gt >= total_tiles) return;
  const int k = find_start(tile_starts, nplumes, gt);
  const MarchPlume& P = table[k];
  const int tile = gt - __ldg(tile_starts + k);
  const int i = ((tile % P.tiles_x) << P.tx_log2) + (lane & ((1 << P.tx_log2) - 1));
  const int j = ((tile / P.tiles_x) << (5 - P.tx_log2)) + (lane >> P.tx_log2);
  if (i >= P.cam.W || j >= P.cam.H) return;
  if (kPass == 1) {
    if (P.staged_half) march_view_pixel<GridH>(P, i, j);
    else march_view_pixel(P, i, j);
  } else {
    march_finish_pixel(P, i, j);
  }
}

// pass 2 over (plume, segment, tile) items: item_starts[p] = first item of plume
// p, whose items are segment-major over its tiles
__global__ void __launch_bounds__(kMarchThreads, kMarchMinBlocks) march_segment_batch_kernel(
    const MarchPlume* __restrict__ table, const int* __restrict__ item_starts,
    const int* __restrict__ tile_counts, int nplumes, int nitems, int* __restrict__ counter) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    const int k = find_start(item_starts, nplumes, item);
    const MarchPlume& P = table[k];
    const int local = item - __ldg(item_starts + k), nt = __ldg(tile_counts + k);
    const int seg = local / nt, tile = local % nt;
    const int i = ((tile % P.tiles_x) << P.tx_log2) + (lane & ((1 << P.tx_log2) - 1));
    const int j = ((tile / P.tiles_x) << (5 - P.tx_log2)) + (lane >> P.tx_log2);
    if (i < P.cam.W && j < P.cam.H) {
      if (P.staged_half) march_segment<false, false, GridH>(P, i, j, seg);   // warp-uniform branch
      else march_segment<false>(P, i, j, seg);
    }
  }
}

cudaError_t launch_march_segmented_batch(const MarchPlume* table_dev, const int* tile_starts_dev,
                                         const int* item_starts_dev, const int* tile_counts_dev,
                                         int nplumes, int total_tiles, int total_items,
                                         int seg_blocks, int* counter, cudaStream_t s) {
  if (total_tiles == 0) return cudaSuccess;
  const int wpb = kMarchThreads / 32;
  const int blocks = (total_tiles + wpb - 1) / wpb;
  cudaError_t e = launch_pdl(march_pass_batch_kernel<1>, dim3(blocks), dim3(kMarchThreads), 0, s, table_dev,
                             tile_starts_dev, nplumes, total_tiles, counter);
  if (e != cudaSuccess) return e;
  if ((e = launch_pdl(march_segment_batch_kernel, dim3(seg_blocks), dim3(kMarchThreads), 0, s, table_dev,
                      item_starts_dev, tile_counts_dev, nplumes, total_items, counter)) != cudaSuccess)
    return e;
  return launch_pdl(march_pass_batch_kernel<3>, dim3(blocks), dim3(kMarchThreads), 0, s, table_dev,
                    tile_starts_dev, nplumes, total_tiles, counter);
}

// Grid-wide barrier of a cooperative launch (every CTA resident): the last CTA
// to arrive resets the arrival count and advances the generation; the others
// wait for the generation to move, for at most ~2 s of clock64, after which
// they record code 0x200 in the error word and return false (no hang).  The
// fences order each phase's stores before the arrival and the next phase's
// loads after it; the scratch written by another CTA is read through L2.
__device__ __forceinline__ bool grid_barrier(unsigned* __restrict__ count, unsigned* gen, unsigned* err) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = atomicAdd(gen, 0u);
    __threadfence();
    int ok = 1;
    if (atomicAdd(count, 1u) + 1u == gridDim.x) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const long long t0 = clock64();
      while (atomicAdd(gen, 0u) == g) {
        if (clock64() - t0 > 4000000000LL) {
          ok = 0;
          if (err) atomicOr_system(err, 0x200u);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// The segment pass of the persistent batched march, kept out of line so that
// its shadow loop gets the register budget of the separate segment kernel.
__device__ __noinline__ void persistent_segment_phase(const MarchPlume* __restrict__ table,
                                                      const int* __restrict__ item_starts,
                                                      const int* __restrict__ tile_counts, int nplumes, int nitems,
                                                      unsigned* __restrict__ queue) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(queue, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= (unsigned)nitems) break;
    const int k = find_start(item_starts, nplumes, (int)item);
    const MarchPlume& P = table[k];
    const int local = (int)item - __ldg(item_starts + k), nt = __ldg(tile_counts + k);
    const int seg = local / nt, tile = local % nt;
    const int i = ((tile % P.tiles_x) << P.tx_log2) + (lane & ((1 << P.tx_log2) - 1));
    const int j = ((tile / P.tiles_x) << (5 - P.tx_log2)) + (lane >> P.tx_log2);
    if (i < P.cam.W && j < P.cam.H) {
      if (P.staged_half) march_segment<false, false, GridH>(P, i, j, seg);
      else march_segment<false>(P, i, j, seg);
    }
  }
}

// The batched march in one persistent launch: the view pass over every
// plume's tiles (grid-stride), a grid-wide barrier, the segment pass from the
// work queue, a barrier, the finish pass.  sync[0] is the work queue, sync[1]
// and sync[2] the barrier's arrival count and generation.
__global__ void __launch_bounds__(kMarchThreads, kMarchMinBlocks) march_persistent_batch_kernel(
    const MarchPlume* __restrict__ table, const int* __restrict__ tile_starts, const int* __restrict__ item_starts,
    const int* __restrict__ tile_counts, int nplumes, int total_tiles, int nitems, unsigned* __restrict__ sync,
    unsigned* err) {
  const int lane = threadIdx.x & 31;
  const int wpb = kMarchThreads / 32, w0 = blockIdx.x * wpb + (threadIdx.x >> 5), nw = gridDim.x * wpb;
  if (blockIdx.x == 0 && threadIdx.x == 0) sync[0] = 0u;
  for (int gt = w0; gt < total_tiles; gt += nw) {
    const int k = find_start(tile_starts, nplumes, gt);
    const MarchPlume& P = table[k];
    const int tile = gt - __ldg(tile_starts + k);
    const int i = ((tile % P.tiles_x) << P.tx_log2) + (lane & ((1 << P.tx_log2) - 1));
    const int j = ((tile / P.tiles_x) << (5 - P.tx_log2)) + (lane >> P.tx_log2);
    if (i < P.cam.W && j < P.cam.H) {
      if (P.staged_half) march_view_pixel<GridH>(P, i, j);
      else march_view_pixel(P, i, j);
    }
  }
  if (!grid_barrier(sync + 1, sync + 2, err)) return;
  persistent_segment_phase(table, item_starts, tile_counts, nplumes, nitems, sync);
  if (!grid_barrier(sync + 1, sync + 2, err)) return;
  for (int gt = w0; gt < total_tiles; gt += nw) {
    const int k = find_start(tile_starts, nplumes, gt);
    const MarchPlume& P = table[k];
    const int tile = gt - __ldg(tile_starts + k);
    const int i = ((tile % P.tiles_x) << P.tx_log2) + (lane & ((1 << P.tx_log2) - 1));
    const int j = ((tile / P.tiles_x) << (5 - P.tx_log2)) + (lane >> P.tx_log2);
    if (i < P.cam.W && j < P.cam.H) march_finish_pixel(P, i, j);
  }
}

// CTAs of the persistent batched march resident at once on the whole GPU.
int march_persistent_blocks_max() {
  static const int blocks = resident_blocks(march_persistent_batch_kernel);
  return blocks;
}

cudaError_t launch_march_persistent_batch(const MarchPlume* table_dev, const int* tile_starts_dev,
                                          const int* item_starts_dev, const int* tile_counts_dev, int nplumes,
                                          int total_tiles, int total_items, int blocks, unsigned* sync,
                                          unsigned* err, cudaStream_t s) {
  if (total_tiles == 0) return cudaSuccess;
  const int most = march_persistent_blocks_max();
  if (blocks < 1 || blocks > most) blocks = most;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kMarchThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, march_persistent_batch_kernel, table_dev, tile_starts_dev, item_starts_dev,
                            tile_counts_dev, nplumes, total_tiles, total_items, sync, err);
}

int march_segment_blocks_max() {
  static const int occ = resident_blocks(march_segment_batch_kernel) / num_sms();
  return occ;
}

// ---------------------------------------------------------------------------
// grid staging: sigma' = scale * rho * [mask == 0], FP16 widened exactly
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

// Staging work units: the quad layout is staged four cells at a time along x
// (one thread loads the 5-voxel windows of its two rows once and writes 64
// contiguous bytes; per cell that is 2.5 loads instead of 8).
// In the y-fastest order the four cells of a unit run along y (one thread reads
// the 5-voxel windows of its two x columns), and consecutive units along x, so
// that a warp's loads of the source rows stay coalesced.
__host__ __device__ __forceinline__ size_t stage_units(int nx, int ny, int nz) {
  if (kMarchOrder == 1) return ((size_t)nx + 1) * (((size_t)ny + 4) / 4) * ((size_t)nz + 2);
  const size_t px = (size_t)nx + 1, rows = ((size_t)ny + 1) * ((size_t)nz + 2);
  return rows * ((px + 3) / 4);
}


// Staging units of one cell plane (quad layouts: the units of plane cz are
// the contiguous range [cz, cz + 1) x stage_units_per_plane).
__host__ __device__ __forceinline__ size_t stage_units_per_plane(int nx, int ny) {
  if (kMarchOrder == 1) return ((size_t)nx + 1) * (((size_t)ny + 4) / 4);
  return ((size_t)ny + 1) * (((size_t)nx + 4) / 4);
}

// Four consecutive cells of staging unit u in the y-fastest order: cell
// (a, b0 + t, cz) holds voxels (a-1, a) x (b0-1+t, b0+t) of slice cz-1, every
// index clamped into the grid; `put(dst_cell, v00, v10, v01, v11)` stores one.
template <class V, class Put>
__device__ __forceinline__ void stage_unit_yfast(int nx, int ny, int nz, size_t u, V val, Put put) {
  const unsigned px = (unsigned)nx + 1u, py = (unsigned)ny + 1u, gpy = (py + 3u) / 4u;
  const unsigned u32 = (unsigned)u;   // staged cells < 2^32 (checked at every entry point)
  const int a = (int)(u32 % px);
  const unsigned rest = u32 / px;
  const int b0 = (int)(4u * (rest % gpy)), cz = (int)(rest / gpy);
  const int i0 = max(a - 1, 0), i1 = min(a, nx - 1);
  const int k0 = min(max(cz - 1, 0), nz - 1);
  decltype(val((size_t)0)) w0[5], w1[5];
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int y = min(max(b0 - 1 + t, 0), ny - 1);
    const size_t row = ((size_t)k0 * ny + y) * nx;
    w0[t] = val(row + i0);
    w1[t] = val(row + i1);
  }
  const unsigned c0 = cell_index(nx, ny, (unsigned)a, (unsigned)b0, (unsigned)cz);
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (b0 + t < (int)py) put(c0 + (unsigned)t, w0[t], w1[t], w0[t + 1], w1[t + 1]);
}

template <typename T>
__device__ __forceinline__ void stage_unit(const T* __restrict__ rho, const uint8_t* __restrict__ mask, int nx,
                                           int ny, int nz, float scale, float* __restrict__ out, size_t u) {
  if constexpr (kMarchOrder == 1) {
    auto val = [&](size_t idx) {
      return (mask && __ldg(mask + idx)) ? 0.f : __fmul_rn(scale, to_f<T>(rho[idx]));
    };
    float4* o4 = reinterpret_cast<float4*>(out);
    stage_unit_yfast(nx, ny, nz, u, val, [&](unsigned c, float v00, float v10, float v01, float v11) {
      o4[c] = make_float4(v00, v10, v01, v11);
    });
  } else {
    auto val = [&](size_t idx) {
      return (mask && __ldg(mask + idx)) ? 0.f : __fmul_rn(scale, to_f<T>(rho[idx]));
    };
    const unsigned px = (unsigned)nx + 1u, py = (unsigned)ny + 1u, gpr = (px + 3u) / 4u;
    const unsigned u32 = (unsigned)u;   // staged cells < 2^32 (checked at every entry point)
    const unsigned r = u32 / gpr;       // row: (slice cz, padded y b)
    const int a0 = (int)(4u * (u32 % gpr));
    const int b = (int)(r % py), cz = (int)(r / py);
    const int j0 = max(b - 1, 0), j1 = min(b, ny - 1);
    const int k0 = min(max(cz - 1, 0), nz - 1);
    const size_t b0 = ((size_t)k0 * ny + j0) * nx, b1 = ((size_t)k0 * ny + j1) * nx;
    // window t holds voxel clamp(a0 - 1 + t): cell a0 + t takes windows t and t + 1
    float w0[5], w1[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const int x = min(max(a0 - 1 + t, 0), nx - 1);
      w0[t] = val(b0 + x);
      w1[t] = val(b1 + x);
    }
    float4* dst = reinterpret_cast<float4*>(out) + ((size_t)r * px + (unsigned)a0);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (a0 + t < (int)px) dst[t] = make_float4(w0[t], w0[t + 1], w1[t], w1[t + 1]);
  }
}


// Staging of sigma' = scale * rho * [mask == 0] in the quad layout, with
// out-of-grid neighbours clamped to the edge: cell (a, b, c) of an (nx+1) x
// (ny+1) x (nz+2) array holds the x/y 2x2 neighbourhood whose low corner is
// voxel (a-1, b-1) of slice c-1, every index clamped into the grid.  Staging
// units [u0, u1).
template <typename T>
__global__ void __launch_bounds__(256) stage_kernel(const T* __restrict__ rho,
                                                    const uint8_t* __restrict__ mask, int nx,
                                                    int ny, int nz, float scale,
                                                    float* __restrict__ out, size_t u0, size_t u1) {
  pdl_wait();      // the previous frame's march may still read the staged grid
  pdl_trigger();
  for (size_t u = u0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < u1; u += (size_t)gridDim.x * blockDim.x)
    stage_unit<T>(rho, mask, nx, ny, nz, scale, out, u);
}

// Unit range of cell planes [c0, c1) (c1 < 0: to the last plane).
static void stage_range(size_t n, size_t per_plane, int c0, int c1, size_t* u0, size_t* u1) {
  *u0 = (size_t)c0 * per_plane;
  *u1 = c1 < 0 ? n : (size_t)c1 * per_plane;
  if (*u1 > n) *u1 = n;
  if (*u0 > *u1) *u0 = *u1;
}

static int stage_blocks(size_t units) {
  int blocks = (int)((units + 255) / 256);
  if (blocks > num_sms() * 16) blocks = num_sms() * 16;
  return blocks < 1 ? 1 : blocks;
}

cudaError_t launch_stage_volume(const void* density, int dtype, const uint8_t* mask, int nx,
                                int ny, int nz, float scale, float* staged, cudaStream_t s, int c0, int c1) {
  size_t u0, u1;
  stage_range(stage_units(nx, ny, nz), stage_units_per_plane(nx, ny), c0, c1, &u0, &u1);
  const int blocks = stage_blocks(u1 - u0);
  if (dtype == NSL_F16)
    return launch_pdl(stage_kernel<__half>, dim3(blocks), dim3(256), 0, s,
                      static_cast<const __half*>(density), mask, nx, ny, nz, scale, staged, u0, u1);
  return launch_pdl(stage_kernel<float>, dim3(blocks), dim3(256), 0, s, static_cast<const float*>(density),
                    mask, nx, ny, nz, scale, staged, u0, u1);
}

// FP16 staging of the quad layout (float16 grids, single plume or batched):
// the raw values rho, masked to 0, four cells per thread as in stage_unit;
// the march multiplies by sigma_scale after the trilinear blend.
__device__ __forceinline__ void stage_half_unit(const __half* __restrict__ rho, const uint8_t* __restrict__ mask,
                                                int nx, int ny, int nz, uint2* __restrict__ out, size_t u) {
  const unsigned px = (unsigned)nx + 1u, py = (unsigned)ny + 1u, gpr = (px + 3u) / 4u;
  const __half zero = __float2half_rn(0.f);
  auto val = [&](size_t idx) { return (mask && __ldg(mask + idx)) ? zero : rho[idx]; };
  if constexpr (kMarchOrder == 1) {
    stage_unit_yfast(nx, ny, nz, u, val, [&](unsigned c, __half v00, __half v10, __half v01, __half v11) {
      const __half2 lo = __halves2half2(v00, v10), hi = __halves2half2(v01, v11);
      out[c] = make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
    });
    return;
  }
  const unsigned u32 = (unsigned)u;   // staged cells < 2^32 (checked at every entry point)
  const unsigned r = u32 / gpr;
  const int a0 = (int)(4u * (u32 % gpr));
  const int b = (int)(r % py), cz = (int)(r / py);
  const int j0 = max(b - 1, 0), j1 = min(b, ny - 1);
  const int k0 = min(max(cz - 1, 0), nz - 1);
  const size_t b0 = ((size_t)k0 * ny + j0) * nx, b1 = ((size_t)k0 * ny + j1) * nx;
  __half w0[5], w1[5];
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int x = min(max(a0 - 1 + t, 0), nx - 1);
    w0[t] = val(b0 + x);
    w1[t] = val(b1 + x);
  }
  uint2* dst = out + ((size_t)r * px + (unsigned)a0);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (a0 + t < (int)px) {
      const __half2 lo = __halves2half2(w0[t], w0[t + 1]), hi = __halves2half2(w1[t], w1[t + 1]);
      dst[t] = make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
    }
  }
}

__global__ void __launch_bounds__(256) stage_half_kernel(const __half* __restrict__ rho,
                                                         const uint8_t* __restrict__ mask, int nx, int ny, int nz,
                                                         uint2* __restrict__ out, size_t u0, size_t u1) {
  pdl_wait();      // the previous frame's march may still read the staged grid
  pdl_trigger();
  for (size_t u = u0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < u1; u += (size_t)gridDim.x * blockDim.x)
    stage_half_unit(rho, mask, nx, ny, nz, out, u);
}

cudaError_t launch_stage_volume_half(const __half* density, const uint8_t* mask, int nx, int ny, int nz,
                                     __half* staged, cudaStream_t s, int c0, int c1) {
  size_t u0, u1;
  stage_range(stage_units(nx, ny, nz), stage_units_per_plane(nx, ny), c0, c1, &u0, &u1);
  return launch_pdl(stage_half_kernel, dim3(stage_blocks(u1 - u0)), dim3(256), 0, s, density, mask, nx, ny, nz,
                    reinterpret_cast<uint2*>(staged), u0, u1);
}

// Octo staging (single-plume float32 contexts): cell (a, b, cz), cz in [0, nz],
// holds the x/y 2x2 neighbourhoods of sigma' = scale * rho * [mask == 0] whose
// low corner is voxel (a-1, b-1) of slice cz - 1 (first float4) and of slice
// cz (second float4), every voxel index clamped into the grid, so that a
// trilinear sample reads its eight corners in one 32-byte load.  A block
// stages tiles of kStTX x kStTY cells of one cell plane: it issues every load
// of the tile's source window (kStTX + 1 voxels of kStTY + 1 rows of both
// slices) into registers at once, puts the window in shared memory with mask
// and scale applied once per voxel, and writes the cells, consecutive threads
// writing consecutive cells, while the next tile's loads are in flight.
// (64 x 8 cells: 30 us for the 68.7 MB of the 128^3 grid; 64 x 32 took 36 us,
// and the four-cells-per-thread scheme of the quad layouts 35 us.)
constexpr int kStTX = 64, kStTY = 8;

template <typename T>
__global__ void __launch_bounds__(256) stage_octo_kernel(const T* __restrict__ rho, const uint8_t* __restrict__ mask,
                                                         int nx, int ny, int nz, float scale, float* __restrict__ out,
                                                         int tiles_x, int tiles_plane, int t0, int t1) {
  pdl_wait();      // the previous frame's march may still read the staged grid
  pdl_trigger();
  constexpr int WX = kStTX + 1, WY = kStTY + 1, NW = 2 * WY * WX;
  constexpr int NE = (NW + 255) / 256;   // window elements per thread
  __shared__ float win[2][WY][WX];
  const int px = nx + 1, py = ny + 1;
  float rv[NE];
  bool rm[NE];
  auto fetch = [&](int t) {
    const int cz = t / tiles_plane, r = t % tiles_plane;
    const int a0 = (r % tiles_x) * kStTX, b0 = (r / tiles_x) * kStTY;
#pragma unroll
    for (int i = 0; i < NE; ++i) {
      const int e = min((int)threadIdx.x + i * 256, NW - 1);
      const int xi = e % WX, rest = e / WX, yi = rest % WY, si = rest / WY;
      const int x = min(max(a0 - 1 + xi, 0), nx - 1), y = min(max(b0 - 1 + yi, 0), ny - 1);
      const int k = si == 0 ? min(max(cz - 1, 0), nz - 1) : min(cz, nz - 1);
      const size_t idx = ((size_t)k * ny + y) * nx + x;
      rm[i] = mask ? __ldg(mask + idx) != 0 : false;
      rv[i] = to_f<T>(__ldg(rho + idx));
    }
  };
  int t = t0 + (int)blockIdx.x;
  if (t < t1) fetch(t);
  for (; t < t1; t += (int)gridDim.x) {
    const int cz = t / tiles_plane, r = t % tiles_plane;
    const int a0 = (r % tiles_x) * kStTX, b0 = (r / tiles_x) * kStTY;
    __syncthreads();   // the previous tile's cells are written
#pragma unroll
    for (int i = 0; i < NE; ++i) {
      const int e = (int)threadIdx.x + i * 256;
      if (e < NW) (&win[0][0][0])[e] = rm[i] ? 0.f : __fmul_rn(scale, rv[i]);
    }
    __syncthreads();
    if (t + (int)gridDim.x < t1) fetch(t + (int)gridDim.x);
    for (int e = threadIdx.x; e < kStTX * kStTY; e += blockDim.x) {
      const int ci = e % kStTX, cj = e / kStTX, a = a0 + ci, b = b0 + cj;
      if (a >= px || b >= py) continue;
      float4* d = reinterpret_cast<float4*>(out) + 2 * (size_t)cell_index(nx, ny, (unsigned)a, (unsigned)b, (unsigned)cz);
      d[0] = make_float4(win[0][cj][ci], win[0][cj][ci + 1], win[0][cj + 1][ci], win[0][cj + 1][ci + 1]);
      d[1] = make_float4(win[1][cj][ci], win[1][cj][ci + 1], win[1][cj + 1][ci], win[1][cj + 1][ci + 1]);
    }
  }
}

cudaError_t launch_stage_volume_octo(const void* density, int dtype, const uint8_t* mask, int nx, int ny, int nz,
                                     float scale, float* staged, cudaStream_t s, int c0, int c1) {
  const int planes = nz + 1;
  const int tiles_x = (nx + 1 + kStTX - 1) / kStTX, tiles_plane = tiles_x * ((ny + 1 + kStTY - 1) / kStTY);
  if (c1 < 0 || c1 > planes) c1 = planes;
  if (c0 < 0) c0 = 0;
  if (c0 >= c1) return cudaSuccess;
  const int t0 = c0 * tiles_plane, t1 = c1 * tiles_plane;
  // four resident blocks per SM, each with one tile's loads in flight while it
  // writes the previous tile (six per SM, all that fit, measured no faster)
  const int most = num_sms() * 4;
  const int blocks = t1 - t0 < most ? t1 - t0 : most;
  if (dtype == NSL_F16)
    return launch_pdl(stage_octo_kernel<__half>, dim3(blocks), dim3(256), 0, s, static_cast<const __half*>(density),
                      mask, nx, ny, nz, scale, staged, tiles_x, tiles_plane, t0, t1);
  return launch_pdl(stage_octo_kernel<float>, dim3(blocks), dim3(256), 0, s, static_cast<const float*>(density), mask,
                    nx, ny, nz, scale, staged, tiles_x, tiles_plane, t0, t1);
}

// Transmittance volumes of the shadow_volume option: one thread per voxel
// centre marches the side lights' two shadow rays exactly as from a view sample
// (consecutive threads along x, so a warp's rays run side by side).
template <class G>
__global__ void __launch_bounds__(256) transmittance_volume_kernel(MarchPlume P, float* __restrict__ outT,
                                                                   float* __restrict__ outB) {
  pdl_wait();      // the staged grid
  pdl_trigger();
  const G g = plume_grid<G>(P);
  const float* sd = P.light_set == NSL_LIGHTS_FLR ? P.cam.r : P.cam.u;
  const size_t n = (size_t)P.nx * P.ny * P.nz;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(v % P.nx), j = (int)((v / P.nx) % P.ny), k = (int)(v / ((size_t)P.nx * P.ny));
    float Tt, Tb;
    unsigned long long ns = 0;
    shadow_pair<false, true>(g, (float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f, sd, P.h, P.tau_lim, Tt, Tb, ns);
    outT[v] = Tt;
    outB[v] = Tb;
  }
}

cudaError_t launch_transmittance_volume(const MarchPlume& p, float* outT, float* outB, cudaStream_t s) {
  const size_t n = (size_t)p.nx * p.ny * p.nz;
  int blocks = (int)((n + 255) / 256);
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  if (p.staged_half)
    return launch_pdl(transmittance_volume_kernel<GridH>, dim3(blocks), dim3(256), 0, s, p, outT, outB);
  if (p.staged_octo)
    return launch_pdl(transmittance_volume_kernel<GridO>, dim3(blocks), dim3(256), 0, s, p, outT, outB);
  return launch_pdl(transmittance_volume_kernel<Grid>, dim3(blocks), dim3(256), 0, s, p, outT, outB);
}

// ---------------------------------------------------------------------------
// six-way shading (Sec. 3): rgb_c = sum_q M[c][q] L_q + E, A = clamp(1 - T, 0, 1)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) shade_kernel(ShadeArgs a) {
  pdl_wait();      // the lightmaps come from the network
  pdl_trigger();
  const size_t P = (size_t)a.W * a.H;
  const size_t P4 = P / 4;
  const float4* lm = reinterpret_cast<const float4*>(a.lm);
  float4* out = reinterpret_cast<float4*>(a.rgba);
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < P4;
       q += (size_t)gridDim.x * blockDim.x) {
    float4 L[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) L[k] = __ldcs(lm + k * P4 + q);
    float4 o[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4 acc = L[7];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        float m = a.M[c][k];
        acc.x = fmaf(m, L[k].x, acc.x); acc.y = fmaf(m, L[k].y, acc.y);
        acc.z = fmaf(m, L[k].z, acc.z); acc.w = fmaf(m, L[k].w, acc.w);
      }
      o[c] = acc;
    }
    o[3].x = fminf(fmaxf(1.f - L[6].x, 0.f), 1.f);
    o[3].y = fminf(fmaxf(1.f - L[6].y, 0.f), 1.f);
    o[3].z = fminf(fmaxf(1.f - L[6].z, 0.f), 1.f);
    o[3].w = fminf(fmaxf(1.f - L[6].w, 0.f), 1.f);
#pragma unroll
    for (int c = 0; c < 4; ++c) __stcs(out + c * P4 + q, o[c]);
  }
}

cudaError_t launch_shade(const ShadeArgs& a, cudaStream_t s) {
  size_t P4 = (size_t)a.W * a.H / 4;
  if (P4 == 0) return cudaSuccess;
  int blocks = (int)((P4 + 255) / 256);
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  return launch_pdl(shade_kernel, dim3(blocks), dim3(256), 0, s, a);
}

// ---------------------------------------------------------------------------
// batched staging and shading: blocks numbered plume after plume
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void stage_units_range(const T* __restrict__ rho, const uint8_t* __restrict__ mask,
                                                  int nx, int ny, int nz, float scale, float* __restrict__ out,
                                                  size_t u0, size_t u1) {
  for (size_t u = u0 + threadIdx.x; u < u1; u += blockDim.x)
    stage_unit<T>(rho, mask, nx, ny, nz, scale, out, u);
}

// staging units per block (2048 cells: 512 four-cell units)
constexpr int kStageChunk = 512;

__global__ void __launch_bounds__(256) stage_batch_kernel(const StageItem* __restrict__ items,
                                                          const int* __restrict__ block_starts,
                                                          int n) {
  pdl_wait();
  pdl_trigger();
  const int k = find_start(block_starts, n, blockIdx.x);
  const StageItem& it = items[k];
  const size_t units = stage_units(it.nx, it.ny, it.nz);
  const size_t u0 = (size_t)(blockIdx.x - __ldg(block_starts + k)) * kStageChunk;
  const size_t u1 = u0 + kStageChunk < units ? u0 + kStageChunk : units;
  if (it.dtype == NSL_F16 && it.half_out) {
    for (size_t u = u0 + threadIdx.x; u < u1; u += blockDim.x)
      stage_half_unit(static_cast<const __half*>(it.density), it.mask, it.nx, it.ny, it.nz,
                      reinterpret_cast<uint2*>(it.out), u);
  } else if (it.dtype == NSL_F16)
    stage_units_range<__half>(static_cast<const __half*>(it.density), it.mask, it.nx, it.ny, it.nz,
                              it.scale, it.out, u0, u1);
  else
    stage_units_range<float>(static_cast<const float*>(it.density), it.mask, it.nx, it.ny, it.nz,
                             it.scale, it.out, u0, u1);
}

int stage_batch_blocks(const StageItem& it) {
  const size_t units = stage_units(it.nx, it.ny, it.nz);
  return (int)((units + kStageChunk - 1) / kStageChunk);
}

cudaError_t launch_stage_batch(const StageItem* items_dev, const int* block_starts_dev, int n,
                               int total_blocks, cudaStream_t s) {
  if (total_blocks == 0) return cudaSuccess;
  return launch_pdl(stage_batch_kernel, dim3(total_blocks), dim3(256), 0, s, items_dev, block_starts_dev, n);
}

__global__ void __launch_bounds__(256) shade_batch_kernel(const ShadeArgs* __restrict__ items,
                                                          const int* __restrict__ block_starts,
                                                          int n) {
  pdl_wait();
  pdl_trigger();
  const int k = find_start(block_starts, n, blockIdx.x);
  const ShadeArgs& a = items[k];
  const size_t P4 = (size_t)a.W * a.H / 4;
  const size_t q = (size_t)(blockIdx.x - __ldg(block_starts + k)) * 256 + threadIdx.x;
  if (q >= P4) return;
  const float4* lm = reinterpret_cast<const float4*>(a.lm);
  float4* out = reinterpret_cast<float4*>(a.rgba);
  float4 L[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) L[c] = __ldcs(lm + c * P4 + q);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float4 acc = L[7];
#pragma unroll
    for (int pl = 0; pl < 6; ++pl) {
      const float m = a.M[c][pl];
      acc.x = fmaf(m, L[pl].x, acc.x); acc.y = fmaf(m, L[pl].y, acc.y);
      acc.z = fmaf(m, L[pl].z, acc.z); acc.w = fmaf(m, L[pl].w, acc.w);
    }
    __stcs(out + c * P4 + q, acc);
  }
  float4 al;
  al.x = fminf(fmaxf(1.f - L[6].x, 0.f), 1.f);
  al.y = fminf(fmaxf(1.f - L[6].y, 0.f), 1.f);
  al.z = fminf(fmaxf(1.f - L[6].z, 0.f), 1.f);
  al.w = fminf(fmaxf(1.f - L[6].w, 0.f), 1.f);
  __stcs(out + 3 * P4 + q, al);
}

cudaError_t launch_shade_batch(const ShadeArgs* items_dev, const int* block_starts_dev, int n,
                               int total_blocks, cudaStream_t s) {
  if (total_blocks == 0) return cudaSuccess;
  return launch_pdl(shade_batch_kernel, dim3(total_blocks), dim3(256), 0, s, items_dev, block_starts_dev, n);
}

}  // namespace nsl
