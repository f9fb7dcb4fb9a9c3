// Sampling of a staged density grid (padded quad or octo layout, FP32 or FP16),
// shared by the guide march and the fine-step reference renderer.
#pragma once
#include "nsl_internal.cuh"

namespace nsl {

// Staged grid layouts.  All are padded by one cell on the low sides with every
// neighbour index clamped to the grid, so a sample inside the box needs no
// clamping:
//   Grid   float4 per cell: the x/y 2x2 neighbourhood of sigma' = scale * rho *
//          [mask == 0] in its slice; a sample reads 2 x 16 bytes
//   GridO  2 x float4 per cell: the 2x2x2 neighbourhood of sigma'; a sample
//          reads one 32-byte vector (twice the memory; single-plume float32
//          contexts whose octo grid fits their L2 share)
//   GridH  the quad layout in FP16 holding rho * [mask == 0], scaled after the
//          blend
struct Grid {
  const float* __restrict__ v;
  int nx, ny, nz;
  float fx, fy, fz;  // box extents
};
struct GridO {
  const float* __restrict__ v;
  int nx, ny, nz;
  float fx, fy, fz;
};
// FP16 quads of the masked density rho (single-plume contexts with an FP16
// grid): values exact, sigma = scl * (trilinear value); half the bytes
struct GridH {
  const __half* __restrict__ v;
  int nx, ny, nz;
  float fx, fy, fz;
  float scl;          // sigma_scale
};
__device__ __forceinline__ float scaled(const Grid&, float v) { return v; }
__device__ __forceinline__ float scaled(const GridO&, float v) { return v; }
__device__ __forceinline__ float scaled(const GridH& g, float v) { return __fmul_rn(g.scl, v); }

// 32-byte load of an octo cell: the 2x2 x/y neighbourhood of slice z (a) and
// of slice z+1 (b), in one 256-bit vector access
__device__ __forceinline__ void ldg_octo(const float* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

// Index of padded cell (X, Y, Z) = (ix + 1, iy + 1, iz + 1) in the staged
// array of an nx x ny x nz grid, in the order kMarchOrder; the cell of the
// next slice is pl = (nx + 1)(ny + 1) cells further on in both orders.
__host__ __device__ __forceinline__ unsigned cell_index(int nx, int ny, unsigned X, unsigned Y, unsigned Z) {
  const unsigned px = (unsigned)nx + 1u, py = (unsigned)ny + 1u;
  if constexpr (kMarchOrder == 1) return (Z * px + X) * py + Y;
  return (Z * py + Y) * px + X;
}

// The two x/y quads of padded cell `cell` (slice z in a, z+1 in b).
__device__ __forceinline__ void load_cell(const Grid& g, unsigned cell, unsigned pl, float4& a, float4& b) {
  const float4* q = reinterpret_cast<const float4*>(g.v) + cell;
  a = __ldg(q);
  b = __ldg(q + pl);
}
__device__ __forceinline__ void load_cell(const GridO& g, unsigned cell, unsigned, float4& a, float4& b) {
  ldg_octo(g.v + 8 * (size_t)cell, a, b);
}
__device__ __forceinline__ float4 half4_to_float4(uint2 u) {
  const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ void load_cell(const GridH& g, unsigned cell, unsigned pl, float4& a, float4& b) {
  const uint2* q = reinterpret_cast<const uint2*>(g.v) + cell;
  a = half4_to_float4(__ldg(q));
  b = half4_to_float4(__ldg(q + pl));
}

// Extinction at p: 0 outside the closed box [0,n]; trilinear interpolation of
// the staged voxels at q = p - 0.5 with clamp-to-edge indices inside it.
template <class G>
__device__ __forceinline__ float sigma_at(const G& g, float px, float py, float pz) {
  if (!(px >= 0.f && px <= g.fx && py >= 0.f && py <= g.fy && pz >= 0.f && pz <= g.fz)) return 0.f;
  float qx = __fsub_rn(px, 0.5f), qy = __fsub_rn(py, 0.5f), qz = __fsub_rn(pz, 0.5f);
  float flx = floorf(qx), fly = floorf(qy), flz = floorf(qz);
  float tx = __fsub_rn(qx, flx), ty = __fsub_rn(qy, fly), tz = __fsub_rn(qz, flz);
  int ix = (int)flx, iy = (int)fly, iz = (int)flz;
  // padded cells: cell (ix+1, iy+1, iz+1) holds the corners, every index of a
  // point inside the box is in range
  const unsigned pl = ((unsigned)g.nx + 1u) * ((unsigned)g.ny + 1u);
  float4 a, b;
  load_cell(g, cell_index(g.nx, g.ny, (unsigned)(ix + 1), (unsigned)(iy + 1), (unsigned)(iz + 1)), pl, a, b);
  const float c00 = fmaf(tx, a.y - a.x, a.x);
  const float c10 = fmaf(tx, a.w - a.z, a.z);
  const float c01 = fmaf(tx, b.y - b.x, b.x);
  const float c11 = fmaf(tx, b.w - b.z, b.z);
  const float c0 = fmaf(ty, c10 - c00, c00);
  const float c1 = fmaf(ty, c11 - c01, c01);
  return scaled(g, fmaf(tz, c1 - c0, c0));
}

}  // namespace nsl
