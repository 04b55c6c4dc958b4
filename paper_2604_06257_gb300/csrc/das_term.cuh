// das_term.cuh -- per-(voxel, element, transmit) delay, index and weight.
//
// The index decision is taken in float32 with one fixed operation sequence (every
// step an explicitly rounded intrinsic, so the compiler cannot fuse or reorder it):
//   d   = v - e                                   (sample units, per axis)
//   rx  = sqrt_rn(fma(dx,dx, fma(dy,dy, dz*dz)))  receive path, Sec. 4.3 "on the fly"
//   s   = s_tx + rx                               s_tx from the per-plan table
//   term kept iff inside the aperture and 0 <= s < S-1   (range rule: both taps exist)
//   i0  = floor(s), w = s - i0 (exact)            linear interpolation, Sec. 4.1
// The window and phase are float32 approximations (errors ~1e-7, far below the
// interpolation's own quantisation):
//   aperture: kept iff dz > 0 and fma(dx,dx, dy*dy) * RN(4F#^2) <= dz*dz (the test
//             rho*2F# <= dz taken squared); window of t = rho F#/dz: boxcar 1,
//             Hann cos^2(pi t), Gaussian exp(-8 t^2)
//   phase:    fc (t0 + s/fs) cycles = frac(fc t0) + i0 frac(fc/fs) + w fc/fs, with the
//             first two terms in 32-bit fixed point (exact wrap-around modulo one cycle)
//             so that large sample indices lose no phase accuracy.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "mach_internal.h"

namespace mach {

struct TermGeo {
  float rx;   // receive delay, samples
  float a;    // window value, or -1 when the element is outside the aperture
};

__device__ __forceinline__ TermGeo term_geometry(const float4 v, const float4 e,
                                                 const DasParams& p) {
  const float dx = __fsub_rn(v.x, e.x);
  const float dy = __fsub_rn(v.y, e.y);
  const float dz = __fsub_rn(v.z, e.z);
  TermGeo g;
  g.rx = __fsqrt_rn(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz))));
  if (p.apod == MACH_APOD_NONE) {
    g.a = 1.0f;
    return g;
  }
  // aperture test squared: rho^2 * 4F#^2 <= dz^2 (and dz > 0) -- no square root decides it
  const float rho2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
  if (!(dz > 0.0f && __fmul_rn(rho2, p.four_f2) <= __fmul_rn(dz, dz))) {
    g.a = -1.0f;
    return g;
  }
  if (p.apod == MACH_APOD_BOXCAR) {
    g.a = 1.0f;
    return g;
  }
  // window of t = rho F# / dz in [0, 1/2]; t^2 = rho^2 F#^2 / dz^2
  const float t2 = __fdividef(rho2 * p.f_num2, dz * dz);
  if (p.apod == MACH_APOD_HANN) {
    const float t = t2 > 0.0f ? t2 * rsqrtf(t2) : 0.0f;
    const float cp = __cosf(3.14159265358979f * t);
    g.a = cp * cp;
  } else {
    g.a = __expf(-8.0f * t2);
  }
  return g;
}

// Record of one term: (a cos phi, a sin phi, w, i0 bits); i0 = -1 marks a dropped term.
__device__ __forceinline__ float4 term_record(const float s_tx, const TermGeo g,
                                              const DasParams& p) {
  const float s = __fadd_rn(s_tx, g.rx);
  if (!(g.a >= 0.0f && s >= 0.0f && s < p.s_max)) return make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
  const float fl = floorf(s);
  const int i0 = static_cast<int>(fl);
  const float w = __fsub_rn(s, fl);
  const uint32_t ph = p.phase_Phi + static_cast<uint32_t>(i0) * p.phase_R;
  float x = __fmaf_rn(w, p.r_f, static_cast<float>(static_cast<int32_t>(ph)) * 2.3283064365386963e-10f);
  x -= rintf(x);                                   // cycles in [-1/2, 1/2]
  float sn, cs;
  __sincosf(6.28318530717958648f * x, &sn, &cs);
  return make_float4(g.a * cs, g.a * sn, w, __int_as_float(i0));
}

// Voxel index of slot q of tile `tile`, or -1 past the grid edge (ragged tiles).
__device__ __forceinline__ int64_t tile_voxel(const DasParams& p, int64_t tile, int q) {
  const int qx = q % p.tile_x;
  const int qr = q / p.tile_x;
  const int qy = qr % p.tile_y;
  const int qz = qr / p.tile_y;
  const int64_t bx = tile % p.tiles_x;
  const int64_t br = tile / p.tiles_x;
  const int64_t by = br % p.tiles_y;
  const int64_t bz = br / p.tiles_y;
  const int64_t gx = bx * p.tile_x + qx, gy = by * p.tile_y + qy, gz = bz * p.tile_z + qz;
  if (gx >= p.nx || gy >= p.ny || gz >= p.nz) return -1;
  return gx + static_cast<int64_t>(p.nx) * (gy + static_cast<int64_t>(p.ny) * gz);
}

// Voxel of slot q when each warp owns a compact wb_x x wb_y x wb_z block of the tile
// (the tile is a whole number of such blocks); -1 past the grid edge.
__device__ __forceinline__ int64_t tile_voxel_blocked(const DasParams& p, int64_t tile, int q) {
  if (p.wb_x == 0) return tile_voxel(p, tile, q);
  const int wbv = p.wb_x * p.wb_y * p.wb_z;
  const int b = q / wbv, r = q % wbv;
  const int nbx = p.tile_x / p.wb_x, nby = p.tile_y / p.wb_y;
  const int lx = (b % nbx) * p.wb_x + r % p.wb_x;
  const int ly = ((b / nbx) % nby) * p.wb_y + (r / p.wb_x) % p.wb_y;
  const int lz = (b / (nbx * nby)) * p.wb_z + r / (p.wb_x * p.wb_y);
  return tile_voxel(p, tile, lx + p.tile_x * (ly + p.tile_y * lz));
}

// Sample rows [lo, lo + rows) of element e that the voxels of a tile can touch for one
// transmit, from the tile's bounding box (sample units) and its transmit-delay range:
// the receive delay over the box lies between the distances from e to the nearest and
// farthest points of the box.  Returns false when no voxel of the tile can have a kept
// term (aperture or range rule), so the pair is skipped.  Two rows of margin on each
// side absorb float rounding of the bounds.
__device__ __forceinline__ bool pair_window(const float4 blo, const float4 bhi, const float2 txr,
                                            const float4 e, const DasParams& p, int& lo, int& rows) {
  const float ax = blo.x - e.x, bx = bhi.x - e.x;
  const float ay = blo.y - e.y, by = bhi.y - e.y;
  const float az = blo.z - e.z, bz = bhi.z - e.z;
  const float nx = fmaxf(fmaxf(ax, -bx), 0.f), ny = fmaxf(fmaxf(ay, -by), 0.f), nz = fmaxf(fmaxf(az, -bz), 0.f);
  const float fx = fmaxf(fabsf(ax), fabsf(bx)), fy = fmaxf(fabsf(ay), fabsf(by)), fz = fmaxf(fabsf(az), fabsf(bz));
  if (p.apod != MACH_APOD_NONE) {
    const float rho_min = sqrtf(nx * nx + ny * ny);
    if (!(bz > 0.f) || rho_min * p.two_f > bz * 1.00001f + 1e-3f) return false;
  }
  const float rmin = sqrtf(nx * nx + ny * ny + nz * nz);
  const float rmax = sqrtf(fx * fx + fy * fy + fz * fz);
  const float smin = txr.x + rmin, smax = txr.y + rmax;
  if (!(smax >= -1.f) || !(smin < p.s_max + 1.f)) return false;
  const float top = static_cast<float>(p.S);
  const int l = max(0, static_cast<int>(floorf(fmaxf(smin, -8.f))) - 2);
  const int h = min(p.S - 1, static_cast<int>(floorf(fminf(smax, top))) + 3);
  if (h < l + 1) return false;
  lo = l;
  rows = h - l + 1;
  return true;
}

}  // namespace mach
