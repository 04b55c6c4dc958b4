// k_das_table.cu -- plan-time term table and the staged kernel that reads it.
//
// Sec. 4.3 weighs precomputing delays against computing them on the fly: the paper keeps
// only the transmit delays in a table (its target GPU has 32 GB) and computes receive
// delays per run.  With 288 GB of HBM a plan can afford, for 2D grids and moderate 3D
// ones, to evaluate every term once -- receive delay, aperture weight, sample index,
// interpolation weight and phase of each (voxel, element, transmit) -- and store it.
// A run then streams each pair's 16-byte records into shared memory with the same bulk
// copy that brings the pair's sample window, and the consumer warps only gather and
// accumulate (das_staged.cuh, TABLE = true).
//
// Layout (pairs in the order the producer copies them: tile by tile, then element, then
// transmit -- the order of the on-the-fly kernel):
//   tile_pairs[tile]      first pair of the tile; tile_pairs[tiles] = number of pairs
//   pair_desc[pair]       (transmit, element, first sample row, rows) of its window
//   term_rec[pair][j]     record of voxel slot j of the block, j = warp * WV + k * G + g
//                         for the voxel that lane group g of consumer warp `warp` holds
//                         as its k-th voxel: (a cos phi, a sin phi, w, i0 bits), i0 = -1
//                         for a dropped term.
// Records are computed by the same device functions (das_term.cuh) as the on-the-fly
// kernel, pairs are accumulated in the same order, so both modes give the same bits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "das_staged.cuh"

namespace mach {

// One thread per (tile, element): the window of every transmit (rows 0 when no voxel of
// the tile can use the pair) and the number of usable transmits.
__global__ void __launch_bounds__(256) k_pair_windows(const DasParams p, int64_t n, int2* win, int* count) {
  const int64_t id = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (id >= n) return;
  const int64_t tile = id / p.C;
  const int c = static_cast<int>(id % p.C);
  const float4 e = __ldg(&p.elem[c]);
  const float4 blo = p.tbox[2 * tile], bhi = p.tbox[2 * tile + 1];
  int used = 0;
  for (int t = 0; t < p.T; ++t) {
    int lo = 0, rows = 0;
    if (pair_window(blo, bhi, __ldg(&p.txr[tile * p.txr_stride + t]), e, p, lo, rows)) {
      rows = min(rows, p.rows_cap);
      ++used;
    } else {
      lo = 0;
      rows = 0;
    }
    win[id * p.T + t] = make_int2(lo, rows);
  }
  count[id] = used;
}

// One block per (tile, element), one thread per voxel slot of the block: the records of
// every usable transmit, written at the pair indices first[id], first[id] + 1, ...
__global__ void __launch_bounds__(128) k_term_records(const DasParams p, int wv, int groups, int vpg, const int2* win,
                                                      const int64_t* first, int4* desc, float4* rec) {
  const int64_t id = blockIdx.x;
  const int64_t tile = id / p.C;
  const int c = static_cast<int>(id % p.C);
  const int j = threadIdx.x;
  const int nrec = blockDim.x;
  const int w = j / wv, pos = j % wv;
  const int k = pos / groups, g = pos % groups;
  const int64_t v = tile_voxel_blocked(p, tile, w * wv + g * vpg + k);
  TermGeo geo;
  geo.rx = 0.f;
  geo.a = -1.f;
  if (v >= 0) geo = term_geometry(p.vox[v], p.elem[c], p);
  int64_t q = first[id];
  for (int t = 0; t < p.T; ++t) {
    const int2 wn = win[id * p.T + t];
    if (wn.y <= 0) continue;
    float4 r = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    if (geo.a >= 0.f) r = term_record(p.tx[static_cast<size_t>(t) * p.V + v], geo, p);
    rec[q * nrec + j] = r;
    if (j == 0) desc[q] = make_int4(t, c, wn.x, wn.y);
    ++q;
  }
}

cudaError_t launch_pair_windows(const DasParams& p, int2* win, int* count, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(p.tiles_x) * p.tiles_y * p.tiles_z * p.C;
  k_pair_windows<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(p, n, win, count);
  return cudaGetLastError();
}

cudaError_t launch_term_records(const DasParams& p, Variant v, const int2* win, const int64_t* first, int4* desc,
                                float4* rec, cudaStream_t s) {
  const VariantShape& sh = variant_shape(v);
  const int groups = 32 / sh.lanes_per_voxel;
  const int vpg = sh.voxels_per_warp / groups;
  const int64_t n = static_cast<int64_t>(p.tiles_x) * p.tiles_y * p.tiles_z * p.C;
  k_term_records<<<static_cast<unsigned>(n), sh.warps * sh.voxels_per_warp, 0, s>>>(p, sh.voxels_per_warp, groups,
                                                                                     vpg, win, first, desc, rec);
  return cudaGetLastError();
}

bool table_supported(Variant v) {
  switch (v) {
    case V_ST32_C64P_V4W7: case V_ST32_C64_V4W7: case V_ST64_C64P_V4: case V_ST64_C64_V4: case V_ST64_C64:
    case V_ST32_H16_V4: case V_ST32_B16_V4: case V_ST64_H16_V4: case V_ST64_H16: case V_ST64_B16_V4:
      return true;
    default:
      return false;
  }
}

cudaError_t launch_das_table(const DasParams& p, Variant v, cudaStream_t s) {
  const size_t sm = staged_smem_bytes(v, p.rows_cap, p.F, p.T, true);
  switch (v) {
    case V_ST32_C64P_V4W7: return go_staged(k_das_staged<C64Planar, 4, 1, 8, 4, 7, kRing, 64, true>, 7, p, sm, s);
    case V_ST32_C64_V4W7: return go_staged(k_das_staged<float2, 2, 2, 8, 4, 7, kRing, 64, true>, 7, p, sm, s);
    case V_ST64_C64P_V4: return go_staged(k_das_staged<C64Planar, 4, 1, 16, 4, 8, 8, 72, true>, 8, p, sm, s);
    case V_ST64_C64_V4: return go_staged(k_das_staged<float2, 2, 2, 16, 4, 8, 8, 72, true>, 8, p, sm, s);
    case V_ST64_C64: return go_staged(k_das_staged<float2, 2, 2, 16, 8, 8, kRing, 112, true>, 8, p, sm, s);
    case V_ST32_H16_V4: return go_staged(k_das_staged<__half2, 4, 1, 8, 4, 8, kRing, 72, true>, 8, p, sm, s);
    case V_ST32_B16_V4: return go_staged(k_das_staged<__nv_bfloat162, 4, 1, 8, 4, 8, kRing, 72, true>, 8, p, sm, s);
    case V_ST64_H16_V4: return go_staged(k_das_staged<__half2, 4, 1, 16, 4, 8, 8, 72, true>, 8, p, sm, s);
    case V_ST64_H16: return go_staged(k_das_staged<__half2, 4, 1, 16, 8, 8, kRing, 112, true>, 8, p, sm, s);
    case V_ST64_B16_V4: return go_staged(k_das_staged<__nv_bfloat162, 4, 1, 16, 4, 8, 8, 72, true>, 8, p, sm, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mach
