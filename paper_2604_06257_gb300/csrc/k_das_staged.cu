// k_das_staged.cu -- the staged delay-and-sum kernel with terms evaluated on the fly
// (Sec. 4.3's hybrid delays), and the plan-time bounds every staged variant needs (per
// tile: voxel bounding box and transmit-delay range, from which each (element,
// transmit) pair's sample window follows).  The kernel itself is in das_staged.cuh.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "das_staged.cuh"

namespace mach {

// ---- plan-time bounds ------------------------------------------------------------------

// One block per tile: bounding box of the tile's voxels and, per transmit, the range of
// the transmit delay over them.
__global__ void __launch_bounds__(256) k_tile_bounds(DasParams p, int per_cta, float4* tbox, float2* txr) {
  const int64_t tile = blockIdx.x;
  __shared__ float red[6][8];
  __shared__ float2 tred[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int q = threadIdx.x; q < per_cta; q += blockDim.x) {
    const int64_t v = tile_voxel(p, tile, q);
    if (v < 0) continue;
    const float4 x = p.vox[v];
    mn[0] = fminf(mn[0], x.x); mn[1] = fminf(mn[1], x.y); mn[2] = fminf(mn[2], x.z);
    mx[0] = fmaxf(mx[0], x.x); mx[1] = fmaxf(mx[1], x.y); mx[2] = fmaxf(mx[2], x.z);
  }
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
      mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
    }
    if (lane == 0) { red[a][warp] = mn[a]; red[3 + a][warp] = mx[a]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f), hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    for (int w = 0; w < (blockDim.x >> 5); ++w) {
      lo.x = fminf(lo.x, red[0][w]); lo.y = fminf(lo.y, red[1][w]); lo.z = fminf(lo.z, red[2][w]);
      hi.x = fmaxf(hi.x, red[3][w]); hi.y = fmaxf(hi.y, red[4][w]); hi.z = fmaxf(hi.z, red[5][w]);
    }
    tbox[2 * tile] = lo;
    tbox[2 * tile + 1] = hi;
  }
  for (int t = 0; t < p.T; ++t) {
    float a = INFINITY, b = -INFINITY;
    for (int q = threadIdx.x; q < per_cta; q += blockDim.x) {
      const int64_t v = tile_voxel(p, tile, q);
      if (v < 0) continue;
      const float s = p.tx[static_cast<int64_t>(t) * p.V + v];
      a = fminf(a, s);
      b = fmaxf(b, s);
    }
    for (int o = 16; o > 0; o >>= 1) {
      a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    __syncthreads();
    if (lane == 0) tred[warp] = make_float2(a, b);
    __syncthreads();
    if (threadIdx.x == 0) {
      float2 r = make_float2(INFINITY, -INFINITY);
      for (int w = 0; w < (blockDim.x >> 5); ++w) { r.x = fminf(r.x, tred[w].x); r.y = fmaxf(r.y, tred[w].y); }
      txr[tile * p.T + t] = r;
    }
  }
}

// Largest window over all (tile, transmit, element) and the number of pairs needing a
// copy: out[0] = max rows, out[1] = pairs (saturating).
__global__ void __launch_bounds__(256) k_window_stats(DasParams p, const float4* tbox, const float2* txr,
                                                      int64_t tiles, int* out) {
  const int64_t id = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (id >= tiles * p.C) return;
  const int64_t tile = id / p.C;
  const int c = static_cast<int>(id % p.C);
  const float4 e = p.elem[c];
  int best = 0, n = 0;
  for (int t = 0; t < p.T; ++t) {
    int lo, rows;
    if (pair_window(tbox[2 * tile], tbox[2 * tile + 1], txr[tile * p.T + t], e, p, lo, rows)) {
      best = max(best, rows);
      ++n;
    }
  }
  if (best) atomicMax(out, best);
  if (n) atomicAdd(out + 1, n);
}

cudaError_t launch_tile_bounds(const DasParams& p, float4* tbox, float2* txr, int* d_out, cudaStream_t s) {
  const int64_t tiles = static_cast<int64_t>(p.tiles_x) * p.tiles_y * p.tiles_z;
  const int per_cta = p.tile_x * p.tile_y * p.tile_z;
  k_tile_bounds<<<static_cast<unsigned>(tiles), 256, 0, s>>>(p, per_cta, tbox, txr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d_out, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
  const int64_t n = tiles * p.C;
  k_window_stats<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(p, tbox, txr, tiles, d_out);
  return cudaGetLastError();
}

// ---- dispatch ------------------------------------------------------------------------------
size_t staged_smem_bytes(Variant v, int rows_cap, int F, int T, bool table) {
  const VariantShape& sh = variant_shape(v);
  if (sh.exact_frames) return exact_smem_bytes(v, rows_cap, T);
  if (sh.ring_slots == 8) return RingLayout<8>(rows_cap, F, sh.iq_bytes, T, sh.warps, sh.voxels_per_warp, table).total();
  return RingLayout<kRing>(rows_cap, F, sh.iq_bytes, T, sh.warps, sh.voxels_per_warp, table).total();
}

cudaError_t launch_das_staged(const DasParams& p, Variant v, cudaStream_t s) {
  if (variant_shape(v).exact_frames) return launch_das_exact(p, v, s);
  const size_t sm = staged_smem_bytes(v, p.rows_cap, p.F, p.T, false);
  switch (v) {
    case V_ST32_C64: return go_staged(k_das_staged<float2, 2, 2, 8, 8, 8, kRing, 112, false>, 8, p, sm, s);
    case V_ST64_C64: return go_staged(k_das_staged<float2, 2, 2, 16, 8, 8, kRing, 112, false>, 8, p, sm, s);
    case V_ST32_H16: return go_staged(k_das_staged<__half2, 4, 1, 8, 8, 8, kRing, 112, false>, 8, p, sm, s);
    case V_ST64_H16: return go_staged(k_das_staged<__half2, 4, 1, 16, 8, 8, kRing, 112, false>, 8, p, sm, s);
    case V_ST32_C64_V4: return go_staged(k_das_staged<float2, 2, 2, 8, 4, 8, kRing, 72, false>, 8, p, sm, s);
    case V_ST32_C64_V4W4: return go_staged(k_das_staged<float2, 2, 2, 8, 4, 4, kRing, 80, false>, 4, p, sm, s);
    case V_ST32_C64_V4R56: return go_staged(k_das_staged<float2, 2, 2, 8, 4, 8, kRing, 56, false>, 8, p, sm, s);
    case V_ST32_C64P_V4: return go_staged(k_das_staged<C64Planar, 4, 1, 8, 4, 8, kRing, 72, false>, 8, p, sm, s);
    case V_ST64_C64P_V4: return go_staged(k_das_staged<C64Planar, 4, 1, 16, 4, 8, 8, 72, false>, 8, p, sm, s);
    case V_ST32_C64P_V4W7: return go_staged(k_das_staged<C64Planar, 4, 1, 8, 4, 7, kRing, 64, false>, 7, p, sm, s);
    case V_ST32_C64_V4W7: return go_staged(k_das_staged<float2, 2, 2, 8, 4, 7, kRing, 64, false>, 7, p, sm, s);
    case V_ST32_H16_V4: return go_staged(k_das_staged<__half2, 4, 1, 8, 4, 8, kRing, 72, false>, 8, p, sm, s);
    case V_ST32_B16_V4: return go_staged(k_das_staged<__nv_bfloat162, 4, 1, 8, 4, 8, kRing, 72, false>, 8, p, sm, s);
    case V_ST64_C64_V4: return go_staged(k_das_staged<float2, 2, 2, 16, 4, 8, 8, 72, false>, 8, p, sm, s);
    case V_ST64_H16_V4: return go_staged(k_das_staged<__half2, 4, 1, 16, 4, 8, 8, 72, false>, 8, p, sm, s);
    case V_ST32_B16: return go_staged(k_das_staged<__nv_bfloat162, 4, 1, 8, 8, 8, kRing, 112, false>, 8, p, sm, s);
    case V_ST64_B16_V4: return go_staged(k_das_staged<__nv_bfloat162, 4, 1, 16, 4, 8, 8, 72, false>, 8, p, sm, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mach
