// k_das.cu -- delay-and-sum kernels (Sec. 2.1 steps 1-3) with fused Power Doppler (Sec. 5).
//
// Data layout (Sec. 4.4): IQ [t][c][s][f] with frames contiguous, so the F frames of one
// (t, c, s) sample are one contiguous row; the two interpolation taps of a term are the
// rows i0 and i0 + 1.
//
// "Frame lanes" kernels (F >= 5):  a warp owns WV voxels; the lanes of a group of FL lanes
// share one voxel and each lane holds FPL frames of it in registers.  Per element (and
// chunk of transmits) every lane evaluates one term (voxel, element, transmit) and
// stores it in a per-warp table in shared memory; the table is then read back as a
// broadcast by the FL lanes of each group and reused across all frames of the tile
// (the paper's delay reuse across frames, Sec. 4.4).  The gather per term is one
// coalesced row segment of FL x FPL frames per tap.
//
// "Channel lanes" kernels (F <= 4): CL lanes share one voxel, lane j takes elements
// j, j + CL, ...; each lane evaluates its own terms, and the partial sums are combined by
// a shuffle tree (pairwise, so rounding grows with log CL).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "das_term.cuh"
#include "tap_mac.cuh"
#include "mach_internal.h"

namespace mach {

template <class IQ, int VEC>
__device__ __forceinline__ void store_y(float2* dst, const float2* acc_m) {
  if constexpr (VEC == 1) {
    dst[0] = acc_m[0];
  } else {
#pragma unroll
    for (int e = 0; e < VEC; e += 2) {
      const float2 a = acc_frame<IQ, VEC>(acc_m, e), b = acc_frame<IQ, VEC>(acc_m, e + 1);
      *reinterpret_cast<float4*>(dst + e) = make_float4(a.x, a.y, b.x, b.y);
    }
  }
}

constexpr int kTxChunk = 8;   // transmits whose terms are staged per element round

// ---- frame-lane kernel ---------------------------------------------------------------
template <class IQ, int VEC, int NV, int FL, int VPG, int NWARP>
__global__ void __launch_bounds__(NWARP * 32) k_das_frames(const DasParams p) {
  constexpr int G = 32 / FL;           // voxel groups per warp
  constexpr int WV = G * VPG;          // voxels per warp
  constexpr int CPR = 32 / WV;         // elements per term round
  constexpr int FPL = VEC * NV;        // frames per lane
  constexpr int FT = FL * FPL;         // frames per block
  static_assert(CPR * WV == 32, "a term round must fill the warp");

  extern __shared__ float4 smem_terms[];   // [NWARP][kTxChunk][32]
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  float4* terms = smem_terms + warp * (kTxChunk * 32);
  const int g = lane / FL;
  const int jl = lane % FL;
  const int f_base = blockIdx.y * FT;
  // deepest tiles (widest apertures, most terms) first: light tiles fill the launch's tail
  const int64_t tile = static_cast<int64_t>(gridDim.x) - 1 - blockIdx.x;
  using E = typename IqStore<IQ>::E;
  const E* __restrict__ iq = static_cast<const E*>(p.iq);
  const int row_elems = p.F * IqStore<IQ>::eps;

  // the term this lane evaluates each round: voxel slot lane % WV, element cc + lane / WV
  const int64_t v_term = tile_voxel(p, tile, warp * WV + (lane % WV));
  const float4 vpos = v_term >= 0 ? p.vox[v_term] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int c_sub = lane / WV;
  // slot (g, k) of element sub-round j is stored at j*WV + k*G + g: the G groups of the
  // warp then read G consecutive entries in one conflict-free broadcast
  const int q_lane = lane % WV;
  const int store_at = c_sub * WV + (q_lane % VPG) * G + (q_lane / VPG);

  float2 acc[VPG][FPL];
#pragma unroll
  for (int k = 0; k < VPG; ++k)
#pragma unroll
    for (int e = 0; e < FPL; ++e) acc[k][e] = make_float2(0.f, 0.f);

  const size_t slab = static_cast<size_t>(p.S) * row_elems;   // samples x frames per (t, c)
  for (int cc = 0; cc < p.C; cc += CPR) {
    const int c = cc + c_sub;
    TermGeo geo;
    geo.rx = 0.f;
    geo.a = -1.f;
    if (v_term >= 0 && c < p.C) geo = term_geometry(vpos, __ldg(&p.elem[c]), p);
    for (int tb = 0; tb < p.T; tb += kTxChunk) {
      const int tn = min(kTxChunk, p.T - tb);
      __syncwarp();
      for (int tt = 0; tt < tn; ++tt) {
        float4 r = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        if (geo.a >= 0.f) r = term_record(__ldg(&p.tx[static_cast<size_t>(tb + tt) * p.V + v_term]), geo, p);
        terms[tt * 32 + store_at] = r;
      }
      __syncwarp();
      for (int tt = 0; tt < tn; ++tt) {
#pragma unroll
        for (int j = 0; j < CPR; ++j) {
          const int c2 = cc + j;
          if (c2 >= p.C) break;
          const E* base = iq + (static_cast<size_t>(tb + tt) * p.C + c2) * slab;
#pragma unroll
          for (int k = 0; k < VPG; ++k) {
            const float4 r = terms[tt * 32 + j * WV + k * G + g];
            const int i0 = __float_as_int(r.w);
            if (i0 >= 0) {
              const float4 cw = tap_weights(r);
              const float c0r = cw.x, c0i = cw.y, c1r = cw.z, c1i = cw.w;
              gather_mac<IQ, VEC, NV, FL, false>(acc[k], base + static_cast<size_t>(i0) * row_elems, row_elems, p.F,
                                                 f_base, jl, c0r, c0i, c1r, c1i);
            }
          }
        }
      }
    }
  }

  // epilogue: complex frames and/or sum_f |y|^2 (Sec. 5), reduced over the FL lanes
#pragma unroll
  for (int k = 0; k < VPG; ++k) {
    const int64_t v = tile_voxel(p, tile, warp * WV + g * VPG + k);
    float pw = 0.f;
#pragma unroll
    for (int m = 0; m < NV; ++m) {
      const int f = f_base + (jl + FL * m) * VEC;
      if (f < p.F) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const float2 a = acc_frame<IQ, VEC>(&acc[k][m * VEC], e);
          pw = fmaf(a.x, a.x, fmaf(a.y, a.y, pw));
        }
        if (v >= 0 && p.y) store_y<IQ, VEC>(p.y + v * p.ystride + f, &acc[k][m * VEC]);
      }
    }
#pragma unroll
    for (int o = FL / 2; o > 0; o >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, o);
    if (jl == 0 && v >= 0 && p.pd) {
      if (p.frame_tiles == 1)
        p.pd[v] = pw;
      else
        p.pd_part[static_cast<int64_t>(blockIdx.y) * p.V + v] = pw;
    }
  }
}

// ---- channel-lane kernel (short ensembles) --------------------------------------------
template <class IQ, int CL, int FMAX, int NWARP>
__global__ void __launch_bounds__(NWARP * 32) k_das_channels(const DasParams p) {
  constexpr int G = 32 / CL;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int g = lane / CL;
  const int jl = lane % CL;
  const int64_t v = tile_voxel(p, static_cast<int64_t>(gridDim.x) - 1 - blockIdx.x, warp * G + g);
  const IQ* __restrict__ iq = static_cast<const IQ*>(p.iq);
  float2 acc[FMAX];
#pragma unroll
  for (int f = 0; f < FMAX; ++f) acc[f] = make_float2(0.f, 0.f);
  if (v >= 0) {
    const float4 vpos = p.vox[v];
    for (int c = jl; c < p.C; c += CL) {
      const TermGeo geo = term_geometry(vpos, __ldg(&p.elem[c]), p);
      if (geo.a < 0.f) continue;
      for (int t = 0; t < p.T; ++t) {
        const float4 r = term_record(__ldg(&p.tx[static_cast<size_t>(t) * p.V + v]), geo, p);
        const int i0 = __float_as_int(r.w);
        if (i0 < 0) continue;
        const float4 cw = tap_weights(r);
        const float c0r = cw.x, c0i = cw.y, c1r = cw.z, c1i = cw.w;
        const IQ* row0 = iq + ((static_cast<size_t>(t) * p.C + c) * p.S + i0) * p.F;
#pragma unroll
        for (int f = 0; f < FMAX; ++f) {
          if (f < p.F) {
            float2 x0[1], x1[1];
            load_vec<IQ, 1, false>(row0 + f, x0);
            load_vec<IQ, 1, false>(row0 + p.F + f, x1);
            mac1(acc[f], c0r, c0i, c1r, c1i, x0[0], x1[0]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int f = 0; f < FMAX; ++f) {
#pragma unroll
    for (int o = CL / 2; o > 0; o >>= 1) {
      acc[f].x += __shfl_xor_sync(0xffffffffu, acc[f].x, o);
      acc[f].y += __shfl_xor_sync(0xffffffffu, acc[f].y, o);
    }
  }
  if (jl == 0 && v >= 0) {
    float pw = 0.f;
#pragma unroll
    for (int f = 0; f < FMAX; ++f) {
      if (f < p.F) {
        pw = fmaf(acc[f].x, acc[f].x, fmaf(acc[f].y, acc[f].y, pw));
        if (p.y) p.y[v * p.ystride + f] = acc[f];
      }
    }
    if (p.pd) p.pd[v] = pw;
  }
}

__global__ void __launch_bounds__(256) k_pd_reduce(const float* __restrict__ part, float* __restrict__ pd,
                                                   int64_t V, int tiles) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float s = 0.f;
  for (int t = 0; t < tiles; ++t) s += part[static_cast<int64_t>(t) * V + v];
  pd[v] = s;
}

// ---- variant table and dispatch -------------------------------------------------------
namespace {
constexpr int kWarps = 8;
//                          name                FPL  lanes vox/warp  FT  warps  ch-lanes
const VariantShape kShapes[] = {
    //  name                      FPL lanes vox/warp FT  warps ch-lanes staged ring bytes type
    {"channels_c64_cl8",           1,  8,   4,    4,  kWarps, true,  false, 0, 8, 0},
    {"frames_c64_ft16",            2,  8,  32,   16,  kWarps, false, false, 0, 8, 0},
    {"frames_c64_ft32",            4,  8,  32,   32,  kWarps, false, false, 0, 8, 0},
    {"frames_c64_ft64",            4, 16,  16,   64,  kWarps, false, false, 0, 8, 0},
    {"frames_c64_scalar_ft32",     1, 32,  16,   32,  kWarps, false, false, 0, 8, 0},
    {"channels_f16_cl8",           1,  8,   4,    4,  kWarps, true,  false, 0, 4, 1},
    {"frames_f16_ft32",            4,  8,  32,   32,  kWarps, false, false, 0, 4, 1},
    {"frames_f16_ft64",            4, 16,  16,   64,  kWarps, false, false, 0, 4, 1},
    {"frames_f16_scalar_ft32",     1, 32,  16,   32,  kWarps, false, false, 0, 4, 1},
    {"staged_c64_ft32",            4,  8,  32,   32,  kWarps, false, true,  4, 8, 0},
    {"staged_c64_ft64",            4, 16,  16,   64,  kWarps, false, true,  4, 8, 0},
    {"staged_f16_ft32",            4,  8,  32,   32,  kWarps, false, true,  4, 4, 1},
    {"staged_f16_ft64",            4, 16,  16,   64,  kWarps, false, true,  4, 4, 1},
    {"staged_c64_ft32_v4",         4,  8,  16,   32,  kWarps, false, true,  4, 8, 0},
    {"staged_c64_ft32_v4w4",       4,  8,  16,   32,  4,      false, true,  4, 8, 0},
    {"staged_c64_ft64_v4",         4, 16,   8,   64,  kWarps, false, true,  8, 8, 0},
    {"staged_f16_ft64_v4",         4, 16,   8,   64,  kWarps, false, true,  8, 4, 1},
    {"channels_b16_cl8",           1,  8,   4,    4,  kWarps, true,  false, 0, 4, 2},
    {"frames_b16_ft32",            4,  8,  32,   32,  kWarps, false, false, 0, 4, 2},
    {"frames_b16_ft64",            4, 16,  16,   64,  kWarps, false, false, 0, 4, 2},
    {"frames_b16_scalar_ft32",     1, 32,  16,   32,  kWarps, false, false, 0, 4, 2},
    {"staged_b16_ft32",            4,  8,  32,   32,  kWarps, false, true,  4, 4, 2},
    {"staged_b16_ft64_v4",         4, 16,   8,   64,  kWarps, false, true,  8, 4, 2},
    {"staged_c64_ft32_v4r56",      4,  8,  16,   32,  kWarps, false, true,  4, 8, 0},
    {"frames_c64p_ft32",           4,  8,  32,   32,  kWarps, false, false, 0, 8, 3},
    {"frames_c64p_ft64",           4, 16,  16,   64,  kWarps, false, false, 0, 8, 3},
    {"staged_c64p_ft32_v4",        4,  8,  16,   32,  kWarps, false, true,  4, 8, 3},
    {"staged_c64p_ft64_v4",        4, 16,   8,   64,  kWarps, false, true,  8, 8, 3},
    {"staged_f16_ft32_v4",         4,  8,  16,   32,  kWarps, false, true,  4, 4, 1},
    {"staged_b16_ft32_v4",         4,  8,  16,   32,  kWarps, false, true,  4, 4, 2},
    {"staged_c64p_ft32_v4w7",      4,  8,  16,   32,  7,      false, true,  4, 8, 3, 8},
    {"staged_c64_ft32_v4w7",       4,  8,  16,   32,  7,      false, true,  4, 8, 0, 8},
    {"staged_c64p_x32_v4w7",       4,  8,  16,   32,  7,      false, true,  4, 8, 3, 8, true},
    {"staged_c64p_x64_v4",         4, 16,   8,   64,  kWarps, false, true,  8, 8, 3, 0, true},
    {"staged_c64p_x32_f4v2w7",     4,  8,   8,   32,  7,      false, true,  8, 8, 3, 4, true},
    {"staged_c64p_x32_f8v1w7",     8,  4,   8,   32,  7,      false, true,  8, 8, 3, 4, true},
    {"staged_c64p_x32_f4v2w15",    4,  8,   8,   32,  15,     false, true,  8, 8, 3, 8, true},
    {"staged_c64p_x32_f8v1w15",    8,  4,   8,   32,  15,     false, true,  8, 8, 3, 8, true},
    {"staged_c64p_x64_f8v2",       8,  8,   8,   64,  kWarps, false, true,  8, 8, 3, 0, true},
    {"staged_c64p_x32_f8v1w15t24", 8,  4,   8,   32,  15,     false, true,  8, 8, 3, 24, true},
    {"staged_c64p_x32_f8v1w15t40", 8,  4,   8,   32,  15,     false, true,  8, 8, 3, 40, true},
    {"staged_c64p_x32_f8v1w15t24s",8,  4,   8,   32,  15,     false, true,  8, 8, 3, 24, true},
    {"staged_c64p_x64_v4s",        4, 16,   8,   64,  kWarps, false, true,  8, 8, 3, 0, true},
    {"staged_c64p_x32_f8v1w7t14",  8,  4,   8,   32,  7,      false, true,  8, 8, 3, 14, true},
    {"staged_c64p_x32_f8v1w7t14e", 8,  4,   8,   32,  7,      false, true,  8, 8, 3, 14, true},
    {"staged_c64p_x32_f4v2w7t14",  4,  8,   8,   32,  7,      false, true,  8, 8, 3, 14, true},
    {"staged_c64p_x32_f8v1w15t30r12",  8, 4, 8,  32,  15,     false, true, 12, 8, 3, 30, true},
    {"staged_c64p_x32_f8v1w15t30r12e", 8, 4, 8,  32,  15,     false, true, 12, 8, 3, 30, true},
    {"staged_c64p_x64_v4e",        4, 16,   8,   64,  kWarps, false, true,  8, 8, 3, 0, true},
    {"staged_c64p_x16_f4v2w7",     4,  4,  16,   16,  7,      false, true,  8, 8, 3, 28, true},
    {"staged_c64p_x16_f4v1w7",     4,  4,   8,   16,  7,      false, true,  8, 8, 3, 14, true},
    {"staged_c64p_x8_f4v1w7",      4,  2,  16,    8,  7,      false, true,  8, 8, 3, 28, true},
    {"channels_c64_cl16",          1, 16,   2,    4,  kWarps, true,  false, 0, 8, 0},
    {"channels_c64_cl32",          1, 32,   1,    4,  kWarps, true,  false, 0, 8, 0},
    {"staged_c64p_x64_v4t16",      4, 16,   8,   64,  kWarps, false, true,  8, 8, 3, 16, true},
    {"staged_c64p_x64_v4t16e",     4, 16,   8,   64,  kWarps, false, true,  8, 8, 3, 16, true},
    {"staged_c64p_x32_v4w7_t8x14", 4,  8,  16,   32,  7,      false, true,  4, 8, 3, 8, true, 8, 14},
    {"staged_c64p_x32_f8v1w7_t8x7e", 8, 4,  8,   32,  7,      false, true,  8, 8, 3, 14, true, 8, 7},
    {"staged_c64p_x64_v4_t8x8",    4, 16,   8,   64,  kWarps, false, true,  8, 8, 3, 16, true, 8, 8},
    {"staged_c64p_x16_f4v2w7_t8x14", 4, 4, 16,   16,  7,      false, true,  8, 8, 3, 28, true, 8, 14},
    {"staged_c64p_x8_f4v1w7_t8x14", 4,  2,  16,    8,  7,      false, true,  8, 8, 3, 28, true, 8, 14},
};
static_assert(sizeof(kShapes) / sizeof(kShapes[0]) == V_COUNT, "one shape row per variant");

template <class K>
cudaError_t go(K kernel, const DasParams& p, size_t smem, cudaStream_t s) {
  const int64_t tiles = static_cast<int64_t>(p.tiles_x) * p.tiles_y * p.tiles_z;
  dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(p.frame_tiles));
  kernel<<<grid, kWarps * 32, smem, s>>>(p);
  return cudaGetLastError();
}
}  // namespace

const VariantShape& variant_shape(Variant v) { return kShapes[v]; }

size_t das_smem_bytes(Variant v) {
  return kShapes[v].channel_lanes ? 0 : static_cast<size_t>(kWarps) * kTxChunk * 32 * sizeof(float4);
}

cudaError_t launch_das(const DasParams& p, Variant v, cudaStream_t s) {
  const size_t sm = das_smem_bytes(v);
  cudaError_t e;
  switch (kShapes[v].staged ? V_COUNT : v) {
    case V_COUNT: e = launch_das_staged(p, v, s); break;
    case V_CH_C64: e = go(k_das_channels<float2, 8, 4, kWarps>, p, sm, s); break;
    case V_CH_C64_L16: e = go(k_das_channels<float2, 16, 4, kWarps>, p, sm, s); break;
    case V_CH_C64_L32: e = go(k_das_channels<float2, 32, 4, kWarps>, p, sm, s); break;
    case V_F16_C64: e = go(k_das_frames<float2, 2, 1, 8, 8, kWarps>, p, sm, s); break;
    case V_F32_C64: e = go(k_das_frames<float2, 2, 2, 8, 8, kWarps>, p, sm, s); break;
    case V_F64_C64: e = go(k_das_frames<float2, 2, 2, 16, 8, kWarps>, p, sm, s); break;
    case V_S32_C64: e = go(k_das_frames<float2, 1, 1, 32, 16, kWarps>, p, sm, s); break;
    case V_CH_H16: e = go(k_das_channels<__half2, 8, 4, kWarps>, p, sm, s); break;
    case V_F32_H16: e = go(k_das_frames<__half2, 4, 1, 8, 8, kWarps>, p, sm, s); break;
    case V_F64_H16: e = go(k_das_frames<__half2, 4, 1, 16, 8, kWarps>, p, sm, s); break;
    case V_S32_H16: e = go(k_das_frames<__half2, 1, 1, 32, 16, kWarps>, p, sm, s); break;
    case V_CH_B16: e = go(k_das_channels<__nv_bfloat162, 8, 4, kWarps>, p, sm, s); break;
    case V_F32_B16: e = go(k_das_frames<__nv_bfloat162, 4, 1, 8, 8, kWarps>, p, sm, s); break;
    case V_F64_B16: e = go(k_das_frames<__nv_bfloat162, 4, 1, 16, 8, kWarps>, p, sm, s); break;
    case V_S32_B16: e = go(k_das_frames<__nv_bfloat162, 1, 1, 32, 16, kWarps>, p, sm, s); break;
    case V_F32_C64P: e = go(k_das_frames<C64Planar, 4, 1, 8, 8, kWarps>, p, sm, s); break;
    case V_F64_C64P: e = go(k_das_frames<C64Planar, 4, 1, 16, 8, kWarps>, p, sm, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (p.frame_tiles > 1 && p.pd) {
    const int64_t blocks = (p.V + 255) / 256;
    k_pd_reduce<<<static_cast<unsigned>(blocks), 256, 0, s>>>(p.pd_part, p.pd, p.V, p.frame_tiles);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace mach
