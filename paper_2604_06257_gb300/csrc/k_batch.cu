// k_batch.cu -- ragged batches: many DAS instances in one persistent launch.
//
// A batch holds instances of different sizes (2D and 3D grids, element, transmit and
// frame counts).  Their voxel tiles form one work list, sorted by decreasing estimated
// cost; a persistent grid (as many blocks as fit on the GPU) pulls (instance, tile) items
// from an atomic counter until the list is exhausted, so large and small instances
// share the machine without a launch per instance.  The last block to finish resets the
// counter, so the launch can be replayed (e.g. from a CUDA graph) without a host step.
//
// Per item, either of two lane mappings (chosen per instance):
//  - frame lanes: FL lanes share a voxel (FL = 4, 8 or 16 at run time), each lane holds
//    4 frames of 4 voxels; per (element, transmit) every lane evaluates one term and the
//    warp's term table is read back by the lane groups (delay reuse across frames).
//    Taps are read through L1, as 16-byte vectors when F % 4 == 0, else one sample at a
//    time.
//  - channel lanes (F <= 4): 8 lanes share a voxel and split its elements; partial sums
//    meet in a shuffle tree.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "das_term.cuh"
#include "mach_internal.h"
#include "tap_mac.cuh"

namespace mach {

constexpr int kBatchWarps = 8;
constexpr int kBatchTx = 4;   // transmits whose terms are staged per element round

template <class IQ, int VEC, int NV>
__device__ __forceinline__ void batch_frames_tile(const DasParams& p, int FL, int64_t tile, float4* terms) {
  constexpr int VPG = 4;
  constexpr int FPL = VEC * NV;   // 4 frames per lane
  static_assert(FPL == 4, "four frames per lane");
  const int G = 32 / FL;
  const int WV = G * VPG;
  const int CPR = 32 / WV;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int g = lane / FL, jl = lane % FL;
  const IQ* __restrict__ iq = static_cast<const IQ*>(p.iq);
  const int64_t v_term = tile_voxel(p, tile, warp * WV + (lane % WV));
  const float4 vpos = v_term >= 0 ? p.vox[v_term] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int c_sub = lane / WV;
  const int q = lane % WV;
  const int store_at = c_sub * WV + (q % VPG) * G + (q / VPG);

  float2 acc[VPG][FPL];
#pragma unroll
  for (int k = 0; k < VPG; ++k)
#pragma unroll
    for (int e = 0; e < FPL; ++e) acc[k][e] = make_float2(0.f, 0.f);

  const size_t slab = static_cast<size_t>(p.S) * p.F;
  for (int cc = 0; cc < p.C; cc += CPR) {
    const int c = cc + c_sub;
    TermGeo geo;
    geo.rx = 0.f;
    geo.a = -1.f;
    if (v_term >= 0 && c < p.C) geo = term_geometry(vpos, __ldg(&p.elem[c]), p);
    for (int tb = 0; tb < p.T; tb += kBatchTx) {
      const int tn = min(kBatchTx, p.T - tb);
      __syncwarp();
      for (int tt = 0; tt < tn; ++tt) {
        float4 r = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        if (geo.a >= 0.f) r = term_record(__ldg(&p.tx[static_cast<size_t>(tb + tt) * p.V + v_term]), geo, p);
        terms[tt * 32 + store_at] = r;
      }
      __syncwarp();
      for (int tt = 0; tt < tn; ++tt) {
        for (int j = 0; j < CPR; ++j) {
          const int c2 = cc + j;
          if (c2 >= p.C) break;
          const IQ* base = iq + (static_cast<size_t>(tb + tt) * p.C + c2) * slab;
#pragma unroll
          for (int k = 0; k < VPG; ++k) {
            const float4 r = terms[tt * 32 + j * WV + k * G + g];
            const int i0 = __float_as_int(r.w);
            if (i0 >= 0) {
              const float4 cw = tap_weights(r);
              const float c0r = cw.x, c0i = cw.y, c1r = cw.z, c1i = cw.w;
              const IQ* row0 = base + static_cast<size_t>(i0) * p.F;
#pragma unroll
              for (int mm = 0; mm < NV; ++mm) {
                const int f = (jl + FL * mm) * VEC;
                if (f < p.F) {
                  float2 x0[VEC], x1[VEC];
                  load_vec<IQ, VEC, false>(row0 + f, x0);
                  load_vec<IQ, VEC, false>(row0 + p.F + f, x1);
#pragma unroll
                  for (int e = 0; e < VEC; ++e) mac1(acc[k][mm * VEC + e], c0r, c0i, c1r, c1i, x0[e], x1[e]);
                }
              }
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < VPG; ++k) {
    const int64_t v = tile_voxel(p, tile, warp * WV + g * VPG + k);
    float pw = 0.f;
#pragma unroll
    for (int mm = 0; mm < NV; ++mm) {
      const int f = (jl + FL * mm) * VEC;
      if (f < p.F) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) pw = fmaf(acc[k][mm * VEC + e].x, acc[k][mm * VEC + e].x,
                                                fmaf(acc[k][mm * VEC + e].y, acc[k][mm * VEC + e].y, pw));
        if (v >= 0 && p.y) {
          if constexpr (VEC == 4) {
            float2* dst = p.y + v * p.F + f;
            *reinterpret_cast<float4*>(dst) = make_float4(acc[k][mm * 4].x, acc[k][mm * 4].y, acc[k][mm * 4 + 1].x,
                                                          acc[k][mm * 4 + 1].y);
            *reinterpret_cast<float4*>(dst + 2) = make_float4(acc[k][mm * 4 + 2].x, acc[k][mm * 4 + 2].y,
                                                              acc[k][mm * 4 + 3].x, acc[k][mm * 4 + 3].y);
          } else {
            p.y[v * p.F + f] = acc[k][mm];
          }
        }
      }
    }
    for (int o = FL / 2; o > 0; o >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, o);
    if (jl == 0 && v >= 0 && p.pd) p.pd[v] = pw;
  }
}

template <class IQ>
__device__ __forceinline__ void batch_channels_tile(const DasParams& p, int64_t tile) {
  constexpr int CL = 8, G = 32 / CL, FMAX = 4;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int g = lane / CL, jl = lane % CL;
  const int64_t v = tile_voxel(p, tile, warp * G + g);
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
        if (p.y) p.y[v * p.F + f] = acc[f];
      }
    }
    if (p.pd) p.pd[v] = pw;
  }
}

// counter[0]: next work item; counter[1]: blocks that have finished.
template <class IQ>
__global__ void __launch_bounds__(kBatchWarps * 32, 2)
    k_das_batch(const BatchInstance* __restrict__ insts, const int2* __restrict__ items, int n_items, int* counter) {
  __shared__ float4 s_terms[kBatchWarps][kBatchTx * 32];
  __shared__ int s_item;
  const int warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&counter[0], 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const int2 w = items[it];
    const BatchInstance& B = insts[w.x];
    const DasParams p = B.p;
    if (B.mode == kBatchChannels) {
      batch_channels_tile<IQ>(p, w.y);
    } else if (p.F % 4 == 0) {
      batch_frames_tile<IQ, 4, 1>(p, B.frame_lanes, w.y, s_terms[warp]);
    } else {
      batch_frames_tile<IQ, 1, 4>(p, B.frame_lanes, w.y, s_terms[warp]);
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&counter[1], 1) == static_cast<int>(gridDim.x) - 1) {
      counter[0] = 0;
      counter[1] = 0;
      __threadfence();
    }
  }
}

template <class IQ>
static cudaError_t go_batch(const BatchInstance* insts, const int2* items, int n_items, int* counter, int grid,
                            cudaStream_t s) {
  k_das_batch<IQ><<<grid, kBatchWarps * 32, 0, s>>>(insts, items, n_items, counter);
  return cudaGetLastError();
}

int batch_blocks_per_sm(int iq_dtype) {
  int n = 0;
  cudaError_t e;
  switch (iq_dtype) {
    case MACH_IQ_F16X2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_das_batch<__half2>, kBatchWarps * 32, 0); break;
    case MACH_IQ_BF16X2:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_das_batch<__nv_bfloat162>, kBatchWarps * 32, 0);
      break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_das_batch<float2>, kBatchWarps * 32, 0); break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_batch(int iq_dtype, const BatchInstance* insts, const int2* items, int n_items, int* counter,
                         int grid, cudaStream_t s) {
  switch (iq_dtype) {
    case MACH_IQ_C64: return go_batch<float2>(insts, items, n_items, counter, grid, s);
    case MACH_IQ_F16X2: return go_batch<__half2>(insts, items, n_items, counter, grid, s);
    case MACH_IQ_BF16X2: return go_batch<__nv_bfloat162>(insts, items, n_items, counter, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mach
