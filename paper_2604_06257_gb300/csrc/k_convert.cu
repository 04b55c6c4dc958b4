// k_convert.cu -- K0: channel data into the frame-contiguous layout and storage type.
//
// Scanners deliver frames one after another ([frame][transmit][element][sample]); the DAS
// kernels want the frames of one sample contiguous ([transmit][element][sample][frame],
// Sec. 4.4's [elements, samples, frames] with a transmit axis in front), optionally stored
// as float16 or bfloat16 pairs (rounded to nearest even) to halve the gathered bytes.
// The reorder is a batched transpose (F x N -> N x F, N = T*C*S), done through 32 x 32
// shared-memory tiles so that both the reads (along N) and the writes (along F) are
// coalesced.  Bound by HBM bandwidth: 8 bytes read and 4 or 8 bytes written per sample.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>

#include "mach_internal.h"

namespace mach {

template <int DT>
__device__ __forceinline__ void put(void* dst, int64_t n, int64_t f, int64_t F, float2 v) {
  const int64_t i = n * F + f;
  if constexpr (DT == MACH_IQ_C64_SPLIT) {
    static_cast<float*>(dst)[2 * n * F + f] = v.x;
    static_cast<float*>(dst)[2 * n * F + F + f] = v.y;
  } else if constexpr (DT == MACH_IQ_C64) {
    static_cast<float2*>(dst)[i] = v;
  } else if constexpr (DT == MACH_IQ_F16X2) {
    static_cast<__half2*>(dst)[i] = __float22half2_rn(v);
  } else {
    static_cast<__nv_bfloat162*>(dst)[i] = __float22bfloat162_rn(v);
  }
}

// src [F][N] -> dst [N][F]; block (32, 8), tile 32 (n) x 32 (f).
template <int DT>
__global__ void __launch_bounds__(256) k_transpose_frames(const float2* __restrict__ src, void* __restrict__ dst,
                                                          int64_t N, int64_t F) {
  __shared__ float2 tile[32][33];
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int64_t f0 = static_cast<int64_t>(blockIdx.y) * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t f = f0 + j, n = n0 + threadIdx.x;
    if (f < F && n < N) tile[j][threadIdx.x] = __ldg(&src[f * N + n]);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t n = n0 + j, f = f0 + threadIdx.x;
    if (n < N && f < F) put<DT>(dst, n, f, F, tile[threadIdx.x][j]);
  }
}

// The same transpose with more bytes in flight per thread: NT (n) x 32 (f) tiles, 16-byte
// loads of two consecutive samples along n (N even, 16-byte aligned source), NT / 8 rows per
// thread on the way out.  NT = 64 measured best (complex64 output 4.9 TB/s against 3.8 TB/s
// for 32 x 32 tiles with 8-byte loads, and 4.6 TB/s for NT = 128).
template <int DT, int NT>
__global__ void __launch_bounds__(256) k_transpose_frames2(const float2* __restrict__ src, void* __restrict__ dst,
                                                           int64_t N, int64_t F) {
  constexpr int L = NT / 64;   // 16-byte loads per thread and f row
  __shared__ float2 tile[32][NT + 1];
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * NT;
  const int64_t f0 = static_cast<int64_t>(blockIdx.y) * 32;
  float4 v[4][L];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t f = f0 + threadIdx.y + 8 * k;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const int64_t n = n0 + 64 * l + 2 * threadIdx.x;
      v[k][l] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (f < F && n < N) v[k][l] = __ldg(reinterpret_cast<const float4*>(src + f * N + n));
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < L; ++l) {
      tile[threadIdx.y + 8 * k][64 * l + 2 * threadIdx.x] = make_float2(v[k][l].x, v[k][l].y);
      tile[threadIdx.y + 8 * k][64 * l + 2 * threadIdx.x + 1] = make_float2(v[k][l].z, v[k][l].w);
    }
  __syncthreads();
  const int64_t f = f0 + threadIdx.x;
#pragma unroll
  for (int k = 0; k < NT / 8; ++k) {
    const int j = threadIdx.y + 8 * k;
    const int64_t nn = n0 + j;
    if (nn < N && f < F) put<DT>(dst, nn, f, F, tile[threadIdx.x][j]);
  }
}

// The 64 x 32 transpose with 16-byte stores as well: a thread writes V consecutive frames of
// one sample (V = 2 for complex64, 4 for the 16-bit pairs and for split rows), so the frame
// count must be a multiple of V and the destination 16-byte aligned (split rows: F % 4 == 0
// puts both rows of every sample on the 16-byte grid).  The tile holds pairs of consecutive
// samples as 16-byte slots, slot p of frame row f stored at p ^ (f / 2): the row-wise
// 16-byte stores of the load phase and the column-wise reads of V frames at one sample both
// spread over all banks.
template <int DT>
__global__ void __launch_bounds__(256) k_transpose_frames3(const float2* __restrict__ src, void* __restrict__ dst,
                                                           int64_t N, int64_t F) {
  constexpr int NT = 64;
  constexpr int V = DT == MACH_IQ_C64 ? 2 : 4;
  constexpr int TPR = 32 / V;            // threads per sample row of 32 frames
  constexpr int RPP = 256 / TPR;         // sample rows per pass
  __shared__ float4 tile4[32][NT / 2];
  const float2(*tile)[NT] = reinterpret_cast<const float2(*)[NT]>(tile4);
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * NT;
  const int64_t f0 = static_cast<int64_t>(blockIdx.y) * 32;
  float4 v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t f = f0 + threadIdx.y + 8 * k;
    const int64_t n = n0 + 2 * threadIdx.x;
    v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (f < F && n < N) v[k] = __ldg(reinterpret_cast<const float4*>(src + f * N + n));
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = threadIdx.y + 8 * k;
    tile4[r][threadIdx.x ^ (r >> 1)] = v[k];
  }
  __syncthreads();
  // sample j of frame row r, in the swizzled tile
  auto at = [&](int r, int j) { return tile[r][2 * ((j >> 1) ^ (r >> 1)) + (j & 1)]; };
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int tc = tid % TPR, tr = tid / TPR;
  const int fl = V * tc;
  const int64_t f = f0 + fl;
  if (f >= F) return;
#pragma unroll
  for (int k = 0; k < NT / RPP; ++k) {
    const int j = tr + k * RPP;
    const int64_t n = n0 + j;
    if (n >= N) continue;
    if constexpr (DT == MACH_IQ_C64) {
      const float2 a = at(fl, j), b = at(fl + 1, j);
      *reinterpret_cast<float4*>(static_cast<float2*>(dst) + n * F + f) = make_float4(a.x, a.y, b.x, b.y);
    } else if constexpr (DT == MACH_IQ_C64_SPLIT) {
      const float2 a = at(fl, j), b = at(fl + 1, j), c = at(fl + 2, j), d = at(fl + 3, j);
      float* row = static_cast<float*>(dst) + 2 * n * F;
      *reinterpret_cast<float4*>(row + f) = make_float4(a.x, b.x, c.x, d.x);
      *reinterpret_cast<float4*>(row + F + f) = make_float4(a.y, b.y, c.y, d.y);
    } else {
      uint32_t h[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 a = at(fl + e, j);
        if constexpr (DT == MACH_IQ_F16X2) {
          const __half2 q = __float22half2_rn(a);
          h[e] = *reinterpret_cast<const uint32_t*>(&q);
        } else {
          const __nv_bfloat162 q = __float22bfloat162_rn(a);
          h[e] = *reinterpret_cast<const uint32_t*>(&q);
        }
      }
      *reinterpret_cast<uint4*>(static_cast<uint32_t*>(dst) + n * F + f) = make_uint4(h[0], h[1], h[2], h[3]);
    }
  }
}

// Same layout, storage type only.
template <int DT>
__global__ void __launch_bounds__(256) k_cast(const float2* __restrict__ src, void* __restrict__ dst, int64_t total,
                                              int64_t F) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    put<DT>(dst, i / F, i % F, F, __ldg(&src[i]));
}

template <int DT>
cudaError_t convert_as(const float2* src, int order, void* dst, int64_t N, int64_t F, cudaStream_t s) {
  const bool src16 = (reinterpret_cast<uintptr_t>(src) & 15u) == 0, dst16 = (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
  if (order == 1 && N % 2 == 0 && src16 && dst16 && F % (DT == MACH_IQ_C64 ? 2 : 4) == 0) {
    const dim3 grid(static_cast<unsigned>((N + 63) / 64), static_cast<unsigned>((F + 31) / 32));
    k_transpose_frames3<DT><<<grid, dim3(32, 8), 0, s>>>(src, dst, N, F);
  } else if (order == 1 && N % 2 == 0 && src16) {
    const dim3 grid(static_cast<unsigned>((N + 63) / 64), static_cast<unsigned>((F + 31) / 32));
    k_transpose_frames2<DT, 64><<<grid, dim3(32, 8), 0, s>>>(src, dst, N, F);
  } else if (order == 1) {
    const dim3 grid(static_cast<unsigned>((N + 31) / 32), static_cast<unsigned>((F + 31) / 32));
    k_transpose_frames<DT><<<grid, dim3(32, 8), 0, s>>>(src, dst, N, F);
  } else {
    const int64_t total = N * F;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_cast<DT><<<static_cast<unsigned>(blocks), 256, 0, s>>>(src, dst, total, F);
  }
  return cudaGetLastError();
}

cudaError_t launch_iq_convert(const float2* src, int src_order, void* dst, int dst_dtype, int64_t T, int64_t C,
                              int64_t S, int64_t F, cudaStream_t s) {
  const int64_t N = T * C * S;
  switch (dst_dtype) {
    case MACH_IQ_C64: return convert_as<MACH_IQ_C64>(src, src_order, dst, N, F, s);
    case MACH_IQ_F16X2: return convert_as<MACH_IQ_F16X2>(src, src_order, dst, N, F, s);
    case MACH_IQ_BF16X2: return convert_as<MACH_IQ_BF16X2>(src, src_order, dst, N, F, s);
    case MACH_IQ_C64_SPLIT: return convert_as<MACH_IQ_C64_SPLIT>(src, src_order, dst, N, F, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mach

using namespace mach;

extern "C" mach_status mach_iq_convert(const void* src_dev, int32_t src_order, void* dst_dev, int32_t dst_dtype,
                                       int32_t n_tx, int32_t n_elem, int32_t n_samples, int32_t n_frames,
                                       void* stream) {
  if (!src_dev || !dst_dev || src_dev == dst_dev) return MACH_ERR_INVALID_ARG;
  if (src_order != MACH_ORDER_TCSF && src_order != MACH_ORDER_FTCS) return MACH_ERR_INVALID_ARG;
  if (dst_dtype < MACH_IQ_C64 || dst_dtype > MACH_IQ_C64_SPLIT) return MACH_ERR_INVALID_ARG;
  if (n_tx < 1 || n_elem < 1 || n_samples < 1 || n_frames < 1) return MACH_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(src_dev) & 7u) || (reinterpret_cast<uintptr_t>(dst_dev) & 3u))
    return MACH_ERR_INVALID_ARG;
  const int64_t N = static_cast<int64_t>(n_tx) * n_elem * n_samples;
  if (src_order == MACH_ORDER_FTCS && (N + 31) / 32 > INT32_MAX) return MACH_ERR_UNSUPPORTED;
  if (src_order == MACH_ORDER_FTCS && (n_frames + 31) / 32 > 65535) return MACH_ERR_UNSUPPORTED;
  const cudaError_t e = launch_iq_convert(static_cast<const float2*>(src_dev), src_order, dst_dev, dst_dtype, n_tx,
                                          n_elem, n_samples, n_frames, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MACH_OK : MACH_ERR_CUDA;
}
