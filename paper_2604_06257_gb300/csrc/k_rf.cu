// k_rf.cu -- RF input: demodulate real RF channel data into the IQ layout the DAS kernels
// read (the method takes RF or IQ data).
//
//   iq[t][c][n][f] = sum_k h[k] rf[t][c][n D + k - (L-1)/2][f] exp(-j 2 pi fc (t0 + (n D + k - (L-1)/2) / fs))
//
// (RF samples outside [0, S_rf) are zero).  Mixing to baseband, a centred FIR low-pass and
// decimation by D in one pass.  The carrier phase of RF sample m is taken in 32-bit fixed
// point, Phi + m R (mod 2^32) with Phi = round(2^32 frac(fc t0)) and R = round(2^32 frac(fc
// / fs)), the same construction the DAS kernels use for the inverse rotation.
//
// Two kernels, both HBM-bound by design (4 bytes read per RF sample, 8 written per IQ
// sample):
//  * k_rf_poly (even ensembles of 16 frames or more, up to 16 taps per polyphase branch,
//    decimation up to 64): the carrier phase is folded into complex taps, the FIR runs in
//    polyphase form with each loaded sample reused for several outputs in registers, two
//    frames per lane and packed FP32 FMAs (details at the kernel).
//  * k_rf_to_iq (the rest): one block per row and run of kRfNB output samples, the mixing
//    phasors once per RF sample in shared memory, threads over (output sample, frame) pairs
//    with every tap read coalesced over the frame axis.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "async_copy.cuh"
#include "mach.h"

namespace mach {

constexpr int kMaxTaps = 128;

struct RfParams {
  const float* rf;
  float2* iq;
  int64_t rows;        // n_tx * n_elem
  int s_rf, s_iq, F, decim, L;
  uint32_t phi, r;     // carrier phase of sample 0 and per-sample increment, 2^-32 cycles
  float h[kMaxTaps];
  float2 g[kMaxTaps];  // h[k] exp(-j 2 pi k r 2^-32): the taps with the carrier's in-window phase
};

constexpr int kRfNB = 64;   // output samples per block

// grid: (rows, runs of kRfNB output samples); dynamic shared memory: the block's phasors
__global__ void __launch_bounds__(256) k_rf_to_iq(const RfParams p) {
  extern __shared__ float2 rot[];   // (cos, sin) of the carrier phase of RF samples m_lo ...
  const int64_t row = blockIdx.x;
  const int n0 = blockIdx.y * kRfNB;
  const int nb = min(kRfNB, p.s_iq - n0);
  const int m_lo = n0 * p.decim - (p.L - 1) / 2;
  const int span = (nb - 1) * p.decim + p.L;   // RF samples the block's outputs reach
  for (int j = threadIdx.x; j < span; j += blockDim.x) {
    const int m = m_lo + j;
    float s = 0.f, c = 0.f;
    if (m >= 0 && m < p.s_rf) {
      // exp(-j 2 pi phase): phase in cycles as a signed 32-bit fraction of a turn
      const uint32_t ph = p.phi + static_cast<uint32_t>(m) * p.r;
      sincospif(static_cast<float>(static_cast<int32_t>(ph)) * 0x1.0p-31f, &s, &c);
    }
    rot[j] = make_float2(c, s);
  }
  __syncthreads();
  const float* base = p.rf + row * static_cast<int64_t>(p.s_rf) * p.F;
  float2* out = p.iq + (row * p.s_iq + n0) * static_cast<int64_t>(p.F);
  const int outputs = nb * p.F;
  for (int o = threadIdx.x; o < outputs; o += blockDim.x) {
    const int nl = o / p.F, f = o - nl * p.F;
    const int j0 = nl * p.decim;                 // rot index of tap 0
    const int m0 = m_lo + j0;                    // RF sample of tap 0
    // taps whose RF sample exists, so that the loop runs without a branch
    const int k_lo = max(0, -m0), k_hi = min(p.L, p.s_rf - m0);
    const float* src = base + f;
    float re = 0.f, im = 0.f;
#pragma unroll 8
    for (int k = k_lo; k < k_hi; ++k) {
      const float x = p.h[k] * __ldg(src + static_cast<int64_t>(m0 + k) * p.F);
      const float2 cs = rot[j0 + k];
      re = fmaf(x, cs.x, re);
      im = fmaf(-x, cs.y, im);
    }
    out[o] = make_float2(re, im);
  }
}

// Shape measured on the 2D Doppler workload from RF (32 taps, D = 4): 8 outputs per
// half-warp and 4 blocks of 4 warps per SM 41 us; 4 outputs at 6 or 8 blocks 45 / 58 us,
// 16 outputs at 2 blocks 45 us.
constexpr int kPolyK = 8;                         // consecutive output samples per half-warp
constexpr int kPolyWarps = 4;
constexpr int kPolyNB = 2 * kPolyK * kPolyWarps;  // output samples per block
constexpr int kPolyMaxP = 16;                     // taps per polyphase branch

// The carrier phase is linear in the sample index, so for m = n D + k - c (c = (L-1)/2)
//   exp(-j phase(m)) = exp(-j theta(n)) exp(-j 2 pi k r 2^-32),  theta(n) = phase(n D - c)
// (exact in the 32-bit fixed-point phase): the FIR runs on the real RF samples with the
// complex taps g[k] = h[k] exp(-j 2 pi k r 2^-32), and each output is rotated once.
//
// Polyphase form, k = q D + r:  iq[n] = exp(-j theta(n)) sum_r sum_q g[q D + r] x[(n + q) D + r - c].
// A lane takes two adjacent frames (one 8-byte load gives both; with the taps' real and
// imaginary parts each duplicated, one packed FMA serves two outputs) and a half-warp 32
// frames and kPolyK consecutive outputs: for each branch r it loads kPolyK + P - 1 samples
// straight from global memory and reuses each for up to P outputs, the next branch's loads
// in flight while this one multiplies.  Neighbouring half-warps
// share most of their windows, which the L1 cache serves; no shared-memory staging, so
// occupancy is set by registers alone.
// grid: (runs of kPolyNB outputs, frame tiles of 32, rows); needs F even and the RF 8-byte aligned.
template <int P>
__device__ __forceinline__ void poly_load(float2 (&w)[kPolyK + P - 1], const float* xb, int m0, int r, int D,
                                          int64_t step, bool interior, int s_rf, int64_t F) {
  const float* xr = xb + static_cast<int64_t>(m0 + r) * F;
  if (interior) {
#pragma unroll
    for (int t = 0; t < kPolyK + P - 1; ++t) w[t] = __ldg(reinterpret_cast<const float2*>(xr + t * step));
  } else {
#pragma unroll
    for (int t = 0; t < kPolyK + P - 1; ++t) {
      const int m = m0 + r + t * D;
      w[t] = (m >= 0 && m < s_rf) ? __ldg(reinterpret_cast<const float2*>(xr + t * step)) : make_float2(0.f, 0.f);
    }
  }
}

template <int P>
__device__ __forceinline__ void poly_mac(const float2 (&w)[kPolyK + P - 1], const float4* gr, float2 (&re)[kPolyK],
                                         float2 (&im)[kPolyK]) {
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const float4 g = gr[q];
    const float2 gre = make_float2(g.x, g.y), gim = make_float2(g.z, g.w);
#pragma unroll
    for (int i = 0; i < kPolyK; ++i) {
      re[i] = __ffma2_rn(gre, w[i + q], re[i]);
      im[i] = __ffma2_rn(gim, w[i + q], im[i]);
    }
  }
}

template <int P>
__global__ void __launch_bounds__(32 * kPolyWarps, P >= 16 ? 3 : 4) k_rf_poly(const RfParams p) {
  __shared__ float4 g4[kPolyMaxP * 64];     // [D][P]: (re, re, im, im); D <= 64 here
  __shared__ float2 rout[kPolyNB];          // exp(-j theta(n))
  const int D = p.decim, c_half = (p.L - 1) / 2;
  const int n0 = blockIdx.x * kPolyNB, f0 = blockIdx.y * 32;
  const int64_t row = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = tid; k < P * D; k += blockDim.x) {
    const int r = k / P, q = k - r * P, tap = q * D + r;
    const float2 g = tap < p.L ? p.g[tap] : make_float2(0.f, 0.f);
    g4[k] = make_float4(g.x, g.x, g.y, g.y);
  }
  for (int t = tid; t < kPolyNB; t += blockDim.x) {
    // exp(-j 2 pi theta): theta in cycles as a signed 32-bit fraction of a turn
    const uint32_t ph = p.phi + static_cast<uint32_t>((n0 + t) * D - c_half) * p.r;
    float sn, cs;
    sincospif(static_cast<float>(static_cast<int32_t>(ph)) * 0x1.0p-31f, &sn, &cs);
    rout[t] = make_float2(cs, -sn);
  }
  __syncthreads();
  const int half = lane >> 4;
  const int nl = (2 * warp + half) * kPolyK;
  const int f = f0 + 2 * (lane & 15);
  if (f >= p.F || n0 + nl >= p.s_iq) return;
  const float* xb = p.rf + row * static_cast<int64_t>(p.s_rf) * p.F + f;
  const int m0 = (n0 + nl) * D - c_half;            // RF sample of output n0 + nl, tap 0
  const bool interior = m0 >= 0 && m0 + (kPolyK + P - 1) * D - 1 < p.s_rf;
  const int64_t step = static_cast<int64_t>(D) * p.F;
  float2 re[kPolyK], im[kPolyK];
#pragma unroll
  for (int i = 0; i < kPolyK; ++i) re[i] = im[i] = make_float2(0.f, 0.f);
  // branches in pairs, the next branch's samples loading while this one's multiply
  float2 wa[kPolyK + P - 1], wb[kPolyK + P - 1];
  poly_load<P>(wa, xb, m0, 0, D, step, interior, p.s_rf, p.F);
  for (int r = 0; r < D; r += 2) {
    if (r + 1 < D) poly_load<P>(wb, xb, m0, r + 1, D, step, interior, p.s_rf, p.F);
    poly_mac<P>(wa, g4 + r * P, re, im);
    if (r + 1 < D) {
      if (r + 2 < D) poly_load<P>(wa, xb, m0, r + 2, D, step, interior, p.s_rf, p.F);
      poly_mac<P>(wb, g4 + (r + 1) * P, re, im);
    }
  }
  float2* out = p.iq + (row * p.s_iq + n0 + nl) * static_cast<int64_t>(p.F) + f;
#pragma unroll
  for (int i = 0; i < kPolyK; ++i) {
    if (n0 + nl + i < p.s_iq) {
      const float2 e = rout[nl + i];
      *reinterpret_cast<float4*>(out) =
          make_float4(fmaf(re[i].x, e.x, -im[i].x * e.y), fmaf(re[i].x, e.y, im[i].x * e.x),
                      fmaf(re[i].y, e.x, -im[i].y * e.y), fmaf(re[i].y, e.y, im[i].y * e.x));
    }
    out += p.F;
  }
}

template <int P>
cudaError_t launch_poly(const RfParams& p, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>((p.s_iq + kPolyNB - 1) / kPolyNB), static_cast<unsigned>((p.F + 31) / 32),
                  static_cast<unsigned>(p.rows));
  k_rf_poly<P><<<grid, 32 * kPolyWarps, 0, s>>>(p);
  return cudaGetLastError();
}

// Whether the polyphase kernel takes these sizes: an even number of frames, 16 or more,
// 16-byte aligned IQ and 8-byte aligned RF, at most kPolyMaxP taps per branch and
// decimation at most 64 (the taps fit the block's table), and the grid's limits.
bool poly_applies(const RfParams& p) {
  if (p.F < 16 || p.F % 2 || (reinterpret_cast<uintptr_t>(p.rf) & 7u) || (reinterpret_cast<uintptr_t>(p.iq) & 15u))
    return false;
  if (p.decim > 64 || (p.L + p.decim - 1) / p.decim > kPolyMaxP) return false;
  if ((p.s_iq + kPolyNB - 1) / kPolyNB > INT32_MAX || (p.F + 31) / 32 > 65535 || p.rows > 65535) return false;
  // RF sample indices n D + k in 32 bits
  return static_cast<int64_t>(p.s_iq + kPolyNB) * p.decim + p.L < INT32_MAX;
}

cudaError_t launch_rf_poly(const RfParams& p, cudaStream_t s) {
  const int P = (p.L + p.decim - 1) / p.decim;
  if (P <= 1) return launch_poly<1>(p, s);
  if (P <= 2) return launch_poly<2>(p, s);
  if (P <= 4) return launch_poly<4>(p, s);
  if (P <= 8) return launch_poly<8>(p, s);
  return launch_poly<16>(p, s);
}

namespace {
uint32_t fixed_turns(double cycles) {
  double fr = cycles - std::floor(cycles);
  double v = std::nearbyint(fr * 4294967296.0);
  if (v >= 4294967296.0) v -= 4294967296.0;
  return static_cast<uint32_t>(v);
}
}  // namespace

}  // namespace mach

using namespace mach;

extern "C" mach_status mach_rf_to_iq(const float* rf, void* iq, int32_t n_tx, int32_t n_elem, int32_t n_rf,
                                     int32_t n_frames, double fs_rf, double fc, double t0, const float* taps,
                                     int32_t n_taps, int32_t decim, void* stream) {
  if (!rf || !iq || !taps || n_tx < 1 || n_elem < 1 || n_rf < 1 || n_frames < 1) return MACH_ERR_INVALID_ARG;
  if (n_taps < 1 || n_taps > kMaxTaps || decim < 1 || decim > n_rf) return MACH_ERR_INVALID_ARG;
  if (!(fs_rf > 0.0) || !std::isfinite(fs_rf) || !(fc >= 0.0) || !std::isfinite(fc) || !std::isfinite(t0))
    return MACH_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(rf) & 3u) || (reinterpret_cast<uintptr_t>(iq) & 7u)) return MACH_ERR_INVALID_ARG;
  RfParams p{};
  p.rf = rf;
  p.iq = static_cast<float2*>(iq);
  p.rows = static_cast<int64_t>(n_tx) * n_elem;
  p.s_rf = n_rf;
  p.s_iq = (n_rf - 1) / decim + 1;
  p.F = n_frames;
  p.decim = decim;
  p.L = n_taps;
  p.phi = fixed_turns(fc * t0);
  p.r = fixed_turns(fc / fs_rf);
  for (int k = 0; k < n_taps; ++k) {
    if (!std::isfinite(taps[k])) return MACH_ERR_INVALID_ARG;
    p.h[k] = taps[k];
    // exp(-j 2 pi k r 2^-32), the phase reduced exactly in 32-bit fixed point
    const double ph = static_cast<double>(static_cast<uint32_t>(static_cast<uint64_t>(k) * p.r)) * 0x1.0p-32;
    p.g[k] = make_float2(static_cast<float>(taps[k] * std::cos(6.283185307179586 * ph)),
                         static_cast<float>(-taps[k] * std::sin(6.283185307179586 * ph)));
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (poly_applies(p)) return launch_rf_poly(p, st) == cudaSuccess ? MACH_OK : MACH_ERR_CUDA;
  const int64_t runs = (p.s_iq + kRfNB - 1) / kRfNB;
  if (runs > 65535 || p.rows > 0x7fffffffLL) return MACH_ERR_UNSUPPORTED;   // grid limits
  if (n_frames > (1 << 24)) return MACH_ERR_UNSUPPORTED;                      // kRfNB * F in 32 bits
  const size_t smem = sizeof(float2) * static_cast<size_t>((kRfNB - 1) * decim + n_taps);
  if (smem > 48 * 1024) return MACH_ERR_UNSUPPORTED;   // (decimation above ~95)
  k_rf_to_iq<<<dim3(static_cast<unsigned>(p.rows), static_cast<unsigned>(runs)), 256, smem, st>>>(p);
  return cudaGetLastError() == cudaSuccess ? MACH_OK : MACH_ERR_CUDA;
}
