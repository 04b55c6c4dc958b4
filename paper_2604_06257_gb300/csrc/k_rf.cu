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
// One block per (transmit, element) row and run of kRfNB output samples.  The mixing
// phasor depends only on the RF sample index, so the block evaluates it once per RF sample
// of its window into shared memory (instead of once per tap of every output); threads then
// take (output sample, frame) pairs, consecutive threads consecutive frames, so every RF tap
// read is coalesced over the frame axis.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

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
  }
  const int64_t runs = (p.s_iq + kRfNB - 1) / kRfNB;
  if (runs > 65535 || p.rows > 0x7fffffffLL) return MACH_ERR_UNSUPPORTED;   // grid limits
  if (n_frames > (1 << 24)) return MACH_ERR_UNSUPPORTED;                      // kRfNB * F in 32 bits
  const size_t smem = sizeof(float2) * static_cast<size_t>((kRfNB - 1) * decim + n_taps);
  if (smem > 48 * 1024) return MACH_ERR_UNSUPPORTED;   // (decimation above ~95)
  k_rf_to_iq<<<dim3(static_cast<unsigned>(p.rows), static_cast<unsigned>(runs)), 256, smem,
               static_cast<cudaStream_t>(stream)>>>(p);
  return cudaGetLastError() == cudaSuccess ? MACH_OK : MACH_ERR_CUDA;
}
