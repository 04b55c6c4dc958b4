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
// One thread per output sample; consecutive threads take consecutive frames, so every RF
// tap read is coalesced over the frame axis.
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

__global__ void __launch_bounds__(256) k_rf_to_iq(const RfParams p) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = p.rows * p.s_iq * p.F;
  if (i >= total) return;
  const int f = static_cast<int>(i % p.F);
  const int64_t q = i / p.F;
  const int n = static_cast<int>(q % p.s_iq);
  const int64_t row = q / p.s_iq;
  const float* src = p.rf + row * static_cast<int64_t>(p.s_rf) * p.F + f;
  const int m0 = n * p.decim - (p.L - 1) / 2;
  float re = 0.f, im = 0.f;
  for (int k = 0; k < p.L; ++k) {
    const int m = m0 + k;
    if (m < 0 || m >= p.s_rf) continue;
    const float x = p.h[k] * __ldg(src + static_cast<int64_t>(m) * p.F);
    // exp(-j 2 pi phase): phase in cycles as a signed 32-bit fraction of a turn
    const uint32_t ph = p.phi + static_cast<uint32_t>(m) * p.r;
    float s, c;
    sincospif(static_cast<float>(static_cast<int32_t>(ph)) * 0x1.0p-31f, &s, &c);
    re = fmaf(x, c, re);
    im = fmaf(-x, s, im);
  }
  p.iq[i] = make_float2(re, im);
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
  const int64_t total = p.rows * p.s_iq * p.F;
  if ((total + 255) / 256 > 0x7fffffffLL) return MACH_ERR_UNSUPPORTED;
  k_rf_to_iq<<<static_cast<unsigned>((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(p);
  return cudaGetLastError() == cudaSuccess ? MACH_OK : MACH_ERR_CUDA;
}
