// host_stream.cpp -- Power Doppler of a sequence of acquisitions held in host memory,
// pipelined: the upload of acquisition k+1 overlaps the conversion (K0) and beamforming of
// acquisition k and the download of k-1.  Two device staging sets, three streams (upload,
// compute, download) ordered by events; the host only enqueues.
#include <cuda_runtime.h>

#include <cstdint>

#include "mach.h"
#include "mach_internal.h"

using namespace mach;

namespace {

struct Pipeline {
  void* raw[2] = {nullptr, nullptr};    // complex64 acquisitions as uploaded
  void* conv[2] = {nullptr, nullptr};   // the plan's IQ layout and storage type
  float* pd[2] = {nullptr, nullptr};
  void* y[2] = {nullptr, nullptr};
  cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
  cudaEvent_t uploaded[2] = {}, converted[2] = {}, beamformed[2] = {}, downloaded[2] = {};

  ~Pipeline() {
    if (up) cudaStreamSynchronize(up);
    if (comp) cudaStreamSynchronize(comp);
    if (down) cudaStreamSynchronize(down);
    for (int b = 0; b < 2; ++b) {
      cudaFree(raw[b]);
      cudaFree(conv[b]);
      cudaFree(pd[b]);
      cudaFree(y[b]);
      for (cudaEvent_t e : {uploaded[b], converted[b], beamformed[b], downloaded[b]})
        if (e) cudaEventDestroy(e);
    }
    for (cudaStream_t s : {up, comp, down})
      if (s) cudaStreamDestroy(s);
  }
};

size_t sample_bytes(int dtype) { return (dtype == MACH_IQ_F16X2 || dtype == MACH_IQ_BF16X2) ? 4 : 8; }

}  // namespace

extern "C" mach_status mach_power_doppler_host_stream(mach_plan p, const void* const* iq_host, int32_t src_order,
                                                      float* const* pd_host, void* const* y_host, int32_t count) {
  if (!p || !iq_host || !pd_host || count < 1) return MACH_ERR_INVALID_ARG;
  if (src_order != -1 && src_order != MACH_ORDER_TCSF && src_order != MACH_ORDER_FTCS) return MACH_ERR_INVALID_ARG;
  for (int k = 0; k < count; ++k)
    if (!iq_host[k] || !pd_host[k] || (y_host && !y_host[k])) return MACH_ERR_INVALID_ARG;
  const DasParams& b = *plan_params(p);
  const int dtype = plan_iq_dtype(p);
  const size_t samples = static_cast<size_t>(b.T) * b.C * b.S * b.F;
  const bool convert = src_order >= 0;
  const size_t conv_bytes = sample_bytes(dtype) * samples;
  const size_t raw_bytes = convert ? 8 * samples : conv_bytes;
  const size_t pd_bytes = sizeof(float) * static_cast<size_t>(b.V);
  const size_t y_bytes = 8 * static_cast<size_t>(b.V) * b.F;

  Pipeline q;
  auto oom = [](cudaError_t e) { return e == cudaErrorMemoryAllocation ? MACH_ERR_OOM : MACH_ERR_CUDA; };
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    if ((e = cudaMalloc(&q.raw[i], raw_bytes)) != cudaSuccess) break;
    if (convert && (e = cudaMalloc(&q.conv[i], conv_bytes)) != cudaSuccess) break;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&q.pd[i]), pd_bytes)) != cudaSuccess) break;
    if (y_host && (e = cudaMalloc(&q.y[i], y_bytes)) != cudaSuccess) break;
    for (cudaEvent_t* ev : {&q.uploaded[i], &q.converted[i], &q.beamformed[i], &q.downloaded[i]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  }
  for (cudaStream_t* s : {&q.up, &q.comp, &q.down})
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return oom(e);
  }

  for (int k = 0; k < count; ++k) {
    const int i = k & 1;
    // staging set i was last used by acquisition k - 2: its upload buffer is free once K0
    // (or, without conversion, the beamformer) has read it, its outputs once they have been
    // downloaded
    if (k >= 2 && (e = cudaStreamWaitEvent(q.up, q.converted[i], 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(q.raw[i], iq_host[k], raw_bytes, cudaMemcpyHostToDevice, q.up)) != cudaSuccess) break;
    if ((e = cudaEventRecord(q.uploaded[i], q.up)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(q.comp, q.uploaded[i], 0)) != cudaSuccess) break;
    mach_status st = MACH_OK;
    if (convert && (st = mach_iq_convert(q.raw[i], src_order, q.conv[i], dtype, b.T, b.C, b.S, b.F, q.comp)) != MACH_OK)
      return st;
    if (convert && (e = cudaEventRecord(q.converted[i], q.comp)) != cudaSuccess) break;
    if (k >= 2 && (e = cudaStreamWaitEvent(q.comp, q.downloaded[i], 0)) != cudaSuccess) break;
    st = mach_power_doppler(p, convert ? q.conv[i] : q.raw[i], q.pd[i], y_host ? q.y[i] : nullptr, q.comp);
    if (st != MACH_OK) return st;
    if ((e = cudaEventRecord(q.beamformed[i], q.comp)) != cudaSuccess) break;
    if (!convert && (e = cudaEventRecord(q.converted[i], q.comp)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(q.down, q.beamformed[i], 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(pd_host[k], q.pd[i], pd_bytes, cudaMemcpyDeviceToHost, q.down)) != cudaSuccess) break;
    if (y_host &&
        (e = cudaMemcpyAsync(y_host[k], q.y[i], y_bytes, cudaMemcpyDeviceToHost, q.down)) != cudaSuccess)
      break;
    if ((e = cudaEventRecord(q.downloaded[i], q.down)) != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(q.down);
  if (e == cudaSuccess) e = cudaStreamSynchronize(q.comp);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MACH_ERR_CUDA;
  }
  return mach_plan_device_status(p, nullptr);
}
