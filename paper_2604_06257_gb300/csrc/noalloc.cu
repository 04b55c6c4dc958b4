// noalloc.cu -- delay-and-sum without any device allocation.
//
// For callers that cannot call cudaMalloc: code running where the allocator is off
// limits (for example inside a host callback, under an external memory budget that
// forbids new allocations, or in a host framework that owns all device memory), or
// that must not pay an allocation on first use.  The per-call tables a plan would own
// (voxel and element positions in sample units, transmit delays, partial Power Doppler
// sums) live instead in one file-scope device array, g_scratch, of kScratchBytes bytes,
// which every GPU that loads this library keeps until the process exits.
//
// The array's name is only a host-side stand-in in host code, so its device address is
// fetched with cudaGetSymbolAddress, once per device, on the first call made with that
// device current; that first call should therefore come before any stream capture.  The
// address is kept for the life of the process (a cudaDeviceReset would make it stale).
// Every call reuses the same array and leaves the last call's tables in it: calls that
// overlap on the GPU (different streams, or different host threads) race on it.  Each
// call rewrites every table entry it reads, so nothing has to start at zero.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "mach.h"
#include "mach_internal.h"

namespace mach {
namespace {

constexpr size_t kScratchBytes = size_t{8} << 20;   // 8 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// A failed CUDA call leaves its error as the runtime's last error; clear it so that the
// caller's next launch check does not report this call's failure again.
mach_status cuda_fail() {
  cudaGetLastError();
  return MACH_ERR_CUDA;
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up on first use).
mach_status scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cuda_fail();
  if (dev < 0 || dev >= kMaxDevices) return MACH_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return cuda_fail();
    g_scratch_dev[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_dev[dev];
  return MACH_OK;
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace
}  // namespace mach

using namespace mach;

extern "C" mach_status mach_das_run_noalloc(const mach_das_desc* d, const void* iq_dev, void* y_dev_or_null,
                                            float* pd_dev_or_null, void* stream) {
  mach_status st = host_validate(d);
  if (st != MACH_OK) return st;
  if (d->term_table) return MACH_ERR_UNSUPPORTED;   // a term table is plan state
  if (!iq_dev || (!y_dev_or_null && !pd_dev_or_null)) return MACH_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(iq_dev) & 15u) || (reinterpret_cast<uintptr_t>(y_dev_or_null) & 15u) ||
      (reinterpret_cast<uintptr_t>(pd_dev_or_null) & 3u))
    return MACH_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  const int C = d->n_elem, T = d->n_tx, S = d->n_samples, F = d->n_frames;
  const bool list = d->vox_pos != nullptr;
  const int64_t V = list ? d->n_vox
                         : static_cast<int64_t>(d->grid_dims[0]) * d->grid_dims[1] * d->grid_dims[2];
  if (list && V > INT32_MAX) return MACH_ERR_UNSUPPORTED;
  const Variant var = host_unstaged_variant(d->iq_dtype, F);

  DasParams b{};
  if (list) {
    b.nx = static_cast<int>(V);
    b.ny = b.nz = 1;
  } else {
    b.nx = d->grid_dims[0];
    b.ny = d->grid_dims[1];
    b.nz = d->grid_dims[2];
  }
  if ((st = host_configure_tiles(b, var, list, V, F)) != MACH_OK) return st;

  // scratch layout; reject anything that does not fit before touching the device
  const size_t off_vox = 0;
  const size_t off_elem = off_vox + align256(sizeof(float4) * static_cast<size_t>(V));
  const size_t off_tx = off_elem + align256(sizeof(float4) * static_cast<size_t>(C));
  const size_t off_u = off_tx + align256(sizeof(float) * static_cast<size_t>(T) * V);
  const size_t off_raw = off_u + align256(d->tx_table_dev ? 0 : sizeof(double) * 3 * static_cast<size_t>(T));
  const size_t off_part = off_raw + align256(list ? sizeof(float) * 3 * static_cast<size_t>(V) : 0);
  const bool need_part = b.frame_tiles > 1 && pd_dev_or_null;
  const size_t end = off_part + align256(need_part ? sizeof(float) * static_cast<size_t>(b.frame_tiles) * V : 0);
  if (end > kScratchBytes) return MACH_ERR_UNSUPPORTED;
  // The host arrays below are copied from this call's own (pageable, short-lived) buffers;
  // a graph captured around the call would read them again at replay, after they are gone.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return cuda_fail();
  if (cap != cudaStreamCaptureStatusNone) return MACH_ERR_UNSUPPORTED;

  unsigned char* base = nullptr;
  if ((st = scratch_address(&base)) != MACH_OK) return st;

  const double k = d->fs / d->c;
  std::vector<float4> elem(C);
  for (int c = 0; c < C; ++c)
    elem[c] = make_float4(static_cast<float>(static_cast<double>(d->elem_pos[3 * c]) * k),
                          static_cast<float>(static_cast<double>(d->elem_pos[3 * c + 1]) * k),
                          static_cast<float>(static_cast<double>(d->elem_pos[3 * c + 2]) * k), 0.0f);
  std::vector<double> u;
  if (!d->tx_table_dev) {
    u.resize(3 * static_cast<size_t>(T));
    for (int t = 0; t < T; ++t) {
      const double az = d->tx_angles[2 * t], el = d->tx_angles[2 * t + 1];
      u[3 * t] = std::sin(az) * std::cos(el);
      u[3 * t + 1] = std::sin(el);
      u[3 * t + 2] = std::cos(az) * std::cos(el);
    }
  }
  float4* d_vox = reinterpret_cast<float4*>(base + off_vox);
  float4* d_elem = reinterpret_cast<float4*>(base + off_elem);
  float* d_tx = reinterpret_cast<float*>(base + off_tx);
  double* d_u = u.empty() ? nullptr : reinterpret_cast<double*>(base + off_u);
  float* d_raw = list ? reinterpret_cast<float*>(base + off_raw) : nullptr;
  float* d_part = need_part ? reinterpret_cast<float*>(base + off_part) : nullptr;

  // host arrays -> scratch (pageable copies return once the host data has been taken)
  if (cudaMemcpyAsync(d_elem, elem.data(), sizeof(float4) * C, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cuda_fail();
  if (d_u && cudaMemcpyAsync(d_u, u.data(), sizeof(double) * u.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cuda_fail();
  if (d_raw && cudaMemcpyAsync(d_raw, d->vox_pos, sizeof(float) * 3 * V, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cuda_fail();

  TableParams tp{};
  tp.raw_vox = d_raw;
  tp.u = d_u;
  tp.tx_seconds = d->tx_table_dev;
  tp.k = k;
  tp.t0fs = d->t0 * d->fs;
  tp.fs = d->fs;
  for (int a = 0; a < 3; ++a) {
    tp.origin[a] = list ? 0.0 : d->grid_origin[a];
    tp.step[a] = list ? 0.0 : d->grid_step[a];
  }
  tp.nx = list ? 1 : d->grid_dims[0];
  tp.ny = list ? 1 : d->grid_dims[1];
  tp.nz = list ? 1 : d->grid_dims[2];
  tp.V = V;
  tp.T = T;
  tp.vox_out = d_vox;
  tp.tx_out = d_tx;
  if (launch_tables(tp, s) != cudaSuccess) return cuda_fail();

  b.vox = d_vox;
  b.elem = d_elem;
  b.tx = d_tx;
  b.pd_part = d_part;
  b.iq = iq_dev;
  b.y = static_cast<float2*>(y_dev_or_null);
  b.pd = pd_dev_or_null;
  b.V = V;
  b.C = C;
  b.T = T;
  b.S = S;
  b.F = F;
  b.ystride = F;
  b.txr_stride = T;
  b.apod = d->apod;
  b.two_f = static_cast<float>(2.0 * d->f_number);
  b.f_num = static_cast<float>(d->f_number);
  b.four_f2 = static_cast<float>(4.0 * d->f_number * d->f_number);
  b.f_num2 = static_cast<float>(d->f_number * d->f_number);
  b.s_max = static_cast<float>(S - 1);
  b.r_f = static_cast<float>(d->fc / d->fs);
  b.phase_R = host_fixed_cycles(d->fc / d->fs);
  b.phase_Phi = host_fixed_cycles(d->fc * d->t0);
  return launch_das(b, var, s) == cudaSuccess ? MACH_OK : cuda_fail();
}
