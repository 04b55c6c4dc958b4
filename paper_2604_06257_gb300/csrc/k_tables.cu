// k_tables.cu -- per-plan tables (hybrid delays, Sec. 4.3) and the term inspector.
//
// K1 builds, once per plan:
//   vox[v] = RN_float(p_v * fs/c)                       (voxel position, samples)
//   tx[t][v] = RN_float(fma(ux,px, fma(uy,py, uz*pz)) * fs/c - t0 fs)   plane wave
//            = RN_float(arrival_s[t][v] * fs - t0 fs)                    user table
// in FP64 (the only FP64 on the device), with p_v = origin + i * step for a grid.
#include <cuda_runtime.h>
#include <cstdint>

#include "das_term.cuh"
#include "mach_internal.h"

namespace mach {

__global__ void __launch_bounds__(256) k_tables(TableParams tp) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= tp.V) return;
  double px, py, pz;
  if (tp.raw_vox) {
    px = static_cast<double>(tp.raw_vox[3 * v + 0]);
    py = static_cast<double>(tp.raw_vox[3 * v + 1]);
    pz = static_cast<double>(tp.raw_vox[3 * v + 2]);
  } else {
    const int64_t ix = v % tp.nx;
    const int64_t iy = (v / tp.nx) % tp.ny;
    const int64_t iz = v / (static_cast<int64_t>(tp.nx) * tp.ny);
    px = __dadd_rn(tp.origin[0], __dmul_rn(static_cast<double>(ix), tp.step[0]));
    py = __dadd_rn(tp.origin[1], __dmul_rn(static_cast<double>(iy), tp.step[1]));
    pz = __dadd_rn(tp.origin[2], __dmul_rn(static_cast<double>(iz), tp.step[2]));
  }
  tp.vox_out[v] = make_float4(__double2float_rn(__dmul_rn(px, tp.k)),
                              __double2float_rn(__dmul_rn(py, tp.k)),
                              __double2float_rn(__dmul_rn(pz, tp.k)), 0.0f);
  for (int t = 0; t < tp.T; ++t) {
    double s;
    if (tp.tx_seconds) {
      s = __fma_rn(static_cast<double>(tp.tx_seconds[static_cast<int64_t>(t) * tp.V + v]), tp.fs, -tp.t0fs);
    } else {
      const double ux = tp.u[3 * t], uy = tp.u[3 * t + 1], uz = tp.u[3 * t + 2];
      const double dot = __fma_rn(ux, px, __fma_rn(uy, py, __dmul_rn(uz, pz)));
      s = __fma_rn(dot, tp.k, -tp.t0fs);
    }
    tp.tx_out[static_cast<int64_t>(t) * tp.V + v] = __double2float_rn(s);
  }
}

cudaError_t launch_tables(const TableParams& tp, cudaStream_t s) {
  const int64_t blocks = (tp.V + 255) / 256;
  k_tables<<<static_cast<unsigned>(blocks), 256, 0, s>>>(tp);
  return cudaGetLastError();
}

// One thread per (listed voxel, element); loops over transmits.  Same device
// functions as the DAS kernels.
__global__ void __launch_bounds__(256) k_terms(DasParams p, const int64_t* vox_idx, int64_t n,
                                               int32_t* i0_out, float* w_out, float* cw_out) {
  const int64_t id = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (id >= n * p.C) return;
  const int64_t j = id / p.C;
  const int c = static_cast<int>(id % p.C);
  const int64_t v = vox_idx[j];
  if (v < 0 || v >= p.V) return;
  const TermGeo g = term_geometry(p.vox[v], p.elem[c], p);
  for (int t = 0; t < p.T; ++t) {
    const float4 r = term_record(p.tx[static_cast<int64_t>(t) * p.V + v], g, p);
    const int64_t o = id * p.T + t;
    if (i0_out) i0_out[o] = __float_as_int(r.w);
    if (w_out) w_out[o] = r.z;
    if (cw_out) {
      cw_out[2 * o] = r.x;
      cw_out[2 * o + 1] = r.y;
    }
  }
}

cudaError_t launch_terms(const DasParams& p, const int64_t* vox_idx, int64_t n, int32_t* i0,
                         float* w, float* cw, cudaStream_t s) {
  const int64_t total = n * p.C;
  if (total == 0) return cudaSuccess;
  const int64_t blocks = (total + 255) / 256;
  k_terms<<<static_cast<unsigned>(blocks), 256, 0, s>>>(p, vox_idx, n, i0, w, cw);
  return cudaGetLastError();
}

}  // namespace mach
