// k_das_staged.cu -- delay-and-sum with the sample windows staged in shared memory.
//
// One block beamforms a compact tile of voxels for all frames of the frame tile.  For
// every (element, transmit) pair that some voxel of the tile can use, the rows of the
// frame-contiguous IQ slab that the tile can touch form ONE contiguous byte range
// (rows lo .. lo+rows-1, all F frames), so a single bulk asynchronous copy (TMA unit)
// brings the window into a ring slot of shared memory.  A producer warp walks the
// pairs, issues the copies and publishes each slot's (transmit, element, lo, rows);
// the consumer warps evaluate their terms (receive delay, index, weight) once per pair
// and reuse them across all frames (Sec. 4.4's delay reuse), reading both taps of every
// frame from shared memory.  Pairs no voxel of the tile can use (outside every voxel's
// aperture, or out of range) are skipped without a copy.
//
// Synchronisation: per slot a "full" mbarrier (producer arrival + transaction bytes)
// and an "empty" mbarrier (one arrival per consumer warp).  Every wait is bounded; on a
// timeout the kernel sets bit 0 of the plan's error word and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "async_copy.cuh"
#include "das_term.cuh"
#include "mach_internal.h"

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

// ---- shared-memory tap loads ------------------------------------------------------------
template <class IQ, int VEC>
struct SmemVec;
template <>
struct SmemVec<float2, 2> {
  static __device__ __forceinline__ void load(const float2* p, float2 (&o)[2]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = make_float2(v.x, v.y);
    o[1] = make_float2(v.z, v.w);
  }
};
template <>
struct SmemVec<__half2, 4> {
  static __device__ __forceinline__ void load(const __half2* p, float2 (&o)[4]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    o[0] = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    o[1] = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    o[2] = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
    o[3] = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
  }
};
template <class IQ, int VEC>
struct GlobVec;
template <>
struct GlobVec<float2, 2> {
  static __device__ __forceinline__ void load(const float2* p, float2 (&o)[2]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = make_float2(v.x, v.y);
    o[1] = make_float2(v.z, v.w);
  }
};
template <>
struct GlobVec<__half2, 4> {
  static __device__ __forceinline__ void load(const __half2* p, float2 (&o)[4]) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    o[0] = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    o[1] = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    o[2] = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
    o[3] = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
  }
};

__device__ __forceinline__ void mac_st(float2& acc, float c0r, float c0i, float c1r, float c1i, float2 x0, float2 x1) {
  acc.x = fmaf(c0r, x0.x, acc.x);
  acc.x = fmaf(-c0i, x0.y, acc.x);
  acc.x = fmaf(c1r, x1.x, acc.x);
  acc.x = fmaf(-c1i, x1.y, acc.x);
  acc.y = fmaf(c0r, x0.y, acc.y);
  acc.y = fmaf(c0i, x0.x, acc.y);
  acc.y = fmaf(c1r, x1.y, acc.y);
  acc.y = fmaf(c1i, x1.x, acc.y);
}

// ---- the staged kernel --------------------------------------------------------------------
constexpr int kTxCache = 16;   // transmits whose delays are cached in shared memory per warp

// Shared memory: [ring slots][term tables][transmit-delay cache][slot metadata][barriers]
template <int NBUF>
struct RingLayout {
  size_t slot_bytes, tx_bytes;
  __host__ __device__ RingLayout(int rows_cap, int F, int iq_bytes, int T, int nwc)
      : slot_bytes(((static_cast<size_t>(rows_cap) * F * iq_bytes) + 127) / 128 * 128),
        tx_bytes(T <= kTxCache ? static_cast<size_t>(nwc) * T * 32 * 4 : 0) {}
  __host__ __device__ size_t terms_off() const { return NBUF * slot_bytes; }
  __host__ __device__ size_t tx_off(int nwc) const { return terms_off() + static_cast<size_t>(nwc) * 32 * 16; }
  __host__ __device__ size_t meta_off(int nwc) const { return tx_off(nwc) + (tx_bytes + 15) / 16 * 16; }
  __host__ __device__ size_t bar_off(int nwc) const { return meta_off(nwc) + NBUF * 32; }
  __host__ __device__ size_t total(int nwc) const { return bar_off(nwc) + 2 * NBUF * 8; }
};

// Slot metadata published by the producer with each window.
struct SlotMeta {
  int t, c, lo, rows;   // c < 0: end of sequence
  float4 e;             // element position (sample units)
};

template <class IQ, int VEC, int NV, int FL>
__device__ __forceinline__ void gather_mac(float2 (&acc)[VEC * NV], const IQ* r0, int F, int f_base, int jl,
                                           float c0r, float c0i, float c1r, float c1i, bool smem) {
#pragma unroll
  for (int mm = 0; mm < NV; ++mm) {
    const int f = f_base + (jl + FL * mm) * VEC;
    if (f < F) {
      float2 x0[VEC], x1[VEC];
      if (smem) {
        SmemVec<IQ, VEC>::load(r0 + f, x0);
        SmemVec<IQ, VEC>::load(r0 + F + f, x1);
      } else {
        GlobVec<IQ, VEC>::load(r0 + f, x0);
        GlobVec<IQ, VEC>::load(r0 + F + f, x1);
      }
#pragma unroll
      for (int e = 0; e < VEC; ++e) mac_st(acc[mm * VEC + e], c0r, c0i, c1r, c1i, x0[e], x1[e]);
    }
  }
}

template <class IQ, int VEC, int NV, int FL, int VPG, int NWC, int NBUF, int MINB>
__global__ void __launch_bounds__((NWC + 1) * 32) __maxnreg__(MINB == 2 ? 112 : (MINB == 3 ? 72 : 168)) k_das_staged(const DasParams p) {
  constexpr int G = 32 / FL;
  constexpr int WV = G * VPG;
  constexpr int FPL = VEC * NV;
  constexpr int FT = FL * FPL;
  static_assert(WV <= 32, "one term per lane and pair");
  extern __shared__ __align__(128) unsigned char smem[];
  const RingLayout<NBUF> L(p.rows_cap, p.F, static_cast<int>(sizeof(IQ)), p.T, NWC);
  IQ* ring = reinterpret_cast<IQ*>(smem);
  float4* terms_all = reinterpret_cast<float4*>(smem + L.terms_off());
  float* txc_all = reinterpret_cast<float*>(smem + L.tx_off(NWC));
  SlotMeta* meta = reinterpret_cast<SlotMeta*>(smem + L.meta_off(NWC));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off(NWC));
  uint64_t* empty = full + NBUF;
  const size_t slot_elems = L.slot_bytes / sizeof(IQ);
  const bool tx_cached = p.T <= kTxCache;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t tile = blockIdx.x;
  const IQ* __restrict__ iq = static_cast<const IQ*>(p.iq);
  const size_t slab = static_cast<size_t>(p.S) * p.F;

  if (threadIdx.x == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], NWC);
    }
    mbar_init_fence();
  }
  __syncthreads();

  // ------------------------------------------------------------------ producer
  if (warp == NWC) {
    if (lane != 0) return;
    const float4 blo = p.tbox[2 * tile], bhi = p.tbox[2 * tile + 1];
    int r = 0;
    bool ok = true;
    for (int c = 0; c < p.C && ok; ++c) {
      const float4 e = __ldg(&p.elem[c]);
      for (int t = 0; t < p.T; ++t) {
        int lo, rows;
        if (!pair_window(blo, bhi, p.txr[tile * p.T + t], e, p, lo, rows)) continue;
        rows = min(rows, p.rows_cap);
        const int slot = r % NBUF;
        if (r >= NBUF && !mbar_wait_bounded(&empty[slot], ((r / NBUF) - 1) & 1, p.wait_limit)) {
          atomicOr(p.err, 1);
          ok = false;
          break;
        }
        meta[slot].t = t;
        meta[slot].c = c;
        meta[slot].lo = lo;
        meta[slot].rows = rows;
        meta[slot].e = e;
        const uint32_t bytes = static_cast<uint32_t>(rows) * p.F * sizeof(IQ);
        mbar_arrive_expect_tx(&full[slot], bytes);
        if (!p.debug_stall)
          bulk_g2s(ring + slot * slot_elems, iq + (static_cast<size_t>(t) * p.C + c) * slab + static_cast<size_t>(lo) * p.F,
                   bytes, &full[slot]);
        ++r;
      }
    }
    if (ok) {   // end-of-sequence marker
      const int slot = r % NBUF;
      if (r >= NBUF && !mbar_wait_bounded(&empty[slot], ((r / NBUF) - 1) & 1, p.wait_limit)) {
        atomicOr(p.err, 1);
      } else {
        meta[slot].c = -1;
        mbar_arrive(&full[slot]);
      }
    } else {    // abandoning: let the copies already issued land before the block can exit
      for (int k = max(0, r - NBUF); k < r; ++k) mbar_wait_bounded(&full[k % NBUF], (k / NBUF) & 1, p.wait_limit);
    }
    return;
  }

  // ------------------------------------------------------------------ consumers
  const int g = lane / FL;
  const int jl = lane % FL;
  const int f_base = blockIdx.y * FT;
  float4* terms = terms_all + warp * 32;
  float* txc = txc_all + warp * (p.T * 32);
  // lane < WV evaluates the terms of voxel slot `lane`; they are stored at k*G + g so
  // that the G groups of the warp read G consecutive entries (no bank conflict)
  const int64_t v_term = lane < WV ? tile_voxel_blocked(p, tile, warp * WV + lane) : -1;
  const float4 vpos = v_term >= 0 ? p.vox[v_term] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int store_at = (lane % VPG) * G + (lane / VPG);
  if (tx_cached) {
    for (int t = 0; t < p.T; ++t) txc[t * 32 + lane] = v_term >= 0 ? p.tx[static_cast<size_t>(t) * p.V + v_term] : 0.f;
  }

  float2 acc[VPG][FPL];
#pragma unroll
  for (int k = 0; k < VPG; ++k)
#pragma unroll
    for (int e = 0; e < FPL; ++e) acc[k][e] = make_float2(0.f, 0.f);

  int cur_c = -1;
  TermGeo geo;
  geo.rx = 0.f;
  geo.a = -1.f;
  bool ok = true;
  for (int r = 0;; ++r) {
    const int slot = r % NBUF;
    if (!mbar_wait_bounded(&full[slot], (r / NBUF) & 1, p.wait_limit)) {
      if (lane == 0) atomicOr(p.err, 1);
      ok = false;
      break;
    }
    const SlotMeta m = meta[slot];
    if (m.c < 0) break;
    if (m.c != cur_c) {
      cur_c = m.c;
      geo.a = -1.f;
      if (v_term >= 0) geo = term_geometry(vpos, m.e, p);
    }
    float4 rec = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    if (geo.a >= 0.f) {
      const float stx = tx_cached ? txc[m.t * 32 + lane] : __ldg(&p.tx[static_cast<size_t>(m.t) * p.V + v_term]);
      rec = term_record(stx, geo, p);
    }
    const int my_i0 = __float_as_int(rec.w);
    const bool active = my_i0 >= 0;
    const bool outside = active && (my_i0 - m.lo < 0 || my_i0 - m.lo + 1 >= m.rows);
    const unsigned any_active = __ballot_sync(0xffffffffu, active);
    const unsigned any_outside = __ballot_sync(0xffffffffu, outside);
    if (any_active) {
      if (lane < WV) terms[store_at] = rec;
      __syncwarp();
      const IQ* win = ring + slot * slot_elems;
      if (!any_outside) {
        // every kept term lies in the staged window: branch-free over the voxels
        // (dropped terms carry zero weights and read row 0)
#pragma unroll
        for (int k = 0; k < VPG; ++k) {
          const float4 tr = terms[k * G + g];
          const int row = max(__float_as_int(tr.w) - m.lo, 0);
          const float c1r = tr.x * tr.z, c1i = tr.y * tr.z;
          const float c0r = tr.x - c1r, c0i = tr.y - c1i;
          gather_mac<IQ, VEC, NV, FL>(acc[k], win + row * p.F, p.F, f_base, jl, c0r, c0i, c1r, c1i, true);
        }
      } else {
        // some kept term falls outside the staged window (not expected): per-term
        // choice between the window and global memory
        const IQ* gsrc = iq + (static_cast<size_t>(m.t) * p.C + m.c) * slab;
#pragma unroll
        for (int k = 0; k < VPG; ++k) {
          const float4 tr = terms[k * G + g];
          const int i0 = __float_as_int(tr.w);
          if (i0 >= 0) {
            const float c1r = tr.x * tr.z, c1i = tr.y * tr.z;
            const float c0r = tr.x - c1r, c0i = tr.y - c1i;
            const int row = i0 - m.lo;
            if (row >= 0 && row + 1 < m.rows)
              gather_mac<IQ, VEC, NV, FL>(acc[k], win + row * p.F, p.F, f_base, jl, c0r, c0i, c1r, c1i, true);
            else
              gather_mac<IQ, VEC, NV, FL>(acc[k], gsrc + static_cast<size_t>(i0) * p.F, p.F, f_base, jl, c0r, c0i,
                                          c1r, c1i, false);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
  }
  if (!ok) return;

#pragma unroll
  for (int k = 0; k < VPG; ++k) {
    const int64_t v = tile_voxel_blocked(p, tile, warp * WV + g * VPG + k);
    float pw = 0.f;
#pragma unroll
    for (int mm = 0; mm < NV; ++mm) {
      const int f = f_base + (jl + FL * mm) * VEC;
      if (f < p.F) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const float2 a = acc[k][mm * VEC + e];
          pw = fmaf(a.x, a.x, fmaf(a.y, a.y, pw));
        }
        if (v >= 0 && p.y) {
          float2* dst = p.y + v * p.F + f;
#pragma unroll
          for (int e = 0; e < VEC; e += 2)
            *reinterpret_cast<float4*>(dst + e) =
                make_float4(acc[k][mm * VEC + e].x, acc[k][mm * VEC + e].y, acc[k][mm * VEC + e + 1].x,
                            acc[k][mm * VEC + e + 1].y);
        }
      }
    }
#pragma unroll
    for (int o = FL / 2; o > 0; o >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, o);
    if (jl == 0 && v >= 0 && p.pd) p.pd[v] = pw;
  }
}

// ---- dispatch ------------------------------------------------------------------------------
namespace {
constexpr int kNWC = 8;     // consumer warps
constexpr int kRing = 4;    // ring slots

template <class K>
cudaError_t go_staged(K kernel, const DasParams& p, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int64_t tiles = static_cast<int64_t>(p.tiles_x) * p.tiles_y * p.tiles_z;
  kernel<<<dim3(static_cast<unsigned>(tiles), 1), (kNWC + 1) * 32, smem, s>>>(p);
  return cudaGetLastError();
}
}  // namespace

size_t staged_smem_bytes(Variant v, int rows_cap, int F, int T) {
  const int b = (v == V_ST32_H16 || v == V_ST64_H16) ? 4 : 8;
  return RingLayout<kRing>(rows_cap, F, b, T, kNWC).total(kNWC);
}

cudaError_t launch_das_staged(const DasParams& p, Variant v, cudaStream_t s) {
  const size_t sm = staged_smem_bytes(v, p.rows_cap, p.F, p.T);
  switch (v) {
    case V_ST32_C64: return go_staged(k_das_staged<float2, 2, 2, 8, 8, kNWC, kRing, 2>, p, sm, s);
    case V_ST64_C64: return go_staged(k_das_staged<float2, 2, 2, 16, 8, kNWC, kRing, 2>, p, sm, s);
    case V_ST32_H16: return go_staged(k_das_staged<__half2, 4, 1, 8, 8, kNWC, kRing, 2>, p, sm, s);
    case V_ST64_H16: return go_staged(k_das_staged<__half2, 4, 1, 16, 8, kNWC, kRing, 2>, p, sm, s);
    case V_ST32_C64_V4: return go_staged(k_das_staged<float2, 2, 2, 8, 4, kNWC, kRing, 3>, p, sm, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mach
