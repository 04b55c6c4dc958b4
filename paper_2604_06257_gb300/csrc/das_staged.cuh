// das_staged.cuh -- the staged delay-and-sum kernel (template), shared by the
// translation unit that instantiates it with receive delays evaluated on the fly
// (k_das_staged.cu) and the one that instantiates it with every term read from a
// plan-time table (k_das_table.cu).
//
// One block beamforms a compact tile of voxels for all frames of the frame tile.  For
// every (element, transmit) pair that some voxel of the tile can use, the rows of the
// frame-contiguous IQ slab that the tile can touch form ONE contiguous byte range
// (rows lo .. lo+rows-1, all F frames), so a single bulk asynchronous copy (TMA unit)
// brings the window into a ring slot of shared memory.  A producer warp walks the
// pairs, issues the copies and publishes each slot's (transmit, element, lo, rows).
//
// Terms (receive delay, index, weight of one voxel for one pair):
//  * on the fly (TABLE = false, Sec. 4.3's hybrid delays): the consumer warps evaluate
//    them once per pair and reuse them across all frames (Sec. 4.4's delay reuse);
//  * from the table (TABLE = true): the plan evaluated every term once, with the same
//    device functions, and stored each pair's records in the order the consumers read
//    them; the producer copies a pair's records into the slot beside its window, so the
//    consumers only gather and accumulate.  Same terms, same order: bitwise the same
//    outputs.
// Either way the consumers read both taps of every frame from shared memory.  Pairs no
// voxel of the tile can use (outside every voxel's aperture, or out of range) are
// skipped without a copy.
//
// Synchronisation: per slot a "full" mbarrier (producer arrival + transaction bytes)
// and an "empty" mbarrier (one arrival per consumer warp).  Every wait is bounded; on a
// timeout the kernel sets bit 0 of the plan's error word and returns.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "async_copy.cuh"
#include "das_term.cuh"
#include "tap_mac.cuh"
#include "mach_internal.h"

namespace mach {

// ---- the staged kernel --------------------------------------------------------------------
constexpr int kTxCache = 16;   // transmits whose delays are cached in shared memory per warp

// Shared memory: [ring slots][term scratch][transmit-delay cache][slot metadata][barriers].
// A ring slot holds one pair's sample window and, in table mode, the pair's term records
// (16 bytes per voxel slot of the block); the term scratch and the delay cache exist only
// when terms are evaluated on the fly.
template <int NBUF>
struct RingLayout {
  size_t win_bytes, rec_bytes, slot_bytes, terms_bytes, tx_bytes;
  __host__ __device__ RingLayout(int rows_cap, int F, int iq_bytes, int T, int nwc, int wv, bool table)
      : win_bytes(((static_cast<size_t>(rows_cap) * F * iq_bytes) + 127) / 128 * 128),
        rec_bytes(table ? static_cast<size_t>(nwc) * wv * 16 : 0),
        slot_bytes((win_bytes + rec_bytes + 127) / 128 * 128),
        terms_bytes(table ? 0 : static_cast<size_t>(nwc) * 32 * 16),
        tx_bytes(!table && T <= kTxCache ? static_cast<size_t>(nwc) * T * 32 * 4 : 0) {}
  __host__ __device__ size_t terms_off() const { return NBUF * slot_bytes; }
  __host__ __device__ size_t tx_off() const { return terms_off() + terms_bytes; }
  __host__ __device__ size_t meta_off() const { return tx_off() + (tx_bytes + 15) / 16 * 16; }
  __host__ __device__ size_t bar_off() const { return meta_off() + NBUF * 32; }
  __host__ __device__ size_t total() const { return bar_off() + 2 * NBUF * 8; }
};

// Slot metadata published by the producer with each window.
struct SlotMeta {
  int t, c, lo, rows;   // c < 0: end of sequence
  float4 e;             // element position (sample units)
};

// ---- producer (shared by the staged kernels) --------------------------------------------
// The producer warp evaluates 32 (element, transmit) pairs at a time (one lane each, loads
// issued together), then lane 0 issues the copies of the usable ones in pair order: it
// claims ring slot r % NBUF once every consumer warp has released the slot's previous use,
// publishes (t, c, lo, rows, element) and copies the window with one bulk copy that
// completes on the slot's "full" barrier.  Returns false when a wait gave up (the error
// word is then set); r counts the slots issued.
template <int NBUF>
__device__ __forceinline__ bool produce_windows(const DasParams& p, int64_t tile, int lane, unsigned char* ring,
                                                size_t slot_bytes, int sample_bytes, SlotMeta* meta, uint64_t* full,
                                                uint64_t* empty, int& r) {
  const unsigned char* iq = static_cast<const unsigned char*>(p.iq);
  const size_t row_bytes = static_cast<size_t>(p.F) * sample_bytes;
  const size_t slab = static_cast<size_t>(p.S) * row_bytes;
  const float4 blo = p.tbox[2 * tile], bhi = p.tbox[2 * tile + 1];
  const int npairs = p.C * p.T;
  bool ok = true;
  for (int pb = 0; pb < npairs && ok; pb += 32) {
    const int pi = pb + lane;
    int t = 0, c = 0, lo = 0, rows = 0;
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    bool use = false;
    if (pi < npairs) {
      c = pi / p.T;
      t = pi - c * p.T;
      e = __ldg(&p.elem[c]);
      use = pair_window(blo, bhi, __ldg(&p.txr[tile * p.txr_stride + t]), e, p, lo, rows);
      rows = min(rows, p.rows_cap);
    }
    unsigned todo = __ballot_sync(0xffffffffu, use);
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      const int tj = __shfl_sync(0xffffffffu, t, j), cj = __shfl_sync(0xffffffffu, c, j);
      const int loj = __shfl_sync(0xffffffffu, lo, j), rowsj = __shfl_sync(0xffffffffu, rows, j);
      float4 ej;
      ej.x = __shfl_sync(0xffffffffu, e.x, j);
      ej.y = __shfl_sync(0xffffffffu, e.y, j);
      ej.z = __shfl_sync(0xffffffffu, e.z, j);
      ej.w = 0.f;
      if (lane == 0) {
        const int slot = r % NBUF;
        if (r >= NBUF && !mbar_wait_bounded(&empty[slot], ((r / NBUF) - 1) & 1, p.wait_limit)) {
          atomicOr(p.err, 1);
          ok = false;
        } else {
          meta[slot].t = tj;
          meta[slot].c = cj;
          meta[slot].lo = loj;
          meta[slot].rows = rowsj;
          meta[slot].e = ej;
          const uint32_t bytes = static_cast<uint32_t>(rowsj * row_bytes);
          mbar_arrive_expect_tx(&full[slot], bytes);
          if (!p.debug_stall)
            bulk_g2s(ring + slot * slot_bytes,
                     iq + (static_cast<size_t>(tj) * p.C + cj) * slab + static_cast<size_t>(loj) * row_bytes, bytes,
                     &full[slot]);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      ++r;
    }
  }
  return ok;
}

// Lane 0 of the producer after its last pair: one end-of-sequence marker per pair a
// consumer round can hold; or, when abandoning after a timeout, a bounded wait for the
// copies already issued, so that none lands after the block has exited.
template <int NBUF, int PB>
__device__ __forceinline__ void finish_producer(const DasParams& p, bool ok, int r, SlotMeta* meta, uint64_t* full,
                                                uint64_t* empty) {
  if (ok) {
    for (int k = 0; k < PB; ++k) {
      const int rr = r + k, slot = rr % NBUF;
      if (rr >= NBUF && !mbar_wait_bounded(&empty[slot], ((rr / NBUF) - 1) & 1, p.wait_limit)) {
        atomicOr(p.err, 1);
        break;
      }
      meta[slot].c = -1;
      mbar_arrive(&full[slot]);
    }
  } else {
    for (int k = max(0, r - NBUF); k < r; ++k) mbar_wait_bounded(&full[k % NBUF], (k / NBUF) & 1, p.wait_limit);
  }
}

// MAXR: register cap per thread, chosen so that the intended number of blocks fits per SM.
// TABLE: terms read from the plan's term table instead of evaluated on the fly.
template <class IQ, int VEC, int NV, int FL, int VPG, int NWC, int NBUF, int MAXR, bool TABLE>
__global__ void __launch_bounds__((NWC + 1) * 32) __maxnreg__(MAXR) k_das_staged(const DasParams p) {
  constexpr int G = 32 / FL;
  constexpr int WV = G * VPG;
  constexpr int FPL = VEC * NV;
  constexpr int FT = FL * FPL;
  constexpr int PB = 32 / WV;          // pairs whose terms one warp evaluates per round
  static_assert(WV * PB == 32, "a round must fill the warp");
  static_assert(NBUF >= PB, "a round must fit in the ring");
  extern __shared__ __align__(128) unsigned char smem[];
  using E = typename IqStore<IQ>::E;
  constexpr int kBytes = static_cast<int>(sizeof(E)) * IqStore<IQ>::eps;   // bytes per complex sample
  constexpr uint32_t kRecBytes = NWC * WV * 16;     // one pair's term records (table mode)
  const RingLayout<NBUF> L(p.rows_cap, p.F, kBytes, p.T, NWC, WV, TABLE);
  E* ring = reinterpret_cast<E*>(smem);
  float4* terms_all = reinterpret_cast<float4*>(smem + L.terms_off());
  float* txc_all = reinterpret_cast<float*>(smem + L.tx_off());
  SlotMeta* meta = reinterpret_cast<SlotMeta*>(smem + L.meta_off());
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off());
  // term records of the pair in ring slot b (table mode)
  auto slot_rec = [&](int b) { return reinterpret_cast<const float4*>(smem + b * L.slot_bytes + L.win_bytes); };
  uint64_t* empty = full + NBUF;
  const size_t slot_elems = L.slot_bytes / sizeof(E);
  const int row_elems = p.F * IqStore<IQ>::eps;     // one sample row, all frames
  const bool tx_cached = !TABLE && p.T <= kTxCache;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // the last tiles (deepest rows of the grid, the widest apertures: the most pairs) start
  // first, so that the light shallow tiles fill the tail of the launch
  const int64_t tile = static_cast<int64_t>(gridDim.x) - 1 - blockIdx.x;
  const E* __restrict__ iq = static_cast<const E*>(p.iq);
  const size_t slab = static_cast<size_t>(p.S) * row_elems;

  if (threadIdx.x == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], NWC);
    }
    mbar_init_fence();
  }
  __syncthreads();

  // ------------------------------------------------------------------ producer
  // The producer warp evaluates 32 (element, transmit) pairs at a time (one lane each,
  // loads issued together), then lane 0 issues the copies of the usable ones in order.
  if (warp == NWC) {
    int r = 0;
    bool ok = true;
    if constexpr (TABLE) {
      // the plan listed the tile's usable pairs in order, with their windows
      const int64_t q0 = p.tile_pairs[tile], q1 = p.tile_pairs[tile + 1];
      for (int64_t qb = q0; qb < q1 && ok; qb += 32) {
        const int n = static_cast<int>(q1 - qb < 32 ? q1 - qb : 32);
        int4 dsc = make_int4(0, 0, 0, 0);
        if (lane < n) dsc = __ldg(&p.pair_desc[qb + lane]);
        for (int j = 0; j < n; ++j) {
          const int tj = __shfl_sync(0xffffffffu, dsc.x, j), cj = __shfl_sync(0xffffffffu, dsc.y, j);
          const int loj = __shfl_sync(0xffffffffu, dsc.z, j), rowsj = __shfl_sync(0xffffffffu, dsc.w, j);
          if (lane == 0) {
            const int slot = r % NBUF;
            if (r >= NBUF && !mbar_wait_bounded(&empty[slot], ((r / NBUF) - 1) & 1, p.wait_limit)) {
              atomicOr(p.err, 1);
              ok = false;
            } else {
              meta[slot].t = tj;
              meta[slot].c = cj;
              meta[slot].lo = loj;
              meta[slot].rows = rowsj;
              const uint32_t bytes = static_cast<uint32_t>(rowsj) * p.F * kBytes;
              mbar_arrive_expect_tx(&full[slot], bytes + kRecBytes);
              if (!p.debug_stall) {
                bulk_g2s(ring + slot * slot_elems,
                         iq + (static_cast<size_t>(tj) * p.C + cj) * slab + static_cast<size_t>(loj) * row_elems,
                         bytes, &full[slot]);
                bulk_g2s(smem + slot * L.slot_bytes + L.win_bytes,
                         p.term_rec + static_cast<size_t>(qb + j) * (NWC * WV), kRecBytes, &full[slot]);
              }
            }
          }
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) break;
          ++r;
        }
      }
    }
    if constexpr (!TABLE)
      ok = produce_windows<NBUF>(p, tile, lane, smem, L.slot_bytes, kBytes, meta, full, empty, r);
    if (lane == 0) finish_producer<NBUF, PB>(p, ok, r, meta, full, empty);
    return;
  }

  // ------------------------------------------------------------------ consumers
  // Each round the warp takes PB consecutive pairs: lane group `sub` (WV lanes) evaluates
  // the terms of pair r + sub for the warp's WV voxels, then the warp consumes the PB
  // pairs one after the other.
  const int g = lane / FL;
  const int jl = lane % FL;
  const int sub = lane / WV;
  const int q = lane % WV;
  const int f_base = blockIdx.y * FT;
  float4* terms = terms_all + warp * 32;
  float* txc = txc_all + warp * (p.T * 32);
  // terms of voxel slot q for pair `sub` are stored at sub*WV + k*G + g (slot q = g*VPG + k),
  // so the G groups of the warp read G consecutive entries (no bank conflict)
  const int64_t v_term = TABLE ? -1 : tile_voxel_blocked(p, tile, warp * WV + q);
  const float4 vpos = v_term >= 0 ? p.vox[v_term] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int rec_at = (q % VPG) * G + (q / VPG);   // position of voxel slot q in a pair's records
  const int store_at = sub * WV + rec_at;
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
  bool ok = true, done = false;
  for (int r = 0; !done; r += PB) {
    const int mine = r + sub, my_slot = mine % NBUF;
    const bool got = mbar_wait_bounded(&full[my_slot], (mine / NBUF) & 1, p.wait_limit);
    if (__any_sync(0xffffffffu, !got)) {
      if (lane == 0) atomicOr(p.err, 1);
      ok = false;
      break;
    }
    const SlotMeta mm = meta[my_slot];
    float4 rec = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    if constexpr (TABLE) {
      if (mm.c >= 0) rec = slot_rec(my_slot)[warp * WV + rec_at];
    } else {
      if (mm.c >= 0) {
        if (mm.c != cur_c) {
          cur_c = mm.c;
          geo.a = -1.f;
          if (v_term >= 0) geo = term_geometry(vpos, mm.e, p);
        }
        if (geo.a >= 0.f) {
          const float stx = tx_cached ? txc[mm.t * 32 + lane] : __ldg(&p.tx[static_cast<size_t>(mm.t) * p.V + v_term]);
          rec = term_record(stx, geo, p);
        }
      }
    }
    const int my_i0 = __float_as_int(rec.w);
    const bool active = my_i0 >= 0;
    const bool outside = active && (my_i0 - mm.lo < 0 || my_i0 - mm.lo + 1 >= mm.rows);
    const unsigned act = __ballot_sync(0xffffffffu, active);
    const unsigned outm = __ballot_sync(0xffffffffu, outside);
    const unsigned ended = __ballot_sync(0xffffffffu, mm.c < 0);
    if (!TABLE) {
      terms[store_at] = rec;
      __syncwarp();
    }
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const unsigned gm = WV == 32 ? 0xffffffffu : (((1u << (WV & 31)) - 1u) << (i * WV));
      if (ended & gm) {   // end marker: every later pair of the round is one too
        done = true;
        break;
      }
      if (!(act & gm)) continue;
      const int slot = (r + i) % NBUF;
      const int lo = meta[slot].lo, rows = meta[slot].rows;
      const E* win = ring + slot * slot_elems;
      const float4* tp = TABLE ? slot_rec(slot) + warp * WV : terms + i * WV;
      if (!(outm & gm)) {
        // every kept term lies in the staged window: branch-free over the voxels
        // (dropped terms carry zero weights and read row 0)
#pragma unroll
        for (int k = 0; k < VPG; ++k) {
          const float4 tr = tp[k * G + g];
          const int row = max(__float_as_int(tr.w) - lo, 0);
          const float4 cw = tap_weights(tr);
          const float c0r = cw.x, c0i = cw.y, c1r = cw.z, c1i = cw.w;
          gather_mac<IQ, VEC, NV, FL, true>(acc[k], win + row * row_elems, row_elems, p.F, f_base, jl, c0r, c0i, c1r,
                                            c1i);
        }
      } else {
        // some kept term falls outside the staged window (not expected): per-term
        // choice between the window and global memory
        const int t = meta[slot].t, c = meta[slot].c;
        const E* gsrc = iq + (static_cast<size_t>(t) * p.C + c) * slab;
#pragma unroll
        for (int k = 0; k < VPG; ++k) {
          const float4 tr = tp[k * G + g];
          const int i0 = __float_as_int(tr.w);
          if (i0 >= 0) {
            const float4 cw = tap_weights(tr);
            const float c0r = cw.x, c0i = cw.y, c1r = cw.z, c1i = cw.w;
            const int row = i0 - lo;
            if (row >= 0 && row + 1 < rows)
              gather_mac<IQ, VEC, NV, FL, true>(acc[k], win + row * row_elems, row_elems, p.F, f_base, jl, c0r, c0i,
                                                c1r, c1i);
            else
              gather_mac<IQ, VEC, NV, FL, false>(acc[k], gsrc + static_cast<size_t>(i0) * row_elems, row_elems, p.F,
                                                 f_base, jl, c0r, c0i, c1r, c1i);
          }
        }
      }
    }
    __syncwarp();
    if (lane < PB) mbar_arrive(&empty[(r + lane) % NBUF]);
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
          const float2 a = acc_frame<IQ, VEC>(&acc[k][mm * VEC], e);
          pw = fmaf(a.x, a.x, fmaf(a.y, a.y, pw));
        }
        if (v >= 0 && p.y) {
          float2* dst = p.y + v * p.ystride + f;
#pragma unroll
          for (int e = 0; e < VEC; e += 2) {
            const float2 a = acc_frame<IQ, VEC>(&acc[k][mm * VEC], e), b = acc_frame<IQ, VEC>(&acc[k][mm * VEC], e + 1);
            *reinterpret_cast<float4*>(dst + e) = make_float4(a.x, a.y, b.x, b.y);
          }
        }
      }
    }
#pragma unroll
    for (int o = FL / 2; o > 0; o >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, o);
    if (jl == 0 && v >= 0 && p.pd) p.pd[v] = pw;
  }
}

// ---- launch ---------------------------------------------------------------------------------
constexpr int kRing = 4;    // ring slots (8 when a round holds 4 pairs)

template <class K>
cudaError_t go_staged(K kernel, int nwc, const DasParams& p, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int64_t tiles = static_cast<int64_t>(p.tiles_x) * p.tiles_y * p.tiles_z;
  kernel<<<dim3(static_cast<unsigned>(tiles), static_cast<unsigned>(p.frame_tiles)), (nwc + 1) * 32, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace mach
