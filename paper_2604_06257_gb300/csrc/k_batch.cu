// k_batch.cu -- ragged batches: many DAS instances in one persistent launch.
//
// A batch holds instances of different sizes (2D and 3D grids, element, transmit and
// frame counts).  Their voxel tiles form one work list, sorted by decreasing estimated
// cost; a persistent grid (as many blocks as fit on the GPU) pulls (instance, tile) items
// from an atomic counter until the list is exhausted, so large and small instances
// share the machine without a launch per instance.  The last block to finish resets the
// counter, so the launch can be replayed (e.g. from a CUDA graph) without a host step.
//
// Per item, one of three lane mappings (chosen per instance):
//  - staged (4 < F <= 64): the staged scheme of das_staged.cuh per item -- a producer warp
//    copies each usable (element, transmit) pair's sample window into a shared-memory
//    ring (one bulk copy; for rows that do not start on a 16-byte boundary the copy starts
//    at the boundary below and the consumers skip the difference), the consumer warps
//    evaluate each term once and accumulate 4 frames per lane from shared memory (16-byte
//    vectors when F % 4 == 0, else one sample per frame).  The ring's barriers are
//    initialised afresh for every item;
//  - frame lanes (F <= 16 or a multiple of 4, and the fallback when an instance's windows
//    exceed the ring): FL lanes share a voxel (FL = 2, 4, 8 or 16 at run time), each lane
//    holds 4 frames of 4 voxels (2 voxels for FL = 2), taps read through L1;
//  - channel lanes (F <= 4): 8 lanes share a voxel and split its elements; partial sums
//    meet in a shuffle tree.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "das_staged.cuh"

namespace mach {

constexpr int kBatchWarps = 8;   // warps of a block; the staged path uses the last one as its producer
constexpr int kBatchConsumers = kBatchWarps - 1;
constexpr int kBatchTx = 4;      // transmits whose terms are staged per element round (frame lanes)
constexpr int kBatchRing = 8;    // ring slots of the staged path

// Frame lanes: FL lanes share a voxel, each holds 4 frames of VPG voxels (VPG = 4, or 2 for
// FL = 2 so that a warp covers 32 voxels, as with FL = 4); a warp covers (32 / FL) VPG voxels.
template <class IQ, int VEC, int NV, int VPG>
__device__ __forceinline__ void batch_frames_tile(const DasParams& p, int FL, int64_t tile, float4* terms) {
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
#pragma unroll
            for (int e = 0; e < VEC; ++e) p.y[v * p.F + f + e] = acc[k][mm * VEC + e];
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

// ---- staged path ---------------------------------------------------------------------------

// Shared memory of a batch block: [ring][per-warp scratch][slot metadata][barriers].  The
// scratch holds the frame-lane path's staged terms, or the staged path's per-warp term
// table and transmit-delay cache (the two paths never share an item).
struct BatchLayout {
  size_t slot_bytes, scratch_bytes;
  __host__ __device__ explicit BatchLayout(size_t slot)
      : slot_bytes(slot),
        scratch_bytes(kBatchWarps * (kBatchTx * 32 * 16 > 32 * 16 + kTxCache * 32 * 4 ? kBatchTx * 32 * 16
                                                                                      : 32 * 16 + kTxCache * 32 * 4)) {}
  __host__ __device__ size_t scratch_off() const { return kBatchRing * slot_bytes; }
  __host__ __device__ size_t meta_off() const { return scratch_off() + scratch_bytes; }
  __host__ __device__ size_t bar_off() const { return meta_off() + kBatchRing * 48; }   // 48 = sizeof(BatchSlotMeta)
  __host__ __device__ size_t total() const { return bar_off() + 2 * kBatchRing * 8; }
};

// Slot metadata of the staged batch path: as SlotMeta, plus the element offset of the
// window's first row inside the slot (copies start on a 16-byte boundary).
struct BatchSlotMeta {
  int t, c, lo, rows;   // c < 0: end of the item's sequence
  float4 e;
  int skip;             // elements (complex samples) before row lo in the slot
  int pad_[3];
};
static_assert(sizeof(BatchSlotMeta) == 48, "slot metadata (BatchLayout reserves 48 bytes per slot)");

// Producer of one staged item: like produce_windows, for rows of any length.  A window is
// rows x F complex samples starting at byte `start` of the IQ array; the bulk copy covers
// [start rounded down to 16 bytes, end rounded up to 16 bytes), clamped so that it never
// reads past the array (a window whose end would be clamped loses its last rows: terms
// there read global memory).
template <class IQ>
__device__ __forceinline__ bool batch_produce(const DasParams& p, int64_t tile, int lane, unsigned char* ring,
                                              size_t slot_bytes, BatchSlotMeta* meta, uint64_t* full, uint64_t* empty,
                                              int& r) {
  constexpr int kBytes = static_cast<int>(sizeof(typename IqStore<IQ>::E)) * IqStore<IQ>::eps;
  const unsigned char* iq = static_cast<const unsigned char*>(p.iq);
  const size_t row_bytes = static_cast<size_t>(p.F) * kBytes;
  const size_t slab = static_cast<size_t>(p.S) * row_bytes;
  const size_t total = slab * p.C * p.T;
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
        const int slot = r % kBatchRing;
        if (r >= kBatchRing && !mbar_wait_bounded(&empty[slot], ((r / kBatchRing) - 1) & 1, p.wait_limit)) {
          atomicOr(p.err, 1);
          ok = false;
        } else {
          const size_t start = (static_cast<size_t>(tj) * p.C + cj) * slab + static_cast<size_t>(loj) * row_bytes;
          const size_t a0 = start & ~static_cast<size_t>(15);
          size_t a1 = (start + rowsj * row_bytes + 15) & ~static_cast<size_t>(15);
          int rows_in = rowsj;
          if (a1 > total) {   // keep the copy inside the array: drop rows that would cross its end
            a1 = total & ~static_cast<size_t>(15);
            rows_in = a1 > start ? static_cast<int>((a1 - start) / row_bytes) : 0;
          }
          meta[slot].t = tj;
          meta[slot].c = cj;
          meta[slot].lo = loj;
          meta[slot].rows = rows_in;
          meta[slot].e = ej;
          meta[slot].skip = static_cast<int>((start - a0) / kBytes);
          const uint32_t bytes = a1 > a0 ? static_cast<uint32_t>(a1 - a0) : 0u;
          mbar_arrive_expect_tx(&full[slot], bytes);
          if (!p.debug_stall && bytes) bulk_g2s(ring + slot * slot_bytes, iq + a0, bytes, &full[slot]);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      ++r;
    }
  }
  return ok;
}

// Consumers of one staged item (generic staged consumer of das_staged.cuh with the
// instance's parameters in shared memory and a per-slot row offset).  FL lanes per voxel,
// 4 frames per lane: VEC = 4 consecutive frames (F % 4 == 0) or VEC = 1 with NV = 4 frames
// FL apart.
template <class IQ, int VEC, int NV, int FL>
__device__ __forceinline__ void batch_consume(const DasParams& p, int64_t tile, int warp, int lane,
                                              const unsigned char* ring, size_t slot_bytes, float4* terms, float* txc,
                                              const BatchSlotMeta* meta, uint64_t* full, uint64_t* empty) {
  constexpr int VPG = 4;
  constexpr int G = 32 / FL;
  constexpr int WV = G * VPG;
  constexpr int FPL = VEC * NV;
  constexpr int PB = 32 / WV;
  static_assert(FPL == 4 && WV * PB == 32 && kBatchRing >= PB, "lane mapping");
  using E = typename IqStore<IQ>::E;
  const E* ringE = reinterpret_cast<const E*>(ring);
  const size_t slot_elems = slot_bytes / sizeof(E);
  const int row_elems = p.F * IqStore<IQ>::eps;
  const E* __restrict__ iq = static_cast<const E*>(p.iq);
  const size_t slab = static_cast<size_t>(p.S) * row_elems;
  const bool tx_cached = p.T <= kTxCache;
  const int g = lane / FL, jl = lane % FL, sub = lane / WV, q = lane % WV;
  const int64_t v_term = tile_voxel(p, tile, warp * WV + q);
  const float4 vpos = v_term >= 0 ? p.vox[v_term] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int rec_at = (q % VPG) * G + (q / VPG);
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
    const int mine = r + sub, my_slot = mine % kBatchRing;
    const bool got = mbar_wait_bounded(&full[my_slot], (mine / kBatchRing) & 1, p.wait_limit);
    if (__any_sync(0xffffffffu, !got)) {
      if (lane == 0) atomicOr(p.err, 1);
      ok = false;
      break;
    }
    const int mc = meta[my_slot].c;
    float4 rec = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    if (mc >= 0) {
      if (mc != cur_c) {
        cur_c = mc;
        geo.a = -1.f;
        if (v_term >= 0) geo = term_geometry(vpos, meta[my_slot].e, p);
      }
      if (geo.a >= 0.f) {
        const int mt = meta[my_slot].t;
        const float stx = tx_cached ? txc[mt * 32 + lane] : __ldg(&p.tx[static_cast<size_t>(mt) * p.V + v_term]);
        rec = term_record(stx, geo, p);
      }
    }
    const int my_i0 = __float_as_int(rec.w);
    const bool active = my_i0 >= 0;
    const int mlo = meta[my_slot].lo, mrows = meta[my_slot].rows;
    const bool outside = active && (my_i0 - mlo < 0 || my_i0 - mlo + 1 >= mrows);
    const unsigned act = __ballot_sync(0xffffffffu, active);
    const unsigned outm = __ballot_sync(0xffffffffu, outside);
    const unsigned ended = __ballot_sync(0xffffffffu, mc < 0);
    terms[store_at] = rec;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const unsigned gm = WV == 32 ? 0xffffffffu : (((1u << (WV & 31)) - 1u) << (i * WV));
      if (ended & gm) {
        done = true;
        break;
      }
      if (!(act & gm)) continue;
      const int slot = (r + i) % kBatchRing;
      const int lo = meta[slot].lo, rows = meta[slot].rows;
      const E* win = ringE + slot * slot_elems + meta[slot].skip * IqStore<IQ>::eps;
      const float4* tp = terms + i * WV;
      if (!(outm & gm)) {
#pragma unroll
        for (int k = 0; k < VPG; ++k) {
          const float4 tr = tp[k * G + g];
          const int row = max(__float_as_int(tr.w) - lo, 0);
          const float4 cw = tap_weights(tr);
          gather_mac<IQ, VEC, NV, FL, true>(acc[k], win + row * row_elems, row_elems, p.F, 0, jl, cw.x, cw.y, cw.z,
                                            cw.w);
        }
      } else {
        const int t = meta[slot].t, c = meta[slot].c;
        const E* gsrc = iq + (static_cast<size_t>(t) * p.C + c) * slab;
#pragma unroll
        for (int k = 0; k < VPG; ++k) {
          const float4 tr = tp[k * G + g];
          const int i0 = __float_as_int(tr.w);
          if (i0 >= 0) {
            const float4 cw = tap_weights(tr);
            const int row = i0 - lo;
            if (row >= 0 && row + 1 < rows)
              gather_mac<IQ, VEC, NV, FL, true>(acc[k], win + row * row_elems, row_elems, p.F, 0, jl, cw.x, cw.y, cw.z,
                                                cw.w);
            else
              gather_mac<IQ, VEC, NV, FL, false>(acc[k], gsrc + static_cast<size_t>(i0) * row_elems, row_elems, p.F,
                                                 0, jl, cw.x, cw.y, cw.z, cw.w);
          }
        }
      }
    }
    __syncwarp();
    if (lane < PB) mbar_arrive(&empty[(r + lane) % kBatchRing]);
  }
  if (!ok) return;
#pragma unroll
  for (int k = 0; k < VPG; ++k) {
    const int64_t v = tile_voxel(p, tile, warp * WV + g * VPG + k);
    float pw = 0.f;
#pragma unroll
    for (int mm = 0; mm < NV; ++mm) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int f = (jl + FL * mm) * VEC + e;
        if (f < p.F) {
          const float2 a = acc_frame<IQ, VEC>(&acc[k][mm * VEC], e);
          pw = fmaf(a.x, a.x, fmaf(a.y, a.y, pw));
          if (v >= 0 && p.y) p.y[v * p.ystride + f] = a;
        }
      }
    }
#pragma unroll
    for (int o = FL / 2; o > 0; o >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, o);
    if (jl == 0 && v >= 0 && p.pd) p.pd[v] = pw;
  }
}

// counter[0]: next work item; counter[1]: blocks that have finished.
template <class IQ>
__global__ void __launch_bounds__(kBatchWarps * 32, 2)
    k_das_batch(const BatchInstance* __restrict__ insts, const int2* __restrict__ items, int n_items, int* counter,
                size_t slot_bytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_item;
  const BatchLayout L(slot_bytes);
  BatchSlotMeta* meta = reinterpret_cast<BatchSlotMeta*>(smem + L.meta_off());
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off());
  uint64_t* empty = full + kBatchRing;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* scratch = smem + L.scratch_off() + warp * (L.scratch_bytes / kBatchWarps);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&counter[0], 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const int2 w = items[it];
    const BatchInstance& B = insts[w.x];
    const DasParams p = B.p;
    const int mode = B.mode, fl = B.frame_lanes;
    if (mode == kBatchStaged) {
      if (threadIdx.x == 0) {   // a fresh ring for this item
        for (int b = 0; b < kBatchRing; ++b) {
          mbar_init(&full[b], 1);
          mbar_init(&empty[b], kBatchConsumers);
        }
        mbar_init_fence();
      }
      __syncthreads();
      if (warp == kBatchConsumers) {
        int r = 0;
        const bool ok = batch_produce<IQ>(p, w.y, lane, smem, slot_bytes, meta, full, empty, r);
        if (lane == 0) {   // end markers (one per pair a consumer round holds), or drain
          const int PB = fl == 16 ? 4 : 2;
          if (ok) {
            for (int k = 0; k < PB; ++k) {
              const int rr = r + k, slot = rr % kBatchRing;
              if (rr >= kBatchRing && !mbar_wait_bounded(&empty[slot], ((rr / kBatchRing) - 1) & 1, p.wait_limit)) {
                atomicOr(p.err, 1);
                break;
              }
              meta[slot].c = -1;
              mbar_arrive(&full[slot]);
            }
          } else {
            for (int k = max(0, r - kBatchRing); k < r; ++k)
              mbar_wait_bounded(&full[k % kBatchRing], (k / kBatchRing) & 1, p.wait_limit);
          }
        }
      } else {
        float4* terms = reinterpret_cast<float4*>(scratch);
        float* txc = reinterpret_cast<float*>(scratch + 32 * 16);
        // 16-byte vectors when F % 4 == 0, 8-byte pairs for the other even F, else single samples
        const int vec = p.F % 4 == 0 ? 4 : (p.F % 2 == 0 ? 2 : 1);
        if (fl == 16) {
          if (vec == 4) batch_consume<IQ, 4, 1, 16>(p, w.y, warp, lane, smem, slot_bytes, terms, txc, meta, full, empty);
          else if (vec == 2) batch_consume<IQ, 2, 2, 16>(p, w.y, warp, lane, smem, slot_bytes, terms, txc, meta, full, empty);
          else batch_consume<IQ, 1, 4, 16>(p, w.y, warp, lane, smem, slot_bytes, terms, txc, meta, full, empty);
        } else {
          if (vec == 4) batch_consume<IQ, 4, 1, 8>(p, w.y, warp, lane, smem, slot_bytes, terms, txc, meta, full, empty);
          else if (vec == 2) batch_consume<IQ, 2, 2, 8>(p, w.y, warp, lane, smem, slot_bytes, terms, txc, meta, full, empty);
          else batch_consume<IQ, 1, 4, 8>(p, w.y, warp, lane, smem, slot_bytes, terms, txc, meta, full, empty);
        }
      }
      __syncthreads();   // the ring is drained before the next item re-initialises it
    } else if (mode == kBatchChannels) {
      batch_channels_tile<IQ>(p, w.y);
    } else if (fl == 2) {
      if (p.F % 4 == 0) batch_frames_tile<IQ, 4, 1, 2>(p, fl, w.y, reinterpret_cast<float4*>(scratch));
      else if (p.F % 2 == 0) batch_frames_tile<IQ, 2, 2, 2>(p, fl, w.y, reinterpret_cast<float4*>(scratch));
      else batch_frames_tile<IQ, 1, 4, 2>(p, fl, w.y, reinterpret_cast<float4*>(scratch));
    } else if (p.F % 4 == 0) {
      batch_frames_tile<IQ, 4, 1, 4>(p, fl, w.y, reinterpret_cast<float4*>(scratch));
    } else if (p.F % 2 == 0) {
      batch_frames_tile<IQ, 2, 2, 4>(p, fl, w.y, reinterpret_cast<float4*>(scratch));
    } else {
      batch_frames_tile<IQ, 1, 4, 4>(p, fl, w.y, reinterpret_cast<float4*>(scratch));
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
                            size_t slot_bytes, cudaStream_t s) {
  const size_t smem = BatchLayout(slot_bytes).total();
  cudaError_t e = cudaFuncSetAttribute(k_das_batch<IQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_das_batch<IQ><<<grid, kBatchWarps * 32, smem, s>>>(insts, items, n_items, counter, slot_bytes);
  return cudaGetLastError();
}

size_t batch_smem_bytes(size_t slot_bytes) { return BatchLayout(slot_bytes).total(); }

int batch_blocks_per_sm(int iq_dtype, size_t slot_bytes) {
  const size_t smem = BatchLayout(slot_bytes).total();
  int n = 0;
  cudaError_t e;
  switch (iq_dtype) {
    case MACH_IQ_F16X2:
      cudaFuncSetAttribute(k_das_batch<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_das_batch<__half2>, kBatchWarps * 32, smem);
      break;
    case MACH_IQ_BF16X2:
      cudaFuncSetAttribute(k_das_batch<__nv_bfloat162>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_das_batch<__nv_bfloat162>, kBatchWarps * 32, smem);
      break;
    default:
      cudaFuncSetAttribute(k_das_batch<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_das_batch<float2>, kBatchWarps * 32, smem);
      break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_batch(int iq_dtype, const BatchInstance* insts, const int2* items, int n_items, int* counter,
                         int grid, size_t slot_bytes, cudaStream_t s) {
  switch (iq_dtype) {
    case MACH_IQ_C64: return go_batch<float2>(insts, items, n_items, counter, grid, slot_bytes, s);
    case MACH_IQ_F16X2: return go_batch<__half2>(insts, items, n_items, counter, grid, slot_bytes, s);
    case MACH_IQ_BF16X2: return go_batch<__nv_bfloat162>(insts, items, n_items, counter, grid, slot_bytes, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mach
