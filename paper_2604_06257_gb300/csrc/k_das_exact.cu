// k_das_exact.cu -- the staged delay-and-sum kernel for split complex64 rows when the
// ensemble fills the frame tile exactly (F = 32 or F = 64), with receive delays evaluated
// on the fly (Sec. 4.3's hybrid delays) and reused across the frames (Sec. 4.4).
//
// Same work, order and arithmetic as k_das_staged<C64Planar, ...> (das_staged.cuh): the
// same producer warp stages each usable (element, transmit) pair's sample window into a
// shared-memory ring with one bulk copy, the same lanes evaluate the same terms, and every
// frame receives the same FMA sequence, so the outputs are bitwise equal.  What differs is
// the consumer's instruction stream, which bounds the generic kernel (about 84 thread
// instructions per 4 term-frames, 16 of them packed FMAs):
//  * the frame count is a compile-time constant, so a sample row is RB = 8 F bytes (F real
//    parts, then F imaginary parts) and the four tap loads of a term are one 32-bit shared
//    address plus constant offsets (0, F*4, RB, RB + F*4); no per-frame bounds tests;
//  * the lane that evaluates a term also forms its two complex tap weights and the byte
//    offset of its first tap row inside the staged window, so a consuming lane reads a
//    16-byte weight record and a 4-byte offset and adds one integer per term;
//  * all shared-memory traffic of the inner loop uses 32-bit shared addresses.
#include <cuda_runtime.h>
#include <cstdint>

#include "das_staged.cuh"

namespace mach {
namespace {

// Shared memory: [ring slots][tap weights][row offsets][transmit-delay cache][slot metadata][barriers].
template <int NBUF>
struct ExactLayout {
  size_t slot_bytes, coef_bytes, offs_bytes, tx_bytes;
  __host__ __device__ ExactLayout(int rows_cap, int row_bytes, int T, int nwc)
      : slot_bytes((static_cast<size_t>(rows_cap) * row_bytes + 127) / 128 * 128),
        coef_bytes(static_cast<size_t>(nwc) * 32 * 16),
        offs_bytes(static_cast<size_t>(nwc) * 32 * 4),
        tx_bytes(T <= kTxCache ? static_cast<size_t>(nwc) * T * 32 * 4 : 0) {}
  __host__ __device__ size_t coef_off() const { return NBUF * slot_bytes; }
  __host__ __device__ size_t offs_off() const { return coef_off() + coef_bytes; }
  __host__ __device__ size_t tx_off() const { return offs_off() + offs_bytes; }
  __host__ __device__ size_t meta_off() const { return tx_off() + (tx_bytes + 15) / 16 * 16; }
  __host__ __device__ size_t bar_off() const { return meta_off() + NBUF * 32; }
  __host__ __device__ size_t total() const { return bar_off() + 2 * NBUF * 8; }
};

__device__ __forceinline__ float4 lds128(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ int lds32(uint32_t a) {
  int v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts128(uint32_t a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
__device__ __forceinline__ void sts32(uint32_t a, int v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// One term into 4 frames of a lane (split rows): taps x0 = (re ar, im ai) at row i0 and
// x1 = (re br, im bi) at row i0 + 1, weights cw = (c0r, c0i, c1r, c1i).  Per frame the
// FMA sequence of tap_mac.cuh: re += c0r x0re - c0i x0im + c1r x1re - c1i x1im and
// im += c0r x0im + c0i x0re + c1r x1im + c1i x1re, two frames per packed FMA.
// acc[2h] = (re of frames 2h, 2h+1), acc[2h+1] = (im of frames 2h, 2h+1).
__device__ __forceinline__ void mac4(float2* acc, const float4 cw, const float4 ar, const float4 ai, const float4 br,
                                     const float4 bi) {
  const float2 C0R = make_float2(cw.x, cw.x), C0N = make_float2(-cw.y, -cw.y), C0I = make_float2(cw.y, cw.y);
  const float2 C1R = make_float2(cw.z, cw.z), C1N = make_float2(-cw.w, -cw.w), C1I = make_float2(cw.w, cw.w);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float2 x0r = h ? make_float2(ar.z, ar.w) : make_float2(ar.x, ar.y);
    const float2 x0i = h ? make_float2(ai.z, ai.w) : make_float2(ai.x, ai.y);
    const float2 x1r = h ? make_float2(br.z, br.w) : make_float2(br.x, br.y);
    const float2 x1i = h ? make_float2(bi.z, bi.w) : make_float2(bi.x, bi.y);
    float2& re = acc[2 * h];
    float2& im = acc[2 * h + 1];
    re = __ffma2_rn(C0R, x0r, re);
    re = __ffma2_rn(C0N, x0i, re);
    re = __ffma2_rn(C1R, x1r, re);
    re = __ffma2_rn(C1N, x1i, re);
    im = __ffma2_rn(C0R, x0i, im);
    im = __ffma2_rn(C0I, x0r, im);
    im = __ffma2_rn(C1R, x1i, im);
    im = __ffma2_rn(C1I, x1r, im);
  }
}

// Frame chunks of a lane: FPL / 4 chunks of 4 consecutive frames.  Chunk c of lane jl of
// lane group g starts at frame 4 (jl + FL (c ^ swz)), swz = g & 1 when FL = 4 and a lane
// holds two chunks: the two lane groups of a quarter warp then read opposite halves of
// their rows first, which keeps every 128-bit load free of bank conflicts.
template <int FL, int FPL>
__device__ __forceinline__ int chunk_swizzle(int g) {
  return (FL == 4 && FPL == 8) ? (g & 1) : 0;
}

// Accumulators of one lane: VPG voxel slots x FPL frames, as packed pairs.
template <int VPG, int FPL>
struct Acc {
  float2 a[VPG][FPL];
};

// The terms of one pair when some kept term falls outside the staged window (not
// expected: the windows carry a margin): such terms read their taps from global memory.
// Out of line, with the accumulators passed and returned by value, so that neither its
// registers nor an address of the accumulators burden the hot loop.
template <int FT, int FPL, int VPG, int G>
__device__ __noinline__ Acc<VPG, FPL> outside_pair(const DasParams& p, Acc<VPG, FPL> acc, const SlotMeta m,
                                                   const unsigned char* wsrc, uint32_t cw_at, uint32_t of_at, int jl,
                                                   int swz) {
  constexpr int RB = FT * 8, IMO = FT * 4, FL = FT / FPL;
  const unsigned char* gsrc =
      static_cast<const unsigned char*>(p.iq) + ((static_cast<size_t>(m.t) * p.C + m.c) * p.S + m.lo) * RB + jl * 16;
#pragma unroll
  for (int k = 0; k < VPG; ++k) {
    const float4 cw = lds128(cw_at + k * G * 16);
    const int off = lds32(of_at + k * G * 4);
    const int rrow = off / RB;
    const unsigned char* src = (rrow >= 0 && rrow + 1 < m.rows ? wsrc : gsrc) + off;
#pragma unroll
    for (int c = 0; c < FPL / 4; ++c) {
      const unsigned char* x = src + (c ^ swz) * FL * 16;
      mac4(&acc.a[k][4 * c], cw, *reinterpret_cast<const float4*>(x), *reinterpret_cast<const float4*>(x + IMO),
           *reinterpret_cast<const float4*>(x + RB), *reinterpret_cast<const float4*>(x + RB + IMO));
    }
  }
  return acc;
}

// FT: frames (= F); FPL frames per lane (4 or 8), FL = FT / FPL lanes per voxel, VPG voxel
// slots per lane group; NWC consumer warps + 1 producer warp; NBUF ring slots; MAXR
// registers per thread.
// FLAGS bit 0: consumers suspended in hardware while waiting for a window; bit 1: a warp
// releases each ring slot right after its last read instead of at the end of the round.
constexpr int kSleep = 1, kEarly = 2;

template <int FT, int FPL, int VPG, int NWC, int NBUF, int MAXR, int FLAGS>
__global__ void __launch_bounds__((NWC + 1) * 32) __maxnreg__(MAXR) k_das_exact(const DasParams p) {
  constexpr int FL = FT / FPL;
  constexpr int G = 32 / FL;
  constexpr int WV = G * VPG;
  constexpr int PB = 32 / WV;           // pairs whose terms one warp evaluates per round
  constexpr int RB = FT * 8;            // bytes per sample row
  constexpr int IMO = FT * 4;           // imaginary parts' offset inside a row
  static_assert(FPL == 4 || FPL == 8, "4 or 8 frames per lane");
  static_assert(WV * PB == 32, "a round must fill the warp");
  static_assert(NBUF >= PB && NBUF % PB == 0, "a round must fit in the ring");
  extern __shared__ __align__(128) unsigned char smem[];
  const ExactLayout<NBUF> L(p.rows_cap, RB, p.T, NWC);
  SlotMeta* meta = reinterpret_cast<SlotMeta*>(smem + L.meta_off());
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off());
  uint64_t* empty = full + NBUF;
  const bool tx_cached = p.T <= kTxCache;
  float* txc_all = reinterpret_cast<float*>(smem + L.tx_off());

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // the last tiles (deepest rows of the grid, the widest apertures: the most pairs) start
  // first, so that the light shallow tiles fill the tail of the launch
  const int64_t tile = static_cast<int64_t>(gridDim.x) - 1 - blockIdx.x;

  if (threadIdx.x == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], NWC);
    }
    mbar_init_fence();
  }
  __syncthreads();

  if (warp == NWC) {   // producer
    int r = 0;
    const bool ok = produce_windows<NBUF>(p, tile, lane, smem, L.slot_bytes, 8, meta, full, empty, r);
    if (lane == 0) finish_producer<NBUF, PB>(p, ok, r, meta, full, empty);
    return;
  }

  // ------------------------------------------------------------------ consumers
  // Lane group g (FL lanes) accumulates the frames of its chunks for the voxel slots
  // g VPG + k.  Each round lane group `sub` (WV lanes) evaluates the terms of pair r + sub
  // for the warp's WV voxels; the weights of voxel slot g VPG + k for pair i sit at entry
  // i WV + k G + g, so the G groups read G consecutive entries (conflict-free broadcast).
  const int g = lane / FL;
  const int jl = lane % FL;
  const int sub = lane / WV;
  const int q = lane % WV;
  const int swz = chunk_swizzle<FL, FPL>(g);
  float* txc = txc_all + warp * (p.T * 32);
  const int64_t v_term = tile_voxel_blocked(p, tile, warp * WV + q);
  const float4 vpos = v_term >= 0 ? p.vox[v_term] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int store_at = sub * WV + (q % VPG) * G + (q / VPG);
  const uint32_t s0 = smem_u32(smem);
  const uint32_t coef_w = s0 + static_cast<uint32_t>(L.coef_off()) + warp * 32 * 16;
  const uint32_t offs_w = s0 + static_cast<uint32_t>(L.offs_off()) + warp * 32 * 4;
  const uint32_t slot_bytes = static_cast<uint32_t>(L.slot_bytes);
  const uint32_t lane_tap = s0 + jl * 16 + swz * FL * 16;   // chunk 0; chunk 1 at +/- FL * 16
  if (tx_cached) {
    for (int t = 0; t < p.T; ++t) txc[t * 32 + lane] = v_term >= 0 ? p.tx[static_cast<size_t>(t) * p.V + v_term] : 0.f;
  }

  Acc<VPG, FPL> acc;
#pragma unroll
  for (int k = 0; k < VPG; ++k)
#pragma unroll
    for (int e = 0; e < FPL; ++e) acc.a[k][e] = make_float2(0.f, 0.f);

  int cur_c = -1;
  TermGeo geo;
  geo.rx = 0.f;
  geo.a = -1.f;
  bool ok = true, done = false;
  for (int r = 0; !done; r += PB) {
    const int mine = r + sub, my_slot = mine % NBUF;
    const bool got = (FLAGS & kSleep) ? mbar_wait_bounded_sleep(&full[my_slot], (mine / NBUF) & 1, p.wait_limit, 1000)
                              : mbar_wait_bounded(&full[my_slot], (mine / NBUF) & 1, p.wait_limit);
    if (__any_sync(0xffffffffu, !got)) {
      if (lane == 0) atomicOr(p.err, 1);
      ok = false;
      break;
    }
    const SlotMeta mm = meta[my_slot];
    float4 rec = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
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
    // dropped terms: zero weights (rec.x = rec.y = rec.z = 0) and row 0 of the window
    const int i0 = __float_as_int(rec.w);
    const bool active = i0 >= 0;
    const int row = active ? i0 - mm.lo : 0;
    const bool outside = active && (row < 0 || row + 1 >= mm.rows);
    sts128(coef_w + store_at * 16, tap_weights(rec));
    sts32(offs_w + store_at * 4, row * RB);
    const unsigned act = __ballot_sync(0xffffffffu, active);
    const unsigned outm = __ballot_sync(0xffffffffu, outside);
    const unsigned ended = __ballot_sync(0xffffffffu, mm.c < 0);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const unsigned gm = WV == 32 ? 0xffffffffu : (((1u << (WV & 31)) - 1u) << (i * WV));
      if (ended & gm) {   // end marker: every later pair of the round is one too
        done = true;
        break;
      }
      const int slot = (r + i) % NBUF;
      if (!(act & gm)) {
        if constexpr ((FLAGS & kEarly) != 0) {
          if (lane == 0) mbar_arrive(&empty[slot]);
        }
        continue;
      }
      const uint32_t win = lane_tap + slot * slot_bytes;
      const uint32_t cw_at = coef_w + (i * WV + g) * 16;
      const uint32_t of_at = offs_w + (i * WV + g) * 4;
      if (!(outm & gm)) {
        // every kept term lies in the staged window: branch-free over the voxels
#pragma unroll
        for (int k = 0; k < VPG; ++k) {
          const float4 cw = lds128(cw_at + k * G * 16);
          const uint32_t a = win + lds32(of_at + k * G * 4);
#pragma unroll
          for (int c = 0; c < FPL / 4; ++c) {
            // chunk c lies (c ^ swz - swz) FL * 16 bytes from chunk 0's lane address
            const uint32_t b = a + ((c ^ swz) - swz) * FL * 16;
            mac4(&acc.a[k][4 * c], cw, lds128(b), lds128(b + IMO), lds128(b + RB), lds128(b + RB + IMO));
          }
        }
      } else {
        acc = outside_pair<FT, FPL, VPG, G>(p, acc, meta[slot], smem + slot * slot_bytes + jl * 16, cw_at, of_at,
                                            jl, swz);
      }
      if constexpr ((FLAGS & kEarly) != 0) {   // every lane has read the slot: release it
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
      }
    }
    if constexpr ((FLAGS & kEarly) == 0) {
      __syncwarp();
      if (lane < PB) mbar_arrive(&empty[(r + lane) % NBUF]);
    }
  }
  if (!ok) return;

  // epilogue: complex frames and sum_f |y|^2 (Sec. 5), reduced over the FL lanes
#pragma unroll
  for (int k = 0; k < VPG; ++k) {
    const int64_t v = tile_voxel_blocked(p, tile, warp * WV + g * VPG + k);
    float pw = 0.f;
#pragma unroll
    for (int c = 0; c < FPL / 4; ++c) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 a = acc_frame<C64Planar, 4>(&acc.a[k][4 * c], e);
        pw = fmaf(a.x, a.x, fmaf(a.y, a.y, pw));
      }
      if (v >= 0 && p.y) {
        float2* dst = p.y + v * p.ystride + 4 * (jl + FL * (c ^ swz));
        const float2 a0 = acc_frame<C64Planar, 4>(&acc.a[k][4 * c], 0), a1 = acc_frame<C64Planar, 4>(&acc.a[k][4 * c], 1);
        const float2 a2 = acc_frame<C64Planar, 4>(&acc.a[k][4 * c], 2), a3 = acc_frame<C64Planar, 4>(&acc.a[k][4 * c], 3);
        *reinterpret_cast<float4*>(dst) = make_float4(a0.x, a0.y, a1.x, a1.y);
        *reinterpret_cast<float4*>(dst + 2) = make_float4(a2.x, a2.y, a3.x, a3.y);
      }
    }
#pragma unroll
    for (int o = FL / 2; o > 0; o >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, o);
    if (jl == 0 && v >= 0 && p.pd) p.pd[v] = pw;
  }
}

}  // namespace

size_t exact_smem_bytes(Variant v, int rows_cap, int T) {
  const VariantShape& sh = variant_shape(v);
  const int rb = sh.frame_tile * 8;
  switch (sh.ring_slots) {
    case 4: return ExactLayout<4>(rows_cap, rb, T, sh.warps).total();
    case 8: return ExactLayout<8>(rows_cap, rb, T, sh.warps).total();
    case 12: return ExactLayout<12>(rows_cap, rb, T, sh.warps).total();
    default: return ExactLayout<16>(rows_cap, rb, T, sh.warps).total();
  }
}

cudaError_t launch_das_exact(const DasParams& p, Variant v, cudaStream_t s) {
  if (p.F != variant_shape(v).frame_tile || p.frame_tiles != 1) return cudaErrorInvalidValue;
  const size_t sm = exact_smem_bytes(v, p.rows_cap, p.T);
  switch (v) {
    //                                        FT FPL VPG NWC NBUF MAXR FLAGS
    case V_SX32_C64P: case V_SX32_C64P_T8X14: return go_staged(k_das_exact<32, 4, 4, 7, 4, 64, 0>, 7, p, sm, s);
    case V_SX32_F4V2W7: return go_staged(k_das_exact<32, 4, 2, 7, 8, 64, 0>, 7, p, sm, s);
    case V_SX32_F8V1W7: return go_staged(k_das_exact<32, 8, 1, 7, 8, 64, 0>, 7, p, sm, s);
    case V_SX32_F4V2W15: return go_staged(k_das_exact<32, 4, 2, 15, 8, 64, 0>, 15, p, sm, s);
    case V_SX32_F8V1W15: case V_SX32_F8V1W15T24: case V_SX32_F8V1W15T40:
      return go_staged(k_das_exact<32, 8, 1, 15, 8, 64, 0>, 15, p, sm, s);
    case V_SX32_F8V1W15T24S: return go_staged(k_das_exact<32, 8, 1, 15, 8, 64, kSleep>, 15, p, sm, s);
    case V_SX32_F8V1W7T14: return go_staged(k_das_exact<32, 8, 1, 7, 8, 64, 0>, 7, p, sm, s);
    case V_SX32_F8V1W7T14E: case V_SX32_F8V1W7_T8X7E:
      return go_staged(k_das_exact<32, 8, 1, 7, 8, 64, kEarly>, 7, p, sm, s);
    case V_SX32_F4V2W7T14: return go_staged(k_das_exact<32, 4, 2, 7, 8, 64, 0>, 7, p, sm, s);
    case V_SX32_F8V1W15T30R12: return go_staged(k_das_exact<32, 8, 1, 15, 12, 64, 0>, 15, p, sm, s);
    case V_SX32_F8V1W15T30R12E: return go_staged(k_das_exact<32, 8, 1, 15, 12, 64, kEarly>, 15, p, sm, s);
    case V_SX64_C64P: case V_SX64_C64P_T16: case V_SX64_C64P_T8X8:
      return go_staged(k_das_exact<64, 4, 4, 8, 8, 72, 0>, 8, p, sm, s);
    case V_SX64_C64P_T16E: return go_staged(k_das_exact<64, 4, 4, 8, 8, 72, kEarly>, 8, p, sm, s);
    case V_SX64_C64PS: return go_staged(k_das_exact<64, 4, 4, 8, 8, 72, kSleep>, 8, p, sm, s);
    case V_SX64_C64PE: return go_staged(k_das_exact<64, 4, 4, 8, 8, 72, kEarly>, 8, p, sm, s);
    case V_SX64_F8V2: return go_staged(k_das_exact<64, 8, 2, 8, 8, 72, 0>, 8, p, sm, s);
    case V_SX16_F4V2W7: case V_SX16_F4V2W7_T8X14:
      return go_staged(k_das_exact<16, 4, 2, 7, 8, 64, kEarly>, 7, p, sm, s);
    case V_SX16_F4V1W7: return go_staged(k_das_exact<16, 4, 1, 7, 8, 64, kEarly>, 7, p, sm, s);
    case V_SX8_F4V1W7: case V_SX8_F4V1W7_T8X14: return go_staged(k_das_exact<8, 4, 1, 7, 8, 64, kEarly>, 7, p, sm, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mach
