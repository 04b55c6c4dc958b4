// k_conv_tc.cu -- 3x3x3 "same" convolution on the 5th-generation tensor cores (tcgen05).
//
// Implicit GEMM: rows = output voxels, columns = output channels, K = 27 taps x input
// channels.  An output tile is 8 (x) x 16 (y) x 1 (z) voxels = 128 GEMM rows (M = 128).
//
//  * A operand: for every 8-channel group the tile's halo brick (10 x 18 x 3 voxels x 16
//    bytes) is loaded once by a 5D TMA tiled copy (out-of-range voxels arrive as zeros,
//    which is the convolution's zero padding).  In shared memory a brick is the
//    no-swizzle K-major canonical layout: 8 consecutive x-voxels of one y-row form an
//    8 x 16-byte core matrix, y-rows are 160 bytes apart (the stride between 8-row
//    groups), the two 8-channel groups of a 16-channel step are one group pitch apart.
//    The A operand of tap (dz, dy, dx) is the same brick seen from another start
//    address, so the 27 taps reuse one load.
//  * B operand: weights pre-packed on the device (mach_nn_pack_weights) so that one tap
//    x 16 input channels is one contiguous block in the same canonical layout (rows =
//    output channels); a bulk copy per tap streams them through an 8-slot ring.
//  * Roles (192 threads, persistent over tiles): warp 0 issues the copies, one thread of
//    warp 1 issues tcgen05.mma (accumulator in tensor memory, two buffers so that the
//    epilogue of one tile overlaps the MMAs of the next), warps 2-5 drain tensor memory
//    (tcgen05.ld), add the bias, apply the leaky ReLU and store bfloat16 / float32.
//  * Every wait is bounded; a wait that gives up sets the device error word, the CTA
//    stops issuing work, waits (bounded) for its MMAs and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <unordered_map>

#include "async_copy.cuh"
#include "mach_nn.h"
#include "nn_internal.h"

namespace mach_nn {

using bf16 = __nv_bfloat16;
using mach::bulk_g2s;
using mach::mbar_arrive;
using mach::mbar_arrive_expect_tx;
using mach::mbar_init;
using mach::mbar_init_fence;
using mach::mbar_wait_bounded;
using mach::smem_u32;

constexpr int kTX = 8, kTY = 16;                             // output tile (x, y) per z plane
constexpr int kHX = kTX + 2, kHY = kTY + 2;                  // halo brick in x, y
constexpr int kNB = 2;                                       // weight ring slots (streamed weights)
constexpr int kThreads = 192;
constexpr uint32_t kDefaultWait = 1u << 24;
constexpr uint32_t kResidentMax = 96 * 1024;                 // weights kept whole in shared memory

__device__ int g_conv_tc_err;   // bit 0: a bounded wait gave up
uint32_t g_wait_limit = 0;      // test hook: polls per bounded wait (0: default)
int g_debug_stall = 0;          // test hook: see ConvTcParams::debug_stall, bit 1: the final wait gave up
int g_conv_fold = 1;            // x-folded kernel for 16 output channels (test hook: 0 = off)
int g_fold_tz = 4;              // z planes per x-folded tile (1, 2 or 4)
int g_fold_stages = 0;          // halo stages of the x-folded kernel (0: as many as fit, up to 4)

struct ConvTcParams {
  const bf16* wpk;      // packed weights [Ci/16][27][2][Co][8]
  const float* bias;    // [Co] or nullptr
  bf16* y;              // [N][D][H][W][Co] or nullptr
  float* yf;            // [N][D][H][W][Co] or nullptr
  int N, D, H, W, Ci, Co;
  int flip, act;
  int tz;               // z planes per tile (1 or 2): one M = 128 MMA per plane and tap
  int resident;         // all weights loaded once per CTA (else 9-tap blocks through a ring)
  int tiles_x, tiles_y, tiles_z;
  int64_t tiles;
  uint32_t group_pitch; // bytes between the two 8-channel groups of a halo stage
  int a_stages;         // halo stages in flight (x-folded kernel: 2 ... 4)
  uint32_t tmem_cols;
  uint32_t wait_limit;
  int debug_stall;      // test hook: the copy warp issues nothing, so every wait runs out
};

// tcgen05 shared-memory matrix descriptor: no swizzle, start address, leading (K
// direction) and stride (M/N direction) byte offsets between core matrices.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
         (static_cast<uint64_t>(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D float32, A and B bfloat16, both K-major, M = 128
__host__ __device__ constexpr uint32_t instr_desc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) | ((128u >> 4) << 24);
}

// Bounded wait for the issuing threads: spins without sleeping first (these threads sit
// on the critical path), then backs off.
__device__ __forceinline__ bool wait_spin(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mach::mbar_try_wait(bar, parity)) return true;
    if (i > 4096) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Three tensor-memory loads of 16 columns each, one wait for all of them.
__device__ __forceinline__ void tmem_ld16x3(uint32_t taddr, uint32_t (&a)[16], uint32_t (&b)[16],
                                            uint32_t (&c)[16]) {
#define MACH_TMEM_LD16(dst, addr)                                                                               \
  asm volatile(                                                                                                \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
      : "=r"(dst[0]), "=r"(dst[1]), "=r"(dst[2]), "=r"(dst[3]), "=r"(dst[4]), "=r"(dst[5]), "=r"(dst[6]),       \
        "=r"(dst[7]), "=r"(dst[8]), "=r"(dst[9]), "=r"(dst[10]), "=r"(dst[11]), "=r"(dst[12]), "=r"(dst[13]),   \
        "=r"(dst[14]), "=r"(dst[15])                                                                           \
      : "r"(addr))
  MACH_TMEM_LD16(a, taddr);
  MACH_TMEM_LD16(b, taddr + 16);
  MACH_TMEM_LD16(c, taddr + 32);
#undef MACH_TMEM_LD16
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TileCoord {
  int n, z0, x0, y0;
};
__device__ __forceinline__ TileCoord tile_coord(const ConvTcParams& p, int64_t tile) {
  TileCoord c;
  const int tx = static_cast<int>(tile % p.tiles_x);
  int64_t r = tile / p.tiles_x;
  const int ty = static_cast<int>(r % p.tiles_y);
  r /= p.tiles_y;
  c.z0 = static_cast<int>(r % p.tiles_z) * p.tz;
  c.n = static_cast<int>(r / p.tiles_z);
  c.x0 = tx * kTX;
  c.y0 = ty * kTY;
  return c;
}

// x-folded tiles: 16 GEMM rows along x starting one voxel before the 14 outputs
__device__ __forceinline__ TileCoord tile_coord_x(const ConvTcParams& p, int64_t tile) {
  TileCoord c;
  const int tx = static_cast<int>(tile % p.tiles_x);
  int64_t r = tile / p.tiles_x;
  const int ty = static_cast<int>(r % p.tiles_y);
  r /= p.tiles_y;
  c.z0 = static_cast<int>(r % p.tiles_z) * p.tz;
  c.n = static_cast<int>(r / p.tiles_z);
  c.x0 = tx * 14 - 1;
  c.y0 = ty * 8;
  return c;
}

template <bool FLIP, int TZ>
__global__ void __launch_bounds__(kThreads, 3) k_conv3d_tc(const __grid_constant__ CUtensorMap xmap,
                                                           const ConvTcParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t tap_bytes = 32u * static_cast<uint32_t>(p.Co);   // one tap x 16 input channels
  const uint32_t a_stage = 2 * p.group_pitch;
  const uint32_t halo_bytes = static_cast<uint32_t>(kHX * kHY * (p.tz + 2) * 16);
  const int NC = p.Ci / 16;
  const uint32_t w_bytes = p.resident ? 27u * NC * tap_bytes : kNB * 9u * tap_bytes;
  uint8_t* sA = sm;
  uint8_t* sW = sm + 2 * a_stage;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sW + w_bytes);
  uint64_t* fullA = bars;          // [2]
  uint64_t* emptyA = bars + 2;     // [2]
  uint64_t* fullB = bars + 4;      // [kNB] (resident: fullB[0] = all weights)
  uint64_t* emptyB = bars + 6;     // [kNB]
  uint64_t* tfull = bars + 8;      // [2]
  uint64_t* tempty = bars + 10;    // [2]
  uint64_t* fin = bars + 12;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 13);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&fullA[i], 1);
      mbar_init(&emptyA[i], 1);
      mbar_init(&fullB[i], 1);
      mbar_init(&emptyB[i], 1);
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 128);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t limit = p.wait_limit;
  const uint32_t acc_cols = static_cast<uint32_t>(p.tz * p.Co);   // one accumulator buffer

  auto give_up = [&]() {
    atomicOr(&g_conv_tc_err, 1);
    *abort_flag = 1;
  };

  if (warp == 0) {
    if (lane == 0 && !p.debug_stall) {   // ----------------------------- copies
      if (p.resident) {
        mbar_arrive_expect_tx(&fullB[0], w_bytes);
        bulk_g2s(sW, p.wpk, w_bytes, &fullB[0]);
      }
      uint32_t a_use = 0, b_use = 0;
      for (int64_t tile = blockIdx.x; tile < p.tiles && !*abort_flag; tile += gridDim.x) {
        const TileCoord tc = tile_coord(p, tile);
        for (int kc = 0; kc < NC && !*abort_flag; ++kc) {
          const uint32_t sa = a_use & 1u, ka = a_use >> 1;
          if (ka >= 1 && !wait_spin(&emptyA[sa], (ka - 1) & 1u, limit)) {
            give_up();
            break;
          }
          mbar_arrive_expect_tx(&fullA[sa], 2 * halo_bytes);
          for (int g = 0; g < 2; ++g)
            tma_load_5d(smem_u32(sA + sa * a_stage + g * p.group_pitch), &xmap, kc * 16 + g * 8, tc.x0 - 1,
                        tc.y0 - 1, tc.z0 - 1, tc.n, &fullA[sa]);
          ++a_use;
          if (p.resident) continue;
          for (int t0 = 0; t0 < 27; t0 += 9) {
            const uint32_t sb = b_use % kNB, kb = b_use / kNB;
            if (kb >= 1 && !wait_spin(&emptyB[sb], (kb - 1) & 1u, limit)) {
              give_up();
              break;
            }
            mbar_arrive_expect_tx(&fullB[sb], 9 * tap_bytes);
            bulk_g2s(sW + sb * 9 * tap_bytes, p.wpk + (static_cast<size_t>(kc) * 27 + t0) * 16 * p.Co,
                     9 * tap_bytes, &fullB[sb]);
            ++b_use;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // ---------------------------------------------- MMAs
      const uint32_t idesc = instr_desc(p.Co);
      bool ok = !p.resident || wait_spin(&fullB[0], 0, limit);
      if (!ok) give_up();
      uint32_t a_use = 0, b_use = 0, acc_use = 0;
      for (int64_t tile = blockIdx.x; ok && tile < p.tiles && !*abort_flag; tile += gridDim.x) {
        const uint32_t buf = acc_use & 1u, ku = acc_use >> 1;
        if (ku >= 1 && !wait_spin(&tempty[buf], (ku - 1) & 1u, limit)) {
          give_up();
          break;
        }
        fence_after();
        const uint32_t d0 = tmem + buf * (p.tmem_cols >> 1);
        for (int kc = 0; kc < NC && ok; ++kc) {
          const uint32_t sa = a_use & 1u, ka = a_use >> 1;
          if (!wait_spin(&fullA[sa], ka & 1u, limit)) {
            give_up();
            ok = false;
            break;
          }
          // descriptors: the taps differ only by start address (16-byte units in the low
          // field), so every MMA costs two additions; the 27 taps unroll at compile time
          const uint64_t ad0 = smem_desc(smem_u32(sA + sa * a_stage), p.group_pitch, kHX * 16);
#pragma unroll
          for (int tb = 0; tb < 3; ++tb) {
            uint32_t w_base;
            uint32_t sb = 0;
            if (p.resident) {
              w_base = smem_u32(sW) + (static_cast<uint32_t>(kc) * 27 + tb * 9) * tap_bytes;
            } else {
              sb = b_use % kNB;
              if (!wait_spin(&fullB[sb], (b_use / kNB) & 1u, limit)) {
                give_up();
                ok = false;
                break;
              }
              w_base = smem_u32(sW + sb * 9 * tap_bytes);
            }
            const uint64_t bd0 = smem_desc(w_base, static_cast<uint32_t>(p.Co) * 16u, 128u);
#pragma unroll
            for (int tt = 0; tt < 9; ++tt) {
              const int t = tb * 9 + tt;
              const int sg = FLIP ? -1 : 1;
              const int dz = sg * (t / 9 - 1), dy = sg * ((t / 3) % 3 - 1), dx = sg * (t % 3 - 1);
              const uint32_t row = static_cast<uint32_t>((dz + 1) * (kHX * kHY) + (dy + 1) * kHX + (dx + 1));
              const uint64_t bd = bd0 + static_cast<uint64_t>(tt) * (tap_bytes >> 4);
              const uint32_t acc = (kc > 0 || t > 0) ? 1u : 0u;
#pragma unroll
              for (int zz = 0; zz < TZ; ++zz)
                mma_f16(d0 + static_cast<uint32_t>(zz * p.Co), ad0 + row + static_cast<uint32_t>(zz * kHX * kHY),
                        bd, idesc, acc);
            }
            if (!p.resident) {
              mma_commit(&emptyB[sb]);
              ++b_use;
            }
          }
          if (!ok) break;
          mma_commit(&emptyA[sa]);
          ++a_use;
        }
        if (!ok) break;
        mma_commit(&tfull[buf]);
        ++acc_use;
      }
      mma_commit(fin);
    }
  } else {   // ---------------------------------------------------------- epilogue
    const int q = warp & 3;            // tensor-memory lanes 32q .. 32q + 31
    const int row = 32 * q + lane;     // GEMM row within a plane
    const int mx = row & 7, my = row >> 3;
    uint32_t acc_use = 0;
    for (int64_t tile = blockIdx.x; tile < p.tiles && !*abort_flag; tile += gridDim.x) {
      const TileCoord tc = tile_coord(p, tile);
      const uint32_t buf = acc_use & 1u, ku = acc_use >> 1;
      // warp-uniform: the tensor-memory loads below are .sync.aligned
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&tfull[buf], ku & 1u, limit))) {
        if (lane == 0) give_up();
        break;
      }
      __syncwarp();
      fence_after();
      const int x = tc.x0 + mx, y = tc.y0 + my;
      for (int zz = 0; zz < TZ; ++zz) {
        const int z = tc.z0 + zz;
        const bool inside = x < p.W && y < p.H && z < p.D;
        const int64_t v = ((static_cast<int64_t>(tc.n) * p.D + z) * p.H + y) * p.W + x;
        const uint32_t taddr = tmem + buf * (p.tmem_cols >> 1) + static_cast<uint32_t>(zz * p.Co) +
                               (static_cast<uint32_t>(32 * q) << 16);
        for (int c0 = 0; c0 < p.Co; c0 += 16) {
          uint32_t r[16];
          tmem_ld16(taddr + static_cast<uint32_t>(c0), r);
          if (inside) {
            float f[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              float val = __uint_as_float(r[i]) + (p.bias ? __ldg(&p.bias[c0 + i]) : 0.f);
              if (p.act) val = val > 0.f ? val : kLeak * val;
              f[i] = val;
            }
            if (p.y) {
              uint32_t h[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
                h[i] = *reinterpret_cast<const uint32_t*>(&b2);
              }
              uint4* dst = reinterpret_cast<uint4*>(p.y + v * p.Co + c0);
              dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
              dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
            }
            if (p.yf) {
              float4* dst = reinterpret_cast<float4*>(p.yf + v * p.Co + c0);
#pragma unroll
              for (int i = 0; i < 4; ++i) dst[i] = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
            }
          }
        }
      }
      fence_before();
      mbar_arrive(&tempty[buf]);
      ++acc_use;
    }
    (void)acc_cols;
  }

  __syncthreads();
  if (warp == 0) {
    if (!mbar_wait_bounded(fin, 0, limit)) atomicOr(&g_conv_tc_err, 2);
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

// ---------------------------------------------------------------------------------------
// x-folded variant for 16 output channels.  With N = 16 each MMA reads a 4 KB A operand for
// 16 columns of work, and the shared-memory operand reads, not the tensor core, set the
// pace.  Folding the three x taps of a (dz, dy) pair into N gives one N = 48 MMA per pair:
//   P_j[x'] = sum_ci W[dz, dy, j - 1][ci] X[x' + .., ci]   (j = 0, 1, 2 -> columns 16 j .. 16 j + 15)
//   Y[x]    = P_0[x - s] + P_1[x] + P_2[x + s]             (s = 1, or -1 with flip)
// so a tile's GEMM rows are 16 consecutive x positions (no x halo in the A brick) of which
// the 14 inner ones are outputs; the epilogue shifts the outer column blocks by one row with
// warp shuffles (rows are x-major, so x +- 1 is lane +- 1).  A tile is 16 (x) x 8 (y) x TZ (z)
// rows, consecutive tiles 14 apart in x.  The weights are rearranged once per CTA into
// per-(kc, dz, dy) blocks [g][j * 16 + co][8] (B operand: N = 48 rows 16 bytes apart, the
// two 8-channel groups 768 bytes apart) and stay resident.
constexpr int kXR = 16;                 // GEMM rows along x per tile
constexpr int kXO = kXR - 2;            // outputs along x per tile
constexpr int kYT = 8;                  // y rows per tile: kXR x kYT = 128
constexpr int kXN = 48;                 // three x taps x 16 output channels
constexpr uint32_t kFoldBlock = 2u * kXN * 16u;   // one (dz, dy) pair x 16 input channels
constexpr int kFoldMaxNC = 6;           // input-channel steps whose weights stay resident

template <bool FLIP, int TZ>
__global__ void __launch_bounds__(kThreads, 2) k_conv3d_tcx(const __grid_constant__ CUtensorMap xmap,
                                                            const ConvTcParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t a_stage = 2 * p.group_pitch;
  constexpr uint32_t halo_bytes = static_cast<uint32_t>(kXR * (kYT + 2) * (TZ + 2) * 16);
  const int NC = p.Ci / 16;
  const uint32_t w_bytes = static_cast<uint32_t>(NC) * 9u * kFoldBlock;
  const uint32_t S = static_cast<uint32_t>(p.a_stages);
  uint8_t* sA = sm;
  uint8_t* sW = sm + S * a_stage;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sW + w_bytes);
  uint64_t* fullA = bars;          // [4]
  uint64_t* emptyA = bars + 4;     // [4]
  uint64_t* tfull = bars + 8;      // [2]
  uint64_t* tempty = bars + 10;    // [2]
  uint64_t* fin = bars + 12;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 13);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // weights: packed [kc][t][g][16][8] -> [kc][dz, dy][g][j * 16 + co][8], t = 3 (dz, dy) + j
  for (int e = threadIdx.x; e < NC * 9 * 2 * 3 * 16; e += blockDim.x) {
    const int co = e & 15;
    int r = e >> 4;
    const int j = r % 3;
    r /= 3;
    const int g = r & 1;
    r >>= 1;
    const int pr = r % 9, kc = r / 9;
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p.wpk) + ((kc * 27 + pr * 3 + j) * 2 + g) * 16 + co);
    *reinterpret_cast<uint4*>(sW + (kc * 9 + pr) * kFoldBlock + (g * kXN + j * 16 + co) * 16) = v;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) {
      mbar_init(&fullA[i], 1);
      mbar_init(&emptyA[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 128);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t limit = p.wait_limit;

  auto give_up = [&]() {
    atomicOr(&g_conv_tc_err, 1);
    *abort_flag = 1;
  };

  if (warp == 0) {
    if (lane == 0 && !p.debug_stall) {   // ----------------------------- copies
      uint32_t a_use = 0;
      for (int64_t tile = blockIdx.x; tile < p.tiles && !*abort_flag; tile += gridDim.x) {
        const TileCoord tc = tile_coord_x(p, tile);
        for (int kc = 0; kc < NC && !*abort_flag; ++kc) {
          const uint32_t sa = a_use % S, ka = a_use / S;
          if (ka >= 1 && !wait_spin(&emptyA[sa], (ka - 1) & 1u, limit)) {
            give_up();
            break;
          }
          mbar_arrive_expect_tx(&fullA[sa], 2 * halo_bytes);
          for (int g = 0; g < 2; ++g)
            tma_load_5d(smem_u32(sA + sa * a_stage + g * p.group_pitch), &xmap, kc * 16 + g * 8, tc.x0, tc.y0 - 1,
                        tc.z0 - 1, tc.n, &fullA[sa]);
          ++a_use;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // ---------------------------------------------- MMAs
      constexpr uint32_t idesc = instr_desc(kXN);
      bool ok = true;
      uint32_t a_use = 0, acc_use = 0;
      for (int64_t tile = blockIdx.x; tile < p.tiles && !*abort_flag; tile += gridDim.x) {
        const uint32_t buf = acc_use & 1u, ku = acc_use >> 1;
        if (ku >= 1 && !wait_spin(&tempty[buf], (ku - 1) & 1u, limit)) {
          give_up();
          break;
        }
        fence_after();
        const uint32_t d0 = tmem + buf * (p.tmem_cols >> 1);
        for (int kc = 0; kc < NC && ok; ++kc) {
          const uint32_t sa = a_use % S, ka = a_use / S;
          if (!wait_spin(&fullA[sa], ka & 1u, limit)) {
            give_up();
            ok = false;
            break;
          }
          // A: 8-row groups (x) 128 bytes apart; the (dz, dy) pairs differ by start address
          const uint64_t ad0 = smem_desc(smem_u32(sA + sa * a_stage), p.group_pitch, 128u);
          const uint64_t bd0 = smem_desc(smem_u32(sW) + static_cast<uint32_t>(kc) * 9u * kFoldBlock, kXN * 16u, 128u);
#pragma unroll
          for (int pr = 0; pr < 9; ++pr) {
            const int sg = FLIP ? -1 : 1;
            const int dz = sg * (pr / 3 - 1), dy = sg * (pr % 3 - 1);
            const uint32_t row = static_cast<uint32_t>((dz + 1) * (kYT + 2) * kXR + (dy + 1) * kXR);
            const uint64_t bd = bd0 + static_cast<uint64_t>(pr) * (kFoldBlock >> 4);
            const uint32_t acc = (kc > 0 || pr > 0) ? 1u : 0u;
#pragma unroll
            for (int zz = 0; zz < TZ; ++zz)
              mma_f16(d0 + static_cast<uint32_t>(zz * kXN), ad0 + row + static_cast<uint32_t>(zz * (kYT + 2) * kXR),
                      bd, idesc, acc);
          }
          mma_commit(&emptyA[sa]);
          ++a_use;
        }
        if (!ok) break;
        mma_commit(&tfull[buf]);
        ++acc_use;
      }
      mma_commit(fin);
    }
  } else {   // ---------------------------------------------------------- epilogue
    const int q = warp & 3;            // tensor-memory lanes 32q .. 32q + 31
    const int row = 32 * q + lane;     // GEMM row within a plane
    const int mx = row & (kXR - 1), my = row / kXR;
    float bias[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) bias[i] = p.bias ? __ldg(&p.bias[i]) : 0.f;
    uint32_t acc_use = 0;
    for (int64_t tile = blockIdx.x; tile < p.tiles && !*abort_flag; tile += gridDim.x) {
      const TileCoord tc = tile_coord_x(p, tile);
      const uint32_t buf = acc_use & 1u, ku = acc_use >> 1;
      // warp-uniform: the tensor-memory loads and shuffles below are .sync.aligned
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&tfull[buf], ku & 1u, limit))) {
        if (lane == 0) give_up();
        break;
      }
      __syncwarp();
      fence_after();
      const int x = tc.x0 + mx, y = tc.y0 + my;
      for (int zz = 0; zz < TZ; ++zz) {
        const int z = tc.z0 + zz;
        const bool inside = mx >= 1 && mx <= kXO && x < p.W && y < p.H && z < p.D;
        const int64_t v = ((static_cast<int64_t>(tc.n) * p.D + z) * p.H + y) * p.W + x;
        const uint32_t taddr = tmem + buf * (p.tmem_cols >> 1) + static_cast<uint32_t>(zz * kXN) +
                               (static_cast<uint32_t>(32 * q) << 16);
        uint32_t r0[16], r1[16], r2[16];
        tmem_ld16x3(taddr, r0, r1, r2);
        float f[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          // column block 0 comes from row x - s, block 2 from row x + s (16-lane segments = one y row)
          const float a = FLIP ? __shfl_down_sync(0xffffffffu, __uint_as_float(r0[i]), 1, 16)
                               : __shfl_up_sync(0xffffffffu, __uint_as_float(r0[i]), 1, 16);
          const float b = FLIP ? __shfl_up_sync(0xffffffffu, __uint_as_float(r2[i]), 1, 16)
                               : __shfl_down_sync(0xffffffffu, __uint_as_float(r2[i]), 1, 16);
          float val = (__uint_as_float(r1[i]) + a) + b + bias[i];
          if (p.act) val = val > 0.f ? val : kLeak * val;
          f[i] = val;
        }
        if (inside) {
          if (p.y) {
            uint32_t h[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
              h[i] = *reinterpret_cast<const uint32_t*>(&b2);
            }
            uint4* dst = reinterpret_cast<uint4*>(p.y + v * 16);
            dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
            dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
          }
          if (p.yf) {
            float4* dst = reinterpret_cast<float4*>(p.yf + v * 16);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
          }
        }
      }
      fence_before();
      mbar_arrive(&tempty[buf]);
      ++acc_use;
    }
  }

  __syncthreads();
  if (warp == 0) {
    if (!mbar_wait_bounded(fin, 0, limit)) atomicOr(&g_conv_tc_err, 2);
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

// bfloat16 weights in the tensor-core layout of both directions:
//   forward  wpk [Ci/16][27][2][Co][8]:  (kc, t, g, co, j) = W[t][16kc + 8g + j][co]
//   flipped  wpkt[Co/16][27][2][Ci][8]:  (kc, t, g, ci, j) = W[t][ci][16kc + 8g + j]
__global__ void k_pack_weights(const float* __restrict__ w, bf16* __restrict__ wpk, bf16* __restrict__ wpkt, int Ci,
                               int Co) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n = 27LL * Ci * Co;
  if (i >= n) return;
  const int co = static_cast<int>(i % Co);
  const int64_t r = i / Co;
  const int ci = static_cast<int>(r % Ci);
  const int t = static_cast<int>(r / Ci);
  const bf16 q = __float2bfloat16_rn(w[i]);
  if (wpk) {
    const int kc = ci / 16, g = (ci / 8) & 1, j = ci & 7;
    wpk[((((static_cast<int64_t>(kc) * 27 + t) * 2 + g) * Co + co) * 8) + j] = q;
  }
  if (wpkt) {
    const int kc = co / 16, g = (co / 8) & 1, j = co & 7;
    wpkt[((((static_cast<int64_t>(kc) * 27 + t) * 2 + g) * Ci + ci) * 8) + j] = q;
  }
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

struct TcShape {
  int tz, resident, a_stages;
  uint32_t group_pitch, w_bytes, tmem_cols;
  size_t smem;
};

TcShape shape_for(int ci, int co, int tz) {
  TcShape t{};
  t.tz = tz;
  const uint32_t halo = static_cast<uint32_t>(kHX * kHY * (tz + 2) * 16);
  t.group_pitch = (halo + 127u) & ~127u;              // TMA destinations are 128-byte aligned
  const uint32_t tap = 32u * static_cast<uint32_t>(co);
  const uint32_t all = 27u * static_cast<uint32_t>(ci / 16) * tap;
  t.resident = all <= kResidentMax ? 1 : 0;
  t.w_bytes = t.resident ? all : kNB * 9u * tap;
  uint32_t c = 32;
  while (c < 2u * static_cast<uint32_t>(tz * co)) c <<= 1;
  t.tmem_cols = c;
  t.smem = 1024 + 4 * static_cast<size_t>(t.group_pitch) + t.w_bytes + 8 * 13 + 16;
  return t;
}

// z planes per tile: more planes share one halo load and its waits, as long as two CTAs
// still fit an SM (shared memory) and tz planes x two buffers of co columns fit the 512
// tensor-memory columns
TcShape tc_shape(int ci, int co) {
  if (co <= 32) {
    const TcShape t4 = shape_for(ci, co, 4);
    if (t4.smem <= 110 * 1024) return t4;
  }
  return shape_for(ci, co, co <= 128 ? 2 : 1);
}

// x-folded kernel (16 output channels): A bricks of 16 x 10 x (tz + 2) voxels, all weights
// resident as nc x 9 blocks of 1536 bytes, tz planes x 48 columns x two accumulator buffers
TcShape shape_fold(int ci, int tz) {
  TcShape t{};
  t.tz = tz;
  const uint32_t halo = static_cast<uint32_t>(kXR * (kYT + 2) * (tz + 2) * 16);
  t.group_pitch = (halo + 127u) & ~127u;
  t.resident = 1;
  t.w_bytes = static_cast<uint32_t>(ci / 16) * 9u * kFoldBlock;
  uint32_t c = 32;
  while (c < 2u * static_cast<uint32_t>(tz * kXN)) c <<= 1;
  t.tmem_cols = c;
  // as many halo stages (up to 4) as keep the CTAs that tensor memory allows on one SM
  const size_t budget = c >= 512 ? 220 * 1024 : 110 * 1024;
  for (t.a_stages = 4; t.a_stages > 2; --t.a_stages)
    if (1024 + 2 * t.a_stages * static_cast<size_t>(t.group_pitch) + t.w_bytes + 8 * 13 + 16 <= budget) break;
  if (g_fold_stages >= 2 && g_fold_stages < t.a_stages) t.a_stages = g_fold_stages;
  t.smem = 1024 + 2 * t.a_stages * static_cast<size_t>(t.group_pitch) + t.w_bytes + 8 * 13 + 16;
  return t;
}

bool use_fold(int ci, int co) { return g_conv_fold && co == 16 && ci / 16 <= kFoldMaxNC; }

}  // namespace

// Per-kernel launch set-up, done once per (device, instantiation) and cached, so that a
// launch makes no runtime calls besides the launch itself (and can be captured in a CUDA
// graph): the dynamic shared-memory limit and carve-out, and the resident CTAs per SM from
// shared memory (1 KB reserved per CTA), registers (allocated per warp in units of 256) and
// tensor memory (512 columns per SM; a CTA beyond that would wait in allocation).
cudaError_t kernel_setup(const void* kern, size_t smem, uint32_t tmem_cols, int* per_sm, int* sms) {
  struct Entry {
    size_t smem_set;
    int regs;
  };
  struct Dev {
    int sms, smem_sm, regs_sm;
  };
  static std::mutex mu;
  static std::unordered_map<const void*, Entry> kernels[64];
  static Dev devs[64];
  static bool dev_known[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!dev_known[dev]) {
    Dev d{};
    if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&d.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
      return e;
    if ((e = cudaDeviceGetAttribute(&d.regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess)
      return e;
    devs[dev] = d;
    dev_known[dev] = true;
  }
  auto it = kernels[dev].find(kern);
  if (it == kernels[dev].end()) {
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
    it = kernels[dev].emplace(kern, Entry{0, fa.numRegs}).first;
  }
  if (it->second.smem_set < smem) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem))) !=
        cudaSuccess)
      return e;
    it->second.smem_set = smem;
  }
  const Dev& d = devs[dev];
  const int by_smem = d.smem_sm / static_cast<int>(smem + 1024);
  const int regs_warp = ((it->second.regs * 32 + 255) / 256) * 256;
  const int by_regs = d.regs_sm / (regs_warp * (kThreads / 32));
  const int by_tmem = static_cast<int>(512 / tmem_cols);
  int n = by_smem < by_regs ? by_smem : by_regs;
  n = n < by_tmem ? n : by_tmem;
  *per_sm = n < 1 ? 1 : n;
  *sms = d.sms;
  return cudaSuccess;
}

bool conv_tc_supported(int ci, int co) { return ci >= 16 && ci % 16 == 0 && co >= 16 && co % 16 == 0 && co <= 256; }

cudaError_t launch_conv_tc(const void* x, const void* wpk, const float* bias, void* y, float* yf, int n, int d,
                           int h, int w, int ci, int co, int flip, int act, cudaStream_t s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[5] = {static_cast<cuuint64_t>(ci), static_cast<cuuint64_t>(w), static_cast<cuuint64_t>(h),
                              static_cast<cuuint64_t>(d), static_cast<cuuint64_t>(n)};
  const cuuint64_t row = 2ull * ci;
  const cuuint64_t strides[4] = {row, row * w, row * w * h, row * w * h * d};
  const bool fold = use_fold(ci, co);
  const int ftz = g_fold_tz == 1 || g_fold_tz == 2 ? g_fold_tz : 4;
  const TcShape shp = fold ? shape_fold(ci, ftz) : tc_shape(ci, co);
  const cuuint32_t box[5] = {8, static_cast<cuuint32_t>(fold ? kXR : kHX), static_cast<cuuint32_t>(fold ? kYT + 2 : kHY),
                             static_cast<cuuint32_t>(shp.tz + 2), 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  ConvTcParams p{};
  p.wpk = static_cast<const bf16*>(wpk);
  p.bias = bias;
  p.y = static_cast<bf16*>(y);
  p.yf = yf;
  p.N = n;
  p.D = d;
  p.H = h;
  p.W = w;
  p.Ci = ci;
  p.Co = co;
  p.flip = flip;
  p.act = act;
  p.tz = shp.tz;
  p.resident = shp.resident;
  p.tiles_x = fold ? (w + kXO - 1) / kXO : (w + kTX - 1) / kTX;
  p.tiles_y = fold ? (h + kYT - 1) / kYT : (h + kTY - 1) / kTY;
  p.tiles_z = (d + shp.tz - 1) / shp.tz;
  p.tiles = static_cast<int64_t>(p.tiles_x) * p.tiles_y * p.tiles_z * n;
  p.group_pitch = shp.group_pitch;
  p.a_stages = fold ? shp.a_stages : 2;
  p.tmem_cols = shp.tmem_cols;
  p.wait_limit = g_wait_limit ? g_wait_limit : kDefaultWait;
  p.debug_stall = g_debug_stall;
  const size_t smem = shp.smem;
  auto kern = fold ? (flip ? (shp.tz == 4 ? k_conv3d_tcx<true, 4> : shp.tz == 2 ? k_conv3d_tcx<true, 2>
                                                                      : k_conv3d_tcx<true, 1>)
                            : (shp.tz == 4 ? k_conv3d_tcx<false, 4> : shp.tz == 2 ? k_conv3d_tcx<false, 2>
                                                                        : k_conv3d_tcx<false, 1>))
                   : flip ? (shp.tz == 4 ? k_conv3d_tc<true, 4> : shp.tz == 2 ? k_conv3d_tc<true, 2>
                                                                     : k_conv3d_tc<true, 1>)
                          : (shp.tz == 4 ? k_conv3d_tc<false, 4>
                                         : shp.tz == 2 ? k_conv3d_tc<false, 2> : k_conv3d_tc<false, 1>);
  int per_sm = 0, sms = 0;
  const cudaError_t e = kernel_setup(reinterpret_cast<const void*>(kern), smem, p.tmem_cols, &per_sm, &sms);
  if (e != cudaSuccess) return e;
  const int64_t grid = p.tiles < static_cast<int64_t>(sms) * per_sm ? p.tiles : static_cast<int64_t>(sms) * per_sm;
  kern<<<static_cast<unsigned>(grid), kThreads, smem, s>>>(map, p);
  return cudaGetLastError();
}

cudaError_t launch_pack_weights(const float* w, void* wpk, void* wpkt, int ci, int co, cudaStream_t s) {
  const int64_t n = 27LL * ci * co;
  k_pack_weights<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(w, static_cast<bf16*>(wpk),
                                                                         static_cast<bf16*>(wpkt), ci, co);
  return cudaGetLastError();
}

}  // namespace mach_nn

using namespace mach_nn;

extern "C" {

mach_status mach_nn_pack_weights(const float* w, void* wpk, void* wpk_flip, int32_t ci, int32_t co, void* stream) {
  if (!w || (!wpk && !wpk_flip) || ci < 16 || ci % 16 || co < 16 || co % 16) return MACH_ERR_INVALID_ARG;
  return launch_pack_weights(w, wpk, wpk_flip, ci, co, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? MACH_OK
             : MACH_ERR_CUDA;
}

mach_status mach_nn_conv3d_tc(const void* x, const void* wpk, const float* bias, void* y, float* y_f32, int32_t n,
                              int32_t nz, int32_t ny, int32_t nx, int32_t ci, int32_t co, int32_t flip, int32_t act,
                              void* stream) {
  if (!x || !wpk || (!y && !y_f32) || n < 1 || nz < 1 || ny < 1 || nx < 1) return MACH_ERR_INVALID_ARG;
  if (!conv_tc_supported(ci, co)) return MACH_ERR_INVALID_ARG;
  const uintptr_t al = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(wpk) |
                       reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(y_f32);
  if (al & 15u) return MACH_ERR_INVALID_ARG;
  if (n > 65535 || static_cast<int64_t>(nz) * ny * nx * n > (1LL << 40)) return MACH_ERR_UNSUPPORTED;
  const cudaError_t e = launch_conv_tc(x, wpk, bias, y, y_f32, n, nz, ny, nx, ci, co, flip, act,
                                       static_cast<cudaStream_t>(stream));
  if (e == cudaErrorNotSupported || e == cudaErrorInvalidValue) {
    cudaGetLastError();
    return MACH_ERR_UNSUPPORTED;
  }
  return e == cudaSuccess ? MACH_OK : MACH_ERR_CUDA;
}

void mach_nn_debug_conv(int32_t stall_copies, uint32_t wait_limit) {
  g_debug_stall = stall_copies ? 1 : 0;
  g_wait_limit = wait_limit;
}

void mach_nn_set_conv_fold(int32_t enable, int32_t z_planes, int32_t halo_stages) {
  g_conv_fold = enable ? 1 : 0;
  g_fold_tz = z_planes == 1 || z_planes == 2 ? z_planes : 4;
  g_fold_stages = halo_stages >= 2 && halo_stages <= 4 ? halo_stages : 0;
}

mach_status mach_nn_device_status(void* stream) {
  int err = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MACH_ERR_CUDA;
  if (cudaMemcpyFromSymbol(&err, g_conv_tc_err, sizeof(int)) != cudaSuccess) return MACH_ERR_CUDA;
  if (err) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_conv_tc_err, &zero, sizeof(int)) != cudaSuccess) return MACH_ERR_CUDA;
    return MACH_ERR_TIMEOUT;
  }
  return MACH_OK;
}

}  // extern "C"
