// k_nn.cu -- kernels of the learned compounding network (a small 3D U-Net).
//
// Activations are channels-last bfloat16 tensors [N][D][H][W][C] with C a multiple of 16;
// weights are bfloat16 [27][Cin][Cout] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)).  Products
// run on the tensor cores (mma.sync m16n8k16, bfloat16 in, float32 accumulate).
//
//  * k_conv3d: 3x3x3 "same" convolution as an implicit GEMM (M = voxels, N = Cout,
//    K = 27 * Cin), 64 voxels x BN output channels per block, K staged 16 channels of one
//    tap at a time through a double-buffered cp.async pipeline; bias, leaky ReLU and the
//    output conversion are fused into the epilogue.  With `flip` the taps are mirrored,
//    which turns it into the data gradient (given the transposed weights [27][Cout][Cin]).
//  * k_conv3d_wgrad: weight gradient dW[t][ci][co] = sum_v X[v + off(t)][ci] dY[v][co]:
//    per block all 27 taps of one (16 input, CT output channel) block over a run of voxel
//    tiles, halo and gradient tiles staged once per tile, partial sums added with float32
//    atomics.
//  * elementwise kernels: leaky-ReLU backward, 2x average pooling and nearest upsampling
//    (and their adjoints), channel-slice copies (concatenation), bias gradient, Adam,
//    and the network boundary (RMS normalisation / packing, loss, output).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "mach_nn.h"
#include "nn_internal.h"

namespace mach_nn {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros (padding).
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
// D += A (16 x 16, row major) * B (16 x 8, column major); bfloat16 in, float32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct Vox {
  int n, z, y, x;
};
__device__ __forceinline__ Vox vox_of(int64_t v, int D, int H, int W) {
  Vox r;
  r.x = static_cast<int>(v % W);
  int64_t q = v / W;
  r.y = static_cast<int>(q % H);
  q /= H;
  r.z = static_cast<int>(q % D);
  r.n = static_cast<int>(q / D);
  return r;
}
__device__ __forceinline__ void tap_offset(int t, int& dz, int& dy, int& dx) {
  dz = t / 9 - 1;
  dy = (t / 3) % 3 - 1;
  dx = t % 3 - 1;
}

// ---------------------------------------------------------------- convolution ----
constexpr int kBM = 64;   // voxels per block
constexpr int kBK = 16;   // input channels per K step

template <int BN>
__global__ void __launch_bounds__(128) k_conv3d(const bf16* __restrict__ X, const bf16* __restrict__ Wt,
                                                const float* __restrict__ bias, bf16* __restrict__ Y,
                                                float* __restrict__ Yf, int N, int D, int H, int W, int Ci, int Co,
                                                int flip, int act) {
  __shared__ __align__(128) bf16 sA[2][kBM][kBK + 8];
  __shared__ __align__(128) bf16 sB[2][kBK][BN + 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t M = static_cast<int64_t>(N) * D * H * W;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * kBM;
  const int n0 = blockIdx.y * BN;

  // the A row (voxel) and 16-byte half this thread copies
  const int ar = tid >> 1, ac = tid & 1;
  const int64_t av = m0 + ar;
  const bool a_in = av < M;
  const Vox a = vox_of(a_in ? av : 0, D, H, W);
  const int cblocks = Ci / kBK;
  const int ksteps = 27 * cblocks;

  auto load = [&](int stage, int ks) {
    const int t = ks / cblocks, cb = ks % cblocks;
    int dz, dy, dx;
    tap_offset(t, dz, dy, dx);
    if (flip) {
      dz = -dz;
      dy = -dy;
      dx = -dx;
    }
    const int z = a.z + dz, y = a.y + dy, x = a.x + dx;
    const bool ok = a_in && z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W;
    const bf16* src = ok ? X + ((((static_cast<int64_t>(a.n) * D + z) * H + y) * W + x) * Ci + cb * kBK + ac * 8) : X;
    cp16(&sA[stage][ar][ac * 8], src, ok ? 16 : 0);
    const bf16* wsrc = Wt + (static_cast<int64_t>(t) * Ci + cb * kBK) * Co + n0;
    for (int c = tid; c < kBK * BN / 8; c += 128) {
      const int r = c / (BN / 8), cc = c % (BN / 8);
      cp16(&sB[stage][r][cc * 8], wsrc + static_cast<int64_t>(r) * Co + cc * 8, 16);
    }
    cp_commit();
  };

  float acc[BN / 8][4];
#pragma unroll
  for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

  load(0, 0);
  for (int ks = 0; ks < ksteps; ++ks) {
    const int st = ks & 1;
    if (ks + 1 < ksteps) {
      load(st ^ 1, ks + 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    uint32_t af[4];
    ldm_x4(af, &sA[st][warp * 16 + (lane & 15)][(lane >> 4) * 8]);
#pragma unroll
    for (int j = 0; j < BN / 16; ++j) {
      uint32_t bfr[4];
      ldm_x4_t(bfr, &sB[st][lane & 15][j * 16 + (lane >> 4) * 8]);
      mma_bf16(acc[2 * j], af, bfr[0], bfr[1]);
      mma_bf16(acc[2 * j + 1], af, bfr[2], bfr[3]);
    }
    __syncthreads();
  }

  // accumulator (j, h): row 16*warp + lane/4 + 8h, columns n0 + 8j + 2*(lane%4) + {0, 1}
#pragma unroll
  for (int j = 0; j < BN / 8; ++j) {
    const int col = n0 + 8 * j + 2 * (lane & 3);
    const float b0 = bias ? bias[col] : 0.f, b1 = bias ? bias[col + 1] : 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t row = m0 + warp * 16 + (lane >> 2) + 8 * h;
      if (row >= M) continue;
      float v0 = acc[j][2 * h] + b0, v1 = acc[j][2 * h + 1] + b1;
      if (act) {
        v0 = v0 > 0.f ? v0 : kLeak * v0;
        v1 = v1 > 0.f ? v1 : kLeak * v1;
      }
      if (Y) *reinterpret_cast<__nv_bfloat162*>(Y + row * Co + col) = __floats2bfloat162_rn(v0, v1);
      if (Yf) *reinterpret_cast<float2*>(Yf + row * Co + col) = make_float2(v0, v1);
    }
  }
}

// Weight gradient, all 27 taps per block.  A block owns one 16-channel input block, one
// CT-channel output block and a run of 8 x 16 x 1 voxel tiles.  Per tile it stages the
// input halo brick (10 x 18 x 3 voxels x 16 channels, zero outside the volume) and the
// output-gradient tile (128 voxels x CT channels, zero outside) in shared memory once,
// and every warp accumulates its taps (warp w: taps w, w + 8, w + 16, w + 24) as
// mma.sync products X_t^T (16 x 16 voxels) x dY (16 voxels x CT) over the tile's voxels.
// Partial sums are added to dW with float32 atomics at the end.
constexpr int kWTaps = 4;              // taps per warp (8 warps cover 27)
constexpr int kHRows = 10 * 18 * 3;    // halo rows of one 8-channel group

template <int CT>
__global__ void __launch_bounds__(256) k_conv3d_wgrad(const bf16* __restrict__ X, const bf16* __restrict__ dY,
                                                      float* __restrict__ dW, int N, int D, int H, int W, int Ci,
                                                      int Co, int64_t tiles, int tiles_x, int tiles_y,
                                                      int64_t tiles_per_block) {
  constexpr int kHaloB = 2 * kHRows * 16;
  constexpr int kGB = (CT / 8) * 128 * 16;
  constexpr int kStage = kHaloB + kGB;
  extern __shared__ __align__(128) uint8_t wsm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cb = blockIdx.y, ob = blockIdx.z;
  const int64_t t_begin = static_cast<int64_t>(blockIdx.x) * tiles_per_block;
  const int64_t t_end = t_begin + tiles_per_block < tiles ? t_begin + tiles_per_block : tiles;

  auto load = [&](int stage, int64_t tile) {
    const int tx = static_cast<int>(tile % tiles_x);
    int64_t r0 = tile / tiles_x;
    const int ty = static_cast<int>(r0 % tiles_y);
    r0 /= tiles_y;
    const int z = static_cast<int>(r0 % D), n = static_cast<int>(r0 / D);
    const int x0 = tx * 8, y0 = ty * 16;
    uint8_t* base = wsm + stage * kStage;
    for (int c = tid; c < 2 * kHRows + (CT / 8) * 128; c += 256) {
      if (c < 2 * kHRows) {
        const int g = c / kHRows, r = c % kHRows;
        const int hz = r / 180, hr = r % 180, hy = hr / 10, hx = hr % 10;
        const int x = x0 - 1 + hx, y = y0 - 1 + hy, zz = z - 1 + hz;
        const bool in = x >= 0 && x < W && y >= 0 && y < H && zz >= 0 && zz < D;
        const bf16* src = in ? X + ((((static_cast<int64_t>(n) * D + zz) * H + y) * W + x) * Ci + cb * 16 + g * 8) : X;
        cp16(base + (g * kHRows + r) * 16, src, in ? 16 : 0);
      } else {
        const int c2 = c - 2 * kHRows;
        const int cg = c2 / 128, k = c2 % 128;
        const int x = x0 + (k & 7), y = y0 + (k >> 3);
        const bool in = x < W && y < H;
        const bf16* src = in ? dY + ((((static_cast<int64_t>(n) * D + z) * H + y) * W + x) * Co + ob * CT + cg * 8) : dY;
        cp16(base + kHaloB + (cg * 128 + k) * 16, src, in ? 16 : 0);
      }
    }
    cp_commit();
  };

  float acc[kWTaps][CT / 8][4];
#pragma unroll
  for (int i = 0; i < kWTaps; ++i)
#pragma unroll
    for (int j = 0; j < CT / 8; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;

  if (t_begin < t_end) load(0, t_begin);
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int st = static_cast<int>((tile - t_begin) & 1);
    if (tile + 1 < t_end) {
      load(st ^ 1, tile + 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const uint8_t* base = wsm + st * kStage;
    const uint8_t* halo = base;
    const uint8_t* gt = base + kHaloB;
#pragma unroll 2
    for (int ks = 0; ks < 8; ++ks) {   // 16 voxels (two x-rows of the tile) per K step
      uint32_t bfr[CT / 16][4];
#pragma unroll
      for (int j = 0; j < CT / 16; ++j)
        ldm_x4_t(bfr[j], gt + ((2 * j + (lane >> 4)) * 128 + ks * 16 + (lane & 15)) * 16);
      const int mat = lane >> 3;
      const int kv = ks * 16 + (mat >> 1) * 8 + (lane & 7);   // voxel of this lane's row address
      const int mx = kv & 7, my = kv >> 3;
#pragma unroll
      for (int i = 0; i < kWTaps; ++i) {
        const int t = warp + 8 * i;
        if (t < 27) {   // warp-uniform
          int dz, dy, dx;
          tap_offset(t, dz, dy, dx);
          const int row = (dz + 1) * 180 + (my + dy + 1) * 10 + (mx + dx + 1);
          uint32_t af[4];
          ldm_x4_t(af, halo + ((mat & 1) * kHRows + row) * 16);
#pragma unroll
          for (int j = 0; j < CT / 16; ++j) {
            mma_bf16(acc[i][2 * j], af, bfr[j][0], bfr[j][1]);
            mma_bf16(acc[i][2 * j + 1], af, bfr[j][2], bfr[j][3]);
          }
        }
      }
    }
    __syncthreads();
  }
  if (t_begin >= t_end) return;
#pragma unroll
  for (int i = 0; i < kWTaps; ++i) {
    const int t = warp + 8 * i;
    if (t >= 27) continue;
#pragma unroll
    for (int j = 0; j < CT / 8; ++j) {
      const int co = ob * CT + 8 * j + 2 * (lane & 3);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ci = cb * 16 + (lane >> 2) + 8 * h;
        float* dst = dW + (static_cast<int64_t>(t) * Ci + ci) * Co + co;
        atomicAdd(dst, acc[i][j][2 * h]);
        atomicAdd(dst + 1, acc[i][j][2 * h + 1]);
      }
    }
  }
}

// ---------------------------------------------------------------- elementwise ----
__global__ void k_lrelu_bwd(bf16* __restrict__ g, const bf16* __restrict__ y, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!(__bfloat162float(y[i]) > 0.f)) g[i] = __float2bfloat16_rn(__bfloat162float(g[i]) * kLeak);
}

// the same, 8 elements (16 bytes) per thread
__global__ void k_lrelu_bwd8(uint4* __restrict__ g, const uint4* __restrict__ y, int64_t n8) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n8) return;
  uint4 gv = g[i];
  const uint4 yv = y[i];
  uint32_t* gw = reinterpret_cast<uint32_t*>(&gv);
  const uint32_t* yw = reinterpret_cast<const uint32_t*>(&yv);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat162 g2 = *reinterpret_cast<const __nv_bfloat162*>(&gw[k]);
    const __nv_bfloat162 y2 = *reinterpret_cast<const __nv_bfloat162*>(&yw[k]);
    const float2 gf = __bfloat1622float2(g2), yf = __bfloat1622float2(y2);
    g2 = __floats2bfloat162_rn(yf.x > 0.f ? gf.x : gf.x * kLeak, yf.y > 0.f ? gf.y : gf.y * kLeak);
    gw[k] = *reinterpret_cast<const uint32_t*>(&g2);
  }
  g[i] = gv;
}

// 2x average pooling [N][D][H][W][C] -> [N][D/2][H/2][W/2][C]
__global__ void k_pool2(const bf16* __restrict__ x, bf16* __restrict__ y, int N, int D, int H, int W, int C) {
  const int d = D / 2, h = H / 2, w = W / 2;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = static_cast<int64_t>(N) * d * h * w * C;
  if (i >= total) return;
  const int c = static_cast<int>(i % C);
  const Vox p = vox_of(i / C, d, h, w);
  float s = 0.f;
  for (int k = 0; k < 8; ++k) {
    const int z = 2 * p.z + (k >> 2), yy = 2 * p.y + ((k >> 1) & 1), xx = 2 * p.x + (k & 1);
    s += __bfloat162float(x[((((static_cast<int64_t>(p.n) * D + z) * H + yy) * W + xx) * C) + c]);
  }
  y[i] = __float2bfloat16_rn(0.125f * s);
}

// adjoint of k_pool2: every child receives dy / 8 (added to dx when accumulating)
__global__ void k_pool2_bwd(const bf16* __restrict__ dy, bf16* __restrict__ dx, int N, int D, int H, int W, int C,
                            int accumulate) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = static_cast<int64_t>(N) * D * H * W * C;
  if (i >= total) return;
  const int c = static_cast<int>(i % C);
  const Vox p = vox_of(i / C, D, H, W);
  const int d = D / 2, h = H / 2, w = W / 2;
  float v = 0.125f * __bfloat162float(dy[((((static_cast<int64_t>(p.n) * d + p.z / 2) * h + p.y / 2) * w + p.x / 2) * C) + c]);
  if (accumulate) v += __bfloat162float(dx[i]);
  dx[i] = __float2bfloat16_rn(v);
}

// nearest 2x upsampling of x [N][d][h][w][C] into channels [off, off + C) of y [N][2d][2h][2w][Cy]
__global__ void k_up2(const bf16* __restrict__ x, bf16* __restrict__ y, int N, int d, int h, int w, int C, int Cy,
                      int off) {
  const int D = 2 * d, H = 2 * h, W = 2 * w;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = static_cast<int64_t>(N) * D * H * W * C;
  if (i >= total) return;
  const int c = static_cast<int>(i % C);
  const int64_t v = i / C;
  const Vox p = vox_of(v, D, H, W);
  y[v * Cy + off + c] = x[((((static_cast<int64_t>(p.n) * d + p.z / 2) * h + p.y / 2) * w + p.x / 2) * C) + c];
}

// adjoint of k_up2: dx = sum over the 8 children of channels [off, off + C) of dy
__global__ void k_up2_bwd(const bf16* __restrict__ dy, bf16* __restrict__ dx, int N, int d, int h, int w, int C,
                          int Cy, int off) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = static_cast<int64_t>(N) * d * h * w * C;
  if (i >= total) return;
  const int c = static_cast<int>(i % C);
  const Vox p = vox_of(i / C, d, h, w);
  const int D = 2 * d, H = 2 * h, W = 2 * w;
  float s = 0.f;
  for (int k = 0; k < 8; ++k) {
    const int z = 2 * p.z + (k >> 2), yy = 2 * p.y + ((k >> 1) & 1), xx = 2 * p.x + (k & 1);
    s += __bfloat162float(dy[((((static_cast<int64_t>(p.n) * D + z) * H + yy) * W + xx) * Cy) + off + c]);
  }
  dx[i] = __float2bfloat16_rn(s);
}

// 16-byte (8-channel) versions of the data-movement kernels, used when every channel
// count and offset is a multiple of 8 (always the case for the network's tensors).
__device__ __forceinline__ void add8(float (&a)[8], uint4 v) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = __bfloat1622float2(h[k]);
    a[2 * k] += f.x;
    a[2 * k + 1] += f.y;
  }
}
__device__ __forceinline__ uint4 pack8(const float (&a)[8], float scale) {
  uint4 v;
  uint32_t* w = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(a[2 * k] * scale, a[2 * k + 1] * scale);
    w[k] = *reinterpret_cast<const uint32_t*>(&b);
  }
  return v;
}

__global__ void k_pool2_v(const uint4* __restrict__ x, uint4* __restrict__ y, int N, int D, int H, int W, int C8) {
  const int d = D / 2, h = H / 2, w = W / 2;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(N) * d * h * w * C8) return;
  const int c = static_cast<int>(i % C8);
  const Vox p = vox_of(i / C8, d, h, w);
  float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < 8; ++k) {
    const int z = 2 * p.z + (k >> 2), yy = 2 * p.y + ((k >> 1) & 1), xx = 2 * p.x + (k & 1);
    add8(a, x[((((static_cast<int64_t>(p.n) * D + z) * H + yy) * W + xx) * C8) + c]);
  }
  y[i] = pack8(a, 0.125f);
}

__global__ void k_pool2_bwd_v(const uint4* __restrict__ dy, uint4* __restrict__ dx, int N, int D, int H, int W, int C8,
                              int accumulate) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(N) * D * H * W * C8) return;
  const int c = static_cast<int>(i % C8);
  const Vox p = vox_of(i / C8, D, H, W);
  const int d = D / 2, h = H / 2, w = W / 2;
  float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  add8(a, dy[((((static_cast<int64_t>(p.n) * d + p.z / 2) * h + p.y / 2) * w + p.x / 2) * C8) + c]);
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] *= 0.125f;
  if (accumulate) add8(a, dx[i]);
  dx[i] = pack8(a, 1.f);
}

__global__ void k_up2_v(const uint4* __restrict__ x, uint4* __restrict__ y, int N, int d, int h, int w, int C8, int Cy8,
                        int off8) {
  const int D = 2 * d, H = 2 * h, W = 2 * w;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(N) * D * H * W * C8) return;
  const int c = static_cast<int>(i % C8);
  const int64_t v = i / C8;
  const Vox p = vox_of(v, D, H, W);
  y[v * Cy8 + off8 + c] = x[((((static_cast<int64_t>(p.n) * d + p.z / 2) * h + p.y / 2) * w + p.x / 2) * C8) + c];
}

__global__ void k_up2_bwd_v(const uint4* __restrict__ dy, uint4* __restrict__ dx, int N, int d, int h, int w, int C8,
                            int Cy8, int off8) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(N) * d * h * w * C8) return;
  const int c = static_cast<int>(i % C8);
  const Vox p = vox_of(i / C8, d, h, w);
  const int D = 2 * d, H = 2 * h, W = 2 * w;
  float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < 8; ++k) {
    const int z = 2 * p.z + (k >> 2), yy = 2 * p.y + ((k >> 1) & 1), xx = 2 * p.x + (k & 1);
    add8(a, dy[((((static_cast<int64_t>(p.n) * D + z) * H + yy) * W + xx) * Cy8) + off8 + c]);
  }
  dx[i] = pack8(a, 1.f);
}

__global__ void k_copy_channels_v(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t voxels, int C8,
                                  int Cy8, int off8, int back) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= voxels * C8) return;
  const int64_t v = i / C8;
  const int c = static_cast<int>(i % C8);
  if (back)
    dst[i] = src[v * Cy8 + off8 + c];
  else
    dst[v * Cy8 + off8 + c] = src[i];
}

__global__ void k_copy_channels(const bf16* __restrict__ src, bf16* __restrict__ dst, int64_t voxels, int C, int Cy,
                                int off, int back) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= voxels * C) return;
  const int64_t v = i / C;
  const int c = static_cast<int>(i % C);
  if (back)
    dst[i] = src[v * Cy + off + c];
  else
    dst[v * Cy + off + c] = src[i];
}

// db[c] += sum_v g[v][c].  Thread t owns channel t % C of rows t / C (+ stride), so a
// warp reads consecutive bytes; per-block sums meet in shared memory.
__global__ void k_bias_grad(const bf16* __restrict__ g, float* __restrict__ db, int64_t voxels, int C) {
  __shared__ float part[256];
  const int tid = threadIdx.x;
  const int rows = blockDim.x / C;
  const int c = tid % C, r = tid / C;
  float s = 0.f;
  for (int64_t v = static_cast<int64_t>(blockIdx.x) * rows + r; v < voxels; v += static_cast<int64_t>(gridDim.x) * rows)
    s += __bfloat162float(g[v * C + c]);
  if (tid < C) part[tid] = 0.f;
  __syncthreads();
  atomicAdd(&part[c], s);
  __syncthreads();
  if (tid < C) atomicAdd(&db[tid], part[tid]);
}

// Adam (float32 master weights); optional bfloat16 copies (same layout, and transposed
// [27][Co][Ci] for the data gradient).
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ gr,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                       bf16* __restrict__ wb, bf16* __restrict__ wbt, int Ci, int Co) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gr[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wb) {
    const bf16 q = __float2bfloat16_rn(wi);
    wb[i] = q;
    if (wbt) {
      const int64_t per_tap = static_cast<int64_t>(Ci) * Co;
      const int64_t t = i / per_tap, r = i % per_tap;
      const int ci = static_cast<int>(r / Co), co = static_cast<int>(r % Co);
      wbt[t * per_tap + static_cast<int64_t>(co) * Ci + ci] = q;
    }
  }
}

__global__ void k_to_bf16(const float* __restrict__ w, int64_t n, bf16* __restrict__ wb, bf16* __restrict__ wbt, int Ci,
                          int Co) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bf16 q = __float2bfloat16_rn(w[i]);
  if (wb) wb[i] = q;
  if (wbt) {
    const int64_t per_tap = static_cast<int64_t>(Ci) * Co;
    const int64_t t = i / per_tap, r = i % per_tap;
    const int ci = static_cast<int>(r / Co), co = static_cast<int>(r % Co);
    wbt[t * per_tap + static_cast<int64_t>(co) * Ci + ci] = q;
  }
}

// ------------------------------------------------------------ network boundary ----
// Sum of |y|^2 per volume in a fixed order (no atomics), so a volume's RMS does not
// depend on the other volumes of the batch or on scheduling.  Pass 1: block b sums its
// contiguous voxel range; thread t owns volume t % N of rows t / N (+ stride), partial sums
// meet in shared memory in thread order.  Pass 2: one thread per volume adds the blocks.
__global__ void k_vol_sumsq_part(const float2* __restrict__ y, float* __restrict__ part, int64_t V, int N,
                                 int64_t rows_per_block) {
  __shared__ float red[256];
  const int tid = threadIdx.x;
  const int lanes = 256 / N;   // threads per volume
  const int n = tid % N, r = tid / N;
  const int64_t v0 = static_cast<int64_t>(blockIdx.x) * rows_per_block;
  const int64_t v1 = v0 + rows_per_block < V ? v0 + rows_per_block : V;
  float acc = 0.f;
  if (r < lanes)
    for (int64_t v = v0 + r; v < v1; v += lanes) {
      const float2 a = y[v * N + n];
      acc = fmaf(a.x, a.x, fmaf(a.y, a.y, acc));
    }
  red[tid] = acc;
  __syncthreads();
  if (tid < N) {
    float s = 0.f;
    for (int k = 0; k < lanes; ++k) s += red[k * N + tid];
    part[static_cast<int64_t>(blockIdx.x) * N + tid] = s;
  }
}

__global__ void k_vol_sumsq_final(const float* __restrict__ part, float* __restrict__ sums, int blocks, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < blocks; ++b) s += part[static_cast<int64_t>(b) * N + n];
  sums[n] = s;
}

__device__ __forceinline__ float rms_of(const float* sums, int n, int64_t V) {
  const float ms = sums[n] / static_cast<float>(V);
  return ms > 0.f ? sqrtf(ms) : 1.f;
}

// Coordinate channel of index i along an axis of n voxels: (2 i + 1 - n) / P, P the
// smallest power of two >= n (an integer over a power of two: exact in float).
__device__ __forceinline__ float coord_of(int64_t i, int n) {
  int P = 1;
  while (P < n) P <<= 1;
  return static_cast<float>(2 * i + 1 - n) / static_cast<float>(P);
}

__global__ void k_pack(const float2* __restrict__ y, const float* __restrict__ sums, int64_t V, int N, int C,
                       int coords, int nx, int ny, int nz, bf16* __restrict__ xin, float2* __restrict__ xf) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;   // = n * V + v
  if (i >= V * N) return;
  const int n = static_cast<int>(i / V);
  const int64_t v = i % V;
  const float inv = 1.f / rms_of(sums, n, V);
  const float2 a = y[v * N + n];
  const float2 x = make_float2(a.x * inv, a.y * inv);
  xf[i] = x;
  uint4* dst = reinterpret_cast<uint4*>(xin + i * C);
  const __nv_bfloat162 q = __floats2bfloat162_rn(x.x, x.y);
  uint4 first = make_uint4(*reinterpret_cast<const uint32_t*>(&q), 0u, 0u, 0u);
  if (coords) {   // channels 2, 3, 4: the voxel's (x, y, z) position
    const int64_t ix = v % nx, iy = (v / nx) % ny, iz = v / (static_cast<int64_t>(nx) * ny);
    const __nv_bfloat162 c01 = __floats2bfloat162_rn(coord_of(ix, nx), coord_of(iy, ny));
    const __nv_bfloat162 c2 = __floats2bfloat162_rn(coord_of(iz, nz), 0.f);
    first.y = *reinterpret_cast<const uint32_t*>(&c01);
    first.z = *reinterpret_cast<const uint32_t*>(&c2);
  }
  dst[0] = first;
  for (int k = 1; k < C / 8; ++k) dst[k] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void k_loss(const float* __restrict__ o, const float2* __restrict__ xf, const float2* __restrict__ target,
                       const float* __restrict__ sums, float gain, int64_t V, int N, int C, bf16* __restrict__ g,
                       float* __restrict__ loss, float inv_count) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;   // = n * V + v
  float e2 = 0.f;
  if (i < V * N) {
    const int n = static_cast<int>(i / V);
    const int64_t v = i % V;
    const float inv = 1.f / rms_of(sums, n, V);
    const float2 t = target[v * N + n];
    const float2 x = xf[i];
    const float er = o[i * C] + gain * x.x - t.x * inv;
    const float ei = o[i * C + 1] + gain * x.y - t.y * inv;
    e2 = fmaf(er, er, ei * ei);
    bf16* gi = g + i * C;
    *reinterpret_cast<__nv_bfloat162*>(gi) = __floats2bfloat162_rn(2.f * er * inv_count, 2.f * ei * inv_count);
    for (int k = 2; k < C; k += 2) *reinterpret_cast<uint32_t*>(gi + k) = 0u;
  }
  for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, off);
  if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, e2 * inv_count);
}

__global__ void k_output(const float* __restrict__ o, const float2* __restrict__ xf, const float* __restrict__ sums,
                         float gain, int64_t V, int N, int C, float2* __restrict__ y) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;   // = n * V + v
  if (i >= V * N) return;
  const int n = static_cast<int>(i / V);
  const int64_t v = i % V;
  const float r = rms_of(sums, n, V);
  const float2 x = xf[i];
  y[v * N + n] = make_float2(r * (o[i * C] + gain * x.x), r * (o[i * C + 1] + gain * x.y));
}

namespace {
inline unsigned blocks_for(int64_t n, int b = 256) { return static_cast<unsigned>((n + b - 1) / b); }
}  // namespace

cudaError_t launch_vol_sumsq(const float2* y, float* sums, float* part, int64_t V, int N, cudaStream_t s) {
  const int64_t rows = (V + kSumBlocks - 1) / kSumBlocks;
  const int blocks = static_cast<int>((V + rows - 1) / rows);
  k_vol_sumsq_part<<<blocks, 256, 0, s>>>(y, part, V, N, rows);
  k_vol_sumsq_final<<<(N + 127) / 128, 128, 0, s>>>(part, sums, blocks, N);
  return cudaGetLastError();
}

cudaError_t launch_pack(const float2* y, const float* sums, int64_t V, int N, int C, int coords, int nx, int ny,
                        int nz, void* xin, float* xf, cudaStream_t s) {
  k_pack<<<blocks_for(V * N), 256, 0, s>>>(y, sums, V, N, C, coords, nx, ny, nz, static_cast<bf16*>(xin),
                                           reinterpret_cast<float2*>(xf));
  return cudaGetLastError();
}

cudaError_t launch_loss(const float* o, const float* xf, const float2* target, const float* sums, float gain,
                        int64_t V, int N, int C, void* g, float* loss, cudaStream_t s) {
  const float inv = 1.f / static_cast<float>(2 * V * N);
  k_loss<<<blocks_for(V * N), 256, 0, s>>>(o, reinterpret_cast<const float2*>(xf), target, sums, gain, V, N, C,
                                           static_cast<bf16*>(g), loss, inv);
  return cudaGetLastError();
}

cudaError_t launch_output(const float* o, const float* xf, const float* sums, float gain, int64_t V, int N, int C,
                          float2* y, cudaStream_t s) {
  k_output<<<blocks_for(V * N), 256, 0, s>>>(o, reinterpret_cast<const float2*>(xf), sums, gain, V, N, C, y);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* w, int64_t count, void* wb, void* wbt, int ci, int co, cudaStream_t s) {
  k_to_bf16<<<blocks_for(count), 256, 0, s>>>(w, count, static_cast<bf16*>(wb), static_cast<bf16*>(wbt), ci, co);
  return cudaGetLastError();
}

}  // namespace mach_nn

// ---------------------------------------------------------------- C ABI ----
using namespace mach_nn;

namespace {
inline unsigned nblocks(int64_t n, int b = 256) { return static_cast<unsigned>((n + b - 1) / b); }
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline mach_status last_status() { return cudaGetLastError() == cudaSuccess ? MACH_OK : MACH_ERR_CUDA; }

template <int CT>
cudaError_t go_wgrad(const bf16* x, const bf16* dy, float* dw, int n, int d, int h, int w, int ci, int co,
                     cudaStream_t s) {
  const int tiles_x = (w + 7) / 8, tiles_y = (h + 15) / 16;
  const int64_t tiles = static_cast<int64_t>(tiles_x) * tiles_y * d * n;
  const int64_t chan_blocks = static_cast<int64_t>(ci / 16) * (co / CT);
  // about four blocks per SM in total, split over runs of tiles
  int64_t splits = (152LL * 4 + chan_blocks - 1) / chan_blocks;
  splits = splits < tiles ? splits : tiles;
  const int64_t per = (tiles + splits - 1) / splits;
  splits = (tiles + per - 1) / per;
  const int smem = 2 * (2 * kHRows * 16 + (CT / 8) * 128 * 16);
  cudaError_t e = cudaFuncSetAttribute(k_conv3d_wgrad<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>(splits), static_cast<unsigned>(ci / 16), static_cast<unsigned>(co / CT));
  k_conv3d_wgrad<CT><<<grid, 256, smem, s>>>(x, dy, dw, n, d, h, w, ci, co, tiles, tiles_x, tiles_y, per);
  return cudaGetLastError();
}
}  // namespace

extern "C" {

mach_status mach_nn_conv3d(const void* x, const void* w, const float* bias, void* y, float* y_f32, int32_t n,
                           int32_t nz, int32_t ny, int32_t nx, int32_t ci, int32_t co, int32_t flip, int32_t act,
                           void* stream) {
  if (!x || !w || (!y && !y_f32) || n < 1 || nz < 1 || ny < 1 || nx < 1) return MACH_ERR_INVALID_ARG;
  if (ci < 16 || ci % 16 || co < 16 || co % 16) return MACH_ERR_INVALID_ARG;
  if (!aligned16(x) || !aligned16(w) || (y && !aligned16(y)) || (y_f32 && !aligned16(y_f32))) return MACH_ERR_INVALID_ARG;
  const int64_t M = static_cast<int64_t>(n) * nz * ny * nx;
  if ((M + kBM - 1) / kBM > 0x7fffffffLL) return MACH_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int bn = co % 128 == 0 ? 128 : (co % 64 == 0 ? 64 : (co % 32 == 0 ? 32 : 16));
  const dim3 grid(static_cast<unsigned>((M + kBM - 1) / kBM), static_cast<unsigned>(co / bn));
  const bf16* X = static_cast<const bf16*>(x);
  const bf16* Wt = static_cast<const bf16*>(w);
  bf16* Y = static_cast<bf16*>(y);
  switch (bn) {
    case 128: k_conv3d<128><<<grid, 128, 0, s>>>(X, Wt, bias, Y, y_f32, n, nz, ny, nx, ci, co, flip, act); break;
    case 64: k_conv3d<64><<<grid, 128, 0, s>>>(X, Wt, bias, Y, y_f32, n, nz, ny, nx, ci, co, flip, act); break;
    case 32: k_conv3d<32><<<grid, 128, 0, s>>>(X, Wt, bias, Y, y_f32, n, nz, ny, nx, ci, co, flip, act); break;
    default: k_conv3d<16><<<grid, 128, 0, s>>>(X, Wt, bias, Y, y_f32, n, nz, ny, nx, ci, co, flip, act); break;
  }
  return last_status();
}

mach_status mach_nn_conv3d_wgrad(const void* x, const void* dy, float* dw, int32_t n, int32_t nz, int32_t ny,
                                 int32_t nx, int32_t ci, int32_t co, void* stream) {
  if (!x || !dy || !dw || n < 1 || nz < 1 || ny < 1 || nx < 1) return MACH_ERR_INVALID_ARG;
  if (ci < 16 || ci % 16 || co < 16 || co % 16) return MACH_ERR_INVALID_ARG;
  if (!aligned16(x) || !aligned16(dy)) return MACH_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bf16* X = static_cast<const bf16*>(x);
  const bf16* G = static_cast<const bf16*>(dy);
  if (ci / 16 > 65535 || co / 16 > 65535) return MACH_ERR_UNSUPPORTED;
  const cudaError_t e = co % 32 == 0 ? go_wgrad<32>(X, G, dw, n, nz, ny, nx, ci, co, s)
                                     : go_wgrad<16>(X, G, dw, n, nz, ny, nx, ci, co, s);
  return e == cudaSuccess ? MACH_OK : MACH_ERR_CUDA;
}

mach_status mach_nn_bias_grad(const void* g, float* db, int64_t voxels, int32_t c, void* stream) {
  if (!g || !db || voxels < 1 || c < 1 || c > 256 || 256 % c) return MACH_ERR_INVALID_ARG;
  const int64_t rows = 256 / c;
  int64_t blocks = (voxels + rows - 1) / rows;
  blocks = blocks < 152 * 8 ? blocks : 152 * 8;
  k_bias_grad<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(g), db, voxels, c);
  return last_status();
}

mach_status mach_nn_lrelu_bwd(void* g, const void* y, int64_t count, void* stream) {
  if (!g || !y || count < 0) return MACH_ERR_INVALID_ARG;
  if (count == 0) return MACH_OK;
  if (count % 8 == 0 && aligned16(g) && aligned16(y))
    k_lrelu_bwd8<<<nblocks(count / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<uint4*>(g), static_cast<const uint4*>(y), count / 8);
  else
    k_lrelu_bwd<<<nblocks(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<bf16*>(g),
                                                                                 static_cast<const bf16*>(y), count);
  return last_status();
}

mach_status mach_nn_pool2(const void* x, void* y, int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t c,
                          int32_t backward, int32_t accumulate, void* stream) {
  if (!x || !y || n < 1 || nz < 2 || ny < 2 || nx < 2 || nz % 2 || ny % 2 || nx % 2 || c < 1) return MACH_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (c % 8 == 0 && aligned16(x) && aligned16(y)) {
    const int c8 = c / 8;
    const int64_t tot = backward ? static_cast<int64_t>(n) * nz * ny * nx * c8
                                 : static_cast<int64_t>(n) * (nz / 2) * (ny / 2) * (nx / 2) * c8;
    if (!backward)
      k_pool2_v<<<nblocks(tot), 256, 0, s>>>(static_cast<const uint4*>(x), static_cast<uint4*>(y), n, nz, ny, nx, c8);
    else
      k_pool2_bwd_v<<<nblocks(tot), 256, 0, s>>>(static_cast<const uint4*>(x), static_cast<uint4*>(y), n, nz, ny, nx,
                                                 c8, accumulate);
    return last_status();
  }
  if (!backward) {
    const int64_t tot = static_cast<int64_t>(n) * (nz / 2) * (ny / 2) * (nx / 2) * c;
    k_pool2<<<nblocks(tot), 256, 0, s>>>(static_cast<const bf16*>(x), static_cast<bf16*>(y), n, nz, ny, nx, c);
  } else {
    const int64_t tot = static_cast<int64_t>(n) * nz * ny * nx * c;
    k_pool2_bwd<<<nblocks(tot), 256, 0, s>>>(static_cast<const bf16*>(x), static_cast<bf16*>(y), n, nz, ny, nx, c,
                                             accumulate);
  }
  return last_status();
}

mach_status mach_nn_up2(const void* x, void* y, int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t c, int32_t cy,
                        int32_t off, int32_t backward, void* stream) {
  if (!x || !y || n < 1 || nz < 1 || ny < 1 || nx < 1 || c < 1 || off < 0 || off + c > cy) return MACH_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (c % 8 == 0 && cy % 8 == 0 && off % 8 == 0 && aligned16(x) && aligned16(y)) {
    const int c8 = c / 8, cy8 = cy / 8, off8 = off / 8;
    if (!backward) {
      const int64_t tot = static_cast<int64_t>(n) * 8 * nz * ny * nx * c8;
      k_up2_v<<<nblocks(tot), 256, 0, s>>>(static_cast<const uint4*>(x), static_cast<uint4*>(y), n, nz, ny, nx, c8, cy8,
                                           off8);
    } else {
      const int64_t tot = static_cast<int64_t>(n) * nz * ny * nx * c8;
      k_up2_bwd_v<<<nblocks(tot), 256, 0, s>>>(static_cast<const uint4*>(x), static_cast<uint4*>(y), n, nz, ny, nx, c8,
                                               cy8, off8);
    }
    return last_status();
  }
  if (!backward) {
    const int64_t tot = static_cast<int64_t>(n) * 8 * nz * ny * nx * c;
    k_up2<<<nblocks(tot), 256, 0, s>>>(static_cast<const bf16*>(x), static_cast<bf16*>(y), n, nz, ny, nx, c, cy, off);
  } else {
    const int64_t tot = static_cast<int64_t>(n) * nz * ny * nx * c;
    k_up2_bwd<<<nblocks(tot), 256, 0, s>>>(static_cast<const bf16*>(x), static_cast<bf16*>(y), n, nz, ny, nx, c, cy,
                                           off);
  }
  return last_status();
}

mach_status mach_nn_copy_channels(const void* src, void* dst, int64_t voxels, int32_t c, int32_t cy, int32_t off,
                                  int32_t back, void* stream) {
  if (!src || !dst || voxels < 1 || c < 1 || off < 0 || off + c > cy) return MACH_ERR_INVALID_ARG;
  if (c % 8 == 0 && cy % 8 == 0 && off % 8 == 0 && aligned16(src) && aligned16(dst)) {
    k_copy_channels_v<<<nblocks(voxels * (c / 8)), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint4*>(src), static_cast<uint4*>(dst), voxels, c / 8, cy / 8, off / 8, back);
    return last_status();
  }
  k_copy_channels<<<nblocks(voxels * c), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const bf16*>(src), static_cast<bf16*>(dst), voxels, c, cy, off, back);
  return last_status();
}

mach_status mach_nn_adam(float* w, float* m, float* v, const float* g, int64_t count, float lr, float beta1,
                         float beta2, float eps, int32_t step, void* w_bf16, void* w_bf16_t, int32_t ci, int32_t co,
                         void* stream) {
  if (!w || !m || !v || !g || count < 1 || step < 1) return MACH_ERR_INVALID_ARG;
  if (w_bf16_t && (!w_bf16 || ci < 1 || co < 1 || count != 27LL * ci * co)) return MACH_ERR_INVALID_ARG;
  const float c1 = 1.f - powf(beta1, static_cast<float>(step)), c2 = 1.f - powf(beta2, static_cast<float>(step));
  k_adam<<<nblocks(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      w, m, v, g, count, lr, beta1, beta2, eps, c1, c2, static_cast<bf16*>(w_bf16), static_cast<bf16*>(w_bf16_t), ci, co);
  return last_status();
}

}  // extern "C"
