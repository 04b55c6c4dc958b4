// nn_internal.h -- launchers shared by the network kernels (k_nn.cu) and the U-Net
// executor (unet.cpp).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace mach_nn {

constexpr float kLeak = 1.0f / 64.0f;   // leaky-ReLU slope (exact in every format used)

// sums[n] = sum_v |y[v][n]|^2 for complex64 y [V][N] (N <= 256), in a fixed order;
// part: scratch of kSumBlocks * N floats
constexpr int kSumBlocks = 608;
cudaError_t launch_vol_sumsq(const float2* y, float* sums, float* part, int64_t V, int N, cudaStream_t s);

// x = y / rms: xin bf16 [N][V][C] (channels 0, 1 = re, im; the rest 0), xf float [N][V][2]
cudaError_t launch_pack(const float2* y, const float* sums, int64_t V, int N, int C, int coords, int nx, int ny,
                        int nz, void* xin, float* xf,
                        cudaStream_t s);

// loss and its gradient for o float [N][V][C] against target complex64 [V][N]
cudaError_t launch_loss(const float* o, const float* xf, const float2* target, const float* sums, float gain,
                        int64_t V, int N, int C, void* g, float* loss, cudaStream_t s);

// y[v][n] = rms_n * (gain * xf + o[.., 0:2])
cudaError_t launch_output(const float* o, const float* xf, const float* sums, float gain, int64_t V, int N, int C,
                          float2* y, cudaStream_t s);

// tensor-core convolution (k_conv_tc.cu); cudaErrorNotSupported without a tensor-map encoder
bool conv_tc_supported(int ci, int co);
cudaError_t launch_conv_tc(const void* x, const void* wpk, const float* bias, void* y, float* yf, int n, int d,
                           int h, int w, int ci, int co, int flip, int act, cudaStream_t s);
cudaError_t launch_pack_weights(const float* w, void* wpk, void* wpkt, int ci, int co, cudaStream_t s);

// bfloat16 copies of float32 weights [27][ci][co]: wb (same layout) and wbt ([27][co][ci])
cudaError_t launch_to_bf16(const float* w, int64_t count, void* wb, void* wbt, int ci, int co, cudaStream_t s);

}  // namespace mach_nn
