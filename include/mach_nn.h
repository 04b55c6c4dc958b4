/*
 * mach_nn.h -- C ABI of the learned compounding network: a 3D U-Net that maps a
 * few-angle compounded DAS volume to the many-angle one.
 *
 * The paper has no counterpart: it only notes that beamformed volumes can stay on the
 * GPU for downstream processing such as machine-learning inference (Sec. 4).  The
 * network is an addition of this library.  Its input and its training targets are
 * volumes produced by the DAS entry points of mach.h.
 *
 * Network (fixed architecture, `levels` = L, `base_ch` = c0):
 *   level l has c_l = c0 * 2^l channels and grid (nz, ny, nx) / 2^l;
 *   encoder l:  a_l = lrelu(conv(in_l)),  e_l = lrelu(conv(a_l)),
 *               in_0 = the packed input, in_l = avgpool2(e_{l-1});
 *   decoder l (L-2 .. 0): cat_l = [up2(d_{l+1}) | e_l]  (d_{L-1} = e_{L-1}),
 *               b_l = lrelu(conv(cat_l)),  d_l = lrelu(conv(b_l));
 *   output:     o = conv(d_0) (no activation, float32), prediction = gain * x + o[:2].
 *   conv = 3x3x3 "same" convolution with zero padding and a bias; lrelu slope 1/64;
 *   avgpool2 = mean of 2x2x2 blocks; up2 = nearest-neighbour 2x upsampling.
 *   x = the input volume divided by its RMS over voxels (per volume); the prediction is
 *   scaled back by the same RMS.  Loss = mean over volumes, voxels and (re, im) of
 *   (prediction / RMS - target / RMS)^2.
 *
 * Numerics: weights and activations are stored as bfloat16, every convolution is a
 * tensor-core implicit GEMM with float32 accumulation; the output layer, the loss and
 * the Adam state are float32 (float32 master weights, bfloat16 copies for the GEMMs).
 *
 * Layouts: activations are channels-last [N][nz][ny][nx][C] bfloat16 with C a multiple
 * of 16; weights [27][C_in][C_out] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1), the tap
 * reading voxel (z+dz, y+dy, x+dx).  Volumes at the network boundary are DAS outputs:
 * complex64 [V][N] with V = nx*ny*nz voxels (v = ix + nx*(iy + ny*iz)) and the N volumes
 * of a batch as the "frames" axis, exactly as mach_das_run writes them.
 *
 * Ownership, streams and errors follow mach.h: device pointers are the caller's, calls
 * are stream-ordered and never synchronise the host except where stated (parameter
 * and gradient copies), arguments are checked before anything is launched.
 */
#ifndef MACH_NN_H
#define MACH_NN_H

#include <stdint.h>

#include "mach.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ single ops --- */
/* 3x3x3 "same" convolution, channels-last bfloat16, float32 accumulation:
 *   Y[n,z,y,x,co] = act(bias[co] + sum_{tap, ci} X[n, z+dz, y+dy, x+dx, ci] * W[tap, ci, co])
 * (out-of-range voxels read as 0).  With flip != 0 the offsets are negated
 * (X[n, z-dz, y-dy, x-dx, ci]); given W transposed to [27][C_out][C_in] and the output
 * gradient as X this is the data gradient of the convolution.  act: 0 none, 1 leaky ReLU
 * (slope 1/64).  Outputs: y (bfloat16) and/or y_f32 (float32), either may be NULL but
 * not both.  bias may be NULL.  ci, co: multiples of 16; x, w, y, y_f32 16-byte
 * aligned. */
mach_status mach_nn_conv3d(const void* x, const void* w, const float* bias, void* y, float* y_f32,
                           int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t ci, int32_t co,
                           int32_t flip, int32_t act, void* stream);

/* The same convolution on the 5th-generation tensor cores (tcgen05.mma, accumulator in
 * tensor memory, operands staged by TMA): w_packed is the output of mach_nn_pack_weights
 * for this direction (the forward copy, or the flipped copy with flip != 0, in which case
 * ci / co are the flipped convolution's input / output channels).  ci, co multiples of
 * 16, co <= 256.  MACH_ERR_UNSUPPORTED if the driver offers no tensor-map encoder.  A
 * bounded wait that gives up is reported by mach_nn_device_status. */
mach_status mach_nn_conv3d_tc(const void* x, const void* w_packed, const float* bias, void* y, float* y_f32,
                              int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t ci, int32_t co,
                              int32_t flip, int32_t act, void* stream);

/* float32 weights [27][ci][co] -> bfloat16 copies in the tensor-core layout: w_packed
 * [ci/16][27][2][co][8] (element (kc, t, g, o, j) = W[t][16kc + 8g + j][o]) for the
 * forward convolution and w_packed_flip [co/16][27][2][ci][8] (= W[t][i][16kc + 8g + j])
 * for its data gradient; either output may be NULL. */
mach_status mach_nn_pack_weights(const float* w, void* w_packed, void* w_packed_flip, int32_t ci, int32_t co,
                                 void* stream);

/* Synchronises `stream` and returns MACH_ERR_TIMEOUT (clearing it) if a tensor-core
 * convolution gave up a bounded wait since the last call, else MACH_OK. */
mach_status mach_nn_device_status(void* stream);

/* Test hook for the tensor-core convolution's bounded waits: with stall_copies != 0 its copy
 * warp issues no copies, so every wait runs out; wait_limit = polls per wait (0: default).
 * A stalled launch gives up, frees its tensor memory and sets the status that
 * mach_nn_device_status reports; the context stays usable.  Not thread-safe. */
void mach_nn_debug_conv(int32_t stall_copies, uint32_t wait_limit);

/* Kernel choice of mach_nn_conv3d_tc (and of the U-Net executor) for 16 output channels with
 * at most 96 input channels: enable != 0 (the default) uses the x-folded kernel, which
 * puts the three x taps of each (dz, dy) pair into one N = 48 MMA and shifts the partial
 * sums by one voxel in its epilogue; enable = 0 the 27-tap kernel.  z_planes: planes per
 * x-folded tile (1, 2 or 4 (default)); halo_stages: input bricks in flight per CTA (2 ... 4,
 * 0: as many as keep the CTAs per SM).  Same results up to float32 summation order.  For
 * tests and measurements; not thread-safe. */
void mach_nn_set_conv_fold(int32_t enable, int32_t z_planes, int32_t halo_stages);

/* Weight gradient, accumulated:  dw[tap, ci, co] += sum_{n,z,y,x} X[n, z+dz, y+dy, x+dx, ci] *
 * dY[n, z, y, x, co]   (float32 dw, caller zeroes it). */
mach_status mach_nn_conv3d_wgrad(const void* x, const void* dy, float* dw, int32_t n, int32_t nz, int32_t ny,
                                 int32_t nx, int32_t ci, int32_t co, void* stream);

/* Bias gradient, accumulated: db[c] += sum over voxels of g[v, c]  (c <= 256, 256 % c == 0). */
mach_status mach_nn_bias_grad(const void* g, float* db, int64_t voxels, int32_t c, void* stream);

/* Leaky-ReLU backward in place: g[i] *= (y[i] > 0 ? 1 : 1/64), y = the layer's output. */
mach_status mach_nn_lrelu_bwd(void* g, const void* y, int64_t count, void* stream);

/* 2x average pooling of x [n][nz][ny][nx][c] into y [n][nz/2][ny/2][nx/2][c]; backward
 * != 0: its adjoint, x = the pooled gradient, y = the full-size gradient, and with
 * accumulate != 0 added to y instead of overwriting it. */
mach_status mach_nn_pool2(const void* x, void* y, int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t c,
                          int32_t backward, int32_t accumulate, void* stream);

/* Nearest 2x upsampling of x [n][nz][ny][nx][c] into channels [off, off+c) of
 * y [n][2nz][2ny][2nx][cy]; backward != 0: its adjoint (x = the gradient of y with cy
 * channels, y = the coarse gradient with c channels). */
mach_status mach_nn_up2(const void* x, void* y, int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t c,
                        int32_t cy, int32_t off, int32_t backward, void* stream);

/* Channel-slice copy: back == 0: src [V][c] -> channels [off, off+c) of dst [V][cy];
 * back != 0: channels [off, off+c) of src [V][cy] -> dst [V][c]. */
mach_status mach_nn_copy_channels(const void* src, void* dst, int64_t voxels, int32_t c, int32_t cy, int32_t off,
                                  int32_t back, void* stream);

/* Adam step on float32 parameters (Kingma & Ba, Algorithm 1, with bias correction):
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;  w -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 * Optional outputs: w_bf16 (same layout, round to nearest even) and w_bf16_t (the
 * [27][ci][co] weights transposed to [27][co][ci]; needs count = 27*ci*co). */
mach_status mach_nn_adam(float* w, float* m, float* v, const float* g, int64_t count, float lr, float beta1,
                         float beta2, float eps, int32_t step, void* w_bf16, void* w_bf16_t, int32_t ci, int32_t co,
                         void* stream);

/* --------------------------------------------------------------- the network --- */
typedef struct mach_unet_s* mach_unet;

typedef struct {
    int32_t levels;     /* L >= 1 (4 for the standard network)                    */
    int32_t base_ch;    /* c0, a multiple of 16 (16)                               */
    int32_t batch;      /* N volumes per call                                      */
    int32_t nx, ny, nz; /* volume dimensions, multiples of 2^(L-1)                 */
    int32_t inference_only; /* non-zero: no gradient, optimiser or data-gradient buffers
                               (about half the memory); backward / train_step then return
                               MACH_ERR_UNSUPPORTED */
    int32_t coords;     /* non-zero: input channels 2, 3, 4 carry the voxel's position,
                           c = (2 i + 1 - n) / P per axis (i the index, n the dimension, P
                           the smallest power of two >= n), so that the network can depend
                           on where a voxel lies (the point-spread function of a finite
                           aperture varies across the volume); zero: channels 2.. are 0 */
} mach_unet_desc;

typedef struct {
    int64_t n_params;        /* float32 parameters (weights + biases)               */
    int64_t flops_forward;   /* multiply-adds x 2 of one forward pass of one volume */
    int64_t device_bytes;    /* device memory the network holds                     */
    int32_t n_convs;         /* 4L - 1 convolutions                                  */
    int32_t in_ch;           /* 2: (re, im), or 5 with coordinates; padded to base_ch */
} mach_unet_info;

/* Creates the network and its buffers for `batch` volumes of the given size.  Weights
 * are drawn from N(0, 2 / (27 * fan_in)) (He initialisation, fan_in = real input
 * channels) by a counter-based generator seeded with `seed`; biases and the output
 * layer start at zero, so an untrained network predicts gain * x.  gain starts at 1. */
mach_status mach_unet_create(const mach_unet_desc* desc, uint64_t seed, mach_unet* out);
mach_status mach_unet_destroy(mach_unet net);
mach_status mach_unet_get_info(mach_unet net, mach_unet_info* info);

/* Parameters as one float32 host array, convolution by convolution in execution order
 * (encoder 0..L-1, decoder L-2..0, output), each as W [27][C_in][C_out] then bias [C_out].
 * Copies synchronise the device.  set_params also refreshes the bfloat16 copies and
 * resets the Adam state. */
mach_status mach_unet_get_params(mach_unet net, float* host, int64_t count);
mach_status mach_unet_set_params(mach_unet net, const float* host, int64_t count);
/* Gradients of the last mach_unet_backward, same order as the parameters. */
mach_status mach_unet_get_grads(mach_unet net, float* host, int64_t count);
mach_status mach_unet_set_gain(mach_unet net, float gain);
/* Convolution kernels: MACH_UNET_TCGEN05 (default) or MACH_UNET_MMA_SYNC (warp-level
 * mma.sync implicit GEMM, kept for comparison). */
typedef enum { MACH_UNET_TCGEN05 = 0, MACH_UNET_MMA_SYNC = 1 } mach_unet_backend;
mach_status mach_unet_set_backend(mach_unet net, int32_t backend);

/* Prediction for `batch` input volumes: x, y complex64 [V][batch] device (y may not
 * alias x). */
mach_status mach_unet_forward(mach_unet net, const void* x, void* y, void* stream);

/* Forward, loss and gradients against target (complex64 [V][batch]); loss (device
 * float, may be NULL) receives the loss. */
mach_status mach_unet_backward(mach_unet net, const void* x, const void* target, float* loss, void* stream);

/* backward, then one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr. */
mach_status mach_unet_train_step(mach_unet net, const void* x, const void* target, float lr, float* loss,
                                 void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MACH_NN_H */
