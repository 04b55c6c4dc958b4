// unet.cpp -- the learned compounding network's executor (host side): parameter layout,
// device buffers (one allocation), initialisation, forward pass, backward pass and Adam,
// all as launches of the kernels in k_nn.cu on the caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "mach_nn.h"
#include "nn_internal.h"

using namespace mach_nn;

namespace {

struct Act {          // bfloat16 [N][level grid][C]
  void* p = nullptr;
  int C = 0;
  int level = 0;
};

struct Conv {
  int ci = 0, co = 0, ci_real = 0, level = 0;
  Act* in = nullptr;
  Act* out = nullptr;  // nullptr: the float32 network output
  bool act = true;
  int64_t w_off = 0, b_off = 0;
  void* wb = nullptr;   // bfloat16 [27][ci][co]
  void* wbt = nullptr;  // bfloat16 [27][co][ci]
  void* wpk = nullptr;  // bfloat16, tensor-core layout of the forward convolution
  void* wpkt = nullptr; // bfloat16, tensor-core layout of the data-gradient convolution
};

uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// standard normal number `k` of stream `seed` (Box-Muller on two counter-based uniforms)
double normal_at(uint64_t seed, uint64_t k) {
  const uint64_t a = splitmix64(seed ^ (2 * k)), b = splitmix64(seed ^ (2 * k + 1));
  const double u1 = (static_cast<double>(a >> 11) + 0.5) * 0x1.0p-53;
  const double u2 = static_cast<double>(b >> 11) * 0x1.0p-53;
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

struct mach_unet_s {
  mach_unet_desc d{};
  int L = 0, c0 = 0, N = 0;
  std::vector<int> nz, ny, nx;   // grid per level
  std::vector<Act> in, a, e, cat, b, dd;
  std::vector<Act> g_in, g_a, g_e, g_cat, g_b, g_d;
  std::vector<Conv> convs;
  float* o = nullptr;     // float32 [N][V0][c0]
  void* g_o = nullptr;    // bfloat16 [N][V0][c0]
  float* xf = nullptr;    // float32 [N][V0][2]
  float* sums = nullptr;  // float32 [N]
  float* sum_part = nullptr;  // float32 [kSumBlocks][N] (fixed-order RMS reduction)
  float* params = nullptr;
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  int64_t n_params = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  float gain = 1.f;
  int step = 0;
  int backend = MACH_UNET_TCGEN05;
  bool training = true;

  int ch(int l) const { return c0 << l; }
  int64_t vox(int l) const { return static_cast<int64_t>(N) * nz[l] * ny[l] * nx[l]; }
  int64_t vox1(int l) const { return static_cast<int64_t>(nz[l]) * ny[l] * nx[l]; }
  int enc(int l, int k) const { return 2 * l + k; }
  int dec(int l, int k) const { return 2 * L + 2 * (L - 2 - l) + k; }
  int out_conv() const { return 4 * L - 2; }
  Act& top() { return L > 1 ? dd[0] : e[0]; }
  Act& g_top() { return L > 1 ? g_d[0] : g_e[0]; }
};

namespace {

mach_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? MACH_OK : MACH_ERR_CUDA; }
#define TRY(x)                               \
  do {                                       \
    const mach_status st_ = (x);             \
    if (st_ != MACH_OK) return st_;          \
  } while (0)

// The tensor-core kernel takes at most 256 output channels.  A convolution's data gradient
// is a convolution from co to ci channels, so the one of a decoder convolution fed by
// 256 + 128 channels (five levels) runs on the warp-MMA kernel, whose bfloat16 weight
// copies are then kept current too.
bool fwd_on_tc(const mach_unet_s* u, const Conv& c) {
  return u->backend == MACH_UNET_TCGEN05 && conv_tc_supported(c.ci, c.co);
}
bool dgrad_on_tc(const mach_unet_s* u, const Conv& c) {
  return u->backend == MACH_UNET_TCGEN05 && conv_tc_supported(c.co, c.ci);
}

mach_status conv_fwd(mach_unet_s* u, const Conv& c, cudaStream_t s) {
  const int l = c.level;
  if (fwd_on_tc(u, c))
    return cuda_ok(launch_conv_tc(c.in->p, c.wpk, u->params + c.b_off, c.out ? c.out->p : nullptr,
                                  c.out ? nullptr : u->o, u->N, u->nz[l], u->ny[l], u->nx[l], c.ci, c.co, 0,
                                  c.act ? 1 : 0, s));
  return mach_nn_conv3d(c.in->p, c.wb, u->params + c.b_off, c.out ? c.out->p : nullptr, c.out ? nullptr : u->o, u->N,
                        u->nz[l], u->ny[l], u->nx[l], c.ci, c.co, 0, c.act ? 1 : 0, s);
}

// gradients of one convolution given the gradient of its (pre-activation) output
mach_status conv_bwd(mach_unet_s* u, const Conv& c, void* gout, void* gin, cudaStream_t s) {
  const int l = c.level;
  TRY(mach_nn_conv3d_wgrad(c.in->p, gout, u->grads + c.w_off, u->N, u->nz[l], u->ny[l], u->nx[l], c.ci, c.co, s));
  TRY(mach_nn_bias_grad(gout, u->grads + c.b_off, u->vox(l), c.co, s));
  if (gin && dgrad_on_tc(u, c))
    TRY(cuda_ok(launch_conv_tc(gout, c.wpkt, nullptr, gin, nullptr, u->N, u->nz[l], u->ny[l], u->nx[l], c.co, c.ci,
                               1, 0, s)));
  else if (gin)
    TRY(mach_nn_conv3d(gout, c.wbt, nullptr, gin, nullptr, u->N, u->nz[l], u->ny[l], u->nx[l], c.co, c.ci, 1, 0, s));
  return MACH_OK;
}

mach_status forward(mach_unet_s* u, const void* x, cudaStream_t s) {
  const int L = u->L, N = u->N;
  TRY(cuda_ok(launch_vol_sumsq(static_cast<const float2*>(x), u->sums, u->sum_part, u->vox1(0), N, s)));
  TRY(cuda_ok(launch_pack(static_cast<const float2*>(x), u->sums, u->vox1(0), N, u->c0, u->d.coords, u->nx[0],
                          u->ny[0], u->nz[0], u->in[0].p, u->xf, s)));
  for (int l = 0; l < L; ++l) {
    if (l > 0)
      TRY(mach_nn_pool2(u->e[l - 1].p, u->in[l].p, N, u->nz[l - 1], u->ny[l - 1], u->nx[l - 1], u->ch(l - 1), 0, 0, s));
    TRY(conv_fwd(u, u->convs[u->enc(l, 0)], s));
    TRY(conv_fwd(u, u->convs[u->enc(l, 1)], s));
  }
  for (int l = L - 2; l >= 0; --l) {
    const Act& src = l == L - 2 ? u->e[L - 1] : u->dd[l + 1];
    const int cy = u->ch(l + 1) + u->ch(l);
    TRY(mach_nn_up2(src.p, u->cat[l].p, N, u->nz[l + 1], u->ny[l + 1], u->nx[l + 1], u->ch(l + 1), cy, 0, 0, s));
    TRY(mach_nn_copy_channels(u->e[l].p, u->cat[l].p, u->vox(l), u->ch(l), cy, u->ch(l + 1), 0, s));
    TRY(conv_fwd(u, u->convs[u->dec(l, 0)], s));
    TRY(conv_fwd(u, u->convs[u->dec(l, 1)], s));
  }
  return conv_fwd(u, u->convs[u->out_conv()], s);
}

mach_status backward(mach_unet_s* u, const void* target, float* loss, cudaStream_t s) {
  const int L = u->L, N = u->N;
  if (loss) TRY(cuda_ok(cudaMemsetAsync(loss, 0, sizeof(float), s)));
  TRY(cuda_ok(launch_loss(u->o, u->xf, static_cast<const float2*>(target), u->sums, u->gain, u->vox1(0), N, u->c0,
                          u->g_o, loss, s)));
  TRY(cuda_ok(cudaMemsetAsync(u->grads, 0, sizeof(float) * u->n_params, s)));
  TRY(conv_bwd(u, u->convs[u->out_conv()], u->g_o, u->g_top().p, s));
  for (int l = 0; l <= L - 2; ++l) {
    const int c = u->ch(l), cy = u->ch(l + 1) + c;
    TRY(mach_nn_lrelu_bwd(u->g_d[l].p, u->dd[l].p, u->vox(l) * c, s));
    TRY(conv_bwd(u, u->convs[u->dec(l, 1)], u->g_d[l].p, u->g_b[l].p, s));
    TRY(mach_nn_lrelu_bwd(u->g_b[l].p, u->b[l].p, u->vox(l) * c, s));
    TRY(conv_bwd(u, u->convs[u->dec(l, 0)], u->g_b[l].p, u->g_cat[l].p, s));
    void* dst = l == L - 2 ? u->g_e[L - 1].p : u->g_d[l + 1].p;
    TRY(mach_nn_up2(u->g_cat[l].p, dst, N, u->nz[l + 1], u->ny[l + 1], u->nx[l + 1], u->ch(l + 1), cy, 0, 1, s));
    TRY(mach_nn_copy_channels(u->g_cat[l].p, u->g_e[l].p, u->vox(l), c, cy, u->ch(l + 1), 1, s));
  }
  for (int l = L - 1; l >= 0; --l) {
    const int c = u->ch(l);
    TRY(mach_nn_lrelu_bwd(u->g_e[l].p, u->e[l].p, u->vox(l) * c, s));
    TRY(conv_bwd(u, u->convs[u->enc(l, 1)], u->g_e[l].p, u->g_a[l].p, s));
    TRY(mach_nn_lrelu_bwd(u->g_a[l].p, u->a[l].p, u->vox(l) * c, s));
    TRY(conv_bwd(u, u->convs[u->enc(l, 0)], u->g_a[l].p, l > 0 ? u->g_in[l].p : nullptr, s));
    if (l > 0)
      TRY(mach_nn_pool2(u->g_in[l].p, u->g_e[l - 1].p, N, u->nz[l - 1], u->ny[l - 1], u->nx[l - 1], u->ch(l - 1), 1, 1,
                        s));
  }
  return MACH_OK;
}

mach_status refresh_bf16(mach_unet_s* u, cudaStream_t s) {
  for (const Conv& c : u->convs) {
    TRY(cuda_ok(launch_to_bf16(u->params + c.w_off, 27LL * c.ci * c.co, c.wb, c.wbt, c.ci, c.co, s)));
    TRY(cuda_ok(launch_pack_weights(u->params + c.w_off, c.wpk, c.wpkt, c.ci, c.co, s)));
  }
  return MACH_OK;
}

void destroy(mach_unet_s* u) {
  if (!u) return;
  cudaFree(u->arena);
  delete u;
}

}  // namespace

extern "C" {

mach_status mach_unet_create(const mach_unet_desc* desc, uint64_t seed, mach_unet* out) {
  if (!desc || !out) return MACH_ERR_INVALID_ARG;
  *out = nullptr;
  const mach_unet_desc d = *desc;
  if (d.levels < 1 || d.levels > 6 || d.batch < 1 || d.batch > 256) return MACH_ERR_INVALID_ARG;
  if (d.base_ch < 16 || d.base_ch % 16) return MACH_ERR_INVALID_ARG;
  const int top_ch = d.base_ch << (d.levels - 1);
  if (top_ch > 256 || 256 % top_ch) return MACH_ERR_UNSUPPORTED;   // bias-gradient kernel limit
  const int q = 1 << (d.levels - 1);
  if (d.nx < q || d.ny < q || d.nz < q || d.nx % q || d.ny % q || d.nz % q) return MACH_ERR_INVALID_ARG;

  mach_unet_s* u = new (std::nothrow) mach_unet_s;
  if (!u) return MACH_ERR_OOM;
  u->d = d;
  u->training = d.inference_only == 0;
  u->L = d.levels;
  u->c0 = d.base_ch;
  u->N = d.batch;
  const int L = u->L;
  for (int l = 0; l < L; ++l) {
    u->nz.push_back(d.nz >> l);
    u->ny.push_back(d.ny >> l);
    u->nx.push_back(d.nx >> l);
  }
  u->in.resize(L);
  u->a.resize(L);
  u->e.resize(L);
  u->g_in.resize(L);
  u->g_a.resize(L);
  u->g_e.resize(L);
  const int nd = L > 1 ? L - 1 : 0;
  u->cat.resize(nd);
  u->b.resize(nd);
  u->dd.resize(nd);
  u->g_cat.resize(nd);
  u->g_b.resize(nd);
  u->g_d.resize(nd);
  for (int l = 0; l < L; ++l) {
    u->in[l] = {nullptr, l == 0 ? u->c0 : u->ch(l - 1), l};
    u->a[l] = u->e[l] = {nullptr, u->ch(l), l};
    u->g_in[l] = u->in[l];
    u->g_a[l] = u->g_e[l] = u->a[l];
  }
  for (int l = 0; l < nd; ++l) {
    u->cat[l] = {nullptr, u->ch(l + 1) + u->ch(l), l};
    u->b[l] = u->dd[l] = {nullptr, u->ch(l), l};
    u->g_cat[l] = u->cat[l];
    u->g_b[l] = u->g_d[l] = u->b[l];
  }

  // convolutions in execution order, with their parameter offsets
  u->convs.resize(4 * L - 1);
  auto set = [&](int idx, int ci, int ci_real, int co, int level, Act* in, Act* outp, bool act) {
    Conv& c = u->convs[idx];
    c.ci = ci;
    c.ci_real = ci_real;
    c.co = co;
    c.level = level;
    c.in = in;
    c.out = outp;
    c.act = act;
  };
  for (int l = 0; l < L; ++l) {
    set(u->enc(l, 0), u->in[l].C, l == 0 ? (d.coords ? 5 : 2) : u->in[l].C, u->ch(l), l, &u->in[l], &u->a[l], true);
    set(u->enc(l, 1), u->ch(l), u->ch(l), u->ch(l), l, &u->a[l], &u->e[l], true);
  }
  for (int l = 0; l < nd; ++l) {
    set(u->dec(l, 0), u->cat[l].C, u->cat[l].C, u->ch(l), l, &u->cat[l], &u->b[l], true);
    set(u->dec(l, 1), u->ch(l), u->ch(l), u->ch(l), l, &u->b[l], &u->dd[l], true);
  }
  set(u->out_conv(), u->c0, u->c0, u->c0, 0, &u->top(), nullptr, false);
  int64_t off = 0;
  for (Conv& c : u->convs) {
    c.w_off = off;
    off += 27LL * c.ci * c.co;
    c.b_off = off;
    off += c.co;
  }
  u->n_params = off;

  // one device allocation, carved in 256-byte pieces
  struct Req {
    void** slot;
    size_t bytes;
  };
  std::vector<Req> reqs;
  auto want = [&](void** slot, size_t bytes) { reqs.push_back({slot, (bytes + 255) / 256 * 256}); };
  const size_t np = sizeof(float) * static_cast<size_t>(u->n_params);
  const bool tr = u->training;
  want(reinterpret_cast<void**>(&u->params), np);
  if (tr) {
    want(reinterpret_cast<void**>(&u->grads), np);
    want(reinterpret_cast<void**>(&u->adam_m), np);
    want(reinterpret_cast<void**>(&u->adam_v), np);
  }
  for (Conv& c : u->convs) {
    want(&c.wb, 2 * 27 * static_cast<size_t>(c.ci) * c.co);
    want(&c.wpk, 2 * 27 * static_cast<size_t>(c.ci) * c.co);
    if (tr) {
      want(&c.wbt, 2 * 27 * static_cast<size_t>(c.ci) * c.co);
      want(&c.wpkt, 2 * 27 * static_cast<size_t>(c.ci) * c.co);
    }
  }
  auto want_act = [&](Act& t) { want(&t.p, 2 * static_cast<size_t>(u->vox(t.level)) * t.C); };
  for (int l = 0; l < L; ++l) {
    want_act(u->in[l]);
    want_act(u->a[l]);
    want_act(u->e[l]);
    if (!tr) continue;
    if (l > 0) want_act(u->g_in[l]);
    want_act(u->g_a[l]);
    want_act(u->g_e[l]);
  }
  for (int l = 0; l < nd; ++l) {
    want_act(u->cat[l]);
    want_act(u->b[l]);
    want_act(u->dd[l]);
    if (!tr) continue;
    want_act(u->g_cat[l]);
    want_act(u->g_b[l]);
    want_act(u->g_d[l]);
  }
  want(reinterpret_cast<void**>(&u->o), sizeof(float) * static_cast<size_t>(u->vox(0)) * u->c0);
  if (tr) want(&u->g_o, 2 * static_cast<size_t>(u->vox(0)) * u->c0);
  want(reinterpret_cast<void**>(&u->xf), sizeof(float) * 2 * static_cast<size_t>(u->vox(0)));
  want(reinterpret_cast<void**>(&u->sums), sizeof(float) * 256);
  want(reinterpret_cast<void**>(&u->sum_part), sizeof(float) * kSumBlocks * 256);
  size_t total = 0;
  for (const Req& r : reqs) total += r.bytes;
  if (cudaMalloc(&u->arena, total) != cudaSuccess) {
    cudaGetLastError();
    delete u;
    return MACH_ERR_OOM;
  }
  u->arena_bytes = total;
  size_t at = 0;
  for (const Req& r : reqs) {
    *r.slot = u->arena + at;
    at += r.bytes;
  }
  // the conv inputs point at the Act objects, whose pointers are now set
  u->convs[u->out_conv()].in = &u->top();

  // He initialisation for the hidden layers; biases and the output layer start at zero
  std::vector<float> h(static_cast<size_t>(u->n_params), 0.f);
  for (size_t i = 0; i + 1 < u->convs.size(); ++i) {
    const Conv& c = u->convs[i];
    const double sd = std::sqrt(2.0 / (27.0 * c.ci_real));
    const uint64_t stream = splitmix64(seed + 0x1000003ull * (i + 1));
    for (int t = 0; t < 27; ++t)
      for (int ci = 0; ci < c.ci_real; ++ci)
        for (int co = 0; co < c.co; ++co) {
          const int64_t k = (static_cast<int64_t>(t) * c.ci + ci) * c.co + co;
          h[static_cast<size_t>(c.w_off + k)] = static_cast<float>(sd * normal_at(stream, static_cast<uint64_t>(k)));
        }
  }
  const mach_status st = mach_unet_set_params(u, h.data(), u->n_params);
  if (st != MACH_OK) {
    destroy(u);
    return st;
  }
  *out = u;
  return MACH_OK;
}

mach_status mach_unet_destroy(mach_unet net) {
  if (!net) return MACH_ERR_INVALID_ARG;
  destroy(net);
  return MACH_OK;
}

mach_status mach_unet_get_info(mach_unet net, mach_unet_info* info) {
  if (!net || !info) return MACH_ERR_INVALID_ARG;
  info->n_params = net->n_params;
  int64_t f = 0;
  for (const Conv& c : net->convs) f += 2LL * 27 * c.ci * c.co * net->vox1(c.level);
  info->flops_forward = f;
  info->device_bytes = static_cast<int64_t>(net->arena_bytes);
  info->n_convs = static_cast<int32_t>(net->convs.size());
  info->in_ch = net->d.coords ? 5 : 2;
  return MACH_OK;
}

mach_status mach_unet_get_params(mach_unet net, float* host, int64_t count) {
  if (!net || !host || count != net->n_params) return MACH_ERR_INVALID_ARG;
  return cuda_ok(cudaMemcpy(host, net->params, sizeof(float) * count, cudaMemcpyDeviceToHost));
}

mach_status mach_unet_get_grads(mach_unet net, float* host, int64_t count) {
  if (!net || !host || count != net->n_params) return MACH_ERR_INVALID_ARG;
  if (!net->training) return MACH_ERR_UNSUPPORTED;
  return cuda_ok(cudaMemcpy(host, net->grads, sizeof(float) * count, cudaMemcpyDeviceToHost));
}

mach_status mach_unet_set_params(mach_unet net, const float* host, int64_t count) {
  if (!net || !host || count != net->n_params) return MACH_ERR_INVALID_ARG;
  const size_t bytes = sizeof(float) * static_cast<size_t>(count);
  TRY(cuda_ok(cudaMemcpy(net->params, host, bytes, cudaMemcpyHostToDevice)));
  if (net->training) {
    TRY(cuda_ok(cudaMemset(net->adam_m, 0, bytes)));
    TRY(cuda_ok(cudaMemset(net->adam_v, 0, bytes)));
  }
  net->step = 0;
  TRY(refresh_bf16(net, nullptr));
  return cuda_ok(cudaDeviceSynchronize());
}

mach_status mach_unet_set_backend(mach_unet net, int32_t backend) {
  if (!net || (backend != MACH_UNET_TCGEN05 && backend != MACH_UNET_MMA_SYNC)) return MACH_ERR_INVALID_ARG;
  net->backend = backend;
  return MACH_OK;
}

mach_status mach_unet_set_gain(mach_unet net, float gain) {
  if (!net || !std::isfinite(gain)) return MACH_ERR_INVALID_ARG;
  net->gain = gain;
  return MACH_OK;
}

mach_status mach_unet_forward(mach_unet net, const void* x, void* y, void* stream) {
  if (!net || !x || !y || x == y) return MACH_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY(forward(net, x, s));
  return cuda_ok(launch_output(net->o, net->xf, net->sums, net->gain, net->vox1(0), net->N, net->c0,
                               static_cast<float2*>(y), s));
}

mach_status mach_unet_backward(mach_unet net, const void* x, const void* target, float* loss, void* stream) {
  if (!net || !x || !target) return MACH_ERR_INVALID_ARG;
  if (!net->training) return MACH_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY(forward(net, x, s));
  return backward(net, target, loss, s);
}

mach_status mach_unet_train_step(mach_unet net, const void* x, const void* target, float lr, float* loss,
                                 void* stream) {
  if (!net || !x || !target || !(lr >= 0.f)) return MACH_ERR_INVALID_ARG;
  if (!net->training) return MACH_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY(forward(net, x, s));
  TRY(backward(net, target, loss, s));
  ++net->step;
  const bool tc = net->backend == MACH_UNET_TCGEN05;
  for (const Conv& c : net->convs) {
    const int64_t nw = 27LL * c.ci * c.co;
    const bool copies = !fwd_on_tc(net, c) || !dgrad_on_tc(net, c);   // warp-MMA kernels read them
    TRY(mach_nn_adam(net->params + c.w_off, net->adam_m + c.w_off, net->adam_v + c.w_off, net->grads + c.w_off, nw,
                     lr, 0.9f, 0.999f, 1e-8f, net->step, copies ? c.wb : nullptr, copies ? c.wbt : nullptr, c.ci,
                     c.co, s));
    if (tc) TRY(cuda_ok(launch_pack_weights(net->params + c.w_off, c.wpk, c.wpkt, c.ci, c.co, s)));
    TRY(mach_nn_adam(net->params + c.b_off, net->adam_m + c.b_off, net->adam_v + c.b_off, net->grads + c.b_off, c.co,
                     lr, 0.9f, 0.999f, 1e-8f, net->step, nullptr, nullptr, 0, 0, s));
  }
  return MACH_OK;
}

}  // extern "C"
