"""Learned compounding network -- Python binding of ``include/mach_nn.h``.

Argument marshalling only: every layer, gradient and optimiser step runs in the
library's CUDA kernels (``csrc/k_nn.cu``) driven by its native executor
(``csrc/unet.cpp``).  Functions carry the C names; ``UNet`` owns a network handle and
accepts torch tensors.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import MachError, _dev_ptr, _stream_ptr, lib

NN_EXPORTS = ("mach_nn_conv3d", "mach_nn_conv3d_tc", "mach_nn_pack_weights", "mach_nn_device_status",
              "mach_nn_debug_conv", "mach_nn_set_conv_fold",
              "mach_unet_set_backend", "mach_nn_conv3d_wgrad", "mach_nn_bias_grad", "mach_nn_lrelu_bwd",
              "mach_nn_pool2", "mach_nn_up2", "mach_nn_copy_channels", "mach_nn_adam",
              "mach_unet_create", "mach_unet_destroy", "mach_unet_get_info", "mach_unet_get_params",
              "mach_unet_set_params", "mach_unet_get_grads", "mach_unet_set_gain", "mach_unet_forward",
              "mach_unet_backward", "mach_unet_train_step")


class mach_unet_desc(C.Structure):
    _fields_ = [("levels", C.c_int32), ("base_ch", C.c_int32), ("batch", C.c_int32),
                ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("inference_only", C.c_int32),
                ("coords", C.c_int32)]


class mach_unet_info(C.Structure):
    _fields_ = [("n_params", C.c_int64), ("flops_forward", C.c_int64), ("device_bytes", C.c_int64),
                ("n_convs", C.c_int32), ("in_ch", C.c_int32)]


_bound = False


def _L():
    global _bound
    L = lib()
    if not _bound:
        vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
        sig = {
            "mach_nn_conv3d": [vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, i32, i32, i32, vp],
            "mach_nn_conv3d_tc": [vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, i32, i32, i32, vp],
            "mach_nn_pack_weights": [vp, vp, vp, i32, i32, vp],
            "mach_nn_device_status": [vp],
            "mach_unet_set_backend": [vp, i32],
            "mach_nn_conv3d_wgrad": [vp, vp, vp, i32, i32, i32, i32, i32, i32, vp],
            "mach_nn_bias_grad": [vp, vp, i64, i32, vp],
            "mach_nn_lrelu_bwd": [vp, vp, i64, vp],
            "mach_nn_pool2": [vp, vp, i32, i32, i32, i32, i32, i32, i32, vp],
            "mach_nn_up2": [vp, vp, i32, i32, i32, i32, i32, i32, i32, i32, vp],
            "mach_nn_copy_channels": [vp, vp, i64, i32, i32, i32, i32, vp],
            "mach_nn_adam": [vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp, vp, i32, i32, vp],
            "mach_unet_create": [C.POINTER(mach_unet_desc), C.c_uint64, C.POINTER(vp)],
            "mach_unet_destroy": [vp],
            "mach_unet_get_info": [vp, C.POINTER(mach_unet_info)],
            "mach_unet_get_params": [vp, vp, i64],
            "mach_unet_set_params": [vp, vp, i64],
            "mach_unet_get_grads": [vp, vp, i64],
            "mach_unet_set_gain": [vp, f32],
            "mach_unet_forward": [vp, vp, vp, vp],
            "mach_unet_backward": [vp, vp, vp, vp, vp],
            "mach_unet_train_step": [vp, vp, vp, f32, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.mach_nn_debug_conv.argtypes = [i32, C.c_uint32]
        L.mach_nn_debug_conv.restype = None
        L.mach_nn_set_conv_fold.argtypes = [i32, i32, i32]
        L.mach_nn_set_conv_fold.restype = None
        _bound = True
    return L


def _check(st: int, where: str):
    if st != 0:
        raise MachError(st, where)


def _bf16(t, what):
    import torch
    return _dev_ptr(t, what, torch.bfloat16)


def _f32(t, what):
    import torch
    return _dev_ptr(t, what, torch.float32)


# ---- single ops (same names as the C entry points) ---------------------------------
def mach_nn_conv3d(x, w, bias, y, y_f32, flip=False, act=False, stream=None):
    """x bf16 [N, nz, ny, nx, ci]; w bf16 [27, ci, co] (or [27, co_x, ci_x] transposed for
    flip); outputs y bf16 and/or y_f32 float32 [N, nz, ny, nx, co]."""
    N, nz, ny, nx, ci = x.shape
    co = w.shape[2]
    _check(_L().mach_nn_conv3d(_bf16(x, "x"), _bf16(w, "w"), _f32(bias, "bias"), _bf16(y, "y"),
                               _f32(y_f32, "y_f32"), N, nz, ny, nx, ci, co, int(flip), int(act),
                               _stream_ptr(stream)), "mach_nn_conv3d")


def mach_nn_pack_weights(w, ci, co, forward=True, flipped=True, stream=None):
    """float32 weights [27, ci, co] -> (forward, flipped) bfloat16 copies in the
    tensor-core layout (flat tensors; None where not requested)."""
    import torch
    n = 27 * ci * co
    wpk = torch.empty(n, dtype=torch.bfloat16, device=w.device) if forward else None
    wpkt = torch.empty(n, dtype=torch.bfloat16, device=w.device) if flipped else None
    _check(_L().mach_nn_pack_weights(_f32(w, "w"), _bf16(wpk, "wpk"), _bf16(wpkt, "wpkt"), ci, co,
                                     _stream_ptr(stream)), "mach_nn_pack_weights")
    return wpk, wpkt


def mach_nn_conv3d_tc(x, w_packed, co, bias, y, y_f32, flip=False, act=False, stream=None):
    """Tensor-core convolution: x bf16 [N, nz, ny, nx, ci], w_packed from mach_nn_pack_weights
    (the flipped copy when flip), outputs [N, nz, ny, nx, co]."""
    N, nz, ny, nx, ci = x.shape
    _check(_L().mach_nn_conv3d_tc(_bf16(x, "x"), _bf16(w_packed, "w_packed"), _f32(bias, "bias"), _bf16(y, "y"),
                                  _f32(y_f32, "y_f32"), N, nz, ny, nx, ci, co, int(flip), int(act),
                                  _stream_ptr(stream)), "mach_nn_conv3d_tc")


def mach_nn_device_status(stream=None) -> int:
    return int(_L().mach_nn_device_status(_stream_ptr(stream)))


def mach_nn_debug_conv(stall_copies: bool, wait_limit: int = 0) -> None:
    _L().mach_nn_debug_conv(int(stall_copies), int(wait_limit))


def mach_nn_set_conv_fold(enable: bool, z_planes: int = 4, halo_stages: int = 0) -> None:
    _L().mach_nn_set_conv_fold(int(enable), int(z_planes), int(halo_stages))


def mach_nn_conv3d_wgrad(x, dy, dw, stream=None):
    N, nz, ny, nx, ci = x.shape
    co = dy.shape[-1]
    _check(_L().mach_nn_conv3d_wgrad(_bf16(x, "x"), _bf16(dy, "dy"), _f32(dw, "dw"), N, nz, ny, nx, ci, co,
                                     _stream_ptr(stream)), "mach_nn_conv3d_wgrad")


def mach_nn_bias_grad(g, db, stream=None):
    c = g.shape[-1]
    _check(_L().mach_nn_bias_grad(_bf16(g, "g"), _f32(db, "db"), g.numel() // c, c, _stream_ptr(stream)),
           "mach_nn_bias_grad")


def mach_nn_lrelu_bwd(g, y, stream=None):
    _check(_L().mach_nn_lrelu_bwd(_bf16(g, "g"), _bf16(y, "y"), g.numel(), _stream_ptr(stream)),
           "mach_nn_lrelu_bwd")


def mach_nn_pool2(x, y, backward=False, accumulate=False, stream=None):
    """Forward: x full size -> y pooled.  Backward: x pooled gradient -> y full-size gradient."""
    full = y if backward else x
    N, nz, ny, nx, c = full.shape
    _check(_L().mach_nn_pool2(_bf16(x, "x"), _bf16(y, "y"), N, nz, ny, nx, c, int(backward), int(accumulate),
                              _stream_ptr(stream)), "mach_nn_pool2")


def mach_nn_up2(x, y, off=0, backward=False, stream=None):
    """Forward: x coarse [.., c] -> channels [off, off+c) of y [.., cy].  Backward: x full
    gradient [.., cy] -> y coarse gradient [.., c]."""
    coarse, full = (y, x) if backward else (x, y)
    N, nz, ny, nx, c = coarse.shape
    _check(_L().mach_nn_up2(_bf16(x, "x"), _bf16(y, "y"), N, nz, ny, nx, c, full.shape[-1], off, int(backward),
                            _stream_ptr(stream)), "mach_nn_up2")


def mach_nn_copy_channels(src, dst, off, back=False, stream=None):
    narrow, wide = (dst, src) if back else (src, dst)
    c, cy = narrow.shape[-1], wide.shape[-1]
    _check(_L().mach_nn_copy_channels(_bf16(src, "src"), _bf16(dst, "dst"), narrow.numel() // c, c, cy, off,
                                      int(back), _stream_ptr(stream)), "mach_nn_copy_channels")


def mach_nn_adam(w, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, w_bf16=None, w_bf16_t=None,
                 ci=0, co=0, stream=None):
    _check(_L().mach_nn_adam(_f32(w, "w"), _f32(m, "m"), _f32(v, "v"), _f32(g, "g"), w.numel(), lr, beta1,
                             beta2, eps, step, _bf16(w_bf16, "w_bf16"), _bf16(w_bf16_t, "w_bf16_t"), ci, co,
                             _stream_ptr(stream)), "mach_nn_adam")


# ---- the network --------------------------------------------------------------------
class UNet:
    """The learned compounding network for `batch` volumes of (nx, ny, nz) voxels.

    Volumes in and out are DAS outputs: complex64 [V, batch] CUDA tensors (the batch as
    the frames axis), V = nx * ny * nz.  ``coords``: the voxel's position enters as three
    extra input channels (mach_unet_desc.coords).
    """

    def __init__(self, nx: int, ny: int, nz: int, batch: int, levels: int = 4, base_ch: int = 16,
                 seed: int = 0, inference_only: bool = False, coords: bool = False):
        self.desc = mach_unet_desc(levels, base_ch, batch, nx, ny, nz, int(inference_only), int(coords))
        h = C.c_void_p()
        _check(_L().mach_unet_create(C.byref(self.desc), C.c_uint64(seed), C.byref(h)), "mach_unet_create")
        self.handle = h.value
        info = mach_unet_info()
        _check(_L().mach_unet_get_info(self.handle, C.byref(info)), "mach_unet_get_info")
        self.n_params = int(info.n_params)
        self.flops_forward = int(info.flops_forward)
        self.device_bytes = int(info.device_bytes)
        self.n_convs = int(info.n_convs)
        self.n_vox = nx * ny * nz
        self.batch = batch
        self.gain = 1.0

    def close(self):
        if getattr(self, "handle", None):
            _L().mach_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _vol(self, t, what):
        import torch
        return _dev_ptr(t, what, torch.complex64, self.n_vox * self.batch)

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(_L().mach_unet_get_params(self.handle, out.ctypes.data, self.n_params), "mach_unet_get_params")
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.size}")
        _check(_L().mach_unet_set_params(self.handle, p.ctypes.data, self.n_params), "mach_unet_set_params")

    def grads(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(_L().mach_unet_get_grads(self.handle, out.ctypes.data, self.n_params), "mach_unet_get_grads")
        return out

    def set_backend(self, backend: str) -> None:
        """'tcgen05' (default) or 'mma.sync'."""
        _check(_L().mach_unet_set_backend(self.handle, {"tcgen05": 0, "mma.sync": 1}[backend]),
               "mach_unet_set_backend")

    def set_gain(self, gain: float) -> None:
        _check(_L().mach_unet_set_gain(self.handle, float(gain)), "mach_unet_set_gain")
        self.gain = float(gain)

    def forward(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(_L().mach_unet_forward(self.handle, self._vol(x, "x"), self._vol(y, "y"), _stream_ptr(stream)),
               "mach_unet_forward")
        return y

    def backward(self, x, target, loss=None, stream=None):
        _check(_L().mach_unet_backward(self.handle, self._vol(x, "x"), self._vol(target, "target"),
                                       _f32(loss, "loss"), _stream_ptr(stream)), "mach_unet_backward")

    def train_step(self, x, target, lr: float, loss=None, stream=None):
        _check(_L().mach_unet_train_step(self.handle, self._vol(x, "x"), self._vol(target, "target"), float(lr),
                                         _f32(loss, "loss"), _stream_ptr(stream)), "mach_unet_train_step")


def _conv_case(argv) -> None:
    """`python -m paper_2604_06257_gb300.nn conv CI CO SIDE BATCH [REPEAT]`: run one tensor-core
    convolution on random bfloat16 data (a fixed launch for profilers)."""
    import torch
    from . import build
    build.build()
    ci, co, side, batch = (int(a) for a in argv[:4])
    repeat = int(argv[4]) if len(argv) > 4 else 4
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(batch, side, side, side, ci, device="cuda", generator=g).to(torch.bfloat16)
    w = torch.randn(27, ci, co, device="cuda", generator=g) * 0.05
    wpk, _ = mach_nn_pack_weights(w, ci, co, flipped=False)
    y = torch.empty(batch, side, side, side, co, device="cuda", dtype=torch.bfloat16)
    for _ in range(repeat):
        mach_nn_conv3d_tc(x, wpk, co, None, y, None)
    torch.cuda.synchronize()
    if mach_nn_device_status() != 0:
        raise MachError(5, "mach_nn_conv3d_tc")
    print(f"conv {ci}->{co} on {batch} x {side}^3: ok")


if __name__ == "__main__":
    import sys
    if len(sys.argv) > 1 and sys.argv[1] == "conv":
        _conv_case(sys.argv[2:])
    else:
        raise SystemExit("usage: python -m paper_2604_06257_gb300.nn conv CI CO SIDE BATCH [REPEAT]")
