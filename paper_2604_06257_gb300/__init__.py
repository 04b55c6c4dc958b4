"""GB300 delay-and-sum beamforming (mach, arXiv 2604.06257) -- Python binding.

A thin ctypes layer over ``libmach_gb300.so`` (the C ABI in ``include/mach.h``).  It only
marshals arguments: every step of the beamforming runs in the library's CUDA kernels.
There is no CPU fallback; importing works without a GPU, but any call needs the built
library and a CUDA device and raises otherwise.

Functions carry the C names (``mach_das_plan``, ``mach_das_run``, ``mach_power_doppler``,
``mach_plan_destroy``, ``mach_status_string`` ...).  ``Plan`` is a small convenience
wrapper that owns a plan handle and accepts torch tensors.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import counts  # noqa: F401  (host-side Eq. 1 / Eq. 2 accounting)

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmach_gb300.so")

MACH_OK, MACH_ERR_INVALID_ARG, MACH_ERR_CUDA, MACH_ERR_OOM, MACH_ERR_UNSUPPORTED, MACH_ERR_TIMEOUT = range(6)
APOD = {"none": 0, "boxcar": 1, "hann": 2, "gauss": 3}
IQ_DTYPE = {"c64": 0, "f16x2": 1, "bf16x2": 2, "c64split": 3}
ORDER = {"tcsf": 0, "ftcs": 1}

EXPORTS = ("mach_das_plan", "mach_das_run", "mach_power_doppler", "mach_plan_destroy",
           "mach_status_string", "mach_plan_get_info", "mach_plan_tx_table", "mach_das_terms",
           "mach_version", "mach_debug_fail_alloc_after", "mach_plan_device_status",
           "mach_debug_force_variant", "mach_debug_set_wait_limit", "mach_debug_stall_producer",
           "mach_das_run_noalloc", "mach_iq_convert", "mach_batch_plan", "mach_batch_bind",
           "mach_batch_run", "mach_batch_get_info", "mach_batch_destroy", "mach_das_run_per_tx",
           "mach_rf_to_iq", "mach_power_doppler_host_stream")


class MachError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__(f"{where}: {mach_status_string(status)} ({status})")


class mach_das_desc(C.Structure):
    _fields_ = [
        ("ndim", C.c_int32), ("n_elem", C.c_int32), ("elem_pos", C.c_void_p),
        ("n_vox", C.c_int64), ("vox_pos", C.c_void_p),
        ("grid_dims", C.c_int32 * 3), ("grid_origin", C.c_double * 3), ("grid_step", C.c_double * 3),
        ("n_tx", C.c_int32), ("tx_angles", C.c_void_p), ("tx_table_dev", C.c_void_p),
        ("fs", C.c_double), ("fc", C.c_double), ("c", C.c_double), ("t0", C.c_double),
        ("f_number", C.c_double), ("apod", C.c_int32), ("n_samples", C.c_int32),
        ("n_frames", C.c_int32), ("iq_dtype", C.c_int32), ("term_table", C.c_int32),
    ]


class mach_plan_info(C.Structure):
    _fields_ = [
        ("variant", C.c_char * 40), ("frames_per_lane", C.c_int32), ("lanes_per_voxel", C.c_int32),
        ("voxels_per_cta", C.c_int32), ("threads_per_cta", C.c_int32), ("tile", C.c_int32 * 3),
        ("frame_tiles", C.c_int32), ("ctas", C.c_int64), ("smem_bytes", C.c_int64),
        ("device_bytes", C.c_int64), ("ring_rows", C.c_int32), ("ring_slots", C.c_int32),
        ("copy_pairs", C.c_int64), ("term_table_bytes", C.c_int64),
    ]

    def as_dict(self):
        return {"variant": self.variant.decode(), "frames_per_lane": self.frames_per_lane,
                "lanes_per_voxel": self.lanes_per_voxel, "voxels_per_cta": self.voxels_per_cta,
                "threads_per_cta": self.threads_per_cta, "tile": list(self.tile),
                "frame_tiles": self.frame_tiles, "ctas": self.ctas, "smem_bytes": self.smem_bytes,
                "device_bytes": self.device_bytes, "ring_rows": self.ring_rows,
                "ring_slots": self.ring_slots, "copy_pairs": self.copy_pairs,
                "term_table_bytes": self.term_table_bytes}


class mach_tile_shape(C.Structure):
    _fields_ = [("mode", C.c_int32), ("frame_lanes", C.c_int32), ("tile", C.c_int32 * 3)]


class mach_batch_info(C.Structure):
    _fields_ = [("instances", C.c_int32), ("items", C.c_int32), ("blocks", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("points", C.c_int64)]


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2604_06257_gb300/build.py "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.mach_das_plan.argtypes = [C.POINTER(mach_das_desc), vp, C.POINTER(vp)]
        L.mach_das_run.argtypes = [vp, vp, vp, vp]
        L.mach_das_run_per_tx.argtypes = [vp, vp, vp, vp]
        L.mach_rf_to_iq.argtypes = [vp, vp, i32, i32, i32, i32, C.c_double, C.c_double, C.c_double, vp, i32,
                                    i32, vp]
        L.mach_rf_to_iq.restype = C.c_int
        L.mach_das_run_per_tx.restype = C.c_int
        L.mach_power_doppler.argtypes = [vp, vp, vp, vp, vp]
        L.mach_power_doppler_host_stream.argtypes = [vp, C.POINTER(vp), i32, C.POINTER(vp), C.POINTER(vp), i32]
        L.mach_power_doppler_host_stream.restype = C.c_int
        L.mach_plan_destroy.argtypes = [vp]
        L.mach_status_string.argtypes = [C.c_int]
        L.mach_status_string.restype = C.c_char_p
        L.mach_plan_get_info.argtypes = [vp, C.POINTER(mach_plan_info)]
        L.mach_plan_tx_table.argtypes = [vp, vp, vp]
        L.mach_das_terms.argtypes = [vp, vp, i64, vp, vp, vp, vp]
        L.mach_version.restype = C.c_char_p
        L.mach_debug_fail_alloc_after.argtypes = [i32]
        L.mach_debug_fail_alloc_after.restype = None
        L.mach_plan_device_status.argtypes = [vp, vp]
        L.mach_plan_device_status.restype = C.c_int
        L.mach_debug_force_variant.argtypes = [C.c_char_p]
        L.mach_debug_force_variant.restype = C.c_int
        L.mach_debug_set_wait_limit.argtypes = [C.c_uint32]
        L.mach_debug_set_wait_limit.restype = None
        L.mach_debug_stall_producer.argtypes = [i32]
        L.mach_debug_stall_producer.restype = None
        L.mach_das_run_noalloc.argtypes = [C.POINTER(mach_das_desc), vp, vp, vp, vp]
        L.mach_iq_convert.argtypes = [vp, i32, vp, i32, i32, i32, i32, i32, vp]
        L.mach_iq_convert.restype = C.c_int
        L.mach_batch_plan.argtypes = [vp, i32, vp, vp, C.POINTER(vp)]
        L.mach_batch_bind.argtypes = [vp, vp, vp, vp, vp]
        L.mach_batch_run.argtypes = [vp, vp]
        L.mach_batch_get_info.argtypes = [vp, C.POINTER(mach_batch_info), vp]
        L.mach_batch_destroy.argtypes = [vp]
        for f in ("mach_batch_plan", "mach_batch_bind", "mach_batch_run", "mach_batch_get_info",
                  "mach_batch_destroy"):
            getattr(L, f).restype = C.c_int
        L.mach_das_run_noalloc.restype = C.c_int
        for f in ("mach_das_plan", "mach_das_run", "mach_power_doppler", "mach_plan_destroy",
                  "mach_plan_get_info", "mach_plan_tx_table", "mach_das_terms"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


# ---- raw ABI wrappers (same names as the C entry points) ---------------------------

def mach_status_string(status: int) -> str:
    return lib().mach_status_string(int(status)).decode()


def mach_version() -> str:
    return lib().mach_version().decode()


def mach_debug_fail_alloc_after(n: int) -> None:
    lib().mach_debug_fail_alloc_after(int(n))


def mach_debug_force_variant(name) -> None:
    st = lib().mach_debug_force_variant(None if not name else name.encode())
    if st != MACH_OK:
        raise MachError(st, "mach_debug_force_variant")


def mach_debug_set_wait_limit(polls: int) -> None:
    lib().mach_debug_set_wait_limit(int(polls))


def mach_debug_stall_producer(on: bool) -> None:
    lib().mach_debug_stall_producer(1 if on else 0)


def mach_plan_device_status(plan: int, stream=None) -> int:
    """Synchronise and return the plan's device status code (MACH_OK or MACH_ERR_TIMEOUT)."""
    return int(lib().mach_plan_device_status(plan, _stream_ptr(stream)))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, what, dtype=None, numel=None):
    """Device pointer of a contiguous CUDA tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{what} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


class _HostArrays:
    """Keeps the host arrays a descriptor points into alive."""

    def __init__(self):
        self.keep = []

    def f32(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        self.keep.append(a)
        return a.ctypes.data

    def f64(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.keep.append(a)
        return a.ctypes.data


def make_desc(*, ndim: int, elem_pos, fs: float, fc: float, c: float, n_samples: int,
              n_frames: int, tx_angles=None, tx_table_dev=None, t0: float = 0.0,
              f_number: float = 1.0, apod: str = "boxcar", vox_pos=None,
              grid_dims: Optional[Sequence[int]] = None, grid_origin=(0.0, 0.0, 0.0),
              grid_step=(0.0, 0.0, 0.0), iq_dtype: str = "c64", term_table: bool = False):
    """Build a ``mach_das_desc`` (plus the host arrays it references).  ``term_table``:
    the plan stores every term instead of computing them per run (mach.h)."""
    h = _HostArrays()
    d = mach_das_desc()
    d.ndim = ndim
    ep = np.asarray(elem_pos)
    d.n_elem = ep.shape[0]
    d.elem_pos = h.f32(ep)
    if vox_pos is not None:
        vp = np.asarray(vox_pos)
        d.n_vox = vp.shape[0]
        d.vox_pos = h.f32(vp)
    else:
        d.grid_dims = (C.c_int32 * 3)(*grid_dims)
        d.grid_origin = (C.c_double * 3)(*grid_origin)
        d.grid_step = (C.c_double * 3)(*grid_step)
        d.n_vox = int(np.prod(grid_dims))
    if tx_angles is not None:
        ta = np.asarray(tx_angles, dtype=np.float64).reshape(-1, 2)
        d.n_tx = ta.shape[0]
        d.tx_angles = h.f64(ta)
    if tx_table_dev is not None:
        d.tx_table_dev = _dev_ptr(tx_table_dev, "tx_table_dev", None)
        if tx_angles is None:
            d.n_tx = tx_table_dev.shape[0]
    d.fs, d.fc, d.c, d.t0, d.f_number = fs, fc, c, t0, f_number
    d.apod = APOD[apod] if isinstance(apod, str) else int(apod)
    d.n_samples, d.n_frames = n_samples, n_frames
    d.iq_dtype = IQ_DTYPE[iq_dtype] if isinstance(iq_dtype, str) else int(iq_dtype)
    d.term_table = int(term_table)
    return d, h


def mach_das_plan(desc, stream=None) -> int:
    """Create a plan; returns the opaque handle (int).  Raises MachError."""
    h = C.c_void_p()
    st = lib().mach_das_plan(C.byref(desc), _stream_ptr(stream), C.byref(h))
    if st != MACH_OK:
        raise MachError(st, "mach_das_plan")
    return h.value


def mach_das_run(plan: int, iq, y, stream=None) -> None:
    st = lib().mach_das_run(plan, _dev_ptr(iq, "iq"), _dev_ptr(y, "y"), _stream_ptr(stream))
    if st != MACH_OK:
        raise MachError(st, "mach_das_run")


def mach_das_run_per_tx(plan: int, iq, y, stream=None) -> None:
    """Uncompounded frames y [V, T, F] complex64 (one volume per transmit)."""
    st = lib().mach_das_run_per_tx(plan, _dev_ptr(iq, "iq"), _dev_ptr(y, "y"), _stream_ptr(stream))
    if st != MACH_OK:
        raise MachError(st, "mach_das_run_per_tx")


def mach_power_doppler(plan: int, iq, pd, y=None, stream=None) -> None:
    st = lib().mach_power_doppler(plan, _dev_ptr(iq, "iq"), _dev_ptr(pd, "pd"), _dev_ptr(y, "y"),
                                  _stream_ptr(stream))
    if st != MACH_OK:
        raise MachError(st, "mach_power_doppler")


def _host_ptr(t, what):
    """Address of a contiguous CPU tensor."""
    if t.is_cuda:
        raise ValueError(f"{what} must be a host tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


def mach_power_doppler_host_stream(plan: int, iq_host, src_order, pd_host, y_host=None) -> None:
    """Pipelined Power Doppler of acquisitions in host memory (lists of CPU tensors, pinned
    for overlap): src_order "ftcs" / "tcsf" (complex64, converted by K0 on the device) or
    None (already in the plan's layout and storage type)."""
    n = len(iq_host)
    if len(pd_host) != n or (y_host is not None and len(y_host) != n):
        raise ValueError("iq_host, pd_host and y_host must have the same length")
    arr = C.c_void_p * max(n, 1)
    iq_a = arr(*[_host_ptr(t, "iq_host") for t in iq_host])
    pd_a = arr(*[_host_ptr(t, "pd_host") for t in pd_host])
    y_a = arr(*[_host_ptr(t, "y_host") for t in y_host]) if y_host is not None else None
    order = -1 if src_order is None else ORDER.get(src_order, src_order)
    st = lib().mach_power_doppler_host_stream(plan, iq_a, order, pd_a, y_a, n)
    if st != MACH_OK:
        raise MachError(st, "mach_power_doppler_host_stream")


def mach_das_run_noalloc(desc, iq, y=None, pd=None, stream=None) -> None:
    """Beamform without any device allocation (tables in the library's fixed 8 MiB
    device array; see include/mach.h)."""
    st = lib().mach_das_run_noalloc(C.byref(desc), _dev_ptr(iq, "iq"), _dev_ptr(y, "y"),
                                    _dev_ptr(pd, "pd"), _stream_ptr(stream))
    if st != MACH_OK:
        raise MachError(st, "mach_das_run_noalloc")


def mach_iq_convert(src, src_order, dst, dst_dtype, n_tx, n_elem, n_samples, n_frames, stream=None) -> None:
    st = lib().mach_iq_convert(_dev_ptr(src, "src"), ORDER.get(src_order, src_order), _dev_ptr(dst, "dst"),
                               IQ_DTYPE.get(dst_dtype, dst_dtype), int(n_tx), int(n_elem), int(n_samples),
                               int(n_frames), _stream_ptr(stream))
    if st != MACH_OK:
        raise MachError(st, "mach_iq_convert")


def mach_rf_to_iq(rf, taps, fs_rf: float, fc: float, t0: float = 0.0, decim: int = 1, iq=None, stream=None):
    """Demodulate real RF [T, C, S_rf, F] (float32 CUDA tensor) into complex64 IQ
    [T, C, (S_rf - 1) // decim + 1, F] (mach.h: mach_rf_to_iq)."""
    import torch
    T, Cn, S, F = rf.shape
    n_iq = (S - 1) // decim + 1
    if iq is None:
        iq = torch.empty((T, Cn, n_iq, F), dtype=torch.complex64, device=rf.device)
    h = np.ascontiguousarray(taps, dtype=np.float32)
    st = lib().mach_rf_to_iq(_dev_ptr(rf, "rf", torch.float32), _dev_ptr(iq, "iq", torch.complex64, T * Cn * n_iq * F),
                             T, Cn, S, F, float(fs_rf), float(fc), float(t0), h.ctypes.data, len(h), int(decim),
                             _stream_ptr(stream))
    if st != MACH_OK:
        raise MachError(st, "mach_rf_to_iq")
    return iq


def prepare_iq(src, src_order="ftcs", dtype="c64", shape=None, stream=None):
    """K0 on a complex64 CUDA tensor: returns the kernels' layout [T, C, S, F] (complex64),
    [T, C, S, F, 2] (float16 / bfloat16) or [T, C, S, 2, F] (float32, split rows).  ``shape`` = (T, C, S, F); defaults from ``src``:
    [F, T, C, S] for "ftcs", [T, C, S, F] for "tcsf"."""
    import torch
    if shape is None:
        shape = (src.shape[1], src.shape[2], src.shape[3], src.shape[0]) if src_order == "ftcs" else tuple(src.shape)
    T, Cn, S, F = shape
    if dtype == "c64":
        out = torch.empty((T, Cn, S, F), dtype=torch.complex64, device=src.device)
    elif dtype == "c64split":
        out = torch.empty((T, Cn, S, 2, F), dtype=torch.float32, device=src.device)
    else:
        out = torch.empty((T, Cn, S, F, 2), dtype=torch.float16 if dtype == "f16x2" else torch.bfloat16,
                          device=src.device)
    mach_iq_convert(src, src_order, out, dtype, T, Cn, S, F, stream)
    return out


def mach_plan_destroy(plan: int) -> None:
    st = lib().mach_plan_destroy(plan)
    if st != MACH_OK:
        raise MachError(st, "mach_plan_destroy")


def mach_plan_get_info(plan: int) -> dict:
    info = mach_plan_info()
    st = lib().mach_plan_get_info(plan, C.byref(info))
    if st != MACH_OK:
        raise MachError(st, "mach_plan_get_info")
    return info.as_dict()


def mach_plan_tx_table(plan: int, out, stream=None) -> None:
    st = lib().mach_plan_tx_table(plan, _dev_ptr(out, "out"), _stream_ptr(stream))
    if st != MACH_OK:
        raise MachError(st, "mach_plan_tx_table")


def mach_das_terms(plan: int, vox_idx, i0=None, w=None, cw=None, stream=None) -> None:
    st = lib().mach_das_terms(plan, _dev_ptr(vox_idx, "vox_idx"), int(vox_idx.numel()),
                              _dev_ptr(i0, "i0"), _dev_ptr(w, "w"), _dev_ptr(cw, "cw"),
                              _stream_ptr(stream))
    if st != MACH_OK:
        raise MachError(st, "mach_das_terms")


# ---- convenience wrapper ------------------------------------------------------------

class Plan:
    """Owns a plan handle.  ``run`` / ``power_doppler`` take CUDA tensors (complex64 or
    float16 [..., 2] IQ [T, C, S, F]) and return CUDA tensors; given CPU tensors they
    stage through reusable device buffers and return CPU tensors."""

    def __init__(self, stream=None, **desc_kw):
        import torch
        self.desc, self._host = make_desc(**desc_kw)
        self.n_vox = int(self.desc.n_vox)
        self.n_frames = int(self.desc.n_frames)
        self.iq_dtype = {0: "c64", 1: "f16x2", 2: "bf16x2", 3: "c64split"}[int(self.desc.iq_dtype)]
        self.iq_shape = (int(self.desc.n_tx), int(self.desc.n_elem), int(self.desc.n_samples),
                         self.n_frames)
        self.handle = mach_das_plan(self.desc, stream)
        self._stage = {}
        self._torch = torch

    # geometry ----------------------------------------------------------------
    def info(self) -> dict:
        return mach_plan_get_info(self.handle)

    def device_status(self, stream=None) -> int:
        return mach_plan_device_status(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            mach_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # checks --------------------------------------------------------------------
    def _check_iq(self, iq):
        torch = self._torch
        if self.iq_dtype == "c64":
            if iq.dtype != torch.complex64 or tuple(iq.shape) != self.iq_shape:
                raise ValueError(f"iq must be complex64 {self.iq_shape}, got {iq.dtype} {tuple(iq.shape)}")
        elif self.iq_dtype == "c64split":
            T, Cn, S, F = self.iq_shape
            if iq.dtype != torch.float32 or tuple(iq.shape) != (T, Cn, S, 2, F):
                raise ValueError(f"iq must be float32 {(T, Cn, S, 2, F)} (split rows)")
        else:
            want = torch.float16 if self.iq_dtype == "f16x2" else torch.bfloat16
            if iq.dtype != want or tuple(iq.shape) != self.iq_shape + (2,):
                raise ValueError(f"iq must be {want} {self.iq_shape + (2,)}")

    def _buf(self, name, shape, dtype):
        torch = self._torch
        b = self._stage.get(name)
        if b is None or b.shape != shape or b.dtype != dtype:
            b = torch.empty(shape, dtype=dtype, device="cuda")
            self._stage[name] = b
        return b

    # compute -------------------------------------------------------------------
    def run(self, iq, y=None, stream=None):
        """Complex frames y [V, F] (complex64)."""
        torch = self._torch
        self._check_iq(iq)
        host = not iq.is_cuda
        if host:
            dev = self._buf("iq", tuple(iq.shape), iq.dtype)
            dev.copy_(iq, non_blocking=True)
            iq = dev
        out = y if y is not None else (self._buf("y", (self.n_vox, self.n_frames), torch.complex64)
                                       if host else torch.empty((self.n_vox, self.n_frames),
                                                                dtype=torch.complex64, device=iq.device))
        mach_das_run(self.handle, iq, out, stream)
        return out.cpu() if host else out

    def run_per_tx(self, iq, y=None, stream=None):
        """Uncompounded frames y [V, T, F] (complex64), CUDA tensors only."""
        torch = self._torch
        self._check_iq(iq)
        T = self.iq_shape[0]
        out = y if y is not None else torch.empty((self.n_vox, T, self.n_frames), dtype=torch.complex64,
                                                  device=iq.device)
        mach_das_run_per_tx(self.handle, iq, out, stream)
        return out

    def power_doppler(self, iq, pd=None, y=None, want_y=False, stream=None):
        """Power Doppler pd [V] (float32) and, if requested, the frames y [V, F]."""
        torch = self._torch
        self._check_iq(iq)
        host = not iq.is_cuda
        if host:
            dev = self._buf("iq", tuple(iq.shape), iq.dtype)
            dev.copy_(iq, non_blocking=True)
            iq = dev
        if pd is None:
            pd = (self._buf("pd", (self.n_vox,), torch.float32) if host else
                  torch.empty((self.n_vox,), dtype=torch.float32, device=iq.device))
        if y is None and want_y:
            y = (self._buf("y", (self.n_vox, self.n_frames), torch.complex64) if host else
                 torch.empty((self.n_vox, self.n_frames), dtype=torch.complex64, device=iq.device))
        mach_power_doppler(self.handle, iq, pd, y, stream)
        if host:
            return pd.cpu(), (y.cpu() if y is not None else None)
        return pd, y

    def power_doppler_host(self, iq_host, pd_host, y_host=None, stream=None, order=None):
        """Host buffers in and out (pinned memory recommended): copies the IQ to the
        device, beamforms, copies Power Doppler (and the frames, if ``y_host`` is given)
        back, and returns once the results are in host memory.  With ``order`` ("ftcs":
        complex64 [F, T, C, S] acquisition order, or "tcsf": complex64 [T, C, S, F]) the
        host data are complex64 and K0 converts them on the device to the plan's layout."""
        torch = self._torch
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            raw = self._buf("raw", tuple(iq_host.shape), iq_host.dtype)
            raw.copy_(iq_host, non_blocking=True)
            if order is None:
                self._check_iq(iq_host)
                dev = raw
            else:
                T, Cn, S, F = self.iq_shape
                shape = (T, Cn, S, 2, F) if self.iq_dtype == "c64split" else (
                    (T, Cn, S, F) if self.iq_dtype == "c64" else (T, Cn, S, F, 2))
                dt = {"c64": torch.complex64, "c64split": torch.float32, "f16x2": torch.float16,
                      "bf16x2": torch.bfloat16}[self.iq_dtype]
                dev = self._buf("iq", shape, dt)
                mach_iq_convert(raw, order, dev, self.iq_dtype, T, Cn, S, F, s)
            pd_d = self._buf("pd", (self.n_vox,), torch.float32)
            y_d = (self._buf("y", (self.n_vox, self.n_frames), torch.complex64)
                   if y_host is not None else None)
            mach_power_doppler(self.handle, dev, pd_d, y_d, s)
            pd_host.copy_(pd_d, non_blocking=True)
            if y_host is not None:
                y_host.copy_(y_d, non_blocking=True)
        s.synchronize()
        return pd_host, y_host

    def power_doppler_host_stream(self, iq_host, pd_host, y_host=None, order=None):
        """Power Doppler of several acquisitions in host memory, pipelined in native code
        (mach.h: mach_power_doppler_host_stream): lists of host tensors shaped as for
        ``power_doppler_host``; returns when every result is in host memory."""
        if order is None:
            for t in iq_host:
                self._check_iq(t)
        else:
            T, Cn, S, F = self.iq_shape
            want = (F, T, Cn, S) if order == "ftcs" else (T, Cn, S, F)
            for t in iq_host:
                if tuple(t.shape) != want or t.dtype != self._torch.complex64:
                    raise ValueError(f"iq_host must be complex64 {want}")
        for t in pd_host:
            if t.numel() != self.n_vox or t.dtype != self._torch.float32:
                raise ValueError("pd_host must be float32 [n_vox]")
        for t in (y_host or []):
            if t.numel() != self.n_vox * self.n_frames or t.dtype != self._torch.complex64:
                raise ValueError("y_host must be complex64 [n_vox, n_frames]")
        mach_power_doppler_host_stream(self.handle, iq_host, order, pd_host, y_host)
        return pd_host, y_host

    def tx_table(self):
        torch = self._torch
        out = torch.empty((self.iq_shape[0], self.n_vox), dtype=torch.float32, device="cuda")
        mach_plan_tx_table(self.handle, out)
        return out

    def terms(self, vox_idx):
        """(i0 int32, w float32, cw complex64) of shape [n, C, T], as the kernels compute them."""
        torch = self._torch
        idx = torch.as_tensor(vox_idx, dtype=torch.int64).cuda().contiguous()
        n, T, Cn = idx.numel(), self.iq_shape[0], self.iq_shape[1]
        i0 = torch.empty((n, Cn, T), dtype=torch.int32, device="cuda")
        w = torch.empty((n, Cn, T), dtype=torch.float32, device="cuda")
        cw = torch.empty((n, Cn, T, 2), dtype=torch.float32, device="cuda")
        mach_das_terms(self.handle, idx, i0, w, cw)
        return i0, w, torch.view_as_complex(cw)


# ---- ragged batches ------------------------------------------------------------------

class Batch:
    """Many instances (``plan_kwargs``-style dicts) beamformed by one persistent launch.
    ``shapes``: optional list of (mode, frame_lanes, (tx, ty, tz)) per instance, e.g. from
    ``autotune.tune_batch``; None uses the library's default lane mapping and tile box."""

    def __init__(self, instances, shapes=None, stream=None):
        self._descs_keep = [make_desc(**kw) for kw in instances]
        n = len(instances)
        arr = (mach_das_desc * n)(*[d for d, _ in self._descs_keep])
        sh = None
        if shapes is not None:
            sh = (mach_tile_shape * n)()
            for i, (mode, fl, tile) in enumerate(shapes):
                sh[i].mode, sh[i].frame_lanes = int(mode), int(fl)
                sh[i].tile = (C.c_int32 * 3)(*(tile if tile is not None else (0, 0, 0)))
        h = C.c_void_p()
        st = lib().mach_batch_plan(C.cast(arr, C.c_void_p), n, None if sh is None else C.cast(sh, C.c_void_p),
                                   _stream_ptr(stream), C.byref(h))
        if st != MACH_OK:
            raise MachError(st, "mach_batch_plan")
        self.handle = h.value
        self.n = n
        self.shapes_in = sh

    def info(self) -> dict:
        inf = mach_batch_info()
        shp = (mach_tile_shape * self.n)()
        st = lib().mach_batch_get_info(self.handle, C.byref(inf), C.cast(shp, C.c_void_p))
        if st != MACH_OK:
            raise MachError(st, "mach_batch_get_info")
        return {"instances": inf.instances, "items": inf.items, "blocks": inf.blocks,
                "blocks_per_sm": inf.blocks_per_sm, "points": inf.points,
                "shapes": [(x.mode, x.frame_lanes, tuple(x.tile)) for x in shp]}

    def bind(self, iqs, ys=None, pds=None, stream=None):
        n = self.n
        ia = (C.c_void_p * n)(*[_dev_ptr(t, "iq") for t in iqs])
        ya = None if ys is None else (C.c_void_p * n)(*[_dev_ptr(t, "y") for t in ys])
        pa = None if pds is None else (C.c_void_p * n)(*[_dev_ptr(t, "pd") for t in pds])
        st = lib().mach_batch_bind(self.handle, C.cast(ia, C.c_void_p),
                                   None if ya is None else C.cast(ya, C.c_void_p),
                                   None if pa is None else C.cast(pa, C.c_void_p), _stream_ptr(stream))
        if st != MACH_OK:
            raise MachError(st, "mach_batch_bind")

    def run(self, stream=None):
        st = lib().mach_batch_run(self.handle, _stream_ptr(stream))
        if st != MACH_OK:
            raise MachError(st, "mach_batch_run")

    def close(self):
        if getattr(self, "handle", None):
            lib().mach_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def plan_kwargs(acq) -> dict:
    """Keyword arguments of ``Plan`` / ``make_desc`` from an object with the attributes of
    an acquisition description (ndim, elem_pos, tx_angles, fs, fc, c, t0, f_number, apod,
    n_samples, n_frames, grid_dims/grid_origin/grid_step or vox_pos, iq_dtype)."""
    kw = dict(ndim=acq.ndim, elem_pos=acq.elem_pos, tx_angles=acq.tx_angles, fs=acq.fs, fc=acq.fc,
              c=acq.c, t0=acq.t0, f_number=acq.f_number, apod=acq.apod, n_samples=acq.n_samples,
              n_frames=acq.n_frames, iq_dtype=acq.iq_dtype)
    if acq.vox_pos is not None:
        kw["vox_pos"] = acq.vox_pos
    else:
        kw.update(grid_dims=acq.grid_dims, grid_origin=acq.grid_origin, grid_step=acq.grid_step)
    return kw
