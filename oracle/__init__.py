"""FP64 CPU oracle for delay-and-sum beamforming and Power Doppler.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg may import this; the product path never does.  It shares no code
with the CUDA library (``paper_2604_06257_gb300``); both read the same seeded inputs
from ``synth``.  The arithmetic lives in ``das_oracle.c``; this module only marshals
arguments through ctypes.

Modes (reading R1): ``"exact"`` evaluates every delay step in FP64; ``"contract"``
takes the index decision in float32 with the fixed operation sequence documented in
``das_oracle.c`` (the precision of the paper's float32 coordinate and arrival-time
arrays, Table 3), then continues in FP64.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_APOD = {"none": 0, "boxcar": 1, "hann": 2, "gauss": 3}
_MODE = {"exact": 0, "contract": 1}


class _Desc(C.Structure):
    _fields_ = [
        ("ndim", C.c_int32), ("n_elem", C.c_int32), ("n_tx", C.c_int32),
        ("n_samples", C.c_int32), ("n_frames", C.c_int32), ("apod", C.c_int32),
        ("mode", C.c_int32), ("pad_", C.c_int32),
        ("n_vox", C.c_int64),
        ("elem_pos", C.c_void_p), ("vox_pos", C.c_void_p),
        ("grid_dims", C.c_int32 * 3), ("pad2_", C.c_int32),
        ("grid_origin", C.c_double * 3), ("grid_step", C.c_double * 3),
        ("tx_angles", C.c_void_p), ("tx_arrival", C.c_void_p),
        ("fs", C.c_double), ("fc", C.c_double), ("c", C.c_double), ("t0", C.c_double),
        ("f_number", C.c_double),
    ]


_lib = None


def configure(L):
    """Declare the C signatures on a loaded oracle library (returns it)."""
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    L.oracle_das.argtypes = [C.POINTER(_Desc), vp, vp, i64, vp, vp, i32]
    L.oracle_terms.argtypes = [C.POINTER(_Desc), vp, i64, vp, vp, vp, vp, vp, vp, i32]
    L.oracle_tx_table.argtypes = [C.POINTER(_Desc), vp]
    L.oracle_tx_exact.argtypes = [C.POINTER(_Desc), vp, i64, vp]
    L.oracle_max_threads.restype = C.c_int
    for f in (L.oracle_das, L.oracle_terms, L.oracle_tx_table, L.oracle_tx_exact):
        f.restype = C.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = configure(C.CDLL(_build.build()))
    return _lib


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Bound:
    """Descriptor plus the numpy arrays it points into (kept alive together)."""

    def __init__(self, acq, mode, tx_arrival=None):
        self.elem = np.ascontiguousarray(acq.elem_pos, dtype=np.float32)
        self.ang = np.ascontiguousarray(acq.tx_angles, dtype=np.float64)
        self.vox = None if acq.vox_pos is None else np.ascontiguousarray(acq.vox_pos, np.float32)
        self.arr = None if tx_arrival is None else np.ascontiguousarray(tx_arrival, np.float32)
        d = _Desc()
        d.ndim, d.n_elem, d.n_tx = acq.ndim, acq.n_elem, acq.n_tx
        d.n_samples, d.n_frames = acq.n_samples, acq.n_frames
        d.apod, d.mode, d.n_vox = _APOD[acq.apod], _MODE[mode], acq.n_vox
        d.elem_pos, d.vox_pos = _ptr(self.elem), _ptr(self.vox)
        if acq.grid_dims is not None:
            d.grid_dims = (C.c_int32 * 3)(*acq.grid_dims)
            d.grid_origin = (C.c_double * 3)(*acq.grid_origin)
            d.grid_step = (C.c_double * 3)(*acq.grid_step)
        d.tx_angles, d.tx_arrival = _ptr(self.ang), _ptr(self.arr)
        d.fs, d.fc, d.c, d.t0, d.f_number = acq.fs, acq.fc, acq.c, acq.t0, acq.f_number
        self.d = d


def _iq_array(iq):
    """complex64 [T,C,S,F] (numpy or torch) -> float32 interleaved numpy."""
    try:
        import torch
        if isinstance(iq, torch.Tensor):
            iq = iq.detach().cpu()
            if iq.dtype in (torch.float16, torch.bfloat16):   # 16-bit pair storage [...,2]
                iq = torch.view_as_complex(iq.float().contiguous())
            iq = iq.to(torch.complex64).numpy()
    except ImportError:
        pass
    iq = np.ascontiguousarray(iq, dtype=np.complex64)
    return iq.view(np.float32)


def _idx(acq, vox_idx):
    if vox_idx is None:
        return np.arange(acq.n_vox, dtype=np.int64)
    return np.ascontiguousarray(vox_idx, dtype=np.int64)


def das(acq, iq, vox_idx=None, mode="contract", threads=0, tx_arrival=None, want_y=True):
    """Beamform: returns (y complex128 [n, F], pd float64 [n]) for voxels ``vox_idx``
    (default all).  ``iq`` complex64 [T,C,S,F] (or float16 [...,2] storage)."""
    b = _Bound(acq, mode, tx_arrival)
    x = _iq_array(iq)
    assert x.size == 2 * acq.n_tx * acq.n_elem * acq.n_samples * acq.n_frames
    idx = _idx(acq, vox_idx)
    n = len(idx)
    y = np.zeros((n, acq.n_frames, 2), dtype=np.float64) if want_y else None
    pd = np.zeros(n, dtype=np.float64)
    rc = lib().oracle_das(C.byref(b.d), _ptr(x), _ptr(idx), n, _ptr(y), _ptr(pd), int(threads))
    assert rc == 0
    yc = None if y is None else y[..., 0] + 1j * y[..., 1]
    return yc, pd


def terms(acq, vox_idx=None, mode="contract", tx_arrival=None, threads=0):
    """Per-term records, arrays of shape [n, C, T]: dict with i0 (int64, -1 out of
    range), valid (bool), w, s, a (window), cw (complex weight)."""
    b = _Bound(acq, mode, tx_arrival)
    idx = _idx(acq, vox_idx)
    n, Cn, T = len(idx), acq.n_elem, acq.n_tx
    shp = (n, Cn, T)
    out = dict(i0=np.zeros(shp, np.int64), valid=np.zeros(shp, np.uint8),
               w=np.zeros(shp), s=np.zeros(shp), a=np.zeros(shp), cw=np.zeros(shp + (2,)))
    rc = lib().oracle_terms(C.byref(b.d), _ptr(idx), n, _ptr(out["i0"]), _ptr(out["valid"]),
                            _ptr(out["w"]), _ptr(out["s"]), _ptr(out["a"]), _ptr(out["cw"]),
                            int(threads))
    assert rc == 0
    out["valid"] = out["valid"].astype(bool)
    out["cw"] = out["cw"][..., 0] + 1j * out["cw"][..., 1]
    return out


def tx_table(acq, tx_arrival=None):
    """Contract-mode transmit delay table, float32 [T, V] in samples."""
    b = _Bound(acq, "contract", tx_arrival)
    out = np.zeros((acq.n_tx, acq.n_vox), dtype=np.float32)
    assert lib().oracle_tx_table(C.byref(b.d), _ptr(out)) == 0
    return out


def tx_exact(acq, vox_idx=None, tx_arrival=None):
    """Exact-mode transmit delay in samples, float64 [T, n]."""
    b = _Bound(acq, "exact", tx_arrival)
    idx = _idx(acq, vox_idx)
    out = np.zeros((acq.n_tx, len(idx)), dtype=np.float64)
    assert lib().oracle_tx_exact(C.byref(b.d), _ptr(idx), len(idx), _ptr(out)) == 0
    return out


def power_doppler(acq, iq, vox_idx=None, mode="contract", threads=0):
    """P[v] = sum_f |y[v][f]|^2 (Sec. 5), float64 [n]."""
    return das(acq, iq, vox_idx, mode, threads, want_y=False)[1]
