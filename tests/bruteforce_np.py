"""A second, independently written FP64 delay-and-sum, vectorised in numpy.

Used only to brute-force the oracle on tiny inputs.  It evaluates every
(voxel, element, transmit) term at once with array broadcasting rather than the
oracle's nested loops, and shares no code with either the oracle or the CUDA path.
Exact (FP64) delays only.
"""
from __future__ import annotations

import numpy as np


def das(acq, iq):
    """y complex128 [V, F] and P [V] for complex IQ [T, C, S, F]."""
    iq = np.asarray(iq, dtype=np.complex128)
    T, C, S, F = iq.shape
    P = acq.voxel_positions()                                  # [V,3]
    E = acq.elem_pos.astype(np.float64)                        # [C,3]
    az, el = acq.tx_angles[:, 0], acq.tx_angles[:, 1]
    U = np.column_stack([np.sin(az) * np.cos(el), np.sin(el), np.cos(az) * np.cos(el)])
    arrival = (P @ U.T) / acq.c                                # [V,T] seconds
    D = P[:, None, :] - E[None, :, :]                          # [V,C,3]
    back = np.sqrt((D ** 2).sum(-1)) / acq.c                   # [V,C] seconds
    t_abs = arrival[:, None, :] + back[:, :, None]             # [V,C,T] absolute time
    s = (t_abs - acq.t0) * acq.fs                              # sample position
    lateral = np.hypot(D[..., 0], D[..., 1])                   # [V,C]
    depth = D[..., 2]
    if acq.apod == "none":
        inside = np.ones_like(depth, dtype=bool)
        frac = np.zeros_like(depth)
    else:
        inside = (depth > 0) & (lateral * 2.0 * acq.f_number <= depth)
        frac = np.where(depth > 0, lateral * acq.f_number / np.where(depth > 0, depth, 1.0), 0.0)
    win = {"none": np.ones_like(frac), "boxcar": np.ones_like(frac),
           "hann": np.cos(np.pi * frac) ** 2, "gauss": np.exp(-8.0 * frac ** 2)}[acq.apod]
    base = np.floor(s)
    frac_s = s - base
    keep = inside[:, :, None] & (base >= 0) & (base + 1 <= S - 1)
    lo = np.clip(base, 0, S - 2).astype(np.int64)
    tt = np.arange(T)[None, None, :]
    cc = np.arange(C)[None, :, None]
    a = iq[tt, cc, lo, :]                                      # [V,C,T,F]
    b = iq[tt, cc, lo + 1, :]
    sample = a + frac_s[..., None] * (b - a)
    rot = np.exp(2j * np.pi * acq.fc * t_abs)                  # = e^{j 2pi fc (t0 + s/fs)}
    weight = np.where(keep, win[:, :, None] * rot, 0.0)
    y = (weight[..., None] * sample).sum(axis=(1, 2))
    return y, (np.abs(y) ** 2).sum(-1)
