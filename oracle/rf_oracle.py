"""FP64 oracle of RF demodulation (the method accepts RF or IQ channel data).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg may import this; the product path never does.  It shares no code with
the CUDA library.  Plain numpy in float64, the definition written out:

  b[m]  = rf[m] exp(-j 2 pi fc (t0 + m / fs))                  (mix to baseband)
  iq[n] = sum_{k < L} h[k] b[n D + k - (L-1)/2]                 (centred FIR, decimate by D)

with RF samples outside [0, S) taken as zero.
"""
from __future__ import annotations

import numpy as np


def rf_to_iq(rf: np.ndarray, taps, fs: float, fc: float, t0: float = 0.0, decim: int = 1) -> np.ndarray:
    """rf float [T, C, S, F] -> complex128 [T, C, (S - 1) // decim + 1, F]."""
    rf = np.asarray(rf, dtype=np.float64)
    h = np.asarray(taps, dtype=np.float64)
    T, C, S, F = rf.shape
    m = np.arange(S)
    b = rf * np.exp(-2j * np.pi * fc * (t0 + m / fs))[None, None, :, None]
    n_iq = (S - 1) // decim + 1
    n = np.arange(n_iq)
    c = (len(h) - 1) // 2
    out = np.zeros((T, C, n_iq, F), dtype=np.complex128)
    for k in range(len(h)):
        idx = n * decim + k - c
        ok = (idx >= 0) & (idx < S)
        out[:, :, ok, :] += h[k] * b[:, :, idx[ok], :]
    return out
