"""Seeded ragged batches: many acquisitions of different shapes.

Sizes are drawn log-uniformly (numpy default_rng(seed)): half 2D linear-array
instances (64-256 elements, 128^2-384^2 pixels at 0.1 mm), half 3D matrix-array
instances (16^2-32^2 = 256-1024 elements, 64^3-112^3 voxels at 0.1 mm); 1-48 frames,
1-15 plane waves spread over +/-10 degrees.  ``scale`` shrinks the grids (tests).
"""
from __future__ import annotations

import math

import numpy as np

from .acquisition import Acquisition, linear_array, matrix_array


def _logu(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def ragged_instances(n: int = 64, seed: int = 4, iq_dtype: str = "f16x2", scale: float = 1.0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        F = int(round(_logu(rng, 1, 48)))
        T = int(round(_logu(rng, 1, 15)))
        ang = np.deg2rad(np.linspace(-10.0, 10.0, T)) if T > 1 else np.zeros(1)
        if i % 2 == 0:      # 2D
            C = int(round(_logu(rng, 64, 256)))
            side = max(8, int(round(_logu(rng, 128, 384) * scale)))
            fs, fc, c = 20e6, 5e6, 1540.0
            depth = 5e-3 + side * 1e-4
            S = int(math.ceil(2.2 * depth * fs / c)) + 32
            acq = Acquisition(name=f"ragged{i}_2d", ndim=2, elem_pos=linear_array(C),
                              tx_angles=np.stack([ang, np.zeros(T)], 1), fs=fs, fc=fc, c=c, t0=0.0,
                              f_number=1.5, apod="hann", n_samples=S, n_frames=F,
                              grid_dims=(side, 1, side), grid_origin=(-(side - 1) * 0.5e-4, 0.0, 5e-3),
                              grid_step=(1e-4, 0.0, 1e-4), iq_dtype=iq_dtype)
        else:               # 3D
            es = int(round(math.sqrt(_logu(rng, 256, 1024))))
            side = max(4, int(round(_logu(rng, 64, 112) * scale)))
            fs, fc, c = 31.2e6, 7.8e6, 1540.0
            depth = 5e-3 + side * 1e-4
            S = int(math.ceil(2.2 * depth * fs / c)) + 32
            tx = np.stack([ang, np.zeros(T)], 1)
            tx[1::2, :] = tx[1::2, ::-1]          # alternate azimuth / elevation tilts
            acq = Acquisition(name=f"ragged{i}_3d", ndim=3, elem_pos=matrix_array(es, es),
                              tx_angles=np.ascontiguousarray(tx), fs=fs, fc=fc, c=c, t0=0.0,
                              f_number=1.0, apod="gauss", n_samples=S, n_frames=F,
                              grid_dims=(side, side, side),
                              grid_origin=(-(side - 1) * 0.5e-4, -(side - 1) * 0.5e-4, 5e-3),
                              grid_step=(1e-4, 1e-4, 1e-4), iq_dtype=iq_dtype)
        out.append(acq)
    return out
