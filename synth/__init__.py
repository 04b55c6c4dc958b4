"""Seeded synthetic workloads: acquisition geometry, phantoms and analytic IQ.

Shared by the tests, the oracle checks and the benchmark as *inputs only*; nothing
here beamforms.  ``make(name, scale)`` returns ``(acquisition, iq)`` with IQ as a
complex64 torch tensor [T, C, S, F] (frames contiguous) on the requested device.

Workloads (full scale):
  ``bmode2d``   128 el linear, 3 plane waves, 1 frame, 1024 samples, 128 x 128 px,
                F# 1.5 Hann; 20 seeded point scatterers + 40 dB SNR noise (seed 1).
  ``doppler2d`` 128 el linear, 1 plane wave, 32 frames @ 10 kHz, 2048 samples,
                256 x 256 px at 0.1 mm, F# 1.0 boxcar; speckle (10 per lambda^2) with a
                10 mm disk rotating at 1 rev/s (seed 2).
  ``volume3d``  32 x 32 matrix, 11 plane waves, 64 frames, 1536 samples, 128^3 voxels
                at 0.1 mm, F# 1.0 Gaussian; speckle (1 per (0.5 mm)^3) + 50 points at
                30x rms; frames = static echo + independent noise at 30 dB (seed 3).
  ``ulm3d``     3D ULM shape (Sec. 6): 32 x 32 matrix at 7.81 MHz, 5 plane waves, 32 frames,
                94 x 94 x 178 voxels at 96 um; speckle + 200 microbubbles at 20x (seed 5).
``small`` scale keeps each workload's structure at sizes the FP64 oracle finishes
in about a second, with grid sides that leave ragged tiles.
"""
from __future__ import annotations

import numpy as np
import torch

from . import acquisition, phantoms, iq as iqmod
from .acquisition import Acquisition, bmode2d, doppler2d, volume3d, linear_array, matrix_array

SEEDS = {"bmode2d": 1, "doppler2d": 2, "volume3d": 3, "ulm3d": 5}


def make_acquisition(name: str, scale: str = "full", iq_dtype: str = "c64") -> Acquisition:
    if name == "bmode2d":
        if scale == "full":
            return bmode2d()
        return bmode2d(nx=45, nz=37)
    if name == "doppler2d":
        if scale == "full":
            return doppler2d(iq_dtype=iq_dtype)
        return doppler2d(nx=61, nz=47, n_frames=32, iq_dtype=iq_dtype).replace(
            grid_origin=(-3.0e-3, 0.0, 18e-3))
    if name == "ulm3d":
        if scale == "full":
            return acquisition.ulm3d(iq_dtype=iq_dtype)
        return acquisition.ulm3d(n_frames=8, iq_dtype=iq_dtype, nx=13, ny=11, nz=17)
    if name == "volume3d":
        if scale == "full":
            return volume3d(iq_dtype=iq_dtype)
        a = volume3d(n=19, n_frames=64, n_side=8, n_samples=768, iq_dtype=iq_dtype)
        return a.replace(grid_dims=(19, 17, 21))
    raise KeyError(name)


def make_phantom(name: str, acq: Acquisition, seed: int, scale: str = "full"):
    if name == "bmode2d":
        return phantoms.points(acq, 20, seed)
    if name == "doppler2d":
        per = 10.0 if scale == "full" else 2.0
        return phantoms.rotating_disk(acq, seed, per_cell=per)
    if name == "volume3d":
        per = 1.0 if scale == "full" else 4.0
        return phantoms.speckle_and_points(acq, seed, per_cell=per)
    if name == "ulm3d":   # tissue speckle plus bright microbubbles
        per = 0.5 if scale == "full" else 4.0
        return phantoms.speckle_and_points(acq, seed, n_points=200, point_gain=20.0, per_cell=per)
    raise KeyError(name)


def make(name: str, scale: str = "full", device="cpu", seed=None, iq_dtype: str = "c64"):
    """(acquisition, IQ complex64 [T,C,S,F]) for a named workload."""
    acq = make_acquisition(name, scale, iq_dtype)
    seed = SEEDS[name] if seed is None else seed
    ph = make_phantom(name, acq, seed, scale)
    if name == "bmode2d":
        iq = iqmod.simulate(acq, ph, seed=seed, snr_db=40.0, device=device)
    elif name == "doppler2d":
        iq = iqmod.simulate(acq, ph, seed=seed, snr_db=None, device=device)
    else:   # volume3d, ulm3d: static echo + independent noise per frame
        accum = torch.complex64 if scale == "full" else torch.complex128
        iq = iqmod.simulate(acq, ph, seed=seed, snr_db=30.0, device=device, accum=accum,
                            static_frames=True)
    return acq, iq


def random_iq(acq: Acquisition, seed: int, device="cpu") -> torch.Tensor:
    """Complex Gaussian IQ (unit power) of the acquisition's shape, for tests whose
    result must not depend on physical structure in the data."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.randn(acq.iq_shape + (2,), generator=g, device=device, dtype=torch.float32)
    return torch.view_as_complex(x * (0.5 ** 0.5))


__all__ = ["Acquisition", "acquisition", "phantoms", "iqmod", "make", "make_acquisition",
           "make_phantom", "random_iq", "bmode2d", "doppler2d", "volume3d", "linear_array",
           "matrix_array", "SEEDS"]
