"""Acquisition descriptions: array geometry, transmit set, sampling and voxel grid.

This module only *describes* workloads (element and voxel positions, plane-wave
angles, sampling parameters).  It holds no beamforming arithmetic; the oracle and
the CUDA library each read these fields and do their own maths.

Workload shapes follow the paper's benchmark and application sections:
  * the rotating-disk Doppler benchmark (Sec. 4.1: 128-element linear array,
    32 plane-wave frames, 0.1 mm grid from 10 to 35 mm depth, F-number 1.0,
    complex64 IQ, linear interpolation);
  * a steered-plane-wave B-mode case (Sec. 2.1: compounding over transmit angles);
  * a 32x32 matrix-array volume (Sec. 6: 1024-channel matrix probe, compounded
    plane waves, 3D grid at ~0.1 mm).
The paper's datasets are not available here, so every input is synthetic and
seeded (see ``synth.phantoms`` and ``synth.iq``).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

APOD_CODES = {"none": 0, "boxcar": 1, "hann": 2, "gauss": 3}
IQ_DTYPES = ("c64", "f16x2", "bf16x2", "c64split")


@dataclasses.dataclass(frozen=True)
class Acquisition:
    """One plane-wave acquisition and its reconstruction grid.

    Units: metres, seconds, hertz, radians.  Axes: x lateral, y elevation, z depth;
    the array lies in the plane z = 0.  Voxels are either a regular grid (x fastest,
    then y, then z) or an explicit float32 list.
    """

    name: str
    ndim: int
    elem_pos: np.ndarray              # float32 [C, 3]
    tx_angles: np.ndarray             # float64 [T, 2] (azimuth, elevation)
    fs: float
    fc: float
    c: float
    t0: float
    f_number: float
    apod: str
    n_samples: int
    n_frames: int
    grid_dims: Optional[Tuple[int, int, int]] = None
    grid_origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    grid_step: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    vox_pos: Optional[np.ndarray] = None   # float32 [V, 3]
    prf: float = 0.0
    iq_dtype: str = "c64"

    def __post_init__(self):
        assert self.ndim in (2, 3)
        assert self.elem_pos.dtype == np.float32 and self.elem_pos.ndim == 2
        assert self.tx_angles.dtype == np.float64 and self.tx_angles.shape[1] == 2
        assert (self.grid_dims is None) != (self.vox_pos is None)
        assert self.apod in APOD_CODES and self.iq_dtype in IQ_DTYPES

    # sizes -----------------------------------------------------------------
    @property
    def n_elem(self) -> int:
        return int(self.elem_pos.shape[0])

    @property
    def n_tx(self) -> int:
        return int(self.tx_angles.shape[0])

    @property
    def n_vox(self) -> int:
        if self.vox_pos is not None:
            return int(self.vox_pos.shape[0])
        nx, ny, nz = self.grid_dims
        return nx * ny * nz

    @property
    def points(self) -> int:
        """Delay-and-sum points, Eq. 1: voxels x channels x transmits x frames."""
        return self.n_vox * self.n_elem * self.n_tx * self.n_frames

    @property
    def iq_shape(self) -> Tuple[int, int, int, int]:
        """IQ layout [transmit][channel][sample][frame], frames contiguous."""
        return (self.n_tx, self.n_elem, self.n_samples, self.n_frames)

    def voxel_positions(self) -> np.ndarray:
        """float64 [V, 3] voxel centres (grid: origin + index * step per axis)."""
        if self.vox_pos is not None:
            return self.vox_pos.astype(np.float64)
        nx, ny, nz = self.grid_dims
        iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        o, s = self.grid_origin, self.grid_step
        p = np.stack([o[0] + ix.astype(np.float64) * s[0],
                      o[1] + iy.astype(np.float64) * s[1],
                      o[2] + iz.astype(np.float64) * s[2]], axis=-1)
        return p.reshape(-1, 3)

    def replace(self, **kw) -> "Acquisition":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------
# arrays
# --------------------------------------------------------------------------

def linear_array(n_elem: int = 128, pitch: float = 0.3e-3) -> np.ndarray:
    """Elements on the x axis, centred on x = 0: x_e = (e - (n-1)/2) * pitch."""
    x = (np.arange(n_elem, dtype=np.float64) - (n_elem - 1) / 2.0) * pitch
    return np.stack([x, np.zeros_like(x), np.zeros_like(x)], axis=1).astype(np.float32)


def matrix_array(nx: int = 32, ny: int = 32, pitch: float = 0.3e-3) -> np.ndarray:
    """Elements on a regular nx x ny lattice at z = 0; element index j*nx + i (x fastest)."""
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = (i.astype(np.float64) - (nx - 1) / 2.0) * pitch
    y = (j.astype(np.float64) - (ny - 1) / 2.0) * pitch
    return np.stack([x.ravel(), y.ravel(), np.zeros(nx * ny)], axis=1).astype(np.float32)


def deg(*a) -> np.ndarray:
    return np.deg2rad(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------
# the three workload shapes (full size) and reduced variants
# --------------------------------------------------------------------------

def bmode2d(nx: int = 128, nz: int = 128, n_elem: int = 128, n_samples: int = 1024,
            n_frames: int = 1) -> Acquisition:
    """Steered-plane-wave 2D B-mode: 128-element linear array (pitch 0.3 mm),
    fc 5 MHz, fs 20 MHz, c 1540 m/s, plane waves at -5/0/+5 degrees, one frame,
    1024 samples, 128 x 128 pixels over x in [-19, 19] mm and z in [5, 40] mm,
    F-number 1.5 with a Hann window."""
    ang = deg(-5.0, 0.0, 5.0)
    return Acquisition(
        name=f"bmode2d_{nx}x{nz}", ndim=2, elem_pos=linear_array(n_elem),
        tx_angles=np.stack([ang, np.zeros(3)], axis=1),
        fs=20e6, fc=5e6, c=1540.0, t0=0.0, f_number=1.5, apod="hann",
        n_samples=n_samples, n_frames=n_frames,
        grid_dims=(nx, 1, nz), grid_origin=(-19e-3, 0.0, 5e-3),
        grid_step=(38e-3 / (nx - 1), 0.0, 35e-3 / (nz - 1)))


def doppler2d(nx: int = 256, nz: int = 256, n_frames: int = 32, n_elem: int = 128,
              n_samples: int = 2048, iq_dtype: str = "c64") -> Acquisition:
    """Rotating-disk ensemble Power Doppler (shape of the paper's Sec. 4.1 benchmark):
    128-element linear array (pitch 0.3 mm), fc 5.2 MHz, fs 20.8 MHz, one 0-degree
    plane wave, 32 frames at 10 kHz PRF, 2048 samples, a 256 x 256 grid at 0.1 mm
    (x in [-12.75, 12.75] mm, z from 10 mm), F-number 1.0 with a flat (boxcar) window."""
    return Acquisition(
        name=f"doppler2d_{nx}x{nz}x{n_frames}", ndim=2, elem_pos=linear_array(n_elem),
        tx_angles=np.zeros((1, 2)), fs=20.8e6, fc=5.2e6, c=1540.0, t0=0.0,
        f_number=1.0, apod="boxcar", n_samples=n_samples, n_frames=n_frames,
        grid_dims=(nx, 1, nz), grid_origin=(-(nx - 1) * 0.5e-4, 0.0, 10e-3),
        grid_step=(1e-4, 0.0, 1e-4), prf=10e3, iq_dtype=iq_dtype)


def volume3d_angles() -> np.ndarray:
    """Eleven plane waves: azimuth-only tilts {-10,-6,-2,2,6,10} degrees and
    elevation-only tilts {-10,-5,0,5,10} degrees."""
    az = deg(-10, -6, -2, 2, 6, 10)
    el = deg(-10, -5, 0, 5, 10)
    return np.concatenate([np.stack([az, np.zeros(6)], 1), np.stack([np.zeros(5), el], 1)])


def volume3d(n: int = 128, n_frames: int = 64, n_side: int = 32, n_samples: int = 1536,
             iq_dtype: str = "c64", tx_angles: Optional[np.ndarray] = None) -> Acquisition:
    """3D volumetric DAS: 32 x 32 matrix array (pitch 0.3 mm), fc 7.8 MHz, fs 31.2 MHz,
    eleven tilted plane waves, 64 frames, 1536 samples, a 128^3 grid at 0.1 mm
    (x, y in [-6.35, 6.35] mm, z from 5 mm), F-number 1.0 with a Gaussian window."""
    ang = volume3d_angles() if tx_angles is None else tx_angles
    return Acquisition(
        name=f"volume3d_{n}^3x{n_frames}_{iq_dtype}", ndim=3,
        elem_pos=matrix_array(n_side, n_side), tx_angles=ang,
        fs=31.2e6, fc=7.8e6, c=1540.0, t0=0.0, f_number=1.0, apod="gauss",
        n_samples=n_samples, n_frames=n_frames,
        grid_dims=(n, n, n), grid_origin=(-(n - 1) * 0.5e-4, -(n - 1) * 0.5e-4, 5e-3),
        grid_step=(1e-4, 1e-4, 1e-4), iq_dtype=iq_dtype)


def grid_extent(acq: Acquisition):
    """(lo, hi) corners of the voxel bounding box, float64 [3] each."""
    p = acq.voxel_positions() if acq.vox_pos is not None else None
    if p is not None:
        return p.min(0), p.max(0)
    o = np.asarray(acq.grid_origin, dtype=np.float64)
    s = np.asarray(acq.grid_step, dtype=np.float64)
    d = np.asarray(acq.grid_dims, dtype=np.float64) - 1.0
    return o, o + d * s


def wavelength(acq: Acquisition) -> float:
    return acq.c / acq.fc


def pulse_sigma_samples(acq: Acquisition) -> float:
    """Standard deviation (in samples) of the Gaussian envelope of a 2-cycle pulse:
    full width at half maximum = 2 / fc."""
    fwhm = 2.0 / acq.fc
    return fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0))) * acq.fs


def ulm3d(n_frames: int = 32, iq_dtype: str = "c64", nx: int = 94, ny: int = 94, nz: int = 178) -> Acquisition:
    """3D ultrasound-localisation-microscopy shape (Sec. 6): 32 x 32 matrix array
    (pitch 0.3 mm) at 7.81 MHz, fs = 4 fc, five plane waves (broadside and +/-5 degrees in
    azimuth and in elevation), a 94 x 94 x 178 grid at 96 um from 3 mm depth, F# 1.0
    Gaussian window."""
    ang = deg(0.0, -5.0, 5.0, 0.0, 0.0)
    el = deg(0.0, 0.0, 0.0, -5.0, 5.0)
    fc = 7.81e6
    fs = 4 * fc
    step = 96e-6
    depth = 3e-3 + (nz - 1) * step
    S = int(math.ceil(2.3 * depth * fs / 1540.0)) + 32
    return Acquisition(
        name=f"ulm3d_{nx}x{ny}x{nz}x{n_frames}", ndim=3, elem_pos=matrix_array(32, 32),
        tx_angles=np.stack([ang, el], 1), fs=fs, fc=fc, c=1540.0, t0=0.0, f_number=1.0,
        apod="gauss", n_samples=S, n_frames=n_frames, grid_dims=(nx, ny, nz),
        grid_origin=(-(nx - 1) * step / 2, -(ny - 1) * step / 2, 3e-3),
        grid_step=(step, step, step), iq_dtype=iq_dtype)
