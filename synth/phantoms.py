"""Seeded scatterer phantoms (positions in metres, real amplitudes).

Each generator draws from ``numpy.random.default_rng(seed)`` so that a given seed
gives the same phantom on every machine.  Frame-dependent phantoms are returned
as a callable ``frame -> (positions, amplitudes)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Optional, Tuple

import numpy as np

from .acquisition import Acquisition, grid_extent, wavelength


@dataclass
class Phantom:
    """Scatterers that do not move (``static``) plus, optionally, scatterers whose
    positions depend on the frame index (``moving(f)``)."""
    static_pos: np.ndarray            # float64 [J, 3]
    static_amp: np.ndarray            # float64 [J]
    moving: Optional[Callable[[int], Tuple[np.ndarray, np.ndarray]]] = None


def _box(acq: Acquisition, margin: float = 0.0):
    lo, hi = grid_extent(acq)
    lo = lo.copy(); hi = hi.copy()
    for k in range(3):
        if hi[k] > lo[k]:
            lo[k] -= margin; hi[k] += margin
    return lo, hi


def points(acq: Acquisition, n: int, seed: int, amplitude: float = 1.0) -> Phantom:
    """``n`` point scatterers uniform in the grid's bounding box, all of amplitude A."""
    rng = np.random.default_rng(seed)
    lo, hi = _box(acq)
    pos = lo + (hi - lo) * rng.random((n, 3))
    return Phantom(pos, np.full(n, float(amplitude)))


def speckle(acq: Acquisition, seed: int, per_cell: float = 10.0,
            cell: Optional[float] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Fully developed speckle: uniformly placed scatterers with N(0, 1) amplitudes.

    2D: ``per_cell`` scatterers per lambda^2 cell over the grid area.
    3D: ``per_cell`` scatterers per ``cell``^3 volume (``cell`` in metres).
    """
    rng = np.random.default_rng(seed)
    lo, hi = _box(acq)
    ext = hi - lo
    if acq.ndim == 2:
        lam = wavelength(acq)
        n = int(round(per_cell * ext[0] * ext[2] / lam ** 2))
    else:
        cell = cell if cell is not None else 0.5e-3
        n = int(round(per_cell * ext[0] * ext[1] * ext[2] / cell ** 3))
    pos = lo + ext * rng.random((n, 3))
    return pos, rng.standard_normal(n)


def rotating_disk(acq: Acquisition, seed: int, per_cell: float = 10.0,
                  radius: float = 10e-3, centre=(0.0, 0.0, 22.5e-3),
                  rev_per_s: float = 1.0, background: bool = True) -> Phantom:
    """Speckle field in which the scatterers inside a disk of ``radius`` (x-z plane)
    rotate about ``centre`` at ``rev_per_s``; frame f is at time f / PRF, so its
    positions are the frame-0 positions rotated by 2*pi*rev_per_s*f/PRF."""
    pos, amp = speckle(acq, seed, per_cell)
    cx, _, cz = centre
    r = np.hypot(pos[:, 0] - cx, pos[:, 2] - cz)
    inside = r < radius
    disk_pos, disk_amp = pos[inside], amp[inside]
    if background:
        stat_pos, stat_amp = pos[~inside], amp[~inside]
    else:
        stat_pos, stat_amp = np.zeros((0, 3)), np.zeros(0)
    prf = acq.prf if acq.prf > 0 else 1.0

    def moving(f: int):
        th = 2.0 * math.pi * rev_per_s * f / prf
        ct, st = math.cos(th), math.sin(th)
        dx, dz = disk_pos[:, 0] - cx, disk_pos[:, 2] - cz
        p = disk_pos.copy()
        p[:, 0] = cx + ct * dx - st * dz
        p[:, 2] = cz + st * dx + ct * dz
        return p, disk_amp

    return Phantom(stat_pos, stat_amp, moving)


def speckle_and_points(acq: Acquisition, seed: int, n_points: int = 50,
                       point_gain: float = 30.0, per_cell: float = 1.0,
                       cell: float = 0.5e-3) -> Phantom:
    """3D speckle (``per_cell`` per ``cell``^3) plus ``n_points`` bright targets whose
    amplitude is ``point_gain`` times the speckle rms."""
    pos, amp = speckle(acq, seed, per_cell=per_cell, cell=cell)
    rng = np.random.default_rng(seed + 7919)
    lo, hi = _box(acq)
    pp = lo + (hi - lo) * rng.random((n_points, 3))
    return Phantom(np.concatenate([pos, pp]),
                   np.concatenate([amp, np.full(n_points, point_gain)]))
