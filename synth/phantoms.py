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


def compounding_base(acq: Acquisition, seed: int) -> Phantom:
    """One building block of the learned-compounding training scenes (3D grids).

    Kinds, drawn with probabilities 0.5 / 0.25 / 0.25:
      * speckle patch: N(0, 1) scatterers at 4 per mm^3, uniform in a random box of
        side 3-9 mm inside the grid;
      * point cluster: 1-5 points of amplitude 5-30 anywhere in the grid;
      * vessel: scatterers at 30 per mm^3 in a tube of radius 0.2-0.6 mm along a random
        segment of length 4-12 mm, amplitudes N(0, 1) x 2.
    Scenes are complex-weighted sums of such blocks; DAS is linear in the scatterer
    amplitudes, so a scene's volume is the same weighted sum of the blocks' volumes.
    """
    rng = np.random.default_rng(seed)
    lo, hi = _box(acq)
    ext = hi - lo
    kind = rng.random()
    if kind < 0.5:
        side = rng.uniform(3e-3, 9e-3, 3)
        side = np.minimum(side, ext)
        c0 = lo + (ext - side) * rng.random(3)
        n = max(1, int(round(4.0 * np.prod(side) / 1e-9)))
        pos = c0 + side * rng.random((n, 3))
        return Phantom(pos, rng.standard_normal(n))
    if kind < 0.75:
        n = int(rng.integers(1, 6))
        pos = lo + ext * rng.random((n, 3))
        return Phantom(pos, rng.uniform(5.0, 30.0, n) * rng.choice([-1.0, 1.0], n))
    radius = rng.uniform(0.2e-3, 0.6e-3)
    length = rng.uniform(4e-3, 12e-3)
    centre = lo + ext * rng.random(3)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    n = max(1, int(round(30.0 * math.pi * radius ** 2 * length / 1e-9)))
    # uniform in the tube: position along the axis plus a uniform point of the disc
    s = (rng.random(n) - 0.5) * length
    u = np.cross(d, [1.0, 0.0, 0.0] if abs(d[0]) < 0.9 else [0.0, 1.0, 0.0])
    u /= np.linalg.norm(u)
    v = np.cross(d, u)
    rr = radius * np.sqrt(rng.random(n))
    th = 2 * math.pi * rng.random(n)
    pos = centre + s[:, None] * d + (rr * np.cos(th))[:, None] * u + (rr * np.sin(th))[:, None] * v
    keep = np.all((pos >= lo) & (pos <= hi), axis=1)
    if not keep.any():
        keep[:1] = True
        pos[:1] = np.clip(pos[:1], lo, hi)
    return Phantom(pos[keep], 2.0 * rng.standard_normal(int(keep.sum())))
