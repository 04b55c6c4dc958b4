"""Autotuner for the per-instance lane mapping and voxel tile of ragged batches.

For one instance, every candidate (lane mapping, tile box) is timed on a one-instance
batch with CUDA events (median of a few launches after a warm-up) and the fastest kept.
Large instances are timed on a slab of their grid (the first ``slab`` z-planes, same
lateral extent, elements, transmits and frames), which has the same per-tile work.
Results are cached per shape signature (dimensionality, grid, elements, transmits,
frames, samples, storage type), so instances of the same shape are tuned once.
"""
from __future__ import annotations

import statistics
from typing import Dict, List, Optional, Tuple

from . import Batch, MachError

Shape = Tuple[int, int, Tuple[int, int, int]]
_CACHE: Dict[tuple, Shape] = {}


def _signature(kw: dict) -> tuple:
    grid = tuple(kw["grid_dims"]) if kw.get("grid_dims") is not None else (len(kw["vox_pos"]), 1, 1)
    return (kw["ndim"], grid, len(kw["elem_pos"]), len(kw["tx_angles"]), kw["n_frames"], kw["n_samples"],
            kw.get("iq_dtype", "c64"))


def _boxes(n: int, ndim: int) -> List[Tuple[int, int, int]]:
    """Compact power-of-two voxel boxes of volume n (a few per lane mapping)."""
    out = []
    if ndim == 2:
        for x in (4, 8, 16):
            if n % x == 0 and n // x <= 64:
                out.append((x, 1, n // x))
    else:
        for x in (4, 8):
            for y in (2, 4):
                if n % (x * y) == 0 and 1 <= n // (x * y) <= 16:
                    out.append((x, y, n // (x * y)))
    return out


def _staged_boxes(n: int, ndim: int) -> List[Tuple[int, int, int]]:
    """Voxel boxes of a staged block (n = 7 x 16 or 7 x 8 voxels): shallow and wide first
    (a window spans ~2 sample rows per voxel of depth, a fraction of a row per voxel of width)."""
    if ndim == 2:
        return [(n // z, 1, z) for z in (2, 4, 7) if n % z == 0]
    return [(x, y, n // (x * y)) for x, y in ((4, 4), (4, 2), (8, 2), (2, 2)) if n % (x * y) == 0 and n // (x * y) >= 1]


def candidates(kw: dict) -> List[Shape]:
    """Lane mappings and voxel boxes an instance can take: staged windows (mode 2, 8 or 16
    frame lanes), frame lanes through L1 (mode 0) and, for F <= 4, channel lanes (mode 1)."""
    F = kw["n_frames"]
    cands: List[Shape] = []
    if F <= 4:
        cands += [(1, 0, b) for b in _boxes(32, kw["ndim"])]
    for fl in (8, 16):
        if 4 * fl >= F:
            n = 7 * 4 * (32 // fl)
            cands += [(2, fl, b) for b in _staged_boxes(n, kw["ndim"])]
    for fl in (2, 4, 8, 16):
        if 4 * fl >= F:
            n = 256 if fl == 2 else 8 * 4 * (32 // fl)
            cands += [(0, fl, b) for b in _boxes(n, kw["ndim"])]
    return cands


def _slab(kw: dict, planes: int) -> dict:
    """The instance restricted to its first ``planes`` z-planes (regular grids only)."""
    if kw.get("grid_dims") is None or kw["grid_dims"][2] <= planes:
        return kw
    nx, ny, nz = kw["grid_dims"]
    return {**kw, "grid_dims": (nx, ny, planes)}


def time_shape(kw: dict, shape: Shape, iq, y, pd, reps: int = 3) -> float:
    import torch
    with Batch([kw], shapes=[shape]) as b:
        b.bind([iq], [y], [pd])
        b.run()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.run()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune_instance(kw: dict, iq, y, pd, max_candidates: Optional[int] = None,
                  slab: int = 32) -> Tuple[Shape, Dict[Shape, float]]:
    sig = _signature(kw)
    if sig in _CACHE:
        return _CACHE[sig], {}
    cands = candidates(kw)
    if max_candidates:
        cands = cands[:max_candidates]
    small = _slab(kw, slab)          # y / pd are large enough for the slab (its voxels come first)
    cands = [c for c in cands]
    times = {}
    for c in cands:
        try:
            times[c] = time_shape(small, c, iq, y, pd)
        except MachError:          # e.g. staged windows that do not fit the ring slot
            continue
    best = min(times, key=times.get)
    _CACHE[sig] = best
    return best, times


def time_batch(instances: List[dict], shapes, iqs, ys, pds, reps: int = 3) -> float:
    import torch
    with Batch(instances, shapes=shapes) as b:
        b.bind(iqs, ys, pds)
        b.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.run()
        e1.record()
        e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(instances: List[dict], iqs, ys, pds) -> Optional[List[Shape]]:
    """Per-instance choices, kept only if the whole batch runs faster with them than with
    the library's default shapes (returns None in that case)."""
    shapes = [tune_instance(kw, iq, y, pd)[0] for kw, iq, y, pd in zip(instances, iqs, ys, pds)]
    if time_batch(instances, shapes, iqs, ys, pds) < time_batch(instances, None, iqs, ys, pds):
        return shapes
    return None
