"""Autotuner for the per-instance lane mapping and voxel tile of ragged batches.

For one instance, every candidate (lane mapping, tile box) is timed on a one-instance
batch with CUDA events (median of a few launches after a warm-up) and the fastest kept.
Results are cached per shape signature (dimensionality, grid, elements, transmits,
frames, samples, storage type), so instances of the same shape are tuned once.
"""
from __future__ import annotations

import statistics
from typing import Dict, List, Optional, Tuple

from . import Batch

Shape = Tuple[int, int, Tuple[int, int, int]]
_CACHE: Dict[tuple, Shape] = {}


def _signature(kw: dict) -> tuple:
    grid = tuple(kw["grid_dims"]) if kw.get("grid_dims") is not None else (len(kw["vox_pos"]), 1, 1)
    return (kw["ndim"], grid, len(kw["elem_pos"]), len(kw["tx_angles"]), kw["n_frames"], kw["n_samples"],
            kw.get("iq_dtype", "c64"))


def _boxes(n: int, ndim: int) -> List[Tuple[int, int, int]]:
    """Power-of-two voxel boxes of volume n."""
    out = []
    if ndim == 2:
        x = 1
        while x <= n:
            if n % x == 0 and 2 <= x <= 64 and n // x <= 64:
                out.append((x, 1, n // x))
            x *= 2
    else:
        for x in (2, 4, 8, 16):
            for y in (1, 2, 4, 8):
                if n % (x * y) == 0 and 1 <= n // (x * y) <= 16:
                    out.append((x, y, n // (x * y)))
    return out


def candidates(kw: dict) -> List[Shape]:
    F = kw["n_frames"]
    cands: List[Shape] = []
    if F <= 4:
        cands += [(1, 0, b) for b in _boxes(32, kw["ndim"])]
    for fl in (4, 8, 16):
        if 4 * fl >= F:
            n = 8 * 4 * (32 // fl)
            cands += [(0, fl, b) for b in _boxes(n, kw["ndim"])]
    return cands


def time_shape(kw: dict, shape: Shape, iq, y, pd, reps: int = 5) -> float:
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


def tune_instance(kw: dict, iq, y, pd, max_candidates: Optional[int] = None) -> Tuple[Shape, Dict[Shape, float]]:
    sig = _signature(kw)
    if sig in _CACHE:
        return _CACHE[sig], {}
    cands = candidates(kw)
    if max_candidates:
        cands = cands[:max_candidates]
    times = {c: time_shape(kw, c, iq, y, pd) for c in cands}
    best = min(times, key=times.get)
    _CACHE[sig] = best
    return best, times


def tune_batch(instances: List[dict], iqs, ys, pds) -> List[Shape]:
    return [tune_instance(kw, iq, y, pd)[0] for kw, iq, y, pd in zip(instances, iqs, ys, pds)]
