"""Multi-GPU layout: independent voxel slabs, no data exchange.

Voxels are independent in delay-and-sum (each output depends only on the shared IQ), so
a job splits into contiguous voxel slabs, one per rank, with no collective on the data
path; Power Doppler is per voxel as well.  The only collective is the timing reduction
(maximum over ranks) used by the benchmark.
"""
from __future__ import annotations

from typing import List, Tuple


def voxel_slabs(n_vox: int, world: int) -> List[Tuple[int, int]]:
    """[start, stop) voxel ranges, contiguous, covering 0..n_vox exactly once, sizes
    differing by at most one."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(int(n_vox), world)
    out, s = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((s, s + n))
        s += n
    return out


def z_slabs(grid_dims, world: int) -> List[Tuple[int, int]]:
    """Split a regular grid along z (whole x-y planes per rank): [z_start, z_stop)."""
    return voxel_slabs(int(grid_dims[2]), world)


def max_over_ranks(x: float) -> float:
    """Maximum of a host scalar over the default process group (identity when not
    distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
