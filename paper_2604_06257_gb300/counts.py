"""Workload accounting: delay-and-sum point counts (Eq. 1) and memory (Eq. 2, Table 3).

Host-side helpers used by the benchmark and the tests; no GPU work here.
"""
from __future__ import annotations

COMPLEX64 = 8
FLOAT32 = 4


def points(voxels: int, channels: int, compounding: int = 1, frames: int = 1) -> int:
    """Eq. 1 numerator: voxels x channels x compounding x frames."""
    return int(voxels) * int(channels) * int(compounding) * int(frames)


def throughput(voxels: int, channels: int, compounding: int, frame_rate: float) -> float:
    """Eq. 1: points per second = voxels x channels x compounding x frame rate."""
    return float(voxels) * channels * compounding * frame_rate


def memory_table(voxels: int, channels: int, samples: int, frames: int,
                 out_frames: int | None = None, transmits: int = 1,
                 iq_bytes: int = COMPLEX64) -> dict:
    """Device arrays of one beamforming call, in bytes (the rows of Table 3).

    Eq. 2: memory grows as voxels x frames (output) + channels x samples x frames (input).
    ``frames`` counts the temporal frames of the channel data (the paper folds the
    compounded transmits into it); ``out_frames`` the output volumes (default frames).
    """
    out_frames = frames if out_frames is None else out_frames
    rows = {
        "channel_data": channels * samples * frames * iq_bytes,
        "element_coords": channels * 3 * FLOAT32,
        "grid_coords": voxels * 3 * FLOAT32,
        "arrival_times": voxels * transmits * FLOAT32,
        "output": voxels * out_frames * COMPLEX64,
    }
    rows["total"] = sum(rows.values())
    return rows


def compulsory_bytes(voxels: int, channels: int, transmits: int, samples: int, frames: int,
                     iq_bytes: int = COMPLEX64, write_y: bool = True,
                     write_pd: bool = False) -> int:
    """Bytes one DAS call must move through HBM at least once: the IQ cube, the
    per-plan transmit table and voxel table (read), and the outputs (written)."""
    b = transmits * channels * samples * frames * iq_bytes      # IQ
    b += transmits * voxels * FLOAT32                           # transmit delay table
    b += voxels * 4 * FLOAT32                                   # voxel coordinates (float4)
    b += channels * 4 * FLOAT32                                 # element coordinates
    if write_y:
        b += voxels * frames * COMPLEX64
    if write_pd:
        b += voxels * FLOAT32
    return int(b)
