"""Window segments for several GPUs without cross-GPU communication.

The paper partitions the alchemical path into small overlapping segments, one
per GPU, duplicating the boundary window so that GPUs never exchange
coordinates, energies or replica information (section "Simulation protocol";
its example: windows [1, 8] on GPU-0 and [8, 15] on GPU-1). MBAR then runs per
segment and the segment free energies are summed.
"""
from __future__ import annotations

from typing import List, Tuple


def segment_windows(n_windows: int, n_gpus: int) -> List[Tuple[int, int]]:
    """Inclusive 0-based window ranges [first, last] per GPU; adjacent segments
    share exactly one window and together they cover 0 .. n_windows-1."""
    if n_windows < 1 or n_gpus < 1:
        raise ValueError("need at least one window and one GPU")
    n = min(n_gpus, max(1, n_windows - 1))
    bounds = [round(i * (n_windows - 1) / n) for i in range(n + 1)]
    segs = [(bounds[i], bounds[i + 1]) for i in range(n)]
    if n_windows == 1:
        segs = [(0, 0)]
    return segs + [segs[-1]] * (n_gpus - n)


def rank_windows(n_windows: int, world_size: int, rank: int) -> List[int]:
    a, b = segment_windows(n_windows, world_size)[rank]
    return list(range(a, b + 1))
