"""Geometric node aggregates on a structured node grid.

Smoothed aggregation groups nodes into disjoint aggregates, one coarse node
each (Sec. 2.2).  The workloads fix aggregates to cubes of 3x3x3 nodes.  Per
direction with m nodes there are n_a = max(1, floor(m/3)) aggregates and node
i belongs to min(floor(i/3), n_a - 1): a remainder of one or two nodes joins
the last aggregate.  Coarse levels apply the same rule to the grid of
aggregates.  Nodes and aggregates are numbered x fastest, then y, then z.
"""
from __future__ import annotations

import numpy as np


def aggregate_1d(m: int) -> tuple[np.ndarray, int]:
    n_a = max(1, m // 3)
    return np.minimum(np.arange(m) // 3, n_a - 1), n_a


def aggregates(grid: tuple[int, int, int]) -> tuple[np.ndarray, tuple[int, int, int]]:
    """Aggregate id of every node of ``grid`` and the coarse grid shape."""
    mx, my, mz = grid
    ax, nax = aggregate_1d(mx)
    ay, nay = aggregate_1d(my)
    az, naz = aggregate_1d(mz)
    n = np.arange(mx * my * mz, dtype=np.int64)
    ix, iy, iz = n % mx, (n // mx) % my, n // (mx * my)
    agg = ax[ix] + nax * (ay[iy] + nay * az[iz])
    return agg.astype(np.int64), (nax, nay, naz)
