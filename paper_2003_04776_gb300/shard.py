"""Sharding of one solve over several GPUs (host logic only).

The task graph of Algorithm 1 is a disjoint union of one sub-graph per block
column (Section 5.3): the eigenvectors are independent units.  A multi-GPU
solve therefore replicates S and T on every rank, gives each rank a selection
of eigenvectors with about equal work, and needs no exchange during the solve;
V comes back column-sharded (or is gathered once).  The work of the
eigenvector whose block starts at diagonal position c is the substitution
over the c rows above it, about 2 c^2 flops per column, so the shares balance
sum c^2, not counts.  A complex pair (a 2x2 block) is one unit: its two
columns always land on the same rank.
"""
from __future__ import annotations

import numpy as np


def block_pattern(subdiag: np.ndarray, n: int) -> np.ndarray:
    """Block pattern from the subdiagonal of S: 0 for a 1x1 block, 1 and 2 for
    the first and second row of a 2x2 block."""
    blk = np.zeros(n, dtype=np.int8)
    i = 0
    while i < n:
        if i + 1 < n and subdiag[i] != 0.0:
            blk[i], blk[i + 1] = 1, 2
            i += 2
        else:
            i += 1
    return blk


def unit_work(blk: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Start position and work (sum over the unit's columns of 2 (c+1)^2) of
    every eigenvector unit in diagonal order."""
    blk = np.asarray(blk)
    starts = np.flatnonzero(blk != 2)
    sizes = np.where(blk[starts] == 1, 2, 1)
    c = starts.astype(np.float64)
    work = 2.0 * (c + 1.0) ** 2
    work = np.where(sizes == 2, work + 2.0 * (c + 2.0) ** 2, work)
    return starts, work


def column_shards(blk: np.ndarray, world: int) -> list[np.ndarray]:
    """Selections (int32[n] masks, nonzero = selected) for `world` ranks:
    contiguous runs of units along the diagonal with about equal work each.
    Every unit is selected on exactly one rank."""
    blk = np.asarray(blk)
    n = blk.size
    starts, work = unit_work(blk)
    masks = [np.zeros(n, dtype=np.int32) for _ in range(world)]
    if starts.size == 0:
        return masks
    cum = np.cumsum(work)
    total = cum[-1]
    # rank r takes the units whose cumulative work ends in (r/world, (r+1)/world] of the total
    owner = np.minimum((np.ceil(cum / total * world) - 1).astype(np.int64), world - 1)
    owner = np.maximum(owner, 0)
    for u, c in enumerate(starts):
        masks[int(owner[u])][c] = 1
    return masks


def shard_balance(blk: np.ndarray, masks: list[np.ndarray]) -> np.ndarray:
    """Work of every rank's selection (for reporting and tests)."""
    starts, work = unit_work(blk)
    return np.array([float(work[m[starts] != 0].sum()) for m in masks])
