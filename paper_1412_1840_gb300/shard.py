"""Sharding of independent lightcurves across processes (one per GPU).

Curves are independent (the paper runs one EROS-2 chip per GPU, Section 8),
so a multi-GPU run gives each rank a contiguous range of curves and needs no
collective on the data path.  Ranges are balanced by the pair-sum cost of a
curve, N(N-1)/2 per trial frequency.  The only collectives are the timing
barrier, the max-over-ranks of elapsed time used for throughput, and (after
the timed work) the gather of each rank's per-curve results in curve order.
"""
from __future__ import annotations

import numpy as np


def curve_ranges(offsets, world: int) -> list:
    """Split curves [0, C) into `world` contiguous ranges of nearly equal total
    cost sum N(N-1)/2 (ranges may be empty when C < world)."""
    off = np.asarray(offsets, dtype=np.int64)
    n = np.diff(off).astype(np.float64)
    cost = np.concatenate([[0.0], np.cumsum(n * (n - 1) / 2)])
    total = cost[-1]
    bounds = [0]
    for r in range(1, world):
        bounds.append(int(np.searchsorted(cost, total * r / world, side="left")))
    bounds.append(len(n))
    bounds = [min(max(b, bounds[i - 1] if i else 0), len(n)) for i, b in enumerate(bounds)]
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def local_csr(times, mags, errs, offsets, rng):
    """The CSR arrays of curves [a, b) with offsets rebased to 0."""
    a, b = rng
    off = np.asarray(offsets, dtype=np.int64)
    lo, hi = int(off[a]), int(off[b])
    return times[lo:hi], mags[lo:hi], errs[lo:hi], off[a:b + 1] - lo


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar (elapsed time) over the default process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(local: dict, world: int) -> dict:
    """Concatenates every rank's per-curve result arrays (a dict of equal-length
    numpy arrays for its contiguous curve range) in rank order, which is the
    global curve order of `curve_ranges`.  Every rank receives the whole
    result.  Runs over the default process group (any backend); a host-side
    object gather, not part of the data path."""
    import torch.distributed as dist
    if world == 1 or not (dist.is_available() and dist.is_initialized()):
        return {k: np.asarray(v) for k, v in local.items()}
    parts = [None] * world
    dist.all_gather_object(parts, {k: np.asarray(v) for k, v in local.items()})
    return {k: np.concatenate([p[k] for p in parts]) for k in local}
