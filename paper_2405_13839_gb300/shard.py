"""Sharding of independent clouds over ranks (one GPU per rank).

The clouds of a batch are independent problems: each rank orients its own
subset, with no exchange on the data path.  The assignment balances the
estimated work (longest processing time first: every cloud goes to the rank
with the least work so far, ties to the lower rank), the cost of a cloud of
n points being n log2 n (the Barnes-Hut evaluation; the all-pairs path of
small clouds is cheaper than that bound).  Results travel only to collect
them on one rank, outside the timed region.
"""
from __future__ import annotations

import math

import numpy as np


def cloud_cost(n: int) -> float:
    return float(n) * math.log2(max(n, 2))


def assign(sizes, world: int):
    """Cloud indices of each rank (each list ascending); every cloud once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    out = [[] for _ in range(world)]
    order = sorted(range(len(sizes)), key=lambda c: (-cloud_cost(int(sizes[c])), c))
    for c in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(c)
        load[r] += cloud_cost(int(sizes[c]))
    return [sorted(v) for v in out]


def sub_batch(points, offsets, clouds):
    """Points and offsets of a subset of the clouds (in the given order)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    parts = [points[offsets[c]:offsets[c + 1]] for c in clouds]
    sub_off = np.zeros(len(clouds) + 1, dtype=np.int64)
    sub_off[1:] = np.cumsum([len(p) for p in parts])
    pts = np.ascontiguousarray(np.vstack(parts)) if parts else np.zeros((0, 3), points.dtype)
    return pts, sub_off


def gather_normals(local, clouds, offsets, total, group=None):
    """Assemble every rank's per-cloud normals into the input layout on all
    ranks (torch.distributed all_gather_object: the host path, used once
    after the timed region)."""
    import torch.distributed as dist
    offsets = np.asarray(offsets, dtype=np.int64)
    world = dist.get_world_size(group)
    items = [None] * world
    dist.all_gather_object(items, (list(clouds), np.asarray(local)), group=group)
    out = np.zeros((total, 3), dtype=np.float32)
    for cl, arr in items:
        o = 0
        for c in cl:
            n = int(offsets[c + 1] - offsets[c])
            out[offsets[c]:offsets[c + 1]] = arr[o:o + n]
            o += n
    return out
