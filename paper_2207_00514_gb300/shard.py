"""Host-side logic of runs on several GPUs, one process per GPU.

A single EMST does not shard: every Boruvka round (Algorithm 1) needs all
component labels and the whole hierarchy, so N GPUs run N independent
replicas.  The batched form does shard: its instances are independent
problems, so they are split across ranks by size, each rank solves its share
with one batched call, and the edge blocks are gathered once at the end.
There is no collective inside the method; the only cross-rank traffic is the
timing reduction and that final gather.

Everything here works on any torch.distributed backend (nccl on GPUs, gloo
on CPU) and on a single process without one.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition_instances(sizes, world: int) -> list[np.ndarray]:
    """Split instances across `world` ranks, balancing the points per rank
    (longest first, each to the least-loaded rank; ties to the lower rank).
    Returns one sorted array of instance indices per rank; every instance is
    in exactly one."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.lexsort((np.arange(len(sizes)), -sizes))  # largest first, stable
    heap = [(0, r) for r in range(world)]
    share: list[list[int]] = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        share[r].append(int(k))
        heapq.heappush(heap, (load + int(sizes[k]), r))
    return [np.array(sorted(s), dtype=np.int64) for s in share]


def local_batch(points, offsets, indices):
    """The rows and offsets of the instances `indices` of a batch (points
    concatenated by instance, offsets[k]..offsets[k+1] = instance k)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    idx = np.asarray(indices, dtype=np.int64)
    if len(idx) == 0:
        return points[:0], np.zeros(1, dtype=np.int64)
    parts = [points[offsets[k]:offsets[k + 1]] for k in idx]
    sizes = offsets[idx + 1] - offsets[idx]
    local_offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    if isinstance(points, np.ndarray):
        return np.concatenate(parts, axis=0), local_offsets
    import torch
    return torch.cat(parts, dim=0), local_offsets


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def max_over_ranks(x: float, device=None) -> float:
    """The largest of every rank's `x` (the job's time is its slowest
    rank's).  `device`: where the reduction tensor lives (a CUDA device for
    nccl, None for gloo)."""
    dist = _dist()
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None) -> None:
    dist = _dist()
    if dist is None:
        return
    if device is not None and getattr(device, "type", None) == "cuda":
        dist.barrier(device_ids=[device.index or 0])
    else:
        dist.barrier()


def gather_edge_blocks(edges: np.ndarray, edge_offsets, indices, num_instances: int):
    """Rank 0 receives every rank's edge blocks and returns the whole batch's
    edges in instance order with their offsets; other ranks return None.
    `edges` / `edge_offsets`: this rank's output for its instances
    `indices` (in that order)."""
    dist = _dist()
    mine = (np.asarray(indices, dtype=np.int64), np.asarray(edges),
            np.asarray(edge_offsets, dtype=np.int64))
    if dist is None:
        parts = [mine]
    else:
        parts = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
        dist.gather_object(mine, parts, dst=0)
        if dist.get_rank() != 0:
            return None
    blocks: list = [None] * num_instances
    for idx, e, eo in parts:
        for slot, k in enumerate(idx):
            blocks[int(k)] = e[eo[slot]:eo[slot + 1]]
    if any(b is None for b in blocks):
        raise ValueError("an instance is missing from every rank's share")
    counts = np.array([len(b) for b in blocks], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    dtype = parts[0][1].dtype
    out = np.concatenate(blocks) if len(blocks) else np.zeros(0, dtype=dtype)
    return out, offs
