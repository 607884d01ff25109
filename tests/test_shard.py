"""The multi-GPU host logic on CPU: the size-balanced split of a batch's
instances, and a world-size-2 gloo run of the batched data flow (split,
solve each share, max-over-ranks timing, one gather of the edge blocks at
rank 0).  The per-rank solve is the oracle here, since these ranks have no
GPU; the GPU path runs the same steps with emst_compute_batched."""
from __future__ import annotations

import os

import numpy as np
import pytest

from paper_2207_00514_gb300 import shard


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_covers_every_instance_once_and_balances(world):
    sizes = np.random.default_rng(world).integers(1, 10_000, size=257)
    parts = shard.partition_instances(sizes, world)
    assert len(parts) == world
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(len(sizes)))
    loads = np.array([sizes[p].sum() for p in parts])
    # longest-first greedy: no rank exceeds another by more than one instance
    assert loads.max() - loads.min() <= sizes.max()
    # deterministic
    again = shard.partition_instances(sizes, world)
    assert all(np.array_equal(a, b) for a, b in zip(parts, again))


def test_partition_edge_cases():
    assert [len(p) for p in shard.partition_instances([], 2)] == [0, 0]
    p = shard.partition_instances([5], 3)
    assert [list(x) for x in p] == [[0], [], []]
    with pytest.raises(ValueError):
        shard.partition_instances([1, 2], 0)


def test_local_batch_slices_instances():
    pts = np.arange(20, dtype=np.float32).reshape(10, 2)
    offs = np.array([0, 3, 3, 7, 10])
    sub, so = shard.local_batch(pts, offs, [2, 0])
    assert np.array_equal(sub, np.concatenate([pts[3:7], pts[0:3]]))
    assert list(so) == [0, 4, 7]
    sub, so = shard.local_batch(pts, offs, [])
    assert len(sub) == 0 and list(so) == [0]


def _solve_share(rank, world, out_dir):
    """One rank: the batched flow with the oracle standing in for the GPU."""
    import torch.distributed as dist

    import oracle
    import synth
    # rendezvous through a file: no port to race for
    dist.init_process_group("gloo", init_method="file://" + os.path.join(out_dir, "rendezvous"),
                            rank=rank, world_size=world)
    try:
        sizes = synth.batched_sizes(24, seed=7, lo=2, hi=300)
        pts, offs = synth.batched_instances(sizes, seed=7)
        mine = shard.partition_instances(sizes, world)[rank]
        lp, lo = shard.local_batch(pts, offs, mine)
        blocks = [oracle.prim(lp[lo[s]:lo[s + 1]]) for s in range(len(mine))]
        eo = np.concatenate([[0], np.cumsum([len(b) for b in blocks])]).astype(np.int64)
        edges = np.concatenate(blocks) if blocks else np.zeros(0, oracle.EDGE_DTYPE)
        slowest = shard.max_over_ranks(1.5 + rank)
        shard.barrier()
        got = shard.gather_edge_blocks(edges, eo, mine, len(sizes))
        np.save(os.path.join(out_dir, f"max_{rank}.npy"), np.array([slowest]))
        if rank == 0:
            e, o = got
            np.save(os.path.join(out_dir, "edges.npy"), e)
            np.save(os.path.join(out_dir, "offs.npy"), o)
        else:
            assert got is None
    finally:
        dist.destroy_process_group()


def test_world_size_2_gloo_batched_flow(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle
    import synth
    mp.start_processes(_solve_share, args=(2, str(tmp_path)), nprocs=2,
                       join=True, start_method="spawn")
    for r in range(2):
        assert float(np.load(tmp_path / f"max_{r}.npy")[0]) == 2.5
    e = np.load(tmp_path / "edges.npy")
    o = np.load(tmp_path / "offs.npy")
    sizes = synth.batched_sizes(24, seed=7, lo=2, hi=300)
    pts, offs = synth.batched_instances(sizes, seed=7)
    for k in range(len(sizes)):
        want = oracle.prim(pts[offs[k]:offs[k + 1]])
        assert np.array_equal(e[o[k]:o[k + 1]].view(np.uint8), want.view(np.uint8)), k
    assert o[-1] == sum(max(int(s) - 1, 0) for s in sizes)
