"""Multi-GPU source sharding, exercised on CPU: world_size-2 gloo ranks each compute the
partial betweenness of their shard of sources (targets stay all of S) with the oracle, one
all-reduce sums the FP64 partials, and the sum must equal the unsharded result.  This is the
host-side logic of the sharded multi-GPU layout (each rank a GPU, one sum-reduce of bc[n])."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def shard_bounds(nsources, rank, world):
    """Contiguous shard of the sources (the library's rule for shard_index/shard_count)."""
    return nsources * rank // world, nsources * (rank + 1) // world


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1406_4173_gb300 import gen
    g = gen.planted_partition(400, 4, 0.05, 0.004, seed=21)
    S = gen.sample_targets(g.n, 150, seed=21)
    s0, s1 = shard_bounds(len(S), rank, world)
    mine = S[s0:s1]
    rest = np.setdiff1d(S, mine)
    order = np.concatenate([mine, rest]).astype(np.int32)
    part, _ = oracle.brandes(g, order, nsrc=len(mine), halve=False)
    t = torch.from_numpy(part)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        full, _ = oracle.brandes(g, S, halve=False)
        np.save(out_path, np.stack([t.numpy(), full]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_source_shards_sum_to_full(tmp_path, world):
    out = str(tmp_path / "res.npy")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    got, full = np.load(out)
    assert np.max(np.abs(got - full) / np.maximum(np.abs(full), 1.0)) < 1e-12


def test_shard_bounds_cover_exactly():
    for nb in (0, 1, 5, 63, 1563, 50000):
        for world in (1, 2, 3, 8):
            cov = []
            for r in range(world):
                a, b = shard_bounds(nb, r, world)
                cov.extend(range(a, b))
            assert cov == list(range(nb))
