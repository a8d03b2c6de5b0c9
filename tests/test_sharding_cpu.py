"""Multi-GPU source sharding, exercised on CPU with world-size-2 and -3 gloo ranks.

Each rank runs the package's sharded driver (``sharded.sharded_sum``) with the CPU oracle as
its per-rank compute: the shard's sources come from the library's own shard rule
(``bcpp_shard_bounds`` through the C ABI, which needs no GPU), the oracle computes their
partial betweenness with all of S as targets, and the driver's FP64 all-reduce sums the
partials.  Every rank must end up with the unsharded oracle result, for plain Brandes and for
Brandes++.  On GPUs the same driver runs the library's sharded calls and reduces over NCCL.
"""
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


def _oracle_shard(fn, g, S, r, R, **kw):
    """The oracle's partial sum over the sources of shard r of R (positions in S's order,
    bounds from the library), with all of S as targets."""
    from paper_1406_4173_gb300 import api
    s0, s1 = api.shard_bounds(len(S), r, R)
    mine = S[s0:s1]
    order = np.concatenate([mine, np.setdiff1d(S, mine)]).astype(np.int32)
    out = fn(g, order, nsrc=len(mine), halve=False, **kw)
    return torch.from_numpy(np.ascontiguousarray(out[0]))


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1406_4173_gb300 import gen, sharded
    g = gen.planted_partition(400, 4, 0.05, 0.004, seed=21, wmax=3)
    S = gen.sample_targets(g.n, 150, seed=21)
    plain = sharded.sharded_sum(lambda r, R: _oracle_shard(oracle.brandes, g, S, r, R))
    pp = sharded.sharded_sum(lambda r, R: _oracle_shard(oracle.brandes_pp, g, S, r, R, part=g.part))
    full, _ = oracle.brandes(g, S, halve=False)
    np.save(out_path + f".{rank}.npy", np.stack([plain.numpy(), pp.numpy(), full]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_driver_sums_to_full(tmp_path, world):
    out = str(tmp_path / "res")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        plain, pp, full = np.load(out + f".{r}.npy")
        assert np.max(np.abs(plain - full) / np.maximum(np.abs(full), 1.0)) < 1e-12
        assert np.max(np.abs(pp - full) / np.maximum(np.abs(full), 1.0)) < 1e-12


def test_library_shard_bounds_cover_exactly():
    """The library's shard rule splits [0, n) into `count` contiguous, disjoint, covering
    ranges whose sizes differ by at most one, and refuses invalid arguments."""
    from paper_1406_4173_gb300 import api
    for ns in (0, 1, 5, 63, 1563, 4096, 50000):
        for world in (1, 2, 3, 7, 8):
            cov, sizes = [], []
            for r in range(world):
                a, b = api.shard_bounds(ns, r, world)
                cov.extend(range(a, b))
                sizes.append(b - a)
            assert cov == list(range(ns))
            assert max(sizes) - min(sizes) <= 1
    assert api.shard_bounds(10, 0, 0) == (0, 10)
    for bad in ((10, 2, 2), (10, -1, 2), (-1, 0, 1)):
        with pytest.raises(api.BcppError):
            api.shard_bounds(*bad)
