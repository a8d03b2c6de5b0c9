"""GPU: the source-sharded driver (sharded.brandes_sharded / brandes_pp_sharded) with two ranks.

This run has one GPU, so the two ranks are two processes on the same device with a gloo process
group (their kernels never wait on each other; the only exchange is the host-side all-reduce of
the FP64 partial sums).  Each rank computes its shard of the sources through the library's C ABI
and must end up with the oracle's full betweenness, for plain Brandes and Brandes++, FP64."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import paper_1406_4173_gb300 as bc
    from paper_1406_4173_gb300 import gen, sharded
    g = gen.chung_lu_communities(3000, [500] * 6, 2.3, 8.0, 0.9, seed=71, wmax=5)
    S = gen.sample_targets(g.n, 900, seed=72)
    G = bc.graph_from_edgelist(g)
    plain = sharded.brandes_sharded(G, S).cpu().numpy()
    pp = sharded.brandes_pp_sharded(G, S, g.part).cpu().numpy()
    mine = bc.brandes(G, S, shard=(rank, world)).cpu().numpy()
    np.save(out_path + f".{rank}.npy", np.stack([plain, pp, mine]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_driver_two_ranks_one_gpu(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from paper_1406_4173_gb300 import gen
    out = str(tmp_path / "res")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    g = gen.chung_lu_communities(3000, [500] * 6, 2.3, 8.0, 0.9, seed=71, wmax=5)
    S = gen.sample_targets(g.n, 900, seed=72)
    ref, _ = oracle.brandes(g, S)
    res = [np.load(out + f".{r}.npy") for r in range(2)]
    for plain, pp, _ in res:
        assert np.max(np.abs(plain - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-12
        assert np.max(np.abs(pp - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-12
    # the ranks computed different shards, which add up
    both = res[0][2] + res[1][2]
    assert np.max(np.abs(both - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-12
    assert np.any(np.abs(res[0][2] - res[1][2]) > 0)
