"""Source-sharded betweenness over several processes, one GPU each.

Betweenness with respect to a target set S is a sum over the sources s in S of independent
single-source dependencies (Sec. 3, Eq. 5-7; Alg. 1 runs Brandes_SK and the Centrality step
per source), so R ranks can split the sources: rank r computes the partial sum of shard r of R
(the library's ``shard=(r, R)`` option, whose bounds ``api.shard_bounds`` returns) on its own
replica of the graph (and, for Brandes++, of the skeleton, which every rank builds), and one
FP64 sum all-reduce of the n partial sums gives every rank the full result.  That all-reduce is
the only exchange.

``sharded_sum`` is the driver: it runs a per-rank compute function and reduces its result
over a ``torch.distributed`` process group (NCCL for GPU tensors; gloo works for CPU tensors).
``brandes_sharded`` and ``brandes_pp_sharded`` plug in the library's calls.  The shard of a
rank covers the targets in the library's batch order, which depends only on the graph and S,
so every rank derives the same order and the shards are disjoint and cover S.
"""
from __future__ import annotations

from typing import Callable

from . import api


def _dist():
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        raise RuntimeError("sharded betweenness needs an initialized torch.distributed process group")
    return dist


def sharded_sum(compute: Callable[[int, int], "object"], group=None):
    """Run ``compute(rank, world)`` on every rank of ``group`` and sum the returned float64
    tensors over the ranks (in place, FP64 all-reduce).  Returns the summed tensor on every
    rank.  ``compute`` returns rank's partial sum: its shard's sources, all of S as targets."""
    import torch
    dist = _dist()
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    part = compute(rank, world)
    if not isinstance(part, torch.Tensor) or part.dtype != torch.float64:
        raise TypeError("the per-rank compute must return a float64 tensor")
    if world > 1:
        dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    return part


def brandes_sharded(G: api.Graph, S=None, precision: str = "fp64", halve: bool = True, group=None,
                    ctx: api.Context | None = None, out=None, **kw):
    """Plain Brandes (Eq. 5-7) with the sources split across the ranks of ``group``: every
    rank passes its replica of G (and the same S) and receives the full result."""
    return sharded_sum(lambda r, R: api.brandes(G, S, precision=precision, halve=halve, ctx=ctx, out=out,
                                                shard=(r, R), **kw), group)


def brandes_pp_sharded(G: api.Graph, S, part, k: int | None = None, precision: str = "fp64", halve: bool = True,
                       group=None, ctx: api.Context | None = None, out=None, **kw):
    """Brandes++ (Alg. 1) with the sources split across the ranks of ``group``: every rank
    builds the skeleton of (G, S, part), runs Brandes_SK and the Centrality step for its shard
    of the sources, and receives the full result."""
    return sharded_sum(lambda r, R: api.brandes_pp(G, S, part, k=k, precision=precision, halve=halve, ctx=ctx,
                                                   out=out, shard=(r, R), **kw), group)
