"""Seeded synthetic graph generators.

This module only produces inputs: edge lists, node partitions and target sets.  It holds
none of the betweenness arithmetic, so the CUDA path and the CPU oracle can both be fed
from it without sharing any of the method's code.

Every generator draws from a numpy PCG64 stream seeded by ``(seed, stream-id)``.  Graphs
are simple: self-loops and repeated edges are rejected and redrawn.  Undirected graphs are
returned with each edge once as ``u < v``; directed graphs as ordered arcs ``u -> v``.
Node ids are laid out community by community, so the planted partition of a graph is a
set of contiguous id ranges.

The workload families stand in for the paper's real datasets (Sec. 6), which are not
available: planted-partition and Chung-Lu graphs with planted communities give the
community structure that the skeleton method relies on (Sec. 6, graph partitioning).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "EdgeList", "rng_for", "path", "star", "cycle", "complete", "complete_bipartite",
    "grid", "erdos_renyi", "planted_partition", "powerlaw_sizes", "chung_lu_communities",
    "er_batch", "with_weights", "sample_targets", "random_partition", "workload", "WORKLOADS",
]


@dataclass
class EdgeList:
    """A simple graph as an edge list.

    n        -- number of nodes
    src, dst -- int32 endpoints (undirected: one entry per edge, src < dst)
    w        -- uint32 weights >= 1, or None for an unweighted graph
    directed -- arcs are src -> dst when True
    part     -- int32 planted community of each node, or None
    """
    n: int
    src: np.ndarray
    dst: np.ndarray
    w: np.ndarray | None = None
    directed: bool = False
    part: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def num_parts(self) -> int:
        return 0 if self.part is None else int(self.part.max()) + 1 if self.n else 0


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def _finish(n, keys, directed, rng, wmax, part=None, meta=None) -> EdgeList:
    src = (keys // n).astype(np.int32)
    dst = (keys % n).astype(np.int32)
    w = None
    if wmax is not None:
        w = rng.integers(1, int(wmax) + 1, size=src.shape[0], dtype=np.int64).astype(np.uint32)
    return EdgeList(n=int(n), src=src, dst=dst, w=w, directed=bool(directed),
                    part=None if part is None else np.ascontiguousarray(part, dtype=np.int32),
                    meta=dict(meta or {}))


def _canon(u, v, n, directed):
    u = u.astype(np.int64)
    v = v.astype(np.int64)
    if not directed:
        lo = np.minimum(u, v)
        hi = np.maximum(u, v)
        u, v = lo, hi
    return u * n + v


def _from_pairs(n, u, v, directed, rng=None, wmax=None, part=None, meta=None) -> EdgeList:
    keys = _canon(np.asarray(u), np.asarray(v), n, directed)
    keys = keys[(keys // n) != (keys % n)]
    keys = np.unique(keys)
    return _finish(n, keys, directed, rng if rng is not None else rng_for(0, 99), wmax, part, meta)


# ----------------------------------------------------------------------------- closed-form families
def path(n: int) -> EdgeList:
    i = np.arange(n - 1)
    return _from_pairs(n, i, i + 1, False)


def star(n: int) -> EdgeList:
    i = np.arange(1, n)
    return _from_pairs(n, np.zeros_like(i), i, False)


def cycle(n: int) -> EdgeList:
    i = np.arange(n)
    return _from_pairs(n, i, (i + 1) % n, False)


def complete(n: int) -> EdgeList:
    u, v = np.triu_indices(n, 1)
    return _from_pairs(n, u, v, False)


def complete_bipartite(a: int, b: int) -> EdgeList:
    u, v = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return _from_pairs(a + b, u.ravel(), v.ravel(), False)


def grid(rows: int, cols: int) -> EdgeList:
    """rows x cols lattice; node (r, c) has id r * cols + c."""
    ids = np.arange(rows * cols).reshape(rows, cols)
    us = [ids[:, :-1].ravel(), ids[:-1, :].ravel()]
    vs = [ids[:, 1:].ravel(), ids[1:, :].ravel()]
    return _from_pairs(rows * cols, np.concatenate(us), np.concatenate(vs), False)


# ----------------------------------------------------------------------------- random families
def _sample_distinct(rng, n, count, draw, directed):
    """Draw edges with ``draw(k) -> (u, v)`` until ``count`` distinct non-loop edges exist.

    Keeps edges in the order they were first drawn, so trimming to ``count`` is stable.
    """
    keys = np.zeros(0, dtype=np.int64)
    rounds = 0
    while keys.shape[0] < count:
        need = count - keys.shape[0]
        u, v = draw(int(need * 1.15) + 16)
        k = _canon(u, v, n, directed)
        k = k[(k // n) != (k % n)]
        allk = np.concatenate([keys, k])
        _, first = np.unique(allk, return_index=True)
        keys = allk[np.sort(first)]
        rounds += 1
        if rounds > 200:
            raise RuntimeError("edge sampler did not converge (graph too dense for its size)")
    return keys[:count]


def erdos_renyi(n: int, p: float, seed: int, directed: bool = False, wmax: int | None = None,
                stream: int = 1) -> EdgeList:
    """G(n, p): the edge count is Binomial(#pairs, p), then that many distinct pairs."""
    rng = rng_for(seed, stream)
    pairs = n * (n - 1) if directed else n * (n - 1) // 2
    count = int(rng.binomial(pairs, p)) if pairs > 0 else 0
    if count == 0:
        return _finish(n, np.zeros(0, np.int64), directed, rng, wmax)

    def draw(k):
        return rng.integers(0, n, k), rng.integers(0, n, k)

    keys = np.sort(_sample_distinct(rng, n, count, draw, directed))
    return _finish(n, keys, directed, rng, wmax)


def planted_partition(n: int, k: int, p_in: float, p_out: float, seed: int,
                      wmax: int | None = None, stream: int = 2) -> EdgeList:
    """k equal communities of contiguous ids; each pair is an edge with p_in inside a
    community and p_out across communities."""
    rng = rng_for(seed, stream)
    size = n // k
    bounds = [(c * size, (c + 1) * size if c < k - 1 else n) for c in range(k)]
    part = np.zeros(n, np.int32)
    for c, (a, b) in enumerate(bounds):
        part[a:b] = c
    keys = []
    for a in range(k):
        for b in range(a, k):
            lo_a, hi_a = bounds[a]
            lo_b, hi_b = bounds[b]
            na, nb = hi_a - lo_a, hi_b - lo_b
            if a == b:
                npairs, p = na * (na - 1) // 2, p_in
            else:
                npairs, p = na * nb, p_out
            cnt = int(rng.binomial(npairs, p)) if npairs else 0
            if cnt == 0:
                continue
            idx = rng.choice(npairs, size=cnt, replace=False)
            if a == b:
                iu, iv = np.triu_indices(na, 1)
                u, v = iu[idx] + lo_a, iv[idx] + lo_a
            else:
                u, v = idx // nb + lo_a, idx % nb + lo_b
            keys.append(_canon(u, v, n, False))
    keys = np.sort(np.concatenate(keys)) if keys else np.zeros(0, np.int64)
    return _finish(n, keys, False, rng, wmax, part,
                   meta=dict(family="planted_partition", k=k, p_in=p_in, p_out=p_out))


def powerlaw_sizes(n: int, k: int, exponent: float, min_size: int, seed: int, stream: int = 3) -> np.ndarray:
    """k community sizes drawn from a power law with the given exponent (Pareto shape
    exponent-1), scaled to sum to n, clamped below at min_size, rounded by largest remainder."""
    rng = rng_for(seed, stream)
    raw = (1.0 - rng.random(k)) ** (-1.0 / (exponent - 1.0))
    frac = raw / raw.sum() * n
    fixed = np.zeros(k, bool)
    for _ in range(k):
        small = (frac < min_size) & ~fixed
        if not small.any():
            break
        fixed |= small
        frac[fixed] = min_size
        rest = ~fixed
        frac[rest] = raw[rest] / raw[rest].sum() * (n - min_size * fixed.sum())
    base = np.floor(frac).astype(np.int64)
    rem = n - base.sum()
    order = np.argsort(-(frac - base), kind="stable")
    base[order[:rem]] += 1
    return np.sort(base)[::-1].copy()


def _powerlaw_weights(rng, n, exponent, mean, cap):
    w = (1.0 - rng.random(n)) ** (-1.0 / (exponent - 1.0))
    w *= mean / w.mean()
    return np.minimum(w, cap)


def chung_lu_communities(n: int, sizes, exponent: float, mean_degree: float, intra: float,
                         seed: int, directed: bool = False, wmax: int | None = None,
                         stream: int = 4) -> EdgeList:
    """Chung-Lu graph with planted communities.

    Expected-degree weights follow a power law with the given exponent, scaled to the mean
    degree and capped at sqrt(n * mean).  The edge count is n*mean/2 (undirected) or n*mean
    (directed, mean = out-degree).  Each edge picks its first endpoint in proportion to the
    (out-)weights; with probability ``intra`` the second endpoint is drawn in proportion to
    the (in-)weights inside the first endpoint's community, otherwise among the other
    communities.  Communities are contiguous id ranges of the given sizes.
    """
    rng = rng_for(seed, stream)
    sizes = np.asarray(sizes, np.int64)
    assert sizes.sum() == n
    k = sizes.shape[0]
    off = np.concatenate([[0], np.cumsum(sizes)])
    part = np.repeat(np.arange(k, dtype=np.int32), sizes)
    cap = math.sqrt(n * mean_degree)
    w_out = _powerlaw_weights(rng, n, exponent, mean_degree, cap)
    w_in = _powerlaw_weights(rng, n, exponent, mean_degree, cap) if directed else w_out
    c_out = np.concatenate([[0.0], np.cumsum(w_out)])
    c_in = np.concatenate([[0.0], np.cumsum(w_in)])
    m = int(round(n * mean_degree)) if directed else int(round(n * mean_degree / 2))

    def pick(cum, lo, hi, r):
        # node in [lo, hi) with probability proportional to its weight (cum = prefix sums)
        x = cum[lo] + r * (cum[hi] - cum[lo])
        v = np.searchsorted(cum, x, side="right") - 1
        return np.clip(v, lo, hi - 1)

    def draw(cnt):
        u = pick(c_out, np.zeros(cnt, np.int64), np.full(cnt, n, np.int64), rng.random(cnt))
        cu = part[u]
        inside = rng.random(cnt) < intra
        v = np.empty(cnt, np.int64)
        lo, hi = off[cu], off[cu + 1]
        v[inside] = pick(c_in, lo[inside], hi[inside], rng.random(int(inside.sum())))
        out = np.nonzero(~inside)[0]
        tries = 0
        while out.size and tries < 64:
            cand = pick(c_in, np.zeros(out.size, np.int64), np.full(out.size, n, np.int64),
                        rng.random(out.size))
            ok = part[cand] != cu[out]
            v[out[ok]] = cand[ok]
            out = out[~ok]
            tries += 1
        v[out] = u[out]          # give up: becomes a self-loop and is rejected
        return u, v

    keys = np.sort(_sample_distinct(rng, n, m, draw, directed))
    return _finish(n, keys, directed, rng, wmax, part,
                   meta=dict(family="chung_lu_communities", exponent=exponent,
                             mean_degree=mean_degree, intra=intra, k=int(k)))


def er_batch(num_graphs: int, median: float, sigma: float, lo: int, hi: int, mean_degree: float,
             seed: int, stream: int = 5) -> list[EdgeList]:
    """Independent undirected G(n, p) graphs with n log-normal (median, sigma) clipped to
    [lo, hi] and p = mean_degree / (n - 1)."""
    rng = rng_for(seed, stream)
    ns = np.clip(np.round(np.exp(rng.normal(math.log(median), sigma, num_graphs))), lo, hi).astype(int)
    out = []
    for g, n in enumerate(ns):
        out.append(erdos_renyi(int(n), mean_degree / (n - 1), seed=seed * 1000003 + g, stream=stream + 1))
    return out


def with_weights(g: EdgeList, wmax: int, seed: int, stream: int = 9) -> EdgeList:
    """A copy of ``g`` with integer edge weights drawn uniformly from [1, wmax]."""
    rng = rng_for(seed, stream)
    w = rng.integers(1, int(wmax) + 1, size=g.m, dtype=np.int64).astype(np.uint32)
    return EdgeList(n=g.n, src=g.src.copy(), dst=g.dst.copy(), w=w, directed=g.directed,
                    part=None if g.part is None else g.part.copy(), meta=dict(g.meta))


def sample_targets(n: int, size: int, seed: int, stream: int = 7) -> np.ndarray:
    """Target set S: ``size`` distinct nodes drawn uniformly, returned sorted."""
    rng = rng_for(seed, stream)
    return np.sort(rng.choice(n, size=size, replace=False)).astype(np.int32)


def random_partition(n: int, k: int, seed: int, stream: int = 8) -> np.ndarray:
    rng = rng_for(seed, stream)
    return rng.integers(0, k, n).astype(np.int32)


# ----------------------------------------------------------------------------- named workloads
def _w_planted_2k(seed=0):
    g = planted_partition(2000, 8, 0.02, 0.0005, seed)
    return g, np.arange(g.n, dtype=np.int32)


def _w_chunglu_50k(seed=0):
    sizes = powerlaw_sizes(50_000, 50, 2.5, 64, seed)
    g = chung_lu_communities(50_000, sizes, 2.3, 10.0, 0.90, seed)
    return g, np.arange(g.n, dtype=np.int32)


def _w_directed_100k(seed=0):
    sizes = np.full(200, 500)
    g = chung_lu_communities(100_000, sizes, 2.3, 12.0, 0.90, seed, directed=True, wmax=16)
    return g, sample_targets(g.n, 2000, seed)


def _w_directed_20k(seed=0):
    sizes = np.full(40, 500)
    g = chung_lu_communities(20_000, sizes, 2.3, 12.0, 0.90, seed, directed=True, wmax=16)
    return g, sample_targets(g.n, 400, seed)


def _w_chunglu_1m(seed=0):
    sizes = np.full(1000, 1000)
    g = chung_lu_communities(1_000_000, sizes, 2.2, 16.0, 0.85, seed)
    return g, sample_targets(g.n, 4096, seed)


def _w_chunglu_100k(seed=0):
    sizes = np.full(100, 1000)
    g = chung_lu_communities(100_000, sizes, 2.2, 16.0, 0.85, seed)
    return g, sample_targets(g.n, 512, seed)


def _w_chunglu_10k(seed=0):
    g = chung_lu_communities(10_000, np.full(10, 1000), 2.3, 10.0, 0.90, seed)
    return g, np.arange(g.n, dtype=np.int32)


def _w_planted_200k(seed=0):
    g = planted_partition(200_000, 100, 0.005, 9e-8, seed)
    return g, sample_targets(g.n, 200, seed)


def _w_er_batch_4096(seed=0):
    return er_batch(4096, 512, 0.75, 64, 4096, 8.0, seed), None


WORKLOADS = {
    # name: (builder, description)
    "planted_2k": (_w_planted_2k, "planted partition n=2,000, 8x250, p_in=0.02, p_out=0.0005, S=V"),
    "chunglu_50k": (_w_chunglu_50k, "Chung-Lu n=50,000, 50 power-law communities (2.5), degree exp 2.3, "
                                    "mean 10, 90% intra, S=V"),
    "directed_100k": (_w_directed_100k, "directed Chung-Lu n=100,000, 200x500 communities, out-degree 12, "
                                        "exp 2.3, 90% intra, w~U[1,16], |S|=2,000"),
    "er_batch_4096": (_w_er_batch_4096, "4,096 G(n, 8/(n-1)) graphs, n log-normal median 512 sigma 0.75 "
                                        "clipped [64,4096], full BC each"),
    "chunglu_10k": (_w_chunglu_10k, "Chung-Lu n=10,000, 10x1,000 communities, degree exp 2.3, mean 10, "
                                    "90% intra, S=V (the small case of full profiler captures)"),
    "planted_200k": (_w_planted_200k, "planted partition n=200,000, 100x2,000, p_in=0.005, p_out=9e-8 "
                                      "(about 1,800 inter-community edges), |S|=200: a small skeleton "
                                      "(N/n about 3%, M/m about 16%)"),
    "directed_20k": (_w_directed_20k, "the directed_100k recipe at n=20,000: 40x500 communities, out-degree 12, "
                                      "exp 2.3, 90% intra, w~U[1,16], |S|=400 (the small case of full profiler "
                                      "captures of the integer-weight passes)"),
    "chunglu_100k": (_w_chunglu_100k, "the chunglu_1m recipe at n=100,000: 100x1,000 communities, degree exp "
                                      "2.2, mean 16, 85% intra, |S|=512 (the small case of full profiler "
                                      "captures of Brandes_SK and Centrality)"),
    "chunglu_1m": (_w_chunglu_1m, "Chung-Lu n=1,000,000, 1,000x1,000 communities, degree exp 2.2, mean 16, "
                                  "85% intra, |S|=4,096"),
}


def workload(name: str, seed: int = 0):
    """Return ``(graph_or_list, S)`` for a named workload (S=None for the batch workload)."""
    return WORKLOADS[name][0](seed)
