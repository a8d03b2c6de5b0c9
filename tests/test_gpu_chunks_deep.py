"""GPU parity on paths that only many batches or deep weighted inputs reach.

- Brandes_SK with Centrality (Sec. 4, Eq. 11-13), with more source batches than slots: by
  default one Brandes_SK launch schedules all batches dynamically, each batch writing its own
  set of rows, and one Centrality launch covers them all; with `pp_chunks=1` (the fallback when
  memory is short) the batches run in static chunks of as many slots as fit, each chunk followed
  by the Centrality step over its slots.  Both are reached here: on small graphs with fewer
  slots (4-CTA clusters, one CTA per SM), and with the default launch shape by a target set of
  10,000 (313 batches of 32).  Brandes++ must equal the oracle's plain Brandes (the method's
  exactness, Sec. 4).
- Integer weights (Sec. 3, Eq. 2): a batch records one step per distinct settled distance, so
  deep weighted graphs (a weighted path, a weighted grid) record tens of thousands of steps per
  batch.  Distances and path counts must match the oracle bit for bit and betweenness to
  1e-12, with no capacity error.
"""
import numpy as np
import pytest

import oracle
from paper_1406_4173_gb300 import gen

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-12
FP32_TOL = 2e-6      # the FP32-delta bar of the small parity graphs


@pytest.fixture(scope="module")
def bc():
    import torch
    import paper_1406_4173_gb300 as m
    from paper_1406_4173_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    return m


def rel_err(x, ref):
    x = np.asarray(x, np.float64)
    return float(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1.0))) if x.size else 0.0


# ----------------------------------------------------------------------------- Brandes_SK chunks
def chunk_graphs():
    und = gen.planted_partition(8000, 16, 0.012, 0.00002, seed=81)
    und_w = gen.with_weights(und, 9, seed=85)
    dirw = gen.chung_lu_communities(6000, [500] * 12, 2.3, 6.0, 0.9, seed=83, directed=True, wmax=16)
    return [("undirected", und), ("undirected-w9", und_w), ("directed-w16", dirw)]


@pytest.mark.parametrize("name,g", chunk_graphs(), ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("pp_chunks", [0, 1])
def test_brandes_pp_many_batches(bc, name, g, pp_chunks):
    """2,000 targets = 63 batches; with 4-CTA clusters and one CTA per SM there are 38 slots on
    152 SMs: one dynamic pass with a row set per batch (pp_chunks=0), or two static chunks of 32
    and 31 batches (pp_chunks=1)."""
    S = gen.sample_targets(g.n, 2000, seed=82)
    G = bc.graph_from_edgelist(g)
    ref, _ = oracle.brandes(g, S)
    for cluster, cps in ((4, 1), (2, 1), (1, 1)):
        got = bc.brandes_pp(G, S, g.part, cluster=cluster, ctas_per_sm=cps, pp_chunks=pp_chunks).cpu().numpy()
        assert rel_err(got, ref) < FP64_TOL, (cluster, cps)
    got32 = bc.brandes_pp(G, S, g.part, cluster=4, ctas_per_sm=1, precision="fp32",
                          pp_chunks=pp_chunks).cpu().numpy()
    assert rel_err(got32, ref) < FP32_TOL
    # shards add up as well
    half = [bc.brandes_pp(G, S, g.part, cluster=4, ctas_per_sm=1, shard=(r, 2), halve=False,
                          pp_chunks=pp_chunks).cpu().numpy() for r in range(2)]
    ref_o, _ = oracle.brandes(g, S, halve=False)
    assert rel_err(half[0] + half[1], ref_o) < FP64_TOL


def test_brandes_pp_default_shape_many_targets(bc):
    """10,000 targets = 313 batches, more than the 304 slots of two CTAs per SM, with the default
    launch shape: one dynamic pass and static chunks."""
    g = gen.planted_partition(30000, 60, 0.012, 0.000005, seed=81)
    S = gen.sample_targets(g.n, 10000, seed=82)
    G = bc.graph_from_edgelist(g)
    ref, _ = oracle.brandes(g, S)
    pp, st = bc.brandes_pp(G, S, g.part, stats=True)
    assert st["table_entries"] > 0            # non-frontier nodes exist: Centrality runs
    assert rel_err(pp.cpu().numpy(), ref) < FP64_TOL
    assert rel_err(bc.brandes_pp(G, S, g.part, pp_chunks=1).cpu().numpy(), ref) < FP64_TOL
    assert rel_err(bc.brandes(G, S).cpu().numpy(), ref) < FP64_TOL


# ----------------------------------------------------------------------------- deep weighted graphs
def _check_sssp(bc, G, g, src):
    dist, sig = bc.sssp(G, src)
    dist, sig = dist.cpu().numpy(), sig.cpu().numpy().view(np.uint64)
    for i, s in enumerate(src):
        d_ref, s_ref, _ = oracle.sssp(g, int(s))
        assert np.array_equal(dist[i], d_ref), s
        assert np.array_equal(sig[i], s_ref), s


def test_weighted_path_3000_deep(bc):
    """A path of 3,000 nodes with weights in [1, 1000]: distances up to about 1.5 million, and
    a batch of 32 sources settles every node at up to 32 distinct distances (up to 96,000 steps
    per batch).  Betweenness on a path does not depend on the weights: i (n - 1 - i)."""
    n = 3000
    g = gen.with_weights(gen.path(n), 1000, seed=91)
    G = bc.graph_from_edgelist(g)
    _check_sssp(bc, G, g, np.array([0, 1, 1499, 2998, 2999], np.int32))
    i = np.arange(n)
    ref, _ = oracle.brandes(g)
    assert rel_err(ref, i * (n - 1 - i)) < FP64_TOL
    assert rel_err(bc.brandes(G).cpu().numpy(), ref) < FP64_TOL
    S = gen.sample_targets(n, 300, seed=92)
    ref_s, _ = oracle.brandes(g, S)
    assert rel_err(bc.brandes(G, S).cpu().numpy(), ref_s) < FP64_TOL
    blocks = (np.arange(n) * 5 // n).astype(np.int32)          # five contiguous parts
    rnd = gen.random_partition(n, 5, seed=93)                   # five random parts
    for part in (blocks, rnd):
        assert rel_err(bc.brandes_pp(G, S, part).cpu().numpy(), ref_s) < FP64_TOL
    assert rel_err(bc.brandes_pp(G, None, rnd).cpu().numpy(), ref) < FP64_TOL


def test_weighted_grid_60x60_deep(bc):
    """A 60 x 60 grid with weights in [1, 500] (distances up to about 30,000)."""
    g = gen.with_weights(gen.grid(60, 60), 500, seed=94)
    G = bc.graph_from_edgelist(g)
    _check_sssp(bc, G, g, np.array([0, 59, 1830, 3599], np.int32))
    ref, _ = oracle.brandes(g)
    assert rel_err(bc.brandes(G).cpu().numpy(), ref) < FP64_TOL
    S = gen.sample_targets(g.n, 400, seed=95)
    ref_s, _ = oracle.brandes(g, S)
    part = ((np.arange(g.n) // 60) // 12 * 5 + (np.arange(g.n) % 60) // 12).astype(np.int32)   # 5 x 5 tiles
    assert rel_err(bc.brandes_pp(G, S, part).cpu().numpy(), ref_s) < FP64_TOL


def test_small_weights_long_distances(bc):
    """Weights in [1, 4] on a 2,000-node path (distances up to about 5,000, thousands of steps per
    batch with few distinct weights) and on a 40 x 40 grid, plain Brandes and Brandes++ in both
    precisions (the Centrality step's distances in 16 bits where they fit, else in 32)."""
    n = 2000
    g = gen.with_weights(gen.path(n), 4, seed=96)
    G = bc.graph_from_edgelist(g)
    i = np.arange(n)
    ref, _ = oracle.brandes(g)
    assert rel_err(ref, i * (n - 1 - i)) < FP64_TOL
    assert rel_err(bc.brandes(G).cpu().numpy(), ref) < FP64_TOL
    assert rel_err(bc.brandes(G, precision="fp32").cpu().numpy(), ref) < FP32_TOL
    _check_sssp(bc, G, g, np.array([0, 999, 1999], np.int32))
    # parts of 10 consecutive nodes: table distances at most 36, distances from the sources to the
    # frontiers up to about 5,000 (the Centrality step's 16-bit path must fall back to 32 bits)
    S1 = gen.sample_targets(n, 100, seed=99)
    ref1, _ = oracle.brandes(g, S1)
    blocks = (np.arange(n) // 10).astype(np.int32)
    for prec, tol in (("fp64", FP64_TOL), ("fp32", FP32_TOL)):
        assert rel_err(bc.brandes_pp(G, S1, blocks, precision=prec).cpu().numpy(), ref1) < tol, prec
    g2 = gen.with_weights(gen.grid(40, 40), 4, seed=97)
    G2 = bc.graph_from_edgelist(g2)
    S = gen.sample_targets(g2.n, 300, seed=98)
    ref2, _ = oracle.brandes(g2, S)
    assert rel_err(bc.brandes(G2, S).cpu().numpy(), ref2) < FP64_TOL
    part = ((np.arange(g2.n) // 40) // 10 * 4 + (np.arange(g2.n) % 40) // 10).astype(np.int32)   # 4 x 4 tiles
    assert rel_err(bc.brandes_pp(G2, S, part).cpu().numpy(), ref2) < FP64_TOL
    assert rel_err(bc.brandes_pp(G2, S, part, precision="fp32").cpu().numpy(), ref2) < FP32_TOL


def _active_lane_counts(g, srcs):
    """Per (node, distance) of one 32-source batch: how many of its sources reach the node at
    that distance (the lanes an entry of that step is active on), from the oracle's distances."""
    d = np.stack([oracle.sssp(g, int(s))[0] for s in srcs], axis=1)
    counts = []
    for row in d:
        r = row[row != np.iinfo(np.int32).max]
        if r.size:
            counts.extend(np.unique(r, return_counts=True)[1].tolist())
    return np.asarray(counts)


@pytest.mark.parametrize("directed", [False, True])
def test_weighted_entries_few_and_many_lanes(bc, directed):
    """Integer weights visit an entry one of two ways: a lane per source when more than 16 of
    the batch's 32 sources are at the step's distance, else (arc, source) pairs over the lanes.
    Weights in {1, 2} give entries of both kinds in the same batch (checked on the first batch
    from the oracle's distances); unsorted sources keep the batches as given."""
    g = gen.chung_lu_communities(1500, [300] * 5, 2.3, 12.0 if directed else 8.0, 0.85, seed=101,
                                 directed=directed, wmax=2)
    S = np.arange(g.n, dtype=np.int32)
    cnt = _active_lane_counts(g, S[:32])
    assert (cnt <= 16).any() and (cnt > 16).any()
    G = bc.graph_from_edgelist(g)
    _check_sssp(bc, G, g, S[:32])
    ref, _ = oracle.brandes(g)
    for order in (False, True):
        assert rel_err(bc.brandes(G, None, order_sources=order).cpu().numpy(), ref) < FP64_TOL, order
    assert rel_err(bc.brandes(G, None, precision="fp32").cpu().numpy(), ref) < FP32_TOL
    T = gen.sample_targets(g.n, 500, seed=102)
    ref_t, _ = oracle.brandes(g, T)
    assert rel_err(bc.brandes_pp(G, T, g.part).cpu().numpy(), ref_t) < FP64_TOL
