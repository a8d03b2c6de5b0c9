"""GPU: the launch-shape autotuner (bcpp_autotune) returns one of its candidates, times each of
them, and the tuned options give the oracle's betweenness."""
import numpy as np
import pytest

import oracle
from paper_1406_4173_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bc():
    import torch
    import paper_1406_4173_gb300 as m
    from paper_1406_4173_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    return m


def rel_err(x, ref):
    return float(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1.0)))


@pytest.mark.parametrize("weighted", [False, True])
def test_autotune_candidates_and_parity(bc, weighted):
    g = gen.chung_lu_communities(2500, [500] * 5, 2.3, 8.0, 0.9, seed=31, wmax=8 if weighted else None)
    G = bc.graph_from_edgelist(g)
    S = gen.sample_targets(g.n, 700, seed=4)
    tuned, times = bc.autotune(G, S)
    assert (tuned["batch"], tuned["cluster"]) in bc.api.AUTOTUNE_CANDIDATES
    assert all(t > 0 for t in times.values()), times
    assert times[(tuned["batch"], tuned["cluster"])] == min(times.values())
    ref, _ = oracle.brandes(g, S)
    x = bc.brandes(G, S, **tuned).cpu().numpy()
    assert rel_err(x, ref) <= 1e-12
    xp = bc.brandes_pp(G, S, g.part, **tuned).cpu().numpy()
    assert rel_err(xp, ref) <= 1e-12


def test_autotune_trivial(bc):
    g = gen.planted_partition(200, 2, 0.05, 0.01, seed=1)
    G = bc.graph_from_edgelist(g)
    tuned, times = bc.autotune(G, np.array([3], np.int32))
    assert all(t == -1.0 for t in times.values())


def test_autotune_directed_weighted(bc):
    g = gen.chung_lu_communities(1200, [300] * 4, 2.3, 6.0, 0.85, seed=19, directed=True, wmax=9)
    G = bc.graph_from_edgelist(g)
    S = gen.sample_targets(g.n, 400, seed=6)
    tuned, times = bc.autotune(G, S, precision="fp32")
    assert (tuned["batch"], tuned["cluster"]) in bc.api.AUTOTUNE_CANDIDATES
    ref, _ = oracle.brandes(g, S)
    x = bc.brandes(G, S, precision="fp32", **tuned).cpu().numpy()
    assert rel_err(x, ref) <= 2e-6       # FP32-delta: measured 1.1e-7


def test_autotune_batched_candidates_and_parity(bc):
    """bcpp_autotune_batched times every (batch, CTAs per SM) candidate on the whole arena and
    the tuned options give the oracle's betweenness for every graph."""
    gs = [gen.erdos_renyi(int(n), min(1.0, 8.0 / max(n - 1, 1)), seed=300 + i) for i, n in
          enumerate([64, 700, 1500, 2, 1, 300, 4096, 90, 129, 33, 650, 512])]
    arena = bc.build_arena(gs)
    tuned, times = bc.autotune_batched(arena)
    assert (tuned["batch"], tuned["ctas_per_sm"]) in bc.api.AUTOTUNE_BATCHED_CANDIDATES
    assert all(t > 0 for t in times.values()), times
    assert times[(tuned["batch"], tuned["ctas_per_sm"])] == min(times.values())
    got = bc.brandes_batched(arena, **tuned).cpu().numpy()
    off = arena.node_ptr_host
    for i, g in enumerate(gs):
        ref, _ = oracle.brandes(g)
        assert rel_err(got[off[i]:off[i + 1]], ref) <= 1e-12, i
