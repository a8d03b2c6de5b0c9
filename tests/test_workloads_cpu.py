"""CPU pins of the seeded workload recipes (the synthetic stand-ins for the paper's datasets):
sizes, target sets, partitions, weight ranges, simple-graph invariants and determinism."""
import numpy as np
import pytest

from paper_1406_4173_gb300 import gen


def _simple(g):
    """No self-loops and no repeated edges (as unordered pairs for undirected graphs)."""
    u, v = np.asarray(g.src, np.int64), np.asarray(g.dst, np.int64)
    assert np.all(u != v)
    a, b = (np.minimum(u, v), np.maximum(u, v)) if not g.directed else (u, v)
    key = a * g.n + b
    assert len(np.unique(key)) == len(key)
    assert u.min() >= 0 and max(u.max(), v.max()) < g.n


@pytest.mark.parametrize("name,n,m,directed,nS,k,wrange", [
    ("planted_2k", 2000, None, False, None, 8, None),
    ("chunglu_10k", 10_000, 50_000, False, None, 10, None),
    ("chunglu_50k", 50_000, 250_000, False, None, 50, None),
    ("directed_100k", 100_000, 1_200_000, True, 2000, 200, (1, 16)),
    ("chunglu_100k", 100_000, 800_000, False, 512, 100, None),
    ("directed_20k", 20_000, 240_000, True, 400, 40, (1, 16)),
    ("planted_200k", 200_000, None, False, 200, 100, None),
])
def test_single_graph_workloads(name, n, m, directed, nS, k, wrange):
    g, S = gen.workload(name)
    assert g.n == n and g.directed == directed
    if m is not None:
        assert g.m == m
    part = np.asarray(g.part)
    assert part.shape == (n,) and part.min() == 0 and part.max() == k - 1
    assert len(np.unique(part)) == k
    if nS is None:
        assert S is None or len(S) == n
    else:
        S = np.asarray(S)
        assert len(S) == nS and len(np.unique(S)) == nS and S.min() >= 0 and S.max() < n
    if wrange is None:
        assert g.w is None
    else:
        w = np.asarray(g.w)
        assert w.min() >= wrange[0] and w.max() <= wrange[1]
    _simple(g)


def test_planted_2k_edge_counts():
    """8 x 250 nodes, p_in = 0.02, p_out = 0.0005: about 8 * C(250,2) * 0.02 = 4,980 intra and
    C(2000,2) - 8 C(250,2) = 1,750,000 pairs * 0.0005 = 875 inter edges."""
    g, _ = gen.workload("planted_2k")
    part = np.asarray(g.part)
    intra = int(np.sum(part[g.src] == part[g.dst]))
    inter = g.m - intra
    assert abs(intra - 4980) < 5 * np.sqrt(4980) and abs(inter - 875) < 5 * np.sqrt(875)


def test_planted_200k_small_cut():
    """The small-skeleton workload: 100 communities of 2,000, intra degree about 10, and only
    about 1,800 edges between communities."""
    g, _ = gen.workload("planted_200k")
    part = np.asarray(g.part)
    assert np.all(np.bincount(part) == 2000)
    inter = int(np.sum(part[g.src] != part[g.dst]))
    assert 1500 < inter < 2100
    assert abs(2 * (g.m - inter) / g.n - 10) < 0.2


def test_er_batch_sizes():
    """4,096 G(n, 8/(n-1)) graphs with log-normal sizes (median 512, clipped to [64, 4096])."""
    gs, S = gen.workload("er_batch_4096")
    assert S is None and len(gs) == 4096
    ns = np.array([g.n for g in gs])
    assert ns.min() >= 64 and ns.max() <= 4096
    assert 450 < np.median(ns) < 580
    mean_deg = np.array([2 * g.m / g.n for g in gs])
    assert abs(np.mean(mean_deg) - 8) < 0.3
    for g in gs[:50]:
        assert not g.directed and g.w is None
        _simple(g)


def test_chunglu_1m_shape():
    g, S = gen.workload("chunglu_1m")
    assert g.n == 1_000_000 and g.m == 8_000_000 and not g.directed and g.w is None
    S = np.asarray(S)
    assert len(S) == 4096 and len(np.unique(S)) == 4096
    part = np.asarray(g.part)
    assert np.all(np.bincount(part) == 1000)


@pytest.mark.parametrize("name", ["planted_2k", "chunglu_10k", "directed_100k"])
def test_workloads_are_deterministic(name):
    g1, S1 = gen.workload(name)
    g2, S2 = gen.workload(name)
    assert np.array_equal(g1.src, g2.src) and np.array_equal(g1.dst, g2.dst)
    assert (g1.w is None and g2.w is None) or np.array_equal(g1.w, g2.w)
    assert np.array_equal(g1.part, g2.part)
    assert (S1 is None and S2 is None) or np.array_equal(S1, S2)
