"""Pins for the CPU oracle, independent of the oracle itself.

Each check comes from the mathematics of Sec. 3-4 rather than from the oracle's code:
exact brute-force enumeration of shortest paths, closed forms of textbook graphs, the
path-length invariant, the exactness of Brandes++ (Brandes++ = Brandes for every S and P),
and the skeleton's preservation of distances and path counts between frontier nodes.
"""
import heapq
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import bruteforce as bf
from paper_1406_4173_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF32 = np.iinfo(np.int32).max


def rel_err(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1.0))) if x.size else 0.0


def small_graphs():
    """Seeded tiny graphs covering directed/undirected x weighted/unweighted."""
    cases = []
    for seed in range(12):
        n = 5 + seed % 6
        for directed in (False, True):
            for wmax in (None, 4):
                p = 0.45 if directed else 0.4
                g = gen.erdos_renyi(n, p, seed=seed, directed=directed, wmax=wmax, stream=11)
                cases.append((f"er{seed}-{'d' if directed else 'u'}-{'w' if wmax else '1'}", g))
    return cases


SMALL = small_graphs()


# ----------------------------------------------------------------------------- brute force
@pytest.mark.parametrize("name,g", SMALL, ids=[c[0] for c in SMALL])
def test_brandes_equals_bruteforce(name, g):
    ref = [float(x) for x in bf.betweenness(g)]
    bc, ovf = oracle.brandes(g)
    assert not ovf
    assert rel_err(bc, ref) < 1e-12
    # a target subset
    rng = np.random.default_rng(len(name))
    S = np.sort(rng.choice(g.n, size=max(2, g.n // 2), replace=False))
    ref_s = [float(x) for x in bf.betweenness(g, S)]
    bc_s, _ = oracle.brandes(g, S)
    assert rel_err(bc_s, ref_s) < 1e-12


@pytest.mark.parametrize("name,g", SMALL[:16], ids=[c[0] for c in SMALL[:16]])
def test_sssp_equals_bruteforce(name, g):
    d, sig = bf.sigma_table(g)
    for s in range(g.n):
        dist, sigma, ovf = oracle.sssp(g, s)
        for t in range(g.n):
            if d[s][t] == bf.INF:
                assert dist[t] == INF32 and sigma[t] == 0
            else:
                assert dist[t] == d[s][t] and int(sigma[t]) == sig[s][t]


def test_golden_bruteforce_fixture():
    """Values stored by tests/golden/make_golden.py (exact brute force)."""
    with open(os.path.join(GOLDEN, "bruteforce_small.json")) as f:
        fx = json.load(f)
    for case in fx["cases"]:
        g = gen.EdgeList(n=case["n"], src=np.array(case["src"], np.int32), dst=np.array(case["dst"], np.int32),
                         w=None if case["w"] is None else np.array(case["w"], np.uint32),
                         directed=case["directed"])
        S = None if case["S"] is None else np.array(case["S"], np.int32)
        bc, _ = oracle.brandes(g, S)
        ref = [float(num) / den for num, den in case["bc"]]
        assert rel_err(bc, ref) < 1e-12, case["name"]


# ----------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [2, 3, 7, 50, 301])
def test_path_closed_form(n):
    bc, _ = oracle.brandes(gen.path(n))
    i = np.arange(n)
    assert rel_err(bc, i * (n - 1 - i)) < 1e-12


@pytest.mark.parametrize("n", [3, 10, 257])
def test_star_closed_form(n):
    bc, _ = oracle.brandes(gen.star(n))
    ref = np.zeros(n)
    ref[0] = (n - 1) * (n - 2) / 2
    assert rel_err(bc, ref) < 1e-12


@pytest.mark.parametrize("n", [5, 6, 11, 40, 101])
def test_cycle_closed_form(n):
    bc, _ = oracle.brandes(gen.cycle(n))
    k = n // 2
    val = k * (k - 1) / 2 if n % 2 else (k - 1) ** 2 / 2
    assert rel_err(bc, np.full(n, val)) < 1e-12


@pytest.mark.parametrize("n", [2, 5, 30])
def test_complete_graph_zero(n):
    bc, _ = oracle.brandes(gen.complete(n))
    assert np.all(bc == 0)


@pytest.mark.parametrize("a,b", [(1, 4), (3, 5), (7, 2), (10, 13)])
def test_complete_bipartite_closed_form(a, b):
    bc, _ = oracle.brandes(gen.complete_bipartite(a, b))
    ref = np.concatenate([np.full(a, math.comb(b, 2) / a), np.full(b, math.comb(a, 2) / b)])
    assert rel_err(bc, ref) < 1e-12


@pytest.mark.parametrize("r,c", [(2, 3), (5, 7), (12, 9)])
def test_grid_sigma_binomial(r, c):
    g = gen.grid(r, c)
    dist, sigma, ovf = oracle.sssp(g, 0)
    for x in range(r):
        for y in range(c):
            assert dist[x * c + y] == x + y
            assert int(sigma[x * c + y]) == math.comb(x + y, x)


def test_grid_sigma_uint64_edge_and_overflow():
    # C(66,33) < 2^64: exact; C(68,34) > 2^64: flagged
    g = gen.grid(34, 34)
    _, sigma, ovf = oracle.sssp(g, 0)
    assert int(sigma[-1]) == math.comb(66, 33) and not ovf
    g = gen.grid(35, 35)
    _, sigma, ovf = oracle.sssp(g, 0)
    assert ovf


# ----------------------------------------------------------------------------- invariants
def _pair_length_sum(g, S):
    """sum over ordered pairs s != t in S, t reachable, of (d(s,t) - 1)."""
    tot = 0
    Sset = set(int(x) for x in S)
    for s in S:
        dist, _, _ = oracle.sssp(g, int(s))
        for t in Sset:
            if t != s and dist[t] != INF32:
                tot += int(dist[t]) - 1
    return tot


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_path_length_invariant_undirected(seed):
    g = gen.erdos_renyi(80, 0.05, seed=seed)
    for S in (np.arange(g.n), gen.sample_targets(g.n, 17, seed)):
        bc, _ = oracle.brandes(g, S)
        # each unordered pair once (halved): sum_v C(v) = sum_{s<t} (d - 1)
        assert abs(bc.sum() - _pair_length_sum(g, S) / 2) < 1e-9 * max(1, bc.sum())


@pytest.mark.parametrize("seed", [0, 1])
def test_path_length_invariant_directed(seed):
    g = gen.erdos_renyi(60, 0.06, seed=seed, directed=True)
    S = np.arange(g.n)
    bc, _ = oracle.brandes(g, S)
    assert abs(bc.sum() - _pair_length_sum(g, S)) < 1e-9 * max(1, bc.sum())


# ----------------------------------------------------------------------------- Brandes++ exactness
def _partitions(n, seed):
    rng = np.random.default_rng(seed)
    return {
        "random4": rng.integers(0, 4, n).astype(np.int32),
        "single": np.zeros(n, np.int32),
        "singletons": np.arange(n, dtype=np.int32),
        "blocks": (np.arange(n) * 5 // max(n, 1)).astype(np.int32),
    }


@pytest.mark.parametrize("name,g", SMALL, ids=[c[0] for c in SMALL])
def test_brandes_pp_equals_bruteforce_tiny(name, g):
    ref = [float(x) for x in bf.betweenness(g)]
    for pname, part in _partitions(g.n, len(name)).items():
        bc, ovf, _ = oracle.brandes_pp(g, np.arange(g.n), part)
        assert rel_err(bc, ref) < 1e-12, pname


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("directed", [False, True])
@pytest.mark.parametrize("wmax", [None, 16])
def test_brandes_pp_equals_brandes(seed, directed, wmax):
    if directed:
        g = gen.chung_lu_communities(300, [60] * 5, 2.3, 5.0, 0.85, seed=seed, directed=True, wmax=wmax)
    else:
        g = gen.planted_partition(300, 6, 0.08, 0.004, seed=seed, wmax=wmax)
    for S in (gen.sample_targets(g.n, 25, seed), np.arange(g.n, dtype=np.int32)):
        ref, _ = oracle.brandes(g, S)
        for pname, part in list(_partitions(g.n, seed).items()) + [("planted", g.part)]:
            bc, ovf, st = oracle.brandes_pp(g, S, part)
            assert rel_err(bc, ref) < 1e-12, (pname, st)


def test_brandes_pp_single_part_and_no_targets_in_part():
    g = gen.planted_partition(120, 3, 0.15, 0.01, seed=3)
    S = np.array([0, 1], np.int32)
    ref, _ = oracle.brandes(g, S)
    bc, _, st = oracle.brandes_pp(g, S, np.zeros(g.n, np.int32))
    assert rel_err(bc, ref) < 1e-12


# ----------------------------------------------------------------------------- skeleton
def _sssp_mult(nodes, arcs, src):
    """Dijkstra with multiplicities on an arc list, written independently for this test."""
    au, av, aw, amu = arcs
    adj = {}
    for a, b, w, m in zip(au.tolist(), av.tolist(), aw.tolist(), amu.tolist()):
        adj.setdefault(a, []).append((b, w, m))
    dist = {src: 0}
    sig = {src: 1}
    done = set()
    pq = [(0, src)]
    while pq:
        d, u = heapq.heappop(pq)
        if u in done or d != dist[u]:
            continue
        done.add(u)
        for v, w, m in adj.get(u, []):
            nd = d + w
            if v not in dist or nd < dist[v]:
                dist[v] = nd
                sig[v] = sig[u] * m
                heapq.heappush(pq, (nd, v))
            elif nd == dist[v]:
                sig[v] += sig[u] * m
    return dist, sig


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("directed", [False, True])
def test_skeleton_preserves_distances_and_counts(seed, directed):
    if directed:
        g = gen.chung_lu_communities(200, [40] * 5, 2.3, 4.0, 0.85, seed=seed, directed=True, wmax=9)
    else:
        g = gen.planted_partition(200, 5, 0.1, 0.006, seed=seed, wmax=5)
    S = gen.sample_targets(g.n, 12, seed)
    nodes, arcs, _ = oracle.skeleton(g, S, g.part)
    assert set(S.tolist()) - set(nodes.tolist()) <= {s for s in S.tolist() if _isolated(g, s)}
    for s in nodes[:: max(1, len(nodes) // 15)]:
        dG, sG, _ = oracle.sssp(g, int(s))
        dK, sK = _sssp_mult(nodes, arcs, int(s))
        for t in nodes.tolist():
            if dG[t] == INF32:
                assert t not in dK
            else:
                assert dK[t] == dG[t] and sK[t] == int(sG[t])


def _isolated(g, v):
    return not (np.any(g.src == v) or np.any(g.dst == v))


def test_skeleton_of_singletons_is_the_graph():
    g = gen.erdos_renyi(40, 0.1, seed=5, wmax=7)
    nodes, (au, av, aw, amu), _ = oracle.skeleton(g, np.arange(g.n), np.zeros(g.n, np.int32))
    assert np.all(amu == 1)
    got = sorted(zip(au.tolist(), av.tolist(), aw.tolist()))
    ref = sorted([(int(a), int(b), int(w)) for a, b, w in zip(g.src, g.dst, g.w)] +
                 [(int(b), int(a), int(w)) for a, b, w in zip(g.src, g.dst, g.w)])
    assert got == ref


def test_skeleton_single_part_no_targets():
    g = gen.erdos_renyi(30, 0.15, seed=2)
    nodes, arcs, _ = oracle.skeleton(g, np.zeros(0, np.int32), np.zeros(g.n, np.int32))
    assert len(nodes) == 0 and arcs[0].size == 0


# ----------------------------------------------------------------------------- input errors
def test_oracle_rejects_bad_inputs():
    g = gen.path(4)
    bad = gen.EdgeList(n=3, src=np.array([0, 1], np.int32), dst=np.array([1, 1], np.int32))
    with pytest.raises(ValueError):
        oracle.brandes(bad)
    dup = gen.EdgeList(n=3, src=np.array([0, 1], np.int32), dst=np.array([1, 0], np.int32))
    with pytest.raises(ValueError):
        oracle.brandes(dup)
    w0 = gen.EdgeList(n=2, src=np.array([0], np.int32), dst=np.array([1], np.int32), w=np.array([0], np.uint32))
    with pytest.raises(ValueError):
        oracle.brandes(w0)
    with pytest.raises(ValueError):
        oracle.brandes(g, np.array([1, 1], np.int32))


def test_distance_sum_matches_definition():
    for seed in range(3):
        g = gen.erdos_renyi(70, 0.06, seed=seed)
        src = np.arange(g.n, dtype=np.int32)
        ref = 0
        for s in src:
            dist, _, _ = oracle.sssp(g, int(s))
            ref += int(np.sum(dist[(dist != INF32) & (np.arange(g.n) != s)] - 1))
        assert oracle.distance_sum(g, src) == ref
    # closed form: path P_n, sum over ordered pairs of (|i-j| - 1)
    n = 40
    ref = sum(abs(i - j) - 1 for i in range(n) for j in range(n) if i != j)
    assert oracle.distance_sum(gen.path(n), np.arange(n, dtype=np.int32)) == ref



# ----------------------------------------------------------------------------- sources -> destinations (Alg. 3 pairs)
@pytest.mark.parametrize("name,g", SMALL[::3], ids=[c[0] for c in SMALL[::3]])
def test_brandes_st_equals_bruteforce(name, g):
    rng = np.random.default_rng(len(name) + 7)
    src = np.sort(rng.choice(g.n, size=max(1, g.n // 2), replace=False))
    dst = np.sort(rng.choice(g.n, size=max(1, g.n // 2), replace=False))
    ref = [float(x) for x in bf.betweenness_st(g, src, dst)]
    got, _ = oracle.brandes_st(g, src, dst)
    assert rel_err(got, ref) < 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_pairs_of_parts_sum_to_full_betweenness(seed):
    """Sec. 5: summing the (P_i -> P_j) pair sets over all ordered pairs of parts gives C."""
    g = gen.planted_partition(120, 4, 0.12, 0.01, seed=seed, wmax=3)
    full, _ = oracle.brandes(g, halve=False)
    tot = np.zeros(g.n)
    for i in range(4):
        for j in range(4):
            Pi, Pj = np.nonzero(g.part == i)[0], np.nonzero(g.part == j)[0]
            x, _ = oracle.brandes_st(g, Pi, Pj, halve=False)
            tot += x
    assert rel_err(tot, full) < 1e-12


# ----------------------------------------------------------------------------- label-propagation partition
# The rule is defined in oracle/bc_oracle.c (not by the paper).  Pins: small cases traced by
# hand from that definition, and properties that any correct implementation of it has.
def test_label_propagation_hand_traced_cases():
    # P4 0-1-2-3.  Round 1, even half: 0 <- 1 (only neighbour), 2 <- min(1, 3) = 1;
    # odd half: 1 keeps 1 (two votes), 3 <- 1.  Round 2 changes nothing: one part, 2 rounds.
    assert [list(x) if hasattr(x, "__len__") else x for x in oracle.label_propagation(gen.path(4))] == \
        [[0, 0, 0, 0], 1, 2]
    # P5 0-1-2-3-4.  Round 1, even: 0 <- 1, 2 <- 1, 4 <- 3 -> [1,1,1,3,3]; odd: 1 keeps 1, 3 keeps 3
    # (tied with 1, own label kept).  Round 2 changes nothing: parts {0,1,2}, {3,4}.
    part, k, r = oracle.label_propagation(gen.path(5))
    assert list(part) == [0, 0, 0, 1, 1] and k == 2 and r == 2
    # star, centre 0 and leaves 1..8.  Round 1, even: 0 <- 1 (eight ties, smallest), even leaves
    # <- 0; odd: odd leaves <- 1.  Round 2, even: centre ties 4:4, keeps 1; even leaves <- 1.
    # Round 3 changes nothing: one part after 3 rounds.
    part, k, r = oracle.label_propagation(gen.star(9))
    assert k == 1 and not part.any() and r == 3
    # directed 3-cycle 0->1->2->0 (in- and out-arcs both count).  Round 1, even: 0 <- min(1,2) = 1,
    # 2 <- min(0,1) = 0; odd: 1 keeps 1 (tie with 0).  Round 2, even: 0 keeps 1, 2 <- 1 (two votes).
    # Round 3 changes nothing.
    cyc = gen.EdgeList(3, np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32), None, True)
    part, k, r = oracle.label_propagation(cyc)
    assert k == 1 and not part.any() and r == 3


def test_label_propagation_cliques_and_isolated_nodes():
    # disjoint cliques with scattered ids: one part per clique; isolated nodes keep their own part
    rng = np.random.default_rng(5)
    sizes = [5, 7, 4, 9]
    n = sum(sizes) + 3
    ids = rng.permutation(n)
    u, v, groups, o = [], [], [], 0
    for s in sizes:
        grp = ids[o:o + s]
        groups.append(grp)
        for a in range(s):
            for b in range(a + 1, s):
                u.append(grp[a]); v.append(grp[b])
        o += s
    g = gen._from_pairs(n, np.array(u), np.array(v), False)
    part, k, _ = oracle.label_propagation(g)
    assert k == len(sizes) + 3
    for grp in groups:
        assert len(set(part[grp])) == 1
    assert len({int(part[grp[0]]) for grp in groups}) == len(sizes)
    for x in ids[o:]:
        assert np.sum(part == part[x]) == 1
    # two 6-cliques joined by one edge: two parts
    u = [a for a in range(6) for b in range(a + 1, 6)] + [6 + a for a in range(6) for b in range(a + 1, 6)] + [5]
    v = [b for a in range(6) for b in range(a + 1, 6)] + [6 + b for a in range(6) for b in range(a + 1, 6)] + [6]
    part, k, _ = oracle.label_propagation(gen._from_pairs(12, np.array(u), np.array(v), False))
    assert k == 2 and len(set(part[:6])) == 1 and len(set(part[6:])) == 1


@pytest.mark.parametrize("seed", range(3))
def test_label_propagation_valid_partition(seed):
    g = gen.chung_lu_communities(600, [150] * 4, 2.3, 6.0, 0.9, seed=seed, directed=bool(seed % 2))
    part, k, r = oracle.label_propagation(g, max_rounds=30)
    assert part.min() == 0 and part.max() == k - 1 and len(np.unique(part)) == k and 1 <= r <= 30
    part2, k2, r2 = oracle.label_propagation(g, max_rounds=30)
    assert np.array_equal(part, part2) and (k, r) == (k2, r2)
