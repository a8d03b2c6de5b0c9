"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Distances and uint64 path counts must match bit for bit; betweenness to a relative 1e-12 in
FP64 mode and to FP32_TOL in FP32-delta mode (relative error max_v |x - ref| / max(|ref|, 1)).
Sizes span several 32-source batches with a ragged last batch.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1406_4173_gb300 import gen

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
# FP32-delta bar of the small parity graphs: 10x the largest error measured on them (1.96e-7,
# `chunglu-u-hub` with S = V; the others 3.1e-8 to 1.4e-7).  The per-source dependencies are
# formed in FP32 in a fixed order per lane, so the error does not vary from run to run.
FP32_TOL = 2e-6
INF32 = np.iinfo(np.int32).max


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
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1.0))) if x.size else 0.0


def graphs():
    out = [
        ("planted-u1", gen.planted_partition(700, 7, 0.03, 0.002, seed=1)),
        ("planted-uw", gen.planted_partition(600, 6, 0.03, 0.003, seed=2, wmax=9)),
        ("chunglu-d1", gen.chung_lu_communities(800, [200] * 4, 2.3, 6.0, 0.85, seed=3, directed=True)),
        ("chunglu-dw", gen.chung_lu_communities(800, [160] * 5, 2.3, 6.0, 0.85, seed=4, directed=True, wmax=16)),
        ("er-sparse-u", gen.erdos_renyi(900, 1.5 / 900, seed=5)),           # many components
        ("chunglu-u-hub", gen.chung_lu_communities(1500, [300] * 5, 2.1, 8.0, 0.9, seed=6)),
    ]
    return out


GRAPHS = graphs()
IDS = [g[0] for g in GRAPHS]


# ----------------------------------------------------------------------------- d and sigma
@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_sssp_bit_exact(bc, name, g):
    G = bc.graph_from_edgelist(g)
    src = np.unique(np.concatenate([np.arange(0, g.n, max(1, g.n // 67)), [g.n - 1]])).astype(np.int32)
    dist, sig = bc.sssp(G, src, allow_overflow=True)
    dist = dist.cpu().numpy()
    sig = sig.cpu().numpy().view(np.uint64)
    for i, s in enumerate(src):
        d_ref, s_ref, _ = oracle.sssp(g, int(s))
        assert np.array_equal(dist[i], d_ref), (name, s)
        assert np.array_equal(sig[i], s_ref), (name, s)


def test_sigma_uint64_limit_and_overflow(bc):
    g = gen.grid(34, 34)
    dist, sig = bc.sssp(bc.graph_from_edgelist(g), np.array([0], np.int32))
    assert int(sig.cpu().numpy().view(np.uint64)[0, -1]) == math.comb(66, 33)
    g = gen.grid(35, 35)
    with pytest.raises(bc.SigmaOverflow):
        bc.sssp(bc.graph_from_edgelist(g), np.array([0], np.int32))


# ----------------------------------------------------------------------------- plain Brandes
def test_brandes_large_path_counts(bc):
    """34 x 34 grid: path counts up to C(66,33) ~ 7.2e18 (the uint64 limit's neighbourhood), so
    the reciprocals 1/sigma of the dependency recursion span 18 decades."""
    g = gen.grid(34, 34)
    G = bc.graph_from_edgelist(g)
    ref, ovf = oracle.brandes(g)
    assert not ovf
    assert rel_err(bc.brandes(G).cpu().numpy(), ref) < FP64_TOL
    assert rel_err(bc.brandes(G, precision="fp32").cpu().numpy(), ref) < FP32_TOL
    S = gen.sample_targets(g.n, 300, seed=71)
    ref_s, _ = oracle.brandes(g, S)
    assert rel_err(bc.brandes(G, S).cpu().numpy(), ref_s) < FP64_TOL


@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_brandes_all_targets(bc, name, g):
    G = bc.graph_from_edgelist(g)
    ref, _ = oracle.brandes(g)
    got = bc.brandes(G).cpu().numpy()
    assert rel_err(got, ref) < FP64_TOL
    got32 = bc.brandes(G, precision="fp32").cpu().numpy()
    assert rel_err(got32, ref) < FP32_TOL


@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_brandes_target_subset(bc, name, g):
    G = bc.graph_from_edgelist(g)
    S = gen.sample_targets(g.n, 75, seed=11)
    ref, _ = oracle.brandes(g, S)
    got = bc.brandes(G, S).cpu().numpy()
    assert rel_err(got, ref) < FP64_TOL
    # unhalved (ordered pairs)
    ref_o, _ = oracle.brandes(g, S, halve=False)
    got_o = bc.brandes(G, S, halve=False).cpu().numpy()
    assert rel_err(got_o, ref_o) < FP64_TOL


@pytest.mark.parametrize("n", [2, 3, 33, 65])
def test_brandes_closed_forms(bc, n):
    i = np.arange(n)
    got = bc.brandes(bc.graph_from_edgelist(gen.path(n))).cpu().numpy()
    assert rel_err(got, i * (n - 1 - i)) < FP64_TOL
    if n >= 3:
        got = bc.brandes(bc.graph_from_edgelist(gen.star(n))).cpu().numpy()
        ref = np.zeros(n)
        ref[0] = (n - 1) * (n - 2) / 2
        assert rel_err(got, ref) < FP64_TOL
        got = bc.brandes(bc.graph_from_edgelist(gen.cycle(n))).cpu().numpy()
        k = n // 2
        assert rel_err(got, np.full(n, k * (k - 1) / 2 if n % 2 else (k - 1) ** 2 / 2)) < FP64_TOL


def test_brandes_degenerate_inputs(bc):
    import torch
    g = gen.erdos_renyi(50, 0.05, seed=9)
    G = bc.graph_from_edgelist(g)
    # |S| < 2: all zeros
    assert torch.all(bc.brandes(G, np.array([3], np.int32)) == 0)
    # a graph without arcs
    e = gen.EdgeList(n=10, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32))
    assert torch.all(bc.brandes(bc.graph_from_edgelist(e)) == 0)
    # isolated targets
    S = np.array([0, 1, 2, 49], np.int32)
    ref, _ = oracle.brandes(g, S)
    assert rel_err(bc.brandes(G, S).cpu().numpy(), ref) < FP64_TOL


def test_brandes_rejects_bad_targets(bc):
    G = bc.graph_from_edgelist(gen.path(10))
    with pytest.raises(bc.BcppError):
        bc.brandes(G, np.array([1, 1], np.int32))
    with pytest.raises(bc.BcppError):
        bc.brandes(G, np.array([1, 10], np.int32))


# ----------------------------------------------------------------------------- CSR build / validation
def test_csr_build_matches_definition(bc):
    g = gen.chung_lu_communities(500, [100] * 5, 2.3, 6.0, 0.8, seed=12, wmax=7)
    G = bc.graph_from_edgelist(g)
    rp = G.row_ptr.cpu().numpy()
    col = G.col.cpu().numpy()
    w = G.w.cpu().numpy().view(np.uint32)
    arcs = sorted([(int(a), int(b), int(c)) for a, b, c in zip(g.src, g.dst, g.w)] +
                  [(int(b), int(a), int(c)) for a, b, c in zip(g.src, g.dst, g.w)])
    got = [(u, int(col[p]), int(w[p])) for u in range(g.n) for p in range(rp[u], rp[u + 1])]
    assert got == arcs
    bc.csr_validate(G)


@pytest.mark.parametrize("case", ["self_loop", "duplicate", "reverse_duplicate", "zero_weight", "range"])
def test_csr_build_rejects(bc, case):
    src, dst, w = np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32), None
    if case == "self_loop":
        dst[2] = 2
    elif case == "duplicate":
        src, dst = np.array([0, 0], np.int32), np.array([1, 1], np.int32)
    elif case == "reverse_duplicate":
        src, dst = np.array([0, 1], np.int32), np.array([1, 0], np.int32)
    elif case == "zero_weight":
        w = np.array([1, 0, 2], np.uint32)
    elif case == "range":
        dst[2] = 4
    with pytest.raises(bc.BcppError):
        bc.csr_build(4, src, dst, w, directed=False)


# ----------------------------------------------------------------------------- Brandes++
def partitions(g, seed):
    rng = np.random.default_rng(seed)
    return {
        "planted": g.part,
        "random": rng.integers(0, 5, g.n).astype(np.int32),
        "single": np.zeros(g.n, np.int32),
        "singletons": np.arange(g.n, dtype=np.int32),
    }


@pytest.mark.parametrize("name,g", GRAPHS[:4] + GRAPHS[5:], ids=IDS[:4] + IDS[5:])
def test_brandes_pp_equals_oracle(bc, name, g):
    G = bc.graph_from_edgelist(g)
    part_all = partitions(g, 5)
    for S in (gen.sample_targets(g.n, 70, seed=13), None):
        ref, _ = oracle.brandes(g, S)
        for pname, part in part_all.items():
            got = bc.brandes_pp(G, S, part).cpu().numpy()
            assert rel_err(got, ref) < FP64_TOL, (pname, S is None)
    S = gen.sample_targets(g.n, 70, seed=14)
    ref, _ = oracle.brandes(g, S)
    got32 = bc.brandes_pp(G, S, g.part, precision="fp32").cpu().numpy()
    assert rel_err(got32, ref) < FP32_TOL


@pytest.mark.parametrize("name,g", GRAPHS[:4], ids=IDS[:4])
def test_skeleton_matches_oracle(bc, name, g):
    G = bc.graph_from_edgelist(g)
    S = gen.sample_targets(g.n, 40, seed=15)
    nodes, (au, av, aw, amu) = bc.skeleton(G, S, g.part)
    onodes, (ou, ov, ow, omu), _ = oracle.skeleton(g, S, g.part)
    assert np.array_equal(nodes, onodes)
    got = sorted(zip(au.tolist(), av.tolist(), aw.tolist(), amu.tolist()))
    ref = sorted(zip(ou.tolist(), ov.tolist(), ow.tolist(), omu.tolist()))
    assert got == ref


def test_brandes_pp_stats(bc):
    g = gen.planted_partition(600, 6, 0.04, 0.002, seed=16)
    S = gen.sample_targets(g.n, 50, seed=16)
    G = bc.graph_from_edgelist(g)
    _, st = bc.brandes_pp(G, S, g.part, stats=True)
    _, _, ost = oracle.brandes_pp(g, S, g.part)
    assert st["skel_nodes"] == ost["N"] and st["skel_edges"] == ost["M"]
    assert st["k"] == ost["k"] and st["lcs"] == ost["LCS"]


# ----------------------------------------------------------------------------- batched graphs
def test_batched_graphs(bc):
    gs = [gen.erdos_renyi(int(n), min(1.0, 6.0 / max(n - 1, 1)), seed=100 + i) for i, n in
          enumerate([64, 100, 37, 512, 2, 1, 300, 90, 129, 33, 700])]
    arena = bc.build_arena(gs)
    got = bc.brandes_batched(arena).cpu().numpy()
    got32 = bc.brandes_batched(arena, precision="fp32").cpu().numpy()
    off = arena.node_ptr_host
    for i, g in enumerate(gs):
        ref, _ = oracle.brandes(g)
        assert rel_err(got[off[i]:off[i + 1]], ref) < FP64_TOL, i
        assert rel_err(got32[off[i]:off[i + 1]], ref) < FP32_TOL, i


# ----------------------------------------------------------------------------- host buffers
def test_host_buffer_calls_match_device(bc):
    g = gen.planted_partition(500, 5, 0.04, 0.003, seed=17, wmax=5)
    S = gen.sample_targets(g.n, 60, seed=17)
    G = bc.graph_from_edgelist(g)
    H = bc.HostCSR.from_device(G)
    dev = bc.brandes(G, S).cpu().numpy()
    host = bc.brandes_host(H, S).numpy()
    assert np.array_equal(dev, host)
    dev_pp = bc.brandes_pp(G, S, g.part).cpu().numpy()
    host_pp = bc.brandes_pp_host(H, S, g.part).numpy()
    assert rel_err(host_pp, dev_pp) < FP64_TOL


# ----------------------------------------------------------------------------- source shards
@pytest.mark.parametrize("world", [2, 3])
def test_source_shards_add_up(bc, world):
    import torch
    g = gen.planted_partition(700, 7, 0.03, 0.002, seed=23, wmax=4)
    S = gen.sample_targets(g.n, 200, seed=23)
    G = bc.graph_from_edgelist(g)
    full = bc.brandes(G, S, halve=False).cpu().numpy()
    parts = sum(bc.brandes(G, S, halve=False, shard=(r, world)).cpu().numpy() for r in range(world))
    assert rel_err(parts, full) < FP64_TOL
    full_pp = bc.brandes_pp(G, S, g.part, halve=False).cpu().numpy()
    parts_pp = sum(bc.brandes_pp(G, S, g.part, halve=False, shard=(r, world)).cpu().numpy() for r in range(world))
    assert rel_err(parts_pp, full_pp) < FP64_TOL
    assert rel_err(full_pp, full) < FP64_TOL


# ----------------------------------------------------------------------------- 64-source batches
@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_brandes_64_source_batches(bc, name, g):
    """Two sources per lane (rows of 64): same results as the oracle, FP64 and FP32."""
    G = bc.graph_from_edgelist(g)
    ref, _ = oracle.brandes(g)
    assert rel_err(bc.brandes(G, batch=64).cpu().numpy(), ref) < FP64_TOL
    assert rel_err(bc.brandes(G, precision="fp32", batch=64).cpu().numpy(), ref) < FP32_TOL
    S = gen.sample_targets(g.n, 101, seed=41)
    ref_s, _ = oracle.brandes(g, S)
    assert rel_err(bc.brandes(G, S, batch=64).cpu().numpy(), ref_s) < FP64_TOL
    # Brandes++ with all-singleton parts has no non-frontier nodes: 64-source Brandes_SK
    assert rel_err(bc.brandes_pp(G, S, np.arange(g.n, dtype=np.int32), batch=64).cpu().numpy(), ref_s) < FP64_TOL


def test_batched_graphs_64_source_batches(bc):
    gs = [gen.erdos_renyi(int(n), min(1.0, 5.0 / max(n - 1, 1)), seed=200 + i) for i, n in
          enumerate([64, 65, 130, 7, 400, 1, 2, 257])]
    arena = bc.build_arena(gs)
    got = bc.brandes_batched(arena, batch=64).cpu().numpy()
    off = arena.node_ptr_host
    for i, g in enumerate(gs):
        ref, _ = oracle.brandes(g)
        assert rel_err(got[off[i]:off[i + 1]], ref) < FP64_TOL, i


def test_source_shards_64(bc):
    g = gen.planted_partition(700, 7, 0.03, 0.002, seed=42)
    S = gen.sample_targets(g.n, 333, seed=42)
    G = bc.graph_from_edgelist(g)
    full, _ = oracle.brandes(g, S, halve=False)
    parts = sum(bc.brandes(G, S, halve=False, shard=(r, 3), batch=64).cpu().numpy() for r in range(3))
    assert rel_err(parts, full) < FP64_TOL


def test_deep_unit_graphs(bc):
    """Deep unit-weight graphs (hundreds of levels) against their closed forms."""
    n = 600
    i = np.arange(n)
    G = bc.graph_from_edgelist(gen.path(n))
    assert rel_err(bc.brandes(G).cpu().numpy(), i * (n - 1 - i)) < FP64_TOL
    arena = bc.build_arena([gen.path(300), gen.cycle(700)])
    got = bc.brandes_batched(arena).cpu().numpy()
    ref_p = np.arange(300) * (299 - np.arange(300))
    k = 350
    assert rel_err(got[:300], ref_p) < FP64_TOL
    assert rel_err(got[300:], np.full(700, (k - 1) ** 2 / 2)) < FP64_TOL



def test_one_byte_distance_boundary(bc):
    """Unit-weight Brandes keeps distances in one byte per source while they stay below 254: a
    path of 254 nodes (longest distance 253) runs in one-byte rows, one of 255 nodes (254) makes
    the batch reaching it abort and the call rerun with int32 rows; both give the closed form,
    plain and batched."""
    for n in (254, 255):
        i = np.arange(n)
        G = bc.graph_from_edgelist(gen.path(n))
        assert rel_err(bc.brandes(G).cpu().numpy(), i * (n - 1 - i)) < FP64_TOL, n
        assert rel_err(bc.brandes(G, precision="fp32").cpu().numpy(), i * (n - 1 - i)) < FP32_TOL, n
    arena = bc.build_arena([gen.path(254), gen.path(255), gen.cycle(600)])
    got = bc.brandes_batched(arena).cpu().numpy()
    assert rel_err(got[:254], np.arange(254) * (253 - np.arange(254))) < FP64_TOL
    assert rel_err(got[254:509], np.arange(255) * (254 - np.arange(255))) < FP64_TOL
    assert rel_err(got[509:], np.full(600, (300 - 1) ** 2 / 2)) < FP64_TOL


# ----------------------------------------------------------------------------- CTA clusters per batch
def test_two_cta_clusters(bc):
    """Between 77 and 152 batches the library runs 2-CTA clusters per batch (4 with fewer,
    1 with more): plain Brandes and Brandes++ against the oracle in that regime."""
    g = gen.planted_partition(4000, 8, 0.006, 0.0004, seed=51, wmax=3)
    G = bc.graph_from_edgelist(g)
    ref, _ = oracle.brandes(g)                      # 125 batches of 32
    assert rel_err(bc.brandes(G).cpu().numpy(), ref) < FP64_TOL
    S = gen.sample_targets(g.n, 3000, seed=52)      # 94 batches
    ref_s, _ = oracle.brandes(g, S)
    assert rel_err(bc.brandes(G, S).cpu().numpy(), ref_s) < FP64_TOL
    assert rel_err(bc.brandes_pp(G, S, g.part).cpu().numpy(), ref_s) < FP64_TOL



# ----------------------------------------------------------------------------- Alg. 3
@pytest.mark.parametrize("name,g", GRAPHS[:4], ids=IDS[:4])
def test_brandes_pp_st_equals_oracle(bc, name, g):
    G = bc.graph_from_edgelist(g)
    src = gen.sample_targets(g.n, 60, seed=61)
    dst = gen.sample_targets(g.n, 90, seed=62)
    ref, _ = oracle.brandes_st(g, src, dst)
    got = bc.brandes_pp_st(G, src, dst, g.part).cpu().numpy()
    assert rel_err(got, ref) < FP64_TOL


@pytest.mark.parametrize("directed,wmax", [(False, None), (False, 5), (True, 7)])
def test_brandes_pp_all_equals_brandes(bc, directed, wmax):
    if directed:
        g = gen.chung_lu_communities(400, [100] * 4, 2.3, 5.0, 0.85, seed=63, directed=True, wmax=wmax)
    else:
        g = gen.planted_partition(400, 5, 0.05, 0.003, seed=64, wmax=wmax)
    G = bc.graph_from_edgelist(g)
    ref, _ = oracle.brandes(g)
    got, st = bc.brandes_pp_all(G, g.part, stats=True)
    assert rel_err(got.cpu().numpy(), ref) < FP64_TOL
    k = int(g.part.max()) + 1
    assert st["skel_edges"] == k * k


def test_brandes_pp_all_uneven_parts(bc):
    """Alg. 3 with an empty part and a one-node part, in both precisions: the pairs that run
    (every ordered pair of non-empty parts except a one-node part with itself) are counted, and
    the sum equals plain Brandes."""
    g = gen.planted_partition(300, 6, 0.06, 0.004, seed=65)
    part = np.asarray(g.part, np.int32).copy()
    part[part == 5] = 7          # part 5 left empty
    part[10] = 6                 # part 6 holds one node
    G = bc.graph_from_edgelist(g)
    ref, _ = oracle.brandes(g)
    got, st = bc.brandes_pp_all(G, part, k=8, stats=True)
    assert rel_err(got.cpu().numpy(), ref) < FP64_TOL
    nonempty = len(np.unique(part))
    assert st["skel_edges"] == nonempty * nonempty - 1
    got32 = bc.brandes_pp_all(G, part, k=8, precision="fp32").cpu().numpy()
    assert rel_err(got32, ref) < FP32_TOL
