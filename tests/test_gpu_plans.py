"""GPU parity of captured plans (bcpp_plan_*): a replayed CUDA graph against the CPU oracle.

Replays must give the oracle's betweenness (FP64 to a relative 1e-12, FP32-delta to the FP32
tolerance of the other parity tests), a plain-Brandes plan must follow in-place rewrites of
its target set, and a plan must refuse (on the device, before computing) a rewritten target
set that is invalid.
"""
import numpy as np
import pytest

import oracle
from paper_1406_4173_gb300 import gen

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-6        # 10x the largest measured error on these graphs (1.96e-7)


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


CASES = [
    ("planted-u", gen.planted_partition(900, 9, 0.03, 0.002, seed=11), None),
    ("planted-w", gen.planted_partition(700, 7, 0.03, 0.003, seed=12, wmax=9), None),
    ("chunglu-dw", gen.chung_lu_communities(800, [160] * 5, 2.3, 6.0, 0.85, seed=13, directed=True, wmax=16), None),
]


@pytest.mark.parametrize("name,g,_", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("allS", [False, True], ids=["S-sub", "S-all"])
def test_plan_plain_replays_match_oracle(bc, name, g, _, allS):
    G = bc.graph_from_edgelist(g)
    S = None if allS else gen.sample_targets(g.n, 301, seed=5)
    ref, _ovf = oracle.brandes(g, S)
    plan = bc.plan_brandes(G, S)
    try:
        x1, st = plan.launch(stats=True)
        x1 = x1.cpu().numpy().copy()
        x2 = plan.launch().cpu().numpy()
        assert rel_err(x1, ref) <= FP64_TOL, name
        assert rel_err(x2, ref) <= FP64_TOL, name
        assert st["kernel_launches"] >= 2
        direct = bc.brandes(G, S).cpu().numpy()
        assert rel_err(x2, direct) <= FP64_TOL
    finally:
        plan.close()


def test_plan_plain_follows_rewritten_targets(bc):
    import torch
    g = gen.planted_partition(1000, 10, 0.03, 0.002, seed=21)
    G = bc.graph_from_edgelist(g)
    S1 = gen.sample_targets(g.n, 200, seed=1)
    S2 = gen.sample_targets(g.n, 200, seed=2)
    plan = bc.plan_brandes(G, S1)
    try:
        assert rel_err(plan.launch().cpu().numpy(), oracle.brandes(g, S1)[0]) <= FP64_TOL
        plan.S.copy_(torch.as_tensor(S2, dtype=torch.int32, device=plan.S.device))
        assert rel_err(plan.launch().cpu().numpy(), oracle.brandes(g, S2)[0]) <= FP64_TOL
        # a repeated target is refused by the device-side check, before any computation
        bad = S2.copy()
        bad[7] = bad[3]
        plan.S.copy_(torch.as_tensor(bad, dtype=torch.int32, device=plan.S.device))
        with pytest.raises(bc.BcppError):
            plan.launch()
        # an out-of-range target as well
        bad = S2.copy()
        bad[0] = g.n + 5
        plan.S.copy_(torch.as_tensor(bad, dtype=torch.int32, device=plan.S.device))
        with pytest.raises(bc.BcppError):
            plan.launch()
        # and a valid set works again afterwards
        plan.S.copy_(torch.as_tensor(S1, dtype=torch.int32, device=plan.S.device))
        assert rel_err(plan.launch().cpu().numpy(), oracle.brandes(g, S1)[0]) <= FP64_TOL
    finally:
        plan.close()


def test_plan_plain_fp32_delta(bc):
    g = gen.chung_lu_communities(1500, [300] * 5, 2.1, 8.0, 0.9, seed=6)
    G = bc.graph_from_edgelist(g)
    ref, _ = oracle.brandes(g, None)
    plan = bc.plan_brandes(G, None, precision="fp32")
    try:
        assert rel_err(plan.launch().cpu().numpy(), ref) <= FP32_TOL
    finally:
        plan.close()


@pytest.mark.parametrize("name,g,_", CASES, ids=[c[0] for c in CASES])
def test_plan_brandes_pp_replays_match_oracle(bc, name, g, _):
    G = bc.graph_from_edgelist(g)
    S = gen.sample_targets(g.n, 150, seed=9)
    ref, _ovf = oracle.brandes(g, S)
    plan = bc.plan_brandes_pp(G, S, g.part)
    try:
        x1, st = plan.launch(stats=True)
        x1 = x1.cpu().numpy().copy()
        x2 = plan.launch().cpu().numpy()
        assert rel_err(x1, ref) <= FP64_TOL, name
        assert rel_err(x2, ref) <= FP64_TOL, name
        assert st["skel_nodes"] > 0
        _, st_direct = bc.brandes_pp(G, S, g.part, stats=True)
        assert st["skel_nodes"] == st_direct["skel_nodes"] and st["skel_edges"] == st_direct["skel_edges"]
    finally:
        plan.close()


def test_plan_trivial_target_set(bc):
    g = gen.planted_partition(300, 3, 0.05, 0.01, seed=3)
    G = bc.graph_from_edgelist(g)
    S = np.array([4], np.int32)          # |S| < 2: all zeros
    for make in (lambda: bc.plan_brandes(G, S), lambda: bc.plan_brandes_pp(G, S, g.part)):
        plan = make()
        try:
            assert not np.any(plan.launch().cpu().numpy())
        finally:
            plan.close()


def test_plan_directed_weighted_fp32_shard(bc):
    """A plan of a directed weighted graph in FP32-delta mode and a source shard: the shard's
    replay equals the oracle's partial over the same sources (batching in the given order)."""
    g = gen.chung_lu_communities(900, [180] * 5, 2.3, 6.0, 0.85, seed=17, directed=True, wmax=12)
    G = bc.graph_from_edgelist(g)
    S = gen.sample_targets(g.n, 320, seed=8)
    ref, _ = oracle.brandes(g, S, nsrc=160)                 # shard 0 of 2: the first 160 targets
    plan = bc.plan_brandes(G, S, precision="fp32", shard=(0, 2), order_sources=False)
    try:
        assert rel_err(plan.launch().cpu().numpy(), ref) <= FP32_TOL
        assert rel_err(plan.launch().cpu().numpy(), ref) <= FP32_TOL
    finally:
        plan.close()
