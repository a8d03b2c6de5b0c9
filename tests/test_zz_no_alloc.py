"""bcpp_brandes_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (a host whose own allocator owns all device memory, or a latency-critical path
that cannot afford an allocation) get plain Brandes with all scratch in a static device
array.  This test calls it through the C ABI and checks it against bcpp_brandes (the
allocating entry point) within the FP64 parity tolerance, on two calls in a row (the second
call must not see the first call's leftovers), and checks that oversized inputs are refused
before any GPU work.  The file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1406_4173_gb300 import gen

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


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
def test_noalloc_matches_brandes_twice(bc, weighted):
    g1 = gen.planted_partition(900, 6, 0.03, 0.002, seed=31, wmax=7 if weighted else None)
    g2 = gen.chung_lu_communities(4096, [1024] * 4, 2.3, 8.0, 0.9, seed=32, wmax=15 if weighted else None)
    for g, S in ((g1, gen.sample_targets(g1.n, 150, seed=33)), (g2, None)):
        G = bc.graph_from_edgelist(g)
        ref = bc.brandes(G, S).cpu().numpy()
        first = bc.brandes_noalloc(G, S).cpu().numpy()
        second = bc.brandes_noalloc(G, S).cpu().numpy()
        assert rel_err(first, ref) < FP64_TOL
        assert rel_err(second, ref) < FP64_TOL


def test_noalloc_rejects_oversized_inputs(bc):
    big = gen.erdos_renyi(4097, 3.0 / 4096, seed=34)
    G = bc.graph_from_edgelist(big)
    with pytest.raises(bc.BcppError):
        bc.brandes_noalloc(G)
    heavy = gen.planted_partition(200, 2, 0.1, 0.01, seed=35, wmax=40)
    with pytest.raises(bc.BcppError):
        bc.brandes_noalloc(bc.graph_from_edgelist(heavy))
    directed = gen.erdos_renyi(100, 0.05, seed=36, directed=True)
    with pytest.raises(bc.BcppError):
        bc.brandes_noalloc(bc.graph_from_edgelist(directed))
