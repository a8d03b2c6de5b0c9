"""bcpp_brandes_noalloc: the entry point for callers that cannot allocate device memory.

Such callers -- a host whose own allocator owns all device memory, or a latency-critical path
that cannot afford an allocation -- get plain Brandes with all scratch in a static device
array.  This test calls it through the C ABI and checks:

- its output against the CPU oracle within the FP64 parity tolerance, on two calls in a row,
  with a smaller graph right after a larger one (the second call must not see the first
  call's leftovers past the smaller size), and on a deep weighted path (every batch records
  tens of thousands of distinct distances);
- that a call allocates nothing: after a warm-up call, the device's free memory is the same
  before and after a call;
- that oversized or invalid inputs and unusable output tensors are refused.

The file is named to be collected last.
"""
import numpy as np
import pytest

import oracle
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
def test_noalloc_matches_oracle_twice(bc, weighted):
    big = gen.chung_lu_communities(4096, [1024] * 4, 2.3, 8.0, 0.9, seed=32, wmax=15 if weighted else None)
    small = gen.planted_partition(900, 6, 0.03, 0.002, seed=31, wmax=7 if weighted else None)
    # the larger graph first, so that the smaller one runs over the larger one's leftovers
    for g, S in ((big, None), (small, gen.sample_targets(small.n, 150, seed=33)), (small, None)):
        ref, _ = oracle.brandes(g, S)
        G = bc.graph_from_edgelist(g)
        first = bc.brandes_noalloc(G, S).cpu().numpy()
        second = bc.brandes_noalloc(G, S).cpu().numpy()
        assert rel_err(first, ref) < FP64_TOL
        assert rel_err(second, ref) < FP64_TOL


def test_noalloc_deep_weighted_path(bc):
    """A path of 4,096 nodes with every weight 15: distances up to 61,425, the deepest input
    the fixed limits admit.  Betweenness on a path is i (n - 1 - i) whatever the weights."""
    n = 4096
    p = gen.path(n)
    g = gen.EdgeList(n=n, src=p.src, dst=p.dst, w=np.full(p.m, 15, np.uint32))
    G = bc.graph_from_edgelist(g)
    i = np.arange(n)
    ref, _ = oracle.brandes(g)
    assert rel_err(ref, i * (n - 1 - i)) < FP64_TOL
    for _ in range(2):
        assert rel_err(bc.brandes_noalloc(G).cpu().numpy(), ref) < FP64_TOL


def test_noalloc_allocates_nothing(bc):
    import torch
    g = gen.planted_partition(2000, 8, 0.01, 0.001, seed=37, wmax=5)
    S = gen.sample_targets(g.n, 300, seed=38)
    G = bc.graph_from_edgelist(g)
    St = torch.as_tensor(S, device=G.row_ptr.device)
    out = torch.empty(g.n, dtype=torch.float64, device=G.row_ptr.device)
    bc.brandes_noalloc(G, St, out=out)            # warm-up: kernels load on their first launch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    bc.brandes_noalloc(G, St, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref, _ = oracle.brandes(g, S)
    assert rel_err(out.cpu().numpy(), ref) < FP64_TOL


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


def test_noalloc_rejects_unusable_output(bc):
    import torch
    g = gen.planted_partition(300, 3, 0.05, 0.01, seed=39)
    G = bc.graph_from_edgelist(g)
    dev = G.row_ptr.device
    for out in (torch.empty(g.n - 1, dtype=torch.float64, device=dev),
                torch.empty(g.n, dtype=torch.float32, device=dev),
                torch.empty(2 * g.n, dtype=torch.float64, device=dev)[::2],
                torch.empty(g.n, dtype=torch.float64)):
        with pytest.raises(bc.BcppError):
            bc.brandes_noalloc(G, out=out)
    # a call after the refusals still gives the right answer
    ref, _ = oracle.brandes(g)
    assert rel_err(bc.brandes_noalloc(G).cpu().numpy(), ref) < FP64_TOL
