"""GPU: the label-propagation partition (bcpp_partition_lp) is the oracle's, label for label,
and Brandes++ on it gives the oracle's betweenness (Brandes++ is exact for every partition)."""
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


CASES = [
    ("path", gen.path(37)),
    ("star-hub", gen.star(200)),                                                    # 199 neighbours
    ("planted", gen.planted_partition(700, 7, 0.03, 0.002, seed=1)),
    ("chunglu-hubs", gen.chung_lu_communities(1500, [300] * 5, 2.1, 8.0, 0.9, seed=6)),
    ("chunglu-directed", gen.chung_lu_communities(800, [200] * 4, 2.3, 6.0, 0.85, seed=3, directed=True)),
    ("er-isolated", gen.erdos_renyi(900, 1.5 / 900, seed=5)),
]


@pytest.mark.parametrize("name,g", CASES, ids=[c[0] for c in CASES])
def test_partition_equals_oracle(bc, name, g):
    ref, k_ref, r_ref = oracle.label_propagation(g, max_rounds=30)
    G = bc.graph_from_edgelist(g)
    part, k, r = bc.partition_lp(G, max_rounds=30)
    assert np.array_equal(part.cpu().numpy(), ref), name
    assert (k, r) == (k_ref, r_ref)


def test_brandes_pp_on_label_propagation_partition(bc):
    g = gen.chung_lu_communities(2000, [400] * 5, 2.3, 8.0, 0.9, seed=12)
    G = bc.graph_from_edgelist(g)
    part, k, _ = bc.partition_lp(G)
    S = gen.sample_targets(g.n, 300, seed=3)
    ref, _ = oracle.brandes(g, S)
    got = bc.brandes_pp(G, S, part, k).cpu().numpy()
    assert float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0))) < 1e-12


def test_partition_host_buffers(bc):
    """The host-buffer form of bcpp_partition_lp gives the device form's labels."""
    import ctypes
    from paper_1406_4173_gb300 import api
    g = gen.planted_partition(500, 5, 0.04, 0.002, seed=9)
    G = bc.graph_from_edgelist(g)
    dev, k, r = bc.partition_lp(G)
    H = bc.HostCSR.from_device(G)
    part = np.empty(g.n, np.int32)
    kk, rr = ctypes.c_int32(0), ctypes.c_int32(0)
    o = api._opts(host=True)
    cg = H.c()
    rc = api.load_library().bcpp_partition_lp(bc.default_context().handle, ctypes.byref(cg), 20, ctypes.byref(o),
                                              part.ctypes.data, ctypes.byref(kk), ctypes.byref(rr))
    assert rc == 0
    assert np.array_equal(part, dev.cpu().numpy()) and (kk.value, rr.value) == (k, r)
