"""Python binding of libbcpp (include/bcpp.h): argument marshalling only.

Every computation runs in the CUDA library; this module passes pointers and sizes.  PyTorch
provides device memory and the stream.  There is no CPU fallback: if the library is missing
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbcpp.so")

BCPP_OK, BCPP_EINVAL, BCPP_ENOMEM, BCPP_ECUDA, BCPP_ETIMEOUT, BCPP_EOVERFLOW_SIGMA, BCPP_ECAPACITY = range(7)
BCPP_FP64, BCPP_FP32_DELTA = 0, 1


class BcppError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bcpp error {code}: {msg}")
        self.code = code


class SigmaOverflow(BcppError):
    """A shortest-path count exceeded 2^64; the results were written but are not exact."""


class c_graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("num_arcs", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("w", ctypes.c_void_p), ("directed", ctypes.c_int32)]


class c_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("halve_undirected", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("validate", ctypes.c_int32), ("host_buffers", ctypes.c_int32),
                ("order_sources", ctypes.c_int32), ("cluster", ctypes.c_int32), ("shard_index", ctypes.c_int32),
                ("shard_count", ctypes.c_int32), ("pp_chunks", ctypes.c_int32)]


class c_stats(ctypes.Structure):
    _fields_ = [("sigma_overflow", ctypes.c_uint32), ("skel_nodes", ctypes.c_int32), ("skel_edges", ctypes.c_int64),
                ("k", ctypes.c_int32), ("lcs", ctypes.c_int32), ("table_entries", ctypes.c_int64),
                ("ms_build_sk", ctypes.c_float), ("ms_brandes_sk", ctypes.c_float),
                ("ms_centrality", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("kernel_launches", ctypes.c_int64), ("ms_batch_forward", ctypes.c_float),
                ("ms_batch_backward", ctypes.c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTS = ["bcpp_default_opts", "bcpp_strerror", "bcpp_create", "bcpp_destroy", "bcpp_workspace_bytes",
           "bcpp_csr_build", "bcpp_csr_validate", "bcpp_brandes", "bcpp_brandes_pp", "bcpp_brandes_batched",
           "bcpp_sssp", "bcpp_skeleton", "bcpp_brandes_noalloc", "bcpp_brandes_pp_st", "bcpp_brandes_pp_all",
           "bcpp_plan_brandes", "bcpp_plan_brandes_pp", "bcpp_plan_launch", "bcpp_plan_destroy", "bcpp_autotune",
           "bcpp_partition_lp", "bcpp_shard_bounds", "bcpp_autotune_batched"]

_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load libbcpp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libbcpp.so not found at {p}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        G, O, ST = ctypes.POINTER(c_graph), ctypes.POINTER(c_opts), ctypes.POINTER(c_stats)
        sig = {
            "bcpp_default_opts": (None, [O]),
            "bcpp_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "bcpp_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), P]),
            "bcpp_destroy": (None, [P]),
            "bcpp_workspace_bytes": (i64, [P]),
            "bcpp_csr_build": (ctypes.c_int, [P, i32, i64, P, P, P, i32, P, P, P, ctypes.POINTER(i64)]),
            "bcpp_csr_validate": (ctypes.c_int, [P, G]),
            "bcpp_brandes": (ctypes.c_int, [P, G, P, i32, O, P, ST]),
            "bcpp_brandes_pp": (ctypes.c_int, [P, G, P, i32, P, i32, O, P, ST]),
            "bcpp_brandes_batched": (ctypes.c_int, [P, i32, P, G, O, P, ST]),
            "bcpp_sssp": (ctypes.c_int, [P, G, P, i32, P, P, O]),
            "bcpp_skeleton": (ctypes.c_int, [P, G, P, i32, P, i32, P, ctypes.POINTER(i32), i64, P, P, P, P,
                                             ctypes.POINTER(i64), O]),
            "bcpp_brandes_noalloc": (ctypes.c_int, [G, P, i32, i32, P, P]),
            "bcpp_brandes_pp_st": (ctypes.c_int, [P, G, P, i32, P, i32, P, i32, O, P, ST]),
            "bcpp_brandes_pp_all": (ctypes.c_int, [P, G, P, i32, O, P, ST]),
            "bcpp_plan_brandes": (ctypes.c_int, [P, G, P, i32, O, P, ctypes.POINTER(ctypes.c_void_p)]),
            "bcpp_plan_brandes_pp": (ctypes.c_int, [P, G, P, i32, P, i32, O, P, ctypes.POINTER(ctypes.c_void_p)]),
            "bcpp_plan_launch": (ctypes.c_int, [P, ST]),
            "bcpp_plan_destroy": (None, [P]),
            "bcpp_autotune": (ctypes.c_int, [P, G, P, i32, O, O, ctypes.POINTER(ctypes.c_float)]),
            "bcpp_partition_lp": (ctypes.c_int, [P, G, i32, O, P, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "bcpp_shard_bounds": (ctypes.c_int, [i64, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
            "bcpp_autotune_batched": (ctypes.c_int, [P, i32, P, G, O, O, ctypes.POINTER(ctypes.c_float)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int, allow_overflow: bool = False):
    if rc == BCPP_OK:
        return
    msg = load_library().bcpp_strerror(rc).decode()
    if rc == BCPP_EOVERFLOW_SIGMA:
        if allow_overflow:
            return
        raise SigmaOverflow(rc, msg)
    raise BcppError(rc, msg)


def _torch():
    import torch
    return torch


class Context:
    """A library context bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("bcpp needs a CUDA device")
        lib = load_library()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.bcpp_create(ctypes.byref(h), ctypes.c_void_p(stream.cuda_stream)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load_library().bcpp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self) -> int:
        return int(load_library().bcpp_workspace_bytes(self.handle))


_default_ctx: dict = {}


def default_context() -> Context:
    torch = _torch()
    key = (torch.cuda.current_device(), torch.cuda.current_stream().cuda_stream)
    ctx = _default_ctx.get(key)
    if ctx is None:
        ctx = Context()
        _default_ctx[key] = ctx
    return ctx


@dataclass
class Graph:
    """CSR graph on the device (torch tensors): row_ptr int64 [n+1], col int32, w uint32-as-int32 or None."""
    n: int
    row_ptr: "object"
    col: "object"
    w: "object | None"
    directed: bool

    @property
    def num_arcs(self) -> int:
        return int(self.col.numel())

    def c(self) -> c_graph:
        return c_graph(self.n, self.num_arcs, self.row_ptr.data_ptr(), self.col.data_ptr() if self.num_arcs else None,
                       None if self.w is None else self.w.data_ptr(), int(self.directed))


def _opts(precision="fp64", halve=True, ctas_per_sm=0, host=False, order_sources=True, shard=None,
          batch=0, cluster=0, pp_chunks=0) -> c_opts:
    o = c_opts()
    load_library().bcpp_default_opts(ctypes.byref(o))
    o.precision = {"fp64": BCPP_FP64, "fp32": BCPP_FP32_DELTA, "fp32_delta": BCPP_FP32_DELTA}[precision]
    o.halve_undirected = 1 if halve else 0
    o.ctas_per_sm = int(ctas_per_sm)
    o.host_buffers = 1 if host else 0
    o.order_sources = 1 if order_sources else 0
    if shard is not None:
        o.shard_index, o.shard_count = int(shard[0]), int(shard[1])
    o.batch = int(batch)
    o.cluster = int(cluster)
    o.pp_chunks = int(pp_chunks)
    return o


def _dev_i32(x, device):
    torch = _torch()
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.int32).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.int32), device=device)


def shard_bounds(num_sources: int, index: int, count: int) -> tuple[int, int]:
    """Source positions [s0, s1) of shard `index` of `count` (bcpp_shard_bounds; host only):
    the rule behind the `shard=(index, count)` option of the betweenness calls."""
    s0, s1 = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load_library().bcpp_shard_bounds(int(num_sources), int(index), int(count), ctypes.byref(s0),
                                            ctypes.byref(s1)))
    return int(s0.value), int(s1.value)


# ----------------------------------------------------------------------------- CSR
def csr_build(n: int, src, dst, w=None, directed: bool = False, ctx: Context | None = None) -> Graph:
    """Device CSR from an edge list (bcpp_csr_build).  src/dst/w may be numpy or torch."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = torch.device("cuda", torch.cuda.current_device())
    eu, ev = _dev_i32(src, dev), _dev_i32(dst, dev)
    m = int(eu.numel())
    ew = None
    if w is not None:
        ew = (w.to(device=dev) if isinstance(w, torch.Tensor) else
              torch.as_tensor(np.ascontiguousarray(w, dtype=np.uint32).view(np.int32), device=dev)).contiguous()
    na = m if directed else 2 * m
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(na, 1), dtype=torch.int32, device=dev)
    wo = torch.empty(max(na, 1), dtype=torch.int32, device=dev) if ew is not None else None
    out_na = ctypes.c_int64(0)
    rc = load_library().bcpp_csr_build(ctx.handle, n, m, eu.data_ptr() if m else None, ev.data_ptr() if m else None,
                                       None if ew is None else ew.data_ptr(), int(directed), rp.data_ptr(),
                                       col.data_ptr(), None if wo is None else wo.data_ptr(), ctypes.byref(out_na))
    _check(rc)
    return Graph(n, rp, col[: out_na.value], None if wo is None else wo[: out_na.value], bool(directed))


def graph_from_edgelist(g, ctx: Context | None = None) -> Graph:
    """Device CSR of a generator EdgeList (built on the GPU)."""
    return csr_build(g.n, g.src, g.dst, g.w, g.directed, ctx)


def csr_validate(G: Graph, ctx: Context | None = None) -> None:
    ctx = ctx or default_context()
    cg = G.c()
    _check(load_library().bcpp_csr_validate(ctx.handle, ctypes.byref(cg)))


# ----------------------------------------------------------------------------- betweenness
def brandes(G: Graph, S=None, precision: str = "fp64", halve: bool = True, ctx: Context | None = None,
            ctas_per_sm: int = 0, out=None, stats: bool = False, allow_overflow: bool = False, shard=None,
            batch: int = 0, order_sources: bool = True, cluster: int = 0):
    """Plain Brandes, target set S (None = all nodes).  Returns a float64 device tensor [n]
    (and the stats dict when stats=True).  shard=(index, count) computes one shard's partial
    sum over the sources (the shards add up to the full result)."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = G.row_ptr.device
    St = _dev_i32(S, dev)
    nS = 0 if St is None else int(St.numel())
    bc = out if out is not None else torch.empty(G.n, dtype=torch.float64, device=dev)
    st = c_stats()
    cg = G.c()
    o = _opts(precision, halve, ctas_per_sm, shard=shard, batch=batch, order_sources=order_sources,
              cluster=cluster)
    rc = load_library().bcpp_brandes(ctx.handle, ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS,
                                     ctypes.byref(o), bc.data_ptr(), ctypes.byref(st))
    _check(rc, allow_overflow)
    return (bc, st.as_dict()) if stats else bc


def brandes_pp(G: Graph, S, part, k: int | None = None, precision: str = "fp64", halve: bool = True,
               ctx: Context | None = None, ctas_per_sm: int = 0, order_sources: bool = True, out=None,
               stats: bool = False, allow_overflow: bool = False, shard=None, batch: int = 0, cluster: int = 0,
               pp_chunks: int = 0):
    """Brandes++ (Build_SK, Brandes_SK, Centrality) for target set S (None = all nodes) and
    node partition `part` with values in [0, k).  pp_chunks=1 runs Brandes_SK in static chunks
    of batches (less memory) instead of one pass with a set of rows per batch."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = G.row_ptr.device
    St = _dev_i32(S, dev)
    nS = 0 if St is None else int(St.numel())
    pt = _dev_i32(part, dev)
    if k is None:
        k = int(pt.max().item()) + 1 if pt.numel() else 0
    bc = out if out is not None else torch.empty(G.n, dtype=torch.float64, device=dev)
    st = c_stats()
    cg = G.c()
    o = _opts(precision, halve, ctas_per_sm, order_sources=order_sources, shard=shard, batch=batch, cluster=cluster,
              pp_chunks=pp_chunks)
    rc = load_library().bcpp_brandes_pp(ctx.handle, ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS,
                                        pt.data_ptr(), int(k), ctypes.byref(o), bc.data_ptr(), ctypes.byref(st))
    _check(rc, allow_overflow)
    return (bc, st.as_dict()) if stats else bc


def brandes_pp_st(G: Graph, Ssrc, Sdst, part, k: int | None = None, precision: str = "fp64", halve: bool = True,
                  ctx: Context | None = None, out=None, stats: bool = False, allow_overflow: bool = False):
    """Brandes++ with separate source and destination sets (Alg. 3's Brandes_SK(G_sk, S_sc, S_dest)
    plus Centrality): sum over s in Ssrc, t in Sdst, s != t."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = G.row_ptr.device
    a, b = _dev_i32(Ssrc, dev), _dev_i32(Sdst, dev)
    pt = _dev_i32(part, dev)
    if k is None:
        k = int(pt.max().item()) + 1 if pt.numel() else 0
    bc = out if out is not None else torch.empty(G.n, dtype=torch.float64, device=dev)
    st = c_stats()
    cg = G.c()
    o = _opts(precision, halve)
    rc = load_library().bcpp_brandes_pp_st(ctx.handle, ctypes.byref(cg), a.data_ptr() if a.numel() else None,
                                           int(a.numel()), b.data_ptr() if b.numel() else None, int(b.numel()),
                                           pt.data_ptr(), int(k), ctypes.byref(o), bc.data_ptr(), ctypes.byref(st))
    _check(rc, allow_overflow)
    return (bc, st.as_dict()) if stats else bc


def brandes_pp_all(G: Graph, part, k: int | None = None, precision: str = "fp64", halve: bool = True,
                   ctx: Context | None = None, out=None, stats: bool = False, allow_overflow: bool = False):
    """Brandes++All (Alg. 3): full betweenness as the sum over all ordered pairs of parts."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = G.row_ptr.device
    pt = _dev_i32(part, dev)
    if k is None:
        k = int(pt.max().item()) + 1 if pt.numel() else 0
    bc = out if out is not None else torch.empty(G.n, dtype=torch.float64, device=dev)
    st = c_stats()
    cg = G.c()
    o = _opts(precision, halve)
    rc = load_library().bcpp_brandes_pp_all(ctx.handle, ctypes.byref(cg), pt.data_ptr(), int(k), ctypes.byref(o),
                                            bc.data_ptr(), ctypes.byref(st))
    _check(rc, allow_overflow)
    return (bc, st.as_dict()) if stats else bc


@dataclass
class Arena:
    """Independent undirected graphs as one disjoint-union CSR (global node ids)."""
    node_ptr: "object"      # int64 device [G+1]
    node_ptr_host: np.ndarray
    graph: Graph


AUTOTUNE_CANDIDATES = [(32, 1), (32, 2), (32, 4), (64, 1)]   # (batch, cluster), as in bcpp_autotune


def autotune(G: Graph, S=None, precision: str = "fp64", ctx: Context | None = None, order_sources: bool = True):
    """Time the launch-shape candidates on a sample of the sources (bcpp_autotune).  Returns
    ({"batch": b, "cluster": c}, {(batch, cluster): ms}) -- pass the first as keyword arguments
    to brandes / brandes_pp / plan_brandes."""
    ctx = ctx or default_context()
    dev = G.row_ptr.device
    St = _dev_i32(S, dev)
    nS = 0 if St is None else int(St.numel())
    o = _opts(precision, True, order_sources=order_sources)
    t = c_opts()
    ms = (ctypes.c_float * len(AUTOTUNE_CANDIDATES))()
    cg = G.c()
    rc = load_library().bcpp_autotune(ctx.handle, ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS,
                                      ctypes.byref(o), ctypes.byref(t), ms)
    _check(rc, allow_overflow=True)
    return {"batch": int(t.batch), "cluster": int(t.cluster)}, dict(zip(AUTOTUNE_CANDIDATES, [float(x) for x in ms]))


AUTOTUNE_BATCHED_CANDIDATES = [(32, 2), (64, 2), (32, 1), (64, 1)]   # (batch, ctas_per_sm)


def autotune_batched(arena: "Arena", precision: str = "fp64", ctx: Context | None = None):
    """Time the batched launch-shape candidates on the whole arena (bcpp_autotune_batched).
    Returns ({"batch": b, "ctas_per_sm": c}, {(batch, ctas_per_sm): ms}) -- pass the first as
    keyword arguments to brandes_batched."""
    ctx = ctx or default_context()
    o = _opts(precision, True)
    t = c_opts()
    ms = (ctypes.c_float * len(AUTOTUNE_BATCHED_CANDIDATES))()
    cg = arena.graph.c()
    rc = load_library().bcpp_autotune_batched(ctx.handle, len(arena.node_ptr_host) - 1, arena.node_ptr.data_ptr(),
                                              ctypes.byref(cg), ctypes.byref(o), ctypes.byref(t), ms)
    _check(rc, allow_overflow=True)
    return ({"batch": int(t.batch), "ctas_per_sm": int(t.ctas_per_sm)},
            dict(zip(AUTOTUNE_BATCHED_CANDIDATES, [float(x) for x in ms])))


def partition_lp(G: Graph, max_rounds: int = 20, ctx: Context | None = None):
    """Label-propagation partition (bcpp_partition_lp).  Returns (part int32 device tensor, k,
    rounds)."""
    torch = _torch()
    ctx = ctx or default_context()
    part = torch.empty(max(G.n, 1), dtype=torch.int32, device=G.row_ptr.device)
    k, r = ctypes.c_int32(0), ctypes.c_int32(0)
    cg = G.c()
    o = _opts()
    _check(load_library().bcpp_partition_lp(ctx.handle, ctypes.byref(cg), int(max_rounds), ctypes.byref(o),
                                            part.data_ptr(), ctypes.byref(k), ctypes.byref(r)))
    return part[: G.n], int(k.value), int(r.value)


class Plan:
    """A captured evaluation (bcpp_plan_brandes / bcpp_plan_brandes_pp): ``launch()`` replays its
    CUDA graph and returns the output tensor.  The plan holds references to the tensors it
    reads (graph arrays, targets ``S``, partition) and writes (``out``).  For a plain-Brandes
    plan, ``S`` (and the graph arrays) may be rewritten in place between launches, keeping their
    sizes; a Brandes++ plan's inputs must not change."""

    def __init__(self, handle, ctx, out, keep):
        self.handle = handle
        self.ctx = ctx
        self.out = out
        self._keep = keep
        self.S = keep.get("S")

    def launch(self, stats: bool = False, allow_overflow: bool = False):
        st = c_stats()
        rc = load_library().bcpp_plan_launch(self.handle, ctypes.byref(st))
        _check(rc, allow_overflow)
        return (self.out, st.as_dict()) if stats else self.out

    def close(self):
        if getattr(self, "handle", None):
            load_library().bcpp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_brandes(G: Graph, S=None, precision: str = "fp64", halve: bool = True, ctx: Context | None = None,
                 out=None, batch: int = 0, order_sources: bool = True, cluster: int = 0, ctas_per_sm: int = 0,
                 shard=None) -> Plan:
    """Capture plain Brandes on (G, S) into a replayable plan (bcpp_plan_brandes)."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = G.row_ptr.device
    St = _dev_i32(S, dev)
    nS = 0 if St is None else int(St.numel())
    bc = out if out is not None else torch.empty(G.n, dtype=torch.float64, device=dev)
    cg = G.c()
    o = _opts(precision, halve, ctas_per_sm, shard=shard, batch=batch, order_sources=order_sources, cluster=cluster)
    h = ctypes.c_void_p()
    rc = load_library().bcpp_plan_brandes(ctx.handle, ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS,
                                          ctypes.byref(o), bc.data_ptr(), ctypes.byref(h))
    _check(rc)
    return Plan(h, ctx, bc, {"G": G, "S": St})


def plan_brandes_pp(G: Graph, S, part, k: int | None = None, precision: str = "fp64", halve: bool = True,
                    ctx: Context | None = None, out=None, batch: int = 0, order_sources: bool = True,
                    cluster: int = 0, ctas_per_sm: int = 0, shard=None) -> Plan:
    """Build the skeleton and capture Brandes++'s per-source work into a plan (bcpp_plan_brandes_pp)."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = G.row_ptr.device
    St = _dev_i32(S, dev)
    nS = 0 if St is None else int(St.numel())
    pt = _dev_i32(part, dev)
    if k is None:
        k = int(pt.max().item()) + 1 if pt.numel() else 0
    bc = out if out is not None else torch.empty(G.n, dtype=torch.float64, device=dev)
    cg = G.c()
    o = _opts(precision, halve, ctas_per_sm, shard=shard, batch=batch, order_sources=order_sources, cluster=cluster)
    h = ctypes.c_void_p()
    rc = load_library().bcpp_plan_brandes_pp(ctx.handle, ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS,
                                             pt.data_ptr(), int(k), ctypes.byref(o), bc.data_ptr(), ctypes.byref(h))
    _check(rc)
    return Plan(h, ctx, bc, {"G": G, "S": St, "part": pt})


def build_arena(graphs, ctx: Context | None = None) -> Arena:
    """Pack generator EdgeLists into one disjoint-union CSR, built on the device."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = torch.device("cuda", torch.cuda.current_device())
    ns = np.array([g.n for g in graphs], np.int64)
    node_ptr = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    offs = np.repeat(node_ptr[:-1], [g.m for g in graphs])
    src = (np.concatenate([g.src for g in graphs]).astype(np.int64) + offs).astype(np.int32)
    dst = (np.concatenate([g.dst for g in graphs]).astype(np.int64) + offs).astype(np.int32)
    G = csr_build(int(node_ptr[-1]), src, dst, None, False, ctx)
    return Arena(torch.as_tensor(node_ptr, device=dev), node_ptr, G)


def brandes_batched(arena: Arena, precision: str = "fp64", halve: bool = True, ctx: Context | None = None,
                    ctas_per_sm: int = 0, out=None, stats: bool = False, allow_overflow: bool = False,
                    batch: int = 0):
    """Full betweenness of every graph of the arena in one launch."""
    torch = _torch()
    ctx = ctx or default_context()
    G = arena.graph
    bc = out if out is not None else torch.empty(G.n, dtype=torch.float64, device=G.row_ptr.device)
    st = c_stats()
    cg = G.c()
    o = _opts(precision, halve, ctas_per_sm, batch=batch)
    rc = load_library().bcpp_brandes_batched(ctx.handle, len(arena.node_ptr_host) - 1, arena.node_ptr.data_ptr(),
                                             ctypes.byref(cg), ctypes.byref(o), bc.data_ptr(), ctypes.byref(st))
    _check(rc, allow_overflow)
    return (bc, st.as_dict()) if stats else bc


def brandes_batched_host(H: "HostCSR", node_ptr_host, precision: str = "fp64", halve: bool = True,
                         ctx: Context | None = None, out=None, stats: bool = False, allow_overflow: bool = False):
    """Batched full betweenness with the arena CSR, its node offsets and the result in (pinned)
    host memory; the library copies in and out."""
    torch = _torch()
    ctx = ctx or default_context()
    off = torch.as_tensor(np.asarray(node_ptr_host, np.int64)).pin_memory()
    bc = out if out is not None else torch.empty(H.n, dtype=torch.float64).pin_memory()
    st = c_stats()
    cg = H.c()
    o = _opts(precision, halve, host=True)
    rc = load_library().bcpp_brandes_batched(ctx.handle, int(off.numel()) - 1, off.data_ptr(), ctypes.byref(cg),
                                             ctypes.byref(o), bc.data_ptr(), ctypes.byref(st))
    _check(rc, allow_overflow)
    return (bc, st.as_dict()) if stats else bc


def sssp(G: Graph, src, ctx: Context | None = None, allow_overflow: bool = False):
    """Distances (int32, INT32_MAX = unreachable) and uint64 path counts (as int64 bits)
    from each source: two device tensors [len(src), n]."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = G.row_ptr.device
    s = _dev_i32(src, dev)
    ns = int(s.numel())
    dist = torch.empty((ns, G.n), dtype=torch.int32, device=dev)
    sig = torch.empty((ns, G.n), dtype=torch.int64, device=dev)
    cg = G.c()
    o = _opts()
    rc = load_library().bcpp_sssp(ctx.handle, ctypes.byref(cg), s.data_ptr() if ns else None, ns,
                                  dist.data_ptr(), sig.data_ptr(), ctypes.byref(o))
    _check(rc, allow_overflow)
    return dist, sig


def skeleton(G: Graph, S, part, k: int | None = None, ctx: Context | None = None):
    """The skeleton of Build_SK: (nodes, (u, v, weight, multiplicity)) as numpy arrays in
    original node ids (S=None or empty: no targets)."""
    torch = _torch()
    ctx = ctx or default_context()
    dev = G.row_ptr.device
    St = _dev_i32(S, dev)
    nS = 0 if St is None else int(St.numel())
    pt = _dev_i32(part, dev)
    if k is None:
        k = int(pt.max().item()) + 1 if pt.numel() else 0
    lib = load_library()
    cg = G.c()
    o = _opts()
    nodes = torch.empty(max(G.n, 1), dtype=torch.int32, device=dev)
    nsk = ctypes.c_int32(0)
    na = ctypes.c_int64(0)
    cap = 0
    rc = lib.bcpp_skeleton(ctx.handle, ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS, pt.data_ptr(),
                           int(k), nodes.data_ptr(), ctypes.byref(nsk), cap, None, None, None, None, ctypes.byref(na),
                           ctypes.byref(o))
    if rc not in (BCPP_OK, BCPP_ECAPACITY):
        _check(rc)
    cap = int(na.value)
    au = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    av = torch.empty_like(au)
    aw = torch.empty_like(au)
    amu = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
    rc = lib.bcpp_skeleton(ctx.handle, ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS, pt.data_ptr(),
                           int(k), nodes.data_ptr(), ctypes.byref(nsk), cap, au.data_ptr(), av.data_ptr(),
                           aw.data_ptr(), amu.data_ptr(), ctypes.byref(na), ctypes.byref(o))
    _check(rc)
    n_sk, n_a = int(nsk.value), int(na.value)
    return (nodes[:n_sk].cpu().numpy(),
            (au[:n_a].cpu().numpy(), av[:n_a].cpu().numpy(), aw[:n_a].cpu().numpy(),
             amu[:n_a].cpu().numpy().view(np.uint64)))


# ----------------------------------------------------------------------------- host buffers (end to end)
class HostCSR:
    """A CSR in pinned host memory, for the end-to-end calls (host_buffers = 1)."""

    def __init__(self, n, row_ptr, col, w, directed):
        torch = _torch()
        self.n = int(n)
        self.directed = bool(directed)
        self.row_ptr = torch.as_tensor(np.asarray(row_ptr, np.int64)).pin_memory()
        self.col = torch.as_tensor(np.asarray(col, np.int32)).pin_memory()
        self.w = None if w is None else torch.as_tensor(np.asarray(w).astype(np.uint32).view(np.int32)).pin_memory()

    def c(self) -> c_graph:
        return c_graph(self.n, int(self.col.numel()), self.row_ptr.data_ptr(),
                       self.col.data_ptr() if self.col.numel() else None,
                       None if self.w is None else self.w.data_ptr(), int(self.directed))

    @staticmethod
    def from_device(G: Graph) -> "HostCSR":
        return HostCSR(G.n, G.row_ptr.cpu().numpy(), G.col.cpu().numpy(),
                       None if G.w is None else G.w.cpu().numpy().view(np.uint32), G.directed)


def brandes_host(H: HostCSR, S=None, precision="fp64", halve=True, ctx: Context | None = None, out=None,
                 stats: bool = False, allow_overflow: bool = False, shard=None):
    """Plain Brandes with every array in (pinned) host memory; the library copies in and out."""
    torch = _torch()
    ctx = ctx or default_context()
    St = None if S is None else torch.as_tensor(np.asarray(S, np.int32)).pin_memory()
    nS = 0 if St is None else int(St.numel())
    bc = out if out is not None else torch.empty(H.n, dtype=torch.float64).pin_memory()
    st = c_stats()
    cg = H.c()
    o = _opts(precision, halve, host=True, shard=shard)
    rc = load_library().bcpp_brandes(ctx.handle, ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS,
                                     ctypes.byref(o), bc.data_ptr(), ctypes.byref(st))
    _check(rc, allow_overflow)
    return (bc, st.as_dict()) if stats else bc


def brandes_pp_host(H: HostCSR, S, part, k=None, precision="fp64", halve=True, ctx: Context | None = None, out=None,
                    stats: bool = False, allow_overflow: bool = False, shard=None):
    """Brandes++ with every array in (pinned) host memory; the library copies in and out."""
    torch = _torch()
    ctx = ctx or default_context()
    St = None if S is None else torch.as_tensor(np.asarray(S, np.int32)).pin_memory()
    nS = 0 if St is None else int(St.numel())
    pt = torch.as_tensor(np.asarray(part, np.int32)).pin_memory()
    if k is None:
        k = int(pt.max().item()) + 1 if pt.numel() else 0
    bc = out if out is not None else torch.empty(H.n, dtype=torch.float64).pin_memory()
    st = c_stats()
    cg = H.c()
    o = _opts(precision, halve, host=True, shard=shard)
    rc = load_library().bcpp_brandes_pp(ctx.handle, ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS,
                                        pt.data_ptr(), int(k), ctypes.byref(o), bc.data_ptr(), ctypes.byref(st))
    _check(rc, allow_overflow)
    return (bc, st.as_dict()) if stats else bc


def brandes_noalloc(G: Graph, S=None, halve: bool = True, out=None, stream=None, allow_overflow: bool = False):
    """Plain Brandes through bcpp_brandes_noalloc: no library allocation (scratch is a static
    device array), for undirected graphs of at most 4,096 nodes and weights <= 15.  For
    callers that cannot allocate device memory; `out` may be a caller-owned float64 tensor."""
    torch = _torch()
    dev = G.row_ptr.device
    St = _dev_i32(S, dev)
    nS = 0 if St is None else int(St.numel())
    if out is not None and (out.dtype != torch.float64 or out.numel() < G.n or not out.is_contiguous()
                            or out.device != dev):
        raise BcppError(BCPP_EINVAL, "out must be a contiguous float64 tensor of at least n elements "
                                     "on the graph's device")
    bc = out if out is not None else torch.empty(G.n, dtype=torch.float64, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream()
    cg = G.c()
    rc = load_library().bcpp_brandes_noalloc(ctypes.byref(cg), None if nS == 0 else St.data_ptr(), nS,
                                             1 if halve else 0, bc.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    _check(rc, allow_overflow)
    return bc
