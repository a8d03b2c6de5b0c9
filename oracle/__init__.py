"""CPU oracle for exact betweenness centrality (plain Brandes and Brandes++).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU-baseline
leg are the only callers.  The product library never imports this package, and this package
imports nothing from the product library.

``bc_oracle.c`` holds the numerics (plain C, FP64, uint64 path counts with an overflow
flag); this module compiles it with gcc on first use and wraps it with ctypes.
``bruteforce.py`` enumerates shortest paths with exact fractions for tiny graphs.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py`` (brute force,
closed forms, invariants, Brandes++ = Brandes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bc_oracle.c")
_LIB = os.path.join(_HERE, "_bc_oracle.so")
_lock = threading.Lock()
_lib = None

_ERR = {1: "EINVAL", 2: "ENOMEM"}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, portable flags: x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.orc_sssp.argtypes = [i32, i64, P, P, P, i32, i32, P, P, P]
            lib.orc_brandes.argtypes = [i32, i64, P, P, P, i32, P, i32, i32, i32, P, P]
            lib.orc_brandes_pp.argtypes = [i32, i64, P, P, P, i32, P, i32, i32, P, i32, i32, P, P, P]
            lib.orc_skeleton.argtypes = [i32, i64, P, P, P, i32, P, i32, P, i32, P, P, i64, P, P, P, P, P, P]
            lib.orc_distance_sum.argtypes = [i32, i64, P, P, i32, P, i32, P]
            lib.orc_brandes_st.argtypes = [i32, i64, P, P, P, i32, P, i32, P, i32, i32, P, P]
            lib.orc_label_propagation.argtypes = [i32, i64, P, P, i32, i32, P, P, P]
            for f in (lib.orc_sssp, lib.orc_brandes, lib.orc_brandes_pp, lib.orc_skeleton, lib.orc_distance_sum,
                      lib.orc_brandes_st, lib.orc_label_propagation):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _edges(g):
    eu = np.ascontiguousarray(g.src, np.int32)
    ev = np.ascontiguousarray(g.dst, np.int32)
    ew = None if g.w is None else np.ascontiguousarray(g.w, np.uint32)
    return eu, ev, ew


def _check(rc, what):
    if rc:
        raise ValueError(f"oracle {what}: {_ERR.get(rc, rc)}")


def sssp(g, src: int):
    """Distances (int32, INT32_MAX = unreachable) and uint64 path counts from one source
    (Eq. 2).  Returns (dist, sigma, overflow)."""
    lib = _load()
    eu, ev, ew = _edges(g)
    dist = np.empty(g.n, np.int32)
    sig = np.empty(g.n, np.uint64)
    ovf = np.zeros(1, np.uint32)
    _check(lib.orc_sssp(g.n, g.m, _ptr(eu), _ptr(ev), _ptr(ew), int(g.directed), int(src),
                        _ptr(dist), _ptr(sig), _ptr(ovf)), "sssp")
    return dist, sig, bool(ovf[0])


def brandes(g, S=None, nsrc: int = -1, halve: bool | None = None):
    """Target-set betweenness C^S (Eq. 5) by Brandes' recursion (Eq. 7).

    S=None means S = V.  Sources are the first ``nsrc`` entries of S (all if negative);
    targets are all of S.  ``halve`` defaults to True for undirected graphs (unordered pairs).
    Returns (bc float64[n], overflow)."""
    lib = _load()
    eu, ev, ew = _edges(g)
    Sa = None if S is None else np.ascontiguousarray(S, np.int32)
    nS = 0 if Sa is None else int(Sa.shape[0])
    if halve is None:
        halve = not g.directed
    bc = np.empty(g.n, np.float64)
    ovf = np.zeros(1, np.uint32)
    _check(lib.orc_brandes(g.n, g.m, _ptr(eu), _ptr(ev), _ptr(ew), int(g.directed), _ptr(Sa), nS,
                           int(nsrc), int(bool(halve)), _ptr(bc), _ptr(ovf)), "brandes")
    return bc, bool(ovf[0])


def brandes_pp(g, S, part, k: int | None = None, nsrc: int = -1, halve: bool | None = None):
    """Brandes++ (Alg. 1): Build_SK, Brandes_SK, Centrality.  Returns (bc, overflow, stats)
    with stats = dict(N, M, k, LCS) of the skeleton and of the partition P'."""
    lib = _load()
    eu, ev, ew = _edges(g)
    Sa = np.ascontiguousarray(np.arange(g.n) if S is None else S, np.int32)
    pa = np.ascontiguousarray(part, np.int32)
    if k is None:
        k = int(pa.max()) + 1 if pa.size else 0
    if halve is None:
        halve = not g.directed
    bc = np.empty(g.n, np.float64)
    ovf = np.zeros(1, np.uint32)
    st = np.zeros(4, np.int64)
    _check(lib.orc_brandes_pp(g.n, g.m, _ptr(eu), _ptr(ev), _ptr(ew), int(g.directed), _ptr(Sa),
                              int(Sa.shape[0]), int(nsrc), _ptr(pa), int(k), int(bool(halve)), _ptr(bc),
                              _ptr(ovf), _ptr(st)), "brandes_pp")
    return bc, bool(ovf[0]), dict(N=int(st[0]), M=int(st[1]), k=int(st[2]), LCS=int(st[3]))


def skeleton(g, S, part, k: int | None = None):
    """Skeleton of Build_SK: (nodes, arcs) with arcs as int arrays (u, v, weight, multiplicity)
    in original node ids; undirected edges appear in both directions."""
    lib = _load()
    eu, ev, ew = _edges(g)
    Sa = np.ascontiguousarray(np.arange(g.n) if S is None else S, np.int32)
    pa = np.ascontiguousarray(part, np.int32)
    if k is None:
        k = int(pa.max()) + 1 if pa.size else 0
    nodes = np.empty(max(g.n, 1), np.int32)
    nsk = np.zeros(1, np.int32)
    cap = 2 * g.m + 16
    while True:
        au = np.empty(cap, np.int32); av = np.empty(cap, np.int32)
        aw = np.empty(cap, np.int32); amu = np.empty(cap, np.uint64)
        na = np.zeros(1, np.int64); ovf = np.zeros(1, np.uint32)
        rc = lib.orc_skeleton(g.n, g.m, _ptr(eu), _ptr(ev), _ptr(ew), int(g.directed), _ptr(Sa),
                              int(Sa.shape[0]), _ptr(pa), int(k), _ptr(nodes), _ptr(nsk), cap, _ptr(au),
                              _ptr(av), _ptr(aw), _ptr(amu), _ptr(na), _ptr(ovf))
        if rc == 1 and na[0] > cap:
            cap = int(na[0])
            continue
        _check(rc, "skeleton")
        n_a = int(na[0])
        return nodes[: int(nsk[0])].copy(), (au[:n_a], av[:n_a], aw[:n_a], amu[:n_a]), bool(ovf[0])


def distance_sum(g, sources) -> int:
    """Sum over the given sources s and reachable t != s of (d(s,t) - 1), unit weights
    (breadth-first search; the right-hand side of the path-length invariant)."""
    lib = _load()
    eu, ev, _ = _edges(g)
    src = np.ascontiguousarray(sources, np.int32)
    out = np.zeros(1, np.int64)
    _check(lib.orc_distance_sum(g.n, g.m, _ptr(eu), _ptr(ev), int(g.directed), _ptr(src), int(src.shape[0]),
                                _ptr(out)), "distance_sum")
    return int(out[0])


def brandes_st(g, src, dst, halve: bool | None = None):
    """Plain Brandes for source set `src` and destination set `dst`: sum over s in src, t in dst,
    s != t, of sigma(s,t|v)/sigma(s,t).  Returns (bc, overflow)."""
    lib = _load()
    eu, ev, ew = _edges(g)
    a = np.ascontiguousarray(src, np.int32)
    b = np.ascontiguousarray(dst, np.int32)
    if halve is None:
        halve = not g.directed
    bc = np.empty(g.n, np.float64)
    ovf = np.zeros(1, np.uint32)
    _check(lib.orc_brandes_st(g.n, g.m, _ptr(eu), _ptr(ev), _ptr(ew), int(g.directed), _ptr(a), int(a.shape[0]),
                              _ptr(b), int(b.shape[0]), int(bool(halve)), _ptr(bc), _ptr(ovf)), "brandes_st")
    return bc, bool(ovf[0])


def label_propagation(g, max_rounds: int = 20):
    """Deterministic label-propagation partition (a heuristic defined in bc_oracle.c, not by the
    paper).  Returns (part int32[n], k, rounds)."""
    lib = _load()
    eu, ev, _ = _edges(g)
    part = np.empty(max(g.n, 1), np.int32)
    k = np.zeros(1, np.int32)
    r = np.zeros(1, np.int32)
    _check(lib.orc_label_propagation(g.n, g.m, _ptr(eu), _ptr(ev), int(g.directed), int(max_rounds), _ptr(part),
                                     _ptr(k), _ptr(r)), "label_propagation")
    return part[: g.n], int(k[0]), int(r[0])
