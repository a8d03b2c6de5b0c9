"""Brute-force betweenness for tiny graphs (n <= 12), in exact rational arithmetic.

TEST INFRASTRUCTURE ONLY (pins the C oracle; never used by the product library).

It follows the definitions of Sec. 3 directly and shares nothing with the Brandes recursion:
distances come from Floyd-Warshall, every shortest s-t path is enumerated explicitly by a
depth-first walk that only follows arcs staying on a shortest path, and the dependency of
the pair (s, t) on v is (#shortest s-t paths through v) / (#shortest s-t paths), summed over
ordered pairs s != t of the target set (Eq. 1 and Eq. 5); endpoints are not credited.
"""
from __future__ import annotations

from fractions import Fraction

INF = float("inf")


def _arcs(g):
    out = [[] for _ in range(g.n)]
    for i in range(g.m):
        u, v = int(g.src[i]), int(g.dst[i])
        w = 1 if g.w is None else int(g.w[i])
        out[u].append((v, w))
        if not g.directed:
            out[v].append((u, w))
    return out


def floyd_warshall(g):
    n = g.n
    d = [[INF] * n for _ in range(n)]
    for v in range(n):
        d[v][v] = 0
    for u, lst in enumerate(_arcs(g)):
        for v, w in lst:
            d[u][v] = min(d[u][v], w)
    for k in range(n):
        dk = d[k]
        for i in range(n):
            dik = d[i][k]
            if dik == INF:
                continue
            di = d[i]
            for j in range(n):
                if dik + dk[j] < di[j]:
                    di[j] = dik + dk[j]
    return d


def shortest_paths(g, d=None):
    """All shortest paths: dict (s, t) -> list of node tuples (s != t, t reachable)."""
    if d is None:
        d = floyd_warshall(g)
    out = _arcs(g)
    res = {}
    for s in range(g.n):
        for t in range(g.n):
            if s == t or d[s][t] == INF:
                continue
            paths = []
            stack = [(s, 0, (s,))]
            while stack:
                u, L, p = stack.pop()
                if u == t:
                    paths.append(p)
                    continue
                for v, w in out[u]:
                    if v not in p and L + w + d[v][t] == d[s][t]:
                        stack.append((v, L + w, p + (v,)))
            res[(s, t)] = paths
    return res


def sigma_table(g):
    """(dist, sigma) as n x n lists: sigma[s][t] = number of shortest s-t paths."""
    d = floyd_warshall(g)
    sp = shortest_paths(g, d)
    n = g.n
    sig = [[0] * n for _ in range(n)]
    for s in range(n):
        sig[s][s] = 1
    for (s, t), paths in sp.items():
        sig[s][t] = len(paths)
    return d, sig


def betweenness(g, S=None, halve=None):
    """Exact C^S(v) as Fractions (Eq. 5), halved for undirected graphs by default."""
    if halve is None:
        halve = not g.directed
    n = g.n
    targets = list(range(n)) if S is None else [int(x) for x in S]
    tset = set(targets)
    sp = shortest_paths(g)
    bc = [Fraction(0)] * n
    for (s, t), paths in sp.items():
        if s not in tset or t not in tset:
            continue
        total = len(paths)
        through = [0] * n
        for p in paths:
            for v in p[1:-1]:
                through[v] += 1
        for v in range(n):
            if through[v]:
                bc[v] += Fraction(through[v], total)
    if halve:
        bc = [x / 2 for x in bc]
    return bc


def betweenness_st(g, src, dst, halve=None):
    """Exact sum over s in src, t in dst, s != t, of (#shortest s-t paths through v) / (#shortest
    s-t paths), as Fractions; halved for undirected graphs by default."""
    if halve is None:
        halve = not g.directed
    sset, tset = set(int(x) for x in src), set(int(x) for x in dst)
    sp = shortest_paths(g)
    bc = [Fraction(0)] * g.n
    for (s, t), paths in sp.items():
        if s not in sset or t not in tset:
            continue
        through = [0] * g.n
        for p in paths:
            for v in p[1:-1]:
                through[v] += 1
        for v in range(g.n):
            if through[v]:
                bc[v] += Fraction(through[v], len(paths))
    if halve:
        bc = [x / 2 for x in bc]
    return bc
