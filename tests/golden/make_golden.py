"""Writes bruteforce_small.json: exact betweenness of a few tiny seeded graphs.

The expected values come only from oracle/bruteforce.py (explicit enumeration of shortest
paths with exact fractions, Eq. 1 / Eq. 5 of the paper); the inputs come from the seeded
generators.  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bruteforce as bf  # noqa: E402
from paper_1406_4173_gb300 import gen  # noqa: E402


def main():
    cases = []
    specs = [
        ("er9-undirected", dict(n=9, p=0.35, seed=101, directed=False, wmax=None), None),
        ("er8-undirected-weighted", dict(n=8, p=0.45, seed=102, directed=False, wmax=3), None),
        ("er8-directed", dict(n=8, p=0.3, seed=103, directed=True, wmax=None), None),
        ("er9-directed-weighted-S", dict(n=9, p=0.35, seed=104, directed=True, wmax=4), [0, 2, 3, 5, 8]),
        ("er10-undirected-S", dict(n=10, p=0.3, seed=105, directed=False, wmax=None), [1, 4, 6, 9]),
    ]
    for name, kw, S in specs:
        g = gen.erdos_renyi(kw["n"], kw["p"], seed=kw["seed"], directed=kw["directed"], wmax=kw["wmax"], stream=21)
        bc = bf.betweenness(g, S)
        cases.append(dict(name=name, n=g.n, directed=g.directed, src=g.src.tolist(), dst=g.dst.tolist(),
                          w=None if g.w is None else g.w.tolist(), S=S,
                          bc=[[x.numerator, x.denominator] for x in bc]))
    out = dict(source="oracle/bruteforce.py: exact shortest-path enumeration (Eq. 1, Eq. 5)", cases=cases)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "bruteforce_small.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
