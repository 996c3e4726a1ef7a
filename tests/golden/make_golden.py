"""Writes tests/golden/tiny_graphs.json from the brute-force enumerator only.

Run:  python tests/golden/make_golden.py
Every value comes from oracle.brute (explicit enumeration of all shortest
paths with exact fractions, following the definitions of Sec. 2.4 and
Table 1); the file stores lambda as exact rationals "p/q".
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
from oracle.brute import brute  # noqa: E402

CASES = [
    # name, n, edges, directed, weights, sources, citation
    ("path5", 5, [(0, 1), (1, 2), (2, 3), (3, 4)], False, None, list(range(5)),
     "Sec. 2.4 lambda over ordered pairs; path P_n gives 2 i (n-1-i)"),
    ("star6", 6, [(0, i) for i in range(1, 6)], False, None, list(range(6)),
     "Sec. 2.4: sigma(s,t,s) = 0, so leaves score 0 and the centre (n-1)(n-2)"),
    ("cycle6", 6, [(i, (i + 1) % 6) for i in range(6)], False, None, list(range(6)),
     "Sec. 2.4; even cycle C_2k gives (k-1)^2 per vertex"),
    ("k23", 5, [(i, 2 + j) for i in range(2) for j in range(3)], False, None, list(range(5)),
     "Sec. 2.4; complete bipartite K_{a,b}: b(b-1)/a and a(a-1)/b"),
    ("weighted_ties", 7, [(0, 1), (0, 2), (1, 3), (2, 3), (3, 4), (1, 4), (4, 5), (2, 6), (6, 5)], True,
     [1, 2, 2, 1, 1, 3, 2, 1, 3], [0, 1, 2, 0, 6],
     "Sec. 4.1 multpath monoid: equal-weight paths of different edge counts are summed (Lemma 1)"),
    ("two_components", 7, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5)], False, [2, 1, 1, 4, 4],
     [0, 3, 6, 5, 5], "Sec. 2.4: unreachable targets contribute 0; duplicate sources count twice"),
    ("directed_unreachable", 6, [(0, 1), (1, 2), (2, 3), (4, 3), (3, 5), (0, 4)], True, None,
     [0, 2, 5, 4], "Sec. 2.4 over directed arcs; vertices unreachable from s carry sigma_bar = 0"),
]


def main():
    out = []
    for name, n, edges, directed, weights, sources, cite in CASES:
        g = gg.from_edges(n, edges, directed=directed, weights=weights)
        tau, sb, lam = brute(g, sources)
        out.append({
            "name": name, "citation": cite, "n": n, "directed": directed,
            "rowptr": g.rowptr.tolist(), "col": g.col.tolist(),
            "w": None if g.w is None else g.w.tolist(),
            "sources": sources,
            "tau": [[-1 if x is None else x for x in tau[s]] for s in sources],
            "sigma_bar": [sb[s] for s in sources],
            "lambda": [f"{x.numerator}/{x.denominator}" for x in lam],
        })
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_graphs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
