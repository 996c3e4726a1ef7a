"""Brute-force betweenness by explicit path enumeration -- TEST INFRASTRUCTURE ONLY.

Independent of Brandes' recurrence: it follows the definitions of the paper's
Sec. 2.4 and Table 1 literally, on graphs of a dozen vertices or fewer.

  tau(s,t)        by Floyd-Warshall over the integer weights;
  sigma_bar(s,t)  by enumerating every simple s -> t path whose weight is
                  tau(s,t) (a prefix of a shortest path is itself shortest,
                  so a branch is cut as soon as its weight exceeds tau(s,x));
  sigma(s,t,v)    the enumerated shortest s -> t paths that pass through an
                  interior vertex v (so sigma(s,s,v) = sigma(s,t,s) =
                  sigma(s,t,t) = 0);
  lambda(v)       sum over listed sources s and all t of sigma(s,t,v)/sigma_bar(s,t),
                  as an exact Fraction (ordered pairs; unreachable t add 0).
"""
from __future__ import annotations

from fractions import Fraction

INF = None


def _arcs(g):
    arcs = {}
    for v in range(g.n):
        for k in range(int(g.rowptr[v]), int(g.rowptr[v + 1])):
            u = int(g.col[k])
            arcs[(v, u)] = 1 if g.w is None else int(g.w[k])
    return arcs


def floyd_warshall(n, arcs):
    d = [[INF] * n for _ in range(n)]
    for v in range(n):
        d[v][v] = 0
    for (u, v), w in arcs.items():
        if d[u][v] is None or w < d[u][v]:
            d[u][v] = w
    for k in range(n):
        dk = d[k]
        for i in range(n):
            dik = d[i][k]
            if dik is None:
                continue
            di = d[i]
            for j in range(n):
                if dk[j] is not None and (di[j] is None or dik + dk[j] < di[j]):
                    di[j] = dik + dk[j]
    return d


def shortest_paths(n, arcs, tau, s):
    """Every shortest path from s, as vertex tuples, grouped by endpoint."""
    adj = [[] for _ in range(n)]
    for (u, v), w in arcs.items():
        adj[u].append((v, w))
    out = {t: [] for t in range(n)}
    path = [s]
    on = [False] * n
    on[s] = True

    def dfs(x, wsum):
        if wsum == tau[s][x]:
            out[x].append(tuple(path))
        for (y, w) in adj[x]:
            if on[y]:
                continue
            ty = tau[s][y]
            if ty is None or wsum + w > ty:
                continue
            on[y] = True
            path.append(y)
            dfs(y, wsum + w)
            path.pop()
            on[y] = False

    dfs(s, 0)
    return out


def brute(g, sources):
    """Return (tau, sigma_bar, lam) with lam a list of Fractions."""
    n = g.n
    arcs = _arcs(g)
    tau = floyd_warshall(n, arcs)
    sigma_bar = [[0] * n for _ in range(n)]
    lam = [Fraction(0)] * n
    cache = {}
    for s in sources:
        s = int(s)
        if s not in cache:
            paths = shortest_paths(n, arcs, tau, s)
            contrib = [Fraction(0)] * n
            for t in range(n):
                P = paths[t]
                sigma_bar[s][t] = len(P)
                if t == s or not P:
                    continue
                through = [0] * n
                for p in P:
                    for v in p[1:-1]:
                        through[v] += 1
                for v in range(n):
                    if through[v]:
                        contrib[v] += Fraction(through[v], len(P))
            cache[s] = contrib
        for v in range(n):
            lam[v] += cache[s][v]
    return tau, sigma_bar, lam
