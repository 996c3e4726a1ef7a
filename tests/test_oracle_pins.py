"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check is independent of the oracle's own code path:
  * closed forms for unweighted graphs (Sec. 2.4 definitions, ordered pairs);
  * exact brute-force enumeration of all shortest paths on tiny graphs;
  * invariants: the unweighted path-length identity, linearity in the source
    list, relabelling invariance, non-negativity;
  * Bellman / Brandes certificates on the oracle's tau, sigma_bar (Lemma 1
    states these are what MFBF returns) and delta;
  * an optional cross-check against networkx (a library implementation).
"""
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.brute import brute

INF = oracle.INF


def _all(n):
    return np.arange(n, dtype=np.int32)


def _rel_close(a, b, tol=1e-12):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.all(np.abs(a - b) <= tol * np.maximum(np.abs(b), 1e-300)) and np.all((b == 0) == (a == 0))


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [2, 3, 5, 8, 13])
def test_path_closed_form(n):
    g = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)], directed=False)
    lam = oracle.bc(g, _all(n))
    assert np.array_equal(lam, [2.0 * i * (n - 1 - i) for i in range(n)])


@pytest.mark.parametrize("n", [3, 6, 11])
def test_directed_path_closed_form(n):
    g = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)], directed=True)
    lam = oracle.bc(g, _all(n))
    assert np.array_equal(lam, [1.0 * i * (n - 1 - i) for i in range(n)])


@pytest.mark.parametrize("n", [3, 4, 9])
def test_star_closed_form(n):
    g = gg.from_edges(n, [(0, i) for i in range(1, n)], directed=False)
    lam = oracle.bc(g, _all(n))
    assert lam[0] == (n - 1) * (n - 2)
    assert np.all(lam[1:] == 0.0)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 10, 11])
def test_cycle_closed_form(n):
    g = gg.from_edges(n, [(i, (i + 1) % n) for i in range(n)], directed=False)
    lam = oracle.bc(g, _all(n))
    k = n // 2
    want = k * (k - 1) if n % 2 else (k - 1) ** 2
    assert np.allclose(lam, want, rtol=1e-14, atol=0)


@pytest.mark.parametrize("n", [2, 4, 7])
def test_complete_graph_zero(n):
    g = gg.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], directed=False)
    assert np.all(oracle.bc(g, _all(n)) == 0.0)


@pytest.mark.parametrize("a,b", [(1, 4), (2, 3), (3, 5), (4, 4)])
def test_complete_bipartite_closed_form(a, b):
    g = gg.from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)], directed=False)
    lam = oracle.bc(g, _all(a + b))
    assert np.allclose(lam[:a], b * (b - 1) / a, rtol=1e-14, atol=0)
    assert np.allclose(lam[a:], a * (a - 1) / b, rtol=1e-14, atol=0)


def _grid_unweighted(L):
    edges = []
    for r in range(L):
        for c in range(L):
            v = r * L + c
            if c + 1 < L:
                edges.append((v, v + 1))
            if r + 1 < L:
                edges.append((v, v + L))
    return gg.from_edges(L * L, edges, directed=False)


@pytest.mark.parametrize("L", [3, 6, 12])
def test_grid_distances_and_path_counts(L):
    g = _grid_unweighted(L)
    srcs = np.array([0, L - 1, (L // 2) * L + L // 2], dtype=np.int32)
    dist, sig, inex = oracle.sssp(g, srcs)
    for i, s in enumerate(srcs):
        sr, sc = divmod(int(s), L)
        for v in range(L * L):
            r, c = divmod(v, L)
            dx, dy = abs(r - sr), abs(c - sc)
            assert dist[i, v] == dx + dy
            assert sig[i, v] == comb(dx + dy, dx)
    assert not inex.any()


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_hypercube_counts(k):
    n = 1 << k
    edges = [(v, v ^ (1 << b)) for v in range(n) for b in range(k) if v < v ^ (1 << b)]
    g = gg.from_edges(n, edges, directed=False)
    dist, sig, _ = oracle.sssp(g, _all(n))
    for s in range(n):
        for v in range(n):
            h = bin(s ^ v).count("1")
            assert dist[s, v] == h and sig[s, v] == factorial(h)


def test_weighted_tree_independent_of_weights():
    rng = np.random.default_rng(5)
    n = 40
    parent = [int(rng.integers(0, i)) for i in range(1, n)]
    edges = [(p, i + 1) for i, p in enumerate(parent)]
    g1 = gg.from_edges(n, edges, directed=False)
    g2 = gg.from_edges(n, edges, directed=False, weights=rng.integers(1, 50, len(edges)))
    assert np.allclose(oracle.bc(g1, _all(n)), oracle.bc(g2, _all(n)), rtol=1e-13, atol=0)


def test_two_components_and_isolated():
    # path 0-1-2 ; edge 3-4 ; isolated 5
    g = gg.from_edges(6, [(0, 1), (1, 2), (3, 4)], directed=False)
    lam = oracle.bc(g, _all(6))
    assert np.array_equal(lam, [0, 2, 0, 0, 0, 0])
    dist, sig, _ = oracle.sssp(g, np.array([0, 5], dtype=np.int32))
    assert dist[0, 3] == INF and sig[0, 3] == 0 and dist[1, 5] == 0 and sig[1, 5] == 1


# --------------------------------------------------------------- brute force
def _random_tiny(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 11))
    directed = bool(rng.integers(0, 2))
    weighted = bool(rng.integers(0, 2))
    p = float(rng.uniform(0.1, 0.7))
    edges, ws = [], []
    for u in range(n):
        for v in range(n):
            if u == v or (not directed and v < u):
                continue
            if rng.random() < p:
                edges.append((u, v))
                ws.append(int(rng.integers(1, 4)))
    g = gg.from_edges(n, edges, directed=directed, weights=ws if weighted else None)
    k = int(rng.integers(0, 2 * n + 1))
    srcs = rng.integers(0, n, size=k).astype(np.int32) if n else np.zeros(0, np.int32)
    return g, srcs


@pytest.mark.parametrize("seed", range(300))
def test_oracle_matches_brute_force(seed):
    g, srcs = _random_tiny(seed)
    tau, sb, lam_exact = brute(g, srcs)
    lam = oracle.bc(g, srcs)
    for v in range(g.n):
        want = lam_exact[v]
        if want == 0:
            assert lam[v] == 0.0
        else:
            assert abs(Fraction(lam[v]) - want) <= Fraction(1, 10**12) * want
    if len(srcs):
        dist, sig, _ = oracle.sssp(g, srcs)
        for i, s in enumerate(srcs):
            for t in range(g.n):
                want_d = tau[s][t]
                assert dist[i, t] == (INF if want_d is None else want_d)
                assert sig[i, t] == sb[s][t]


# ---------------------------------------------------------------- invariants
def test_unweighted_path_length_identity():
    # sum_v lambda(v) = sum_{s in S} sum_{t != s reachable} (tau(s,t) - 1)
    for g in (gg.erdos_renyi(300, 4, seed=11), gg.rmat(10, 8, seed=3),
              gg.rmat(9, 8, directed=True, seed=4)):
        srcs = gg.sample_sources(g, 64, seed=5)
        lam = oracle.bc(g, srcs)
        dist, _, _ = oracle.sssp(g, srcs)
        reach = (dist != INF) & (dist > 0)
        rhs = float(np.sum(dist[reach].astype(np.int64) - 1))
        assert abs(lam.sum() - rhs) <= 1e-9 * rhs


def test_linearity_in_sources():
    g = gg.rmat(10, 8, directed=True, weights=(1, 9), seed=7)
    s1 = gg.sample_sources(g, 40, seed=1)
    s2 = gg.sample_sources(g, 25, seed=2)
    both = oracle.bc(g, np.concatenate([s1, s2]))
    sep = oracle.bc(g, s1) + oracle.bc(g, s2)
    assert np.allclose(both, sep, rtol=1e-12, atol=0)
    assert np.all(both >= 0)


def test_relabel_invariance():
    g = gg.erdos_renyi(200, 5, weights=(1, 5), seed=9)
    rng = np.random.default_rng(0)
    perm = rng.permutation(g.n)                    # old id -> new id
    edges = []
    ws = []
    for v in range(g.n):
        for k in range(g.rowptr[v], g.rowptr[v + 1]):
            u = int(g.col[k])
            if v < u:
                edges.append((int(perm[v]), int(perm[u])))
                ws.append(int(g.w[k]))
    h = gg.from_edges(g.n, edges, directed=False, weights=ws)
    srcs = np.arange(g.n, dtype=np.int32)
    lam_g = oracle.bc(g, srcs)
    lam_h = oracle.bc(h, perm[srcs].astype(np.int32))
    assert np.allclose(lam_h[perm], lam_g, rtol=1e-11, atol=1e-12)


def test_bellman_and_brandes_certificates():
    """tau, sigma_bar satisfy the Bellman recurrences (Lemma 1) and delta the
    Brandes recurrence (Sec. 2.4), checked arc by arc."""
    for g in (gg.rmat(9, 8, directed=True, weights=(1, 20), seed=13), gg.erdos_renyi(150, 6, seed=2)):
        srcs = gg.sample_sources(g, 8, seed=3)
        dist, sig, _ = oracle.sssp(g, srcs)
        w = g.w if g.w is not None else np.ones(g.nnz, dtype=np.int32)
        src_of = np.repeat(np.arange(g.n), np.diff(g.rowptr))
        for i, s in enumerate(srcs):
            d = dist[i].astype(np.int64)
            ds, dt = d[src_of], d[g.col]
            fin = ds != INF
            assert np.all(dt[fin] <= ds[fin] + w[fin])
            tight = fin & (dt == ds + w)
            acc = np.zeros(g.n)
            np.add.at(acc, g.col[tight], sig[i][src_of[tight]])
            acc[s] = 1.0
            reach = d != INF
            assert np.array_equal(acc[reach], sig[i][reach])
            assert np.all(sig[i][~reach] == 0)
            de = oracle.delta(g, int(s))
            rhs = np.zeros(g.n)
            np.add.at(rhs, src_of[tight], sig[i][src_of[tight]] / sig[i][g.col[tight]] * (1 + de[g.col[tight]]))
            assert np.allclose(de, rhs, rtol=1e-12, atol=1e-12)


def test_sigma_inexact_flag_on_large_grid():
    # corner-to-corner path counts of an L x L grid are C(2L-2, L-1)
    g = _grid_unweighted(25)          # C(48,24) ~ 3.2e13 < 2^53
    _, sig, inex = oracle.sssp(g, np.array([0], dtype=np.int32))
    assert sig[0, -1] == comb(48, 24) and not inex[0]
    g = _grid_unweighted(30)          # C(58,29) ~ 3.0e16 > 2^53
    _, _, inex = oracle.sssp(g, np.array([0], dtype=np.int32))
    assert inex[0]


def test_networkx_cross_check():
    nx = pytest.importorskip("networkx")
    cases = [gg.erdos_renyi(120, 5, seed=21), gg.erdos_renyi(100, 6, weights=(1, 4), seed=22),
             gg.rmat(7, 6, directed=True, weights=(1, 3), seed=23), gg.rmat(7, 6, directed=True, seed=24)]
    for g in cases:
        G = nx.DiGraph() if g.directed else nx.Graph()
        G.add_nodes_from(range(g.n))
        for v in range(g.n):
            for k in range(g.rowptr[v], g.rowptr[v + 1]):
                G.add_edge(v, int(g.col[k]), weight=1 if g.w is None else int(g.w[k]))
        ref = nx.betweenness_centrality(G, normalized=False, weight="weight")
        ref = np.array([ref[v] for v in range(g.n)]) * (1 if g.directed else 2)
        lam = oracle.bc(g, np.arange(g.n, dtype=np.int32))
        assert np.allclose(lam, ref, rtol=1e-9, atol=1e-9)


# ------------------------------------------------------------ golden fixtures
def test_oracle_matches_golden_fixtures():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_graphs.json")
    for case in json.load(open(path)):
        g = gg.CSRGraph(n=case["n"], rowptr=np.array(case["rowptr"], np.int64),
                        col=np.array(case["col"], np.int32),
                        w=None if case["w"] is None else np.array(case["w"], np.int32),
                        directed=case["directed"])
        srcs = np.array(case["sources"], np.int32)
        lam = oracle.bc(g, srcs)
        for v, q in enumerate(case["lambda"]):
            want = Fraction(q)
            assert abs(Fraction(lam[v]) - want) <= Fraction(1, 10**12) * want
        dist, sig, _ = oracle.sssp(g, srcs)
        tau = np.array(case["tau"], np.int64)
        assert np.array_equal(np.where(dist == INF, -1, dist), tau)
        assert np.array_equal(sig, np.array(case["sigma_bar"], np.float64))
