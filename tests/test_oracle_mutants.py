"""The oracle's pins are sensitive: plausible single mistakes are caught.

Each mutant is a textual edit of a temporary copy of oracle/brandes.c (the
committed oracle is never modified), compiled with gcc on the CPU and run
through a subset of the pins: brute-force enumeration on tiny graphs and the
closed forms.  Every mutant must fail at least one of them.
"""
import ctypes
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.brute import brute

SRC = os.path.join(os.path.dirname(oracle.__file__), "brandes.c")

MUTANTS = {
    "drop_one_plus": ("(1.0 + S->delta[wv])", "(S->delta[wv])"),
    "transposed_ratio": ("S->sigma[v] / S->sigma[wv]", "S->sigma[wv] / S->sigma[v]"),
    "source_not_excluded": ("if (v != s) J->lambda[v]", "if (1) J->lambda[v]"),
    "no_reset_on_improve": ("S->dist[u] = (int32_t)nd; S->sigma[u] = S->sigma[v];",
                            "S->dist[u] = (int32_t)nd; S->sigma[u] += S->sigma[v];"),
    "ties_dropped": ("} else if (nd == S->dist[u]) {", "} else if (0) {"),
    "weight_ignored_backward": ("(int64_t)S->dist[v] + a)", "(int64_t)S->dist[v] + 1)"),
    "bfs_counts_all_arcs": ("if (S->dist[u] == S->dist[v] + 1) {", "if (S->dist[u] != 0) {"),
}


def _build_mutant(name, tmp):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, name
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as f:
        f.write(text.replace(old, new))
    so = os.path.join(tmp, f"{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", path, "-o", so])
    lib = ctypes.CDLL(so)
    vp = ctypes.c_void_p
    lib.oracle_bc.argtypes = [ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int32, ctypes.c_int, vp, vp]
    lib.oracle_sssp.argtypes = [ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int32, ctypes.c_int, vp, vp, vp]
    return lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _bc(lib, g, srcs):
    lam = np.zeros(g.n)
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.int32)
    s = np.ascontiguousarray(srcs, dtype=np.int32)
    lib.oracle_bc(g.n, _p(g.rowptr), _p(g.col), _p(w), _p(s), len(s), 1, _p(lam), None)
    return lam


def _sigma(lib, g, srcs):
    s = np.ascontiguousarray(srcs, dtype=np.int32)
    dist = np.empty((len(s), g.n), np.int32)
    sig = np.empty((len(s), g.n))
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.int32)
    lib.oracle_sssp(g.n, _p(g.rowptr), _p(g.col), _p(w), _p(s), len(s), 1, _p(dist), _p(sig), None)
    return dist, sig


def _pins_pass(lib):
    # closed forms
    n = 6
    g = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)], directed=False)
    if not np.array_equal(_bc(lib, g, np.arange(n)), [2.0 * i * (n - 1 - i) for i in range(n)]):
        return False
    g = gg.from_edges(5, [(0, i) for i in range(1, 5)], directed=False)
    lam = _bc(lib, g, np.arange(5))
    if lam[0] != 12 or np.any(lam[1:] != 0):
        return False
    g = gg.from_edges(6, [(i, (i + 1) % 6) for i in range(6)], directed=False)
    if not np.allclose(_bc(lib, g, np.arange(6)), 4.0):
        return False
    # brute force on tiny random graphs (weighted and unweighted)
    for seed in range(80):
        rng = np.random.default_rng(1000 + seed)
        nn = int(rng.integers(3, 9))
        directed = bool(seed % 2)
        edges, ws = [], []
        for u in range(nn):
            for v in range(nn):
                if u != v and (directed or u < v) and rng.random() < 0.45:
                    edges.append((u, v)); ws.append(int(rng.integers(1, 4)))
        g = gg.from_edges(nn, edges, directed=directed, weights=ws if seed % 4 < 2 else None)
        srcs = np.arange(nn, dtype=np.int32)
        tau, sb, lam_exact = brute(g, srcs)
        lam = _bc(lib, g, srcs)
        _, sig = _sigma(lib, g, srcs)
        for v in range(nn):
            if abs(Fraction(lam[v]) - lam_exact[v]) > Fraction(1, 10**9) * max(lam_exact[v], 1):
                return False
            for s in range(nn):
                if sig[s, v] != sb[s][v]:
                    return False
    return True


def test_committed_oracle_passes_the_mutant_pins():
    oracle.build()
    with tempfile.TemporaryDirectory() as tmp:
        old = MUTANTS["drop_one_plus"][0]
        MUTANTS["identity"] = (old, old)
        try:
            assert _pins_pass(_build_mutant("identity", tmp))
        finally:
            del MUTANTS["identity"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    with tempfile.TemporaryDirectory() as tmp:
        assert not _pins_pass(_build_mutant(name, tmp)), f"mutant {name} survived the pins"
