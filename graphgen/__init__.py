"""Seeded synthetic inputs for the MFBC workloads (inputs only).

This package generates graphs and source lists; it contains none of the
betweenness-centrality arithmetic.  Both the CPU oracle and the CUDA library
consume what it produces, and neither is imported here.

Workloads (the paper's experimental section, Sec. 6):
  * R-MAT power-law graphs (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), edge factor E,
    with a seeded random relabelling of the vertices;
  * Erdos-Renyi G(n, p) "uniform random" graphs with p = k / (n - 1);
  * weighted 4-neighbour 2D grids (serving pool).
Self-loops are dropped, duplicate arcs merged (minimum weight kept), rows
sorted; undirected graphs store both arcs with one weight per edge.

The C core (graphgen.c) is compiled on first use with gcc into
``graphgen/_build/libgraphgen.so``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_SRC = os.path.join(_HERE, "graphgen.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator core with gcc (portable flags only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            i64p, i32p = P(ctypes.c_int64), P(ctypes.c_int32)
            out = [P(i64p), P(i32p), P(i32p), P(ctypes.c_int64)]
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_uint64, ctypes.c_int] + out
            lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_uint64] + out
            lib.gg_grid.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_uint64] + out
            lib.gg_sample_sources.argtypes = [ctypes.c_int32, i64p, ctypes.c_int32,
                                              ctypes.c_uint64, i32p]
            lib.gg_free.argtypes = [ctypes.c_void_p]
            for f in (lib.gg_rmat, lib.gg_er, lib.gg_grid, lib.gg_sample_sources):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclasses.dataclass
class CSRGraph:
    """Adjacency A in CSR: row v lists the arcs v -> col[k] with weight w[k].

    ``w is None`` means unweighted (every arc has weight 1)."""
    n: int
    rowptr: np.ndarray          # int64 [n+1]
    col: np.ndarray             # int32 [nnz]
    w: np.ndarray | None        # int32 [nnz] or None
    directed: bool
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def m(self) -> int:
        """Edges as counted for TEPS: arcs if directed, undirected edges otherwise."""
        return self.nnz if self.directed else self.nnz // 2

    def out_degree(self) -> np.ndarray:
        return np.diff(self.rowptr)


def _collect(rc, rp, cp, wp, nnz, n, directed, name):
    lib = _load()
    if rc == -2:
        raise ValueError("graphgen: invalid generator parameters")
    if rc != 0:
        raise MemoryError("graphgen: allocation failed")
    m = nnz.value
    rowptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(cp, shape=(max(m, 1),))[:m].copy()
    w = np.ctypeslib.as_array(wp, shape=(max(m, 1),))[:m].copy() if wp else None
    for p in (rp, cp, wp):
        if p:
            lib.gg_free(ctypes.cast(p, ctypes.c_void_p))
    return CSRGraph(n=n, rowptr=rowptr, col=col, w=w, directed=directed, name=name)


def _outs():
    P = ctypes.POINTER
    return P(ctypes.c_int64)(), P(ctypes.c_int32)(), P(ctypes.c_int32)(), ctypes.c_int64(0)


def rmat(scale: int, edge_factor: int = 16, *, a=0.57, b=0.19, c=0.19, directed=False,
         weights: tuple[int, int] | None = None, seed: int = 1,
         nthreads: int | None = None) -> CSRGraph:
    """R-MAT with 2**scale vertices and edge_factor * 2**scale edge draws."""
    lib = _load()
    rp, cp, wp, nnz = _outs()
    wlo, whi = weights if weights else (0, 0)
    nth = nthreads or max(1, min(os.cpu_count() or 1, 32))
    rc = lib.gg_rmat(scale, edge_factor << scale, a, b, c, int(directed), wlo, whi, seed, nth,
                     ctypes.byref(rp), ctypes.byref(cp), ctypes.byref(wp), ctypes.byref(nnz))
    nm = f"rmat{scale}_e{edge_factor}_{'dir' if directed else 'und'}" + (f"_w{wlo}-{whi}" if weights else "")
    return _collect(rc, rp, cp, wp, nnz, 1 << scale, directed, nm)


def erdos_renyi(n: int, avg_degree: float, *, directed=False,
                weights: tuple[int, int] | None = None, seed: int = 1) -> CSRGraph:
    """G(n, p) with p = avg_degree / (n - 1)."""
    lib = _load()
    rp, cp, wp, nnz = _outs()
    wlo, whi = weights if weights else (0, 0)
    rc = lib.gg_er(n, float(avg_degree), int(directed), wlo, whi, seed,
                   ctypes.byref(rp), ctypes.byref(cp), ctypes.byref(wp), ctypes.byref(nnz))
    nm = f"er{n}_k{avg_degree:g}_{'dir' if directed else 'und'}" + (f"_w{wlo}-{whi}" if weights else "")
    return _collect(rc, rp, cp, wp, nnz, n, directed, nm)


def grid2d(L: int, *, weights: tuple[int, int] | None = (1, 16), seed: int = 1) -> CSRGraph:
    """L x L 4-neighbour grid, undirected; vertex (r, c) has id r * L + c."""
    lib = _load()
    rp, cp, wp, nnz = _outs()
    wlo, whi = weights if weights else (0, 0)
    rc = lib.gg_grid(L, wlo, whi, seed, ctypes.byref(rp), ctypes.byref(cp), ctypes.byref(wp),
                     ctypes.byref(nnz))
    nm = f"grid{L}" + (f"_w{wlo}-{whi}" if weights else "")
    return _collect(rc, rp, cp, wp, nnz, L * L, False, nm)


def sample_sources(g: CSRGraph, k: int, seed: int = 2) -> np.ndarray:
    """k distinct sources, uniform among vertices with out-degree >= 1."""
    lib = _load()
    out = np.empty(k, dtype=np.int32)
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    rc = lib.gg_sample_sources(g.n, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), k, seed,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc == -3:
        raise ValueError(f"graphgen: only fewer than {k} vertices have out-degree >= 1")
    if rc != 0:
        raise MemoryError("graphgen: allocation failed")
    return out


def from_edges(n: int, edges, *, directed: bool, weights=None, name: str = "") -> CSRGraph:
    """Small hand-written graphs: edges is a list of (u, v) pairs (both arcs are
    added when undirected), weights an optional parallel list of integers."""
    src, dst, ww = [], [], []
    for i, (u, v) in enumerate(edges):
        if u == v:
            raise ValueError("self-loop")
        wv = 1 if weights is None else int(weights[i])
        src.append(u); dst.append(v); ww.append(wv)
        if not directed:
            src.append(v); dst.append(u); ww.append(wv)
    best: dict[tuple[int, int], int] = {}
    for u, v, wv in zip(src, dst, ww):
        if (u, v) not in best or wv < best[(u, v)]:
            best[(u, v)] = wv
    keys = sorted(best)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    for u, _ in keys:
        rowptr[u + 1] += 1
    rowptr = np.cumsum(rowptr).astype(np.int64)
    col = np.array([v for _, v in keys], dtype=np.int32)
    w = None if weights is None else np.array([best[k] for k in keys], dtype=np.int32)
    return CSRGraph(n=n, rowptr=rowptr, col=col, w=w, directed=directed, name=name)


# The five workload shapes used by the tests and the benchmark.
def workload(name: str) -> tuple[CSRGraph, np.ndarray, int]:
    """Return (graph, sources, n_b) for a named workload."""
    if name == "er1024":          # unweighted undirected ER n=1024, k=8; all sources
        g = erdos_renyi(1024, 8, seed=1)
        return g, np.arange(g.n, dtype=np.int32), 128
    if name == "rmat16w":         # weighted directed R-MAT scale 16, w ~ U[1,255]
        g = rmat(16, 16, directed=True, weights=(1, 255), seed=1)
        return g, sample_sources(g, 4096, seed=2), 512
    if name == "rmat22":          # unweighted undirected R-MAT scale 22
        g = rmat(22, 16, seed=1)
        return g, sample_sources(g, 16384, seed=2), 0
    if name == "er20k32":         # unweighted undirected ER n=2^20, k=32
        g = erdos_renyi(1 << 20, 32, seed=1)
        return g, sample_sources(g, 16384, seed=2), 0
    if name == "er16k1024w":      # weighted undirected ER n=2^16, k=1024, w ~ U[1,100]
        g = erdos_renyi(1 << 16, 1024, weights=(1, 100), seed=1)
        return g, np.arange(g.n, dtype=np.int32), 0
    raise KeyError(name)
