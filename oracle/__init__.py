"""CPU oracle for MFBC -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  The CUDA library (paper_1609_07008_gb300) never
imports it, and the two share no code: the only thing both see is the input
produced by the separate ``graphgen`` package.

  * ``bc`` / ``sssp`` / ``delta``: plain C Brandes (brandes.c), BFS for unit
    weights and binary-heap Dijkstra for integer weights, FP64, with an exact
    128-bit shadow of every path count (Sec. 2.4; Theorem 1 makes its lambda
    the result MFBC must reproduce).
  * ``brute``: explicit enumeration of all shortest paths with exact
    fractions for graphs of a dozen vertices (definitions of Sec. 2.4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "brandes.c")
_lock = threading.Lock()
_lib = None

INF = np.iinfo(np.int32).max


def build(force: bool = False) -> str:
    """Compile brandes.c with gcc (no fast-math: IEEE FP64 throughout)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.oracle_bc.argtypes = [ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int32, ctypes.c_int, vp, vp]
            lib.oracle_sssp.argtypes = [ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int32, ctypes.c_int,
                                        vp, vp, vp]
            lib.oracle_delta.argtypes = [ctypes.c_int32, vp, vp, vp, ctypes.c_int32, vp]
            for f in (lib.oracle_bc, lib.oracle_sssp, lib.oracle_delta):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _graph_arrays(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.int32)
    return rp, col, w


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def bc(g, sources, nthreads: int | None = None, return_inexact: bool = False):
    """lambda(v) = sum over sources s of delta(s, v), v != s (ordered pairs)."""
    lib = _load()
    rp, col, w = _graph_arrays(g)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    lam = np.zeros(g.n, dtype=np.float64)
    inex = np.zeros(max(len(src), 1), dtype=np.uint8)
    rc = lib.oracle_bc(g.n, _ptr(rp), _ptr(col), _ptr(w), _ptr(src), len(src),
                       nthreads or default_threads(), _ptr(lam), _ptr(inex))
    if rc != 0:
        raise MemoryError("oracle_bc failed")
    return (lam, inex[:len(src)].astype(bool)) if return_inexact else lam


def sssp(g, sources, nthreads: int | None = None):
    """(dist [nsrc, n] int32 with INF = INT32_MAX, sigma_bar [nsrc, n] f64, inexact [nsrc] bool)."""
    lib = _load()
    rp, col, w = _graph_arrays(g)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    dist = np.empty((len(src), g.n), dtype=np.int32)
    sig = np.empty((len(src), g.n), dtype=np.float64)
    inex = np.zeros(max(len(src), 1), dtype=np.uint8)
    rc = lib.oracle_sssp(g.n, _ptr(rp), _ptr(col), _ptr(w), _ptr(src), len(src),
                         nthreads or default_threads(), _ptr(dist), _ptr(sig), _ptr(inex))
    if rc != 0:
        raise MemoryError("oracle_sssp failed")
    return dist, sig, inex[:len(src)].astype(bool)


def delta(g, s: int):
    """delta(s, .) for one source."""
    lib = _load()
    rp, col, w = _graph_arrays(g)
    out = np.zeros(g.n, dtype=np.float64)
    rc = lib.oracle_delta(g.n, _ptr(rp), _ptr(col), _ptr(w), int(s), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_delta failed")
    return out
