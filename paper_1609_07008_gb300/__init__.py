"""MFBC on one GB300: Python binding of the C ABI in include/mfbc.h.

Maximal Frontier Betweenness Centrality (Solomonik, Besta, Vella, Hoefler,
SC17, arXiv:1609.07008): MFBF (Algorithm 1) computes distances and
shortest-path multiplicities for a batch of sources, MFBr (Algorithm 2) the
partial centrality factors, and Algorithm 3 accumulates betweenness over
batches.  Every step runs in the CUDA kernels of libmfbc.so; this module only
marshals arguments (numpy arrays for host buffers, torch CUDA tensors for
device buffers, torch streams).  There is no CPU fallback: if libmfbc.so is
missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MFBC_LIBRARY may point at another build of the same ABI (e.g. a tuning variant)
LIB_PATH = os.environ.get("MFBC_LIBRARY") or os.path.join(_HERE, "_build", "libmfbc.so")

MFBC_OK = 0
MFBC_ERR_INVALID = 1
MFBC_ERR_OOM = 2
MFBC_ERR_CUDA = 3
MFBC_ERR_OVERFLOW = 4
MFBC_ERR_NO_CONVERGENCE = 5
MFBC_ERR_TIMEOUT = 6
MFBC_CSR = 0
MFBC_CSC = 1
MFBC_DIRECTED = 0
MFBC_UNDIRECTED = 2
MFBC_WARN_SIGMA_INEXACT = 1
PATH_AUTO, PATH_GENERAL, PATH_LEVEL, PATH_DIST, PATH_SMALL = 0, 1, 2, 3, 4
MFBC_OPT_COUNT_BYTES = 1
MFBC_OPT_KEEP_ORDER = 2
MFBC_OPT_TEST_STALL = 4
MFBC_OPT_TEST_SMALL_ROUNDS = 16
MFBC_OPT_ACCUMULATE = 8
ACCUM_AUTO, ACCUM_ATOMIC, ACCUM_SEGMENTED, ACCUM_HASH = 0, 1, 2, 3
INF = np.iinfo(np.int32).max
MAX_KSTATS = 24


class MFBCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mfbc status {status}: {msg}")
        self.status = status


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_uint64),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("nkernels", ctypes.c_int32), ("k", KernelStat * MAX_KSTATS),
                ("batches", ctypes.c_uint64), ("fwd_iters", ctypes.c_uint64),
                ("bwd_iters", ctypes.c_uint64), ("n_b", ctypes.c_int32), ("path", ctypes.c_int32),
                ("stat", ctypes.c_uint64 * 4)]

    def as_dict(self) -> dict:
        return {
            "kernels": {self.k[i].name.decode(): {"launches": int(self.k[i].launches), "ms": self.k[i].ms,
                                                   "bytes": self.k[i].bytes}
                        for i in range(self.nkernels)},
            "batches": int(self.batches), "fwd_iters": int(self.fwd_iters),
            "bwd_iters": int(self.bwd_iters), "n_b": int(self.n_b), "path": int(self.path),
            "pairs_fwd": int(self.stat[0]), "pairs_bwd": int(self.stat[1]),
            "values_fwd": int(self.stat[2]), "values_bwd": int(self.stat[3]),
        }


class Options(ctypes.Structure):
    _fields_ = [("n_b", ctypes.c_int32), ("path", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_uint64),
                ("warn_out", ctypes.POINTER(ctypes.c_uint32)), ("profile", ctypes.POINTER(Profile)),
                ("flags", ctypes.c_uint32), ("lambda_rows", ctypes.c_void_p), ("accumulator", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    """mfbc_tuning (include/mfbc.h)."""
    _fields_ = [("n_b", ctypes.c_int32), ("path", ctypes.c_int32), ("arcs", ctypes.c_int32),
                ("tried", ctypes.c_int32), ("ms_per_source", ctypes.c_double), ("accumulator", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libmfbc.so (built by paper_1609_07008_gb300.build).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libmfbc.so not found at {p}: run `python -m paper_1609_07008_gb300.build`"
                               " (the CUDA library is required; there is no fallback)")
        lib = ctypes.CDLL(p)
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        st = ctypes.c_int
        sig = {
            "mfbc_graph_create": [i32, i64, vp, vp, vp, u32, vp, ctypes.POINTER(vp)],
            "mfbc_graph_create_device": [i32, i64, vp, vp, vp, u32, vp, ctypes.POINTER(vp)],
            "mfbc_graph_info": [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(u32),
                                ctypes.POINTER(i32)],
            "mfbc_bc": [vp, vp, i32, vp, ctypes.POINTER(Options)],
            "mfbc_bc_device": [vp, vp, i32, vp, ctypes.POINTER(Options)],
            "mfbc_bc_multi_device": [vp, vp, i32, vp, i32, vp, ctypes.POINTER(Options)],
            "mfbc_autotune": [vp, vp, i32, ctypes.POINTER(Options), ctypes.POINTER(Tuning)],
            "mfbc_sssp_batch": [vp, vp, i32, vp, vp, ctypes.POINTER(Options)],
            "mfbc_sssp_batch_device": [vp, vp, i32, vp, vp, ctypes.POINTER(Options)],
            "mfbc_workspace_size": [vp, i32, i32, ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_uint64)],
            "mfbc_graph_release_scratch": [vp],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = st
        lib.mfbc_graph_destroy.argtypes = [vp]
        lib.mfbc_graph_destroy.restype = None
        for name in ("mfbc_status_string",):
            getattr(lib, name).argtypes = [st]
            getattr(lib, name).restype = ctypes.c_char_p
        lib.mfbc_last_error.argtypes = []
        lib.mfbc_last_error.restype = ctypes.c_char_p
        lib.mfbc_version.argtypes = []
        lib.mfbc_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(status: int):
    if status != MFBC_OK:
        lib = load()
        detail = lib.mfbc_last_error().decode() or lib.mfbc_status_string(status).decode()
        raise MFBCError(status, detail)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _hptr(a) -> ctypes.c_void_p | None:
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _dptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream) -> ctypes.c_void_p | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _options(n_b, path, stream, workspace, warn, profile, count_bytes=False, keep_order=False,
             test_stall=False, accumulator=ACCUM_AUTO, test_small_rounds=False) -> Options:
    o = Options()
    o.accumulator = int(accumulator)
    o.flags = (MFBC_OPT_COUNT_BYTES if count_bytes else 0) | (MFBC_OPT_KEEP_ORDER if keep_order else 0) | \
        (MFBC_OPT_TEST_STALL if test_stall else 0) | (MFBC_OPT_TEST_SMALL_ROUNDS if test_small_rounds else 0)
    o.n_b = int(n_b)
    o.path = int(path)
    o.stream = _stream_handle(stream)
    if workspace is not None:
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    if warn is not None:
        o.warn_out = ctypes.pointer(warn)
    if profile is not None:
        o.profile = ctypes.pointer(profile)
    return o


class Graph:
    """A device-resident graph (CSR of the adjacency matrix A, Sec. 2.1).

    rowptr/col/w are numpy arrays (host) or torch CUDA tensors (device);
    w None means unit weights.  directed=False asserts A is symmetric.
    csc=True: the arrays are the rows of A^T (row v lists the tails of the
    arcs into v) instead of the rows of A."""

    def __init__(self, rowptr, col, w=None, *, directed: bool, stream=None, csc: bool = False):
        lib = load()
        self._h = ctypes.c_void_p()
        flags = (MFBC_DIRECTED if directed else MFBC_UNDIRECTED) | (MFBC_CSC if csc else MFBC_CSR)
        if _is_torch(rowptr):
            n = rowptr.numel() - 1
            nnz = col.numel()
            st = lib.mfbc_graph_create_device(n, nnz, _dptr(rowptr), _dptr(col), None if w is None else _dptr(w),
                                              flags, _stream_handle(stream), ctypes.byref(self._h))
        else:
            rp = _host(rowptr, np.int64)
            c = _host(col, np.int32)
            ww = None if w is None else _host(w, np.int32)
            n = len(rp) - 1
            st = lib.mfbc_graph_create(n, len(c), _hptr(rp), _hptr(c), _hptr(ww), flags,
                                       _stream_handle(stream), ctypes.byref(self._h))
        _check(st)
        self.n = n
        self.nnz = nnz if _is_torch(rowptr) else len(c)
        self.directed = directed
        u = ctypes.c_int32()
        _check(lib.mfbc_graph_info(self._h, None, None, None, ctypes.byref(u)))
        self.unit_weights = bool(u.value)

    @classmethod
    def from_csr(cls, g, stream=None) -> "Graph":
        """From any object with n, rowptr, col, w, directed attributes."""
        return cls(g.rowptr, g.col, g.w, directed=g.directed, stream=stream)

    def release_scratch(self):
        """Free the device scratch cached on this handle (mfbc_graph_release_scratch)."""
        _check(load().mfbc_graph_release_scratch(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().mfbc_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ----------------------------------------------------------- entry points
    def bc(self, sources, *, n_b: int = 0, path: int = PATH_AUTO, out=None, stream=None, workspace=None,
           profile: bool = False, count_bytes: bool = False, keep_order: bool = False,
           return_warn: bool = False, test_stall: bool = False, accumulator: int = ACCUM_AUTO,
           test_small_rounds: bool = False):
        """Betweenness centrality summed over `sources` (Algorithm 3).

        Host (numpy) sources -> numpy lambda via mfbc_bc; torch CUDA sources
        -> torch CUDA lambda via mfbc_bc_device (into `out` when given).
        test_stall and test_small_rounds set the MFBC_OPT_TEST_STALL and
        MFBC_OPT_TEST_SMALL_ROUNDS test hooks."""
        lib = load()
        warn = ctypes.c_uint32(0)
        prof = Profile() if (profile or count_bytes) else None
        opt = _options(n_b, path, stream, workspace, warn, prof, count_bytes, keep_order, test_stall, accumulator,
                       test_small_rounds)
        if _is_torch(sources):
            import torch
            src = sources.to(dtype=torch.int32).contiguous()
            lam = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=src.device)
            st = lib.mfbc_bc_device(self._h, _dptr(src), src.numel(), _dptr(lam), ctypes.byref(opt))
        else:
            src = _host(sources, np.int32)
            lam = out if out is not None else np.empty(self.n, dtype=np.float64)
            st = lib.mfbc_bc(self._h, _hptr(src), len(src), _hptr(lam), ctypes.byref(opt))
        _check(st)
        res = [lam]
        if return_warn:
            res.append(int(warn.value))
        if profile or count_bytes:
            res.append(prof.as_dict())
        return res[0] if len(res) == 1 else tuple(res)

    def bc_multi(self, source_lists, *, n_b: int = 0, path: int = PATH_AUTO, out=None, stream=None,
                 workspace=None, profile: bool = False, rows=None, accumulate: bool = False,
                 test_small_rounds: bool = False):
        """One lambda row per request: `source_lists` is a sequence of torch
        CUDA int tensors (or one concatenated tensor with a host `offsets`
        pair: (sources, offsets)).  Returns a [nreq, n] float64 CUDA tensor
        (mfbc_bc_multi_device), or `out` ([rows, n]) when given.  rows: the
        row of `out` for each request (default: request r -> row r);
        accumulate: add into those rows instead of overwriting them."""
        import torch
        lib = load()
        if isinstance(source_lists, tuple) and len(source_lists) == 2 and not _is_torch(source_lists[1]):
            src, offs = source_lists
            src = src.to(dtype=torch.int32).contiguous()
            off = np.ascontiguousarray(offs, dtype=np.int32)
        else:
            parts = [t.to(dtype=torch.int32).reshape(-1) for t in source_lists]
            if not parts:
                raise ValueError("no requests")
            src = torch.cat(parts).contiguous()
            off = np.zeros(len(parts) + 1, dtype=np.int32)
            off[1:] = np.cumsum([p.numel() for p in parts])
        nreq = len(off) - 1
        lam = out if out is not None else torch.empty((nreq, self.n), dtype=torch.float64, device=src.device)
        prof = Profile() if profile else None
        opt = _options(n_b, path, stream, workspace, None, prof, test_small_rounds=test_small_rounds)
        rws = None
        if rows is not None:
            rws = np.ascontiguousarray(rows, dtype=np.int32)
            if len(rws) != nreq or (len(rws) and (rws.min() < 0 or rws.max() >= lam.shape[0])):
                raise ValueError("rows must name one row of out per request")
            opt.lambda_rows = ctypes.c_void_p(rws.ctypes.data)
        if accumulate:
            opt.flags |= MFBC_OPT_ACCUMULATE
        _check(lib.mfbc_bc_multi_device(self._h, _dptr(src), src.numel(), _hptr(off), nreq, _dptr(lam),
                                        ctypes.byref(opt)))
        return (lam, prof.as_dict()) if profile else lam

    def autotune(self, sources, *, path: int = PATH_AUTO) -> dict:
        """Time the candidate batch widths (and, on the general kernels, arcs
        per step) on host `sources` and keep the fastest on this handle
        (mfbc_autotune)."""
        lib = load()
        src = _host(sources, np.int32)
        t = Tuning()
        opt = _options(0, path, None, None, None, None)
        _check(lib.mfbc_autotune(self._h, _hptr(src), len(src), ctypes.byref(opt), ctypes.byref(t)))
        return {"n_b": t.n_b, "path": t.path, "arcs": t.arcs, "tried": t.tried, "ms_per_source": t.ms_per_source,
                "accumulator": t.accumulator}

    def sssp(self, sources, *, n_b: int = 0, path: int = PATH_AUTO, with_sigma: bool = True, stream=None,
             workspace=None, profile: bool = False, return_warn: bool = False, accumulator: int = ACCUM_AUTO,
             test_small_rounds: bool = False):
        """MFBF alone (Algorithm 1): (dist [nsrc, n] int32, sigma [nsrc, n] f64 or None)."""
        lib = load()
        warn = ctypes.c_uint32(0)
        prof = Profile() if profile else None
        opt = _options(n_b, path, stream, workspace, warn, prof, accumulator=accumulator,
                       test_small_rounds=test_small_rounds)
        if _is_torch(sources):
            import torch
            src = sources.to(dtype=torch.int32).contiguous()
            dist = torch.empty((src.numel(), self.n), dtype=torch.int32, device=src.device)
            sig = torch.empty((src.numel(), self.n), dtype=torch.float64, device=src.device) if with_sigma else None
            st = lib.mfbc_sssp_batch_device(self._h, _dptr(src), src.numel(), _dptr(dist),
                                            None if sig is None else _dptr(sig), ctypes.byref(opt))
        else:
            src = _host(sources, np.int32)
            dist = np.empty((len(src), self.n), dtype=np.int32)
            sig = np.empty((len(src), self.n), dtype=np.float64) if with_sigma else None
            st = lib.mfbc_sssp_batch(self._h, _hptr(src), len(src), _hptr(dist), _hptr(sig), ctypes.byref(opt))
        _check(st)
        res = [dist, sig]
        if return_warn:
            res.append(int(warn.value))
        if profile:
            res.append(prof.as_dict())
        return tuple(res)

    def workspace_size(self, nsrc: int, mode: int = 0, *, n_b: int = 0, path: int = PATH_AUTO) -> int:
        lib = load()
        opt = _options(n_b, path, None, None, None, None)
        out = ctypes.c_uint64()
        _check(lib.mfbc_workspace_size(self._h, nsrc, mode, ctypes.byref(opt), ctypes.byref(out)))
        return int(out.value)


def bc(graph: Graph, sources, **kw):
    return graph.bc(sources, **kw)


def sssp_batch(graph: Graph, sources, **kw):
    return graph.sssp(sources, **kw)


def version() -> str:
    return load().mfbc_version().decode()
