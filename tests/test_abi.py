"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point.

No CUDA device is needed: these calls are rejected by host-side argument
checks before the library touches the GPU.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1609_07008_gb300 as mfbc
from paper_1609_07008_gb300 import build as mbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mfbc.h")


@pytest.fixture(scope="module")
def lib():
    mbuild.build()
    return mfbc.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mfbc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mfbc_graph_create", "mfbc_graph_destroy", "mfbc_bc", "mfbc_sssp_batch",
                     "mfbc_bc_device", "mfbc_sssp_batch_device", "mfbc_status_string", "mfbc_last_error"):
        assert required in names


def test_binding_constants_match_the_header():
    # every MFBC_* constant the binding names has the header's value
    text = open(HEADER).read()
    defs = {k: int(v.rstrip("uU"), 0) for k, v in re.findall(r"#define\s+(MFBC_\w+)\s+(0x[0-9a-fA-F]+u?|\d+u?)\b", text)}
    aliases = {"PATH_": "MFBC_PATH_", "ACCUM_": "MFBC_ACCUM_"}
    checked = 0
    for name in dir(mfbc):
        hname = name
        for short, full in aliases.items():
            if name.startswith(short):
                hname = full + name[len(short):]
        if hname in defs:
            assert getattr(mfbc, name) == defs[hname], f"{name} = {getattr(mfbc, name)}, header {defs[hname]}"
            checked += 1
    assert checked >= 15


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(mbuild.LIB)
    for name in declared_functions():
        assert hasattr(raw, name), f"{name} declared in mfbc.h but not exported"


def test_library_is_built_for_sm_103a():
    assert any("sm_103a" in a for a in mbuild.ARCH)
    assert os.path.getsize(mbuild.LIB) > 0


def test_status_strings_and_version(lib):
    assert lib.mfbc_status_string(0) == b"ok"
    assert lib.mfbc_status_string(1) == b"invalid argument"
    assert b"sm_103a" in lib.mfbc_version()


def _create(lib, n, rowptr, col, w=None, flags=0):
    h = ctypes.c_void_p()
    rp = None if rowptr is None else np.ascontiguousarray(rowptr, np.int64)
    c = None if col is None else np.ascontiguousarray(col, np.int32)
    nnz = 0 if c is None else len(c)
    st = lib.mfbc_graph_create(n, nnz, None if rp is None else ctypes.c_void_p(rp.ctypes.data),
                               None if c is None else ctypes.c_void_p(c.ctypes.data),
                               None if w is None else ctypes.c_void_p(w.ctypes.data), flags, None,
                               ctypes.byref(h))
    return st, h


def test_host_side_argument_checks(lib):
    st, h = _create(lib, -1, [0], [])
    assert st == mfbc.MFBC_ERR_INVALID and not h.value
    assert b"n must be" in lib.mfbc_last_error()
    st, h = _create(lib, 3, None, [])
    assert st == mfbc.MFBC_ERR_INVALID
    st, h = _create(lib, 2, [0, 1, 3], [1, 0])          # rowptr[n] != nnz
    assert st == mfbc.MFBC_ERR_INVALID and b"rowptr" in lib.mfbc_last_error()
    st, h = _create(lib, 2, [1, 1, 2], [1, 0])          # rowptr[0] != 0
    assert st == mfbc.MFBC_ERR_INVALID
    for bad_flags in (4, 8, 0x80000000):                   # unknown flag bits
        st, h = _create(lib, 2, [0, 1, 2], [1, 0], flags=bad_flags)
        assert st == mfbc.MFBC_ERR_INVALID and b"flag" in lib.mfbc_last_error()
    # CSC arrays (rows of A^T) are checked as rows before they are transposed,
    # on the host
    csc = mfbc.MFBC_CSC | mfbc.MFBC_DIRECTED
    st, h = _create(lib, 3, [0, 2, 3, 4], [2, 1, 0, 0], flags=csc)
    assert st == mfbc.MFBC_ERR_INVALID and b"sorted" in lib.mfbc_last_error()
    st, h = _create(lib, 3, [0, 1, 2, 3], [1, 7, 0], flags=csc)
    assert st == mfbc.MFBC_ERR_INVALID and b"range" in lib.mfbc_last_error()
    st, h = _create(lib, 3, [0, 2, 1, 3], [1, 2, 0], flags=csc)
    assert st == mfbc.MFBC_ERR_INVALID and b"rowptr" in lib.mfbc_last_error()
    assert lib.mfbc_bc(None, None, 0, None, None) == mfbc.MFBC_ERR_INVALID
    assert lib.mfbc_graph_release_scratch(None) == mfbc.MFBC_ERR_INVALID
    assert lib.mfbc_sssp_batch(None, None, 0, None, None, None) == mfbc.MFBC_ERR_INVALID
    out = ctypes.c_uint64()
    assert lib.mfbc_workspace_size(None, 1, 0, None, ctypes.byref(out)) == mfbc.MFBC_ERR_INVALID


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="no fallback"):
        mfbc_mod = __import__("paper_1609_07008_gb300")
        saved = mfbc_mod._lib
        try:
            mfbc_mod._lib = None
            mfbc_mod.load(str(tmp_path / "missing.so"))
        finally:
            mfbc_mod._lib = saved
