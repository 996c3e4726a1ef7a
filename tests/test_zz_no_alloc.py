"""mfbc_bc_static: betweenness centrality for callers that must not allocate.

Some callers cannot call cudaMalloc when they need a result -- a serving
process whose device memory is fully partitioned by its own pool, code inside
an allocator callback, a plug-in whose framework owns all device memory.
mfbc_bc_static keeps its scratch in a fixed __device__ array instead.  These
tests call it through the C ABI twice in a row and check each result against
the allocating entry point mfbc_bc_device (lambda within 1e-9 relative, exact
zeros equal), that the second call leaves the device's free memory exactly
as it was, that it reports path counts of 2^53 and more as the other entry
points do, and that graphs larger than its array are rejected.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import paper_1609_07008_gb300 as mfbc

pytestmark = pytest.mark.gpu
RTOL = 1e-9


@pytest.fixture(scope="module")
def lib():
    from paper_1609_07008_gb300 import build
    build.build()
    lib = mfbc.load()
    lib.mfbc_bc_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]
    lib.mfbc_bc_static.restype = ctypes.c_int
    lib.mfbc_static_max_vertices.argtypes = []
    lib.mfbc_static_max_vertices.restype = ctypes.c_uint64
    return lib


def _close(got, want):
    zero = want == 0
    assert np.array_equal(got[zero], want[zero])
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.size == 0 or rel.max() <= RTOL, rel.max()


@pytest.mark.parametrize("weighted", [False, True])
def test_static_matches_allocating_entry_point_twice(lib, weighted):
    import torch
    g = gg.rmat(12, 8, directed=weighted, weights=(1, 9) if weighted else None, seed=11)
    assert g.n <= lib.mfbc_static_max_vertices()
    G = mfbc.Graph.from_csr(g)
    for call, seed in enumerate((1, 2)):
        srcs = torch.from_numpy(gg.sample_sources(g, 83 + 20 * call, seed=seed)).cuda()
        want = G.bc(srcs).cpu().numpy()
        lam = torch.full((g.n,), -1.0, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        warn = ctypes.c_uint32(7)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = lib.mfbc_bc_static(G._h, ctypes.c_void_p(srcs.data_ptr()), srcs.numel(),
                                ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(stream), ctypes.byref(warn))
        assert st == mfbc.MFBC_OK, lib.mfbc_last_error()
        torch.cuda.synchronize()
        if call == 1:
            # the first call looked up the array's address; later calls must
            # not take or give back any device memory
            assert torch.cuda.mem_get_info()[0] == free_before
        assert warn.value == 0
        _close(lam.cpu().numpy(), want)
    G.close()


def _grid(L):
    edges = [(r * L + c, r * L + c + 1) for r in range(L) for c in range(L - 1)]
    edges += [(r * L + c, (r + 1) * L + c) for r in range(L - 1) for c in range(L)]
    return gg.from_edges(L * L, edges, directed=False)


def test_static_reports_inexact_path_counts(lib):
    # unweighted L x L grid from a corner: sigma_bar of the far corner is
    # C(2L-2, L-1), 2^47.3 for L = 25 and 2^54.7 (past 2^53) for L = 30
    import torch
    for L, inexact in ((25, False), (30, True)):
        G = mfbc.Graph.from_csr(_grid(L))
        srcs = torch.tensor([0, L * L - 1], dtype=torch.int32, device="cuda")
        want, want_warn = G.bc(srcs, return_warn=True)
        lam = torch.empty(L * L, dtype=torch.float64, device="cuda")
        warn = ctypes.c_uint32(0)
        st = lib.mfbc_bc_static(G._h, ctypes.c_void_p(srcs.data_ptr()), 2, ctypes.c_void_p(lam.data_ptr()),
                                None, ctypes.byref(warn))
        assert st == mfbc.MFBC_OK, lib.mfbc_last_error()
        torch.cuda.synchronize()
        assert bool(warn.value & mfbc.MFBC_WARN_SIGMA_INEXACT) == inexact == bool(want_warn)
        _close(lam.cpu().numpy(), want.cpu().numpy())
        G.close()


def test_static_rejects_graphs_beyond_its_array(lib):
    import torch
    n = int(lib.mfbc_static_max_vertices()) + 1
    g = gg.erdos_renyi(n, 2, seed=3)
    G = mfbc.Graph.from_csr(g)
    srcs = torch.zeros(1, dtype=torch.int32, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    st = lib.mfbc_bc_static(G._h, ctypes.c_void_p(srcs.data_ptr()), 1, ctypes.c_void_p(lam.data_ptr()), None, None)
    assert st == mfbc.MFBC_ERR_INVALID
    assert b"too large" in lib.mfbc_last_error()
    bad = torch.tensor([n + 5], dtype=torch.int32, device="cuda")
    small = mfbc.Graph.from_csr(gg.erdos_renyi(100, 3, seed=1))
    lam2 = torch.empty(100, dtype=torch.float64, device="cuda")
    st = lib.mfbc_bc_static(small._h, ctypes.c_void_p(bad.data_ptr()), 1, ctypes.c_void_p(lam2.data_ptr()), None,
                            None)
    assert st == mfbc.MFBC_ERR_INVALID
    G.close()
    small.close()
