"""GPU parity at the widths and magnitudes the benchmarks run, through the C ABI.

  * the distance-ordered kernels (MFBC_PATH_DIST) at n_b = 1024 and 4096 --
    32 and 128 words per vertex, the n*W-slot bucket lists and the
    n*n_b-entry settled list at full size -- on the weighted 256^2 grid with
    4096 sources and on the dense weighted Erdos-Renyi graph (n = 2^16,
    k = 1024) with 1024 sources; the general kernels at the same widths;
  * path counts between 2^48 and 2^55: unweighted L x L grids (L = 28, 29,
    30) from their four corners, where sigma_bar of the opposite corner is
    C(2L-2, L-1) (2^50.8, 2^52.8, 2^54.7).  The level kernels carry these
    counts as exact 64-bit integers and convert them to double-float for
    MFBr; every family is compared with the oracle.

Bars: tau bit-exact; sigma_bar bit-exact below 2^53 (above it, within 1e-12
relative: FP64 sums round, Sec. 4.1.1's counts are integers); lambda within
1e-9 relative with exact zeros equal.  Lemma 1 and Theorem 1 (Sec. 4.1.3,
Sec. 4.3) fix these results.
"""
from math import comb

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1609_07008_gb300 as mfbc

pytestmark = pytest.mark.gpu
RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_07008_gb300 import build
    build.build()
    mfbc.load()


def assert_lambda_close(got, want, rtol=RTOL):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    zero = want == 0
    assert np.array_equal(got[zero], want[zero]), "exact zeros differ"
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.size == 0 or rel.max() <= rtol, f"max rel err {rel.max():.3e}"


def check_rows(G, srcs, rows, n_b, path, g):
    """MFBF of the whole source list on the device at width n_b; the sampled
    rows (indices into srcs, spread over every batch) against the oracle."""
    import torch
    d_src = torch.from_numpy(np.ascontiguousarray(srcs)).cuda()
    dist, sig = G.sssp(d_src, n_b=n_b, path=path)
    idx = torch.from_numpy(np.asarray(rows, np.int64)).cuda()
    got_d = dist[idx].cpu().numpy()
    got_s = sig[idx].cpu().numpy()
    del dist, sig
    torch.cuda.empty_cache()
    wd, ws, _ = oracle.sssp(g, srcs[rows])
    assert np.array_equal(got_d, wd), f"dist mismatch (path {path}, n_b {n_b})"
    assert np.array_equal(got_s, ws), f"sigma mismatch (path {path}, n_b {n_b})"


def spread(nsrc, n_b, per_batch):
    """per_batch row indices from each batch of n_b columns (first, last, between)."""
    rows = []
    for b0 in range(0, nsrc, n_b):
        b1 = min(nsrc, b0 + n_b)
        rows += np.unique(np.linspace(b0, b1 - 1, per_batch).astype(np.int64)).tolist()
    return np.array(rows, np.int64)


@pytest.fixture(scope="module")
def grid256w():
    g = gg.grid2d(256, weights=(1, 16), seed=1)
    srcs = gg.sample_sources(g, 4096, seed=2)
    return g, srcs, oracle.bc(g, srcs)


@pytest.mark.parametrize("n_b", [1024, 4096])
def test_dist_kernels_wide_batches_weighted_grid(grid256w, n_b):
    g, srcs, want = grid256w
    G = mfbc.Graph.from_csr(g)
    assert_lambda_close(G.bc(srcs, n_b=n_b, path=mfbc.PATH_DIST), want)
    check_rows(G, srcs, spread(len(srcs), n_b, 32 if n_b == 4096 else 8), n_b, mfbc.PATH_DIST, g)
    G.close()


def test_general_kernels_wide_batch_weighted_grid(grid256w):
    g, srcs, want = grid256w
    G = mfbc.Graph.from_csr(g)
    assert_lambda_close(G.bc(srcs, n_b=4096, path=mfbc.PATH_GENERAL), want)
    G.close()


@pytest.fixture(scope="module")
def dense_er():
    g = gg.erdos_renyi(1 << 16, 1024, weights=(1, 100), seed=1)
    srcs = gg.sample_sources(g, 1024, seed=3)
    return g, srcs, oracle.bc(g, srcs)


@pytest.mark.parametrize("n_b", [1024, 4096])
def test_dist_kernels_wide_batches_dense_weighted_er(dense_er, n_b):
    # n_b = 4096 with 1024 sources: one batch of 128 words, 96 of them padding
    g, srcs, want = dense_er
    G = mfbc.Graph.from_csr(g)
    assert_lambda_close(G.bc(srcs, n_b=n_b, path=mfbc.PATH_DIST), want)
    check_rows(G, srcs, np.array([0, 1, 511, 777, 1022, 1023]), n_b, mfbc.PATH_DIST, g)
    G.close()


def _grid(L):
    edges = [(r * L + c, r * L + c + 1) for r in range(L) for c in range(L - 1)]
    edges += [(r * L + c, (r + 1) * L + c) for r in range(L - 1) for c in range(L)]
    return gg.from_edges(L * L, edges, directed=False)


@pytest.mark.parametrize("L", [28, 29, 30])
@pytest.mark.parametrize("path", [mfbc.PATH_LEVEL, mfbc.PATH_GENERAL, mfbc.PATH_DIST])
def test_large_path_counts_unweighted_grid_corners(L, path):
    g = _grid(L)
    corners = np.array([0, L - 1, L * (L - 1), L * L - 1], np.int32)
    G = mfbc.Graph.from_csr(g)
    lam, warn = G.bc(corners, path=path, return_warn=True)
    assert_lambda_close(lam, oracle.bc(g, corners))
    assert bool(warn & mfbc.MFBC_WARN_SIGMA_INEXACT) == (comb(2 * L - 2, L - 1) >= 2**53)
    d, s = G.sssp(corners[:1], path=path)
    # from corner (0, 0): tau = r + c and sigma_bar = C(r + c, r) on every vertex
    r, c = np.divmod(np.arange(L * L), L)
    assert np.array_equal(d[0], (r + c).astype(np.int32))
    exact = np.array([float(comb(int(a + b), int(a))) for a, b in zip(r, c)])
    if path == mfbc.PATH_LEVEL:
        # exact 64-bit integer counts, rounded once to FP64
        assert np.array_equal(s[0], exact)
    else:
        small = exact < 2**53
        assert np.array_equal(s[0][small], exact[small])
        assert np.max(np.abs(s[0] - exact) / exact) <= 1e-12
    G.close()


def test_dist_kernels_width_cap_at_a_million_vertices():
    # the distance kernels address their settled list (up to n * n_b
    # entries) with 32-bit offsets, so the planner keeps n * n_b < 2^32: on
    # the weighted 1024^2 grid (n = 2^20) n_b is at most 4064.  The widest
    # batch must give the lambda of four 1024-column batches.
    g = gg.grid2d(1024, weights=(1, 16), seed=1)
    srcs = gg.sample_sources(g, 4064, seed=2)
    G = mfbc.Graph.from_csr(g)
    with pytest.raises(mfbc.MFBCError) as e:
        G.bc(srcs[:64], n_b=4096, path=mfbc.PATH_DIST)
    assert e.value.status == mfbc.MFBC_ERR_INVALID and "4064" in str(e.value)
    wide, prof = G.bc(srcs, path=mfbc.PATH_DIST, profile=True)
    assert prof["n_b"] == 4064 and prof["batches"] == 1
    narrow = G.bc(srcs, n_b=1024, path=mfbc.PATH_DIST)
    assert_lambda_close(wide, narrow, rtol=1e-12)
    G.close()
