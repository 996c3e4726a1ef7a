"""The persistent small-graph kernel (MFBC_PATH_SMALL) against the oracle,
through the C ABI, on what is particular to it:

  * its bounded waits: with the MFBC_OPT_TEST_STALL hook every group barrier
    waits for an arrival that never comes; each wait runs out of its budget,
    the launch returns and the call reports MFBC_ERR_TIMEOUT.  No fault, no
    hang: the same handle then computes the right answer;
  * the batch queue: many batches over few block groups, ragged last batch,
    several requests packed into shared batches (one lambda row each);
  * batches it hands to the general kernels: deeper than 254 levels (a long
    path) and path counts of 2^58 and more (a 40 x 40 grid from its corners,
    sigma_bar up to C(78, 39) ~ 2^75), with the inexact-count warning;
  * MFBF output rows (tau, sigma_bar) bit-exact.
Bars: tau and sigma_bar bit-exact below 2^53, lambda within 1e-9 relative
with exact zeros equal.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1609_07008_gb300 as mfbc

pytestmark = pytest.mark.gpu
SMALL = mfbc.PATH_SMALL


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_07008_gb300 import build
    build.build()
    mfbc.load()


def close(got, want, rtol=1e-9):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    zero = want == 0
    assert np.array_equal(got[zero], want[zero]), "exact zeros differ"
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.size == 0 or rel.max() <= rtol, f"max rel err {rel.max():.3e}"


def test_wait_budget_runs_out_and_the_call_reports_timeout():
    g = gg.erdos_renyi(1024, 8, seed=1)
    srcs = np.arange(0, 1024, 3, dtype=np.int32)
    G = mfbc.Graph.from_csr(g)
    with pytest.raises(mfbc.MFBCError) as e:
        G.bc(srcs, n_b=128, path=SMALL, test_stall=True)
    assert e.value.status == mfbc.MFBC_ERR_TIMEOUT
    assert "budget" in str(e.value)
    # the context and the handle are still usable
    close(G.bc(srcs, n_b=128, path=SMALL), oracle.bc(g, srcs))
    G.close()


@pytest.mark.parametrize("n_b", [32, 64, 128, 256])
def test_queue_of_batches_ragged_and_mfbf_rows(n_b):
    g = gg.rmat(12, 8, seed=3)
    srcs = gg.sample_sources(g, 1000, seed=4)          # ragged: 1000 is no multiple of 64..256
    G = mfbc.Graph.from_csr(g)
    close(G.bc(srcs, n_b=n_b, path=SMALL), oracle.bc(g, srcs))
    d, s = G.sssp(srcs[:70], n_b=n_b, path=SMALL)
    wd, ws, _ = oracle.sssp(g, srcs[:70])
    assert np.array_equal(d, wd) and np.array_equal(s, ws)
    G.close()


def test_directed_graph_with_unreachable_pairs():
    g = gg.rmat(11, 8, directed=True, seed=5)
    srcs = gg.sample_sources(g, 300, seed=6)
    G = mfbc.Graph.from_csr(g)
    close(G.bc(srcs, n_b=64, path=SMALL), oracle.bc(g, srcs))
    d, s = G.sssp(srcs[:50], n_b=64, path=SMALL)
    wd, ws, _ = oracle.sssp(g, srcs[:50])
    assert np.array_equal(d, wd) and np.array_equal(s, ws)
    G.close()


def test_packed_requests_each_equal_alone():
    import torch
    g = gg.rmat(12, 8, seed=7)
    rng = np.random.default_rng(8)
    lists = [gg.sample_sources(g, int(k), seed=int(i) + 10) for i, k in enumerate(rng.integers(1, 300, 9))]
    G = mfbc.Graph.from_csr(g)
    lam = G.bc_multi([torch.from_numpy(x).cuda() for x in lists], n_b=128, path=SMALL).cpu().numpy()
    for r, x in enumerate(lists):
        close(lam[r], oracle.bc(g, x))
    G.close()


def _grid(L):
    edges = [(r * L + c, r * L + c + 1) for r in range(L) for c in range(L - 1)]
    edges += [(r * L + c, (r + 1) * L + c) for r in range(L - 1) for c in range(L)]
    return gg.from_edges(L * L, edges, directed=False)


def test_counts_past_2p58_go_to_the_general_kernels():
    g = _grid(40)
    corners = np.array([0, 39, 40 * 39, 40 * 40 - 1, 20 * 40 + 20], np.int32)
    G = mfbc.Graph.from_csr(g)
    for p in (SMALL, mfbc.PATH_LEVEL):
        lam, warn = G.bc(corners, n_b=32, path=p, return_warn=True)
        assert warn & mfbc.MFBC_WARN_SIGMA_INEXACT
        close(lam, oracle.bc(g, corners))
    G.close()


def test_deeper_than_byte_levels_goes_to_the_general_kernels():
    n = 700
    g = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)], directed=False)
    srcs = np.array([0, 1, 350, 699, 5, 5], np.int32)      # depths up to 699 > 254; a shallow batch too
    G = mfbc.Graph.from_csr(g)
    close(G.bc(srcs, n_b=32, path=SMALL), oracle.bc(g, srcs))
    d, s = G.sssp(srcs, n_b=32, path=SMALL)
    wd, ws, _ = oracle.sssp(g, srcs)
    assert np.array_equal(d, wd) and np.array_equal(s, ws)
    G.close()
