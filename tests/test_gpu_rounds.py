"""The level kernels' product rounds when their buffers run out, and level
state across batches, against the oracle through the C ABI.

* MFBC_OPT_TEST_SMALL_ROUNDS gives the pair and segment buffers 2^16 slots,
  so MFBF and MFBr rounds overflow: an unchecked round's gather then does
  nothing (MFBr: the rest of the sweep returns at once) and the host redoes
  it over halves of the work items.  tau and sigma_bar must stay bit-exact
  and lambda within 1e-9 (Lemma 1, Theorem 1: the products do not depend on
  how the work is split).
* Graphs deep enough that the distance profiles ordering the sources (128
  landmarks) fill the level lists: every later batch must start from clean
  masks.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1609_07008_gb300 as mfbc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_07008_gb300 import build
    build.build()
    mfbc.load()


def close(got, want, rtol=1e-9):
    zero = want == 0
    assert np.array_equal(got[zero], want[zero]), "exact zeros differ"
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.size == 0 or rel.max() <= rtol, f"max rel err {rel.max():.3e}"


@pytest.mark.parametrize("n_b", [128, 512])
def test_overflowing_rounds_are_redone_over_halves(n_b):
    g = gg.rmat(12, 16, seed=3)
    srcs = gg.sample_sources(g, 600, seed=4)
    G = mfbc.Graph.from_csr(g)
    want = oracle.bc(g, srcs)
    lam, prof = G.bc(srcs, n_b=n_b, path=mfbc.PATH_LEVEL, test_small_rounds=True, profile=True)
    close(lam, want)
    assert prof["kernels"]["level_round_split"]["launches"] > 0
    # the same call without the hook agrees to rounding
    close(G.bc(srcs, n_b=n_b, path=mfbc.PATH_LEVEL), lam, rtol=1e-12)
    d, s = G.sssp(srcs[:80], n_b=n_b, path=mfbc.PATH_LEVEL, test_small_rounds=True)
    wd, ws, _ = oracle.sssp(g, srcs[:80])
    assert np.array_equal(d, wd) and np.array_equal(s, ws)
    G.close()


def test_packed_requests_with_overflowing_rounds():
    import torch
    g = gg.erdos_renyi(3000, 24, seed=5)
    rng = np.random.default_rng(6)
    reqs = [rng.choice(g.n, k, replace=False).astype(np.int32) for k in (70, 200, 33)]
    G = mfbc.Graph.from_csr(g)
    lam = G.bc_multi([torch.from_numpy(r).cuda() for r in reqs], n_b=128, path=mfbc.PATH_LEVEL,
                     test_small_rounds=True).cpu().numpy()
    for r, x in zip(reqs, lam):
        close(x, oracle.bc(g, r))
    G.close()


def _grid(L):
    edges = [(r * L + c, r * L + c + 1) for r in range(L) for c in range(L - 1)]
    edges += [(r * L + c, (r + 1) * L + c) for r in range(L - 1) for c in range(L)]
    return gg.from_edges(L * L, edges, directed=False)


@pytest.mark.parametrize("L", [20, 30, 36])
def test_deep_grids_with_ordered_sources(L):
    # more sources than one batch: the sources are ordered by their distances
    # to 128 landmarks first (an MFBF pass on the level kernels whose level
    # lists can overflow on deep graphs); the batches after it start clean
    g = _grid(L)
    srcs = np.random.default_rng(L).choice(g.n, min(g.n, 400), replace=False).astype(np.int32)
    G = mfbc.Graph.from_csr(g)
    want = oracle.bc(g, srcs)
    close(G.bc(srcs, n_b=256, path=mfbc.PATH_LEVEL), want)
    close(G.bc(srcs, n_b=256, path=mfbc.PATH_LEVEL, test_small_rounds=True), want)
    G.close()
