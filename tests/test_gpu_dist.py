"""GPU parity of the distance-ordered kernels (MFBC_PATH_DIST) on the cases
their structure makes special, against the CPU oracle through the C ABI:

  * weights with large gaps: a ring of w_max + 1 = 129 buckets (five flag
    words per item) with most distance values empty, so the step kernels
    skip buckets on the device;
  * ragged batches: source counts that are not multiples of 32 (padding
    columns that never hold a pair);
  * a hub of degree n - 1: per-lane arc walks far longer than a warp, and
    the automatic choice must avoid these kernels there;
  * average degree >= 32: the one-item-at-a-time scan variant;
  * sources repeated in the list (lambda is linear in the source list).

Bars as in test_gpu_parity: tau and sigma_bar bit-exact, lambda within 1e-9
relative with exact zeros.
"""
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


def random_weighted(n, deg, weights, seed, directed=True):
    rng = np.random.default_rng(seed)
    m = n * deg // (1 if directed else 2)
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)
    keep = u != v
    w = rng.choice(np.asarray(weights), m)
    return gg.from_edges(n, list(zip(u[keep].tolist(), v[keep].tolist())), directed=directed,
                         weights=w[keep].tolist())


def check_dist(g, srcs, n_b=0):
    G = mfbc.Graph.from_csr(g)
    try:
        want = oracle.bc(g, srcs)
        wd, ws, _ = oracle.sssp(g, srcs)
        lam = G.bc(srcs, n_b=n_b, path=mfbc.PATH_DIST)
        assert_lambda_close(lam, want)
        d, s = G.sssp(srcs, n_b=n_b, path=mfbc.PATH_DIST)
        assert np.array_equal(d, wd)
        assert np.array_equal(s, ws)
        _, prof = G.bc(srcs, n_b=n_b, profile=True)
        return prof["path"]
    finally:
        G.close()


def test_weight_gaps_span_several_flag_words():
    g = random_weighted(3000, 6, [1, 40, 77, 128], seed=11)
    srcs = gg.sample_sources(g, 100, seed=3)
    assert check_dist(g, srcs, n_b=64) == mfbc.PATH_DIST      # weights <= 128, no hub


def test_ragged_single_word_batches():
    g = gg.grid2d(24, weights=(1, 16), seed=4)
    srcs = gg.sample_sources(g, 45, seed=5)
    check_dist(g, srcs, n_b=32)                                 # 32 + 13 columns


def test_hub_forced_and_avoided_by_auto():
    rng = np.random.default_rng(7)
    n = 2000
    edges = [(0, v) for v in range(1, n)]
    extra = rng.integers(1, n, (3000, 2))
    edges += [(int(a), int(b)) for a, b in extra if a != b]
    w = rng.integers(1, 6, len(edges)).tolist()
    g = gg.from_edges(n, edges, directed=False, weights=w)
    srcs = gg.sample_sources(g, 70, seed=8)
    assert check_dist(g, srcs) == mfbc.PATH_GENERAL             # a hub: not for the distance kernels


def test_dense_graph_takes_the_one_item_scan():
    g = gg.erdos_renyi(2000, 40, weights=(1, 10), seed=9)
    srcs = gg.sample_sources(g, 96, seed=10)
    assert check_dist(g, srcs) == mfbc.PATH_DIST


def test_repeated_sources_count_once_each():
    g = gg.grid2d(16, weights=(1, 16), seed=12)
    G = mfbc.Graph.from_csr(g)
    try:
        one = G.bc(np.array([5, 77], np.int32), path=mfbc.PATH_DIST)
        rep = G.bc(np.array([5, 77, 5, 5, 77], np.int32), path=mfbc.PATH_DIST)
        want = oracle.bc(g, np.array([5, 77, 5, 5, 77], np.int32))
        assert_lambda_close(rep, want)
        a = oracle.bc(g, np.array([5], np.int32))
        b = oracle.bc(g, np.array([77], np.int32))
        assert_lambda_close(one, a + b)
    finally:
        G.close()
