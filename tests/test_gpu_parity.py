"""GPU parity: the CUDA path against the CPU oracle, through the C ABI.

Bars (written here, checked element by element):
  * distances tau                 -- bit-exact;
  * multiplicities sigma_bar      -- bit-exact (integers below 2^53);
  * centrality lambda             -- |gpu - oracle| <= 1e-9 * |oracle|, and
                                     oracle == 0 exactly where gpu == 0.
Both kernel families are exercised: the level kernels (unit weights) and the
general kernels (any integer weights; also forced on unit-weight graphs).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1609_07008_gb300 as mfbc

pytestmark = pytest.mark.gpu
RTOL = 1e-9
PATHS = [mfbc.PATH_LEVEL, mfbc.PATH_GENERAL, mfbc.PATH_DIST, mfbc.PATH_SMALL]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_07008_gb300 import build
    build.build()
    mfbc.load()


def assert_lambda_close(got, want, rtol=RTOL):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape
    zero = want == 0
    assert np.array_equal(got[zero], want[zero]), "exact zeros differ"
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.size == 0 or rel.max() <= rtol, f"max rel err {rel.max():.3e}"


def paths_for(g):
    return PATHS if g.w is None else [mfbc.PATH_GENERAL, mfbc.PATH_DIST]


def check_graph(g, srcs, n_b=0, sssp=True, paths=None):
    G = mfbc.Graph.from_csr(g)
    want_lam = oracle.bc(g, srcs)
    if sssp:
        wd, ws, _ = oracle.sssp(g, srcs)
    for p in (paths or paths_for(g)):
        lam = G.bc(srcs, n_b=n_b, path=p)
        assert_lambda_close(lam, want_lam)
        if sssp:
            d, s = G.sssp(srcs, n_b=n_b, path=p)
            assert np.array_equal(d, wd), f"dist mismatch on path {p}"
            assert np.array_equal(s, ws), f"sigma mismatch on path {p}"
    G.close()


# ------------------------------------------------------------ golden fixtures
def test_golden_fixtures_exact():
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_graphs.json")
    for case in json.load(open(path)):
        g = gg.CSRGraph(n=case["n"], rowptr=np.array(case["rowptr"], np.int64),
                        col=np.array(case["col"], np.int32),
                        w=None if case["w"] is None else np.array(case["w"], np.int32),
                        directed=case["directed"])
        G = mfbc.Graph.from_csr(g)
        srcs = np.array(case["sources"], np.int32)
        for p in paths_for(g):
            lam = G.bc(srcs, path=p)
            for v, q in enumerate(case["lambda"]):
                want = Fraction(q)
                if want == 0:
                    assert lam[v] == 0.0, case["name"]
                else:
                    assert abs(Fraction(lam[v]) - want) <= Fraction(1, 10**9) * want, case["name"]
            d, s = G.sssp(srcs, path=p)
            tau = np.array(case["tau"], np.int64)
            assert np.array_equal(np.where(d == mfbc.INF, -1, d), tau), case["name"]
            assert np.array_equal(s, np.array(case["sigma_bar"], np.float64)), case["name"]
        G.close()


# ----------------------------------------------------------- random small graphs
def _random_graph(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 90))
    directed = bool(rng.integers(0, 2))
    weighted = bool(rng.integers(0, 2))
    k = float(rng.uniform(0.5, 6))
    g = gg.erdos_renyi(n, k, directed=directed, weights=(1, int(rng.integers(1, 5))) if weighted else None,
                       seed=seed + 1)
    nsrc = int(rng.integers(0, 3 * n))
    srcs = rng.integers(0, n, size=nsrc).astype(np.int32)
    n_b = int(rng.choice([0, 32, 64, 96]))
    return g, srcs, n_b


@pytest.mark.parametrize("seed", range(60))
def test_random_graphs_match_oracle(seed):
    g, srcs, n_b = _random_graph(seed)
    check_graph(g, srcs, n_b=n_b)


# ------------------------------------------------------------- workloads
def test_er1024_all_sources_nb128():
    g, srcs, nb = gg.workload("er1024")
    check_graph(g, srcs, n_b=nb)


def test_rmat16_weighted_directed_nb512():
    g, srcs, nb = gg.workload("rmat16w")
    G = mfbc.Graph.from_csr(g)
    lam = G.bc(srcs, n_b=nb)
    assert_lambda_close(lam, oracle.bc(g, srcs))
    sub = srcs[:96]
    d, s = G.sssp(sub, n_b=nb)
    wd, ws, _ = oracle.sssp(g, sub)
    assert np.array_equal(d, wd) and np.array_equal(s, ws)
    G.close()


def test_er_2p20_k32_sampled_sources():
    g = gg.erdos_renyi(1 << 20, 32, seed=1)
    srcs = gg.sample_sources(g, 160, seed=2)
    G = mfbc.Graph.from_csr(g)
    for p in PATHS:
        assert_lambda_close(G.bc(srcs, n_b=128, path=p), oracle.bc(g, srcs))
    d, s = G.sssp(srcs[:8])
    wd, ws, _ = oracle.sssp(g, srcs[:8])
    assert np.array_equal(d, wd) and np.array_equal(s, ws)
    G.close()


def test_rmat22_bench_launch_configuration():
    # the bench's graph and sources at its batch width (n_b = 1024, level
    # kernels, landmark ordering on): 1056 sources = two batches, lambda
    # against the oracle element by element; then MFBF of the same 1056
    # sources (a full 1024-column batch and a ragged 32-column one) with 40
    # rows spread over both batches compared bit-exactly
    import torch
    g = gg.rmat(22, 16, seed=1)
    srcs = gg.sample_sources(g, 16384, seed=2)[:1056]
    G = mfbc.Graph.from_csr(g)
    assert_lambda_close(G.bc(srcs, n_b=1024), oracle.bc(g, srcs))
    dist, sig = G.sssp(torch.from_numpy(srcs).cuda(), n_b=1024)
    pick = np.concatenate([np.linspace(0, 1023, 24).astype(np.int64), np.arange(1024, 1056, 2)])
    assert len(np.unique(pick)) == 40
    idx = torch.from_numpy(pick).cuda()
    got_d, got_s = dist[idx].cpu().numpy(), sig[idx].cpu().numpy()
    del dist, sig
    torch.cuda.empty_cache()
    wd, ws, _ = oracle.sssp(g, srcs[pick])
    assert np.array_equal(got_d, wd)
    assert np.array_equal(got_s, ws)
    G.close()


def test_dense_weighted_er_2p16_k1024():
    g = gg.erdos_renyi(1 << 16, 1024, weights=(1, 100), seed=1)
    srcs = gg.sample_sources(g, 40, seed=3)
    G = mfbc.Graph.from_csr(g)
    assert_lambda_close(G.bc(srcs, n_b=64), oracle.bc(g, srcs))
    d, s = G.sssp(srcs[:4], n_b=32)
    wd, ws, _ = oracle.sssp(g, srcs[:4])
    assert np.array_equal(d, wd) and np.array_equal(s, ws)
    G.close()


def test_weighted_grid_sampled():
    g = gg.grid2d(96, weights=(1, 16), seed=1)
    srcs = np.array([0, 95, 48 * 96 + 48, 96 * 96 - 1], np.int32)
    check_graph(g, srcs, n_b=32)


# ------------------------------------------------------------ edge cases
def test_empty_source_list_and_empty_graph():
    g = gg.erdos_renyi(50, 3, seed=4)
    G = mfbc.Graph.from_csr(g)
    for p in PATHS:
        assert np.all(G.bc(np.zeros(0, np.int32), path=p) == 0.0)
        d, s = G.sssp(np.zeros(0, np.int32), path=p)
        assert d.shape == (0, 50)
    G.close()
    e = gg.CSRGraph(n=5, rowptr=np.zeros(6, np.int64), col=np.zeros(0, np.int32), w=None, directed=True)
    check_graph(e, np.array([0, 3, 3], np.int32))
    one = gg.CSRGraph(n=1, rowptr=np.zeros(2, np.int64), col=np.zeros(0, np.int32), w=None, directed=False)
    check_graph(one, np.array([0], np.int32))


def test_ragged_batches_duplicates_and_isolated_sources():
    g = gg.rmat(10, 8, seed=5)
    deg = g.out_degree()
    iso = np.flatnonzero(deg == 0)[:3]
    srcs = np.concatenate([gg.sample_sources(g, 77, seed=1), iso, [5, 5, 5]]).astype(np.int32)
    for n_b in (32, 64, 0):
        check_graph(g, srcs, n_b=n_b)


def test_n_b_independence_and_determinism():
    g = gg.rmat(11, 8, directed=True, seed=6)
    srcs = gg.sample_sources(g, 200, seed=3)
    G = mfbc.Graph.from_csr(g)
    ref_d, ref_s = G.sssp(srcs, n_b=32, path=mfbc.PATH_GENERAL)
    ref_l = G.bc(srcs, n_b=32, path=mfbc.PATH_GENERAL)
    for p in PATHS:
        for n_b in (64, 224, 256):
            d, s = G.sssp(srcs, n_b=n_b, path=p)
            assert np.array_equal(d, ref_d) and np.array_equal(s, ref_s)
            assert_lambda_close(G.bc(srcs, n_b=n_b, path=p), ref_l, rtol=1e-12)
    d2, s2 = G.sssp(srcs, n_b=64)
    d3, s3 = G.sssp(srcs, n_b=64)
    assert np.array_equal(d2, d3) and np.array_equal(s2, s3)
    G.close()


def test_long_path_exceeds_level_capacity_and_falls_back():
    n = 300                                  # depth 299 > the level kernels' 64-level capacity
    g = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)], directed=False)
    srcs = np.arange(0, n, 7, dtype=np.int32)
    check_graph(g, srcs, n_b=32, paths=[mfbc.PATH_LEVEL, mfbc.PATH_SMALL])


def _grid(L):
    edges = [(r * L + c, r * L + c + 1) for r in range(L) for c in range(L - 1)]
    edges += [(r * L + c, (r + 1) * L + c) for r in range(L - 1) for c in range(L)]
    return gg.from_edges(L * L, edges, directed=False)


def test_sigma_exactness_warning():
    from math import comb
    for p in PATHS:
        g = _grid(25)
        G = mfbc.Graph.from_csr(g)
        d, s, warn = G.sssp(np.array([0], np.int32), path=p, return_warn=True)
        assert s[0, -1] == comb(48, 24) and warn == 0
        _, warn = G.bc(np.array([0], np.int32), path=p, return_warn=True)
        assert warn == 0
        G.close()
        g = _grid(30)
        G = mfbc.Graph.from_csr(g)
        _, _, warn = G.sssp(np.array([0], np.int32), path=p, return_warn=True)
        assert warn & mfbc.MFBC_WARN_SIGMA_INEXACT
        _, warn = G.bc(np.array([0], np.int32), path=p, return_warn=True)
        assert warn & mfbc.MFBC_WARN_SIGMA_INEXACT
        G.close()


def test_invalid_inputs_are_rejected():
    bad = [
        (3, [0, 2, 3, 4], [2, 1, 0, 0], None, mfbc.MFBC_DIRECTED),     # unsorted row
        (3, [0, 2, 3, 4], [1, 1, 0, 0], None, mfbc.MFBC_DIRECTED),     # duplicate arc
        (3, [0, 1, 2, 3], [0, 2, 0], None, mfbc.MFBC_DIRECTED),        # self-loop
        (3, [0, 1, 2, 3], [1, 5, 0], None, mfbc.MFBC_DIRECTED),        # out of range
        (3, [0, 1, 2, 3], [1, 2, 0], [1, 0, 1], mfbc.MFBC_DIRECTED),   # zero weight
        (3, [0, 1, 2, 2], [1, 2], None, mfbc.MFBC_UNDIRECTED),         # asymmetric
        (2, [0, 1, 2], [1, 0], [3, 4], mfbc.MFBC_UNDIRECTED),          # asymmetric weights
        (3, [0, 2, 1, 3], [1, 2, 0], None, mfbc.MFBC_DIRECTED),        # decreasing rowptr
    ]
    for n, rp, col, w, fl in bad:
        with pytest.raises(mfbc.MFBCError) as e:
            mfbc.Graph(np.array(rp), np.array(col), None if w is None else np.array(w),
                       directed=fl == mfbc.MFBC_DIRECTED)
        assert e.value.status == mfbc.MFBC_ERR_INVALID
    with pytest.raises(mfbc.MFBCError) as e:      # (n-1) * w_max overflows int32 distances
        mfbc.Graph(np.array([0, 1, 1]), np.array([1]), np.array([2**31 - 1]), directed=True)
    assert e.value.status == mfbc.MFBC_ERR_OVERFLOW
    g = gg.erdos_renyi(20, 3, seed=1)
    G = mfbc.Graph.from_csr(g)
    for srcs in ([20], [-1]):
        with pytest.raises(mfbc.MFBCError) as e:
            G.bc(np.array(srcs, np.int32))
        assert e.value.status == mfbc.MFBC_ERR_INVALID
    with pytest.raises(mfbc.MFBCError):
        G.bc(np.array([1], np.int32), n_b=2048, path=mfbc.PATH_LEVEL)
    Gw = mfbc.Graph.from_csr(gg.erdos_renyi(20, 3, weights=(1, 3), seed=1))
    with pytest.raises(mfbc.MFBCError):
        Gw.bc(np.array([1], np.int32), path=mfbc.PATH_LEVEL)
    G.close()
    Gw.close()


def test_device_entry_points_match_host():
    import torch
    g = gg.rmat(11, 8, directed=True, weights=(1, 7), seed=8)
    srcs = gg.sample_sources(g, 70, seed=1)
    G = mfbc.Graph.from_csr(g)
    lam_h = G.bc(srcs, n_b=32)
    d_src = torch.from_numpy(srcs).cuda()
    lam_d = G.bc(d_src, n_b=32)
    torch.cuda.synchronize()
    assert np.array_equal(lam_d.cpu().numpy(), lam_h) or np.allclose(lam_d.cpu().numpy(), lam_h, rtol=1e-12, atol=0)
    dd, sd = G.sssp(d_src[:20], n_b=32)
    dh, sh = G.sssp(srcs[:20], n_b=32)
    assert np.array_equal(dd.cpu().numpy(), dh) and np.array_equal(sd.cpu().numpy(), sh)
    # graph built from device arrays, caller-provided workspace
    G2 = mfbc.Graph(torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda(),
                    torch.from_numpy(g.w).cuda(), directed=True)
    ws = torch.empty(G2.workspace_size(70, 0, n_b=32), dtype=torch.uint8, device="cuda")
    lam_w = G2.bc(srcs, n_b=32, workspace=ws)
    assert_lambda_close(lam_w, oracle.bc(g, srcs))
    G.close()
    G2.close()


def test_profile_reports_kernels():
    g = gg.rmat(12, 8, seed=2)
    srcs = gg.sample_sources(g, 64, seed=1)
    G = mfbc.Graph.from_csr(g)
    for p in PATHS:
        lam, prof = G.bc(srcs, n_b=64, path=p, profile=True, count_bytes=True)
        assert prof["batches"] == 1 and prof["fwd_iters"] > 0 and prof["bwd_iters"] > 0
        ks = prof["kernels"]
        main = {mfbc.PATH_LEVEL: "level_mfbf_gather", mfbc.PATH_GENERAL: "mfbf_relax_min",
                mfbc.PATH_DIST: "dist_mfbf", mfbc.PATH_SMALL: "small_persistent"}[p]
        assert ks[main]["launches"] > 0 and ks[main]["ms"] > 0 and ks[main]["bytes"] > 0
    G.close()


def test_source_ordering_with_few_landmarks_and_duplicates():
    # 12 non-isolated vertices (fewer than the 128 landmarks the ordering
    # wants), 40 isolated ones, and 300 sources with repeats across 3 batches
    edges = [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (4, 5), (5, 6), (6, 7), (7, 4), (8, 9), (9, 10), (10, 11)]
    g = gg.from_edges(52, edges, directed=False)
    rng = np.random.default_rng(3)
    srcs = rng.integers(0, 52, size=300).astype(np.int32)
    want = oracle.bc(g, srcs)
    G = mfbc.Graph.from_csr(g)
    a = G.bc(srcs, n_b=128, path=mfbc.PATH_LEVEL)
    b = G.bc(srcs, n_b=128, path=mfbc.PATH_LEVEL, keep_order=True)
    assert_lambda_close(a, want)
    assert_lambda_close(b, want)
    G.close()


def test_source_ordering_over_disconnected_components():
    # two R-MAT components side by side: sources of the second one are
    # unreachable from every landmark of the first and sort last
    g1 = gg.rmat(11, 8, seed=4)
    g2 = gg.erdos_renyi(1500, 6, seed=5)
    e = [(int(u), int(v)) for u in range(g1.n) for v in g1.col[g1.rowptr[u]:g1.rowptr[u + 1]] if u < v]
    e += [(int(u) + g1.n, int(v) + g1.n) for u in range(g2.n) for v in g2.col[g2.rowptr[u]:g2.rowptr[u + 1]] if u < v]
    g = gg.from_edges(g1.n + g2.n, e, directed=False)
    srcs = gg.sample_sources(g, 700, seed=6)
    want = oracle.bc(g, srcs)
    G = mfbc.Graph.from_csr(g)
    for n_b in (128, 256):
        assert_lambda_close(G.bc(srcs, n_b=n_b), want)
    G.close()


def test_l2_fetch_hint_is_restored():
    # the calls set the context's L2 fetch granularity to 32 bytes while they
    # run; the caller's value must be back afterwards
    import ctypes
    rt = None
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            pass
    if rt is None:
        pytest.skip("no libcudart to query the limit")
    import torch
    torch.zeros(1, device="cuda")
    limit = 5                                    # cudaLimitMaxL2FetchGranularity
    v = ctypes.c_size_t(0)
    assert rt.cudaDeviceSetLimit(limit, ctypes.c_size_t(128)) == 0
    assert rt.cudaDeviceGetLimit(ctypes.byref(v), limit) == 0
    before = v.value
    g = gg.rmat(10, 8, seed=2)
    G = mfbc.Graph.from_csr(g)
    srcs = gg.sample_sources(g, 200, seed=1)
    assert_lambda_close(G.bc(srcs), oracle.bc(g, srcs))
    G.sssp(srcs[:10])
    assert rt.cudaDeviceGetLimit(ctypes.byref(v), limit) == 0
    assert v.value == before
    G.close()


def test_source_ordering_does_not_change_lambda():
    g = gg.rmat(13, 8, seed=9)
    srcs = gg.sample_sources(g, 300, seed=5)
    want = oracle.bc(g, srcs)
    G = mfbc.Graph.from_csr(g)
    for n_b in (32, 96):
        a = G.bc(srcs, n_b=n_b)
        b = G.bc(srcs, n_b=n_b, keep_order=True)
        assert_lambda_close(a, want)
        assert_lambda_close(b, want)
        assert_lambda_close(a, b, rtol=1e-12)
    G.close()


@pytest.mark.parametrize("weighted", [False, True])
def test_autotune_picks_a_candidate_and_results_are_unchanged(weighted):
    g = gg.rmat(12, 8, directed=weighted, weights=(1, 9) if weighted else None, seed=31)
    srcs = gg.sample_sources(g, 600, seed=1)
    G = mfbc.Graph.from_csr(g)
    t = G.autotune(srcs)
    if weighted:
        # general kernels (3 widths x {atomic x 2 arc steps, segmented, hash, per product})
        # and distance kernels (3 widths)
        assert t["path"] in (mfbc.PATH_GENERAL, mfbc.PATH_DIST) and t["tried"] == 18
        assert t["arcs"] in ((0, 1, 8) if t["path"] == mfbc.PATH_GENERAL else (0,))
        assert t["accumulator"] in ((0, 1, 2, 3) if t["path"] == mfbc.PATH_GENERAL else (0,))
    else:
        # level kernels (3 widths) and the persistent small-graph kernel (4 widths)
        assert t["path"] in (mfbc.PATH_LEVEL, mfbc.PATH_SMALL) and t["tried"] == 7 and t["arcs"] == 0
    assert t["n_b"] in {32, 64, 128, 256, 512} and t["ms_per_source"] > 0
    lam, prof = G.bc(srcs, profile=True)
    assert prof["path"] == t["path"]
    widest = 256 if t["path"] == mfbc.PATH_SMALL else 512
    if t["n_b"] < widest:                   # a wider width was tried and lost: it caps later calls
        assert prof["n_b"] <= t["n_b"]
    assert_lambda_close(lam, oracle.bc(g, srcs))
    G.close()


def test_release_scratch_frees_the_cached_workspace():
    # mfbc_graph_release_scratch gives the handle's cached scratch back; the
    # next call allocates it again and computes the same result
    import torch
    g = gg.rmat(14, 8, seed=12)
    srcs = gg.sample_sources(g, 512, seed=3)
    G = mfbc.Graph.from_csr(g)
    a = G.bc(srcs, n_b=512, path=mfbc.PATH_LEVEL)
    torch.cuda.synchronize()
    held = torch.cuda.mem_get_info()[0]
    G.release_scratch()
    freed = torch.cuda.mem_get_info()[0] - held
    assert freed >= G.workspace_size(512, 0, n_b=512, path=mfbc.PATH_LEVEL) // 2
    G.release_scratch()                           # nothing cached: a no-op
    assert_lambda_close(G.bc(srcs, n_b=512, path=mfbc.PATH_LEVEL), a, rtol=1e-12)
    assert_lambda_close(a, oracle.bc(g, srcs))
    G.close()
