"""Several requests in one pass (mfbc_bc_multi_device) and the serving loop
on the GPU: every request's lambda must be the one it gets alone (oracle and
mfbc_bc_device, 1e-9 relative, exact zeros), whatever it was packed with."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1609_07008_gb300 as mfbc
from paper_1609_07008_gb300.serve import Server, latency_stats, make_requests, run_served

pytestmark = pytest.mark.gpu
RTOL = 1e-9


def _close(got, want, rtol=RTOL):
    got, want = np.asarray(got), np.asarray(want)
    zero = want == 0
    assert np.array_equal(got[zero], want[zero])
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.size == 0 or rel.max() <= rtol, rel.max()


def _lists(g, sizes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in sizes:
        out.append(rng.integers(0, g.n, size=k).astype(np.int32))   # repeats allowed
    return out


CASES = [
    ("level", False, mfbc.PATH_LEVEL),
    ("general-unit", False, mfbc.PATH_GENERAL),
    ("general-weighted", True, mfbc.PATH_GENERAL),
    ("dist-weighted", True, mfbc.PATH_DIST),
]


@pytest.mark.parametrize("name,weighted,path", CASES)
def test_bc_multi_rows_equal_each_request_alone(name, weighted, path):
    import torch
    g = gg.rmat(11, 8, directed=weighted, weights=(1, 9) if weighted else None, seed=21)
    # sizes chosen to mix requests inside 128-column quads, leave words
    # partly empty, include an empty request, and span several batches
    sizes = [1, 31, 32, 33, 0, 70, 200, 5, 300, 17]
    lists = _lists(g, sizes, seed=5)
    G = mfbc.Graph.from_csr(g)
    lam = G.bc_multi([torch.from_numpy(x).cuda() for x in lists], n_b=128, path=path).cpu().numpy()
    assert lam.shape == (len(lists), g.n)
    for r, x in enumerate(lists):
        want = oracle.bc(g, x) if len(x) else np.zeros(g.n)
        _close(lam[r], want)
        if len(x):
            _close(lam[r], G.bc(x, n_b=128, path=path))
    G.close()


def test_bc_multi_single_request_equals_bc_and_rejects_bad_offsets():
    import torch
    g = gg.rmat(10, 8, seed=3)
    G = mfbc.Graph.from_csr(g)
    x = torch.from_numpy(gg.sample_sources(g, 150, seed=1)).cuda()
    lam = G.bc_multi([x])
    _close(lam[0].cpu().numpy(), G.bc(x, keep_order=True).cpu().numpy())
    with pytest.raises(mfbc.MFBCError):
        G.bc_multi((x, np.array([0, 10, 5, 150], dtype=np.int32)))
    with pytest.raises(mfbc.MFBCError):
        G.bc_multi((x, np.array([0, 149], dtype=np.int32)))
    G.close()


def test_server_answers_each_request_as_if_alone():
    g_r = gg.rmat(10, 8, seed=11)
    g_e = gg.erdos_renyi(800, 6, seed=12)
    g_w = gg.grid2d(20, weights=(1, 16), seed=13)
    host = {"rmat": g_r, "er": g_e, "grid": g_w}
    graphs = {k: mfbc.Graph.from_csr(g) for k, g in host.items()}
    reqs = make_requests({k: g.n for k, g in host.items()}, 36, rate=400.0, lo=8, hi=300, seed=9)
    srv = Server(graphs, budget_bytes=8 << 30, max_cols=512, n_b=256).start()
    run_served(srv, reqs, timeout=300)
    srv.close()
    assert any(gl.nreq > 1 for gl in srv.log)          # requests were packed together
    for r in reqs:
        _close(r.result, oracle.bc(host[r.graph], r.sources))
        _close(r.result, graphs[r.graph].bc(r.sources, keep_order=True))
    st = latency_stats(reqs, {k: g.m for k, g in host.items()})
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"] and st["gteps"] > 0
    for G in graphs.values():
        G.close()


@pytest.mark.parametrize("path", [mfbc.PATH_LEVEL, mfbc.PATH_SMALL, mfbc.PATH_GENERAL])
def test_requests_split_over_calls_accumulate_into_their_rows(path):
    # the serving loop's use of mfbc_bc_multi_device: each request owns a row
    # of a pool (lambda_rows, in any order), and a request split over several
    # calls (MFBC_OPT_ACCUMULATE) sums to its answer alone
    import torch
    g = gg.rmat(11, 8, seed=31)
    lists = _lists(g, [300, 45, 128, 7], seed=6)
    G = mfbc.Graph.from_csr(g)
    pool = torch.full((6, g.n), 123.0, dtype=torch.float64, device="cuda")
    rows = [4, 0, 2, 5]
    pool[rows] = 0.0
    cuts = [(0, 100), (100, 300)]
    for lo, hi in cuts:
        parts = [torch.from_numpy(x[min(lo, len(x)):min(hi, len(x))]).cuda() for x in lists]
        G.bc_multi(parts, n_b=128, path=path, out=pool, rows=rows, accumulate=True)
    got = pool.cpu().numpy()
    for r, x in zip(rows, lists):
        _close(got[r], oracle.bc(g, x))
    assert np.all(got[[1, 3]] == 123.0)                # rows no request names are untouched
    # without accumulate the named rows are overwritten
    G.bc_multi([torch.from_numpy(x).cuda() for x in lists], n_b=128, path=path, out=pool, rows=rows)
    got = pool.cpu().numpy()
    for r, x in zip(rows, lists):
        _close(got[r], oracle.bc(g, x))
    G.close()
