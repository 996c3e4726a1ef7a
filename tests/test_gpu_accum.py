"""The general kernels' accumulators against the oracle, through the C ABI.

MFBC_ACCUM_ATOMIC pushes candidates from the frontier and reduces them with
atomics at the target; MFBC_ACCUM_SEGMENTED pulls them per target row and
reduces each (vertex, 32-column word) segment in registers, a block per row
longer than 256 arcs; MFBC_ACCUM_HASH pushes, but first reduces a block's
candidates for high-degree targets in a shared-memory hash table and merges
each slot column once.  All compute the multpath product (min distance, tied
multiplicities summed, Sec. 4.1.1) and the centpath product of MFBr (Sec.
4.2), so tau and sigma_bar must be bit-exact and lambda within 1e-9 relative
(exact zeros equal), on every kind of graph, on rows on both sides of the
block threshold, and with more hot targets per block than the hash table
holds.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1609_07008_gb300 as mfbc

pytestmark = pytest.mark.gpu
ACCS = [mfbc.ACCUM_ATOMIC, mfbc.ACCUM_SEGMENTED, mfbc.ACCUM_HASH, mfbc.ACCUM_AUTO]


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


def check(g, srcs, n_b, accs=ACCS):
    G = mfbc.Graph.from_csr(g)
    want = oracle.bc(g, srcs)
    wd, ws, _ = oracle.sssp(g, srcs[:64])
    for acc in accs:
        close(G.bc(srcs, n_b=n_b, path=mfbc.PATH_GENERAL, accumulator=acc), want)
        d, s = G.sssp(srcs[:64], n_b=n_b, path=mfbc.PATH_GENERAL, accumulator=acc)
        assert np.array_equal(d, wd) and np.array_equal(s, ws), f"MFBF mismatch, accumulator {acc}"
    G.close()


@pytest.mark.parametrize("seed", range(16))
def test_random_graphs(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 400))
    directed = bool(seed % 2)
    weights = (1, int(rng.integers(1, 6))) if seed % 4 < 2 else None
    g = gg.erdos_renyi(n, float(rng.uniform(1, 12)), directed=directed, weights=weights, seed=seed + 7)
    srcs = rng.integers(0, n, size=int(rng.integers(1, 3 * n))).astype(np.int32)
    check(g, srcs, n_b=int(rng.choice([32, 64, 160])))


def test_hub_rows_past_the_block_threshold():
    # vertex 0 has arcs to and from every other vertex (rows of 1499 arcs,
    # block-reduced), a middle vertex has 200 (warp-reduced); small weights
    # make many ties
    rng = np.random.default_rng(5)
    n = 1500
    edges = [(0, v) for v in range(1, n)] + [(v, 0) for v in range(1, n)]
    edges += [(7, v) for v in range(8, 208)]
    edges += [(int(a), int(b)) for a, b in rng.integers(1, n, size=(6000, 2)) if a != b]
    edges = sorted(set(edges))
    w = rng.integers(1, 4, size=len(edges)).tolist()
    g = gg.from_edges(n, edges, directed=True, weights=w)
    srcs = rng.integers(0, n, size=300).astype(np.int32)
    check(g, srcs, n_b=128)


def test_weighted_rmat16_directed_segmented():
    g, srcs, nb = gg.workload("rmat16w")
    srcs = srcs[:1024]
    G = mfbc.Graph.from_csr(g)
    want = oracle.bc(g, srcs)
    for acc in (mfbc.ACCUM_SEGMENTED, mfbc.ACCUM_HASH, mfbc.ACCUM_AUTO):
        close(G.bc(srcs, n_b=nb, path=mfbc.PATH_GENERAL, accumulator=acc), want)
    wd, ws, _ = oracle.sssp(g, srcs[:40])
    for acc in (mfbc.ACCUM_SEGMENTED, mfbc.ACCUM_HASH):
        d, s = G.sssp(srcs[:40], n_b=nb, path=mfbc.PATH_GENERAL, accumulator=acc)
        assert np.array_equal(d, wd) and np.array_equal(s, ws), f"MFBF mismatch, accumulator {acc}"
    G.close()


def _many_hubs(directed, weights, seed):
    # 300 hubs: every other vertex has 40 arcs to hubs and 2 to non-hubs,
    # every hub 400 arcs to non-hubs and 5 to hubs, so hubs are hot targets of
    # both products (in- and out-degree far above twice the average) and the
    # 32 items of a hash block meet a few hundred distinct hot keys: more than
    # the table's 128 slots (probe collisions and the atomic fallback)
    rng = np.random.default_rng(seed)
    n, H = 3000, 300
    edges = set()
    for v in range(H, n):
        for h in rng.choice(H, 40, replace=False):
            edges.add((v, int(h)))
        for u in rng.integers(H, n, size=2):
            if u != v:
                edges.add((v, int(u)))
    for h in range(H):
        for u in rng.choice(np.arange(H, n), 400, replace=False):
            edges.add((h, int(u)))
        for u in rng.integers(0, H, size=5):
            if u != h:
                edges.add((h, int(u)))
    if not directed:
        edges |= {(b, a) for a, b in edges}
    edges = sorted(edges)
    w = None
    if weights:
        wd = {}
        for a, b in edges:
            k = (min(a, b), max(a, b)) if not directed else (a, b)
            if k not in wd:
                wd[k] = int(rng.integers(1, weights + 1))
        w = [wd[(min(a, b), max(a, b)) if not directed else (a, b)] for a, b in edges]
    return gg.from_edges(n, edges, directed=directed, weights=w)


@pytest.mark.parametrize("directed,weights,n_b", [(True, 3, 128), (True, None, 64), (False, 2, 256)])
def test_hash_accumulator_with_more_hot_keys_than_slots(directed, weights, n_b):
    g = _many_hubs(directed, weights, seed=11 + n_b)
    srcs = np.random.default_rng(3).choice(g.n, 400, replace=False).astype(np.int32)
    G = mfbc.Graph.from_csr(g)
    want = oracle.bc(g, srcs)
    close(G.bc(srcs, n_b=n_b, path=mfbc.PATH_GENERAL, accumulator=mfbc.ACCUM_HASH), want)
    wd, ws, _ = oracle.sssp(g, srcs[:96])
    d, s = G.sssp(srcs[:96], n_b=n_b, path=mfbc.PATH_GENERAL, accumulator=mfbc.ACCUM_HASH)
    assert np.array_equal(d, wd) and np.array_equal(s, ws)
    # the same per-product work on the atomic path: identical tau and sigma_bar
    d2, s2 = G.sssp(srcs[:96], n_b=n_b, path=mfbc.PATH_GENERAL, accumulator=mfbc.ACCUM_ATOMIC)
    assert np.array_equal(d, d2) and np.array_equal(s, s2)
    G.close()
