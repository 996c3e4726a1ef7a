"""Both input orientations of mfbc_graph_create give the same graph.

The arrays may hold the rows of A (MFBC_CSR, Sec. 2.1) or of A^T (MFBC_CSC:
row v lists the tails of the arcs into v, the operand of Algorithm 2's
products, Sec. 4.2).  A graph built from each, through the C ABI, must give
bit-identical tau and sigma_bar on every kernel family, lambda equal up to the
order of floating-point atomic sums (1e-12 relative), and match the oracle.
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


def transpose(g):
    """Rows of A^T from the rows of A (numpy, stable: rows stay sorted)."""
    src = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(g.rowptr))
    order = np.lexsort((src, g.col))
    rp = np.zeros(g.n + 1, np.int64)
    np.cumsum(np.bincount(g.col, minlength=g.n), out=rp[1:])
    return rp, src[order], None if g.w is None else g.w[order]


@pytest.mark.parametrize("kind", ["directed_weighted", "directed_unit", "undirected"])
def test_csc_and_csr_inputs_agree(kind):
    import torch
    if kind == "directed_weighted":
        g = gg.rmat(12, 8, directed=True, weights=(1, 9), seed=21)
    elif kind == "directed_unit":
        g = gg.rmat(12, 8, directed=True, seed=22)
    else:
        g = gg.rmat(12, 8, seed=23)
    srcs = gg.sample_sources(g, 300, seed=4)
    rpt, colt, wt = transpose(g)
    A = mfbc.Graph.from_csr(g)
    At = mfbc.Graph(rpt, colt, wt, directed=g.directed, csc=True)
    At_dev = mfbc.Graph(torch.from_numpy(rpt).cuda(), torch.from_numpy(colt).cuda(),
                        None if wt is None else torch.from_numpy(wt).cuda(), directed=g.directed, csc=True)
    want = oracle.bc(g, srcs)
    wd, ws, _ = oracle.sssp(g, srcs[:40])
    paths = [mfbc.PATH_GENERAL, mfbc.PATH_DIST] + ([] if g.w is not None else [mfbc.PATH_LEVEL])
    for p in paths:
        la = A.bc(srcs, n_b=128, path=p)
        for H in (At, At_dev):
            lb = H.bc(srcs, n_b=128, path=p)
            nz = la != 0
            assert np.array_equal(la[~nz], lb[~nz]), f"exact zeros differ between orientations (path {p})"
            assert np.max(np.abs(la[nz] - lb[nz]) / la[nz]) <= 1e-12, f"lambda differs (path {p})"
            d, s = H.sssp(srcs[:40], n_b=64, path=p)
            assert np.array_equal(d, wd) and np.array_equal(s, ws)
        nz = want != 0
        assert np.array_equal(la[~nz], want[~nz])
        assert np.max(np.abs(la[nz] - want[nz]) / want[nz]) <= 1e-9
    for G in (A, At, At_dev):
        G.close()


def test_csc_input_is_validated_as_rows():
    bad = [
        (3, [0, 2, 3, 4], [2, 1, 0, 0]),     # unsorted row of A^T
        (3, [0, 2, 3, 4], [1, 1, 0, 0]),     # duplicate arc
        (3, [0, 1, 2, 3], [1, 5, 0]),        # tail out of range
        (3, [0, 1, 2, 3], [0, 2, 0]),        # self-loop (found on A)
    ]
    for n, rp, col in bad:
        with pytest.raises(mfbc.MFBCError) as e:
            mfbc.Graph(np.array(rp), np.array(col), None, directed=True, csc=True)
        assert e.value.status == mfbc.MFBC_ERR_INVALID
