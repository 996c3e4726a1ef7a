"""Input generators: determinism and the structural rules every workload obeys."""
import numpy as np
import pytest

import graphgen as gg


def _check_csr(g):
    assert g.rowptr[0] == 0 and np.all(np.diff(g.rowptr) >= 0)
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    assert np.all((g.col >= 0) & (g.col < g.n))
    assert not np.any(src == g.col), "self-loop"
    key = src.astype(np.int64) * g.n + g.col
    assert np.all(np.diff(key) > 0), "rows must be sorted without duplicates"
    if g.w is not None:
        assert g.w.min() >= 1
    if not g.directed:
        rev = g.col.astype(np.int64) * g.n + src
        order = np.argsort(rev)
        assert np.array_equal(rev[order], key)
        if g.w is not None:
            assert np.array_equal(g.w[order], g.w)


@pytest.mark.parametrize("make", [
    lambda: gg.rmat(12, 16, seed=1),
    lambda: gg.rmat(12, 16, directed=True, weights=(1, 255), seed=1),
    lambda: gg.erdos_renyi(2000, 8, seed=1),
    lambda: gg.erdos_renyi(500, 20, directed=True, weights=(1, 100), seed=3),
    lambda: gg.grid2d(17, weights=(1, 16)),
])
def test_structure_and_determinism(make):
    g1, g2 = make(), make()
    _check_csr(g1)
    assert np.array_equal(g1.rowptr, g2.rowptr) and np.array_equal(g1.col, g2.col)
    if g1.w is not None:
        assert np.array_equal(g1.w, g2.w)


def test_thread_count_does_not_change_rmat():
    a = gg.rmat(11, 8, seed=5, nthreads=1)
    b = gg.rmat(11, 8, seed=5, nthreads=7)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.rowptr, b.rowptr)


def test_er_mean_degree():
    g = gg.erdos_renyi(1 << 14, 32, seed=1)
    assert abs(g.nnz / g.n - 32) < 0.5


def test_rmat_skew_and_weight_range():
    g = gg.rmat(14, 16, directed=True, weights=(1, 255), seed=1)
    d = g.out_degree()
    assert d.max() > 50 * d.mean()
    assert g.w.min() == 1 and g.w.max() == 255


def test_sample_sources():
    g = gg.rmat(10, 4, seed=2)
    s = gg.sample_sources(g, 100, seed=2)
    assert len(np.unique(s)) == 100
    assert np.all(g.out_degree()[s] > 0)
    assert np.array_equal(s, gg.sample_sources(g, 100, seed=2))
    with pytest.raises(ValueError):
        gg.sample_sources(g, g.n + 1)


def test_grid_is_four_neighbour_with_the_weight_range():
    L = 20
    g = gg.grid2d(L, weights=(1, 16), seed=1)
    assert g.n == L * L and g.nnz == 2 * 2 * L * (L - 1)          # 2L(L-1) edges, both arcs
    deg = g.out_degree()
    assert deg.min() == 2 and deg.max() == 4 and np.sum(deg == 2) == 4
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    dx = np.abs(src % L - g.col % L)
    dy = np.abs(src // L - g.col // L)
    assert np.all(dx + dy == 1)                                      # only lattice neighbours
    assert g.w.min() == 1 and g.w.max() == 16
    assert len(np.unique(g.w)) == 16                                 # every weight occurs


def test_dense_er_degree_spread_suits_the_distance_kernels():
    # the automatic choice takes the distance kernels when no degree exceeds
    # max(64, 4x the average): true of uniform random graphs, false of R-MAT
    er = gg.erdos_renyi(1 << 12, 256, weights=(1, 100), seed=1)
    assert er.out_degree().max() <= 4 * er.nnz / er.n
    rm = gg.rmat(12, 16, directed=True, weights=(1, 255), seed=1)
    assert rm.out_degree().max() > max(64, 4 * rm.nnz / rm.n)
