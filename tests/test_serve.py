"""Host logic of the serving loop, without a GPU: a fake executor adds each
batch part's oracle lambda into its request's pool row, so batching,
admission and the latency bookkeeping are checked on their own."""
import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1609_07008_gb300.serve import Request, Server, align32, latency_stats, make_requests, run_served


def _graphs():
    return {"a": gg.rmat(8, 8, seed=1), "b": gg.erdos_renyi(300, 5, seed=2)}


class Recorder:
    """Executor stand-in: oracle lambda per request, optional delay, and a
    record of the bytes held while each group ran."""

    def __init__(self, graphs, server_ref, delay=0.0):
        self.graphs, self.server_ref, self.delay = graphs, server_ref, delay
        self.held_seen = []
        self.lock = threading.Lock()

    def __call__(self, key, parts, nb, pool, rows, stream, handle):
        with self.lock:
            self.held_seen.append(self.server_ref[0]._held)
        assert sum(align32(k) for _, _, k in parts) <= nb
        if self.delay:
            time.sleep(self.delay)
        for (r, a, k), row in zip(parts, rows):
            if k:
                pool[row] += oracle.bc(self.graphs[key], r.sources[a:a + k], nthreads=1)


def test_groups_respect_columns_and_results_match_the_oracle():
    graphs = _graphs()
    ref = []
    rec = Recorder(graphs, ref)
    srv = Server(graphs, budget_bytes=1 << 40, max_cols=256, executor=rec,
                 sizer=lambda k, nb, slots: nb * 100)
    ref.append(srv)
    reqs = make_requests({k: g.n for k, g in graphs.items()}, 40, rate=0, lo=5, hi=200, seed=3)
    srv.start()
    run_served(srv, reqs, timeout=120)
    srv.close()
    for r in reqs:
        np.testing.assert_allclose(r.result, oracle.bc(graphs[r.graph], r.sources), rtol=1e-12, atol=0)
        assert r.arrival <= r.start <= r.done
    # every batch fits its columns (requests larger than a batch are split)
    for g in srv.log:
        assert g.cols <= 256
    # all requests arrived at once: several share a batch (continuous batching)
    assert max(g.nreq for g in srv.log) > 1
    assert sum(g.new for g in srv.log) == len(reqs)
    st = srv.stats()
    assert st["batches"] == len(srv.log) and st["batches_with_several_requests"] > 0


def test_admission_never_exceeds_the_budget():
    graphs = _graphs()
    ref = []
    rec = Recorder(graphs, ref, delay=0.02)
    # a worker holds 1000 bytes per column; the budget lets one worker of
    # 1024 columns run, so the two graphs' workers must take turns
    srv = Server(graphs, budget_bytes=1024 * 1000, max_cols=1024, executor=rec,
                 sizer=lambda k, nb, slots: nb * 1000)
    ref.append(srv)
    reqs = make_requests({k: g.n for k, g in graphs.items()}, 30, rate=0, lo=200, hi=300, seed=4)
    srv.start()
    run_served(srv, reqs, timeout=120)
    srv.close()
    for g in srv.log:
        assert g.bytes <= 1024 * 1000
    assert max(rec.held_seen) <= 1024 * 1000
    # the groups of the two graphs never overlap in time
    spans = sorted((g.t0, g.t1) for g in srv.log)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1 - 1e-9


def test_groups_run_concurrently_when_the_budget_allows():
    graphs = _graphs()
    ref = []
    rec = Recorder(graphs, ref, delay=0.05)
    srv = Server(graphs, budget_bytes=1 << 40, max_cols=64, executor=rec,
                 sizer=lambda k, nb, slots: nb)
    ref.append(srv)
    reqs = [Request(i, "a" if i % 2 else "b", np.arange(10, dtype=np.int32), 0.0) for i in range(8)]
    srv.start()
    run_served(srv, reqs, timeout=60)
    srv.close()
    spans = [(g.t0, g.t1, g.graph) for g in srv.log]
    overlap = any(a[2] != b[2] and a[0] < b[1] and b[0] < a[1] for a in spans for b in spans)
    assert overlap


def test_oversize_worker_lowers_n_b_until_it_fits():
    graphs = _graphs()
    seen = []

    def sizer(k, nb, slots):
        return nb * 10

    def ex(key, parts, nb, pool, rows, stream, handle):
        seen.append(nb)

    srv = Server(graphs, budget_bytes=300 * 10, max_cols=4096, n_b=0, executor=ex, sizer=sizer)
    srv.start()
    run_served(srv, [Request(0, "a", np.arange(50, dtype=np.int32), 0.0)], timeout=30)
    srv.close()
    assert seen == [256]


def test_executor_errors_reach_the_caller():
    graphs = _graphs()

    def ex(*a):
        raise RuntimeError("device lost")

    srv = Server(graphs, budget_bytes=1 << 30, executor=ex, sizer=lambda *a: 1)
    srv.start()
    with pytest.raises(RuntimeError, match="device lost"):
        run_served(srv, [Request(0, "a", np.arange(3, dtype=np.int32), 0.0)], timeout=30)
    srv.close()


def test_make_requests_shapes_and_latency_stats():
    sizes = {"x": 5000, "y": 100}
    reqs = make_requests(sizes, 200, rate=50.0, lo=64, hi=4096, seed=7)
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) >= 0) and arr[-1] > 0
    for r in reqs:
        assert 1 <= len(r.sources) <= min(4096, sizes[r.graph])
        assert len(np.unique(r.sources)) == len(r.sources)
        assert r.sources.min() >= 0 and r.sources.max() < sizes[r.graph]
    # mean inter-arrival close to 1/rate
    assert 0.01 < np.diff(arr).mean() < 0.04
    for i, r in enumerate(reqs):
        r.start, r.done = r.arrival, r.arrival + 0.001 * (i % 10 + 1)
    st = latency_stats(reqs, {"x": 10, "y": 10})
    assert st["requests"] == 200 and st["p50_ms"] <= st["p99_ms"] <= 10.0 + 1e-9
    assert align32(1) == 32 and align32(64) == 64 and align32(65) == 96


def test_replica_handles_let_groups_of_one_graph_overlap():
    graphs = _graphs()
    ref = []
    rec = Recorder(graphs, ref, delay=0.05)
    srv = Server(graphs, budget_bytes=1 << 40, max_cols=32, executor=rec, sizer=lambda k, nb, slots: nb,
                 replicas={"a": [object(), object()]})
    ref.append(srv)
    assert len(srv._threads) == 4                   # three workers for "a", one for "b"
    reqs = [Request(i, "a", np.arange(20, dtype=np.int32), 0.0) for i in range(6)]
    srv.start()
    run_served(srv, reqs, timeout=60)
    srv.close()
    spans = [(g.t0, g.t1) for g in srv.log]
    assert any(a[0] < b[1] and b[0] < a[1] for i, a in enumerate(spans) for b in spans[i + 1:])
    for r in reqs:
        np.testing.assert_allclose(r.result, oracle.bc(graphs["a"], r.sources), rtol=1e-12, atol=0)


def test_request_arriving_during_a_batch_joins_the_next_one():
    # one worker, 256-column batches: a 1000-source request needs four; a
    # small request arriving while the first runs is admitted into the
    # second and answered long before the large one
    graphs = {"a": gg.rmat(9, 8, seed=5)}
    ref = []
    rec = Recorder(graphs, ref, delay=0.1)
    srv = Server(graphs, budget_bytes=1 << 40, max_cols=256, executor=rec, sizer=lambda k, nb, slots: nb)
    ref.append(srv)
    big = Request(0, "a", gg.sample_sources(graphs["a"], 300, seed=1).repeat(4)[:1000].astype(np.int32), 0.0)
    small = Request(1, "a", np.arange(40, dtype=np.int32), 0.05)
    srv.start()
    run_served(srv, [big, small], timeout=60)
    srv.close()
    assert len(srv.log) == 5                         # 4 batches of the big one; the small shares the 2nd
    assert small.group == 1 and srv.log[1].nreq == 2 and srv.log[1].new == 1
    assert small.done < big.done
    for r in (big, small):
        np.testing.assert_allclose(r.result, oracle.bc(graphs["a"], r.sources), rtol=1e-12, atol=0)


def test_a_graph_no_width_fits_is_reported():
    graphs = _graphs()

    def sizer(k, nb, slots):
        raise ValueError("wider than the library takes")

    srv = Server(graphs, budget_bytes=1 << 30, executor=lambda *a: None, sizer=sizer)
    srv.start()
    with pytest.raises(ValueError, match="no batch width fits"):
        run_served(srv, [Request(0, "a", np.arange(3, dtype=np.int32), 0.0)], timeout=30)
    srv.close()
