"""Host-side helpers of bench.py (no GPU): the gating of the stored DRAM
traffic figure on the kernel source, the whole-step traffic model of the
unweighted path, the L2 note of a run's config, the bench workloads' shapes
and the bounded CPU-oracle baseline."""
import hashlib
import os

import numpy as np
import pytest

import bench
import graphgen as gg


def test_traffic_figure_is_gated_on_the_kernel_source(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel v1\n")
    sha = hashlib.sha1(src.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC", {("w", "k"): {"per_alg_byte": 1.5, "sha1": sha, "source": "kernel.cu"}})
    assert bench.traffic_per_launch("w", "k", 10.0) == pytest.approx(15.0)
    assert bench.traffic_per_launch("w", "other", 10.0) is None
    assert bench.traffic_per_launch("other", "k", 10.0) is None
    src.write_text("// kernel v2\n")                      # changed since the capture
    assert bench.traffic_per_launch("w", "k", 10.0) is None


def test_committed_traffic_entries_name_existing_sources():
    for (workload, kernel), t in bench.TRAFFIC.items():
        assert workload in bench.WORKLOADS
        assert os.path.exists(os.path.join(bench.ROOT, t["source"]))
        assert t["per_alg_byte"] >= 1.0                 # DRAM traffic cannot undercut the compulsory bytes


def test_product_byte_model_terms_on_a_small_graph():
    # two components: a path 0-1-2-3 and an edge 4-5
    g = gg.from_edges(6, [(0, 1), (1, 2), (2, 3), (4, 5)], directed=False)
    srcs = np.array([0, 4], np.int32)
    prof = {"values_bwd": 7}
    m = bench.product_byte_model(g, srcs, prof, step_s=1.0, peak_gbs=1.0)
    R = 4 + 2                                            # reachable pairs, sources included
    F = 6 + 2                                            # arcs in each source's component
    D = 7
    G = 2 * R
    total = (12 * R + 4 * F + 16 * D + 24 * G) + (4 * R + 4 * g.nnz + 4 * F + 8 * D) + (12 * R + 4 * F + 24 * D) \
        + (16 * R + 16 * g.n)
    assert m["reachable_pairs"] == R and m["arc_visits"] == F and m["tight_arcs"] == D
    assert m["bytes_per_step"] == pytest.approx(total)
    assert m["bytes_per_tep"] == pytest.approx(total / (len(srcs) * g.m))
    assert m["measured_over_model"] == pytest.approx(total / 1e9)
    w = gg.from_edges(3, [(0, 1), (1, 2)], directed=False, weights=[1, 2])
    assert bench.product_byte_model(w, srcs[:1], prof, 1.0, 1.0) is None


def test_l2_note_follows_the_state_size():
    assert bench.l2_note(1 << 22, 1024).startswith("state much larger than L2")
    assert "may stay in L2" in bench.l2_note(1 << 16, 64)
    # the general kernels keep 32 bytes per pair: R-MAT 16 at n_b = 512 is 1 GiB
    assert bench.l2_note(1 << 16, 512, path=1).startswith("state much larger than L2")
    assert "may stay in L2" in bench.l2_note(1 << 16, 512)


def test_grid_workload_shape():
    g, srcs = bench.make_workload("grid256w")
    assert g.n == 256 * 256 and not g.directed
    assert g.w is not None and g.w.min() >= 1 and g.w.max() <= 16
    assert len(srcs) == 4096 and len(np.unique(srcs)) == 4096


def test_cpu_baseline_is_bounded_and_states_its_sample():
    g = gg.erdos_renyi(512, 8, seed=1)
    srcs = gg.sample_sources(g, 64, seed=2)
    r = bench.cpu_baseline(g, srcs, budget_s=0.5)
    assert r["kind"] == "oracle" and r["cores"] >= 1 and r["value"] > 0
    assert "of the 64 sources" in r["sample"]
