"""Benchmark: betweenness centrality GTEPS of MFBC on one GB300 (or N, one process per GPU).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mfbc|reference] [--workload rmat22]

One step = one whole MFBC pass (Algorithm 3: every batch of MFBF + MFBr +
lambda accumulation) over the workload's full source list on the
device-resident graph.  Default workload: unweighted undirected R-MAT scale 22
(edge factor 16, a,b,c,d = .57,.19,.19,.05, seeded relabelling), 16384 sources
sampled among vertices of degree >= 1.  GTEPS = sources * m / seconds with m
the number of undirected edges.

Printed JSON line (rank 0):
  value       device-resident throughput over K timed steps (CUDA events on the
              launching stream, barrier + synchronize on both sides, max over ranks);
  e2e         the same metric through the C ABI with HOST buffers: graph upload
              and construction (mfbc_graph_create from pinned host CSR),
              mfbc_bc with host sources, lambda copied back to the host;
  roofline    the dominant kernel's algorithmic bytes per launch (device-counted
              in an untimed pass) over its average launch time (CUDA events
              recorded by the library on the launching stream during the timed
              steps), against the measured HBM copy bandwidth;
  cpu_baseline  the CPU oracle (plain C Brandes) on a bounded sample of the
              same workload on all host cores, rank 0 only.
  workloads   the other benchmark configurations (Erdos-Renyi n=1024 all
              sources; weighted directed R-MAT 16; Erdos-Renyi n=2^20 k=32;
              dense weighted Erdos-Renyi n=2^16 k=1024 on its first 4096
              sources), one short measurement each with its own roofline
              and oracle baseline (all cores and one thread).
Multi-GPU (torchrun): each rank runs its own sample of sources (weak scaling),
or with --shard one contiguous part of the same list (strong scaling); lambda
is summed across ranks with one all-reduce per step.
The headline state (n x n_b x 8 bytes and more) is far larger than the 129 MB
L2, so no explicit L2 flush is done between its steps; configurations whose
state could stay in L2 are timed step by step with an L2-sized buffer
overwritten between steps.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "rmat22": dict(kind="rmat", scale=22, ef=16, nsrc=16384,
                   desc="R-MAT scale 22, edge factor 16, undirected, unweighted, 16384 sampled sources"),
    "er1024": dict(kind="er1024", nsrc=1024,
                   desc="Erdos-Renyi n=1024, k=8, undirected, unweighted, all 1024 sources, n_b=128"),
    "rmat20": dict(kind="rmat", scale=20, ef=16, nsrc=4096,
                   desc="R-MAT scale 20, edge factor 16, undirected, unweighted, 4096 sampled sources (profiling size)"),
    "er20k32": dict(kind="er", n=1 << 20, k=32, nsrc=16384,
                    desc="Erdos-Renyi n=2^20, k=32, undirected, unweighted, 16384 sampled sources"),
    "rmat16w": dict(kind="rmat16w", nsrc=4096,
                    desc="R-MAT scale 16, edge factor 16, directed, weights U[1,255], 4096 sources, n_b=512"),
    "er16k1024w": dict(kind="er16k1024w", nsrc=1 << 16,
                       desc="Erdos-Renyi n=2^16, k=1024, undirected, weights U[1,100], all 65536 sources"),
    "grid256w": dict(kind="grid", L=256, nsrc=4096,
                     desc="2D grid 256^2, 4-neighbour, undirected, weights U[1,16], 4096 sampled sources"),
}


def make_workload(name, rank=0):
    import graphgen as gg
    w = WORKLOADS[name]
    if w["kind"] == "rmat":
        g = gg.rmat(w["scale"], w["ef"], seed=1)
    elif w["kind"] == "er":
        g = gg.erdos_renyi(w["n"], w["k"], seed=1)
    elif w["kind"] == "er1024":
        g = gg.erdos_renyi(1024, 8, seed=1)
        return g, np.arange(g.n, dtype=np.int32)          # all-source exact BC
    elif w["kind"] == "er16k1024w":
        g = gg.erdos_renyi(1 << 16, 1024, weights=(1, 100), seed=1)
        return g, np.arange(g.n, dtype=np.int32)          # all-source exact BC
    elif w["kind"] == "grid":
        g = gg.grid2d(w["L"], weights=(1, 16), seed=1)
    else:
        g = gg.rmat(16, 16, directed=True, weights=(1, 255), seed=1)
    srcs = gg.sample_sources(g, w["nsrc"], seed=2 + rank)
    return g, srcs


# DRAM traffic of the dominant kernel: dram__bytes_read.sum + dram__bytes_write.sum
# per launch from one ncu capture of the timed gathers on the first 2048 sources of
# the same workload (two batches of the same width), expressed per
# algorithmic byte so that it scales with the launches this run makes.  Each entry
# records the SHA-1 of the kernel source it was taken on; once that source changes
# the figure is reported as null.
TRAFFIC = {
    ("rmat22", "level_mfbr_gather"): {"per_alg_byte": 61.808 / 39.2486, "sha1": "d5dd8751004112c8e375901701fa3fe389f416bd",
                                      "source": "paper_1609_07008_gb300/csrc/level.cu"},
    ("rmat22", "level_mfbf_gather"): {"per_alg_byte": 25.330 / 24.839, "sha1": "d5dd8751004112c8e375901701fa3fe389f416bd",
                                      "source": "paper_1609_07008_gb300/csrc/level.cu"},
}


def traffic_per_launch(workload, kernel, alg_bytes):
    import hashlib
    t = TRAFFIC.get((workload, kernel))
    if not t:
        return None
    with open(os.path.join(ROOT, t["source"]), "rb") as f:
        if hashlib.sha1(f.read()).hexdigest() != t["sha1"]:
            return None
    return t["per_alg_byte"] * alg_bytes


def product_byte_model(g, srcs, prof_bytes, step_s, peak_gbs):
    """A per-TEP byte model of the paper's products for MFBF + counters + MFBr + lambda
    (unweighted graphs, 4-byte arcs).  It is an algorithmic-byte model of the
    paper's products with stored distances and counters, not a ceiling of the
    level kernels: those replace the 4-byte distance check per arc visit by
    frontier bit rows shared by 32 columns per word and keep no counters, so
    a run can exceed the model's rate (`measured_over_model` > 1).  Per step
      B_fwd = 12 R + 4 F + 16 D + 24 G,  B_cnt = 4 R + 4 nnz + 4 F + 8 D,
      B_bwd = 12 R + 4 F + 24 D,         B_acc = 16 R + 16 n,
    with R reachable (source, vertex) pairs, F arc visits from reachable pairs
    (sum over sources of the arcs in the source's component), D tight-arc hits
    (the values the MFBr gathers read, counted on the device) and G the entries touched
    by the products, taken as 2 R (it lies between R and 3 R).  The frontier-row
    terms (a few bytes per vertex and level) are left out.  Returns None for
    weighted or directed workloads."""
    if g.w is not None or g.directed:
        return None
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    a = sp.csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col, g.rowptr), shape=(g.n, g.n))
    _, lab = connected_components(a, directed=False)
    size = np.bincount(lab).astype(np.float64)
    arcs = np.bincount(lab, weights=np.diff(g.rowptr).astype(np.float64))
    R = float(size[lab[srcs]].sum())
    F = float(arcs[lab[srcs]].sum())
    D = float(prof_bytes["values_bwd"])
    G = 2.0 * R
    total = (12 * R + 4 * F + 16 * D + 24 * G) + (4 * R + 4 * g.nnz + 4 * F + 8 * D) + (12 * R + 4 * F + 24 * D) \
        + (16 * R + 16 * g.n)
    teps = len(srcs) * g.m
    at_peak = peak_gbs * 1e9 / (total / teps) / 1e9
    return {"bytes_per_step": total, "bytes_per_tep": total / teps, "gteps_if_model_bytes_at_peak": at_peak,
            "measured_over_model": (total / (peak_gbs * 1e9)) / step_s, "reachable_pairs": R, "arc_visits": F,
            "tight_arcs": D}


# The serving pool of the request-loop configuration: R-MAT scales 10-20 (edge
# factor 16, undirected, unweighted), Erdos-Renyi n = 2^14..2^20 (k = 16,
# undirected, unweighted), weighted 2D grids 256^2..2048^2 (w U[1,16]).
SERVE_FULL = ["rmat10", "rmat12", "rmat14", "rmat16", "rmat18", "rmat20", "er14", "er16", "er18", "er20",
              "grid256w", "grid512w", "grid1024w", "grid2048w"]
# the default bench line's pool: the same families up to about 2^18 vertices
SERVE_DEFAULT = ["rmat10", "rmat12", "rmat14", "rmat16", "rmat18", "er14", "er16", "er18", "grid256w", "grid512w"]


def serve_graph(name):
    import graphgen as gg
    if name.startswith("rmat"):
        return gg.rmat(int(name[4:]), 16, seed=1)
    if name.startswith("er"):
        return gg.erdos_renyi(1 << int(name[2:]), 16, seed=1)
    return gg.grid2d(int(name[4:-1]), weights=(1, 16), seed=1)


def serving_bench(pool=SERVE_DEFAULT, n_requests=300, seed=5, loads=(0.5, 0.8, 1.2)):
    """Served (continuous batching at batch granularity, memory-budget
    admission, several workers and CUDA streams per graph) against plain (one
    mfbc_bc_device call per request, in arrival order) on the same requests:
    saturated (every request at t = 0: capacity), then Poisson arrivals at
    each offered load (a multiple of the plain form's capacity): p50/p99
    latency, throughput, the batches' packing, and the largest relative
    difference between the two forms' lambdas (equal accuracy).  A request
    picks graph g with probability proportional to 1/sqrt(n_g) (small graphs
    are asked more often) and log-uniform [64, 4096] sources (at most the
    graph's vertices of degree >= 1)."""
    import torch
    import paper_1609_07008_gb300 as mfbc
    from paper_1609_07008_gb300 import serve
    host = {k: serve_graph(k) for k in pool}
    graphs = {k: mfbc.Graph.from_csr(g) for k, g in host.items()}
    # three more workers (handles, streams) per graph up to 2^18 vertices, one more above
    replicas = {k: [mfbc.Graph.from_csr(g) for _ in range(3 if g.n <= (1 << 18) else 1)] for k, g in host.items()}
    edges = {k: g.m for k, g in host.items()}
    elig = {k: np.flatnonzero(g.out_degree() > 0).astype(np.int32) for k, g in host.items()}
    sizes = {k: g.n for k, g in host.items()}
    weights = {k: 1.0 / np.sqrt(g.n) for k, g in host.items()}
    # batch width per graph: the level kernels take at most 1024 columns; the
    # distance kernels (weighted grids) pay per distance step whatever the
    # width, so their batches are as wide as a request gets
    max_cols = {k: 4096 if g.w is not None else 1024 for k, g in host.items()}
    handles = list(graphs.values()) + [R for rs_ in replicas.values() for R in rs_]
    budget = 0

    def release():
        # the plain form's calls leave scratch cached on the handles, the
        # server's workers their tensors in torch's cache: give both back
        for G in handles:
            G.release_scratch()
        torch.cuda.empty_cache()

    def reqs(rate, count=n_requests, lo=64, hi=4096, sd=seed):
        return serve.make_requests(sizes, count, rate, lo=lo, hi=hi, seed=sd, eligible=elig, weights=weights)

    def served(rs):
        nonlocal budget
        release()
        free, _ = torch.cuda.mem_get_info()
        budget = int(0.7 * free)
        srv = serve.Server(graphs, budget_bytes=budget, max_cols=max_cols, replicas=replicas).start()
        try:
            serve.run_served(srv, rs, timeout=3600)
        finally:
            srv.close()
        return dict(serve.latency_stats(rs, edges), **srv.stats())

    def diff(a_list, b_list):
        d = 0.0
        for a, b in zip(sorted(a_list, key=lambda r: r.rid), sorted(b_list, key=lambda r: r.rid)):
            nz = b.result != 0
            if np.any(a.result[~nz] != 0):
                return float("inf")
            if nz.any():
                d = max(d, float(np.max(np.abs(a.result[nz] - b.result[nz]) / np.abs(b.result[nz]))))
        return d

    # warm both forms once (library scratch, torch allocator, module load)
    serve.run_plain(graphs, reqs(0, count=2 * len(pool), hi=256, sd=seed + 1))
    served(reqs(0, count=2 * len(pool), hi=256, sd=seed + 1))
    release()
    sat_plain_reqs = serve.run_plain(graphs, reqs(0))
    sat_plain = serve.latency_stats(sat_plain_reqs, edges)
    sat_served_reqs = reqs(0)
    sat_served = served(sat_served_reqs)
    worst = diff(sat_plain_reqs, sat_served_reqs)
    cap = n_requests / sat_plain["span_s"]
    rows = []
    for load in loads:
        release()
        rp = serve.run_plain(graphs, reqs(load * cap))
        rs = reqs(load * cap)
        row = {"offered_load_vs_plain_capacity": load, "rate_per_s": load * cap,
               "plain": serve.latency_stats(rp, edges), "served": served(rs)}
        worst = max(worst, diff(rp, rs))
        rows.append(row)
    for G in handles:
        G.close()
    return {"pool": {k: {"n": host[k].n, "m": int(host[k].m), "weighted": host[k].w is not None} for k in pool},
            "graph_choice": "probability proportional to 1/sqrt(n)", "sources_per_request": "log-uniform [64, 4096]",
            "requests": n_requests, "workers_per_graph": {k: 1 + len(v) for k, v in replicas.items()},
            "batch_columns": max_cols, "budget_bytes": budget,
            "saturated": {"plain_gteps": sat_plain["gteps"], "served_gteps": sat_served["gteps"],
                          "plain_span_s": sat_plain["span_s"], "served_span_s": sat_served["span_s"],
                          "served_packing": {k: sat_served[k] for k in sat_served if k.startswith(("batches",
                                                                                                     "requests_per",
                                                                                                     "columns"))}},
            "plain_capacity_per_s": cap, "loads": rows, "max_rel_diff": worst}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mfbc_clocks_{os.getpid()}_{device_index}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(g, srcs, budget_s=15.0, single_budget_s=5.0):
    """The oracle as it stands on a bounded sample of sources: on all host
    cores (the line's value) and on one thread (single_thread)."""
    import oracle
    nth = oracle.default_threads()
    k = max(nth, 1)
    t0 = time.perf_counter()
    oracle.bc(g, srcs[:k], nthreads=nth)
    dt = time.perf_counter() - t0
    per_src = dt / k
    k2 = int(min(len(srcs), max(k, (budget_s / max(per_src, 1e-6)) // nth * nth)))
    if k2 > k:
        t0 = time.perf_counter()
        oracle.bc(g, srcs[:k2], nthreads=nth)
        dt = time.perf_counter() - t0
        k = k2
    out = {"value": k * g.m / dt / 1e9, "unit": "GTEPS", "cores": nth, "kind": "oracle",
           "sample": f"first {k} of the {len(srcs)} sources, {dt:.1f} s"}
    t0 = time.perf_counter()
    oracle.bc(g, srcs[:1], nthreads=1)
    d1 = time.perf_counter() - t0
    k1 = int(min(len(srcs), max(1, single_budget_s / max(d1, 1e-6))))
    if k1 > 1:
        t0 = time.perf_counter()
        oracle.bc(g, srcs[:k1], nthreads=1)
        d1 = time.perf_counter() - t0
    out["single_thread"] = {"value": k1 * g.m / d1 / 1e9, "unit": "GTEPS", "cores": 1,
                            "sample": f"first {k1} of the {len(srcs)} sources, {d1:.1f} s"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    g, srcs = make_workload(args.workload)
    import oracle
    nth = oracle.default_threads()
    per_step = max(nth, args.ref_sources)
    for _ in range(args.warmup):
        oracle.bc(g, srcs[:nth], nthreads=nth)
    t0 = time.perf_counter()
    for i in range(args.steps):
        sl = srcs[(i * per_step) % len(srcs):][:per_step]
        oracle.bc(g, sl, nthreads=nth)
    dt = time.perf_counter() - t0
    val = args.steps * per_step * g.m / dt / 1e9
    line = {"impl": "reference", "metric": "BC GTEPS", "value": val, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "strong" if args.shard else "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config_of(args, g, len(srcs), None),
            "cpu_baseline": {"value": val, "unit": "GTEPS", "cores": nth, "kind": "oracle",
                             "sample": f"{per_step} sources per step of the {len(srcs)}-source workload"},
            "e2e": {"value": val, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


L2_BYTES = 129 << 20


STATE_BYTES_PER_PAIR = {1: 32, 2: 8, 3: 20}   # general, level, distance kernels


def l2_note(n, n_b, path=None):
    """How the timed steps relate to the L2: the kernel family's state per
    (source, vertex) pair (the smallest, 8 bytes, when the family is not
    known) times n * n_b, against the L2 size."""
    state = STATE_BYTES_PER_PAIR.get(path, 8) * int(n) * int(n_b or 0)
    if state > 2 * L2_BYTES:
        return "state much larger than L2 (no flush)"
    return f"state of {state / 2**20:.0f} MB may stay in L2 (no flush: a probe, not a bench line)"


def needs_flush(n, n_b, path):
    return STATE_BYTES_PER_PAIR.get(path, 8) * int(n) * int(n_b or 0) <= 2 * L2_BYTES


def config_of(args, g, nsrc, n_b, path=None):
    par = f"one source list sharded x{args.gpus}" if args.shard else f"sources sampled per rank x{args.gpus}"
    return {"workload": WORKLOADS[args.workload]["desc"], "name": args.workload, "n": g.n, "nnz": g.nnz,
            "m": g.m, "sources": nsrc, "n_b": n_b, "parallelism": par,
            "l2": l2_note(g.n, n_b if n_b else min(nsrc, 1024), path)}   # the reference arm has no n_b


DTYPE = {1: "f64 (sigma, zeta, lambda)", 2: "u64 sigma / fp32x2 zeta / f64 lambda", 3: "f64 (sigma, zeta, lambda)"}


def roofline_of(kstats, prof_bytes, peak, peak_kind, workload, step_s):
    """Dominant kernel's algorithmic bytes per launch over its mean launch time,
    plus the whole step: every kernel's device-counted bytes over the step time."""
    dom = max(kstats.items(), key=lambda kv: kv[1]["ms"])[0]
    kb = prof_bytes["kernels"].get(dom, {})
    per_launch_bytes = kb.get("bytes", 0.0) / max(kb.get("launches", 1), 1)
    avg_ms = kstats[dom]["ms"] / kstats[dom]["launches"]
    achieved = per_launch_bytes / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else 0.0
    step_bytes = sum(v.get("bytes", 0.0) for v in prof_bytes["kernels"].values())
    traffic = {}
    for k, v in prof_bytes["kernels"].items():
        t = traffic_per_launch(workload, k, v.get("bytes", 0.0) / max(v.get("launches", 1), 1))
        if t is not None:
            traffic[k] = t
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
            "peak_kind": f"{peak_kind} copy bandwidth", "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic.get(dom), "bytes_per_launch": per_launch_bytes, "avg_launch_ms": avg_ms,
            "kernel_bytes_per_launch": {k: v.get("bytes", 0.0) / max(v.get("launches", 1), 1)
                                        for k, v in prof_bytes["kernels"].items() if v.get("bytes")},
            "whole_step": {"bytes": step_bytes, "achieved": step_bytes / step_s / 1e9,
                           "frac": step_bytes / step_s / 1e9 / peak}}
    if len(traffic) > 1 or (traffic and dom not in traffic):
        roof["traffic_other_kernels"] = {k: v for k, v in traffic.items() if k != dom}
    return roof


def time_steps(step, steps, stream, flush=None):
    """K timed steps with CUDA events on the launching stream; with flush, an
    L2-sized buffer is overwritten between steps (outside the timed spans)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kstats = {}
    for a, b in ev:
        if flush is not None:
            flush.fill_(1)
        a.record(stream)
        prof = step()
        b.record(stream)
        for k, v in prof["kernels"].items():
            x = kstats.setdefault(k, {"launches": 0, "ms": 0.0})
            x["launches"] += v["launches"]
            x["ms"] += v["ms"]
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / 1e3, kstats


# The benchmark configurations besides the headline, one short measurement
# each on the default run (name, batch width, timed steps, source cap).
EXTRA_WORKLOADS = [("er1024", 128, 20, None), ("rmat16w", 512, 2, None), ("er20k32", 0, 1, None),
                   ("er16k1024w", 0, 1, 4096)]


def extra_workload(name, n_b, steps, cap, peak, peak_kind, args):
    """One configuration: untimed byte-counting pass, one warm-up step, then
    `steps` timed steps (L2 flushed between steps when the state could stay
    in L2), its roofline and the oracle on the host cores."""
    import torch
    import paper_1609_07008_gb300 as mfbc
    g, srcs = make_workload(name)
    if cap:
        srcs = srcs[:cap]
    G = mfbc.Graph.from_csr(g)
    d_src = torch.from_numpy(srcs).cuda()
    lam = torch.empty(g.n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    _, prof_bytes = G.bc(d_src, n_b=n_b, out=lam, count_bytes=True)
    G.bc(d_src, n_b=n_b, out=lam)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda") \
        if needs_flush(g.n, prof_bytes["n_b"], prof_bytes["path"]) else None
    t, kstats = time_steps(lambda: G.bc(d_src, n_b=n_b, out=lam, profile=True)[1], steps, stream, flush)
    G.close()
    flushed = flush is not None
    del flush
    torch.cuda.empty_cache()
    desc = WORKLOADS[name]["desc"] + (f" (first {cap} of them)" if cap else "")
    roof = roofline_of(kstats, prof_bytes, peak, peak_kind, name, t / steps)
    if flushed:
        roof["note"] = ("the state fits in the L2: after the flush the kernel's per-use bytes are served mostly by "
                        "the L2, so the fraction of the HBM copy bandwidth can pass 1")
    return {"value": steps * len(srcs) * g.m / t / 1e9, "unit": "GTEPS", "steps": steps,
            "ms_per_step": t / steps * 1e3, "dtype": DTYPE.get(prof_bytes["path"], "f64"),
            "config": {"workload": desc, "name": name, "n": g.n, "nnz": g.nnz, "m": g.m, "sources": len(srcs),
                       "n_b": prof_bytes["n_b"], "path": prof_bytes["path"],
                       "l2": "L2 flushed between steps (2x L2 buffer written)" if flushed
                       else l2_note(g.n, prof_bytes["n_b"], prof_bytes["path"])},
            "roofline": roof,
            "cpu_baseline": None if args.no_cpu_baseline else cpu_baseline(g, srcs, budget_s=4.0, single_budget_s=2.0)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mfbc", choices=["mfbc", "reference"])
    ap.add_argument("--workload", default="rmat22", choices=sorted(WORKLOADS))
    ap.add_argument("--n-b", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-sources", type=int, default=64)
    ap.add_argument("--shard", action="store_true",
                    help="split the one source list across ranks (strong scaling) instead of a sample per rank")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-workloads", action="store_true", help="skip the other benchmark configurations")
    ap.add_argument("--serve-only", action="store_true", help="print only the serving measurement")
    ap.add_argument("--serve-full", action="store_true",
                    help="serving over the whole pool (R-MAT 10-20, ER 2^14-2^20, grids 256^2-2048^2)")
    ap.add_argument("--serve-requests", type=int, default=0)
    ap.add_argument("--serve-loads", default="0.5,0.8,1.2", help="offered loads (x plain capacity) to measure")
    ap.add_argument("--sources", type=int, default=0, help="use only the first N sources (probing)")
    ap.add_argument("--keep-order", action="store_true", help="batch sources in the given order")
    ap.add_argument("--accumulator", type=int, default=0, help="general kernels: MFBC_ACCUM_* (0 = auto)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve_only:
        import torch
        import paper_1609_07008_gb300 as mfbc
        from paper_1609_07008_gb300 import build as mbuild
        torch.cuda.set_device(0)
        mbuild.build()
        mfbc.load()
        pool = SERVE_FULL if args.serve_full else SERVE_DEFAULT
        res = serving_bench(pool, n_requests=args.serve_requests or (2000 if args.serve_full else 300),
                            loads=tuple(float(x) for x in args.serve_loads.split(",")))
        print(json.dumps({"serving": res}), flush=True)
        return

    import torch
    import paper_1609_07008_gb300 as mfbc
    from paper_1609_07008_gb300 import build as mbuild
    from paper_1609_07008_gb300.shard import shard_sources

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        mbuild.build()
    if dist:
        dist.barrier()
    mfbc.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # weak scaling: every rank its own sample; --shard: one list split across ranks
    g, srcs_all = make_workload(args.workload, 0 if args.shard else rank)
    if args.sources:
        srcs_all = srcs_all[:args.sources]
    srcs = shard_sources(srcs_all, rank, world) if args.shard else srcs_all
    nb_req = args.n_b or (512 if args.workload == "rmat16w" else 0)
    G = mfbc.Graph.from_csr(g)
    d_src = torch.from_numpy(np.ascontiguousarray(srcs)).to(dev)
    lam = torch.empty(g.n, dtype=torch.float64, device=dev)

    def step(profile=False):
        out = G.bc(d_src, n_b=nb_req, out=lam, profile=profile, keep_order=args.keep_order,
                   accumulator=args.accumulator)
        if dist:
            dist.all_reduce(lam)
        return out

    def barrier_sync():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # untimed pass that counts algorithmic bytes per kernel on the device
    _, prof_bytes = G.bc(d_src, n_b=nb_req, out=lam, count_bytes=True, keep_order=args.keep_order,
                         accumulator=args.accumulator)
    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    barrier_sync()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kstats = {}
    ev0.record(stream)
    for _ in range(args.steps):
        _, prof = step(profile=True)
        for k, v in prof["kernels"].items():
            a = kstats.setdefault(k, {"launches": 0, "ms": 0.0})
            a["launches"] += v["launches"]
            a["ms"] += v["ms"]
    ev1.record(stream)
    barrier_sync()
    clk = clocks.stop()
    t = ev0.elapsed_time(ev1) / 1e3
    if dist:
        tt = torch.tensor([t], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    total_sources = len(srcs_all) if args.shard else len(srcs_all) * world
    units = args.steps * total_sources * g.m
    value = units / t / 1e9

    # end to end through the host-buffer C ABI
    rp = torch.from_numpy(g.rowptr).pin_memory().numpy()
    cl = torch.from_numpy(g.col).pin_memory().numpy()
    wt = torch.from_numpy(g.w).pin_memory().numpy() if g.w is not None else None
    hs = torch.from_numpy(np.ascontiguousarray(srcs)).pin_memory().numpy()
    hl = torch.empty(g.n, dtype=torch.float64).pin_memory().numpy()
    h2d = rp.nbytes + cl.nbytes + hs.nbytes + (wt.nbytes if wt is not None else 0)
    G.close()
    del G
    torch.cuda.empty_cache()
    barrier_sync()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        with mfbc.Graph(rp, cl, wt, directed=g.directed) as Ge:
            Ge.bc(hs, n_b=nb_req, out=hl, keep_order=args.keep_order)
        if dist:
            x = torch.from_numpy(hl).to(dev)
            dist.all_reduce(x)
            hl[:] = x.cpu().numpy()
    barrier_sync()
    te = time.perf_counter() - t0
    if dist:
        tt = torch.tensor([te], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        te = float(tt.item())
    e2e = args.e2e_steps * total_sources * g.m / te / 1e9 if args.e2e_steps else None

    if rank == 0:
        peak, peak_kind = load_peaks()
        launches = sum(v["launches"] for v in kstats.values())
        line = {
            "metric": "BC GTEPS", "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "strong" if args.shard else "weak", "vs_baseline": None,
            "dtype": DTYPE.get(prof_bytes.get("path"), "f64"), "data": "synthetic",
            "config": config_of(args, g, total_sources, prof_bytes["n_b"], prof_bytes.get("path")),
            "clocks": clk,
            "e2e": {"value": e2e, "unit": "GTEPS", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(hl.nbytes)},
            "gpu_launches": int(launches),
            "roofline": roofline_of(kstats, prof_bytes, peak, peak_kind, args.workload, t / args.steps),
            "product_byte_model": product_byte_model(g, srcs, prof_bytes, t / args.steps, peak),
            "gather_stats": {k: prof_bytes.get(k) for k in ("pairs_fwd", "pairs_bwd", "values_fwd", "values_bwd",
                                                            "fwd_iters", "bwd_iters", "batches")},
            "kernels_ms_share": {k: round(v["ms"] / sum(x["ms"] for x in kstats.values()), 4)
                                 for k, v in sorted(kstats.items(), key=lambda kv: -kv[1]["ms"])},
        }
        if world == 1 and not args.no_workloads:
            line["workloads"] = {name: extra_workload(name, nb, k, cap, peak, peak_kind, args)
                                 for name, nb, k, cap in EXTRA_WORKLOADS}
        if world == 1 and not args.no_serve:
            line["serving"] = serving_bench()
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g, srcs)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
