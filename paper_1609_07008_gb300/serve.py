"""Serving loop for approximate-BC requests over resident graphs.

A request is (graph, sampled source list); its answer is the lambda of
Algorithm 3 over that list.  The paper runs one source list at a time; a
server receives many independent lists and can pack their columns into the
same MFBF/MFBr batches (Algorithm 3's batch dimension), which amortises the
per-level costs of small requests.

`Server` keeps the graphs resident on the device and runs one worker thread
per graph:

* continuous batching -- a worker takes, in arrival order, the pending
  requests of its graph up to `max_cols` packed columns (each request rounded
  up to 32) and runs them in one `mfbc_bc_multi_device` call, which returns
  one lambda row per request; requests that arrive meanwhile wait for the
  worker's next group;
* memory-budget admission -- a group holds the device bytes of its scratch
  (`mfbc_workspace_size`, mode 2) plus its lambda rows; a group starts only
  when the bytes held by running groups leave room for it, and its n_b is
  lowered until a lone group fits;
* overlap -- every worker issues its work on its own CUDA stream, so groups
  of different graphs run on the device at once; extra handles of one graph
  (`replicas`) give it more workers, so that several of its groups overlap
  too (a graph whose batches leave the device idle between their short
  kernels, such as a weighted grid on the general kernels, gains most).

`run_plain` is the one-request-at-a-time form (one mfbc_bc_device call per
request, in arrival order) that the server is compared against.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np


def align32(k: int) -> int:
    return (k + 31) // 32 * 32


@dataclass
class Request:
    rid: int
    graph: str
    sources: np.ndarray                  # int32 vertex ids
    arrival: float = 0.0                 # seconds, on the run's clock
    start: float = math.nan
    done: float = math.nan
    result: np.ndarray | None = None     # lambda, float64[n]
    group: int = -1


@dataclass
class GroupLog:
    graph: str
    nreq: int
    cols: int
    n_b: int
    bytes: int
    t0: float
    t1: float


class Server:
    """Resident graphs, memory-budget admission, continuous batching.

    graphs: name -> paper_1609_07008_gb300.Graph.  executor(name, group,
    n_b, ws_bytes, stream) -> list of lambda arrays may replace the GPU call
    (host-logic tests); sizer(name, cols, nreq, n_b) -> bytes likewise."""

    def __init__(self, graphs: dict, *, budget_bytes: int, max_cols: int = 4096, n_b: int = 0,
                 executor=None, sizer=None, clock=time.perf_counter, replicas: dict | None = None):
        self.graphs = graphs
        # extra handles of the same graphs: one more worker (and CUDA stream)
        # each, so that several groups of one graph can run at once
        self.handles = {k: [G] + list((replicas or {}).get(k, [])) for k, G in graphs.items()}
        self.budget = int(budget_bytes)
        self.max_cols = int(max_cols)
        self.n_b = int(n_b)
        self.clock = clock
        self.executor = executor or self._execute_gpu
        self.sizer = sizer or self._group_bytes
        self._cv = threading.Condition()
        self._pending = {k: collections.deque() for k in graphs}
        self._held = 0
        self._stop = False
        self._inflight = 0
        self.log: list[GroupLog] = []
        self.errors: list[BaseException] = []
        self._threads = [threading.Thread(target=self._worker, args=(k, h), daemon=True)
                         for k in graphs for h in self.handles[k]]

    # ------------------------------------------------------------ public
    def start(self) -> "Server":
        for t in self._threads:
            t.start()
        return self

    def submit(self, req: Request) -> None:
        with self._cv:
            if self._stop:
                raise RuntimeError("server is closed")
            self._pending[req.graph].append(req)
            self._inflight += 1
            self._cv.notify_all()

    def drain(self, timeout: float | None = None) -> bool:
        """Wait until every submitted request is answered."""
        end = None if timeout is None else self.clock() + timeout
        with self._cv:
            while self._inflight and not self.errors:
                left = None if end is None else end - self.clock()
                if left is not None and left <= 0:
                    return False
                self._cv.wait(left)
            if self.errors:
                raise self.errors[0]
        return True

    def close(self) -> None:
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        for t in self._threads:
            t.join()

    # ------------------------------------------------------------ internals
    def _take_group(self, key):
        q = self._pending[key]
        group, cols = [], 0
        while q:
            c = align32(len(q[0].sources))
            if group and cols + c > self.max_cols:
                break
            group.append(q.popleft())
            cols += c
        return group, cols

    def _fit(self, key, cols, nreq):
        """The group's n_b and bytes: self.n_b (0 = the library's own choice
        for the group's columns), lowered in steps of 128 while the group
        alone would not fit the budget."""
        nb = self.n_b
        need = self.sizer(key, cols, nreq, nb)
        if need > self.budget and nb == 0:
            nb = 1024
            need = self.sizer(key, cols, nreq, nb)
        while need > self.budget and nb > 128:
            nb -= 128
            need = self.sizer(key, cols, nreq, nb)
        return nb, need

    def _worker(self, key, handle):
        stream = None
        try:
            import torch
            if torch.cuda.is_available() and self.executor == self._execute_gpu:
                stream = torch.cuda.Stream()
        except ImportError:
            pass
        while True:
            with self._cv:
                while not self._pending[key] and not self._stop:
                    self._cv.wait()
                if not self._pending[key]:
                    return
                group, cols = self._take_group(key)
                nb, need = self._fit(key, cols, len(group))
                # admission: wait until the running groups leave room
                while self._held and self._held + need > self.budget:
                    self._cv.wait()
                self._held += need
                gid = len(self.log)
                self.log.append(GroupLog(key, len(group), cols, nb, need, self.clock(), math.nan))
            t0 = self.clock()
            for r in group:
                r.start, r.group = t0, gid
            try:
                results = self.executor(key, group, nb, need, stream) if self.executor != self._execute_gpu \
                    else self._execute_gpu(key, group, nb, need, stream, handle)
            except BaseException as e:             # surface to drain()
                with self._cv:
                    self.errors.append(e)
                    self._held -= need
                    self._cv.notify_all()
                return
            t1 = self.clock()
            with self._cv:
                for r, lam in zip(group, results):
                    r.result, r.done = lam, t1
                self.log[gid].t1 = t1
                self._held -= need
                self._inflight -= len(group)
                self._cv.notify_all()

    def _group_bytes(self, key, cols, nreq, nb):
        G = self.graphs[key]
        return G.workspace_size(cols, 2, n_b=nb) + 8 * nreq * G.n

    def _execute_gpu(self, key, group, nb, ws_bytes, stream, handle=None):
        import torch
        G = handle if handle is not None else self.graphs[key]
        with torch.cuda.stream(stream):
            srcs = [torch.from_numpy(np.ascontiguousarray(r.sources, dtype=np.int32)).to("cuda", non_blocking=True)
                    for r in group]
            ws = torch.empty(ws_bytes - 8 * len(group) * G.n, dtype=torch.uint8, device="cuda")
            lam = G.bc_multi(srcs, n_b=nb, stream=stream, workspace=ws)
            host = lam.to("cpu")
        return [host[i].numpy() for i in range(len(group))]


def run_served(server: Server, requests: list[Request], clock=time.perf_counter, timeout=None):
    """Submit each request at its arrival time (relative to the call) and wait
    for all answers; arrival/start/done are rewritten on the run's clock."""
    t0 = clock()
    for r in sorted(requests, key=lambda r: r.arrival):
        wait = t0 + r.arrival - clock()
        if wait > 0:
            time.sleep(wait)
        r.arrival = t0 + r.arrival
        server.submit(r)
    server.drain(timeout)
    for r in requests:
        r.arrival -= t0
        r.start -= t0
        r.done -= t0
    return requests


def run_plain(graphs: dict, requests: list[Request], clock=time.perf_counter, n_b: int = 0):
    """One request at a time in arrival order (mfbc_bc_device per request)."""
    import torch
    t0 = clock()
    for r in sorted(requests, key=lambda r: r.arrival):
        wait = t0 + r.arrival - clock()
        if wait > 0:
            time.sleep(wait)
        r.start = clock() - t0
        G = graphs[r.graph]
        src = torch.from_numpy(np.ascontiguousarray(r.sources, dtype=np.int32)).to("cuda")
        r.result = G.bc(src, n_b=n_b).to("cpu").numpy()
        r.done = clock() - t0
    return requests


def make_requests(graph_sizes: dict, count: int, rate: float, *, lo: int = 64, hi: int = 4096,
                  seed: int = 0, eligible: dict | None = None) -> list[Request]:
    """Poisson arrivals at `rate` per second; each request picks a graph
    uniformly and log-uniform [lo, hi] sources (at most the graph's eligible
    vertices), sampled without replacement."""
    rng = np.random.default_rng(seed)
    names = sorted(graph_sizes)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        name = names[int(rng.integers(len(names)))]
        pool = eligible[name] if eligible else np.arange(graph_sizes[name], dtype=np.int32)
        k = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        k = max(1, min(k, len(pool)))
        src = np.sort(rng.choice(pool, size=k, replace=False)).astype(np.int32)
        out.append(Request(rid=i, graph=name, sources=src, arrival=t))
    return out


def latency_stats(requests: list[Request], edges: dict) -> dict:
    """p50/p99/mean latency (arrival to answer) and throughput over the run."""
    lat = np.array([r.done - r.arrival for r in requests])
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    teps = sum(len(r.sources) * edges[r.graph] for r in requests)
    return {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "span_s": float(span), "gteps": float(teps / span / 1e9)}
