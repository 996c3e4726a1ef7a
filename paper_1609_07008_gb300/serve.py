"""Serving loop for approximate-BC requests over resident graphs.

A request is (graph, sampled source list); its answer is the lambda of
Algorithm 3 over that list.  The paper runs one source list at a time; a
server receives many independent lists and can pack their columns into the
same MFBF/MFBr batches (Algorithm 3's batch dimension), which amortises the
per-level costs of small requests.

`Server` keeps the graphs resident on the device and runs workers (one CUDA
stream each; `replicas` gives a graph more of them):

* continuous batching at batch granularity -- a worker runs one batch of
  n_b columns at a time.  Before each batch it fills the columns, in arrival
  order, first with the next sources of the requests it already serves, then
  with newly arrived requests of its graph (each request's part starts on a
  32-column word).  A request that arrives while a batch runs joins the next
  batch; a large request is spread over several batches and shares them
  with others.  Each batch is one `mfbc_bc_multi_device` call that adds
  every part's lambda into its request's row of the worker's lambda pool
  (lambda is linear in the source list, MFBC_OPT_ACCUMULATE); a request is
  answered when the batch holding its last sources completes;
* memory-budget admission -- a worker holds its batch scratch
  (`mfbc_workspace_size`, mode 2) and one lambda row per request it can
  serve at once (n_b / 32 rows); it takes this memory from the budget when
  it has work and gives it back when idle, so the workers of other graphs
  wait while the budget is spent; n_b is lowered until one worker fits;
* overlap -- every worker issues its work on its own CUDA stream, so the
  batches of different graphs (and of one graph's replicas) run on the device
  at once.

`run_plain` is the one-request-at-a-time form (one mfbc_bc_device call per
request, in arrival order) that the server is compared against.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from dataclasses import dataclass

import numpy as np


def align32(k: int) -> int:
    return (k + 31) // 32 * 32


@dataclass
class Request:
    rid: int
    graph: str
    sources: np.ndarray                  # int32 vertex ids
    arrival: float = 0.0                 # seconds, on the run's clock
    start: float = math.nan              # its first batch began
    done: float = math.nan
    result: np.ndarray | None = None     # lambda, float64[n]
    group: int = -1                      # index of its first batch in Server.log
    placed: int = 0                      # sources already given to batches
    slot: int = -1                       # its row in the worker's lambda pool


@dataclass
class GroupLog:
    """One batch: the requests it held (nreq), how many of them started in it
    (new), the columns used, its width and the bytes its worker held."""
    graph: str
    nreq: int
    cols: int
    n_b: int
    bytes: int
    t0: float
    t1: float
    new: int = 0
    worker: int = 0


class _Worker:
    def __init__(self, wid, key, handle):
        self.wid, self.key, self.handle = wid, key, handle
        self.bound: collections.deque = collections.deque()   # requests served, arrival order
        self.free_slots: list[int] = []
        self.active = False
        self.nb = 0
        self.need = 0
        self.pool = None                   # [slots, n] lambda rows
        self.ws = None                     # batch scratch (GPU)
        self.stream = None


class Server:
    """Resident graphs, memory-budget admission, continuous batching.

    graphs: name -> paper_1609_07008_gb300.Graph.  For host-logic tests,
    executor(key, parts, n_b, pool, rows, stream, handle) may replace the GPU
    call (it must add each part's lambda into pool[row]; parts are (request,
    first source, count)), and sizer(key, n_b, slots) -> bytes the
    library's scratch size; the pool is then a numpy array."""

    def __init__(self, graphs: dict, *, budget_bytes: int, max_cols=1024, n_b: int = 0,
                 executor=None, sizer=None, clock=time.perf_counter, replicas: dict | None = None):
        self.graphs = graphs
        self.handles = {k: [G] + list((replicas or {}).get(k, [])) for k, G in graphs.items()}
        self.budget = int(budget_bytes)
        # columns per batch: one width, or one per graph (a dict)
        self.max_cols = dict(max_cols) if isinstance(max_cols, dict) else {k: int(max_cols) for k in graphs}
        self.n_b = int(n_b)
        self.clock = clock
        self._gpu = executor is None
        self.executor = executor or self._execute_gpu
        self.sizer = sizer or self._worker_bytes
        self._cv = threading.Condition()
        self._pending = {k: collections.deque() for k in graphs}
        self._held = 0
        self._stop = False
        self._inflight = 0
        self.log: list[GroupLog] = []
        self.errors: list[BaseException] = []
        self._workers = [_Worker(i, k, h) for i, (k, h) in
                         enumerate((k, h) for k in graphs for h in self.handles[k])]
        self._threads = [threading.Thread(target=self._run, args=(w,), daemon=True) for w in self._workers]

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

    def stats(self) -> dict:
        """Packing of the batches run so far: requests per batch, columns
        used per batch, batches that held several requests."""
        if not self.log:
            return {"batches": 0}
        nreq = np.array([g.nreq for g in self.log])
        cols = np.array([g.cols / g.n_b for g in self.log])
        return {"batches": len(self.log), "requests_per_batch_mean": float(nreq.mean()),
                "requests_per_batch_max": int(nreq.max()),
                "batches_with_several_requests": float((nreq > 1).mean()),
                "columns_used_mean": float(cols.mean())}

    # ------------------------------------------------------------ internals
    def _width(self, key):
        """The worker's n_b and bytes: n_b (or the graph's max_cols), lowered
        in steps of 128 while one worker would not fit the budget."""
        nb = self.n_b or self.max_cols[key]
        while True:
            try:
                need = self.sizer(key, nb, max(1, nb // 32))
            except ValueError:                  # wider than the library takes for this graph
                need = None
            if (need is not None and need <= self.budget) or nb <= 128:
                break
            nb = max(128, nb - 128)
        if need is None:
            raise ValueError(f"no batch width fits graph {key}")
        return nb, need

    def _fill(self, w: _Worker):
        """Columns of the next batch.  The requests the worker serves that
        still have sources, then newly arrived ones (while pool rows and
        32-column words are free), share the batch's words equally as far as
        each needs them (water filling), so a request that arrives while a
        large one runs gets its share of the very next batch."""
        words = max(1, w.nb // 32)
        cands = [r for r in w.bound if len(r.sources) > r.placed]
        new = 0
        q = self._pending[w.key]
        while q and w.free_slots and len(cands) < words:
            r = q.popleft()
            r.slot = w.free_slots.pop()
            r.start, r.group = self.clock(), len(self.log)
            w.bound.append(r)
            new += 1
            if len(r.sources):
                cands.append(r)
        need = [-(-(len(r.sources) - r.placed) // 32) for r in cands]
        alloc = [0] * len(cands)
        left = words
        order = sorted(range(len(cands)), key=lambda i: need[i])
        for k, i in enumerate(order):           # smallest needs first, the rest share what remains
            share = min(need[i], left // (len(order) - k))
            alloc[i] = share
            left -= share
        for i in order[::-1]:                   # words left by rounding go to the largest needs
            extra = min(left, need[i] - alloc[i])
            alloc[i] += extra
            left -= extra
        parts, cols = [], 0
        for r, a in zip(cands, alloc):
            if a:
                take = min(len(r.sources) - r.placed, 32 * a)
                parts.append((r, r.placed, take))
                r.placed += take
                cols += align32(take)
        for r in w.bound:                       # requests without sources are answered with this batch
            if len(r.sources) == 0 and r.group == len(self.log):
                parts.append((r, 0, 0))
        return parts, cols, new

    def _has_work(self, w: _Worker) -> bool:
        if any(len(r.sources) > r.placed for r in w.bound):
            return True
        return bool(self._pending[w.key]) and (not w.active or bool(w.free_slots))

    def _run(self, w: _Worker):
        try:
            import torch
            if self._gpu and torch.cuda.is_available():
                w.stream = torch.cuda.Stream()
        except ImportError:
            pass
        while True:
            with self._cv:
                while True:
                    if self._has_work(w):
                        if w.active:
                            break
                        try:
                            nb, need = self._width(w.key)
                        except BaseException as e:     # surface to drain()
                            self.errors.append(e)
                            self._cv.notify_all()
                            return
                        # admission: start when the active workers leave room
                        if not self._held or self._held + need <= self.budget:
                            w.active, w.nb, w.need = True, nb, need
                            w.free_slots = list(range(max(1, nb // 32)))[::-1]
                            self._held += need
                            break
                    elif w.active and not w.bound:
                        # idle: give the memory back to the budget
                        w.active = False
                        self._held -= w.need
                        w.pool = w.ws = None
                        self._cv.notify_all()
                    elif self._stop and not w.bound and not self._pending[w.key]:
                        return
                    self._cv.wait()
                parts, cols, new = self._fill(w)
                gid = len(self.log)
                self.log.append(GroupLog(w.key, len({id(p[0]) for p in parts}), cols, w.nb, w.need,
                                         self.clock(), math.nan, new, w.wid))
            try:
                self._ensure_memory(w)
                for r, first, _ in parts:
                    if first == 0:
                        self._zero_row(w, r.slot)
                rows = [r.slot for r, _, _ in parts]
                if self._gpu:
                    self._execute_gpu(w, parts, rows)
                else:
                    self.executor(w.key, parts, w.nb, w.pool, rows, None, None)
                finished = [r for r in w.bound if r.placed >= len(r.sources)]
                results = [self._read_row(w, r.slot) for r in finished]
            except BaseException as e:             # surface to drain()
                with self._cv:
                    self.errors.append(e)
                    if w.active:
                        self._held -= w.need
                    w.active = False
                    self._cv.notify_all()
                return
            t1 = self.clock()
            with self._cv:
                for r, lam in zip(finished, results):
                    r.result, r.done = lam, t1
                    w.bound.remove(r)
                    w.free_slots.append(r.slot)
                self.log[gid].t1 = t1
                self._inflight -= len(finished)
                self._cv.notify_all()

    def _ensure_memory(self, w: _Worker):
        n = self.graphs[w.key].n
        slots = max(1, w.nb // 32)
        if w.pool is not None and w.pool.shape[0] == slots:
            return
        if not self._gpu:
            w.pool = np.zeros((slots, n))
            return
        import torch
        G = self.graphs[w.key]
        with torch.cuda.stream(w.stream):
            w.pool = torch.zeros((slots, n), dtype=torch.float64, device="cuda")
            w.ws = torch.empty(max(1, G.workspace_size(w.nb, 2, n_b=w.nb)), dtype=torch.uint8, device="cuda")

    def _zero_row(self, w: _Worker, slot: int):
        if self._gpu:
            import torch
            with torch.cuda.stream(w.stream):
                w.pool[slot].zero_()
        else:
            w.pool[slot] = 0.0

    def _read_row(self, w: _Worker, slot: int):
        if self._gpu:
            import torch
            with torch.cuda.stream(w.stream):
                return w.pool[slot].to("cpu").numpy()
        return w.pool[slot].copy()

    def _worker_bytes(self, key, nb, slots):
        from . import MFBCError, MFBC_ERR_INVALID
        G = self.graphs[key]
        try:
            return G.workspace_size(nb, 2, n_b=nb) + 8 * slots * G.n
        except MFBCError as e:
            if e.status == MFBC_ERR_INVALID:
                raise ValueError(str(e)) from e
            raise

    def _execute_gpu(self, w: _Worker, parts, rows):
        """One batch: every part's lambda added into its request's pool row."""
        import torch
        src = np.concatenate([r.sources[a:a + k] for r, a, k in parts]).astype(np.int32)
        off = np.zeros(len(parts) + 1, dtype=np.int32)
        off[1:] = np.cumsum([k for _, _, k in parts])
        with torch.cuda.stream(w.stream):
            d_src = torch.from_numpy(src).to("cuda")
            w.handle.bc_multi((d_src, off), n_b=w.nb, stream=w.stream, workspace=w.ws, out=w.pool, rows=rows,
                              accumulate=True)


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
                  seed: int = 0, eligible: dict | None = None, weights: dict | None = None) -> list[Request]:
    """Poisson arrivals at `rate` per second; each request picks a graph
    (uniformly, or with probability proportional to `weights`) and
    log-uniform [lo, hi] sources (at most the graph's eligible vertices),
    sampled without replacement."""
    rng = np.random.default_rng(seed)
    names = sorted(graph_sizes)
    p = None
    if weights:
        p = np.array([float(weights[k]) for k in names])
        p = p / p.sum()
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        name = names[int(rng.choice(len(names), p=p))] if p is not None else names[int(rng.integers(len(names)))]
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
