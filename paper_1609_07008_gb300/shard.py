"""Source sharding across ranks (one process per GPU).

Sources are independent in Algorithm 3 (the batch loop over columns of the
n x n_b frontier), and lambda is linear in the source list, so a multi-GPU
run gives each rank a disjoint part of the source list, runs MFBC on a full
replica of the graph (the paper's replicate-A decomposition, Sec. 5.2.1
variant A and the replication of Theorem 2's proof), and sums the per-rank
lambda vectors with one all-reduce.  These helpers hold only that host logic;
the per-rank computation is the C ABI's mfbc_bc.
"""
from __future__ import annotations

import numpy as np


def shard_sources(sources, rank: int, world: int) -> np.ndarray:
    """Contiguous, near-equal slice of the source list for `rank` of `world`.

    The slices partition the list exactly (every occurrence lands on one rank)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    src = np.asarray(sources)
    lo = (len(src) * rank) // world
    hi = (len(src) * (rank + 1)) // world
    return src[lo:hi]


def allreduce_lambda(lam, group=None):
    """Sum a per-rank lambda (torch tensor) over the process group in place
    (a no-op without an initialised process group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(lam, op=dist.ReduceOp.SUM, group=group)
    return lam


def _device_bc(graph, shard, **kw):
    """This rank's lambda on its GPU: mfbc_bc_device over the shard."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    return graph.bc(torch.from_numpy(np.ascontiguousarray(shard, dtype=np.int32)).to(dev), **kw)


def sharded_bc(graph, sources, rank: int, world: int, *, group=None, compute=None, **kw):
    """lambda over all `sources`, computed as this rank's shard plus an all-reduce.

    `graph` is this rank's replica of the graph (a paper_1609_07008_gb300.Graph
    on its GPU); `sources` is the full list (host array), the same on every
    rank.  `compute(graph, shard, **kw)` returns the shard's lambda as a torch
    tensor; by default it is the library's device call.  Returns the summed
    lambda (a torch tensor on the compute's device)."""
    mine = shard_sources(sources, rank, world)
    lam = (compute or _device_bc)(graph, mine, **kw)
    return allreduce_lambda(lam, group)
