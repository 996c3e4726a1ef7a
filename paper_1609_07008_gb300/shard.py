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
    """Sum a per-rank lambda (torch tensor) over the process group in place."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(lam, op=dist.ReduceOp.SUM, group=group)
    return lam


def sharded_bc(graph, sources, rank: int, world: int, *, group=None, **kw):
    """lambda over all `sources`, computed as this rank's shard plus an all-reduce.

    `graph` is a paper_1609_07008_gb300.Graph replica on this rank's GPU;
    `sources` is the full list (host array); returns a torch CUDA tensor."""
    import torch
    mine = shard_sources(sources, rank, world)
    dev = torch.device("cuda", torch.cuda.current_device())
    lam = graph.bc(torch.from_numpy(np.ascontiguousarray(mine, dtype=np.int32)).to(dev), **kw)
    return allreduce_lambda(lam, group)
