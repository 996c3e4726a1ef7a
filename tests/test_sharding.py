"""Multi-rank host logic on CPU: world_size-2 gloo ranks run the product's
sharded_bc (shard the source list, compute the shard's lambda, sum by one
all-reduce).  Only the per-rank computation is replaced, through sharded_bc's
`compute` argument, by the oracle on the CPU; the sharding and the reduction
are the code a multi-GPU run executes."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import graphgen as gg
import oracle
from paper_1609_07008_gb300.shard import shard_sources, sharded_bc


def test_shards_partition_the_list():
    src = np.arange(103)
    for world in (1, 2, 3, 8):
        parts = [shard_sources(src, r, world) for r in range(world)]
        assert np.array_equal(np.concatenate(parts), src)
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        shard_sources(src, 2, 2)


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = gg.rmat(9, 8, directed=True, weights=(1, 5), seed=3)
    src = gg.sample_sources(g, 77, seed=4)
    seen = []

    def on_cpu(graph, shard):
        seen.append(len(shard))
        return torch.from_numpy(oracle.bc(graph, shard, nthreads=1))

    lam = sharded_bc(g, src, rank, world, compute=on_cpu)
    assert seen == [len(shard_sources(src, rank, world))]
    if rank == 0:
        np.save(out, lam.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2_allreduce_matches_single_rank(tmp_path):
    out = str(tmp_path / "lam.npy")
    port = 29500 + (os.getpid() % 2000)
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    g = gg.rmat(9, 8, directed=True, weights=(1, 5), seed=3)
    src = gg.sample_sources(g, 77, seed=4)
    want = oracle.bc(g, src)
    got = np.load(out)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
