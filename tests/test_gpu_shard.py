"""The multi-GPU entry sharded_bc on this GPU: world size 1 with a real NCCL
process group (the all-reduce runs), and two emulated ranks whose shards are
summed by hand, against the oracle (lambda within 1e-9 relative, exact zeros
equal).  Sources are independent (Algorithm 3's batch loop), so the sum of
the shards' lambdas is the list's lambda."""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1609_07008_gb300 as mfbc
from paper_1609_07008_gb300.shard import shard_sources, sharded_bc

pytestmark = pytest.mark.gpu


def _close(got, want):
    zero = want == 0
    assert np.array_equal(got[zero], want[zero])
    rel = np.abs(got[~zero] - want[~zero]) / want[~zero]
    assert rel.size == 0 or rel.max() <= 1e-9


def test_sharded_bc_world1_nccl_and_two_emulated_ranks():
    import datetime

    import torch
    import torch.distributed as dist
    from paper_1609_07008_gb300 import build
    build.build()
    g = gg.rmat(13, 8, seed=7)
    src = gg.sample_sources(g, 700, seed=8)
    want = oracle.bc(g, src)
    G = mfbc.Graph.from_csr(g)
    torch.cuda.set_device(0)
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", str(29700 + os.getpid() % 1000))
    dist.init_process_group("nccl", rank=0, world_size=1, timeout=datetime.timedelta(seconds=120),
                            device_id=torch.device("cuda", 0))
    try:
        lam = sharded_bc(G, src, 0, 1, n_b=256)
        torch.cuda.synchronize()
        _close(lam.cpu().numpy(), want)
    finally:
        dist.destroy_process_group()
    # two ranks' shards on one GPU, one after the other (no collective)
    parts = [sharded_bc(G, src, r, 2, n_b=256).cpu().numpy() for r in range(2)]
    assert sum(len(shard_sources(src, r, 2)) for r in range(2)) == len(src)
    _close(parts[0] + parts[1], want)
    G.close()
