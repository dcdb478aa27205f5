"""Multi-rank slice sharding on CPU (gloo, world_size 2): shards partition the
stack, the timing reduction takes the max, and sharded solves reassemble to
the unsharded result (slices are independent)."""

import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2006_09808_gb300.sharding import max_over_ranks, slice_shard


@pytest.mark.parametrize("n,world", [(0, 2), (7, 2), (64, 8), (5, 8), (96, 3)])
def test_shards_partition(n, world):
    ranges = [slice_shard(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle import pd_oracle as O

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(0)
    f = rng.standard_normal((5, 12, 10))
    m = (rng.random((5, 12, 10)) > 0.2).astype(np.uint8)
    a, b = slice_shard(5, rank, world)
    chi = O.pd_solve(f[a:b], m[a:b], 0.5, 1 / 2.9, 1 / 2.9, 30)
    np.save(os.path.join(out_dir, f"shard{rank}.npy"), chi)
    t = max_over_ranks(1.0 + rank)
    np.save(os.path.join(out_dir, f"max{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2_sharded_solve(tmp_path):
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    from oracle import pd_oracle as O

    rng = np.random.default_rng(0)
    f = rng.standard_normal((5, 12, 10))
    m = (rng.random((5, 12, 10)) > 0.2).astype(np.uint8)
    full = O.pd_solve(f, m, 0.5, 1 / 2.9, 1 / 2.9, 30)
    parts = np.concatenate([np.load(tmp_path / f"shard{r}.npy") for r in range(2)])
    assert np.allclose(parts, full, rtol=0, atol=1e-14)
    assert [float(np.load(tmp_path / f"max{r}.npy")[0]) for r in range(2)] == [2.0, 2.0]
