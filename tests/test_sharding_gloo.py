"""Sharded lookups across two ranks (gloo, CPU): each rank filters its contiguous
share of the queries with query_offset = share start (here through the oracle, the
CPU stand-in for a rank's GPU), and the shares concatenate to the single-process
result.  No data is exchanged on the lookup path; the gather below only checks."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2305_05810_gb300.sharding import shard


def test_shard_ranges_cover_everything_once():
    for n in (0, 1, 7, 1000, 33177600):
        for world in (1, 2, 3, 8):
            ranges = [shard(n, r, world) for r in range(world)]
            assert sum(c for _, c in ranges) == n
            assert all(ranges[k][0] + ranges[k][1] == ranges[k + 1][0] for k in range(world - 1))
            assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    from oracle import codecs, filters, textures
    vals = synth.dense_density(n=32, seed=3, period=8.0)
    grid = textures.Dense3D(codecs.f16_decode(codecs.f16_encode(vals.astype(np.float64))))
    pts = (synth.uniform(3 * 5001, 6).reshape(-1, 3) * np.float32(36) - np.float32(2)).astype(np.float32)
    start, count = shard(pts.shape[0], rank, world)
    qid = np.arange(start, start + count, dtype=np.uint64)   # query_offset = start
    v, _, _ = filters.lookup_3d(grid, pts[start:start + count], "bspline3", stochastic_form=True,
                                seed=9, qid=qid)
    parts = [None] * world
    dist.all_gather_object(parts, v)
    if rank == 0:
        whole, _, _ = filters.lookup_3d(grid, pts, "bspline3", stochastic_form=True, seed=9)
        q.put(bool(np.array_equal(np.concatenate(parts), whole)))
    dist.destroy_process_group()


def test_two_rank_shards_concatenate_to_single_process_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True
