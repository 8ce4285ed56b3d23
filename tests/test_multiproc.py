"""Multi-process (gloo, world size 2, CPU) coverage of the env-sharded path:
the shard plan covers every env exactly once with balanced cost, and the
envs stepped by two ranks and gathered equal a single-process run (the step
has no cross-env exchange).  The per-rank stepping here uses the oracle, so
the test needs no GPU."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import scenegen
from paper_2410_00425_b300 import shard


def test_shard_ranges_cover_and_balance():
    g = np.random.default_rng(0)
    for E in (1, 2, 3, 7, 64, 1000):
        for world in (1, 2, 3, 4, 8):
            costs = g.integers(1, 100, E)
            rs = shard.shard_ranges(costs, world)
            assert len(rs) == world
            assert rs[0][0] == 0 and rs[-1][1] == E
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c and a <= b
            if E >= world:
                assert all(b > a for a, b in rs)
                sums = [costs[a:b].sum() for a, b in rs]
                assert max(sums) <= costs.sum() / world + costs.max() + 1e-9


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    sc = scenegen.make_scene("clutter", n_envs=24)
    mine = shard.local_envs(sc, rank, world)
    sub = sc.subset(mine)
    o = oracle.Oracle(sub)
    o.step(3)
    st = torch.from_numpy(o.state())
    # gather variable-size shards: sizes first, then padded states
    n = torch.tensor([st.shape[0]])
    sizes = [torch.zeros(1, dtype=torch.long) for _ in range(world)]
    dist.all_gather(sizes, n)
    mx = int(max(s.item() for s in sizes))
    pad = torch.zeros((mx, 13), dtype=torch.float64)
    pad[:st.shape[0]] = st
    bufs = [torch.zeros((mx, 13), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(bufs, pad)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)          # the bench's max-over-ranks timing
    if rank == 0:
        full = torch.cat([b[:int(s.item())] for b, s in zip(bufs, sizes)]).numpy()
        np.save(out_path, full)
        assert t.item() == world
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo_sharded_step_equals_single_process(tmp_path):
    import oracle
    world = 2
    port = 29500 + (os.getpid() % 2000)
    out = str(tmp_path / "gathered.npy")
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    gathered = np.load(out)
    sc = scenegen.make_scene("clutter", n_envs=24)
    o = oracle.Oracle(sc)
    o.step(3)
    assert np.array_equal(gathered, o.state())
