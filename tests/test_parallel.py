"""The multi-rank paths on CPU: pattern shards all-reduced over a
world-size-2 gloo group equal the unsharded result (the oracle stands in
for each rank's GPU evaluation), and the bench's replica mode combines
per-rank timings with a MAX all-reduce only."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_2303_04390_gb300.parallel import pattern_shard


def test_pattern_shards_partition_the_patterns():
    for C in [0, 1, 7, 100, 10001]:
        for world in [1, 2, 3, 8]:
            ranges = [pattern_shard(C, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == C
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from oracle import phylo_oracle as O
    from paper_2303_04390_gb300.parallel import sharded_evaluate
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.small_workload(12, 4, 4, 101, seed=90)

    def oracle_shard(shard):
        ll, g, _ = O.evaluate(shard.parent, shard.t, shard.Q, shard.pi,
                              shard.rates, shard.weights,
                              shard.pattern_weights,
                              tip_states=shard.tip_states)
        return torch.tensor(np.concatenate([[ll], g]), dtype=torch.float64)

    vec = sharded_evaluate(w, evaluator=oracle_shard)
    # replica-mode timing combine: MAX over ranks
    tt = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    out.put((rank, vec.numpy(), float(tt.item())))
    dist.destroy_process_group()


def test_sharded_sum_equals_unsharded_over_gloo():
    import multiprocessing as mp
    from oracle import phylo_oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.small_workload(12, 4, 4, 101, seed=90)
    ll, g, _ = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                          w.pattern_weights, tip_states=w.tip_states)
    ref = np.concatenate([[ll], g])
    for rank, vec, tmax in got:
        np.testing.assert_allclose(vec, ref, rtol=1e-12, atol=1e-10)
        assert tmax == 2.0
