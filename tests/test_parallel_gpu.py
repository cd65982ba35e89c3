"""The pattern-shard path on the GPU: a resident ShardedContext (the library
evaluating its shard on this rank's GPU, then an NCCL all-reduce) at world
size 1, over several steps with new branch lengths, against the oracle."""
import socket

import numpy as np
import pytest

import synth
from parity import compare, oracle_eval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_resident_shard_with_nccl_all_reduce_world_1():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.distributed as dist
    from paper_2303_04390_gb300 import build as B
    B.build()
    from paper_2303_04390_gb300.parallel import ShardedContext
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}",
                            rank=0, world_size=1)
    try:
        w = synth.small_workload(40, 4, 4, 500, seed=91)
        sc = ShardedContext(w, "fp32", device="cuda")
        rng = np.random.default_rng(3)
        for _ in range(3):
            t = w.t * np.exp(0.1 * rng.standard_normal(w.t.shape))
            vec = sc.evaluate(t).cpu().numpy()
            compare(vec[0], vec[1:], oracle_eval(w, t=t), "fp32", "shard world 1")
        sc.close()
    finally:
        dist.destroy_process_group()
