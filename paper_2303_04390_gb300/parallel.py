"""One problem across several GPUs by pattern shards.

Site patterns are conditionally independent (paper, Methods), so log P(Y)
and every gradient entry are sums over patterns (Eqs. 3 and 7): each rank
evaluates a contiguous range of patterns on its own GPU and one all-reduce
(sum) of the 2N-1 FP64 values [log P(Y), gradient] combines them -- the
only exchange step of the path.  Independent problems (many HMC chains)
need no collective at all and run as replicas instead.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple


def pattern_shard(n_patterns: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous, balanced range [lo, hi) of patterns for `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_patterns, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def _gpu_evaluator(precision: str, device) -> Callable:
    def run(shard):
        import torch
        from .context import from_workload
        ctx = from_workload(shard, precision, device=device)
        out = ctx.evaluate_device()
        ctx.check()
        res = out.clone()
        ctx.close()
        return res
    return run


def sharded_evaluate(w, precision: str = "fp32", group=None, device=None,
                     evaluator: Optional[Callable] = None):
    """[log P(Y), d log P(Y)/d t_0 .. t_{2N-3}] of workload `w` (a
    synth.Workload-like object) summed over the ranks of `group`, each rank
    evaluating its pattern shard.  `evaluator(shard) -> tensor [2N-1]`
    defaults to this library on the rank's GPU; the all-reduce runs on
    whatever device that tensor lives on (NCCL for CUDA tensors)."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    lo, hi = pattern_shard(w.n_patterns, rank, world)
    shard = w.with_patterns(lo, hi)
    run = evaluator or _gpu_evaluator(precision, device)
    vec = run(shard)
    dist.all_reduce(vec, op=dist.ReduceOp.SUM, group=group)
    return vec
