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


class ShardedContext:
    """One problem across the ranks of a process group: each rank keeps its
    pattern shard resident in a library context on its own GPU (tree
    schedule, eigendecomposition, tip data, graph), so a step pays only the
    branch-length upload, one graph replay and one all-reduce (sum) of the
    2N-1 FP64 values."""

    def __init__(self, w, precision: str = "fp32", group=None, device=None):
        import torch.distributed as dist
        from .context import from_workload
        self.group = group
        rank = dist.get_rank(group)
        world = dist.get_world_size(group)
        self.lo, self.hi = pattern_shard(w.n_patterns, rank, world)
        self.ctx = from_workload(w.with_patterns(self.lo, self.hi), precision,
                                 device=device)

    def evaluate(self, t=None):
        """[log P(Y), gradient] summed over the ranks (a CUDA FP64 tensor of
        2N-1 values); t (host array or CUDA tensor) replaces the branch
        lengths first."""
        import torch.distributed as dist
        if t is not None:
            self.ctx.set_branch_lengths(t)
        vec = self.ctx.evaluate_device()
        dist.all_reduce(vec, op=dist.ReduceOp.SUM, group=self.group)
        self.ctx.check()
        return vec

    def close(self):
        self.ctx.close()


def sharded_evaluate(w, precision: str = "fp32", group=None, device=None,
                     evaluator: Optional[Callable] = None):
    """One-shot [log P(Y), d log P(Y)/d t_0 .. t_{2N-3}] of workload `w` (a
    synth.Workload-like object) summed over the ranks of `group`, each rank
    evaluating its pattern shard.  `evaluator(shard) -> tensor [2N-1]`
    replaces this library's evaluation of the shard (the CPU tests pass the
    oracle); the all-reduce runs on whatever device that tensor lives on
    (NCCL for CUDA tensors).  Repeated evaluations of one problem use
    ShardedContext, which keeps the shard resident."""
    import torch.distributed as dist
    if evaluator is None:
        sc = ShardedContext(w, precision, group=group, device=device)
        try:
            return sc.evaluate().clone()
        finally:
            sc.close()
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    lo, hi = pattern_shard(w.n_patterns, rank, world)
    vec = evaluator(w.with_patterns(lo, hi))
    dist.all_reduce(vec, op=dist.ReduceOp.SUM, group=group)
    return vec
