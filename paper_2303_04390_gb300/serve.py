"""Continuous-batching request loop for likelihood-and-gradient evaluations.

Each request is one problem (tree, alignment, model, branch lengths) whose
log P(Y) and full branch-length gradient are wanted -- e.g. one leapfrog
step of one of many concurrent HMC chains, or a one-shot evaluation.  The
loop:
  - takes requests as they arrive (wall-clock arrival times);
  - admits a waiting request when a slot is free and its device footprint
    (phylo_workspace_bytes) fits in the memory budget next to the requests
    already resident; a request larger than the whole budget is rejected;
  - sets admitted requests up on worker threads (context, uploads) and
    launches each evaluation asynchronously on its own CUDA stream, so the
    work of different requests overlaps on the device while earlier ones
    are still running;
  - polls completion with CUDA events, returns the result, frees the slot
    and its memory, and admits more -- new arrivals join between polls, not
    at batch boundaries;
  - records per-request latency (arrival to result on the host).

A request that fails (malformed input, device-side numeric flag) returns
its error and does not disturb the others.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Result:
    request_id: int
    log_likelihood: Optional[float]
    gradient: Optional[np.ndarray]
    latency_s: float
    error: Optional[str] = None


class Admission:
    """Slot and memory-budget bookkeeping (host logic only)."""

    def __init__(self, budget_bytes: int, max_active: int):
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.used = 0
        self.active = 0
        self.peak_used = 0
        self.peak_active = 0

    def fits_ever(self, footprint: int) -> bool:
        return footprint <= self.budget

    def try_admit(self, footprint: int) -> bool:
        if self.active >= self.max_active or self.used + footprint > self.budget:
            return False
        self.used += footprint
        self.active += 1
        self.peak_used = max(self.peak_used, self.used)
        self.peak_active = max(self.peak_active, self.active)
        return True

    def release(self, footprint: int) -> None:
        self.used -= footprint
        self.active -= 1
        assert self.used >= 0 and self.active >= 0


class _Slot:
    __slots__ = ("rid", "arrival", "footprint", "future", "ctx", "host", "event")

    def __init__(self, rid, arrival, footprint, future):
        self.rid, self.arrival, self.footprint = rid, arrival, footprint
        self.future = future
        self.ctx = self.host = self.event = None


class Server:
    """See the module docstring.  `precision` applies to every request."""

    def __init__(self, memory_budget_bytes: int, max_active: int = 32,
                 n_streams: int = 16, setup_workers: int = 4,
                 precision: str = "fp32", device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        self.admission = Admission(memory_budget_bytes, max_active)
        self.precision = precision
        self.streams = [torch.cuda.Stream(device=self.device)
                        for _ in range(n_streams)]
        self._next_stream = 0
        self.pool = cf.ThreadPoolExecutor(max_workers=setup_workers)
        self._lock = threading.Lock()

    def close(self):
        self.pool.shutdown(wait=True)

    # -- one request ---------------------------------------------------------
    def _setup_and_launch(self, w, stream):
        from .context import from_workload
        torch = self.torch
        # The workspace comes from the allocator's default-stream pool (so
        # any request can reuse it); it is released only after this
        # request's event has completed.
        ctx = from_workload(w, self.precision, device=self.device,
                            stream=stream, use_graph=False)
        out = torch.empty(2 * w.n_tips - 1, dtype=torch.float64,
                          device=self.device)
        ctx.evaluate_device(out)
        host = torch.empty(out.numel(), dtype=torch.float64, pin_memory=True)
        with torch.cuda.stream(stream):
            host.copy_(out, non_blocking=True)
            event = torch.cuda.Event()
            event.record(stream)
        ctx._serve_out = out  # keep alive until the event completes
        return ctx, host, event

    def footprint(self, w) -> int:
        from .context import workspace_bytes
        return workspace_bytes(w.n_tips, w.n_patterns, w.n_states,
                               w.n_categories, self.precision) + 256

    # -- the loop ------------------------------------------------------------
    def run(self, workloads, arrivals: Optional[List[float]] = None,
            poll_sleep_s: float = 50e-6) -> List[Result]:
        """Serve `workloads` (synth.Workload-like objects) arriving at the
        given offsets in seconds from now (all at 0 when None).  Returns
        the results in request order."""
        n = len(workloads)
        arrivals = [0.0] * n if arrivals is None else list(arrivals)
        order = sorted(range(n), key=lambda i: arrivals[i])
        future_q = collections.deque(order)
        waiting = collections.deque()
        active: List[_Slot] = []
        results: List[Optional[Result]] = [None] * n
        t0 = time.perf_counter()
        while future_q or waiting or active:
            now = time.perf_counter() - t0
            while future_q and arrivals[future_q[0]] <= now:
                waiting.append(future_q.popleft())
            # admit in arrival order while slots and memory allow
            while waiting:
                rid = waiting[0]
                try:
                    fp = self.footprint(workloads[rid])
                except Exception as e:  # invalid shape
                    waiting.popleft()
                    results[rid] = Result(rid, None, None, now - arrivals[rid],
                                          f"rejected: {e}")
                    continue
                if not self.admission.fits_ever(fp):
                    waiting.popleft()
                    results[rid] = Result(
                        rid, None, None, now - arrivals[rid],
                        f"rejected: needs {fp} bytes, budget "
                        f"{self.admission.budget}")
                    continue
                if not self.admission.try_admit(fp):
                    break
                waiting.popleft()
                stream = self.streams[self._next_stream % len(self.streams)]
                self._next_stream += 1
                fut = self.pool.submit(self._setup_and_launch, workloads[rid],
                                       stream)
                active.append(_Slot(rid, arrivals[rid], fp, fut))
            # completions
            still = []
            for s in active:
                if s.ctx is None and s.future.done():
                    try:
                        s.ctx, s.host, s.event = s.future.result()
                    except Exception as e:
                        results[s.rid] = Result(
                            s.rid, None, None,
                            time.perf_counter() - t0 - s.arrival, str(e))
                        self.admission.release(s.footprint)
                        continue
                if s.event is not None and s.event.query():
                    err = None
                    try:
                        s.ctx.check()
                    except Exception as e:
                        err = str(e)
                    vals = s.host.numpy()
                    lat = time.perf_counter() - t0 - s.arrival
                    results[s.rid] = Result(
                        s.rid, None if err else float(vals[0]),
                        None if err else vals[1:].copy(), lat, err)
                    s.ctx.close()
                    s.ctx = s.host = s.event = None
                    self.admission.release(s.footprint)
                    continue
                still.append(s)
            active = still
            if active or waiting or future_q:
                time.sleep(poll_sleep_s)
        return results


def latency_summary(results: List[Result], elapsed_s: float) -> dict:
    ok = [r for r in results if r.error is None]
    lat = np.array([r.latency_s for r in ok]) if ok else np.zeros(1)
    return {
        "requests": len(results),
        "completed": len(ok),
        "failed": len(results) - len(ok),
        "evals_per_s": len(ok) / elapsed_s if elapsed_s > 0 else None,
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "max_ms": float(lat.max() * 1e3),
    }


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 0) -> List[float]:
    rng = np.random.default_rng(seed)
    return list(np.cumsum(rng.exponential(1.0 / rate_per_s, size=n)))
