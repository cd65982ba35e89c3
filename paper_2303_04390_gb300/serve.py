"""Continuous-batching request loop for likelihood-and-gradient evaluations.

Each request asks for log P(Y) and the full branch-length gradient of one
problem (tree, alignment, model, branch lengths) -- one leapfrog step of
one of many concurrent HMC chains, or a one-shot evaluation.  The loop:
  - takes requests as they arrive (wall-clock arrival times, or submitted
    by a client while the loop runs);
  - keeps a session's problem resident on the device: a request carrying a
    session key (a client, a chain) reuses that session's library context
    (workspace, tree schedule, eigen split, tip data, CUDA graph), so a
    repeated step costs one branch-length upload, one graph replay and one
    read-back; idle sessions are evicted least-recently-used when memory
    is needed;
  - admits a waiting request when a slot is free and its device footprint
    (phylo_workspace_bytes) fits in the memory budget beside everything
    resident; a request larger than the whole budget is rejected;
  - sets new contexts up on worker threads and launches each evaluation
    asynchronously on its own CUDA stream, so the work of different
    requests overlaps on the device while earlier ones are still running;
  - polls completion with CUDA events, returns the result, frees one-shot
    contexts, and admits more -- new arrivals join between polls, not at
    batch boundaries;
  - fails a request, without touching the others, when its deadline
    passes, when it is cancelled, when its context cannot be allocated,
    or when its input or the device flags it; a request already on the
    device when its deadline passes or it is cancelled gets its error at
    once, and its slot and memory are released when its device work ends;
  - records per-request latency (arrival to result on the host).

Requests of different problems are not fused into shared launches: each
problem's level schedule differs (tree shape, pattern count, state count),
and the level kernels already fill the GPU at the sizes served here, so
concurrent streams recover the device time that one small problem leaves
idle (the bench reports the served throughput beside the sum of the
requests' device times measured alone).

The device work goes through a backend (TorchBackend: the library on the
current GPU); tests of the host logic substitute a fake.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Any, Dict, Hashable, List, Optional

import numpy as np


@dataclasses.dataclass
class Result:
    request_id: int
    log_likelihood: Optional[float]
    gradient: Optional[np.ndarray]
    latency_s: float
    error: Optional[str] = None
    session_hit: bool = False  # served by a resident session context


@dataclasses.dataclass
class Request:
    """One evaluation.  `workload` is the problem (a synth.Workload-like
    object: parent, tip_states, pattern_weights, Q, pi, rates, weights, t);
    `t` replaces its branch lengths; requests with the same `session` key
    are steps of one client on the same problem (same tree, data and
    model), served by a context kept resident between them; `deadline_s`
    (from arrival) bounds the wait for the result."""
    workload: Any
    t: Optional[np.ndarray] = None
    session: Optional[Hashable] = None
    deadline_s: Optional[float] = None


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

    def fits_now(self, footprint: int) -> bool:
        return self.used + footprint <= self.budget

    def take_memory(self, footprint: int) -> None:
        self.used += footprint
        self.peak_used = max(self.peak_used, self.used)

    def give_memory(self, footprint: int) -> None:
        self.used -= footprint
        assert self.used >= 0

    def take_slot(self) -> bool:
        if self.active >= self.max_active:
            return False
        self.active += 1
        self.peak_active = max(self.peak_active, self.active)
        return True

    def give_slot(self) -> None:
        self.active -= 1
        assert self.active >= 0

    def try_admit(self, footprint: int) -> bool:
        if self.active >= self.max_active or not self.fits_now(footprint):
            return False
        self.take_slot()
        self.take_memory(footprint)
        return True

    def release(self, footprint: int) -> None:
        self.give_memory(footprint)
        self.give_slot()


class TorchBackend:
    """The library on the current CUDA device: contexts over workspaces
    from PyTorch's allocator, one stream per slot, CUDA events."""

    def __init__(self, n_streams: int, precision: str, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        self.precision = precision
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_streams)]

    def footprint(self, w) -> int:
        from .context import workspace_bytes
        return workspace_bytes(w.n_tips, w.n_patterns, w.n_states,
                               w.n_categories, self.precision) + 256

    def create(self, w, stream_index: int, resident: bool):
        """A context with every input of `w` set (graph capture for a
        resident session; direct launches for a one-shot context).  Raises
        on invalid input or when the workspace cannot be allocated."""
        from .context import from_workload
        stream = self.streams[stream_index]
        ctx = from_workload(w, self.precision, device=self.device, stream=stream,
                            use_graph=resident)
        torch = self.torch
        ctx._serve_out = torch.empty(2 * w.n_tips - 1, dtype=torch.float64,
                                     device=self.device)
        ctx._serve_host = torch.empty(2 * w.n_tips - 1, dtype=torch.float64,
                                      pin_memory=True)
        ctx._serve_t = torch.empty(2 * w.n_tips - 2, dtype=torch.float64,
                                   pin_memory=True)
        ctx._serve_stream = stream
        return ctx

    def launch(self, ctx, t):
        """Asynchronous: new branch lengths (None: keep), one evaluation,
        and the read-back; returns a handle for poll/result."""
        torch = self.torch
        if t is not None:
            ctx._serve_t.copy_(torch.from_numpy(np.ascontiguousarray(t, dtype=np.float64)))
            ctx.set_branch_lengths(ctx._serve_t)
        ctx.evaluate_device(ctx._serve_out)
        with torch.cuda.stream(ctx._serve_stream):
            ctx._serve_host.copy_(ctx._serve_out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(ctx._serve_stream)
        return ev

    def done(self, handle) -> bool:
        return handle.query()

    def result(self, ctx):
        ctx.check()  # the stream has reached the event: no wait
        vals = ctx._serve_host.numpy()
        return float(vals[0]), vals[1:].copy()

    def close(self, ctx) -> None:
        ctx.close()


class _Session:
    __slots__ = ("key", "ctx", "footprint", "shape", "busy", "ready", "stream")

    def __init__(self, key, footprint, shape, stream):
        self.key, self.footprint, self.shape, self.stream = key, footprint, shape, stream
        self.ctx = None
        self.busy = False   # a request of this session is being served
        self.ready = False  # context set up


class _Slot:
    __slots__ = ("rid", "arrival", "deadline", "footprint", "future", "ctx", "handle",
                 "session", "hit", "answered", "t")

    def __init__(self, rid, arrival, deadline, footprint, session, t):
        self.rid, self.arrival, self.deadline = rid, arrival, deadline
        self.footprint, self.session, self.t = footprint, session, t
        self.future = self.ctx = self.handle = None
        self.hit = False
        self.answered = False  # its Result was already given (deadline, cancel)


def _shape(w):
    return (w.n_tips, w.n_patterns, w.n_states, w.n_categories)


class Server:
    """See the module docstring.  `precision` applies to every request.
    `session_budget_bytes` caps the memory resident sessions may keep
    between their requests (default: the whole budget)."""

    def __init__(self, memory_budget_bytes: int, max_active: int = 32,
                 n_streams: int = 16, setup_workers: int = 4,
                 precision: str = "fp32", device=None, backend=None):
        self.backend = backend or TorchBackend(n_streams, precision, device)
        self.n_streams = n_streams
        self.admission = Admission(memory_budget_bytes, max_active)
        self.precision = precision
        self._next_stream = 0
        self.pool = cf.ThreadPoolExecutor(max_workers=setup_workers)
        self._sessions: "collections.OrderedDict[Hashable, _Session]" = collections.OrderedDict()
        self._cancel_lock = threading.Lock()
        self._cancelled: set = set()
        self.evictions = 0
        self.session_hits = 0

    # -- public --------------------------------------------------------------
    def cancel(self, request_id: int) -> None:
        """Cancel a request (thread-safe; takes effect at the next poll)."""
        with self._cancel_lock:
            self._cancelled.add(request_id)

    def resident_sessions(self) -> List[Hashable]:
        return [k for k, s in self._sessions.items() if s.ready]

    def drop_session(self, key) -> None:
        """Release a session's resident context (it must be idle)."""
        s = self._sessions.get(key)
        if s is not None and not s.busy:
            self._evict(s)

    def close(self):
        self.pool.shutdown(wait=True)
        for s in list(self._sessions.values()):
            if s.ready and not s.busy:
                self._evict(s)

    def footprint(self, w) -> int:
        return self.backend.footprint(w)

    # -- internals -----------------------------------------------------------
    def _stream_index(self) -> int:
        i = self._next_stream % self.n_streams
        self._next_stream += 1
        return i

    def _evict(self, s: _Session) -> None:
        if s.ctx is not None:
            self.backend.close(s.ctx)
            s.ctx = None
        self.admission.give_memory(s.footprint)
        del self._sessions[s.key]
        self.evictions += 1

    def _make_room(self, need: int) -> bool:
        """Evict idle sessions, least recently used first, until `need`
        bytes fit; False if they cannot."""
        while not self.admission.fits_now(need):
            victim = next((s for s in self._sessions.values()
                           if s.ready and not s.busy), None)
            if victim is None:
                return False
            self._evict(victim)
        return True

    def _setup(self, w, stream_index, resident):
        return self.backend.create(w, stream_index, resident)

    def run(self, requests, arrivals: Optional[List[float]] = None,
            poll_sleep_s: float = 50e-6, follow_up=None) -> List[Result]:
        """Serve `requests` (Request objects, or bare workloads for one-shot
        evaluations) arriving at the given offsets in seconds from now (all
        at 0 when None).  `follow_up(request_id, result)` may return a new
        Request, which arrives at once and gets the next request id (a
        closed-loop client: an HMC chain's next step).  Returns the results
        in request-id order."""
        reqs = [r if isinstance(r, Request) else Request(r) for r in requests]
        n = len(reqs)
        arrivals = [0.0] * n if arrivals is None else list(arrivals)
        order = sorted(range(n), key=lambda i: arrivals[i])
        future_q = collections.deque(order)
        waiting: "collections.deque[int]" = collections.deque()
        new_arrivals: List[int] = []
        active: List[_Slot] = []
        results: List[Optional[Result]] = [None] * n
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def answer(rid, ll, g, err, hit=False):
            if results[rid] is not None:
                return
            results[rid] = Result(rid, ll, g, now() - arrivals[rid], err, hit)
            nxt = follow_up(rid, results[rid]) if follow_up else None
            if nxt is not None:
                reqs.append(nxt)
                arrivals.append(now())
                results.append(None)
                new_arrivals.append(len(reqs) - 1)

        while future_q or waiting or active or new_arrivals:
            tnow = now()
            while future_q and arrivals[future_q[0]] <= tnow:
                waiting.append(future_q.popleft())
            waiting.extend(new_arrivals)
            new_arrivals.clear()
            with self._cancel_lock:
                cancelled = set(self._cancelled)
            # -- waiting requests: cancellation, deadlines, admission ------
            still_waiting = collections.deque()
            blocked = False
            for rid in waiting:
                rq = reqs[rid]
                if rid in cancelled:
                    answer(rid, None, None, "cancelled")
                    continue
                if rq.deadline_s is not None and tnow > arrivals[rid] + rq.deadline_s:
                    answer(rid, None, None, "deadline exceeded before launch")
                    continue
                if blocked:
                    still_waiting.append(rid)
                    continue
                admitted = self._admit(rid, rq, arrivals[rid], active, answer)
                if admitted is None:  # cannot start now: keep arrival order
                    still_waiting.append(rid)
                    blocked = True
            waiting = still_waiting
            # -- active requests ------------------------------------------
            still = []
            for s in active:
                rq = reqs[s.rid]
                if not s.answered:
                    if s.rid in cancelled:
                        answer(s.rid, None, None, "cancelled")
                        s.answered = True
                    elif s.deadline is not None and now() > s.deadline:
                        answer(s.rid, None, None, "deadline exceeded")
                        s.answered = True
                if s.handle is None and s.future is not None and s.future.done():
                    try:
                        ctx = s.future.result()
                    except Exception as e:  # invalid input, allocation failure
                        answer(s.rid, None, None, _describe(e))
                        self._finish(s, failed=True)
                        continue
                    s.future = None
                    s.ctx = ctx
                    if s.session is not None:
                        s.session.ctx = ctx
                        s.session.ready = True
                    try:
                        s.handle = self.backend.launch(ctx, s.t)
                    except Exception as e:
                        answer(s.rid, None, None, _describe(e))
                        self._finish(s, failed=True)
                        continue
                if s.handle is not None and self.backend.done(s.handle):
                    try:
                        ll, g = self.backend.result(s.ctx)
                        answer(s.rid, ll, g, None, s.hit)
                    except Exception as e:  # device-side numeric flag
                        answer(s.rid, None, None, _describe(e))
                    self._finish(s, failed=False)
                    continue
                still.append(s)
            active = still
            if (active or waiting or future_q) and not new_arrivals:
                time.sleep(poll_sleep_s)
        with self._cancel_lock:
            self._cancelled.clear()
        return results

    def _admit(self, rid, rq: Request, arrival: float, active: List[_Slot], answer):
        """Start request `rid` if a slot and memory allow.  Returns True if
        started, False if it was answered (rejected), None if it must wait."""
        w = rq.workload
        deadline = None if rq.deadline_s is None else arrival + rq.deadline_s
        try:
            fp = self.footprint(w)
        except Exception as e:  # invalid shape
            answer(rid, None, None, f"rejected: {_describe(e)}")
            return False
        if not self.admission.fits_ever(fp):
            answer(rid, None, None,
                   f"rejected: needs {fp} bytes, budget {self.admission.budget}")
            return False
        if rq.session is not None:
            s = self._sessions.get(rq.session)
            if s is not None and s.shape != _shape(w):
                answer(rid, None, None, "rejected: session problem shape changed")
                return False
            if s is not None:
                if s.busy:
                    return None  # the session's previous step is still running
                if not self.admission.take_slot():
                    return None
                s.busy = True
                self._sessions.move_to_end(s.key)
                slot = _Slot(rid, arrival, deadline, 0, s, rq.t)
                slot.ctx, slot.hit = s.ctx, True
                self.session_hits += 1
                try:
                    slot.handle = self.backend.launch(s.ctx, rq.t)
                except Exception as e:
                    answer(rid, None, None, _describe(e))
                    self._finish(slot, failed=True)
                    return False
                active.append(slot)
                return True
            # a new session: its memory stays taken until evicted
            if self.admission.active >= self.admission.max_active or not self._make_room(fp):
                return None
            self.admission.take_slot()
            self.admission.take_memory(fp)
            s = _Session(rq.session, fp, _shape(w), self._stream_index())
            s.busy = True
            self._sessions[rq.session] = s
            slot = _Slot(rid, arrival, deadline, 0, s, rq.t)
            slot.future = self.pool.submit(self._setup, w, s.stream, True)
            active.append(slot)
            return True
        # one shot
        if self.admission.active >= self.admission.max_active or not self._make_room(fp):
            return None
        self.admission.try_admit(fp)
        slot = _Slot(rid, arrival, deadline, fp, None, rq.t)
        slot.future = self.pool.submit(self._setup, w, self._stream_index(), False)
        active.append(slot)
        return True

    def _finish(self, s: _Slot, failed: bool) -> None:
        """Release a request's slot; one-shot contexts and their memory go,
        a session's context stays resident unless its setup failed."""
        if s.session is not None:
            sess = s.session
            sess.busy = False
            if failed and not sess.ready:  # setup failed: nothing resident
                if s.ctx is not None:
                    self.backend.close(s.ctx)
                self.admission.give_memory(sess.footprint)
                self._sessions.pop(sess.key, None)
            self.admission.give_slot()
            return
        if s.ctx is not None:
            self.backend.close(s.ctx)
            s.ctx = None
        self.admission.release(s.footprint)


def _describe(e: Exception) -> str:
    name = type(e).__name__
    if "OutOfMemory" in name or isinstance(e, MemoryError):
        return f"device memory: {e}"
    return str(e) or name


def latency_summary(results: List[Result], elapsed_s: float) -> Dict[str, Any]:
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
