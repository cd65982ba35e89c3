"""The serving loop: admission bookkeeping on the host (CPU tests), and on
the GPU that every result is the same alone and in a concurrent mix, that
the memory budget holds, and that a failing request does not disturb the
others."""
import numpy as np
import pytest

import synth
from paper_2303_04390_gb300.serve import Admission, poisson_arrivals


def test_admission_budget_and_slots():
    a = Admission(budget_bytes=100, max_active=2)
    assert a.try_admit(60)
    assert not a.try_admit(50)          # memory
    assert a.try_admit(40)
    assert not a.try_admit(0)           # slots
    a.release(60)
    assert a.try_admit(10)
    assert a.peak_used == 100 and a.peak_active == 2
    assert not a.fits_ever(101) and a.fits_ever(100)
    a.release(40)
    a.release(10)
    assert a.used == 0 and a.active == 0


def test_poisson_arrivals_are_increasing_with_the_right_rate():
    t = poisson_arrivals(20000, rate_per_s=500.0, seed=3)
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 500.0) / 500.0 < 0.03


# --------------------------------------------------------------------------
# Host logic of the server with a fake backend (no GPU): sessions, LRU
# eviction, deadlines, cancellation, allocation failure, closed-loop chains.
# --------------------------------------------------------------------------

class _FakeOOM(Exception):
    """Stands in for torch.cuda.OutOfMemoryError (matched by name)."""


_FakeOOM.__name__ = "OutOfMemoryError"


class _Prob:
    """A fake problem: its footprint, set-up and run times, and its value."""

    def __init__(self, name, footprint=100, setup_s=0.0, run_s=0.002, fail_alloc=False,
                 flag=False, shape=(8, 10, 4, 4)):
        self.name, self.fp, self.setup_s, self.run_s = name, footprint, setup_s, run_s
        self.fail_alloc, self.flag = fail_alloc, flag
        self.n_tips, self.n_patterns, self.n_states, self.n_categories = shape
        self.t = np.ones(2 * self.n_tips - 2)


class _FakeBackend:
    def __init__(self):
        import threading
        self.created, self.closed, self.launched = [], [], []
        self.lock = threading.Lock()

    def footprint(self, w):
        return w.fp

    def create(self, w, stream_index, resident):
        import time
        time.sleep(w.setup_s)
        if w.fail_alloc:
            raise _FakeOOM("fake: no device memory for the workspace")
        with self.lock:
            self.created.append((w.name, resident))
        return {"w": w, "t": w.t.copy()}

    def launch(self, ctx, t):
        import time
        if t is not None:
            ctx["t"] = np.asarray(t, dtype=float).copy()
        self.launched.append(ctx["w"].name)
        return time.perf_counter() + ctx["w"].run_s

    def done(self, handle):
        import time
        return time.perf_counter() >= handle

    def result(self, ctx):
        if ctx["w"].flag:
            raise RuntimeError("[-5] device flagged: zero-gradient-denominator")
        return float(np.sum(ctx["t"])), ctx["t"] * 2.0

    def close(self, ctx):
        self.closed.append(ctx["w"].name)


def _server(budget=1000, max_active=8):
    from paper_2303_04390_gb300.serve import Server
    be = _FakeBackend()
    return Server(memory_budget_bytes=budget, max_active=max_active, n_streams=4,
                  backend=be), be


def test_sessions_stay_resident_and_are_reused():
    from paper_2303_04390_gb300.serve import Request
    srv, be = _server()
    a, b = _Prob("a"), _Prob("b")
    reqs = [Request(a, t=np.full(14, 1.0), session="A"),
            Request(b, t=np.full(14, 2.0), session="B"),
            Request(a, t=np.full(14, 3.0), session="A"),
            Request(a, t=np.full(14, 4.0), session="A")]
    res = srv.run(reqs, arrivals=[0.0, 0.0, 0.02, 0.04])
    assert [r.error for r in res] == [None] * 4
    assert [r.log_likelihood for r in res] == [14.0, 28.0, 42.0, 56.0]
    assert [r.session_hit for r in res] == [False, False, True, True]
    assert sorted(be.created) == [("a", True), ("b", True)]  # one context each
    assert srv.resident_sessions() == ["A", "B"] or set(srv.resident_sessions()) == {"A", "B"}
    assert srv.admission.used == 200 and srv.admission.active == 0
    srv.close()
    assert srv.admission.used == 0 and sorted(be.closed) == ["a", "b"]


def test_idle_sessions_are_evicted_least_recently_used():
    from paper_2303_04390_gb300.serve import Request
    srv, be = _server(budget=250)
    p = {k: _Prob(k, footprint=100) for k in "abc"}
    order = ["a", "b", "a", "c", "b"]  # c evicts b (a was used after b); b evicts a
    res = srv.run([Request(p[k], session=k) for k in order],
                  arrivals=[0.01 * i for i in range(len(order))])
    assert all(r.error is None for r in res)
    assert srv.admission.peak_used <= 250
    assert be.closed == ["b", "a"]
    assert set(srv.resident_sessions()) == {"c", "b"}
    assert [r.session_hit for r in res] == [False, False, True, False, False]
    srv.close()


def test_deadlines_before_and_after_launch():
    from paper_2303_04390_gb300.serve import Request
    srv, be = _server(max_active=1)
    slow = _Prob("slow", run_s=0.20)
    quick = _Prob("quick", run_s=0.001)
    reqs = [Request(slow, deadline_s=0.05),   # on the device past its deadline
            Request(quick, deadline_s=0.03),  # waits for the slot past its deadline
            Request(quick)]                   # no deadline: served after the slow one
    res = srv.run(reqs)
    assert res[0].error == "deadline exceeded" and 0.05 <= res[0].latency_s < 0.15
    assert res[1].error == "deadline exceeded before launch"
    assert res[2].error is None and res[2].latency_s >= 0.19  # the slot came back
    assert srv.admission.active == 0 and srv.admission.used == 0
    assert be.launched == ["slow", "quick"]
    srv.close()


def test_cancellation_of_waiting_and_running_requests():
    import threading
    from paper_2303_04390_gb300.serve import Request
    srv, be = _server(max_active=1)
    long_ = _Prob("long", run_s=0.15)
    reqs = [Request(long_), Request(_Prob("w")), Request(_Prob("x"))]
    timer = threading.Timer(0.03, lambda: (srv.cancel(0), srv.cancel(1)))
    timer.start()
    res = srv.run(reqs)
    timer.join()
    assert res[0].error == "cancelled" and res[0].latency_s < 0.12
    assert res[1].error == "cancelled"
    assert res[2].error is None
    assert "w" not in be.launched
    assert srv.admission.active == 0 and srv.admission.used == 0
    srv.close()


def test_allocation_failure_and_flags_are_isolated():
    from paper_2303_04390_gb300.serve import Request
    srv, be = _server()
    good = [_Prob(f"g{k}") for k in range(4)]
    reqs = [Request(good[0]), Request(_Prob("oom", fail_alloc=True)),
            Request(good[1], session="s"), Request(_Prob("oom2", fail_alloc=True), session="t"),
            Request(_Prob("bad", flag=True)), Request(good[2]), Request(good[3])]
    res = srv.run(reqs)
    assert res[1].error.startswith("device memory:") and res[3].error.startswith("device memory:")
    assert "zero-gradient-denominator" in res[4].error
    for k in (0, 2, 5, 6):
        assert res[k].error is None
    assert srv.resident_sessions() == ["s"]  # the failed session left nothing resident
    assert srv.admission.used == 100 and srv.admission.active == 0
    srv.close()


def test_a_session_cannot_change_its_problem_shape():
    from paper_2303_04390_gb300.serve import Request
    srv, _ = _server()
    res = srv.run([Request(_Prob("a"), session="A"),
                   Request(_Prob("a2", shape=(9, 10, 4, 4)), session="A")],
                  arrivals=[0.0, 0.01])
    assert res[0].error is None and "shape changed" in res[1].error
    srv.close()


def test_closed_loop_chains_follow_up():
    from paper_2303_04390_gb300.serve import Request
    srv, be = _server()
    probs = [_Prob(f"c{k}") for k in range(3)]
    steps = {k: 0 for k in range(3)}
    owner = {}

    def follow(rid, res):
        k = owner[rid]
        steps[k] += 1
        if steps[k] < 5:
            return Request(probs[k], t=np.full(14, float(steps[k])), session=k)
        return None

    first = [Request(probs[k], session=k) for k in range(3)]
    for k in range(3):
        owner[k] = k
    # ids of follow-ups are assigned in answer order: track them as they come
    orig = follow

    def follow_tracked(rid, res):
        nxt = orig(rid, res)
        if nxt is not None:
            owner[len(owner)] = owner[rid]
        return nxt

    res = srv.run(first, follow_up=follow_tracked)
    assert len(res) == 15 and all(r.error is None for r in res)
    assert sum(r.session_hit for r in res) == 12 and len(be.created) == 3
    srv.close()


def _requests(n, seed=50):
    out = []
    for k in range(n):
        S = 4 if k % 3 else 20
        out.append(synth.small_workload(8 + 5 * k, S, 4, 60 + 37 * k,
                                        seed=seed + k))
    return out


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_04390_gb300 as pg
    from paper_2303_04390_gb300.serve import Server
    reqs = _requests(9)
    alone = []
    for w in reqs:
        ctx = pg.from_workload(w, "fp32")
        alone.append(ctx.evaluate())
        ctx.close()
    srv = Server(memory_budget_bytes=1 << 30, max_active=6, n_streams=4)
    arrivals = poisson_arrivals(len(reqs), rate_per_s=2000.0, seed=1)
    res = srv.run(reqs, arrivals)
    srv.close()
    assert srv.admission.peak_active > 1  # they did overlap
    for (ll, g), r in zip(alone, res):
        assert r.error is None, r.error
        assert r.log_likelihood == ll
        assert np.array_equal(r.gradient, g)


@pytest.mark.gpu
def test_budget_rejection_and_failure_isolation():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_04390_gb300 as pg
    from paper_2303_04390_gb300.serve import Server
    reqs = _requests(5, seed=70)
    big = synth.small_workload(200, 20, 4, 3000, seed=71)
    bad = synth.small_workload(10, 4, 4, 50, seed=72)
    bad.parent = bad.parent.copy()
    bad.parent[0] = 3  # a tip as parent: rejected by validation
    fp_small = max(pg.workspace_bytes(w.n_tips, w.n_patterns, w.n_states,
                                      w.n_categories) for w in reqs)
    budget = 2 * fp_small + 1024
    srv = Server(memory_budget_bytes=budget, max_active=8, n_streams=4)
    res = srv.run(reqs[:2] + [big, bad] + reqs[2:])
    srv.close()
    assert srv.admission.peak_used <= budget
    assert res[2].error and "rejected" in res[2].error
    assert res[3].error and "internal node" in res[3].error
    for r in res[:2] + res[4:]:
        assert r.error is None, r.error


@pytest.mark.gpu
def test_session_steps_equal_fresh_evaluations():
    """Chains served as sessions (resident contexts, graph replays, new branch
    lengths each step) give the same results, bit for bit, as a fresh
    context evaluated alone at the same branch lengths."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_04390_gb300 as pg
    from paper_2303_04390_gb300.serve import Request, Server
    probs = _requests(4, seed=80)
    rng = np.random.default_rng(3)
    steps = {k: [w.t * np.exp(0.05 * rng.standard_normal(w.t.shape)) for _ in range(4)]
             for k, w in enumerate(probs)}
    srv = Server(memory_budget_bytes=1 << 30, max_active=8, n_streams=4)
    owner, done = {}, {k: 0 for k in range(len(probs))}

    def follow(rid, res):
        k = owner[rid]
        done[k] += 1
        if done[k] < len(steps[k]):
            owner[len(owner)] = k
            return Request(probs[k], t=steps[k][done[k]], session=k)
        return None

    first = []
    for k, w in enumerate(probs):
        owner[k] = k
        first.append(Request(w, t=steps[k][0], session=k))
    res = srv.run(first, follow_up=follow)
    srv.close()
    assert len(res) == 16 and sum(r.session_hit for r in res) == 12
    seen = {k: 0 for k in range(len(probs))}
    for rid, r in enumerate(res):
        assert r.error is None, r.error
        k = owner[rid]
        ctx = pg.from_workload(probs[k], "fp32")
        ctx.set_branch_lengths(steps[k][seen[k]])
        ll, g = ctx.evaluate()
        ctx.close()
        seen[k] += 1
        assert r.log_likelihood == ll and np.array_equal(r.gradient, g)
