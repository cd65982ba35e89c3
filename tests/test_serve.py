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
