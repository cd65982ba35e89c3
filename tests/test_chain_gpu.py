"""GPU chain-rule epilogues (branch parameterisations of the Methods: rate x
time, node heights, strict-clock sums) through the C ABI, against the
oracle's chain rule applied to the oracle's gradient.  Tolerances are the
gradient's (tests/parity.py), propagated through the chain rule: a
derivative that combines branches i with coefficients a_i is held to
max(rel |ref|, cond * sum_i |a_i| B_i)."""
import numpy as np
import pytest

import synth
from oracle import phylo_oracle as O
from parity import TOL, oracle_eval

pytestmark = pytest.mark.gpu


def _setup(S, seed):
    rng = np.random.default_rng(seed)
    w = synth.small_workload(24, S, 4, 150, seed=seed)
    kids, root = O.tree_children(w.parent)
    n = len(w.parent)
    heights = np.zeros(n)
    heights[:w.n_tips] = rng.uniform(0.0, 0.05, w.n_tips)
    for v in O.postorder_list(w.parent):
        if kids[v]:
            heights[v] = max(heights[c] for c in kids[v]) + rng.exponential(0.06)
    rates = rng.uniform(0.5, 2.0, n - 1)
    return w, heights, rates


def _check(got, ref, scale, precision, what):
    tol = TOL[precision]
    got, ref, scale = np.asarray(got), np.asarray(ref), np.asarray(scale)
    bound = np.maximum(tol["g_rel"] * np.abs(ref), tol["g_cond"] * scale)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (what, float(np.max(err / np.maximum(bound, 1e-300))))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("S", [4, 20, 61])
def test_chain_rules_match_oracle(S, precision):
    import paper_2303_04390_gb300 as pg
    w, heights, rates = _setup(S, seed=40 + S)
    times = O.lengths_from_heights(w.parent, heights)
    t = rates * times
    _, g_ref, _, B = oracle_eval(w, t=t)
    ctx = pg.from_workload(w, precision)
    ctx.set_branch_lengths(t)
    ctx.evaluate()
    dr, dt = ctx.gradient_rate_time(rates, times)
    r_ref, t_ref = O.chain_rate_time(g_ref, rates, times)
    _check(dr, r_ref, np.abs(times) * B, precision, "d/d rates")
    _check(dt, t_ref, np.abs(rates) * B, precision, "d/d times")
    dh = ctx.gradient_heights(rates)
    h_ref = O.chain_heights(w.parent, g_ref, rates)
    h_scale = np.zeros(len(w.parent))
    for i, p in enumerate(w.parent):  # sum of |coefficient| B over the branches at each node
        if p >= 0:
            h_scale[i] += abs(rates[i]) * B[i]
            h_scale[p] += abs(rates[i]) * B[i]
    _check(dh, h_ref, h_scale, precision, "d/d heights")
    allb = np.arange(len(t))
    s = ctx.gradient_branch_sum(allb, times)
    _check([s], [O.branch_sum(g_ref, allb, times)], [np.sum(np.abs(times) * B)], precision,
           "strict clock")
    sub = np.array([3, 0, 7, 3], dtype=np.int32)
    s2 = ctx.gradient_branch_sum(sub)
    _check([s2], [O.branch_sum(g_ref, sub)], [np.sum(B[sub])], precision, "subset sum")
    ctx.close()


def test_device_form_equals_host_form():
    import torch
    import paper_2303_04390_gb300 as pg
    w, heights, rates = _setup(4, seed=60)
    times = O.lengths_from_heights(w.parent, heights)
    ctx = pg.from_workload(w, "fp32")
    ctx.set_branch_lengths(rates * times)
    ctx.evaluate()
    dr, dt = ctx.gradient_rate_time(rates, times)
    dh = ctx.gradient_heights(rates)
    s = ctx.gradient_branch_sum(np.arange(len(times)), times)
    dev = torch.device("cuda")
    r_d = torch.tensor(rates, device=dev)
    t_d = torch.tensor(times, device=dev)
    dr_d, dt_d = ctx.gradient_rate_time(r_d, t_d)
    dh_d = ctx.gradient_heights(r_d)
    s_d = ctx.gradient_branch_sum(torch.arange(len(times), device=dev), t_d)
    torch.cuda.synchronize()
    assert np.array_equal(dr_d.cpu().numpy(), dr) and np.array_equal(dt_d.cpu().numpy(), dt)
    assert np.array_equal(dh_d.cpu().numpy(), dh)
    assert float(s_d.cpu()[0]) == s
    ctx.close()


def test_chain_rules_need_an_evaluation_and_valid_branches():
    import paper_2303_04390_gb300 as pg
    from paper_2303_04390_gb300._native import PHYLO_EINVAL, PHYLO_ESTATE, PhyloError
    w, heights, rates = _setup(4, seed=61)
    ctx = pg.from_workload(w, "fp32")
    with pytest.raises(PhyloError) as e:
        ctx.gradient_heights(rates)
    assert e.value.code == PHYLO_ESTATE
    ctx.evaluate()
    with pytest.raises(PhyloError) as e:
        ctx.gradient_branch_sum(np.array([0, 2 * w.n_tips - 2], dtype=np.int32))
    assert e.value.code == PHYLO_EINVAL
    with pytest.raises(PhyloError) as e:
        ctx.gradient_rate_time(np.full(2 * w.n_tips - 2, np.nan), np.ones(2 * w.n_tips - 2))
    assert e.value.code == PHYLO_EINVAL
    assert ctx.gradient_branch_sum(np.zeros(0, dtype=np.int32)) == 0.0
    ctx.close()
