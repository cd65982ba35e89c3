"""Pins for the oracle's branch-parameterisation chain rules (Methods: a
branch length is the difference of the parent's and the child's node
heights times a possibly branch-specific rate; a strict clock reduces the
branch derivatives over a set of branches): central finite differences of
the oracle's log-likelihood in the heights, rates, times and the clock rate,
and the invariance of log P to a common shift of every node height."""
import numpy as np

import synth
from oracle import phylo_oracle as O


def _problem(seed=3, n_tips=7):
    rng = np.random.default_rng(seed)
    w = synth.small_workload(n_tips, 4, 4, 40, seed=seed)
    parent = w.parent
    n = len(parent)
    kids, root = O.tree_children(parent)
    heights = np.zeros(n)
    heights[:n_tips] = rng.uniform(0.0, 0.05, n_tips)  # tips sampled at different times
    for v in O.postorder_list(parent):
        if kids[v]:
            heights[v] = max(heights[c] for c in kids[v]) + rng.exponential(0.08)
    rates = rng.uniform(0.5, 2.0, n - 1)
    return w, heights, rates


def _logl(w, t):
    return O.log_likelihood(w.parent, t, w.Q, w.pi, w.rates, w.weights,
                            w.pattern_weights, tip_states=w.tip_states)


def _grad(w, t):
    return O.evaluate(w.parent, t, w.Q, w.pi, w.rates, w.weights,
                      w.pattern_weights, tip_states=w.tip_states)[1]


def _central(f, x, i, h):
    xp, xm = x.copy(), x.copy()
    xp[i] += h
    xm[i] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_heights_chain_rule_matches_finite_differences():
    w, heights, rates = _problem()
    t = O.lengths_from_heights(w.parent, heights, rates)
    dh = O.chain_heights(w.parent, _grad(w, t), rates)
    f = lambda h: _logl(w, O.lengths_from_heights(w.parent, h, rates))
    for k in range(len(heights)):
        fd = _central(f, heights, k, 1e-6)
        assert abs(fd - dh[k]) <= 1e-6 * max(1.0, abs(dh[k])), (k, fd, dh[k])


def test_heights_gradient_sums_to_zero():
    # shifting every height (tips included) leaves every branch length alone
    w, heights, rates = _problem(seed=4)
    t = O.lengths_from_heights(w.parent, heights, rates)
    g = _grad(w, t)
    dh = O.chain_heights(w.parent, g, rates)
    assert abs(dh.sum()) <= 1e-12 * np.sum(np.abs(rates * g))


def test_rate_time_chain_rule_matches_finite_differences():
    w, heights, rates = _problem(seed=5)
    times = O.lengths_from_heights(w.parent, heights)  # durations
    g = _grad(w, rates * times)
    d_rates, d_times = O.chain_rate_time(g, rates, times)
    for i in [0, 3, len(rates) - 1]:
        fd_r = _central(lambda r: _logl(w, r * times), rates, i, 1e-6)
        fd_t = _central(lambda tt: _logl(w, rates * tt), times, i, 1e-7)
        assert abs(fd_r - d_rates[i]) <= 1e-6 * max(1.0, abs(d_rates[i]))
        assert abs(fd_t - d_times[i]) <= 1e-6 * max(1.0, abs(d_times[i]))


def test_strict_clock_reduction_matches_finite_differences():
    w, heights, _ = _problem(seed=6)
    times = O.lengths_from_heights(w.parent, heights)
    rho = 1.7
    g = _grad(w, rho * times)
    d_rho = O.branch_sum(g, np.arange(len(times)), times)
    fd = (_logl(w, (rho + 1e-6) * times) - _logl(w, (rho - 1e-6) * times)) / 2e-6
    assert abs(fd - d_rho) <= 1e-6 * max(1.0, abs(d_rho))
    # Euler: a common scale of every length, so rho d/d rho = sum_i t_i g_i
    assert abs(rho * d_rho - np.sum(rho * times * g)) <= 1e-12 * np.sum(np.abs(rho * times * g))


def test_branch_sum_of_a_subset():
    g = np.array([1.0, -2.0, 4.0, 0.5])
    assert O.branch_sum(g, [2, 0, 2]) == 9.0
    assert O.branch_sum(g, [1, 3], [2.0, -4.0]) == -6.0
