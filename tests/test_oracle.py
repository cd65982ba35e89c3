"""Pins for the FP64 CPU oracle: each test checks it against something other
than itself (closed forms, a library matrix exponential, brute-force
summation, finite differences, the O(N^2) substitution route, the any-node
identity of Eq. 5, rerooting, normalisation and limits). The last group
plants mistakes in the oracle and checks that a pin catches each one."""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import phylo_oracle as O


def _models(rng):
    out = [synth.jc69(), synth.hky85(4.0, rng.dirichlet([10.0] * 4)),
           synth.random_reversible(20, rng)]
    pi = rng.dirichlet(np.ones(61))
    pi = np.maximum(pi, 1e-4)
    out.append(synth.codon_gy94(2.0, 0.3, pi / pi.sum()))
    return out


# --------------------------------------------------------------- Eq. 1 ----

def test_expm_matches_library_routine():
    rng = np.random.default_rng(1)
    for Q, _ in _models(rng):
        for t in [0.0, 1e-4, 0.002, 0.05, 0.3, 2.0, 25.0]:
            ref = scipy.linalg.expm(t * Q)
            got = O.expm_taylor(t * Q)
            assert np.max(np.abs(got - ref)) < 1e-13 * max(1.0, t)


def test_jc69_closed_form():
    Q, _ = synth.jc69()
    for t in [0.0, 0.01, 0.1, 1.0, 3.0]:
        P = O.expm_taylor(t * Q)
        same = 0.25 + 0.75 * math.exp(-4.0 * t / 3.0)
        diff = 0.25 - 0.25 * math.exp(-4.0 * t / 3.0)
        expect = np.full((4, 4), diff)
        np.fill_diagonal(expect, same)
        np.testing.assert_allclose(P, expect, rtol=0, atol=1e-15)


def test_transition_matrix_properties():
    rng = np.random.default_rng(2)
    for Q, pi in _models(rng):
        S = Q.shape[0]
        np.testing.assert_array_equal(O.expm_taylor(0.0 * Q), np.eye(S))
        for s, t in [(0.01, 0.3), (0.2, 0.7), (1.0, 2.5)]:
            Ps, Pt, Pst = (O.expm_taylor(x * Q) for x in (s, t, s + t))
            np.testing.assert_allclose(Ps @ Pt, Pst, atol=1e-13)
            np.testing.assert_allclose(Pt.sum(axis=1), 1.0, atol=1e-13)
            np.testing.assert_allclose(pi @ Pt, pi, atol=1e-13)
            D = pi[:, None] * Pt
            np.testing.assert_allclose(D, D.T, atol=1e-14)
            assert Pt.min() > -1e-15


def test_large_state_spaces():
    """The 122-state Markov-modulated codon model and a 256-state model:
    P from the oracle against the library matrix exponential, P(0) = I,
    rows summing to 1, stationarity and detailed balance."""
    rng = np.random.default_rng(9)
    pi = rng.dirichlet(np.ones(61))
    pi = np.maximum(pi, 1e-4)
    for Q, pi_ in [synth.codon_mmm(2.0, (0.1, 1.0), pi / pi.sum()),
                   synth.random_reversible(256, rng)]:
        S = Q.shape[0]
        assert np.allclose(Q.sum(axis=1), 0.0, atol=1e-13)
        assert abs(-np.dot(pi_, np.diag(Q)) - 1.0) < 1e-12
        np.testing.assert_array_equal(O.expm_taylor(0.0 * Q), np.eye(S))
        for t in [1e-3, 0.05, 0.7]:
            P = O.expm_taylor(t * Q)
            np.testing.assert_allclose(P, scipy.linalg.expm(t * Q), atol=1e-13)
            np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-13)
            np.testing.assert_allclose(pi_ @ P, pi_, atol=1e-13)
            D = pi_[:, None] * P
            np.testing.assert_allclose(D, D.T, atol=1e-14)


def test_transition_derivative_by_finite_difference():
    rng = np.random.default_rng(3)
    rates = np.array([0.3, 1.7])
    for Q, _ in _models(rng):
        t, h = 0.13, 1e-5
        d = O.transition_derivatives(Q, rates, t)
        fd = (O.transition_matrices(Q, rates, t + h)
              - O.transition_matrices(Q, rates, t - h)) / (2 * h)
        np.testing.assert_allclose(d, fd, atol=1e-8)


# ------------------------------------------------------ Eqs. 2, 3, 6-8 ----

def _two_taxon_jc(rates, weights, y0, y1, t0, t1):
    """P(Y_c) and dP/dt0 for a root with two tips under JC69 (+ categories):
    L = sum_r w_r 1/4 P_{y0 y1}(gamma_r (t0 + t1))."""
    L = dL = 0.0
    for g, w in zip(rates, weights):
        e = math.exp(-4.0 * g * (t0 + t1) / 3.0)
        if y0 == y1:
            L += w * 0.25 * (0.25 + 0.75 * e)
            dL += w * 0.25 * (-g * e)
        else:
            L += w * 0.25 * (0.25 - 0.25 * e)
            dL += w * 0.25 * (g * e / 3.0)
    return L, dL


@pytest.mark.parametrize("ncat", [1, 4])
def test_two_taxon_jc69_closed_form(ncat):
    Q, pi = synth.jc69()
    rates, weights = synth.discrete_gamma(0.5, ncat)
    parent = np.array([2, 2, -1], dtype=np.int32)
    t = np.array([0.07, 0.31])
    states = np.array([[0, 0, 1, 3, 2], [0, 2, 1, 0, 2]], dtype=np.uint8)
    W = np.array([3.0, 1.0, 2.0, 5.0, 1.0])
    logL, grad, _ = O.evaluate(parent, t, Q, pi, rates, weights, W,
                               tip_states=states)
    exp_ll = exp_g = 0.0
    for c in range(states.shape[1]):
        L, dL = _two_taxon_jc(rates, weights, states[0, c], states[1, c],
                              t[0], t[1])
        exp_ll += W[c] * math.log(L)
        exp_g += W[c] * dL / L
    assert abs(logL - exp_ll) < 1e-13 * abs(exp_ll)
    # both branches enter only through t0 + t1
    np.testing.assert_allclose(grad, [exp_g, exp_g], rtol=1e-12)
    # the single-category, same-state formula written out
    if ncat == 1:
        T = t.sum()
        e = math.exp(-4 * T / 3)
        g_same = -e / (0.25 + 0.75 * e)
        g_diff = (e / 3.0) / (0.25 - 0.25 * e)
        n_same = sum(W[c] for c in range(5) if states[0, c] == states[1, c])
        n_diff = W.sum() - n_same
        assert abs(grad[0] - (n_same * g_same + n_diff * g_diff)) < 1e-12


def _golden_jc69():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "jc69_two_taxon.txt")
    return [tuple(float(x) for x in line.split()) for line in open(path)
            if line.strip() and not line.startswith("#")]


def test_golden_jc69_two_taxon():
    """The stored closed-form values (tests/golden/jc69_two_taxon.txt): one
    same-state and one different-state site on a two-taxon tree with both
    branches T/2."""
    Q, pi = synth.jc69()
    parent = np.array([2, 2, -1], dtype=np.int32)
    states = np.array([[0, 0], [0, 1]], dtype=np.uint8)
    for T, ls, dls, ld, dld in _golden_jc69():
        if ld == 0.0:
            continue
        logL, grad, _ = O.evaluate(parent, np.array([T / 2, T / 2]), Q, pi, np.ones(1),
                                   np.ones(1), np.ones(2), tip_states=states)
        want = math.log(ls) + math.log(ld)
        assert abs(logL - want) <= 1e-13 * abs(want)
        g = dls / ls + dld / ld
        np.testing.assert_allclose(grad, [g, g], rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("n_tips,n_states,ncat", [(6, 4, 2), (5, 4, 4),
                                                   (4, 20, 2), (3, 61, 2)])
def test_likelihood_matches_brute_force(n_tips, n_states, ncat):
    w = synth.small_workload(n_tips, n_states, ncat, 7, seed=11, mean_t=0.2)
    states = w.tip_states.copy()
    states[0, 1] = n_states  # a gap
    ll_sites = O.site_log_likelihoods(
        w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
        O.tip_partial_vectors(n_states, states))
    bf = O.brute_force_site_likelihoods(w.parent, w.t, w.Q, w.pi, w.rates,
                                        w.weights, tip_states=states)
    np.testing.assert_allclose(np.exp(ll_sites), bf, rtol=1e-12)


def test_pattern_probabilities_sum_to_one():
    rng = np.random.default_rng(5)
    parent = synth.yule_tree(4, rng)
    t = synth.exponential_branch_lengths(4, 0.3, rng)
    Q, pi = synth.hky85(4.0, rng.dirichlet([3.0] * 4))
    rates, weights = synth.discrete_gamma(0.5, 4)
    pats = np.array(list(itertools.product(range(4), repeat=4)),
                    dtype=np.uint8).T
    ll = O.site_log_likelihoods(parent, t, Q, pi, rates, weights,
                                O.tip_partial_vectors(4, pats))
    assert abs(np.exp(ll).sum() - 1.0) < 1e-13


@pytest.mark.parametrize("n_tips,n_states", [(12, 4), (6, 122)])
def test_any_node_identity(n_tips, n_states):
    w = synth.small_workload(n_tips, n_states, 4, 40, seed=3)
    _, _, _, det = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                              w.pattern_weights, tip_states=w.tip_states,
                              return_details=True)
    for node in range(len(w.parent)):
        np.testing.assert_allclose(
            O.node_site_log_likelihoods(det, w.weights, node),
            det["site_ll"], rtol=1e-12, atol=1e-12)


def _fd_gradient(w, h_rel=1e-4):
    """Richardson-extrapolated central differences of log P(Y)."""
    def f(tt):
        return O.log_likelihood(w.parent, tt, w.Q, w.pi, w.rates, w.weights,
                                w.pattern_weights, tip_states=w.tip_states)
    g = np.zeros_like(w.t)
    for b in range(len(w.t)):
        h = h_rel * max(w.t[b], 1e-2)

        def D(hh):
            tp, tm = w.t.copy(), w.t.copy()
            tp[b] += hh
            tm[b] -= hh
            return (f(tp) - f(tm)) / (2 * hh)
        g[b] = (4 * D(h / 2) - D(h)) / 3
    return g


@pytest.mark.parametrize("n_tips,n_states,ncat", [(8, 4, 4), (5, 20, 2),
                                                   (4, 61, 2), (4, 122, 2)])
def test_gradient_matches_finite_differences(n_tips, n_states, ncat):
    w = synth.small_workload(n_tips, n_states, ncat, 25, seed=4, mean_t=0.15)
    _, grad, abs_sum = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates,
                                  w.weights, w.pattern_weights,
                                  tip_states=w.tip_states)
    fd = _fd_gradient(w)
    assert np.all(np.abs(grad - fd) <= 1e-6 * np.maximum(abs_sum, 1.0))


def test_gradient_matches_substitution_route():
    w = synth.small_workload(16, 4, 4, 30, seed=8, mean_t=0.1)
    w.tip_states[3, 5] = 4  # gap
    _, grad, abs_sum = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates,
                                  w.weights, w.pattern_weights,
                                  tip_states=w.tip_states)
    sub = O.gradient_by_substitution(w.parent, w.t, w.Q, w.pi, w.rates,
                                     w.weights, w.pattern_weights,
                                     tip_states=w.tip_states)
    assert np.all(np.abs(grad - sub) <= 1e-12 * np.maximum(abs_sum, 1.0))


def test_root_branches_have_equal_gradient():
    """Reversible model with root = pi: only the sum of the two root branch
    lengths is identifiable, so both derivatives agree."""
    w = synth.small_workload(10, 20, 4, 30, seed=9)
    _, grad, _ = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                            w.pattern_weights, tip_states=w.tip_states)
    root = len(w.parent) - 1
    a, b = np.nonzero(w.parent == root)[0]
    assert abs(grad[a] - grad[b]) < 1e-11 * max(1.0, abs(grad[a]))


def test_zero_length_branch():
    """An unrooted tree nested in the rooted form by a zero root branch:
    P(0) = I, and the gradient there is still defined."""
    w = synth.small_workload(7, 4, 2, 20, seed=10)
    root = len(w.parent) - 1
    a, b = np.nonzero(w.parent == root)[0]
    t = w.t.copy()
    t[b] += t[a]
    t[a] = 0.0
    ll0 = O.log_likelihood(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                           w.pattern_weights, tip_states=w.tip_states)
    ll1, grad, _ = O.evaluate(w.parent, t, w.Q, w.pi, w.rates, w.weights,
                              w.pattern_weights, tip_states=w.tip_states)
    assert abs(ll0 - ll1) < 1e-11 * abs(ll0)
    sub = O.gradient_by_substitution(w.parent, t, w.Q, w.pi, w.rates,
                                     w.weights, w.pattern_weights,
                                     tip_states=w.tip_states)
    np.testing.assert_allclose(grad, sub, rtol=1e-11, atol=1e-11)


def _reroot(parent, t, new_child, frac):
    """Move the root of (parent, t) onto the branch above ``new_child``,
    splitting it frac : 1-frac. The old root's two branches merge into one
    edge. Tip labels are kept; internal nodes are renumbered."""
    n = len(parent)
    n_tips = (n + 1) // 2
    root = int(np.nonzero(parent < 0)[0][0])
    adj = {v: {} for v in range(n) if v != root}
    a, b = [v for v in range(n) if parent[v] == root]
    for v in range(n):
        if v == root or parent[v] == root:
            continue
        adj[v][int(parent[v])] = t[v]
        adj[int(parent[v])][v] = t[v]
    adj[a][b] = t[a] + t[b]
    adj[b][a] = t[a] + t[b]
    up = int(parent[new_child]) if parent[new_child] != root else (
        b if new_child == a else a)
    L = adj[new_child][up]
    del adj[new_child][up]
    del adj[up][new_child]
    new_parent = np.full(n, -1, dtype=np.int32)
    new_t = np.zeros(n - 1)
    ids = {}
    next_id = [n_tips]

    def assign(v):
        if v < n_tips:
            return v
        ids[v] = next_id[0]
        next_id[0] += 1
        return ids[v]

    new_root = n - 1
    out_edges = [(new_child, frac * L), (up, (1 - frac) * L)]
    stack = []
    for v, length in out_edges:
        stack.append((v, None, new_root, length))
    order = []
    while stack:
        v, from_v, par_id, length = stack.pop()
        order.append((v, from_v, par_id, length))
        vid = assign(v) if v >= n_tips else v
        for w2, l2 in adj[v].items():
            if w2 != from_v:
                stack.append((w2, v, vid, l2))
    for v, _, par_id, length in order:
        vid = v if v < n_tips else ids[v]
        new_parent[vid] = par_id
        new_t[vid] = length
    assert next_id[0] == n - 1
    return new_parent, new_t


@pytest.mark.parametrize("n_states", [4, 122])
def test_reroot_invariance(n_states):
    """Rerooting under a reversible model with root = pi (also the 122-state
    Markov-modulated codon model)."""
    w = synth.small_workload(9, n_states, 4 if n_states == 4 else 2, 30, seed=12)
    ll0, g0, _ = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                            w.pattern_weights, tip_states=w.tip_states)
    root = len(w.parent) - 1
    for child in [0, 3, 10, 12]:
        if w.parent[child] == root:
            continue
        p2, t2 = _reroot(w.parent, w.t, child, 0.3)
        ll1, g1, _ = O.evaluate(p2, t2, w.Q, w.pi, w.rates, w.weights,
                                w.pattern_weights, tip_states=w.tip_states)
        assert abs(ll0 - ll1) < 1e-11 * abs(ll0)
        # tip edges that exist unchanged in both trees keep their derivative
        for tip in range(9):
            if tip == child or w.parent[tip] == root:
                continue
            assert abs(g0[tip] - g1[tip]) < 1e-9 * max(1.0, abs(g0[tip]))


def test_long_branch_limit_needs_rescaling():
    """With very long branches P -> 1 pi', so P(Y_c) = prod_n pi[y_nc].
    On 300 tips with 20 states that is ~1e-400: it underflows FP64 unless
    the partials are rescaled."""
    rng = np.random.default_rng(13)
    n = 300
    parent = synth.caterpillar_tree(n)
    t = np.full(2 * n - 2, 60.0)
    Q, pi = synth.random_reversible(20, rng)
    rates, weights = np.array([1.0]), np.array([1.0])
    states = rng.integers(0, 20, size=(n, 6)).astype(np.uint8)
    W = np.arange(1, 7, dtype=np.float64)
    logL, grad, _ = O.evaluate(parent, t, Q, pi, rates, weights, W,
                               tip_states=states)
    expect = float(np.dot(W, np.log(pi)[states].sum(axis=0)))
    assert expect < -1000
    assert abs(logL - expect) < 1e-10 * abs(expect)
    assert np.max(np.abs(grad)) < 1e-9


def test_gap_tip_equals_pruned_tip():
    """A tip that is all gaps contributes P 1 = 1: the likelihood equals
    that of the tree with the tip removed (its sibling's branch absorbs the
    parent's branch)."""
    w = synth.small_workload(6, 4, 2, 15, seed=14)
    n = len(w.parent)
    root = n - 1
    x = next(v for v in range(6) if w.parent[v] != root)
    k = int(w.parent[x])
    sib = next(v for v in range(n) if w.parent[v] == k and v != x)
    states_gap = w.tip_states.copy()
    states_gap[x, :] = 4
    ll_gap = O.log_likelihood(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                              w.pattern_weights, tip_states=states_gap)
    tips = [v for v in range(6) if v != x]
    ints = [v for v in range(6, n) if v != k]
    lab = {v: i for i, v in enumerate(tips + ints)}
    p2 = np.full(n - 2, -1, dtype=np.int32)
    t2 = np.zeros(n - 3)
    for v in tips + ints:
        if v == root:
            continue
        p_old = int(w.parent[v])
        length = w.t[v]
        if v == sib:
            p_old = int(w.parent[k])
            length = w.t[v] + w.t[k]
        p2[lab[v]] = lab[p_old]
        t2[lab[v]] = length
    assert p2[-1] == -1
    ll_pruned = O.log_likelihood(p2, t2, w.Q, w.pi, w.rates, w.weights,
                                 w.pattern_weights,
                                 tip_states=w.tip_states[tips])
    assert abs(ll_gap - ll_pruned) < 1e-11 * abs(ll_pruned)


def test_tip_partials_equal_tip_states():
    w = synth.small_workload(7, 20, 2, 12, seed=15)
    a = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                   w.pattern_weights, tip_states=w.tip_states)
    b = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                   w.pattern_weights,
                   tip_partials=O.tip_partial_vectors(20, w.tip_states))
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])


# ---------------------------------------------- planted mistakes ----------

def _pins_pass(w):
    """Any-node identity + finite differences on workload w."""
    _, grad, abs_sum, det = O.evaluate(
        w.parent, w.t, w.Q, w.pi, w.rates, w.weights, w.pattern_weights,
        tip_states=w.tip_states, return_details=True)
    ok_nodes = all(np.allclose(O.node_site_log_likelihoods(det, w.weights, v),
                               det["site_ll"], rtol=1e-10, atol=1e-10)
                   for v in range(len(w.parent)))
    fd = _fd_gradient(w)
    ok_fd = bool(np.all(np.abs(grad - fd)
                        <= 1e-6 * np.maximum(abs_sum, 1.0)))
    return ok_nodes and ok_fd


def _asym_workload():
    w = synth.small_workload(6, 4, 4, 20, seed=16, mean_t=0.2)
    w.Q, w.pi = synth.hky85(4.0, np.array([0.1, 0.2, 0.3, 0.4]))
    return w


def test_pins_pass_on_correct_oracle():
    assert _pins_pass(_asym_workload())


def test_planted_transposed_gradient_rate_matrix_is_caught(monkeypatch):
    def wrong(p_i, Q, q_i, rates):
        return np.asarray(rates)[:, None] * np.einsum("rcs,su,rcu->rc",
                                                      p_i, Q, q_i)
    monkeypatch.setattr(O, "gradient_numerator", wrong)
    assert not _pins_pass(_asym_workload())


def test_planted_dropped_category_rate_is_caught(monkeypatch):
    def wrong(p_i, Q, q_i, rates):
        return np.einsum("rcs,us,rcu->rc", p_i, Q, q_i)
    monkeypatch.setattr(O, "gradient_numerator", wrong)
    assert not _pins_pass(_asym_workload())


def test_planted_untransposed_preorder_matrix_is_caught(monkeypatch):
    monkeypatch.setattr(O, "apply_matrix_transposed", O.apply_matrix)
    assert not _pins_pass(_asym_workload())


def test_planted_transposed_postorder_matrix_is_caught():
    w = synth.small_workload(5, 4, 2, 7, seed=17, mean_t=0.3)
    w.Q, w.pi = synth.hky85(4.0, np.array([0.1, 0.2, 0.3, 0.4]))
    orig = O.apply_matrix
    try:
        O.apply_matrix = O.apply_matrix_transposed
        ll = O.site_log_likelihoods(w.parent, w.t, w.Q, w.pi, w.rates,
                                    w.weights,
                                    O.tip_partial_vectors(4, w.tip_states))
    finally:
        O.apply_matrix = orig
    bf = O.brute_force_site_likelihoods(w.parent, w.t, w.Q, w.pi, w.rates,
                                        w.weights, tip_states=w.tip_states)
    assert not np.allclose(np.exp(ll), bf, rtol=1e-6)


def _two_taxon_jc_B(rates, weights, x, y, T):
    """B of either branch of the two-taxon JC69 tree for one site (x, y):
    q of branch 0 is (1/4) P(gamma T)[., y], p is the one-hot e_x, and JC69
    has |Q[u, s]| = 1 on the diagonal and 1/3 off it, so the absolute
    numerator is gamma (1/4) [P_xy + (1 - P_xy) / 3] and the denominator
    (1/4) P_xy (column sums of the symmetric P are 1).  With
    P_same = 1/4 + 3/4 e and P_diff = 1/4 - 1/4 e (e = exp(-4 gamma T / 3))
    the bracket is P_same + P_diff (x = y) or P_diff + 1/4 + e/12 (x != y)."""
    num = den = 0.0
    for g, w in zip(rates, weights):
        e = math.exp(-4.0 * g * T / 3.0)
        p_same, p_diff = 0.25 + 0.75 * e, 0.25 - 0.25 * e
        if x == y:
            num += w * g * (p_same + p_diff)
            den += w * p_same
        else:
            num += w * g * (p_diff + 0.25 + e / 12.0)
            den += w * p_diff
    return num / den


@pytest.mark.parametrize("ncat", [1, 4])
def test_conditioning_scale_two_taxon_closed_form(ncat):
    """B (the sum over patterns of the Eq. 8 terms in absolute value, over
    the denominator) of the two-taxon JC69 tree in closed form."""
    Q, pi = synth.jc69()
    rates, weights = synth.discrete_gamma(0.5, ncat)
    parent = np.array([2, 2, -1], dtype=np.int32)
    t = np.array([0.07, 0.31])
    states = np.array([[0, 0, 1, 3, 2, 1], [0, 2, 1, 0, 2, 3]], dtype=np.uint8)
    W = np.array([3.0, 1.0, 2.0, 5.0, 1.0, 4.0])
    _, _, _, B = O.evaluate_with_scales(parent, t, Q, pi, rates, weights, W,
                                        tip_states=states)
    want = sum(W[c] * _two_taxon_jc_B(rates, weights, states[0, c],
                                      states[1, c], t.sum())
               for c in range(states.shape[1]))
    np.testing.assert_allclose(B, [want, want], rtol=1e-13)


def _scale_by_substitution(w):
    """B_i by a second route: one pruning pass per branch with P_i replaced
    by gamma_r P_i |Q| gives, at the root, sum_r w_r gamma_r a_i' P_i |Q| p_i
    (= the absolute Eq. 8 numerator, since p, q >= 0 and q_i = P_i' a_i);
    dividing by P(Y_c) and summing with the pattern weights gives B_i."""
    Q = np.asarray(w.Q)
    tips = O.tip_partial_vectors(Q.shape[0], w.tip_states)
    P = O.branch_matrices(w.parent, w.t, Q, w.rates)
    p, scale, root = O.postorder(w.parent, P, w.rates, tips)
    base = np.log(np.einsum("rc,r->c", np.einsum("rcs,s->rc", p[root], w.pi),
                            w.weights)) + scale[root]
    B = np.zeros(len(w.parent) - 1)
    for b in range(len(w.parent)):
        if b == root:
            continue
        M = np.stack([g * P[b][r] @ np.abs(Q) for r, g in enumerate(w.rates)])
        pd, sd, _ = O.postorder(w.parent, P, w.rates, tips, substitute=b, dP=M)
        val = np.einsum("rc,r->c", np.einsum("rcs,s->rc", pd[root], w.pi),
                        w.weights)
        B[b] = float(np.dot(w.pattern_weights, val * np.exp(sd[root] - base)))
    return B


def _scale_workloads():
    w4 = synth.small_workload(7, 4, 4, 25, seed=19, mean_t=0.2)
    w4.Q, w4.pi = synth.hky85(4.0, np.array([0.1, 0.2, 0.3, 0.4]))
    w4.tip_states[2, 3] = 4  # gap
    w20 = synth.small_workload(5, 20, 2, 12, seed=20, mean_t=0.3)
    return [w4, w20]


def test_conditioning_scale_matches_substitution_route():
    for w in _scale_workloads():
        _, _, _, B = O.evaluate_with_scales(w.parent, w.t, w.Q, w.pi, w.rates,
                                            w.weights, w.pattern_weights,
                                            tip_states=w.tip_states)
        np.testing.assert_allclose(B, _scale_by_substitution(w), rtol=1e-11)


@pytest.mark.parametrize("mistake", ["times_S", "signed_Q", "abs_after_sum",
                                     "transposed_Q"])
def test_planted_scale_mistake_is_caught(monkeypatch, mistake):
    """A wrong conditioning scale (which would silently widen every parity
    bound) fails the substitution-route pin."""
    right = O.gradient_numerator_abs

    def wrong(p_i, Q, q_i, rates):
        g = np.asarray(rates)[:, None]
        if mistake == "times_S":
            return right(p_i, Q, q_i, rates) * np.asarray(Q).shape[0]
        if mistake == "signed_Q":
            return g * np.einsum("rcs,us,rcu->rc", np.abs(p_i), Q, np.abs(q_i))
        if mistake == "abs_after_sum":
            return np.abs(g * np.einsum("rcs,us,rcu->rc", p_i, Q, q_i))
        return g * np.einsum("rcs,su,rcu->rc", np.abs(p_i), np.abs(Q), np.abs(q_i))

    monkeypatch.setattr(O, "gradient_numerator_abs", wrong)
    caught = False
    for w in _scale_workloads():
        _, _, _, B = O.evaluate_with_scales(w.parent, w.t, w.Q, w.pi, w.rates,
                                            w.weights, w.pattern_weights,
                                            tip_states=w.tip_states)
        caught |= not np.allclose(B, _scale_by_substitution(w), rtol=1e-11)
    assert caught


def test_conditioning_scales():
    """The conditioning scales bound the entries: B_i >= A_i >= |grad_i|."""
    w = synth.small_workload(9, 4, 4, 30, seed=18)
    ll, g, A, B = O.evaluate_with_scales(w.parent, w.t, w.Q, w.pi, w.rates,
                                         w.weights, w.pattern_weights,
                                         tip_states=w.tip_states)
    ll2, g2, A2 = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                             w.pattern_weights, tip_states=w.tip_states)
    assert ll == ll2 and np.array_equal(g, g2) and np.array_equal(A, A2)
    assert np.all(B >= A * (1 - 1e-12)) and np.all(A >= np.abs(g) * (1 - 1e-12))
