"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: trees, branch lengths, substitution models
(generator matrices Q and their stationary distributions), discrete-Gamma rate
categories, simulated alignments and compressed site patterns. It computes no
likelihood, no partial and no gradient; both the CUDA path and the CPU oracle
take its output as given.

The paper's datasets (dengue, carnivores, yeast, West Nile virus; Results
section) are not available, so every workload here is synthetic: Yule trees
with i.i.d. exponential branch lengths and alignments simulated along them.

Conventions (paper, Methods): tips are nodes 0..N-1, internal nodes
N..2N-2 numbered in post-order, the root is node 2N-2, and branch i is the
branch above node i. ``parent[root] == -1``.

Alignment simulation uses uniformisation of the continuous-time Markov chain
(jumps at rate mu = max_i -Q_ii, each jump drawn from I + Q/mu), so it never
forms a transition matrix exp(tQ).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# ---------------------------------------------------------------------------
# Trees
# ---------------------------------------------------------------------------


def yule_tree(n_tips: int, rng: np.random.Generator) -> np.ndarray:
    """Random rooted binary topology by repeated splitting of a uniformly
    chosen current leaf (pure-birth / Yule process on topologies).

    Returns ``parent`` (int32, length 2N-1) with tips 0..N-1 in random order,
    internal nodes N..2N-2 numbered in post-order and the root = 2N-2.
    """
    if n_tips < 2:
        raise ValueError("a tree needs at least 2 tips")
    # Grow with temporary ids: node 0 is the root.
    children = {0: None}
    leaves = [0]
    next_id = 1
    while len(leaves) < n_tips:
        k = int(rng.integers(len(leaves)))
        leaf = leaves[k]
        a, b = next_id, next_id + 1
        next_id += 2
        children[leaf] = (a, b)
        children[a] = None
        children[b] = None
        leaves[k] = a
        leaves.append(b)
    # Post-order numbering of internal nodes; random labels for tips.
    tip_labels = rng.permutation(n_tips)
    tip_iter = iter(tip_labels.tolist())
    new_id = {}
    internal_counter = n_tips
    stack = [(0, False)]
    while stack:
        node, done = stack.pop()
        ch = children[node]
        if ch is None:
            new_id[node] = next(tip_iter)
        elif done:
            new_id[node] = internal_counter
            internal_counter += 1
        else:
            stack.append((node, True))
            stack.append((ch[1], False))
            stack.append((ch[0], False))
    parent = np.full(2 * n_tips - 1, -1, dtype=np.int32)
    for node, ch in children.items():
        if ch is not None:
            for c in ch:
                parent[new_id[c]] = new_id[node]
    assert new_id[0] == 2 * n_tips - 2
    return parent


def caterpillar_tree(n_tips: int) -> np.ndarray:
    """Fully unbalanced (ladder) tree: height N-1, the worst case for
    level-batched traversals. Internal nodes in post-order, root 2N-2."""
    parent = np.full(2 * n_tips - 1, -1, dtype=np.int32)
    parent[0] = n_tips
    parent[1] = n_tips
    for k in range(2, n_tips):
        parent[n_tips + k - 2] = n_tips + k - 1
        parent[k] = n_tips + k - 1
    return parent


def balanced_tree(n_tips: int) -> np.ndarray:
    """Balanced tree built by pairing neighbouring subtrees level by level."""
    parent = np.full(2 * n_tips - 1, -1, dtype=np.int32)
    layer = list(range(n_tips))
    nxt = n_tips
    while len(layer) > 1:
        new_layer = []
        for i in range(0, len(layer) - 1, 2):
            parent[layer[i]] = nxt
            parent[layer[i + 1]] = nxt
            new_layer.append(nxt)
            nxt += 1
        if len(layer) % 2:
            new_layer.append(layer[-1])
        layer = new_layer
    assert nxt == 2 * n_tips - 1
    return parent


def exponential_branch_lengths(n_tips: int, mean: float,
                               rng: np.random.Generator) -> np.ndarray:
    """i.i.d. Exp(mean) lengths for the 2N-2 branches (indexed by child)."""
    return rng.exponential(mean, size=2 * n_tips - 2).astype(np.float64)


# ---------------------------------------------------------------------------
# Substitution models: every Q is reversible w.r.t. pi and scaled to mean
# rate 1 (-sum_i pi_i Q_ii = 1), so branch lengths are expected numbers of
# substitutions per site (paper, Methods).
# ---------------------------------------------------------------------------


def _reversible_q(exch: np.ndarray, pi: np.ndarray) -> np.ndarray:
    """Q_ij = exch_ij * pi_j for i != j, rows summing to 0, mean rate 1."""
    s = pi.shape[0]
    ex = np.array(exch, dtype=np.float64)
    assert ex.shape == (s, s) and np.allclose(ex, ex.T)
    q = ex * pi[None, :]
    np.fill_diagonal(q, 0.0)
    np.fill_diagonal(q, -q.sum(axis=1))
    mean_rate = -float(np.dot(pi, np.diag(q)))
    return q / mean_rate


def jc69():
    pi = np.full(4, 0.25)
    return _reversible_q(np.ones((4, 4)), pi), pi


_PURINES = {0, 2}  # A, G in the order A, C, G, T


def _is_transition(a: int, b: int) -> bool:
    return (a in _PURINES) == (b in _PURINES)


def hky85(kappa: float, pi: np.ndarray):
    pi = np.asarray(pi, dtype=np.float64)
    ex = np.ones((4, 4))
    for a in range(4):
        for b in range(4):
            if a != b and _is_transition(a, b):
                ex[a, b] = kappa
    return _reversible_q(ex, pi), pi


def gtr(rates6: np.ndarray, pi: np.ndarray):
    """rates6 in the order AC, AG, AT, CG, CT, GT."""
    pi = np.asarray(pi, dtype=np.float64)
    ex = np.zeros((4, 4))
    k = 0
    for a in range(4):
        for b in range(a + 1, 4):
            ex[a, b] = ex[b, a] = rates6[k]
            k += 1
    return _reversible_q(ex, pi), pi


def random_reversible(n_states: int, rng: np.random.Generator,
                      exch_shape: float = 1.0, pi_alpha: float = 1.0):
    """General reversible model: exchangeabilities ~ Gamma(shape, 1),
    frequencies ~ Dirichlet(pi_alpha * 1). Used for the 20-state amino-acid
    workload and for arbitrary state counts."""
    ex = np.zeros((n_states, n_states))
    iu = np.triu_indices(n_states, 1)
    ex[iu] = rng.gamma(exch_shape, 1.0, size=len(iu[0]))
    ex = ex + ex.T
    pi = rng.dirichlet(np.full(n_states, pi_alpha))
    pi = np.maximum(pi, 1e-6)
    pi = pi / pi.sum()
    return _reversible_q(ex, pi), pi


# Standard genetic code, codons enumerated with nucleotides in T, C, A, G order.
_NUC_TCAG = "TCAG"
_AA_TCAG = "FFLLSSSSYY**CC*WLLLLPPPPHHQQRRRRIIIMTTTTNNKKSSRRVVVVAAAADDEEGGGG"


def sense_codons():
    """(codon strings, amino acids) of the 61 sense codons of the standard
    genetic code."""
    codons, aas = [], []
    k = 0
    for a in _NUC_TCAG:
        for b in _NUC_TCAG:
            for c in _NUC_TCAG:
                if _AA_TCAG[k] != "*":
                    codons.append(a + b + c)
                    aas.append(_AA_TCAG[k])
                k += 1
    return codons, aas


def codon_gy94(kappa: float, omega: float, pi: np.ndarray):
    """GY94-style codon model on the 61 sense codons: codons differing at one
    position exchange at rate kappa (if a transition) times omega (if
    non-synonymous); others do not exchange directly."""
    codons, aas = sense_codons()
    s = len(codons)
    pi = np.asarray(pi, dtype=np.float64)
    assert pi.shape == (s,)
    purine = set("AG")
    ex = np.zeros((s, s))
    for i in range(s):
        for j in range(i + 1, s):
            diff = [(x, y) for x, y in zip(codons[i], codons[j]) if x != y]
            if len(diff) != 1:
                continue
            x, y = diff[0]
            rate = 1.0
            if (x in purine) == (y in purine):
                rate *= kappa
            if aas[i] != aas[j]:
                rate *= omega
            ex[i, j] = ex[j, i] = rate
    return _reversible_q(ex, pi), pi


def markov_modulated(components, pis_class, switch_rate: float):
    """Markov-modulated model (the paper's 122-state MMM of two codon
    models, Results): K reversible component generators on the same S
    states and frequencies pi, combined on the K*S states (k, i).  Within
    class k substitutions follow Q_k; the class switches (k, i) -> (l, i)
    at rate switch_rate * rho_l.  The stationary distribution is
    rho_k pi_i and the combined generator is reversible; it is rescaled to
    mean rate 1 like every model here."""
    K = len(components)
    S = components[0][0].shape[0]
    pi = np.asarray(components[0][1], dtype=np.float64)
    rho = np.asarray(pis_class, dtype=np.float64)
    assert rho.shape == (K,) and abs(rho.sum() - 1.0) < 1e-12
    ex = np.zeros((K * S, K * S))
    for k, (Qk, pik) in enumerate(components):
        assert np.allclose(pik, pi)
        exk = Qk / pi[None, :]  # Q_k[i][j] = ex_k[i][j] pi_j off the diagonal
        np.fill_diagonal(exk, 0.0)
        ex[k * S:(k + 1) * S, k * S:(k + 1) * S] = exk / rho[k]
    for k in range(K):
        for l in range(K):
            if k != l:
                idx = np.arange(S)
                ex[k * S + idx, l * S + idx] = switch_rate / pi
    pi_full = (rho[:, None] * pi[None, :]).reshape(-1)
    return _reversible_q(ex, pi_full), pi_full


def codon_mmm(kappa: float, omegas, pi: np.ndarray, switch_rate: float = 0.5):
    """Two (or more) GY94-style codon models differing in omega, modulated
    with equal class weights: 61 * len(omegas) states."""
    comps = [codon_gy94(kappa, om, pi) for om in omegas]
    return markov_modulated(comps, np.full(len(omegas), 1.0 / len(omegas)),
                            switch_rate)


def discrete_gamma(alpha: float, n_cat: int):
    """Yang (1994) discrete Gamma: equal-probability bins of Gamma(alpha,
    rate alpha), each category rate the mean of its bin (mean rate 1).
    Returns (rates, weights)."""
    from scipy.special import gammainc, gammaincinv
    if n_cat == 1:
        return np.ones(1), np.ones(1)
    edges = [0.0]
    for k in range(1, n_cat):
        edges.append(gammaincinv(alpha, k / n_cat) / alpha)
    edges.append(math.inf)
    cum = [0.0]
    for k in range(1, n_cat):
        cum.append(gammainc(alpha + 1.0, alpha * edges[k]))
    cum.append(1.0)
    rates = np.array([n_cat * (cum[k + 1] - cum[k]) for k in range(n_cat)])
    weights = np.full(n_cat, 1.0 / n_cat)
    return rates, weights


# ---------------------------------------------------------------------------
# Alignment simulation and pattern compression
# ---------------------------------------------------------------------------


def preorder_nodes(parent: np.ndarray):
    """Nodes ordered so that every parent precedes its children."""
    n = parent.shape[0]
    kids = [[] for _ in range(n)]
    root = -1
    for v in range(n):
        if parent[v] < 0:
            root = v
        else:
            kids[parent[v]].append(v)
    order, stack = [], [root]
    while stack:
        v = stack.pop()
        order.append(v)
        stack.extend(kids[v])
    return order


def simulate_sites(parent, t, Q, pi, rates, weights, n_sites,
                   rng: np.random.Generator) -> np.ndarray:
    """Simulate ``n_sites`` columns along the tree; returns tip states
    (uint8 [N, n_sites]). Each site draws a rate category, the root state
    from pi, then jumps down each branch by uniformisation."""
    s = Q.shape[0]
    n_nodes = parent.shape[0]
    n_tips = (n_nodes + 1) // 2
    mu = float(np.max(-np.diag(Q)))
    jump = np.eye(s) + Q / mu
    jump = np.maximum(jump, 0.0)
    jump /= jump.sum(axis=1, keepdims=True)
    cum = np.cumsum(jump, axis=1)
    cat = rng.choice(len(rates), size=n_sites, p=weights)
    site_rate = np.asarray(rates)[cat]
    state = np.zeros((n_nodes, n_sites), dtype=np.int64)
    for v in preorder_nodes(parent):
        if parent[v] < 0:
            state[v] = rng.choice(s, size=n_sites, p=pi)
            continue
        x = state[parent[v]].copy()
        k = rng.poisson(mu * site_rate * t[v])
        kmax = int(k.max()) if n_sites else 0
        for step in range(kmax):
            live = np.nonzero(k > step)[0]
            u = rng.random(live.shape[0])
            x[live] = np.minimum((u[:, None] > cum[x[live]]).sum(axis=1), s - 1)
        state[v] = x
    return state[:n_tips].astype(np.uint8)


def compress_patterns(tip_states: np.ndarray):
    """Unique columns in order of first appearance and their counts."""
    cols = np.ascontiguousarray(tip_states.T)
    _, first, counts = np.unique(cols, axis=0, return_index=True,
                                 return_counts=True)
    order = np.argsort(first)
    uniq = cols[first[order]].T.copy()
    return uniq.astype(np.uint8), counts[order].astype(np.float64)


def unique_patterns(parent, t, Q, pi, rates, weights, n_patterns,
                    rng: np.random.Generator, batch: int = 4096,
                    max_batches: int = 200) -> np.ndarray:
    """Simulate sites in batches until ``n_patterns`` distinct columns are
    collected; keep the first ``n_patterns`` in order of appearance."""
    seen = {}
    out = []
    for _ in range(max_batches):
        sites = simulate_sites(parent, t, Q, pi, rates, weights, batch, rng)
        for col in np.ascontiguousarray(sites.T):
            key = col.tobytes()
            if key not in seen:
                seen[key] = len(out)
                out.append(col)
                if len(out) == n_patterns:
                    return np.stack(out, axis=1).astype(np.uint8)
    raise RuntimeError("could not collect %d unique patterns" % n_patterns)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Workload:
    name: str
    parent: np.ndarray          # int32 [2N-1]
    t: np.ndarray               # float64 [2N-2]
    Q: np.ndarray               # float64 [S, S], reversible, mean rate 1
    pi: np.ndarray              # float64 [S], stationary = root distribution
    rates: np.ndarray           # float64 [R]  category rates gamma_r
    weights: np.ndarray         # float64 [R]  category weights P(gamma_r)
    tip_states: np.ndarray      # uint8 [N, C]
    pattern_weights: np.ndarray  # float64 [C]
    precision: str = "fp32"

    @property
    def n_tips(self):
        return (self.parent.shape[0] + 1) // 2

    @property
    def n_patterns(self):
        return self.tip_states.shape[1]

    @property
    def n_states(self):
        return self.Q.shape[0]

    @property
    def n_categories(self):
        return self.rates.shape[0]

    def with_patterns(self, lo: int, hi: int) -> "Workload":
        """A contiguous range of site patterns (shards are independent)."""
        return dataclasses.replace(
            self, name=f"{self.name}[{lo}:{hi}]",
            tip_states=np.ascontiguousarray(self.tip_states[:, lo:hi]),
            pattern_weights=np.ascontiguousarray(self.pattern_weights[lo:hi]))


def workload_jc69_8(seed: int = 0) -> Workload:
    """8-taxon Yule tree, Exp(mean 0.1) branches, JC69, one category,
    1,000 simulated sites compressed to unique patterns (weights = counts);
    FP64."""
    rng = np.random.default_rng([seed, 1])
    parent = yule_tree(8, rng)
    t = exponential_branch_lengths(8, 0.1, rng)
    Q, pi = jc69()
    rates, w = discrete_gamma(1.0, 1)
    sites = simulate_sites(parent, t, Q, pi, rates, w, 1000, rng)
    pats, counts = compress_patterns(sites)
    return Workload("jc69-8taxa-1000sites", parent, t, Q, pi, rates, w,
                    pats, counts, "fp64")


def workload_hky_1024(seed: int = 0, n_tips: int = 1024,
                      n_patterns: int = 10000) -> Workload:
    """1,024-taxon Yule tree, Exp(mean 0.002) branches, HKY85 (kappa 4,
    frequencies ~ Dirichlet(10,10,10,10)) + discrete Gamma(0.5) 4 categories,
    10,000 unique simulated patterns with weights uniform on 1..5."""
    rng = np.random.default_rng([seed, 2])
    parent = yule_tree(n_tips, rng)
    t = exponential_branch_lengths(n_tips, 0.002, rng)
    Q, pi = hky85(4.0, rng.dirichlet([10.0] * 4))
    rates, w = discrete_gamma(0.5, 4)
    pats = unique_patterns(parent, t, Q, pi, rates, w, n_patterns, rng)
    pw = rng.integers(1, 6, size=n_patterns).astype(np.float64)
    return Workload(f"hky85-g4-{n_tips}taxa-{n_patterns}patterns", parent, t,
                    Q, pi, rates, w, pats, pw, "fp32")


def workload_codon_128(seed: int = 0, n_tips: int = 128,
                       n_patterns: int = 2000) -> Workload:
    """128-taxon Yule tree, Exp(mean 0.05) branches, GY94-style 61-state
    codon model (omega 0.3, kappa 2, codon frequencies ~ Dirichlet(61 x 1))
    + Gamma 4 categories (alpha 0.5), 2,000 unique patterns, weights 1..5."""
    rng = np.random.default_rng([seed, 3])
    parent = yule_tree(n_tips, rng)
    t = exponential_branch_lengths(n_tips, 0.05, rng)
    pi = rng.dirichlet(np.ones(61))
    pi = np.maximum(pi, 1e-4)
    pi /= pi.sum()
    Q, pi = codon_gy94(2.0, 0.3, pi)
    rates, w = discrete_gamma(0.5, 4)
    pats = unique_patterns(parent, t, Q, pi, rates, w, n_patterns, rng)
    pw = rng.integers(1, 6, size=n_patterns).astype(np.float64)
    return Workload(f"gy94-codon61-g4-{n_tips}taxa-{n_patterns}patterns",
                    parent, t, Q, pi, rates, w, pats, pw, "fp32")


def workload_aa_256(seed: int = 0, n_tips: int = 256,
                    n_patterns: int = 5000) -> Workload:
    """256-taxon Yule tree, Exp(mean 0.1) branches, 20-state reversible
    model (exchangeabilities ~ Gamma(1,1), frequencies ~ Dirichlet(20 x 1))
    + Gamma 4 categories (alpha 0.5), 5,000 unique patterns, weights 1..5."""
    rng = np.random.default_rng([seed, 4])
    parent = yule_tree(n_tips, rng)
    t = exponential_branch_lengths(n_tips, 0.1, rng)
    Q, pi = random_reversible(20, rng, 1.0, 1.0)
    rates, w = discrete_gamma(0.5, 4)
    pats = unique_patterns(parent, t, Q, pi, rates, w, n_patterns, rng)
    pw = rng.integers(1, 6, size=n_patterns).astype(np.float64)
    return Workload(f"aa20-g4-{n_tips}taxa-{n_patterns}patterns", parent, t,
                    Q, pi, rates, w, pats, pw, "fp32")


def workload_mmm_122(seed: int = 0, n_tips: int = 128,
                     n_patterns: int = 2000) -> Workload:
    """The codon workload's shape with the paper's Markov-modulated model:
    two GY94-style codon models (kappa 2, omega 0.1 and 1.0, codon
    frequencies ~ Dirichlet(61 x 1)) switching at rate 0.5, 122 states;
    128-taxon Yule tree, Exp(mean 0.05) branches, Gamma 4 categories
    (alpha 0.5), 2,000 unique patterns, weights 1..5."""
    rng = np.random.default_rng([seed, 6])
    parent = yule_tree(n_tips, rng)
    t = exponential_branch_lengths(n_tips, 0.05, rng)
    pi = rng.dirichlet(np.ones(61))
    pi = np.maximum(pi, 1e-4)
    pi /= pi.sum()
    Q, pi = codon_mmm(2.0, (0.1, 1.0), pi)
    rates, w = discrete_gamma(0.5, 4)
    pats = unique_patterns(parent, t, Q, pi, rates, w, n_patterns, rng)
    pw = rng.integers(1, 6, size=n_patterns).astype(np.float64)
    return Workload(f"mmm-codon122-g4-{n_tips}taxa-{n_patterns}patterns",
                    parent, t, Q, pi, rates, w, pats, pw, "fp32")


def small_workload(n_tips: int, n_states: int, n_cat: int, n_patterns: int,
                   seed: int, mean_t: float = 0.1,
                   tree: str = "yule", unique: bool = False) -> Workload:
    """Small seeded workload of any shape (parity tests)."""
    rng = np.random.default_rng([seed, 77, n_tips, n_states, n_cat])
    if tree == "yule":
        parent = yule_tree(n_tips, rng)
    elif tree == "caterpillar":
        parent = caterpillar_tree(n_tips)
    else:
        parent = balanced_tree(n_tips)
    t = exponential_branch_lengths(n_tips, mean_t, rng)
    if n_states == 4:
        Q, pi = hky85(4.0, rng.dirichlet([10.0] * 4))
    elif n_states in (61, 122):
        pi = rng.dirichlet(np.ones(61))
        pi = np.maximum(pi, 1e-4)
        pi /= pi.sum()
        if n_states == 61:
            Q, pi = codon_gy94(2.0, 0.3, pi)
        else:
            Q, pi = codon_mmm(2.0, (0.1, 1.0), pi)
    else:
        Q, pi = random_reversible(n_states, rng)
    rates, w = discrete_gamma(0.5, n_cat)
    if unique:
        pats = unique_patterns(parent, t, Q, pi, rates, w, n_patterns, rng)
    else:
        pats = simulate_sites(parent, t, Q, pi, rates, w, n_patterns, rng)
    pw = rng.integers(1, 6, size=n_patterns).astype(np.float64)
    return Workload(f"small-n{n_tips}-s{n_states}-r{n_cat}-c{n_patterns}",
                    parent, t, Q, pi, rates, w, pats, pw, "fp32")


CONFIGS = {
    "jc69-8": workload_jc69_8,
    "hky-1024": workload_hky_1024,
    "codon-128": workload_codon_128,
    "aa-256": workload_aa_256,
    "mmm-122": workload_mmm_122,
}


def served_request(k: int, seed: int = 0):
    """Request k of the served stream: Yule tree with N ~ logU[16, 2048]
    taxa, C ~ logU[100, 20000] patterns, 4 states (p = 0.7, HKY85 as the
    1,024-taxon workload) or 20 states (the amino-acid model), Gamma 4
    categories (alpha 0.5), Exp(mean 0.05) branches, weights 1..5."""
    rng = np.random.default_rng([seed, 5, k])
    n_tips = int(round(math.exp(rng.uniform(math.log(16), math.log(2048)))))
    n_pat = int(round(math.exp(rng.uniform(math.log(100), math.log(20000)))))
    four = rng.random() < 0.7
    parent = yule_tree(n_tips, rng)
    t = exponential_branch_lengths(n_tips, 0.05, rng)
    if four:
        Q, pi = hky85(4.0, rng.dirichlet([10.0] * 4))
    else:
        Q, pi = random_reversible(20, rng, 1.0, 1.0)
    rates, w = discrete_gamma(0.5, 4)
    # Sites, not unique patterns: cheap to draw for large requests.
    pats = simulate_sites(parent, t, Q, pi, rates, w, n_pat, rng)
    pw = rng.integers(1, 6, size=n_pat).astype(np.float64)
    return Workload(f"req{k}-n{n_tips}-s{Q.shape[0]}-c{n_pat}", parent, t, Q,
                    pi, rates, w, pats, pw, "fp32")
