"""Plain FP64 CPU oracle for the phylogenetic log-likelihood and its gradient
with respect to all 2N-2 branch lengths (arXiv 2303.04390).

TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the bench's
CPU-baseline leg may import this module; the library never routes through it.
It shares no code with the CUDA path: it builds transition matrices by
scaling-and-squaring of a Taylor series of gamma*t*Q (never an
eigendecomposition), carries its own log-scale factors (not powers of two),
and evaluates the gradient in the paper's Eq. 8 form p' Q' q (the CUDA path
uses the equivalent a' (dP) p form).

Notation (paper, Methods): tips 0..N-1, internal nodes N..2N-2, the root
is the node whose parent is -1; branch i is the branch above node i, with
length t[i]. For each node i, category r and pattern c:
  p[i][r, c, :]  post-order partial  (Eq. 2)
  q[i][r, c, :]  pre-order partial   (Eq. 4)
P^(r)(t) = exp(gamma_r t Q) with entry (s, u) = Pr(child u | parent s) (Eq. 1).

Tip data: ``tip_states`` (uint8 [N, C]); a value equal to S marks a gap or an
unknown character (all-ones partial). Or ``tip_partials`` (float [N, C, S]).

Every vector is kept with a per-(node, pattern) natural-log scale that is
shared by all categories and states, so nothing underflows.

Parity is pinned by tests/test_oracle.py (closed forms, brute force,
finite differences, the O(N^2) substitution route, the any-node identity,
rerooting and normalisation).
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Eq. 1: transition matrices
# ---------------------------------------------------------------------------


def expm_taylor(A: np.ndarray) -> np.ndarray:
    """exp(A) by scaling and squaring of a truncated Taylor series, FP64.

    A is scaled by 2^-j until its 1-norm is at most 1/2, the series is summed
    until terms stop changing the sum, then squared j times.
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    norm = float(np.max(np.sum(np.abs(A), axis=0))) if n else 0.0
    j = 0
    while norm > 0.5:
        norm /= 2.0
        j += 1
    B = A / (2.0 ** j)
    E = np.eye(n)
    term = np.eye(n)
    for k in range(1, 40):
        term = term @ B / k
        E = E + term
        if np.max(np.abs(term)) < 1e-18:
            break
    for _ in range(j):
        E = E @ E
    return E


def transition_matrices(Q, rates, t):
    """P^(r)(t) = exp(gamma_r t Q) for every category r (Eq. 1).
    Returns [R, S, S]."""
    return np.stack([expm_taylor(g * t * np.asarray(Q)) for g in rates])


def transition_derivatives(Q, rates, t):
    """d/dt P^(r)(t) = gamma_r Q P^(r)(t). Returns [R, S, S]."""
    P = transition_matrices(Q, rates, t)
    return np.stack([g * np.asarray(Q) @ P[r] for r, g in enumerate(rates)])


# ---------------------------------------------------------------------------
# Tree helpers
# ---------------------------------------------------------------------------


def tree_children(parent):
    parent = np.asarray(parent)
    n = parent.shape[0]
    kids = [[] for _ in range(n)]
    root = None
    for v in range(n):
        if parent[v] < 0:
            root = v
        else:
            kids[int(parent[v])].append(v)
    return kids, root


def postorder_list(parent):
    """Nodes with every child before its parent."""
    kids, root = tree_children(parent)
    out, stack = [], [(root, False)]
    while stack:
        v, done = stack.pop()
        if done or not kids[v]:
            out.append(v)
        else:
            stack.append((v, True))
            for c in kids[v]:
                stack.append((c, False))
    return out


def tip_partial_vectors(n_states, tip_states=None, tip_partials=None):
    """One-hot (or all-ones for the gap code S) tip vectors, [N, C, S]."""
    if tip_partials is not None:
        return np.asarray(tip_partials, dtype=np.float64)
    ts = np.asarray(tip_states).astype(np.int64)
    n, c = ts.shape
    out = np.zeros((n, c, n_states))
    obs = ts < n_states
    ii, cc = np.nonzero(obs)
    out[ii, cc, ts[ii, cc]] = 1.0
    out[~obs] = 1.0
    return out


# The two matrix-vector products of the traversals, for all r and c at once.
# Kept as named helpers so that the tests can plant mistakes in them.


def apply_matrix(P, v):
    """(P v) for each r, c:  out[r,c,s] = sum_u P[r,s,u] v[r,c,u]."""
    return np.einsum("rsu,rcu->rcs", P, v)


def apply_matrix_transposed(P, v):
    """(P' v) for each r, c: out[r,c,u] = sum_s P[r,s,u] v[r,c,s]."""
    return np.einsum("rsu,rcs->rcu", P, v)


def _rescale(v, allow_zero=False):
    """Divide each (c) slice by its max |.| over (r, s); return
    (v, log max). A slice that is exactly zero is an error (data
    incompatible with the model) unless ``allow_zero``, where it stays 0."""
    m = np.max(np.abs(v), axis=(0, 2))
    if np.any(~(m > 0)):
        if not allow_zero or np.any(np.isnan(m)):
            raise ValueError("a partial vector is zero for some pattern "
                             "(data incompatible with the model)")
        m = np.where(m > 0, m, 1.0)
    return v / m[None, :, None], np.log(m)


# ---------------------------------------------------------------------------
# Eq. 2 and 3: post-order partials and the likelihood
# ---------------------------------------------------------------------------


def branch_matrices(parent, t, Q, rates):
    """P^(r)(t_b) for every branch b (Eq. 1), as a dict b -> [R, S, S]."""
    root = int(np.nonzero(np.asarray(parent) < 0)[0][0])
    return {b: transition_matrices(Q, rates, t[b])
            for b in range(len(parent)) if b != root}


def postorder(parent, P, rates, tips, substitute=None, dP=None):
    """Post-order partials p[i] ([R, C, S], rescaled) and their log scales
    for every node (Eq. 2). Tip partials are the data vectors.

    ``substitute`` = branch b uses ``dP`` (dP_b/dt) in place of P_b (the
    O(N^2) route).
    """
    kids, root = tree_children(parent)
    n_tips = tips.shape[0]
    R = len(rates)
    C = tips.shape[1]
    p, scale = {}, {}
    for v in postorder_list(parent):
        if v < n_tips:
            p[v] = np.broadcast_to(tips[v][None], (R,) + tips[v].shape).copy()
            scale[v] = np.zeros(C)
            continue
        prod = None
        log_s = np.zeros(C)
        for ch in kids[v]:
            M = dP if ch == substitute else P[ch]
            u = apply_matrix(M, p[ch])
            prod = u if prod is None else prod * u
            log_s = log_s + scale[ch]
        prod, s = _rescale(prod, allow_zero=substitute is not None)
        p[v], scale[v] = prod, log_s + s
    return p, scale, root


def site_log_likelihoods(parent, t, Q, pi, rates, weights, tips):
    """log P(Y_c) for every pattern c (Eq. 3)."""
    P = branch_matrices(parent, t, Q, rates)
    p, scale, root = postorder(parent, P, rates, tips)
    per_r = np.einsum("rcs,s->rc", p[root], pi)
    return np.log(np.einsum("rc,r->c", per_r, weights)) + scale[root]


def log_likelihood(parent, t, Q, pi, rates, weights, pattern_weights,
                   tip_states=None, tip_partials=None):
    """log P(Y) = sum_c W_c log sum_r w_r p_root,r,c' pi (Eq. 3)."""
    tips = tip_partial_vectors(np.asarray(Q).shape[0], tip_states,
                               tip_partials)
    ll = site_log_likelihoods(parent, t, Q, pi, rates, weights, tips)
    return float(np.dot(pattern_weights, ll))


# ---------------------------------------------------------------------------
# Eq. 4: pre-order partials
# ---------------------------------------------------------------------------


def preorder(parent, P, pi, rates, p, pscale):
    """Pre-order partials q[i] and their log scales for every node (Eq. 4):
    q_root = pi; q_i = P_i' (q_k o P_j p_j) for parent k and sibling j."""
    kids, root = tree_children(parent)
    R = len(rates)
    C = p[root].shape[1]
    S = len(pi)
    q, qscale = {}, {}
    q[root] = np.broadcast_to(np.asarray(pi, float)[None, None, :],
                              (R, C, S)).copy()
    qscale[root] = np.zeros(C)
    order = list(reversed(postorder_list(parent)))  # parents first
    for k in order:
        if not kids[k]:
            continue
        for i in kids[k]:
            a = q[k].copy()
            log_s = qscale[k].copy()
            for j in kids[k]:
                if j == i:
                    continue
                a = a * apply_matrix(P[j], p[j])
                log_s = log_s + pscale[j]
            qi, s = _rescale(apply_matrix_transposed(P[i], a))
            q[i], qscale[i] = qi, log_s + s
    return q, qscale


# ---------------------------------------------------------------------------
# Eqs. 5-8: any-node identity and the gradient
# ---------------------------------------------------------------------------


def gradient_numerator(p_i, Q, q_i, rates):
    """gamma_r p_i' Q' q_i for every r, c (the numerator terms of Eq. 8)."""
    return np.asarray(rates)[:, None] * np.einsum("rcs,us,rcu->rc",
                                                  p_i, Q, q_i)


def node_likelihood_terms(p_i, q_i):
    """p_i' q_i for every r, c (Eq. 5 and the denominator of Eq. 8)."""
    return np.einsum("rcs,rcs->rc", p_i, q_i)


def evaluate(parent, t, Q, pi, rates, weights, pattern_weights,
             tip_states=None, tip_partials=None, return_details=False):
    """log P(Y) and d log P(Y) / d t_i for all 2N-2 branches (Eqs. 3, 7, 8).

    Returns (logL, grad[2N-2], abs_sum[2N-2]) where
    abs_sum[i] = sum_c W_c |d log P(Y_c) / d t_i| is the conditioning scale
    of entry i (used by the tolerance on near-zero entries).
    """
    Q = np.asarray(Q, dtype=np.float64)
    pi = np.asarray(pi, dtype=np.float64)
    rates = np.asarray(rates, dtype=np.float64)
    weights = np.asarray(weights, dtype=np.float64)
    W = np.asarray(pattern_weights, dtype=np.float64)
    tips = tip_partial_vectors(Q.shape[0], tip_states, tip_partials)
    P = branch_matrices(parent, t, Q, rates)
    p, pscale, root = postorder(parent, P, rates, tips)
    per_r = np.einsum("rcs,s->rc", p[root], pi)
    site_ll = np.log(np.einsum("rc,r->c", per_r, weights)) + pscale[root]
    logL = float(np.dot(W, site_ll))
    q, qscale = preorder(parent, P, pi, rates, p, pscale)
    n_br = len(parent) - 1
    grad = np.zeros(n_br)
    abs_sum = np.zeros(n_br)
    for i in range(len(parent)):
        if i == root:
            continue
        num = np.einsum("rc,r->c", gradient_numerator(p[i], Q, q[i], rates),
                        weights)
        den = np.einsum("rc,r->c", node_likelihood_terms(p[i], q[i]),
                        weights)
        g_c = num / den
        grad[i] = float(np.dot(W, g_c))
        abs_sum[i] = float(np.dot(W, np.abs(g_c)))
    if return_details:
        return logL, grad, abs_sum, dict(p=p, pscale=pscale, q=q,
                                         qscale=qscale, root=root,
                                         site_ll=site_ll)
    return logL, grad, abs_sum


def gradient_numerator_abs(p_i, Q, q_i, rates):
    """gamma_r |p_i|' |Q|' |q_i| for every r, c: the numerator of Eq. 8
    with every term taken in absolute value (its rounding-error scale)."""
    return np.asarray(rates)[:, None] * np.einsum(
        "rcs,us,rcu->rc", np.abs(p_i), np.abs(Q), np.abs(q_i))


def evaluate_with_scales(parent, t, Q, pi, rates, weights, pattern_weights,
                         tip_states=None, tip_partials=None):
    """evaluate() plus the conditioning scale of every gradient entry:

    returns (logL, grad, A, B) with
      A_i = sum_c W_c |g_ic|                       (cross-pattern cancellation)
      B_i = sum_c W_c sum_r w_r |Eq. 8 numerator terms| / den_c
                                        (cross-pattern and within-pattern)
    B_i >= A_i.  A finite-precision evaluation of entry i carries an error
    proportional to B_i, not to |grad_i|.
    """
    logL, grad, A, det = evaluate(parent, t, Q, pi, rates, weights,
                                  pattern_weights, tip_states=tip_states,
                                  tip_partials=tip_partials,
                                  return_details=True)
    Qa = np.asarray(Q, dtype=np.float64)
    wts = np.asarray(weights, dtype=np.float64)
    W = np.asarray(pattern_weights, dtype=np.float64)
    B = np.zeros_like(A)
    for i in range(len(parent)):
        if i == det["root"]:
            continue
        p_i, q_i = det["p"][i], det["q"][i]
        num = np.einsum("rc,r->c", gradient_numerator_abs(p_i, Qa, q_i, rates),
                        wts)
        den = np.einsum("rc,r->c", node_likelihood_terms(p_i, q_i), wts)
        B[i] = float(np.dot(W, num / den))
    return logL, grad, A, B


def node_site_log_likelihoods(details, weights, node):
    """log sum_r w_r p_i' q_i for every c at ``node`` (Eq. 5); equals the
    site log-likelihood at every node."""
    terms = node_likelihood_terms(details["p"][node], details["q"][node])
    return (np.log(np.einsum("rc,r->c", terms, np.asarray(weights)))
            + details["pscale"][node] + details["qscale"][node])


# ---------------------------------------------------------------------------
# Independent routes used as pins
# ---------------------------------------------------------------------------


def gradient_by_substitution(parent, t, Q, pi, rates, weights,
                             pattern_weights, tip_states=None,
                             tip_partials=None):
    """O(N^2) route: for each branch b one full pruning pass with P_b
    replaced by dP_b/dt gives dP(Y_c)/dt_b; the gradient entry is
    sum_c W_c P'(Y_c) / P(Y_c)."""
    Q = np.asarray(Q, dtype=np.float64)
    pi = np.asarray(pi, dtype=np.float64)
    tips = tip_partial_vectors(Q.shape[0], tip_states, tip_partials)
    W = np.asarray(pattern_weights, dtype=np.float64)
    P = branch_matrices(parent, t, Q, rates)
    p, scale, root = postorder(parent, P, rates, tips)
    base = np.log(np.abs(np.einsum("rc,r->c", np.einsum(
        "rcs,s->rc", p[root], pi), weights))) + scale[root]
    grad = np.zeros(len(parent) - 1)
    for b in range(len(parent)):
        if b == root:
            continue
        dP = transition_derivatives(Q, rates, t[b])
        pd, sd, _ = postorder(parent, P, rates, tips, substitute=b, dP=dP)
        val = np.einsum("rc,r->c", np.einsum("rcs,s->rc", pd[root], pi),
                        weights)
        ratio = val * np.exp(sd[root] - base)
        grad[b] = float(np.dot(W, ratio))
    return grad


def brute_force_site_likelihoods(parent, t, Q, pi, rates, weights,
                                 tip_states=None, tip_partials=None):
    """P(Y_c) by explicit summation over every joint assignment of states to
    the internal nodes (no pruning): sum over assignments x of
    pi[x_root] * prod over branches of P_b[x_parent, x_child], with tip
    branches summed against the tip vectors. Tiny trees only."""
    Q = np.asarray(Q, dtype=np.float64)
    S = Q.shape[0]
    tips = tip_partial_vectors(S, tip_states, tip_partials)
    parent = np.asarray(parent)
    n = parent.shape[0]
    n_tips = (n + 1) // 2
    internal = list(range(n_tips, n))
    n_int = len(internal)
    pos = {v: k for k, v in enumerate(internal)}
    # all assignments: [S^n_int, n_int]
    grids = np.indices((S,) * n_int).reshape(n_int, -1).T
    C = tips.shape[1]
    total = np.zeros(C)
    root = int(np.nonzero(parent < 0)[0][0])
    for r, (g, w) in enumerate(zip(rates, weights)):
        prod = np.asarray(pi)[grids[:, pos[root]]][:, None] * np.ones((1, C))
        for b in range(n):
            if b == root:
                continue
            Pb = expm_taylor(g * t[b] * Q)
            xs = grids[:, pos[int(parent[b])]]
            if b < n_tips:
                # sum over the tip's state against its data vector
                prod = prod * (Pb[xs] @ tips[b].T)
            else:
                prod = prod * Pb[xs, grids[:, pos[b]]][:, None]
        total += w * prod.sum(axis=0)
    return total


# ---------------------------------------------------------------------------
# Branch parameterisations (Methods): a branch length is the difference of
# the parent's and the child's node heights in time units times a (possibly
# branch-specific) rate; a strict clock reduces the branch derivatives over
# a set of branches.  Plain chain rule on the gradient g = d log P / d t.
# ---------------------------------------------------------------------------


def lengths_from_heights(parent, heights, rates=None):
    """t_i = rate_i (h_parent(i) - h_i) for every non-root node i."""
    parent = np.asarray(parent)
    n = len(parent)
    t = np.zeros(n - 1)
    for i in range(n):
        if parent[i] >= 0:
            r = 1.0 if rates is None else rates[i]
            t[i] = r * (heights[parent[i]] - heights[i])
    return t


def chain_rate_time(g, rates, times):
    """(d/d rate_i, d/d time_i) of log P for t_i = rate_i time_i."""
    g = np.asarray(g, dtype=np.float64)
    return np.asarray(times) * g, np.asarray(rates) * g


def chain_heights(parent, g, rates=None):
    """d log P / d h_k for t_i = rate_i (h_parent(i) - h_i): branch i
    contributes -rate_i g_i to its child node i and +rate_i g_i to its
    parent node."""
    parent = np.asarray(parent)
    dh = np.zeros(len(parent))
    for i in range(len(parent)):
        p = parent[i]
        if p < 0:
            continue
        r = 1.0 if rates is None else rates[i]
        dh[i] -= r * g[i]
        dh[p] += r * g[i]
    return dh


def branch_sum(g, branches, weights=None):
    """sum_j weights_j g[branches_j] (a strict clock over a set of branches)."""
    g = np.asarray(g, dtype=np.float64)
    b = np.asarray(branches, dtype=np.int64)
    w = np.ones(len(b)) if weights is None else np.asarray(weights, dtype=np.float64)
    return float(np.sum(w * g[b]))
