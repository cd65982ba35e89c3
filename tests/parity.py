"""Shared helpers for the parity tests: the oracle run (optionally over
pattern shards in a spawn process pool) and the tolerance check.

Tolerances:
  FP64 path: |logL - logL*| <= 1e-12 |logL*|;
             |g - g*| <= max(1e-12 |g*|, 1e-11 B)
  FP32 path: |logL - logL*| <= 1e-5 |logL*|;
             |g - g*| <= max(1e-4 |g*|,  1e-6 B)
where B is the entry's conditioning scale from the oracle: the sum over
patterns and categories of the absolute values of the Eq. 8 numerator terms
over the denominator (pinned independently by the oracle tests: a closed
form on two taxa and a substitution route).  An entry that cancels across
patterns or inside a pattern (|g*| << B) cannot be held to a bound relative
to |g*| by any finite-precision evaluation -- two FP64 evaluations in
different but exact orders already differ by ~1e-14 B -- so the bound falls
back to a fraction of B.  FP32: the measured worst on the full-size
workloads is 4.1e-7 B (codon-128; mmm-122 3.6e-7 B, hky-1024 1.5e-7 B,
aa-256 4e-8 B).  FP64: the eigen route of Eq. 1
leaves an absolute error of order S u sqrt(pi_max / pi_min) in the small
entries of P (two- and three-nucleotide codon changes on short branches),
which the 61-state workload turns into ~3e-12 B; the Taylor route of the
oracle does not share it.

compare() returns the figures the tests print: the relative error of log
P(Y), the worst error over its bound, the worst relative error over the
entries with |g*| >= 1e-3 B (those the relative bound governs), the worst
error in units of B, and how many entries pass only through the B fallback.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

from oracle import phylo_oracle as O

TOL = {
    "fp64": dict(ll_rel=1e-12, g_rel=1e-12, g_cond=1e-11),
    "fp32": dict(ll_rel=1e-5, g_rel=1e-4, g_cond=1e-6),
}


def _oracle_shard(args):
    (parent, t, Q, pi, rates, weights, W, states, partials) = args
    return O.evaluate_with_scales(parent, t, Q, pi, rates, weights, W,
                                  tip_states=states, tip_partials=partials)


def oracle_eval(w, t=None, tip_partials=None, shards=1):
    """(logL, grad, A, B) from the oracle.  With shards > 1 the patterns are
    split into contiguous ranges evaluated in a spawn process pool; the
    results are summed (every output is a sum over patterns, Eq. 7)."""
    t = w.t if t is None else t
    C = w.n_patterns
    if shards <= 1 or C < 2 * shards:
        tp = tip_partials
        return O.evaluate_with_scales(w.parent, t, w.Q, w.pi, w.rates,
                                      w.weights, w.pattern_weights,
                                      tip_states=w.tip_states,
                                      tip_partials=tp)
    bounds = np.linspace(0, C, shards + 1).astype(int)
    jobs = []
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        tp = None if tip_partials is None else tip_partials[:, lo:hi]
        jobs.append((w.parent, t, w.Q, w.pi, w.rates, w.weights,
                     w.pattern_weights[lo:hi], w.tip_states[:, lo:hi], tp))
    with ProcessPoolExecutor(max_workers=shards,
                             mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_oracle_shard, jobs))
    logL = sum(p[0] for p in parts)
    grad = sum(p[1] for p in parts)
    A = sum(p[2] for p in parts)
    B = sum(p[3] for p in parts)
    return logL, grad, A, B


def compare(logL, grad, ref, precision, what=""):
    """Assert the tolerances above; return the error figures (a dict)."""
    ll_ref, g_ref, A, B = ref
    tol = TOL[precision]
    ll_err = abs(logL - ll_ref)
    assert ll_err <= tol["ll_rel"] * abs(ll_ref), (
        f"{what}: logL {logL!r} vs oracle {ll_ref!r} (rel err "
        f"{ll_err / max(abs(ll_ref), 1e-300):.3e})")
    err = np.abs(np.asarray(grad) - g_ref)
    rel_bound = tol["g_rel"] * np.abs(g_ref)
    bound = np.maximum(rel_bound, tol["g_cond"] * B)
    ratio = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0),
                     np.where(err > 0, np.inf, 0.0))
    worst = int(np.argmax(ratio)) if ratio.size else 0
    assert ratio.size == 0 or ratio[worst] <= 1.0, (
        f"{what}: gradient entry {worst}: {grad[worst]!r} vs oracle "
        f"{g_ref[worst]!r} (|err| {err[worst]:.3e}, bound {bound[worst]:.3e},"
        f" B {B[worst]:.3e}, A {A[worst]:.3e})")
    big = np.abs(g_ref) >= 1e-3 * B
    rel = err[big] / np.abs(g_ref[big]) if np.any(big) else np.zeros(1)
    in_b = err / np.where(B > 0, B, 1.0)
    stats = {
        "ll_rel_err": ll_err / max(abs(ll_ref), 1e-300),
        "worst_err_over_bound": float(ratio[worst]) if ratio.size else 0.0,
        "worst_rel_err_large_entries": float(np.max(rel)),
        "worst_err_in_B": float(np.max(in_b)) if in_b.size else 0.0,
        "n_entries": int(err.size),
        "n_fallback_only": int(np.sum(err > rel_bound)),
    }
    log = os.environ.get("PHYLO_PARITY_LOG")
    if log:  # one JSON line per comparison, for the error tables
        with open(log, "a") as f:
            f.write(json.dumps({"what": what, "precision": precision,
                                **stats}) + "\n")
    return stats


def describe(stats):
    return (f"logL rel err {stats['ll_rel_err']:.2e}; gradient: worst "
            f"err/bound {stats['worst_err_over_bound']:.3f}, worst rel err "
            f"(|g*| >= 1e-3 B) {stats['worst_rel_err_large_entries']:.2e}, "
            f"worst err/B {stats['worst_err_in_B']:.2e}, "
            f"{stats['n_fallback_only']} of {stats['n_entries']} entries pass "
            f"only through the B fallback")
