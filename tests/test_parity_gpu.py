"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element (log P(Y) and every gradient
entry), for both precisions, over shapes that span several pattern tiles
with a ragged tail, every padded state class, idle category lanes, deep
and shallow trees, gaps, tip partials, zero-length branches, empty inputs,
device-side error flags, and the full-size workloads."""
import numpy as np
import pytest

import synth
from parity import TOL, compare, describe, oracle_eval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04390_gb300 import build as B
    B.build()
    import paper_2303_04390_gb300 as pg
    return pg


def _gpu(w, precision, tip_partials=None, t=None):
    import paper_2303_04390_gb300 as pg
    ctx = pg.from_workload(w, precision, tip_partials=tip_partials is not None)
    if tip_partials is not None:
        for tip in range(w.n_tips):
            if not np.all(tip_partials[tip] == _onehot(w, tip)):
                ctx.set_tip_partials(tip, tip_partials[tip])
    if t is not None:
        ctx.set_branch_lengths(t)
    logL, grad = ctx.evaluate()
    return ctx, logL, grad


def _onehot(w, tip):
    from oracle import phylo_oracle as O
    return O.tip_partial_vectors(w.n_states, w.tip_states[tip:tip + 1])[0]


SMALL = [
    # (n_tips, n_states, n_cat, n_patterns, tree)
    (2, 4, 1, 5, "yule"),
    (3, 4, 4, 33, "yule"),
    (17, 4, 4, 300, "yule"),
    (40, 4, 2, 100, "caterpillar"),
    (32, 4, 4, 257, "balanced"),
    (12, 3, 3, 70, "yule"),
    (10, 7, 5, 50, "yule"),
    (12, 20, 4, 150, "yule"),
    (9, 20, 8, 40, "caterpillar"),
    (9, 61, 4, 70, "yule"),
    (6, 33, 2, 20, "balanced"),
    (5, 64, 1, 17, "yule"),
    (24, 61, 4, 37, "caterpillar"),
    (14, 61, 4, 300, "yule"),          # several 128-pattern tiles, ragged tail
    (6, 45, 3, 129, "caterpillar"),    # a tail of one pattern
    (40, 61, 4, 1, "yule"),
    (120, 61, 4, 130, "caterpillar"),  # deep chain: rescaling at every node
    # 65..256 states (S_pad 128, 256): matrices streamed through shared memory
    (6, 122, 4, 40, "yule"),
    (9, 122, 2, 33, "caterpillar"),
    (20, 122, 4, 50, "yule"),
    (7, 90, 3, 17, "balanced"),
    (5, 256, 2, 19, "yule"),
    (8, 200, 1, 9, "caterpillar"),
    (5, 65, 8, 21, "yule"),            # smallest S of S_pad 128, eight categories
    (4, 129, 3, 18, "balanced"),       # smallest S of S_pad 256
    (30, 122, 2, 17, "caterpillar"),   # deep chain at 122 states: rescaling at every node
    # the U form (FP32, 5-128 states): two-taxon trees (the root level alone)
    # and the largest and smallest state counts of each padded size
    (2, 20, 4, 9, "yule"),
    (2, 61, 2, 130, "yule"),
    (2, 122, 1, 7, "yule"),
    (3, 21, 4, 129, "caterpillar"),
    (4, 128, 2, 40, "balanced"),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", SMALL, ids=lambda s: "n%d-s%d-r%d-c%d-%s" % s)
def test_small_parity(shape, precision):
    n, S, R, C, tree = shape
    w = synth.small_workload(n, S, R, C, seed=21, mean_t=0.15, tree=tree)
    rng = np.random.default_rng(5)
    gaps = rng.random(w.tip_states.shape) < 0.05
    if S < 256:  # 256 states use every byte value: no gap code
        w.tip_states[gaps] = S
    ref = oracle_eval(w)
    _, logL, grad = _gpu(w, precision)
    compare(logL, grad, ref, precision, w.name)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("S", [4, 20, 61, 122])
def test_tip_partials(S, precision):
    w = synth.small_workload(11, S, 4, 45, seed=22)
    from oracle import phylo_oracle as O
    tp = O.tip_partial_vectors(S, w.tip_states)
    rng = np.random.default_rng(S)
    for tip in [0, 3, 7]:
        tp[tip] = rng.random((45, S)) ** 3 + 0.01  # ambiguity / error model
    ref = oracle_eval(w, tip_partials=tp)
    _, logL, grad = _gpu(w, precision, tip_partials=tp)
    compare(logL, grad, ref, precision, "tip partials")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("S", [20, 61, 122])
def test_tip_partials_two_taxa(S, precision):
    """Both tips of a two-taxon tree carry partial vectors: the U form's
    first post-order launch (the tips' U) feeds the root level directly."""
    w = synth.small_workload(2, S, 4, 33, seed=31)
    from oracle import phylo_oracle as O
    tp = O.tip_partial_vectors(S, w.tip_states)
    rng = np.random.default_rng(S + 1)
    for tip in [0, 1]:
        tp[tip] = rng.random((33, S)) ** 3 + 0.01
    ref = oracle_eval(w, tip_partials=tp)
    _, logL, grad = _gpu(w, precision, tip_partials=tp)
    compare(logL, grad, ref, precision, "tip partials, two taxa")


@pytest.mark.parametrize("S", [20, 61, 122])
def test_tip_level_launch(S):
    """On the U-form FP32 paths a tip with partials adds one post-order
    launch (its U = P p, formed before the first level); the result still
    matches the oracle."""
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(9, S, 2, 40, seed=33)
    plain = pg.from_workload(w, "fp32")
    n0, (p0, q0) = plain.launches_per_evaluation(), plain.level_counts()
    plain.close()
    from oracle import phylo_oracle as O
    tp = O.tip_partial_vectors(S, w.tip_states)
    tp[4] = np.random.default_rng(S).random((40, S)) + 0.05
    ctx, logL, grad = _gpu(w, "fp32", tip_partials=tp)
    assert ctx.launches_per_evaluation() == n0 + 1
    assert ctx.level_counts() == (p0 + 1, q0)
    ctx.close()
    compare(logL, grad, oracle_eval(w, tip_partials=tp), "fp32", "tip level")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("S", [4, 61, 122])
def test_zero_length_branches(S, precision):
    w = synth.small_workload(15, S, 4, 80, seed=23)
    t = w.t.copy()
    root = 2 * w.n_tips - 2
    a = int(np.nonzero(w.parent == root)[0][0])
    t[a] = 0.0  # unrooted tree nested in the rooted form
    t[w.n_tips] = 0.0  # an internal branch
    ref = oracle_eval(w, t=t)
    _, logL, grad = _gpu(w, precision, t=t)
    compare(logL, grad, ref, precision, "zero-length branches")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("S", [4, 20, 61, 256])
def test_empty_alignment(S, precision):
    w = synth.small_workload(6, S, 2, 10, seed=24)
    w = w.with_patterns(0, 0)
    _, logL, grad = _gpu(w, precision)
    assert logL == 0.0 and np.all(grad == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_golden_jc69_two_taxon(precision):
    """The CUDA path against the stored closed-form JC69 values
    (tests/golden/jc69_two_taxon.txt), independently of the oracle."""
    import math
    import os
    import paper_2303_04390_gb300 as pg
    path = os.path.join(os.path.dirname(__file__), "golden", "jc69_two_taxon.txt")
    rows = [tuple(float(x) for x in line.split()) for line in open(path)
            if line.strip() and not line.startswith("#")]
    Q, pi = synth.jc69()
    for T, ls, dls, ld, dld in rows:
        if ld == 0.0:
            continue
        w = synth.Workload("jc69-two-taxon", np.array([2, 2, -1], dtype=np.int32),
                           np.array([T / 2, T / 2]), Q, pi, np.ones(1), np.ones(1),
                           np.array([[0, 0], [0, 1]], dtype=np.uint8), np.ones(2), precision)
        ctx = pg.from_workload(w, precision)
        logL, grad = ctx.evaluate()
        ctx.close()
        want = math.log(ls) + math.log(ld)
        g = dls / ls + dld / ld
        B = abs(dls / ls) + abs(dld / ld)
        tol = TOL[precision]
        assert abs(logL - want) <= tol["ll_rel"] * abs(want) + 1e-300
        assert np.all(np.abs(grad - g) <= np.maximum(tol["g_rel"] * abs(g), tol["g_cond"] * B))


def test_single_pattern_many_tips():
    w = synth.small_workload(300, 4, 4, 1, seed=25, tree="yule")
    ref = oracle_eval(w)
    for precision in ("fp64", "fp32"):
        _, logL, grad = _gpu(w, precision)
        compare(logL, grad, ref, precision, "C=1")


@pytest.mark.parametrize("S", [4, 20, 61])
def test_impossible_data_is_flagged_and_recoverable(S):
    """Two tips on zero-length branches under one parent with different
    states: the likelihood is exactly 0, the device flags it and the call
    returns PHYLO_ENUMERIC; the context still works afterwards."""
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(4, S, 2, 6, seed=26)
    root = 2 * w.n_tips - 2
    k = next(v for v in range(w.n_tips, root)
             if np.sum(w.parent[:w.n_tips] == v) == 2)
    i, j = np.nonzero(w.parent[:w.n_tips] == k)[0]
    w.tip_states[i, 2] = 0
    w.tip_states[j, 2] = 1
    t = w.t.copy()
    t[i] = t[j] = 0.0
    ctx = pg.from_workload(w, "fp32")
    ctx.set_branch_lengths(t)
    with pytest.raises(pg.PhyloError) as e:
        ctx.evaluate()
    assert e.value.code == -5
    ctx.set_branch_lengths(w.t)
    ref = oracle_eval(w)
    logL, grad = ctx.evaluate()
    compare(logL, grad, ref, "fp32", "after recovery")


def test_device_branch_lengths_and_validation():
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(20, 4, 4, 64, seed=27)
    ctx = pg.from_workload(w, "fp64")
    ref = oracle_eval(w)
    t_dev = torch.tensor(w.t, dtype=torch.float64, device="cuda")
    ctx.set_branch_lengths(t_dev)
    out = ctx.evaluate_device()
    ctx.check()
    res = out.cpu().numpy()
    compare(res[0], res[1:], ref, "fp64", "device pointers")
    bad = t_dev.clone()
    bad[3] = -1.0
    ctx.set_branch_lengths(bad)
    ctx.evaluate_device()
    with pytest.raises(pg.PhyloError) as e:
        ctx.check()
    assert e.value.code == -5
    ctx.set_branch_lengths(t_dev)
    logL, grad = ctx.evaluate()
    compare(logL, grad, ref, "fp64", "after bad device lengths")


def test_deterministic_and_stream_ordered():
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(64, 20, 4, 500, seed=28)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = pg.from_workload(w, "fp32", stream=s)
        a = ctx.evaluate()
        b = ctx.evaluate()
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    outs = []
    with torch.cuda.stream(s):
        for _ in range(3):
            outs.append(ctx.evaluate_device(
                torch.empty(2 * w.n_tips - 1, dtype=torch.float64,
                            device="cuda")))
    s.synchronize()
    for o in outs:
        assert o[0].item() == a[0]
        assert np.array_equal(o[1:].cpu().numpy(), a[1])


def test_launch_count_matches_level_schedule():
    """One launch per non-empty level.  On the FP32 4-state path a cherry
    (non-root node whose two children are tips) is fused into its parent's
    post-order step and has no post-order level of its own."""
    import paper_2303_04390_gb300 as pg
    from oracle import phylo_oracle as O
    for tree in ["yule", "caterpillar", "balanced"]:
        w = synth.small_workload(33, 4, 2, 40, seed=29, tree=tree)
        kids, root = O.tree_children(w.parent)
        height = {}
        for v in O.postorder_list(w.parent):
            height[v] = 0 if not kids[v] else 1 + max(height[c] for c in kids[v])
        depth = {root: 0}
        for v in reversed(O.postorder_list(w.parent)):
            for c in kids[v]:
                depth[c] = depth[v] + 1
        internal = range(w.n_tips, len(w.parent))
        cherry = {v for v in internal
                  if v != root and all(c < w.n_tips for c in kids[v])}
        for precision, fused in (("fp32", cherry), ("fp64", set())):
            ctx = pg.from_workload(w, precision)
            keep = [v for v in internal if v not in fused]
            n_post = len({height[v] for v in keep})
            n_pre = len({depth[v] for v in internal})
            assert ctx.launches_per_evaluation() == 2 + n_post + n_pre, (tree, precision)
            assert ctx.level_counts() == (n_post, n_pre)
            ctx.close()


FULL = {
    "jc69-8": ("fp64", 1),
    "hky-1024": ("fp32", 8),
    "codon-128": ("fp32", 8),
    "aa-256": ("fp32", 8),
    "mmm-122": ("fp32", 8),  # the 122-state Markov-modulated model, codon shape
}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_workloads(name):
    """The full-size workloads, in the configuration the bench times, against
    the oracle on every output; the FP64 path is checked on each too."""
    import paper_2303_04390_gb300 as pg
    precision, shards = FULL[name]
    w = synth.CONFIGS[name](0)
    ref = oracle_eval(w, shards=shards)
    for prec in sorted({precision, "fp64"}):
        ctx = pg.from_workload(w, prec)
        logL, grad = ctx.evaluate()
        stats = compare(logL, grad, ref, prec, f"{name} {prec}")
        print(f"{name} {prec}: {describe(stats)}")
        # pulley principle on the device result (reversible, root = pi)
        root = 2 * w.n_tips - 2
        a, b = np.nonzero(w.parent == root)[0]
        assert abs(grad[a] - grad[b]) <= 2 * max(
            TOL[prec]["g_rel"] * abs(ref[1][a]), TOL[prec]["g_cond"] * ref[3][a])
        ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("S", [61, 122, 256])
def test_general_eigen_form(precision, S):
    """Eigenvector columns rescaled: the same P(t), but not the symmetric
    decomposition of a reversible model, so the matrix build takes its
    general form (the symmetric one is what set_rate_matrix produces)."""
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(14 if S < 256 else 6, S, 4, 150 if S < 256 else 30, seed=77)
    V, Vi, lam = pg.eigen_reversible(w.Q, w.pi)
    c = np.random.default_rng(7).uniform(0.5, 2.0, S)
    ref = oracle_eval(w)
    ctx = pg.from_workload(w, precision)
    ctx.set_eigen(V * c, Vi / c[:, None], lam, w.pi)
    logL, grad = ctx.evaluate()
    compare(logL, grad, ref, precision, "general eigen form")
    ctx.close()
