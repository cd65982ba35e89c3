"""The autograd Function over log branch lengths: forward = post-order pass,
backward = pre-order pass with the fused gradient kernel.  Checked against
finite differences (gradcheck in FP64 on small trees; central differences
of the FP64 path on sampled entries at full size) and against the oracle
gradient with the chain rule for t = exp(log t)."""
import numpy as np
import pytest

import synth
from parity import TOL, oracle_eval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04390_gb300 import build as B
    B.build()


def test_gradcheck_fp64_small_tree():
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(6, 20, 2, 30, seed=31)
    ctx = pg.from_workload(w, "fp64")
    log_t = torch.tensor(np.log(w.t), dtype=torch.float64, device="cuda",
                         requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: pg.branch_loglik(x, ctx),
                                    (log_t,), eps=1e-6, atol=1e-6, rtol=1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_backward_matches_oracle_with_chain_rule(precision):
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(30, 20, 4, 200, seed=32)
    ctx = pg.from_workload(w, precision)
    log_t = torch.tensor(np.log(w.t), dtype=torch.float64, device="cuda",
                         requires_grad=True)
    ll = pg.branch_loglik(log_t, ctx)
    ll.backward()
    ll_ref, g_ref, A, B = oracle_eval(w)
    tol = TOL[precision]
    assert abs(ll.item() - ll_ref) <= tol["ll_rel"] * abs(ll_ref)
    got = log_t.grad.cpu().numpy()
    want = g_ref * w.t
    bound = np.maximum(tol["g_rel"] * np.abs(want), tol["g_cond"] * B * w.t)
    assert np.all(np.abs(got - want) <= bound)


def test_backward_needs_forward():
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(8, 4, 2, 20, seed=33)
    ctx = pg.from_workload(w, "fp32")
    g = torch.empty(2 * w.n_tips - 2, dtype=torch.float64, device="cuda")
    import ctypes
    from paper_2303_04390_gb300 import _native as N
    rc = N.load().phylo_backward_device(ctx._ctx, ctypes.c_void_p(g.data_ptr()), 0)
    assert rc == N.PHYLO_ESTATE


def test_two_forwards_then_backward():
    """Two forwards on one context before a backward: the C ABI refuses the
    first forward's backward (its partials were overwritten), and the
    autograd Function then recomputes that forward, so each graph gets its
    own gradient, in either order."""
    import ctypes
    import paper_2303_04390_gb300 as pg
    from paper_2303_04390_gb300 import _native as N
    w = synth.small_workload(16, 4, 4, 90, seed=35)
    ctx = pg.from_workload(w, "fp32")
    lib = N.load()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(2 * w.n_tips - 2, dtype=torch.float64, device="cuda")
    gens = []
    for scale in (1.0, 1.3):
        ctx.set_branch_lengths(w.t * scale)
        gen = ctypes.c_uint64(0)
        assert lib.phylo_forward_device(ctx._ctx, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.byref(gen)) == 0
        gens.append(gen.value)
    assert gens[1] > gens[0]
    assert lib.phylo_backward_device(ctx._ctx, ctypes.c_void_p(g.data_ptr()),
                                     gens[0]) == N.PHYLO_ESTATE
    assert lib.phylo_backward_device(ctx._ctx, ctypes.c_void_p(g.data_ptr()),
                                     gens[1]) == 0
    tol = TOL["fp32"]
    for order in ((0, 1), (1, 0)):
        lts = [torch.tensor(np.log(w.t * s), dtype=torch.float64, device="cuda",
                            requires_grad=True) for s in (1.0, 1.3)]
        lls = [pg.branch_loglik(lt, ctx) for lt in lts]
        for k in order:
            lls[k].backward()
        for lt, s in zip(lts, (1.0, 1.3)):
            ref = oracle_eval(w, t=w.t * s)
            want = ref[1] * w.t * s
            bound = np.maximum(tol["g_rel"] * np.abs(want),
                               tol["g_cond"] * ref[3] * w.t * s)
            assert np.all(np.abs(lt.grad.cpu().numpy() - want) <= bound), (order, s)


def test_forward_backward_agree_with_evaluate_over_steps():
    """An HMC-like sequence of forward/backward calls gives what full
    evaluations give, bit for bit (same kernels, same order)."""
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(40, 4, 4, 300, seed=34)
    a = pg.from_workload(w, "fp32")
    b = pg.from_workload(w, "fp32")
    rng = np.random.default_rng(0)
    for _ in range(3):
        t = w.t * np.exp(0.1 * rng.standard_normal(w.t.shape))
        log_t = torch.tensor(np.log(t), dtype=torch.float64, device="cuda",
                             requires_grad=True)
        ll = pg.branch_loglik(log_t, a)
        ll.backward()
        b.set_branch_lengths(torch.tensor(t, dtype=torch.float64, device="cuda"))
        ll2, g2 = b.evaluate()
        assert ll.item() == ll2
        np.testing.assert_allclose(log_t.grad.cpu().numpy(),
                                   g2 * torch.tensor(t).numpy(), rtol=1e-15)


def test_full_size_amino_acid_against_finite_differences():
    """The 256-taxon, 20-state workload: the FP32 autograd gradient w.r.t.
    log t against central differences of the FP64 path on sampled
    branches (Richardson-extrapolated)."""
    import paper_2303_04390_gb300 as pg
    w = synth.workload_aa_256(0)
    ctx32 = pg.from_workload(w, "fp32")
    ctx64 = pg.from_workload(w, "fp64")
    log_t = torch.tensor(np.log(w.t), dtype=torch.float64, device="cuda",
                         requires_grad=True)
    pg.branch_loglik(log_t, ctx32).backward()
    got = log_t.grad.cpu().numpy()

    def f(lt):
        ctx64.set_branch_lengths(np.exp(lt))
        return ctx64.evaluate(gradient=False)

    B = oracle_eval(w, shards=8)[3]  # conditioning scales (d/dt)
    base = np.log(w.t)
    rng = np.random.default_rng(7)
    for b in rng.choice(len(base), size=6, replace=False):
        def D(h):
            tp, tm = base.copy(), base.copy()
            tp[b] += h
            tm[b] -= h
            return (f(tp) - f(tm)) / (2 * h)
        fd = (4 * D(5e-4) - D(1e-3)) / 3
        tol = TOL["fp32"]
        bound = max(tol["g_rel"] * abs(fd), tol["g_cond"] * B[b] * w.t[b])
        assert abs(got[b] - fd) <= bound, (b, got[b], fd, bound)
