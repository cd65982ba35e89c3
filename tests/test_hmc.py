"""HMC over log branch lengths (the paper's use case): the generic
integrator on CPU against a Gaussian target, and on the GPU the library-
backed posterior's gradient against the oracle, concurrent chains against
solo runs, and acceptance."""
import numpy as np
import pytest
import torch

from paper_2303_04390_gb300.hmc import (ChainState, accept, hamiltonian, leapfrog,
                                         propose)


def _gauss(prec):
    P = torch.tensor(prec, dtype=torch.float64)

    def logp_grad(theta):
        g = -(P @ theta)
        return 0.5 * torch.dot(theta, g), g
    return logp_grad


PREC = np.array([[2.0, 0.3, 0.0], [0.3, 1.0, 0.2], [0.0, 0.2, 0.5]])


def test_leapfrog_is_reversible_and_second_order():
    f = _gauss(PREC)
    th0 = torch.tensor([0.3, -1.2, 0.8], dtype=torch.float64)
    p0 = torch.tensor([0.5, 0.1, -0.7], dtype=torch.float64)
    lp0, g0 = f(th0)
    th1, p1, lp1, g1 = leapfrog(f, th0, p0, g0, 0.05, 20)
    th2, p2, _, _ = leapfrog(f, th1, -p1, g1, 0.05, 20)
    assert torch.allclose(th2, th0, atol=1e-12) and torch.allclose(-p2, p0, atol=1e-12)
    errs = []
    for eps in (0.04, 0.02):
        n = int(round(0.8 / eps))
        _, p, lp, _ = leapfrog(f, th0, p0, g0, eps, n)
        errs.append(abs(float(hamiltonian(lp, p) - hamiltonian(lp0, p0))))
    assert 3.0 < errs[0] / errs[1] < 5.0  # energy error O(eps^2)


def test_sampler_recovers_a_gaussian():
    f = _gauss(PREC)
    th = torch.zeros(3, dtype=torch.float64)
    lp, g = f(th)
    st = ChainState(th, lp, g)
    gen = torch.Generator().manual_seed(5)
    rng = np.random.default_rng(5)
    draws = []
    for _ in range(3000):
        accept(st, propose(f, st, 0.3, 8, gen), float(rng.uniform()))
        draws.append(st.theta.numpy().copy())
    x = np.array(draws[500:])
    cov = np.linalg.inv(PREC)
    assert np.all(np.abs(x.mean(0)) < 0.15)
    assert np.all(np.abs(np.cov(x.T) - cov) < 0.25 * np.max(np.abs(cov)))
    assert st.accepted / st.proposed > 0.6


@pytest.mark.gpu
def test_branch_posterior_matches_oracle():
    import synth
    import paper_2303_04390_gb300 as pg
    from oracle import phylo_oracle as O
    from paper_2303_04390_gb300.hmc import BranchPosterior
    w = synth.small_workload(16, 4, 4, 120, seed=71)
    ctx = pg.from_workload(w, "fp64")
    post = BranchPosterior(ctx, prior_rate=5.0)
    theta = torch.tensor(np.log(w.t), dtype=torch.float64, device="cuda")
    lp, g = post(theta)
    ll, g_ref, _ = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                              w.pattern_weights, tip_states=w.tip_states)
    lp_ref = ll - 5.0 * w.t.sum() + np.log(w.t).sum()
    gt_ref = (g_ref - 5.0) * w.t + 1.0
    assert abs(float(lp) - lp_ref) <= 1e-10 * abs(lp_ref)
    assert np.allclose(g.cpu().numpy(), gt_ref, rtol=1e-9, atol=1e-9 * np.abs(gt_ref).max())
    ctx.close()


@pytest.mark.gpu
def test_concurrent_chains_equal_solo_chains_and_accept():
    import synth
    from paper_2303_04390_gb300.hmc import make_chain, run_chains
    ws = [synth.small_workload(20, 4, 4, 200, seed=72),
          synth.small_workload(12, 20, 4, 150, seed=73)]

    def chains():
        return [make_chain(w, np.log(w.t), seed=100 + i) for i, w in enumerate(ws)]

    together = chains()
    rates = run_chains(together, 8, 0.02, 5)
    solo = []
    for ch in chains():
        run_chains([ch], 8, 0.02, 5)
        solo.append(ch)
    for a, b in zip(together, solo):
        assert a.state.trace == b.state.trace
        assert torch.equal(a.state.theta, b.state.theta)
    assert all(r >= 0.5 for r in rates), rates
    for ch in together + solo:
        ch.post.ctx.close()
