"""Hamiltonian Monte Carlo over log branch lengths: the use the paper builds
its gradient for (Introduction and Results: HMC transition kernels that
need d log P(Y) / d t at every leapfrog step).  Each leapfrog step costs one
library evaluation (log P(Y) and all 2N-2 derivatives); many independent
chains run concurrently, each on its own CUDA stream, so their evaluations
overlap on the GPU the way served requests do.

The integrator (leapfrog, Metropolis correction) is generic: it takes a
callable returning (log density, gradient) and works on CPU or CUDA
tensors.  BranchPosterior supplies that callable for a tree:

  log p(theta | Y) = log P(Y | t) + sum_i log Exp(t_i; lambda) + sum_i theta_i,
  t = exp(theta),

the last sum being the Jacobian of t = exp(theta), so that
  d/d theta_i = (d log P / d t_i - lambda) t_i + 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional, Tuple

import numpy as np
import torch

LogpGrad = Callable[[torch.Tensor], Tuple[torch.Tensor, torch.Tensor]]


def leapfrog(logp_grad: LogpGrad, theta, p, grad, eps: float, n_steps: int):
    """n_steps leapfrog steps of size eps from (theta, p) with gradient
    `grad` at theta; returns (theta, p, logp, grad) at the end."""
    p = p + 0.5 * eps * grad
    logp = None
    for s in range(n_steps):
        theta = theta + eps * p
        logp, grad = logp_grad(theta)
        if s + 1 < n_steps:
            p = p + eps * grad
    p = p + 0.5 * eps * grad
    return theta, p, logp, grad


def hamiltonian(logp, p):
    return -logp + 0.5 * torch.sum(p * p)


@dataclass
class ChainState:
    theta: torch.Tensor
    logp: torch.Tensor
    grad: torch.Tensor
    accepted: int = 0
    proposed: int = 0
    trace: List[float] = field(default_factory=list)


def propose(logp_grad: LogpGrad, st: ChainState, eps: float, n_steps: int,
            gen: torch.Generator):
    """One HMC proposal from st (asynchronous on the current stream):
    returns (theta', logp', grad', log acceptance ratio) as tensors."""
    p0 = torch.randn(st.theta.shape, generator=gen, dtype=st.theta.dtype,
                     device=st.theta.device)
    h0 = hamiltonian(st.logp, p0)
    th, p1, lp, gr = leapfrog(logp_grad, st.theta, p0, st.grad, eps, n_steps)
    log_ratio = h0 - hamiltonian(lp, p1)
    return th, lp, gr, log_ratio


def accept(st: ChainState, prop, u: float) -> bool:
    """Metropolis correction with a uniform draw u (host)."""
    th, lp, gr, log_ratio = prop
    st.proposed += 1
    lr = float(log_ratio)
    ok = bool(np.isfinite(lr)) and np.log(u) < min(0.0, lr)
    if ok:
        st.theta, st.logp, st.grad = th, lp, gr
        st.accepted += 1
    st.trace.append(float(st.logp))
    return ok


class BranchPosterior:
    """log p(theta | Y) for theta = log t on a PhyloContext whose data,
    model and tree are set; gradients from the library (one evaluation per
    call, on the context's stream)."""

    def __init__(self, ctx, prior_rate: float = 10.0):
        self.ctx = ctx
        self.prior_rate = float(prior_rate)

    def __call__(self, theta: torch.Tensor):
        t = torch.exp(theta)
        self.ctx.set_branch_lengths(t)
        out = self.ctx.evaluate_device(
            torch.empty(theta.numel() + 1, dtype=torch.float64, device=theta.device))
        logp = out[0] - self.prior_rate * torch.sum(t) + torch.sum(theta)
        grad = (out[1:] - self.prior_rate) * t + 1.0
        return logp, grad


@dataclass
class Chain:
    """One chain: its posterior, CUDA stream, state and generators."""
    post: BranchPosterior
    stream: object
    state: ChainState
    gen: torch.Generator
    rng: np.random.Generator


def make_chain(w, theta0: np.ndarray, seed: int, precision: str = "fp32",
               prior_rate: float = 10.0, device: Optional[torch.device] = None) -> Chain:
    """A chain for workload w (synth.Workload-like) on its own stream."""
    from .context import from_workload
    device = device or torch.device("cuda")
    stream = torch.cuda.Stream(device=device)
    ctx = from_workload(w, precision, device=device, stream=stream)
    post = BranchPosterior(ctx, prior_rate)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    with torch.cuda.stream(stream):
        theta = torch.tensor(theta0, dtype=torch.float64, device=device)
        logp, grad = post(theta)
    return Chain(post, stream, ChainState(theta, logp.clone(), grad.clone()), gen,
                 np.random.default_rng(seed))


def run_chains(chains: List[Chain], n_iter: int, eps: float, n_steps: int):
    """n_iter HMC transitions of every chain.  Each iteration issues every
    chain's proposal on its own stream first (the trajectories overlap on
    the GPU), then reads back the acceptance ratios and decides on the
    host.  Returns the acceptance rate of each chain."""
    for _ in range(n_iter):
        props = []
        for ch in chains:
            with torch.cuda.stream(ch.stream):
                props.append(propose(ch.post, ch.state, eps, n_steps, ch.gen))
        for ch, prop in zip(chains, props):
            ch.stream.synchronize()
            accept(ch.state, prop, float(ch.rng.uniform()))
    for ch in chains:
        ch.post.ctx.check()
    return [ch.state.accepted / max(ch.state.proposed, 1) for ch in chains]
