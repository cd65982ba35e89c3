"""torch.autograd.Function over branch lengths, with the library's
pre-order pass as the hand-written backward.

forward(log_t):  t = exp(log_t); the matrix build, the post-order pass and
                 the log-likelihood reduction (phylo_forward_device)
backward(g):     the pre-order pass with the fused gradient kernel
                 (phylo_backward_device) gives d log P(Y) / d t; the chain
                 rule for t = exp(log_t) multiplies by t.

Both run on the context's stream; the log-likelihood and the gradient stay
on the device.  Each forward carries the generation number the library
gave its post-order pass; backward passes it back, and the library refuses
(PHYLO_ESTATE) if another pass has rewritten the context's partials since.
Backward then runs this graph's forward again from its saved branch
lengths and differentiates that, so two forwards on one context before a
backward (as torch.autograd.gradcheck does) give each graph its own
gradient, never the later forward's.  The context is left holding the
branch lengths of the graph differentiated last.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class BranchLogLik(torch.autograd.Function):
    """log P(Y) as a function of log branch lengths (FP64 CUDA tensor of
    2N-2 entries) for a PhyloContext whose other inputs are set."""

    @staticmethod
    def forward(fctx, log_t, phylo_ctx):
        assert log_t.is_cuda and log_t.dtype == torch.float64
        t = torch.exp(log_t).contiguous()
        phylo_ctx.set_branch_lengths(t)
        out = torch.empty(1, dtype=torch.float64, device=log_t.device)
        gen = ctypes.c_uint64(0)
        phylo_ctx._check(N.load().phylo_forward_device(
            phylo_ctx._ctx, _ptr(out), ctypes.byref(gen)))
        fctx.phylo_ctx = phylo_ctx
        fctx.generation = gen.value
        fctx.save_for_backward(t)
        return out[0]

    @staticmethod
    def backward(fctx, grad_out):
        (t,) = fctx.saved_tensors
        pc = fctx.phylo_ctx
        lib = N.load()
        g = torch.empty_like(t)
        rc = lib.phylo_backward_device(pc._ctx, _ptr(g), fctx.generation)
        if rc == N.PHYLO_ESTATE:
            # a later pass rewrote the partials: recompute this forward
            pc.set_branch_lengths(t)
            out = torch.empty(1, dtype=torch.float64, device=t.device)
            gen = ctypes.c_uint64(0)
            pc._check(lib.phylo_forward_device(pc._ctx, _ptr(out),
                                               ctypes.byref(gen)))
            rc = lib.phylo_backward_device(pc._ctx, _ptr(g), gen.value)
        pc._check(rc)
        return grad_out * g * t, None


def branch_loglik(log_t: torch.Tensor, phylo_ctx) -> torch.Tensor:
    """Differentiable log P(Y) of log branch lengths."""
    return BranchLogLik.apply(log_t, phylo_ctx)
