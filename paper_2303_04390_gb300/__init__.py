"""GB300-native log-likelihood and branch-length gradient on phylogenetic
trees (arXiv 2303.04390): a CUDA library for sm_103a behind a C ABI
(include/phylo_api.h) with a thin Python binding."""
from .context import PhyloContext, eigen_reversible, from_workload, workspace_bytes  # noqa: F401
from ._native import PhyloError  # noqa: F401


def branch_loglik(log_t, phylo_ctx):
    """Differentiable log P(Y) of log branch lengths (see autograd.py)."""
    from .autograd import branch_loglik as f
    return f(log_t, phylo_ctx)

__all__ = ["PhyloContext", "PhyloError", "branch_loglik", "eigen_reversible",
           "from_workload", "workspace_bytes"]
