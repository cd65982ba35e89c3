"""FP64 CPU oracle (test infrastructure only; see phylo_oracle)."""
from .phylo_oracle import *  # noqa: F401,F403
