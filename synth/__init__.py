"""Seeded synthetic input generators shared by the CUDA path, the oracle,
the tests and the bench. Holds no likelihood or gradient arithmetic."""
from .workloads import *  # noqa: F401,F403
from .workloads import Workload, CONFIGS  # noqa: F401
