"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle's tests."""
from .lofar import SPECS, ProblemSpec, make_problem, pack_uniform, agent_slices, user_layout

__all__ = ["SPECS", "ProblemSpec", "make_problem", "pack_uniform", "agent_slices", "user_layout"]
