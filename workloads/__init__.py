"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds only input generation (points, targets, partitions,
support sets, hyperparameters).  None of the LMA arithmetic lives here, so
both the oracle and the GPU library can consume the same arrays without
sharing any of the method's code.
"""
from .synth import Problem, make_problem, make_random_problem, make_replicated, make_toy, CONFIG_NAMES  # noqa: F401
