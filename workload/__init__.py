"""Seeded synthetic workload generators shared by the tests, the benchmark and the oracle's callers.

This package holds no arithmetic of the FliX method itself: it only draws keys, values, operation
mixes and batch sizes.  Both the CUDA path and the CPU oracle receive its arrays as plain inputs.
"""
from .gen import *  # noqa: F401,F403
