"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package describes problems (mesh shape, refinement lists, boundary
conditions) and evaluates input fields (right-hand side, coefficient,
boundary values) at cell and face centres.  It contains none of the
multigrid arithmetic: no operator, smoother, transfer or cycle.
"""
from .workloads import *  # noqa: F401,F403
