"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Holds random draws and determinant bookkeeping only; no SA-DSRG arithmetic.
"""
from .problems import Problem, make_problem, workload, WORKLOADS, CUTS, batch_sizes, batch_problem  # noqa: F401
