"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Holds random draws and determinant bookkeeping only; no SA-DSRG arithmetic.
"""
from .problems import (  # noqa: F401
    Problem, make_problem, workload, WORKLOADS, CUTS, batch_sizes, batch_problem, random_density3, random_cumulant3,
)
