"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the trace-estimation method: it only draws
gauge fields, generic test vectors and the workload parameter sets.  The
random numbers that the method itself draws (the Z(4) noise) are not made
here; each side implements the counter-based generator on its own.
"""
from .gauge import random_gauge, unit_gauge, random_spinor, gauge_transform_matrices
from .workloads import WORKLOADS, Workload

__all__ = ["random_gauge", "unit_gauge", "random_spinor", "gauge_transform_matrices",
           "WORKLOADS", "Workload"]
