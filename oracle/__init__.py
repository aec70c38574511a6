"""Oracle: plain, slow, FP64 CPU implementation of the Multipolynomial Monte
Carlo hot path, written from the paper (Lashomb, Morgan, Whyte, Wilcox,
"Multipolynomial Monte Carlo Trace Estimation", Lattice 2023).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; it
is used by the tests, by ``__graft_entry__.smoke()`` and by the benchmark's
CPU-baseline leg.  It shares no code with the CUDA path: the only common
module is ``synth`` (seeded gauge fields and workload numbers).

Every function cites the passage of the paper it follows.  Where the paper
is silent the reading taken is stated in the function's docstring.
"""
