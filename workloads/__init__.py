"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds problem inputs only: the trilinear (Q1) hexahedral
elasticity mesh, its element stiffness, the blocked COO value stream, the
load vector, seeded perturbations and right-hand sides.  It holds none of the
multigrid method's arithmetic (no assembly sums, no aggregation, no Galerkin
product, no smoothing): the oracle and the CUDA library each do those
themselves from the same stream.
"""
