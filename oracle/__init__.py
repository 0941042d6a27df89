"""Plain FP64 CPU oracle for the blocked SA-AMG reuse phase (test infrastructure).

This package is test infrastructure, not part of the library.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA path: it works on scalar CSR matrices
(``scipy.sparse``), builds everything from the plain definitions in the paper
(arxiv 2606.24748, Adams, "A Natively Blocked, Device-Resident Algebraic
Multigrid GPU Path in PETSc"), and uses library primitives (sparse and dense
matrix products, LAPACK QR, LU and Cholesky) only as whole steps.

Modules
  assembly     blocked COO -> scalar CSR with duplicate summation (Sec. 3.4, Sec. 5)
  aggregation  geometric 3x3x3 node aggregates (aggregation, Sec. 2.2)
  prolongator  rigid-body near-null space, tentative P by QR, smoothed P (Sec. 2.2)
  galerkin     A_c = P^T A P with the structural block pattern (Sec. 2.2, Sec. 3.1)
  smoother     point-block Jacobi inverse, eigenvalue estimate, Chebyshev (Sec. 4.1)
  multigrid    hierarchy setup / reuse update / V-cycle (Sec. 2.1, Sec. 3.1)
  krylov       preconditioned CG (Sec. 4.1)
  splitmix     the splitmix64 counter-based generator (start vectors)
  learned      features, targets, MLP and Adam of the learned smoother weights
  multi_rhs    many right-hand sides: the cycle and CG column by column
  strength     block-norm strength graph, Luby MIS and MIS aggregates (Sec. 2.2, 3.2, 6)
"""
