"""Many right-hand sides: the V-cycle and PCG applied to k vectors.

Test infrastructure.  The multi-vector forms compute, per column, exactly the
single-vector operations (Sec. 2.1 V-cycle, Sec. 4.1 PCG): the cycle is one
fixed linear operator M applied to every column, and the CG recurrences are
independent, each with its own step lengths, stopping test and iteration
count.  Written here as plain loops over the columns of B (n x k).
"""
from __future__ import annotations

import numpy as np

from . import krylov
from . import multigrid as omg


def vcycle_columns(h: omg.Hierarchy, B: np.ndarray) -> np.ndarray:
    """X[:, j] = M B[:, j]."""
    return np.stack([omg.vcycle(h, B[:, j]) for j in range(B.shape[1])], axis=1)


def pcg_columns(h: omg.Hierarchy, B: np.ndarray, rtol: float = 1e-8, maxit: int = 500):
    """Independent PCG solves of A x_j = b_j; returns (X, iterations, infos)."""
    As = h.levels[0].As
    X = np.zeros_like(B)
    its, infos = [], []
    for j in range(B.shape[1]):
        x, it, info = krylov.pcg(As, B[:, j], lambda r: omg.vcycle(h, r), rtol, maxit)
        X[:, j] = x
        its.append(it)
        infos.append(info)
    return X, its, infos
