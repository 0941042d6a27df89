"""Point-block Jacobi, the largest-eigenvalue estimate and the Chebyshev smoother.

The paper's smoother is point-block Jacobi (``pbjacobi``, Sec. 4.1); the
workloads run it under Chebyshev acceleration of degree 2 in each of the pre-
and post-smoothing steps, V(2,2).

* Point-block Jacobi: D_b is the block diagonal of A (bs x bs per block row);
  its inverse is taken block by block with LU and partial pivoting.
* Eigenvalue estimate: 15 power iterations on D^{-1} A from the splitmix64
  start vector, 2-norm normalised, then the Rayleigh quotient
  v^T A v / v^T D v (the quotient of the generalised problem A v = lam D v).
* Chebyshev (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
  Algorithm 12.1, preconditioned by D): interval [alpha, beta] =
  [0.1 lam, 1.1 lam], theta = (beta + alpha) / 2, delta = (beta - alpha) / 2,
  sigma = theta / delta.  From r_0 = b - A x_0: d_0 = D^{-1} r_0 / theta,
  rho_0 = 1 / sigma, and for k = 0, 1, ...:
      x_{k+1} = x_k + d_k,     r_{k+1} = r_k - A d_k,
      rho_{k+1} = 1 / (2 sigma - rho_k),
      d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) D^{-1} r_{k+1}.
  Degree m takes m steps; the error is multiplied by
  T_m((theta - D^{-1}A) / delta) / T_m(theta / delta).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .assembly import BlockMatrix
from .splitmix import start_vector

CHEB_LOWER = 0.1
CHEB_UPPER = 1.1
POWER_ITS = 15


def diagonal_blocks(A: BlockMatrix) -> np.ndarray:
    D = np.zeros((A.nbr, A.bs_r, A.bs_c))
    for I in range(A.nbr):
        k = A.find(I, I)
        if k < 0:
            raise ValueError(f"block row {I} has no diagonal block")
        D[I] = A.vals[k]
    return D


def block_diag_inverse(A: BlockMatrix) -> np.ndarray:
    """Inverse of each diagonal block (LU with partial pivoting, via LAPACK)."""
    return np.linalg.inv(diagonal_blocks(A))


def apply_blocks(Db: np.ndarray, v: np.ndarray) -> np.ndarray:
    n, bs, _ = Db.shape
    return np.einsum("nij,nj->ni", Db, v.reshape(n, bs)).reshape(-1)


def power_lambda(As: sp.spmatrix, apply_dinv, quad_d, its: int = POWER_ITS) -> float:
    """Largest eigenvalue estimate of D^{-1} A (power iteration + Rayleigh quotient)."""
    v = start_vector(As.shape[0])
    for _ in range(its):
        w = apply_dinv(As @ v)
        v = w / np.linalg.norm(w)
    return float((v @ (As @ v)) / quad_d(v))


def block_jacobi_lambda(A: BlockMatrix, As: sp.spmatrix | None = None,
                        Dinv: np.ndarray | None = None, weights: np.ndarray | None = None) -> float:
    """Largest eigenvalue estimate of W D^{-1} A (W = per-block-row weights, I if None):
    the Rayleigh quotient of A v = lam M v with M = D W^{-1}."""
    As = A.scalar() if As is None else As
    D = diagonal_blocks(A)
    Dinv = np.linalg.inv(D) if Dinv is None else Dinv
    bs = D.shape[1]
    wr = np.ones(A.nbr) if weights is None else np.asarray(weights, dtype=np.float64)
    wd = np.repeat(wr, bs)
    return power_lambda(As, lambda v: wd * apply_blocks(Dinv, v),
                        lambda v: float(v @ (apply_blocks(D, v) / wd)))


def chebyshev(As: sp.spmatrix, Dinv: np.ndarray, b: np.ndarray, x0: np.ndarray | None,
              lam: float, degree: int = 2, want_residual: bool = False,
              weights: np.ndarray | None = None):
    """Degree-``degree`` Chebyshev smoothing of A x = b from x0 (None = zero),
    preconditioned by W D^{-1} (W = per-block-row weights, I if None).

    Returns x, and also r = b - A x (carried by the recurrence) when
    ``want_residual``; in that case one more product A d is taken.
    """
    if weights is not None:
        wd = np.repeat(np.asarray(weights, dtype=np.float64), Dinv.shape[1])
        apply = lambda v: wd * apply_blocks(Dinv, v)  # noqa: E731
    else:
        apply = lambda v: apply_blocks(Dinv, v)  # noqa: E731
    alpha, beta = CHEB_LOWER * lam, CHEB_UPPER * lam
    theta = 0.5 * (beta + alpha)
    delta = 0.5 * (beta - alpha)
    sigma = theta / delta
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - As @ x
    d = apply(r) / theta
    rho = 1.0 / sigma
    for k in range(degree):
        x = x + d
        if k == degree - 1 and not want_residual:
            break
        r = r - As @ d
        if k == degree - 1:
            break
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * apply(r)
        rho = rho_new
    return (x, r) if want_residual else x
