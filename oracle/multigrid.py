"""Smoothed-aggregation hierarchy: cold setup, hot reuse update, V-cycle.

Setup (Sec. 2.2): on each level, aggregate, build the tentative prolongator
from the near-null space, smooth it, and form A_c = P^T A P; coarsen while the
level has more than ``max_coarse_dofs`` dofs (2,100 reproduces every
workload's level count) or until ``max_levels``.

Reuse update (Sec. 3.1, Sec. 3.5): with the prolongators fixed, recompute the
Galerkin products on every level from a new fine operator, then refresh the
smoother data (block-diagonal inverses, eigenvalue estimates) and factor the
coarsest operator (dense Cholesky).

V-cycle (Sec. 2.1): from x = 0, pre-smooth, restrict the residual with P^T,
recurse (the coarsest level solves exactly), prolong and add the correction,
post-smooth.  Pre- and post-smoothing are the same degree-2 Chebyshev /
point-block Jacobi polynomial, so the cycle is a symmetric operator.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .aggregation import aggregates
from .assembly import BlockMatrix
from .galerkin import galerkin
from .prolongator import rigid_body_modes, smoothed_prolongator, tentative_prolongator
from .smoother import block_diag_inverse, block_jacobi_lambda, chebyshev

MAX_COARSE_DOFS = 2100


@dataclasses.dataclass
class Level:
    A: BlockMatrix
    grid: tuple[int, int, int]
    As: sp.csr_matrix | None = None
    P: BlockMatrix | None = None       # prolongator to this level from the next coarser
    Ps: sp.csr_matrix | None = None
    agg: np.ndarray | None = None
    omega: float = 0.0
    Dinv: np.ndarray | None = None
    lam: float = 0.0
    chol: np.ndarray | None = None     # lower Cholesky factor (coarsest level)
    Bc: np.ndarray | None = None
    weights: np.ndarray | None = None  # per-block-row smoother weights (None = plain)


@dataclasses.dataclass
class Hierarchy:
    levels: list[Level]
    degree: int = 2

    @property
    def n_levels(self) -> int:
        return len(self.levels)


def setup(A: BlockMatrix, coords: np.ndarray, dirichlet: np.ndarray,
          grid: tuple[int, int, int], max_coarse_dofs: int = MAX_COARSE_DOFS,
          max_levels: int = 10, degree: int = 2, aggregation: str = "geometric",
          eps: float = 0.02, seed: int = 1) -> Hierarchy:
    """aggregation: "geometric" (3x3x3 node cubes on the structured grid) or
    "mis" (MIS aggregates of each level's block strength graph, Sec. 3.2 and
    Sec. 6, with the readings of strength.hierarchy_aggregates; seed + level
    seeds the vertex weights of level l)."""
    levels = [Level(A=A, grid=grid)]
    Bn = None
    while (levels[-1].A.nbr * levels[-1].A.bs_r > max_coarse_dofs
           and len(levels) < max_levels):
        L = levels[-1]
        if aggregation == "mis":
            from .strength import hierarchy_aggregates
            l = len(levels) - 1
            if Bn is None:
                def near_null(m):  # rigid-body rows of the members about their centroid
                    sub = rigid_body_modes(coords[m], np.zeros(len(m), dtype=np.int64), 1, dirichlet[m])
                    return sub.reshape(-1, 6)
            else:
                Bprev = Bn
                near_null = lambda m: Bprev[m].reshape(-1, 6)  # noqa: E731
            agg, n_agg = hierarchy_aggregates(L.A, eps, seed + l, near_null)
            cgrid = None
        else:
            agg, cgrid = aggregates(L.grid)
            n_agg = int(np.prod(cgrid))
        if Bn is None:
            Bn = rigid_body_modes(coords, agg, n_agg, dirichlet)
        Pt, Bc = tentative_prolongator(Bn, agg, n_agg)
        P, omega = smoothed_prolongator(L.A, Pt)
        L.P, L.agg, L.omega, L.Bc = P, agg, omega, Bc
        levels.append(Level(A=galerkin(L.A, P), grid=cgrid))
        Bn = Bc
    h = Hierarchy(levels, degree)
    refresh(h)
    return h


def refresh(h: Hierarchy) -> None:
    """Smoother data on every non-coarsest level; Cholesky factor on the coarsest."""
    for L in h.levels:
        L.As = L.A.scalar()
        if L.P is not None:
            L.Ps = L.P.scalar()
    for L in h.levels[:-1]:
        L.Dinv = block_diag_inverse(L.A)
        L.lam = block_jacobi_lambda(L.A, L.As, L.Dinv, L.weights)
    C = h.levels[-1]
    C.chol = np.linalg.cholesky(C.A.dense())


def update(h: Hierarchy, A_new: BlockMatrix) -> Hierarchy:
    """Hot reuse step: same prolongators, new fine operator, new Galerkin products."""
    levels = [dataclasses.replace(L) for L in h.levels]
    levels[0].A = A_new
    for l in range(len(levels) - 1):
        levels[l + 1].A = galerkin(levels[l].A, levels[l].P)
    out = Hierarchy(levels, h.degree)
    refresh(out)
    return out


def coarse_solve(L: Level, b: np.ndarray) -> np.ndarray:
    y = sla.solve_triangular(L.chol, b, lower=True)
    return sla.solve_triangular(L.chol.T, y, lower=False)


def vcycle(h: Hierarchy, b: np.ndarray, level: int = 0) -> np.ndarray:
    L = h.levels[level]
    if level == h.n_levels - 1:
        return coarse_solve(L, b)
    x, r = chebyshev(L.As, L.Dinv, b, None, L.lam, h.degree, want_residual=True, weights=L.weights)
    ec = vcycle(h, L.Ps.T @ r, level + 1)
    x = x + L.Ps @ ec
    return chebyshev(L.As, L.Dinv, b, x, L.lam, h.degree, weights=L.weights)


def set_weights(h: Hierarchy, weights: list) -> None:
    """Per-block-row smoother weights for the non-coarsest levels (None entries
    keep the plain smoother); the eigen-estimates are refreshed for W D^{-1} A."""
    for L, w in zip(h.levels[:-1], weights):
        L.weights = None if w is None else np.asarray(w, dtype=np.float32).astype(np.float64)
    refresh(h)


def stationary(h: Hierarchy, b: np.ndarray, its: int) -> list[float]:
    """Residual norms of x_{k+1} = x_k + M (b - A x_k), x_0 = 0."""
    As = h.levels[0].As
    x = np.zeros_like(b)
    r = b.copy()
    out = [float(np.linalg.norm(r))]
    for _ in range(its):
        x = x + vcycle(h, r)
        r = b - As @ x
        out.append(float(np.linalg.norm(r)))
    return out
