"""Near-null space, tentative prolongator and prolongator smoothing (Sec. 2.2).

* Near-null space of 3D elasticity: the six rigid-body modes.  For a fine node
  at x relative to its aggregate's centroid, the 3x6 block is
  [I_3 | (-y, x, 0) (0, -z, y) (z, 0, -x)] (translations, then rotations about
  z, x and y).  Rows of clamped nodes are zero.  On coarse levels the near-null
  block of a coarse node is the 6x6 R factor of its aggregate.
* Tentative prolongator (Sec. 2.2): per aggregate, the thin QR factorisation of
  the stacked near-null blocks B_agg = Q R with diag(R) > 0 (unique for full
  rank).  The rows of Q are the prolongator's blocks (one per node, in the
  aggregate's column), so P~ reproduces the near-null space exactly:
  P~ B_c = B.  Rows that are zero in B are zero in Q = B R^{-1}.
* Smoothed prolongator (Sec. 2.2): P = (I - omega D^{-1} A) P~ with D the
  (scalar) diagonal of A and omega = 4 / (3 lam), lam the largest-eigenvalue
  estimate of D^{-1} A.  The structural pattern of P is that of P~ united with
  pattern(A) * pattern(P~).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .assembly import BlockMatrix, to_blocks
from .smoother import power_lambda

OMEGA_NUMERATOR = 4.0 / 3.0


def rigid_body_modes(coords: np.ndarray, agg: np.ndarray, n_agg: int,
                     dirichlet: np.ndarray) -> np.ndarray:
    """(n_nodes, 3, 6) rigid-body blocks centred on each aggregate's centroid
    (nodes outside every aggregate, agg = -1, get zero blocks)."""
    inside = agg >= 0
    a = np.where(inside, agg, 0)
    counts = np.bincount(agg[inside], minlength=n_agg).astype(np.float64)
    cen = np.stack([np.bincount(agg[inside], weights=coords[inside, d], minlength=n_agg) for d in range(3)], 1)
    cen /= np.maximum(counts, 1.0)[:, None]
    rel = coords - cen[a]
    x, y, z = rel[:, 0], rel[:, 1], rel[:, 2]
    B = np.zeros((coords.shape[0], 3, 6))
    B[:, 0, 0] = B[:, 1, 1] = B[:, 2, 2] = 1.0
    B[:, 0, 3], B[:, 1, 3] = -y, x
    B[:, 1, 4], B[:, 2, 4] = -z, y
    B[:, 0, 5], B[:, 2, 5] = z, -x
    B[np.asarray(dirichlet).astype(bool)] = 0.0
    B[~inside] = 0.0
    return B


def tentative_prolongator(Bn: np.ndarray, agg: np.ndarray, n_agg: int) -> tuple[BlockMatrix, np.ndarray]:
    """P~ (one bs x 6 block per aggregated node, column = its aggregate; no
    block for a node outside every aggregate, agg = -1) and coarse blocks R."""
    n_nodes, bs, k = Bn.shape
    Q_nodes = np.zeros((n_nodes, bs, k))
    Bc = np.zeros((n_agg, k, k))
    order = np.argsort(agg, kind="stable")
    order = order[agg[order] >= 0]
    starts = np.searchsorted(agg[order], np.arange(n_agg + 1))
    for a in range(n_agg):
        nodes = order[starts[a]:starts[a + 1]]
        Bagg = Bn[nodes].reshape(-1, k)
        if Bagg.shape[0] < k:
            raise ValueError(f"aggregate {a} has fewer rows than near-null vectors")
        Q, R = np.linalg.qr(Bagg, mode="reduced")
        s = np.sign(np.diag(R))
        if np.any(s == 0) or np.min(np.abs(np.diag(R))) < 1e-12 * np.max(np.abs(np.diag(R))):
            raise ValueError(f"aggregate {a}: near-null space is rank deficient")
        Q = Q * s[None, :]
        R = R * s[:, None]
        zero_rows = ~np.any(Bagg != 0.0, axis=1)
        Q[zero_rows] = 0.0
        Q_nodes[nodes] = Q.reshape(-1, bs, k)
        Bc[a] = R
    inside = agg >= 0
    rowptr = np.zeros(n_nodes + 1, dtype=np.int64)
    np.cumsum(inside, out=rowptr[1:])
    P = BlockMatrix(n_nodes, n_agg, bs, k, rowptr, agg[inside].astype(np.int64), Q_nodes[inside])
    return P, Bc


def scalar_diagonal_lambda(As: sp.spmatrix) -> float:
    Ds = As.diagonal()
    return power_lambda(As, lambda v: v / Ds, lambda v: float(v @ (Ds * v)))


def smoothed_prolongator(A: BlockMatrix, Pt: BlockMatrix) -> tuple[BlockMatrix, float]:
    """P = P~ - omega D^{-1} (A P~) on pattern(P~) U pattern(A) pattern(P~); returns (P, omega)."""
    As = A.scalar()
    Ds = As.diagonal()
    lam = scalar_diagonal_lambda(As)
    omega = OMEGA_NUMERATOR / lam
    Pts = Pt.scalar()
    vals = Pts - sp.diags(omega / Ds) @ (As @ Pts)
    struct = A.structure() @ Pt.structure() + Pt.structure()
    return to_blocks(vals, struct, A.bs_r, Pt.bs_c), omega
