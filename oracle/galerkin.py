"""Galerkin coarse operator A_c = P^T A P (Sec. 2.1, Sec. 2.2, Sec. 3.1).

Values are the scalar triple product.  The structural pattern is the product
of the scalar structures (every stored tile entry counts, explicit zeros
included; no value-based pruning), read off as 6x6 tiles.
"""
from __future__ import annotations

from .assembly import BlockMatrix, to_blocks


def ap_pattern(A: BlockMatrix, P: BlockMatrix):
    """Structure of the intermediate product A P (for pattern checks)."""
    return A.structure() @ P.structure()


def galerkin(A: BlockMatrix, P: BlockMatrix) -> BlockMatrix:
    As, Ps = A.scalar(), P.scalar()
    vals = Ps.T @ (As @ Ps)
    Ss = P.structure()
    struct = Ss.T @ (A.structure() @ Ss)
    return to_blocks(vals, struct, P.bs_c, P.bs_c)
