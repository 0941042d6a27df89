"""Blocked COO assembly and block patterns, written on scalar CSR.

Blocked COO (Sec. 3.4 and Sec. 5): each coordinate (bi, bj) addresses a dense
bs_r x bs_c block; duplicates are summed.  The oracle expands every block into
its bs_r*bs_c scalar entries (keeping explicit zeros as structural entries) and
lets the scalar COO -> CSR conversion sum duplicates.  Entries with a negative
block coordinate are ignored.

The block pattern of a scalar matrix is the set of bs_r x bs_c tiles that hold
at least one structural scalar; block values are read back tile by tile.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class BlockMatrix:
    """Oracle block matrix: sorted block CSR pattern and dense tile values."""
    nbr: int
    nbc: int
    bs_r: int
    bs_c: int
    rowptr: np.ndarray     # int64 (nbr + 1,)
    colidx: np.ndarray     # int64 (nnzb,)
    vals: np.ndarray       # float64 (nnzb, bs_r, bs_c)

    @property
    def nnzb(self) -> int:
        return int(self.colidx.shape[0])

    def block_rows(self) -> np.ndarray:
        return np.repeat(np.arange(self.nbr), np.diff(self.rowptr))

    def scalar(self) -> sp.csr_matrix:
        """Scalar CSR with every tile entry structural (zeros kept)."""
        return _scalar_from_blocks(self.block_rows(), self.colidx, self.vals,
                                   self.nbr, self.nbc, self.bs_r, self.bs_c)

    def structure(self) -> sp.csr_matrix:
        """Scalar structure with value 1 on every structural entry."""
        return _scalar_from_blocks(self.block_rows(), self.colidx,
                                   np.ones_like(self.vals), self.nbr, self.nbc,
                                   self.bs_r, self.bs_c)

    def dense(self) -> np.ndarray:
        return self.scalar().toarray()

    def find(self, I: int, J: int) -> int:
        lo, hi = self.rowptr[I], self.rowptr[I + 1]
        k = lo + np.searchsorted(self.colidx[lo:hi], J)
        if k < hi and self.colidx[k] == J:
            return int(k)
        return -1


def _scalar_from_blocks(brow, bcol, vals, nbr, nbc, bs_r, bs_c) -> sp.csr_matrix:
    r = np.arange(bs_r)[None, :, None]
    c = np.arange(bs_c)[None, None, :]
    rows = np.broadcast_to(brow.astype(np.int64)[:, None, None] * bs_r + r, vals.shape)
    cols = np.broadcast_to(bcol.astype(np.int64)[:, None, None] * bs_c + c, vals.shape)
    A = sp.coo_matrix((vals.reshape(-1), (rows.reshape(-1), cols.reshape(-1))),
                      shape=(nbr * bs_r, nbc * bs_c)).tocsr()
    A.sort_indices()
    return A


def coo_assemble(nbr: int, nbc: int, bs_r: int, bs_c: int, bi, bj, vals) -> sp.csr_matrix:
    """Scalar CSR of a blocked COO stream: duplicates summed, zeros structural."""
    bi = np.asarray(bi, dtype=np.int64)
    bj = np.asarray(bj, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64).reshape(-1, bs_r, bs_c)
    keep = (bi >= 0) & (bj >= 0)
    return _scalar_from_blocks(bi[keep], bj[keep], vals[keep], nbr, nbc, bs_r, bs_c)


def block_pattern(structure: sp.spmatrix, bs_r: int, bs_c: int) -> tuple[np.ndarray, np.ndarray]:
    """(rowptr, colidx) of the tiles that contain a structural scalar."""
    S = structure.tocoo()
    nbr = S.shape[0] // bs_r
    nbc = S.shape[1] // bs_c
    key = np.unique((S.row.astype(np.int64) // bs_r) * nbc + S.col.astype(np.int64) // bs_c)
    I, J = key // nbc, key % nbc
    rowptr = np.zeros(nbr + 1, dtype=np.int64)
    np.add.at(rowptr, I + 1, 1)
    return np.cumsum(rowptr), J


def to_blocks(values: sp.spmatrix, structure: sp.spmatrix, bs_r: int, bs_c: int) -> BlockMatrix:
    """Block matrix on the tile pattern of ``structure`` with entries of ``values``.

    ``values`` may omit structural entries that happen to be zero; they read
    back as 0.0.
    """
    rowptr, colidx = block_pattern(structure, bs_r, bs_c)
    nbr = structure.shape[0] // bs_r
    nbc = structure.shape[1] // bs_c
    key_blocks = np.repeat(np.arange(nbr), np.diff(rowptr)) * nbc + colidx
    out = np.zeros((colidx.shape[0], bs_r, bs_c))
    V = values.tocoo()
    if V.nnz:
        kb = (V.row.astype(np.int64) // bs_r) * nbc + V.col.astype(np.int64) // bs_c
        slot = np.searchsorted(key_blocks, kb)
        if np.any(slot >= key_blocks.shape[0]) or np.any(key_blocks[np.minimum(slot, key_blocks.shape[0] - 1)] != kb):
            raise ValueError("value entry outside the structural pattern")
        np.add.at(out, (slot, V.row % bs_r, V.col % bs_c), V.data)
    return BlockMatrix(nbr, nbc, bs_r, bs_c, rowptr, colidx, out)


def coo_assemble_blocks(nbr: int, nbc: int, bs_r: int, bs_c: int, bi, bj, vals) -> BlockMatrix:
    A = coo_assemble(nbr, nbc, bs_r, bs_c, bi, bj, vals)
    return to_blocks(A, A, bs_r, bs_c)
