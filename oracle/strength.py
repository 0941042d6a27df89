"""Strength-of-connection graph and MIS aggregation from block norms (test infrastructure).

Smoothed aggregation couples node i to node j strongly when
|a_ij| >= eps sqrt(a_ii a_jj) (Sec. 2.2).  The blocked path takes that test on
the bs x bs blocks themselves, with the block norm as the coupling weight
(Sec. 3.2: one graph edge per stored block, weighted by its norm), and the
device coarsener is a Luby-round maximal independent set with deterministic
hash weights (Sec. 6).

Readings (the paper states the formula for scalars and names the norm only):
* The block norm is the Frobenius norm.  The test is taken on squares so that
  no square root enters a decision: with s = sum of the squared entries of a
  block, summed in row-major order, j is a strong neighbour of i when j != i,
  s_ij > 0 (a stored zero block is no coupling) and s_ij * s_ij >=
  (eps^4 * s_ii) * s_jj, with eps^4 = (eps * eps) * (eps * eps).  Every step is
  one IEEE double operation, rounded separately, so the decision is exact and
  reproducible.
* Vertex weights: w_i = splitmix64(i, seed), ties broken by the vertex number:
  (w_i, i) is a total order.
* The independent set is the fixed point of Luby rounds with these weights; it
  equals the greedy set that takes vertices in descending (w, i) order.
* Aggregates: one per selected vertex (a root), numbered by root in
  increasing vertex order; every other vertex joins its strong neighbour root
  of largest (w, j).  A vertex without strong neighbours is a root of its own.
The operators here are symmetric, so the row-wise graph is symmetric.
"""
from __future__ import annotations

import numpy as np

from .assembly import BlockMatrix
from .splitmix import splitmix64


def block_sumsq(A: BlockMatrix) -> np.ndarray:
    """Sum of squared entries of every stored block, accumulated in row-major order."""
    v = A.vals.reshape(A.nnzb, -1)
    s = np.zeros(A.nnzb)
    for e in range(v.shape[1]):
        s = s + v[:, e] * v[:, e]
    return s


def frobenius_norm(A: BlockMatrix) -> float:
    """Frobenius norm of the whole matrix (MatNorm over the blocks)."""
    return float(np.sqrt(np.sum(block_sumsq(A))))


def inf_norm(A: BlockMatrix) -> float:
    """Largest absolute row sum of the scalar matrix."""
    rows = np.zeros(A.nbr * A.bs_r)
    br = A.block_rows()
    absrow = np.abs(A.vals).sum(axis=2)  # (nnzb, bs_r)
    for a in range(A.bs_r):
        np.add.at(rows, br * A.bs_r + a, absrow[:, a])
    return float(rows.max()) if rows.size else 0.0


def strength_graph(A: BlockMatrix, eps: float) -> tuple[np.ndarray, np.ndarray]:
    """CSR graph (rowptr, col) of the strong couplings, columns in stored order."""
    if A.nbr != A.nbc or A.bs_r != A.bs_c:
        raise ValueError("the strength graph needs a square operator")
    s = block_sumsq(A)
    br = A.block_rows()
    diag = np.zeros(A.nbr)
    is_diag = A.colidx == br
    diag[br[is_diag]] = s[is_diag]
    eps2 = eps * eps
    eps4 = eps2 * eps2
    rhs = (eps4 * diag[br]) * diag[A.colidx]
    strong = (A.colidx != br) & (s > 0.0) & (s * s >= rhs)
    counts = np.bincount(br[strong], minlength=A.nbr)
    rowptr = np.zeros(A.nbr + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, A.colidx[strong].astype(np.int64)


def weights(n: int, seed: int) -> np.ndarray:
    return splitmix64(np.arange(n, dtype=np.uint64), seed)


def _key(w: np.ndarray, i: int) -> tuple[int, int]:
    return int(w[i]), i


def mis_greedy(rowptr: np.ndarray, col: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Greedy maximal independent set taking vertices in descending (w, i) order."""
    n = rowptr.size - 1
    order = sorted(range(n), key=lambda i: _key(w, i), reverse=True)
    state = np.zeros(n, dtype=np.int8)  # 0 free, 1 in the set, 2 blocked
    for i in order:
        if state[i] != 0:
            continue
        state[i] = 1
        for j in col[rowptr[i]:rowptr[i + 1]]:
            if state[j] == 0:
                state[j] = 2
    return state == 1


def mis_luby(rowptr: np.ndarray, col: np.ndarray, w: np.ndarray) -> tuple[np.ndarray, int]:
    """Luby rounds with fixed weights: an undecided vertex enters when its (w, i)
    beats every undecided neighbour; then the undecided neighbours of entered
    vertices leave.  Returns the set and the number of rounds."""
    n = rowptr.size - 1
    state = np.zeros(n, dtype=np.int8)  # 0 undecided, 1 in, 2 out
    rounds = 0
    while (state == 0).any():
        rounds += 1
        enter = []
        for i in np.flatnonzero(state == 0):
            ki = _key(w, i)
            if all(state[j] != 0 or _key(w, j) < ki for j in col[rowptr[i]:rowptr[i + 1]]):
                enter.append(i)
        state[enter] = 1
        for i in np.flatnonzero(state == 0):
            if (state[col[rowptr[i]:rowptr[i + 1]]] == 1).any():
                state[i] = 2
    return state == 1, rounds


def mis_aggregates(rowptr: np.ndarray, col: np.ndarray, w: np.ndarray, in_set: np.ndarray) -> np.ndarray:
    """Aggregate of every vertex: roots numbered in vertex order; others join the
    neighbour root of largest (w, j)."""
    n = rowptr.size - 1
    root_id = np.cumsum(in_set) - 1
    agg = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        if in_set[i]:
            agg[i] = root_id[i]
            continue
        best = -1
        for j in col[rowptr[i]:rowptr[i + 1]]:
            if in_set[j] and (best < 0 or _key(w, j) > _key(w, best)):
                best = j
        if best < 0:
            raise ValueError(f"vertex {i} has no neighbour in the set: the set is not maximal")
        agg[i] = root_id[best]
    return agg


def _rank_ok(Bagg: np.ndarray) -> bool:
    """Full column rank by the QR test the tentative prolongator applies."""
    if Bagg.shape[0] < Bagg.shape[1]:
        return False
    R = np.linalg.qr(Bagg, mode="r")
    d = np.abs(np.diag(R))
    return bool(d.min() >= 1e-12 * d.max())


def hierarchy_aggregates(A: BlockMatrix, eps: float, seed: int, near_null) -> tuple[np.ndarray, int]:
    """Aggregates of one level of the MIS-driven hierarchy (readings of Sec. 3.2
    and Sec. 6 where the paper is silent):

    1. MIS aggregates of the strength graph with weights splitmix64(i, seed).
    2. A vertex with no strong neighbour (a clamped node, or one decoupled by
       eps) is left out of every aggregate (-1): its prolongator row is empty.
    3. An aggregate whose near-null block (its members' rows, in vertex order,
       centred on the members' centroid at the fine level) is rank deficient
       is dissolved: each of its vertices joins, among the surviving
       aggregates of its strong neighbours, the one whose root has the largest
       (weight, root); a vertex with no such neighbour is left out.
    4. The surviving aggregates are renumbered in root order.

    near_null(members) returns the stacked near-null rows of those vertices.
    Returns (aggregate of every vertex or -1, number of aggregates)."""
    rowptr, col = strength_graph(A, eps)
    w = weights(A.nbr, seed)
    in_set = mis_greedy(rowptr, col, w)
    agg = mis_aggregates(rowptr, col, w, in_set)
    roots = np.flatnonzero(in_set)
    deg = np.diff(rowptr)
    agg[deg == 0] = -1
    n_agg = roots.size
    members = [[] for _ in range(n_agg)]
    for v in range(A.nbr):
        if agg[v] >= 0:
            members[agg[v]].append(v)
    dissolved = np.array([len(m) > 0 and not _rank_ok(near_null(np.array(m))) for m in members], dtype=bool)
    out = agg.copy()
    for v in range(A.nbr):
        if agg[v] < 0 or not dissolved[agg[v]]:
            continue
        best = -1
        for j in col[rowptr[v]:rowptr[v + 1]]:
            a = agg[j]
            if a >= 0 and not dissolved[a] and (best < 0 or _key(w, roots[a]) > _key(w, roots[best])):
                best = a
        out[v] = best
    keep = np.array([len(m) > 0 and not d for m, d in zip(members, dissolved)], dtype=bool)
    if not keep.any():
        raise ValueError("no aggregate survives: every aggregate's near-null block is rank deficient")
    renum = np.cumsum(keep) - 1
    out = np.where(out >= 0, renum[np.maximum(out, 0)], -1)
    return out.astype(np.int64), int(keep.sum())
