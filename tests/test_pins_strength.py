"""Pins of the oracle's strength graph, MIS and MIS aggregates (Sec. 2.2, 3.2, 6)."""
import numpy as np
import pytest

from oracle.assembly import BlockMatrix, coo_assemble_blocks
from oracle import strength as st

from oracle_cases import problem


def block_matrix(blocks: dict, n: int, bs: int) -> BlockMatrix:
    rowptr = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        js = sorted(j for (r, j) in blocks if r == i)
        rowptr[i + 1] = rowptr[i] + len(js)
        cols += js
        vals += [np.asarray(blocks[(i, j)], dtype=float) for j in js]
    return BlockMatrix(n, n, bs, bs, rowptr, np.asarray(cols, dtype=np.int64), np.asarray(vals).reshape(-1, bs, bs))


def test_block_sums_of_squares_are_squared_frobenius_norms():
    rng = np.random.default_rng(0)
    blocks = {(i, j): rng.standard_normal((3, 3)) for i in range(4) for j in range(4) if abs(i - j) <= 1}
    A = block_matrix(blocks, 4, 3)
    s = st.block_sumsq(A)
    ref = np.array([np.linalg.norm(b, "fro") ** 2 for b in A.vals])
    assert np.allclose(s, ref, rtol=1e-15, atol=0)
    assert st.frobenius_norm(A) == pytest.approx(np.linalg.norm(A.dense(), "fro"), rel=1e-15)
    assert st.inf_norm(A) == pytest.approx(np.abs(A.dense()).sum(axis=1).max(), rel=1e-15)


def test_hand_example_takes_the_threshold_inclusively():
    # s_DD = 8, s_B = 2, s_C = 0.02; eps = 0.5: eps^4 s_ii s_jj = 4 = s_B^2 -> strong (>=), C weak
    D, Bb, C = 2 * np.eye(2), np.eye(2), 0.1 * np.eye(2)
    A = block_matrix({(0, 0): D, (0, 1): Bb, (1, 0): Bb, (1, 1): D, (1, 2): C, (2, 1): C, (2, 2): D}, 3, 2)
    rowptr, col = st.strength_graph(A, 0.5)
    assert rowptr.tolist() == [0, 1, 2, 2] and col.tolist() == [1, 0]
    rowptr, col = st.strength_graph(A, 0.1)   # rhs = 1e-4 * 64 = 0.0064 > 0.0004: C still weak
    assert col.tolist() == [1, 0]
    rowptr, col = st.strength_graph(A, 0.0)   # every nonzero off-diagonal block
    assert col.tolist() == [1, 0, 2, 1]


def test_scalar_blocks_reduce_to_the_papers_formula():
    """With 1 x 1 blocks the test is |a_ij| >= eps sqrt(a_ii a_jj) (Sec. 2.2)."""
    rng = np.random.default_rng(4)
    n = 40
    M = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.2)
    M = M + M.T + n * np.eye(n)
    blocks = {(i, j): [[M[i, j]]] for i in range(n) for j in range(n) if M[i, j] != 0}
    A = block_matrix(blocks, n, 1)
    for eps in (0.02, 0.08, 0.25):
        rowptr, col = st.strength_graph(A, eps)
        want = {(i, j) for i in range(n) for j in range(n)
                if i != j and M[i, j] != 0 and abs(M[i, j]) >= eps * np.sqrt(M[i, i] * M[j, j])}
        got = {(i, int(j)) for i in range(n) for j in col[rowptr[i]:rowptr[i + 1]]}
        assert got == want


def random_symmetric_graph(rng, n, p):
    adj = np.triu(rng.random((n, n)) < p, 1)
    adj = adj | adj.T
    rowptr = np.zeros(n + 1, dtype=np.int64)
    cols = []
    for i in range(n):
        js = np.flatnonzero(adj[i])
        cols += js.tolist()
        rowptr[i + 1] = rowptr[i] + js.size
    return adj, rowptr, np.asarray(cols, dtype=np.int64)


@pytest.mark.parametrize("seed", range(6))
def test_mis_is_independent_maximal_and_the_luby_fixed_point(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 60))
    adj, rowptr, col = random_symmetric_graph(rng, n, float(rng.uniform(0.02, 0.3)))
    w = st.weights(n, seed)
    mis = st.mis_greedy(rowptr, col, w)
    luby, rounds = st.mis_luby(rowptr, col, w)
    assert np.array_equal(mis, luby) and 1 <= rounds <= n
    S = np.flatnonzero(mis)
    assert not adj[np.ix_(S, S)].any()                                   # independent
    assert all(mis[i] or adj[i, S].any() for i in range(n))              # maximal
    key = lambda i: (int(w[i]), i)
    for i in range(n):   # every excluded vertex is beaten by a set neighbour: the greedy order
        if not mis[i]:
            assert any(key(j) > key(i) for j in S if adj[i, j])
    agg = st.mis_aggregates(rowptr, col, w, mis)
    assert agg.min() == 0 and agg.max() == S.size - 1
    assert np.array_equal(agg[S], np.arange(S.size))                      # roots numbered in order
    for i in np.flatnonzero(~mis):
        nb = [j for j in S if adj[i, j]]
        assert agg[i] == agg[max(nb, key=key)]


def test_mis_hand_example_on_a_path():
    # path 0-1-2-3-4 with weights favouring 1 and 3: MIS {1, 3} (0 joins 1, 2 the heavier of 1 and 3, 4 joins 3)
    rowptr = np.array([0, 1, 3, 5, 7, 8])
    col = np.array([1, 0, 2, 1, 3, 2, 4, 3])
    w = np.array([10, 50, 20, 40, 30], dtype=np.uint64)
    mis = st.mis_greedy(rowptr, col, w)
    assert np.flatnonzero(mis).tolist() == [1, 3]
    assert st.mis_aggregates(rowptr, col, w, mis).tolist() == [0, 0, 0, 1, 1]


def test_elasticity_graph_is_symmetric_and_clamped_nodes_stand_alone():
    mesh, _, A = problem(4)
    rowptr, col = st.strength_graph(A, 0.01)
    edges = {(i, int(j)) for i in range(A.nbr) for j in col[rowptr[i]:rowptr[i + 1]]}
    assert all((j, i) in edges for (i, j) in edges)
    clamped = np.flatnonzero(mesh.dirichlet())
    assert all(rowptr[i + 1] == rowptr[i] for i in clamped)   # zeroed couplings are no edges
    w = st.weights(A.nbr, 1)
    mis = st.mis_greedy(rowptr, col, w)
    assert mis[clamped].all()
    agg = st.mis_aggregates(rowptr, col, w, mis)
    assert np.bincount(agg).min() >= 1
