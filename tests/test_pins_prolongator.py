"""Pins of the aggregation and prolongator oracle (Sec. 2.2)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.aggregation import aggregate_1d, aggregates
from oracle.prolongator import (rigid_body_modes, scalar_diagonal_lambda, smoothed_prolongator,
                                tentative_prolongator)

from oracle_cases import problem, rigid_modes_global


@pytest.mark.parametrize("m", list(range(1, 20)) + [65, 128, 49, 42, 21, 17, 16, 14])
def test_aggregates_1d_properties(m):
    a, n_a = aggregate_1d(m)
    assert n_a == max(1, m // 3)
    assert a[0] == 0 and np.all(np.diff(a) >= 0) and np.all(np.diff(a) <= 1)
    sizes = np.bincount(a)
    assert sizes.size == n_a
    if m >= 3:
        assert np.all(sizes[:-1] == 3) and 3 <= sizes[-1] <= 5
    else:
        assert sizes[0] == m


@pytest.mark.parametrize("m,levels", [(9, [27]), (65, [21 ** 3, 7 ** 3]),
                                      (128, [42 ** 3, 14 ** 3, 4 ** 3]), (49, [16 ** 3, 5 ** 3])])
def test_aggregate_counts_of_workloads(m, levels):
    grid = (m, m, m)
    for n in levels:
        agg, grid = aggregates(grid)
        assert int(np.prod(grid)) == n
        assert agg.max() + 1 == n


def test_aggregates_3d_are_boxes():
    agg, cgrid = aggregates((7, 5, 11))
    n = np.arange(7 * 5 * 11)
    ijk = np.stack([n % 7, (n // 7) % 5, n // 35], 1)
    for a in range(int(np.prod(cgrid))):
        box = ijk[agg == a]
        lo, hi = box.min(0), box.max(0)
        assert box.shape[0] == np.prod(hi - lo + 1)


def test_rigid_body_mode_columns():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (10, 3))
    agg = np.array([0] * 4 + [1] * 6)
    B = rigid_body_modes(x, agg, 2, np.zeros(10, np.uint8))
    cen = np.stack([x[:4].mean(0), x[4:].mean(0)])
    rel = x - cen[agg]
    assert np.allclose(B, rigid_modes_global(rel), rtol=0, atol=1e-15)
    B2 = rigid_body_modes(x, agg, 2, np.array([1] + [0] * 9, np.uint8))
    assert np.all(B2[0] == 0.0) and np.array_equal(B2[1:], B[1:])


def fine_tentative(ne=8):
    mesh, _, A = problem(ne)
    agg, cgrid = aggregates(mesh.grid)
    n_agg = int(np.prod(cgrid))
    B = rigid_body_modes(mesh.coords(), agg, n_agg, mesh.dirichlet())
    Pt, Bc = tentative_prolongator(B, agg, n_agg)
    return mesh, A, agg, n_agg, B, Pt, Bc


def test_tentative_qr_properties():
    mesh, A, agg, n_agg, B, Pt, Bc = fine_tentative()
    assert Pt.nnzb == mesh.n_nodes and np.array_equal(Pt.colidx, agg)
    for a in range(n_agg):
        nodes = np.nonzero(agg == a)[0]
        Q = Pt.vals[nodes].reshape(-1, 6)
        R = Bc[a]
        assert np.allclose(Q.T @ Q, np.eye(6), atol=1e-14)
        assert np.allclose(Q @ R, B[nodes].reshape(-1, 6), atol=1e-14)
        assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) > 0)
    dn = mesh.dirichlet().astype(bool)
    assert np.all(Pt.vals[dn] == 0.0)


def coarse_coefficients(Pt, agg, n_agg, U):
    """Per-aggregate coarse vectors c with P~ c reproducing U on the aggregate."""
    C = np.zeros((n_agg, 6, U.shape[-1]))
    for a in range(n_agg):
        nodes = np.nonzero(agg == a)[0]
        Q = Pt.vals[nodes].reshape(-1, 6)
        C[a] = Q.T @ U[nodes].reshape(-1, U.shape[-1])
    return C


def test_tentative_reproduces_global_rigid_modes():
    mesh, A, agg, n_agg, B, Pt, Bc = fine_tentative()
    U = rigid_modes_global(mesh.coords())
    U[mesh.dirichlet().astype(bool)] = 0.0
    C = coarse_coefficients(Pt, agg, n_agg, U)
    rec = np.einsum("nij,njk->nik", Pt.vals, C[agg])
    assert np.abs(rec - U).max() < 1e-13


def test_smoothed_prolongator_dense_formula_and_interior_modes():
    mesh, A, agg, n_agg, B, Pt, Bc = fine_tentative()
    P, omega = smoothed_prolongator(A, Pt)
    Ad, Ptd = A.dense(), Pt.dense()
    D = np.diag(Ad)
    ref = Ptd - omega * (Ad @ Ptd) / D[:, None]
    assert np.abs(P.dense() - ref).max() < 1e-14 * np.abs(ref).max()
    lam = sla.eigh(Ad, np.diag(D), eigvals_only=True).max()
    assert 0.9 * lam <= 4.0 / (3.0 * omega) <= lam * (1 + 1e-12)
    # interior rows: P c = u because A u = 0 there
    U = rigid_modes_global(mesh.coords())
    U[mesh.dirichlet().astype(bool)] = 0.0
    C = coarse_coefficients(Pt, agg, n_agg, U).reshape(-1, 6)
    PU = P.dense() @ C
    ijk = mesh.node_ijk()
    m = mesh.m
    inner = np.all((ijk >= 2) & (ijk <= m - 3), axis=1)
    rows = (3 * np.nonzero(inner)[0][:, None] + np.arange(3)).reshape(-1)
    assert rows.size > 0
    assert np.abs(PU[rows] - U.reshape(-1, 6)[rows]).max() < 1e-12


def count_1d(m):
    """Brute-force 1-D pattern sizes: A (|i-j|<=1), P, AP, and A_c."""
    a, n_a = aggregate_1d(m)
    nbr = [set(j for j in (i - 1, i, i + 1) if 0 <= j < m) for i in range(m)]
    P = [set(a[j] for j in nbr[i]) for i in range(m)]
    AP = [set().union(*(P[k] for k in nbr[i])) for i in range(m)]
    Ac = set()
    for i in range(m):
        for I in P[i]:
            for J in AP[i]:
                Ac.add((I, J))
    return sum(len(s) for s in nbr), sum(len(s) for s in P), sum(len(s) for s in AP), len(Ac)


@pytest.mark.parametrize("ne", [8, 10])
def test_pattern_counts_are_products_of_1d_counts(ne):
    from oracle.galerkin import ap_pattern, galerkin
    from oracle.assembly import block_pattern
    mesh, A, agg, n_agg, B, Pt, Bc = fine_tentative(ne)
    P, _ = smoothed_prolongator(A, Pt)
    nA, nP, nAP, nAc = count_1d(mesh.m)
    assert A.nnzb == nA ** 3 and P.nnzb == nP ** 3
    assert block_pattern(ap_pattern(A, P), 3, 6)[1].size == nAP ** 3
    assert galerkin(A, P).nnzb == nAc ** 3


def test_config1_pattern_counts():
    assert count_1d(9) == (25, 13, 17, 7)   # 15,625 / 2,197 / 4,913 / 343 blocks in 3-D


def test_scalar_lambda_is_lower_bound():
    mesh, _, A = problem(4)
    As = A.scalar()
    D = As.diagonal()
    lam = sla.eigh(As.toarray(), np.diag(D), eigvals_only=True).max()
    est = scalar_diagonal_lambda(As)
    assert 0.9 * lam <= est <= lam * (1 + 1e-12)
