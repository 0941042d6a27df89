"""Pins of the V-cycle and CG oracle (Sec. 2.1, Sec. 4.1)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import krylov
from oracle import multigrid as omg
from oracle.aggregation import aggregate_1d
from oracle.smoother import diagonal_blocks

from oracle_cases import hierarchy, problem
from test_pins_smoother import cheb_error_poly


def smoother_error(L, degree):
    Ad = L.A.dense()
    D = sla.block_diag(*diagonal_blocks(L.A))
    w, V = sla.eigh(Ad, D)
    return V @ np.diag(cheb_error_poly(L.lam, degree)(w)) @ V.T @ D


def test_two_level_vcycle_equals_dense_error_operator():
    h = hierarchy(8)
    L0, L1 = h.levels
    Ad, Pd = L0.A.dense(), L0.P.dense()
    S = smoother_error(L0, h.degree)
    Ac = L1.A.dense()
    CGC = np.eye(Ad.shape[0]) - Pd @ np.linalg.solve(Ac, Pd.T @ Ad)
    E = S @ CGC @ S
    rng = np.random.default_rng(7)
    b = rng.standard_normal(Ad.shape[0])
    ref = (np.eye(Ad.shape[0]) - E) @ np.linalg.solve(Ad, b)
    got = omg.vcycle(h, b)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_three_level_vcycle_is_symmetric():
    h = hierarchy(8, max_coarse_dofs=100)
    assert h.n_levels == 3 and h.levels[-1].A.nbr == 1
    rng = np.random.default_rng(8)
    x, y = rng.standard_normal((2, h.levels[0].A.nbr * 3))
    a = omg.vcycle(h, x) @ y
    b = x @ omg.vcycle(h, y)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_single_level_is_exact_solve():
    mesh, _, A = problem(3)
    h = omg.setup(A, mesh.coords(), mesh.dirichlet(), mesh.grid, max_coarse_dofs=10 ** 6)
    assert h.n_levels == 1
    b = np.random.default_rng(0).standard_normal(A.nbr * 3)
    assert np.allclose(A.dense() @ omg.vcycle(h, b), b, atol=1e-11)


@pytest.mark.parametrize("m,levels", [(9, 2), (65, 3), (128, 4), (49, 3), (17, 2), (41, 3)])
def test_level_count_rule(m, levels):
    dofs, bs, n = [], 3, m
    count = 1
    while n ** 3 * bs > omg.MAX_COARSE_DOFS:
        n = aggregate_1d(n)[1]
        bs = 6
        count += 1
    assert count == levels


def test_cg_distinct_eigenvalues():
    ev = np.repeat([1.0, 2.0, 5.0, 11.0, 40.0], 20)
    A = sp.diags(ev).tocsr()
    b = np.random.default_rng(1).standard_normal(ev.size)
    x, its, info = krylov.pcg(A, b, lambda r: r.copy(), rtol=1e-12, maxit=50)
    assert its == 5 and info["converged"]
    assert np.allclose(x, b / ev, rtol=1e-10)


def test_cg_exact_preconditioner_one_iteration():
    _, _, A = problem(3)
    Ad = A.dense()
    b = np.random.default_rng(2).standard_normal(Ad.shape[0])
    x, its, info = krylov.pcg(A.scalar(), b, lambda r: np.linalg.solve(Ad, r), 1e-8, 10)
    assert its == 1


def test_cg_with_vcycle_reaches_tolerance():
    h = hierarchy(8)
    As = h.levels[0].A.scalar()
    b = np.random.default_rng(3).standard_normal(As.shape[0])
    x, its, info = krylov.pcg(As, b, lambda r: omg.vcycle(h, r), 1e-8, 100)
    assert info["converged"] and info["true_residual"] <= 1.01e-8 * np.linalg.norm(b)
    x_star = np.linalg.solve(As.toarray(), b)
    assert np.linalg.norm(x - x_star) <= 1e-5 * np.linalg.norm(x_star)
    assert its < 30
