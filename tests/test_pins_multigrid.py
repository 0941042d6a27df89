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


def dense_two_level_error(h):
    """E = S (I - P A_c^{-1} P^T A) S of a two-level hierarchy, from dense
    matrices and the Chebyshev error polynomial (no call into the V-cycle)."""
    L0, L1 = h.levels
    Ad, Pd = L0.A.dense(), L0.P.dense()
    S = smoother_error(L0, h.degree)
    CGC = np.eye(Ad.shape[0]) - Pd @ np.linalg.solve(L1.A.dense(), Pd.T @ Ad)
    return Ad, S @ CGC @ S


def stationary_reference(Ad, E, b, its):
    """||r_k|| of x_{k+1} = x_k + M r_k with M = (I - E) A^{-1}: the residual
    obeys r_{k+1} = (I - A M) r_k = A E A^{-1} r_k."""
    T = Ad @ E @ np.linalg.inv(Ad)
    r = b.copy()
    out = [float(np.linalg.norm(r))]
    for _ in range(its):
        r = T @ r
        out.append(float(np.linalg.norm(r)))
    return np.array(out)


def test_stationary_iteration_equals_dense_error_operator_powers():
    h = hierarchy(8)
    Ad, E = dense_two_level_error(h)
    b = np.random.default_rng(11).standard_normal(Ad.shape[0])
    its = 6
    ref = stationary_reference(Ad, E, b, its)
    got = np.array(omg.stationary(h, b, its))
    assert got.shape == ref.shape
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-12 * ref[0])
    # the factor that rates the learned smoother follows from the same powers
    assert (got[-1] / got[0]) ** (1 / its) < 1.0


def test_stationary_pin_rejects_a_planted_mistake():
    """A stationary loop that applies the cycle to b instead of the current
    residual differs from the error-operator powers (the pin can tell)."""
    h = hierarchy(8)
    Ad, E = dense_two_level_error(h)
    b = np.random.default_rng(12).standard_normal(Ad.shape[0])
    As = h.levels[0].As
    x = np.zeros_like(b)
    wrong = [float(np.linalg.norm(b))]
    for _ in range(4):
        x = x + omg.vcycle(h, b)           # planted: b in place of r
        wrong.append(float(np.linalg.norm(b - As @ x)))
    ref = stationary_reference(Ad, E, b, 4)
    assert not np.allclose(wrong, ref, rtol=1e-3)
