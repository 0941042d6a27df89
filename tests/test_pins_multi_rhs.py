"""Pins of the many-right-hand-side oracle: the cycle is one linear operator
applied column by column, and the CG recurrences are independent and
homogeneous (scaling a right-hand side by a power of two scales its iterates
exactly)."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import multi_rhs as OM
from workloads.elasticity import Mesh, gaussian_rhs

from oracle_cases import hierarchy


def test_cycle_commutes_with_column_mixing():
    h = hierarchy(6)
    m = h.levels[0].A.nbr * 3
    rng = np.random.default_rng(1)
    B = rng.standard_normal((m, 3))
    C = rng.standard_normal((3, 4))
    lhs = OM.vcycle_columns(h, B @ C)
    rhs = OM.vcycle_columns(h, B) @ C
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)
    # symmetric operator: B^T M B is a symmetric matrix
    G = B.T @ OM.vcycle_columns(h, B)
    assert np.allclose(G, G.T, rtol=1e-12, atol=1e-12 * np.abs(G).max())


def test_cg_columns_are_independent_and_homogeneous():
    ne = 6
    h = hierarchy(ne)
    b = gaussian_rhs(Mesh(ne), 0)
    B = np.stack([b, 2.0 * b, -0.5 * b, np.zeros_like(b)], axis=1)
    X, its, infos = OM.pcg_columns(h, B, 1e-8, 100)
    assert np.array_equal(X[:, 1], 2.0 * X[:, 0])
    assert np.array_equal(X[:, 2], -0.5 * X[:, 0])
    assert its[0] == its[1] == its[2] > 0 and its[3] == 0 and not X[:, 3].any()
    assert all(i["converged"] for i in infos)


def test_cg_columns_solve_the_system():
    ne = 6
    h = hierarchy(ne)
    As = h.levels[0].As.tocsc()
    B = np.stack([gaussian_rhs(Mesh(ne), s) for s in range(3)], axis=1)
    X, its, infos = OM.pcg_columns(h, B, 1e-10, 200)
    for j in range(3):
        xd = spla.spsolve(As, B[:, j])
        assert np.linalg.norm(X[:, j] - xd) <= 1e-7 * np.linalg.norm(xd)
        assert np.linalg.norm(B[:, j] - As @ X[:, j]) <= 1e-10 * np.linalg.norm(B[:, j])
