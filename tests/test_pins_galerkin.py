"""Pins of the Galerkin product oracle A_c = P^T A P (Sec. 2.2, Sec. 3.1)."""
import numpy as np

from oracle import multigrid as omg
from oracle.galerkin import galerkin

from oracle_cases import hierarchy, problem


def test_dense_brute_force_config1():
    h = hierarchy(8)
    L0, L1 = h.levels
    Ad, Pd = L0.A.dense(), L0.P.dense()
    ref = Pd.T @ Ad @ Pd
    got = L1.A.dense()
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)
    # the pattern is the tile set of the dense boolean product of the structures
    Sa = L0.A.structure().toarray() != 0
    Sp = L0.P.structure().toarray() != 0
    Sc = (Sp.T.astype(int) @ Sa.astype(int) @ Sp.astype(int)) != 0
    tiles = Sc.reshape(L1.A.nbr, 6, L1.A.nbc, 6).any(axis=(1, 3))
    I, J = np.nonzero(tiles)
    assert np.array_equal(np.bincount(I, minlength=L1.A.nbr), np.diff(L1.A.rowptr))
    assert np.array_equal(J, L1.A.colidx)


def test_galerkin_identity_symmetry_spd():
    h = hierarchy(8)
    L0, L1 = h.levels
    rng = np.random.default_rng(5)
    xc, yc = rng.standard_normal((2, L1.A.nbr * 6))
    Ps, As = L0.P.scalar(), L0.A.scalar()
    lhs = xc @ (L1.A.scalar() @ yc)
    rhs = (Ps @ xc) @ (As @ (Ps @ yc))
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs)
    Ac = L1.A.dense()
    assert np.linalg.norm(Ac - Ac.T) <= 1e-15 * np.linalg.norm(Ac)
    np.linalg.cholesky(Ac)


def test_hot_update_matches_dense_product_and_is_reproducible():
    mesh, _, A2 = problem(8, seed=3)
    h = hierarchy(8)
    h2 = omg.update(h, A2)
    Pd = h.levels[0].P.dense()
    ref = Pd.T @ A2.dense() @ Pd
    got = h2.levels[1].A.dense()
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)
    h1 = omg.update(h, h.levels[0].A)
    assert np.array_equal(h1.levels[1].A.vals, h.levels[1].A.vals)


def test_rectangular_general_galerkin():
    # a non-symmetric A and an arbitrary block P: the product is still P^T A P
    from oracle.assembly import coo_assemble_blocks
    rng = np.random.default_rng(2)
    n, nc = 7, 3
    bi, bj = rng.integers(0, n, 40), rng.integers(0, n, 40)
    A = coo_assemble_blocks(n, n, 3, 3, bi, bj, rng.standard_normal((40, 3, 3)))
    pi, pj = rng.integers(0, n, 12), rng.integers(0, nc, 12)
    P = coo_assemble_blocks(n, nc, 3, 6, pi, pj, rng.standard_normal((12, 3, 6)))
    Ac = galerkin(A, P)
    ref = P.dense().T @ A.dense() @ P.dense()
    assert np.linalg.norm(Ac.dense() - ref) <= 1e-14 * np.linalg.norm(ref)
