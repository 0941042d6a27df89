"""Pins of the point-block Jacobi / eigenvalue / Chebyshev oracle."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
from numpy.polynomial import chebyshev as npcheb

from oracle.smoother import (CHEB_LOWER, CHEB_UPPER, apply_blocks, block_diag_inverse,
                             block_jacobi_lambda, chebyshev, diagonal_blocks)
from oracle.splitmix import splitmix64, start_vector

from oracle_cases import hierarchy, problem


def test_splitmix64_published_outputs(root):
    with open(os.path.join(root, "tests", "golden", "splitmix64_seed0.json")) as f:
        g = json.load(f)
    got = splitmix64(np.arange(3, dtype=np.uint64))
    assert [int(v) for v in got] == [int(s, 16) for s in g["outputs_hex"]]
    v = start_vector(1000)
    assert v.min() >= -1.0 and v.max() < 1.0 and abs(v.mean()) < 0.1


def test_block_inverse():
    _, _, A = problem(4)
    D = diagonal_blocks(A)
    Dinv = block_diag_inverse(A)
    assert np.abs(np.einsum("nij,njk->nik", Dinv, D) - np.eye(3)).max() < 1e-13


def dense_block_diag(Db):
    return sla.block_diag(*Db)


def test_block_jacobi_lambda_bounds():
    for h in (hierarchy(8),):
        for L in h.levels[:-1]:
            D = dense_block_diag(diagonal_blocks(L.A))
            lam = sla.eigh(L.A.dense(), D, eigvals_only=True).max()
            assert 0.9 * lam <= L.lam <= lam * (1 + 1e-12)
    _, _, A = problem(3)
    D = dense_block_diag(diagonal_blocks(A))
    lam = sla.eigh(A.dense(), D, eigvals_only=True).max()
    est = block_jacobi_lambda(A)
    assert 0.9 * lam <= est <= lam * (1 + 1e-12)


def cheb_error_poly(lam_hat, degree):
    a, b = CHEB_LOWER * lam_hat, CHEB_UPPER * lam_hat
    theta, delta = (a + b) / 2, (b - a) / 2
    T = npcheb.Chebyshev.basis(degree)
    return lambda t: T((theta - t) / delta) / T(theta / delta)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_chebyshev_matches_closed_form_polynomial(degree):
    _, _, A = problem(3, seed=4)
    Ad = A.dense()
    Db = diagonal_blocks(A)
    Dinv = np.linalg.inv(Db)
    D = dense_block_diag(Db)
    lam_hat = 0.97 * sla.eigh(Ad, D, eigvals_only=True).max()
    w, V = sla.eigh(Ad, D)               # D^{-1} A = V diag(w) V^T D
    p = cheb_error_poly(lam_hat, degree)(w)
    E = V @ np.diag(p) @ V.T @ D          # error propagation p(D^{-1} A)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(Ad.shape[0])
    x_star = np.linalg.solve(Ad, b)
    As = A.scalar()
    x = chebyshev(As, Dinv, b, None, lam_hat, degree)
    assert np.linalg.norm(x - (x_star - E @ x_star)) <= 1e-10 * np.linalg.norm(x_star)
    x0 = rng.standard_normal(Ad.shape[0])
    x, r = chebyshev(As, Dinv, b, x0, lam_hat, degree, want_residual=True)
    assert np.linalg.norm(x - (x_star + E @ (x0 - x_star))) <= 1e-10 * np.linalg.norm(x_star)
    assert np.linalg.norm(r - (b - Ad @ x)) <= 1e-12 * np.linalg.norm(b)


def test_apply_blocks():
    rng = np.random.default_rng(0)
    Db = rng.standard_normal((4, 6, 6))
    v = rng.standard_normal(24)
    assert np.allclose(apply_blocks(Db, v), dense_block_diag(Db) @ v, atol=1e-14)
