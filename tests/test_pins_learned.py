"""Pins of the learned-smoother oracle: bf16 rounding, MLP gradients, Adam,
features, targets and the weighted Chebyshev smoother."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import learned as OL
from oracle import multigrid as omg
from oracle.assembly import coo_assemble_blocks
from oracle.smoother import block_jacobi_lambda, chebyshev, diagonal_blocks

from oracle_cases import hierarchy, problem


def test_bf16_rounding_matches_torch_and_ties_to_even():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(10000) * 10.0 ** rng.uniform(-6, 6, 10000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(OL.bf16(x), ref)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8)], dtype=np.float32)
    assert np.array_equal(OL.bf16(ties), np.array([1.0, 1 + 2 ** -6, -1.0], dtype=np.float32))


def random_theta(seed, scale=0.3):
    return np.random.default_rng(seed).standard_normal(OL.N_PARAMS) * scale


def test_fp64_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((40, OL.N_FEATURES))
    t = rng.uniform(0.5, 2.0, 40)
    theta = random_theta(2)
    _, g = OL.loss_and_grad(theta, X, t, emulate_bf16=False)
    idx = rng.choice(OL.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [OL.N_PARAMS - 1, 0, 520]])
    h = 1e-6
    for k in idx:
        e = np.zeros(OL.N_PARAMS)
        e[k] = h
        fd = (OL.loss_and_grad(theta + e, X, t, False)[0] - OL.loss_and_grad(theta - e, X, t, False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g).max()), k


def test_bf16_forward_close_to_fp64():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((500, OL.N_FEATURES))
    theta = random_theta(4)
    w16, _ = OL.forward(theta, X, True)
    w64, _ = OL.forward(theta, X, False)
    assert np.all((w16 > 0.5) & (w16 < 2.0))
    assert np.linalg.norm(w16 - w64) / np.linalg.norm(w64) < 2e-2


def test_adam_matches_torch():
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(5)]
    opt = OL.Adam(50, lr=1e-2)
    p = torch.nn.Parameter(torch.from_numpy(theta.copy()))
    topt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    th = theta.copy()
    for g in grads:
        th = opt.step(th, g)
        p.grad = torch.from_numpy(g.copy())
        topt.step()
    assert np.allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_features_on_a_hand_built_matrix():
    # block row 0: diag 2 I (norm 2 sqrt 3), one off-diagonal block of ones (norm 3)
    bi = np.array([0, 0, 1])
    bj = np.array([0, 1, 1])
    vals = np.stack([2 * np.eye(3), np.ones((3, 3)), np.eye(3)])
    A = coo_assemble_blocks(2, 2, 3, 3, bi, bj, vals)
    F = OL.block_features(A, level=1)
    d = 2 * np.sqrt(3)
    assert F[0, 0] == pytest.approx(np.log(d), rel=1e-6)
    assert F[0, 1] == pytest.approx(3 / d, rel=1e-6)
    assert F[0, 2] == pytest.approx(np.log(d / 3), rel=1e-6)    # max / min block norm
    assert F[0, 3] == pytest.approx(2 / 27, rel=1e-6) and F[0, 4] == 0.0
    assert F[0, 5] == pytest.approx(np.log(np.sqrt(3) + 1.5), rel=1e-6)   # ||I||=sqrt3, ||ones/2||=1.5
    assert F[1, 4] == 1.0 and F[1, 2] == 0.0 and F[1, 6] == 1.0 and F[1, 7] == 1.0


@pytest.mark.parametrize("c,expect", [(1.0, 1.0), (1.5, 1 / 1.5), (0.25, 2.0), (4.0, 0.5)])
def test_local_damping_of_a_scaled_diagonal(c, expect):
    rng = np.random.default_rng(6)
    D = rng.standard_normal((5, 3, 3))
    D = np.einsum("nij,nkj->nik", D, D) + 3 * np.eye(3)
    A = sp.block_diag([sp.csr_matrix(c * d) for d in D]).tocsr()
    R = [rng.standard_normal(15) for _ in range(3)]
    w = OL.local_damping(A, np.linalg.inv(D), R)
    assert np.allclose(w, expect, rtol=1e-6)


def test_uniform_weight_equals_rescaled_plain_smoother():
    _, _, A = problem(3, seed=4)
    As = A.scalar()
    Dinv = np.linalg.inv(diagonal_blocks(A))
    lam = block_jacobi_lambda(A, As, Dinv)
    wgt = 1.3
    lam_w = block_jacobi_lambda(A, As, Dinv, np.full(A.nbr, wgt))
    assert lam_w == pytest.approx(wgt * lam, rel=1e-12)
    b = np.random.default_rng(7).standard_normal(As.shape[0])
    x1 = chebyshev(As, Dinv, b, None, lam, 2)
    x2 = chebyshev(As, Dinv, b, None, lam_w, 2, weights=np.full(A.nbr, wgt))
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)


def test_weighted_vcycle_symmetric_and_targets_in_range():
    import copy
    h = copy.deepcopy(hierarchy(8))
    rng = np.random.default_rng(9)
    w0 = rng.uniform(0.6, 1.6, h.levels[0].A.nbr)
    omg.set_weights(h, [w0])
    x, y = rng.standard_normal((2, h.levels[0].A.nbr * 3))
    a = omg.vcycle(h, x) @ y
    b = x @ omg.vcycle(h, y)
    assert abs(a - b) <= 1e-12 * abs(a)
    T = OL.smoother_targets(h, rng.standard_normal((2, h.levels[0].A.nbr * 3)))
    assert len(T) == h.n_levels - 1
    assert np.all((T[0] >= 0.5) & (T[0] <= 2.0))


def dense_presmoothing_residual(L, degree, rhs, weights=None):
    """Residual after degree-m Chebyshev pre-smoothing from x = 0, from the
    generalised eigenpairs A V = M V Lam (V^T M V = I, M = D W^{-1}): the
    residual operator is M V p(Lam) V^T, p the Chebyshev error polynomial."""
    import scipy.linalg as sla
    from test_pins_smoother import cheb_error_poly
    Db = diagonal_blocks(L.A)
    if weights is not None:
        Db = Db / np.asarray(weights, dtype=np.float64)[:, None, None]
    M = sla.block_diag(*Db)
    lam, V = sla.eigh(L.A.dense(), M)
    return M @ (V @ (cheb_error_poly(L.lam, degree)(lam) * (V.T @ rhs)))


def expected_targets(h, B, restrict_residual=True):
    res = [[] for _ in range(h.n_levels - 1)]
    for b in B:
        rhs = b
        for l in range(h.n_levels - 1):
            L = h.levels[l]
            r = dense_presmoothing_residual(L, h.degree, rhs, L.weights)
            res[l].append(r)
            rhs = L.P.dense().T @ (r if restrict_residual else rhs)
    return [OL.local_damping(h.levels[l].As, h.levels[l].Dinv, res[l]) for l in range(h.n_levels - 1)]


def test_smoother_targets_follow_the_level_composition():
    """Level l's targets come from the residual after its pre-smoothing, with
    the restricted pre-smoothed residual of level l-1 as right-hand side; on
    a three-level hierarchy both levels are checked against the dense
    spectral form of the pre-smoothing residual."""
    h = hierarchy(8, max_coarse_dofs=100)
    assert h.n_levels == 3
    B = np.random.default_rng(21).standard_normal((3, h.levels[0].A.nbr * 3))
    got = OL.smoother_targets(h, B)
    ref = expected_targets(h, B)
    assert len(got) == 2
    for g, r in zip(got, ref):
        assert np.allclose(g, r, rtol=1e-5, atol=1e-6)
        assert np.ptp(r) > 0.05            # the targets are not all the same value
    # planted mistake: restricting the level's input instead of its residual
    wrong = expected_targets(h, B, restrict_residual=False)
    assert not np.allclose(wrong[1], got[1], rtol=1e-3, atol=1e-3)


def test_smoother_targets_with_weights_use_the_weighted_smoother():
    import copy
    h = copy.deepcopy(hierarchy(8, max_coarse_dofs=100))
    rng = np.random.default_rng(22)
    omg.set_weights(h, [rng.uniform(0.6, 1.6, h.levels[0].A.nbr), None])
    B = rng.standard_normal((2, h.levels[0].A.nbr * 3))
    got = OL.smoother_targets(h, B)
    ref = expected_targets(h, B)
    for g, r in zip(got, ref):
        assert np.allclose(g, r, rtol=1e-5, atol=1e-6)
