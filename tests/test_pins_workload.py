"""Pins of the seeded elasticity generator against closed forms and invariants."""
import numpy as np
import pytest

from workloads.elasticity import (Mesh, body_force, coo_indices, coo_values, element_scale,
                                  element_stiffness, gauss_rule, lame, reference_blocks)


def unit_cube_nodes():
    return np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.float64)


def rigid_modes(x):
    """Global rigid-body modes at points x (n, 3): translations and omega x r."""
    n = x.shape[0]
    U = np.zeros((n, 3, 6))
    U[:, :, :3] = np.eye(3)
    for col, w in ((3, [0, 0, 1]), (4, [1, 0, 0]), (5, [0, 1, 0])):
        U[:, :, col] = np.cross(np.array(w, dtype=float), x)
    return U.reshape(3 * n, 6)


@pytest.mark.parametrize("nu", [0.2, 0.3, 0.45])
def test_element_stiffness_closed_form_entries(nu):
    # For the unit cube: int (dN0/dx)^2 = 1/9 and int dN0/dx dN0/dy = 1/12 (exact
    # under 2-point Gauss), so K[0,0] = (lam + 4 mu)/9 and K[0,1] = (lam + mu)/12.
    lam, mu = lame(1.0, nu)
    K = element_stiffness(1.0, nu)
    assert K[0, 0] == pytest.approx((lam + 4.0 * mu) / 9.0, rel=1e-14)
    assert K[0, 1] == pytest.approx((lam + mu) / 12.0, rel=1e-14)


@pytest.mark.parametrize("nu", [0.2, 0.3, 0.45])
def test_element_stiffness_rigid_modes_and_rank(nu):
    K = element_stiffness(1.0, nu)
    assert np.allclose(K, K.T, rtol=0, atol=1e-15 * np.abs(K).max())
    U = rigid_modes(unit_cube_nodes() + np.array([0.3, -1.2, 2.0]))
    assert np.abs(K @ U).max() < 1e-13 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev < 1e-12 * ev.max()) == 6
    assert np.all(ev > -1e-13 * ev.max())


def test_gauss_rules_integrate_exactly():
    for order, deg in ((2, 3), (3, 5)):
        p, w = gauss_rule(order)
        for k in range(deg + 1):
            assert np.dot(w, p ** k) == pytest.approx(1.0 / (k + 1), rel=1e-14)


def test_three_point_gauss_gives_same_stiffness():
    K2 = element_stiffness(1.0, 0.3, 1.0, 2)
    K3 = element_stiffness(1.0, 0.3, 1.0, 3)
    assert np.abs(K2 - K3).max() < 1e-14 * np.abs(K2).max()


def test_stiffness_scales_with_E_and_h():
    K = element_stiffness(2.5, 0.3, 0.125)
    ref = 2.5 * 0.125 * element_stiffness(1.0, 0.3)
    assert np.abs(K - ref).max() < 1e-14 * np.abs(ref).max()


def test_reference_blocks_layout():
    K = element_stiffness(1.0, 0.3)
    kb = reference_blocks(0.3)
    for a in range(8):
        for b in range(8):
            assert np.array_equal(kb[8 * a + b], K[3 * a:3 * a + 3, 3 * b:3 * b + 3])


def test_body_force_total():
    mesh = Mesh(6)
    b = body_force(mesh).reshape(-1, 3)
    assert np.all(b[:, :2] == 0.0)
    # unit volume, unit force; clamped nodes (ix = 0) would receive h/2 of it
    assert b[:, 2].sum() == pytest.approx(-(1.0 - mesh.h / 2.0), rel=1e-13)
    assert np.all(b[mesh.dirichlet().astype(bool)] == 0.0)


def test_coo_stream_layout():
    mesh = Mesh(3)
    bi, bj = coo_indices(mesh)
    scale = element_scale(mesh, delta=np.linspace(-0.01, 0.01, mesh.n_el))
    v = coo_values(mesh, 0.3, scale).numpy()
    n_dir = int(mesh.dirichlet().sum())
    assert bi.shape[0] == 64 * mesh.n_el + n_dir == v.shape[0]
    conn = mesh.connectivity()
    kb = reference_blocks(0.3)
    dn = mesh.dirichlet().astype(bool)
    for e in (0, 7, mesh.n_el - 1):
        for a in range(8):
            for b in range(8):
                k = 64 * e + 8 * a + b
                assert bi[k] == conn[e, a] and bj[k] == conn[e, b]
                if dn[conn[e, a]] or dn[conn[e, b]]:
                    assert np.all(v[k] == 0.0)
                else:
                    assert np.array_equal(v[k], scale[e] * kb[8 * a + b])
    tail = v[64 * mesh.n_el:]
    assert np.array_equal(tail, np.broadcast_to(np.eye(3), tail.shape))
    assert np.array_equal(bi.numpy()[64 * mesh.n_el:], np.nonzero(dn)[0])
