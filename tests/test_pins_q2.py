"""Pins of the Q2 (27-node hexahedron) workload: the element stiffness and
load against closed forms and an independent quadrature, and the mesh."""
import numpy as np
import pytest

from workloads.elasticity import Mesh, body_force, coo_stream, element_scale, element_stiffness_q, lame

from test_pins_workload import rigid_modes


def q2_nodes():
    a = np.arange(27)
    return np.stack([a % 3, (a // 3) % 3, a // 9], axis=1) * 0.5


def voigt_D(nu):
    lam, mu = lame(1.0, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[[0, 1, 2], [0, 1, 2]] += 2.0 * mu
    D[[3, 4, 5], [3, 4, 5]] = mu
    return D


@pytest.mark.parametrize("nu", [0.25, 0.3, 0.45])
def test_q2_stiffness_is_symmetric_psd_with_the_rigid_modes_as_kernel(nu):
    K = element_stiffness_q(1.0, nu, 1.0, 2, 3)
    assert K.shape == (81, 81) and np.allclose(K, K.T, atol=1e-14)
    ev = np.linalg.eigvalsh(K)
    assert ev[:6].max() < 1e-12 * ev[-1] and ev[6] > 1e-6 * ev[-1]
    U = rigid_modes(q2_nodes())
    assert np.abs(K @ U).max() < 1e-12 * np.abs(K).max()


def strain_energy(grad_u, nu, n=6):
    """sum over an n^3 Gauss rule of eps_v^T D eps_v for the displacement gradient grad_u(x) (3x3)."""
    t, w = np.polynomial.legendre.leggauss(n)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    D = voigt_D(nu)
    e = 0.0
    for i in range(n):
        for j in range(n):
            for k in range(n):
                G = grad_u(np.array([t[i], t[j], t[k]]))
                ev = np.array([G[0, 0], G[1, 1], G[2, 2], G[0, 1] + G[1, 0], G[1, 2] + G[2, 1], G[0, 2] + G[2, 0]])
                e += w[i] * w[j] * w[k] * ev @ D @ ev
    return e


def test_q2_reproduces_the_energy_of_quadratic_fields():
    """A Q2 element represents every quadratic displacement exactly, so
    u^T K u equals the continuum energy (an independent 6-point rule)."""
    nu = 0.3
    K = element_stiffness_q(1.0, nu, 1.0, 2, 3)
    X = q2_nodes()
    rng = np.random.default_rng(2)
    for _ in range(3):
        C1 = rng.standard_normal((3, 3))
        C2 = rng.standard_normal((3, 3, 3))   # u_c = sum C1[c,d] x_d + C2[c,d,e] x_d x_e
        u = np.array([[C1[c] @ x + x @ C2[c] @ x for c in range(3)] for x in X]).reshape(-1)
        grad = lambda x: C1 + np.einsum("cde,e->cd", C2, x) + np.einsum("cde,d->ce", C2, x)
        assert u @ K @ u == pytest.approx(strain_energy(grad, nu), rel=1e-12)


def test_q2_mesh_and_load():
    mesh = Mesh(3, order=2)
    assert mesh.m == 7 and mesh.n_nodes == 343 and mesh.nodes_per_element == 27
    conn = mesh.connectivity()
    assert conn.shape == (27, 27) and np.unique(conn).size == mesh.n_nodes
    xc = mesh.coords()[conn].mean(axis=1)
    assert np.allclose(xc, mesh.element_centroids())
    b = body_force(mesh).reshape(-1, 3)
    # x = 0 nodes are clamped: they carry 1/6 of the first element layer's load
    assert b[:, 2].sum() == pytest.approx(-(1.0 - mesh.h / 6.0), rel=1e-13)
    s = coo_stream(mesh, 0.3, element_scale(mesh))
    assert s.n == 27 * 27 * mesh.n_el + int(mesh.dirichlet().sum())
