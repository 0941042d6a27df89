"""Pins of the oracle's blocked COO assembly (Sec. 3.4, Sec. 5)."""
import numpy as np
import pytest

from oracle.assembly import coo_assemble_blocks
from workloads.elasticity import Mesh, coo_stream, element_scale

from test_pins_workload import rigid_modes


def test_coo_brute_force_rectangular_blocks():
    rng = np.random.default_rng(3)
    nbr, nbc, br, bc, n = 5, 4, 2, 3, 60
    bi = rng.integers(-1, nbr, n)
    bj = rng.integers(-1, nbc, n)
    bi[0], bj[0] = -1, 2          # ignored entries
    bi[1], bj[1] = 3, -5
    vals = rng.standard_normal((n, br, bc))
    vals[5] = 0.0                  # an all-zero block stays structural
    dense = np.zeros((nbr * br, nbc * bc))
    present = set()
    for k in range(n):
        if bi[k] < 0 or bj[k] < 0:
            continue
        present.add((bi[k], bj[k]))
        for r in range(br):
            for c in range(bc):
                dense[bi[k] * br + r, bj[k] * bc + c] += vals[k, r, c]
    A = coo_assemble_blocks(nbr, nbc, br, bc, bi, bj, vals)
    assert np.allclose(A.dense(), dense, rtol=0, atol=1e-14)
    got = {(I, int(J)) for I in range(nbr) for J in A.colidx[A.rowptr[I]:A.rowptr[I + 1]]}
    assert got == present
    for I in range(nbr):
        row = A.colidx[A.rowptr[I]:A.rowptr[I + 1]]
        assert np.all(np.diff(row) > 0)


def assemble(ne, nu=0.3, delta=None):
    mesh = Mesh(ne)
    s = coo_stream(mesh, nu, element_scale(mesh, delta=delta))
    return mesh, coo_assemble_blocks(mesh.n_nodes, mesh.n_nodes, 3, 3,
                                     s.bi.numpy(), s.bj.numpy(), s.vals.numpy())


@pytest.mark.parametrize("ne", [2, 5, 8])
def test_pattern_is_full_node_adjacency(ne):
    mesh, A = assemble(ne)
    m = mesh.m
    assert A.nnzb == (3 * m - 2) ** 3
    ijk = mesh.node_ijk()
    rows = A.block_rows()
    d = np.abs(ijk[rows] - ijk[A.colidx])
    assert d.max() <= 1


def interior_rows(mesh, margin_x=2):
    ijk = mesh.node_ijk()
    m = mesh.m
    ok = (ijk[:, 0] >= margin_x) & (ijk[:, 0] <= m - 2)
    ok &= (ijk[:, 1] >= 1) & (ijk[:, 1] <= m - 2) & (ijk[:, 2] >= 1) & (ijk[:, 2] <= m - 2)
    return np.nonzero(ok)[0]


def test_symmetric_clamped_identity_and_rigid_modes():
    delta = np.random.default_rng(1).uniform(-0.01, 0.01, Mesh(6).n_el)
    mesh, A = assemble(6, delta=delta)
    D = A.dense()
    assert np.abs(D - D.T).max() <= 1e-15 * np.abs(D).max()
    dn = np.nonzero(mesh.dirichlet())[0]
    dofs = (3 * dn[:, None] + np.arange(3)).reshape(-1)
    sub = D[dofs]
    assert np.array_equal(sub[:, dofs], np.eye(dofs.size))
    mask = np.ones(D.shape[1], bool)
    mask[dofs] = False
    assert np.all(sub[:, mask] == 0.0) and np.all(D[mask][:, dofs] == 0.0)
    U = rigid_modes(mesh.coords())
    rows = (3 * interior_rows(mesh)[:, None] + np.arange(3)).reshape(-1)
    assert np.abs((D @ U)[rows]).max() < 1e-13 * np.abs(D).max()


def test_patch_test_linear_fields():
    mesh, A = assemble(5, nu=0.35)
    D = A.dense()
    x = mesh.coords()
    rows = (3 * interior_rows(mesh)[:, None] + np.arange(3)).reshape(-1)
    for comp in range(3):
        for dirn in range(3):
            u = np.zeros_like(x)
            u[:, comp] = x[:, dirn]
            assert np.abs((D @ u.reshape(-1))[rows]).max() < 1e-13 * np.abs(D).max()
        u = np.zeros_like(x)
        u[:, comp] = 1.0
        assert np.abs((D @ u.reshape(-1))[rows]).max() < 1e-13 * np.abs(D).max()
