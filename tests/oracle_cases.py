"""Small cached oracle problems shared by the pin and parity tests."""
import functools

import numpy as np

from oracle import multigrid as omg
from oracle.assembly import coo_assemble_blocks
from workloads.elasticity import Mesh, coo_stream, element_scale


@functools.lru_cache(maxsize=None)
def problem(ne: int, nu: float = 0.3, seed: int | None = None, order: int = 1):
    mesh = Mesh(ne, order)
    delta = None
    if seed is not None:
        from workloads.elasticity import perturbation
        delta = perturbation(mesh.n_el, seed)
    s = coo_stream(mesh, nu, element_scale(mesh, delta=delta))
    A = coo_assemble_blocks(mesh.n_nodes, mesh.n_nodes, 3, 3,
                            s.bi.numpy(), s.bj.numpy(), s.vals.numpy())
    return mesh, s, A


@functools.lru_cache(maxsize=None)
def hierarchy(ne: int, nu: float = 0.3, max_coarse_dofs: int = omg.MAX_COARSE_DOFS, order: int = 1,
              aggregation: str = "geometric", eps: float = 0.02, seed: int = 1):
    mesh, _, A = problem(ne, nu, order=order)
    return omg.setup(A, mesh.coords(), mesh.dirichlet(), mesh.grid, max_coarse_dofs,
                     aggregation=aggregation, eps=eps, seed=seed)


def rigid_modes_global(x: np.ndarray) -> np.ndarray:
    n = x.shape[0]
    U = np.zeros((n, 3, 6))
    U[:, :, :3] = np.eye(3)
    for col, w in ((3, [0, 0, 1]), (4, [1, 0, 0]), (5, [0, 1, 0])):
        U[:, :, col] = np.cross(np.array(w, dtype=float), x)
    return U
