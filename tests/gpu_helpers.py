"""Helpers for the GPU tests: build problems through the C ABI binding and read
library matrices back for comparison with the oracle."""
import numpy as np
import torch

from oracle.assembly import BlockMatrix
from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import Mesh, coo_indices, coo_values, element_scale, perturbation

# FP64 parity bar: normwise relative error ||X_gpu - X_oracle|| / ||X_oracle||.
TOL64 = 1e-12


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def read_bsr(ctx, A) -> BlockMatrix:
    info = B.bamg_bsr_info(A)
    rp = torch.empty(info["nbr"] + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(max(info["nnzb"], 1), dtype=torch.int32, device="cuda")
    B.bamg_bsr_get_pattern(ctx, A, rp, ci)
    v = torch.empty(max(info["nnzb"], 1) * info["bs_r"] * info["bs_c"], dtype=torch.float64, device="cuda")
    B.bamg_bsr_get_values(ctx, A, v)
    torch.cuda.synchronize()
    nnzb = info["nnzb"]
    return BlockMatrix(info["nbr"], info["nbc"], info["bs_r"], info["bs_c"], rp.cpu().numpy().astype(np.int64),
                       ci.cpu().numpy()[:nnzb].astype(np.int64),
                       v.cpu().numpy()[: nnzb * info["bs_r"] * info["bs_c"]].reshape(nnzb, info["bs_r"],
                                                                                      info["bs_c"]))


def same_pattern(a: BlockMatrix, b: BlockMatrix) -> bool:
    return (a.nbr == b.nbr and a.nbc == b.nbc and np.array_equal(a.rowptr, b.rowptr)
            and np.array_equal(a.colidx, b.colidx))


class GpuProblem:
    """Elasticity problem assembled on the GPU through blocked COO, with an
    optional hierarchy."""

    def __init__(self, ne, nu=0.3, seed=None, precision=B.BAMG_FP64, max_coarse_dofs=2100, setup=True,
                 E_el=None, coarse_solver=0, order=1, aggregation=B.BAMG_AGG_GEOMETRIC, mis_eps=0.02, mis_seed=1):
        self.mesh = Mesh(ne, order)
        self.nu = nu
        self.ctx = B.bamg_ctx_create(torch.cuda.current_stream())
        n = self.mesh.n_nodes
        self.bi, self.bj = coo_indices(self.mesh, "cuda")
        self.A = B.bamg_bsr_create(self.ctx, 3, 3, n, n)
        B.bamg_bsr_coo_preallocate(self.ctx, self.A, self.bi, self.bj)
        delta = None if seed is None else perturbation(self.mesh.n_el, seed)
        self.scale = element_scale(self.mesh, E_el=E_el, delta=delta)
        self.vals = coo_values(self.mesh, nu, self.scale, "cuda")
        B.bamg_bsr_coo_set_values(self.ctx, self.A, self.vals, 0)
        self.mg = None
        if setup:
            o = B.bamg_mg_opts_default()
            o.grid[0] = o.grid[1] = o.grid[2] = self.mesh.m
            o.precision = precision
            o.max_coarse_dofs = max_coarse_dofs
            o.coarse_solver = coarse_solver
            o.aggregation = aggregation
            o.mis_eps = mis_eps
            o.mis_seed = mis_seed
            self.mg = B.bamg_mg_setup(self.ctx, self.A, self.mesh.coords(), self.mesh.dirichlet(), o)

    def reassemble(self, seed):
        delta = perturbation(self.mesh.n_el, seed)
        self.scale = element_scale(self.mesh, delta=delta)
        coo_values(self.mesh, self.nu, self.scale, "cuda", out=self.vals)
        B.bamg_bsr_coo_set_values(self.ctx, self.A, self.vals, 0)

    def close(self):
        if self.mg is not None:
            B.bamg_mg_destroy(self.mg)
        B.bamg_bsr_destroy(self.A)
        B.bamg_ctx_destroy(self.ctx)
