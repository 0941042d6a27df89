"""Parity at the large benchmark size (127^3 elements, 6,291,456 dofs, 4
levels), in the configuration bench.py times (autotuned lanes and splits),
through properties that hold at any size: the rigid-body modes in the kernel
of the interior rows, the Galerkin identity x_c^T A_c y_c = (P x_c)^T A (P y_c)
and the symmetry of A_c on every level, and both CG forms reaching rtol 1e-8
with the residual recomputed by a plain product.  (The 9.6 GB COO stream of
this size is too large for the oracle to sum rows from on the host; the 64^3
module checks sampled rows.)"""
import numpy as np
import pytest
import torch

from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import body_force

from gpu_helpers import GpuProblem
from test_pins_workload import rigid_modes

pytestmark = pytest.mark.gpu
NE = 127


@pytest.fixture(scope="module")
def large():
    gp = GpuProblem(NE)
    yield gp
    gp.close()


def mv(ctx, M, v, m):
    out = torch.zeros(m, dtype=torch.float64, device="cuda")
    B.bamg_bsr_spmv(ctx, M, v, out)
    return out


def test_hierarchy_shape(large):
    nl = B.bamg_mg_num_levels(large.mg)
    assert nl == 4
    rows = [B.bamg_bsr_info(B.bamg_mg_get_level(large.mg, l)[0])["nbr"] for l in range(nl)]
    assert rows == [128 ** 3, 42 ** 3, 14 ** 3, 4 ** 3]


def test_rigid_modes_are_in_the_kernel_of_interior_rows(large):
    x = rigid_modes(large.mesh.coords())
    clamp = np.repeat(large.mesh.dirichlet().astype(bool), 3)
    ijk = large.mesh.node_ijk()
    inner = np.repeat(((ijk > 1) & (ijk < large.mesh.m - 1)).all(axis=1), 3) & ~clamp
    for k in range(6):
        y = mv(large.ctx, large.A, torch.from_numpy(np.ascontiguousarray(x[:, k])).cuda(), x.shape[0]).cpu().numpy()
        assert np.abs(y[inner]).max() <= 1e-12 * np.abs(y).max() + 1e-14, k


def test_galerkin_identity_on_every_level(large):
    rng = np.random.default_rng(127)
    nl = B.bamg_mg_num_levels(large.mg)
    for l in range(nl - 1):
        A, P = B.bamg_mg_get_level(large.mg, l)
        Ac, _ = B.bamg_mg_get_level(large.mg, l + 1)
        ic, ia = B.bamg_bsr_info(Ac), B.bamg_bsr_info(A)
        nc, nf = ic["nbr"] * ic["bs_r"], ia["nbr"] * ia["bs_r"]
        xc = torch.from_numpy(rng.standard_normal(nc)).cuda()
        yc = torch.from_numpy(rng.standard_normal(nc)).cuda()
        lhs = float(xc @ mv(large.ctx, Ac, yc, nc))
        lhs_t = float(yc @ mv(large.ctx, Ac, xc, nc))
        px, py = mv(large.ctx, P, xc, nf), mv(large.ctx, P, yc, nf)
        apy = mv(large.ctx, A, py, nf)
        rhs = float(px @ apy)
        scale = float(torch.linalg.norm(px) * torch.linalg.norm(apy))
        assert abs(lhs - rhs) <= 1e-12 * scale, l
        assert abs(lhs - lhs_t) <= 1e-12 * scale, l


@pytest.mark.parametrize("precision", [B.BAMG_FP64, B.BAMG_FP32])
def test_cg_reaches_the_tolerance_with_the_true_residual(large, precision):
    gp = large if precision == B.BAMG_FP64 else GpuProblem(NE, precision=precision)
    try:
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        x = torch.zeros_like(b)
        out = B.bamg_cg_solve(gp.ctx, gp.mg, b, x, 1e-8, 200)
        assert out["converged"] and out["iterations"] <= 50
        r = mv(gp.ctx, gp.A, x, b.numel())   # b - A x with the plain product, not CG's recurrence
        true_rel = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
        assert true_rel <= 1.05e-8
        assert out["true_rnorm"] / out["bnorm"] == pytest.approx(true_rel, rel=1e-6, abs=1e-12)
    finally:
        if gp is not large:
            gp.close()
