"""GPU parity of the many-right-hand-side cycle and CG (blocked SpMM form)
against the oracle, the single-vector path, and exact invariants."""
import numpy as np
import pytest
import torch

from oracle import multi_rhs as OM
from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import gaussian_rhs

from gpu_helpers import TOL64, GpuProblem, rel
from oracle_cases import hierarchy

pytestmark = pytest.mark.gpu


def rhs(mesh, k, first_seed=0):
    return np.stack([gaussian_rhs(mesh, first_seed + s) for s in range(k)], axis=1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("k", [1, 5, 16])
def test_multi_vcycle_matches_oracle(k):
    ne = 13
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        Bh = rhs(gp.mesh, k)
        X = torch.zeros_like(dev(Bh))
        B.bamg_mg_vcycle_multi(gp.ctx, gp.mg, dev(Bh), X, k)
        ref = OM.vcycle_columns(h, Bh)
        got = X.cpu().numpy()
        for j in range(k):
            assert rel(got[:, j], ref[:, j]) <= TOL64, j
    finally:
        gp.close()


def test_multi_vcycle_equals_single_vector_cycles_bitwise():
    ne = 13
    gp = GpuProblem(ne)
    try:
        B.bamg_mg_set_lanes(gp.ctx, gp.mg, 1)
        k = 7
        Bh = rhs(gp.mesh, k, 3)
        X = torch.zeros_like(dev(Bh))
        B.bamg_mg_vcycle_multi(gp.ctx, gp.mg, dev(Bh), X, k)
        for j in range(k):
            x = torch.zeros(Bh.shape[0], dtype=torch.float64, device="cuda")
            B.bamg_vcycle(gp.ctx, gp.mg, dev(Bh[:, j]), x)
            assert torch.equal(X[:, j], x), j
    finally:
        gp.close()


def test_multi_cg_matches_oracle_per_column():
    ne = 13
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        k = 16
        Bh = rhs(gp.mesh, k)
        X = torch.zeros_like(dev(Bh))
        infos = B.bamg_cg_solve_multi(gp.ctx, gp.mg, dev(Bh), X, k, 1e-8, 200)
        Xr, its, _ = OM.pcg_columns(h, Bh, 1e-8, 200)
        got = X.cpu().numpy()
        for j in range(k):
            assert infos[j]["converged"]
            assert abs(infos[j]["iterations"] - its[j]) <= 1, j
            bn = np.linalg.norm(Bh[:, j])
            assert infos[j]["bnorm"] == pytest.approx(bn, rel=1e-12)
            assert infos[j]["true_rnorm"] <= 1.05e-8 * bn
            assert rel(got[:, j], Xr[:, j]) <= 1e-7, j
    finally:
        gp.close()


def test_multi_cg_agrees_with_single_vector_cg():
    ne = 13
    gp = GpuProblem(ne)
    try:
        k = 4
        Bh = rhs(gp.mesh, k, 20)
        X = torch.zeros_like(dev(Bh))
        infos = B.bamg_cg_solve_multi(gp.ctx, gp.mg, dev(Bh), X, k, 1e-8, 200)
        for j in range(k):
            x = torch.zeros(Bh.shape[0], dtype=torch.float64, device="cuda")
            out = B.bamg_cg_solve(gp.ctx, gp.mg, dev(Bh[:, j]), x, 1e-8, 200)
            assert abs(out["iterations"] - infos[j]["iterations"]) <= 1
            assert rel(X[:, j].cpu().numpy(), x.cpu().numpy()) <= 1e-7
    finally:
        gp.close()


@pytest.mark.parametrize("precision", [B.BAMG_FP64, B.BAMG_FP32])
def test_multi_cg_scaling_and_zero_columns_exact(precision):
    ne = 13
    gp = GpuProblem(ne, precision=precision)
    try:
        b = gaussian_rhs(gp.mesh, 0)
        Bh = np.stack([b, 2.0 * b, np.zeros_like(b), -0.25 * b, b], axis=1)
        X = torch.zeros_like(dev(Bh))
        infos = B.bamg_cg_solve_multi(gp.ctx, gp.mg, dev(Bh), X, 5, 1e-8, 200)
        assert torch.equal(X[:, 1], 2.0 * X[:, 0])
        assert torch.equal(X[:, 3], -0.25 * X[:, 0])
        assert torch.equal(X[:, 4], X[:, 0])
        assert not X[:, 2].any() and infos[2]["iterations"] == 0 and infos[2]["converged"]
        assert infos[0]["iterations"] == infos[1]["iterations"] == infos[3]["iterations"] > 0
    finally:
        gp.close()


def test_multi_mixed_precision_reaches_tolerance():
    ne = 13
    h = hierarchy(ne)
    gp = GpuProblem(ne, precision=B.BAMG_FP32)
    try:
        k = 16
        Bh = rhs(gp.mesh, k)
        X = torch.zeros_like(dev(Bh))
        infos = B.bamg_cg_solve_multi(gp.ctx, gp.mg, dev(Bh), X, k, 1e-8, 200)
        Xr, its, _ = OM.pcg_columns(h, Bh, 1e-8, 200)
        got = X.cpu().numpy()
        for j in range(k):
            bn = np.linalg.norm(Bh[:, j])
            assert infos[j]["converged"] and infos[j]["true_rnorm"] <= 1.05e-8 * bn
            assert abs(infos[j]["iterations"] - its[j]) <= 2
            assert rel(got[:, j], Xr[:, j]) <= 1e-6
        # the FP32 cycle is close to, not equal to, the FP64 one
        Y = torch.zeros_like(X)
        B.bamg_mg_vcycle_multi(gp.ctx, gp.mg, dev(Bh), Y, k)
        ref = OM.vcycle_columns(h, Bh)
        d = rel(Y.cpu().numpy(), ref)
        assert 1e-12 < d < 1e-4
        # and equal to the single-vector FP32 cycle column by column
        B.bamg_mg_set_lanes(gp.ctx, gp.mg, 1)
        B.bamg_mg_vcycle_multi(gp.ctx, gp.mg, dev(Bh), Y, k)
        for j in (0, 7, 15):
            y = torch.zeros(Bh.shape[0], dtype=torch.float64, device="cuda")
            B.bamg_vcycle(gp.ctx, gp.mg, dev(Bh[:, j]), y)
            assert torch.equal(Y[:, j], y), j
    finally:
        gp.close()


def test_multi_column_count_limits_and_maxit():
    ne = 8
    gp = GpuProblem(ne)
    try:
        m = gp.mesh.n_dofs
        Bh = rhs(gp.mesh, 32)
        X = torch.zeros_like(dev(Bh))
        infos = B.bamg_cg_solve_multi(gp.ctx, gp.mg, dev(Bh), X, 32, 1e-8, 200)
        assert all(i["converged"] for i in infos)
        for k in (0, 33):
            st = B.lib().bamg_cg_solve_multi(gp.mg, B._ptr(X), B._ptr(X), k, 1e-8, 10, None)
            assert st == B.BAMG_ERR_INVALID
        # a tolerance that cannot be met in 2 iterations: every column stops at maxit
        X2 = torch.zeros((m, 3), dtype=torch.float64, device="cuda")
        out = B.bamg_cg_solve_multi(gp.ctx, gp.mg, dev(Bh[:, :3]), X2, 3, 1e-14, 2, check=False)
        assert out[0]["status"] == B.BAMG_ERR_NOT_CONVERGED
        assert all(o["iterations"] == 2 and not o["converged"] for o in out)
        # a smaller column count reuses the larger work arrays
        infos = B.bamg_cg_solve_multi(gp.ctx, gp.mg, dev(Bh[:, :5]), X2.new_zeros((m, 5)), 5, 1e-8, 200)
        assert all(i["converged"] for i in infos)
    finally:
        gp.close()


def test_spmm_four_wide_matches_oracle_products():
    ne = 13
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        As = h.levels[0].As
        for k in (4, 16, 3):
            Xh = np.random.default_rng(k).standard_normal((As.shape[0], k))
            Y = torch.zeros_like(dev(Xh))
            B.bamg_bsr_spmm(gp.ctx, gp.A, dev(Xh), Y, k, B.BAMG_FP64)
            assert rel(Y.cpu().numpy(), As @ Xh) <= TOL64
    finally:
        gp.close()


@pytest.mark.parametrize("ne,k", [(13, 16), (13, 8), (8, 16), (13, 12)])
def test_spmm_fp32_matches_oracle_products(ne, k):
    """FP32 products of 8, 12 and 16 right-hand sides (8^3 has its fine
    operator stored with rows sorted by length): against the FP64 product of
    the oracle, at FP32 rounding, and against the FP32 product of the same
    values taken one column at a time."""
    h = hierarchy(ne)
    gp = GpuProblem(ne, precision=B.BAMG_FP32)
    try:
        As = h.levels[0].As
        n = As.shape[0]
        Xh = np.random.default_rng(k + ne).standard_normal((n, k)).astype(np.float32)
        Y = torch.zeros(n * k, dtype=torch.float32, device="cuda")
        B.bamg_bsr_spmm(gp.ctx, gp.A, torch.from_numpy(Xh.copy()).cuda(), Y, k, B.BAMG_FP32)
        got = Y.cpu().numpy().reshape(n, k).astype(np.float64)
        assert rel(got, As @ Xh.astype(np.float64)) <= 2e-6
        for j in (0, k - 1):
            y = torch.zeros(n, dtype=torch.float32, device="cuda")
            B.bamg_bsr_spmv(gp.ctx, gp.A, torch.from_numpy(np.ascontiguousarray(Xh[:, j])).cuda(), y, B.BAMG_FP32)
            assert rel(got[:, j], y.cpu().numpy().astype(np.float64)) <= 2e-6
    finally:
        gp.close()
