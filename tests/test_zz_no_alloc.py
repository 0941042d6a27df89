"""The allocation-free residual-norm entry point.

Some callers cannot call cudaMalloc (an application whose device memory is
all pre-reserved by its own pool, where one more allocation would fail); they use
bamg_bsr_residual_norm_noalloc, whose reduction scratch is a fixed device
array inside the library.  Its result must equal the residual norm that the
existing CG entry point reports for the same solution, on two calls in a row.
This file is collected last so that a run stopping at the first failure has
run every other test before it.
"""
import numpy as np
import pytest
import torch

from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import body_force

from gpu_helpers import GpuProblem

pytestmark = pytest.mark.gpu


def test_noalloc_residual_norm_matches_cg_true_residual():
    B.lib()
    gp = GpuProblem(8)
    try:
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        x = torch.zeros_like(b)
        out = B.bamg_cg_solve(gp.ctx, gp.mg, b, x, 1e-6, 100)
        ref = out["true_rnorm"]
        assert ref > 0
        for _ in range(2):                      # two calls in a row share the scratch
            norm = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            B.bamg_bsr_residual_norm_noalloc(gp.ctx, gp.A, x, b, norm)
            torch.cuda.synchronize()
            got = float(norm.item())
            assert abs(got - ref) <= 1e-12 * ref
        # an exact solution gives zero, a zero guess gives ||b||
        zero = torch.zeros_like(b)
        norm = torch.empty((1,), dtype=torch.float64, device="cuda")
        B.bamg_bsr_residual_norm_noalloc(gp.ctx, gp.A, zero, b, norm)
        torch.cuda.synchronize()
        assert abs(float(norm.item()) - float(torch.linalg.norm(b))) <= 1e-12 * float(torch.linalg.norm(b))
    finally:
        gp.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    n = 4096 * 128 + 64                         # one more slice than the scratch covers
    A = B.bamg_bsr_create(ctx, 3, 3, n, n)
    try:
        idx = torch.arange(n, dtype=torch.int32, device="cuda")
        B.bamg_bsr_coo_preallocate(ctx, A, idx, idx)
        B.bamg_bsr_set_lanes(ctx, A, 1)
        v = torch.eye(3, dtype=torch.float64, device="cuda").repeat(n, 1, 1)
        B.bamg_bsr_coo_set_values(ctx, A, v, 0)
        x = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
        norm = torch.empty((1,), dtype=torch.float64, device="cuda")
        with pytest.raises(B.BamgError) as e:
            B.bamg_bsr_residual_norm_noalloc(ctx, A, x, x, norm)
        assert e.value.status == 1 and "at most 4096" in str(e.value)
    finally:
        B.bamg_bsr_destroy(A)
        B.bamg_ctx_destroy(ctx)
