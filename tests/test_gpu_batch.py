"""GPU tests of the batch solver: one graph launch with a device-controlled
loop solves every problem exactly as a standalone solve would."""
import numpy as np
import pytest
import torch

from oracle import krylov
from oracle import multigrid as omg
from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import body_force, gaussian_rhs

from gpu_helpers import GpuProblem, rel
from oracle_cases import hierarchy

pytestmark = pytest.mark.gpu

CASES = [(6, 0.30), (10, 0.25), (8, 0.42), (13, 0.33), (7, 0.21), (9, 0.38)]


@pytest.fixture(scope="module")
def batch_set():
    probs = [GpuProblem(ne, nu=nu) for ne, nu in CASES]
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    bt = B.bamg_batch_create(ctx, [p.mg for p in probs])
    bs = [torch.from_numpy(gaussian_rhs(p.mesh, 40 + i)).cuda() for i, p in enumerate(probs)]
    yield ctx, bt, probs, bs
    B.bamg_batch_destroy(bt)
    B.bamg_ctx_destroy(ctx)
    for p in probs:
        p.close()


def standalone(probs, bs):
    xs, outs = [], []
    for p, b in zip(probs, bs):
        x = torch.zeros_like(b)
        outs.append(B.bamg_cg_solve(p.ctx, p.mg, b, x, 1e-8, 200))
        xs.append(x)
    return xs, outs


def test_batch_equals_standalone_solves_bitwise(batch_set):
    ctx, bt, probs, bs = batch_set
    xs = [torch.zeros_like(b) for b in bs]
    infos, loops = B.bamg_batch_cg_solve(ctx, bt, bs, xs, 1e-8, 200)
    ref_x, ref = standalone(probs, bs)
    for i in range(len(probs)):
        assert infos[i]["iterations"] == ref[i]["iterations"], i
        assert torch.equal(xs[i], ref_x[i]), i
        assert infos[i]["true_rnorm"] == ref[i]["true_rnorm"]
    assert loops == max(i["iterations"] for i in infos)
    # a second launch of the same graph gives the same answer
    xs2 = [torch.zeros_like(b) for b in bs]
    B.bamg_batch_cg_solve(ctx, bt, bs, xs2, 1e-8, 200)
    assert all(torch.equal(a, c) for a, c in zip(xs, xs2))


def test_batch_matches_oracle(batch_set):
    ctx, bt, probs, bs = batch_set
    xs = [torch.zeros_like(b) for b in bs]
    infos, _ = B.bamg_batch_cg_solve(ctx, bt, bs, xs, 1e-8, 200)
    for i in (0, 2, 3):
        ne, nu = CASES[i]
        h = hierarchy(ne, nu)
        b = bs[i].cpu().numpy()
        xr, its, _ = krylov.pcg(h.levels[0].As, b, lambda r: omg.vcycle(h, r), 1e-8, 200)
        assert abs(infos[i]["iterations"] - its) <= 1
        assert infos[i]["true_rnorm"] <= 1.05e-8 * np.linalg.norm(b)
        assert rel(xs[i].cpu().numpy(), xr) <= 1e-7


def test_batch_branch_counts_and_autotune(batch_set):
    ctx, bt, probs, bs = batch_set
    ref = None
    for nb in (1, 2, 3, len(probs)):
        B.bamg_batch_set_branches(ctx, bt, nb)
        assert B.bamg_batch_get_branches(bt) == nb
        xs = [torch.zeros_like(b) for b in bs]
        B.bamg_batch_cg_solve(ctx, bt, bs, xs, 1e-8, 200)
        if ref is None:
            ref = xs
        assert all(torch.equal(a, c) for a, c in zip(xs, ref))
    xs = [torch.zeros_like(b) for b in bs]
    ms = B.bamg_batch_autotune(ctx, bt, bs, xs, 1e-8, 200)
    assert ms > 0 and 1 <= B.bamg_batch_get_branches(bt) <= len(probs)
    B.bamg_batch_cg_solve(ctx, bt, bs, xs, 1e-8, 200)
    assert all(torch.equal(a, c) for a, c in zip(xs, ref))


def test_batch_zero_rhs_and_iteration_limit(batch_set):
    ctx, bt, probs, bs = batch_set
    bz = list(bs)
    bz[1] = torch.zeros_like(bs[1])
    xs = [torch.full_like(b, 7.0) for b in bs]
    infos, _ = B.bamg_batch_cg_solve(ctx, bt, bz, xs, 1e-8, 200)
    assert infos[1]["iterations"] == 0 and infos[1]["converged"] and not xs[1].any()
    infos, loops = B.bamg_batch_cg_solve(ctx, bt, bs, xs, 1e-14, 2, check=False)
    assert infos[0]["status"] == B.BAMG_ERR_NOT_CONVERGED
    # meshes of 6^3 and 7^3 elements have one level (a direct solve): one iteration
    assert loops == 2
    for (ne, _), i in zip(CASES, infos):
        if ne <= 7:
            assert i["iterations"] == 1 and i["converged"]
        else:
            assert i["iterations"] == 2 and not i["converged"]


def test_batch_mixes_precision_forms_and_rejects_shared_contexts():
    p64 = GpuProblem(8)
    p32 = GpuProblem(9, precision=B.BAMG_FP32)
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    try:
        bt = B.bamg_batch_create(ctx, [p64.mg, p32.mg])
        bs = [torch.from_numpy(body_force(p.mesh)).cuda() for p in (p64, p32)]
        xs = [torch.zeros_like(b) for b in bs]
        infos, _ = B.bamg_batch_cg_solve(ctx, bt, bs, xs, 1e-8, 200)
        ref_x, ref = standalone([p64, p32], bs)
        for i in range(2):
            assert infos[i]["converged"] and infos[i]["iterations"] == ref[i]["iterations"]
            assert torch.equal(xs[i], ref_x[i])
        B.bamg_batch_destroy(bt)
        with pytest.raises(B.BamgError) as e:
            B.bamg_batch_create(ctx, [p64.mg, p64.mg])
        assert e.value.status == B.BAMG_ERR_INVALID
    finally:
        B.bamg_ctx_destroy(ctx)
        p64.close()
        p32.close()
