"""Q2 elements (27-node hexahedra, up to 125 blocks per row): the whole
reuse path against the oracle (the paper's nonzeros-per-row study, Sec. 4.6)."""
import numpy as np
import pytest
import torch

from oracle import krylov
from oracle import learned as OL
from oracle import multigrid as omg
from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import body_force

from gpu_helpers import TOL64, GpuProblem, read_bsr, rel, same_pattern
from oracle_cases import hierarchy, problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ne", [4, 12])
def test_q2_hierarchy_and_cycle_match_oracle(ne):
    mesh, _, Aref = problem(ne, order=2)
    h = hierarchy(ne, order=2)
    gp = GpuProblem(ne, order=2)
    try:
        A = read_bsr(gp.ctx, gp.A)
        assert same_pattern(A, Aref) and rel(A.vals, Aref.vals) <= 1e-15
        assert int(np.diff(A.rowptr).max()) == 125
        nl = B.bamg_mg_num_levels(gp.mg)
        assert nl == h.n_levels >= 2
        for l in range(nl):
            Al, _ = B.bamg_mg_get_level(gp.mg, l)
            ga = read_bsr(gp.ctx, Al)
            assert same_pattern(ga, h.levels[l].A) and rel(ga.vals, h.levels[l].A.vals) <= TOL64, l
        b = np.random.default_rng(ne).standard_normal(mesh.n_dofs)
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x)
        assert rel(x.cpu().numpy(), omg.vcycle(h, b)) <= TOL64
        f = body_force(mesh)
        xr, its, _ = krylov.pcg(h.levels[0].As, f, lambda r: omg.vcycle(h, r), 1e-8, 200)
        x = torch.zeros(f.size, dtype=torch.float64, device="cuda")
        out = B.bamg_cg_solve(gp.ctx, gp.mg, torch.from_numpy(f).cuda(), x, 1e-8, 200)
        assert out["converged"] and abs(out["iterations"] - its) <= 1
        assert rel(x.cpu().numpy(), xr) <= 1e-7
    finally:
        gp.close()


def unsorted_slots(rowptr) -> int:
    """Slots of the plain sliced layout: every 32-row slice padded to its
    longest row (the storage without a row sort)."""
    lens = np.diff(rowptr)
    pad = np.zeros(-(-lens.size // 32) * 32, dtype=np.int64)
    pad[:lens.size] = lens
    return int(pad.reshape(-1, 32).max(axis=1).sum()) * 32


def test_q2_rows_sorted_by_length_in_every_row_kernel():
    """Q2's vertex and mid-edge rows (125 and fewer blocks) alternate along x:
    the library stores the fine operator with rows sorted by length (slot_row
    maps positions to rows).  Every row kernel that walks it by position must
    still write by row: the SpMV, the multi-vector cycle (bitwise equal to
    single cycles), the allocation-free residual, the CG exit residual, the
    mixed-precision cycle and the learned features."""
    ne = 12
    mesh, _, Aref = problem(ne, order=2)
    h = hierarchy(ne, order=2)
    gp = GpuProblem(ne, order=2)
    gq = None
    try:
        st = B.bamg_bsr_storage(gp.A)
        plain = unsorted_slots(Aref.rowptr)
        assert st["rows_sorted"]
        assert Aref.nnzb <= st["stored_slots"] <= 0.9 * plain
        A1, _ = B.bamg_mg_get_level(gp.mg, 1)
        assert B.bamg_bsr_storage(A1)["rows_sorted"]  # the 6x6 split kernels too
        rng = np.random.default_rng(5)
        xh = rng.standard_normal(mesh.n_dofs)
        y = torch.empty(mesh.n_dofs, dtype=torch.float64, device="cuda")
        B.bamg_bsr_spmv(gp.ctx, gp.A, torch.from_numpy(xh).cuda(), y)
        assert rel(y.cpu().numpy(), Aref.scalar() @ xh) <= 1e-14
        # multi-vector cycle against single-vector cycles, bit for bit
        B.bamg_mg_set_lanes(gp.ctx, gp.mg, 1)
        k = 5
        Bh = np.ascontiguousarray(rng.standard_normal((mesh.n_dofs, k)))
        X = torch.zeros(Bh.shape, dtype=torch.float64, device="cuda")
        B.bamg_mg_vcycle_multi(gp.ctx, gp.mg, torch.from_numpy(Bh).cuda(), X, k)
        for j in range(k):
            x = torch.zeros(mesh.n_dofs, dtype=torch.float64, device="cuda")
            B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(np.ascontiguousarray(Bh[:, j])).cuda(), x)
            assert torch.equal(X[:, j], x), j
            assert rel(x.cpu().numpy(), omg.vcycle(h, Bh[:, j])) <= TOL64, j
        # residual norms: allocation-free entry and the CG exit
        f = body_force(mesh)
        fd = torch.from_numpy(f).cuda()
        x = torch.zeros_like(fd)
        out = B.bamg_cg_solve(gp.ctx, gp.mg, fd, x, 1e-8, 200)
        res = float(np.linalg.norm(f - Aref.scalar() @ x.cpu().numpy()))
        assert abs(out["true_rnorm"] - res) <= 1e-9 * np.linalg.norm(f)
        norm = torch.empty(1, dtype=torch.float64, device="cuda")
        B.bamg_bsr_residual_norm_noalloc(gp.ctx, gp.A, x, fd, norm)
        torch.cuda.synchronize()
        assert abs(float(norm.item()) - out["true_rnorm"]) <= 1e-12 * out["true_rnorm"]
        # learned-smoother features, row by row
        for l in range(h.n_levels - 1):
            L = h.levels[l]
            Xf = torch.empty((L.A.nbr, 8), dtype=torch.float32, device="cuda")
            B.bamg_mg_block_features(gp.ctx, gp.mg, l, Xf)
            assert np.allclose(Xf.cpu().numpy(), OL.block_features(L.A, l, L.Dinv), rtol=1e-5, atol=1e-6), l
        # the mixed form (FP32 cycle) reaches the same tolerance
        gq = GpuProblem(ne, order=2, precision=B.BAMG_FP32)
        xq = torch.zeros_like(fd)
        outq = B.bamg_cg_solve(gq.ctx, gq.mg, fd, xq, 1e-8, 200)
        assert outq["converged"] and abs(outq["iterations"] - out["iterations"]) <= 2
        assert outq["true_rnorm"] <= 1.05e-8 * np.linalg.norm(f)
    finally:
        gp.close()
        if gq is not None:
            gq.close()


@pytest.mark.parametrize("precision", [B.BAMG_FP64, B.BAMG_FP32])
def test_q2_full_size_properties(precision):
    """32^3 Q2 elements, the bench's Q2 size (823,875 dofs, 16.97 M blocks,
    3 levels), in the autotuned configuration: the fine operator stored
    sorted by row length, the Galerkin identity and symmetry on every level,
    and CG to rtol 1e-8 with the true residual."""
    ne = 32
    gp = GpuProblem(ne, order=2, precision=precision)
    try:
        nl = B.bamg_mg_num_levels(gp.mg)
        assert nl == 3
        assert B.bamg_bsr_storage(gp.A)["rows_sorted"]
        rng = np.random.default_rng(32)

        def mv(M, v, m):
            out = torch.zeros(m, dtype=torch.float64, device="cuda")
            B.bamg_bsr_spmv(gp.ctx, M, v, out)
            return out

        if precision == B.BAMG_FP64:
            for l in range(nl - 1):
                A, P = B.bamg_mg_get_level(gp.mg, l)
                Ac, _ = B.bamg_mg_get_level(gp.mg, l + 1)
                ic, ia = B.bamg_bsr_info(Ac), B.bamg_bsr_info(A)
                nc, nf = ic["nbr"] * ic["bs_r"], ia["nbr"] * ia["bs_r"]
                xc = torch.from_numpy(rng.standard_normal(nc)).cuda()
                yc = torch.from_numpy(rng.standard_normal(nc)).cuda()
                lhs, lhs_t = float(xc @ mv(Ac, yc, nc)), float(yc @ mv(Ac, xc, nc))
                px, py = mv(P, xc, nf), mv(P, yc, nf)
                apy = mv(A, py, nf)
                scale = float(torch.linalg.norm(px) * torch.linalg.norm(apy))
                assert abs(lhs - float(px @ apy)) <= 1e-12 * scale, l
                assert abs(lhs - lhs_t) <= 1e-12 * scale, l
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        x = torch.zeros_like(b)
        out = B.bamg_cg_solve(gp.ctx, gp.mg, b, x, 1e-8, 200)
        assert out["converged"] and out["iterations"] <= 40
        r = mv(gp.A, x, b.numel())
        assert float(torch.linalg.norm(b - r) / torch.linalg.norm(b)) <= 1.05e-8
    finally:
        gp.close()
