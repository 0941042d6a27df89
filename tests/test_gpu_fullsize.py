"""Parity at the full benchmark size (64^3 elements, 823,875 dofs, 3 levels), in
the configuration bench.py times (autotuned lanes and splits): sampled block
rows that the oracle computes one by one from the COO stream, and properties
that hold at any size."""
import numpy as np
import pytest
import torch

from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import Mesh, body_force, coo_stream, element_scale

from gpu_helpers import TOL64, GpuProblem, rel
from test_pins_workload import rigid_modes

pytestmark = pytest.mark.gpu
NE = 64


@pytest.fixture(scope="module")
def big():
    gp = GpuProblem(NE)
    yield gp
    gp.close()


@pytest.fixture(scope="module")
def big32():
    gp = GpuProblem(NE, precision=B.BAMG_FP32)
    yield gp
    gp.close()


@pytest.fixture(scope="module")
def stream():
    mesh = Mesh(NE)
    s = coo_stream(mesh, 0.3, element_scale(mesh))
    bi, bj, v = s.bi.numpy(), s.bj.numpy(), s.vals.numpy().reshape(-1, 3, 3)
    order = np.argsort(bi, kind="stable")
    return bi, bj, v, order, np.searchsorted(bi[order], np.arange(mesh.n_nodes + 1))


def oracle_block_row(stream, I):
    """Block row I of the assembled operator: the sum of the stream's
    contributions to each (I, J), J ascending."""
    bi, bj, v, order, start = stream
    idx = order[start[I]:start[I + 1]]
    cols = np.unique(bj[idx])
    return cols, np.array([v[idx[bj[idx] == J]].sum(axis=0) for J in cols])


def test_sampled_rows_of_assembly_and_product(big, stream):
    rng = np.random.default_rng(64)
    n = big.mesh.n_nodes
    x = rng.standard_normal(3 * n)
    y = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    B.bamg_bsr_spmv(big.ctx, big.A, torch.from_numpy(x).cuda(), y)
    y = y.cpu().numpy()
    rows = rng.choice(n, 300, replace=False)
    rows[:3] = [0, n // 2, n - 1]
    for I in rows:
        cols, blocks = oracle_block_row(stream, I)
        want = sum(blocks[k] @ x[3 * J:3 * J + 3] for k, J in enumerate(cols))
        # rounding bound of a sum of products: a small multiple of eps * sum |a| |x|
        bound = sum(np.abs(blocks[k]) @ np.abs(x[3 * J:3 * J + 3]) for k, J in enumerate(cols))
        assert np.all(np.abs(y[3 * I:3 * I + 3] - want) <= 1e-13 * bound), I


def test_rigid_modes_are_in_the_kernel_of_interior_rows(big):
    x = rigid_modes(big.mesh.coords())
    clamp = np.repeat(big.mesh.dirichlet().astype(bool), 3)
    for k in range(6):
        y = torch.zeros(x.shape[0], dtype=torch.float64, device="cuda")
        B.bamg_bsr_spmv(big.ctx, big.A, torch.from_numpy(np.ascontiguousarray(x[:, k])).cuda(), y)
        y = y.cpu().numpy()
        ijk = big.mesh.node_ijk()
        inner = np.repeat(((ijk > 1) & (ijk < big.mesh.m - 1)).all(axis=1), 3) & ~clamp
        assert np.abs(y[inner]).max() <= 1e-12 * np.abs(y).max() + 1e-14


def test_galerkin_identity_on_every_level(big):
    """x_c^T A_c y_c = (P x_c)^T A (P y_c) and A_c symmetric, with the library's own products."""
    rng = np.random.default_rng(3)
    nl = B.bamg_mg_num_levels(big.mg)
    assert nl == 3
    for l in range(nl - 1):
        A, P = B.bamg_mg_get_level(big.mg, l)
        Ac, _ = B.bamg_mg_get_level(big.mg, l + 1)
        ic, ia = B.bamg_bsr_info(Ac), B.bamg_bsr_info(A)
        nc, nf = ic["nbr"] * ic["bs_r"], ia["nbr"] * ia["bs_r"]

        def mv(M, v, m):
            out = torch.zeros(m, dtype=torch.float64, device="cuda")
            B.bamg_bsr_spmv(big.ctx, M, v, out)
            return out

        xc = torch.from_numpy(rng.standard_normal(nc)).cuda()
        yc = torch.from_numpy(rng.standard_normal(nc)).cuda()
        lhs = float(xc @ mv(Ac, yc, nc))
        lhs_t = float(yc @ mv(Ac, xc, nc))
        px, py = mv(P, xc, nf), mv(P, yc, nf)
        rhs = float(px @ mv(A, py, nf))
        scale = float(torch.linalg.norm(px) * torch.linalg.norm(mv(A, py, nf)))
        assert abs(lhs - rhs) <= 1e-12 * scale, l
        assert abs(lhs - lhs_t) <= 1e-12 * scale, l


@pytest.mark.parametrize("precision", [B.BAMG_FP64, B.BAMG_FP32])
def test_cg_reaches_the_tolerance_with_the_true_residual(big, big32, precision):
    gp = big if precision == B.BAMG_FP64 else big32
    b = torch.from_numpy(body_force(gp.mesh)).cuda()
    x = torch.zeros_like(b)
    out = B.bamg_cg_solve(gp.ctx, gp.mg, b, x, 1e-8, 200)
    assert out["converged"] and out["iterations"] <= 40
    r = torch.zeros_like(b)   # b - A x with the plain product, not CG's recurrence
    B.bamg_bsr_spmv(gp.ctx, gp.A, x, r)
    true_rel = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
    assert true_rel <= 1.05e-8
    assert out["true_rnorm"] / out["bnorm"] == pytest.approx(true_rel, rel=1e-6, abs=1e-12)


def test_finest_restriction_in_its_tuned_forms(big32):
    """The finest restriction (9,261 rows of 6x3 blocks) in the forms the
    autotuner chose for the mixed cycle: the FP64 product equals a host sum of
    its own blocks on sampled rows, and the FP32 product (the block split,
    where the tuner keeps it) stays within FP32 rounding of the FP64 one."""
    gp = big32
    R = B.bamg_mg_get_restriction(gp.mg, 0)
    info = B.bamg_bsr_info(R)
    assert (info["bs_r"], info["bs_c"]) == (6, 3)
    nbr, nbc, nnzb = info["nbr"], info["nbc"], info["nnzb"]
    rowptr = torch.zeros(nbr + 1, dtype=torch.int32, device="cuda")
    colidx = torch.zeros(nnzb, dtype=torch.int32, device="cuda")
    vals = torch.zeros(nnzb * 18, dtype=torch.float64, device="cuda")
    B.bamg_bsr_get_pattern(gp.ctx, R, rowptr, colidx)
    B.bamg_bsr_get_values(gp.ctx, R, vals)
    rowptr, colidx, vals = rowptr.cpu().numpy(), colidx.cpu().numpy(), vals.cpu().numpy().reshape(-1, 6, 3)
    x = np.random.default_rng(11).standard_normal(nbc * 3)
    y64 = torch.zeros(nbr * 6, dtype=torch.float64, device="cuda")
    B.bamg_bsr_spmv(gp.ctx, R, torch.from_numpy(x).cuda(), y64)
    y32 = torch.zeros(nbr * 6, dtype=torch.float32, device="cuda")
    B.bamg_bsr_spmv(gp.ctx, R, torch.from_numpy(x).float().cuda(), y32, B.BAMG_FP32)
    y64, y32 = y64.cpu().numpy(), y32.double().cpu().numpy()
    xb = x.reshape(-1, 3)
    for I in np.random.default_rng(12).choice(nbr, 48, replace=False):
        k0, k1 = rowptr[I], rowptr[I + 1]
        ref = np.einsum("krc,kc->r", vals[k0:k1], xb[colidx[k0:k1]])
        assert rel(y64[6 * I:6 * I + 6], ref) <= 1e-13
    assert rel(y32, y64) <= 1e-5


def test_booked_vcycles_equal_fine_chebyshev_launches(big):
    """The bench's byte count books bench.vcycles_per_solve(its) V-cycles per
    solve; each V-cycle launches the fine Chebyshev step three times (two
    pre-smoothing steps, one post-smoothing step after the residual start)."""
    import bench
    b = torch.from_numpy(body_force(big.mesh)).cuda()
    x = torch.zeros_like(b)
    B.bamg_mg_update(big.ctx, big.mg)
    B.bamg_cg_solve(big.ctx, big.mg, b, x, 1e-8, 500)      # captures the graphs
    B.bamg_ctx_profile_slots(big.ctx, ["cheb_step_l0"])
    try:
        out = B.bamg_cg_solve(big.ctx, big.mg, b, x, 1e-8, 500)
        torch.cuda.synchronize()
        _, launches = B.bamg_ctx_profile_read(big.ctx, B.PROF_SLOTS["cheb_step_l0"])
    finally:
        B.bamg_ctx_profile_slots(big.ctx, [])
    assert launches == 3 * bench.vcycles_per_solve(out["iterations"])


def test_mis_hierarchy_properties_at_full_size(big):
    """The hierarchy built from device MIS aggregates of the same operator
    (4 levels, coarse operators of 67 and 244 blocks per row, stored sorted
    by row length): Galerkin identity and symmetry on every level, and CG to
    rtol 1e-8 with the true residual."""
    o = B.bamg_mg_opts_default()
    o.grid[0] = o.grid[1] = o.grid[2] = big.mesh.m
    o.aggregation = B.BAMG_AGG_MIS
    mg = B.bamg_mg_setup(big.ctx, big.A, big.mesh.coords(), big.mesh.dirichlet(), o)
    try:
        nl = B.bamg_mg_num_levels(mg)
        assert nl == 4
        rng = np.random.default_rng(5)
        for l in range(nl - 1):
            A, P = B.bamg_mg_get_level(mg, l)
            Ac, _ = B.bamg_mg_get_level(mg, l + 1)
            ic, ia = B.bamg_bsr_info(Ac), B.bamg_bsr_info(A)
            nc, nf = ic["nbr"] * ic["bs_r"], ia["nbr"] * ia["bs_r"]

            def mv(M, v, m):
                out = torch.zeros(m, dtype=torch.float64, device="cuda")
                B.bamg_bsr_spmv(big.ctx, M, v, out)
                return out

            xc = torch.from_numpy(rng.standard_normal(nc)).cuda()
            yc = torch.from_numpy(rng.standard_normal(nc)).cuda()
            lhs, lhs_t = float(xc @ mv(Ac, yc, nc)), float(yc @ mv(Ac, xc, nc))
            px, py = mv(P, xc, nf), mv(P, yc, nf)
            apy = mv(A, py, nf)
            scale = float(torch.linalg.norm(px) * torch.linalg.norm(apy))
            assert abs(lhs - float(px @ apy)) <= 1e-12 * scale, l
            assert abs(lhs - lhs_t) <= 1e-12 * scale, l
        assert B.bamg_bsr_storage(B.bamg_mg_get_level(mg, 1)[0])["rows_sorted"]
        b = torch.from_numpy(body_force(big.mesh)).cuda()
        x = torch.zeros_like(b)
        out = B.bamg_cg_solve(big.ctx, mg, b, x, 1e-8, 200)
        assert out["converged"]
        r = torch.zeros_like(b)
        B.bamg_bsr_spmv(big.ctx, big.A, x, r)
        assert float(torch.linalg.norm(b - r) / torch.linalg.norm(b)) <= 1.05e-8
    finally:
        B.bamg_mg_destroy(mg)
