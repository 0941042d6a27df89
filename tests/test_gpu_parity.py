"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Patterns and aggregates must match bit-exactly; FP64 values to 1e-12
normwise relative error (||X_gpu - X_oracle|| / ||X_oracle||)."""
import numpy as np
import pytest
import torch

from oracle import krylov, multigrid as omg
from oracle.assembly import coo_assemble_blocks
from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import Mesh, body_force

from gpu_helpers import TOL64, GpuProblem, read_bsr, rel, same_pattern
from oracle_cases import hierarchy, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.lib()


def random_stream(rng, nbr, nbc, br, bc, n, neg=True):
    bi = rng.integers(-1 if neg else 0, nbr, n).astype(np.int32)
    bj = rng.integers(-1 if neg else 0, nbc, n).astype(np.int32)
    v = rng.standard_normal((n, br, bc))
    return bi, bj, v


@pytest.mark.parametrize("br,bc", [(3, 3), (6, 6), (3, 6), (6, 3), (2, 5)])
def test_coo_assembly_and_spmv(br, bc):
    rng = np.random.default_rng(br * 10 + bc)
    nbr, nbc, n = 77, 53, 2000       # several slices and a ragged tail
    bi, bj, v = random_stream(rng, nbr, nbc, br, bc, n)
    ref = coo_assemble_blocks(nbr, nbc, br, bc, bi, bj, v)
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    A = B.bamg_bsr_create(ctx, br, bc, nbr, nbc)
    try:
        B.bamg_bsr_coo_preallocate(ctx, A, torch.from_numpy(bi).cuda(), torch.from_numpy(bj).cuda())
        vt = torch.from_numpy(v).cuda()
        B.bamg_bsr_coo_set_values(ctx, A, vt, 0)
        got = read_bsr(ctx, A)
        assert same_pattern(got, ref)
        assert rel(got.vals, ref.vals) <= 1e-15
        B.bamg_bsr_coo_set_values(ctx, A, vt, 1)          # ADD mode doubles every block
        assert rel(read_bsr(ctx, A).vals, 2 * ref.vals) <= 1e-15
        B.bamg_bsr_coo_set_values(ctx, A, vt, 0)
        x = rng.standard_normal(nbc * bc)
        y = torch.zeros(nbr * br, dtype=torch.float64, device="cuda")
        B.bamg_bsr_spmv(ctx, A, torch.from_numpy(x).cuda(), y)
        yref = ref.scalar() @ x
        assert rel(y.cpu().numpy(), yref) <= 1e-14
        y32 = torch.zeros(nbr * br, dtype=torch.float32, device="cuda")
        B.bamg_bsr_spmv(ctx, A, torch.from_numpy(x.astype(np.float32)).cuda(), y32, B.BAMG_FP32)
        assert rel(y32.cpu().numpy(), yref) <= 1e-5
        if (br, bc) != (2, 5):
            k = 5
            X = rng.standard_normal((nbc * bc, k))
            Y = torch.zeros(nbr * br * k, dtype=torch.float64, device="cuda")
            B.bamg_bsr_spmm(ctx, A, torch.from_numpy(X.copy()).cuda(), Y, k)
            assert rel(Y.cpu().numpy().reshape(-1, k), ref.scalar() @ X) <= 1e-14
    finally:
        B.bamg_bsr_destroy(A)
        B.bamg_ctx_destroy(ctx)


def test_coo_rejects_out_of_range_index():
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    A = B.bamg_bsr_create(ctx, 3, 3, 4, 4)
    try:
        bi = torch.tensor([0, 1, 4], dtype=torch.int32, device="cuda")
        bj = torch.tensor([0, 1, 1], dtype=torch.int32, device="cuda")
        with pytest.raises(B.BamgError) as e:
            B.bamg_bsr_coo_preallocate(ctx, A, bi, bj)
        assert e.value.status == 1
    finally:
        B.bamg_bsr_destroy(A)
        B.bamg_ctx_destroy(ctx)


@pytest.mark.parametrize("case", ["empty", "all_dropped", "single", "one_long_row"])
def test_coo_degenerate_streams(case):
    """Blocked COO (Sec. 3.4) on the degenerate streams: no entries, entries
    that all carry a negative index (dropped), one contribution in the last
    row, and one row of many duplicates beside empty rows.  Pattern and
    values as the oracle's, the product A x as the oracle's (zero where A is
    empty), in INSERT and ADD mode."""
    rng = np.random.default_rng(11)
    br = bc = 3
    nbr, nbc = 40, 40
    if case == "empty":
        bi = bj = np.zeros(0, dtype=np.int32)
    elif case == "all_dropped":
        bi = np.full(10, -1, dtype=np.int32)
        bj = np.arange(10, dtype=np.int32)
    elif case == "single":
        bi = np.array([nbr - 1], dtype=np.int32)
        bj = np.array([0], dtype=np.int32)
    else:
        bi = np.full(300, 5, dtype=np.int32)
        bj = rng.integers(0, nbc, 300).astype(np.int32)
    v = rng.standard_normal((bi.size, br, bc))
    ref = coo_assemble_blocks(nbr, nbc, br, bc, bi, bj, v)
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    A = B.bamg_bsr_create(ctx, br, bc, nbr, nbc)
    try:
        B.bamg_bsr_coo_preallocate(ctx, A, torch.from_numpy(bi).cuda(), torch.from_numpy(bj).cuda())
        vt = torch.from_numpy(v.reshape(-1)).cuda()
        for add, scale in ((0, 1.0), (1, 2.0)):
            B.bamg_bsr_coo_set_values(ctx, A, vt, add)
            got = read_bsr(ctx, A)
            assert same_pattern(got, ref)
            assert got.nnzb == ref.nnzb
            if ref.nnzb:
                assert rel(got.vals, scale * ref.vals) <= 1e-15
        B.bamg_bsr_coo_set_values(ctx, A, vt, 0)
        x = rng.standard_normal(nbc * bc)
        y = torch.full((nbr * br,), 7.0, dtype=torch.float64, device="cuda")
        B.bamg_bsr_spmv(ctx, A, torch.from_numpy(x).cuda(), y)
        yref = ref.scalar() @ x
        assert np.allclose(y.cpu().numpy(), yref, rtol=1e-14, atol=1e-14 * max(1.0, np.abs(yref).max(initial=0.0)))
    finally:
        B.bamg_bsr_destroy(A)
        B.bamg_ctx_destroy(ctx)


def test_general_galerkin_product_through_the_abi():
    from oracle.galerkin import galerkin
    rng = np.random.default_rng(11)
    for (bs, bsp, n, nc) in ((3, 6, 150, 40), (6, 6, 90, 33)):
        bi, bj, v = random_stream(rng, n, n, bs, bs, 1500, neg=False)
        pi, pj, pv = random_stream(rng, n, nc, bs, bsp, 400, neg=False)
        Aref = coo_assemble_blocks(n, n, bs, bs, bi, bj, v)
        Pref = coo_assemble_blocks(n, nc, bs, bsp, pi, pj, pv)
        ref = galerkin(Aref, Pref)
        ctx = B.bamg_ctx_create(torch.cuda.current_stream())
        A = B.bamg_bsr_create(ctx, bs, bs, n, n)
        P = B.bamg_bsr_create(ctx, bs, bsp, n, nc)
        plan = Ac = None
        try:
            B.bamg_bsr_coo_preallocate(ctx, A, torch.from_numpy(bi).cuda(), torch.from_numpy(bj).cuda())
            B.bamg_bsr_coo_set_values(ctx, A, torch.from_numpy(v).cuda(), 0)
            B.bamg_bsr_coo_preallocate(ctx, P, torch.from_numpy(pi).cuda(), torch.from_numpy(pj).cuda())
            B.bamg_bsr_coo_set_values(ctx, P, torch.from_numpy(pv).cuda(), 0)
            plan, Ac = B.bamg_ptap_symbolic(ctx, A, P)
            B.bamg_ptap_numeric(ctx, plan, A, P, Ac)
            got = read_bsr(ctx, Ac)
            assert same_pattern(got, ref)
            assert rel(got.vals, ref.vals) <= TOL64
            first = got.vals.copy()
            B.bamg_ptap_numeric(ctx, plan, A, P, Ac)      # deterministic: bitwise equal
            assert np.array_equal(read_bsr(ctx, Ac).vals, first)
            B.bamg_ptap_numeric_prec(ctx, plan, A, P, Ac, B.BAMG_FP32)
            with pytest.raises(B.BamgError):
                B.bamg_bsr_get_values(ctx, Ac, torch.empty(10, dtype=torch.float64, device="cuda"))
            B.bamg_ptap_numeric(ctx, plan, A, P, Ac)
            assert np.array_equal(read_bsr(ctx, Ac).vals, first)
        finally:
            if plan is not None:
                B.bamg_ptap_destroy(plan)
                B.bamg_bsr_destroy(Ac)
            B.bamg_bsr_destroy(P)
            B.bamg_bsr_destroy(A)
            B.bamg_ctx_destroy(ctx)


@pytest.mark.parametrize("ne", [8, 13, 24])
def test_hierarchy_matches_oracle(ne):
    """Assembled A, P and A_c of every level, eigen-estimates, damping and Dinv."""
    mesh, s, Aref = problem(ne)
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        A = read_bsr(gp.ctx, gp.A)
        assert same_pattern(A, Aref) and rel(A.vals, Aref.vals) <= 1e-15
        nl = B.bamg_mg_num_levels(gp.mg)
        assert nl == h.n_levels
        for l in range(nl):
            Al, Pl = B.bamg_mg_get_level(gp.mg, l)
            ga = read_bsr(gp.ctx, Al)
            assert same_pattern(ga, h.levels[l].A), f"level {l} operator pattern"
            assert rel(ga.vals, h.levels[l].A.vals) <= TOL64, f"level {l} operator values"
            if l + 1 < nl:
                gpP = read_bsr(gp.ctx, Pl)
                assert same_pattern(gpP, h.levels[l].P), f"level {l} prolongator pattern"
                assert rel(gpP.vals, h.levels[l].P.vals) <= TOL64, f"level {l} prolongator values"
                lam, om = B.bamg_mg_get_level_scalars(gp.ctx, gp.mg, l)
                assert abs(om - h.levels[l].omega) <= 1e-12 * h.levels[l].omega
                assert abs(lam - h.levels[l].lam) <= 1e-12 * h.levels[l].lam
                d = torch.empty(h.levels[l].A.nbr * h.levels[l].A.bs_r ** 2, dtype=torch.float64, device="cuda")
                B.bamg_mg_get_dinv(gp.ctx, gp.mg, l, d)
                assert rel(d.cpu().numpy(), h.levels[l].Dinv.reshape(-1)) <= TOL64
    finally:
        gp.close()


@pytest.mark.parametrize("ne", [8, 24])
def test_vcycle_matches_oracle(ne):
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        rng = np.random.default_rng(ne)
        b = rng.standard_normal(gp.mesh.n_dofs)
        x = torch.zeros_like(torch.from_numpy(b)).cuda()
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x)
        ref = omg.vcycle(h, b)
        assert rel(x.cpu().numpy(), ref) <= TOL64
    finally:
        gp.close()


@pytest.mark.parametrize("ne", [13, 16, 20])
@pytest.mark.parametrize("form", [1, 2])
def test_coarsest_solve_forms_match_oracle(ne, form):
    """Dense and banded (block-tridiagonal) coarsest factorisations give the
    oracle's cycle; 20^3 elements has the 7^3-node coarsest level of the
    64^3-element workload (2,058 dofs, six 352-row chunks)."""
    h = hierarchy(ne)
    gp = GpuProblem(ne, coarse_solver=form)
    try:
        rng = np.random.default_rng(100 + ne)
        b = rng.standard_normal(gp.mesh.n_dofs)
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x)
        assert rel(x.cpu().numpy(), omg.vcycle(h, b)) <= TOL64
        # the coarsest operator itself
        nl = B.bamg_mg_num_levels(gp.mg)
        Ac, _ = B.bamg_mg_get_level(gp.mg, nl - 1)
        C = read_bsr(gp.ctx, Ac)
        L = h.levels[-1]
        assert rel(C.vals, L.A.vals) <= TOL64
        # FP32 precision form on the same structure
        if form == 2:
            g32 = GpuProblem(ne, precision=B.BAMG_FP32, coarse_solver=form)
            try:
                y = torch.zeros_like(x)
                B.bamg_vcycle(g32.ctx, g32.mg, torch.from_numpy(b).cuda(), y)
                assert rel(y.cpu().numpy(), omg.vcycle(h, b)) < 1e-3   # FP32 cycle
            finally:
                g32.close()
    finally:
        gp.close()


@pytest.mark.parametrize("ne,form", [(6, 1), (6, 2), (9, 0), (9, 1)])
def test_one_level_cycle_is_the_exact_solve(ne, form):
    """With a single level the cycle is the coarsest solve of the fine 3x3-block
    operator: compare with a sparse direct solve (banded: 6 or 9 chunks)."""
    import scipy.sparse.linalg as spla
    _, _, A = problem(ne)
    gp = GpuProblem(ne, max_coarse_dofs=10 ** 6, coarse_solver=form)
    try:
        assert B.bamg_mg_num_levels(gp.mg) == 1
        b = np.random.default_rng(ne).standard_normal(gp.mesh.n_dofs)
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x)
        ref = spla.spsolve(A.scalar().tocsc(), b)
        assert rel(x.cpu().numpy(), ref) <= 1e-11
    finally:
        gp.close()


@pytest.mark.parametrize("ne", [8, 24])
def test_cg_matches_oracle(ne):
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        b = body_force(gp.mesh)
        xr, its, info = krylov.pcg(h.levels[0].As, b, lambda r: omg.vcycle(h, r), 1e-8, 200)
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        out = B.bamg_cg_solve(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x, 1e-8, 200)
        assert out["converged"]
        assert abs(out["iterations"] - its) <= 1
        assert out["true_rnorm"] <= 1.05e-8 * np.linalg.norm(b)
        assert rel(x.cpu().numpy(), xr) <= 1e-7
    finally:
        gp.close()


def test_profiling_slots_time_only_the_chosen_kernels():
    """A slot mask brackets only the chosen launches; the solve is unchanged."""
    ne = 16
    gp = GpuProblem(ne)
    try:
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        x0 = torch.zeros_like(b)
        out0 = B.bamg_cg_solve(gp.ctx, gp.mg, b, x0, 1e-8, 200)
        B.bamg_ctx_profile_slots(gp.ctx, ["cheb_step_l0", "cg_ap"])
        x1 = torch.zeros_like(b)
        out1 = B.bamg_cg_solve(gp.ctx, gp.mg, b, x1, 1e-8, 200)
        got = {k: B.bamg_ctx_profile_read(gp.ctx, s) for k, s in B.PROF_SLOTS.items()}
        B.bamg_ctx_profile(gp.ctx, 0)
        its = out1["iterations"]
        assert abs(got["cg_ap"][1] - its) <= 1 and got["cg_ap"][0] > 0
        assert got["cheb_step_l0"][1] > 0
        assert all(v[1] == 0 for k, v in got.items() if k not in ("cheb_step_l0", "cg_ap"))
        assert its == out0["iterations"] and torch.equal(x0, x1)
    finally:
        gp.close()


def test_sampling_slot_takes_the_pre_smoothing_pair():
    """The sampling slot brackets the finest pre-smoothing pair of every cycle
    (one bracket, two launches); slot 0 then keeps only the post-smoothing
    step.  The all-slot profile leaves the sampling slot off."""
    gp = GpuProblem(16)
    try:
        b = torch.from_numpy(body_force(gp.mesh)).cuda()

        def solve():
            x = torch.zeros_like(b)
            return B.bamg_cg_solve(gp.ctx, gp.mg, b, x, 1e-8, 200)["iterations"]

        def launches(name):
            return B.bamg_ctx_profile_read(gp.ctx, B.PROF_SLOTS[name])[1]

        B.bamg_ctx_profile_slots(gp.ctx, ["cheb_step_l0"])
        its = solve()
        full = launches("cheb_step_l0")
        B.bamg_ctx_profile_slots(gp.ctx, ["cheb_step_l0", "cheb_pre_l0"])
        assert solve() == its
        post, pre = launches("cheb_step_l0"), launches("cheb_pre_l0")
        assert full > 0 and pre == 2 * post and pre + post == full
        B.bamg_ctx_profile_slots(gp.ctx, ["cheb_pre_l0"])
        assert solve() == its
        assert launches("cheb_pre_l0") == pre and launches("cheb_step_l0") == 0
        B.bamg_ctx_profile(gp.ctx, 1)
        assert solve() == its
        assert launches("cheb_pre_l0") == 0 and launches("cheb_step_l0") == full
        B.bamg_ctx_profile(gp.ctx, 0)
    finally:
        gp.close()


def test_device_memory_counts_the_library_allocations():
    """The pool counters see a hierarchy's allocations and their high-water mark."""
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    try:
        used0, _ = B.bamg_device_memory(ctx, reset_peak=True)
        gp = GpuProblem(12)
        try:
            used1, peak1 = B.bamg_device_memory(gp.ctx)
            assert used1 > used0 and peak1 >= used1
        finally:
            gp.close()
        used2, peak2 = B.bamg_device_memory(ctx)
        assert used2 < used1 and peak2 >= peak1
    finally:
        B.bamg_ctx_destroy(ctx)


@pytest.mark.parametrize("ne", [5, 12])
def test_element_by_element_assembly_matches_oracle(ne):
    """Atomic scatter of the COO stream gives the oracle's operator (up to the
    order of the additions); add = 1 accumulates."""
    _, _, Ao = problem(ne)
    gp = GpuProblem(ne, setup=False)
    try:
        B.bamg_bsr_coo_scatter_values(gp.ctx, gp.A, gp.vals, 0)
        import scipy.sparse.linalg as spla
        ref = Ao.scalar()
        got = read_bsr(gp.ctx, gp.A).scalar()
        assert spla.norm(got - ref) <= TOL64 * spla.norm(ref)
        B.bamg_bsr_coo_scatter_values(gp.ctx, gp.A, gp.vals, 1)
        got2 = read_bsr(gp.ctx, gp.A).scalar()
        assert spla.norm(got2 - 2 * ref) <= TOL64 * spla.norm(2 * ref)
    finally:
        gp.close()


def test_hot_update_matches_oracle():
    ne = 13
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        for seed in (1, 2):
            gp.reassemble(seed)
            B.bamg_mg_update(gp.ctx, gp.mg)
            _, _, A2 = problem(ne, seed=seed)
            h2 = omg.update(h, A2)
            for l in range(h2.n_levels):
                Al, _ = B.bamg_mg_get_level(gp.mg, l)
                assert rel(read_bsr(gp.ctx, Al).vals, h2.levels[l].A.vals) <= TOL64
            b = body_force(gp.mesh)
            x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
            B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x)
            assert rel(x.cpu().numpy(), omg.vcycle(h2, b)) <= TOL64
    finally:
        gp.close()


def test_mixed_precision_cg_reaches_tolerance():
    ne = 24
    h = hierarchy(ne)
    gp = GpuProblem(ne, precision=B.BAMG_FP32)
    try:
        b = body_force(gp.mesh)
        xr, its, _ = krylov.pcg(h.levels[0].As, b, lambda r: omg.vcycle(h, r), 1e-8, 200)
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        out = B.bamg_cg_solve(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x, 1e-8, 200)
        assert out["converged"] and out["true_rnorm"] <= 1.05e-8 * np.linalg.norm(b)
        assert out["iterations"] <= its + 3
        assert rel(x.cpu().numpy(), xr) <= 1e-6
        z = torch.zeros_like(x)
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), z)
        assert rel(z.cpu().numpy(), omg.vcycle(h, b)) <= 1e-4
    finally:
        gp.close()


def test_nan_values_are_reported():
    gp = GpuProblem(4)
    try:
        gp.vals[5, 1, 1] = float("nan")
        B.bamg_bsr_coo_set_values(gp.ctx, gp.A, gp.vals, 0)
        with pytest.raises(B.BamgError) as e:
            B.bamg_ctx_sync(gp.ctx)
        assert e.value.status == 5
    finally:
        gp.close()


def test_cg_maxit_reports_not_converged():
    gp = GpuProblem(8)
    try:
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        x = torch.zeros_like(b)
        out = B.bamg_cg_solve(gp.ctx, gp.mg, b, x, 1e-12, 3, check=False)
        assert out["status"] == 7 and out["iterations"] == 3 and not out["converged"]
    finally:
        gp.close()


@pytest.mark.parametrize("br,bc", [(3, 3), (6, 6), (6, 3), (3, 6)])
def test_lane_choice_invariance(br, bc):
    """Every lanes-per-row width gives the oracle's product; the tuner picks one of them."""
    rng = np.random.default_rng(7 + br + bc)
    nbr, nbc, n = 45, 300, 6000                 # few, long rows
    bi, bj, v = random_stream(rng, nbr, nbc, br, bc, n, neg=False)
    ref = coo_assemble_blocks(nbr, nbc, br, bc, bi, bj, v)
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    A = B.bamg_bsr_create(ctx, br, bc, nbr, nbc)
    try:
        B.bamg_bsr_coo_preallocate(ctx, A, torch.from_numpy(bi).cuda(), torch.from_numpy(bj).cuda())
        B.bamg_bsr_coo_set_values(ctx, A, torch.from_numpy(v).cuda(), 0)
        x = rng.standard_normal(nbc * bc)
        yref = ref.scalar() @ x
        # -1, -2, -4: component split; -32, -64, -128: one CTA per row;
        # -(256 + VB): block split (6x3 only; 45 rows leave the second slice ragged)
        choices = (1, 2, 4, 8, 16, 32) + ((-1, -2, -4, -32, -64, -128) if br == 6 else ())
        block_split = (-258, -260, -264, -272, -288)
        if (br, bc) == (6, 3):
            choices += block_split
        for lanes in choices:
            B.bamg_bsr_set_lanes(ctx, A, lanes)
            assert B.bamg_bsr_get_lanes(A) == lanes
            y = torch.zeros(nbr * br, dtype=torch.float64, device="cuda")
            B.bamg_bsr_spmv(ctx, A, torch.from_numpy(x).cuda(), y)
            assert rel(y.cpu().numpy(), yref) <= 1e-14, lanes
            y32 = torch.zeros(nbr * br, dtype=torch.float32, device="cuda")
            B.bamg_bsr_spmv(ctx, A, torch.from_numpy(x).float().cuda(), y32, B.BAMG_FP32)
            assert rel(y32.double().cpu().numpy(), yref) <= 1e-5, lanes
        lanes, ms = B.bamg_bsr_autotune(ctx, A)
        assert lanes in choices and ms > 0
        assert B.bamg_bsr_get_lanes_prec(A, B.BAMG_FP64) == lanes
        assert B.bamg_bsr_get_lanes_prec(A, B.BAMG_FP32) in choices
        # one copy at a time: the FP32 choice moves, the FP64 one stays
        other = next(c for c in choices if c != lanes)
        B.bamg_bsr_set_lanes_prec(ctx, A, B.BAMG_FP32, other)
        assert B.bamg_bsr_get_lanes_prec(A, B.BAMG_FP32) == other and B.bamg_bsr_get_lanes(A) == lanes
        y32 = torch.zeros(nbr * br, dtype=torch.float32, device="cuda")
        B.bamg_bsr_spmv(ctx, A, torch.from_numpy(x).float().cuda(), y32, B.BAMG_FP32)
        assert rel(y32.double().cpu().numpy(), yref) <= 1e-5
        with pytest.raises(B.BamgError):
            B.bamg_bsr_set_lanes_prec(ctx, A, 2, 1)
        with pytest.raises(B.BamgError):
            B.bamg_bsr_set_lanes(ctx, A, 3)
        if (br, bc) != (6, 3):
            for code in block_split:
                with pytest.raises(B.BamgError):
                    B.bamg_bsr_set_lanes(ctx, A, code)
        if br == 3:
            with pytest.raises(B.BamgError):
                B.bamg_bsr_set_lanes(ctx, A, 0)
    finally:
        B.bamg_bsr_destroy(A)
        B.bamg_ctx_destroy(ctx)


@pytest.mark.parametrize("precision", [B.BAMG_FP64, B.BAMG_FP32])
def test_component_split_hierarchy_gives_same_cycle(precision):
    """The component-split kernels (6-row blocks: R, coarse A and P) change
    only the summation order of the cycle."""
    ne = 16
    h = hierarchy(ne)
    gp = GpuProblem(ne, precision=precision)
    try:
        b = np.random.default_rng(6).standard_normal(gp.mesh.n_dofs)
        ys = []
        for lanes in (1, 0):
            B.bamg_mg_set_lanes(gp.ctx, gp.mg, lanes)
            y = torch.zeros(b.size, dtype=torch.float64, device="cuda")
            B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), y)
            ys.append(y.cpu().numpy())
        ref = omg.vcycle(h, b)
        tol = TOL64 if precision == B.BAMG_FP64 else 1e-3
        assert rel(ys[1], ref) <= tol and rel(ys[0], ref) <= tol
        assert rel(ys[1], ys[0]) <= (1e-13 if precision == B.BAMG_FP64 else 1e-5)
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        out = B.bamg_cg_solve(gp.ctx, gp.mg, torch.from_numpy(body_force(gp.mesh)).cuda(), x, 1e-8, 200)
        assert out["converged"]
    finally:
        gp.close()


@pytest.mark.parametrize("precision,lanes", [(B.BAMG_FP64, -32), (B.BAMG_FP64, -128), (B.BAMG_FP32, -64),
                                             (B.BAMG_FP64, -258), (B.BAMG_FP64, -272), (B.BAMG_FP64, -288),
                                             (B.BAMG_FP32, -260), (B.BAMG_FP32, -288)])
def test_row_form_restriction_gives_same_cycle(precision, lanes):
    """The restriction's row form (a CTA per coarse row) and its block split
    (VB warps per slice of 6x3 rows) change only the summation order of the
    cycle.  The block split exists for 6x3 blocks only: it is set on the
    finest restriction, and 6x6 restrictions refuse it."""
    ne = 16
    h = hierarchy(ne)
    gp = GpuProblem(ne, precision=precision)
    try:
        b = np.random.default_rng(8).standard_normal(gp.mesh.n_dofs)
        B.bamg_mg_set_lanes(gp.ctx, gp.mg, 1)
        y0 = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), y0)
        for l in range(B.bamg_mg_num_levels(gp.mg) - 1):
            R = B.bamg_mg_get_restriction(gp.mg, l)
            assert R is not None
            if lanes <= -258 and l > 0:
                with pytest.raises(RuntimeError):
                    B.bamg_bsr_set_lanes(gp.ctx, R, lanes)
                continue
            B.bamg_bsr_set_lanes(gp.ctx, R, lanes)
            assert B.bamg_bsr_get_lanes(R) == lanes
        y1 = torch.zeros_like(y0)
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), y1)
        ref = omg.vcycle(h, b)
        tol = TOL64 if precision == B.BAMG_FP64 else 1e-3
        assert rel(y1.cpu().numpy(), ref) <= tol
        assert rel(y1.cpu().numpy(), y0.cpu().numpy()) <= (1e-13 if precision == B.BAMG_FP64 else 1e-5)
    finally:
        gp.close()


def test_autotuned_hierarchy_gives_same_cycle():
    """The tuned lane widths change only the summation order."""
    ne = 13
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        b = np.random.default_rng(5).standard_normal(gp.mesh.n_dofs)
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x)
        for l in range(B.bamg_mg_num_levels(gp.mg)):
            Al, Pl = B.bamg_mg_get_level(gp.mg, l)
            B.bamg_bsr_set_lanes(gp.ctx, Al, 1)
            if Pl is not None:
                B.bamg_bsr_set_lanes(gp.ctx, Pl, 32)
        x1 = torch.zeros_like(x)
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x1)
        ref = omg.vcycle(h, b)
        assert rel(x.cpu().numpy(), ref) <= TOL64 and rel(x1.cpu().numpy(), ref) <= TOL64
    finally:
        gp.close()


def test_sorted_prolongator_products_match_oracle():
    """Prolongators are stored with rows sorted by length inside each window
    of slices; every product still writes each block row in place."""
    ne = 13
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        for l in range(B.bamg_mg_num_levels(gp.mg) - 1):
            _, P = B.bamg_mg_get_level(gp.mg, l)
            Ps = h.levels[l].P.scalar()
            info = B.bamg_bsr_info(P)
            rng = np.random.default_rng(l)
            x = rng.standard_normal(Ps.shape[1])
            choices = (1, 2, 4, 8) + ((-1, -2, -4) if info["bs_r"] == 6 else ())
            for lanes in choices:
                B.bamg_bsr_set_lanes(gp.ctx, P, lanes)
                y = torch.zeros(Ps.shape[0], dtype=torch.float64, device="cuda")
                B.bamg_bsr_spmv(gp.ctx, P, torch.from_numpy(x).cuda(), y)
                assert rel(y.cpu().numpy(), Ps @ x) <= TOL64, (l, lanes)
            for k in (3, 8):
                X = rng.standard_normal((Ps.shape[1], k))
                Y = torch.zeros((Ps.shape[0], k), dtype=torch.float64, device="cuda")
                B.bamg_bsr_spmm(gp.ctx, P, torch.from_numpy(X).cuda(), Y, k, B.BAMG_FP64)
                assert rel(Y.cpu().numpy(), Ps @ X) <= TOL64, (l, k)
    finally:
        gp.close()
