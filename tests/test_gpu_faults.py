"""Failure reporting and the state gate, through the C ABI.

Every failure here is made on the host: an indefinite operator (negated
element values) and a bounded device wait told to give up at once.  No kernel
faults, traps or waits without a limit; after each failure the same context
solves a valid problem again.  The state gate (Sec. 3.5): the prolongator-side
caches (block-ordered P inside the Galerkin plan, R = P^T) are rebuilt when
P's version changes and never otherwise."""
import numpy as np
import pytest
import torch

from oracle import krylov, multigrid as omg
from oracle.assembly import coo_assemble_blocks
from oracle.galerkin import galerkin
from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import body_force

from gpu_helpers import TOL64, GpuProblem, read_bsr, rel
from oracle_cases import hierarchy

pytestmark = pytest.mark.gpu
DEFAULT_WAIT = 1 << 22


def solves_cleanly(gp, b):
    x = torch.zeros_like(b)
    out = B.bamg_cg_solve(gp.ctx, gp.mg, b, x, 1e-8, 200)
    assert out["converged"] and out["true_rnorm"] <= 1.05e-8 * out["bnorm"]
    return x


def test_indefinite_operator_reports_breakdown_in_cg():
    """CG on -A with the hierarchy of A: p^T (-A) p < 0 at the first
    iteration, as in the oracle, which stops there too."""
    gp = GpuProblem(8)
    try:
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        B.bamg_bsr_coo_set_values(gp.ctx, gp.A, -gp.vals, 0)
        x = torch.zeros_like(b)
        out = B.bamg_cg_solve(gp.ctx, gp.mg, b, x, 1e-8, 100, check=False)
        assert out["status"] == B.BAMG_ERR_BREAKDOWN and not out["converged"]
        h = hierarchy(8)
        As = h.levels[0].As
        bh = body_force(gp.mesh)
        _, its, info = krylov.pcg(-As, bh, lambda r: omg.vcycle(h, r), 1e-8, 100)
        assert not info["converged"] and its == out["iterations"] == 0
        # the context is usable again once the operator is valid
        B.bamg_bsr_coo_set_values(gp.ctx, gp.A, gp.vals, 0)
        B.bamg_ctx_sync(gp.ctx)
        solves_cleanly(gp, b)
    finally:
        gp.close()


def test_indefinite_operator_reports_breakdown_in_update():
    """Refreshing the smoother of -A: its diagonal blocks are negative
    definite, so the block Cholesky of point-block Jacobi fails."""
    gp = GpuProblem(8)
    try:
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        B.bamg_bsr_coo_set_values(gp.ctx, gp.A, -gp.vals, 0)
        with pytest.raises(B.BamgError) as e:
            B.bamg_mg_update(gp.ctx, gp.mg)
            B.bamg_ctx_sync(gp.ctx)
        assert e.value.status == B.BAMG_ERR_BREAKDOWN
        try:                      # clear anything a later kernel of the update recorded
            B.bamg_ctx_sync(gp.ctx)
        except B.BamgError:
            pass
        B.bamg_bsr_coo_set_values(gp.ctx, gp.A, gp.vals, 0)
        B.bamg_mg_update(gp.ctx, gp.mg)
        B.bamg_ctx_sync(gp.ctx)
        solves_cleanly(gp, b)
    finally:
        gp.close()


def test_exhausted_device_wait_reports_timeout_and_context_recovers():
    """With a wait limit of zero polls the coarsest factorisation's bounded
    wait gives up at once: the kernel records BAMG_ERR_TIMEOUT and returns
    (every CTA still meets the grid barriers); the host reads the status,
    restores the limit, and the same hierarchy solves again."""
    gp = GpuProblem(16)        # 750 coarsest dofs: several 32-wide tile columns, one wait each
    try:
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        x_ref = solves_cleanly(gp, b)
        with pytest.raises(B.BamgError):
            B.bamg_ctx_set_wait_limit(gp.ctx, -1)
        B.bamg_ctx_set_wait_limit(gp.ctx, 0)
        try:
            B.bamg_mg_update(gp.ctx, gp.mg)
            with pytest.raises(B.BamgError) as e:
                B.bamg_ctx_sync(gp.ctx)
            assert e.value.status == B.BAMG_ERR_TIMEOUT
        finally:
            B.bamg_ctx_set_wait_limit(gp.ctx, DEFAULT_WAIT)
        B.bamg_ctx_sync(gp.ctx)            # the error word was cleared by the read above
        B.bamg_mg_update(gp.ctx, gp.mg)
        B.bamg_ctx_sync(gp.ctx)
        x = solves_cleanly(gp, b)
        assert rel(x.cpu().numpy(), x_ref.cpu().numpy()) <= 1e-12
    finally:
        gp.close()


def test_hierarchy_state_gate_rebuilds_only_when_p_changes():
    gp = GpuProblem(16)
    try:
        nl = B.bamg_mg_num_levels(gp.mg)
        assert nl >= 2
        before = [B.bamg_mg_get_gate_counts(gp.mg, l) for l in range(nl - 1)]
        r_versions = [B.bamg_bsr_info(B.bamg_mg_get_restriction(gp.mg, l))["version"] for l in range(nl - 1)]
        for seed in (3, 4):                      # hot updates: P fixed, nothing rebuilt
            gp.reassemble(seed)
            B.bamg_mg_update(gp.ctx, gp.mg)
        B.bamg_ctx_sync(gp.ctx)
        assert [B.bamg_mg_get_gate_counts(gp.mg, l) for l in range(nl - 1)] == before
        assert [B.bamg_bsr_info(B.bamg_mg_get_restriction(gp.mg, l))["version"] for l in range(nl - 1)] == r_versions
        B.bamg_mg_resetup(gp.ctx, gp.mg)         # P re-smoothed: new version, one rebuild of each cache
        B.bamg_ctx_sync(gp.ctx)
        after = [B.bamg_mg_get_gate_counts(gp.mg, l) for l in range(nl - 1)]
        assert after == [(p + 1, r + 1) for p, r in before]
        # the rebuilt caches give the oracle's hierarchy for the new operator
        h = omg.setup(read_bsr(gp.ctx, gp.A), gp.mesh.coords(), gp.mesh.dirichlet(), gp.mesh.grid)
        A1 = read_bsr(gp.ctx, B.bamg_mg_get_level(gp.mg, 1)[0])
        assert rel(A1.vals, h.levels[1].A.vals) <= TOL64
    finally:
        gp.close()


def test_plan_state_gate_counts_p_versions():
    rng = np.random.default_rng(31)
    n, nc, bs, bsp = 120, 30, 3, 6
    bi = rng.integers(0, n, 1200).astype(np.int32)
    bj = rng.integers(0, n, 1200).astype(np.int32)
    v = rng.standard_normal((1200, bs, bs))
    pi = rng.integers(0, n, 300).astype(np.int32)
    pj = rng.integers(0, nc, 300).astype(np.int32)
    pv = rng.standard_normal((300, bs, bsp))
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
        assert B.bamg_ptap_get_refreshes(plan) == 0
        B.bamg_ptap_numeric(ctx, plan, A, P, Ac)
        B.bamg_ptap_numeric(ctx, plan, A, P, Ac)
        assert B.bamg_ptap_get_refreshes(plan) == 1          # one P version: one rebuild
        v2 = v * rng.uniform(0.5, 1.5, (1200, 1, 1))
        B.bamg_bsr_coo_set_values(ctx, A, torch.from_numpy(v2).cuda(), 0)
        B.bamg_ptap_numeric(ctx, plan, A, P, Ac)
        assert B.bamg_ptap_get_refreshes(plan) == 1          # A changed, P did not
        pv2 = pv * rng.uniform(0.5, 1.5, (300, 1, 1))
        B.bamg_bsr_coo_set_values(ctx, P, torch.from_numpy(pv2).cuda(), 0)
        B.bamg_ptap_numeric(ctx, plan, A, P, Ac)
        assert B.bamg_ptap_get_refreshes(plan) == 2          # new P version: rebuilt
        ref = galerkin(coo_assemble_blocks(n, n, bs, bs, bi, bj, v2), coo_assemble_blocks(n, nc, bs, bsp, pi, pj, pv2))
        assert rel(read_bsr(ctx, Ac).vals, ref.vals) <= TOL64
    finally:
        if plan is not None:
            B.bamg_ptap_destroy(plan)
            B.bamg_bsr_destroy(Ac)
        B.bamg_bsr_destroy(P)
        B.bamg_bsr_destroy(A)
        B.bamg_ctx_destroy(ctx)
