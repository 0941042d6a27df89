"""The MIS-driven hierarchy on the GPU (Sec. 3.2, Sec. 6 feeding Sec. 2.2)
against the oracle: aggregates bit-exact on every level (including the rows
left out, -1), prolongator and coarse-operator patterns bit-exact, FP64 values
to 1e-12, and PCG iterations within one of the oracle's."""
import numpy as np
import pytest
import torch

from oracle import krylov, multigrid as omg
from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import body_force

from gpu_helpers import TOL64, GpuProblem, read_bsr, rel, same_pattern
from oracle_cases import hierarchy

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ne,seed", [(8, 1), (13, 1), (16, 5)])
def test_mis_hierarchy_matches_oracle(ne, seed):
    h = hierarchy(ne, aggregation="mis", seed=seed)
    gp = GpuProblem(ne, aggregation=B.BAMG_AGG_MIS, mis_seed=seed)
    try:
        assert B.bamg_mg_num_levels(gp.mg) == h.n_levels
        for l, L in enumerate(h.levels):
            A, P = B.bamg_mg_get_level(gp.mg, l)
            a = read_bsr(gp.ctx, A)
            assert same_pattern(a, L.A), l
            assert rel(a.vals, L.A.vals) <= TOL64, l
            if L.P is None:
                continue
            agg = torch.empty(L.A.nbr, dtype=torch.int32, device="cuda")
            B.bamg_mg_get_aggregates(gp.ctx, gp.mg, l, agg)
            assert np.array_equal(agg.cpu().numpy(), L.agg), l
            p = read_bsr(gp.ctx, P)
            assert same_pattern(p, L.P), l
            assert rel(p.vals, L.P.vals) <= TOL64, l
        b = body_force(gp.mesh)
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        out = B.bamg_cg_solve(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x, 1e-8, 200)
        xr, its, info = krylov.pcg(h.levels[0].As, b, lambda r: omg.vcycle(h, r), 1e-8, 200)
        assert out["converged"] and abs(out["iterations"] - its) <= 1
        assert rel(x.cpu().numpy(), xr) <= 1e-7
    finally:
        gp.close()


def test_mis_hierarchy_reuse_step_and_options():
    """The hot reuse step on an MIS hierarchy (same aggregates and P, new
    operator) and the option checks."""
    ne = 13
    gp = GpuProblem(ne, aggregation=B.BAMG_AGG_MIS)
    try:
        gp.reassemble(9)
        B.bamg_mg_update(gp.ctx, gp.mg)
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        x = torch.zeros_like(b)
        out = B.bamg_cg_solve(gp.ctx, gp.mg, b, x, 1e-8, 200)
        assert out["converged"] and out["true_rnorm"] <= 1.05e-8 * out["bnorm"]
        o = B.bamg_mg_opts_default()
        assert o.aggregation == B.BAMG_AGG_GEOMETRIC and o.mis_eps == pytest.approx(0.02) and o.mis_seed == 1
        o.aggregation = 7
        with pytest.raises(B.BamgError):
            B.bamg_mg_setup(gp.ctx, gp.A, gp.mesh.coords(), gp.mesh.dirichlet(), o)
    finally:
        gp.close()
