"""Q2 elements (27-node hexahedra, up to 125 blocks per row): the whole
reuse path against the oracle (the paper's nonzeros-per-row study, Sec. 4.6)."""
import numpy as np
import pytest
import torch

from oracle import krylov
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
