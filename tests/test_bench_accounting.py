"""The bench books as many V-cycles per solve as PCG applies (host logic)."""
import numpy as np

import bench
from oracle import krylov
from oracle import multigrid as omg

from oracle_cases import hierarchy


def test_pcg_applies_the_preconditioner_once_per_iteration():
    h = hierarchy(8)
    As = h.levels[0].As
    b = np.random.default_rng(5).standard_normal(As.shape[0])
    calls = []

    def M(r):
        calls.append(1)
        return omg.vcycle(h, r)

    _, its, info = krylov.pcg(As, b, M, 1e-8, 100)
    assert info["converged"] and its > 3
    assert len(calls) == bench.vcycles_per_solve(its) == its


def test_step_bytes_count_one_vcycle_per_iteration():
    lv = bench.oracle_levels(hierarchy(8))
    t20, p20, vc = bench.step_bytes(lv, 1000, 20, False)
    t21, p21, _ = bench.step_bytes(lv, 1000, 21, False)
    assert p20["vcycles"] == 20 * vc
    assert t21 - t20 == vc + (p21["cg"] - p20["cg"])
