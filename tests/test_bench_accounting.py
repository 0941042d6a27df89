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


class _FakeLanes:
    """Stand-in for the binding's hierarchy accessors and per-copy lanes."""
    BAMG_FP64, BAMG_FP32 = 0, 1

    def __init__(self, levels):
        self.levels = levels       # list of (A, P, R) names, P and R None on the coarsest
        self.lanes = {}

    def bamg_mg_num_levels(self, mg):
        return len(self.levels)

    def bamg_mg_get_level(self, mg, l):
        return self.levels[l][0], self.levels[l][1]

    def bamg_mg_get_restriction(self, mg, l):
        return self.levels[l][2]

    def bamg_bsr_get_lanes_prec(self, M, p):
        return self.lanes.get((M, p), 1)

    def bamg_bsr_set_lanes_prec(self, ctx, M, p, v):
        self.lanes[(M, p)] = v


def test_tune_cache_keeps_both_copies(tmp_path):
    """The tune cache saves every level matrix's FP64 and FP32 lanes and puts
    them back, copy by copy."""
    levels = [("A0", "P0", "R0"), ("A1", "P1", "R1"), ("A2", None, None)]
    src = _FakeLanes(levels)
    src.lanes = {("R0", 0): -4, ("R0", 1): -288, ("A1", 0): 16, ("A1", 1): -4, ("P0", 0): 2}
    path = str(tmp_path / "tune.json")
    bench.apply_tune_cache(src, None, None, path)          # no file yet: saves
    dst = _FakeLanes(levels)
    bench.apply_tune_cache(dst, None, None, path)          # file present: restores
    for M in ("A0", "P0", "R0", "A1", "P1", "R1", "A2"):
        for p in (0, 1):
            assert dst.lanes[(M, p)] == src.bamg_bsr_get_lanes_prec(M, p)
    assert dst.lanes[("R0", 1)] == -288 and dst.lanes[("R0", 0)] == -4


class _FakeWorkload:
    def __init__(self, mixed):
        import types
        self.mixed = mixed
        self.mesh = types.SimpleNamespace(ne=64)
        self.levels = [{"A": {"nbr": 274625, "nnzb": 7189057}, "P": None}, {"A": {"nbr": 9261, "nnzb": 226981}}]


def test_roofline_takes_the_sampled_slot_and_the_form_s_traffic():
    """The roofline times the sampled pre-smoothing pair when that slot ran,
    books the mean bytes of those two steps, and reports the DRAM traffic
    recorded for the same form."""
    from paper_2606_24748_gb300 import bytes_model as bm
    nnzb, n = 7189057, 274625
    alu = {"fp64_peak_tflops": bench.FP64_PEAK_DERIVED_TFLOPS, "fp64_probe_tflops": None}
    for mixed in (False, True):
        prof = {k: (0.0, 0) for k in ("cheb_step_l0", "ptap_stage1_l0", "ptap_stage2_l0", "cg_ap")}
        prof["cheb_pre_l0"] = (46 * 0.1, 46)
        r = bench.roofline(_FakeWorkload(mixed), prof, None, alu)
        s = 4 if mixed else 8
        want = (bm.cheb_step_bytes(nnzb, n, 3, s, True) + bm.cheb_step_bytes(nnzb, n, 3, s, False)) / 2
        assert r["kernel"] == "cheb_step_l0" and r["launches"] == 46
        assert r["bytes_per_launch"] == int(want)
        assert r["traffic"] == int(bench.TRAFFIC[("cheb_step_l0", 64, mixed)][0])
        assert r["bound"] == ("hbm" if mixed else "alu")
