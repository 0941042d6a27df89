"""The row-sharded operator on the GPU (Sec. 3.3, Sec. 3.5): every part of a
partition runs in turn on the one device, and the sharded SpMV and Galerkin
product must equal the oracle's (patterns bit-exact, FP64 values to 1e-12
normwise); P_oth is gathered once per version of P."""
import numpy as np
import pytest
import torch

from oracle.galerkin import galerkin
from paper_2606_24748_gb300 import bamg as B

from gpu_helpers import TOL64, GpuProblem, read_bsr, rel, same_pattern
from oracle_cases import hierarchy

pytestmark = pytest.mark.gpu


def starts_for(n, nparts):
    return np.array([round(k * n / nparts) for k in range(nparts + 1)], dtype=np.int64)


@pytest.mark.parametrize("ne,level,nparts", [(8, 0, 1), (8, 0, 2), (13, 0, 3), (16, 0, 5), (24, 1, 4)])
def test_sharded_spmv_and_galerkin_match_oracle(ne, level, nparts):
    gp = GpuProblem(ne)
    sh = Ac = None
    try:
        h = hierarchy(ne)
        A, P = B.bamg_mg_get_level(gp.mg, level)
        Ao, Po = h.levels[level].A, h.levels[level].P
        sh, Ac = B.bamg_sharded_create(gp.ctx, A, P, starts_for(Ao.nbr, nparts))
        rng = np.random.default_rng(ne + nparts)
        x = rng.standard_normal(Ao.nbr * Ao.bs_r)
        y = torch.zeros_like(torch.from_numpy(x)).cuda()
        B.bamg_sharded_spmv(gp.ctx, sh, torch.from_numpy(x).cuda(), y)
        assert rel(y.cpu().numpy(), Ao.scalar() @ x) <= 1e-14
        B.bamg_sharded_ptap(gp.ctx, sh, A, P, Ac)
        got, ref = read_bsr(gp.ctx, Ac), galerkin(Ao, Po)
        assert same_pattern(got, ref)
        assert rel(got.vals, ref.vals) <= TOL64
        st = B.bamg_sharded_stats(sh)
        assert st["poth_gathers"] == 1
        if nparts == 1:
            assert st["ghost_rows"] == st["poth_blocks"] == st["reduce_blocks"] == 0
        else:
            assert st["halo_bytes_per_spmv"] == st["ghost_rows"] * Ao.bs_r * 8 > 0
    finally:
        if sh is not None:
            B.bamg_sharded_destroy(sh)
            B.bamg_bsr_destroy(Ac)
        gp.close()


def test_sharded_state_gate_and_reuse():
    """A new operator (hot reuse) needs no new P_oth; a re-smoothed P does."""
    ne, nparts = 13, 3
    gp = GpuProblem(ne)
    sh = Ac = None
    try:
        A, P = B.bamg_mg_get_level(gp.mg, 0)
        n = B.bamg_bsr_info(A)["nbr"]
        sh, Ac = B.bamg_sharded_create(gp.ctx, A, P, starts_for(n, nparts))
        B.bamg_sharded_ptap(gp.ctx, sh, A, P, Ac)
        gp.reassemble(7)                           # hot reuse: A changes, P stays
        B.bamg_sharded_ptap(gp.ctx, sh, A, P, Ac)
        assert B.bamg_sharded_stats(sh)["poth_gathers"] == 1
        a = read_bsr(gp.ctx, A)
        p = read_bsr(gp.ctx, P)
        assert rel(read_bsr(gp.ctx, Ac).vals, galerkin(a, p).vals) <= TOL64
        B.bamg_mg_resetup(gp.ctx, gp.mg)           # P re-smoothed for the new A: new version
        B.bamg_sharded_ptap(gp.ctx, sh, A, P, Ac)
        assert B.bamg_sharded_stats(sh)["poth_gathers"] == 2
        p2 = read_bsr(gp.ctx, P)
        assert rel(p2.vals, p.vals) > 1e-8
        got = read_bsr(gp.ctx, Ac)
        assert rel(got.vals, galerkin(a, p2).vals) <= TOL64
        # and equals the hierarchy's own (unsharded) product of the same level
        assert rel(got.vals, read_bsr(gp.ctx, B.bamg_mg_get_level(gp.mg, 1)[0]).vals) <= TOL64
        with pytest.raises(B.BamgError):            # a matrix it was not built for
            B.bamg_sharded_ptap(gp.ctx, sh, A, P, B.bamg_mg_get_level(gp.mg, 1)[0])
    finally:
        if sh is not None:
            B.bamg_sharded_destroy(sh)
            B.bamg_bsr_destroy(Ac)
        gp.close()


def test_sharded_full_size_equals_unsharded():
    """64^3 elements, four parts: the sharded products against the library's
    unsharded ones on the same operators (the oracle checks the latter at
    this size through sampled rows and identities, test_gpu_fullsize.py)."""
    gp = GpuProblem(64)
    sh = Ac = None
    try:
        A, P = B.bamg_mg_get_level(gp.mg, 0)
        n = B.bamg_bsr_info(A)["nbr"]
        sh, Ac = B.bamg_sharded_create(gp.ctx, A, P, starts_for(n, 4))
        x = torch.randn(n * 3, dtype=torch.float64, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
        y1, y2 = torch.empty_like(x), torch.empty_like(x)
        B.bamg_sharded_spmv(gp.ctx, sh, x, y1)
        B.bamg_bsr_spmv(gp.ctx, A, x, y2)
        assert float(torch.linalg.norm(y1 - y2) / torch.linalg.norm(y2)) <= 1e-14
        B.bamg_mg_update(gp.ctx, gp.mg)
        B.bamg_sharded_ptap(gp.ctx, sh, A, P, Ac)
        got, ref = read_bsr(gp.ctx, Ac), read_bsr(gp.ctx, B.bamg_mg_get_level(gp.mg, 1)[0])
        assert same_pattern(got, ref)
        assert rel(got.vals, ref.vals) <= TOL64
    finally:
        if sh is not None:
            B.bamg_sharded_destroy(sh)
            B.bamg_bsr_destroy(Ac)
        gp.close()
