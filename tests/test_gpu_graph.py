"""Block norms, strength graph and device MIS aggregation against the oracle
(Sec. 2.2, Sec. 3.2, Sec. 6), through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import strength as st
from paper_2606_24748_gb300 import bamg as B

from gpu_helpers import TOL64, GpuProblem
from oracle_cases import hierarchy, problem

pytestmark = pytest.mark.gpu


def gpu_graph(ctx, A, eps):
    info = B.bamg_bsr_info(A)
    rp = torch.empty(info["nbr"] + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(max(info["nnzb"], 1), dtype=torch.int32, device="cuda")
    ne = B.bamg_strength_graph(ctx, A, eps, rp, col)
    torch.cuda.synchronize()
    return rp.cpu().numpy().astype(np.int64), col.cpu().numpy()[:ne].astype(np.int64), rp, col


def edges(rowptr, col):
    return {(i, int(j)) for i in range(rowptr.size - 1) for j in col[rowptr[i]:rowptr[i + 1]]}


def assert_same_graph(A_oracle, eps, rp_g, col_g):
    """Equal edge sets; an edge may differ only where the oracle's own test is
    a tie to 1e-10 (the GPU's values differ from the oracle's in the last bits)."""
    rp_o, col_o = st.strength_graph(A_oracle, eps)
    diff = edges(rp_o, col_o) ^ edges(rp_g, col_g)
    if diff:
        s = st.block_sumsq(A_oracle)
        br = A_oracle.block_rows()
        d = {int(i): s[k] for k, i in enumerate(br) if A_oracle.colidx[k] == i}
        for (i, j) in diff:
            k = A_oracle.find(i, j)
            lhs = s[k] * s[k]
            rhs = (eps ** 4) * d[i] * d[j]
            assert abs(lhs - rhs) <= 1e-10 * max(rhs, 1e-300), (i, j, lhs, rhs)
    for i in range(rp_g.size - 1):   # ascending columns
        assert np.all(np.diff(col_g[rp_g[i]:rp_g[i + 1]]) > 0)
    return rp_o, col_o, not diff


@pytest.mark.parametrize("ne", [6, 12])
def test_block_norms_and_matrix_norms_match_oracle(ne):
    mesh, _, Ao = problem(ne)
    gp = GpuProblem(ne, setup=False)
    try:
        info = B.bamg_bsr_info(gp.A)
        out = torch.empty(info["nnzb"], dtype=torch.float64, device="cuda")
        B.bamg_bsr_block_norms(gp.ctx, gp.A, out)
        rp = torch.empty(info["nbr"] + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(info["nnzb"], dtype=torch.int32, device="cuda")
        B.bamg_bsr_get_pattern(gp.ctx, gp.A, rp, ci)
        rp, ci, out = rp.cpu().numpy(), ci.cpu().numpy(), out.cpu().numpy()
        so = np.sqrt(st.block_sumsq(Ao))
        got = {(i, int(ci[k])): out[k] for i in range(info["nbr"]) for k in range(rp[i], rp[i + 1])}
        want = {(i, int(Ao.colidx[k])): so[k] for i in range(Ao.nbr) for k in range(Ao.rowptr[i], Ao.rowptr[i + 1])}
        for key, v in got.items():   # blocks the oracle's scalar form dropped are zero
            assert abs(v - want.get(key, 0.0)) <= 1e-14 * max(1.0, abs(v)), key
        assert B.bamg_bsr_norm(gp.ctx, gp.A, B.BAMG_NORM_FROBENIUS) == pytest.approx(st.frobenius_norm(Ao), rel=TOL64)
        assert B.bamg_bsr_norm(gp.ctx, gp.A, B.BAMG_NORM_INFINITY) == pytest.approx(st.inf_norm(Ao), rel=TOL64)
    finally:
        gp.close()


@pytest.mark.parametrize("ne,eps", [(6, 0.0), (12, 0.01), (12, 0.08)])
def test_strength_graph_matches_oracle(ne, eps):
    _, _, Ao = problem(ne)
    gp = GpuProblem(ne, setup=False)
    try:
        rp, col, _, _ = gpu_graph(gp.ctx, gp.A, eps)
        assert_same_graph(Ao, eps, rp, col)
    finally:
        gp.close()


def upload_graph(rowptr, col):
    return (torch.from_numpy(rowptr.astype(np.int32)).cuda(),
            torch.from_numpy(np.asarray(col, dtype=np.int32) if col.size else np.zeros(1, np.int32)).cuda())


@pytest.mark.parametrize("ne,eps,seed", [(6, 0.01, 1), (12, 0.01, 7), (12, 0.08, 3)])
def test_mis_aggregates_match_oracle_bit_for_bit(ne, eps, seed):
    _, _, Ao = problem(ne)
    rp_o, col_o = st.strength_graph(Ao, eps)
    w = st.weights(Ao.nbr, seed)
    mis = st.mis_greedy(rp_o, col_o, w)
    _, rounds = st.mis_luby(rp_o, col_o, w)
    agg_o = st.mis_aggregates(rp_o, col_o, w, mis)
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    try:
        rp, col = upload_graph(rp_o, col_o)
        agg = torch.empty(Ao.nbr, dtype=torch.int32, device="cuda")
        n_agg, r = B.bamg_mis_aggregate(ctx, Ao.nbr, rp, col, seed, agg)
        assert n_agg == int(mis.sum()) and r == rounds
        assert np.array_equal(agg.cpu().numpy(), agg_o)
    finally:
        B.bamg_ctx_destroy(ctx)


def test_device_graph_to_aggregates_end_to_end_on_a_coarse_level():
    """6x6 blocks: level 1 of the hierarchy, graph and aggregates on the device."""
    ne, eps, seed = 16, 0.01, 5
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        A1, _ = B.bamg_mg_get_level(gp.mg, 1)
        rp, col, rp_d, col_d = gpu_graph(gp.ctx, A1, eps)
        rp_o, col_o, same = assert_same_graph(h.levels[1].A, eps, rp, col)
        n = rp.size - 1
        agg = torch.empty(n, dtype=torch.int32, device="cuda")
        n_agg, _ = B.bamg_mis_aggregate(gp.ctx, n, rp_d, col_d, seed, agg)
        agg = agg.cpu().numpy()
        # every vertex in one of aggregates 0 .. n_agg - 1, each aggregate a star of the graph
        assert agg.min() == 0 and agg.max() == n_agg - 1 and np.bincount(agg).min() >= 1
        E = edges(rp, col)
        for a in range(n_agg):
            members = np.flatnonzero(agg == a)
            assert any(all(m == c or (c, int(m)) in E for m in members) for c in members), a
        if same:   # the usual case: the oracle's graph, MIS and aggregates exactly
            w = st.weights(n, seed)
            mis_o = st.mis_greedy(rp_o, col_o, w)
            assert np.array_equal(agg, st.mis_aggregates(rp_o, col_o, w, mis_o))
    finally:
        gp.close()


def test_graph_errors_are_reported():
    gp = GpuProblem(4, setup=False)
    try:
        info = B.bamg_bsr_info(gp.A)
        rp = torch.empty(info["nbr"] + 1, dtype=torch.int32, device="cuda")
        small = torch.empty(3, dtype=torch.int32, device="cuda")
        with pytest.raises(B.BamgError):
            B.bamg_strength_graph(gp.ctx, gp.A, -1.0, rp, small)
        with pytest.raises(B.BamgError):
            B.bamg_strength_graph(gp.ctx, gp.A, 0.0, rp, small)
    finally:
        gp.close()
