"""Pins of the MIS-driven hierarchy of the oracle (Sec. 3.2, Sec. 6 aggregates
feeding Sec. 2.2 smoothed aggregation), against properties the method fixes:
the aggregation rules, exact reproduction of the near-null space by the
tentative prolongator, the Galerkin identity, SPD coarse operators, the
two-level cycle as the dense error operator, and PCG convergence."""
import numpy as np
import pytest

from oracle import krylov, multigrid as omg, strength as S
from oracle.prolongator import rigid_body_modes, tentative_prolongator

from oracle_cases import hierarchy, problem
from test_pins_multigrid import dense_two_level_error, stationary_reference


def fine_near_null(mesh):
    coords, dirc = mesh.coords(), mesh.dirichlet()
    return lambda m: rigid_body_modes(coords[m], np.zeros(len(m), dtype=np.int64), 1, dirc[m]).reshape(-1, 6)


@pytest.mark.parametrize("ne", [8, 12])
def test_aggregation_rules(ne):
    mesh, _, A = problem(ne)
    eps, seed = 0.08, 3
    nn = fine_near_null(mesh)
    agg, n_agg = S.hierarchy_aggregates(A, eps, seed, nn)
    rp, col = S.strength_graph(A, eps)
    w = S.weights(A.nbr, seed)
    in_set = S.mis_greedy(rp, col, w)
    agg0 = S.mis_aggregates(rp, col, w, in_set)
    roots = np.flatnonzero(in_set)
    deg = np.diff(rp)
    # isolated vertices (the clamped face) join nothing; they are exactly the clamped nodes here
    assert np.array_equal(deg == 0, mesh.dirichlet().astype(bool))
    assert np.all(agg[deg == 0] == -1)
    # aggregates are numbered 0..n_agg-1, all used, every one of full rank
    assert set(agg[agg >= 0]) == set(range(n_agg))
    for a in range(n_agg):
        m = np.flatnonzero(agg == a)
        Bm = nn(m)
        assert np.linalg.matrix_rank(Bm) == 6
    # survivors are the full-rank original aggregates, in root order, with their members kept
    survivors = [a for a in range(roots.size) if deg[roots[a]] > 0 and np.linalg.matrix_rank(nn(np.flatnonzero(agg0 == a))) == 6]
    assert len(survivors) == n_agg
    assert len(survivors) < roots.size - int((deg == 0).sum())      # some aggregates were dissolved
    for new, old in enumerate(survivors):
        assert np.all(agg[agg0 == old] == new)
    # a vertex of a dissolved aggregate joins its strong neighbour's aggregate of largest root key
    key = lambda a: (int(w[roots[a]]), int(roots[a]))  # noqa: E731
    surv = set(survivors)
    for v in np.flatnonzero((agg0 >= 0) & (deg > 0)):
        if agg0[v] in surv:
            continue
        cands = {agg0[j] for j in col[rp[v]:rp[v + 1]] if agg0[j] in surv}
        if not cands:
            assert agg[v] == -1
        else:
            assert agg[v] == survivors.index(max(cands, key=key))


def test_tentative_prolongator_reproduces_the_near_null_space():
    mesh, _, A = problem(8)
    agg, n_agg = S.hierarchy_aggregates(A, 0.08, 1, fine_near_null(mesh))
    B = rigid_body_modes(mesh.coords(), agg, n_agg, mesh.dirichlet())
    Pt, Bc = tentative_prolongator(B, agg, n_agg)
    Pd = Pt.dense()
    assert np.allclose(Pd.T @ Pd, np.eye(6 * n_agg), atol=1e-12)      # orthonormal columns per aggregate
    Bd = np.zeros((A.nbr * 3, n_agg * 6))
    Bcd = np.zeros((n_agg * 6, 6 * n_agg))
    for a in range(n_agg):
        Bcd[6 * a:6 * a + 6, 6 * a:6 * a + 6] = Bc[a]
    for v in range(A.nbr):
        if agg[v] >= 0:
            Bd[3 * v:3 * v + 3, 6 * agg[v]:6 * agg[v] + 6] = B[v]
    assert np.allclose(Pd @ Bcd, Bd, atol=1e-12)                         # P~ B_c = B
    assert np.all(np.abs(Pd[np.repeat(agg < 0, 3)]) == 0)               # rows outside every aggregate


@pytest.mark.parametrize("ne", [8, 16])
def test_mis_hierarchy_galerkin_identity_and_spd(ne):
    h = hierarchy(ne, aggregation="mis")
    rng = np.random.default_rng(ne)
    for l in range(h.n_levels - 1):
        L, C = h.levels[l], h.levels[l + 1]
        xc, yc = rng.standard_normal((2, C.A.nbr * 6))
        Ps = L.P.scalar()
        lhs = xc @ (C.A.scalar() @ yc)
        rhs = (Ps @ xc) @ (L.A.scalar() @ (Ps @ yc))
        assert abs(lhs - rhs) <= 1e-12 * np.sqrt(abs(xc @ (C.A.scalar() @ xc)) * abs(yc @ (C.A.scalar() @ yc)))
        Ac = C.A.dense()
        assert np.allclose(Ac, Ac.T, atol=1e-13 * np.abs(Ac).max())
        np.linalg.cholesky(Ac)


def test_mis_two_level_cycle_is_the_dense_error_operator_and_cg_converges():
    h = hierarchy(8, aggregation="mis")
    assert h.n_levels == 2
    Ad, E = dense_two_level_error(h)
    b = np.random.default_rng(4).standard_normal(Ad.shape[0])
    ref = (np.eye(Ad.shape[0]) - E) @ np.linalg.solve(Ad, b)
    assert np.linalg.norm(omg.vcycle(h, b) - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.allclose(omg.stationary(h, b, 4), stationary_reference(Ad, E, b, 4), rtol=1e-9)
    x, its, info = krylov.pcg(h.levels[0].As, b, lambda r: omg.vcycle(h, r), 1e-8, 100)
    assert info["converged"] and its < 25
