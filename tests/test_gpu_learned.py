"""GPU parity of the learned-smoother kernels against the oracle (features,
MLP forward, gradients, Adam, targets, weighted V-cycle, stationary
iteration) and a short training run."""
import copy

import numpy as np
import pytest
import torch

from oracle import learned as OL
from oracle import multigrid as omg
from paper_2606_24748_gb300 import bamg as B
from workloads.elasticity import body_force

from gpu_helpers import TOL64, GpuProblem, rel
from oracle_cases import hierarchy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.lib()
    c = B.bamg_ctx_create(torch.cuda.current_stream())
    yield c
    B.bamg_ctx_destroy(c)


def test_block_features_match_oracle():
    ne = 24
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        for l in range(h.n_levels - 1):
            L = h.levels[l]
            X = torch.empty((L.A.nbr, 8), dtype=torch.float32, device="cuda")
            B.bamg_mg_block_features(gp.ctx, gp.mg, l, X)
            ref = OL.block_features(L.A, l, L.Dinv)
            got = X.cpu().numpy()
            assert np.allclose(got, ref, rtol=1e-5, atol=1e-6), l
    finally:
        gp.close()


@pytest.mark.parametrize("N", [3000, 100003])
def test_mlp_forward_gradient_and_adam_match_oracle(ctx, N):
    """Tensor-core forward and fused backward (BF16 operands, FP32
    accumulation) against the oracle's BF16-emulating MLP; 3,000 rows fill a
    dozen CTAs with a ragged last chunk, 100,003 rows every CTA slot."""
    n = B.bamg_mlp_num_params()
    assert n == OL.N_PARAMS
    mlp = B.bamg_mlp_create(ctx, 7)
    try:
        rng = np.random.default_rng(3)
        theta = (rng.standard_normal(n) * 0.3).astype(np.float32)
        B.bamg_mlp_set_params(ctx, mlp, torch.from_numpy(theta).cuda())
        X = rng.standard_normal((N, 8)).astype(np.float32)
        t = rng.uniform(0.5, 2.0, N).astype(np.float32)
        Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
        w = torch.empty(N, dtype=torch.float32, device="cuda")
        B.bamg_mlp_forward(ctx, mlp, Xd, w)
        wref, _ = OL.forward(theta.astype(np.float64), X, True)
        assert np.abs(w.cpu().numpy() - wref).max() < 2e-2
        assert rel(w.cpu().numpy(), wref) < 1e-3
        g = torch.empty(n, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        B.bamg_mlp_gradient(ctx, mlp, Xd, td, w, g, loss)
        lref, gref = OL.loss_and_grad(theta.astype(np.float64), X, t, True)
        assert float(loss.item()) == pytest.approx(lref, rel=1e-3)
        assert rel(g.cpu().numpy(), gref) < 2e-2
        # one Adam step equals the oracle's Adam on the same gradient
        B.bamg_mlp_train_step(ctx, mlp, Xd, td, w, 1e-3, loss)
        p1 = torch.empty(n, dtype=torch.float32, device="cuda")
        B.bamg_mlp_get_params(ctx, mlp, p1)
        opt = OL.Adam(n, lr=1e-3)
        ref1 = opt.step(theta.astype(np.float64), g.cpu().numpy().astype(np.float64))
        assert rel(p1.cpu().numpy(), ref1) < 1e-6
        # deterministic: the same gradient twice
        g2 = torch.empty_like(g)
        B.bamg_mlp_set_params(ctx, mlp, torch.from_numpy(theta).cuda())
        B.bamg_mlp_gradient(ctx, mlp, Xd, td, w, g2, None)
        assert torch.equal(g, g2)
    finally:
        B.bamg_mlp_destroy(mlp)


def test_smoother_targets_match_oracle():
    ne = 13
    h = hierarchy(ne)
    gp = GpuProblem(ne)
    try:
        rng = np.random.default_rng(4)
        Bk = rng.standard_normal((3, gp.mesh.n_dofs))
        n = sum(L.A.nbr for L in h.levels[:-1])
        t = torch.empty(n, dtype=torch.float32, device="cuda")
        B.bamg_mg_smoother_targets(gp.ctx, gp.mg, torch.from_numpy(Bk).cuda(), 3, t)
        ref = np.concatenate(OL.smoother_targets(h, Bk))
        assert np.allclose(t.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
    finally:
        gp.close()


def test_weighted_vcycle_and_stationary_match_oracle():
    ne = 13
    h = copy.deepcopy(hierarchy(ne))
    gp = GpuProblem(ne)
    try:
        rng = np.random.default_rng(5)
        w0 = rng.uniform(0.6, 1.6, h.levels[0].A.nbr).astype(np.float32)
        omg.set_weights(h, [w0])
        wd = torch.from_numpy(w0).cuda()
        B.bamg_mg_set_smoother_weights(gp.ctx, gp.mg, 0, wd)
        B.bamg_mg_update(gp.ctx, gp.mg)
        lam, _ = B.bamg_mg_get_level_scalars(gp.ctx, gp.mg, 0)
        assert abs(lam - h.levels[0].lam) <= 1e-12 * h.levels[0].lam
        b = body_force(gp.mesh)
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        B.bamg_vcycle(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x)
        assert rel(x.cpu().numpy(), omg.vcycle(h, b)) <= TOL64
        rn = B.bamg_mg_stationary(gp.ctx, gp.mg, torch.from_numpy(b).cuda(), x, 5)
        ref = omg.stationary(h, b, 5)
        assert np.allclose(rn, ref, rtol=1e-9)
    finally:
        gp.close()


def test_attached_mlp_predicts_the_weights_on_update(ctx):
    ne = 13
    gp = GpuProblem(ne)
    mlp = B.bamg_mlp_create(gp.ctx, 11)
    try:
        n0 = B.bamg_bsr_info(B.bamg_mg_get_level(gp.mg, 0)[0])["nbr"]
        X = torch.empty((n0, 8), dtype=torch.float32, device="cuda")
        B.bamg_mg_block_features(gp.ctx, gp.mg, 0, X)
        w = torch.empty(n0, dtype=torch.float32, device="cuda")
        B.bamg_mlp_forward(gp.ctx, mlp, X, w)
        b = torch.from_numpy(body_force(gp.mesh)).cuda()
        # manual weights on every level
        nl = B.bamg_mg_num_levels(gp.mg)
        ws = [w]
        for l in range(1, nl - 1):
            nl_rows = B.bamg_bsr_info(B.bamg_mg_get_level(gp.mg, l)[0])["nbr"]
            Xl = torch.empty((nl_rows, 8), dtype=torch.float32, device="cuda")
            B.bamg_mg_block_features(gp.ctx, gp.mg, l, Xl)
            wl = torch.empty(nl_rows, dtype=torch.float32, device="cuda")
            B.bamg_mlp_forward(gp.ctx, mlp, Xl, wl)
            ws.append(wl)
        for l, wl in enumerate(ws):
            B.bamg_mg_set_smoother_weights(gp.ctx, gp.mg, l, wl)
        B.bamg_mg_update(gp.ctx, gp.mg)
        x1 = torch.zeros_like(b)
        B.bamg_vcycle(gp.ctx, gp.mg, b, x1)
        # the same weights predicted inside mg_update
        B.bamg_mg_attach_mlp(gp.ctx, gp.mg, mlp)
        B.bamg_mg_update(gp.ctx, gp.mg)
        x2 = torch.zeros_like(b)
        B.bamg_vcycle(gp.ctx, gp.mg, b, x2)
        assert torch.equal(x1, x2)
        out = B.bamg_cg_solve(gp.ctx, gp.mg, b, x2, 1e-8, 200)
        assert out["converged"]
        B.bamg_mg_attach_mlp(gp.ctx, gp.mg, None)
    finally:
        B.bamg_mlp_destroy(mlp)
        gp.close()


def test_training_reduces_the_loss():
    from paper_2606_24748_gb300 import learned
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    mlp = B.bamg_mlp_create(ctx, 3)
    try:
        Xs, ts = [], []
        probs = learned.InclusionProblems(ctx, 12)
        for s in range(2):
            X, t = probs.load(s).data()
            Xs.append(X)
            ts.append(t)
        probs.close()
        X, t = torch.cat(Xs), torch.cat(ts)
        before = learned.mse(ctx, mlp, X, t)
        hist = learned.train(ctx, mlp, X, t, epochs=40, batch=2048, lr=3e-3)
        after = learned.mse(ctx, mlp, X, t)
        assert after < 0.5 * before and hist[-1] < hist[0]
    finally:
        B.bamg_mlp_destroy(mlp)
        B.bamg_ctx_destroy(ctx)


def test_numeric_resetup_equals_a_fresh_setup():
    from gpu_helpers import read_bsr, same_pattern
    ne = 13
    fresh = GpuProblem(ne, seed=21)
    reuse = GpuProblem(ne, seed=5)
    try:
        reuse.reassemble(21)
        B.bamg_mg_resetup(reuse.ctx, reuse.mg)
        for l in range(B.bamg_mg_num_levels(fresh.mg)):
            Af, Pf = B.bamg_mg_get_level(fresh.mg, l)
            Ar, Pr = B.bamg_mg_get_level(reuse.mg, l)
            a, b = read_bsr(fresh.ctx, Af), read_bsr(reuse.ctx, Ar)
            assert same_pattern(a, b) and rel(b.vals, a.vals) <= 1e-13
            if Pf is not None:
                pa, pb = read_bsr(fresh.ctx, Pf), read_bsr(reuse.ctx, Pr)
                assert rel(pb.vals, pa.vals) <= 1e-13
        h = hierarchy(ne)   # the unperturbed problem differs: resetup really recomputed P
        pr = read_bsr(reuse.ctx, B.bamg_mg_get_level(reuse.mg, 0)[1])
        assert rel(pr.vals, h.levels[0].P.vals) > 1e-8
    finally:
        fresh.close()
        reuse.close()


def test_train_epoch_equals_train_steps_on_gathered_batches(ctx):
    """bamg_mlp_train_epoch gathers each batch's rows through the permutation
    inside the kernel; it must give bit for bit the parameters (and the loss)
    of bamg_mlp_train_step on the same batches gathered beforehand."""
    rng = np.random.default_rng(12)
    n, batch = 10000, 3000                          # three full batches and a ragged one
    X = torch.from_numpy(rng.standard_normal((n, 8)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.uniform(0.5, 2.0, n).astype(np.float32)).cuda()
    perm = torch.from_numpy(rng.permutation(n)).cuda()
    a = B.bamg_mlp_create(ctx, 5)
    b = B.bamg_mlp_create(ctx, 5)
    try:
        loss_sum = torch.zeros(1, dtype=torch.float64, device="cuda")
        B.bamg_mlp_train_epoch(ctx, a, X, t, perm, batch, 1e-3, loss_sum)
        w = torch.empty(batch, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        tot = 0.0
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            B.bamg_mlp_train_step(ctx, b, X[idx].contiguous(), t[idx].contiguous(), w, 1e-3, loss)
            tot += float(loss.item()) * idx.numel()
        pa = torch.empty(OL.N_PARAMS, dtype=torch.float32, device="cuda")
        pb = torch.empty_like(pa)
        B.bamg_mlp_get_params(ctx, a, pa)
        B.bamg_mlp_get_params(ctx, b, pb)
        assert torch.equal(pa, pb)
        assert float(loss_sum.item()) == pytest.approx(tot, rel=1e-6)
    finally:
        B.bamg_mlp_destroy(a)
        B.bamg_mlp_destroy(b)
