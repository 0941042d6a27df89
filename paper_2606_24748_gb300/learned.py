"""Training and evaluation driver for the learned smoother weights.

Builds inclusion-mesh instances (3D elasticity with a heterogeneous Young's
modulus), generates (features, target) pairs with the plain V-cycle, trains
the MLP on the GPU with the library's own forward/backward/Adam kernels, and
compares the learned and the plain smoother on held-out instances: V-cycle
convergence factor of the stationary iteration and CG iterations / time to
rtol 1e-8.  Every numerical step runs in libbamg; this module only moves
tensors and calls the C ABI.

    python -m paper_2606_24748_gb300.learned --ne 48 --train 200 --test 50
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import bamg as B

K_RHS = 4
RHO_CYCLES = 10
RHO_SKIP = 2


def convergence_factor(rnorms, skip: int = RHO_SKIP) -> float:
    """(||r_n|| / ||r_skip||)^(1 / (n - skip)) of a residual-norm history r_0 .. r_n."""
    n = len(rnorms) - 1
    return float((rnorms[n] / rnorms[skip]) ** (1.0 / (n - skip)))


class InclusionProblems:
    """Inclusion meshes of one size, assembled through blocked COO; the first
    load builds the hierarchy, later loads re-set it up numerically for the
    new operator (same pattern, so every symbolic structure is reused)."""

    def __init__(self, ctx, ne: int, nu: float = 0.3, precision: int = B.BAMG_FP64):
        from workloads.elasticity import Mesh, body_force, coo_indices
        self.ctx, self.nu, self.precision = ctx, nu, precision
        self.mesh = Mesh(ne)
        m = self.mesh
        bi, bj = coo_indices(m, "cuda")
        self.A = B.bamg_bsr_create(ctx, 3, 3, m.n_nodes, m.n_nodes)
        B.bamg_bsr_coo_preallocate(ctx, self.A, bi, bj)
        self.mg = None
        self.b = torch.from_numpy(body_force(m)).cuda()
        self.seed = None

    def load(self, seed: int):
        from workloads.elasticity import coo_values, element_scale, gaussian_rhs, inclusion_moduli
        m = self.mesh
        vals = coo_values(m, self.nu, element_scale(m, E_el=inclusion_moduli(m, seed)), "cuda")
        B.bamg_bsr_coo_set_values(self.ctx, self.A, vals, 0)
        del vals
        if self.mg is None:
            o = B.bamg_mg_opts_default()
            o.grid[0] = o.grid[1] = o.grid[2] = m.m
            o.precision = self.precision
            self.mg = B.bamg_mg_setup(self.ctx, self.A, m.coords(), m.dirichlet(), o)
            self.nl = B.bamg_mg_num_levels(self.mg)
            self.rows = [B.bamg_bsr_info(B.bamg_mg_get_level(self.mg, l)[0])["nbr"] for l in range(self.nl - 1)]
        else:
            B.bamg_mg_attach_mlp(self.ctx, self.mg, None)
            B.bamg_mg_resetup(self.ctx, self.mg)
        self.rhs = torch.from_numpy(np.stack([gaussian_rhs(m, 10_000 + 31 * seed + k)
                                              for k in range(K_RHS)])).cuda()
        self.seed = seed
        return self

    def data(self):
        """(features, targets) of every non-coarsest level, stacked."""
        n = sum(self.rows)
        X = torch.empty((n, 8), dtype=torch.float32, device="cuda")
        t = torch.empty(n, dtype=torch.float32, device="cuda")
        off = 0
        for l, nr in enumerate(self.rows):
            B.bamg_mg_block_features(self.ctx, self.mg, l, X[off:off + nr])
            off += nr
        B.bamg_mg_smoother_targets(self.ctx, self.mg, self.rhs, K_RHS, t)
        return X, t

    def measure(self, its: int = RHO_CYCLES, skip: int = RHO_SKIP):
        """Convergence factor of the stationary V-cycle iteration and CG to 1e-8
        (iterations, ms).  The factor is the mean residual reduction per cycle
        over cycles skip+1 .. skip+its: under a large modulus contrast the
        first cycle raises ||b - A x|| (the energy norm of the error still
        falls), and that transient would otherwise dominate the mean."""
        x = torch.zeros_like(self.b)
        rn = B.bamg_mg_stationary(self.ctx, self.mg, self.b, x, skip + its)
        rho = convergence_factor(rn, skip)
        B.bamg_cg_solve(self.ctx, self.mg, self.b, x, 1e-8, 500, check=False)   # warm the graph
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = B.bamg_cg_solve(self.ctx, self.mg, self.b, x, 1e-8, 500, check=False)
        ms = (time.perf_counter() - t0) * 1e3
        return {"rho": rho, "cg_its": out["iterations"], "cg_ms": ms, "converged": out["converged"]}

    def close(self):
        if self.mg is not None:
            B.bamg_mg_destroy(self.mg)
        B.bamg_bsr_destroy(self.A)


def train(ctx, mlp, X, t, epochs: int = 30, batch: int = 32768, lr: float = 1e-3, seed: int = 0):
    """Mini-batch Adam on (X, t), one library call per epoch over a seeded
    device permutation (rows gathered inside the kernel); returns the mean
    loss of every epoch."""
    n = X.shape[0]
    g = torch.Generator(device="cuda").manual_seed(seed)
    sums = torch.zeros(epochs, dtype=torch.float64, device="cuda")
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g, device="cuda")
        B.bamg_mlp_train_epoch(ctx, mlp, X, t, perm, batch, lr, sums[ep:ep + 1])
    return [float(v) / n for v in sums.cpu()]


def train_step_rate(ctx, mlp, n: int = 1 << 20, reps: int = 20, seed: int = 0) -> dict:
    """Rows per second of one training step (fused forward + backward on the
    tensor cores, gradient reduction, Adam) on n seeded N(0,1) feature rows,
    CUDA events on the current stream; the parameters are restored after."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    X = torch.randn((n, 8), generator=gen).cuda()
    t = (0.5 + 1.5 * torch.rand(n, generator=gen)).cuda()
    w = torch.empty(n, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    saved = torch.empty(B.bamg_mlp_num_params(), dtype=torch.float32, device="cuda")
    B.bamg_mlp_get_params(ctx, mlp, saved)
    for _ in range(3):
        B.bamg_mlp_train_step(ctx, mlp, X, t, w, 1e-6, loss)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        B.bamg_mlp_train_step(ctx, mlp, X, t, w, 1e-6, loss)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    B.bamg_mlp_set_params(ctx, mlp, saved)
    # multiply-adds per row: 8x64 + 64x64 + 64 forward, 64x64 for d1, 64x64 + 8x64 + 3x64 for the gradients
    flop_row = 2 * (8 * 64 + 64 * 64 + 64) + 2 * 64 * 64 + 2 * (64 * 64 + 8 * 64 + 3 * 64)
    return {"rows": n, "ms_per_step": round(ms, 4), "rows_per_s": round(n / ms * 1e3, 1),
            "tflops": round(flop_row * n / ms / 1e9, 3), "flop_per_row": flop_row}


def mse(ctx, mlp, X, t) -> float:
    w = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    B.bamg_mlp_forward(ctx, mlp, X, w)
    return float(torch.mean((w - t) ** 2).item())


def run(ne: int = 48, n_train: int = 200, n_test: int = 50, epochs: int = 30, seed0_train: int = 0,
        seed0_test: int = 1000, log=print) -> dict:
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    mlp = B.bamg_mlp_create(ctx, 12345)
    probs = InclusionProblems(ctx, ne)
    Xs, ts = [], []
    t0 = time.perf_counter()
    for k in range(n_train):
        X, t = probs.load(seed0_train + k).data()
        Xs.append(X)
        ts.append(t)
    X, t = torch.cat(Xs), torch.cat(ts)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t1 = time.perf_counter()
    hist = train(ctx, mlp, X, t, epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    log(f"training set {X.shape[0]} rows from {n_train} instances in {t_data:.1f} s; "
        f"{epochs} epochs in {t_train:.2f} s, loss {hist[0]:.4f} -> {hist[-1]:.4f}")
    rate = train_step_rate(ctx, mlp)
    var = float(torch.mean((t - t.mean()) ** 2).item())
    res = []
    for k in range(n_test):
        p = probs.load(seed0_test + k)
        Xt, tt = p.data()
        plain = p.measure()
        B.bamg_mg_attach_mlp(ctx, p.mg, mlp)
        B.bamg_mg_update(ctx, p.mg)
        learned = p.measure()
        res.append({"plain": plain, "learned": learned, "mse": mse(ctx, mlp, Xt, tt)})
    probs.close()
    B.bamg_mlp_destroy(mlp)
    B.bamg_ctx_destroy(ctx)

    def agg(key, f):
        return float(np.mean([r[key][f] for r in res]))
    out = {
        "ne": ne, "train_instances": n_train, "test_instances": n_test, "train_rows": int(X.shape[0]),
        "epochs": epochs, "train_seconds": round(t_train, 3), "data_seconds": round(t_data, 1),
        "train_rows_per_s": round(X.shape[0] * epochs / t_train, 1), "train_step_kernels": rate,
        "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1], "target_variance": var,
        "test_mse": float(np.mean([r["mse"] for r in res])),
        "rho_plain": agg("plain", "rho"), "rho_learned": agg("learned", "rho"),
        "cg_its_plain": agg("plain", "cg_its"), "cg_its_learned": agg("learned", "cg_its"),
        "cg_ms_plain": agg("plain", "cg_ms"), "cg_ms_learned": agg("learned", "cg_ms"),
        "learned_better_fraction": float(np.mean([r["learned"]["rho"] < r["plain"]["rho"] for r in res])),
        "all_converged": bool(all(r[k]["converged"] for r in res for k in ("plain", "learned"))),
        "per_instance": [{"rho_plain": r["plain"]["rho"], "rho_learned": r["learned"]["rho"],
                          "cg_its_plain": r["plain"]["cg_its"], "cg_its_learned": r["learned"]["cg_its"]}
                         for r in res],
    }
    # the plain smoother stays the fallback unless the learned one converges faster
    out["use_learned"] = out["rho_learned"] < out["rho_plain"] and out["cg_its_learned"] <= out["cg_its_plain"]
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--ne", type=int, default=48)
    p.add_argument("--train", type=int, default=200)
    p.add_argument("--test", type=int, default=50)
    p.add_argument("--epochs", type=int, default=30)
    a = p.parse_args()
    print(json.dumps(run(a.ne, a.train, a.test, a.epochs)))


if __name__ == "__main__":
    main()
