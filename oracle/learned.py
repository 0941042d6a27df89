"""Learned per-block-row smoother weights: features, targets, MLP, Adam.

Reference for the learned part of the smoother (not in the paper; specified
by the workload: an MLP with two hidden layers of 64 predicts one weight per
block row from local block features; it is trained on residual-reduction
data from the plain V-cycle; the plain smoother stays the fallback).

Features of block row i (level l), FP32:
  f0 = log ||A_ii||_F
  f1 = sum_{j != i} ||A_ij||_F / ||A_ii||_F
  f2 = log(max_j ||A_ij||_F / min_{j: ||A_ij|| > 0} ||A_ij||_F)
  f3 = (number of stored blocks in the row) / 27
  f4 = 1 if every off-diagonal block is zero (a clamped row), else 0
  f5 = log sum_j ||D_i^{-1} A_ij||_F   (a Gershgorin-type bound of the scaled row)
  f6 = l (level index)
  f7 = 1
Target of block row i: the local least-squares damping of a Richardson step
on the preconditioned residual, w_i = clip(sum_k <r_i, q_i> / sum_k ||q_i||^2,
0.5, 2) with q = A D^{-1} r and r the residual after pre-smoothing on that
level inside plain V-cycles, summed over k seeded right-hand sides.
MLP: z = w3 . relu(W2^T relu(W1^T x + b1) + b2) + b3, weight
w = 0.5 + 1.5 sigmoid(z); inputs, parameters and hidden activations rounded
to bfloat16 (round to nearest even), products accumulated in FP32; loss MSE.
Adam (Kingma and Ba, ICLR 2015) with beta1 0.9, beta2 0.999, eps 1e-8 on FP32
master parameters.
"""
from __future__ import annotations

import numpy as np

from .assembly import BlockMatrix
from .smoother import apply_blocks, diagonal_blocks

N_FEATURES = 8
HIDDEN = 64
LAYOUT = (("W1", (N_FEATURES, HIDDEN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (HIDDEN,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in LAYOUT)
W_LO, W_HI = 0.5, 2.0


def bf16(x) -> np.ndarray:
    """Round float32 values to bfloat16 precision (nearest, ties to even), as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def unpack(theta: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in LAYOUT:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in LAYOUT])


# ------------------------------------------------------------------ features
def block_features(A: BlockMatrix, level: int, Dinv: np.ndarray | None = None) -> np.ndarray:
    D = diagonal_blocks(A)
    Dinv = np.linalg.inv(D) if Dinv is None else Dinv
    rows = A.block_rows()
    norms = np.sqrt(np.sum(A.vals.astype(np.float64) ** 2, axis=(1, 2)))
    scaled = np.einsum("nij,njk->nik", Dinv[rows], A.vals)
    snorm = np.sqrt(np.sum(scaled ** 2, axis=(1, 2)))
    F = np.zeros((A.nbr, N_FEATURES))
    for i in range(A.nbr):
        lo, hi = A.rowptr[i], A.rowptr[i + 1]
        cols = A.colidx[lo:hi]
        nr = norms[lo:hi]
        d = nr[cols == i][0]
        off = nr[cols != i]
        F[i, 0] = np.log(d)
        F[i, 1] = off.sum() / d
        pos = nr[nr > 0]
        F[i, 2] = np.log(pos.max() / pos.min())
        F[i, 3] = (hi - lo) / 27.0
        F[i, 4] = 1.0 if not np.any(off > 0) else 0.0
        F[i, 5] = np.log(snorm[lo:hi].sum())
        F[i, 6] = level
        F[i, 7] = 1.0
    return F.astype(np.float32)


# ------------------------------------------------------------------- targets
def local_damping(As, Dinv: np.ndarray, R: list[np.ndarray]) -> np.ndarray:
    """clip(sum_k <r_i, q_i> / sum_k ||q_i||^2, 0.5, 2), q = A D^{-1} r, per block row."""
    n, bs, _ = Dinv.shape
    num = np.zeros(n)
    den = np.zeros(n)
    for r in R:
        q = As @ apply_blocks(Dinv, r)
        num += np.sum((r * q).reshape(n, bs), axis=1)
        den += np.sum((q * q).reshape(n, bs), axis=1)
    w = np.where(den > 0, num / np.where(den > 0, den, 1.0), 1.0)
    return np.clip(w, W_LO, W_HI).astype(np.float32)


def smoother_targets(h, B: np.ndarray) -> list[np.ndarray]:
    """Targets of every non-coarsest level from plain V-cycle pre-smoothing on
    the right-hand sides B (k x n0): level l uses the residual after its
    pre-smoothing, with the restricted residual of level l-1 as right-hand side."""
    from .smoother import chebyshev
    nl = h.n_levels
    res = [[] for _ in range(nl - 1)]
    for b in B:
        rhs = np.asarray(b, dtype=np.float64)
        for l in range(nl - 1):
            L = h.levels[l]
            _, r = chebyshev(L.As, L.Dinv, rhs, None, L.lam, h.degree, want_residual=True,
                             weights=L.weights)
            res[l].append(r)
            rhs = L.Ps.T @ r
    return [local_damping(h.levels[l].As, h.levels[l].Dinv, res[l]) for l in range(nl - 1)]


# ----------------------------------------------------------------------- MLP
def forward(theta: np.ndarray, X: np.ndarray, emulate_bf16: bool = True):
    """Returns (w, cache).  FP32 arithmetic on bfloat16-rounded operands, or
    plain FP64 when emulate_bf16 is False."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    if emulate_bf16:
        r = bf16
        f = np.float32
    else:
        r = (lambda a: np.asarray(a, dtype=np.float64))
        f = np.float64
    x = r(X)
    W1, b1, W2, b2 = r(p["W1"]), r(p["b1"]), r(p["W2"]), r(p["b2"])
    W3, b3 = r(p["W3"]), r(p["b3"])
    a1 = (x.astype(f) @ W1.astype(f) + b1.astype(f)).astype(f)
    h1 = r(np.maximum(a1, 0))
    a2 = (h1.astype(f) @ W2.astype(f) + b2.astype(f)).astype(f)
    h2 = r(np.maximum(a2, 0))
    z = (h2.astype(f) @ W3.astype(f) + b3.astype(f)[0]).astype(f)
    s = 1.0 / (1.0 + np.exp(-z.astype(np.float64)))
    w = W_LO + (W_HI - W_LO) * s
    cache = dict(x=x, a1=a1, h1=h1, a2=a2, h2=h2, z=z, s=s, W2=W2, W3=W3)
    return w, cache


def loss_and_grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray, emulate_bf16: bool = True):
    """MSE loss mean((w - t)^2) and its gradient with respect to theta."""
    w, c = forward(theta, X, emulate_bf16)
    n = X.shape[0]
    e = w - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(e ** 2))
    dz = (2.0 / n) * e * (W_HI - W_LO) * c["s"] * (1.0 - c["s"])
    g = {}
    g["b3"] = np.array([dz.sum()])
    g["W3"] = c["h2"].astype(np.float64).T @ dz
    d2 = np.outer(dz, c["W3"].astype(np.float64)) * (c["a2"] > 0)
    g["b2"] = d2.sum(axis=0)
    g["W2"] = c["h1"].astype(np.float64).T @ d2
    d1 = (d2 @ c["W2"].astype(np.float64).T) * (c["a1"] > 0)
    g["b1"] = d1.sum(axis=0)
    g["W1"] = c["x"].astype(np.float64).T @ d1
    return loss, pack(g)


class Adam:
    def __init__(self, n: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta: np.ndarray, g: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
