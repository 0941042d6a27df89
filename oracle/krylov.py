"""Preconditioned conjugate gradients (Sec. 4.1: CG accelerator, stopping test on
the unpreconditioned residual norm).

x_0 = 0.  Each iteration: q = A p, alpha = (r, z) / (p, q), x += alpha p,
r -= alpha q; stop when ||r||_2 <= rtol ||b||_2; else z' = M r,
beta = (r, z' - z) / (r_old, z) (Polak-Ribiere form, which tolerates a
preconditioner that is not exactly symmetric, e.g. one applied in FP32), and
p = z' + beta p.  The true residual ||b - A x|| is recomputed at exit.
"""
from __future__ import annotations

import numpy as np


def pcg(As, b: np.ndarray, M, rtol: float = 1e-8, maxit: int = 500):
    """Returns (x, iterations, info) with info = residual history and flags."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = float(np.linalg.norm(b))
    hist = [float(np.linalg.norm(r))]
    if bnorm == 0.0 or hist[0] <= rtol * bnorm:
        return x, 0, {"history": hist, "converged": True, "true_residual": hist[0]}
    z = M(r)
    p = z.copy()
    rz = float(r @ z)
    converged = False
    its = 0
    for k in range(1, maxit + 1):
        q = As @ p
        pq = float(p @ q)
        if pq <= 0.0:
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        its = k
        hist.append(float(np.linalg.norm(r)))
        if hist[-1] <= rtol * bnorm:
            converged = True
            break
        z_new = M(r)
        beta = float(r @ (z_new - z)) / rz
        rz = float(r @ z_new)
        p = z_new + beta * p
        z = z_new
    true_res = float(np.linalg.norm(b - As @ x))
    return x, its, {"history": hist, "converged": converged, "true_residual": true_res}
