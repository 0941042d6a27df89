"""Algorithmic bytes and flops of the reuse-phase kernels.

Algorithmic bytes are what an operation must move at least: every matrix
value and index once, every vector it reads or writes once.  Re-reads,
intermediates (the A P product of the Galerkin triple product), padding of
the sliced storage and scatter maps are not counted, so a kernel that moves
more shows up as a lower achieved bandwidth.

The per-block figures follow the paper's byte accounting for blocked storage
(Sec. 4.2): a 3x3 block with FP64 values and one int32 column index moves
72 + 4 = 76 B against 108 B for the same nine entries in scalar CSR.
"""
from __future__ import annotations

IDX = 4  # int32 indices


def block_bytes(bs_r: int, bs_c: int, s: int = 8, idx: int = IDX) -> int:
    """Bytes of one stored block: values plus one column index (Sec. 4.2)."""
    return bs_r * bs_c * s + idx


def scalar_csr_bytes(bs_r: int, bs_c: int, s: int = 8, idx: int = IDX) -> int:
    """Bytes of the same entries in scalar CSR: one index per value (Sec. 4.2)."""
    return bs_r * bs_c * (s + idx)


def matrix_bytes(nnzb: int, nbr: int, bs_r: int, bs_c: int, s: int = 8) -> int:
    """Values, one index per block and the row pointers."""
    return nnzb * block_bytes(bs_r, bs_c, s) + IDX * (nbr + 1)


def spmv_bytes(nnzb: int, nbr: int, nbc: int, bs_r: int, bs_c: int, s: int = 8) -> int:
    """y = A x: the matrix once, x once, y written once."""
    return matrix_bytes(nnzb, nbr, bs_r, bs_c, s) + s * (bs_c * nbc + bs_r * nbr)


def spmv_flops(nnzb: int, bs_r: int, bs_c: int) -> int:
    return 2 * nnzb * bs_r * bs_c


def spmm_bytes(nnzb: int, nbr: int, nbc: int, bs_r: int, bs_c: int, k: int, s: int = 8) -> int:
    """Y = A X for k vectors: the matrix once, X once, Y written once."""
    return matrix_bytes(nnzb, nbr, bs_r, bs_c, s) + s * k * (bs_c * nbc + bs_r * nbr)


def ptap_bytes(A: dict, P: dict, Ac: dict, s: int = 8) -> int:
    """A_c = P^T A P: A and P read once (values, indices, row pointers), A_c values written."""
    return (matrix_bytes(A["nnzb"], A["nbr"], A["bs_r"], A["bs_c"], s)
            + matrix_bytes(P["nnzb"], P["nbr"], P["bs_r"], P["bs_c"], s)
            + s * Ac["nnzb"] * Ac["bs_r"] * Ac["bs_c"])


def ptap_flops(pairs_stage1: int, pairs_stage2: int, bs: int, bsp: int) -> int:
    """Multiply-adds of the two gather stages x 2: stage 1 pairs (A_ik, P_kJ)
    cost bs*bs*bsp FMA, stage 2 pairs (P_iI, Z_iJ) bs*bsp*bsp FMA."""
    return 2 * (pairs_stage1 * bs * bs * bsp + pairs_stage2 * bs * bsp * bsp)


def coo_bytes(n_coo: int, nnzb: int, bs_r: int, bs_c: int, s: int = 8) -> int:
    """Blocked COO numeric assembly: the value stream read once, the matrix
    values written once, the permutation and segment offsets read once."""
    return n_coo * bs_r * bs_c * s + nnzb * bs_r * bs_c * s + IDX * n_coo + IDX * (nnzb + 1)


def cheb_step_bytes(nnzb: int, n: int, bs: int, s: int, has_next: bool) -> int:
    """Fused Chebyshev step: A and the gathered direction once; x, r read and
    written; the next direction written and D^-1 read when has_next."""
    b = matrix_bytes(nnzb, n, bs, bs, s) + s * n * bs * (1 + 4)
    if has_next:
        b += s * n * bs + s * n * bs * bs
    return b


def vcycle_level_bytes(A: dict, P: dict | None, R: dict | None, s: int, degree: int = 2) -> int:
    """One V-cycle visit of a non-coarsest level (pre/post smoothing, transfers)."""
    n, bs, nnzb = A["nbr"], A["bs_r"], A["nnzb"]
    v = s * n * bs
    dinv = s * n * bs * bs
    total = 4 * v + dinv                                              # init: b -> r, d, x
    total += sum(cheb_step_bytes(nnzb, n, bs, s, k + 1 < degree) for k in range(degree))
    total += spmv_bytes(R["nnzb"], R["nbr"], R["nbc"], R["bs_r"], R["bs_c"], s)   # restrict
    total += spmv_bytes(P["nnzb"], P["nbr"], P["nbc"], P["bs_r"], P["bs_c"], s) + v  # prolong (x r/w)
    total += matrix_bytes(nnzb, n, bs, bs, s) + 4 * v + dinv          # residual init
    total += sum(cheb_step_bytes(nnzb, n, bs, s, True) for _ in range(degree - 1))
    total += 3 * v                                                    # final x += d
    return total


def coarse_solve_bytes(n: int) -> int:
    """Two dense triangular matrix-vector products with W = L^-1 (FP64)."""
    return 2 * (8 * n * (n + 1) // 2) + 8 * 4 * n


def cg_iteration_bytes(A: dict) -> int:
    """FP64 CG vector work and the A p product of one iteration (without the preconditioner)."""
    n = A["nbr"] * A["bs_r"]
    v = 8 * n
    return spmv_bytes(A["nnzb"], A["nbr"], A["nbc"], A["bs_r"], A["bs_c"]) + v * (2 + 4 + 3 + 4)
