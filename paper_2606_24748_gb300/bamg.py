"""Thin Python binding of libbamg (the C ABI declared in include/bamg.h).

Every function here has the name of the C entry point it calls and only
marshals arguments: device buffers are passed as torch CUDA tensors (their
data pointers), host buffers as numpy arrays, and handles as opaque
ctypes pointers.  A non-zero status raises :class:`BamgError` with the
library's last-error message.  All compute runs in the CUDA library; there is
no fallback: if libbamg.so is missing or cannot be loaded, importing the
library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbamg.so")

BAMG_OK = 0
STATUS_NAMES = {0: "BAMG_OK", 1: "BAMG_ERR_INVALID", 2: "BAMG_ERR_OOM", 3: "BAMG_ERR_CUDA", 4: "BAMG_ERR_STATE",
                5: "BAMG_ERR_NAN", 6: "BAMG_ERR_BREAKDOWN", 7: "BAMG_ERR_NOT_CONVERGED", 8: "BAMG_ERR_TIMEOUT"}
(BAMG_ERR_INVALID, BAMG_ERR_OOM, BAMG_ERR_CUDA, BAMG_ERR_STATE, BAMG_ERR_NAN, BAMG_ERR_BREAKDOWN,
 BAMG_ERR_NOT_CONVERGED, BAMG_ERR_TIMEOUT) = range(1, 9)
BAMG_FP64 = 0
BAMG_FP32 = 1
BAMG_AGG_GEOMETRIC = 0
BAMG_AGG_MIS = 1
BAMG_NORM_FROBENIUS = 0
BAMG_NORM_INFINITY = 1
PROF_SLOTS = {"cheb_step_l0": 0, "cheb_rinit_l0": 1, "ptap_stage1_l0": 2, "ptap_stage2_l0": 3, "cg_ap": 4,
              "coo": 5, "coarse_factor": 6, "smooth_coarse": 7, "transfer": 8, "coarse_solve": 9,
              "l0_vector": 10, "cg_xr": 11, "cg_vector": 12, "refresh": 13, "cheb_pre_l0": 14}


class BamgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class bamg_mg_opts(ctypes.Structure):
    _fields_ = [("max_levels", ctypes.c_int), ("max_coarse_dofs", ctypes.c_int64),
                ("grid", ctypes.c_int * 3), ("cheb_degree", ctypes.c_int),
                ("cheb_lower", ctypes.c_double), ("cheb_upper", ctypes.c_double),
                ("power_its", ctypes.c_int), ("precision", ctypes.c_int), ("autotune", ctypes.c_int),
                ("coarse_solver", ctypes.c_int), ("aggregation", ctypes.c_int), ("mis_eps", ctypes.c_double),
                ("mis_seed", ctypes.c_uint64)]


class bamg_shard_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("ghost_rows", "halo_bytes_per_spmv", "poth_blocks", "poth_bytes",
                                              "poth_gathers", "reduce_blocks", "reduce_bytes_per_ptap",
                                              "max_owned_rows")]


class bamg_cg_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rnorm", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("true_rnorm", ctypes.c_double)]


_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_I64 = ctypes.c_int64
_SIGS = {
    "bamg_ctx_create": [_P, _PP],
    "bamg_ctx_destroy": [_P],
    "bamg_ctx_sync": [_P],
    "bamg_probe_fma_rate": [_P, ctypes.c_int, _P],
    "bamg_halo_create": [_I64, _P, _P, ctypes.c_int, _P, _PP],
    "bamg_halo_destroy": [_P],
    "bamg_halo_part_info": [_P, ctypes.c_int, _P, _P, _P],
    "bamg_halo_part_pattern": [_P, ctypes.c_int, _P, _P, _P],
    "bamg_halo_part_ghosts": [_P, ctypes.c_int, _P, _P],
    "bamg_halo_sends": [_P, ctypes.c_int, ctypes.c_int, _P, _P],
    "bamg_sharded_create": [_P, _P, ctypes.c_int, _P, _PP, _PP],
    "bamg_sharded_spmv": [_P, _P, _P],
    "bamg_sharded_ptap": [_P, _P, _P, _P],
    "bamg_sharded_stats": [_P, _P],
    "bamg_sharded_destroy": [_P],
    "bamg_mlp_train_epoch": [_P, _P, _P, _P, _I64, _I64, ctypes.c_float, _P],
    "bamg_ctx_set_wait_limit": [_P, _I64],
    "bamg_mg_get_aggregates": [_P, ctypes.c_int, _P],
    "bamg_mg_get_gate_counts": [_P, ctypes.c_int, _P, _P],
    "bamg_ptap_get_refreshes": [_P, _P],
    "bamg_ctx_profile": [_P, ctypes.c_int],
    "bamg_ctx_profile_slots": [_P, ctypes.c_uint],
    "bamg_device_memory": [_P, _P, _P, ctypes.c_int],
    "bamg_ctx_profile_read": [_P, ctypes.c_int, _P, _P],
    "bamg_bsr_create": [_P, ctypes.c_int, ctypes.c_int, _I64, _I64, _PP],
    "bamg_bsr_destroy": [_P],
    "bamg_bsr_coo_preallocate": [_P, _I64, _P, _P],
    "bamg_bsr_coo_set_values": [_P, _P, ctypes.c_int],
    "bamg_bsr_info": [_P, _P, _P, _P, _P, _P, _P],
    "bamg_bsr_storage": [_P, _P, _P],
    "bamg_bsr_get_pattern": [_P, _P, _P],
    "bamg_bsr_get_values": [_P, _P],
    "bamg_bsr_set_symmetric": [_P, ctypes.c_int],
    "bamg_bsr_spmv": [_P, _P, _P, ctypes.c_int, ctypes.c_int],
    "bamg_bsr_autotune": [_P, _P, _P],
    "bamg_bsr_residual_norm_noalloc": [_P, _P, _P, _P],
    "bamg_bsr_set_lanes": [_P, ctypes.c_int],
    "bamg_bsr_get_lanes": [_P, _P],
    "bamg_bsr_set_lanes_prec": [_P, ctypes.c_int, ctypes.c_int],
    "bamg_bsr_get_lanes_prec": [_P, ctypes.c_int, _P],
    "bamg_bsr_block_norms": [_P, _P],
    "bamg_bsr_coo_scatter_values": [_P, _P, ctypes.c_int],
    "bamg_bsr_norm": [_P, ctypes.c_int, _P],
    "bamg_strength_graph": [_P, ctypes.c_double, _P, _P, ctypes.c_int64, _P],
    "bamg_mis_aggregate": [_P, ctypes.c_int64, _P, _P, ctypes.c_uint64, _P, _P, _P],
    "bamg_bsr_spmm": [_P, _P, _P, ctypes.c_int, ctypes.c_int],
    "bamg_ptap_symbolic": [_P, _P, _PP, _PP],
    "bamg_ptap_numeric": [_P, _P, _P, _P],
    "bamg_ptap_numeric_prec": [_P, _P, _P, _P, ctypes.c_int],
    "bamg_ptap_destroy": [_P],
    "bamg_mg_setup": [_P, _P, _P, _P, ctypes.POINTER(bamg_mg_opts), _PP],
    "bamg_mg_update": [_P],
    "bamg_mg_resetup": [_P],
    "bamg_vcycle": [_P, _P, _P],
    "bamg_cg_solve": [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(bamg_cg_info)],
    "bamg_mg_vcycle_multi": [_P, _P, _P, ctypes.c_int],
    "bamg_cg_solve_multi": [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(bamg_cg_info)],
    "bamg_batch_create": [_P, ctypes.c_int, _P, _PP],
    "bamg_batch_destroy": [_P],
    "bamg_batch_set_branches": [_P, ctypes.c_int],
    "bamg_batch_get_branches": [_P, ctypes.POINTER(ctypes.c_int)],
    "bamg_batch_cg_solve": [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(bamg_cg_info),
                            ctypes.POINTER(ctypes.c_int)],
    "bamg_batch_autotune": [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_float)],
    "bamg_mg_set_smoother_weights": [_P, ctypes.c_int, _P],
    "bamg_mg_set_lanes": [_P, ctypes.c_int],
    "bamg_mg_num_levels": [_P, ctypes.POINTER(ctypes.c_int)],
    "bamg_mg_get_level": [_P, ctypes.c_int, _PP, _PP],
    "bamg_mg_get_restriction": [_P, ctypes.c_int, _PP],
    "bamg_mg_get_level_scalars": [_P, ctypes.c_int, _P, _P],
    "bamg_mg_get_dinv": [_P, ctypes.c_int, _P],
    "bamg_mg_destroy": [_P],
    "bamg_mlp_num_params": [_P],
    "bamg_mlp_create": [_P, ctypes.c_uint64, _PP],
    "bamg_mlp_destroy": [_P],
    "bamg_mlp_get_params": [_P, _P],
    "bamg_mlp_set_params": [_P, _P],
    "bamg_mlp_forward": [_P, _P, _I64, _P],
    "bamg_mlp_gradient": [_P, _P, _P, _I64, _P, _P, _P],
    "bamg_mlp_train_step": [_P, _P, _P, _I64, _P, ctypes.c_float, _P],
    "bamg_mg_block_features": [_P, ctypes.c_int, _P],
    "bamg_mg_smoother_targets": [_P, _P, ctypes.c_int, _P],
    "bamg_mg_attach_mlp": [_P, _P],
    "bamg_mg_stationary": [_P, _P, _P, ctypes.c_int, _P],
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libbamg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libbamg.so not found at {LIB_PATH}: run paper_2606_24748_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.bamg_last_error.argtypes = [_P]
        L.bamg_last_error.restype = ctypes.c_char_p
        L.bamg_mg_opts_default.argtypes = [ctypes.POINTER(bamg_mg_opts)]
        L.bamg_mg_opts_default.restype = None
        L.bamg_kernel_launches.argtypes = []
        L.bamg_kernel_launches.restype = ctypes.c_uint64
        _lib = L
    return _lib


def _ptr(t) -> int | None:
    """Device pointer of a torch tensor (None passes NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _check(status: int, ctx) -> None:
    if status != BAMG_OK:
        msg = lib().bamg_last_error(ctx).decode() if ctx else ""
        raise BamgError(status, msg)


# ------------------------------------------------------------------ context
def bamg_ctx_create(stream=None):
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (legacy default)."""
    s = getattr(stream, "cuda_stream", stream)
    h = ctypes.c_void_p()
    _check(lib().bamg_ctx_create(s, ctypes.byref(h)), None)
    return h


def bamg_ctx_destroy(ctx):
    _check(lib().bamg_ctx_destroy(ctx), None)


def bamg_last_error(ctx) -> str:
    return lib().bamg_last_error(ctx).decode()


def bamg_ctx_sync(ctx):
    _check(lib().bamg_ctx_sync(ctx), ctx)


def bamg_ctx_profile(ctx, enable: int):
    _check(lib().bamg_ctx_profile(ctx, int(enable)), ctx)


def bamg_ctx_profile_slots(ctx, slots):
    """Time only the named slots (names of PROF_SLOTS or slot numbers); empty disables."""
    mask = 0
    for s in slots:
        mask |= 1 << (PROF_SLOTS[s] if isinstance(s, str) else int(s))
    _check(lib().bamg_ctx_profile_slots(ctx, mask), ctx)


def bamg_ctx_profile_read(ctx, slot: int) -> tuple[float, int]:
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(lib().bamg_ctx_profile_read(ctx, int(slot), ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def bamg_device_memory(ctx, reset_peak: bool = False) -> tuple[int, int]:
    """(bytes in use, high-water mark) of the library's device allocations."""
    used, peak = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().bamg_device_memory(ctx, ctypes.byref(used), ctypes.byref(peak), int(reset_peak)), ctx)
    return used.value, peak.value


def bamg_kernel_launches() -> int:
    return int(lib().bamg_kernel_launches())


def bamg_mg_get_aggregates(ctx, mg, level: int, out):
    """Aggregate of every block row of a level (-1: in none) into a device int32 tensor."""
    _check(lib().bamg_mg_get_aggregates(mg, int(level), _ptr(out)), ctx)


def bamg_ctx_set_wait_limit(ctx, polls: int):
    _check(lib().bamg_ctx_set_wait_limit(ctx, int(polls)), ctx)


def bamg_mg_get_gate_counts(mg, level: int) -> tuple[int, int]:
    """(rebuilds of the plan's block-ordered P, rebuilds of R) of a level."""
    p, r = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().bamg_mg_get_gate_counts(mg, int(level), ctypes.byref(p), ctypes.byref(r)), None)
    return p.value, r.value


def bamg_ptap_get_refreshes(plan) -> int:
    p = ctypes.c_uint64()
    _check(lib().bamg_ptap_get_refreshes(plan, ctypes.byref(p)), None)
    return p.value


def bamg_probe_fma_rate(ctx, precision: int) -> float:
    """Measured FMA throughput (TFLOP/s) of the FP64 or FP32 pipe."""
    out = ctypes.c_double()
    _check(lib().bamg_probe_fma_rate(ctx, int(precision), ctypes.byref(out)), ctx)
    return out.value


# ---------------------------------------------------------- block matrices
def bamg_bsr_create(ctx, bs_r: int, bs_c: int, nbr: int, nbc: int):
    h = ctypes.c_void_p()
    _check(lib().bamg_bsr_create(ctx, bs_r, bs_c, nbr, nbc, ctypes.byref(h)), ctx)
    return h


def bamg_bsr_destroy(A):
    _check(lib().bamg_bsr_destroy(A), None)


def bamg_bsr_coo_preallocate(ctx, A, bi, bj):
    """bi, bj: int32 CUDA tensors of block coordinates."""
    _check(lib().bamg_bsr_coo_preallocate(A, int(bi.numel()), _ptr(bi), _ptr(bj)), ctx)


def bamg_bsr_coo_set_values(ctx, A, v, add: int = 0):
    """v: float64 CUDA tensor of n row-major blocks."""
    _check(lib().bamg_bsr_coo_set_values(A, _ptr(v), int(add)), ctx)


def bamg_bsr_info(A) -> dict:
    bs_r, bs_c = ctypes.c_int(), ctypes.c_int()
    nbr, nbc, nnzb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    ver = ctypes.c_uint64()
    _check(lib().bamg_bsr_info(A, ctypes.byref(bs_r), ctypes.byref(bs_c), ctypes.byref(nbr), ctypes.byref(nbc),
                               ctypes.byref(nnzb), ctypes.byref(ver)), None)
    return {"bs_r": bs_r.value, "bs_c": bs_c.value, "nbr": nbr.value, "nbc": nbc.value, "nnzb": nnzb.value,
            "version": ver.value}


def bamg_bsr_storage(A) -> dict:
    slots, sorted_ = ctypes.c_int64(), ctypes.c_int()
    _check(lib().bamg_bsr_storage(A, ctypes.byref(slots), ctypes.byref(sorted_)), None)
    return {"stored_slots": slots.value, "rows_sorted": bool(sorted_.value)}


def bamg_bsr_get_pattern(ctx, A, rowptr, colidx):
    _check(lib().bamg_bsr_get_pattern(A, _ptr(rowptr), _ptr(colidx)), ctx)


def bamg_bsr_get_values(ctx, A, vals):
    _check(lib().bamg_bsr_get_values(A, _ptr(vals)), ctx)


def bamg_bsr_set_symmetric(ctx, A, symmetric: int):
    _check(lib().bamg_bsr_set_symmetric(A, int(symmetric)), ctx)


def bamg_bsr_autotune(ctx, A) -> tuple[int, float]:
    lanes, ms = ctypes.c_int(), ctypes.c_float()
    _check(lib().bamg_bsr_autotune(A, ctypes.byref(lanes), ctypes.byref(ms)), ctx)
    return lanes.value, ms.value


def bamg_bsr_set_lanes(ctx, A, lanes: int):
    _check(lib().bamg_bsr_set_lanes(A, int(lanes)), ctx)


def bamg_bsr_coo_scatter_values(ctx, A, v, add: int = 0):
    """Element-by-element (atomic) assembly of the COO stream v."""
    _check(lib().bamg_bsr_coo_scatter_values(A, _ptr(v), int(add)), ctx)


def bamg_bsr_block_norms(ctx, A, out):
    """Frobenius norm of every stored block (block-CSR order) into the device tensor out."""
    _check(lib().bamg_bsr_block_norms(A, _ptr(out)), ctx)


def bamg_bsr_norm(ctx, A, kind: int = BAMG_NORM_FROBENIUS) -> float:
    v = ctypes.c_double()
    _check(lib().bamg_bsr_norm(A, int(kind), ctypes.byref(v)), ctx)
    return v.value


def bamg_strength_graph(ctx, A, eps: float, rowptr, col) -> int:
    """Strong-coupling graph into device int32 tensors rowptr (nbr + 1) and col; returns the edge count."""
    ne = ctypes.c_int64()
    _check(lib().bamg_strength_graph(A, float(eps), _ptr(rowptr), _ptr(col), int(col.numel()), ctypes.byref(ne)), ctx)
    return ne.value


def bamg_mis_aggregate(ctx, n: int, rowptr, col, seed: int, agg) -> tuple[int, int]:
    """MIS aggregates of a device CSR graph into the int32 tensor agg; returns (aggregates, rounds)."""
    na, rounds = ctypes.c_int64(), ctypes.c_int()
    _check(lib().bamg_mis_aggregate(ctx, int(n), _ptr(rowptr), _ptr(col), ctypes.c_uint64(seed), _ptr(agg),
                                    ctypes.byref(na), ctypes.byref(rounds)), ctx)
    return na.value, rounds.value


def bamg_bsr_get_lanes(A) -> int:
    v = ctypes.c_int()
    _check(lib().bamg_bsr_get_lanes(A, ctypes.byref(v)), None)
    return v.value


def bamg_bsr_set_lanes_prec(ctx, A, prec: int, lanes: int):
    _check(lib().bamg_bsr_set_lanes_prec(A, int(prec), int(lanes)), ctx)


def bamg_bsr_get_lanes_prec(A, prec: int) -> int:
    v = ctypes.c_int()
    _check(lib().bamg_bsr_get_lanes_prec(A, int(prec), ctypes.byref(v)), None)
    return v.value


def bamg_bsr_residual_norm_noalloc(ctx, A, x, b, norm):
    """||b - A x||_2 into the one-element float64 CUDA tensor `norm`, without
    any device allocation (see include/bamg.h)."""
    _check(lib().bamg_bsr_residual_norm_noalloc(A, _ptr(x), _ptr(b), _ptr(norm)), ctx)


def bamg_bsr_spmv(ctx, A, x, y, prec: int = BAMG_FP64, transpose: int = 0):
    _check(lib().bamg_bsr_spmv(A, _ptr(x), _ptr(y), int(prec), int(transpose)), ctx)


def bamg_bsr_spmm(ctx, A, X, Y, k: int, prec: int = BAMG_FP64):
    _check(lib().bamg_bsr_spmm(A, _ptr(X), _ptr(Y), int(k), int(prec)), ctx)


# ------------------------------------------------------------ Galerkin
def bamg_ptap_symbolic(ctx, A, P):
    plan, Ac = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().bamg_ptap_symbolic(A, P, ctypes.byref(plan), ctypes.byref(Ac)), ctx)
    return plan, Ac


def bamg_ptap_numeric(ctx, plan, A, P, Ac):
    _check(lib().bamg_ptap_numeric(plan, A, P, Ac), ctx)


def bamg_ptap_numeric_prec(ctx, plan, A, P, Ac, prec: int):
    _check(lib().bamg_ptap_numeric_prec(plan, A, P, Ac, int(prec)), ctx)


def bamg_ptap_destroy(plan):
    _check(lib().bamg_ptap_destroy(plan), None)


# ------------------------------------------------------------ multigrid
def bamg_mg_opts_default() -> bamg_mg_opts:
    o = bamg_mg_opts()
    lib().bamg_mg_opts_default(ctypes.byref(o))
    return o


def bamg_mg_setup(ctx, A, coords: np.ndarray, dirichlet: np.ndarray, opts: bamg_mg_opts):
    c = np.ascontiguousarray(coords, dtype=np.float64)
    d = np.ascontiguousarray(dirichlet, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(lib().bamg_mg_setup(ctx, A, c.ctypes.data, d.ctypes.data, ctypes.byref(opts), ctypes.byref(h)), ctx)
    return h


def bamg_mg_update(ctx, mg):
    _check(lib().bamg_mg_update(mg), ctx)


def bamg_mg_resetup(ctx, mg):
    _check(lib().bamg_mg_resetup(mg), ctx)


def bamg_vcycle(ctx, mg, b, x):
    _check(lib().bamg_vcycle(mg, _ptr(b), _ptr(x)), ctx)


def bamg_cg_solve(ctx, mg, b, x, rtol: float, maxit: int, check: bool = True) -> dict:
    info = bamg_cg_info()
    st = lib().bamg_cg_solve(mg, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(info))
    out = {"status": st, "iterations": info.iterations, "converged": bool(info.converged),
           "rnorm": info.rnorm, "bnorm": info.bnorm, "true_rnorm": info.true_rnorm}
    if check:
        _check(st, ctx)
    return out


def bamg_mg_vcycle_multi(ctx, mg, B, X, k: int):
    """X = M B for k fine vectors stored RHS-minor (B[d * k + j])."""
    _check(lib().bamg_mg_vcycle_multi(mg, _ptr(B), _ptr(X), int(k)), ctx)


def bamg_cg_solve_multi(ctx, mg, B, X, k: int, rtol: float, maxit: int, check: bool = True) -> list:
    """k simultaneous PCG solves; returns one info dict per column."""
    info = (bamg_cg_info * max(1, int(k)))()
    st = lib().bamg_cg_solve_multi(mg, _ptr(B), _ptr(X), int(k), float(rtol), int(maxit), info)
    out = [{"status": st, "iterations": i.iterations, "converged": bool(i.converged), "rnorm": i.rnorm,
            "bnorm": i.bnorm, "true_rnorm": i.true_rnorm} for i in info[:int(k)]]
    if check:
        _check(st, ctx)
    return out


def _ptr_array(ts):
    return (ctypes.c_void_p * len(ts))(*[(_ptr(t) if t is not None else None) for t in ts])


def bamg_batch_create(ctx, mgs):
    arr = (ctypes.c_void_p * len(mgs))(*mgs)
    out = ctypes.c_void_p()
    _check(lib().bamg_batch_create(ctx, len(mgs), arr, ctypes.byref(out)), ctx)
    return out.value


def bamg_batch_destroy(bt):
    lib().bamg_batch_destroy(bt)


def bamg_batch_set_branches(ctx, bt, n: int):
    _check(lib().bamg_batch_set_branches(bt, int(n)), ctx)


def bamg_batch_get_branches(bt) -> int:
    n = ctypes.c_int()
    _check(lib().bamg_batch_get_branches(bt, ctypes.byref(n)), None)
    return n.value


def bamg_batch_cg_solve(ctx, bt, bs, xs, rtol: float, maxit: int, check: bool = True):
    """One graph launch solving every problem; returns (infos, loop iterations)."""
    n = len(bs)
    info = (bamg_cg_info * n)()
    loops = ctypes.c_int()
    st = lib().bamg_batch_cg_solve(bt, _ptr_array(bs), _ptr_array(xs) if xs is not None else None,
                                   float(rtol), int(maxit), info, ctypes.byref(loops))
    out = [{"status": st, "iterations": i.iterations, "converged": bool(i.converged), "rnorm": i.rnorm,
            "bnorm": i.bnorm, "true_rnorm": i.true_rnorm} for i in info]
    if check:
        _check(st, ctx)
    return out, loops.value


def bamg_batch_autotune(ctx, bt, bs, xs, rtol: float, maxit: int) -> float:
    ms = ctypes.c_float()
    _check(lib().bamg_batch_autotune(bt, _ptr_array(bs), _ptr_array(xs), float(rtol), int(maxit), ctypes.byref(ms)),
           ctx)
    return ms.value


def bamg_mg_set_smoother_weights(ctx, mg, level: int, w):
    _check(lib().bamg_mg_set_smoother_weights(mg, int(level), _ptr(w)), ctx)


def bamg_mg_set_lanes(ctx, mg, lanes: int):
    _check(lib().bamg_mg_set_lanes(mg, int(lanes)), ctx)


def bamg_mg_num_levels(mg) -> int:
    n = ctypes.c_int()
    _check(lib().bamg_mg_num_levels(mg, ctypes.byref(n)), None)
    return n.value


def bamg_mg_get_level(mg, level: int):
    A, P = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().bamg_mg_get_level(mg, int(level), ctypes.byref(A), ctypes.byref(P)), None)
    return A, (P if P.value else None)


def bamg_mg_get_restriction(mg, level: int):
    R = ctypes.c_void_p()
    _check(lib().bamg_mg_get_restriction(mg, int(level), ctypes.byref(R)), None)
    return R if R.value else None


def bamg_mg_get_level_scalars(ctx, mg, level: int) -> tuple[float, float]:
    lam, om = ctypes.c_double(), ctypes.c_double()
    _check(lib().bamg_mg_get_level_scalars(mg, int(level), ctypes.byref(lam), ctypes.byref(om)), ctx)
    return lam.value, om.value


def bamg_mg_get_dinv(ctx, mg, level: int, out):
    _check(lib().bamg_mg_get_dinv(mg, int(level), _ptr(out)), ctx)


def bamg_mg_destroy(mg):
    _check(lib().bamg_mg_destroy(mg), None)


# ------------------------------------------------- learned smoother weights
def bamg_mlp_num_params() -> int:
    n = ctypes.c_int()
    _check(lib().bamg_mlp_num_params(ctypes.byref(n)), None)
    return n.value


def bamg_mlp_create(ctx, seed: int = 0):
    h = ctypes.c_void_p()
    _check(lib().bamg_mlp_create(ctx, ctypes.c_uint64(seed), ctypes.byref(h)), ctx)
    return h


def bamg_mlp_destroy(mlp):
    _check(lib().bamg_mlp_destroy(mlp), None)


def bamg_mlp_get_params(ctx, mlp, out):
    _check(lib().bamg_mlp_get_params(mlp, _ptr(out)), ctx)


def bamg_mlp_set_params(ctx, mlp, params):
    _check(lib().bamg_mlp_set_params(mlp, _ptr(params)), ctx)


def bamg_mlp_train_epoch(ctx, mlp, X, t, perm, batch: int, lr: float, loss_sum):
    """One epoch over the rows perm (device int64) in batches, loss summed into loss_sum (device double)."""
    _check(lib().bamg_mlp_train_epoch(mlp, _ptr(X), _ptr(t), _ptr(perm), int(perm.numel()), int(batch),
                                      float(lr), _ptr(loss_sum)), ctx)


def bamg_mlp_forward(ctx, mlp, X, w):
    _check(lib().bamg_mlp_forward(mlp, _ptr(X), int(X.shape[0]), _ptr(w)), ctx)


def bamg_mlp_gradient(ctx, mlp, X, t, w_tmp, grad=None, loss=None):
    _check(lib().bamg_mlp_gradient(mlp, _ptr(X), _ptr(t), int(X.shape[0]), _ptr(w_tmp), _ptr(grad), _ptr(loss)), ctx)


def bamg_mlp_train_step(ctx, mlp, X, t, w_tmp, lr: float, loss=None):
    _check(lib().bamg_mlp_train_step(mlp, _ptr(X), _ptr(t), int(X.shape[0]), _ptr(w_tmp), ctypes.c_float(lr),
                                     _ptr(loss)), ctx)


def bamg_mg_block_features(ctx, mg, level: int, X):
    _check(lib().bamg_mg_block_features(mg, int(level), _ptr(X)), ctx)


def bamg_mg_smoother_targets(ctx, mg, B, k: int, targets):
    _check(lib().bamg_mg_smoother_targets(mg, _ptr(B), int(k), _ptr(targets)), ctx)


def bamg_mg_attach_mlp(ctx, mg, mlp):
    _check(lib().bamg_mg_attach_mlp(mg, mlp), ctx)


def bamg_mg_stationary(ctx, mg, b, x, its: int) -> list:
    out = (ctypes.c_double * (its + 1))()
    _check(lib().bamg_mg_stationary(mg, _ptr(b), _ptr(x), int(its), ctypes.byref(out)), ctx)
    return list(out)


def exported_symbols() -> list[str]:
    """Names of the C entry points this binding declares."""
    return sorted(list(_SIGS) + ["bamg_last_error", "bamg_mg_opts_default", "bamg_kernel_launches"])


# ---------------------------------------------------------- row-sharded operator
def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


class Halo:
    """Host-only partition plan of a square block pattern (no GPU needed)."""

    def __init__(self, rowptr, colidx, row_starts):
        rp, prp = _host(rowptr, np.int32)
        ci, pci = _host(colidx, np.int32)
        rs, prs = _host(row_starts, np.int64)
        self.nparts = len(rs) - 1
        h = ctypes.c_void_p()
        st = lib().bamg_halo_create(int(len(rp) - 1), prp, pci, int(self.nparts), prs, ctypes.byref(h))
        if st != BAMG_OK:
            raise BamgError(st, "bamg_halo_create")
        self.h = h

    def close(self):
        if self.h:
            lib().bamg_halo_destroy(self.h)
            self.h = None

    def info(self, p: int) -> tuple[int, int, int]:
        n, g, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().bamg_halo_part_info(self.h, int(p), ctypes.byref(n), ctypes.byref(g), ctypes.byref(nb)), None)
        return n.value, g.value, nb.value

    def pattern(self, p: int):
        """(rowptr, local colidx, global block index of each local block)."""
        n, _, nb = self.info(p)
        rp, prp = _host(np.zeros(n + 1), np.int32)
        ci, pci = _host(np.zeros(nb), np.int32)
        src, psrc = _host(np.zeros(nb), np.int64)
        _check(lib().bamg_halo_part_pattern(self.h, int(p), prp, pci, psrc), None)
        return rp, ci, src

    def ghosts(self, p: int):
        _, g, _ = self.info(p)
        gh, pgh = _host(np.zeros(g), np.int64)
        ow, pow_ = _host(np.zeros(g), np.int32)
        _check(lib().bamg_halo_part_ghosts(self.h, int(p), pgh, pow_), None)
        return gh, ow

    def sends(self, src: int, dst: int):
        cnt = ctypes.c_int64()
        _check(lib().bamg_halo_sends(self.h, int(src), int(dst), ctypes.byref(cnt), None), None)
        out, pout = _host(np.zeros(cnt.value), np.int64)
        _check(lib().bamg_halo_sends(self.h, int(src), int(dst), None, pout), None)
        return out


def bamg_sharded_create(ctx, A, P, row_starts):
    rs, prs = _host(row_starts, np.int64)
    sh, Ac = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().bamg_sharded_create(A, P, int(len(rs) - 1), prs, ctypes.byref(sh), ctypes.byref(Ac)), ctx)
    return sh, Ac


def bamg_sharded_spmv(ctx, sh, x, y):
    _check(lib().bamg_sharded_spmv(sh, _ptr(x), _ptr(y)), ctx)


def bamg_sharded_ptap(ctx, sh, A, P, Ac):
    _check(lib().bamg_sharded_ptap(sh, A, P, Ac), ctx)


def bamg_sharded_stats(sh) -> dict:
    o = bamg_shard_stats()
    _check(lib().bamg_sharded_stats(sh, ctypes.byref(o)), None)
    return {k: getattr(o, k) for k, _ in o._fields_}


def bamg_sharded_destroy(sh):
    _check(lib().bamg_sharded_destroy(sh), None)
