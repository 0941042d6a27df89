#!/usr/bin/env python3
"""Benchmark of the blocked SA-AMG reuse phase (3D elasticity, Q1 hexahedra).

One step = one reuse step of the hot path on fresh synthetic input: blocked
COO re-assembly of the perturbed operator, the Galerkin recompute
A_c = P^T A P on every level, the smoother refresh (block-diagonal inverses,
eigen-estimates, coarsest factorisation) and CG with the V(2,2) Chebyshev /
point-block Jacobi V-cycle to rtol 1e-8.  Default workload: 64^3 elements
(274,625 nodes, 823,875 dofs), 3 levels, FP64; the mixed-precision form is
measured on the same workload for comparison.

metric: algorithmic bytes of the step (byte model in
paper_2606_24748_gb300/bytes_model.py) / step time, in GB/s, over all ranks.
Multi-GPU runs are independent replicas (one problem per rank).
"""
import os
import sys

if "--impl" in sys.argv and "reference" in sys.argv:
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"

import argparse  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_24748_gb300 import bytes_model as bm  # noqa: E402
from workloads.elasticity import (Mesh, body_force, coo_indices, coo_values, element_scale,  # noqa: E402
                                  perturbation)

METRIC = "PtAP+V-cycle HBM GB/s; CG time to rtol 1e-8, FP64 vs mixed/learned"
# FP64 FMA peak from unit counts and the maximum clock: SMs x DFMA/clk/SM x
# flop/FMA x 2.07 GHz.  The roofline's denominator for FP64-bound kernels.  A
# pure-FMA probe (bamg_probe_fma_rate) is measured beside it: it stays below
# this figure (as does every FP64 kernel measured here), but also below what
# the fused Chebyshev step sustains at 127^3, so it is not itself the peak.
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
RTOL = 1e-8
MAXIT = 500
# DRAM bytes per launch of the dominant kernel from one ncu capture each
# (profiles/traffic_cheb_step_l0_64cubed_fp64.md, _mixed.md): the mean of the
# two pre-smoothing steps, the launches the timed steps sample.  Each carries
# a fingerprint of the kernel's source at capture time and is reported as
# null once it changes.  The source is device.cuh (the row products) and the
# span of cycle.cu from the block-diagonal apply through the end of the fused
# Chebyshev step.
TRAFFIC = {("cheb_step_l0", 64, False): (587.2e6, "f5d61c966d397dd7"),
           ("cheb_step_l0", 64, True): (307.6e6, "f5d61c966d397dd7")}
TRAFFIC_SOURCES = (("paper_2606_24748_gb300/csrc/device.cuh", None, None),
                   ("paper_2606_24748_gb300/csrc/cycle.cu", "__device__ __forceinline__ void dinv_apply",
                    "// r = b - A x; d = w Dinv r / theta"))


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--ne", type=int, default=None, help="elements per direction (default 64 for Q1, 32 for Q2)")
    p.add_argument("--element", default="q1", choices=["q1", "q2"],
                   help="q2: 27-node hexahedra (up to 125 blocks per row; 32^3 has the dofs of Q1 64^3)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    p.add_argument("--no-compare", action="store_true", help="skip the mixed-precision comparison run")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                   help="0: lanes per row from the size heuristic instead of timing (for runs under a profiler)")
    p.add_argument("--tune-cache", default="",
                   help="JSON file of the tuned lanes per level matrix: applied if it exists (no tuning), "
                        "else written after tuning; makes a run under a profiler use the timed run's choices")
    p.add_argument("--no-multi", action="store_true", help="skip the 16-right-hand-side measurement")
    p.add_argument("--no-batch", action="store_true", help="skip the 32-problem batch measurement")
    p.add_argument("--step-only", action="store_true",
                   help="only the timed reuse steps and their per-kernel table (for runs under a profiler)")
    p.add_argument("--no-large", action="store_true",
                   help="skip the 127^3 FP64-vs-mixed comparison (4 levels, 6.3 M dofs)")
    p.add_argument("--only", default="", choices=["", "multi", "batch", "peaks", "large", "ptap", "mis"],
                   help="run only that measurement (its own JSON object; used for profiling)")
    return p.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------- byte model
def level_sizes(B, mg):
    out = []
    nl = B.bamg_mg_num_levels(mg)
    for l in range(nl):
        A, P = B.bamg_mg_get_level(mg, l)
        a = B.bamg_bsr_info(A)
        p = B.bamg_bsr_info(P) if P is not None else None
        r = None
        if p is not None:
            r = {"nnzb": p["nnzb"], "nbr": p["nbc"], "nbc": p["nbr"], "bs_r": p["bs_c"], "bs_c": p["bs_r"]}
        out.append({"A": a, "P": p, "R": r})
    return out


def vcycles_per_solve(cg_its):
    """V-cycles of a PCG solve that took cg_its iterations: one before the
    first iteration and one after every iteration that did not converge
    (the last iteration's test ends the solve before its preconditioner)."""
    return cg_its


def step_bytes(levels, n_coo, cg_its, mixed, power_its=15):
    """Algorithmic bytes of one reuse step (see bytes_model)."""
    precond_applications = vcycles_per_solve(cg_its)
    s = 4 if mixed else 8
    A0 = levels[0]["A"]
    parts = {}
    parts["coo"] = bm.coo_bytes(n_coo, A0["nnzb"], 3, 3) + (A0["nnzb"] * 9 * 4 if mixed else 0)
    ptap = 0
    for l in range(len(levels) - 1):
        ptap += bm.ptap_bytes(levels[l]["A"], levels[l]["P"], levels[l + 1]["A"], s)
    parts["ptap"] = ptap
    refresh = 0
    for l in range(len(levels) - 1):
        a = levels[l]["A"]
        sa = 8 if (l == 0 or not mixed) else 4
        n, bs = a["nbr"], a["bs_r"]
        refresh += n * bs * bs * (sa + 8 + (4 if mixed else 0))                 # Dinv
        refresh += (power_its + 1) * bm.spmv_bytes(a["nnzb"], n, n, bs, bs, sa)  # eigen-estimate
    nc = levels[-1]["A"]["nbr"] * levels[-1]["A"]["bs_r"]
    npad = -(-nc // 32) * 32
    refresh += 3 * npad * npad * 8
    parts["refresh"] = refresh
    vc = sum(bm.vcycle_level_bytes(levels[l]["A"], levels[l]["P"], levels[l]["R"], s)
             for l in range(len(levels) - 1)) + bm.coarse_solve_bytes(nc)
    parts["vcycles"] = precond_applications * vc
    parts["cg"] = cg_its * bm.cg_iteration_bytes(A0) + 4 * 8 * A0["nbr"] * 3
    return sum(parts.values()), parts, vc


def level_count(ne, max_coarse_dofs=2100, order=1):
    """Levels of the hierarchy: coarsen (3x3x3 node aggregates) while a level has more dofs."""
    m, bs, n = order * ne + 1, 3, 1
    while bs * m ** 3 > max_coarse_dofs:
        m, bs, n = max(1, m // 3), 6, n + 1
    return n


def blocks_1d(ne, order):
    """Node couplings along one direction: every node couples to the nodes of
    the elements it belongs to (the block count of A is this number cubed)."""
    if order == 1:
        return 3 * ne + 1             # 27-point adjacency: 3m - 2, m = ne + 1
    m = 2 * ne + 1
    return sum(min(m - 1, i + (2 if i % 2 == 0 else 1)) - max(0, i - (2 if i % 2 == 0 else 1)) + 1 for i in range(m))


def workload_config(ne, precision, world, order=1):
    mesh = Mesh(ne, order)
    nl = level_count(ne, order=order)
    n_coo = mesh.nodes_per_element ** 2 * ne ** 3 + mesh.m ** 2
    nnzb = blocks_1d(ne, order) ** 3
    return {"workload": f"elasticity {ne}^3 Q{order} elements, {mesh.n_dofs} dofs, {nl}-level SA-AMG, reuse step "
                        f"(COO re-assembly, PtAP all levels, smoother refresh, PCG V(2,2) Chebyshev to rtol 1e-8), "
                        f"{'mixed FP32/FP64' if precision == 'mixed' else 'FP64'}",
            "elements": ne, "dofs": mesh.n_dofs, "levels": nl, "precision": precision,
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (value stream %.2f GB, fine operator %.2f GB)" % (
                n_coo * 72 / 1e9, nnzb * 76 / 1e9)}


# ---------------------------------------------------------------- our arm
def hierarchy_matrices(B, mg):
    out = []
    for l in range(B.bamg_mg_num_levels(mg)):
        A, P = B.bamg_mg_get_level(mg, l)
        out += [(f"A{l}", A), (f"P{l}", P), (f"R{l}", B.bamg_mg_get_restriction(mg, l))]
    return [(k, M) for k, M in out if M is not None]


def apply_tune_cache(B, ctx, mg, path):
    """Lanes of every level matrix, FP64 and FP32 copies (the product's and the
    smoothers' tuned choices), from `path` if it exists, else save them there."""
    if not path:
        return
    mats = hierarchy_matrices(B, mg)
    precs = (B.BAMG_FP64, B.BAMG_FP32)
    if os.path.exists(path):
        with open(path) as f:
            lanes = json.load(f)
        for k, M in mats:
            for p, v in zip(precs, lanes.get(k, [])):
                B.bamg_bsr_set_lanes_prec(ctx, M, p, v)
    else:
        with open(path, "w") as f:
            json.dump({k: [B.bamg_bsr_get_lanes_prec(M, p) for p in precs] for k, M in mats}, f)


class Workload:
    def __init__(self, B, torch, ne, nu, precision, n_inputs, seed0=1000, autotune=1, tune_cache="", order=1):
        self.B, self.torch = B, torch
        self.mesh = Mesh(ne, order)
        m = self.mesh
        self.ctx = B.bamg_ctx_create(torch.cuda.current_stream())
        self.bi, self.bj = coo_indices(m, "cuda")
        self.n_coo = int(self.bi.numel())
        self.A = B.bamg_bsr_create(self.ctx, 3, 3, m.n_nodes, m.n_nodes)
        B.bamg_bsr_coo_preallocate(self.ctx, self.A, self.bi, self.bj)
        v0 = coo_values(m, nu, element_scale(m), "cuda")
        B.bamg_bsr_coo_set_values(self.ctx, self.A, v0, 0)
        o = B.bamg_mg_opts_default()
        o.grid[0] = o.grid[1] = o.grid[2] = m.m
        o.precision = B.BAMG_FP32 if precision == "mixed" else B.BAMG_FP64
        o.autotune = 0 if (tune_cache and os.path.exists(tune_cache)) else autotune
        self.mg = B.bamg_mg_setup(self.ctx, self.A, m.coords(), m.dirichlet(), o)
        apply_tune_cache(B, self.ctx, self.mg, tune_cache)
        del v0
        # per-step inputs (perturbed operators), resident in HBM
        self.inputs = [coo_values(m, nu, element_scale(m, delta=perturbation(m.n_el, seed0 + k)), "cuda")
                       for k in range(n_inputs)]
        self.b = torch.from_numpy(body_force(m)).cuda()
        self.x = torch.zeros_like(self.b)
        self.levels = level_sizes(B, self.mg)
        self.mixed = precision == "mixed"

    def step(self, k):
        B = self.B
        B.bamg_bsr_coo_set_values(self.ctx, self.A, self.inputs[k % len(self.inputs)], 0)
        B.bamg_mg_update(self.ctx, self.mg)
        return B.bamg_cg_solve(self.ctx, self.mg, self.b, self.x, RTOL, MAXIT)

    def close(self):
        B = self.B
        B.bamg_mg_destroy(self.mg)
        B.bamg_bsr_destroy(self.A)
        B.bamg_ctx_destroy(self.ctx)


def slowest_rank_ms(torch, dist, ms_step, device="cuda"):
    """Per-step time of the slowest rank: every rank runs a replica, and the
    job ends with the last one (the maximum over ranks)."""
    if not dist:
        return ms_step
    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, bytes_step, ms_step):
    """Whole-job GB/s: the algorithmic bytes of all replicas over the slowest rank's step time."""
    return world * bytes_step / (ms_step / 1e3) / 1e9


def timed(torch, dist, fn, K):
    st = torch.cuda.current_stream()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    outs = [fn(k) for k in range(K)]
    e1.record(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return e0.elapsed_time(e1), outs


def run_ours(args):
    import torch
    from paper_2606_24748_gb300 import bamg as B

    if not os.path.exists(B.LIB_PATH):
        from paper_2606_24748_gb300.build import build
        build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    K, W = args.steps, args.warmup
    pctx = B.bamg_ctx_create(torch.cuda.current_stream())
    alu = alu_peaks(B, pctx) if not args.step_only else {"fp64_peak_tflops": round(FP64_PEAK_DERIVED_TFLOPS, 4),
                                                          "fp64_probe_tflops": None}
    B.bamg_ctx_destroy(pctx)
    stream_bytes = 72 * Mesh(args.ne, args.order).nodes_per_element ** 2 * args.ne ** 3
    wl = Workload(B, torch, args.ne, 0.3, args.precision, order=args.order,
                  n_inputs=min(K + W, 8, max(2, int(16e9 // stream_bytes))), autotune=args.autotune,
                  tune_cache=args.tune_cache)
    # inside the timed region only the roofline candidates are bracketed by
    # events (each bracket costs the kernel its overlap with its neighbours);
    # enabled before the warm-up, so that the CG graphs are captured with
    # them outside the timed region, and re-enabled after it (resets totals)
    B.bamg_ctx_profile_slots(wl.ctx, ROOFLINE_SLOTS)
    for k in range(W):
        wl.step(k)
    clocks = Clocks(local)
    B.bamg_ctx_profile_slots(wl.ctx, ROOFLINE_SLOTS)
    lib_setup_bytes, _ = B.bamg_device_memory(wl.ctx, reset_peak=True)
    launches0 = B.bamg_kernel_launches()
    clocks.start()
    ms, outs = timed(torch, dist, lambda k: wl.step(W + k), K)
    clk = clocks.stop()
    launches = B.bamg_kernel_launches() - launches0
    _, lib_peak_bytes = B.bamg_device_memory(wl.ctx)
    prof = {name: B.bamg_ctx_profile_read(wl.ctx, slot) for name, slot in B.PROF_SLOTS.items()}
    # every slot, in a separate untimed pass (the per-kernel breakdown)
    B.bamg_ctx_profile(wl.ctx, 1)
    for k in range(KERNEL_TABLE_STEPS):
        wl.step(W + K + k)
    table = {name: B.bamg_ctx_profile_read(wl.ctx, slot) for name, slot in B.PROF_SLOTS.items()}
    B.bamg_ctx_profile(wl.ctx, 0)
    its = [o["iterations"] for o in outs]
    ms_step = slowest_rank_ms(torch, dist, ms / K)
    per_step = [step_bytes(wl.levels, wl.n_coo, i, wl.mixed)[0] for i in its]
    bytes_step = float(np.mean(per_step))
    value = replica_value(world, bytes_step, ms_step)
    _, parts, vc_bytes = step_bytes(wl.levels, wl.n_coo, its[-1], wl.mixed)

    roof = roofline(wl, prof, B, alu)
    if roof is not None:
        # the single kernel with the largest share of the step in the all-slot
        # pass (the Galerkin stages counted together, as the roofline candidate
        # takes them; the slots that group several kernels are left out)
        shares = {k: table[k][0] for k in ("cheb_step_l0", "cheb_rinit_l0", "cg_ap", "coo", "cg_xr")}
        shares["ptap_l0"] = table["ptap_stage1_l0"][0] + table["ptap_stage2_l0"][0]
        roof["largest_kernel_in_all_slot_pass"] = max(shares, key=shares.get)
    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if wl.mixed else "f64",
        "data": f"synthetic: seeded Q{args.order} elasticity, per-element stiffness perturbed by U[-1%,1%] each step",
        "config": workload_config(args.ne, args.precision, world, args.order),
        "cg_iterations": its, "bytes_per_step": int(bytes_step),
        "bytes_parts": {k: int(v) for k, v in parts.items()},
        "gpu_launches": int(launches),
        "roofline": roof,
        "alu_peaks": alu,
        "clocks": clk,
        "kernel_ms": {k: {"total_ms": round(v[0], 3), "launches": v[1]} for k, v in table.items()},
        "kernel_ms_steps": KERNEL_TABLE_STEPS,
    }
    free_b, total_b = torch.cuda.mem_get_info()
    result["memory_gb"] = {
        "library_after_setup": round(lib_setup_bytes / 1e9, 3),
        "library_peak_in_timed_steps": round(lib_peak_bytes / 1e9, 3),
        "resident_inputs": round(torch.cuda.max_memory_allocated() / 1e9, 3),
        "device_used": round((total_b - free_b) / 1e9, 3),
        "note": "library = its stream-ordered pool allocations (hierarchy, plans, vectors); "
                "inputs = the value streams and vectors bench.py keeps resident through torch"}
    stor = B.bamg_bsr_storage(wl.A)
    result["fine_operator"] = {"lanes": B.bamg_bsr_get_lanes(wl.A), "stored_slots": stor["stored_slots"],
                               "padding": round(1 - B.bamg_bsr_info(wl.A)["nnzb"] / stor["stored_slots"], 4),
                               "rows_sorted": stor["rows_sorted"]}
    if args.step_only:
        wl.close()
        if dist:
            dist.destroy_process_group()
        return result if rank == 0 else None
    # phases (separate, untimed pass for the breakdown)
    result["phases_ms"] = phases(wl, torch, B)
    result["ptap_reuse"] = ptap_reuse(wl, torch, B)
    result["aggregation_graph"] = aggregation_graph(wl, torch, B)
    result["assembly"] = assembly_compare(wl, torch, B)
    result["sharded"] = sharded_compare(wl, torch, B)
    if rank == 0 and world == 1:
        result["mis_hierarchy"] = mis_hierarchy(wl, torch, B)
    if not args.no_e2e:
        result["e2e"] = e2e(wl, torch, B, dist, K, W, world, per_step)
    if not args.no_multi and args.precision == "fp64" and rank == 0 and world == 1:
        result["multi_rhs"] = multi_rhs(wl, torch, B, alu)
    if not args.no_batch and rank == 0 and world == 1:
        result["batch"] = batch_solve(torch, B)
    if rank == 0 and world == 1:
        result["mlp_training"] = mlp_training(torch, B)
    if not args.no_compare and args.precision == "fp64" and rank == 0 and world == 1:
        out0 = wl.step(0)
        x64 = wl.x.clone()
        result["fp64_input0"] = {"cg_iterations": out0["iterations"],
                                 "true_residual_rel": out0["true_rnorm"] / out0["bnorm"]}
        wl.close()
        wl = None
        result["mixed"] = compare_mixed(args, torch, B, x64, alu)
    if not args.no_large and args.order == 1 and args.ne < 127 and rank == 0 and world == 1:
        if wl is not None:
            wl.close()
            wl = None
        result["large"] = large_compare(torch, B, alu)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(ne=24 // args.order, order=args.order)
    if wl is not None:
        wl.close()
    if dist:
        dist.destroy_process_group()
    return result if rank == 0 else None


# Bracketed inside the timed region: the finest Chebyshev step through its
# sampling slot (the pre-smoothing pair of every cycle: one bracket per cycle,
# where the full slot takes two, and each bracket costs the kernel its
# programmatic overlap with its neighbours) and the finest Galerkin stages.
# The all-slot pass after the timed region shows which kernel dominates.
ROOFLINE_SLOTS = ("cheb_pre_l0", "ptap_stage1_l0", "ptap_stage2_l0")
KERNEL_TABLE_STEPS = 3  # steps of the untimed all-slot pass behind kernel_ms


def sources_fingerprint() -> str:
    import hashlib
    h = hashlib.sha256()
    for f, start, end in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = fh.read()
        if start is not None:
            i = text.index(start)
            text = text[i:text.index(end, i)]
        h.update(text.encode())
    return h.hexdigest()[:16]


def alu_peaks(B, ctx, reps=1, clocks_index=None):
    """FMA rates of the FP64 and FP32 pipes (TFLOP/s) from the library's probe
    (best of `reps` launches of >= 0.1 s), with the SM clock sampled during
    each when clocks_index is given, and the derived FP64 peak."""
    out = {}
    for name, prec in (("fp64", B.BAMG_FP64), ("fp32", B.BAMG_FP32)):
        clk = Clocks(clocks_index) if clocks_index is not None else None
        if clk:
            clk.start()
        out[f"{name}_probe_tflops"] = round(max(B.bamg_probe_fma_rate(ctx, prec) for _ in range(reps)), 4)
        if clk:
            out[f"{name}_probe_clocks"] = clk.stop()
    out["fp64_peak_tflops"] = round(FP64_PEAK_DERIVED_TFLOPS, 4)
    out["how"] = ("peak: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz; probe: bamg_probe_fma_rate, 8 independent "
                  "FMA chains per thread at full occupancy, one launch of >= 0.1 s timed with CUDA events")
    return out


def roofline(wl, prof, B, alu):
    """Dominant kernel of the timed region: algorithmic bytes/flops per launch / mean duration."""
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    lv = wl.levels
    A0 = lv[0]["A"]
    s = 4 if wl.mixed else 8
    n, nnzb = A0["nbr"], A0["nnzb"]
    cand = {}
    fl = 2 * nnzb * 9 + n * (2 * 9 + 8)
    if prof.get("cheb_pre_l0", (0, 0))[1]:
        # the sampled pre-smoothing pair: step 0 with a next direction, then the last pre step
        bts = (bm.cheb_step_bytes(nnzb, n, 3, s, True) + bm.cheb_step_bytes(nnzb, n, 3, s, False)) / 2
        cand["cheb_step_l0"] = (prof["cheb_pre_l0"], bts, fl)
    elif prof["cheb_step_l0"][1]:
        # launches alternate between has_next (pre-smoothing step 0, post step 0) and the last pre step
        bts = (2 * bm.cheb_step_bytes(nnzb, n, 3, s, True) + bm.cheb_step_bytes(nnzb, n, 3, s, False)) / 3
        cand["cheb_step_l0"] = (prof["cheb_step_l0"], bts, fl)
    if prof["ptap_stage1_l0"][1]:
        P0, A1 = lv[0]["P"], lv[1]["A"]
        bts = bm.ptap_bytes(A0, P0, A1, s)
        cand["ptap_l0"] = ((prof["ptap_stage1_l0"][0] + prof["ptap_stage2_l0"][0], prof["ptap_stage1_l0"][1]), bts,
                           None)
    if prof["cg_ap"][1]:
        bts = bm.spmv_bytes(nnzb, n, n, 3, 3, 8) + 8 * 3 * n
        cand["cg_ap"] = (prof["cg_ap"], bts, 2 * nnzb * 9 + 6 * n)
    if not cand:
        return None
    name = max(cand, key=lambda k: cand[k][0][0])
    (tot, cnt), bts, fl = cand[name]
    avg_s = tot / cnt / 1e3
    gbs = bts / avg_s / 1e9
    traffic = None
    rec = TRAFFIC.get((name, wl.mesh.ne, wl.mixed))
    if rec is not None and rec[1] == sources_fingerprint():
        traffic = int(rec[0])
    out = {"kernel": name, "launches": cnt, "avg_ms": round(avg_s * 1e3, 4), "bytes_per_launch": int(bts),
           "sample": ("pre-smoothing steps of every cycle (2 of the 3 launches per cycle)"
                      if name == "cheb_step_l0" and prof.get("cheb_pre_l0", (0, 0))[1] else "every launch"),
           "hbm_achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3), "traffic": traffic}
    peak64 = alu["fp64_peak_tflops"]
    fp64_bound = (not wl.mixed) and fl is not None and (fl / (peak64 * 1e12)) > (bts / (hbm * 1e9))
    if fp64_bound:
        tf = fl / avg_s / 1e12
        out.update({"bound": "alu", "achieved": round(tf, 4), "peak": peak64,
                    "unit": "TFLOP/s", "frac": round(tf / peak64, 3),
                    "peak_source": "FP64 FMA pipe from unit counts and the maximum clock (152 x 2 DFMA/clk x "
                                   "2 flop x 2.07 GHz); no FP64 rate measured on this part exceeds it",
                    "probe_tflops": alu["fp64_probe_tflops"]})
    else:
        out.update({"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(gbs / hbm, 3), "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"})
    return out


def ptap_reuse(wl, torch, B):
    """Finest-level Galerkin product with a fresh symbolic plan (symbolic plus
    the first numeric pass) against the numeric pass alone on a cached plan."""
    A0, P0 = B.bamg_mg_get_level(wl.mg, 0)
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan, Ac = B.bamg_ptap_symbolic(wl.ctx, A0, P0)
    B.bamg_ptap_numeric(wl.ctx, plan, A0, P0, Ac)
    torch.cuda.synchronize()
    both = (time.perf_counter() - t0) * 1e3
    ts = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        B.bamg_ptap_numeric(wl.ctx, plan, A0, P0, Ac)
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    B.bamg_ptap_destroy(plan)
    B.bamg_bsr_destroy(Ac)
    num = sorted(ts)[2]
    return {"level": 0, "symbolic_plus_numeric_ms": round(both, 2), "numeric_ms": round(num, 3),
            "ratio": round(both / num, 1),
            "timing": "symbolic + first numeric: host clock around synchronised calls; numeric: CUDA events, median of 5"}


def mis_hierarchy(wl, torch, B, eps=0.02, seed=1):
    """The same operator with the hierarchy built from device MIS aggregates
    of the block strength graph (instead of 3x3x3 node cubes): cold setup
    time, level sizes, and the reuse step's update and CG to rtol 1e-8 (CUDA
    events, median of 3) against the geometric hierarchy's."""
    m = wl.mesh
    o = B.bamg_mg_opts_default()
    o.grid[0] = o.grid[1] = o.grid[2] = m.m
    o.aggregation = B.BAMG_AGG_MIS
    o.mis_eps = eps
    o.mis_seed = seed
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mg = B.bamg_mg_setup(wl.ctx, wl.A, m.coords(), m.dirichlet(), o)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    try:
        out = {"eps": eps, "seed": seed, "setup_s": round(setup_s, 2), "levels": []}
        for l in range(B.bamg_mg_num_levels(mg)):
            info = B.bamg_bsr_info(B.bamg_mg_get_level(mg, l)[0])
            out["levels"].append({"block_rows": info["nbr"], "blocks": info["nnzb"]})
        for name, h in (("mis", mg), ("geometric", wl.mg)):
            res = {}
            B.bamg_mg_update(wl.ctx, h)
            B.bamg_cg_solve(wl.ctx, h, wl.b, wl.x, RTOL, MAXIT)
            t_up = sorted(event_ms(torch, lambda: B.bamg_mg_update(wl.ctx, h), 1) for _ in range(3))[1]
            t_cg = sorted(event_ms(torch, lambda: res.__setitem__(
                "o", B.bamg_cg_solve(wl.ctx, h, wl.b, wl.x, RTOL, MAXIT)), 1) for _ in range(3))[1]
            out[name] = {"update_ms": round(t_up, 3), "cg_ms": round(t_cg, 3), "cg_iterations": res["o"]["iterations"],
                         "true_residual_rel": res["o"]["true_rnorm"] / res["o"]["bnorm"]}
        return out
    finally:
        B.bamg_mg_destroy(mg)


def sharded_compare(wl, torch, B, nparts=4):
    """The finest level as a row-sharded operator of `nparts` contiguous parts
    run in turn on this GPU: SpMV and numeric Galerkin product through the
    parts (halo gathers, cached P_oth, per-part products, reduce) against the
    unsharded kernels, CUDA events, median of 5, and the partition's
    communication profile (what a multi-GPU run would move)."""
    A0, P0 = B.bamg_mg_get_level(wl.mg, 0)
    n = B.bamg_bsr_info(A0)["nbr"]
    starts = np.array([round(k * n / nparts) for k in range(nparts + 1)], dtype=np.int64)
    t0 = time.perf_counter()
    sh, Ac = B.bamg_sharded_create(wl.ctx, A0, P0, starts)
    build_s = time.perf_counter() - t0
    plan, Ac1 = B.bamg_ptap_symbolic(wl.ctx, A0, P0)
    x = torch.randn(n * 3, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    try:
        B.bamg_sharded_ptap(wl.ctx, sh, A0, P0, Ac)
        B.bamg_ptap_numeric(wl.ctx, plan, A0, P0, Ac1)

        def med(fn):
            return sorted(event_ms(torch, fn, 1) for _ in range(5))[2]
        out = {"parts": nparts, "build_s": round(build_s, 2),
               "spmv_ms": round(med(lambda: B.bamg_sharded_spmv(wl.ctx, sh, x, y)), 4),
               "spmv_unsharded_ms": round(med(lambda: B.bamg_bsr_spmv(wl.ctx, A0, x, y)), 4),
               "ptap_ms": round(med(lambda: B.bamg_sharded_ptap(wl.ctx, sh, A0, P0, Ac)), 4),
               "ptap_unsharded_ms": round(med(lambda: B.bamg_ptap_numeric(wl.ctx, plan, A0, P0, Ac1)), 4)}
        v1 = torch.empty(B.bamg_bsr_info(Ac)["nnzb"] * 36, dtype=torch.float64, device="cuda")
        v2 = torch.empty_like(v1)
        B.bamg_bsr_get_values(wl.ctx, Ac, v1)
        B.bamg_bsr_get_values(wl.ctx, Ac1, v2)
        out["ptap_rel_diff"] = float(torch.linalg.norm(v1 - v2) / torch.linalg.norm(v2))
        out.update(B.bamg_sharded_stats(sh))
        return out
    finally:
        B.bamg_ptap_destroy(plan)
        B.bamg_bsr_destroy(Ac1)
        B.bamg_sharded_destroy(sh)
        B.bamg_bsr_destroy(Ac)


def assembly_compare(wl, torch, B):
    """Blocked COO assembly (sorted gather-sum) against element-by-element
    assembly (an FP64 atomic per contribution) of the same value streams:
    CUDA events, median of 5, each repetition on the next resident stream
    (1.2 GB at 64^3, larger than L2).  The operator is left as blocked COO
    assembled it from the first stream."""
    st = torch.cuda.current_stream()
    info = B.bamg_bsr_info(wl.A)

    def timeit(fn):
        ts = []
        for r in range(5):
            v = wl.inputs[(r + 1) % len(wl.inputs)]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn(v)
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[2]

    t_coo = timeit(lambda v: B.bamg_bsr_coo_set_values(wl.ctx, wl.A, v, 0))
    B.bamg_bsr_coo_scatter_values(wl.ctx, wl.A, wl.inputs[0], 0)   # builds the per-entry slot map
    t_ebe = timeit(lambda v: B.bamg_bsr_coo_scatter_values(wl.ctx, wl.A, v, 0))
    n = info["nnzb"] * 9
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    B.bamg_bsr_coo_scatter_values(wl.ctx, wl.A, wl.inputs[0], 0)
    B.bamg_bsr_get_values(wl.ctx, wl.A, x)
    B.bamg_bsr_coo_set_values(wl.ctx, wl.A, wl.inputs[0], 0)
    B.bamg_bsr_get_values(wl.ctx, wl.A, y)
    diff = float(torch.linalg.norm(x - y) / torch.linalg.norm(y))
    nb = bm.coo_bytes(wl.n_coo, info["nnzb"], 3, 3)
    return {"entries": wl.n_coo, "blocks": info["nnzb"], "blocked_coo_ms": round(t_coo, 3),
            "element_by_element_ms": round(t_ebe, 3), "speedup": round(t_ebe / t_coo, 2),
            "blocked_coo_gbs": round(nb / t_coo / 1e6, 1), "rel_diff": diff}


def aggregation_graph(wl, torch, B, eps=0.01, seed=1):
    """Cold-setup graph phase on the finest operator: block-norm strength graph
    and device MIS aggregation, host clock around synchronised calls (each
    call waits for the stream itself), best of 3."""
    info = B.bamg_bsr_info(wl.A)
    n = info["nbr"]
    rp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(info["nnzb"], dtype=torch.int32, device="cuda")
    agg = torch.empty(n, dtype=torch.int32, device="cuda")
    tg, tm = [], []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ne = B.bamg_strength_graph(wl.ctx, wl.A, eps, rp, col)
        t1 = time.perf_counter()
        n_agg, rounds = B.bamg_mis_aggregate(wl.ctx, n, rp, col, seed, agg)
        t2 = time.perf_counter()
        tg.append((t1 - t0) * 1e3)
        tm.append((t2 - t1) * 1e3)
    return {"eps": eps, "seed": seed, "vertices": n, "edges": ne, "aggregates": n_agg, "luby_rounds": rounds,
            "strength_graph_ms": round(min(tg), 3), "mis_aggregation_ms": round(min(tm), 3)}


def phases(wl, torch, B):
    st = torch.cuda.current_stream()
    out = {}
    for name, fn in (("coo_assembly", lambda: B.bamg_bsr_coo_set_values(wl.ctx, wl.A, wl.inputs[0], 0)),
                     ("mg_update", lambda: B.bamg_mg_update(wl.ctx, wl.mg)),
                     ("cg_solve", lambda: B.bamg_cg_solve(wl.ctx, wl.mg, wl.b, wl.x, RTOL, MAXIT))):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        out[name] = round(e0.elapsed_time(e1), 3)
    return out


def e2e(wl, torch, B, dist, K, W, world, per_step):
    """Same step through the C ABI with host buffers: the value stream and b
    copied from pinned host memory, the solution read back, every step.  The
    next step's inputs are copied on a second stream while the current step
    solves (two device buffers of each); each step's copy is inside the timed
    region.  The main stream issues no host-to-device copy of its own, so no
    small copy of it queues behind the value stream on a copy engine, and the
    value stream moves in pieces of about 128 MB."""
    n_host = min(2 if wl.n_coo * 72 < 4e9 else 1, len(wl.inputs))
    host_in = [t.cpu().pin_memory() for t in wl.inputs[:n_host]]
    host_b = wl.b.cpu().pin_memory()
    host_x = torch.empty_like(host_b).pin_memory()
    dev_in = [torch.empty_like(wl.inputs[0]) for _ in range(2)]
    dev_b = [torch.empty_like(wl.b) for _ in range(2)]
    piece = max(1, (128 << 20) // 8)
    copy_stream = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    main = torch.cuda.current_stream()
    state = {"n": 0, "spans": [], "waits": [], "host_s": 0.0}

    def fetch(k):
        src, dst = host_in[k % n_host].view(-1), dev_in[k % 2].view(-1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(copy_stream):
            e0.record(copy_stream)
            dev_b[k % 2].copy_(host_b, non_blocking=True)
            for i in range(0, src.numel(), piece):
                dst[i:i + piece].copy_(src[i:i + piece], non_blocking=True)
            e1.record(copy_stream)
            ready[k % 2].record(copy_stream)
        state["spans"].append((e0, e1))

    def run(k, last):
        t0 = time.perf_counter()
        if k == 0 or state["n"] == 0:
            fetch(k)
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(main)
        main.wait_event(ready[k % 2])
        w1.record(main)
        state["waits"].append((w0, w1))
        B.bamg_bsr_coo_set_values(wl.ctx, wl.A, dev_in[k % 2], 0)
        if not last:
            copy_stream.wait_stream(main)   # the other buffers' last readers were the previous step
            fetch(k + 1)
        state["host_s"] += time.perf_counter() - t0
        B.bamg_mg_update(wl.ctx, wl.mg)
        out = B.bamg_cg_solve(wl.ctx, wl.mg, dev_b[k % 2], wl.x, RTOL, MAXIT)
        host_x.copy_(wl.x, non_blocking=True)
        state["n"] += 1
        return out

    def step(k):
        return run(k, k + 1 >= K)

    for k in range(min(W, 2)):
        state["n"] = 0
        run(k, True)
    state["n"] = 0
    state["spans"], state["waits"], state["host_s"] = [], [], 0.0
    ms, outs = timed(torch, dist, step, K)
    ms_step = slowest_rank_ms(torch, dist, ms / K)
    copy_ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in state["spans"]]))
    wait_ms = [w0.elapsed_time(w1) for w0, w1 in state["waits"]]
    its = [o["iterations"] for o in outs]
    bytes_step = float(np.mean([step_bytes(wl.levels, wl.n_coo, i, wl.mixed)[0] for i in its]))
    h2d = int(host_in[0].numel() * 8 + host_b.numel() * 8)
    return {"value": round(replica_value(world, bytes_step, ms_step), 2), "unit": "GB/s",
            "ms_per_step": round(ms_step, 4),
            "h2d_bytes_per_step": h2d,
            "h2d_ms_per_step": round(copy_ms, 3),
            "h2d_gbs": round(h2d / copy_ms / 1e6, 1),
            # where an end-to-end step loses time against the device step: the
            # main stream waiting for the step's inputs (the first step's copy
            # is never overlapped), and the host enqueueing the copies
            "copy_wait_ms": {"first_step": round(wait_ms[0], 3),
                             "later_steps_mean": round(float(np.mean(wait_ms[1:])), 3) if K > 1 else None},
            "host_enqueue_ms_per_step": round(state["host_s"] * 1e3 / K, 3),
            "overlap": "next step's value stream and b copied on a second stream during the current step",
            "d2h_bytes_per_step": int(host_x.numel() * 8)}


def event_ms(torch, fn, reps):
    """Device time of fn() per call (CUDA events on the current stream)."""
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def multi_rhs(wl, torch, B, alu, k=16):
    """k seeded N(0,1) right-hand sides (clamped dofs zeroed) on the workload's
    operator: blocked SpMM against k SpMVs, and the k-column PCG against k
    single-vector solves, in the FP64 form and the mixed form."""
    from workloads.elasticity import gaussian_rhs
    m = wl.mesh
    n = m.n_dofs
    a = wl.levels[0]["A"]
    Bh = np.stack([gaussian_rhs(m, s) for s in range(k)], axis=1)
    Bd = torch.from_numpy(Bh).cuda()
    X = torch.zeros_like(Bd)
    out = {"k": k, "rhs": "N(0,1) seeds 0..%d, clamped dofs zeroed" % (k - 1)}
    # SpMM vs k SpMVs on the fine operator (operator 0.55 GB FP64: larger than L2)
    cols = [Bd[:, j].contiguous() for j in range(k)]
    ys = [torch.empty_like(c) for c in cols]
    for prec, s, name in ((B.BAMG_FP64, 8, "fp64"), (B.BAMG_FP32, 4, "fp32")):
        if prec == B.BAMG_FP32:
            Xs, Ys = Bd.float(), torch.empty(n, k, dtype=torch.float32, device="cuda")
            cs = [c.float() for c in cols]
            yss = [y.float() for y in ys]
        else:
            Xs, Ys, cs, yss = Bd, X, cols, ys
        f_mm = lambda: B.bamg_bsr_spmm(wl.ctx, wl.A, Xs, Ys, k, prec)  # noqa: E731
        f_mv = lambda: [B.bamg_bsr_spmv(wl.ctx, wl.A, c, y, prec) for c, y in zip(cs, yss)]  # noqa: E731
        for _ in range(3):
            f_mm()
            f_mv()
        t_mm = event_ms(torch, f_mm, 10)
        t_mv = event_ms(torch, f_mv, 3)
        byts = bm.spmm_bytes(a["nnzb"], a["nbr"], a["nbc"], 3, 3, k, s)
        flops = bm.spmv_flops(a["nnzb"], 3, 3) * k
        out[f"spmm_{name}"] = {"ms": round(t_mm, 4), "gbs": round(byts / t_mm / 1e6, 1),
                               "tflops": round(flops / t_mm / 1e9, 4),
                               "k_spmv_ms": round(t_mv, 4), "speedup_vs_k_spmv": round(t_mv / t_mm, 2)}
        if prec == B.BAMG_FP64:
            out[f"spmm_{name}"]["frac_fp64_peak"] = round(flops / t_mm / 1e9 / alu["fp64_peak_tflops"], 3)
    # k-column PCG vs k single solves: FP64 hierarchy (the workload's) and a mixed one
    ctx, A = wl.ctx, wl.A
    o = B.bamg_mg_opts_default()
    o.grid[0] = o.grid[1] = o.grid[2] = m.m
    o.precision = B.BAMG_FP32
    mg32 = B.bamg_mg_setup(ctx, A, m.coords(), m.dirichlet(), o)
    for name, mg in (("fp64", wl.mg), ("mixed", mg32)):
        B.bamg_mg_update(ctx, mg)
        B.bamg_cg_solve_multi(ctx, mg, Bd, X, k, RTOL, MAXIT)   # warm-up (allocates, captures)
        B.bamg_cg_solve(ctx, mg, cols[0], ys[0], RTOL, MAXIT)
        res = {}
        t_blk = event_ms(torch, lambda: res.__setitem__("i", B.bamg_cg_solve_multi(ctx, mg, Bd, X, k, RTOL, MAXIT)), 2)
        infos = res["i"]
        seq = []
        t_seq = event_ms(torch, lambda: seq.append([B.bamg_cg_solve(ctx, mg, c, y, RTOL, MAXIT) for c, y in zip(cols, ys)]), 1)
        its_b = [i["iterations"] for i in infos]
        its_s = [o["iterations"] for o in seq[-1]]
        worst = max(i["true_rnorm"] / i["bnorm"] for i in infos)
        diff = max(float(torch.linalg.norm(X[:, j] - ys[j]) / torch.linalg.norm(ys[j])) for j in range(k))
        out[f"cg_{name}"] = {"block_ms": round(t_blk, 3), "sequential_ms": round(t_seq, 3),
                             "speedup": round(t_seq / t_blk, 2), "iterations_block": its_b,
                             "iterations_sequential": its_s, "max_true_residual_rel": worst,
                             "max_solution_rel_diff_block_vs_single": diff}
    B.bamg_mg_destroy(mg32)
    return out


def batch_solve(torch, B, seed=7, count=32):
    """A batch of uneven problems (elements per direction U{16..40}, Poisson
    ratio U[0.2, 0.45], each with its own hierarchy and context, unit body
    force): one graph launch solving all of them to rtol 1e-8 (branch count
    autotuned) against the same solves one after another."""
    from workloads.elasticity import batch_problems
    probs = []
    for ne, nu in batch_problems(seed, count):
        m = Mesh(ne)
        ctx = B.bamg_ctx_create(torch.cuda.current_stream())
        bi, bj = coo_indices(m, "cuda")
        A = B.bamg_bsr_create(ctx, 3, 3, m.n_nodes, m.n_nodes)
        B.bamg_bsr_coo_preallocate(ctx, A, bi, bj)
        B.bamg_bsr_coo_set_values(ctx, A, coo_values(m, nu, element_scale(m), "cuda"), 0)
        o = B.bamg_mg_opts_default()
        o.grid[0] = o.grid[1] = o.grid[2] = m.m
        mg = B.bamg_mg_setup(ctx, A, m.coords(), m.dirichlet(), o)
        b = torch.from_numpy(body_force(m)).cuda()
        probs.append({"ne": ne, "nu": nu, "ctx": ctx, "A": A, "mg": mg, "b": b, "x": torch.zeros_like(b),
                      "levels": level_sizes(B, mg), "n_coo": int(bi.numel())})
    lctx = B.bamg_ctx_create(torch.cuda.current_stream())
    bt = B.bamg_batch_create(lctx, [p["mg"] for p in probs])
    bs, xs = [p["b"] for p in probs], [p["x"] for p in probs]
    tune_ms = B.bamg_batch_autotune(lctx, bt, bs, xs, RTOL, MAXIT)
    res = {}
    B.bamg_batch_cg_solve(lctx, bt, bs, xs, RTOL, MAXIT)
    l0 = B.bamg_kernel_launches()
    t_batch = event_ms(torch, lambda: res.__setitem__("r", B.bamg_batch_cg_solve(lctx, bt, bs, xs, RTOL, MAXIT)), 3)
    kernels = (B.bamg_kernel_launches() - l0) // 3
    infos, loops = res["r"]
    seq = []
    for p in probs:
        B.bamg_cg_solve(p["ctx"], p["mg"], p["b"], p["x"], RTOL, MAXIT)
    t_seq = event_ms(torch, lambda: seq.append([B.bamg_cg_solve(p["ctx"], p["mg"], p["b"], p["x"], RTOL, MAXIT)
                                                for p in probs]), 3)
    its = [i["iterations"] for i in infos]
    same = all(i["iterations"] == o["iterations"] for i, o in zip(infos, seq[-1]))
    nbytes = 0
    for p, it in zip(probs, its):
        _, parts, _ = step_bytes(p["levels"], p["n_coo"], it, False)
        nbytes += parts["vcycles"] + parts["cg"]
    out = {"problems": count, "seed": seed,
           "dofs_total": int(sum(p["b"].numel() for p in probs)),
           "levels": [len(p["levels"]) for p in probs],
           "branches": B.bamg_batch_get_branches(bt), "autotune_best_ms": round(tune_ms, 3),
           "batch_ms": round(t_batch, 3), "sequential_ms": round(t_seq, 3),
           "speedup": round(t_seq / t_batch, 2),
           "gbs_batch": round(nbytes / t_batch / 1e6, 1), "gbs_sequential": round(nbytes / t_seq / 1e6, 1),
           "graph_launches_per_solve": 1, "loop_iterations": loops, "kernels_per_solve": int(kernels),
           "iterations": its, "iterations_equal_sequential": same,
           "max_true_residual_rel": max(i["true_rnorm"] / i["bnorm"] for i in infos)}
    B.bamg_batch_destroy(bt)
    B.bamg_ctx_destroy(lctx)
    for p in probs:
        B.bamg_mg_destroy(p["mg"])
        B.bamg_bsr_destroy(p["A"])
        B.bamg_ctx_destroy(p["ctx"])
    return out


def mlp_training(torch, B):
    """One training step of the learned-weight MLP (fused forward and
    backward on the tensor cores, gradient reduction, Adam) on 2^20 seeded
    feature rows: rows/s and its BF16 tensor rate against the measured burst
    peak (the kernels are timed alone)."""
    from paper_2606_24748_gb300 import learned
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    mlp = B.bamg_mlp_create(ctx, 12345)
    try:
        out = learned.train_step_rate(ctx, mlp)
    finally:
        B.bamg_mlp_destroy(mlp)
        B.bamg_ctx_destroy(ctx)
    peak = float(measured_peaks().get("bf16_tflops", 1932.6))
    out["tensor_frac_of_bf16_peak"] = round(out["tflops"] / peak, 4)
    out["bf16_peak_tflops"] = peak
    return out


def compare_mixed(args, torch, B, x64, alu, ne=None, steps=None):
    """Time to rtol 1e-8 of the mixed-precision form on the same workload, its
    roofline, and its solution against the FP64 form's for the same input."""
    ne = args.ne if ne is None else ne
    K = max(3, min(args.steps, 10)) if steps is None else steps
    stream_bytes = 72 * Mesh(ne, args.order).nodes_per_element ** 2 * ne ** 3
    wl = Workload(B, torch, ne, 0.3, "mixed", n_inputs=min(K, max(2, int(16e9 // stream_bytes))),
                  order=args.order)
    B.bamg_ctx_profile_slots(wl.ctx, ROOFLINE_SLOTS)   # CG graphs captured with the slots in the warm-up
    for k in range(3):
        wl.step(k)
    B.bamg_ctx_profile_slots(wl.ctx, ROOFLINE_SLOTS)
    ms, outs = timed(torch, None, lambda k: wl.step(k), K)
    prof = {name: B.bamg_ctx_profile_read(wl.ctx, slot) for name, slot in B.PROF_SLOTS.items()}
    B.bamg_ctx_profile_slots(wl.ctx, [])
    ph = phases(wl, torch, B)
    its = [o["iterations"] for o in outs]
    bytes_step = float(np.mean([step_bytes(wl.levels, wl.n_coo, i, True)[0] for i in its]))
    res = {"ms_per_step": round(ms / K, 4), "steps": K, "cg_iterations": its,
           "value": round(bytes_step / (ms / K / 1e3) / 1e9, 2), "unit": "GB/s", "phases_ms": ph,
           "roofline": roofline(wl, prof, B, alu),
           "true_residual_rel": outs[-1]["true_rnorm"] / outs[-1]["bnorm"]}
    if x64 is not None:
        out0 = wl.step(0)
        d = torch.linalg.norm(wl.x - x64) / torch.linalg.norm(x64)
        res["input0"] = {"cg_iterations": out0["iterations"],
                         "true_residual_rel": out0["true_rnorm"] / out0["bnorm"],
                         "solution_rel_diff_vs_fp64": float(d.item())}
    wl.close()
    return res


def large_compare(torch, B, alu, ne=127, steps=5, warmup=3):
    """The 127^3-element problem (128^3 nodes, 6,291,456 dofs, 4 levels): the
    FP64 reuse step against the mixed one (FP32 V-cycle under FP64 CG), each
    timed over `steps` steps after `warmup`, with the rooflines of their
    dominant kernels and the mixed solution's distance from the FP64 one for
    the same input (both recompute the true residual at exit)."""
    args = parse_args_for_test(["--ne", str(ne), "--steps", str(steps)])
    stream_bytes = 72 * 64 * ne ** 3
    wl = Workload(B, torch, ne, 0.3, "fp64", n_inputs=min(steps, max(2, int(16e9 // stream_bytes))))
    B.bamg_ctx_profile_slots(wl.ctx, ROOFLINE_SLOTS)   # CG graphs captured with the slots in the warm-up
    for k in range(warmup):
        wl.step(k)
    B.bamg_ctx_profile_slots(wl.ctx, ROOFLINE_SLOTS)
    ms, outs = timed(torch, None, lambda k: wl.step(k), steps)
    prof = {name: B.bamg_ctx_profile_read(wl.ctx, slot) for name, slot in B.PROF_SLOTS.items()}
    B.bamg_ctx_profile_slots(wl.ctx, [])
    its = [o["iterations"] for o in outs]
    bytes_step = float(np.mean([step_bytes(wl.levels, wl.n_coo, i, False)[0] for i in its]))
    fp64 = {"ms_per_step": round(ms / steps, 4), "steps": steps, "cg_iterations": its,
            "value": round(bytes_step / (ms / steps / 1e3) / 1e9, 2), "unit": "GB/s",
            "roofline": roofline(wl, prof, B, alu),
            "true_residual_rel": outs[-1]["true_rnorm"] / outs[-1]["bnorm"]}
    out0 = wl.step(0)
    x64 = wl.x.clone()
    fp64["input0"] = {"cg_iterations": out0["iterations"], "true_residual_rel": out0["true_rnorm"] / out0["bnorm"]}
    levels = len(wl.levels)
    wl.close()
    mixed = compare_mixed(args, torch, B, x64, alu, ne=ne, steps=steps)
    return {"workload": f"elasticity {ne}^3 Q1 elements, {3 * (ne + 1) ** 3} dofs, {levels}-level SA-AMG, "
                        f"reuse step, FP64 against mixed FP32/FP64",
            "fp64": fp64, "mixed": mixed,
            "mixed_speedup": round(fp64["ms_per_step"] / mixed["ms_per_step"], 3)}


# ---------------------------------------------------------------- CPU baseline (oracle)
def oracle_levels(h2):
    levels = []
    for L in h2.levels:
        a = {"nnzb": L.A.nnzb, "nbr": L.A.nbr, "nbc": L.A.nbc, "bs_r": L.A.bs_r, "bs_c": L.A.bs_c}
        p = r = None
        if L.P is not None:
            p = {"nnzb": L.P.nnzb, "nbr": L.P.nbr, "nbc": L.P.nbc, "bs_r": L.P.bs_r, "bs_c": L.P.bs_c}
            r = {"nnzb": L.P.nnzb, "nbr": L.P.nbc, "nbc": L.P.nbr, "bs_r": L.P.bs_c, "bs_c": L.P.bs_r}
        levels.append({"A": a, "P": p, "R": r})
    return levels


class OracleSample:
    """The oracle's reuse step on a smaller mesh of the same problem: cold
    setup once (untimed), then per step COO assembly of a perturbed operator,
    the Galerkin products on every level, the smoother refresh and PCG."""

    def __init__(self, ne, order=1):
        from oracle import multigrid as omg
        from oracle.assembly import coo_assemble_blocks
        self.omg, self.coo = omg, coo_assemble_blocks
        self.m = m = Mesh(ne, order)
        bi, bj = coo_indices(m)
        self.bi, self.bj = bi.numpy(), bj.numpy()
        v0 = coo_values(m, 0.3, element_scale(m)).numpy()
        self.h = omg.setup(coo_assemble_blocks(m.n_nodes, m.n_nodes, 3, 3, self.bi, self.bj, v0),
                           m.coords(), m.dirichlet(), m.grid)
        self.b = body_force(m)

    def step(self, seed):
        """Returns (seconds, algorithmic bytes, iterations)."""
        from oracle import krylov
        m, omg = self.m, self.omg
        v = coo_values(m, 0.3, element_scale(m, delta=perturbation(m.n_el, seed))).numpy()
        t0 = time.perf_counter()
        A = self.coo(m.n_nodes, m.n_nodes, 3, 3, self.bi, self.bj, v)
        h2 = omg.update(self.h, A)
        x, its, info = krylov.pcg(h2.levels[0].As, self.b, lambda r: omg.vcycle(h2, r), RTOL, MAXIT)
        dt = time.perf_counter() - t0
        nbytes = step_bytes(oracle_levels(h2), int(self.bi.size), its, False)[0]
        return dt, nbytes, its


def cpu_baseline(steps=8, ne=24, order=1):
    s = OracleSample(ne, order)
    tot_t, tot_b = 0.0, 0.0
    for k in range(steps):
        dt, nb, _ = s.step(seed=k + 1)
        tot_t += dt
        tot_b += nb
    out = {"value": round(tot_b / tot_t / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"{steps} oracle reuse steps (COO assembly, Galerkin products, smoother refresh, "
                     f"PCG to 1e-8) of the same elasticity problem at {ne}^3 Q{order} elements "
                     f"({3 * (order * ne + 1) ** 3} dofs), single-threaded scipy/numpy on the host",
           "seconds": round(tot_t, 2)}
    try:
        out["all_cores"] = cpu_baseline_all_cores(ne, order)
    except Exception as e:  # the single-thread figure above stands on its own
        out["all_cores"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def _oracle_replica(ne, order, steps, seed0, barrier, queue):
    """One single-threaded oracle process of the all-core baseline.  A failure
    breaks the barrier, so that no sibling waits for it, and is reported."""
    try:
        s = OracleSample(ne, order)
        barrier.wait(timeout=300)
        t0, nb = time.time(), 0.0
        for k in range(steps):
            nb += s.step(seed=seed0 + k)[1]
        queue.put((t0, time.time(), nb))
    except Exception as e:
        try:
            barrier.abort()
        except Exception:
            pass
        queue.put(("error", f"{type(e).__name__}: {e}", 0.0))


def cpu_baseline_all_cores(ne, order, steps=2, max_procs=64):
    """The same oracle steps in one single-threaded process per host core (a
    spawned pool: the parent already holds a CUDA context), timed from the
    common start to the last finish."""
    import multiprocessing as mpm
    procs = max(1, min(os.cpu_count() or 1, max_procs))
    ctx = mpm.get_context("spawn")
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        barrier, queue = ctx.Barrier(procs), ctx.Queue()
        ps = [ctx.Process(target=_oracle_replica, args=(ne, order, steps, 1 + 100 * i, barrier, queue))
              for i in range(procs)]
        for p in ps:
            p.start()
        try:
            res = [queue.get(timeout=600) for _ in ps]
        finally:
            for p in ps:
                p.join(timeout=30)
                if p.is_alive():
                    p.terminate()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    errors = [r[1] for r in res if r[0] == "error"]
    if errors:
        raise RuntimeError(errors[0])
    t0, t1 = min(r[0] for r in res), max(r[1] for r in res)
    return {"value": round(sum(r[2] for r in res) / (t1 - t0) / 1e9, 4), "unit": "GB/s", "cores": procs,
            "sample": f"{procs} single-threaded oracle processes, {steps} reuse steps each, same problem",
            "seconds": round(t1 - t0, 2)}


def run_reference(args):
    """The oracle on the host cores (one thread), each step one reuse step of
    the same problem on a 24^3-element sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    K, W = args.steps, args.warmup
    ne = 24 // args.order   # the same dofs for Q1 and Q2
    sample = OracleSample(ne, args.order)
    for k in range(W):
        sample.step(seed=100 + k)
    tt, tb = 0.0, 0.0
    for k in range(K):
        dt, nb, _ = sample.step(seed=k + 1)
        tt += dt
        tb += nb
    value = tb / tt / 1e9
    desc = (f"oracle reuse step (COO assembly, Galerkin products, smoother refresh, PCG to 1e-8) per step "
            f"on a {ne}^3-element Q{args.order} sample ({3 * (args.order * ne + 1) ** 3} dofs) of the same problem, "
            f"single-threaded")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": round(tt / K * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": f"synthetic: seeded Q{args.order} elasticity, per-element stiffness perturbed by U[-1%,1%] each step",
            "config": dict(workload_config(ne, args.precision, args.gpus, args.order),
                           sample_of=workload_config(args.ne, args.precision, args.gpus, args.order)["workload"],
                           l2="host run (no GPU cache)",
                           note="the oracle runs a smaller mesh of the same problem; GB/s of algorithmic "
                                "bytes is compared across the two sizes"),
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "kind": "oracle", "cores": 1, "sample": desc},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_only(args):
    """One of the extra measurements on its own (for profiling runs)."""
    import torch
    from paper_2606_24748_gb300 import bamg as B
    if not os.path.exists(B.LIB_PATH):
        from paper_2606_24748_gb300.build import build
        build()
    if args.only == "batch":
        return {"only": "batch", "batch": batch_solve(torch, B)}
    if args.only in ("ptap", "mis"):
        wl = Workload(B, torch, args.ne, 0.3, "fp64", n_inputs=1)
        if args.only == "ptap":
            out = {"only": "ptap", "ptap_reuse": ptap_reuse(wl, torch, B)}
        else:
            out = {"only": "mis", "mis_hierarchy": mis_hierarchy(wl, torch, B)}
        wl.close()
        return out
    if args.only in ("peaks", "large"):
        ctx = B.bamg_ctx_create(torch.cuda.current_stream())
        alu = alu_peaks(B, ctx, reps=10 if args.only == "peaks" else 1, clocks_index=0)
        B.bamg_ctx_destroy(ctx)
        if args.only == "peaks":
            return {"only": "peaks", "alu_peaks": alu}
        return {"only": "large", "alu_peaks": alu, "large": large_compare(torch, B, alu, ne=args.ne, steps=args.steps)}
    ctx = B.bamg_ctx_create(torch.cuda.current_stream())
    alu = alu_peaks(B, ctx)
    B.bamg_ctx_destroy(ctx)
    wl = Workload(B, torch, args.ne, 0.3, "fp64", n_inputs=1)
    out = {"only": "multi", "multi_rhs": multi_rhs(wl, torch, B, alu)}
    wl.close()
    return out


def finish_args(args):
    args.order = 2 if args.element == "q2" else 1
    if args.ne is None:
        args.ne = 64 // args.order
    return args


def parse_args_for_test(argv):
    """The parsed command line for ``argv`` (tests call the arms directly)."""
    saved = sys.argv
    try:
        sys.argv = ["bench.py", *argv]
        return finish_args(parse())
    finally:
        sys.argv = saved


def main():
    args = finish_args(parse())
    if args.only and args.impl == "ours":
        print(json.dumps(run_only(args)), flush=True)
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
