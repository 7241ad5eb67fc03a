#!/usr/bin/env python
"""Benchmark of the deflated-CG hot path on one GB300 (or N replicas).

Workload (default): 2D unit square, 1024 x 1024 Q1 pseudo-stress elements
(N = 4,186,116 unknowns, BSR 4x4, 9 blocks per row), nu = 1, right-hand side
uniform[-1, 1) from seed 0, solved to true relative residual 1e-8 (FP64) for
dt in {1e-6, 1e-5, 1e-4} (dt at most ~100 h^2, where deflation pays; plain CG
is reported over the whole sweep 1e-6..1e-1). One step = one complete
deflated-CG solve (W-cycle multigrid with RAS 8x8 cores, overlap 2, 2+2
smoothing steps, 4 levels; FCG(1) outer; fixed inner tolerance c_F = 0.01)
at the next dt of the sweep. The headline runs the W-cycle in FP32 and
everything else in FP64 (--precision fp64 runs all in FP64).

Printed: one JSON line (rank 0) with the contract keys, plus "roofline"
(dominant kernel class, measured live with CUDA events during the timed
steps), "cpu_baseline" (the FP64 oracle on the host: one SpMV and one
W-cycle at this size, composed with the iteration counts of the timed
solves), "e2e" (same solves through the host-array entry point, copies
included), "clocks" (nvidia-smi samples during the timed region) and
"extra" (per-dt iterations and times, plain CG, kernel breakdown).

--impl reference times the oracle alone on a bounded sample of the same
workload (one SpMV and one W-cycle per step), scaled to seconds per solve
with the outer/inner iteration counts this bench measured on GB300.
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

DTS = [1e-6, 1e-5, 1e-4]          # timed deflated-CG solves (one dt per step, cycling)
DTS_CG = [1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1]   # plain CG reported over the whole sweep
WORKLOAD = ("2D unit square 1024x1024 Q1 pseudo-stress (4 comps/node, N=4,186,116, BSR 4x4 FP64), nu=1, "
            "deflated CG at dt in {1e-6,1e-5,1e-4} (one dt per step, cycling), RHS uniform[-1,1) seed 0, "
            "tol 1e-8 true residual; DCG: FCG(1), c_F=0.01, W-cycle (levels autotuned), RAS 8x8 cores overlap 2, m1=m2=2; "
            "plain CG over dt 1e-6..1e-1 reported in extra")
# Outer / in-iteration W-cycle counts per dt of this workload (mixed precision),
# measured on GB300 by this bench; the parity tests hold device and oracle
# counts within +-2 at sizes the oracle finishes. Used only to scale the
# oracle's per-kernel timings to seconds per solve in the reference arm.
REF_COUNTS = {1e-6: (34, 170), 1e-5: (106, 530), 1e-4: (335, 1675)}

FP32_LANES_PER_SM = 128
NUM_SMS = 152


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# --------------------------------------------------------------------------- clocks


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- distributed


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_time(local_ms, steps, ws, torch, device="cuda"):
    """Whole-job timing of N replicas: the slowest rank's time (MAX over
    ranks; every rank gets it) and the job's seconds per solve, i.e. that
    time over the steps * N solves all ranks completed."""
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    elapsed_ms = float(t.item())
    return elapsed_ms, elapsed_ms / 1e3 / (steps * ws)


# --------------------------------------------------------------------------- oracle timing


def oracle_kernel_times(n=1024, P=8, o=2, dt=1e-6, levels=2):
    """Time the FP64 oracle at the bench size: one BSR SpMV and one W-cycle
    (single thread). Returns seconds for each and the sample description."""
    from oracle import fem, mg
    from paper_2606_13429_gb300 import inputs
    asm = fem.assemble(2, n, dt)
    A = asm.matrix().tocsr()
    V = fem.V_matrix(asm.mesh)
    H = mg.Hierarchy(2, n, mg.inner_matrix(V, A), mg.MGOptions(patch=P, overlap=o, m1=2, m2=2, max_levels=levels))
    x = inputs.rhs(0, asm.mesh.n_unknowns)
    g = inputs.rhs(1, asm.mesh.n_nodes)
    t0 = time.perf_counter()
    y = A @ x
    t_spmv = time.perf_counter() - t0
    t0 = time.perf_counter()
    z = H.wcycle(g, np.zeros_like(g))
    t_wc = time.perf_counter() - t0
    del y, z
    return t_spmv, t_wc


def compose_solve_time(t_spmv, t_wc, counts, n_unknowns):
    """Seconds per solve from per-kernel times: per outer iteration two SpMVs
    and its W-cycles, plus about ten vector passes; the f_D and reconstruction
    inner solves add ~2 inner solves of W-cycles and two SpMVs."""
    t_vec = 10 * n_unknowns * 8 / 5e9  # ~5 GB/s single-thread numpy streaming
    total = 0.0
    for outer, cycles in counts:
        inner = cycles / max(1, outer)
        total += outer * (2 * t_spmv + t_vec) + cycles * t_wc + 2 * (inner * t_wc + t_spmv)
    return total / len(counts)


# --------------------------------------------------------------------------- main arm


def run_ours(args):
    global DTS
    if args.dts:  # profiling runs: a subset of the step sizes
        DTS = list(args.dts)
    import torch
    import torch.distributed as dist
    from paper_2606_13429_gb300 import build as B
    from paper_2606_13429_gb300 import dcg, inputs

    ws, rank, local = dist_init()
    if ws > 1:
        dist.init_process_group("nccl")
        # replicas: the headline solve only; the single-GPU characterisations
        # (plain CG sweep, FP64 solver, batched, matrix-free, 3D) stay at N = 1
        args.skip_cg = args.skip_fp64 = args.skip_batched = args.skip_mf = args.skip_3d = True
    torch.cuda.set_device(local)
    B.build()
    dcg.load()
    prec = dcg.DCG_MIXED if args.precision == "mixed" else dcg.DCG_FP64
    opts = dcg.options(patch=8, overlap=2, m1=2, m2=2, max_levels=4, precision=prec, inner_rule=dcg.DCG_INNER_FIXED,
                       c=0.01, recurrence=dcg.DCG_FCG1)
    n = args.n
    probs = {}
    for dt in DTS:
        probs[dt] = dcg.dcg_assemble(2, n, dt)
    # autotune the hierarchy depth on the first problem: time one inner solve
    # to 1e-10 for each candidate level count and keep the fastest
    tune = {}
    g = torch.from_numpy(inputs.rhs(1, probs[DTS[0]].n_nodes)).cuda()
    invs = [dcg.DCG_INV_FP32, dcg.DCG_INV_BF16] if prec == dcg.DCG_MIXED else [dcg.DCG_INV_FP32]
    for levels, inv in [(lv, iv) for lv in args.levels for iv in invs]:
        o = dcg.options(patch=8, overlap=2, m1=2, m2=2, max_levels=levels, precision=prec,
                        inner_rule=dcg.DCG_INNER_FIXED, c=0.01, recurrence=dcg.DCG_FCG1, ras_inverse=inv)
        try:
            dcg.dcg_setup(probs[DTS[0]], o)
        except dcg.DCGError:
            continue
        best = None
        for _ in range(3):
            z = torch.zeros_like(g)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dcg.dcg_mg_solve(probs[DTS[0]], g, z, 1e-10)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            best = t if best is None else min(best, t)
        tune[(levels, inv)] = best
    best_levels, best_inv = min(tune, key=tune.get)
    opts.max_levels = best_levels
    opts.ras_inverse = best_inv
    for dt in DTS:
        dcg.dcg_setup(probs[dt], opts)
    N = probs[DTS[0]].N
    f = torch.from_numpy(inputs.rhs(0, N)).cuda()
    x = torch.zeros_like(f)
    stream = torch.cuda.current_stream()

    def step(k, record=None):
        dt = DTS[k % len(DTS)]
        x.zero_()
        st = dcg.dcg_solve(probs[dt], f, x, tol=1e-8, max_it=args.max_it)
        if record is not None:
            record.append((dt, st))
        return st

    # warm-up: every class timed, to find the dominant one
    for p in probs.values():
        dcg.dcg_profile_enable(p, dcg.PROF_CLASSES)
    warm = []
    for k in range(args.warmup):
        step(k, warm)
    breakdown = {c: {"ms": 0.0, "launches": 0, "flops": 0.0, "bytes": 0.0} for c in dcg.PROF_CLASSES}
    for p in probs.values():
        r = dcg.dcg_profile_read(p)
        for c in dcg.PROF_CLASSES:
            for key in breakdown[c]:
                breakdown[c][key] += r[c][key]
    dominant = max(breakdown, key=lambda c: breakdown[c]["ms"])
    for p in probs.values():
        dcg.dcg_profile_enable(p, [dominant])

    # timed region
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = dcg.dcg_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    timed = []
    for k in range(args.steps):
        step(k, timed)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = dcg.dcg_kernel_launches() - launches0
    clk = clocks.stop() if rank == 0 else None
    elapsed_ms, value = job_time(ev0.elapsed_time(ev1), args.steps, ws, torch, device="cuda")
    dom = {"ms": 0.0, "launches": 0, "flops": 0.0, "bytes": 0.0}
    for p in probs.values():
        r = dcg.dcg_profile_read(p)[dominant]
        for key in dom:
            dom[key] += r[key]
        dcg.dcg_profile_enable(p, [])
    ok = all(st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8 for _, st in timed)

    # end to end: host arrays in pinned memory, copies inside the timed region
    f_h = torch.from_numpy(inputs.rhs(0, N)).pin_memory()
    x_h = torch.zeros(N, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e0 = time.perf_counter()
    e2e_stats = []
    for k in range(args.steps):
        dt = DTS[k % len(DTS)]
        x_h.zero_()
        e2e_stats.append(dcg.dcg_solve_host(probs[dt], f_h, x_h, tol=1e-8, max_it=args.max_it))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    _, e2e_s = job_time((time.perf_counter() - e0) * 1e3, args.steps, ws, torch, device="cuda")

    # plain CG, FP64, at each dt (reported, outside the timed region)
    extra = {"per_dt": {}}
    if not args.skip_cg:
        copt = dcg.options(deflate=0)
        for dt in DTS_CG:
            pc = dcg.dcg_assemble(2, n, dt)
            dcg.dcg_setup(pc, copt)
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = dcg.dcg_solve(pc, f, x, tol=1e-8, max_it=args.max_it)
            torch.cuda.synchronize()
            extra["per_dt"].setdefault(str(dt), {})["plain_cg"] = {
                "s": time.perf_counter() - t0, "outer_its": st["outer_its"], "true_relres": st["true_relres"]}
            pc.close()
    if args.dcg_sweep:
        # deflated CG at the large step sizes (thousands of outer iterations;
        # not part of the default run)
        sweep_opts = dcg.options(**{k: getattr(opts, k) for k, _ in opts._fields_})
        sweep_opts.c = args.sweep_c if args.sweep_c else opts.c
        for dt in [d for d in DTS_CG if d not in DTS]:
            pd = dcg.dcg_assemble(2, n, dt)
            dcg.dcg_setup(pd, sweep_opts)
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = dcg.dcg_solve(pd, f, x, tol=1e-8, max_it=args.max_it)
            torch.cuda.synchronize()
            extra["per_dt"].setdefault(str(dt), {})["dcg"] = {
                "s": time.perf_counter() - t0, "outer_its": st["outer_its"], "total_mg_cycles": st["total_mg_cycles"],
                "restarts": st["restarts"], "true_relres": st["true_relres"], "status": st["status"],
                "c_F": sweep_opts.c}
            pd.close()
    for dt, st in timed:
        extra["per_dt"].setdefault(str(dt), {})["dcg"] = {
            "s": st["solve_ms"] / 1e3, "outer_its": st["outer_its"], "total_mg_cycles": st["total_mg_cycles"],
            "avg_inner": round(st["avg_inner"], 2), "true_relres": st["true_relres"], "restarts": st["restarts"]}

    # SpMV bandwidth on this operator (FP64, plain product)
    p0 = probs[DTS[0]]
    dcg.dcg_profile_enable(p0, ["spmv"])
    y = torch.empty_like(f)
    for _ in range(20):
        dcg.dcg_spmv(p0, f, y)
    sp = dcg.dcg_profile_read(p0)["spmv"]
    dcg.dcg_profile_enable(p0, [])
    # all-FP64 deflated CG at the smallest dt (W-cycle in FP64 too)
    if not args.skip_fp64:
        pf = dcg.dcg_assemble(2, n, DTS[0])
        fp64_levels = best_levels
        while True:  # FP64 coarse panels need twice the shared memory: deepen if needed
            try:
                dcg.dcg_setup(pf, dcg.options(patch=8, overlap=2, m1=2, m2=2, max_levels=fp64_levels,
                                              precision=dcg.DCG_FP64))
                break
            except dcg.DCGError:
                fp64_levels += 1
                if fp64_levels > 8:
                    raise
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = dcg.dcg_solve(pf, f, x, tol=1e-8, max_it=args.max_it)
        torch.cuda.synchronize()
        extra["dcg_all_fp64_dt1e-6"] = {"s": time.perf_counter() - t0, "outer_its": st["outer_its"], "mg_levels": fp64_levels,
                                        "total_mg_cycles": st["total_mg_cycles"], "true_relres": st["true_relres"]}
        pf.close()
    for key, skip, fn in [("batched", args.skip_batched, batched_extra), ("matrix_free_3d_256", args.skip_mf, mf_extra),
                          ("bsr_3d_128", args.skip_3d, bsr3d_extra)]:
        if skip:
            continue
        try:
            extra[key] = fn(args, opts, dcg, inputs, torch)
        except Exception as exc:  # an extra must not cost the headline line
            extra[key] = {"error": "%s: %s" % (type(exc).__name__, exc)}
        torch.cuda.empty_cache()
    extra["spmv_fp64"] = {"GB_per_s": sp["bytes"] / (sp["ms"] / 1e3) / 1e9, "ms": sp["ms"] / max(1, sp["launches"])}
    extra["kernel_breakdown_warmup_ms"] = {c: round(v["ms"], 3) for c, v in breakdown.items()}

    peaks, peak_src = load_peaks()
    roof = roofline(dominant, dom, peaks, peak_src, tensor=(best_inv == dcg.DCG_INV_BF16))

    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        t_spmv, t_wc = oracle_kernel_times(n, levels=best_levels)
        counts = [(st["outer_its"], st["iter_mg_cycles"]) for _, st in timed]
        cpu = {"value": compose_solve_time(t_spmv, t_wc, counts, N), "unit": "s/solve", "cores": 1,
               "kind": "oracle",
               "sample": "FP64 oracle at 1024^2 on the host: one BSR SpMV (%.3f s) and one W-cycle (%.2f s), "
                         "single thread, composed with the outer/inner iteration counts of the timed solves"
                         % (t_spmv, t_wc)}

    if rank == 0:
        line = {
            "metric": "time-to-1e-8 true residual, deflated CG (W-cycle MG + RAS inner), 2D Q1 pseudo-stress 1024^2, "
                      "dt in {1e-6,1e-5,1e-4}",
            "value": value, "unit": "s/solve", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64 outer CG, f32 W-cycle" if prec == dcg.DCG_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": "replicas" if ws > 1 else "single GPU",
                       "mg_levels": best_levels, "dts": DTS,
                       "ras_products": "tcgen05 BF16 x BF16 -> FP32" if best_inv == dcg.DCG_INV_BF16 else "FP32 SIMT",
                       "autotune_inner_solve_s": {"levels=%d,%s" % (k[0], "bf16" if k[1] else "fp32"): v
                                                  for k, v in tune.items()},
                       "l2": "inputs larger than L2 (BSR matrix 1.2 GB per dt)", "precision": args.precision,
                       "all_converged": ok},
            "e2e": {"value": e2e_s, "unit": "s/solve", "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": N * 8},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
            "extra": extra,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def _timed(torch, fn, reps):
    """Mean ms of fn() over reps calls, CUDA events on the current stream."""
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def mf_extra(args, opts, dcg, inputs, torch):
    """Matrix-free 3D operator on 256^3 hexahedra (149,232,375 unknowns),
    lognormal(0,1) element viscosity, dt = 1e-5: the product in FP32 and FP64
    arithmetic, and one deflated-CG solve (FP32 products and W-cycle, FP64
    outer recurrences and true residual)."""
    n, dt = 256, 1e-5
    nu = inputs.nu_elements(4, n ** 3)
    prob = dcg.dcg_assemble(3, n, dt, nu_elem=nu, matrix_free=True)
    N, nn = prob.N, prob.n_nodes
    x = torch.from_numpy(inputs.rhs(0, N)).cuda()
    y = torch.empty_like(x)
    flops = 2.0 * (243 + 243 + 216) * nn
    by = (72 + 72 + 8) * nn
    out = {"n": n, "unknowns": N, "dt": dt, "nu": "lognormal(0,1) per element"}
    for name, prec in [("fp32", dcg.DCG_MIXED), ("fp64", dcg.DCG_FP64)]:
        ms = _timed(torch, lambda: dcg.dcg_spmv_prec(prob, x, y, prec), 10 if prec == dcg.DCG_MIXED else 3)
        out["spmv_" + name] = {"ms": ms, "TFLOP_per_s": flops / (ms * 1e-3) / 1e12,
                               "GB_per_s": by / (ms * 1e-3) / 1e9}
    if not args.skip_mf_solve:
        o = dcg.options(patch=4, overlap=1, m1=2, m2=2, max_levels=4, precision=dcg.DCG_MIXED,
                        ras_inverse=dcg.DCG_INV_BF16)
        t0 = time.perf_counter()
        dcg.dcg_setup(prob, o)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        xs = torch.zeros_like(x)
        t0 = time.perf_counter()
        st = dcg.dcg_solve(prob, x, xs, tol=1e-8, max_it=args.max_it)
        torch.cuda.synchronize()
        out["dcg_mixed"] = {"s": time.perf_counter() - t0, "setup_s": setup_s, "levels": prob.levels,
                            "outer_its": st["outer_its"], "total_mg_cycles": st["total_mg_cycles"],
                            "restarts": st["restarts"], "true_relres": st["true_relres"], "status": st["status"]}
    prob.close()
    return out


def bsr3d_extra(args, opts, dcg, inputs, torch):
    """Assembled 3D operator on 128^3 hexahedra (18,458,712 unknowns, BSR
    9x9), dt = 1e-4: deflated CG with the FP32 W-cycle and BF16 RAS inverses
    on tensor cores against the all-FP64 solver."""
    n, dt = 128, 1e-4
    prob = dcg.dcg_assemble(3, n, dt)
    f = torch.from_numpy(inputs.rhs(0, prob.N)).cuda()
    out = {"n": n, "unknowns": prob.N, "dt": dt}
    for name, prec, inv in [("mixed_bf16", dcg.DCG_MIXED, dcg.DCG_INV_BF16), ("fp64", dcg.DCG_FP64, dcg.DCG_INV_FP32)]:
        dcg.dcg_setup(prob, dcg.options(patch=4, overlap=1, m1=2, m2=2, max_levels=4, precision=prec,
                                        ras_inverse=inv))
        x = torch.zeros_like(f)
        t0 = time.perf_counter()
        st = dcg.dcg_solve(prob, f, x, tol=1e-8, max_it=args.max_it)
        torch.cuda.synchronize()
        out[name] = {"s": time.perf_counter() - t0, "outer_its": st["outer_its"],
                     "total_mg_cycles": st["total_mg_cycles"], "true_relres": st["true_relres"],
                     "status": st["status"]}
    y = torch.empty_like(f)
    sp_ms = _timed(torch, lambda: dcg.dcg_spmv(prob, f, y), 10)
    out["spmv_fp64_ms"] = sp_ms
    out["spmv_fp64_GB_per_s"] = (prob.nnzb * 81 * 8 + prob.nnzb * 4 + 2 * prob.N * 8) / (sp_ms * 1e-3) / 1e9
    prob.close()
    return out


def batched_extra(args, opts, dcg, inputs, torch):
    """Independent 2D problems (n log-uniform in [64, 512], dt log-uniform in
    [1e-6, 1e-1]), 4 right-hand sides each: one batched call against the
    same solves one after another on one stream."""
    nrhs = args.batched_rhs
    plist = inputs.batched_problems(11, args.batched_problems)
    probs, fs = [], []
    tuned, choices = {}, {}
    t_tune = time.perf_counter()
    for p, (nb, dtb) in enumerate(plist):
        pr = dcg.dcg_assemble(2, nb, dtb)
        f0 = torch.from_numpy(inputs.rhs(5, pr.N, p=p, r=0)).cuda()
        if args.batched_no_tune:
            dcg.dcg_setup(pr, opts)
        elif nb not in tuned:
            # the library's autotuner (hierarchy depth, RAS tile and overlap,
            # inverse precision) once per mesh size: the inner system does not
            # depend on dt, so one problem of each size stands for the others
            best, _ = dcg.dcg_autotune(pr, f0, opts, inner_tol=1e-10, reps=2)
            tuned[nb] = best
        else:
            dcg.dcg_setup(pr, tuned[nb])
        if nb in tuned:
            b = tuned[nb]
            key = "levels=%d,P=%d,o=%d,%s" % (b.max_levels, b.patch, b.overlap,
                                              "bf16" if b.ras_inverse == dcg.DCG_INV_BF16 else "fp32")
            choices[key] = choices.get(key, 0) + 1
        probs.append(pr)
        fs.append(f0)
        for r in range(1, nrhs):
            fs.append(torch.from_numpy(inputs.rhs(5, pr.N, p=p, r=r)).cuda())
    torch.cuda.synchronize()
    t_tune = time.perf_counter() - t_tune
    xs = [torch.zeros_like(f) for f in fs]
    # one outer iteration per problem, untimed: builds every W-cycle graph
    dcg.dcg_solve_batched(probs, 1, fs[::nrhs], xs[::nrhs], tol=1e-8, max_it=1)
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    code, stats = dcg.dcg_solve_batched(probs, nrhs, fs, xs, tol=1e-8, max_it=args.max_it)
    torch.cuda.synchronize()
    t_batched = time.perf_counter() - t0
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = [dcg.dcg_solve(probs[k // nrhs], fs[k], xs[k], tol=1e-8, max_it=args.max_it) for k in range(len(fs))]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    unknowns = sum(pr.N for pr in probs) * nrhs
    out = {"problems": len(probs), "rhs_per_problem": nrhs, "unknowns_total": unknowns,
           "n_range": [min(n for n, _ in plist), max(n for n, _ in plist)],
           "batched_s": t_batched, "sequential_s": t_seq, "speedup": t_seq / t_batched,
           "batched_unknowns_per_s": unknowns / t_batched,
           "all_converged": code == dcg.DCG_OK and all(st["true_relres"] <= 1e-8 for st in stats),
           "same_iterations_as_sequential": all(a["outer_its"] == b["outer_its"] for a, b in zip(stats, seq)),
           "setup_and_autotune_s": t_tune, "autotuned_options_per_problem": choices or "not tuned"}
    for pr in probs:
        pr.close()
    return out


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_13429_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def roofline(dominant, dom, peaks, peak_src, tensor=False):
    """Roofline of the dominant kernel class over the timed region."""
    secs = dom["ms"] / 1e3
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tr = json.load(fh)
        ent = tr.get(dominant)
        if ent and ent.get("source_hash") == kernel_source_hash():
            traffic = ent["dram_bytes_per_launch"]
    except Exception:
        pass
    if dominant == "inner_res" and secs > 0:
        # FP64 stencil residual: bound by FP64 issue (ncu: FP64 pipe ~83% busy),
        # against the nominal GB300 FP64 rate (2 FMA / clock / SM)
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = NUM_SMS * 4 * mhz * 1e6 / 1e12
        achieved = dom["flops"] / secs / 1e12
        return {"kernel": dominant, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": "FP64 FMA: 152 SMs x 2 FMA x 2 flops x %.0f MHz (nominal 1.26 TFLOP/s)" % mhz,
                "launches": dom["launches"], "algorithmic_flops_per_launch": dom["flops"] / max(1, dom["launches"])}
    if dominant in ("spmv", "vec", "ras_update", "transfer", "inner_res") or secs <= 0:
        achieved = dom["bytes"] / secs / 1e9 if secs > 0 else 0.0
        peak = peaks["hbm_gbs"]
        return {"kernel": dominant, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src + " copy bandwidth",
                "launches": dom["launches"],
                "algorithmic_bytes_per_launch": dom["bytes"] / max(1, dom["launches"])}
    if dominant == "ras_solve" and tensor and secs > 0:
        # BF16 inverse x BF16 residual products on tcgen05: the sustained
        # measured BF16 peak (the kernel runs inside a long step)
        peak = peaks["bf16_tflops_sustained"]
        achieved = dom["flops"] / secs / 1e12
        return {"kernel": dominant, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": peak_src + " bf16 sustained (cuBLAS GEMM)",
                "launches": dom["launches"], "algorithmic_flops_per_launch": dom["flops"] / max(1, dom["launches"])}
    # FP32 SIMT products (RAS patch inverses, coarse passes): plain ALU bound
    mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = NUM_SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    achieved = dom["flops"] / secs / 1e12
    return {"kernel": dominant, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flops x %.0f MHz (max SM clock)" % mhz,
            "launches": dom["launches"], "algorithmic_flops_per_launch": dom["flops"] / max(1, dom["launches"])}


# --------------------------------------------------------------------------- reference arm


def run_reference(args):
    ws, rank, local = dist_init()
    if rank != 0:
        return
    t0 = time.perf_counter()
    samples = []
    for k in range(args.warmup + args.steps):
        t_spmv, t_wc = oracle_kernel_times(args.n, levels=args.ref_levels)
        if k >= args.warmup:
            samples.append((t_spmv, t_wc))
    t_spmv = statistics.median(s[0] for s in samples)
    t_wc = statistics.median(s[1] for s in samples)
    counts = [REF_COUNTS[DTS[k % len(DTS)]] for k in range(args.steps)]
    N = 4 * (args.n - 1) ** 2
    value = compose_solve_time(t_spmv, t_wc, counts, N)
    sample = ("FP64 oracle at 1024^2, single thread: per step one BSR SpMV and one W-cycle (medians %.3f s, %.2f s), "
              "scaled to seconds per solve with the sweep's outer/inner iteration counts" % (t_spmv, t_wc))
    line = {
        "metric": "time-to-1e-8 true residual, deflated CG (W-cycle MG + RAS inner), 2D Q1 pseudo-stress 1024^2, "
                  "dt in {1e-6,1e-5,1e-4}",
        "value": value, "unit": "s/solve", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (time.perf_counter() - t0) * 1e3 / (args.steps + args.warmup),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "host oracle"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "s/solve", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "s/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--max-it", type=int, default=20000)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-cg", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-mf", action="store_true")
    ap.add_argument("--skip-mf-solve", action="store_true")
    ap.add_argument("--skip-3d", action="store_true")
    ap.add_argument("--dcg-sweep", action="store_true", help="also time deflated CG at dt 1e-3..1e-1")
    ap.add_argument("--sweep-c", type=float, default=None, help="inner tolerance factor c_F of that sweep")
    ap.add_argument("--dts", type=float, nargs="+", default=None,
                    help="step sizes of the timed solves (default 1e-6 1e-5 1e-4); for profiling runs")
    ap.add_argument("--batched-problems", type=int, default=64)
    ap.add_argument("--batched-rhs", type=int, default=4)
    ap.add_argument("--batched-no-tune", action="store_true")
    ap.add_argument("--levels", type=int, nargs="+", default=[2, 3, 4], help="hierarchy depths to autotune over")
    ap.add_argument("--ref-levels", type=int, default=2, help="hierarchy depth of the oracle in the reference arm")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
