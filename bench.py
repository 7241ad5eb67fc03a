#!/usr/bin/env python
"""Benchmark of the deflated-CG hot path on one GB300 (or N replicas).

Workload (default, the 2D sweep): unit square, 1024 x 1024 Q1 pseudo-stress
elements (N = 4,186,116 unknowns, BSR 4x4, 9 blocks per row), nu = 1,
right-hand side uniform[-1, 1) from seed 0, solved to true relative residual
1e-8 for dt in {1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1}, everything in FP64.
One step = one complete deflated-CG solve (FCG(1), fixed inner tolerance
c_F = 0.01, W-cycle multigrid with RAS 8x8 cores, overlap 2, 2+2 smoothing
steps, hierarchy depth autotuned among 2-4 levels) at the next dt of the sweep
(step k solves dt number k mod 6). value = the mean over the six dt of the
time to solution (each dt's time the mean of its timed steps), so every dt
counts once whatever the step count.

Printed: one JSON line (rank 0) with the contract keys, plus "roofline"
(dominant kernel class, measured live with CUDA events during the timed
steps), "cpu_baseline" (the FP64 oracle on the host cores), "e2e" (one sweep
through the host-array entry point, copies included), "clocks" (nvidia-smi
samples during the timed region) and "extra": plain CG at every dt, the
mixed-precision solver (FP32 W-cycle, BF16 RAS on tensor cores) at every dt
with its speed-up and error against the FP64 solution, the error of each
mixed component against FP64, per-class kernel rooflines against the measured
HBM and FP64 peaks, and the 3D, matrix-free and batched workloads.

--impl reference times the oracle alone on a bounded sample of the same
workload, scaled to seconds per solve (see run_reference).
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")
# hardware queues for concurrent streams and graph branches (the batched
# workload's problems run as independent branches); read at context creation
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

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

DTS = [1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1]  # the sweep: step k solves DTS[k % 6]
WORKLOAD = ("2D unit square 1024x1024 Q1 pseudo-stress (4 comps/node, N=4,186,116, BSR 4x4), nu=1, "
            "dt in {1e-6,1e-5,1e-4,1e-3,1e-2,1e-1} (step k solves dt k mod 6), RHS uniform[-1,1) seed 0, "
            "tol 1e-8 true residual, all FP64: deflated CG (FCG(1), c_F=0.01, W-cycle MG with levels autotuned, "
            "RAS 8x8 cores overlap 2, m1=m2=2) vs plain CG")
MG_OPTS = dict(patch=8, overlap=2, m1=2, m2=2, inner_rule=0, c=0.01, recurrence=0)

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
    """Time the FP64 oracle at the bench size (single thread): one BSR product,
    one W-cycle (Algorithm 4) of the bench hierarchy and the vector work of one
    outer iteration (Algorithm 1 updates and the embed/extract of M_D)."""
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
    t0 = time.perf_counter()
    d, r, xh = x.copy(), y.copy(), np.zeros_like(x)
    q = y - V @ (V.T @ y)
    dq = d @ q
    a = (d @ r) / dq
    xh = xh + a * d
    r = r - a * q
    d = r - ((r @ q) / dq) * d
    t_vec = time.perf_counter() - t0
    del y, z
    return t_spmv, t_wc, t_vec


def compose_solve_time(t_spmv, t_wc, t_vec, stats):
    """Seconds per solve of the oracle from its timed pieces and the counts of
    a solve: per outer iteration one product A d, the V^T / V and the vector
    updates (t_vec) and its W-cycles; the f_D and reconstruction products."""
    total = 0.0
    for st in stats:
        passes = 1 + st["restarts"]
        total += (st["outer_its"] * (t_spmv + t_vec) + st["total_mg_cycles"] * t_wc
                  + passes * 3 * t_spmv)
    return total / max(1, len(stats))


def _oracle_full_solve(args):
    """One full FP64 oracle solve (deflated CG with the bench hierarchy) in a
    fresh process; returns (dt, seconds, outer iterations, W-cycles)."""
    n, dt, levels = args
    from oracle import fem, mg, solvers
    from paper_2606_13429_gb300 import inputs
    asm = fem.assemble(2, n, dt)
    f = inputs.rhs(0, asm.mesh.n_unknowns)
    S = solvers.FDCG(asm, solvers.FDCGOptions(mg=mg.MGOptions(patch=8, overlap=2, m1=2, m2=2, max_levels=levels)))
    t0 = time.perf_counter()
    x, st = S.solve(f, tol=1e-8, max_it=20000)
    return dt, time.perf_counter() - t0, st.outer_its, st.total_mg_cycles, bool(st.converged)


def oracle_full_solves(n=32, dts=None, parallel=True):
    """Real oracle solves of the sweep on an n x n mesh: one after another in
    this process (one thread), and the same solves spread over the host
    cores (one process each, started with spawn)."""
    dts = list(dts or DTS)
    t0 = time.perf_counter()
    seq = [_oracle_full_solve((n, dt, 2)) for dt in dts]
    t_seq = time.perf_counter() - t0
    out = {"n": n, "dts": dts, "single_thread_s_per_solve": t_seq / len(dts),
           "per_dt": {str(r[0]): {"s": r[1], "outer_its": r[2], "total_mg_cycles": r[3], "converged": r[4]}
                      for r in seq}}
    if parallel:
        import multiprocessing as mpr
        cores = min(len(dts), os.cpu_count() or 1)
        t0 = time.perf_counter()
        with mpr.get_context("spawn").Pool(cores) as pool:
            pool.map(_oracle_full_solve, [(n, dt, 2) for dt in dts])
        out["all_cores_s_per_solve"] = (time.perf_counter() - t0) / len(dts)
        out["cores"] = cores
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


# --------------------------------------------------------------------------- main arm


def _event_solve(torch, fn):
    """Run fn() between two CUDA events on the current stream; (result, ms)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = fn()
    e1.record()
    e1.synchronize()
    return res, e0.elapsed_time(e1)


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
        # replicas: the headline sweep only; the single-GPU characterisations
        # stay at N = 1
        args.skip_cg = args.skip_mixed = args.skip_batched = args.skip_mf = args.skip_3d = True
    torch.cuda.set_device(local)
    B.build()
    dcg.load()
    peaks, peak_src = load_peaks()
    fp64_peak = dcg.dcg_measure_fma_rate(dcg.DCG_FP64)   # TFLOP/s, measured on this GPU
    fp32_peak = dcg.dcg_measure_fma_rate(dcg.DCG_MIXED)
    n = args.n
    probs = {dt: dcg.dcg_assemble(2, n, dt) for dt in DTS}
    # hierarchy depth: one inner solve to 1e-10 per candidate (the inner
    # system does not depend on dt), fastest kept
    tune = {}
    g = torch.from_numpy(inputs.rhs(1, probs[DTS[0]].n_nodes)).cuda()
    for levels in args.levels:
        try:
            dcg.dcg_setup(probs[DTS[0]], dcg.options(max_levels=levels, precision=dcg.DCG_FP64, **MG_OPTS))
        except dcg.DCGError:
            continue
        best = None
        for _ in range(3):
            z = torch.zeros_like(g)
            _, ms = _event_solve(torch, lambda: dcg.dcg_mg_solve(probs[DTS[0]], g, z, 1e-10))
            best = ms if best is None else min(best, ms)
        tune[levels] = best
    best_levels = min(tune, key=tune.get)
    opts = dcg.options(max_levels=best_levels, precision=dcg.DCG_FP64, **MG_OPTS)
    for dt in DTS:
        dcg.dcg_setup(probs[dt], opts)
    N = probs[DTS[0]].N
    f = torch.from_numpy(inputs.rhs(0, N)).cuda()
    x = torch.zeros_like(f)
    stream = torch.cuda.current_stream()

    def step(k, record):
        dt = DTS[k % len(DTS)]
        x.zero_()
        st, ms = _event_solve(torch, lambda: dcg.dcg_solve(probs[dt], f, x, tol=1e-8, max_it=args.max_it))
        record.append((dt, st, ms))
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
    elapsed_ms, _ = job_time(ev0.elapsed_time(ev1), args.steps, ws, torch, device="cuda")
    # value: mean over the dt of the sweep of the time to solution (slowest
    # rank per step), over all ranks' solves
    step_ms = torch.tensor([ms for _, _, ms in timed], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(step_ms, op=dist.ReduceOp.MAX)
    per_dt = {}
    for (dt, _, _), ms in zip(timed, step_ms.tolist()):
        per_dt.setdefault(dt, []).append(ms)
    value = statistics.mean(statistics.mean(v) for v in per_dt.values()) / 1e3 / ws
    dom = {"ms": 0.0, "launches": 0, "flops": 0.0, "bytes": 0.0}
    for p in probs.values():
        r = dcg.dcg_profile_read(p)[dominant]
        for key in dom:
            dom[key] += r[key]
        dcg.dcg_profile_enable(p, [])
    ok = all(st["status"] == dcg.DCG_OK and st["true_relres"] <= 1e-8 for _, st, _ in timed)

    # end to end: one sweep through the host-array entry point, pinned host
    # memory, copies inside the timed region
    f_h = torch.from_numpy(inputs.rhs(0, N)).pin_memory()
    x_h = torch.zeros(N, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e2e_ms = []
    for dt in DTS:
        x_h.zero_()
        t0 = time.perf_counter()
        dcg.dcg_solve_host(probs[dt], f_h, x_h, tol=1e-8, max_it=args.max_it)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_t = torch.tensor(e2e_ms, dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_s = float(e2e_t.mean().item()) / 1e3 / ws

    extra = {"per_dt": {}, "fp64_fma_peak_tflops": fp64_peak, "fp32_fma_peak_tflops": fp32_peak,
             "autotune_inner_solve_ms": {"levels=%d" % k: v for k, v in tune.items()}}
    for dt, st, ms in timed:
        e = extra["per_dt"].setdefault(str(dt), {})
        if "dcg_fp64" not in e:
            e["dcg_fp64"] = {"s": ms / 1e3, "outer_its": st["outer_its"], "total_mg_cycles": st["total_mg_cycles"],
                             "avg_inner": round(st["avg_inner"], 2), "restarts": st["restarts"],
                             "true_relres": st["true_relres"]}
    x64 = {}
    if not args.skip_cg or not args.skip_mixed:
        for dt in DTS:  # FP64 reference solutions for the mixed arm's error
            xx = torch.zeros_like(f)
            dcg.dcg_solve(probs[dt], f, xx, tol=1e-8, max_it=args.max_it)
            x64[dt] = xx
    # plain CG, FP64, at every dt (same matrix, same right-hand side)
    if not args.skip_cg:
        for dt in DTS:
            pc = dcg.dcg_assemble(2, n, dt)
            dcg.dcg_setup(pc, dcg.options(deflate=0))
            x.zero_()
            st, ms = _event_solve(torch, lambda: dcg.dcg_solve(pc, f, x, tol=1e-8, max_it=args.max_it))
            e = extra["per_dt"][str(dt)]
            e["plain_cg_fp64"] = {"s": ms / 1e3, "outer_its": st["outer_its"], "true_relres": st["true_relres"]}
            if "dcg_fp64" in e:
                e["dcg_speedup_vs_cg"] = e["plain_cg_fp64"]["s"] / e["dcg_fp64"]["s"]
            pc.close()
    # mixed precision (FP32 W-cycle, BF16 inverses on tcgen05; FP64 outer CG)
    if not args.skip_mixed:
        mopts = dcg.options(max_levels=2, precision=dcg.DCG_MIXED, ras_inverse=dcg.DCG_INV_BF16, **MG_OPTS)
        for dt in DTS:
            dcg.dcg_setup(probs[dt], mopts)
            x.zero_()
            dcg.dcg_solve(probs[dt], f, x, tol=1e-8, max_it=30)  # builds the graph
            x.zero_()
            st, ms = _event_solve(torch, lambda: dcg.dcg_solve(probs[dt], f, x, tol=1e-8, max_it=args.max_it))
            e = extra["per_dt"][str(dt)]
            err = float(torch.linalg.norm(x - x64[dt]) / torch.linalg.norm(x64[dt]))
            e["dcg_mixed"] = {"s": ms / 1e3, "outer_its": st["outer_its"], "total_mg_cycles": st["total_mg_cycles"],
                              "restarts": st["restarts"], "true_relres": st["true_relres"],
                              "rel_error_vs_fp64_solution": err}
            if "dcg_fp64" in e:
                e["mixed_speedup_vs_fp64"] = e["dcg_fp64"]["s"] / e["dcg_mixed"]["s"]
        extra["mixed_component_errors"] = mixed_component_errors(dcg, inputs, torch, n)
        extra["four_level_wcycle"] = four_level_wcycle(dcg, inputs, torch, n, best_levels)
    for p in probs.values():
        p.close()
    probs.clear()
    torch.cuda.empty_cache()

    # SpMV bandwidth on this operator (FP64, plain product) and the per-class rooflines
    extra["spmv_fp64"] = spmv_rate(dcg, inputs, torch, n, peaks)
    extra["class_rooflines"] = class_rooflines(breakdown, peaks, fp64_peak)
    extra["kernel_breakdown_warmup_ms"] = {c: round(v["ms"], 3) for c, v in breakdown.items()}
    # the batched workload runs its multigrid in FP32 (BF16 inverses) with
    # FP64 outer CG; its options are autotuned per mesh size from these
    bopts = dcg.options(max_levels=2, precision=dcg.DCG_MIXED, ras_inverse=dcg.DCG_INV_BF16, **MG_OPTS)
    for key, skip, fn in [("batched", args.skip_batched, batched_extra), ("matrix_free_3d_256", args.skip_mf, mf_extra),
                          ("bsr_3d_%d" % args.n3, args.skip_3d, bsr3d_extra)]:
        if skip:
            continue
        try:
            extra[key] = fn(args, bopts, dcg, inputs, torch)
        except Exception as exc:  # an extra must not cost the headline line
            extra[key] = {"error": "%s: %s" % (type(exc).__name__, exc)}
        torch.cuda.empty_cache()

    roof = roofline(dominant, dom, peaks, peak_src, fp64_peak)

    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        t_spmv, t_wc, t_vec = oracle_kernel_times(n, levels=best_levels)
        stats = [st for _, st, _ in timed]
        full = oracle_full_solves(32)
        cpu = {"value": compose_solve_time(t_spmv, t_wc, t_vec, stats), "unit": "s/solve", "cores": 1,
               "kind": "oracle",
               "sample": ("FP64 oracle at 1024^2, one thread: one BSR product (%.3f s), one W-cycle of the bench "
                          "hierarchy (%.2f s) and the vector work of one outer iteration (%.3f s) timed, scaled to "
                          "s/solve with the outer iterations and W-cycles of the timed solves (whose counts the "
                          "parity tests hold within 2 of the oracle's)" % (t_spmv, t_wc, t_vec)),
               "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
               "real_full_solves_32": full}

    if rank == 0:
        line = {
            "metric": "time-to-1e-8 true residual, deflated CG (W-cycle MG + RAS inner) vs plain CG, FP64 (mixed in "
                      "extra), 2D Q1 pseudo-stress 1024^2, dt in {1e-6..1e-1}",
            "value": value, "unit": "s/solve", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": "replicas" if ws > 1 else "single GPU",
                       "mg_levels": best_levels, "dts": DTS,
                       "value": "mean over the six dt of the time to solution (each dt the mean of its timed steps)",
                       "smoother": "RAS, FP64 local solves by fast diagonalisation (sine transforms + line solves)",
                       "l2": "inputs larger than L2 (BSR matrix 1.2 GB per dt, 6 matrices)",
                       "all_converged": ok},
            "e2e": {"value": e2e_s, "unit": "s/solve", "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": N * 8,
                    "steps": len(DTS), "note": "one sweep (each dt once) through dcg_solve_host"},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
            "extra": extra,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def spmv_rate(dcg, inputs, torch, n, peaks):
    """The FP64 BSR product alone (20 launches after one warm-up): GB/s of the
    algorithmic bytes against the measured copy bandwidth."""
    p = dcg.dcg_assemble(2, n, 1e-6)
    f = torch.from_numpy(inputs.rhs(0, p.N)).cuda()
    y = torch.empty_like(f)
    dcg.dcg_spmv(p, f, y)
    dcg.dcg_profile_enable(p, ["spmv"])
    for _ in range(20):
        dcg.dcg_spmv(p, f, y)
    sp = dcg.dcg_profile_read(p)["spmv"]
    dcg.dcg_profile_enable(p, [])
    p.close()
    gbs = sp["bytes"] / (sp["ms"] / 1e3) / 1e9
    return {"GB_per_s": gbs, "ms": sp["ms"] / max(1, sp["launches"]), "frac_of_hbm": gbs / peaks["hbm_gbs"],
            "algorithmic_bytes_per_launch": sp["bytes"] / max(1, sp["launches"])}


def class_rooflines(breakdown, peaks, fp64_peak):
    """Per kernel class over the warm-up solves: algorithmic GB/s and TFLOP/s
    against the measured HBM copy bandwidth and FP64 FMA rate; the roof of a
    class is the smaller of the two times its work needs."""
    out = {}
    for c, v in breakdown.items():
        if v["ms"] <= 0:
            continue
        secs = v["ms"] / 1e3
        gbs = v["bytes"] / secs / 1e9
        tf = v["flops"] / secs / 1e12
        t_hbm = v["bytes"] / (peaks["hbm_gbs"] * 1e9)
        t_alu = v["flops"] / (fp64_peak * 1e12)
        out[c] = {"ms": round(v["ms"], 3), "launches": v["launches"], "GB_per_s": gbs, "TFLOP_per_s": tf,
                  "frac_hbm": gbs / peaks["hbm_gbs"], "frac_fp64": tf / fp64_peak,
                  "frac_of_roof": max(t_hbm, t_alu) / secs}
    return out


def mixed_component_errors(dcg, inputs, torch, n):
    """Error of each mixed-precision component against its FP64 counterpart at
    the bench size (element-wise, max |mixed - fp64| / max |fp64|): one
    W-cycle (FP32 with BF16 tensor-core RAS) and one RAS step (BF16 inverse
    x BF16 residual, FP32 accumulation) on the bench hierarchy."""
    out = {}
    p64 = dcg.dcg_assemble(2, n, 1e-6)
    pmx = dcg.dcg_assemble(2, n, 1e-6)
    dcg.dcg_setup(p64, dcg.options(max_levels=2, precision=dcg.DCG_FP64, **MG_OPTS))
    dcg.dcg_setup(pmx, dcg.options(max_levels=2, precision=dcg.DCG_MIXED, ras_inverse=dcg.DCG_INV_BF16, **MG_OPTS))
    g = torch.from_numpy(inputs.rhs(13, p64.n_nodes)).cuda()
    z64, zmx = torch.zeros_like(g), torch.zeros_like(g)
    dcg.dcg_mg_cycles(p64, g, z64, 1)
    dcg.dcg_mg_cycles(pmx, g, zmx, 1)
    out["wcycle_fp32_bf16"] = float((zmx - z64).abs().max() / z64.abs().max())
    nn = p64.level_nodes(2)
    fr = torch.from_numpy(inputs.rhs(20, nn)).cuda()
    zr = torch.from_numpy(inputs.rhs(21, nn)).cuda()
    a, b = zr.clone(), zr.clone()
    dcg.dcg_ras_step(p64, 2, fr, a)
    dcg.dcg_ras_step(pmx, 2, fr, b)
    out["ras_step_bf16_update"] = float(((b - zr) - (a - zr)).abs().max() / (a - zr).abs().max())
    zc = torch.zeros_like(g)
    cyc = dcg.dcg_mg_solve(pmx, g, zc, 1e-10)
    zc64 = torch.zeros_like(g)
    cyc64 = dcg.dcg_mg_solve(p64, g, zc64, 1e-10)
    out["inner_solve_1e-10_fp32_vs_fp64"] = {"rel_error": float((zc - zc64).abs().max() / zc64.abs().max()),
                                             "cycles_mixed": cyc, "cycles_fp64": cyc64}
    p64.close()
    pmx.close()
    return out


def four_level_wcycle(dcg, inputs, torch, n, best_levels):
    """Time per inner solve (to 1e-10) of the paper's four-level 2D hierarchy
    next to the autotuned depth, FP64 and mixed."""
    out = {}
    p = dcg.dcg_assemble(2, n, 1e-6)
    g = torch.from_numpy(inputs.rhs(1, p.n_nodes)).cuda()
    for name, prec, inv in [("fp64", dcg.DCG_FP64, dcg.DCG_INV_FP32), ("mixed_bf16", dcg.DCG_MIXED, dcg.DCG_INV_BF16)]:
        for lv in sorted({best_levels, 2, 4}):
            dcg.dcg_setup(p, dcg.options(max_levels=lv, precision=prec, ras_inverse=inv, **MG_OPTS))
            z = torch.zeros_like(g)
            dcg.dcg_mg_solve(p, g, z, 1e-10)
            z.zero_()
            cyc, ms = _event_solve(torch, lambda: dcg.dcg_mg_solve(p, g, z, 1e-10))
            out["%s_levels=%d" % (name, lv)] = {"ms_per_inner_solve": ms, "cycles": cyc}
    p.close()
    return out


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
    n, dt = args.n3, 1e-4
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
    # bytes of the product in the stored BSR format (81 values per block): the
    # kernel skips the 48 structural zeros of a block, but DRAM still moves
    # the whole blocks (ncu: DRAM reads equal the stored bytes), at a read
    # rate above the copy bandwidth (which mixes reads and writes)
    fmt = prob.nnzb * 81 * 8 + prob.nnzb * 4 + 2 * prob.N * 8
    out["spmv_fp64_GB_per_s"] = fmt / (sp_ms * 1e-3) / 1e9
    out["spmv_fp64_frac_of_copy_bw"] = out["spmv_fp64_GB_per_s"] / load_peaks()[0]["hbm_gbs"]
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
    seq, per_problem = [], [0.0] * len(probs)
    for k in range(len(fs)):
        tk = time.perf_counter()
        seq.append(dcg.dcg_solve(probs[k // nrhs], fs[k], xs[k], tol=1e-8, max_it=args.max_it))
        per_problem[k // nrhs] += time.perf_counter() - tk  # dcg_solve returns after its solve ended
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    unknowns = sum(pr.N for pr in probs) * nrhs
    crit = max(range(len(probs)), key=lambda i: per_problem[i])
    out = {"problems": len(probs), "rhs_per_problem": nrhs, "unknowns_total": unknowns,
           "n_range": [min(n for n, _ in plist), max(n for n, _ in plist)],
           "batched_s": t_batched, "sequential_s": t_seq, "speedup": t_seq / t_batched,
           # a problem's right-hand sides run in sequence (they share its
           # work vectors): the slowest problem bounds the batch from below
           "critical_path_s": per_problem[crit],
           "critical_problem": {"n": plist[crit][0], "dt": plist[crit][1],
                                "outer_its": [st["outer_its"] for st in seq[crit * nrhs:(crit + 1) * nrhs]]},
           "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
           "batched_unknowns_per_s": unknowns / t_batched,
           "all_converged": code == dcg.DCG_OK and all(st["true_relres"] <= 1e-8 for st in stats),
           "same_iterations_as_sequential": all(a["outer_its"] == b["outer_its"] for a, b in zip(stats, seq)),
           "setup_and_autotune_s": t_tune, "autotuned_options_per_problem": choices or "not tuned"}
    for pr in probs:
        pr.close()
    return out


def kernel_source_hash(files=None, functions=None):
    """Hash of kernel sources: all of csrc/ (or the named files), or only the
    text of the named device functions in them (from the line that declares
    the function to its closing brace in column 0). A DRAM traffic figure in
    profiles/traffic.json counts only while the code it was captured on is
    unchanged."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_13429_gb300", "csrc")
    for fn in sorted(files or os.listdir(csrc)):
        with open(os.path.join(csrc, fn), "r", encoding="utf-8") as fh:
            text = fh.read()
        if not functions:
            h.update(text.encode())
            continue
        for name in functions:
            for mt in re.finditer(r"^(?:template <[^\n]*>\n)?(?:__global__|__device__)[^\n]*\b%s\(" % re.escape(name),
                                  text, re.M):
                end = text.find("\n}\n", mt.start())
                h.update(text[mt.start():end + 3].encode())
    return h.hexdigest()[:16]


def roofline(dominant, dom, peaks, peak_src, fp64_peak):
    """Roofline of the dominant kernel class over the timed region: its
    algorithmic bytes and FP64 flops against the measured HBM copy bandwidth
    and the measured FP64 FMA rate; the bound is whichever needs more time."""
    secs = dom["ms"] / 1e3
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tr = json.load(fh)
        ent = tr.get(dominant)
        if ent and ent.get("source_hash") == kernel_source_hash(ent.get("source_files"), ent.get("functions")):
            traffic = ent["dram_bytes_per_launch"]
    except Exception:
        pass
    base = {"kernel": dominant, "traffic": traffic, "launches": dom["launches"],
            "algorithmic_bytes_per_launch": dom["bytes"] / max(1, dom["launches"]),
            "algorithmic_flops_per_launch": dom["flops"] / max(1, dom["launches"])}
    if secs <= 0:
        return dict(base, bound="hbm", achieved=0.0, peak=peaks["hbm_gbs"], unit="GB/s", frac=0.0)
    t_hbm = dom["bytes"] / (peaks["hbm_gbs"] * 1e9)
    t_alu = dom["flops"] / (fp64_peak * 1e12)
    if t_alu > t_hbm:
        achieved = dom["flops"] / secs / 1e12
        return dict(base, bound="alu", achieved=achieved, peak=fp64_peak, unit="TFLOP/s", frac=achieved / fp64_peak,
                    peak_source="FP64 FMA rate measured on this GPU by dcg_measure_fma_rate (independent FMA chains "
                                "on all SMs); an FMA counts 2 flops")
    achieved = dom["bytes"] / secs / 1e9
    return dict(base, bound="hbm", achieved=achieved, peak=peaks["hbm_gbs"], unit="GB/s",
                frac=achieved / peaks["hbm_gbs"], peak_source=peak_src + " copy bandwidth (MEASURED_PEAKS.json)")


# --------------------------------------------------------------------------- reference arm


def load_counts():
    """Outer iterations, W-cycles and restarts of each dt's FP64 solve at 1024^2
    (profiles/iteration_counts_1024.json, written from a bench run on GB300:
    the oracle cannot run these solves to convergence within a bench, and the
    parity tests hold the GPU solver's counts within 2 of the oracle's)."""
    with open(os.path.join(ROOT, "profiles", "iteration_counts_1024.json")) as fh:
        return {float(k): v for k, v in json.load(fh)["per_dt"].items()}


def run_reference(args):
    ws, rank, local = dist_init()
    if rank != 0:
        return
    counts = load_counts()
    from oracle import fem, mg
    from paper_2606_13429_gb300 import inputs
    n = args.n
    asm = fem.assemble(2, n, 1e-6)
    A = asm.matrix().tocsr()
    V = fem.V_matrix(asm.mesh)
    H = mg.Hierarchy(2, n, mg.inner_matrix(V, A), mg.MGOptions(patch=8, overlap=2, m1=2, m2=2,
                                                                max_levels=args.ref_levels))
    xv = inputs.rhs(0, asm.mesh.n_unknowns)
    g = inputs.rhs(1, asm.mesh.n_nodes)
    samples = []
    t_start = time.perf_counter()
    for k in range(args.warmup + args.steps):
        # one bounded sample per step: a BSR product, a W-cycle of the bench
        # hierarchy and the vector work of an outer iteration, real oracle code
        t0 = time.perf_counter()
        y = A @ xv
        t_spmv = time.perf_counter() - t0
        t0 = time.perf_counter()
        H.wcycle(g, np.zeros_like(g))
        t_wc = time.perf_counter() - t0
        t0 = time.perf_counter()
        q = y - V @ (V.T @ y)
        dq = xv @ q
        r = y - ((xv @ y) / dq) * q
        _ = r - ((r @ q) / dq) * xv
        t_vec = time.perf_counter() - t0
        if k >= args.warmup:
            dt = DTS[k % len(DTS)]
            samples.append((dt, compose_solve_time(t_spmv, t_wc, t_vec, [counts[dt]])))
    per_dt = {}
    for dt, v in samples:
        per_dt.setdefault(dt, []).append(v)
    value = statistics.mean(statistics.mean(v) for v in per_dt.values())
    sample = ("FP64 oracle at 1024^2, one thread: per step one BSR product, one W-cycle of the bench hierarchy "
              "(levels=%d) and the vector work of an outer iteration, timed and scaled to s/solve with the "
              "counts of profiles/iteration_counts_1024.json" % args.ref_levels)
    line = {
        "metric": "time-to-1e-8 true residual, deflated CG (W-cycle MG + RAS inner) vs plain CG, FP64 (mixed in "
                  "extra), 2D Q1 pseudo-stress 1024^2, dt in {1e-6..1e-1}",
        "value": value, "unit": "s/solve", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (time.perf_counter() - t_start) * 1e3 / (args.steps + args.warmup),
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
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--max-it", type=int, default=20000)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-cg", action="store_true")
    ap.add_argument("--skip-mixed", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-mf", action="store_true")
    ap.add_argument("--skip-mf-solve", action="store_true")
    ap.add_argument("--skip-3d", action="store_true")
    ap.add_argument("--n3", type=int, default=128, help="mesh of the 3D assembled workload (cfg3: 128)")
    ap.add_argument("--dts", type=float, nargs="+", default=None,
                    help="step sizes of the timed solves (default: the sweep 1e-6..1e-1); for profiling runs")
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
