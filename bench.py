#!/usr/bin/env python3
"""Benchmark: CG time-to-1e-10 true residual for the Wilson-Dirac normal equations on GB300.

Workload (the paper's largest lattice): 14^4 sites, kappa = 0.12, links exp(i 0.4 H) re-unitarised
to SU(3) (gauge seed 1), complex Gaussian source (seed 2), antiperiodic time, chiral gamma basis,
plain FP64 CG (CGLS form, two dslash per iteration) to a true relative residual of 1e-10, 1 RHS.

One step = load the gauge field into the device layout + one complete solve from x = 0 + the true
residual recomputation, with inputs resident in HBM. The L2 (129 MB) is flushed before every step
by writing a 512 MB buffer outside the timed interval.

Extra measurements on the same line: the dominant kernel against its roofline (the FP64 ceiling
measured in the same run), the same solve end to end from host buffers, plain FP32 CG and mixed
precision, a dslash bandwidth sweep, and the CPU oracle's whole solve of the same system on one host
core (a baseline, not a target).

``--impl reference`` times the FP64 CPU oracle (the plain definition of the method) instead, one
whole solve per timed step. ``--profile-case ...`` runs one small workload for an ncu capture (see
profile_case below) instead of the benchmark.
Multi-GPU: the solver does not shard here, so ``--gpus N`` runs N independent replicas (one per
rank, weak scaling) and reports the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (14, 14, 14, 14)
KAPPA = 0.12
EPS = 0.4
TOL = 1e-10
MAXIT = 4000
GAUGE_SEED, SOURCE_SEED = 1, 2
BC = (1, 1, 1, -1)
FLOPS_PER_SITE = 1320          # hopping part of one dslash, the usual convention
BYTES_SITE_F64_18 = 192 + 576 + 192  # spinor in + 4 links + spinor out (FP64, 18-real links)
BLAS_FLOPS_PER_SITE_ITER = 288        # per CG iteration: 3 norms + 3 axpy-type updates, 24 FMA each


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# The FP64 roofline ceiling from the unit count: SMs x 2 DFMA per clock x 2 flop x the maximum SM clock
# (152 x 2 x 2 x 2.07 GHz = 1.259 TFLOP/s on GB300). The library's DFMA probe (wd_measure_fp64_peak),
# run beside it, reads about 84 % of that, but the FP64 dslash at 32^4 retires its mixed stream of
# FMAs, adds and multiplies at about 95 % of the unit count, so the probe is not the pipe's ceiling.
FP64_DFMA_PER_CLK_PER_SM = 2


def _fp64_unit_peak(dev) -> tuple:
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(_peaks().get("sm_max_mhz", 2070.0))
    tf = sms * FP64_DFMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12
    return tf, (f"unit count: {sms} SMs x {FP64_DFMA_PER_CLK_PER_SM} DFMA/clk x 2 flop x {mhz:.0f} MHz "
                f"(maximum SM clock) = {tf:.3f} TFLOP/s")

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the kernels the line
# reports, from one ncu capture each; the summary file holds the full command. None = not captured
# for the kernel as it now stands.
NCU_TRAFFIC = {
    "cg_loop_f64_14x4": (70633984, "profiles/cg_loop_f64_14x4.md"),
    "dslash_f64_14x4": (29587712, "profiles/dslash_f64_14x4.md"),
}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "window": "warm-up start to timed-region end, 100 ms period"}


def make_inputs(dims, eps=EPS, gseed=GAUGE_SEED, sseed=SOURCE_SEED):
    import synthetic
    return synthetic.gauge_field(dims, eps, gseed), synthetic.gaussian_source(dims, sseed)


# ---------------------------------------------------------------------------- reference arm

REFERENCE_MAX_TIMED_SOLVES = 3  # full oracle solves of the 14^4 workload timed per run (~30 s each)


def run_reference(args, rank, world):
    """The FP64 CPU oracle, as it stands, solving the same workload to the same tolerance.

    Each timed step is one whole oracle solve of the 14^4 system (CGLS to a 1e-10 true residual,
    about 30 s on one host core), so the value is a measurement, not an extrapolation. To end within
    a few minutes the run times at most REFERENCE_MAX_TIMED_SOLVES of them: the line's `steps` is
    the number timed and `steps_requested` the number asked for. Warm-up steps run one CGLS
    iteration each (numpy has no JIT or cache to warm; they only page in the code and the fields).
    """
    if rank != 0:
        return 0
    from oracle import cg as ocg
    U, eta = make_inputs(DIMS)
    for _ in range(args.warmup):
        ocg.cgls(U, eta, KAPPA, 0.0, 1)
    n_timed = max(1, min(args.steps, REFERENCE_MAX_TIMED_SOLVES))
    times, iters, res = [], None, None
    c0 = time.process_time()
    for _ in range(n_timed):
        t0 = time.perf_counter()
        _, iters, res, _ = ocg.cgls(U, eta, KAPPA, TOL, MAXIT)
        times.append(1e3 * (time.perf_counter() - t0))
    busy = (time.process_time() - c0) / (1e-3 * sum(times))
    ms = statistics.mean(times)
    sample = (f"{n_timed} whole oracle solves of the 14^4 workload (FP64 numpy CGLS, {iters} iterations, "
              f"true residual {res:.2e}); {args.steps} steps requested; numpy's dot products run on "
              f"OpenBLAS threads over the host's {os.cpu_count()} cores, {busy:.1f} cores busy on average")
    line = {
        "impl": "reference", "metric": "CG time-to-1e-10 residual", "value": ms, "unit": "ms",
        "n_gpus": world, "steps": n_timed, "steps_requested": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(), "iterations": iters, "true_rel_residual": res,
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": os.cpu_count(), "avg_busy_cores": busy,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config():
    return {"workload": "plain FP64 CG on D^dag D, 14^4, kappa 0.12, eps 0.4, tol 1e-10, 1 RHS",
            "lattice": list(DIMS), "kappa": KAPPA, "eps": EPS, "tol": TOL, "rhs": 1,
            "l2": "flushed before every step (512 MB write, untimed)"}


# ---------------------------------------------------------------------------- native arm

def max_over_ranks(ms, world, device):
    """The slowest replica's time: every rank solves its own system (weak scaling)."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def run_native(args, rank, world):
    import torch
    from paper_2111_14958_gb300 import wd

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    U, eta = make_inputs(DIMS)
    Ud = torch.from_numpy(U).to(dev)
    etad = torch.from_numpy(eta).to(dev)
    x = torch.zeros_like(etad)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    op = wd.WilsonDirac(DIMS, KAPPA, BC, wd.WD_PREC_F64, stream=stream)
    op.load_gauge(Ud)
    if args.no_graph:
        op.set_option(wd.WD_OPT_USE_GRAPH, 0)

    def step():
        op.load_gauge(Ud)
        x.zero_()
        return wd.cg_solve(op.ctx, etad, x, TOL, MAXIT)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters_seen, res_seen, loop_ms_seen = [], [], []
    # clocks are sampled from the start of the warm-up to the end of the timed region
    with ClockSampler(local) as clk:
        for _ in range(max(args.warmup, 3)):
            step()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            st, it, rr = step()
            ev[i][1].record(stream)
            iters_seen.append(it)
            res_seen.append(rr)
            loop_ms_seen.append(op.stats()["loop_ms"])  # host read of the finished solve's record
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(statistics.mean(step_ms), world, dev)
    stats = op.stats()
    iters = iters_seen[-1]
    # our kernels per step: gauge load 1, parameter set 1, pack 2, unpack 1, and per pass of the
    # solver (1 + restarts) prologue 4 (init, two dslash, check) + true residual 1 + the loop: one
    # persistent kernel, or 4 per iteration (two dslash, two updates)
    passes = 1 + stats["restarts"]
    if stats["loop_mode"] == 2:
        launches = len(iters_seen) * (5 + 6 * passes)
    else:
        launches = sum(5 + 5 * passes + 4 * it for it in iters_seen)

    # dominant kernel: the FP64 dslash as the solver launches it, timed with CUDA events on the
    # solver's stream over 200 back-to-back launches on the resident workload
    dslash_ms = op.time_dslash(False, 200)
    V = int(np.prod(DIMS))
    flops = FLOPS_PER_SITE * V
    achieved_tflops = flops / (dslash_ms * 1e-3) / 1e12
    achieved_gbs = BYTES_SITE_F64_18 * V / (dslash_ms * 1e-3) / 1e9
    share = 2 * iters * dslash_ms / ms
    # the FP64 compute ceiling from the unit count, and the DFMA probe's rate measured now beside it
    fp64_peak, peak_source = _fp64_unit_peak(dev)
    fma_probe = wd.wd_measure_fp64_peak(stream, 5)
    peak_source += (f"; the library's DFMA probe (wd_measure_fp64_peak, best of 5 launches, CUDA events) "
                    f"read {fma_probe:.3f} TFLOP/s in this run")
    traffic, traffic_src = NCU_TRAFFIC["dslash_f64_14x4"]
    dslash_roof = {"bound": "alu", "achieved": achieved_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                   "frac": achieved_tflops / fp64_peak, "traffic": traffic, "traffic_source": traffic_src,
                   "kernel": "dslash_kernel<FP64, 18r> (q = D p with fused |q|^2), the launch shape the "
                             "solver uses",
                   "algorithmic": f"{FLOPS_PER_SITE} flop/site x {V} sites per launch; "
                                  f"{BYTES_SITE_F64_18} B/site",
                   "peak_source": peak_source, "frac_of_fma_probe": achieved_tflops / fma_probe,
                   "achieved_hbm_gbs": achieved_gbs, "launch_ms": dslash_ms,
                   "share_of_step": share}
    if stats["loop_mode"] == 2:
        # the whole CG loop is one persistent kernel: its own launch is the unit. FP64 flops per site
        # and iteration: two dslash (2 x 1320) + the BLAS-1 steps (|q|^2, |s|^2, r -= alpha q with
        # |r|^2, x += alpha p, p = s + beta p: 6 x 24 real FMA = 288)
        loop_ms = statistics.mean(loop_ms_seen)
        loop_flops = (2 * FLOPS_PER_SITE + BLAS_FLOPS_PER_SITE_ITER) * V * iters
        ach = loop_flops / (loop_ms * 1e-3) / 1e12
        traffic, traffic_src = NCU_TRAFFIC["cg_loop_f64_14x4"]
        roofline = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": ach / fp64_peak, "traffic": traffic, "traffic_source": traffic_src,
                    "kernel": f"cg_loop_kernel<FP64> (the whole CG loop in one cooperative launch: {iters} "
                              f"iterations of q = D p, r update, s = D^dag r, x and p update)",
                    "algorithmic": f"(2 x {FLOPS_PER_SITE} dslash + {BLAS_FLOPS_PER_SITE_ITER} BLAS-1) flop/site x "
                                   f"{V} sites x {iters} iterations per launch",
                    "peak_source": peak_source, "frac_of_fma_probe": ach / fma_probe,
                    "launch_ms": loop_ms, "share_of_step": loop_ms / ms,
                    "dslash_standalone": dslash_roof}
    else:
        roofline = dslash_roof

    out = {
        "metric": "CG time-to-1e-10 residual", "value": ms, "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(), "iterations": iters, "true_rel_residual": res_seen[-1],
        "cg_loop": {0: "host loop", 1: "CUDA graph with a device-side while node",
                    2: "one persistent cooperative kernel"}[stats["loop_mode"]],
        "gpu_launches": launches, "roofline": roofline, "clocks": clk.summary(),
        "solve_stats": stats,
    }
    if rank == 0 and not args.quick:
        out["e2e"] = _e2e(args, op, U, eta, dev, stream)
        out["fp32_cg"] = _variant(wd, U, eta, dev, stream, wd.WD_PREC_F32, 1e-6, c12=True)
        # the paper's own CG form (on D D^dag, Sec. 2) with the same kernels and stopping rule
        out["paper_cg_form_f64"] = _variant(wd, U, eta, dev, stream, wd.WD_PREC_F64, TOL, c12=False,
                                            options={wd.WD_OPT_CG_FORM: 1})
        out["mixed_f32"] = _variant(wd, U, eta, dev, stream, wd.WD_PREC_MIXED_F32, TOL, c12=True)
        out["mixed_f16"] = _variant(wd, U, eta, dev, stream, wd.WD_PREC_MIXED_F16, TOL, c12=True)
        out["dslash_sweep"] = _sweep(wd, dev, stream, args.sweep)
        out["paper_sizes_f64_cg"] = _paper_sizes(wd, stream)
        out["mixed_32x64"] = _mixed_32x64(wd, dev, stream)
        out["multi_rhs_24x48"] = _multi_24x48(wd, dev, stream)
        out["even_odd"] = _even_odd(wd, dev, stream)
        out["paper_coo_14x4"] = _paper_coo(wd, dev, stream)
        out["serving"] = _serving(wd)
        out["cpu_baseline"] = _cpu_baseline(iters)
    op.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def _e2e(args, op, U, eta, dev, stream):
    """Same solve through the public API from pinned host buffers, copies inside the timing."""
    import torch
    from paper_2111_14958_gb300 import wd
    Uh = torch.from_numpy(U).pin_memory()
    etah = torch.from_numpy(eta).pin_memory()
    xh = torch.empty_like(etah).pin_memory()
    etad = torch.empty_like(etah, device=dev)
    xd = torch.empty_like(etah, device=dev)
    times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op.load_gauge(Uh)                       # host pointer: staged H2D inside the library
        etad.copy_(etah, non_blocking=True)
        xd.zero_()
        wd.cg_solve(op.ctx, etad, xd, TOL, MAXIT)
        xh.copy_(xd, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        t1 = time.perf_counter()
        if i >= args.warmup:
            times.append(1e3 * (t1 - t0))
    return {"value": statistics.mean(times), "unit": "ms",
            "h2d_bytes_per_step": U.nbytes + eta.nbytes, "d2h_bytes_per_step": eta.nbytes}


def _variant(wd, U, eta, dev, stream, prec, tol, c12, options=None):
    import torch
    op = wd.WilsonDirac(DIMS, KAPPA, BC, prec, stream=stream)
    op.load_gauge(torch.from_numpy(U).to(dev), compress12=c12)
    for k, v in (options or {}).items():
        op.set_option(k, v)
    etad = torch.from_numpy(eta).to(dev)
    x = torch.zeros_like(etad)
    for _ in range(3):
        x.zero_()
        wd.cg_solve(op.ctx, etad, x, tol, MAXIT)
    ts = []
    for _ in range(5):
        x.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, it, res = wd.cg_solve(op.ctx, etad, x, tol, MAXIT)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    s = op.stats()
    dms = op.time_dslash(False, 200)
    op.close()
    return {"ms": statistics.mean(ts), "iterations": it, "true_rel_residual": res, "tol": tol,
            "reliable_updates": s["reliable_updates"], "dslash_launch_ms": dms}


def _sweep(wd, dev, stream, sizes):
    """Stand-alone dslash bandwidth sweep (links generated on the device, same recipe)."""
    out = []
    for L in sizes:
        dims = (L, L, L, L)
        V = L ** 4
        row = {"L": L, "V": V}
        for name, prec, c12, bps in (("f64_18r", wd.WD_PREC_F64, False, 960), ("f32_18r", wd.WD_PREC_F32, False, 480),
                                     ("f32_12r", wd.WD_PREC_F32, True, 384), ("f16_12r", wd.WD_PREC_MIXED_F16, True, 296)):
            op = wd.WilsonDirac(dims, KAPPA, BC, prec, stream=stream)
            op.generate_gauge(EPS, GAUGE_SEED, compress12=c12)
            ms = op.time_dslash(False, 50 if L >= 24 else 200)
            op.close()
            row[name] = {"ms": ms, "gbs": bps * V / (ms * 1e-3) / 1e9,
                         "gflops": FLOPS_PER_SITE * V / (ms * 1e-3) / 1e9}
        out.append(row)
    return out


def _paper_sizes(wd, stream):
    """Plain FP64 CG to 1e-10 over the paper's lattice sizes (4^4 to 14^4), same generator."""
    out = []
    for L in (4, 8, 12, 14):
        dims = (L, L, L, L)
        op = wd.WilsonDirac(dims, KAPPA, BC, wd.WD_PREC_F64, stream=stream)
        op.generate_gauge(EPS, GAUGE_SEED)
        eta = op.generate_source(SOURCE_SEED)
        _, rec = _timed_solve(op, wd, eta, TOL, repeats=3)
        st = op.stats()
        rec["L"] = L
        rec["gflops_1320"] = 2 * FLOPS_PER_SITE * L ** 4 * rec["iterations"] / (rec["ms"] * 1e-3) / 1e9
        rec["cg_loop"] = {0: "host loop", 1: "graph", 2: "persistent kernel"}[st["loop_mode"]]
        op.close()
        out.append(rec)
    return out


def _timed_solve(op, wd, eta, tol, repeats=1):
    import torch
    x = torch.zeros_like(eta)
    best = None
    for _ in range(repeats):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it, res = wd.cg_solve(op.ctx, eta, x, tol, 20000)
        t1 = time.perf_counter()
        best = min(best, t1 - t0) if best is not None else t1 - t0
    return x, {"ms": 1e3 * best, "iterations": it, "true_rel_residual": res, "status": st,
               "reliable_updates": op.stats()["reliable_updates"]}


def _mixed_32x64(wd, dev, stream):
    """Mixed precision at 32^3 x 64 (kappa 0.124) against plain FP64 CG on the same GPU."""
    import torch
    dims, kappa = (32, 32, 32, 64), 0.124
    out = {"workload": "32^3x64, kappa 0.124, eps 0.4, tol 1e-10, 1 RHS, FP32 12-real inner links",
           "reliable_delta": 0.1,
           "updates": "mixed_*: reliable-update residual and solution in double-float (FP32 pairs, ~48 bits); "
                      "mixed_*_fp64_updates: the same in native FP64; the final true residual is FP64 in both"}
    ref = wd.WilsonDirac(dims, kappa, BC, wd.WD_PREC_F64, stream=stream)
    ref.generate_gauge(EPS, GAUGE_SEED)
    eta = ref.generate_source(SOURCE_SEED)
    x64, out["plain_f64"] = _timed_solve(ref, wd, eta, TOL)
    for name, prec in (("mixed_f32", wd.WD_PREC_MIXED_F32), ("mixed_f16", wd.WD_PREC_MIXED_F16)):
        op = wd.WilsonDirac(dims, kappa, BC, prec, stream=stream)
        op.generate_gauge(EPS, GAUGE_SEED, compress12=True)
        x, rec = _timed_solve(op, wd, eta, TOL, repeats=2)
        rec["rel_diff_vs_f64_solution"] = float(torch.linalg.vector_norm(x - x64) / torch.linalg.vector_norm(x64))
        rec["speedup_vs_f64"] = out["plain_f64"]["ms"] / rec["ms"]
        out[name] = rec
        # the same solve with a reliable update every 100x drop of |r| instead of 10x
        op.set_option(wd.WD_OPT_RELIABLE_DELTA, 0.01)
        _, rec = _timed_solve(op, wd, eta, TOL, repeats=2)
        rec["speedup_vs_f64"] = out["plain_f64"]["ms"] / rec["ms"]
        out[name + "_delta_0.01"] = rec
        # reliable updates in native FP64 (residual recomputation and solution accumulation), as the
        # mixed-precision workload states them; the default above uses double-float for both
        op.set_option(wd.WD_OPT_RELIABLE_DELTA, 0.1)
        op.set_option(wd.WD_OPT_DF_UPDATES, 0)
        x, rec = _timed_solve(op, wd, eta, TOL, repeats=2)
        rec["rel_diff_vs_f64_solution"] = float(torch.linalg.vector_norm(x - x64) / torch.linalg.vector_norm(x64))
        rec["speedup_vs_f64"] = out["plain_f64"]["ms"] / rec["ms"]
        out[name + "_fp64_updates"] = rec
        op.close()
    ref.close()
    return out


def _multi_24x48(wd, dev, stream):
    """12 RHS at 24^3 x 48: spin-colour point sources at the origin, then 12 Gaussian sources."""
    import torch
    dims = (24, 24, 24, 48)
    lx, ly, lz, lt = dims
    out = {"workload": "24^3x48, kappa 0.12, eps 0.4, tol 1e-10 per RHS, FP32 inner + FP64 reliable updates"}
    op = wd.WilsonDirac(dims, KAPPA, BC, wd.WD_PREC_MIXED_F32, stream=stream)
    op.generate_gauge(EPS, GAUGE_SEED, compress12=True)
    point = torch.zeros((12, lt, lz, ly, lx, 4, 3), dtype=torch.complex128, device=dev)
    for k in range(12):
        point[k, 0, 0, 0, 0, k // 3, k % 3] = 1.0
    gauss = torch.stack([op.generate_source(100 + k) for k in range(12)])
    for name, src in (("point_sources", point), ("gaussian_sources", gauss)):
        x = torch.zeros_like(src)
        wd.cg_solve_multi(op.ctx, src, x, TOL, 20000)   # autotune + graph build on the first call
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, iters, res = wd.cg_solve_multi(op.ctx, src, x, TOL, 20000)
        t1 = time.perf_counter()
        ms = wd.wd_get_multi_stats(op.ctx)
        out[name] = {"ms": 1e3 * (t1 - t0), "status": st, "iterations_max": max(iters),
                     "iterations_min": min(iters), "true_rel_residual_max": max(res),
                     "reliable_updates": ms["reliable_updates"], "group_K": ms["group"],
                     "sites_per_block": ms["sites_per_block"], "multi_dslash_ms": ms["dslash_ms"]}
    # one right-hand side at a time with the same solver, for comparison
    x = torch.zeros_like(gauss[0])
    wd.cg_solve(op.ctx, gauss[0], x, TOL, 20000)
    t = []
    for k in range(12):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        wd.cg_solve(op.ctx, gauss[k], x, TOL, 20000)
        t.append(time.perf_counter() - t0)
    out["gaussian_one_at_a_time_mixed_ms"] = 1e3 * sum(t)
    op.close()
    # the same with FP16 spinors (per-site norm) in the inner solver
    op = wd.WilsonDirac(dims, KAPPA, BC, wd.WD_PREC_MIXED_F16, stream=stream)
    op.generate_gauge(EPS, GAUGE_SEED, compress12=True)
    x = torch.zeros_like(gauss)
    wd.cg_solve_multi(op.ctx, gauss, x, TOL, 20000)
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, iters, res = wd.cg_solve_multi(op.ctx, gauss, x, TOL, 20000)
    t1 = time.perf_counter()
    ms = wd.wd_get_multi_stats(op.ctx)
    out["f16_gaussian_sources"] = {"ms": 1e3 * (t1 - t0), "status": st, "iterations_max": max(iters),
                                   "true_rel_residual_max": max(res), "reliable_updates": ms["reliable_updates"],
                                   "group_K": ms["group"], "sites_per_block": ms["sites_per_block"]}
    x1 = torch.zeros_like(gauss[0])
    wd.cg_solve(op.ctx, gauss[0], x1, TOL, 20000)
    t = []
    for k in range(12):
        x1.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        wd.cg_solve(op.ctx, gauss[k], x1, TOL, 20000)
        t.append(time.perf_counter() - t0)
    out["f16_gaussian_one_at_a_time_ms"] = 1e3 * sum(t)
    op.close()
    # plain FP64, one right-hand side (x 12 for the batch-equivalent time)
    ref = wd.WilsonDirac(dims, KAPPA, BC, wd.WD_PREC_F64, stream=stream)
    ref.generate_gauge(EPS, GAUGE_SEED)
    _, rec = _timed_solve(ref, wd, gauss[0], TOL)
    out["plain_f64_one_rhs"] = rec
    out["plain_f64_x12_ms"] = 12 * rec["ms"]
    ref.close()
    return out


def _paper_coo(wd, dev, stream):
    """The paper's COO SpMV (Sec. 2) on this GPU at its largest lattice, 14^4, FP64."""
    import torch
    op = wd.WilsonDirac(DIMS, KAPPA, BC, wd.WD_PREC_F64, stream=stream)
    U = op.generate_gauge(EPS, GAUGE_SEED, return_field=True)
    row, col, val = wd.wd_coo_build(op.ctx, U)
    psi = op.generate_source(SOURCE_SEED)
    out = torch.empty_like(psi)
    for _ in range(3):
        wd.wd_coo_spmv(op.ctx, row, col, val, psi, out)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    a.record(stream)
    for _ in range(reps):
        wd.wd_coo_spmv(op.ctx, row, col, val, psi, out)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    nnz = row.numel()
    V = int(np.prod(DIMS))
    stencil_ms = op.time_dslash(False, 100)
    op.close()
    return {"workload": "14^4 FP64, D in COO (49 non-zeros per row), one thread per non-zero, atomic adds",
            "nnz": nnz, "spmv_ms": ms, "gflops_8_per_nonzero": 8 * nnz / (ms * 1e-3) / 1e9,
            "gflops_1320_per_site": FLOPS_PER_SITE * V / (ms * 1e-3) / 1e9,
            "stencil_dslash_ms": stencil_ms, "stencil_speedup": ms / stencil_ms,
            "paper_a100_gflops": 65}


def _even_odd(wd, dev, stream):
    """Even-odd (Schur) preconditioned solves against the unpreconditioned ones."""
    import torch
    out = {}
    for name, dims, kappa, prec in (("14x4_f64", DIMS, KAPPA, wd.WD_PREC_F64),
                                    ("14x4_mixed_f32", DIMS, KAPPA, wd.WD_PREC_MIXED_F32),
                                    ("32x64_mixed_f32", (32, 32, 32, 64), 0.124, wd.WD_PREC_MIXED_F32),
                                    ("32x64_mixed_f16", (32, 32, 32, 64), 0.124, wd.WD_PREC_MIXED_F16)):
        rec = {}
        for tag, flag in (("plain", 0), ("even_odd", wd.WD_EVEN_ODD)):
            op = wd.WilsonDirac(dims, kappa, BC, prec | flag, stream=stream)
            op.generate_gauge(EPS, GAUGE_SEED, compress12=prec != wd.WD_PREC_F64)
            eta = op.generate_source(SOURCE_SEED)
            _, r = _timed_solve(op, wd, eta, TOL, repeats=2)
            rec[tag] = r
            op.close()
        rec["speedup"] = rec["plain"]["ms"] / rec["even_odd"]["ms"]
        out[name] = rec
    return out


SERVE_SIZES = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (16, 16, 16, 32), (24, 24, 24, 48),
               (32, 32, 32, 64)]


def _serve_requests(n_req, rate, seed):
    """A seeded Poisson stream: sizes uniform over SERVE_SIZES, kappa U[0.115, 0.124], tol in
    {1e-8, 1e-10}, eps U[0.3, 0.5], a seeded gauge field and source per request."""
    rng = np.random.default_rng(seed)
    reqs, t = [], 0.0
    for i in range(n_req):
        t += rng.exponential(1.0 / rate)
        reqs.append(dict(t=t, dims=SERVE_SIZES[int(rng.integers(6))], kappa=float(rng.uniform(0.115, 0.124)),
                         tol=float([1e-8, 1e-10][int(rng.integers(2))]), eps=float(rng.uniform(0.3, 0.5)),
                         gauge_seed=10000 + i, source_seed=20000 + i))
    return reqs


def _serve_run(wd, reqs, precision, slots, max_batch, policy=0):
    srv = wd.Server(150e9, slots, max_batch=max_batch)
    srv.set_policy(policy, 1000.0)
    # one untimed request per size and slot first: the resident contexts, tuned launch shapes, graphs
    warm = [srv.submit(dims=d, kappa=0.12, eps=0.4, gauge_seed=1, source_seed=2, tol=1e-8, precision=precision)
            for d in SERVE_SIZES for _ in range(slots)]
    for w in warm:
        srv.wait(w)
    base = srv.stats()
    t0 = time.perf_counter()
    ids = []
    for q in reqs:
        dt = q["t"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(dims=q["dims"], kappa=q["kappa"], eps=q["eps"], gauge_seed=q["gauge_seed"],
                              source_seed=q["source_seed"], tol=q["tol"], precision=precision))
    res = [srv.wait(i) for i in ids]
    t1 = time.perf_counter()
    st = srv.stats()
    srv.close()
    lat = np.array([r["latency_ms"] for r in res])
    worst = max((r["true_rel_residual"] / q["tol"]) for r, q in zip(res, reqs))
    by_size = {}
    for d in SERVE_SIZES:
        sel = [r for r, q in zip(res, reqs) if q["dims"] == d]
        if sel:
            ls = np.array([r["latency_ms"] for r in sel])
            by_size["x".join(str(v) for v in d)] = {
                "requests": len(sel), "p50_ms": float(np.percentile(ls, 50)), "p99_ms": float(np.percentile(ls, 99)),
                "mean_solve_ms": float(np.mean([r["solve_ms"] for r in sel])),
                "mean_batch": float(np.mean([r["batch"] for r in sel]))}
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_solve_ms": float(np.mean([r["solve_ms"] for r in res])),
            "solves_per_s": len(res) / (t1 - t0), "wall_s": t1 - t0,
            "completed_ok": sum(1 for r in res if r["status"] == 0), "requests": len(res),
            "max_true_residual_over_tol": float(worst), "slots": slots, "max_batch": max_batch,
            "policy": ["oldest first", "least work first, oldest first after 1 s"][policy],
            "batches": st["batches"] - base["batches"],
            "batched_requests": st["batched_requests"] - base["batched_requests"],
            "warm_hits": st["warm_hits"] - base["warm_hits"], "evictions": st["evictions"],
            "peak_gb": st["peak_bytes"] / 1e9, "by_size": by_size}


def _serving(wd, seed=7):
    """Poisson streams of single-RHS solves through the serving runtime (continuous admission, batches of
    same-operator requests where the persistent loop serves them: 8^4 and 12^4 in mixed precision).
    Above saturation (200 requests/s offered, 500 requests) and below it (15/s, 300 requests); mixed
    precision on 4 slots with and without batching, with least-work-first admission (aging after
    1 s), on 1 slot, with even-odd preconditioning, and
    plain FP64 one at a time (a 100-request sample: it serves about 4 solves/s). 150 GB budget."""
    hi = _serve_requests(500, 200.0, seed)
    lo = _serve_requests(300, 15.0, seed + 1)
    out = {"workload": "Poisson arrivals, sizes uniform over 8^4, 12^4, 16^4, 16^3x32, 24^3x48, 32^3x64, "
                       "kappa U[0.115,0.124], tol {1e-8,1e-10}, eps U[0.3,0.5], 150 GB budget"}
    out["mixed_f32_4_slots_batched_200_per_s"] = _serve_run(wd, hi, wd.WD_PREC_MIXED_F32, 4, 8)
    out["mixed_f32_4_slots_unbatched_200_per_s"] = _serve_run(wd, hi, wd.WD_PREC_MIXED_F32, 4, 1)
    out["mixed_f32_4_slots_batched_least_work_first_200_per_s"] = _serve_run(wd, hi, wd.WD_PREC_MIXED_F32, 4, 8,
                                                                            policy=1)
    out["mixed_f32_1_slot_batched_200_per_s"] = _serve_run(wd, hi, wd.WD_PREC_MIXED_F32, 1, 8)
    out["mixed_f32_4_slots_batched_15_per_s"] = _serve_run(wd, lo, wd.WD_PREC_MIXED_F32, 4, 8)
    out["mixed_f32_even_odd_4_slots_200_per_s"] = _serve_run(wd, hi, wd.WD_PREC_MIXED_F32 | wd.WD_EVEN_ODD, 4, 8)
    out["plain_f64_1_slot_200_per_s_100_requests"] = _serve_run(wd, hi[:100], wd.WD_PREC_F64, 1, 1)
    return out


def _cpu_baseline(gpu_iters):
    """The oracle on the host cores: the whole 14^4 solve (the headline workload, ~30 s), the whole
    4^4 solve, and one oracle dslash per sweep volume (unit links: the oracle's arithmetic does not
    depend on the link values)."""
    import synthetic
    from oracle import cg as ocg
    from oracle import wilson as owil
    U, eta = make_inputs(DIMS)
    c0 = time.process_time()
    t0 = time.perf_counter()
    _, it, res, _ = ocg.cgls(U, eta, KAPPA, TOL, MAXIT)
    wall = time.perf_counter() - t0
    busy = (time.process_time() - c0) / wall
    ms = 1e3 * wall
    out = {"value": ms, "unit": "ms", "cores": os.cpu_count(), "avg_busy_cores": busy, "kind": "oracle",
           "sample": f"one whole oracle solve of the 14^4 workload (FP64 numpy CGLS: einsum contractions on "
                     f"one thread, dot products on OpenBLAS threads; {busy:.1f} of {os.cpu_count()} cores busy "
                     f"on average): {it} iterations (GPU: {gpu_iters}), true residual {res:.2e}",
           "iterations": int(it), "true_rel_residual": float(res)}
    U4, eta4 = make_inputs((4, 4, 4, 4))
    t0 = time.perf_counter()
    _, it4, res4 = ocg.cgls(U4, eta4, KAPPA, TOL, 2000)[:3]
    out["solve_4x4_ms"] = 1e3 * (time.perf_counter() - t0)
    out["solve_4x4_iterations"] = int(it4)
    out["solve_4x4_true_rel_residual"] = float(res4)
    sweep = {}
    for L in (8, 12, 14, 16, 24, 32):
        d = (L, L, L, L)
        Ul, psi = synthetic.unit_gauge(d), synthetic.gaussian_source(d, SOURCE_SEED)
        t0 = time.perf_counter()
        owil.apply_D(Ul, psi, KAPPA)
        sweep[str(L)] = 1e3 * (time.perf_counter() - t0)
        del Ul, psi
    out["dslash_ms_by_L"] = sweep
    return out


# ---------------------------------------------------------------------------- profiling cases

# Small, self-contained workloads for capturing one kernel under ncu (the commands in profiles/):
#   python bench.py --profile-case --prec 64 --dims 14,14,14,14 --launches 5
#   python bench.py --profile-case --prec 32 --c12 --dims 32,32,32,32 --launches 3
#   python bench.py --profile-case --prec 64 --dims 14,14,14,14 --launches 0 --solve
#   python bench.py --profile-case --prec 6432 --c12 --dims 16,16,16,16 --launches 0 --apply 3 --apply-df
#   python bench.py --profile-case --prec 6432 --c12 --dims 16,16,16,32 --launches 0 --multi 12
#   python bench.py --profile-case --prec 6432 --c12 --dims 24,24,24,48 --launches 0 --device-fields --msolve 12
# Fields come from the seeded generators (links exp(i 0.4 H), Gaussian source; on the host, or with
# --device-fields from the library's own generators on the device); the program prints the timing
# of the dslash as the solver launches it (CUDA events) and, with --solve, one CG solve.

def profile_case(argv):
    ap = argparse.ArgumentParser(prog="bench.py --profile-case")
    ap.add_argument("--prec", type=int, default=64, help="64, 32, 6432 or 6416")
    ap.add_argument("--dims", default="14,14,14,14")
    ap.add_argument("--c12", action="store_true")
    ap.add_argument("--launches", type=int, default=5)
    ap.add_argument("--dagger", action="store_true")
    ap.add_argument("--solve", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--kappa", type=float, default=0.12)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--variant", type=int, default=0, help="WD_OPT_DSLASH_VARIANT (FP64: 1..5 = 1..16 lanes per site)")
    ap.add_argument("--apply", type=int, default=0, help="wd_apply calls on a Gaussian field")
    ap.add_argument("--apply-df", action="store_true",
                    help="mixed-precision contexts: wd_apply through the double-float operator")
    ap.add_argument("--even-odd", action="store_true")
    ap.add_argument("--multi", type=int, default=0, help="wd_apply_multi calls on this many Gaussian fields")
    ap.add_argument("--mgroup", type=int, default=0, help="multi-RHS group size K (0 = tuned)")
    ap.add_argument("--msites", type=int, default=0, help="multi-RHS sites per block (0 = tuned)")
    ap.add_argument("--mkt", type=int, default=0, help="multi-RHS right-hand sides per thread (0 = tuned)")
    ap.add_argument("--msolve", type=int, default=0, help="one cg_solve_multi on this many Gaussian sources")
    ap.add_argument("--device-fields", action="store_true", help="generate links and sources on the device")
    ap.add_argument("--graph", type=int, default=-1,
                    help="WD_OPT_USE_GRAPH for the solves (0 = plain launches, which ncu lists one by one)")
    ap.add_argument("--tma", type=int, default=0, help="WD_OPT_DSLASH_TMA (FP32 12-real: 1 or 2 = TMA-staged tiles)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="WD_OPT_DSLASH_SCHEDULE (FP32 / FP16: 1 hop by hop, 2 two sites per thread, "
                         "3 both hops of a direction loaded together; 0 = tuned)")
    ap.add_argument("--apply-inner", action="store_true",
                    help="mixed-precision contexts: wd_apply through the inner FP32 / FP16 operator")
    args = ap.parse_args(argv)

    import torch

    import synthetic
    from paper_2111_14958_gb300 import wd

    dims = tuple(int(v) for v in args.dims.split(","))
    prec = args.prec | (wd.WD_EVEN_ODD if args.even_odd else 0)
    op = wd.WilsonDirac(dims, args.kappa, (1, 1, 1, -1), prec)
    if args.device_fields:
        op.generate_gauge(0.4, 1, compress12=args.c12)
    else:
        op.load_gauge(torch.from_numpy(synthetic.gauge_field(dims, 0.4, 1)).cuda(), compress12=args.c12)

    def source(seed):
        if args.device_fields:
            return op.generate_source(seed)
        return torch.from_numpy(synthetic.gaussian_source(dims, seed)).cuda()
    if args.block:
        op.set_option(wd.WD_OPT_BLOCK_DSLASH, args.block)
    if args.variant:
        op.set_option(wd.WD_OPT_DSLASH_VARIANT, args.variant)
    if args.tma:
        op.set_option(wd.WD_OPT_DSLASH_TMA, args.tma)
    if args.schedule:
        op.set_option(wd.WD_OPT_DSLASH_SCHEDULE, args.schedule)
    if args.graph >= 0:
        op.set_option(wd.WD_OPT_USE_GRAPH, args.graph)
    if args.launches:
        ms = op.time_dslash(args.dagger, args.launches)
        print(f"dslash dims={dims} prec={args.prec} c12={args.c12}: {ms * 1e3:.2f} us per launch")
    if args.apply:
        if args.apply_df:
            op.set_option(wd.WD_OPT_APPLY_DF, 1)
        if args.apply_inner:
            op.set_option(wd.WD_OPT_APPLY_INNER, 1)
        psi = source(3)
        if args.prec == wd.WD_PREC_F32:
            psi = psi.to(torch.complex64)
        out = torch.empty_like(psi)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.apply):
            op.apply(psi, out=out)
        b.record()
        torch.cuda.synchronize()
        print(f"wd_apply x{args.apply}: {a.elapsed_time(b) / args.apply * 1e3:.2f} us per call (with packing)")
    if args.multi:
        if args.mgroup:
            op.set_option(wd.WD_OPT_MULTI_GROUP, args.mgroup)
        if args.msites:
            op.set_option(wd.WD_OPT_MULTI_SITES, args.msites)
        if args.mkt:
            op.set_option(wd.WD_OPT_MULTI_RHS_PER_THREAD, args.mkt)
        psi = torch.stack([source(10 + i) for i in range(args.multi)])
        out = op.apply_multi(psi)  # tunes the launch shape
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            out = op.apply_multi(psi)
        b.record()
        torch.cuda.synchronize()
        st = op.multi_stats()
        print(f"wd_apply_multi x3 ({args.multi} RHS): {a.elapsed_time(b) / 3 * 1e3:.1f} us per call with packing; "
              f"tuned group {st['group']} sites/block {st['sites_per_block']} dslash {st['dslash_ms'] * 1e3:.1f} us")
    if args.msolve:
        eta = torch.stack([source(100 + i) for i in range(args.msolve)])
        x = torch.zeros_like(eta)
        wd.cg_solve_multi(op.ctx, eta, x, args.tol, 20000)  # tunes the launch shapes
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, iters, res = wd.cg_solve_multi(op.ctx, eta, x, args.tol, 20000)
        t1 = time.perf_counter()
        ms = wd.wd_get_multi_stats(op.ctx)
        print(f"cg_solve_multi ({args.msolve} RHS): status {st} iterations {max(iters)} "
              f"max true residual {max(res):.3e} reliable updates {ms['reliable_updates']} "
              f"group {ms['group']} sites/block {ms['sites_per_block']} ms {1e3 * (t1 - t0):.1f}")
    if args.solve:
        eta = source(2)
        x, iters, res, status = op.solve(eta, tol=args.tol, maxit=4000)
        s = op.stats()
        print(f"solve: status {status} iterations {iters} true residual {res:.3e} "
              f"reliable updates {s['reliable_updates']} host ms {s['solve_ms']:.3f}")
    op.close()
    return 0



def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--profile-case":
        return profile_case(sys.argv[2:])
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--quick", action="store_true", help="only the headline step (for profiling)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the solver's kernels one by one instead of as a CUDA graph (for "
                         "ncu launch lists, which do not list kernels inside conditional graph nodes)")
    ap.add_argument("--sweep", default="4,8,12,14,16,24,32")
    args = ap.parse_args()
    args.sweep = [int(v) for v in args.sweep.split(",") if v]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "native":
        import torch
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_native(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
