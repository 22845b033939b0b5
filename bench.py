#!/usr/bin/env python
"""Benchmark of the RAPRAL hot path on GB300.

A step is one whole solve of the stagnation-line workload (200 two-temperature
cells, 20,000 atomic + 300,000 molecular lines, 1,000,000-point grid over
50-2000 nm, 16-direction tangent slab plus the normal ray): populations ->
line binning -> line-by-line kappa / j -> ray march -> wall flux, with inputs
resident in HBM.  The FP32-chosen arithmetic is the headline; the FP64-plain
path on the same workload is measured beside it.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "cell·λ coeff points/s and ray·λ segments/s; served q_rad p50/p99 vs FP64 plain"
WORKLOAD = "stagnation line: 200 cells, 20k atomic + 300k molecular lines, 1e6-point grid 50-2000 nm, 16-mu tangent slab"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 20 for the stagnation-line step, 5 for the other workloads)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["rapral", "reference"], default="rapral")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-plain side measurement")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-serve", action="store_true", help="skip the served-requests measurement")
    ap.add_argument("--serve-requests", type=int, default=40)
    ap.add_argument("--serve-fp64-requests", type=int, default=4)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default tiling)")
    ap.add_argument("--workload", choices=["stagnation", "afterbody", "batch", "fibonacci", "qss", "continuum", "voigt"],
                    default="stagnation",
                    help="stagnation line (the bench line); afterbody / batch / fibonacci / qss / continuum / "
                         "voigt (the stagnation step with the exact Voigt shape): one-off measurements")
    ap.add_argument("--cont-levels", type=int, default=100, help="continuum workload: levels per atom (N, O)")
    ap.add_argument("--cont-points", type=int, default=1_000_000,
                    help="continuum workload: grid points (fewer only for profiler captures)")
    ap.add_argument("--fib-points", type=int, default=8, help="fibonacci workload: surface points")
    ap.add_argument("--fib-los", type=int, default=128, help="fibonacci workload: Fibonacci directions per point")
    ap.add_argument("--ab-small", action="store_true",
                    help="afterbody workload at 100 x 50 cells, 20 points, 2e5 grid points (profiler captures)")
    ap.add_argument("--cells", type=int, default=200,
                    help="cells of the stagnation line (fewer only for profiler captures)")
    ap.add_argument("--oracle-phases", action="store_true",
                    help="with --impl reference: the oracle's time per phase, all threads and one thread")
    args = ap.parse_args()
    if args.steps is None:   # the stagnation step takes ~31 ms: 20 steps give the clock sampler a few samples
        args.steps = 20 if (args.impl == "rapral" and args.workload == "stagnation") else 5
    return args


# DRAM bytes (read + write) of one timed FP32 line-sum launch on the stagnation line
# at full size (200 cells x 1e6 points, tiling 128 x 2), from a one-pass ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel source
# with this digest (source_digest).  Other cell / point counts scale in proportion (the bytes are
# the kappa / j rows written); a different source (comments aside) gives null.
LINE_SUM_TRAFFIC = {"sha1": "ee162f14b8a843d46ca76ea6702ffe0ac1880911", "cells": 200, "grid_points": 1_000_000,
                    "bytes": 55_467_776 + 1_546_483_712}


# DRAM bytes of one FP32 continuum level-sum launch at full size (200 cells x
# 1e6 points, N and O with 100 levels each), from a one-pass ncu capture of the
# kernel source with this digest (source_digest); a different source gives null.
CONT_TRAFFIC = {"sha1": "5acd74ef87910912678c8d6546c788ab0f5e87b0", "cells": 200, "grid_points": 1_000_000, "levels": 100,
                "bytes": 1_782_956_800 + 1_538_739_456}


def source_digest(name):
    """SHA-1 of a kernel source with its comments and white space removed, so
    that only a change of the code itself invalidates a stored measurement."""
    import hashlib
    import re
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2604_11856_gb300", "csrc", name)
    try:
        text = open(src).read()
    except OSError:
        return None
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return hashlib.sha1(re.sub(r"\s+", "", text).encode()).hexdigest()


def continuum_traffic(cells, grid_points, levels):
    digest = source_digest("k_continuum.cu")
    t = CONT_TRAFFIC
    if digest != t["sha1"] or (cells, grid_points, levels) != (t["cells"], t["grid_points"], t["levels"]):
        return None
    return t["bytes"]


def line_sum_traffic(cells, grid_points):
    digest = source_digest("k_lines.cu")
    if digest != LINE_SUM_TRAFFIC["sha1"]:
        return None
    t = LINE_SUM_TRAFFIC
    return t["bytes"] * (cells / t["cells"]) * (grid_points / t["grid_points"])


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower().startswith("active")})
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def measured_peaks():
    try:
        return json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def cpu_baseline(problem, seconds, precision_note="f64"):
    """The oracle as it stands, on the host cores, on a bounded sample of the
    workload: every line, the whole grid, a few cells (one per thread), for
    about `seconds`; reported as coefficient cell*lambda points per second."""
    import oracle
    from paper_2604_11856_gb300 import synth
    threads = oracle.lib().orc_num_threads()
    p = problem
    # first estimate with one cell per thread on a 1/20 slice of the grid
    n_cells = max(1, threads)
    idx = np.linspace(0, len(p.cells) - 1, n_cells).round().astype(int)
    cells = synth.Cells(Ttr=p.cells.Ttr[idx], Tve=p.cells.Tve[idx], n=p.cells.n[idx])
    sub = synth.Problem(p.name, p.species, p.lines, cells, p.grid, p.geometry)
    lnp = oracle.lnpref(sub)
    nk = p.grid.n // 20
    t0 = time.perf_counter()
    oracle.spectral_coeffs(sub, lnp, 0, nk)
    dt = time.perf_counter() - t0
    # grow the slice towards the time budget
    nk2 = int(min(p.grid.n, nk * max(1.0, seconds / max(dt, 1e-3))))
    k0 = (p.grid.n - nk2) // 2
    t0 = time.perf_counter()
    oracle.spectral_coeffs(sub, lnp, k0, nk2)
    dt2 = time.perf_counter() - t0
    return {"value": n_cells * nk2 / dt2, "unit": "cell·λ points/s", "cores": threads, "kind": "oracle",
            "sample": f"{n_cells} of {len(p.cells)} cells x {nk2} of {p.grid.n} grid points, all "
                      f"{len(p.lines)} lines, kappa and j in FP64 ({dt2:.1f} s)", "seconds": dt2}


def served(p, args, device):
    """Open-loop served requests (line-of-sight and slab solves, config-4
    sizes) sharing the resident stagnation-line lists; FP32-chosen vs FP64
    plain on the same requests (FP64 on the first few only: it is ~80x
    slower)."""
    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import serve, synth
    pool = (p.lines, p.species, {})
    gen = synth.served_requests(seed=1004, n_requests=args.serve_requests, rate=args.serve_rate, pool=pool)
    res = {"offered_rate_req_s": args.serve_rate, "slots": 4, "budget_bytes": 150 << 30}
    q32 = {}
    for prec, n, name in ((R.FP32, args.serve_requests, "fp32"), (R.FP64, args.serve_fp64_requests, "fp64")):
        if n <= 0:
            continue
        reqs = [serve.Request(rid=i, problem=g["problem"], arrival=g["t"], precision=prec)
                for i, g in enumerate(gen[:n])]
        srv = serve.Server(p.lines, p.species, device=device, slots=4)
        res[name] = serve.run_open_loop(srv, reqs)
        if prec == R.FP32:
            q32 = {r.rid: r.q for r in reqs if r.status == "done"}
        else:
            errs = [float(np.max(np.abs(q32[r.rid] / r.q - 1))) for r in reqs if r.status == "done" and r.rid in q32]
            res["q_rel_err_fp32_vs_fp64_max"] = max(errs) if errs else None
    return res


def run_reference(args):
    """--impl reference: the oracle on the host cores, bounded samples of the
    bench workload per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2604_11856_gb300 import synth
    p = synth.stagnation_line()
    per_step = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(p, per_step / 4)
    vals, secs = [], []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(p, per_step)
        vals.append(last["value"])
        secs.append(last.pop("seconds"))
    v = float(np.mean(vals))
    # a step here is one bounded sample of the workload, not the whole 200-cell step
    line = {"metric": METRIC, "value": v, "unit": "cell·λ points/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3, "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": last["sample"]},
            "cpu_baseline": {**last, "value": v},
            "e2e": {"value": v, "unit": "cell·λ points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def oracle_phases(args):
    """--impl reference --oracle-phases: wall-clock of the oracle as it stands,
    per phase (populations, coefficients, march with the angular sum, spectral
    integral), with all OpenMP threads and with one.  The uniform slab runs
    whole.  On the stagnation line the populations run whole, the
    coefficients on a sample of cells over the whole grid (one cell per
    thread; two cells on one thread), projected by the cell ratio, and the
    march and spectral integral over every cell and direction on a
    5,000-point slice in the middle of the grid, projected by the column
    ratio.  One JSON line per (workload, threads)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2604_11856_gb300 import synth
    lib = oracle.lib()
    n_all = lib.orc_num_threads()
    cases = (("uniform slab: 20 cells, 1,500 atomic lines, 2e5-point grid, 16-mu tangent slab + normal ray",
              synth.uniform_slab(), False),
             ("stagnation line: 200 cells, 20k atomic + 300k molecular lines, 1e6-point grid, 16-mu tangent slab",
              synth.stagnation_line(), True))
    for name, p, sampled in cases:
        K, C = p.grid.n, len(p.cells)
        geo = p.geometry
        order = np.asarray(geo.cell_order, np.int64)
        w = 2.0 * np.pi * np.asarray(geo.wmu) * np.asarray(geo.mu)
        lnp = oracle.lnpref(p)
        k0, nk = ((K - 5000) // 2, 5000) if sampled else (0, K)
        kap, em = oracle.spectral_coeffs(p, lnp, k0, nk)    # the march's input (timed below when whole)
        for threads in (n_all, 1):
            lib.orc_set_threads(threads)
            t, full, sample = {}, {}, {}
            t0 = time.perf_counter()
            lnp = oracle.lnpref(p)
            t["populations"] = full["populations"] = time.perf_counter() - t0
            if sampled:
                n_c = threads if threads > 1 else 2
                idx = np.linspace(0, C - 1, n_c).round().astype(int)
                sub = synth.Problem(p.name, p.species, p.lines,
                                    synth.Cells(Ttr=p.cells.Ttr[idx], Tve=p.cells.Tve[idx], n=p.cells.n[idx]),
                                    p.grid, geo)
                t0 = time.perf_counter()
                oracle.spectral_coeffs(sub, lnp[idx], 0, K)
                t["coefficients"] = time.perf_counter() - t0
                full["coefficients"] = t["coefficients"] * C / n_c
                sample["coefficients"] = f"{n_c} of {C} cells, whole grid"
            else:
                t0 = time.perf_counter()
                oracle.spectral_coeffs(p, lnp, 0, K)
                t["coefficients"] = full["coefficients"] = time.perf_counter() - t0
            t0 = time.perf_counter()
            qlam = np.zeros(nk)
            for m, mu in enumerate(geo.mu):
                qlam += w[m] * oracle.march(order, geo.dx, 1.0 / mu, kap, em, p.grid, k0, geo.wall_start, geo.T_wall)
            if geo.normal_ray:
                oracle.march(order, geo.dx, 1.0, kap, em, p.grid, k0, geo.wall_start, geo.T_wall)
            t["march_angular"] = time.perf_counter() - t0
            t0 = time.perf_counter()
            oracle.spectral_integral(qlam, p.grid, k0)
            t["spectral_integral"] = time.perf_counter() - t0
            for k in ("march_angular", "spectral_integral"):
                full[k] = t[k] * K / nk
                if sampled:
                    sample[k] = f"all cells and directions, {nk} of {K} grid points"
            print(json.dumps({"impl": "reference", "kind": "oracle phases", "workload": name, "threads": threads,
                              "seconds_run": t, "sample": sample, "seconds_projected_full": full,
                              "total_projected_s": sum(full.values()),
                              "cell_lambda_per_s": C * K / full["coefficients"]}))
    lib.orc_set_threads(n_all)
    return 0


def run_afterbody(args):
    """The axisymmetric afterbody (80,000 cells, 1e6 points in 65,536-point
    chunks, 102,400 rays): one FP32 solve with the two-stream chunk pipeline."""
    import torch
    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import solver, synth
    if args.ab_small:
        p = synth.afterbody(nx=100, nr=50, n_points=20, n_grid=200_000)
    else:
        p = synth.afterbody()
    ctx = R.Context(0)
    ctx2 = R.Context(0, stream=torch.cuda.Stream())
    dp = solver.DeviceProblem(p, ctx)
    ctx.sync()
    bufs = [(torch.empty((dp.C, p.chunk), dtype=torch.float32, device=ctx.device),
             torch.empty((dp.C, p.chunk), dtype=torch.float32, device=ctx.device)) for _ in range(2)]
    for _ in range(args.warmup):
        solver.solve(dp, ctx, R.FP32, chunk=p.chunk, ctx2=ctx2, buffers=bufs)
    ctx.sync(); ctx2.sync()
    ms = []
    with ClockSampler(0) as clk:
        for i in range(max(1, args.steps)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream)
            out = solver.solve(dp, ctx, R.FP32, chunk=p.chunk, ctx2=ctx2, buffers=bufs)
            b.record(ctx.stream)
            ctx.sync(); ctx2.sync()
            ms.append(a.elapsed_time(b))
    t = float(np.mean(ms)) * 1e-3
    nseg = dp.rays.struct.n_segments
    # the march alone on one full chunk (its kappa / j computed first, untimed), L2
    # flushed before each repetition: segment-wavelengths per second and the
    # effective gather bandwidth (8 B of kappa + j per segment-wavelength)
    nk = min(p.chunk, p.grid.n)
    kap, em = bufs[0]
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, nk, R.FP32, kap, em)
    qlam = torch.empty((dp.P, nk), dtype=torch.float32, device=ctx.device)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=ctx.device)
    mm = []
    for rep in range(4):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(ctx.stream)
        R.trace_rays(ctx, dp.rays, dp.C, kap, em, p.grid, 0, nk, R.FP32, qlam)
        b.record(ctx.stream)
        ctx.sync()
        if rep:
            mm.append(a.elapsed_time(b))
    tm = float(np.mean(mm)) * 1e-3
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gather = nseg * nk * 8 / tm / 1e9
    march = {"kernel": "k_march (single-direction rays)", "chunk_points": nk, "kernel_ms": tm * 1e3,
             "ray_lambda_segments_per_s": nseg * nk / tm, "gather_GBps_effective": gather,
             "hbm_peak_GBps": hbm, "gather_over_hbm_peak": gather / hbm,
             "unique_kappa_j_bytes": dp.C * nk * 8,
             "note": "kappa / j rows are gathered from L2 (one DRAM pass per chunk): bound by issue, not HBM"}
    g = p.geometry
    desc = (f"afterbody {len(g.xf) - 1}x{len(g.rf) - 1} cells, {len(p.lines) // 1000}k lines, {p.grid.n:.0e} points "
            f"in {p.chunk}-point chunks, {len(g.surf_x)} points x {len(g.mu) * g.n_phi} rays")
    print(json.dumps({"workload": desc, "warmup": args.warmup, "steps": max(1, args.steps), "ms_per_solve": t * 1e3,
                      "cell_lambda_per_s": dp.C * p.grid.n / t, "ray_lambda_segments_per_s": nseg * p.grid.n / t,
                      "segments": int(nseg), "q_mean_W_cm2": float(out["q"].mean().item()), "clocks": clk.summary(),
                      "march": march}))
    return 0


def run_batch(args):
    """64 uneven uniform-slab solves (FP32): one persistent line-sum launch per
    spectral round, the whole run captured in one CUDA graph, against the
    same solves run one after another."""
    import torch
    from paper_2604_11856_gb300 import autotune, batch, rapral as R, solver, synth
    probs = synth.batch_slabs()
    ctx = R.Context(0)
    tw, wpb, times = autotune.tune(ctx, max(probs, key=lambda q: len(q.lines)))
    bs = batch.BatchSolver(probs, ctx, chunk=65536)
    bs.run(); ctx.sync()
    bs.capture()
    bs.replay(); torch.cuda.synchronize()
    ms = []
    for _ in range(max(1, args.steps)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(); bs.replay(); b.record(); torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.mean(ms)) * 1e-3
    cl = sum(len(q.cells) * q.grid.n for q in probs)
    # the same solves one after another through the regular entry points
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dps = [solver.DeviceProblem(q, ctx) for q in probs]
    ctx.sync()
    a.record(ctx.stream)
    for dp in dps:
        solver.solve(dp, ctx, R.FP32, chunk=65536)
    b.record(ctx.stream)
    ctx.sync()
    t_seq = a.elapsed_time(b) * 1e-3
    print(json.dumps({"workload": "64 uneven slab solves (cells 20-2000, 1e5-2e6 points, 1e3-5e4 atomic + "
                                  "0-3e5 molecular lines)", "tiling": [tw, wpb], "graph_ms": t * 1e3,
                      "cell_lambda_per_s": cl / t, "sequential_ms": t_seq * 1e3,
                      "sequential_cell_lambda_per_s": cl / t_seq, "rounds": len(bs.handles),
                      "units": bs.units()[:3]}))
    return 0


def run_qss(args):
    """QSS collisional-radiative populations of atomic N and O (32 solved +
    4 lumped levels each, 496 transitions) in every cell of the 400 x 200
    afterbody: one FP64 LU-solved system per (cell, atom)."""
    import torch
    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import synth
    p = synth.afterbody(n_points=2, n_grid=11)
    ctx = R.Context(0)
    models = [R.DeviceCrModel(synth.cr_model(species=s, n_levels=32, n_lumped=4, seed=1005 + i), ctx.device)
              for i, s in enumerate(("N", "O"))]
    dc = R.DeviceCells(p.cells, 8, ctx.device)
    C = len(p.cells.Ttr)
    outs = [torch.empty((C, m.l), dtype=torch.float64, device=ctx.device) for m in models]
    run = lambda: [R.qss_populations(ctx, m, dc, o) for m, o in zip(models, outs)]
    for _ in range(max(1, args.warmup)):
        run()
    ctx.sync()
    ms = []
    with ClockSampler(0) as clk:
        for _ in range(max(1, args.steps)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream)
            run()
            b.record(ctx.stream)
            ctx.sync()
            ms.append(a.elapsed_time(b))
    t = float(np.mean(ms)) * 1e-3
    systems = C * len(models)
    l = models[0].l
    # LU of an l x l system: 2 l^3 / 3 flops (the rate assembly, 2 pow + 2 exp a transition, not counted)
    print(json.dumps({"workload": f"QSS populations, {C} afterbody cells x 2 atoms (N, O), {l} levels + 4 lumped, "
                                  f"{l * (l - 1) // 2} transitions, FP64", "warmup": args.warmup,
                      "steps": max(1, args.steps), "ms_per_solve": t * 1e3, "systems_per_s": systems / t,
                      "lu_gflops": systems * 2.0 * l ** 3 / 3.0 / t / 1e9, "clocks": clk.summary()}))
    return 0


def continuum_terms(models, grid, C, W=128):
    """(cell, level, point) terms of the continuum level sums: per tile of W
    points the levels whose table reaches the tile's first wavelength."""
    last = np.concatenate([m["node_lam"][m["node_off"][1:] - 1] for m in models])
    h = (grid.lam_max - grid.lam_min) / (grid.n - 1)
    T = (grid.n + W - 1) // W
    lam0 = grid.lam_min + (np.arange(T) * W).astype(np.float64) * h
    n = (last[None, :] >= lam0[:, None]).sum(1)
    return int(C * n.sum() * W), int(n.sum() * W)


def run_continuum(args):
    """Atomic continuum (bound-free + free-free of N and O, 100 levels each)
    added to the coefficients of the 200-cell, 1e6-point stagnation line."""
    import torch
    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import solver, synth
    p = synth.stagnation_line(n_cells=args.cells, n_atomic=200, n_molecular=300, n_grid=args.cont_points)
    ctx = R.Context(0)
    models = [synth.continuum_model(species=s, n_levels=args.cont_levels, seed=1007 + i)
              for i, s in enumerate(("N", "O"))]
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    dc = R.DeviceContinuum(models, ctx.device)
    C, K = dp.C, p.grid.n
    out = {}
    terms, table_entries = continuum_terms(models, p.grid, C)
    for prec, dt, name in ((R.FP32, torch.float32, "fp32"), (R.FP64, torch.float64, "fp64")):
        kap = torch.zeros((C, K), dtype=dt, device=ctx.device)
        em = torch.zeros_like(kap)
        run = lambda: R.continuum_coeffs(ctx, dc, dp.species.S, dp.cells, p.grid, 0, K, prec, kap, em)
        for _ in range(max(3, args.warmup)):
            run()
        ctx.sync()
        steps = max(1, args.steps)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in kev:
            a.record(ctx.stream); b.record(ctx.stream)
        ctx.sync()
        with ClockSampler(0) as clk:
            for i in range(steps):
                ev[i][0].record(ctx.stream)
                ctx.set_profile_events(*kev[i])
                run()
                ctx.set_profile_events(None, None)
                ev[i][1].record(ctx.stream)
            ctx.sync()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        kms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
        esz = 4 if prec == R.FP32 else 8
        # algorithmic bytes of the level-sum kernel: kappa and j read and written once, the resampled tables read once
        nbytes = C * K * 4 * esz + table_entries * esz
        peaks = measured_peaks()
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        out[name] = {"ms_per_call": ms, "value": C * K / (ms * 1e-3), "kernel_ms": kms,
                     "roofline": {"bound": "hbm", "achieved": nbytes / (kms * 1e-3) / 1e9, "peak": hbm,
                                  "unit": "GB/s", "frac": nbytes / (kms * 1e-3) / 1e9 / hbm,
                                  "traffic": continuum_traffic(C, K, args.cont_levels) if esz == 4 else None,
                                  "kernel": f"k_continuum<{'float, 4, 4' if esz == 4 else 'double, 4, 2'}>",
                                  "algorithmic_bytes": nbytes,
                                  "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback"},
                     "clocks": clk.summary()}
        del kap, em
    print(json.dumps({"workload": f"atomic continuum (bound-free + free-free, N and O, {args.cont_levels} levels "
                                  f"each) on the stagnation line, {C} cells x {K} points",
                      "metric": "cell·λ points/s", "terms_per_call": terms, "warmup": args.warmup,
                      "steps": max(1, args.steps), **out}))
    return 0


def run_voigt(args):
    """The stagnation-line step (200 cells, 320k lines, 1e6 points) with the
    exact Voigt line shape instead of Whiting's: FP32 step and line-sum
    times, and one FP64 step."""
    import torch
    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import solver, synth
    p = synth.stagnation_line(n_cells=args.cells)
    ctx = R.Context(0)
    ctx.set_profile(R.PROFILE_VOIGT)
    dp = solver.DeviceProblem(p, ctx)
    C, K = dp.C, p.grid.n
    out = {}
    for prec, dt, name, steps in ((R.FP32, torch.float32, "fp32", max(1, args.steps)), (R.FP64, torch.float64, "fp64", 1)):
        bufs = [(torch.empty((C, K), dtype=dt, device=ctx.device), torch.empty((C, K), dtype=dt, device=ctx.device))]
        for _ in range(max(3, args.warmup) if prec == R.FP32 else 1):
            solver.solve(dp, ctx, prec, buffers=bufs)
        ctx.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in kev:
            a.record(ctx.stream); b.record(ctx.stream)
        ctx.sync()
        with ClockSampler(0) as clk:
            for i in range(steps):
                ev[i][0].record(ctx.stream)
                ctx.set_profile_events(*kev[i])
                r = solver.solve(dp, ctx, prec, buffers=bufs)
                ctx.set_profile_events(None, None)
                ev[i][1].record(ctx.stream)
            ctx.sync()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        kms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
        out[name] = {"ms_per_step": ms, "value": C * K / (ms * 1e-3), "line_sum_ms": kms, "q_W_cm2": float(r["q"].item()),
                     "clocks": clk.summary()}
        del bufs
    out["fp32_q_rel_err"] = abs(out["fp32"]["q_W_cm2"] / out["fp64"]["q_W_cm2"] - 1)
    print(json.dumps({"workload": f"stagnation line with the exact Voigt shape: {C} cells, {len(p.lines)} lines, "
                                  f"{K} points", "metric": "cell·λ points/s", "warmup": args.warmup,
                      "steps": max(1, args.steps), **out}))
    return 0


def run_fibonacci(args):
    """The paper's own angular path on the afterbody at 100 x 50 cells (2e5
    points in 65,536-point chunks): Fibonacci lines of sight from
    --fib-points surface points, flow variables at their nodes, kappa / j at
    every node, the node march, and the flux from a 33 x 65 (phi, theta)
    grid; FP32.  For comparison the same points with 16-mu x 32-azimuth rays
    through per-cell coefficients."""
    import torch
    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import solver, synth
    P = args.fib_points
    p = synth.afterbody(nx=100, nr=50, n_points=P, n_grid=200_000)
    ctx = R.Context(0)
    sp = R.DeviceSpecies(p.species, ctx.device)
    ln = R.DeviceLines(p.lines, ctx.device)
    run = lambda: solver.solve_fibonacci(p, ctx, args.fib_los, 33, 65, R.FP32, chunk=p.chunk, species=sp, lines=ln)
    for _ in range(max(1, args.warmup)):
        out = run()
    ctx.sync()
    ms = []
    with ClockSampler(0) as clk:
        for _ in range(max(1, args.steps)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream)
            out = run()
            b.record(ctx.stream)
            ctx.sync()
            ms.append(a.elapsed_time(b))
    t = float(np.mean(ms)) * 1e-3
    rays = out["rays"]
    # the per-cell path on the same points: coefficients once per cell, shared by all rays
    dp = solver.DeviceProblem(p, ctx, lines=ln, species=sp)
    bufs = [(torch.empty((dp.C, p.chunk), dtype=torch.float32, device=ctx.device),
             torch.empty((dp.C, p.chunk), dtype=torch.float32, device=ctx.device))]
    solver.solve(dp, ctx, R.FP32, chunk=p.chunk, buffers=bufs)
    ctx.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(ctx.stream)
    cell = solver.solve(dp, ctx, R.FP32, chunk=p.chunk, buffers=bufs)
    b.record(ctx.stream)
    ctx.sync()
    tc = a.elapsed_time(b) * 1e-3
    print(json.dumps({
        "workload": f"afterbody 100x50 cells, {len(p.lines) // 1000}k lines, {p.grid.n:.0e} points in "
                    f"{p.chunk}-point chunks; {P} points x {args.fib_los} Fibonacci LOS ({rays.n_dirs // max(P, 1)} "
                    f"leave the body), 33 x 65 (phi, theta) grid, FP32",
        "warmup": args.warmup, "steps": max(1, args.steps), "ms_per_solve": t * 1e3,
        "nodes": int(rays.n_nodes), "lines_of_sight": int(rays.n_dirs), "segments": int(rays.struct.n_segments),
        "node_lambda_per_s": rays.n_nodes * p.grid.n / t,
        "ray_lambda_segments_per_s": rays.struct.n_segments * p.grid.n / t,
        "q_mean_W_cm2": float(out["q"].mean().item()), "clocks": clk.summary(),
        "per_cell_path": {"rays": "16 mu x 32 azimuths", "ms_per_solve": tc * 1e3, "cells": dp.C,
                          "q_mean_W_cm2": float(cell["q"].mean().item())}}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return oracle_phases(args) if args.oracle_phases else run_reference(args)
    if args.workload == "afterbody":
        return run_afterbody(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "fibonacci":
        return run_fibonacci(args)
    if args.workload == "qss":
        return run_qss(args)
    if args.workload == "continuum":
        return run_continuum(args)
    if args.workload == "voigt":
        return run_voigt(args)
    import torch
    import torch.distributed as dist

    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import solver, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    precision = R.FP32 if args.precision == "fp32" else R.FP64

    p = synth.stagnation_line(n_cells=args.cells)
    ctx = R.Context(local)
    tuned = None
    if args.tile:
        ctx.set_tiling(tile_width=args.tile)
    elif precision == R.FP32 and not args.no_tune:
        from paper_2604_11856_gb300 import autotune
        tw, wpb, times = autotune.tune(ctx, p)
        tuned = {"tile_width": tw, "cells_per_block": wpb, "candidates_ms": times}
    dp = solver.DeviceProblem(p, ctx)
    C, K = dp.C, p.grid.n
    n_dirs = dp.rays.n_dirs
    seg_lambda = C * n_dirs * K          # segments x directions x wavelengths per step
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    dt = torch.float32 if precision == R.FP32 else torch.float64
    bufs = [(torch.empty((C, K), dtype=dt, device=dev), torch.empty((C, K), dtype=dt, device=dev))]
    stream = ctx.stream

    def step(ev_pair=None):
        if ev_pair is not None:
            ctx.set_profile_events(*ev_pair)
        out = solver.solve(dp, ctx, precision, buffers=bufs)
        if ev_pair is not None:
            ctx.set_profile_events(None, None)
        return out

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    # one untimed step with the work counters on (evaluations, XU terms), then
    # the timed steps without them
    ctx.set_counters(True)
    ctx.reset_stats()
    step()
    stats = ctx.get_stats()
    ctx.set_counters(False)
    ctx.sync()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in k3:   # materialise the events before handing them to the library
        a.record(stream); b.record(stream)
    barrier()
    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))              # evict L2 between steps (outside the timed window)
            starts[i].record(stream)
            step(k3[i])
            ends[i].record(stream)
        barrier()
    t_wall = time.perf_counter() - t_wall
    ctx.sync()
    step_ms = [starts[i].elapsed_time(ends[i]) for i in range(args.steps)]
    k3_ms = [k3[i][0].elapsed_time(k3[i][1]) for i in range(args.steps)]
    total_ms = float(np.sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * C * K / (ms_per_step * 1e-3)
    evals_per_step = stats["evaluations"]
    k3_mean = float(np.mean(k3_ms))

    # roofline of the line sum: transcendental (XU / MUFU) work the FP32
    # profile needs: rcp + 2 rsqrt per evaluation, + ex2 for the Gaussian core
    # and + ex2 for the correction term where they do not underflow
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    if precision == R.FP32:
        traffic = line_sum_traffic(C, K)
        xu_ops = 3 * stats["evaluations"] + stats["gauss_terms"] + stats["correction_terms"]
        peak = n_sm * 16 * sm_max / 1e9               # Gop/s: 16 XU lanes per SM per clock
        achieved = xu_ops / (k3_mean * 1e-3) / 1e9
        roof = {"bound": "alu", "pipe": "xu (MUFU ex2/rsqrt/rcp)", "achieved": achieved, "peak": peak,
                "unit": "Gop/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_algorithmic_bytes": C * K * 8,   # kappa and j written once, FP32
                "kernel": "k_line_sum_f32", "kernel_ms": k3_mean, "evaluations": evals_per_step,
                "peak_source": f"{n_sm} SMs x 16 XU lanes x {sm_max / 1e6:.0f} MHz (max SM clock)"}
    else:
        # FP64: about 40 FP64 operations per evaluation (two exponentials, two square roots, the bracket),
        # 2 FP64 FMA lanes per SM per clock
        fp64_ops = 40.0 * evals_per_step
        peak = n_sm * 2 * 2 * sm_max / 1e9
        achieved = fp64_ops / (k3_mean * 1e-3) / 1e9
        roof = {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_line_sum_f64", "kernel_ms": k3_mean,
                "evaluations": evals_per_step}

    out = {"metric": METRIC, "value": value, "unit": "cell·λ points/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if precision == R.FP32 else "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": args.precision + ("-chosen" if precision == R.FP32 else "-plain"),
                      "cells": C, "lines": len(p.lines), "grid_points": K, "directions": n_dirs,
                      "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}",
                      "tiling": tuned},
           "secondary": {"ray_lambda_segments_per_s": world * seg_lambda / (ms_per_step * 1e-3),
                         "profile_evaluations_per_s": world * evals_per_step / (ms_per_step * 1e-3),
                         "line_sum_ms": k3_mean, "wall_s": t_wall,
                         "pairs_per_step": stats["pairs"],
                         "gauss_terms_per_step": stats["gauss_terms"],
                         "correction_terms_per_step": stats["correction_terms"]},
           "roofline": roof, "clocks": clk.summary(), "gpu_launches": None}
    # launches per step (checked against the ncu launch list): populations + its cell
    # validation; line and cell validation, line prep, cell prep, bin bounds, count, scan,
    # fill, line sum; ray validation, march, flux part + sum; FP32 adds three copies of ray
    # data to float.  The slab rays are built once, before the timed region.
    out["gpu_launches"] = (18 if precision == R.FP32 else 15) * args.steps

    if not args.no_fp64 and precision == R.FP32:
        bufs64 = [(torch.empty((C, K), dtype=torch.float64, device=dev),
                   torch.empty((C, K), dtype=torch.float64, device=dev))]
        r64 = solver.solve(dp, ctx, R.FP64, buffers=bufs64)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record(stream)
        r64 = solver.solve(dp, ctx, R.FP64, buffers=bufs64)
        e1.record(stream)
        ctx.sync()
        ms64 = e0.elapsed_time(e1)
        r32 = step()
        ctx.sync()
        q32, q64 = float(r32["q"].item()), float(r64["q"].item())
        out["fp64_plain"] = {"value": C * K / (ms64 * 1e-3), "ms_per_step": ms64, "q_W_cm2": q64,
                             "fp32_q_W_cm2": q32, "fp32_q_rel_err": abs(q32 / q64 - 1)}
        del bufs64

    if not args.no_e2e:
        # end to end through the public API: host arrays -> pinned staging -> device -> q on the host
        ectx = R.Context(local)
        solver.solve_host(p, precision, ctx=ectx)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        n_e2e = max(1, min(3, args.steps))
        for _ in range(n_e2e):
            qh, bi, bo = solver.solve_host(p, precision, ctx=ectx)
        te = (time.perf_counter() - t0) / n_e2e
        out["e2e"] = {"value": world * C * K / te, "unit": "cell·λ points/s", "h2d_bytes_per_step": bi,
                      "d2h_bytes_per_step": bo, "ms_per_step": te * 1e3}
        ectx.close()
    if not args.no_serve:
        out["served"] = served(p, args, local)
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
        out["cpu_baseline"].pop("seconds")
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
