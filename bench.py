#!/usr/bin/env python
"""Benchmark of the RAPRAL hot path on GB300.

Headline (default): the axisymmetric afterbody stand-in of the paper's
Fire II case (Sec. 3.2): 400 x 200 two-temperature cells, 20,000 atomic +
300,000 molecular lines, a 1,000,000-point grid over 50-2000 nm in 65,536-point
chunks, 200 surface points x 512 rays (16 mu x 32 azimuths), FP32-chosen
arithmetic.  A step is one spectral chunk of that solve, through every step of
the path: line binning -> line-by-line kappa / j of all 80,000 cells -> ray
march of all 102,400 rays with the angular sum -> wall flux; populations at
the first chunk of each solve.  Steps run back to back through the chunk
pipeline on one stream (`--streams 2`: the line sum of chunk i + 1 beside the
march of chunk i, which takes the same time on this workload), cycling
through the 16 chunks, so 16 steps are one whole solve.  The ray
segments depend on the geometry only and are built once, before timing.
Inputs are resident in HBM when timing starts; each step's kappa / j table
(42 GB) is far larger than L2.

Secondary blocks: the stagnation-line step (FP32 and FP64 plain), the served
request loop.  `--impl reference` times the CPU oracle instead, on a bounded
sample of the same workload.  Prints one JSON line (rank 0).
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
WORKLOAD = ("afterbody: 400x200 cells, 20k atomic + 300k molecular lines, 1e6-point grid 50-2000 nm "
            "in 65,536-point chunks, 200 points x 512 rays (16 mu x 32 azimuths)")
STAG_WORKLOAD = "stagnation line: 200 cells, 20k atomic + 300k molecular lines, 1e6-point grid 50-2000 nm, 16-mu tangent slab"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
SERVE_RATES = (50.0, 100.0, 200.0, 500.0, 1000.0, 2000.0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 20 for the afterbody chunks and the stagnation step, 5 otherwise)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["rapral", "reference"], default="rapral")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="seconds of oracle work in the cpu_baseline sample (and at most per reference-arm step)")
    ap.add_argument("--no-secondary", action="store_true", help="headline only: skip the stagnation and served blocks")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-requests block")
    ap.add_argument("--serve-requests", type=int, default=100, help="FP32 requests per offered rate")
    ap.add_argument("--serve-fp64-requests", type=int, default=4, help="FP64 requests per offered rate (the first ones)")
    ap.add_argument("--serve-rates", type=str, default="4,50,2000",
                    help=f"offered rates, req/s (the whole study: {','.join(str(int(r)) for r in SERVE_RATES)})")
    ap.add_argument("--serve-fp64-rates", type=str, default="2000")
    ap.add_argument("--serve-slots", type=int, default=4, help="served block: concurrent request slots")
    ap.add_argument("--stag-chunks", type=str, default="",
                    help="stagnation block: also time the FP32 step in spectral chunks of these sizes (comma list)")
    ap.add_argument("--pairs-per-pass", type=int, choices=[32, 64], default=32,
                    help="afterbody: (line, cell) pairs a warp of the FP32 line sum stages per sweep pass")
    ap.add_argument("--serve-solo", action="store_true",
                    help="served block: also run each rate's FP32 requests back to back on one stream (no "
                         "arrival gaps, one at a time), the capacity the served loop compares with")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default tiling)")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32", help="stagnation workload only")
    ap.add_argument("--no-fp64", action="store_true", help="stagnation: skip the FP64-plain side measurement")
    ap.add_argument("--workload", choices=["afterbody", "stagnation", "serve", "batch", "fibonacci", "qss", "continuum",
                                           "voigt"],
                    default="afterbody",
                    help="afterbody (the bench line); stagnation / serve / batch / fibonacci / qss / continuum / "
                         "voigt (the stagnation step with the exact Voigt shape): one-off measurements")
    ap.add_argument("--cont-levels", type=int, default=100, help="continuum workload: levels per atom (N, O)")
    ap.add_argument("--cont-points", type=int, default=1_000_000,
                    help="continuum workload: grid points (fewer only for profiler captures)")
    ap.add_argument("--fib-points", type=int, default=8, help="fibonacci workload: surface points")
    ap.add_argument("--fib-los", type=int, default=128, help="fibonacci workload: Fibonacci directions per point")
    ap.add_argument("--streams", type=int, choices=[1, 2], default=1,
                    help="afterbody: chunk pipeline on one stream, or two (line sum of the next chunk beside the "
                         "march)")
    ap.add_argument("--ab-small", action="store_true",
                    help="afterbody at 100 x 50 cells, 20 points, 2e5 grid points (profiler captures)")
    ap.add_argument("--ab-cells", type=str, default="",
                    help="afterbody cells as NXxNR (smaller only for profiler captures; all 200 points kept)")
    ap.add_argument("--cells", type=int, default=200,
                    help="cells of the stagnation line (fewer only for profiler captures)")
    ap.add_argument("--oracle-phases", action="store_true",
                    help="with --impl reference: the oracle's time per phase, all threads and one thread")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 20 if (args.impl == "rapral" and args.workload in ("afterbody", "stagnation")) else 5
    return args


# DRAM bytes (read + write) of one timed FP32 line-sum launch on the stagnation line
# at full size (200 cells x 1e6 points, tiling 128 x 2, the persistent launch), from a
# one-pass ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel
# source with this digest (source_digest).  Other cell / point counts scale in proportion (the
# bytes are the kappa / j rows written); a different source (comments aside) gives null.
LINE_SUM_TRAFFIC = {"sha1": "9cb401bd4549a6eaf0a40186c4f84d5e3c0dda4c", "cells": 200, "grid_points": 1_000_000,
                    "bytes": 53_932_288 + 1_543_667_712}


# DRAM bytes of one FP32 continuum level-sum launch at full size (200 cells x
# 1e6 points, N and O with 100 levels each), from a one-pass ncu capture of the
# kernel source with this digest (source_digest); a different source gives null.
CONT_TRAFFIC = {"sha1": "b20ff15bc5d2a99674fcbc6991e7a0c6b0701352", "cells": 200, "grid_points": 1_000_000, "levels": 100,
                "bytes": 1_782_987_520 + 1_539_120_640}

# DRAM bytes (read + write) of one FP32 march launch (k_march1) on a full
# 65,536-point afterbody chunk (80,000 cells, 26,697,080 ray segments), from a
# one-pass ncu capture of the kernel source with this digest (source_digest);
# another source or ray set gives null.
MARCH_TRAFFIC = {"sha1": "156f11f3f01ceca0c87329b7dcd4e547185c0877", "cells": 80_000, "segments": 26_697_080,
                 "grid_points": 65_536, "bytes": 356_842_381_824 + 468_259_328}


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


# L2 gather-bandwidth probe (a roofline denominator for the march, whose
# gathers L2 serves): warps load 256-byte rows (8 bytes a lane) at
# pseudo-random row indices of an L2-resident table; every index is reduced
# modulo the row count, so every access stays inside the table.
GATHER_PROBE_SRC = r"""
#include <cuda_runtime.h>
extern "C" __global__ void k_gather_probe(const float2* __restrict__ tab, long long rows, int iters, float* out) {
    const int lane = threadIdx.x & 31;
    unsigned x = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 2654435761u + 12345u;
    float s = 0.f;
    for (int i = 0; i < iters; i += 4) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x = x * 1664525u + 1013904223u;
            v[u] = tab[(long long)(x % (unsigned)rows) * 32 + lane];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s += v[u].x + v[u].y;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
extern "C" float gather_probe_ms(const void* tab, long long bytes, int blocks, int iters, float* out) {
    const long long rows = bytes / 256;
    cudaEvent_t a, b;
    cudaEventCreate(&a); cudaEventCreate(&b);
    k_gather_probe<<<blocks, 256>>>((const float2*)tab, rows, iters, out);
    cudaEventRecord(a);
    k_gather_probe<<<blocks, 256>>>((const float2*)tab, rows, iters, out);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a); cudaEventDestroy(b);
    return ms;
}
"""


def l2_gather_peak(dev_index):
    """Measured L2 gather bandwidth (GB/s): the best of a few block counts on
    48 MB and 96 MB tables (both L2-resident), built with nvcc for sm_103a."""
    import ctypes
    import torch
    from paper_2604_11856_gb300 import build as B
    os.makedirs(B.BUILD, exist_ok=True)
    src = os.path.join(B.BUILD, "gather_probe.cu")
    lib = os.path.join(B.BUILD, "gather_probe.so")
    stale = not (os.path.exists(lib) and os.path.exists(src) and open(src).read() == GATHER_PROBE_SRC)
    if stale:
        with open(src, "w") as f:
            f.write(GATHER_PROBE_SRC)
        subprocess.run([B.nvcc(), *B.ARCH, "-O3", "-shared", "-Xcompiler", "-fPIC", src, "-o", lib], check=True)
    L = ctypes.CDLL(lib)
    L.gather_probe_ms.restype = ctypes.c_float
    L.gather_probe_ms.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    best = {}
    n_sm = torch.cuda.get_device_properties(dev_index).multi_processor_count
    for mb in (48, 96):
        nbytes = mb << 20
        tab = torch.ones(nbytes // 4, dtype=torch.float32, device=f"cuda:{dev_index}")
        for blocks in (4 * n_sm, 8 * n_sm):
            out = torch.empty(blocks * 256, dtype=torch.float32, device=f"cuda:{dev_index}")
            iters = 4096
            ms = L.gather_probe_ms(tab.data_ptr(), nbytes, blocks, iters, out.data_ptr())
            best[mb] = max(best.get(mb, 0.0), blocks * 256 * iters * 8 / (ms * 1e-3) / 1e9)
    return {"GBps_48MB_table": best[48], "GBps_96MB_table": best[96],
            "how": "warps loading 256-byte rows at random row indices of an L2-resident table (bench.py)"}


def march_traffic(cells, segments, grid_points):
    """The stored DRAM bytes of one march launch, scaled to the launch's columns
    (the segment lists are read once per wavelength tile); None for another ray
    set or another kernel source."""
    digest = source_digest("k_rays.cu")
    t = MARCH_TRAFFIC
    if t["bytes"] is None or digest != t["sha1"] or cells != t["cells"] or segments != t["segments"]:
        return None
    return t["bytes"] * (grid_points / t["grid_points"])


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
            "sample": f"{n_cells} of {len(p.cells)} cells spread over the domain x {nk2} of {p.grid.n} grid points, "
                      f"all {len(p.lines)} lines, kappa and j in FP64 ({dt2:.1f} s)", "seconds": dt2}


def served(p, args, device):
    """Open-loop served requests (config-4 sizes: line-of-sight and slab
    solves, cells 10-5000, 1e5-1e6 points, 1-256 rays) sharing the resident
    stagnation-line lists, at several offered Poisson rates.  At each rate
    the FP32-chosen path serves the whole request stream and the FP64-plain
    path the same stream's first requests (it is ~80x slower); the q error of
    FP32 is taken against FP64 on the requests both served."""
    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import serve, synth
    pool = (p.lines, p.species, {})
    rates = [float(r) for r in args.serve_rates.split(",") if r]
    rates64 = {float(r) for r in args.serve_fp64_rates.split(",") if r}
    res = {"slots": args.serve_slots, "admission": "device free memory at start minus a 16 GiB reserve", "rates": []}
    errs_all = []
    for i, rate in enumerate(rates):
        gen = synth.served_requests(seed=1004 + i, n_requests=args.serve_requests, rate=rate, pool=pool)
        row = {"offered_rate_req_s": rate}
        q32 = {}
        for prec, n, name in ((R.FP32, args.serve_requests, "fp32"), (R.FP64, args.serve_fp64_requests, "fp64")):
            if n <= 0 or (prec == R.FP64 and rate not in rates64):
                continue
            reqs = [serve.Request(rid=j, problem=g["problem"], arrival=g["t"], precision=prec)
                    for j, g in enumerate(gen[:n])]
            srv = serve.Server(p.lines, p.species, device=device, slots=args.serve_slots)
            row[name] = serve.run_open_loop(srv, reqs)
            res["budget_bytes"] = srv.budget
            if prec == R.FP32:
                q32 = {r.rid: r.q for r in reqs if r.status == "done"}
                if args.serve_solo:
                    t0 = time.perf_counter()
                    solo = serve.solo(reqs, p.lines, p.species, device=device)
                    dt = time.perf_counter() - t0
                    row["fp32_back_to_back"] = {"requests": len(solo), "seconds": dt, "req_s": len(solo) / dt,
                                                "max_q_rel_diff_vs_served": float(max(
                                                    np.max(np.abs(q32[k] / solo[k] - 1)) for k in q32))}
            else:
                errs = [float(np.max(np.abs(q32[r.rid] / r.q - 1))) for r in reqs
                        if r.status == "done" and r.rid in q32]
                row["q_rel_err_fp32_vs_fp64_max"] = max(errs) if errs else None
                errs_all += errs
        res["rates"].append(row)
    res["q_rel_err_fp32_vs_fp64_max"] = max(errs_all) if errs_all else None
    sat = [r["fp32"]["throughput_req_s"] for r in res["rates"] if "fp32" in r]
    res["fp32_saturation_req_s"] = max(sat) if sat else None
    return res


def run_reference(args):
    """--impl reference: the oracle on the host cores, bounded samples of the
    bench workload (the afterbody) per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = afterbody_problem(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    per_step = max(2.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(p, per_step / 4)
    vals, secs = [], []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(p, per_step)
        vals.append(last["value"])
        secs.append(last.pop("seconds"))
    v = float(np.mean(vals))
    # a step here is one bounded sample of the workload, not a whole chunk
    line = {"metric": METRIC, "value": v, "unit": "cell·λ points/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3, "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": headline_config(args, p, world),
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


def run_batch(args):
    """64 uneven uniform-slab solves (FP32): one persistent line-sum launch per
    spectral round, the whole run captured in one CUDA graph, against the
    same solves run one after another."""
    import torch
    from paper_2604_11856_gb300 import autotune, batch, rapral as R, solver, synth
    probs = synth.batch_slabs()
    ctx = R.Context(0)
    tw, wpb, pb, times = autotune.tune(ctx, max(probs, key=lambda q: len(q.lines)))
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
                                  "0-3e5 molecular lines)", "tiling": [tw, wpb, pb], "graph_ms": t * 1e3,
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


def dist_setup():
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(dev, world):
    import torch
    import torch.distributed as dist
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()


def afterbody_problem(args):
    from paper_2604_11856_gb300 import synth
    if args.ab_small:
        return synth.afterbody(nx=100, nr=50, n_points=20, n_grid=200_000)
    if args.ab_cells:
        nx, nr = (int(v) for v in args.ab_cells.lower().split("x"))
        return synth.afterbody(nx=nx, nr=nr)
    return synth.afterbody()


def headline_config(args, p, world):
    """The bench line's `config`: the afterbody workload as the arguments
    select it (both arms print the same one)."""
    geo = p.geometry
    C, P = len(p.cells), len(geo.surf_x)
    return {"workload": WORKLOAD if not (args.ab_small or args.ab_cells) else f"reduced afterbody {C} cells",
            "precision": "fp32-chosen", "cells": C, "lines": len(p.lines), "grid_points": p.grid.n,
            "chunk_points": p.chunk, "surface_points": P, "rays": P * len(geo.mu) * int(geo.n_phi),
            "step": f"one {p.chunk:,}-point spectral chunk of the solve ({-(-p.grid.n // p.chunk)} steps = one "
                    f"solve), {'two-stream' if args.streams == 2 else 'one-stream'} pipeline, populations at each "
                    f"solve's first chunk",
            "l2": "inputs larger than L2 (a 42 GB kappa / j table per step)",
            "parallelism": f"spectral shards x{world} (every {world}-th chunk a rank, one FP64 "
                           f"all-reduce of the wall flux)" if world > 1 else "one GPU"}


def run_headline(args):
    """The afterbody chunk steps (module docstring).  With N ranks each rank
    takes every N-th chunk of the solve (a spectral shard: the chunks are
    independent, populations are replicated) and the P partial fluxes are
    summed by one FP64 all-reduce at the end."""
    import torch
    import torch.distributed as dist
    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import solver

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    p = afterbody_problem(args)
    sa = torch.cuda.Stream(dev)
    ctx = R.Context(local, stream=sa)
    ctx2 = R.Context(local, stream=torch.cuda.Stream(dev)) if args.streams == 2 else None
    ctx.set_line_batch(args.pairs_per_pass)
    dp = solver.DeviceProblem(p, ctx)   # ray segments: built once per geometry
    ctx.sync()
    C, P, n, chunk = dp.C, dp.P, p.grid.n, p.chunk
    nseg = int(dp.rays.struct.n_segments)
    mine = solver.shard_ranges(n, rank, world, chunk)   # this rank's spectral shard: every world-th chunk
    pipe = solver.ChunkPipeline(dp, ctx, R.FP32, chunk, ctx2=ctx2)
    solves = []          # (flux of each completed pass over this rank's chunks)
    launches = [0]

    def enqueue(s, kev=None, mev=None):
        j = s % len(mine)
        if j == 0:
            pipe.begin()
            launches[0] += 2                    # cell validation + populations
        k0, nk = mine[j]
        if kev is not None:
            ctx.set_profile_events(*kev)
        pipe.step(k0, nk, march_events=mev)
        if kev is not None:
            ctx.set_profile_events(None, None)
        # coefficients: cell and line validation, line prep, cell prep, bin bounds, count, scan, fill,
        # line sum; march: ray validation, three FP32 copies, march, group sum; flux: part + sum
        launches[0] += 9 + 6 + 2
        if j == len(mine) - 1:
            pipe.end()
            with torch.cuda.stream(sa):
                solves.append(pipe.q.clone())
        return nk

    for s in range(args.warmup):
        enqueue(s)
    pipe.end()
    barrier(dev, world)
    solves.clear()
    pipe.i = 0
    K = args.steps
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in kev:   # materialise the events before handing them to the library
        a.record(sa); b.record(sa)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev_solve = torch.cuda.Event(enable_timing=True)
    barrier(dev, world)
    launches[0] = 0
    cell_lambda = 0
    seg_lambda = 0
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        t0.record(sa)
        for s in range(K):
            nk = enqueue(s, kev[s], mev[s])
            cell_lambda += C * nk
            seg_lambda += nseg * nk
            if s == len(mine) - 1:
                ev_solve.record(sa)   # after the join of the first whole pass
        pipe.end()
        qsum = pipe.q if len(solves) == 0 else solves[0]
        if world > 1:   # the only exchange: the P partial fluxes of the shards
            with torch.cuda.stream(sa):
                qred = qsum.clone()
                dist.all_reduce(qred, op=dist.ReduceOp.SUM)
        t1.record(sa)
        barrier(dev, world)
        t_wall = time.perf_counter() - t_wall
    total_ms = t0.elapsed_time(t1)
    solve_ms = t0.elapsed_time(ev_solve) if K >= len(mine) else None
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        w = torch.tensor([float(cell_lambda), float(seg_lambda)], dtype=torch.float64, device=dev)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
        cell_lambda, seg_lambda = float(w[0].item()), float(w[1].item())
    ms_per_step = total_ms / K
    value = cell_lambda / (total_ms * 1e-3)
    k_ms = [a.elapsed_time(b) for a, b in kev]
    m_ms = [a.elapsed_time(b) for a, b in mev]
    march_mean, lsum_mean = float(np.mean(m_ms)), float(np.mean(k_ms))
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # march: per launch it reads each cell's kappa / j columns once from DRAM and writes q_lambda
    steps_nk = [mine[s % len(mine)][1] for s in range(K)]
    nk_mean = float(np.mean(steps_nk))
    uniq = C * nk_mean * 8 + P * nk_mean * 4
    seglam_launch = nseg * nk_mean
    gather = seglam_launch * 8 / (march_mean * 1e-3) / 1e9
    l2 = l2_gather_peak(local)
    l2_peak = max(l2["GBps_48MB_table"], l2["GBps_96MB_table"])
    march = {"kernel": "k_march1 (single-direction rays, FP32; + ray validation, FP32 copies, bundle plan, "
                       "group sum)",
             "kernel_ms": march_mean, "segments": nseg, "segment_lambda_per_launch": seglam_launch,
             "ray_lambda_segments_per_s": seglam_launch / (march_mean * 1e-3),
             "gather_bytes_per_launch": seglam_launch * 8, "gather_GBps": gather,
             "l2_gather_peak": l2, "frac_of_l2_gather_peak": gather / l2_peak,
             "dram_unique_bytes_per_launch": uniq,
             "dram_traffic_bytes_per_launch": march_traffic(C, nseg, nk_mean),
             "dram_frac_of_hbm_peak": uniq / (march_mean * 1e-3) / 1e9 / hbm,
             "timed_inside": ("the two-stream pipeline (overlaps the next chunk's line sum)" if ctx2 is not None
                              else "the one-stream pipeline (the kernel alone on the GPU)")}
    roof = {"bound": "hbm", "achieved": gather, "peak": hbm, "unit": "GB/s", "frac": gather / hbm,
            "traffic": march_traffic(C, nseg, nk_mean),
            "kernel": "k_march1 (single-direction rays, FP32)", "kernel_ms": march_mean,
            "algorithmic_bytes": seglam_launch * 8,
            "algorithmic_unit": "8 B (FP32 kappa + j of the next cell) gathered per segment-wavelength, x the "
                                "launch's segments x columns",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback",
            "served_from": "L2: the gathers hit L2, whose measured gather bandwidth is in march.l2_gather_peak; "
                           "DRAM (traffic) sees the chunk's kappa / j once and the segment lists once per "
                           "64-column wavelength tile",
            "frac_of_l2_gather_peak": gather / l2_peak}
    out = {"metric": METRIC, "value": value, "unit": "cell·λ points/s", "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": headline_config(args, p, world),
           "secondary": {"segments": nseg, "ray_lambda_segments_per_s": seg_lambda / (total_ms * 1e-3),
                         "solve_s": solve_ms * 1e-3 if solve_ms else None,
                         "line_sum_ms_mean": lsum_mean, "march_ms_mean": march_mean, "wall_s": t_wall,
                         "q_mean_W_cm2": float(qsum.mean().item()) if world == 1 else None},
           "roofline": roof, "march": march, "clocks": clk.summary(), "gpu_launches": launches[0]}

    # XU work of the timed steps: each distinct chunk of the timed sequence once more, untimed, with the
    # library's work counters on (they cost time, so the timed steps run without them)
    ctx.set_counters(True)
    kap, em = pipe.buffers[0]
    per_chunk = {}
    for s in range(K):
        j = s % len(mine)
        if j in per_chunk:
            continue
        k0, nk = mine[j]
        ctx.reset_stats()
        R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, k0, nk, R.FP32, kap, em)
        st = ctx.get_stats()
        per_chunk[j] = (3 * st["evaluations"] + st["gauss_terms"] + st["correction_terms"], st["evaluations"])
    ctx.set_counters(False)
    xu = sum(per_chunk[s % len(mine)][0] for s in range(K))
    ev_total = sum(per_chunk[s % len(mine)][1] for s in range(K))
    xu_peak = n_sm * 16 * sm_max / 1e9
    out["line_sum"] = {"kernel": "k_line_sum_f32_persist", "bound": "alu", "pipe": "xu (MUFU ex2/rsqrt/rcp)",
                       "evaluations_per_step": ev_total / K,
                       "ms_mean": lsum_mean,
                       "xu_frac": xu / (float(np.sum(k_ms)) * 1e-3) / 1e9 / xu_peak,
                       "peak_gops": xu_peak,
                       "peak_source": f"{n_sm} SMs x 16 XU lanes x {sm_max / 1e6:.0f} MHz (max SM clock)",
                       "timed_inside": march["timed_inside"].replace("(the kernel alone on the GPU)", "(alone)"),
                       "note": "time: the line-sum kernel of each timed step (CUDA events the library records "
                               "around the launch, on its stream); XU "
                               "operations: 3 per evaluation + one per Gaussian and correction term, from the "
                               "library's work counters in an untimed pass over the same chunks"}

    if not args.no_e2e:
        # end to end through the public API: host arrays -> pinned staging -> device -> q on the host,
        # one chunk a call (with --streams 2 cut in two halves, pipelined on the two streams), over one
        # whole pass of this rank's chunks, so that its chunk mix is the solve's (the chunks' line-sum
        # costs differ 60-fold)
        n_e2e = len(mine)
        sub = chunk if ctx2 is None else chunk // 2
        k0, nk = mine[-1]
        solver.solve_host(p, R.FP32, sub, ctx=ctx, ctx2=ctx2, k_start=k0, k_stop=k0 + nk)
        barrier(dev, world)
        t0w = time.perf_counter()
        cl_e2e = 0
        for s in range(n_e2e):
            k0, nk = mine[s]
            _qh, bi, bo = solver.solve_host(p, R.FP32, sub, ctx=ctx, ctx2=ctx2, k_start=k0, k_stop=k0 + nk)
            cl_e2e += C * nk
        barrier(dev, world)
        te = time.perf_counter() - t0w
        if world > 1:
            t = torch.tensor([te], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
            w = torch.tensor([float(cl_e2e)], dtype=torch.float64, device=dev)
            dist.all_reduce(w, op=dist.ReduceOp.SUM)
            cl_e2e = float(w.item())
        out["e2e"] = {"value": cl_e2e / te, "unit": "cell·λ points/s", "h2d_bytes_per_step": bi,
                      "d2h_bytes_per_step": bo, "ms_per_step": te / n_e2e * 1e3, "steps": n_e2e,
                      "device_ms_per_step_same_chunks": solve_ms / len(mine) if solve_ms else None,
                      "note": "one whole pass over the chunks (the solve's chunk mix), one chunk a call; each "
                              "call also builds the ray segments from the geometry"}
    if not args.no_secondary and world == 1:
        ctx.close()
        if ctx2 is not None:
            ctx2.close()
        del pipe, dp, solves
        torch.cuda.empty_cache()
        out["stagnation"] = stagnation_block(args, local, world, rank)
        if not args.no_serve:
            from paper_2604_11856_gb300 import synth
            pst = synth.stagnation_line()
            out["served"] = served(pst, args, local)
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
        out["cpu_baseline"].pop("seconds")
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


def stagnation_block(args, local, world, rank, fp64=True):
    """The stagnation-line step (200 cells, 320k lines, 1e6 points, 16-mu
    tangent slab + normal ray, one whole solve a step): FP32-chosen with
    autotuned tiling, the line sum's XU roofline, and one FP64-plain step."""
    import torch
    from paper_2604_11856_gb300 import autotune
    from paper_2604_11856_gb300 import rapral as R
    from paper_2604_11856_gb300 import solver, synth

    dev = torch.device("cuda", local)
    p = synth.stagnation_line(n_cells=args.cells)
    ctx = R.Context(local)
    if args.no_tune:   # the library's default tiling (128-point tiles, 4 cells a block, 32 lines a pass)
        tuned = {"tile_width": 128, "cells_per_block": 4, "pairs_per_pass": 32, "candidates_ms": None}
    else:
        tw, wpb, pb, times = autotune.tune(ctx, p)
        tuned = {"tile_width": tw, "cells_per_block": wpb, "pairs_per_pass": pb, "candidates_ms": times}
    dp = solver.DeviceProblem(p, ctx)
    C, K = dp.C, p.grid.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    bufs = [(torch.empty((C, K), dtype=torch.float32, device=dev), torch.empty((C, K), dtype=torch.float32, device=dev))]
    stream = ctx.stream
    for _ in range(3):
        solver.solve(dp, ctx, R.FP32, buffers=bufs)
    ctx.set_counters(True)
    ctx.reset_stats()
    solver.solve(dp, ctx, R.FP32, buffers=bufs)
    stats = ctx.get_stats()
    ctx.set_counters(False)
    ctx.sync()
    steps = 20
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    k3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in k3:
        a.record(stream); b.record(stream)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            ctx.set_profile_events(*k3[i])
            r32 = solver.solve(dp, ctx, R.FP32, buffers=bufs)
            ctx.set_profile_events(None, None)
            ev[i][1].record(stream)
        ctx.sync()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    kms = float(np.mean([a.elapsed_time(b) for a, b in k3]))
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    xu_ops = 3 * stats["evaluations"] + stats["gauss_terms"] + stats["correction_terms"]
    peak = n_sm * 16 * sm_max / 1e9
    out = {"workload": STAG_WORKLOAD, "precision": "fp32-chosen", "steps": steps, "warmup": 3, "ms_per_step": ms,
           "value": C * K / (ms * 1e-3), "unit": "cell·λ points/s", "tiling": tuned,
           "ray_lambda_segments_per_s": C * dp.rays.n_dirs * K / (ms * 1e-3),
           "profile_evaluations_per_s": stats["evaluations"] / (ms * 1e-3),
           "l2": "flushed between steps (512 MB write)",
           "line_sum_roofline": {"bound": "alu", "pipe": "xu (MUFU ex2/rsqrt/rcp)", "achieved": xu_ops / (kms * 1e-3) / 1e9,
                                 "peak": peak, "unit": "Gop/s", "frac": xu_ops / (kms * 1e-3) / 1e9 / peak,
                                 "traffic": line_sum_traffic(C, K), "traffic_algorithmic_bytes": C * K * 8,
                                 "kernel": "k_line_sum_f32_persist", "kernel_ms": kms, "evaluations": stats["evaluations"],
                                 "peak_source": f"{n_sm} SMs x 16 XU lanes x {sm_max / 1e6:.0f} MHz (max SM clock)"},
           "clocks": clk.summary()}
    q32 = float(r32["q"].item())
    chunked = {}
    for ch in (int(v) for v in args.stag_chunks.split(",") if v):
        # the same step through the chunk pipeline: per-chunk buffers, planning and flux per chunk
        cb = [(torch.empty((C, ch), dtype=torch.float32, device=dev), torch.empty((C, ch), dtype=torch.float32, device=dev))]
        solver.solve(dp, ctx, R.FP32, chunk=ch, buffers=cb)
        ctx.sync()
        cms = []
        for i in range(5):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rc = solver.solve(dp, ctx, R.FP32, chunk=ch, buffers=cb)
            b.record(stream)
            ctx.sync()
            cms.append(a.elapsed_time(b))
        chunked[str(ch)] = {"ms_per_step": float(np.mean(cms)), "q_rel_diff_vs_whole": abs(float(rc["q"].item()) / q32 - 1)}
        del cb
    if chunked:
        out["chunked"] = chunked
    if fp64:
        bufs64 = [(torch.empty((C, K), dtype=torch.float64, device=dev),
                   torch.empty((C, K), dtype=torch.float64, device=dev))]
        solver.solve(dp, ctx, R.FP64, buffers=bufs64)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record(stream)
        r64 = solver.solve(dp, ctx, R.FP64, buffers=bufs64)
        e1.record(stream)
        ctx.sync()
        ms64 = e0.elapsed_time(e1)
        q64 = float(r64["q"].item())
        out["fp64_plain"] = {"value": C * K / (ms64 * 1e-3), "ms_per_step": ms64, "q_W_cm2": q64,
                             "fp32_q_W_cm2": q32, "fp32_q_rel_err": abs(q32 / q64 - 1)}
        del bufs64
    del bufs
    ctx.close()
    torch.cuda.empty_cache()
    return out


def run_stagnation(args):
    """--workload stagnation: the stagnation-line block on its own."""
    world, rank, local = dist_setup()
    out = stagnation_block(args, local, world, rank, fp64=not args.no_fp64)
    print(json.dumps(out))
    return 0


def run_serve(args):
    """--workload serve: the served-request study on its own."""
    from paper_2604_11856_gb300 import synth
    world, rank, local = dist_setup()
    print(json.dumps({"workload": "served requests", **served(synth.stagnation_line(), args, local)}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return oracle_phases(args) if args.oracle_phases else run_reference(args)
    runs = {"afterbody": run_headline, "stagnation": run_stagnation, "serve": run_serve, "batch": run_batch,
            "fibonacci": run_fibonacci, "qss": run_qss, "continuum": run_continuum, "voigt": run_voigt}
    return runs[args.workload](args)


if __name__ == "__main__":
    sys.exit(main())
