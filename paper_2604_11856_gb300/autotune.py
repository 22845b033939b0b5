"""Autotuner of the FP32 line sum: spectral tile width, cells (warps) per
block and lines (line, cell pairs) a warp stages per sweep pass.

For a workload class (GPU, line count, grid spacing) it times the
coefficient step of a representative sample -- a chunk from the middle of
the grid and a spread of cells -- under every candidate setting, keeps the
fastest by median of a few repetitions, and caches the choice in a JSON file
next to the built library.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import build as _build
from . import rapral as R
from . import solver, synth

CANDIDATES = [(tw, wpb, pb) for pb in (32, 64) for tw in (128, 256) for wpb in (2, 4, 8)]
CACHE = os.path.join(_build.BUILD, "autotune.json")


def _key(problem, precision):
    name = torch.cuda.get_device_name().replace(" ", "_")
    h = (problem.grid.lam_max - problem.grid.lam_min) / (problem.grid.n - 1)
    lb = int(round(math.log2(max(1, len(problem.lines)))))
    hb = int(round(math.log2(h * 1e4)))
    return f"{name}|p{precision}|L2^{lb}|h2^{hb}"


def _load():
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def _store(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, CACHE)


def sample_problem(problem, n_cells=48):
    """A spread of the problem's cells (same lines, grid, geometry type)."""
    C = len(problem.cells)
    idx = np.unique(np.linspace(0, C - 1, min(C, n_cells)).round().astype(int))
    cells = synth.Cells(Ttr=problem.cells.Ttr[idx], Tve=problem.cells.Tve[idx], n=problem.cells.n[idx])
    geo = synth.SlabGeometry(cell_order=np.arange(len(idx), dtype=np.int64), dx=np.ones(len(idx)),
                             mu=np.array([1.0]), wmu=np.array([1.0]), normal_ray=False)
    return synth.Problem(problem.name, problem.species, problem.lines, cells, problem.grid, geo)


def tune(ctx, problem, precision=R.FP32, nk=65536, reps=3, use_cache=True, candidates=CANDIDATES):
    """Returns (tile_width, cells_per_block, pairs_per_pass, timings) and
    applies the choice to `ctx`."""
    key = _key(problem, precision)
    cache = _load() if use_cache else {}
    if use_cache and key in cache and len(cache[key]["choice"]) == 3:
        tw, wpb, pb = cache[key]["choice"]
        ctx.set_tiling(tw, wpb)
        ctx.set_line_batch(pb)
        return tw, wpb, pb, cache[key]["ms"]
    sp = sample_problem(problem)
    dp = solver.DeviceProblem(sp, ctx)
    R.populations(ctx, dp.species, dp.cells)
    nk = min(nk, sp.grid.n)
    k0 = (sp.grid.n - nk) // 2
    kap = torch.empty((dp.C, nk), dtype=torch.float32, device=ctx.device)
    em = torch.empty_like(kap)
    times = {}
    for tw, wpb, pb in candidates:
        ctx.set_tiling(tw, wpb)
        ctx.set_line_batch(pb)
        R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, sp.grid, k0, nk, precision, kap, em)   # warm
        ctx.sync()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream); b.record(ctx.stream)
            ctx.set_profile_events(a, b)
            R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, sp.grid, k0, nk, precision, kap, em)
            ctx.set_profile_events(None, None)
            ctx.sync()
            ms.append(a.elapsed_time(b))
        times[f"{tw}x{wpb}x{pb}"] = float(np.median(ms))
    best = min(times, key=times.get)
    tw, wpb, pb = (int(x) for x in best.split("x"))
    ctx.set_tiling(tw, wpb)
    ctx.set_line_batch(pb)
    if use_cache:
        cache = _load()
        cache[key] = {"choice": [tw, wpb, pb], "ms": times}
        _store(cache)
    return tw, wpb, pb, times
