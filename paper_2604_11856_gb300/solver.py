"""Whole solves over the C-ABI: populations -> spectral coefficients (per
spectral chunk) -> ray march -> wall flux.

`DeviceProblem` holds a problem's inputs resident on the device; `solve`
runs the path on them (optionally in spectral chunks, with the line sum of
chunk k+1 overlapping the march of chunk k on a second stream);
`solve_host` is the end-to-end call that starts from host arrays, copies
them in, and returns the wall flux on the host.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rapral as R
from . import synth


class DeviceProblem:
    """A problem's species, lines, cells, rays and grid on one device."""

    def __init__(self, problem, ctx, points=None, lines=None, species=None):
        dev = ctx.device
        self.problem = problem
        self.grid = problem.grid
        self.species = species if species is not None else R.DeviceSpecies(problem.species, dev)
        self.lines = lines if lines is not None else R.DeviceLines(problem.lines, dev)
        self.cells = R.DeviceCells(problem.cells, self.species.S, dev)
        geo = problem.geometry
        if isinstance(geo, synth.SlabGeometry):
            self.rays = R.slab_rays(ctx, geo, dev)
        elif isinstance(geo, synth.AxisymGeometry):
            self.rays = R.axisym_rays(ctx, geo, dev, points=points)
        else:
            raise TypeError(f"unknown geometry {type(geo)}")
        self.C = self.cells.C
        self.P = self.rays.n_points


def _dtype(precision):
    return torch.float64 if precision == R.FP64 else torch.float32


def shard_range(n, rank, world, align=512):
    """Contiguous part [k0, k0 + nk) of an n-point grid for `rank` of
    `world`, boundaries on multiples of `align` (a tile width)."""
    blocks = (n + align - 1) // align
    b0 = blocks * rank // world
    b1 = blocks * (rank + 1) // world
    k0 = min(n, b0 * align)
    k1 = min(n, b1 * align)
    return k0, k1 - k0


class ChunkPipeline:
    """A problem's spectral chunks enqueued one at a time on two streams:
    chunk i's coefficients on ctx's stream (A), its march and flux on ctx2's
    stream (B), with two kappa / j buffers, so that the line sum of chunk
    i + 1 overlaps the march of chunk i.  `begin` starts a pass over the
    grid (zeroes q on B, populations on A); `step(k0, nk)` enqueues one chunk;
    `end` joins B into A.  Nothing allocates or synchronises the host after
    construction.  Without ctx2 every step runs on A."""

    def __init__(self, dp, ctx, precision, chunk, ctx2=None, buffers=None, continuum=None, I=None):
        self.dp, self.ctx, self.ctx2, self.precision = dp, ctx, ctx2, precision
        self.continuum, self.I = continuum, I
        dev = ctx.device
        dt = _dtype(precision)
        nbuf = 2 if ctx2 is not None else 1
        if buffers is None:
            buffers = [(torch.empty((dp.C, chunk), dtype=dt, device=dev),
                        torch.empty((dp.C, chunk), dtype=dt, device=dev)) for _ in range(nbuf)]
        self.buffers = buffers[:nbuf]
        self.qlam = torch.empty((dp.P, chunk), dtype=dt, device=dev)
        self.q = torch.zeros(dp.P, dtype=torch.float64, device=dev)
        self.i = 0
        self.used = [False] * nbuf
        if ctx2 is not None:
            self.free = [torch.cuda.Event() for _ in range(nbuf)]
            self.ready = torch.cuda.Event()
            self.ev = torch.cuda.Event()

    @property
    def march_ctx(self):
        return self.ctx2 if self.ctx2 is not None else self.ctx

    def begin(self, q=None):
        """Starts a pass: q (default: the pipeline's own) is zeroed on the
        march stream after its earlier uses, populations run on stream A."""
        if q is not None:
            self.q = q
        dp, ctx = self.dp, self.ctx
        if self.ctx2 is not None:   # earlier readers of q on stream A come first
            self.ev.record(ctx.stream)
            self.ctx2.stream.wait_event(self.ev)
        with torch.cuda.stream(self.march_ctx.stream):
            self.q.zero_()
        R.populations(ctx, dp.species, dp.cells)
        if self.ctx2 is not None:
            self.ev.record(ctx.stream)
            self.ctx2.stream.wait_event(self.ev)

    def step(self, k0, nk, march_events=None):
        """Enqueues grid points [k0, k0 + nk); `march_events` (a pair of
        torch.cuda.Event) are recorded around the march on its stream."""
        dp, ctx, prec = self.dp, self.ctx, self.precision
        b = self.i % len(self.buffers)
        kap, em = self.buffers[b]
        if self.ctx2 is not None and self.used[b]:
            ctx.stream.wait_event(self.free[b])
        R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, dp.grid, k0, nk, prec, kap, em)
        if self.continuum is not None:
            R.continuum_coeffs(ctx, self.continuum, dp.species.S, dp.cells, dp.grid, k0, nk, prec, kap, em)
        mc = self.march_ctx
        if self.ctx2 is not None:
            self.ready.record(ctx.stream)
            self.ctx2.stream.wait_event(self.ready)
        if march_events is not None:
            march_events[0].record(mc.stream)
        R.trace_rays(mc, dp.rays, dp.C, kap, em, dp.grid, k0, nk, prec, self.qlam, self.I)
        if march_events is not None:
            march_events[1].record(mc.stream)
        R.wall_flux(mc, self.qlam, prec, dp.grid, k0, nk, dp.P, self.q)
        if self.ctx2 is not None:
            self.free[b].record(self.ctx2.stream)
            self.used[b] = True
        self.i += 1
        return kap, em

    def end(self):
        if self.ctx2 is not None:
            self.ev.record(self.ctx2.stream)
            self.ctx.stream.wait_event(self.ev)
        return self.q


def solve(dp, ctx, precision=R.FP64, chunk=None, keep_coeffs=False, keep_intensity=False, ctx2=None,
          buffers=None, k_start=0, k_stop=None, continuum=None):
    """Runs the whole path on device-resident inputs over the grid points
    [k_start, k_stop) (default: all).  Returns a dict with q [P] (FP64,
    device; the range's part of the flux with the whole grid's trapezoid
    weights) and, on request, kappa / emis [C, nk] and q_lambda [P, nk] /
    I [n_dirs, nk] (single chunk only).  With ctx2 (a second context on
    another stream) chunk k+1's line sum overlaps chunk k's march.  With
    continuum (an R.DeviceContinuum) the atomic bound-free and free-free
    continuum is added to every chunk's coefficients before the march."""
    k_stop = dp.grid.n if k_stop is None else k_stop
    n_range = k_stop - k_start
    chunk = n_range if not chunk else min(chunk, n_range)
    I = None
    if keep_intensity:
        I = torch.empty((dp.rays.n_dirs, chunk), dtype=_dtype(precision), device=ctx.device)
    pipe = ChunkPipeline(dp, ctx, precision, chunk, ctx2=ctx2, buffers=buffers, continuum=continuum, I=I)
    starts = list(range(k_start, k_stop, chunk))
    pipe.begin()
    for k0 in starts:
        kap, em = pipe.step(k0, min(chunk, k_stop - k0))
    pipe.end()
    out = {"q": pipe.q}
    if len(starts) == 1:
        if keep_coeffs:
            out["kappa"], out["emis"] = kap, em
        out["q_lambda"] = pipe.qlam
        if keep_intensity:
            out["I"] = I
    return out


def shard_ranges(n, rank, world, chunk=None):
    """Grid ranges [(k0, nk), ...] of `rank`'s spectral shard.  With `chunk`,
    the grid is cut into chunk-point chunks dealt round-robin (chunk i to
    rank i mod world), which spreads the heavier short-wavelength chunks over
    the ranks; without, one contiguous tile-aligned range (shard_range)."""
    if chunk:
        return [(k0, min(chunk, n - k0)) for i, k0 in enumerate(range(0, n, chunk)) if i % world == rank]
    k0, nk = shard_range(n, rank, world)
    return [(k0, nk)] if nk > 0 else []


def solve_sharded(dp, ctx, rank, world, precision=R.FP32, chunk=None, group=None, ctx2=None, dealt=False,
                  reduce=True):
    """Spectral sharding across ranks (Sec. 2.3 parallelises the spectral
    evaluation): each rank solves its shard of the grid (shard_ranges; dealt
    chunks with `dealt`, else one contiguous range cut into `chunk`-point
    chunks), populations replicated, no data exchange; then one FP64 sum of
    the P partial fluxes over the process group (skipped with reduce=False or
    world == 1) finishes the job.  Returns q [P] (device)."""
    ranges = shard_ranges(dp.grid.n, rank, world, chunk if dealt else None)
    span = max((nk for _k0, nk in ranges), default=1)
    step = min(chunk, span) if chunk else span
    pipe = ChunkPipeline(dp, ctx, precision, step, ctx2=ctx2)
    pipe.begin()
    for k0, nk in ranges:
        for c0 in range(k0, k0 + nk, step):
            pipe.step(c0, min(step, k0 + nk - c0))
    q = pipe.end()
    if reduce and world > 1:
        import torch.distributed as dist
        with torch.cuda.stream(ctx.stream):
            dist.all_reduce(q, op=dist.ReduceOp.SUM, group=group)
    return q


def solve_host(problem, precision=R.FP64, chunk=None, ctx=None, device=None, ctx2=None, k_start=0, k_stop=None):
    """End-to-end: host arrays in, wall flux out.  Inputs are staged through
    pinned host memory and copied on the context's stream; the result (the
    flux of grid points [k_start, k_stop), default all) is read back to the
    host.  With ctx2 the chunks are pipelined on two streams as in `solve`.
    Returns (q numpy array, bytes in, bytes out)."""
    if ctx is None:
        ctx = R.Context(device)
    dev = ctx.device
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()
    with torch.cuda.stream(ctx.stream):
        sp = problem.species
        hs = dict(kind=pin(sp.kind, np.int32), density_col=pin(sp.density_col, np.int32), mass=pin(sp.mass, np.float64),
                  atom_off=pin(sp.atom_off, np.int64), atom_E=pin(sp.atom_E, np.float64),
                  atom_g=pin(sp.atom_g, np.float64), st_off=pin(sp.st_off, np.int64), st_E=pin(sp.st_E, np.float64),
                  st_g=pin(sp.st_g, np.float64), st_sigma=pin(sp.st_sigma, np.float64),
                  st_Lalt=pin(sp.st_Lalt, np.float64), st_nv=pin(sp.st_nv, np.int32), st_nj=pin(sp.st_nj, np.int32),
                  st_vib_off=pin(sp.st_vib_off, np.int64), st_rot_off=pin(sp.st_rot_off, np.int64),
                  vib_E=pin(sp.vib_E, np.float64), rot_E=pin(sp.rot_E, np.float64))
        hl = {k: pin(getattr(problem.lines, k), np.float64) for k in R.LINE_KEYS}
        hl["species"] = pin(problem.lines.species, np.int32)
        hc = dict(Ttr=pin(problem.cells.Ttr, np.float64), Tve=pin(problem.cells.Tve, np.float64),
                  n=pin(problem.cells.n, np.float64))
        nbytes = sum(t.numel() * t.element_size() for d in (hs, hl, hc) for t in d.values())
        dl = {k: v.to(dev, non_blocking=True) for k, v in hl.items()}
        dc = {k: v.to(dev, non_blocking=True) for k, v in hc.items()}
        dsp = R.DeviceSpecies.__new__(R.DeviceSpecies)
        dsp.t = {k: v.to(dev, non_blocking=True) for k, v in hs.items()}
        s = R.Species()
        s.n_species = len(sp.names)
        for k, v in dsp.t.items():
            setattr(s, k, v.data_ptr() if v.numel() else None)
        s.n_atom_levels, s.n_states = int(sp.atom_E.shape[0]), int(sp.st_E.shape[0])
        s.n_vib, s.n_rot = int(sp.vib_E.shape[0]), int(sp.rot_E.shape[0])
        dsp.struct, dsp.S = s, s.n_species
        dp = DeviceProblem.__new__(DeviceProblem)
        dp.problem, dp.grid, dp.species = problem, problem.grid, dsp
        dp.lines = R.DeviceLines(None, dev, tensors=dl)
        dp.cells = R.DeviceCells(problem.cells, dsp.S, dev, tensors=dc)
        geo = problem.geometry
        dp.rays = R.slab_rays(ctx, geo, dev) if isinstance(geo, synth.SlabGeometry) else R.axisym_rays(ctx, geo, dev)
        dp.C, dp.P = dp.cells.C, dp.rays.n_points
        res = solve(dp, ctx, precision, chunk, ctx2=ctx2, k_start=k_start, k_stop=k_stop)
        q_host = torch.empty(res["q"].shape, dtype=torch.float64).pin_memory()
        q_host.copy_(res["q"], non_blocking=True)
    ctx.sync()
    return q_host.numpy().copy(), nbytes, q_host.numel() * 8


def solve_fibonacci(problem, ctx, n_los, n_phi, n_theta, precision=R.FP64, chunk=None, points=None,
                    species=None, lines=None):
    """The paper's own angular path (Sec. 2.2.3) for an axisymmetric problem:
    Fibonacci lines of sight from the surface points (or the selected ones),
    flow variables interpolated to their nodes, kappa / j at the nodes, the
    node march, the per-line wavelength integral S and the flux from S on a
    uniform (phi, theta) grid.  Returns a dict with q [P] (FP64, device), S
    [lines] (FP64, device), the rays and the node cells; with one chunk also
    the intensities I [lines, n] and the node tables kappa / emis."""
    dev = ctx.device
    geo = problem.geometry
    sp = species if species is not None else R.DeviceSpecies(problem.species, dev)
    ln = lines if lines is not None else R.DeviceLines(problem.lines, dev)
    gcells = R.DeviceCells(problem.cells, sp.S, dev)
    rays = R.fibonacci_rays(ctx, geo, n_los, dev, points)
    ncells = R.los_node_states(ctx, geo, gcells, rays, sp.S, dev)
    R.populations(ctx, sp, ncells)
    N, B, P = rays.n_nodes, rays.n_dirs, rays.n_points
    n = problem.grid.n
    chunk = n if not chunk else min(chunk, n)
    dt = _dtype(precision)
    kap = torch.empty((max(N, 1), chunk), dtype=dt, device=dev)
    em = torch.empty_like(kap)
    Ibuf = torch.empty(max(B, 1) * chunk, dtype=dt, device=dev)
    qbuf = torch.empty(max(P, 1) * chunk, dtype=dt, device=dev)
    S = torch.zeros(max(B, 1), dtype=torch.float64, device=dev)
    for k0 in range(0, n, chunk):
        nk = min(chunk, n - k0)
        I = Ibuf[:B * nk].view(B, nk)
        R.spectral_coeffs(ctx, sp, ln, ncells, problem.grid, k0, nk, precision, kap, em)
        R.trace_rays(ctx, rays, N, kap, em, problem.grid, k0, nk, precision, qbuf[:P * nk].view(P, nk), I)
        R.wall_flux(ctx, I, precision, problem.grid, k0, nk, B, S)
    q = torch.empty(max(P, 1), dtype=torch.float64, device=dev)
    R.fibonacci_flux(ctx, rays, S, n_phi, n_theta, q)
    out = dict(q=q[:P], S=S[:B], rays=rays, node_cells=ncells)
    if chunk == n:
        out["I"] = Ibuf[:B * n].view(B, n)
        out["kappa"], out["emis"] = kap[:N], em[:N]
    return out
