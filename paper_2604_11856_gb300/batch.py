"""Batched solves: many independent, uneven slab / line-of-sight solves
planned together and run as one persistent line-sum launch per spectral
round, optionally captured in a CUDA graph.

Each solve's grid is cut into chunks of `chunk` points; round r holds chunk
r of every solve that has one.  A round is one rapral_batch (planned once:
line records and tile lists of every request); a run is: zero the fluxes,
populations of every solve, then every round's rapral_batch_run.  Nothing
in a run allocates or synchronises, so the whole run is captured in one
CUDA graph and replayed.
"""
from __future__ import annotations

import ctypes as ct

import torch

from . import rapral as R
from . import solver


class BatchSolver:
    def __init__(self, problems, ctx, chunk=65536, species=None, tile_width=None, cells_per_block=None):
        self.ctx = ctx
        dev = ctx.device
        if tile_width or cells_per_block:
            ctx.set_tiling(tile_width or 0, cells_per_block or 0)
        sp = species if species is not None else R.DeviceSpecies(problems[0].species, dev)
        self.dps = [solver.DeviceProblem(p, ctx, species=sp) for p in problems]
        self.chunk = chunk
        self.bufs, self.q, self.grids = [], [], []
        for dp in self.dps:
            nk = min(chunk, dp.grid.n)
            self.bufs.append((torch.empty((dp.C, nk), dtype=torch.float32, device=dev),
                              torch.empty((dp.C, nk), dtype=torch.float32, device=dev),
                              torch.empty((dp.P, nk), dtype=torch.float32, device=dev)))
            self.q.append(torch.zeros(dp.P, dtype=torch.float64, device=dev))
            self.grids.append(R.grid_struct(dp.grid))
        self.handles = []
        self._keep = []
        n_rounds = max((dp.grid.n + chunk - 1) // chunk for dp in self.dps)
        for r in range(n_rounds):
            items = []
            for i, dp in enumerate(self.dps):
                k0 = r * chunk
                if k0 >= dp.grid.n:
                    continue
                nk = min(chunk, dp.grid.n - k0)
                kap, em, ql = self.bufs[i]
                it = R.BatchItem()
                it.species = ct.addressof(dp.species.struct)
                it.lines = ct.addressof(dp.lines.struct)
                it.cells = ct.addressof(dp.cells.struct)
                it.grid = ct.addressof(self.grids[i])
                it.rays = ct.addressof(dp.rays.struct)
                it.k0, it.nk = k0, nk
                it.kappa, it.emis, it.ld = kap.data_ptr(), em.data_ptr(), kap.shape[1]
                it.q_lambda, it.q = ql.data_ptr(), self.q[i].data_ptr()
                items.append(it)
            arr = (R.BatchItem * len(items))(*items)
            self._keep.append(arr)
            # populations first: planning reads the cells, the run reads lnpref
            if r == 0:
                for dp in self.dps:
                    R.populations(ctx, dp.species, dp.cells)
            h = ct.c_void_p()
            ctx.check(ctx.lib.rapral_batch_create(ctx.h, len(items), arr, R.FP32, ct.byref(h)))
            self.handles.append(h)
        self.graph = None

    def units(self):
        out = []
        for h in self.handles:
            u, b = ct.c_int64(), ct.c_int()
            self.ctx.lib.rapral_batch_units(h, ct.byref(u), ct.byref(b))
            out.append((u.value, b.value))
        return out

    def _enqueue(self):
        for q in self.q:
            q.zero_()
        for dp in self.dps:
            R.populations(self.ctx, dp.species, dp.cells)
        for h in self.handles:
            self.ctx.check(self.ctx.lib.rapral_batch_run(self.ctx.h, h))

    def run(self):
        """Eager run on the context's stream."""
        with torch.cuda.stream(self.ctx.stream):
            self._enqueue()
        return self.q

    def capture(self):
        """Captures one whole run in a CUDA graph."""
        torch.cuda.synchronize(self.ctx.device)
        g = torch.cuda.CUDAGraph()
        old = self.ctx.stream
        with torch.cuda.graph(g):
            self.ctx.set_stream(torch.cuda.current_stream())
            self._enqueue()
        self.ctx.set_stream(old)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.q

    def close(self):
        for h in self.handles:
            self.ctx.lib.rapral_batch_destroy(h)
        self.handles = []
