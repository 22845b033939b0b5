"""Serving loop: radiation solves of different sizes arriving over time.

Requests (slab or line-of-sight solves with their own cells, spectral grid
and rays) share line lists that stay resident on the device.  A scheduler
admits queued requests in arrival order whenever a slot is free and the
request's device-memory estimate fits in the budget; each slot is a worker
thread with its own CUDA stream and library context, so admitted requests
run concurrently on the GPU while new ones keep arriving (continuous
batching at the request level).  The queue is bounded: beyond it requests
are shed and counted.  Results carry per-request latency (arrival to result
on the host) and the served flux.
"""
from __future__ import annotations

import collections
import dataclasses
import queue
import threading
import time

import numpy as np
import torch

from . import rapral as R
from . import solver, synth

CHUNK = 65536


@dataclasses.dataclass
class Request:
    rid: int
    problem: synth.Problem
    arrival: float = 0.0             # seconds after the start of the run
    precision: int = R.FP32
    status: str = "queued"           # queued / admitted / done / shed / failed
    q: np.ndarray | None = None
    t_admit: float = 0.0
    t_done: float = 0.0
    nbytes: int = 0
    error: str = ""

    @property
    def latency(self):
        return self.t_done - self.arrival


def request_bytes(problem, precision, chunk=CHUNK):
    """Device bytes a request holds while it runs: kappa / j chunk buffers,
    q_lambda, cell arrays and the library workspace."""
    C = len(problem.cells)
    nk = min(chunk, problem.grid.n)
    esz = 8 if precision == R.FP64 else 4
    geo = problem.geometry
    P = 1 if isinstance(geo, synth.SlabGeometry) else len(geo.surf_x)
    b = 2 * C * nk * esz + P * nk * esz + C * (8 * 13 + 8 * 8)
    b += R.workspace_bytes(len(problem.lines), C, nk)
    return int(b)


class Server:
    """`slots` concurrent workers on one GPU, admission by a byte budget.

    The budget defaults to the device's free memory once the resident line
    list is loaded, less `reserve_bytes`, capped at `cap_bytes` (150 GB, the
    served configuration's HBM budget)."""

    def __init__(self, lines, species, device=0, slots=4, budget_bytes=None, queue_limit=512, chunk=CHUNK,
                 reserve_bytes=16 << 30, cap_bytes=150 * 10 ** 9):
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.chunk = chunk
        self.queue_limit = queue_limit
        boot = R.Context(device)
        # resident line list and species database, shared by every request
        self.dlines = R.DeviceLines(lines, self.device)
        self.dspecies = R.DeviceSpecies(species, self.device)
        torch.cuda.synchronize(self.device)
        boot.close()
        if budget_bytes is None:
            free, _total = torch.cuda.mem_get_info(self.device)
            budget_bytes = min(cap_bytes, max(0, free - reserve_bytes))
        self.budget = int(budget_bytes)
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.in_use = 0
        self.high_water = 0
        self.free_slots = slots
        self.shed = 0
        self.done = []
        self.t0 = None
        self.stop = False
        self.workq = queue.Queue()
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        self.sched = threading.Thread(target=self._scheduler, daemon=True)

    def now(self):
        return time.perf_counter() - self.t0

    def start(self):
        self.t0 = time.perf_counter()
        for w in self.workers:
            w.start()
        self.sched.start()

    def submit(self, req: Request):
        req.nbytes = request_bytes(req.problem, req.precision, self.chunk)
        with self.cv:
            if req.nbytes > self.budget or len(self.pending) >= self.queue_limit:
                req.status = "shed"
                req.t_done = self.now()
                self.shed += 1
                self.done.append(req)
                return False
            self.pending.append(req)
            self.cv.notify_all()
        return True

    def _admissible(self):
        return bool(self.pending) and self.free_slots > 0 and self.in_use + self.pending[0].nbytes <= self.budget

    def _scheduler(self):
        while True:
            with self.cv:
                # wait (never spin) until the head of the queue fits, or the
                # server is closing with nothing left to admit
                while not self._admissible() and not (self.stop and not self.pending):
                    self.cv.wait(0.05)
                if not self._admissible():   # closing and the queue is empty
                    break
                req = self.pending.popleft()
                self.in_use += req.nbytes
                self.high_water = max(self.high_water, self.in_use)
                self.free_slots -= 1
                req.status = "admitted"
                req.t_admit = self.now()
            self.workq.put(req)
        for _ in self.workers:
            self.workq.put(None)

    def _worker(self, i):
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device)
        ctx = R.Context(self.device.index, stream=stream)
        while True:
            req = self.workq.get()
            if req is None:
                break
            try:
                with torch.cuda.stream(stream):
                    dp = solver.DeviceProblem(req.problem, ctx, lines=self.dlines, species=self.dspecies)
                    out = solver.solve(dp, ctx, req.precision, chunk=self.chunk)
                    q = out["q"].cpu()   # synchronises this stream only
                ctx.sync()
                req.q = q.numpy()
                req.status = "done"
            except Exception as e:   # a failed request does not stop the server
                req.status = "failed"
                req.error = str(e)
                ctx.clear_status()
            req.t_done = self.now()
            with self.cv:
                self.in_use -= req.nbytes
                self.free_slots += 1
                self.done.append(req)
                self.cv.notify_all()
        ctx.close()

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        self.sched.join()
        for w in self.workers:
            w.join()


def run_open_loop(server, requests):
    """Submits each request at its arrival time (open loop) and waits for all."""
    server.start()
    for r in sorted(requests, key=lambda r: r.arrival):
        dt = r.arrival - server.now()
        if dt > 0:
            time.sleep(dt)
        server.submit(r)
    server.close()
    return summarize(server, requests)


def summarize(server, requests):
    done = [r for r in requests if r.status == "done"]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    span = max((r.t_done for r in done), default=0.0) - min((r.arrival for r in requests), default=0.0)
    cl = sum(len(r.problem.cells) * r.problem.grid.n for r in done)
    return {"requests": len(requests), "done": len(done), "shed": sum(r.status == "shed" for r in requests),
            "failed": sum(r.status == "failed" for r in requests),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "throughput_req_s": len(done) / span if span > 0 else 0.0,
            "cell_lambda_per_s": cl / span if span > 0 else 0.0,
            "budget_bytes": server.budget, "high_water_bytes": server.high_water}


def solo(requests, lines, species, device=0, chunk=CHUNK):
    """Each request alone on an idle GPU (reference for the mix)."""
    dev = torch.device("cuda", device)
    ctx = R.Context(device)
    dl = R.DeviceLines(lines, dev)
    ds = R.DeviceSpecies(species, dev)
    out = {}
    for r in requests:
        dp = solver.DeviceProblem(r.problem, ctx, lines=dl, species=ds)
        q = solver.solve(dp, ctx, r.precision, chunk=chunk)["q"].cpu().numpy()
        ctx.sync()
        out[r.rid] = q
    ctx.close()
    return out
