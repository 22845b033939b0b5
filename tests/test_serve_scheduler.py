"""The serving loop's scheduler on the CPU, with stand-in workers (no GPU):
requests are admitted in arrival order within the slot count and the byte
budget, every request is served, and while the server is closing with
requests still queued behind busy slots the scheduler waits for a slot
instead of spinning (a spinning scheduler holds the interpreter lock away
from the workers)."""
import collections
import queue
import threading
import time
import types

from paper_2604_11856_gb300 import serve


def _problem(nbytes):
    return types.SimpleNamespace(cells=[0], grid=types.SimpleNamespace(n=1), nbytes=nbytes)


class CountingCondition(threading.Condition):
    def __init__(self):
        super().__init__()
        self.entries = 0

    def __enter__(self):
        self.entries += 1
        return super().__enter__()


def _server(slots, budget):
    srv = serve.Server.__new__(serve.Server)
    srv.chunk, srv.queue_limit, srv.budget = serve.CHUNK, 512, budget
    srv.pending, srv.cv = collections.deque(), CountingCondition()
    srv.in_use = srv.high_water = srv.shed = 0
    srv.free_slots, srv.done, srv.stop = slots, [], False
    srv.workq, srv.t0 = queue.Queue(), time.perf_counter()
    order, live = [], [0, 0]

    def worker():
        while True:
            req = srv.workq.get()
            if req is None:
                break
            with srv.cv:
                order.append(req.rid)
                live[0] += 1
                live[1] = max(live[1], live[0])
            time.sleep(0.02)              # the request's GPU work
            req.status, req.t_done = "done", srv.now()
            with srv.cv:
                live[0] -= 1
                srv.in_use -= req.nbytes
                srv.free_slots += 1
                srv.done.append(req)
                srv.cv.notify_all()

    srv.workers = [threading.Thread(target=worker, daemon=True) for _ in range(slots)]
    srv.sched = threading.Thread(target=srv._scheduler, daemon=True)
    return srv, order, live


def test_scheduler_admits_in_order_and_waits_while_closing(monkeypatch):
    sizes = [30, 50, 20, 60, 10, 40, 30, 20, 50, 10, 30, 40]
    monkeypatch.setattr(serve, "request_bytes", lambda problem, precision, chunk=serve.CHUNK: problem.nbytes)
    srv, order, live = _server(slots=2, budget=100)
    reqs = [serve.Request(rid=i, problem=_problem(b), arrival=0.0) for i, b in enumerate(sizes)]
    stats = serve.run_open_loop(srv, reqs)   # all arrive at once: close() runs with a full queue
    assert stats["done"] == len(sizes) and stats["shed"] == 0
    assert order == list(range(len(sizes)))          # FIFO admission
    assert live[1] <= 2 and srv.high_water <= 100    # slots and budget respected
    assert srv.in_use == 0 and srv.free_slots == 2
    # 12 requests of 20 ms on two slots take ~0.15 s; waiting in 50 ms steps
    # plus the wake-ups of the workers' notifications is a few dozen entries,
    # a spinning loop hundreds of thousands
    assert srv.cv.entries < 500, srv.cv.entries


def test_oversized_request_is_shed(monkeypatch):
    monkeypatch.setattr(serve, "request_bytes", lambda problem, precision, chunk=serve.CHUNK: problem.nbytes)
    srv, order, _live = _server(slots=1, budget=100)
    reqs = [serve.Request(rid=0, problem=_problem(150), arrival=0.0),
            serve.Request(rid=1, problem=_problem(40), arrival=0.0)]
    stats = serve.run_open_loop(srv, reqs)
    assert stats["shed"] == 1 and stats["done"] == 1 and order == [1]
