"""Serving loop on the GPU: continuous admission under a memory budget,
concurrent requests on several streams, each served result equal to the
same request solved alone, and served results of both kinds (slab and line
of sight) equal to the oracle's within the tolerance of their arithmetic."""
import numpy as np
import pytest

import oracle
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    return synth._air_lines(np.random.default_rng(1001), 2000, 20000)


def _requests(pool, n, rate, precision, seed=1004, scale=0.02):
    reqs = synth.served_requests(seed=seed, n_requests=n, rate=rate, pool=pool, scale=scale)
    return [serve.Request(rid=i, problem=r["problem"], arrival=r["t"], precision=precision) for i, r in enumerate(reqs)]


@pytest.mark.parametrize("precision", [R.FP32, R.FP64])
def test_served_results_equal_solo(pool, precision):
    lines, species, _ = pool
    reqs = _requests(pool, 24, 400.0, precision)
    largest = max(serve.request_bytes(r.problem, precision) for r in reqs)
    srv = serve.Server(lines, species, slots=4, budget_bytes=3 * largest)
    stats = serve.run_open_loop(srv, reqs)
    bad = [(r.rid, r.status, r.error) for r in reqs if r.status != "done"]
    assert not bad, (stats, bad[:5])
    assert stats["high_water_bytes"] <= stats["budget_bytes"]
    ref = serve.solo(reqs, lines, species)
    bitwise = 0
    for r in reqs:
        np.testing.assert_allclose(r.q, ref[r.rid], rtol=1e-12, atol=0)
        bitwise += bool(np.array_equal(r.q, ref[r.rid]))
    print(f"  {stats}; bitwise equal {bitwise}/{len(reqs)}")


def test_bounded_queue_sheds(pool):
    lines, species, _ = pool
    reqs = _requests(pool, 30, 1e6, R.FP32)   # a burst
    srv = serve.Server(lines, species, slots=1, queue_limit=3)
    stats = serve.run_open_loop(srv, reqs)
    assert stats["shed"] > 0
    assert stats["done"] + stats["shed"] == len(reqs)


@pytest.mark.parametrize("precision,tol", [(R.FP32, 1e-4), (R.FP64, 1e-10)])
def test_served_results_match_oracle(pool, precision, tol):
    """Requests served in a concurrent mix: at least two tangent-slab and two
    single line-of-sight requests are checked against the oracle's whole
    solve of the same problem (heat flux within 1e-4 for FP32, 1e-10 for
    FP64)."""
    lines, species, _ = pool
    reqs = _requests(pool, 16, 400.0, precision, seed=2024)
    srv = serve.Server(lines, species, slots=4)
    stats = serve.run_open_loop(srv, reqs)
    assert stats["done"] == len(reqs), stats
    slab = [r for r in reqs if len(r.problem.geometry.mu) > 1][:2]
    los = [r for r in reqs if len(r.problem.geometry.mu) == 1][:2]
    assert len(slab) == 2 and len(los) == 2
    for r in slab + los:
        ref = oracle.solve_slab(r.problem)["q"]
        err = abs(r.q[0] / ref - 1)
        print(f"  request {r.rid} ({len(r.problem.cells)} cells, {r.problem.grid.n} points, "
              f"{len(r.problem.geometry.mu)} directions): q {r.q[0]!r} oracle {ref!r} rel {err:.2e}")
        assert err <= tol
