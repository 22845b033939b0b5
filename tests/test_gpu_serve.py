"""Serving loop on the GPU: continuous admission under a memory budget,
concurrent requests on several streams, and each served result equal to
the same request solved alone."""
import numpy as np
import pytest

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
