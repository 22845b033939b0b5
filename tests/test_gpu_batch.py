"""Batched persistent solves: many uneven slab solves in one persistent
line-sum launch per spectral round, eager and replayed from a CUDA graph;
every solve equals the same solve run alone (same chunking) and the
oracle within the FP32 tolerance."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_11856_gb300 import batch, rapral as R, solver, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problems():
    pool = synth._air_lines(np.random.default_rng(1001), 2000, 20000)
    probs = synth.batch_slabs(n_solves=6, pool=pool, scale=0.01)
    probs += synth.batch_slabs(seed=77, n_solves=3, pool=pool, scale=0.01, iid_cells=True)
    return probs


@pytest.mark.parametrize("pb", [32, 64])
def test_batch_equals_solo_and_graph_replays(problems, pb):
    ctx = R.Context(0)
    ctx.set_line_batch(pb)   # lines staged per sweep pass, in the batch and in the solo runs
    chunk = 3000
    bs = batch.BatchSolver(problems, ctx, chunk=chunk)
    assert len(bs.handles) >= 2   # several spectral rounds
    q_eager = [q.cpu().numpy().copy() for q in bs.run()]
    ctx.sync()
    bs.capture()
    q_g1 = [q.cpu().numpy().copy() for q in bs.replay()]
    q_g2 = [q.cpu().numpy().copy() for q in bs.replay()]
    torch.cuda.synchronize()
    ctx.sync()
    for i, p in enumerate(problems):
        dp = solver.DeviceProblem(p, ctx)
        solo = solver.solve(dp, ctx, R.FP32, chunk=chunk)["q"].cpu().numpy()
        ctx.sync()
        np.testing.assert_allclose(q_eager[i], solo, rtol=1e-12, atol=0)
        assert np.array_equal(q_g1[i], q_eager[i]) and np.array_equal(q_g2[i], q_eager[i])
    bs.close()


def test_batch_matches_oracle(problems):
    ctx = R.Context(0)
    p = problems[0]
    bs = batch.BatchSolver([p], ctx, chunk=2500)
    q = bs.run()[0].cpu().numpy()
    ctx.sync()
    ref = oracle.solve_slab(p)["q"]
    assert abs(q[0] / ref - 1) <= 1e-4, (q, ref)
    bs.close()


def test_mixed_slab_and_line_of_sight_batch():
    """One batch mixing tangent-slab solves with an axisymmetric
    line-of-sight solve (3 surface points x 32 single-direction rays): every
    solve equals the same solve run alone, and the line-of-sight solve's
    wall fluxes equal the oracle's within the FP32 heat-flux tolerance."""
    import types
    ctx = R.Context(0)
    pool = synth._air_lines(np.random.default_rng(1001), 2000, 20000)
    lines_all, species, _ = pool
    slabs = synth.batch_slabs(n_solves=3, pool=pool, scale=0.01)
    los = synth.afterbody(nx=40, nr=20, x_len=20.0, r_body=3.35, r_len=15.0, n_points=3, n_mu=4, n_phi=8,
                          n_grid=8001, lines_from=types.SimpleNamespace(lines=lines_all, species=species), chunk=0)
    probs = [slabs[0], los] + slabs[1:]
    chunk = 3000
    bs = batch.BatchSolver(probs, ctx, chunk=chunk)
    q = [x.cpu().numpy().copy() for x in bs.run()]
    ctx.sync()
    bs.capture()
    q_g = [x.cpu().numpy().copy() for x in bs.replay()]
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        dp = solver.DeviceProblem(p, ctx)
        solo = solver.solve(dp, ctx, R.FP32, chunk=chunk)["q"].cpu().numpy()
        ctx.sync()
        np.testing.assert_allclose(q[i], solo, rtol=1e-12, atol=0)
        assert np.array_equal(q_g[i], q[i])
    rk, re = oracle.spectral_coeffs(los)
    _ql, ref = oracle.solve_axisym_points(los, range(len(los.geometry.surf_x)), rk, re)
    err = np.abs(q[1] / ref - 1)
    print(f"  line-of-sight solve in the batch: max |q / q_oracle - 1| = {err.max():.2e}")
    assert err.max() <= 1e-4
    bs.close()
