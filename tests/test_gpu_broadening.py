"""The optional Lorentz terms of Sec. 2.2.1 (Stark coefficient from the
ionisation gap, resonance and van der Waals widths) on the GPU against the
oracle: FP64 to 1e-10 relative, FP32 to the FP32 tolerance with the same
window decisions as FP64, and the batched path equal to the single call."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu

ALL = R.BROAD_STARK_IONIZE | R.BROAD_RESONANCE | R.BROAD_VDW


@pytest.fixture()
def ctx():
    c = R.Context(0)
    yield c
    c.set_broadening(0)


def _problem():
    return synth.stagnation_line(n_cells=24, n_atomic=3000, n_molecular=20000, n_grid=60001)


def _gpu(ctx, p, precision, flags):
    ctx.set_broadening(flags, synth.RAD_E_IONIZE, synth.FLOW_MASS)
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    dt = torch.float64 if precision == R.FP64 else torch.float32
    kap = torch.empty((dp.C, p.grid.n), dtype=dt, device=ctx.device)
    em = torch.empty_like(kap)
    ctx.reset_stats()
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, p.grid.n, precision, kap, em)
    ctx.sync()
    return kap.double().cpu().numpy(), em.double().cpu().numpy(), ctx.get_stats()["evaluations"]


def _oracle(p, flags):
    oracle.set_broadening(flags, synth.RAD_E_IONIZE, synth.FLOW_MASS)
    try:
        return oracle.spectral_coeffs(p, with_abs=True)
    finally:
        oracle.set_broadening(0)


@pytest.mark.parametrize("flags", [R.BROAD_STARK_IONIZE, R.BROAD_RESONANCE, R.BROAD_VDW, ALL])
def test_broadening_fp64_matches_oracle(ctx, flags):
    p = _problem()
    kap, em, _ = _gpu(ctx, p, R.FP64, flags)
    rk, re, ra = _oracle(p, flags)
    den = np.maximum(np.abs(re), 1e-300)
    assert np.max(np.abs(em - re) / den) <= 1e-10
    scale = np.maximum(np.abs(rk), ra)
    m = scale > 0
    assert np.max(np.abs(kap - rk)[m] / scale[m]) <= 1e-10
    # the terms do change the result
    rk0, re0, _ = _oracle(p, 0)
    assert np.max(np.abs(re - re0) / np.maximum(re0, 1e-300)) > 1e-6


def test_broadening_fp32_within_tolerance_and_same_windows(ctx):
    p = _problem()
    kap, em, n32 = _gpu(ctx, p, R.FP32, ALL)
    _, _, n64 = _gpu(ctx, p, R.FP64, ALL)
    assert n32 == n64 > 0
    rk, re, ra = _oracle(p, ALL)
    big = re >= 1e-6 * re.max(axis=1, keepdims=True)
    err = (np.abs(em - re) / np.maximum(re, 1e-300))[big]
    print(f"  j: max rel err {err.max():.3e}")
    assert err.max() <= 1e-3
    scale = np.maximum(np.abs(rk), ra)
    bigk = scale >= 1e-6 * scale.max(axis=1, keepdims=True)
    assert np.max((np.abs(kap - rk) / np.maximum(scale, 1e-300))[bigk]) <= 1e-3


def test_broadening_batch_equals_single_call(ctx):
    from paper_2604_11856_gb300 import batch
    ctx.set_broadening(ALL, synth.RAD_E_IONIZE, synth.FLOW_MASS)
    pool = synth._air_lines(np.random.default_rng(1001), 2000, 20000)
    probs = synth.batch_slabs(n_solves=3, pool=pool, scale=0.01)
    chunk = 3000
    bs = batch.BatchSolver(probs, ctx, chunk=chunk)
    q_batch = [q.cpu().numpy().copy() for q in bs.run()]
    ctx.sync()
    for i, p in enumerate(probs):
        dp = solver.DeviceProblem(p, ctx)
        solo = solver.solve(dp, ctx, R.FP32, chunk=chunk)["q"].cpu().numpy()
        ctx.sync()
        np.testing.assert_allclose(q_batch[i], solo, rtol=1e-12, atol=0)
    bs.close()


def test_set_broadening_checks(ctx):
    with pytest.raises(R.RapralError):
        ctx.set_broadening(8)
    with pytest.raises(R.RapralError):
        ctx.set_broadening(R.BROAD_STARK_IONIZE)          # no ionisation energies
    with pytest.raises(R.RapralError):
        ctx.set_broadening(R.BROAD_VDW, synth.RAD_E_IONIZE)   # no column masses
    ctx.set_broadening(0)
