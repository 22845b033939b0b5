"""The exact Voigt line shape on the GPU (rapral_set_profile, the optional
profile of Sec. 2.2.1's full broadening) against the oracle of
oracle/voigt.py: FP64 to 1e-10 relative, FP32 to the FP32 tolerance, alone
and with the optional Lorentz terms; the windows are Whiting's."""
import numpy as np
import pytest
import torch

import oracle
from oracle import voigt
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu

ALL = R.BROAD_STARK_IONIZE | R.BROAD_RESONANCE | R.BROAD_VDW


@pytest.fixture()
def ctx():
    c = R.Context(0)
    yield c
    c.set_profile(R.PROFILE_WHITING)
    c.set_broadening(0)


def _problem():
    return synth.stagnation_line(n_cells=8, n_atomic=1500, n_molecular=6000, n_grid=40001)


def _gpu(ctx, p, precision, flags=0, tile=0):
    ctx.set_profile(R.PROFILE_VOIGT)
    ctx.set_broadening(flags, synth.RAD_E_IONIZE, synth.FLOW_MASS)
    if tile:
        ctx.set_tiling(tile_width=tile)
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    dt = torch.float64 if precision == R.FP64 else torch.float32
    kap = torch.empty((dp.C, p.grid.n), dtype=dt, device=ctx.device)
    em = torch.empty_like(kap)
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, p.grid.n, precision, kap, em)
    ctx.sync()
    return kap.double().cpu().numpy(), em.double().cpu().numpy()


def _oracle(p, flags=0):
    oracle.set_broadening(flags, synth.RAD_E_IONIZE, synth.FLOW_MASS)
    try:
        return voigt.spectral_coeffs(p, with_abs=True)
    finally:
        oracle.set_broadening(0)


@pytest.mark.parametrize("flags,tile", [(0, 0), (ALL, 256)])
def test_voigt_fp64_matches_oracle(ctx, flags, tile):
    p = _problem()
    kap, em = _gpu(ctx, p, R.FP64, flags, tile)
    rk, re, ra = _oracle(p, flags)
    ej = np.max(np.abs(em - re) / np.maximum(np.abs(re), 1e-300))
    scale = np.maximum(np.abs(rk), ra)
    m = scale > 0
    ek = np.max(np.abs(kap - rk)[m] / scale[m])
    print(f"  j {ej:.3e}  kappa {ek:.3e}")
    assert ej <= 1e-10 and ek <= 1e-10
    wk, wj = oracle.spectral_coeffs(p)
    assert np.max(np.abs(re - wj) / np.maximum(wj, 1e-300)) > 1e-3          # the shape does change j


@pytest.mark.parametrize("flags", [0, ALL])
def test_voigt_fp32_within_tolerance(ctx, flags):
    p = _problem()
    kap, em = _gpu(ctx, p, R.FP32, flags)
    rk, re, ra = _oracle(p, flags)
    big = re >= 1e-6 * re.max(axis=1, keepdims=True)
    err = (np.abs(em - re) / np.maximum(re, 1e-300))[big]
    print(f"  j: max rel err {err.max():.3e} (p99 {np.quantile(err, 0.99):.3e})")
    assert err.max() <= 1e-3
    scale = np.maximum(np.abs(rk), ra)
    bigk = scale >= 1e-6 * scale.max(axis=1, keepdims=True)
    assert np.max((np.abs(kap - rk) / np.maximum(scale, 1e-300))[bigk]) <= 1e-3


def test_profile_checks(ctx):
    with pytest.raises(R.RapralError):
        ctx.set_profile(7)
