"""Non-Boltzmann populations on the GPU (Sec. 2.1): QSS populations turned
into departure coefficients (rapral_qss_departures) and fed to the line sum
(rapral_set_departures), against the oracle's departures and line strengths:
ln b to 1e-12 absolute, coefficients FP64 to 1e-10 relative, FP32 to the
FP32 tolerance."""
import numpy as np
import pytest
import torch

import oracle
from oracle import qss
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu

SPECIES = "N"


@pytest.fixture()
def ctx():
    c = R.Context(0)
    yield c
    c.set_departures()


def _problem(n_cells=24):
    base = synth.stagnation_line(n_cells=n_cells, n_atomic=3000, n_molecular=20000, n_grid=60001)
    m = synth.cr_model(species=SPECIES, n_levels=16, n_lumped=3)
    lines, lev_u, lev_l = synth.cr_lines(m, SPECIES, base=base.lines)
    p = synth.Problem("cr", base.species, lines, base.cells, base.grid, base.geometry, chunk=0)
    return p, m, lev_u.astype(np.int32), lev_l.astype(np.int32)


def _gpu_departures(ctx, p, m, dp, n_lev):
    dm = R.DeviceCrModel(m, ctx.device)
    nq = torch.empty((dp.C, dm.l), dtype=torch.float64, device=ctx.device)
    R.qss_populations(ctx, dm, dp.cells, nq)
    ln_b = torch.zeros((dp.C, dp.species.S, n_lev), dtype=torch.float64, device=ctx.device)
    R.qss_departures(ctx, dm, dp.cells, synth.RAD_SPECIES.index(SPECIES), nq, ln_b)
    return ln_b


def _oracle_departures(p, m, n_lev, S):
    lnp = oracle.lnpref(p)
    s = synth.RAD_SPECIES.index(SPECIES)
    n_qss = qss.solve_cells(m, p.cells, ion_col=m["ion_col"])
    ln_b = np.zeros((len(p.cells.Tve), S, n_lev))
    ln_b[:, s, :] = qss.departures(m, p.cells, lnp, s, n_qss, n_lev)
    return ln_b


def _gpu(ctx, p, precision, m, lu, ll, n_lev):
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    ln_b = _gpu_departures(ctx, p, m, dp, n_lev)
    ctx.set_departures(ln_b, torch.from_numpy(lu).to(ctx.device), torch.from_numpy(ll).to(ctx.device))
    dt = torch.float64 if precision == R.FP64 else torch.float32
    kap = torch.empty((dp.C, p.grid.n), dtype=dt, device=ctx.device)
    em = torch.empty_like(kap)
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, p.grid.n, precision, kap, em)
    ctx.sync()
    ctx.set_departures()
    return kap.double().cpu().numpy(), em.double().cpu().numpy(), ln_b.cpu().numpy()


def _oracle(p, ln_b, lu, ll):
    oracle.set_departures(ln_b, lu, ll)
    try:
        return oracle.spectral_coeffs(p, with_abs=True)
    finally:
        oracle.set_departures()


def test_departures_match_oracle():
    p, m, lu, ll = _problem(12)
    c = R.Context(0)
    dp = solver.DeviceProblem(p, c)
    R.populations(c, dp.species, dp.cells)
    got = _gpu_departures(c, p, m, dp, 20).cpu().numpy()
    c.sync()
    ref = _oracle_departures(p, m, 20, dp.species.S)
    print(f"  ln b: max abs err {np.max(np.abs(got - ref)):.3e}, range {ref.min():.2f} .. {ref.max():.2f}")
    assert np.max(np.abs(got - ref)) <= 1e-12
    assert np.ptp(ref) > 1.0                     # the populations do depart from Boltzmann


def test_coefficients_with_departures_fp64(ctx):
    p, m, lu, ll = _problem()
    kap, em, ln_b = _gpu(ctx, p, R.FP64, m, lu, ll, 20)
    rk, re, ra = _oracle(p, _oracle_departures(p, m, 20, ln_b.shape[1]), lu, ll)
    den = np.maximum(np.abs(re), 1e-300)
    err = np.max(np.abs(em - re) / den)
    scale = np.maximum(np.abs(rk), ra)
    mk = scale > 0
    errk = np.max(np.abs(kap - rk)[mk] / scale[mk])
    print(f"  j: {err:.3e}  kappa: {errk:.3e}")
    assert err <= 1e-10 and errk <= 1e-10
    rk0, re0, _ = oracle.spectral_coeffs(p, with_abs=True)
    assert np.max(np.abs(re - re0) / np.maximum(re0, 1e-300)) > 1e-3     # the departures do change j


def test_coefficients_with_departures_fp32(ctx):
    p, m, lu, ll = _problem()
    kap, em, ln_b = _gpu(ctx, p, R.FP32, m, lu, ll, 20)
    rk, re, ra = _oracle(p, _oracle_departures(p, m, 20, ln_b.shape[1]), lu, ll)
    big = re >= 1e-6 * re.max(axis=1, keepdims=True)
    err = (np.abs(em - re) / np.maximum(re, 1e-300))[big]
    print(f"  j: max rel err {err.max():.3e}")
    assert err.max() <= 1e-3
    scale = np.maximum(np.abs(rk), ra)
    bigk = scale >= 1e-6 * scale.max(axis=1, keepdims=True)
    assert np.max((np.abs(kap - rk) / np.maximum(scale, 1e-300))[bigk]) <= 1e-3


def test_zero_table_is_boltzmann(ctx):
    p, m, lu, ll = _problem(6)
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    out = []
    for dep in (False, True):
        if dep:
            z = torch.zeros((dp.C, dp.species.S, 16), dtype=torch.float64, device=ctx.device)
            ctx.set_departures(z, torch.from_numpy(lu).to(ctx.device), torch.from_numpy(ll).to(ctx.device))
        kap = torch.empty((dp.C, p.grid.n), dtype=torch.float64, device=ctx.device)
        em = torch.empty_like(kap)
        R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, p.grid.n, R.FP64, kap, em)
        ctx.sync()
        out.append((kap.cpu().numpy(), em.cpu().numpy()))
    ctx.set_departures()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_departure_checks(ctx):
    p, m, lu, ll = _problem(4)
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    kap = torch.empty((dp.C, p.grid.n), dtype=torch.float64, device=ctx.device)
    em = torch.empty_like(kap)
    u = torch.from_numpy(lu).to(ctx.device)
    lo = torch.from_numpy(ll).to(ctx.device)
    # a table of another cell count
    ctx.set_departures(torch.zeros((dp.C + 1, dp.species.S, 16), dtype=torch.float64, device=ctx.device), u, lo)
    with pytest.raises(R.RapralError):
        R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, p.grid.n, R.FP64, kap, em)
    # a level index past the table: caught on the device, nothing read
    ctx.set_departures(torch.zeros((dp.C, dp.species.S, 4), dtype=torch.float64, device=ctx.device), u, lo)
    with pytest.raises(R.RapralError):
        R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, p.grid.n, R.FP64, kap, em)
        ctx.sync()
    ctx.clear_status()
    ctx.set_departures()
    ctx.sync()


@pytest.mark.parametrize("precision", [R.FP64, R.FP32])
@pytest.mark.parametrize("voigt_shape", [False, True])
def test_departures_with_broadening_and_line_shape(ctx, precision, voigt_shape):
    """Departures together with the optional Lorentz terms, with Whiting's
    shape and with the exact Voigt shape (every combination of the line
    sums' optional flags)."""
    from oracle import voigt
    ALL = R.BROAD_STARK_IONIZE | R.BROAD_RESONANCE | R.BROAD_VDW
    p, m, lu, ll = _problem(6)
    ctx.set_broadening(ALL, synth.RAD_E_IONIZE, synth.FLOW_MASS)
    ctx.set_profile(R.PROFILE_VOIGT if voigt_shape else R.PROFILE_WHITING)
    try:
        kap, em, ln_b = _gpu(ctx, p, precision, m, lu, ll, 20)
    finally:
        ctx.set_broadening(0)
        ctx.set_profile(R.PROFILE_WHITING)
    oracle.set_broadening(ALL, synth.RAD_E_IONIZE, synth.FLOW_MASS)
    oracle.set_departures(_oracle_departures(p, m, 20, ln_b.shape[1]), lu, ll)
    try:
        rk, re, ra = (voigt.spectral_coeffs(p, with_abs=True) if voigt_shape
                      else oracle.spectral_coeffs(p, with_abs=True))
    finally:
        oracle.set_departures()
        oracle.set_broadening(0)
    scale = np.maximum(np.abs(rk), ra)
    if precision == R.FP64:
        assert np.max(np.abs(em - re) / np.maximum(np.abs(re), 1e-300)) <= 1e-10
        m_ = scale > 0
        assert np.max(np.abs(kap - rk)[m_] / scale[m_]) <= 1e-10
    else:
        big = re >= 1e-6 * re.max(axis=1, keepdims=True)
        assert np.max((np.abs(em - re) / np.maximum(re, 1e-300))[big]) <= 1e-3
        bigk = scale >= 1e-6 * scale.max(axis=1, keepdims=True)
        assert np.max((np.abs(kap - rk) / np.maximum(scale, 1e-300))[bigk]) <= 1e-3
