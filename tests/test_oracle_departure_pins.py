"""Pins of the oracle's non-Boltzmann populations (Sec. 2.1: departure
coefficients b = N / N_Boltzmann of collisional-radiative levels entering the
line strengths).  No departure changes nothing; the QSS solution at its
Boltzmann limit gives one departure for every level, which scales j and
kappa alike; j is linear in the upper level's b and kappa is affine in it."""
import numpy as np
import pytest

import oracle
from oracle import qss
from paper_2604_11856_gb300 import synth


@pytest.fixture(autouse=True)
def _reset():
    oracle.set_departures()
    yield
    oracle.set_departures()


def _problem():
    base = synth.stagnation_line(n_cells=4, n_atomic=200, n_molecular=300, n_grid=3001)
    m = synth.cr_model(species="N", n_levels=12)
    lines, lev_u, lev_l = synth.cr_lines(m, "N", base=base.lines)
    p = synth.Problem("cr", base.species, lines, base.cells, base.grid, base.geometry, chunk=0)
    return p, m, lev_u, lev_l


def _coeffs(p, ln_b=None, lev_u=None, lev_l=None):
    if ln_b is not None:
        oracle.set_departures(ln_b, lev_u, lev_l)
    try:
        return oracle.spectral_coeffs(p)
    finally:
        oracle.set_departures()


def test_zero_departures_change_nothing():
    p, m, lu, ll = _problem()
    k0, j0 = _coeffs(p)
    k1, j1 = _coeffs(p, np.zeros((len(p.cells), 8, m["l"])), lu, ll)
    assert np.array_equal(k0, k1) and np.array_equal(j0, j1)


def test_boltzmann_limit_of_qss_scales_cr_lines_uniformly():
    p, m, lu, ll = _problem()
    mm = dict(m)
    mm["A"] = np.zeros_like(m["A"]); mm["ii_C"] = np.zeros_like(m["ii_C"])
    cells = synth.Cells(Ttr=p.cells.Tve.copy(), Tve=p.cells.Tve.copy(), n=p.cells.n)
    p2 = synth.Problem("cr", p.species, p.lines, cells, p.grid, p.geometry, chunk=0)
    lnp = oracle.lnpref(p2)
    s = synth.RAD_SPECIES.index("N")
    n_qss = qss.solve_cells(mm, cells)
    d = qss.departures(mm, cells, lnp, s, n_qss)
    # one value per cell: ln(Z_species / Z_model)
    assert np.max(np.ptp(d, axis=1)) < 1e-10
    ln_b = np.zeros((len(cells.Tve), 8, m["l"])); ln_b[:, s, :] = d
    # only the model's lines: their kappa and j both scale by b
    only = synth.Lines(**{k: getattr(p.lines, k)[lu >= 0] for k in synth.Lines.__dataclass_fields__})
    p3 = synth.Problem("cr", p.species, only, cells, p.grid, p.geometry, chunk=0)
    k0, j0 = _coeffs(p3)
    k1, j1 = _coeffs(p3, ln_b, lu[lu >= 0], ll[lu >= 0])
    b = np.exp(d[:, 0])[:, None]
    big = j0 > 1e-12 * j0.max()
    assert np.max(np.abs(j1[big] / (b * j0)[big] - 1)) < 1e-12
    bigk = np.abs(k0) > 1e-12 * np.abs(k0).max()
    assert np.max(np.abs(k1[bigk] / (b * k0)[bigk] - 1)) < 1e-10


def test_upper_level_departure_linear_in_j_affine_in_kappa():
    p, m, lu, ll = _problem()
    s = synth.RAD_SPECIES.index("N")
    out = []
    for b in (1.0, 2.0, 3.0):
        ln_b = np.zeros((len(p.cells), 8, m["l"]))
        ln_b[:, s, 5] = np.log(b)                      # level 5 only
        out.append(_coeffs(p, ln_b, lu, ll))
    (k1, j1), (k2, j2), (k3, j3) = out
    touched = np.abs(j2 - j1) > 0
    assert touched.any()
    # j: the part from lines with upper level 5 doubles and triples
    dj = j2 - j1
    np.testing.assert_allclose(j3 - j1, 2 * dj, rtol=1e-9, atol=1e-30 * j1.max())
    # kappa: affine in b (lines with level 5 as upper or lower level)
    np.testing.assert_allclose(k3 - k2, k2 - k1, rtol=1e-8, atol=1e-12 * np.abs(k1).max())


def test_lower_level_departure_moves_kappa_only():
    """A line absorbs from its lower level and emits from its upper one
    (Sec. 2.2.1): a departure on the lower level alone leaves j unchanged and
    scales the absorbing part of kappa, so kappa grows with b, affinely."""
    p, m, lu, ll = _problem()
    s = synth.RAD_SPECIES.index("N")
    sel = (ll == 5) & (lu != 5)
    assert sel.sum() >= 1
    only = synth.Lines(**{k: getattr(p.lines, k)[sel] for k in synth.Lines.__dataclass_fields__})
    p2 = synth.Problem("cr", p.species, only, p.cells, p.grid, p.geometry, chunk=0)
    out = []
    for b in (1.0, 2.0, 3.0):
        ln_b = np.zeros((len(p.cells), 8, m["l"]))
        ln_b[:, s, 5] = np.log(b)
        out.append(_coeffs(p2, ln_b, lu[sel], ll[sel]))
    (k1, j1), (k2, j2), (k3, j3) = out
    assert np.array_equal(j1, j2) and np.array_equal(j1, j3)
    assert np.all(k2 >= k1) and (k2 > k1).any()
    np.testing.assert_allclose(k3 - k2, k2 - k1, rtol=1e-8, atol=1e-12 * np.abs(k1).max())
