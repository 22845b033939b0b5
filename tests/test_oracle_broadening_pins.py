"""Pins of the oracle's optional Lorentz terms (Sec. 2.2.1 full broadening:
Stark coefficient from the ionisation gap, resonance and van der Waals
widths).  A literature value fixes the oscillator strength; scaling laws
and limits fix the rest; the wiring into the line widths is checked against
the separate terms."""
import numpy as np
import pytest

import oracle
from paper_2604_11856_gb300 import synth


@pytest.fixture(autouse=True)
def _reset():
    oracle.set_broadening(0)
    yield
    oracle.set_broadening(0)
    oracle.lib().orc_set_codata(0)


def test_oscillator_strength_of_lyman_alpha():
    """H Lyman alpha (1s - 2p, 121.567 nm, A = 6.2649e8 s^-1, g_u = 6,
    g_l = 2) has f_lu = 0.41641 (NIST)."""
    assert abs(oracle.oscillator_strength(121.567, 6.2649e8, 6, 2) / 0.41641 - 1) < 6e-4   # printed 4-digit constants
    oracle.lib().orc_set_codata(1)
    assert abs(oracle.oscillator_strength(121.567, 6.2649e8, 6, 2) / 0.41641 - 1) < 1e-4


def test_stark_coefficient_from_ionisation_gap():
    Eion = 117225.7
    floor = 109678.77 / 25.0
    a = oracle.stark_coeff_ionize(500.0, 90000.0, Eion)
    assert abs(oracle.stark_coeff_ionize(1000.0, 90000.0, Eion) / a - 4.0) < 1e-13          # lam^2
    # gap halved -> coefficient x 2^2.623
    b = oracle.stark_coeff_ionize(500.0, Eion - (Eion - 90000.0) / 2, Eion)
    assert abs(b / a - 2 ** 2.623) < 1e-12
    # at and above E_ionize - E_H/25 the gap is held at E_H/25: continuous and constant
    top = oracle.stark_coeff_ionize(500.0, Eion + 5000.0, Eion)
    assert oracle.stark_coeff_ionize(500.0, Eion - floor + 1e-6, Eion) == top
    assert abs(oracle.stark_coeff_ionize(500.0, Eion - floor, Eion) / top - 1) < 1e-12
    assert abs(oracle.stark_coeff_ionize(500.0, Eion - floor - 1e-3, Eion) / top - 1) < 1e-6
    assert abs(top - 1.69e3 * 500.0 ** 2 / floor ** 2.623) < 1e-14 * top


def test_van_der_waals_scalings():
    w = oracle.vdw_hwhm(500.0, 8000.0, 1e16, 14.0, 0.0, 1.0)
    assert abs(oracle.vdw_hwhm(1000.0, 8000.0, 1e16, 14.0, 0.0, 1.0) / w - 4.0) < 1e-13     # lam^2
    assert abs(oracle.vdw_hwhm(500.0, 32000.0, 1e16, 14.0, 0.0, 1.0) / w - 2.0) < 1e-13     # T^0.5
    assert abs(oracle.vdw_hwhm(500.0, 8000.0, 3e16, 14.0, 0.0, 1.0) / w - 3.0) < 1e-13      # N
    assert abs(oracle.vdw_hwhm(500.0, 8000.0, 1e16, 56.0, 0.0, 1.0) / w - 0.5) < 1e-13      # M^-0.5
    # the other particles add their own term, with the printed coefficient ratio
    o = oracle.vdw_hwhm(500.0, 8000.0, 0.0, 14.0, 1e16, 14.0)
    assert abs(o / w - 2.925 / 6.65) < 1e-13
    assert abs(oracle.vdw_hwhm(500.0, 8000.0, 1e16, 14.0, 1e16, 14.0) / (w + o) - 1) < 1e-13


def test_resonance_width_scalings():
    r = oracle.resonance_hwhm(120.0, 1e8, 6, 2, 1e15)
    assert abs(oracle.resonance_hwhm(120.0, 1e8, 6, 2, 2e15) / r - 2.0) < 1e-13             # N_0
    assert abs(oracle.resonance_hwhm(240.0, 1e8, 6, 2, 1e15) / r - 32.0) < 1e-12            # lam f lam^2, f ~ lam^2
    assert abs(oracle.resonance_hwhm(120.0, 2e8, 6, 2, 1e15) / r - 2.0) < 1e-13             # A
    # g_u / g_l enters f, (g_l / g_u)^0.5 the width: net (g_u / g_l)^0.5
    assert abs(oracle.resonance_hwhm(120.0, 1e8, 8, 2, 1e15) / r - np.sqrt(4.0 / 3.0)) < 1e-13


def _states(p, flags):
    oracle.set_broadening(flags, synth.RAD_E_IONIZE, synth.FLOW_MASS)
    lnp = oracle.lnpref(p)
    out = [oracle.line_states(p, lnp, c) for c in range(len(p.cells))]
    oracle.set_broadening(0)
    return lnp, out


def test_terms_enter_the_lorentz_width_of_atomic_lines_only():
    p = synth.stagnation_line(n_cells=3, n_atomic=400, n_molecular=400, n_grid=1001)
    ln, sp = p.lines, p.species
    lnp, base = _states(p, 0)
    atom = sp.kind[ln.species] == 0
    reso = atom & (ln.El_el == 0) & (ln.El_v == 0) & (ln.El_j == 0)
    assert reso.any() and (atom & ~reso).any()
    for flags in (1, 2, 4, 7):
        _, st = _states(p, flags)
        for c in range(len(p.cells)):
            lamL0, lamL = base[c]["lamL"], st[c]["lamL"]
            assert np.array_equal(lamL[~atom], lamL0[~atom])               # molecules untouched
            extra = np.zeros(len(ln))
            ne = p.cells.n[c, synth.NE_COL]
            stc = (p.cells.Tve[c] / 1e4) ** 0.33 * (ne / 1e16)
            if flags & 1:
                s0 = np.array([oracle.stark_coeff_ionize(ln.lam0[l], ln.Eu_el[l], synth.RAD_E_IONIZE[ln.species[l]])
                               for l in range(len(ln))])
                extra[atom] += (s0[atom] - ln.lamS0[atom]) * stc
            if flags & 2:
                for l in np.nonzero(reso)[0]:
                    s = ln.species[l]
                    g0 = synth.ATOM_GROUND_G[synth.RAD_SPECIES[s]]
                    N0 = np.exp(lnp[c, s] + np.log(g0))
                    extra[l] += oracle.resonance_hwhm(ln.lam0[l], ln.A[l], ln.gu[l], ln.gl[l], N0)
            if flags & 4:
                for l in np.nonzero(atom)[0]:
                    s = ln.species[l]
                    col = synth.RAD_DENSITY_COL[s]
                    others = [k for k in range(11) if k != col and synth.FLOW_MASS[k] > 0]
                    No = p.cells.n[c, others].sum()
                    Mo = (p.cells.n[c, others] * synth.FLOW_MASS[others]).sum() / No
                    extra[l] += oracle.vdw_hwhm(ln.lam0[l], p.cells.Ttr[c], p.cells.n[c, col], sp.mass[s], No, Mo)
            np.testing.assert_allclose(lamL[atom], lamL0[atom] + extra[atom], rtol=1e-10)
