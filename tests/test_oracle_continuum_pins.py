"""Pins of the oracle's atomic continuum (Sec. 2.2.1 bound-free and
free-free): Kirchhoff's law at LTE with the ions at a textbook Saha
equilibrium, the free-free Saha ratio against the same textbook form, the
cross-section tables at and between their nodes and past the edge, the
Table 3 fit against Kramers' hydrogenic free-free, bilinear D, and zero
ions.  None of them retypes the oracle's formulas."""
import os

import numpy as np
import pytest

import oracle
from oracle import continuum as ct
from paper_2604_11856_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table3_ff_fit.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            out[f[0]] = np.array([float(x) for x in f[1:]])
    return out


def test_table3_coefficients_are_the_printed_ones():
    g = _golden()
    for a in ("N", "O"):
        assert np.array_equal(synth.FF_FIT[a], g[a])
        assert np.array_equal(synth.continuum_model(species=a, n_levels=3)["ff_c"], g[a])


def _saha_textbook_si(Qp, Qa, E_ion_cm, T):
    """N_+ N_e / N_a in cm^-3 from the SI Saha equation (thermal de Broglie
    wavelength form), written independently of the oracle's cgs factors."""
    h, k, me, c = 6.626e-34, 1.380e-23, 9.109e-31, 2.998e8
    lam_th = h / np.sqrt(2 * np.pi * me * k * T)           # m
    chi = h * c * E_ion_cm * 100.0                          # J
    return 2.0 * Qp / Qa / lam_th ** 3 * np.exp(-chi / (k * T)) * 1e-6


def _lte_problem(T, species="N"):
    base = synth.stagnation_line(n_cells=3, n_atomic=50, n_molecular=50, n_grid=4001)
    s = synth.RAD_SPECIES.index(species)
    m = synth.continuum_model(species=species, n_levels=30)
    n = base.cells.n.copy()
    cells = synth.Cells(Ttr=np.full(3, T), Tve=np.full(3, T), n=n)
    p = synth.Problem("lte", base.species, base.lines, cells, base.grid, base.geometry, chunk=0)
    Qa = oracle.partition(p, s, T, T)
    R = _saha_textbook_si(ct.ion_Q(m, T), Qa, m["E_ion"], T)
    n[:, m["ion_col"]] = n[:, m["atom_col"]] * R / n[:, synth.NE_COL]
    return p, m, s


@pytest.mark.parametrize("T,species", [(6000.0, "N"), (11000.0, "N"), (9000.0, "O")])
def test_kirchhoff_at_lte_with_textbook_saha(T, species):
    p, m, s = _lte_problem(T, species)
    lnp = oracle.lnpref(p)
    kap, em = ct.continuum([m], p.cells, lnp, p.grid)
    h = (p.grid.lam_max - p.grid.lam_min) / (p.grid.n - 1)
    lam = p.grid.lam_min + np.arange(p.grid.n) * h
    B = ct.planck(lam, T)
    big = kap > 1e-30 * kap.max()
    assert np.max(np.abs(em[:, big[0]] / (B * kap)[:, big[0]] - 1)) < 1e-11
    # the free-free Saha ratio equals the textbook one: kappa_ff = N_+ N_e sigma^H (1 + D)
    ff_only = dict(m, node_sigma=np.zeros_like(m["node_sigma"]))
    kff, _ = ct.continuum([ff_only], p.cells, lnp, p.grid)
    n = p.cells.n
    ref = (n[:, m["ion_col"]] * n[:, synth.NE_COL])[:, None] * ct.sigma_ff_H(m, lam, T) * \
        (1.0 + ct.D_value(m, ct.LAM_H / lam, T))[None, :]
    assert np.allclose(kff, ref, rtol=1e-11, atol=0)


def test_tables_at_and_between_nodes_and_past_the_edge():
    base = synth.stagnation_line(n_cells=2, n_atomic=50, n_molecular=50, n_grid=1001)
    g = base.grid
    h = (g.lam_max - g.lam_min) / (g.n - 1)
    lam = g.lam_min + np.arange(g.n) * h
    nodes = lam[[100, 300, 301, 600]]
    vals = np.array([2e-18, 5e-18, 1e-18, 3e-18])
    E1, g1, E_ion = 80000.0, 6.0, 117225.7
    m = dict(species=0, atom_col=3, ion_col=8, E_ion=E_ion, E=np.array([E1]), g=np.array([g1]),
             node_off=np.array([0, 4]), node_lam=nodes, node_sigma=vals, ion_E=np.array([0.0]),
             ion_g=np.array([9.0]), ff_c=np.zeros(8), D_sigma=np.array([0.1, 1.0]), D_T=np.array([1e3, 1e4]),
             D=np.zeros((2, 2)))
    lnp = oracle.lnpref(base)
    kap, _ = ct.continuum([m], base.cells, lnp, g)
    for c in range(2):
        T = base.cells.Tve[c]
        N1 = np.exp(oracle.lib().orc_ln_level_pop(lnp[c, 0], g1, E1, 0.0, 0.0, T, T))
        assert np.allclose(kap[c, [100, 300, 301, 600]], N1 * vals, rtol=1e-13, atol=0)
        assert np.isclose(kap[c, 200], N1 * 0.5 * (vals[0] + vals[1]), rtol=1e-12)
        assert np.all(kap[c, :100] == 0) and np.all(kap[c, 601:] == 0)     # outside the table


@pytest.mark.parametrize("species", ["N", "O"])
def test_table3_fit_against_kramers(species):
    """Kramers' hydrogenic free-free absorption per N_+ N_e (no stimulated
    emission) times a Gaunt factor of 0.8-1.35 brackets the fit over
    100-2000 nm and 5000-20000 K."""
    e, me, h, k, c = 4.803e-10, 9.109e-28, 6.626e-27, 1.380e-16, 2.998e10
    m = synth.continuum_model(species=species, n_levels=2)
    for T in (5000.0, 10000.0, 20000.0):
        lam = np.array([100.0, 300.0, 1000.0, 2000.0])
        nu = c / (lam * 1e-7)
        kr = 4 * e ** 6 / (3 * me * h * c) * np.sqrt(2 * np.pi / (3 * k * me)) / np.sqrt(T) / nu ** 3
        ratio = ct.sigma_ff_H(m, lam, T) / kr
        assert np.all((ratio > 0.8) & (ratio < 1.35)), ratio


def test_D_is_bilinear_and_clamped():
    m = synth.continuum_model(species="N", n_levels=2)
    xs, ts = m["D_sigma"], m["D_T"]
    f = lambda s, T: 0.03 + 0.1 * s - 2e-6 * T + 3e-6 * s * T
    m["D"] = f(xs[None, :], ts[:, None])
    rng = np.random.default_rng(2)
    for s, T in zip(rng.uniform(xs[0], xs[-1], 20), rng.uniform(ts[0], ts[-1], 20)):
        assert abs(ct.D_value(m, s, T) - f(s, T)) < 1e-14
    assert abs(ct.D_value(m, 10.0, 1e5) - f(xs[-1], ts[-1])) < 1e-14
    assert abs(ct.D_value(m, 1e-4, 10.0) - f(xs[0], ts[0])) < 1e-14


def test_zero_ions_leave_only_free_free_emission():
    p, m, s = _lte_problem(9000.0)
    lnp = oracle.lnpref(p)
    k1, _ = ct.continuum([m], p.cells, lnp, p.grid)
    p.cells.n[:, m["ion_col"]] = 0.0
    k0, j0 = ct.continuum([m], p.cells, lnp, p.grid)
    assert np.array_equal(k0, k1)                       # absorption does not see the ions
    ff_only = dict(m, node_sigma=np.zeros_like(m["node_sigma"]))
    kff, jff = ct.continuum([ff_only], p.cells, lnp, p.grid)
    assert np.allclose(j0, jff, rtol=1e-14, atol=0)


def test_planck_equals_the_wall_planck_and_integrates_to_sigma_T4():
    lam = np.geomspace(60.0, 1e6, 200001)
    for T in (3000.0, 12000.0):
        for l in (80.0, 500.0, 1900.0):
            assert abs(ct.planck(l, T) / oracle.lib().orc_planck(l, T) - 1) < 1e-14
        # integral over wavelength (W/cm^2/sr/um * um) -> sigma T^4 / pi (W/cm^2/sr)
        B = ct.planck(lam, T)
        tot = np.trapezoid(B, lam * 1e-3)
        sig = 2 * np.pi ** 5 * (1.380e-23) ** 4 / (15 * (6.626e-34) ** 3 * (2.998e8) ** 2) * 1e-4   # W/cm^2/K^4
        assert abs(tot / (sig * T ** 4 / np.pi) - 1) < 2e-3


@pytest.mark.parametrize("T,species", [(7000.0, "N"), (12000.0, "O")])
def test_saha_boltzmann_equals_boltzmann_at_saha_equilibrium(T, species):
    """With the ions at the textbook Saha equilibrium of the atom, the
    Saha-Boltzmann prefactor is the Boltzmann one, ln(N_a / Q_a)."""
    p, m, s = _lte_problem(T, species)
    lnp = oracle.lnpref(p)
    sb = ct.saha_lnpref(p.cells, m["ion_col"], m["E_ion"], m["ion_E"], m["ion_g"])
    assert np.max(np.abs(sb - lnp[:, s])) < 1e-11
    # twice the ions: twice the populations
    p.cells.n[:, m["ion_col"]] *= 2.0
    sb2 = ct.saha_lnpref(p.cells, m["ion_col"], m["E_ion"], m["ion_E"], m["ion_g"])
    assert np.allclose(sb2 - sb, np.log(2.0), atol=1e-13)
    p.cells.n[0, m["ion_col"]] = 0.0
    assert ct.saha_lnpref(p.cells, m["ion_col"], m["E_ion"], m["ion_E"], m["ion_g"])[0] == -np.inf
