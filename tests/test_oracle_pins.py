"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/paper_constants.json), closed forms, physical
laws, arbitrary-precision evaluation, an ODE integrator, the exact Voigt
profile, or brute force on tiny inputs.  Each is chosen so that a plausible
mistake (a dropped term, a swapped coefficient, a wrong temperature or
index) fails it.

Parity unpinned: the Whiting shape between the Gaussian and Lorentzian
limits is an empirical fit; it is held only to its measured distance from
the exact Voigt profile (test_whiting_vs_exact_voigt).
"""
import json
import math
import os

import mpmath
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq
from scipy.special import expn, voigt_profile

import oracle
from paper_2604_11856_gb300 import synth

G = {k: v["value"] for k, v in json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                                           "paper_constants.json"))).items()
     if not k.startswith("_")}
L = oracle.lib()


# ------------------------------------------------------------------ constants

def test_constants_as_printed():
    assert L.orc_const(0) == G["k_cgs"] and L.orc_const(1) == G["c_cgs"] and L.orc_const(2) == G["h_cgs"]
    assert L.orc_c2() == pytest.approx(G["h_cgs"] * G["c_cgs"] / G["k_cgs"], rel=1e-15)
    # the printed constants are within their 4-digit rounding of CODATA
    assert G["h_cgs"] * G["c_cgs"] / G["k_cgs"] == pytest.approx(1.438776877, rel=2e-3)


def test_doppler_constant_from_kinetic_theory():
    # HWHM of a Maxwellian line: lam * sqrt(2 ln2 k T / (m c^2)), SI, m = M * amu
    k, amu, c = 1.380649e-23, 1.66053906660e-27, 2.99792458e8
    coef = math.sqrt(2 * math.log(2) * k / (amu * c * c))
    assert G["doppler_coefficient"] / 2 == pytest.approx(coef, rel=2e-4)
    lam0, T, M = 500.0, 12000.0, 14.0
    assert L.orc_doppler_hwhm(lam0, T, M) == pytest.approx(coef * lam0 * math.sqrt(T / M), rel=2e-4)
    # scales as sqrt(T / M) and linearly in lam0
    assert L.orc_doppler_hwhm(2 * lam0, 4 * T, M) == pytest.approx(4 * L.orc_doppler_hwhm(lam0, T, M), rel=1e-14)


def test_stark_reference_point_and_scaling():
    lamS0 = 0.0123
    assert L.orc_stark_hwhm(lamS0, G["stark_T_ref"], G["stark_ne_ref"]) == pytest.approx(lamS0, rel=1e-15)
    assert L.orc_stark_hwhm(lamS0, 2e4, 1e16) == pytest.approx(lamS0 * 2 ** G["stark_T_exponent"], rel=1e-14)
    assert L.orc_stark_hwhm(lamS0, 1e4, 3e16) == pytest.approx(3 * lamS0, rel=1e-14)
    # Lorentz width = natural + Stark
    assert L.orc_lorentz_hwhm(0.0) == G["natural_hwhm_nm"]


# ------------------------------------------------------------- Voigt widths

def test_voigt_hwhm_limits():
    # d = +1: pure Lorentz; d = -1: pure Gauss; d = 0: equal widths
    assert L.orc_voigt_hwhm(0.37, 0.0) == pytest.approx(0.37, rel=1e-14)
    assert L.orc_voigt_hwhm(0.0, 0.21) == pytest.approx(0.21, rel=1e-14)
    assert L.orc_voigt_hwhm(0.5, 0.5) == pytest.approx((1 - G["voigt_hwhm_c1"]) * 1.0, rel=1e-14)


def _exact_voigt_hwhm(lamL, lamG):
    sigma = lamG / math.sqrt(2 * math.log(2))
    f0 = voigt_profile(0.0, sigma, lamL)
    return brentq(lambda x: voigt_profile(x, sigma, lamL) - f0 / 2, 0.0, 10 * (lamL + lamG), xtol=1e-15)


def test_voigt_hwhm_vs_exact_voigt():
    # the printed fit reproduces the exact Voigt half width to ~1e-4 for every
    # mix; a wrong sign or coefficient in any of its three terms is >= 1e-3 off
    worst = 0.0
    for d in np.linspace(-0.995, 0.995, 81):
        lamL, lamG = (1 + d) / 2, (1 - d) / 2
        worst = max(worst, abs(L.orc_voigt_hwhm(lamL, lamG) / _exact_voigt_hwhm(lamL, lamG) - 1))
    assert worst < 2e-4


# -------------------------------------------------------------- line shape

def _phi(dlam, lamL, lamV):
    return np.array([L.orc_whiting_phi(float(x), lamL, lamV) for x in np.atleast_1d(dlam)])


def test_whiting_peak():
    for lamL, lamG in [(0.0, 0.3), (0.3, 0.0), (0.1, 0.2), (0.25, 0.05)]:
        lamV = L.orc_voigt_hwhm(lamL, lamG)
        r = lamL / lamV
        a, b, c = G["whiting_norm"]
        assert _phi(0.0, lamL, lamV)[0] == pytest.approx(1e3 / (2 * lamV * (a + b * r + c * r * r)), rel=1e-14)


def _simpson_area(f, W, n=200_001):
    x = np.linspace(-W, W, n)
    y = np.array([f(abs(v)) for v in x])
    h = x[1] - x[0]
    return h / 3 * (y[0] + y[-1] + 4 * y[1:-1:2].sum() + 2 * y[2:-1:2].sum())


def test_whiting_area_gauss_and_lorentz_limits():
    lamV = 0.02
    # r = 0: 1e3 / (2 lamV 1.065) * int exp(-2.772 (x/2lamV)^2) dx, x in nm -> um (1e-3)
    area0 = _simpson_area(lambda x: L.orc_whiting_phi(x, 0.0, lamV), 12 * lamV) * 1e-3
    assert area0 == pytest.approx(math.sqrt(math.pi / G["whiting_gauss"]) / G["whiting_norm"][0], rel=1e-9)
    # r = 1, cut at |x| <= 100 lamV: atan(100) / (1.065 + 0.447 + 0.058)
    area1 = _simpson_area(lambda x: L.orc_whiting_phi(x, lamV, lamV), 100 * lamV, n=2_000_001) * 1e-3
    assert area1 == pytest.approx(math.atan(100.0) / sum(G["whiting_norm"]), rel=1e-9)


@pytest.mark.parametrize("r_target,bound", [(0.1, 0.13), (0.3, 0.10), (0.5, 0.075), (0.7, 0.045), (0.9, 0.016)])
def test_whiting_vs_exact_voigt(r_target, bound):
    """Pointwise over |u| <= 50 the fit stays within `bound` of the exact
    Voigt profile (measured deviation + ~20%); dropping the 0.016 correction
    term or flipping its sign leaves 2-8x that."""
    d = brentq(lambda d: (1 + d) / 2 / L.orc_voigt_hwhm((1 + d) / 2, (1 - d) / 2) - r_target, -0.9999, 0.9999)
    lamL, lamG = (1 + d) / 2, (1 - d) / 2
    lamV = L.orc_voigt_hwhm(lamL, lamG)
    x = np.linspace(0, 100 * lamV, 2001)
    exact = voigt_profile(x, lamG / math.sqrt(2 * math.log(2)), lamL) * 1e3
    assert np.max(np.abs(_phi(x, lamL, lamV) / exact - 1)) < bound


# ----------------------------------------------------------- Planck function

def test_planck_stefan_boltzmann():
    # int B dlam (um) = sigma T^4 / pi with sigma in W/cm^2/K^4; printed constants are 4-digit
    T = 8000.0
    lam = np.linspace(20.0, 2e5, 2_000_001)   # nm
    B = np.array([L.orc_planck(float(x), T) for x in lam[::10]])
    integral = np.trapezoid(B, lam[::10] * 1e-3)
    sigma = 2 * math.pi ** 5 * G["k_cgs"] ** 4 / (15 * G["h_cgs"] ** 3 * G["c_cgs"] ** 2) * 1e-7  # W/cm^2/K^4
    assert integral == pytest.approx(sigma * T ** 4 / math.pi, rel=1e-4)
    # Wien limit at short wavelength
    lam0 = 100.0
    x = G["h_cgs"] * G["c_cgs"] / (lam0 * 1e-7 * G["k_cgs"] * 3000.0)
    wien = 1e-7 * 2 * G["h_cgs"] * G["c_cgs"] ** 2 / (1e4 * (lam0 * 1e-7) ** 5) * math.exp(-x)
    assert L.orc_planck(lam0, 3000.0) == pytest.approx(wien, rel=1e-12)


# -------------------------------------------------------------- populations

def _species(atom_levels=None, mol=None):
    """A one-species database: atom (E, g) or molecule dict."""
    if atom_levels is not None:
        E, g = atom_levels
        return synth.Species(names=["X"], kind=np.array([0], np.int32), mass=np.array([14.0]),
                             density_col=np.array([0], np.int32), atom_off=np.array([0, len(E)], np.int64),
                             atom_E=np.asarray(E, float), atom_g=np.asarray(g, float),
                             st_off=np.array([0, 0], np.int64), st_E=np.zeros(0), st_g=np.zeros(0),
                             st_sigma=np.zeros(0), st_Lalt=np.zeros((0, 2)), st_nv=np.zeros(0, np.int32),
                             st_nj=np.zeros(0, np.int32), st_vib_off=np.zeros(0, np.int64),
                             st_rot_off=np.zeros(0, np.int64), vib_E=np.zeros(0), rot_E=np.zeros(0))
    states = mol["states"]
    vib, rot, vo, ro = [], [], [], []
    nv_, nj_ = 0, 0
    for st in states:
        vo.append(nv_); ro.append(nj_)
        vib.append(st["vib"]); rot.append(st["rot"].ravel())
        nv_ += st["rot"].shape[0]; nj_ += st["rot"].size
    return synth.Species(
        names=["M"], kind=np.array([1], np.int32), mass=np.array([28.0]), density_col=np.array([0], np.int32),
        atom_off=np.array([0, 0], np.int64), atom_E=np.zeros(0), atom_g=np.zeros(0),
        st_off=np.array([0, len(states)], np.int64), st_E=np.array([s["E"] for s in states]),
        st_g=np.array([s["g"] for s in states]), st_sigma=np.array([s["sigma"] for s in states]),
        st_Lalt=np.array([s.get("Lalt", (1.0, 1.0)) for s in states], float),
        st_nv=np.array([s["rot"].shape[0] for s in states], np.int32),
        st_nj=np.array([s["rot"].shape[1] for s in states], np.int32),
        st_vib_off=np.array(vo, np.int64), st_rot_off=np.array(ro, np.int64),
        vib_E=np.concatenate(vib), rot_E=np.concatenate(rot))


class _P:
    def __init__(self, species, cells=None, lines=None, grid=None):
        self.species, self.cells, self.lines, self.grid = species, cells, lines, grid


def test_partition_atom_two_level_closed_form():
    c2 = L.orc_c2()
    sp = _species(atom_levels=([0.0, 83000.0], [4.0, 12.0]))
    for T in [3000.0, 10000.0, 30000.0]:
        Z = oracle.partition(_P(sp), 0, 500.0, T)   # T_tr must not matter for atoms
        assert Z == pytest.approx(4.0 + 12.0 * math.exp(-c2 * 83000.0 / T), rel=1e-14)


def test_partition_harmonic_vibration_rigid_rotor():
    """Separable ladder: Q_vr = [finite geometric sum over V at T_v] x
    [rigid-rotor sum at T_r]; the rotor sum is checked against its
    high-temperature (Mulholland) expansion, the vibrational sum exactly.
    Swapping T_v and T_r, or dropping (2J+1) or 1/sigma, fails it."""
    c2 = L.orc_c2()
    we, B, sigma, g, Te = 1500.0, 0.2, 2.0, 3.0, 1000.0
    nv, nj = 11, 400
    V = np.arange(nv); J = np.arange(nj)
    EV = we * (V + 0.5)
    EJ = np.tile(B * J * (J + 1.0), (nv, 1))
    sp = _species(mol=dict(states=[dict(E=Te, g=g, sigma=sigma, vib=EV, rot=EJ)]))
    Ttr, Tve = 2500.0, 9000.0
    x = c2 * we / Tve
    qv = math.exp(-x / 2) * (1 - math.exp(-nv * x)) / (1 - math.exp(-x))
    y = c2 * B / Ttr
    qr = 1 / y + 1 / 3 + y / 15 + 4 * y * y / 315
    Z = oracle.partition(_P(sp), 0, Ttr, Tve)
    assert Z == pytest.approx(g * math.exp(-c2 * Te / Tve) * qv * qr / sigma, rel=1e-7)


def test_line_alternation_factor_is_applied_by_parity():
    c2 = L.orc_c2()
    EJ = np.array([[0.0, 10.0, 30.0]])
    sp = _species(mol=dict(states=[dict(E=0.0, g=1.0, sigma=1.0, vib=np.array([0.0]), rot=EJ, Lalt=(6.0, 3.0))]))
    T = 100.0
    expect = 6.0 * 1 + 3.0 * 3 * math.exp(-c2 * 10 / T) + 6.0 * 5 * math.exp(-c2 * 30 / T)
    assert oracle.partition(_P(sp), 0, T, 5000.0) == pytest.approx(expect, rel=1e-14)


def test_population_normalisation_atoms_and_molecules():
    """Summed over every level of the partition function, the level
    populations return the species density (Sec. 2.1, S_multi = 1)."""
    p = synth.stagnation_line(n_atomic=400, n_molecular=2000, n_cells=5, n_grid=1000)
    lnp = oracle.lnpref(p)
    sp = p.species
    for c in range(len(p.cells)):
        Ttr, Tve = p.cells.Ttr[c], p.cells.Tve[c]
        for s in range(len(sp.names)):
            n_s = p.cells.n[c, sp.density_col[s]]
            if n_s == 0:
                continue
            tot = 0.0
            if sp.kind[s] == 0:
                for E, g in zip(sp.atom_E[sp.atom_off[s]:sp.atom_off[s + 1]], sp.atom_g[sp.atom_off[s]:sp.atom_off[s + 1]]):
                    tot += math.exp(L.orc_ln_level_pop(lnp[c, s], g, E, 0.0, 0.0, Tve, Ttr))
            else:
                for i in range(sp.st_off[s], sp.st_off[s + 1]):
                    nv, nj = sp.st_nv[i], sp.st_nj[i]
                    for v in range(nv):
                        for J in range(nj):
                            w = sp.st_g[i] * (2 * J + 1) * sp.st_Lalt[i, J & 1] / sp.st_sigma[i]
                            EJ = sp.rot_E[sp.st_rot_off[i] + v * nj + J]
                            tot += math.exp(L.orc_ln_level_pop(lnp[c, s], w, sp.st_E[i],
                                                               sp.vib_E[sp.st_vib_off[i] + v], EJ, Tve, Ttr))
            assert tot == pytest.approx(n_s, rel=1e-12)


def test_lnpref_absent_species_is_minus_inf():
    p = synth.uniform_slab(n_lines=20, n_grid=1000)
    lnp = oracle.lnpref(p)
    assert np.all(np.isfinite(lnp[:, :2]))
    assert np.all(np.isneginf(lnp[:, 2:]))


# ------------------------------------------------------------ line strengths

def _consistent_slab(n_lines=40, T=9000.0, n_grid=20000, seed=7, n_cells=4, dx=1.0, scale_n=1.0):
    """Single-temperature atomic slab whose lines are energy consistent:
    E_u - E_l = 1e7 / lam0 exactly, E_l > 0."""
    rng = np.random.default_rng(seed)
    lam0 = np.sort(rng.uniform(300.0, 900.0, n_lines))
    Eu = rng.uniform(11.0, 14.0, n_lines) * synth.EV_TO_CM
    El = Eu - 1e7 / lam0
    assert np.all(El > 0)
    lines = synth.Lines(lam0=lam0, A=10 ** rng.uniform(6, 8, n_lines), lamS0=10 ** rng.uniform(-3, -2, n_lines),
                        species=np.zeros(n_lines, np.int32), Eu_el=Eu, Eu_v=np.zeros(n_lines),
                        Eu_j=np.zeros(n_lines), gu=rng.integers(2, 10, n_lines).astype(float), El_el=El,
                        El_v=np.zeros(n_lines), El_j=np.zeros(n_lines),
                        gl=rng.integers(2, 10, n_lines).astype(float))
    E = np.concatenate([[0.0], Eu, El]); g = np.concatenate([[4.0], lines.gu, lines.gl])
    sp = synth.Species(names=["N"], kind=np.array([0], np.int32), mass=np.array([14.0]),
                       density_col=np.array([3], np.int32), atom_off=np.array([0, len(E)], np.int64),
                       atom_E=E, atom_g=g, st_off=np.array([0, 0], np.int64), st_E=np.zeros(0), st_g=np.zeros(0),
                       st_sigma=np.zeros(0), st_Lalt=np.zeros((0, 2)), st_nv=np.zeros(0, np.int32),
                       st_nj=np.zeros(0, np.int32), st_vib_off=np.zeros(0, np.int64),
                       st_rot_off=np.zeros(0, np.int64), vib_E=np.zeros(0), rot_E=np.zeros(0))
    n = np.zeros((n_cells, 11)); n[:, 3] = 1e17 * scale_n; n[:, 10] = 1e15
    cells = synth.Cells(Ttr=np.full(n_cells, T), Tve=np.full(n_cells, T), n=n)
    mu, w = synth.gauss_legendre_01(16)
    geo = synth.SlabGeometry(cell_order=np.arange(n_cells, dtype=np.int64), dx=np.full(n_cells, dx), mu=mu, wmu=w)
    return synth.Problem("consistent", sp, lines, cells, synth.Grid(300.0, 900.0, n_grid), geo)


def test_kirchhoff_per_line():
    """Single temperature, energy-consistent lines: S_j / S_kappa equals the
    Planck function in temperature form at the line centre."""
    p = _consistent_slab()
    lnp = oracle.lnpref(p)
    st = oracle.line_states(p, lnp, 0)
    T = p.cells.Tve[0]
    for l in range(len(p.lines)):
        assert st["Sj"][l] / st["Sk"][l] == pytest.approx(L.orc_planck(p.lines.lam0[l], T), rel=1e-12)


def test_emitted_power_is_photon_energy_rate():
    """4 pi S_j = N_u A h c / lam (erg -> W by 1e-7): the line's total
    emitted power per volume (unit-area profile)."""
    p = _consistent_slab(n_lines=10)
    lnp = oracle.lnpref(p)
    st = oracle.line_states(p, lnp, 1)
    for l in range(len(p.lines)):
        lnNu = L.orc_ln_level_pop(lnp[1, 0], p.lines.gu[l], p.lines.Eu_el[l], 0.0, 0.0, p.cells.Tve[1], p.cells.Ttr[1])
        power = 1e-7 * math.exp(lnNu) * p.lines.A[l] * G["h_cgs"] * G["c_cgs"] / (p.lines.lam0[l] * 1e-7)
        assert 4 * math.pi * st["Sj"][l] == pytest.approx(power, rel=1e-13)


# --------------------------------------------------------------- line sum

def test_windowed_sum_equals_brute_force():
    """Tiny lists: the windowed line sum equals the sum over every (line,
    grid point) pair that passes the window test, including windows cut by
    the grid ends and a range that starts inside the grid (k0 > 0)."""
    p = synth.uniform_slab(n_lines=12, n_cells=3, n_grid=2000, lam=(50.0, 60.0), seed=5)
    p.lines.lam0[:] = np.sort(np.random.default_rng(3).uniform(49.0, 61.0, 12))
    p.cells.n[:, synth.NE_COL] = 3e16   # wide Stark windows, several cut by the ends
    lnp = oracle.lnpref(p)
    for k0, nk in [(0, 2000), (700, 600)]:
        kap, em = oracle.spectral_coeffs(p, lnp, k0, nk)
        for c in range(3):
            st = oracle.line_states(p, lnp, c)
            for k in range(k0, k0 + nk, 7):
                lk = oracle.grid_lambda(p.grid, k)
                tj, tk = [], []
                for l in range(len(p.lines)):
                    if L.orc_in_window(lk, p.lines.lam0[l], st["lamV"][l]):
                        ph = L.orc_whiting_phi(abs(lk - p.lines.lam0[l]), st["lamL"][l], st["lamV"][l])
                        tj.append(st["Sj"][l] * ph); tk.append(st["Sk"][l] * ph)
                assert em[c, k - k0] == pytest.approx(math.fsum(tj), rel=1e-15, abs=1e-300)
                assert kap[c, k - k0] == pytest.approx(math.fsum(tk), rel=1e-15, abs=1e-300)


def test_evaluation_count_is_the_in_window_triples():
    """The oracle's count of profile evaluations (the work unit of the line
    sum's roofline) is the number of (line, cell, grid point) triples with
    |lam_k - lam0| <= 100 lamV, counted here by brute force over every grid
    point of the range, windows cut by the grid ends included."""
    p = synth.uniform_slab(n_lines=12, n_cells=3, n_grid=2000, lam=(50.0, 60.0), seed=5)
    p.lines.lam0[:] = np.sort(np.random.default_rng(3).uniform(49.0, 61.0, 12))
    p.cells.n[:, synth.NE_COL] = 3e16
    p.cells.Ttr[:] = [4000.0, 9000.0, 25000.0]
    lnp = oracle.lnpref(p)
    h = (p.grid.lam_max - p.grid.lam_min) / (p.grid.n - 1)
    for k0, nk in [(0, 2000), (700, 600)]:
        oracle.spectral_coeffs(p, lnp, k0, nk)
        got = oracle.last_evaluations()
        lam = p.grid.lam_min + np.arange(k0, k0 + nk) * h
        want = 0
        for c in range(3):
            lamV = oracle.line_states(p, lnp, c)["lamV"]
            want += int((np.abs(lam[None, :] - p.lines.lam0[:, None]) <= 100.0 * lamV[:, None]).sum())
        assert got == want > 0


def test_window_is_fifty_full_widths_each_side():
    """The line wings are cut at |lam - lam0| = 100 lamV, fifty Voigt FWHM on
    each side (reading A3).  One line whose window lies inside a fine grid:
    its emission summed over the grid, divided by its strength, is the area of
    Whiting's shape over exactly that interval (Simpson, independent of the
    oracle's window test).  A cut at 50 lamV would lose about 0.6 % of it."""
    p = synth.uniform_slab(n_lines=1, n_cells=1, n_grid=8001, lam=(53.0, 57.0), seed=11)
    p.lines.lam0[:] = 55.0
    p.lines.lamS0[:] = 0.008           # Stark-dominated: lamV ~ 0.0085 nm at n_e = 1e16
    p.cells.n[:, synth.NE_COL] = 1e16
    lnp = oracle.lnpref(p)
    st = oracle.line_states(p, lnp, 0)
    lamL, lamV, Sj = st["lamL"][0], st["lamV"][0], st["Sj"][0]
    h = (p.grid.lam_max - p.grid.lam_min) / (p.grid.n - 1)
    assert 100 * lamV < 2.0 - 2 * h and lamV / h > 10     # window inside the grid, well resolved
    _, em = oracle.spectral_coeffs(p, lnp)
    area_grid = em[0].sum() * h * 1e-3 / Sj            # um^-1 x um
    area_100 = _simpson_area(lambda x: L.orc_whiting_phi(x, lamL, lamV), 100 * lamV, n=400_001) * 1e-3
    area_50 = _simpson_area(lambda x: L.orc_whiting_phi(x, lamL, lamV), 50 * lamV, n=400_001) * 1e-3
    assert area_grid == pytest.approx(area_100, rel=1e-5)     # measured 7e-8
    assert abs(area_100 / area_50 - 1) > 1e-3                 # 6.4e-3


def test_coeffs_at_points_matches_full_table():
    p = synth.uniform_slab(n_lines=200, n_cells=2, n_grid=5000, seed=9)
    lnp = oracle.lnpref(p)
    kap, em = oracle.spectral_coeffs(p, lnp)
    rng = np.random.default_rng(0)
    c = rng.integers(0, 2, 300); k = rng.integers(0, 5000, 300)
    k2, e2, _ = oracle.coeffs_at(p, c, k, lnp)
    np.testing.assert_allclose(k2, kap[c, k], rtol=1e-15, atol=0)
    np.testing.assert_allclose(e2, em[c, k], rtol=1e-15, atol=0)


# ------------------------------------------------------------------- march

def _exact_coeffs(dtau, s):
    mp = mpmath.mp
    mp.dps = 50
    dt = mpmath.mpf(dtau); s = mpmath.mpf(s)
    if dt == 0:
        return float(s / 2), float(s / 2)
    kap = dt / s
    e = mpmath.exp(-dt)
    f = (1 - e) / dt
    return float((f - e) / kap), float((1 - f) / kap)


@pytest.mark.parametrize("dtau", [0.0, 1e-9, 3e-5, 3.99e-4, 4.01e-4, 1e-3, 0.05, 0.7, 3.0, 30.0, -2e-4, -0.3, -2.0])
def test_segment_coefficients_vs_high_precision(dtau):
    s = 0.37
    a, b = oracle.segment_coeffs(dtau / s, s)
    ea, eb = _exact_coeffs(dtau, s)
    assert a == pytest.approx(ea, rel=1e-11, abs=0)
    assert b == pytest.approx(eb, rel=1e-11, abs=0)


def test_segment_branches_meet_at_threshold():
    t = oracle.THIN_FP64
    s = 1.0
    for sign in (1.0, -1.0):
        lo = oracle.segment_coeffs(sign * t * (1 - 1e-12), s)
        hi = oracle.segment_coeffs(sign * t * (1 + 1e-12), s)
        assert lo[0] == pytest.approx(hi[0], rel=1e-11)
        assert lo[1] == pytest.approx(hi[1], rel=1e-11)


def test_march_matches_ode_with_linear_emission():
    """Two cells: node values are cell values at the ends and the cell mean
    at the shared face; along each segment kappa is the far node's value and
    j is linear.  The march must equal the ODE dI/ds = j(s) - kappa(s) I
    integrated to 1e-13 (this fixes which coefficient multiplies which
    node)."""
    kA, kB, jA, jB = 0.8, 0.1, 2.0, 7.0
    dsA, dsB = 0.9, 1.6
    kap = np.array([[kA], [kB]]); em = np.array([[jA], [jB]])
    grid = synth.Grid(500.0, 501.0, 2)
    I = oracle.march([0, 1], [dsA, dsB], 1.0, kap, em, grid)[0]
    jm, km = 0.5 * (jA + jB), 0.5 * (kA + kB)

    def rhs(s, y):
        if s < dsA:
            return [jA + (jm - jA) * s / dsA - kA * y[0]]
        x = s - dsA
        return [jm + (jB - jm) * x / dsB - km * y[0]]
    y1 = solve_ivp(rhs, (0, dsA), [0.0], method="DOP853", rtol=1e-13, atol=1e-15).y[0, -1]
    y2 = solve_ivp(lambda s, y: rhs(s + dsA, y), (0, dsB), [y1], method="DOP853", rtol=1e-13, atol=1e-15).y[0, -1]
    assert I == pytest.approx(y2, rel=1e-11)


@pytest.mark.parametrize("kap", [0.0, 1e-7, 0.013, 0.4, 10.0])
def test_uniform_slab_closed_form(kap):
    j, m, ds = 3.3, 20, 0.25
    Lx = m * ds
    I = oracle.march(np.arange(m), np.full(m, ds), 1.0, np.full((m, 1), kap), np.full((m, 1), j),
                     synth.Grid(400.0, 401.0, 2))[0]
    expect = j * Lx if kap == 0 else j / kap * -math.expm1(-kap * Lx)
    assert I == pytest.approx(expect, rel=1e-12)


def test_wall_start_is_planck_attenuated():
    T = 1560.0
    grid = synth.Grid(600.0, 601.0, 2)
    kap = 0.3; m = 5; ds = 0.2
    I = oracle.march(np.arange(m), np.full(m, ds), 1.0, np.full((m, 2), kap), np.zeros((m, 2)), grid,
                     wall_start=True, T_wall=T)
    assert I[1] == pytest.approx(L.orc_planck(601.0, T) * math.exp(-kap * m * ds), rel=1e-13)


@pytest.mark.parametrize("n_mu,tol", [(64, [2e-6, 1e-10, 1e-13, 1e-13]), (16, [1e-3, 1e-5, 1e-9, 1e-13])])
def test_tangent_slab_flux_E3(n_mu, tol):
    """Uniform slab: q_lambda = 2 pi S (1/2 - E3(kappa L)), S = j / kappa.
    The Gauss-Legendre error grows as kappa L -> 0 (a boundary layer of
    width kappa L at mu -> 0); the tolerances follow that measured error."""
    p = _consistent_slab(n_lines=3, n_grid=200, n_cells=10, dx=0.5)
    p.geometry.mu, p.geometry.wmu = synth.gauss_legendre_01(n_mu)
    kap = np.array([1e-3, 0.02, 0.3, 2.0]); j = np.array([1.0, 5.0, 2.0, 0.7])
    K = np.tile(kap, (10, 1)); J = np.tile(j, (10, 1))
    out = oracle.solve_slab(p, 0, 4, coeffs=(K, J))
    tau = kap * 5.0
    expect = 2 * math.pi * j / kap * (0.5 - expn(3, tau))
    assert np.all(np.abs(out["q_lambda"] / expect - 1) <= np.asarray(tol))
    # isotropic field of intensity S: flux pi S  (optically thick limit)
    out2 = oracle.solve_slab(p, 0, 4, coeffs=(np.full((10, 4), 50.0), np.full((10, 4), 50.0 * 2.0)))
    np.testing.assert_allclose(out2["q_lambda"], math.pi * 2.0, rtol=1e-12)


def test_planck_limit_thick_single_temperature():
    """Energy-consistent lines in a thick single-temperature slab: at each
    line centre the emerging intensity approaches B(lam0, T) (the source
    function of an isolated line is the Planck function at its centre)."""
    p = _consistent_slab(n_lines=15, n_grid=60001, n_cells=8, dx=2.0, scale_n=100.0)
    out = oracle.solve_slab(p)
    T = p.cells.Tve[0]
    h = (p.grid.lam_max - p.grid.lam_min) / (p.grid.n - 1)
    hits = 0
    for l in range(len(p.lines)):
        k = int(round((p.lines.lam0[l] - p.grid.lam_min) / h))
        if out["kappa"][0, k] * 16.0 > 40.0:
            assert out["I_normal"][k] == pytest.approx(L.orc_planck(p.lines.lam0[l], T), rel=1e-12)
            hits += 1
    assert hits >= 5


def test_spectral_integral_trapezoid():
    grid = synth.Grid(50.0, 2000.0, 1001)
    c = 3.7
    assert oracle.spectral_integral(np.full(1001, c), grid) == pytest.approx(c * 1950.0 * 1e-3, rel=1e-14)
    lam = np.linspace(50.0, 2000.0, 1001)
    assert oracle.spectral_integral(2.0 * lam, grid) == pytest.approx((2000.0 ** 2 - 50.0 ** 2) * 1e-3, rel=1e-13)
    q = np.random.default_rng(1).uniform(0, 1, 1001)
    parts = oracle.spectral_integral(q[:400], grid, 0) + oracle.spectral_integral(q[400:], grid, 400)
    assert parts == pytest.approx(oracle.spectral_integral(q, grid), rel=1e-14)


# ---------------------------------------------------------------- geometry

def _chord(geo, x0, d):
    """Distance to the exit of the (x, r) box, by bisection on the path."""
    dx, dn, dt = d
    def outside(t):
        x = x0 + t * dx
        r = math.hypot(geo.r_body + t * dn, t * dt)
        return x < geo.xf[0] or x > geo.xf[-1] or r > geo.rf[-1]
    lo, hi = 0.0, 1.0
    while not outside(hi):
        hi *= 2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (lo, mid) if outside(mid) else (mid, hi)
    return 0.5 * (lo + hi)


def test_axisym_segments_cover_the_chord_and_sit_in_their_cells():
    geo = synth.AxisymGeometry(xf=np.linspace(0, 20, 41), rf=np.linspace(3.0, 18.0, 21), surf_x=np.array([5.0]),
                               r_body=3.0, mu=np.array([0.3]), wmu=np.array([1.0]), n_phi=4)
    rng = np.random.default_rng(2)
    nx, nr = 40, 20
    for _ in range(30):
        mu = rng.uniform(0.05, 1.0); psi = rng.uniform(0, 2 * math.pi); x0 = rng.uniform(0.1, 19.9)
        st = math.sqrt(1 - mu * mu)
        d = (st * math.cos(psi), mu, st * math.sin(psi))
        cells, ds = oracle.axisym_segments(geo, x0, d)
        assert np.all(ds > 0) and np.all((cells >= 0) & (cells < nx * nr))
        assert ds.sum() == pytest.approx(_chord(geo, x0, d), rel=1e-12)
        # walk from the surface point outward: each segment's interior lies in its cell
        t = 0.0
        for c, s in zip(cells[::-1], ds[::-1]):
            for frac in (0.1, 0.5, 0.9):
                tt = t + frac * s
                x = x0 + tt * d[0]; r = math.hypot(3.0 + tt * d[1], tt * d[2])
                ix, jr = divmod(int(c), nr)
                assert geo.xf[ix] - 1e-9 <= x <= geo.xf[ix + 1] + 1e-9
                assert geo.rf[jr] - 1e-9 <= r <= geo.rf[jr + 1] + 1e-9
            t += s


# -------------------------------------------------------------- generator

@pytest.mark.parametrize("kind,Lu", [("SS", 0), ("DL0", 1), ("DL+", 1), ("DL-", 0)])
def test_hoenl_london_sum_rule(kind, Lu):
    """Table 4 columns: for fixed J_u the branch factors sum to 2 J_u + 1."""
    J = np.arange(2, 151)
    hl = synth._hl_factors(kind, J, Lu)
    np.testing.assert_allclose(hl.sum(axis=1), 2 * J + 1, rtol=1e-13)
