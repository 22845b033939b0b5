"""Pins of the QSS collisional-radiative oracle (Sec. 2.1): detailed balance
must give the Boltzmann distribution (and Saha-consistent ionisation must
not disturb it), the closure must hold, a two-level atom must match its
closed form, and collisions must win at high density."""
import numpy as np
import pytest

from oracle import qss
from paper_2604_11856_gb300 import synth


def _state(T, n_M=1e17, n_e=1e15, n_ion=0.0, n_tot=1e16):
    return dict(Ttr=T, Tve=T, n_M=n_M, n_e=n_e, n_ion=n_ion, n_total=n_tot)


def _solve(m, st):
    R, b = qss.rate_matrix(m, st["Ttr"], st["Tve"], st["n_M"], st["n_e"], st["n_ion"], st["n_total"])
    return np.linalg.solve(R, b)


def _boltzmann(m, T, n_tot):
    Q = qss.level_Q(m, T)
    return n_tot * Q[: m["l"]] / Q.sum()


@pytest.mark.parametrize("lumped", [0, 5])
def test_detailed_balance_without_radiation_gives_boltzmann(lumped):
    m = synth.cr_model(n_levels=12, n_lumped=lumped)
    m["A"][:] = 0.0
    m["ii_C"][:] = 0.0
    for T in (5000.0, 9000.0, 15000.0):
        n = _solve(m, _state(T))
        np.testing.assert_allclose(n, _boltzmann(m, T, 1e16), rtol=1e-10)


@pytest.mark.parametrize("kind", ["electrons", "heavy"])
def test_each_collision_partner_thermalises_at_its_own_temperature(kind):
    """Two temperatures, no radiation and no ionisation: with electron
    collisions alone the levels take the Boltzmann distribution at T_ve, with
    heavy-particle collisions alone at T_tr (Sec. 2.1: electron rates at the
    electron temperature, heavy-particle rates at the translational one)."""
    m = synth.cr_model(n_levels=10)
    m["A"][:] = 0.0
    m["ii_C"][:] = 0.0
    m["hp_C" if kind == "electrons" else "e_C"][:] = 0.0
    st = dict(Ttr=6000.0, Tve=12000.0, n_M=1e17, n_e=1e15, n_ion=0.0, n_total=1e16)
    n = _solve(m, st)
    T = st["Tve"] if kind == "electrons" else st["Ttr"]
    np.testing.assert_allclose(n, _boltzmann(m, T, 1e16), rtol=1e-10)


def test_saha_consistent_ions_keep_boltzmann():
    m = synth.cr_model(n_levels=10)
    m["A"][:] = 0.0
    T, n_e, n_tot = 11000.0, 3e15, 1e16
    Q = qss.level_Q(m, T)
    Qp = m["g_ion"] * np.exp(-qss.C2 * m["E_ion"] / T)
    Qe = 2.0 * (2.0 * np.pi * qss.ME * qss.KB * T / (qss.H * qss.H)) ** 1.5
    n_ion = n_tot * Qp * Qe / (Q.sum() * n_e)          # Saha with the Boltzmann atom
    n = _solve(m, _state(T, n_e=n_e, n_ion=n_ion, n_tot=n_tot))
    np.testing.assert_allclose(n, _boltzmann(m, T, n_tot), rtol=1e-9)
    # and away from Saha the excited levels move (the source term is live)
    n2 = _solve(m, _state(T, n_e=n_e, n_ion=10 * n_ion, n_tot=n_tot))
    assert np.max(np.abs(n2[1:] / n[1:] - 1)) > 1e-3


def test_closure_and_two_level_closed_form():
    m = synth.cr_model(n_levels=2)
    m["ii_C"][:] = 0.0
    m["A"][:] = 3e7
    m["lam"][:] = 500.0                                 # optically thin: escapes
    st = _state(8000.0, n_M=1e16, n_e=1e14)
    n = _solve(m, st)
    assert abs(n.sum() / 1e16 - 1) < 1e-13
    # n1 / n0 = (collisional up) / (collisional down + A), per particle
    th = qss.C2 * (m["E"][1] - m["E"][0])
    up = (m["hp_C"][0] * 8000.0 ** m["hp_n"][0] * np.exp(-th / 8000.0) * 1e16 +
          m["e_C"][0] * 8000.0 ** m["e_n"][0] * np.exp(-th / 8000.0) * 1e14) / qss.N_A
    Q = qss.level_Q(m, 8000.0)
    dn = up * Q[0] / Q[1] + 3e7
    assert abs(n[1] / n[0] / (up / dn) - 1) < 1e-12
    # in the VUV (below 200 nm) the line is trapped: Boltzmann again
    m["lam"][:] = 150.0
    n = _solve(m, st)
    assert abs(n[1] / n[0] / (Q[1] / Q[0]) - 1) < 1e-12


def test_two_level_closed_form_at_two_temperatures():
    """Two temperatures and both partners: the two-level balance
    n1 / n0 = (heavy up + electron up) / (heavy down + electron down + A), with
    heavy-particle rates at T_tr and electron rates at T_ve (Sec. 2.1), and each
    downward rate from its upward one by detailed balance at the partner's
    temperature."""
    m = synth.cr_model(n_levels=2)
    m["ii_C"][:] = 0.0
    m["A"][:] = 3e7
    m["lam"][:] = 500.0
    Ttr, Tve, n_M, n_e = 6000.0, 14000.0, 1e16, 1e14
    n = _solve(m, dict(Ttr=Ttr, Tve=Tve, n_M=n_M, n_e=n_e, n_ion=0.0, n_total=1e16))
    th = qss.C2 * (m["E"][1] - m["E"][0])
    kh = m["hp_C"][0] * Ttr ** m["hp_n"][0] * np.exp(-th / Ttr)
    ke = m["e_C"][0] * Tve ** m["e_n"][0] * np.exp(-th / Tve)
    Qh, Qe = qss.level_Q(m, Ttr), qss.level_Q(m, Tve)
    up = (kh * n_M + ke * n_e) / qss.N_A
    dn = (kh * Qh[0] / Qh[1] * n_M + ke * Qe[0] / Qe[1] * n_e) / qss.N_A + 3e7
    assert abs(n[1] / n[0] / (up / dn) - 1) < 1e-12


def test_collisions_win_at_high_density():
    m = synth.cr_model(n_levels=15)
    m["ii_C"][:] = 0.0
    T = 9000.0
    lo = _solve(m, _state(T, n_M=1e14, n_e=1e11))
    hi = _solve(m, _state(T, n_M=1e22, n_e=1e20))
    ref = _boltzmann(m, T, 1e16)
    assert np.max(np.abs(hi / ref - 1)) < 1e-3
    assert np.max(np.abs(lo[1:] / ref[1:] - 1)) > 0.1      # radiation depletes excited levels
    assert np.all(lo[1:] < ref[1:])


def test_cells_wiring_boltzmann_in_every_cell():
    m = synth.cr_model(n_levels=8)
    m["A"][:] = 0.0
    m["ii_C"][:] = 0.0
    p = synth.stagnation_line(n_cells=5, n_atomic=10, n_molecular=10, n_grid=11)
    cells = synth.Cells(Ttr=p.cells.Tve.copy(), Tve=p.cells.Tve.copy(), n=p.cells.n)
    n = qss.solve_cells(m, cells, ion_col=m["ion_col"])
    for c in range(5):
        np.testing.assert_allclose(n[c], _boltzmann(m, cells.Tve[c], cells.n[c, m["col"]]), rtol=1e-9)
