"""CPU oracle of the atomic continuum of Sec. 2.2.1 (bound-free and free-free
absorption and emission) -- test infrastructure only, like the rest of this
package.

Per cell (T = T_ee = T_ve) and atomic radiator with levels i (E_i, g_i):

  bound-free  kappa = sum_i N_i sigma_i(lam),  N_i = (N_a / Q_a) g_i e^{-c2 E_i / T}
              j     = sum_i N_+ N_e B_lam(T) sigma_i(lam) S_i(T),
              S_i   = (h^2 / (2 pi m_e k T))^1.5 g_i e^{c2 (E_ion - E_i) / T} / (2 Q_+)
              (the Saha-Boltzmann N_i,eq / (N_+ N_e); Kirchhoff's law fixes j)
  free-free   kappa = N_a (N_+ N_e / N_a)_Saha sigma^H(lam, T) [1 + D(sigma, T)],
              (N_+ N_e / N_a)_Saha = 2 (Q_+ / Q_a) (2 pi m_e k T / h^2)^1.5 e^{-c2 E_ion / T}
              sigma^3 sigma^H 1e40 = A1 / sigma + A2 (z = 1), sigma = 91.1267 / lam,
              A1 = c1 + c2 e^{-c3 T}, A2 = c4 + c5 e^{-c6 T} + c7 e^{-c8 T}
              j     = B_lam(T) kappa

sigma_i(lam) is the level's table, linear between its nodes and zero outside
them; D(sigma, T) is bilinear in its table and constant beyond its edges;
Q_+ sums the ion's terms; N_a / Q_a is exp(lnpref) of the main path.  The
cgs form of the Saha factors equals the paper's SI form with its unit
conversions.  Both emissions are formed in log space so that the Saha factor
and the Planck function, which over- and underflow separately at low T, are
multiplied as exponents.  Printed constants (Sec. 2.1).

Pinned in tests/test_oracle_continuum_pins.py: Kirchhoff's law at LTE with
the ions at a textbook Saha equilibrium, the tables' nodes and interpolation,
the edge, Kramers' hydrogenic free-free within the fit's Gaunt band, a
bilinear D, and zero ions.
"""
from __future__ import annotations

import numpy as np

KB, CL, H, ME = 1.380e-16, 2.998e10, 6.626e-27, 9.109e-28   # Sec. 2.1 printed constants (cgs)
C2 = H * CL / KB
LAM_H = 91.1267   # nm, hydrogen's bound-free edge (Sec. 2.2.1)


def planck(lam_nm, T):
    """Planck function, W/cm^2/sr/um (the form of Sec. 2.2)."""
    lcm = np.asarray(lam_nm) * 1e-7
    with np.errstate(over="ignore"):   # cold gas: expm1 overflows to inf and B to 0, as it should
        return 1e-7 * 2.0 * H * CL * CL / (1e4 * lcm ** 5 * np.expm1(H * CL / (lcm * KB * T)))


def ln_planck(lam_nm, T):
    lcm = np.asarray(lam_nm) * 1e-7
    x = H * CL / (lcm * KB * T)
    return np.log(1e-7 * 2.0 * H * CL * CL / (1e4 * lcm ** 5)) - x - np.log(-np.expm1(-x))


def sigma_bf(model, i, lam):
    """Level i's photoionisation cross section at lam (cm^2)."""
    a, b = model["node_off"][i], model["node_off"][i + 1]
    return np.interp(lam, model["node_lam"][a:b], model["node_sigma"][a:b], left=0.0, right=0.0)


def ion_Q(model, T):
    return float(np.sum(model["ion_g"] * np.exp(-C2 * model["ion_E"] / T)))


def D_value(model, sig, T):
    """Bilinear D(sigma, T), clamped to the table's range."""
    xs, ts, D = model["D_sigma"], model["D_T"], model["D"]
    sig = np.clip(sig, xs[0], xs[-1])
    T = min(max(T, ts[0]), ts[-1])
    j = np.clip(np.searchsorted(xs, sig, side="right") - 1, 0, len(xs) - 2)
    w = (sig - xs[j]) / (xs[j + 1] - xs[j])
    it = min(max(int(np.searchsorted(ts, T, side="right")) - 1, 0), len(ts) - 2)
    t = (T - ts[it]) / (ts[it + 1] - ts[it])
    row0 = (1 - w) * D[it, j] + w * D[it, j + 1]
    row1 = (1 - w) * D[it + 1, j] + w * D[it + 1, j + 1]
    return (1 - t) * row0 + t * row1


def sigma_ff_H(model, lam, T):
    """Hydrogenic free-free cross section of the Table 3 fit (cm^5), z = 1."""
    c = model["ff_c"]
    s = LAM_H / np.asarray(lam)
    A1 = c[0] + c[1] * np.exp(-c[2] * T)
    A2 = c[3] + c[4] * np.exp(-c[5] * T) + c[6] * np.exp(-c[7] * T)
    return (A1 / s + A2) / (s ** 3 * 1e40)


def coeffs_cell(model, lnpref_s, Tve, n_row, lam, ne_col):
    """Bound-free + free-free (kappa, j) of one model in one cell on lam."""
    T = float(Tve)
    kap = np.zeros_like(lam)
    em = np.zeros_like(lam)
    n_ion, n_e = n_row[model["ion_col"]], n_row[ne_col]
    ln_pe = np.log(n_ion * n_e) if n_ion * n_e > 0 else -np.inf
    Qp = ion_Q(model, T)
    lnB = ln_planck(lam, T)
    for i in range(len(model["E"])):
        sig = sigma_bf(model, i, lam)
        lnN = lnpref_s + np.log(model["g"][i]) - C2 * model["E"][i] / T
        kap += np.exp(lnN) * sig
        lnS = (1.5 * np.log(H * H / (2.0 * np.pi * ME * KB * T)) + np.log(model["g"][i])
               + C2 * (model["E_ion"] - model["E"][i]) / T - np.log(2.0 * Qp))
        em += sig * np.exp(ln_pe + lnS + lnB)
    lnR = np.log(2.0 * Qp) + 1.5 * np.log(2.0 * np.pi * ME * KB * T / (H * H)) - C2 * model["E_ion"] / T
    D = D_value(model, LAM_H / lam, T)
    kff = np.exp(lnpref_s + lnR) * sigma_ff_H(model, lam, T) * (1.0 + D)
    return kap + kff, em + planck(lam, T) * kff


def continuum(models, cells, lnpref, grid, k0=0, nk=None, ne_col=10):
    """Continuum kappa, j [C, nk] of every model over grid points [k0, k0+nk)."""
    nk = grid.n - k0 if nk is None else nk
    h = (grid.lam_max - grid.lam_min) / (grid.n - 1)
    lam = grid.lam_min + np.arange(k0, k0 + nk, dtype=np.float64) * h
    C = len(cells.Tve)
    kap = np.zeros((C, nk))
    em = np.zeros((C, nk))
    for c in range(C):
        for m in models:
            k, j = coeffs_cell(m, lnpref[c, m["species"]], cells.Tve[c], cells.n[c], lam, ne_col)
            kap[c] += k
            em[c] += j
    return kap, em


def saha_lnpref(cells, s_col_ion, E_ion, ion_E, ion_g, ne_col=10):
    """Saha-Boltzmann populations of an atomic radiator (Sec. 2.1),
    N_i = N_+ N_e (h^2 / (2 pi m_e k T))^1.5 g_i e^{c2 (E_ion - E_i) / T} / (2 Q_+),
    written as the prefactor of the Boltzmann form N_i = e^{lnpref} g_i
    e^{-c2 E_i / T}: lnpref = ln(N_+ N_e) + 1.5 ln(h^2 / (2 pi m_e k T)) + c2
    E_ion / T - ln(2 Q_+), per cell (T = T_ve); -inf without ions or electrons."""
    out = np.empty(len(cells.Tve))
    m = dict(ion_E=np.asarray(ion_E, float), ion_g=np.asarray(ion_g, float))
    for c, T in enumerate(cells.Tve):
        pe = cells.n[c, s_col_ion] * cells.n[c, ne_col]
        if pe <= 0:
            out[c] = -np.inf
            continue
        out[c] = (np.log(cells.n[c, s_col_ion]) + np.log(cells.n[c, ne_col])
                  + 1.5 * np.log(H * H / (2.0 * np.pi * ME * KB * T)) + C2 * E_ion / T - np.log(2.0 * ion_Q(m, T)))
    return out
