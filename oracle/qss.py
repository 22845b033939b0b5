"""CPU oracle of the quasi-steady-state (QSS) collisional-radiative
populations of Sec. 2.1 -- test infrastructure only, like the rest of this
package.

For one radiating atom and one cell the excited levels 1 .. l-1 obey
0 = gains - losses (the QSS form of the master equation) with heavy-particle
impact excitation (HPIE), electron impact excitation (EIE), spontaneous
emission with an escape factor (RT) and electron impact ionisation with its
three-body recombination (EII); the ground level closes the system with the
total density.  The matrix R and source b follow the paper's assembly:

  R[0, j] = 1 (j < l-1),  R[0, l-1] = 1 + sum_{p >= l} Q_p / Q_{l-1}
  R[i, i] = - sum_{m != i} (k_HPIE(i,m) N_M + k_EIE(i,m) N_e) / N_A
            - sum_{m < i} Lambda A(i,m) - k_EII(i,c) N_e / N_A
  R[i, j] = (k_HPIE(j,i) N_M + k_EIE(j,i) N_e) / N_A + [j > i] Lambda A(j,i)
  b[0] = N_total,  b[i] = - k_EII(c,i) N_+ N_e N_e / N_A

with forward (upward) rates k = C T^n exp(-theta/T), theta the level gap
(or the ionisation gap) in K, backward rates by detailed balance
k(j,i) = k(i,j) Q_i / Q_j with Q_i = g_i exp(-hc E_i / k T), and the
recombination k(c,i) = k(i,c) Q_i / (Q_+ Q_e), Q_+ = g_+ exp(-hc E_ion / kT),
Q_e = 2 (2 pi m_e k T / h^2)^1.5.  Heavy-particle rates at T_tr, electron
rates at T_ve; N_M the summed density of every non-electron column; the
escape factor Lambda = 0 below 200 nm (optically thick VUV), 1 above.
numpy.linalg.solve (LU with partial pivoting) is the solve step.

Pinned in tests/test_oracle_qss_pins.py: detailed balance gives the
Boltzmann distribution at one temperature without radiation (with and
without ionisation at Saha equilibrium), the closure holds, a two-level
system matches its closed form, and collisions dominate at high density.
"""
from __future__ import annotations

import numpy as np

N_A = 6.022e23          # 1/mol
C2 = 6.626e-27 * 2.998e10 / 1.380e-16   # hc/k, cm K (Sec. 2.1 printed constants)
KB, H, ME = 1.380e-16, 6.626e-27, 9.109e-28


def level_Q(model, T):
    """Q_i = g_i exp(-hc E_i / k T) for every level of the model (l* levels)."""
    return model["g"] * np.exp(-C2 * model["E"] / T)


def rate_matrix(model, Ttr, Tve, n_M, n_e, n_ion, n_total):
    """R (l x l) and b (l) of one cell, as in the module docstring."""
    l = int(model["l"])
    E, g = model["E"], model["g"]
    lo, up = model["lo"], model["up"]
    R = np.zeros((l, l))
    b = np.zeros(l)
    Qh, Qe_lv = level_Q(model, Ttr), level_Q(model, Tve)

    def k_fwd(C, n, theta, T):
        return C * T ** n * np.exp(-theta / T)

    for t in range(len(lo)):
        i, j = int(lo[t]), int(up[t])                   # i < j
        theta = C2 * (E[j] - E[i])
        kh_up = k_fwd(model["hp_C"][t], model["hp_n"][t], theta, Ttr)
        kh_dn = kh_up * Qh[i] / Qh[j]
        ke_up = k_fwd(model["e_C"][t], model["e_n"][t], theta, Tve)
        ke_dn = ke_up * Qe_lv[i] / Qe_lv[j]
        rad = model["A"][t] * (1.0 if model["lam"][t] >= 200.0 else 0.0)
        up_rate = (kh_up * n_M + ke_up * n_e) / N_A      # i -> j, per particle in i
        dn_rate = (kh_dn * n_M + ke_dn * n_e) / N_A + rad   # j -> i, per particle in j
        # losses on the diagonal, gains off it (rows 1 .. l-1 only)
        if i > 0:
            R[i, i] -= up_rate
            R[i, j] += dn_rate
        if j > 0:
            R[j, j] -= dn_rate
            R[j, i] += up_rate
    # ionisation and three-body recombination
    Qp = model["g_ion"] * np.exp(-C2 * model["E_ion"] / Tve)
    Qel = 2.0 * (2.0 * np.pi * ME * KB * Tve / (H * H)) ** 1.5
    for i in range(1, l):
        kf = model["ii_C"][i] * Tve ** model["ii_n"][i] * np.exp(-C2 * (model["E_ion"] - E[i]) / Tve)
        kr = kf * Qe_lv[i] / (Qp * Qel)
        R[i, i] -= kf * n_e / N_A
        b[i] = -kr * n_ion * n_e * n_e / N_A
    # closure with the lumped levels above l - 1 (Boltzmann with level l - 1 at T_ve)
    R[0, :] = 1.0
    if len(E) > l:
        R[0, l - 1] = 1.0 + np.sum(Qe_lv[l:]) / Qe_lv[l - 1]
    b[0] = n_total
    return R, b


def solve_cells(model, cells, ion_col=None):
    """Populations n [C, l] of the model's species in every cell."""
    col, ne_col = int(model["col"]), int(getattr(cells, "ne_col", 10))
    C = len(cells.Ttr)
    out = np.zeros((C, int(model["l"])))
    for c in range(C):
        dens = np.asarray(cells.n[c], dtype=np.float64)
        n_M = float(np.sum(np.delete(dens, ne_col)))
        n_e = float(dens[ne_col])
        n_ion = float(dens[ion_col]) if ion_col is not None and ion_col >= 0 else 0.0
        R, b = rate_matrix(model, cells.Ttr[c], cells.Tve[c], n_M, n_e, n_ion, float(dens[col]))
        out[c] = np.linalg.solve(R, b)
    return out


def departures(model, cells, lnpref, s, n_qss, n_lev=None):
    """ln b_i = ln N_i(QSS) - ln N_i(Boltzmann) of the model's levels for
    species s in every cell, with N_i(Boltzmann) = exp(lnpref[c][s] + ln g_i
    - c2 E_i / T_ve) (the main path's populations); returns [C, n_lev]
    (zero past the model's levels)."""
    l = int(model["l"])
    n_lev = l if n_lev is None else n_lev
    out = np.zeros((len(cells.Tve), n_lev))
    for c in range(len(cells.Tve)):
        lnB = lnpref[c, s] + np.log(model["g"][:l]) - C2 * model["E"][:l] / cells.Tve[c]
        out[c, :l] = np.log(n_qss[c]) - lnB
    return out
