"""CPU oracle of the line sum with the exact Voigt line shape (the optional
profile of Sec. 2.2.1's full broadening) -- test infrastructure only, like
the rest of this package.

  phi(dlam) = 1e3 Re w(z) / (sigma sqrt(2 pi))  um^-1,
  z = (dlam + i lamL) / (sigma sqrt 2),  sigma = lamG / sqrt(2 ln 2),

the convolution of the Doppler Gaussian (HWHM lamG) with the Lorentzian
(HWHM lamL), normalised to 1 over wavelength in um; w is the Faddeeva
function, taken from scipy.special.wofz (a library routine).  Strengths,
widths and windows (|lam_k - lam0| <= 100 lamV, lamV Olivero's HWHM) are
the main oracle's (oracle.line_states), so only the shape differs from
oracle.spectral_coeffs.

Pinned in tests/test_oracle_voigt_pins.py: the Gaussian and Lorentzian
limits, the normalisation, the half width against Olivero's formula, and
the line sum against Whiting's within that fit's accuracy.
"""
from __future__ import annotations

import numpy as np
from scipy.special import wofz

from . import line_states, lnpref as _lnpref

WINDOW = 100.0


def voigt_phi(dlam, lamL, lamG):
    """The exact Voigt shape, um^-1, at offsets dlam (nm)."""
    sig = lamG / np.sqrt(2.0 * np.log(2.0))
    z = (np.asarray(dlam, dtype=np.float64) + 1j * lamL) / (sig * np.sqrt(2.0))
    return 1e3 * wofz(z).real / (sig * np.sqrt(2.0 * np.pi))


def spectral_coeffs(problem, lnp=None, k0=0, nk=None, with_abs=False):
    """kappa, j [C, nk] over grid points [k0, k0+nk) with the exact Voigt shape."""
    if lnp is None:
        lnp = _lnpref(problem)
    g = problem.grid
    nk = g.n - k0 if nk is None else nk
    h = (g.lam_max - g.lam_min) / (g.n - 1)
    C = len(problem.cells)
    kap = np.zeros((C, nk)); em = np.zeros((C, nk)); ab = np.zeros((C, nk))
    lam0 = problem.lines.lam0
    for c in range(C):
        st = line_states(problem, lnp, c)
        for l in np.nonzero((st["Sj"] > 0) | (st["Sk"] != 0))[0]:
            half = WINDOW * st["lamV"][l]
            a = max(int(np.floor((lam0[l] - half - g.lam_min) / h)) - 2, k0)
            b = min(int(np.ceil((lam0[l] + half - g.lam_min) / h)) + 2, k0 + nk - 1)
            if a > b:
                continue
            k = np.arange(a, b + 1)
            lk = g.lam_min + k.astype(np.float64) * h
            m = np.abs(lk - lam0[l]) <= WINDOW * st["lamV"][l]
            if not m.any():
                continue
            phi = voigt_phi(lk[m] - lam0[l], st["lamL"][l], st["lamG"][l])
            idx = k[m] - k0
            em[c, idx] += st["Sj"][l] * phi
            kap[c, idx] += st["Sk"][l] * phi
            ab[c, idx] += np.abs(st["Sk"][l] * phi)
    return (kap, em, ab) if with_abs else (kap, em)
