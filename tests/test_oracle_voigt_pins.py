"""Pins of the oracle's exact Voigt line shape (Sec. 2.2.1, the optional
profile of the full broadening): the Gaussian and Lorentzian limits, the
normalisation over wavelength, the half width against Olivero's formula
(the paper's Voigt HWHM, accurate to 0.02 %), and the line sum against the
Whiting fit of the main oracle."""
import numpy as np
import pytest

import oracle
from oracle import voigt
from paper_2604_11856_gb300 import synth


def test_gaussian_limit():
    lamG = 0.013
    d = np.linspace(0.0, 3 * lamG, 301)
    g = 1e3 * np.sqrt(np.log(2) / np.pi) / lamG * np.exp(-np.log(2) * (d / lamG) ** 2)
    assert np.max(np.abs(voigt.voigt_phi(d, 1e-12 * lamG, lamG) / g - 1)) < 1e-8


def test_lorentzian_limit():
    lamL = 0.02
    d = np.linspace(0.0, 50 * lamL, 501)
    lor = 1e3 * (lamL / np.pi) / (d * d + lamL * lamL)
    assert np.max(np.abs(voigt.voigt_phi(d, lamL, 1e-7 * lamL) / lor - 1)) < 1e-6


@pytest.mark.parametrize("lamL,lamG", [(0.01, 0.01), (0.002, 0.03), (0.05, 0.004)])
def test_normalised_over_wavelength(lamL, lamG):
    X = 2e4 * (lamL + lamG)
    d = np.concatenate([np.linspace(0, 20 * (lamL + lamG), 200001)[:-1], np.geomspace(20 * (lamL + lamG), X, 200001)])
    phi = voigt.voigt_phi(d, lamL, lamG)
    area = 2 * np.trapezoid(phi, d) * 1e-3 + 2 * lamL / (np.pi * X)    # um^-1 x um, plus the Lorentz tails
    assert abs(area - 1) < 2e-6


@pytest.mark.parametrize("lamL,lamG", [(0.01, 0.01), (0.002, 0.03), (0.05, 0.004), (1e-4, 0.02), (0.03, 1e-4)])
def test_half_width_matches_olivero(lamL, lamG):
    p0 = voigt.voigt_phi(0.0, lamL, lamG)
    lo, hi = 0.0, 10 * (lamL + lamG)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if voigt.voigt_phi(mid, lamL, lamG) > 0.5 * p0:
            lo = mid
        else:
            hi = mid
    ref = oracle.lib().orc_voigt_hwhm(lamL, lamG)
    assert abs(lo / ref - 1) < 3e-4


def test_line_sum_against_whiting():
    p = synth.stagnation_line(n_cells=3, n_atomic=400, n_molecular=1500, n_grid=20001)
    lnp = oracle.lnpref(p)
    k1, j1 = oracle.spectral_coeffs(p, lnp)
    k2, j2 = voigt.spectral_coeffs(p, lnp)
    # the same lines and windows, shapes within Whiting's accuracy: the spectra integrate alike
    assert np.all(np.abs(j2.sum(axis=1) / j1.sum(axis=1) - 1) < 0.02)
    big = j1 > 0.1 * j1.max(axis=1, keepdims=True)
    assert np.max(np.abs(j2[big] / j1[big] - 1)) < 0.05
    assert np.array_equal(j1 > 0, j2 > 0)    # identical windows
