"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle (a flipped sign, a
swapped coefficient, a wrong temperature, a dropped term, a changed
constant) and runs the pins against the copy; at least one pin must fail for
every mistake.  Mistakes in oracle/rapral_oracle.cpp are built with the
oracle's own flags and loaded through RAPRAL_ORACLE_LIB by
tests/test_oracle_pins.py.  Mistakes in the numpy modules (QSS populations,
continuum, exact Voigt shape, the Fibonacci angular path) go into a copy of
the oracle package in a scratch tree, where that module's pin file runs.
CPU only: nothing here touches a GPU."""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rapral_oracle.cpp")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, text in the oracle, planted mistake[, pin file; test_oracle_pins.py by default])
MUTATIONS = [
    ("whiting correction sign (Sec. 2.2.1)",
     "+ 0.016 * r * (1.0 - r)", "- 0.016 * r * (1.0 - r)"),
    ("whiting Gaussian exponent (Sec. 2.2.1)",
     "std::exp(-2.772 * u * u)", "std::exp(-2.0 * u * u)"),
    ("whiting normalisation (Sec. 2.2.1)",
     "(1.065 + 0.447 * r + 0.058 * r * r)", "(1.065 + 0.447 * r - 0.058 * r * r)"),
    ("Doppler width temperature over mass inverted (Sec. 2.2.1)",
     "std::sqrt(Ttr / M)", "std::sqrt(M / Ttr)"),
    ("Stark temperature exponent (Sec. 2.2.1)",
     "std::pow(Tve / 10000.0, 0.33)", "std::pow(Tve / 10000.0, 0.5)"),
    ("Voigt half width, sign inside the 0.18121 term (Sec. 2.2.1)",
     "0.18121 * (1.0 - d * d)", "0.18121 * (1.0 + d * d)"),
    ("segment coefficients attached to the wrong nodes (Sec. 2.2.3)",
     "*a = (f - e) / kap;\n        *b = (1.0 - f) / kap;", "*a = (1.0 - f) / kap;\n        *b = (f - e) / kap;"),
    ("thin-segment series, first-order term (Sec. 2.2.3)",
     "*a = s * (0.5 - dtau / 3.0 + dtau * dtau / 8.0);", "*a = s * (0.5 - dtau / 6.0 + dtau * dtau / 8.0);"),
    ("node values not face-averaged (Sec. 2.2.3)",
     "return 0.5 * (tab[cell[i - 1] * ld + k] + tab[cell[i] * ld + k]);", "return tab[cell[i] * ld + k];"),
    ("trapezoid end weights (Sec. 2.2.3)",
     "? 0.5 : 1.0;", "? 1.0 : 1.0;"),
    ("rotational ladder at the vibrational-electronic temperature (Sec. 2.1)",
     "std::exp(-c2 * EJ / Ttr)", "std::exp(-c2 * EJ / Tve)"),
    ("vibrational level energy at the translational temperature (Sec. 2.1)",
     "E_v / Tve + E_j / Ttr", "E_v / Ttr + E_j / Ttr"),
    ("line-wing window of 50 instead of 100 half widths",
     "WINDOW_HWHM = 100.0", "WINDOW_HWHM = 50.0"),
    ("stimulated emission dropped from the absorption strength (Sec. 2.2.1)",
     "std::expm1(lnNl + std::log(ln->gu[l]) - std::log(ln->gl[l]) - lnNu)",
     "std::exp(lnNl + std::log(ln->gu[l]) - std::log(ln->gl[l]) - lnNu)"),
    ("Planck function, power of the wavelength (Sec. 2.2)",
     "(1e4 * std::pow(lcm, 5) * std::expm1(x))", "(1e4 * std::pow(lcm, 4) * std::expm1(x))"),
    ("emission strength prefactor hc/4pi (Sec. 2.2.1)",
     "(hP * cL / (4.0 * M_PI))", "(hP * cL / (2.0 * M_PI))"),
    ("Stark coefficient, exponent of the ionisation gap (Sec. 2.2.1)",
     "std::pow(dE, 2.623)", "std::pow(dE, 2.5)", "test_oracle_broadening_pins.py"),
    ("Stark coefficient, floor of the ionisation gap (Sec. 2.2.1)",
     "E_IONIZE_H / 25.0", "E_IONIZE_H / 16.0", "test_oracle_broadening_pins.py"),
    ("oscillator strength with the weights inverted (Sec. 2.2.1)",
     "* gu / gl * A;", "* gl / gu * A;", "test_oracle_broadening_pins.py"),
    ("resonance width, weight ratio inverted (Sec. 2.2.1)",
     "std::sqrt(gl / gu)", "std::sqrt(gu / gl)", "test_oracle_broadening_pins.py"),
    ("van der Waals width without the factor 2 in the speed (Sec. 2.2.1)",
     "6.65e-29 * N * std::sqrt(2.0 * Ttr / M)", "6.65e-29 * N * std::sqrt(Ttr / M)",
     "test_oracle_broadening_pins.py"),
    ("departure of the lower level taken from the upper level's index (Sec. 2.1)",
     "departure(sp, c, s, DEP_LEV_L, l)", "departure(sp, c, s, DEP_LEV_U, l)", "test_oracle_departure_pins.py"),
    ("ln(N_s / Z_s) with the partition function multiplied in (Sec. 2.1)",
     "std::log(N) - std::log(Z);", "std::log(N) + std::log(Z);"),
    ("rotational sum multiplied by the symmetry number instead of divided (Sec. 2.1)",
     "* rot / sp->st_sigma[i];", "* rot * sp->st_sigma[i];"),
    ("ray's radial distance with the body radius dropped (ray-cell segments)",
     "const double y = r_body + t * dn, z = t * dt;", "const double y = t * dn, z = t * dt;"),
    ("departure of the upper level with the wrong sign (Sec. 2.1)",
     "departure(sp, c, s, DEP_LEV_U, l);", "-departure(sp, c, s, DEP_LEV_U, l);", "test_oracle_departure_pins.py"),
]


def _run(case, tmp):
    name, old, new = case[:3]
    pins = os.path.join(ROOT, "tests", case[3]) if len(case) > 3 else PINS
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique or missing: {name}"
    tag = str(MUTATIONS.index(case))
    cpp = os.path.join(tmp, f"mutant{tag}.cpp")
    so = os.path.join(tmp, f"mutant{tag}.so")
    with open(cpp, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", cpp, "-o", so],
                   check=True)
    env = dict(os.environ, RAPRAL_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    return name, r.returncode, r.stdout[-400:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        results = list(ex.map(lambda c: _run(c, str(tmp_path)), MUTATIONS))
    survived = [(name, out) for name, rc, out in results if rc == 0]
    assert not survived, "mistakes no pin caught:\n" + "\n".join(f"{n}\n{o}" for n, o in survived)
    # a return code other than 1 (tests failed) means the run itself broke
    broken = [(name, rc, out) for name, rc, out in results if rc not in (0, 1)]
    assert not broken, broken


def test_unmutated_copy_passes_the_pins(tmp_path):
    """The harness itself: the same build of the unchanged source passes."""
    so = os.path.join(str(tmp_path), "same.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", SRC, "-o", so],
                   check=True)
    env = dict(os.environ, RAPRAL_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-2000:]


# (module, name, text in the module, planted mistake, pin file).  Not here: the
# A1 / sigma term of the Table 3 free-free fit.  It is at most ~7 % of the fit
# over 100-2000 nm, inside the Kramers-Gaunt band that is the only check
# independent of the printed formula, so no pin can tell it from A1 sigma.
PY_MUTATIONS = [
    ("qss.py", "detailed balance inverted (Sec. 2.1)",
     "kh_dn = kh_up * Qh[i] / Qh[j]", "kh_dn = kh_up * Qh[j] / Qh[i]", "test_oracle_qss_pins.py"),
    ("qss.py", "three-body recombination by the wrong partition ratio (Sec. 2.1)",
     "kr = kf * Qe_lv[i] / (Qp * Qel)", "kr = kf * Qe_lv[i] * Qp / Qel", "test_oracle_qss_pins.py"),
    ("qss.py", "electron-impact rates at the translational temperature (Sec. 2.1, reading Q2)",
     'theta, Tve)\n        ke_dn', 'theta, Ttr)\n        ke_dn', "test_oracle_qss_pins.py"),
    ("qss.py", "VUV lines not trapped (escape factor, Sec. 2.1 reading Q4)",
     "(1.0 if model[\"lam\"][t] >= 200.0 else 0.0)", "1.0", "test_oracle_qss_pins.py"),
    ("qss.py", "closure without the lumped levels' Boltzmann ratio (Sec. 2.1)",
     "1.0 + np.sum(Qe_lv[l:]) / Qe_lv[l - 1]", "1.0 + np.sum(Qe_lv[l:])", "test_oracle_qss_pins.py"),
    ("continuum.py", "free-free emission without the Planck factor (Kirchhoff, Sec. 2.2.1)",
     "em + planck(lam, T) * kff", "em + kff", "test_oracle_continuum_pins.py"),
    ("continuum.py", "bound-free emission, sign of the ionisation gap (Sec. 2.2.1)",
     "+ C2 * (model[\"E_ion\"] - model[\"E\"][i]) / T", "- C2 * (model[\"E_ion\"] - model[\"E\"][i]) / T",
     "test_oracle_continuum_pins.py"),
    ("continuum.py", "free-free correction D with the wrong sign (Sec. 2.2.1)",
     "* (1.0 + D)", "* (1.0 - D)", "test_oracle_continuum_pins.py"),
    ("continuum.py", "cross sections extrapolated past the table edge (Sec. 2.2.1)",
     "left=0.0, right=0.0", "left=None, right=None", "test_oracle_continuum_pins.py"),
    ("continuum.py", "Saha factor without the electron spin weight 2 (Sec. 2.1)",
     "- np.log(2.0 * ion_Q(m, T))", "- np.log(ion_Q(m, T))", "test_oracle_continuum_pins.py"),
    ("continuum.py", "Saha-Boltzmann populations, thermal de Broglie exponent (Sec. 2.1)",
     "+ 1.5 * np.log(H * H / (2.0 * np.pi * ME * KB * T)) + C2 * E_ion / T",
     "+ 1.0 * np.log(H * H / (2.0 * np.pi * ME * KB * T)) + C2 * E_ion / T", "test_oracle_continuum_pins.py"),
    ("voigt.py", "Gaussian sigma from the half width (Sec. 2.2.1)",
     "sig = lamG / np.sqrt(2.0 * np.log(2.0))", "sig = lamG / np.sqrt(np.log(2.0))", "test_oracle_voigt_pins.py"),
    ("voigt.py", "Voigt normalisation (Sec. 2.2.1)",
     "(sig * np.sqrt(2.0 * np.pi))", "(sig * np.sqrt(np.pi))", "test_oracle_voigt_pins.py"),
    ("voigt.py", "Lorentz half width doubled in the Faddeeva argument (Sec. 2.2.1)",
     "1j * lamL", "1j * 2.0 * lamL", "test_oracle_voigt_pins.py"),
    ("los.py", "Fibonacci azimuth step (Sec. 2.2.3)",
     "(np.sqrt(5.0) - 1.0) * np.pi", "(np.sqrt(5.0) - 1.0) * 0.5 * np.pi", "test_oracle_los_pins.py"),
    ("los.py", "four-point sum with the printed weight (Sec. 2.2.3, reading F5)",
     "0.5 * (np.cos(phi[p]) ** 2 - np.cos(phi[p + 1]) ** 2)", "(np.cos(phi[p + 1]) - np.cos(phi[p]))",
     "test_oracle_los_pins.py"),
    ("los.py", "azimuth grid spacing (Sec. 2.2.3)",
     "2.0 * np.pi * np.arange(n_theta) / (n_theta - 1)", "2.0 * np.pi * np.arange(n_theta) / n_theta",
     "test_oracle_los_pins.py"),
]


def _run_py(idx, case, tmp, lib):
    module, name, old, new, pins = case
    root = os.path.join(tmp, f"tree{idx}")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(root, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    pkg = os.path.join(root, "paper_2604_11856_gb300")
    os.makedirs(pkg)
    for f in glob.glob(os.path.join(ROOT, "paper_2604_11856_gb300", "*.py")):
        shutil.copy(f, pkg)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(root, "tests", "golden"))
    for f in ("conftest.py", pins):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(root, "tests", f))
    path = os.path.join(root, "oracle", module)
    src = open(path).read()
    assert src.count(old) == 1, f"mutation site not unique or missing: {name}"
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    env = dict(os.environ, RAPRAL_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", pins), "-x", "-q", "-p",
                        "no:cacheprovider"], cwd=root, env=env, capture_output=True, text=True)
    return name, r.returncode, r.stdout[-400:]


def test_every_planted_mistake_in_the_numpy_modules_fails_a_pin(tmp_path):
    import oracle
    lib = oracle.build()
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        results = list(ex.map(lambda ic: _run_py(ic[0], ic[1], str(tmp_path), lib), enumerate(PY_MUTATIONS)))
    survived = [(name, out) for name, rc, out in results if rc == 0]
    assert not survived, "mistakes no pin caught:\n" + "\n".join(f"{n}\n{o}" for n, o in survived)
    broken = [(name, rc, out) for name, rc, out in results if rc not in (0, 1)]
    assert not broken, broken
