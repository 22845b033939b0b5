"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/rapral_oracle.cpp (a flipped
sign, a swapped coefficient, a wrong temperature, a dropped term, a changed
constant), builds the copy with the oracle's own flags, and runs
tests/test_oracle_pins.py against it (RAPRAL_ORACLE_LIB).  At least one pin
must fail for every mistake.  CPU only: nothing here touches a GPU."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rapral_oracle.cpp")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, text in the oracle, planted mistake)
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
]


def _run(case, tmp):
    name, old, new = case
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
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
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
