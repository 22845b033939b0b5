"""CPU oracle for the RAPRAL hot path -- test infrastructure only.

A plain FP64 restatement of the method (C++ with OpenMP over cells, the
paper's own parallel axis, plus numpy glue for sums that are one line).  Only
the tests, the package smoke check and the benchmark's CPU-baseline leg may
import it.  It shares no code with the CUDA library and never imports it; the
two meet only through the seeded inputs of the generator module.

Pinned functions and what pins them are listed in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rapral_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

# thin-segment thresholds of the march (|dtau| below which the series is used)
THIN_FP64 = 4e-4


def build(force=False):
    """Compile the oracle with g++ (-ffp-contract=off keeps x86 and Arm
    rounding identical)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Species(ct.Structure):
    _fields_ = [("S", ct.c_int32), ("kind", ct.c_void_p), ("dens_col", ct.c_void_p), ("mass", ct.c_void_p),
                ("atom_off", ct.c_void_p), ("atom_E", ct.c_void_p), ("atom_g", ct.c_void_p),
                ("st_off", ct.c_void_p), ("st_E", ct.c_void_p), ("st_g", ct.c_void_p),
                ("st_sigma", ct.c_void_p), ("st_Lalt", ct.c_void_p), ("st_nv", ct.c_void_p),
                ("st_nj", ct.c_void_p), ("st_vib_off", ct.c_void_p), ("st_rot_off", ct.c_void_p),
                ("vib_E", ct.c_void_p), ("rot_E", ct.c_void_p)]


class _Lines(ct.Structure):
    _fields_ = [("L", ct.c_int64)] + [(k, ct.c_void_p) for k in
                                       ["lam0", "A", "lamS0", "species", "Eu_el", "Eu_v", "Eu_j", "gu",
                                        "El_el", "El_v", "El_j", "gl"]]


class _Cells(ct.Structure):
    _fields_ = [("C", ct.c_int64), ("Ttr", ct.c_void_p), ("Tve", ct.c_void_p), ("n", ct.c_void_p),
                ("ncol", ct.c_int32), ("ne_col", ct.c_int32)]


class _Grid(ct.Structure):
    _fields_ = [("lam_min", ct.c_double), ("lam_max", ct.c_double), ("n", ct.c_int64)]


def lib():
    """The oracle library, built on first use.  RAPRAL_ORACLE_LIB names a
    different build of the same source to load instead: the mutation tests use
    it to run the pins against copies with planted mistakes."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = ct.CDLL(os.environ.get("RAPRAL_ORACLE_LIB") or build())
            d, i64, i32, vp = ct.c_double, ct.c_int64, ct.c_int32, ct.c_void_p
            P = ct.POINTER
            sig = {
                "orc_set_codata": (None, [ct.c_int]),
                "orc_c2": (d, []),
                "orc_const": (d, [ct.c_int]),
                "orc_partition": (d, [P(_Species), i32, d, d]),
                "orc_lnpref": (None, [P(_Species), P(_Cells), vp]),
                "orc_ln_level_pop": (d, [d, d, d, d, d, d, d]),
                "orc_planck": (d, [d, d]),
                "orc_doppler_hwhm": (d, [d, d, d]),
                "orc_stark_hwhm": (d, [d, d, d]),
                "orc_lorentz_hwhm": (d, [d]),
                "orc_voigt_hwhm": (d, [d, d]),
                "orc_whiting_phi": (d, [d, d, d]),
                "orc_line_states": (None, [P(_Species), P(_Lines), P(_Cells), vp, i64, vp, vp, vp, vp, vp]),
                "orc_grid_lambda": (d, [P(_Grid), i64]),
                "orc_in_window": (ct.c_int, [d, d, d]),
                "orc_spectral_coeffs": (None, [P(_Species), P(_Lines), P(_Cells), vp, P(_Grid), i64, i64,
                                               vp, vp, vp]),
                "orc_coeffs_at": (None, [P(_Species), P(_Lines), P(_Cells), vp, P(_Grid), i64, vp, vp,
                                         vp, vp, vp]),
                "orc_axisym_segments": (i64, [vp, i32, vp, i32, d, d, d, d, d, i64, vp, vp]),
                "orc_march": (None, [i64, vp, vp, d, vp, vp, i64, i64, i32, d, P(_Grid), i64, d, vp]),
                "orc_march_nodes": (None, [i64, vp, vp, vp, vp, i64, i64, i32, d, P(_Grid), i64, d, vp]),
                "orc_set_broadening": (None, [ct.c_int, ct.c_int, vp, ct.c_int, vp]),
                "orc_set_departures": (None, [i64, vp, vp, vp]),
                "orc_stark_coeff_ionize": (d, [d, d, d]),
                "orc_oscillator_strength": (d, [d, d, d, d]),
                "orc_resonance_hwhm": (d, [d, d, d, d, d]),
                "orc_vdw_hwhm": (d, [d, d, d, d, d, d]),
                "orc_spectral_integral": (d, [vp, P(_Grid), i64, i64]),
                "orc_segment_coeffs": (None, [d, d, d, P(d), P(d)]),
                "orc_last_evaluations": (i64, []),
                "orc_num_threads": (ct.c_int, []),
                "orc_set_threads": (None, [ct.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(_lib, name)
                f.restype = res
                f.argtypes = args
    return _lib


def _p(a):
    return a.ctypes.data_as(ct.c_void_p) if a is not None else None


class _Keep:
    """Holds contiguous numpy copies alive while a ctypes struct points at them."""

    def __init__(self):
        self.arrs = []

    def __call__(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.arrs.append(a)
        return _p(a)


def species_struct(sp, keep):
    s = _Species()
    s.S = len(sp.names)
    s.kind = keep(sp.kind, np.int32); s.dens_col = keep(sp.density_col, np.int32)
    s.mass = keep(sp.mass, np.float64)
    s.atom_off = keep(sp.atom_off, np.int64); s.atom_E = keep(sp.atom_E, np.float64)
    s.atom_g = keep(sp.atom_g, np.float64)
    s.st_off = keep(sp.st_off, np.int64); s.st_E = keep(sp.st_E, np.float64)
    s.st_g = keep(sp.st_g, np.float64); s.st_sigma = keep(sp.st_sigma, np.float64)
    s.st_Lalt = keep(sp.st_Lalt, np.float64); s.st_nv = keep(sp.st_nv, np.int32)
    s.st_nj = keep(sp.st_nj, np.int32); s.st_vib_off = keep(sp.st_vib_off, np.int64)
    s.st_rot_off = keep(sp.st_rot_off, np.int64); s.vib_E = keep(sp.vib_E, np.float64)
    s.rot_E = keep(sp.rot_E, np.float64)
    return s


def lines_struct(ln, keep):
    s = _Lines()
    s.L = len(ln)
    for k in ["lam0", "A", "lamS0", "Eu_el", "Eu_v", "Eu_j", "gu", "El_el", "El_v", "El_j", "gl"]:
        setattr(s, k, keep(getattr(ln, k), np.float64))
    s.species = keep(ln.species, np.int32)
    return s


def cells_struct(cells, keep):
    s = _Cells()
    s.C = len(cells)
    s.Ttr = keep(cells.Ttr, np.float64); s.Tve = keep(cells.Tve, np.float64)
    n = np.ascontiguousarray(cells.n, np.float64)
    s.n = keep(n, np.float64)
    s.ncol = n.shape[1]; s.ne_col = cells.ne_col
    return s


def grid_struct(g):
    s = _Grid()
    s.lam_min, s.lam_max, s.n = float(g.lam_min), float(g.lam_max), int(g.n)
    return s


# ----------------------------------------------------------------------------
# steps of the path
# ----------------------------------------------------------------------------

# Sec. 2.2.1 full Lorentz broadening switches (see orc_set_broadening)
BROAD_STARK_IONIZE, BROAD_RESONANCE, BROAD_VDW = 1, 2, 4


def set_broadening(flags, E_ionize=None, column_mass=None):
    """Turns the optional Lorentz terms on for every later call (flags 0: the
    natural + Stark width with the lines' own Stark coefficients).  E_ionize:
    per radiating species, cm^-1; column_mass: per density column, g/mol (0
    for electrons)."""
    E = np.ascontiguousarray(E_ionize if E_ionize is not None else np.zeros(0), np.float64)
    M = np.ascontiguousarray(column_mass if column_mass is not None else np.zeros(0), np.float64)
    lib().orc_set_broadening(int(flags), E.shape[0], _p(E) if E.size else None, M.shape[0],
                             _p(M) if M.size else None)
    set_broadening._keep = (E, M)


def set_departures(ln_b=None, lev_u=None, lev_l=None):
    """Departure coefficients for every later call: ln_b [C][S][n_lev] (ln of
    N / N_Boltzmann per collisional-radiative level), lev_u / lev_l [L] the
    level index of each line's upper / lower level (-1: Boltzmann).  No
    argument: off."""
    if ln_b is None:
        lib().orc_set_departures(0, None, None, None)
        set_departures._keep = None
        return
    b = np.ascontiguousarray(ln_b, np.float64)
    u = np.ascontiguousarray(lev_u, np.int32)
    lo = np.ascontiguousarray(lev_l, np.int32)
    lib().orc_set_departures(b.shape[2], _p(b), _p(u), _p(lo))
    set_departures._keep = (b, u, lo)


def stark_coeff_ionize(lam0, Eu, Eion):
    return lib().orc_stark_coeff_ionize(float(lam0), float(Eu), float(Eion))


def oscillator_strength(lam0, A, gu, gl):
    return lib().orc_oscillator_strength(float(lam0), float(A), float(gu), float(gl))


def resonance_hwhm(lam0, A, gu, gl, N0):
    return lib().orc_resonance_hwhm(float(lam0), float(A), float(gu), float(gl), float(N0))


def vdw_hwhm(lam0, Ttr, N, M, No, Mo):
    return lib().orc_vdw_hwhm(float(lam0), float(Ttr), float(N), float(M), float(No), float(Mo))


def lnpref(problem):
    """ln N_s - ln Z_s, [C, S] (Sec. 2.1 Boltzmann distributions)."""
    keep = _Keep()
    sp = species_struct(problem.species, keep)
    ce = cells_struct(problem.cells, keep)
    out = np.zeros((len(problem.cells), sp.S))
    lib().orc_lnpref(ct.byref(sp), ct.byref(ce), _p(out))
    return out


def partition(problem, s, Ttr, Tve):
    keep = _Keep()
    sp = species_struct(problem.species, keep)
    return lib().orc_partition(ct.byref(sp), int(s), float(Ttr), float(Tve))


def line_states(problem, lnp, cell):
    """Per-line strengths (S_j, S_kappa) and HWHMs (G, L, V) in one cell."""
    keep = _Keep()
    sp = species_struct(problem.species, keep)
    ln = lines_struct(problem.lines, keep)
    ce = cells_struct(problem.cells, keep)
    L = len(problem.lines)
    out = [np.zeros(L) for _ in range(5)]
    lnp = np.ascontiguousarray(lnp, np.float64)
    lib().orc_line_states(ct.byref(sp), ct.byref(ln), ct.byref(ce), _p(lnp), int(cell), *[_p(o) for o in out])
    return dict(Sj=out[0], Sk=out[1], lamG=out[2], lamL=out[3], lamV=out[4])


def last_evaluations():
    """In-window (line, cell, grid point) triples the last spectral_coeffs
    call evaluated the profile at."""
    return int(lib().orc_last_evaluations())


def line_widths_all_cells(problem, lnp):
    """HWHMs (G, L, V) of every line in every cell, [C, L] each (for short
    line lists: one orc_line_states call per cell)."""
    keep = _Keep()
    sp = species_struct(problem.species, keep)
    ln = lines_struct(problem.lines, keep)
    ce = cells_struct(problem.cells, keep)
    C, L = len(problem.cells), len(problem.lines)
    lnp = np.ascontiguousarray(lnp, np.float64)
    out = [np.zeros((C, L)) for _ in range(5)]
    f = lib().orc_line_states
    for c in range(C):
        f(ct.byref(sp), ct.byref(ln), ct.byref(ce), _p(lnp), c, *[_p(o[c]) for o in out])
    return dict(lamG=out[2], lamL=out[3], lamV=out[4])


def spectral_coeffs(problem, lnp=None, k0=0, nk=None, with_abs=False):
    """kappa, j over grid points [k0, k0+nk) for every cell, [C, nk]."""
    if lnp is None:
        lnp = lnpref(problem)
    nk = problem.grid.n - k0 if nk is None else nk
    keep = _Keep()
    sp = species_struct(problem.species, keep)
    ln = lines_struct(problem.lines, keep)
    ce = cells_struct(problem.cells, keep)
    g = grid_struct(problem.grid)
    C = len(problem.cells)
    kap = np.zeros((C, nk)); em = np.zeros((C, nk))
    ab = np.zeros((C, nk)) if with_abs else None
    lnp = np.ascontiguousarray(lnp, np.float64)
    lib().orc_spectral_coeffs(ct.byref(sp), ct.byref(ln), ct.byref(ce), _p(lnp), ct.byref(g),
                              int(k0), int(nk), _p(kap), _p(em), _p(ab))
    return (kap, em, ab) if with_abs else (kap, em)


def coeffs_at(problem, cells_idx, ks, lnp=None):
    """kappa, j, sum|kappa terms| at individual (cell, k) points."""
    if lnp is None:
        lnp = lnpref(problem)
    keep = _Keep()
    sp = species_struct(problem.species, keep)
    ln = lines_struct(problem.lines, keep)
    ce = cells_struct(problem.cells, keep)
    g = grid_struct(problem.grid)
    pc = np.ascontiguousarray(cells_idx, np.int64)
    pk = np.ascontiguousarray(ks, np.int64)
    n = pc.shape[0]
    kap, em, ab = np.zeros(n), np.zeros(n), np.zeros(n)
    lnp = np.ascontiguousarray(lnp, np.float64)
    lib().orc_coeffs_at(ct.byref(sp), ct.byref(ln), ct.byref(ce), _p(lnp), ct.byref(g), n,
                        _p(pc), _p(pk), _p(kap), _p(em), _p(ab))
    return kap, em, ab


def grid_lambda(grid, k):
    g = grid_struct(grid)
    return lib().orc_grid_lambda(ct.byref(g), int(k))


def march(cells_far_to_near, ds, scale, kappa, emis, grid, k0=0, wall_start=False, T_wall=0.0,
          thin=THIN_FP64):
    """Intensity at the near end of one ray for every column of the tables."""
    cc = np.ascontiguousarray(cells_far_to_near, np.int64)
    ds = np.ascontiguousarray(ds, np.float64)
    kappa = np.ascontiguousarray(kappa, np.float64)
    emis = np.ascontiguousarray(emis, np.float64)
    nk = kappa.shape[1]
    out = np.zeros(nk)
    g = grid_struct(grid)
    lib().orc_march(cc.shape[0], _p(cc), _p(ds), float(scale), _p(kappa), _p(emis), nk, nk,
                    int(bool(wall_start)), float(T_wall), ct.byref(g), int(k0), float(thin), _p(out))
    return out


def march_nodes(nodes_far_to_near, ds, kappa, emis, grid, k0=0, wall_start=False, T_wall=0.0, thin=THIN_FP64):
    """Intensity at the near end of one LOS whose kappa / j are given at its
    len(ds) + 1 nodes (rows of the tables), for every column."""
    nn = np.ascontiguousarray(nodes_far_to_near, np.int64)
    ds = np.ascontiguousarray(ds, np.float64)
    kappa = np.ascontiguousarray(kappa, np.float64)
    emis = np.ascontiguousarray(emis, np.float64)
    assert nn.shape[0] == ds.shape[0] + 1
    nk = kappa.shape[1]
    out = np.zeros(nk)
    g = grid_struct(grid)
    lib().orc_march_nodes(ds.shape[0], _p(nn), _p(ds), _p(kappa), _p(emis), nk, nk, int(bool(wall_start)),
                          float(T_wall), ct.byref(g), int(k0), float(thin), _p(out))
    return out


def segment_coeffs(kappa, ds, thin=THIN_FP64):
    """(far, near) coefficients of one march segment."""
    a, b = ct.c_double(), ct.c_double()
    lib().orc_segment_coeffs(float(kappa), float(ds), float(thin), ct.byref(a), ct.byref(b))
    return a.value, b.value


def spectral_integral(q_lambda, grid, k0=0):
    q = np.ascontiguousarray(q_lambda, np.float64)
    g = grid_struct(grid)
    return lib().orc_spectral_integral(_p(q), ct.byref(g), int(k0), q.shape[0])


def axisym_segments(geo, x0, direction, max_seg=100_000):
    """(cells, ds) of one ray from the surface point x0, far boundary first."""
    xf = np.ascontiguousarray(geo.xf, np.float64)
    rf = np.ascontiguousarray(geo.rf, np.float64)
    cell = np.zeros(max_seg, np.int64)
    ds = np.zeros(max_seg)
    dx, dn, dt = direction
    m = lib().orc_axisym_segments(_p(xf), xf.shape[0] - 1, _p(rf), rf.shape[0] - 1, float(x0),
                                  float(geo.r_body), float(dx), float(dn), float(dt), max_seg,
                                  _p(cell), _p(ds))
    if m < 0:
        raise RuntimeError("segment buffer too small")
    return cell[:m].copy(), ds[:m].copy()


def hemisphere_directions(geo):
    """Ray directions about the outward normal and their flux weights
    w_m mu_m dphi (Sec. 2.2.3 solid-angle integral with mu = cos(polar))."""
    dphi = 2.0 * np.pi / geo.n_phi
    dirs, wts = [], []
    for m, mu in enumerate(geo.mu):
        st = np.sqrt(1.0 - mu * mu)
        for a in range(geo.n_phi):
            psi = (a + 0.5) * dphi
            dirs.append((st * np.cos(psi), mu, st * np.sin(psi)))
            wts.append(geo.wmu[m] * mu * dphi)
    return dirs, np.asarray(wts)


# ----------------------------------------------------------------------------
# whole solves
# ----------------------------------------------------------------------------

def solve_slab(problem, k0=0, nk=None, coeffs=None, thin=THIN_FP64):
    """Uniform / stratified slab: kappa, j; intensities along the normal ray
    and each direction mu_m (path ds/mu); tangent-slab spectral flux
    q_lambda = 2 pi sum_m w_m mu_m I(mu_m); wall flux q (W/cm^2)."""
    geo = problem.geometry
    nk = problem.grid.n - k0 if nk is None else nk
    if coeffs is None:
        lnp = lnpref(problem)
        kap, em = spectral_coeffs(problem, lnp, k0, nk)
    else:
        lnp = None
        kap, em = coeffs
    order = np.asarray(geo.cell_order, np.int64)
    out = dict(kappa=kap, emis=em, lnpref=lnp)
    I_mu = np.stack([march(order, geo.dx, 1.0 / mu, kap, em, problem.grid, k0, geo.wall_start, geo.T_wall,
                           thin) for mu in geo.mu])
    out["I_mu"] = I_mu
    if geo.normal_ray:
        out["I_normal"] = march(order, geo.dx, 1.0, kap, em, problem.grid, k0, geo.wall_start, geo.T_wall,
                                thin)
    w = 2.0 * np.pi * np.asarray(geo.wmu) * np.asarray(geo.mu)
    qlam = (w[:, None] * I_mu).sum(axis=0)
    out["q_lambda"] = qlam
    out["q"] = spectral_integral(qlam, problem.grid, k0)
    return out


def solve_axisym_points(problem, points, kappa, emis, k0=0, thin=THIN_FP64, rows=None):
    """Afterbody rays of the given surface points over the columns of the
    (kappa, emis) tables (which cover grid points [k0, k0 + ncol)):
    q_lambda[p] = sum_rays w_m mu_m dphi I, and the chunk's flux part.
    Row c of the tables belongs to cell c, or, with `rows` (an array over the
    grid's cells), to the cells c with rows[c] = that row (tables of only the
    cells the rays cross)."""
    geo = problem.geometry
    dirs, wts = hemisphere_directions(geo)
    qlam = np.zeros((len(points), kappa.shape[1]))
    for ip, p in enumerate(points):
        for d, w in zip(dirs, wts):
            cells, ds = axisym_segments(geo, geo.surf_x[p], d)
            if rows is not None:
                cells = rows[cells]
            qlam[ip] += w * march(cells, ds, 1.0, kappa, emis, problem.grid, k0, False, 0.0, thin)
    q = np.array([spectral_integral(qlam[i], problem.grid, k0) for i in range(len(points))])
    return qlam, q
