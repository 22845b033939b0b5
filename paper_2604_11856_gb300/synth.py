"""Seeded synthetic inputs shaped after the paper's workloads.

This module only draws data: line lists, level tables, flowfields and ray-set
geometry specifications.  It contains none of the radiation method's
arithmetic (no populations, no line strengths, widths or profiles, no
transport).  Both the CPU oracle and the CUDA path consume its output.

The paper's own inputs (the Fire II flowfield, NIST / TOPbase / Liang et al.
spectroscopic databases) are not available, so every workload is synthetic.
The species database the paper builds with Python utilities (Sec. 2.3, first
layer: energy levels and transition probabilities) is stood in for by the
generators below:

* atomic lines (Sec. 2.2.1) with centres, Einstein coefficients, upper/lower
  energies, degeneracies and Stark coefficients drawn from fixed distributions;
* diatomic rovibronic lines (Sec. 2.2.2) built from randomly drawn molecular
  constants with the energy expressions of Sec. 2.2.2 (vibrational ladder and
  Hund's case (a) rotational ladder), Hoenl-London factors of Table 4 and a
  proportional form of the molecular Einstein coefficient;
* cell states (two-temperature gas, 11 air species) for a uniform slab, a
  stagnation line and an axisymmetric afterbody.

Energies are in cm^-1, wavelengths in nm, number densities in cm^-3.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

EV_TO_CM = 8065.544  # eV -> cm^-1 conversion used for the drawn energies

# Flowfield species, in the column order of the cell density array.
FLOW_SPECIES = ["N2", "O2", "NO", "N", "O", "N2+", "O2+", "NO+", "N+", "O+", "e-"]
NE_COL = 10

# Radiating species, in the order of every per-species array.
RAD_SPECIES = ["N", "O", "N+", "O+", "N2", "O2", "NO", "N2+"]
RAD_KIND = np.array([0, 0, 0, 0, 1, 1, 1, 1], dtype=np.int32)  # 0 atom, 1 diatomic
RAD_MASS = np.array([14.0, 16.0, 14.0, 16.0, 28.0, 32.0, 30.0, 28.0])  # g/mol
RAD_DENSITY_COL = np.array([FLOW_SPECIES.index(s) for s in RAD_SPECIES], dtype=np.int32)
ATOM_GROUND_G = {"N": 4.0, "O": 9.0, "N+": 9.0, "O+": 4.0}  # ground-term weights
# Ionisation energies of the radiating species, cm^-1 (N I, O I, N II, O II
# from their ground terms; molecules 0: the full-broadening options use atoms
# only) and molar masses of the flow columns, g/mol (electrons 0), for the
# optional Stark-from-ionisation-gap and van der Waals widths (Sec. 2.2.1).
RAD_E_IONIZE = np.array([117225.7, 109837.02, 238750.2, 283270.9, 0.0, 0.0, 0.0, 0.0])
FLOW_MASS = np.array([28.0, 32.0, 30.0, 14.0, 16.0, 28.0, 32.0, 30.0, 14.0, 16.0, 0.0])

# Molecular electronic states: (name, Lambda).  The first entry is the ground state.
MOL_STATES = {
    "N2": [("X", 0), ("A", 0), ("B", 1), ("C", 1)],
    "O2": [("X", 0), ("B", 0)],
    "NO": [("X", 1), ("A", 0), ("B", 1)],
    "N2+": [("X", 0), ("B", 0)],
}
MOL_SIGMA = {"N2": 2.0, "O2": 2.0, "NO": 1.0, "N2+": 2.0}  # homo- / heteronuclear
# Band systems (Table 8 names): (name, species, upper, lower, spin multiplicity)
MOL_SYSTEMS = [
    ("N2 1+", "N2", "B", "A", 3),
    ("N2 2+", "N2", "C", "B", 3),
    ("N2+ 1-", "N2+", "B", "X", 2),
    ("NO gamma", "NO", "A", "X", 2),
    ("NO beta", "NO", "B", "X", 2),
    ("O2 SR", "O2", "B", "X", 3),
]
N_V = 11      # vibrational quantum numbers 0..10
N_J = 152     # rotational quantum numbers 0..151 in the partition function
J_U_MAX = 150  # upper-level J range of the line list


@dataclass
class Species:
    """Radiating-species database: atomic level lists and molecular ladders."""
    names: list
    kind: np.ndarray          # int32 [S]
    mass: np.ndarray          # f64 [S] g/mol
    density_col: np.ndarray   # int32 [S] column in the cell density array
    atom_off: np.ndarray      # int64 [S+1] level ranges (empty for molecules)
    atom_E: np.ndarray        # f64 [n_lev] cm^-1
    atom_g: np.ndarray        # f64 [n_lev]
    st_off: np.ndarray        # int64 [S+1] electronic-state ranges (empty for atoms)
    st_E: np.ndarray          # f64 [n_st] electronic term energy, cm^-1
    st_g: np.ndarray          # f64 [n_st] electronic degeneracy
    st_sigma: np.ndarray      # f64 [n_st] symmetry factor
    st_Lalt: np.ndarray       # f64 [n_st, 2] line-alternation factor for even / odd J
    st_nv: np.ndarray         # int32 [n_st] vibrational levels
    st_nj: np.ndarray         # int32 [n_st] rotational levels per vibrational level
    st_vib_off: np.ndarray    # int64 [n_st] offset into vib_E
    st_rot_off: np.ndarray    # int64 [n_st] offset into rot_E (nv*nj entries per state)
    vib_E: np.ndarray         # f64 vibrational energies E_V, cm^-1
    rot_E: np.ndarray         # f64 rotational energies E_J(V), cm^-1, [V][J] per state


@dataclass
class Lines:
    """Line list, sorted by centre wavelength.  Level weights g are the
    statistical weights that multiply the Boltzmann factor of the level."""
    lam0: np.ndarray      # f64 [L] nm
    A: np.ndarray         # f64 [L] s^-1
    lamS0: np.ndarray     # f64 [L] nm, Stark HWHM at N_e = 1e16 cm^-3, T = 1e4 K
    species: np.ndarray   # int32 [L] radiating-species index
    Eu_el: np.ndarray
    Eu_v: np.ndarray
    Eu_j: np.ndarray
    gu: np.ndarray
    El_el: np.ndarray
    El_v: np.ndarray
    El_j: np.ndarray
    gl: np.ndarray

    def __len__(self):
        return int(self.lam0.shape[0])


@dataclass
class Cells:
    Ttr: np.ndarray   # f64 [C] K
    Tve: np.ndarray   # f64 [C] K
    n: np.ndarray     # f64 [C, 11] cm^-3 (columns FLOW_SPECIES)
    ne_col: int = NE_COL

    def __len__(self):
        return int(self.Ttr.shape[0])


@dataclass
class Grid:
    lam_min: float
    lam_max: float
    n: int


@dataclass
class SlabGeometry:
    """Plane-parallel slab: cells listed far -> near (wall last)."""
    cell_order: np.ndarray   # int64 [m] cell indices, far boundary first
    dx: np.ndarray           # f64 [m] cell thickness along the normal, cm
    mu: np.ndarray           # f64 [n_mu] Gauss-Legendre nodes on (0, 1)
    wmu: np.ndarray          # f64 [n_mu] weights, sum 1
    normal_ray: bool = True  # also march mu = 1 (intensity output only)
    wall_start: bool = False # far end is a wall at T_wall (else far field, I = 0)
    T_wall: float = 0.0


@dataclass
class AxisymGeometry:
    """Rectilinear (x, r) grid around a cylinder of radius r_body; surface
    points on r = r_body; rays on the outward hemisphere."""
    xf: np.ndarray      # f64 [nx+1] x faces, cm
    rf: np.ndarray      # f64 [nr+1] r faces, cm (rf[0] = r_body)
    surf_x: np.ndarray  # f64 [P]
    r_body: float
    mu: np.ndarray      # f64 [n_mu] polar-cosine nodes about the outward normal
    wmu: np.ndarray     # f64 [n_mu]
    n_phi: int          # azimuths at midpoints of 2*pi/n_phi


@dataclass
class Problem:
    name: str
    species: Species
    lines: Lines
    cells: Cells
    grid: Grid
    geometry: object
    chunk: int = 0   # spectral chunk length (0: whole grid)
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# distributions
# ----------------------------------------------------------------------------

def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def gauss_legendre_01(n):
    """Gauss-Legendre nodes and weights mapped to (0, 1); weights sum to 1."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def atomic_lines(rng, n_lines, species_idx):
    """Atomic lines with the common distribution: centres log-uniform
    50-1000 nm, A log-uniform 1e4-1e9 s^-1, E_u uniform 10-14.5 eV,
    E_l = max(0, E_u - 1e7/lam0), integer g in [2, 20], Stark HWHM at
    N_e = 1e16 log-uniform 1e-4-1e-1 nm.  `species_idx` is an int array of
    length n_lines."""
    lam0 = _loguniform(rng, 50.0, 1000.0, n_lines)
    A = _loguniform(rng, 1e4, 1e9, n_lines)
    Eu = rng.uniform(10.0, 14.5, n_lines) * EV_TO_CM
    El = np.maximum(0.0, Eu - 1e7 / lam0)
    gu = rng.integers(2, 21, n_lines).astype(np.float64)
    gl = rng.integers(2, 21, n_lines).astype(np.float64)
    lamS0 = _loguniform(rng, 1e-4, 1e-1, n_lines)
    z = np.zeros(n_lines)
    return dict(lam0=lam0, A=A, lamS0=lamS0, species=np.asarray(species_idx, np.int32),
                Eu_el=Eu, Eu_v=z.copy(), Eu_j=z.copy(), gu=gu,
                El_el=El, El_v=z.copy(), El_j=z.copy(), gl=gl)


def _atom_levels(lines, s):
    """Level set of atomic species s: ground (E = 0, ground-term weight)
    together with every distinct (E, g) of the lines' upper levels and of
    the lower levels with E_l > 0."""
    m = lines["species"] == s
    E = np.concatenate([lines["Eu_el"][m], lines["El_el"][m][lines["El_el"][m] > 0]])
    g = np.concatenate([lines["gu"][m], lines["gl"][m][lines["El_el"][m] > 0]])
    pairs = np.unique(np.stack([E, g], axis=1), axis=0)
    g0 = ATOM_GROUND_G[RAD_SPECIES[s]]
    E = np.concatenate([[0.0], pairs[:, 0]])
    g = np.concatenate([[g0], pairs[:, 1]])
    return E, g


def _hl_factors(kind, Ju, Lu):
    """Hoenl-London factors of Table 4 (Hund's case (a)) for branches
    P (J_l = J_u + 1), Q (J_l = J_u), R (J_l = J_u - 1).
    kind: 'SS' (Lambda_u = Lambda_l = 0), 'DL0' (Delta Lambda = 0, Lambda > 0),
    'DL+' (Lambda_u = Lambda_l + 1), 'DL-' (Lambda_u = Lambda_l - 1).
    Entries that are not defined (J below Lambda) are returned as 0."""
    J = Ju.astype(np.float64)
    L = float(Lu)
    with np.errstate(divide="ignore", invalid="ignore"):
        if kind == "SS":
            P = J + 1.0
            Q = np.zeros_like(J)
            R = J.copy()
        elif kind == "DL0":
            P = (J + 1 + L) * (J + 1 - L) / (J + 1)
            Q = (2 * J + 1) * L * L / (J * (J + 1))
            R = (J + L) * (J - L) / J
        elif kind == "DL+":
            P = (J + 1 - L) * (J + 2 - L) / (2 * (J + 1))
            Q = (J + L) * (J + 1 - L) * (2 * J + 1) / (2 * J * (J + 1))
            R = (J + L) * (J - 1 + L) / (2 * J)
        elif kind == "DL-":
            P = (J + 1 + L) * (J + 2 + L) / (2 * (J + 1))
            Q = (J - L) * (J + 1 + L) * (2 * J + 1) / (2 * J * (J + 1))
            R = (J - L) * (J - 1 - L) / (2 * J)
        else:
            raise ValueError(kind)
    out = np.stack([P, Q, R], axis=1)
    out[~np.isfinite(out)] = 0.0
    return np.maximum(out, 0.0)


def _hl_kind(Lu, Ll):
    if Lu == 0 and Ll == 0:
        return "SS"
    if Lu == Ll:
        return "DL0"
    return "DL+" if Lu == Ll + 1 else "DL-"


def _mol_state_constants(rng):
    we = rng.uniform(1000.0, 2400.0)
    wexe = we / rng.uniform(60.0, 120.0)
    Be = rng.uniform(1.0, 2.0)
    ae = rng.uniform(0.01, 0.02)
    return dict(we=we, wexe=wexe, weye=0.0, Be=Be, ae=ae, De=5e-6, be=0.0,
                g=float(rng.integers(2, 7)), spin_a=rng.uniform(5.0, 40.0))


def _vib_energy(c, v):
    x = v + 0.5
    return c["we"] * x - c["wexe"] * x * x + c["weye"] * x ** 3


def _rot_energy(c, v, J):
    Bv = c["Be"] - c["ae"] * (v + 0.5)
    Dv = c["De"] + c["be"] * (v + 0.5)
    JJ = J * (J + 1.0)
    return Bv * JJ - Dv * JJ * JJ


def molecular_database(rng, n_target):
    """Six band systems with v', v'' in 0..10, J_u in 0..150, P/Q/R branches
    (Table 4 columns chosen by the states' Lambda) and one sub-band per spin
    component (S_multi = 1/multiplicity).  Lines with centres outside
    [50, 2000] nm are dropped and a seeded subsample of exactly n_target
    lines is kept.  Returns (lines dict, per-species state tables)."""
    consts = {sp: [_mol_state_constants(rng) for _ in st] for sp, st in MOL_STATES.items()}
    Te = {sp: [None] * len(st) for sp, st in MOL_STATES.items()}
    for sp in MOL_STATES:
        Te[sp][0] = 0.0
    Te["N2"][1] = rng.uniform(40000.0, 60000.0)   # N2 A: not an upper state of any system
    origins = {}
    for name, sp, up, lo, _m in MOL_SYSTEMS:
        iu = [s[0] for s in MOL_STATES[sp]].index(up)
        il = [s[0] for s in MOL_STATES[sp]].index(lo)
        lam_org = rng.uniform(150.0, 1200.0)
        origins[name] = lam_org
        cu, cl = consts[sp][iu], consts[sp][il]
        # term energy of the upper state so that the (0,0) band origin is lam_org
        Te[sp][iu] = Te[sp][il] + _vib_energy(cl, 0) - _vib_energy(cu, 0) + 1e7 / lam_org

    rad_index = {s: i for i, s in enumerate(RAD_SPECIES)}
    cols = {k: [] for k in ["lam0", "A", "species", "Eu_el", "Eu_v", "Eu_j", "gu",
                            "El_el", "El_v", "El_j", "gl"]}
    Ju_all = np.arange(0, J_U_MAX + 1, dtype=np.float64)
    for name, sp, up, lo, mult in MOL_SYSTEMS:
        names = [s[0] for s in MOL_STATES[sp]]
        iu, il = names.index(up), names.index(lo)
        Lu, Ll = MOL_STATES[sp][iu][1], MOL_STATES[sp][il][1]
        cu, cl = consts[sp][iu], consts[sp][il]
        sig = MOL_SIGMA[sp]
        hl = _hl_factors(_hl_kind(Lu, Ll), Ju_all, Lu)         # [J, 3]
        Jl_all = np.stack([Ju_all + 1, Ju_all, Ju_all - 1], axis=1)
        ok = (hl > 0) & (Jl_all >= Ll) & (Ju_all[:, None] >= Lu)
        for vu in range(N_V):
            for vl in range(N_V):
                A_band = _loguniform(rng, 1e5, 1e7, 1)[0]
                Ebu = Te[sp][iu] + _vib_energy(cu, vu)
                Ebl = Te[sp][il] + _vib_energy(cl, vl)
                if Ebu - Ebl <= 0.0:
                    continue
                lam_band = 1e7 / (Ebu - Ebl)
                for k in range(mult):
                    off_u = cu["spin_a"] * (k - 0.5 * (mult - 1))
                    off_l = cl["spin_a"] * (k - 0.5 * (mult - 1))
                    for b in range(3):
                        sel = ok[:, b]
                        Ju = Ju_all[sel]
                        Jl = Jl_all[sel, b]
                        EJu = _rot_energy(cu, vu, Ju) + off_u
                        EJl = _rot_energy(cl, vl, Jl) + off_l
                        dE = (Ebu + EJu) - (Ebl + EJl)
                        good = dE > 0
                        lam0 = np.full(Ju.shape, np.inf)
                        lam0[good] = 1e7 / dE[good]
                        keep = good & (lam0 >= 50.0) & (lam0 <= 2000.0)
                        if not np.any(keep):
                            continue
                        Ju, Jl, EJu, EJl, lam0 = Ju[keep], Jl[keep], EJu[keep], EJl[keep], lam0[keep]
                        S = hl[sel, b][keep]
                        A = A_band * S / (2 * Ju + 1) * (lam_band / lam0) ** 3
                        n = Ju.shape[0]
                        cols["lam0"].append(lam0)
                        cols["A"].append(A)
                        cols["species"].append(np.full(n, rad_index[sp], np.int32))
                        cols["Eu_el"].append(np.full(n, Te[sp][iu]))
                        cols["Eu_v"].append(np.full(n, _vib_energy(cu, vu)))
                        cols["Eu_j"].append(EJu)
                        cols["gu"].append(cu["g"] * (1.0 / mult) * (2 * Ju + 1) / sig)
                        cols["El_el"].append(np.full(n, Te[sp][il]))
                        cols["El_v"].append(np.full(n, _vib_energy(cl, vl)))
                        cols["El_j"].append(EJl)
                        cols["gl"].append(cl["g"] * (1.0 / mult) * (2 * Jl + 1) / sig)
    pool = {k: np.concatenate(v) for k, v in cols.items()}
    n_pool = pool["lam0"].shape[0]
    if n_pool < n_target:
        raise RuntimeError(f"molecular pool {n_pool} < {n_target}")
    pick = np.sort(rng.choice(n_pool, size=n_target, replace=False))
    lines = {k: v[pick] for k, v in pool.items()}
    lines["lamS0"] = np.zeros(n_target)   # Doppler-dominated: natural width only
    tables = {}
    for sp, st in MOL_STATES.items():
        rows = []
        for i, (_nm, _L) in enumerate(st):
            c = consts[sp][i]
            v = np.arange(N_V, dtype=np.float64)
            J = np.arange(N_J, dtype=np.float64)
            rows.append(dict(E=Te[sp][i], g=c["g"], sigma=MOL_SIGMA[sp], Lalt=(1.0, 1.0),
                             vib=_vib_energy(c, v),
                             rot=np.stack([_rot_energy(c, vv, J) for vv in range(N_V)])))
        tables[sp] = rows
    return lines, tables, dict(pool=int(n_pool), origins=origins)


def _species_db(atom_levels, mol_tables):
    S = len(RAD_SPECIES)
    atom_off = [0]
    aE, ag = [], []
    st_off = [0]
    st = dict(E=[], g=[], sigma=[], Lalt=[], nv=[], nj=[], vib_off=[], rot_off=[])
    vibE, rotE = [], []
    nvib = nrot = 0
    for s, name in enumerate(RAD_SPECIES):
        if RAD_KIND[s] == 0:
            E, g = atom_levels.get(s, (np.zeros(0), np.zeros(0)))
            aE.append(E)
            ag.append(g)
            atom_off.append(atom_off[-1] + E.shape[0])
            st_off.append(st_off[-1])
        else:
            atom_off.append(atom_off[-1])
            rows = mol_tables.get(name, [])
            for r in rows:
                st["E"].append(r["E"]); st["g"].append(r["g"]); st["sigma"].append(r["sigma"])
                st["Lalt"].append(r["Lalt"])
                nv, nj = r["rot"].shape
                st["nv"].append(nv); st["nj"].append(nj)
                st["vib_off"].append(nvib); st["rot_off"].append(nrot)
                vibE.append(r["vib"]); rotE.append(r["rot"].ravel())
                nvib += nv; nrot += nv * nj
            st_off.append(st_off[-1] + len(rows))
    cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0)
    return Species(
        names=list(RAD_SPECIES), kind=RAD_KIND.copy(), mass=RAD_MASS.copy(),
        density_col=RAD_DENSITY_COL.copy(),
        atom_off=np.asarray(atom_off, np.int64), atom_E=cat(aE), atom_g=cat(ag),
        st_off=np.asarray(st_off, np.int64), st_E=np.asarray(st["E"], np.float64),
        st_g=np.asarray(st["g"], np.float64), st_sigma=np.asarray(st["sigma"], np.float64),
        st_Lalt=np.asarray(st["Lalt"], np.float64).reshape(-1, 2),
        st_nv=np.asarray(st["nv"], np.int32), st_nj=np.asarray(st["nj"], np.int32),
        st_vib_off=np.asarray(st["vib_off"], np.int64), st_rot_off=np.asarray(st["rot_off"], np.int64),
        vib_E=cat(vibE), rot_E=cat(rotE))


def _merge_lines(parts):
    keys = ["lam0", "A", "lamS0", "species", "Eu_el", "Eu_v", "Eu_j", "gu",
            "El_el", "El_v", "El_j", "gl"]
    cat = {k: np.concatenate([p[k] for p in parts]) for k in keys}
    order = np.argsort(cat["lam0"], kind="stable")
    cat = {k: np.ascontiguousarray(v[order]) for k, v in cat.items()}
    cat["species"] = cat["species"].astype(np.int32)
    return Lines(**cat)


def composition(Tve, n_total):
    """Eleven-species number densities from a smooth dissociation /
    ionisation rule driven by T_ve (a stand-in for a CFD solution):
    delta = 1/(1+exp(-(T-7000)/1000)), iota = 0.1/(1+exp(-(T-12000)/1500));
    molecules (1-delta)(1-iota) n as N2:O2:NO = 0.78:0.20:0.02; atoms
    delta(1-iota) n as N:O = 0.79:0.21; ions iota n/2 as
    N+:O+:N2+:O2+:NO+ = 0.70:0.20:0.05:0.02:0.03; electrons iota n/2."""
    Tve = np.asarray(Tve, np.float64)
    n_total = np.broadcast_to(np.asarray(n_total, np.float64), Tve.shape)
    d = 1.0 / (1.0 + np.exp(-(Tve - 7000.0) / 1000.0))
    io = 0.1 / (1.0 + np.exp(-(Tve - 12000.0) / 1500.0))
    n = np.zeros(Tve.shape + (11,))
    mol = (1 - d) * (1 - io) * n_total
    atm = d * (1 - io) * n_total
    ion = io * n_total / 2
    col = FLOW_SPECIES.index
    n[..., col("N2")] = 0.78 * mol
    n[..., col("O2")] = 0.20 * mol
    n[..., col("NO")] = 0.02 * mol
    n[..., col("N")] = 0.79 * atm
    n[..., col("O")] = 0.21 * atm
    n[..., col("N+")] = 0.70 * ion
    n[..., col("O+")] = 0.20 * ion
    n[..., col("N2+")] = 0.05 * ion
    n[..., col("O2+")] = 0.02 * ion
    n[..., col("NO+")] = 0.03 * ion
    n[..., col("e-")] = ion
    return n


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def uniform_slab(seed=1000, n_lines=1500, n_cells=20, n_grid=200_000, lam=(50.0, 1000.0),
                 T=10000.0, nN=1e16, nO=1e16, ne=1e15, dx=0.25, n_mu=16):
    """Plain uniform slab: one gas state repeated over n_cells cells of
    thickness dx; 1,500 atomic lines alternating N / O; one normal ray and a
    tangent-slab flux with n_mu Gauss-Legendre directions."""
    rng = np.random.default_rng(seed)
    sp = np.where(np.arange(n_lines) % 2 == 0, 0, 1)
    al = atomic_lines(rng, n_lines, sp)
    lines = _merge_lines([al])
    raw = {k: getattr(lines, k) for k in ["species", "Eu_el", "El_el", "gu", "gl"]}
    levels = {s: _atom_levels(raw, s) for s in range(4)}
    species = _species_db(levels, {})
    n = np.zeros((n_cells, 11))
    n[:, FLOW_SPECIES.index("N")] = nN
    n[:, FLOW_SPECIES.index("O")] = nO
    n[:, NE_COL] = ne
    cells = Cells(Ttr=np.full(n_cells, T), Tve=np.full(n_cells, T), n=n)
    mu, w = gauss_legendre_01(n_mu)
    geo = SlabGeometry(cell_order=np.arange(n_cells, dtype=np.int64), dx=np.full(n_cells, dx),
                       mu=mu, wmu=w)
    return Problem("uniform_slab", species, lines, cells, Grid(lam[0], lam[1], n_grid), geo,
                   meta=dict(seed=seed))


def stagnation_profiles(x):
    """Stagnation-line temperatures: T_tr rises from 2000 K to a 30000 K peak
    at x = 0.2 cm then relaxes towards 10000 K; T_ve lags it (peak 15000 K
    at x = 0.6 cm)."""
    x = np.asarray(x, np.float64)
    Ttr = np.where(x < 0.2, 2000.0 + 28000.0 * (x / 0.2) ** 2,
                   10000.0 + 20000.0 * np.exp(-(x - 0.2) / 0.5))
    Tve = np.where(x < 0.6, 2000.0 + 13000.0 * (1.0 - (1.0 - x / 0.6) ** 2),
                   10000.0 + 5000.0 * np.exp(-(x - 0.6) / 0.5))
    return Ttr, Tve


def _air_lines(rng, n_atomic, n_molecular):
    per = n_atomic // 4
    sp = np.repeat(np.arange(4), per)
    al = atomic_lines(rng, per * 4, sp)
    levels = {s: _atom_levels(al, s) for s in range(4)}
    if n_molecular > 0:
        ml, tables, info = molecular_database(rng, n_molecular)
        parts = [al, ml]
    else:
        tables, info = {}, {}
        parts = [al]
    lines = _merge_lines(parts)
    species = _species_db(levels, tables)
    return lines, species, info


def stagnation_line(seed=1001, n_cells=200, length=3.0, n_atomic=20_000, n_molecular=300_000,
                    n_grid=1_000_000, lam=(50.0, 2000.0), n_total=1e17, n_mu=16):
    """Two-temperature stagnation line: n_cells cells over `length` cm, far
    field at x = 0, wall at x = length; 11 species from the composition rule;
    20,000 atomic (N, O, N+, O+) and 300,000 molecular lines."""
    rng = np.random.default_rng(seed)
    lines, species, info = _air_lines(rng, n_atomic, n_molecular)
    dx = length / n_cells
    x = (np.arange(n_cells) + 0.5) * dx
    Ttr, Tve = stagnation_profiles(x)
    cells = Cells(Ttr=Ttr, Tve=Tve, n=composition(Tve, n_total))
    mu, w = gauss_legendre_01(n_mu)
    geo = SlabGeometry(cell_order=np.arange(n_cells, dtype=np.int64), dx=np.full(n_cells, dx),
                       mu=mu, wmu=w)
    return Problem("stagnation_line", species, lines, cells, Grid(lam[0], lam[1], n_grid), geo,
                   meta=dict(seed=seed, **info))


def afterbody_fields(xc, yc):
    """Smooth afterbody temperature / density fields on cell centres
    (x along the axis, y = r - r_body), with a recirculation blob centred
    at (40, 15) cm of radius 30 cm where T_tr spans 3000-8000 K;
    T_ve >= T_tr outside the blob; total density log-linear from 1e17
    (x = 0) to 1e15 (x = 200 cm)."""
    X, Y = np.meshgrid(xc, yc, indexing="ij")
    base = 2500.0 + 7500.0 * np.exp(-X / 60.0) * (1.0 - 0.3 * Y / 150.0)
    rho = np.sqrt((X - 40.0) ** 2 + (Y - 15.0) ** 2) / 30.0
    w = np.clip(1.0 - rho ** 2, 0.0, None) ** 2
    blob = 8000.0 - 5000.0 * np.clip(rho, 0.0, 1.0) ** 2
    Ttr = base * (1.0 - w) + blob * w
    Tve = Ttr + (200.0 + 2000.0 * np.exp(-X / 80.0)) * (1.0 - w)
    ntot = 10.0 ** (17.0 - 2.0 * X / 200.0)
    return Ttr, Tve, ntot


def afterbody(seed=1002, nx=400, nr=200, x_len=200.0, r_body=33.5, r_len=150.0,
              n_points=200, n_mu=16, n_phi=32, n_atomic=20_000, n_molecular=300_000,
              n_grid=1_000_000, lam=(50.0, 2000.0), chunk=65536, lines_from=None):
    """Axisymmetric afterbody stand-in: nx x nr rectilinear cells in (x, r)
    around a cylinder of radius r_body; surface points uniform in
    x in [1, x_len - 1]; n_mu x n_phi rays per point; the stagnation-line
    line lists (pass `lines_from` to share an existing problem's lists)."""
    rng = np.random.default_rng(seed)
    if lines_from is None:
        lines, species, info = _air_lines(np.random.default_rng(1001), n_atomic, n_molecular)
    else:
        lines, species, info = lines_from.lines, lines_from.species, {}
    xf = np.linspace(0.0, x_len, nx + 1)
    rf = np.linspace(r_body, r_body + r_len, nr + 1)
    xc = 0.5 * (xf[1:] + xf[:-1])
    yc = 0.5 * (rf[1:] + rf[:-1]) - r_body
    Ttr, Tve, ntot = afterbody_fields(xc, yc)
    cells = Cells(Ttr=Ttr.ravel(), Tve=Tve.ravel(), n=composition(Tve.ravel(), ntot.ravel()))
    surf_x = np.linspace(1.0, x_len - 1.0, n_points)
    mu, w = gauss_legendre_01(n_mu)
    geo = AxisymGeometry(xf=xf, rf=rf, surf_x=surf_x, r_body=r_body, mu=mu, wmu=w, n_phi=n_phi)
    _ = rng  # the afterbody draws nothing beyond the shared line lists
    return Problem("afterbody", species, lines, cells, Grid(lam[0], lam[1], n_grid), geo,
                   chunk=chunk, meta=dict(seed=seed, nx=nx, nr=nr, **info))


def subset_lines(lines: Lines, idx):
    idx = np.sort(np.asarray(idx, dtype=np.int64))
    return Lines(**{k: np.ascontiguousarray(getattr(lines, k)[idx]) for k in Lines.__dataclass_fields__})


def batch_slabs(seed=1003, n_solves=64, pool=None, iid_cells=False, scale=1.0):
    """Uneven uniform-slab solves: cells uniform-int [20, 2000], spectral
    points log-uniform [1e5, 2e6] on [50, 2000] nm, atomic lines
    uniform-int [1e3, 5e4] and molecular lines uniform-int [0, 3e5] drawn
    from the stagnation-line pools, T_tr, T_ve uniform [5000, 30000] K,
    total density log-uniform [1e14, 1e18] cm^-3, slab thickness 5 cm.
    `scale` < 1 shrinks every size (for quick tests)."""
    rng = np.random.default_rng(seed)
    if pool is None:
        pool = _air_lines(np.random.default_rng(1001), 20_000, 300_000)
    lines_all, species, _info = pool
    atom_idx = np.nonzero(lines_all.species < 4)[0]
    mol_idx = np.nonzero(lines_all.species >= 4)[0]
    out = []
    for i in range(n_solves):
        C = max(2, int(rng.integers(20, 2001) * scale))
        K = max(1000, int(_loguniform(rng, 1e5, 2e6, 1)[0] * scale))
        na = max(10, int(rng.integers(1000, 50_001) * scale))
        nm = int(rng.integers(0, 300_001) * scale)
        na = min(na, atom_idx.shape[0]); nm = min(nm, mol_idx.shape[0])
        pick = np.concatenate([rng.choice(atom_idx, na, replace=False),
                               rng.choice(mol_idx, nm, replace=False)])
        lines = subset_lines(lines_all, pick)
        if iid_cells:
            Ttr = rng.uniform(5000.0, 30000.0, C)
            Tve = rng.uniform(5000.0, 30000.0, C)
            ntot = _loguniform(rng, 1e14, 1e18, C)
        else:
            Ttr = np.full(C, rng.uniform(5000.0, 30000.0))
            Tve = np.full(C, rng.uniform(5000.0, 30000.0))
            ntot = np.full(C, _loguniform(rng, 1e14, 1e18, 1)[0])
        cells = Cells(Ttr=Ttr, Tve=Tve, n=composition(Tve, ntot))
        mu, w = gauss_legendre_01(16)
        geo = SlabGeometry(cell_order=np.arange(C, dtype=np.int64), dx=np.full(C, 5.0 / C), mu=mu, wmu=w,
                           normal_ray=False)
        out.append(Problem(f"batch_slab_{i}", species, lines, cells, Grid(50.0, 2000.0, K), geo,
                           meta=dict(seed=seed, index=i)))
    return out


def served_requests(seed=1004, n_requests=2000, rate=100.0, pool=None, scale=1.0):
    """Open-loop Poisson request stream: arrival times at `rate` per second;
    cells log-uniform int [10, 5000], spectral points log-uniform
    [1e5, 1e6], rays log-uniform int [1, 256]; half slab solves (mu rays),
    half line-of-sight solves; states as the batched slabs; all requests
    share the stagnation-line line lists.  Returns a list of dicts with the
    arrival time and a Problem."""
    rng = np.random.default_rng(seed)
    if pool is None:
        pool = _air_lines(np.random.default_rng(1001), 20_000, 300_000)
    lines_all, species, _info = pool
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    reqs = []
    for i in range(n_requests):
        C = max(2, int(np.round(_loguniform(rng, 10, 5000, 1)[0] * scale)))
        K = max(1000, int(_loguniform(rng, 1e5, 1e6, 1)[0] * scale))
        n_rays = int(np.round(_loguniform(rng, 1, 256, 1)[0]))
        slab = bool(rng.integers(0, 2))
        Ttr = rng.uniform(5000.0, 30000.0, C)
        Tve = rng.uniform(5000.0, 30000.0, C)
        ntot = _loguniform(rng, 1e14, 1e18, C)
        cells = Cells(Ttr=Ttr, Tve=Tve, n=composition(Tve, ntot))
        n_mu = max(1, n_rays) if slab else 1
        mu, w = gauss_legendre_01(n_mu) if slab else (np.ones(1), np.ones(1))
        geo = SlabGeometry(cell_order=np.arange(C, dtype=np.int64), dx=np.full(C, 5.0 / C), mu=mu, wmu=w,
                           normal_ray=False)
        reqs.append(dict(t=float(t[i]), slab=slab, problem=Problem(
            f"req_{i}", species, lines_all, cells, Grid(50.0, 2000.0, K), geo, meta=dict(index=i))))
    return reqs


def cr_model(seed=1005, species="N", n_levels=20, n_lumped=0, radiative_fraction=0.5):
    """Synthetic collisional-radiative level model of an atomic radiator
    (Sec. 2.1 QSS populations; the paper's rate databases are not available):
    a ground level with the species' ground-term weight and n_levels - 1
    excited levels uniform in 15-95 % of the ionisation energy (plus
    n_lumped levels above them that only enter the closure), weights 2-20;
    every level pair is a transition with upward Arrhenius rates
    C T^n e^{-theta/T}: heavy-particle impact C log-uniform 1e10-1e13
    cm^3/mol/s, electron impact 1e13-1e16, n uniform 0-0.5; a fraction of
    the pairs radiate with A log-uniform 1e4-1e8 s^-1 at lam = 1e7 / dE nm;
    electron-impact ionisation of each level C log-uniform 1e12-1e14, n = 0.5."""
    rng = np.random.default_rng(seed)
    s = RAD_SPECIES.index(species)
    E_ion = float(RAD_E_IONIZE[s])
    n_all = n_levels + n_lumped
    E = np.concatenate([[0.0], np.sort(rng.uniform(0.15, 0.95, n_all - 1)) * E_ion])
    g = np.concatenate([[ATOM_GROUND_G[species]], rng.integers(2, 21, n_all - 1).astype(np.float64)])
    lo, up = np.triu_indices(n_levels, k=1)
    T = lo.shape[0]
    lu = lambda a, b, n: 10.0 ** rng.uniform(np.log10(a), np.log10(b), n)
    A = np.where(rng.uniform(size=T) < radiative_fraction, lu(1e4, 1e8, T), 0.0)
    ion = {"N": "N+", "O": "O+"}.get(species)
    return dict(l=n_levels, E=E, g=g, lo=lo.astype(np.int32), up=up.astype(np.int32),
                hp_C=lu(1e10, 1e13, T), hp_n=rng.uniform(0.0, 0.5, T), e_C=lu(1e13, 1e16, T),
                e_n=rng.uniform(0.0, 0.5, T), A=A, lam=1e7 / (E[up] - E[lo]),
                ii_C=lu(1e12, 1e14, n_levels), ii_n=np.full(n_levels, 0.5), E_ion=E_ion,
                g_ion=float(ATOM_GROUND_G[ion]) if ion else 1.0, col=int(RAD_DENSITY_COL[s]),
                ion_col=FLOW_SPECIES.index(ion) if ion else -1)


def cr_lines(model, species, base=None, seed=1006):
    """Lines of a collisional-radiative model's radiating transitions (A > 0,
    centre 50-2000 nm) for the atomic radiator `species`, merged with an
    optional base line list and sorted by centre; returns (Lines, lev_u,
    lev_l) with the model-level index of every line's upper / lower level
    (-1 for the base lines)."""
    rng = np.random.default_rng(seed)
    s = RAD_SPECIES.index(species)
    keep = np.nonzero((model["A"] > 0) & (model["lam"] >= 50.0) & (model["lam"] <= 2000.0))[0]
    n = len(keep)
    lo, up = model["lo"][keep], model["up"][keep]
    z = np.zeros(n)
    new = Lines(lam0=model["lam"][keep].astype(np.float64), A=model["A"][keep].astype(np.float64),
                lamS0=10.0 ** rng.uniform(-4, -1, n), species=np.full(n, s, np.int32),
                Eu_el=model["E"][up].astype(np.float64), Eu_v=z.copy(), Eu_j=z.copy(), gu=model["g"][up].astype(np.float64),
                El_el=model["E"][lo].astype(np.float64), El_v=z.copy(), El_j=z.copy(), gl=model["g"][lo].astype(np.float64))
    lev_u, lev_l = up.astype(np.int32), lo.astype(np.int32)
    if base is not None:
        new = Lines(**{k: np.concatenate([getattr(base, k), getattr(new, k)]) for k in Lines.__dataclass_fields__})
        m = len(base)
        lev_u = np.concatenate([np.full(m, -1, np.int32), lev_u])
        lev_l = np.concatenate([np.full(m, -1, np.int32), lev_l])
    order = np.argsort(new.lam0, kind="stable")
    new = Lines(**{k: np.ascontiguousarray(getattr(new, k)[order]) for k in Lines.__dataclass_fields__})
    return new, lev_u[order], lev_l[order]


# Free-free fit coefficients c1..c8 of the hydrogenic cross section for N and
# O (Sec. 2.2.1, Table 3).
FF_FIT = {
    "N": np.array([0.006805, -0.00934, 0.000116, 0.508, 1.046, 5.77e-5, 1.85, 0.000343]),
    "O": np.array([0.001905, -0.005105, 8.176e-5, 0.4554, 1.0238, 5.329e-5, 1.7587, 0.003121]),
}
# Low terms of the ions (cm^-1, weight) for their partition functions.
ION_TERMS = {"N": ([0.0, 15316.2, 32688.8], [9.0, 5.0, 1.0]),
             "O": ([0.0, 26810.6, 40468.0], [4.0, 10.0, 6.0])}


def continuum_model(seed=1007, species="N", n_levels=100, n_nodes=120, n_resonances=3, D="synthetic"):
    """Synthetic atomic continuum model (Sec. 2.2.1 bound-free and free-free;
    the TOPbase cross sections and Peach's D table are not available):
    a ground level with the ground-term weight and n_levels - 1 levels
    uniform in 15-99.5 % of the ionisation energy, weights 2-18; per level a
    photoionisation table of n_nodes wavelengths, geometric from 10 nm to the
    edge 1e7 / (E_ion - E_i) nm, with sigma = s0 (lam / edge)^3 (Kramers
    shape), s0 log-uniform 1e-19-2e-17 cm^2, times up to n_resonances
    Lorentzian bumps; the ion's low terms for Q_+; Table 3's free-free fit;
    a D(sigma, T) table on 12 sigma x 8 T nodes, smooth with |D| <= 0.2
    ("synthetic") or zero ("zero")."""
    rng = np.random.default_rng(seed)
    s = RAD_SPECIES.index(species)
    E_ion = float(RAD_E_IONIZE[s])
    E = np.concatenate([[0.0], np.sort(rng.uniform(0.15, 0.995, n_levels - 1)) * E_ion])
    g = np.concatenate([[ATOM_GROUND_G[species]], 2.0 * rng.integers(1, 10, n_levels - 1)])
    off = np.zeros(n_levels + 1, np.int64)
    lam_parts, sig_parts = [], []
    for i in range(n_levels):
        edge = 1e7 / (E_ion - E[i])
        lam = np.geomspace(10.0, edge, n_nodes)
        lam[-1] = edge
        s0 = 10.0 ** rng.uniform(np.log10(1e-19), np.log10(2e-17))
        bump = np.ones(n_nodes)
        for _ in range(rng.integers(0, n_resonances + 1)):
            lr, w, a = rng.uniform(0.2, 0.98) * edge, rng.uniform(0.002, 0.02) * edge, rng.uniform(0.5, 5.0)
            bump += a / (1.0 + ((lam - lr) / w) ** 2)
        lam_parts.append(lam)
        sig_parts.append(s0 * (lam / edge) ** 3 * bump)
        off[i + 1] = off[i] + n_nodes
    D_sigma = np.geomspace(0.02, 2.5, 12)
    D_T = np.linspace(2000.0, 30000.0, 8)
    if D == "zero":
        Dv = np.zeros((8, 12))
    else:
        ph = rng.uniform(0, 2 * np.pi)
        Dv = 0.2 * np.sin(ph + 2.0 * np.log(D_sigma)[None, :] + (D_T[:, None] / 12000.0)) * \
            np.exp(-D_T[:, None] / 40000.0)
    ion = {"N": "N+", "O": "O+"}[species]
    iE, ig = ION_TERMS[species]
    return dict(species=s, atom_col=int(RAD_DENSITY_COL[s]), ion_col=FLOW_SPECIES.index(ion), E_ion=E_ion,
                E=E, g=g, node_off=off, node_lam=np.concatenate(lam_parts), node_sigma=np.concatenate(sig_parts),
                ion_E=np.array(iE), ion_g=np.array(ig), ff_c=FF_FIT[species].copy(),
                D_sigma=D_sigma, D_T=D_T, D=Dv)
