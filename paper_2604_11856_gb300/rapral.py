"""Thin ctypes binding of librapral (include/rapral.h).

Argument marshalling only: device memory and streams come from PyTorch, every
step of the path runs in the library's CUDA kernels.  Functions carry the
C-ABI names without the `rapral_` prefix.  There is no CPU fallback: without
the built library or a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np
import torch

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ECANCELED = range(6)
FP64, FP32 = 0, 1
MAX_DIRS = 65
SLAB_DIRS = 17   # directions per tangent-slab bundle
_ERRNAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT", ECANCELED: "ECANCELED"}

_lib = None
_lock = threading.Lock()


BROAD_STARK_IONIZE, BROAD_RESONANCE, BROAD_VDW = 1, 2, 4   # rapral_set_broadening flags
PROFILE_WHITING, PROFILE_VOIGT = 0, 1                     # rapral_set_profile


class RapralError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Stats(ct.Structure):
    _fields_ = [("evaluations", ct.c_int64), ("gauss_terms", ct.c_int64), ("correction_terms", ct.c_int64),
                ("pairs", ct.c_int64)]


class Species(ct.Structure):
    _fields_ = [("n_species", ct.c_int32), ("kind", ct.c_void_p), ("density_col", ct.c_void_p),
                ("mass", ct.c_void_p), ("atom_off", ct.c_void_p), ("atom_E", ct.c_void_p),
                ("atom_g", ct.c_void_p), ("st_off", ct.c_void_p), ("st_E", ct.c_void_p), ("st_g", ct.c_void_p),
                ("st_sigma", ct.c_void_p), ("st_Lalt", ct.c_void_p), ("st_nv", ct.c_void_p),
                ("st_nj", ct.c_void_p), ("st_vib_off", ct.c_void_p), ("st_rot_off", ct.c_void_p),
                ("vib_E", ct.c_void_p), ("rot_E", ct.c_void_p), ("n_atom_levels", ct.c_int64),
                ("n_states", ct.c_int64), ("n_vib", ct.c_int64), ("n_rot", ct.c_int64)]


class Lines(ct.Structure):
    _fields_ = [("n_lines", ct.c_int64)] + [(k, ct.c_void_p) for k in
                                             ["lam0", "A", "lamS0", "species", "Eu_el", "Eu_v", "Eu_j", "gu",
                                              "El_el", "El_v", "El_j", "gl"]]


class Cells(ct.Structure):
    _fields_ = [("n_cells", ct.c_int64), ("Ttr", ct.c_void_p), ("Tve", ct.c_void_p), ("n", ct.c_void_p),
                ("n_cols", ct.c_int32), ("ne_col", ct.c_int32), ("lnpref", ct.c_void_p)]


class Grid(ct.Structure):
    _fields_ = [("lam_min", ct.c_double), ("lam_max", ct.c_double), ("n", ct.c_int64)]


class Rays(ct.Structure):
    _fields_ = [("n_bundles", ct.c_int64), ("n_points", ct.c_int64), ("n_segments", ct.c_int64),
                ("n_dirs", ct.c_int64), ("max_dirs", ct.c_int32), ("max_bundles_per_point", ct.c_int32),
                ("point_off", ct.c_void_p), ("seg_off", ct.c_void_p), ("seg_cell", ct.c_void_p),
                ("seg_ds", ct.c_void_p), ("dir_off", ct.c_void_p), ("dir_scale", ct.c_void_p),
                ("dir_weight", ct.c_void_p), ("bundle_wall", ct.c_void_p), ("T_wall", ct.c_double),
                ("node_values", ct.c_int32)]


class CrModel(ct.Structure):
    _fields_ = [("n_levels", ct.c_int32), ("n_levels_all", ct.c_int32), ("E", ct.c_void_p), ("g", ct.c_void_p),
                ("n_trans", ct.c_int32), ("lo", ct.c_void_p), ("up", ct.c_void_p), ("hp_C", ct.c_void_p),
                ("hp_n", ct.c_void_p), ("e_C", ct.c_void_p), ("e_n", ct.c_void_p), ("A", ct.c_void_p),
                ("lam", ct.c_void_p), ("ii_C", ct.c_void_p), ("ii_n", ct.c_void_p), ("E_ionize", ct.c_double),
                ("g_ion", ct.c_double), ("col", ct.c_int32), ("ion_col", ct.c_int32)]


class Continuum(ct.Structure):
    _fields_ = [("species", ct.c_int32), ("atom_col", ct.c_int32), ("ion_col", ct.c_int32),
                ("E_ionize", ct.c_double), ("n_levels", ct.c_int32), ("E", ct.c_void_p), ("g", ct.c_void_p),
                ("n_nodes", ct.c_int64), ("node_off", ct.c_void_p), ("node_lam", ct.c_void_p),
                ("node_sigma", ct.c_void_p), ("n_ion_terms", ct.c_int32), ("ion_E", ct.c_void_p),
                ("ion_g", ct.c_void_p), ("ff_c", ct.c_double * 8), ("n_D_sigma", ct.c_int32),
                ("n_D_T", ct.c_int32), ("D_sigma", ct.c_void_p), ("D_T", ct.c_void_p), ("D", ct.c_void_p)]


class BatchItem(ct.Structure):
    _fields_ = [("species", ct.c_void_p), ("lines", ct.c_void_p), ("cells", ct.c_void_p), ("grid", ct.c_void_p),
                ("rays", ct.c_void_p), ("k0", ct.c_int64), ("nk", ct.c_int64), ("kappa", ct.c_void_p),
                ("emis", ct.c_void_p), ("ld", ct.c_int64), ("q_lambda", ct.c_void_p), ("q", ct.c_void_p)]


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Loads librapral.so (building it with nvcc when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"librapral.so is not built ({path}); run __graft_entry__.build()")
        L = ct.CDLL(path)
        i, i32, i64, vp, d = ct.c_int, ct.c_int32, ct.c_int64, ct.c_void_p, ct.c_double
        P = ct.POINTER
        sig = {
            "rapral_create": (i, [P(vp), i, vp]),
            "rapral_destroy": (None, [vp]),
            "rapral_last_error": (ct.c_char_p, [vp]),
            "rapral_set_stream": (i, [vp, vp]),
            "rapral_sync": (i, [vp]),
            "rapral_clear_status": (i, [vp]),
            "rapral_set_constants": (i, [vp, i]),
            "rapral_set_tiling": (i, [vp, i, i]),
            "rapral_set_line_sum_blocks": (i, [vp, i]),
            "rapral_set_line_batch": (i, [vp, i]),
            "rapral_workspace_bytes": (i, [i64, i64, i64, P(ct.c_size_t)]),
            "rapral_get_stats": (i, [vp, P(Stats)]),
            "rapral_reset_stats": (i, [vp]),
            "rapral_set_counters": (i, [vp, i]),
            "rapral_set_profile_events": (i, [vp, vp, vp]),
            "rapral_populations": (i, [vp, P(Species), P(Cells), vp]),
            "rapral_batch_create": (i, [vp, i, P(BatchItem), i, P(vp)]),
            "rapral_batch_run": (i, [vp, vp]),
            "rapral_batch_units": (i, [vp, P(i64), P(i)]),
            "rapral_batch_destroy": (None, [vp]),
            "rapral_spectral_coeffs": (i, [vp, P(Species), P(Lines), P(Cells), P(Grid), i64, i64, i, vp, vp, i64]),
            "rapral_trace_rays": (i, [vp, P(Rays), i64, vp, vp, i64, P(Grid), i64, i64, i, vp, vp]),
            "rapral_wall_flux": (i, [vp, vp, i, P(Grid), i64, i64, i64, vp]),
            "rapral_slab_rays": (i, [vp, vp, vp, i32, vp, vp, i32, i32, i32, d, vp, vp, vp, vp, vp, vp, vp, vp,
                                     P(Rays)]),
            "rapral_axisym_rays": (i, [vp, vp, i32, vp, i32, vp, i32, vp, vp, i32, i32, vp, P(i64), vp, vp, vp,
                                       vp, vp, vp, vp, P(Rays)]),
            "rapral_fibonacci_rays": (i, [vp, vp, i32, vp, i32, vp, i32, i32, vp, P(i64), vp, vp, vp, vp, vp, vp,
                                          vp, vp, vp, vp, P(Rays)]),
            "rapral_los_node_states": (i, [vp, vp, i32, vp, i32, P(Cells), i64, vp, vp, vp, vp, vp]),
            "rapral_fibonacci_flux": (i, [vp, i64, vp, vp, i32, vp, i32, i32, vp]),
            "rapral_set_broadening": (i, [vp, i32, i32, vp, i32, vp]),
            "rapral_set_profile": (i, [vp, i32]),
            "rapral_qss_populations": (i, [vp, P(CrModel), P(Cells), vp]),
            "rapral_continuum_coeffs": (i, [vp, vp, i32, i32, P(Cells), P(Grid), i64, i64, i, vp, vp, i64]),
            "rapral_saha_populations": (i, [vp, P(Cells), i32, i32, d, i32, i32, vp, vp, vp]),
            "rapral_qss_departures": (i, [vp, P(CrModel), P(Cells), i32, i32, vp, vp, i32]),
            "rapral_set_departures": (i, [vp, i32, vp, i64, i32, vp, vp, i64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _ptr(t):
    return ct.c_void_p(t.data_ptr()) if t is not None else None


class Context:
    """A librapral context bound to a CUDA device and stream."""

    def __init__(self, device=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("librapral needs a CUDA device; there is no CPU fallback")
        self.lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ct.c_void_p()
        rc = self.lib.rapral_create(ct.byref(h), self.device.index, ct.c_void_p(self.stream.cuda_stream))
        if rc != OK:
            raise RapralError(rc, "rapral_create failed")
        self.h = h

    def check(self, rc):
        if rc != OK:
            raise RapralError(rc, self.lib.rapral_last_error(self.h).decode())

    def set_broadening(self, flags, E_ionize=None, column_mass=None):
        """Optional Lorentz terms (BROAD_* flags) for later coefficient calls:
        E_ionize per radiating species (cm^-1), column_mass per density column
        (g/mol, 0 for electrons)."""
        E = np.ascontiguousarray(E_ionize if E_ionize is not None else np.zeros(0), np.float64)
        M = np.ascontiguousarray(column_mass if column_mass is not None else np.zeros(0), np.float64)
        self.check(self.lib.rapral_set_broadening(self.h, int(flags), E.shape[0],
                                                  E.ctypes.data_as(ct.c_void_p) if E.size else None, M.shape[0],
                                                  M.ctypes.data_as(ct.c_void_p) if M.size else None))

    def set_departures(self, ln_b=None, lev_u=None, lev_l=None):
        """Departure coefficients for later coefficient calls: device tensors
        ln_b [C, S, n_lev] (float64), lev_u / lev_l [L] (int32, -1: none);
        kept referenced while set.  No argument: off."""
        if ln_b is None:
            self.check(self.lib.rapral_set_departures(self.h, 0, None, 0, 0, None, None, 0))
            self._dep = None
            return
        C, S, n = ln_b.shape
        self._dep = (ln_b.contiguous(), lev_u.contiguous(), lev_l.contiguous())
        b, u, lo = self._dep
        self.check(self.lib.rapral_set_departures(self.h, int(n), _ptr(b), int(C), int(S), _ptr(u), _ptr(lo),
                                                  int(u.shape[0])))

    def set_profile(self, profile):
        """Line shape of later coefficient calls: PROFILE_WHITING (default) or PROFILE_VOIGT."""
        self.check(self.lib.rapral_set_profile(self.h, int(profile)))

    def set_stream(self, stream):
        self.stream = stream
        self.check(self.lib.rapral_set_stream(self.h, ct.c_void_p(stream.cuda_stream)))

    def sync(self):
        self.check(self.lib.rapral_sync(self.h))

    def clear_status(self):
        self.check(self.lib.rapral_clear_status(self.h))

    def set_tiling(self, tile_width=0, cells_per_block=0):
        self.check(self.lib.rapral_set_tiling(self.h, tile_width, cells_per_block))

    def set_line_sum_blocks(self, blocks_per_sm=-1):
        """FP32 line-sum launch: -1 persistent at full occupancy (default),
        n > 0 persistent with n blocks a SM, 0 one block per work unit."""
        self.check(self.lib.rapral_set_line_sum_blocks(self.h, blocks_per_sm))

    def set_line_batch(self, pairs=32):
        """FP32 line sum: (line, cell) pairs a warp stages per sweep pass, 32 or 64."""
        self.check(self.lib.rapral_set_line_batch(self.h, pairs))

    def get_stats(self):
        st = Stats()
        self.check(self.lib.rapral_get_stats(self.h, ct.byref(st)))
        return dict(evaluations=st.evaluations, gauss_terms=st.gauss_terms,
                    correction_terms=st.correction_terms, pairs=st.pairs)

    def set_counters(self, on):
        self.check(self.lib.rapral_set_counters(self.h, int(bool(on))))

    def reset_stats(self):
        self.check(self.lib.rapral_reset_stats(self.h))

    def set_profile_events(self, before=None, after=None):
        """torch.cuda.Event pair recorded around every line-sum launch (None: off)."""
        b = ct.c_void_p(before.cuda_event) if before is not None else None
        a = ct.c_void_p(after.cuda_event) if after is not None else None
        self.check(self.lib.rapral_set_profile_events(self.h, b, a))

    def set_constants(self, codata):
        self.check(self.lib.rapral_set_constants(self.h, int(codata)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.rapral_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workspace_bytes(n_lines, n_cells, nk):
    out = ct.c_size_t()
    rc = load().rapral_workspace_bytes(int(n_lines), int(n_cells), int(nk), ct.byref(out))
    if rc != OK:
        raise RapralError(rc, "rapral_workspace_bytes")
    return out.value


# ----------------------------------------------------------------------------
# device-resident inputs
# ----------------------------------------------------------------------------

def _t(a, dtype, device):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(device, non_blocking=True)


class DeviceSpecies:
    """Species database on the device plus its rapral_species struct."""

    def __init__(self, sp, device):
        f8, i4, i8 = np.float64, np.int32, np.int64
        self.t = dict(kind=_t(sp.kind, i4, device), density_col=_t(sp.density_col, i4, device),
                      mass=_t(sp.mass, f8, device), atom_off=_t(sp.atom_off, i8, device),
                      atom_E=_t(sp.atom_E, f8, device), atom_g=_t(sp.atom_g, f8, device),
                      st_off=_t(sp.st_off, i8, device), st_E=_t(sp.st_E, f8, device), st_g=_t(sp.st_g, f8, device),
                      st_sigma=_t(sp.st_sigma, f8, device), st_Lalt=_t(sp.st_Lalt, f8, device),
                      st_nv=_t(sp.st_nv, i4, device), st_nj=_t(sp.st_nj, i4, device),
                      st_vib_off=_t(sp.st_vib_off, i8, device), st_rot_off=_t(sp.st_rot_off, i8, device),
                      vib_E=_t(sp.vib_E, f8, device), rot_E=_t(sp.rot_E, f8, device))
        s = Species()
        s.n_species = len(sp.names)
        for k, v in self.t.items():
            setattr(s, k, v.data_ptr() if v.numel() else None)
        s.n_atom_levels = int(sp.atom_E.shape[0]); s.n_states = int(sp.st_E.shape[0])
        s.n_vib = int(sp.vib_E.shape[0]); s.n_rot = int(sp.rot_E.shape[0])
        self.struct = s
        self.S = s.n_species


LINE_KEYS = ["lam0", "A", "lamS0", "Eu_el", "Eu_v", "Eu_j", "gu", "El_el", "El_v", "El_j", "gl"]


class DeviceLines:
    def __init__(self, ln, device, tensors=None):
        if tensors is None:
            tensors = {k: _t(getattr(ln, k), np.float64, device) for k in LINE_KEYS}
            tensors["species"] = _t(ln.species, np.int32, device)
        self.t = tensors
        s = Lines()
        s.n_lines = int(tensors["lam0"].shape[0])
        for k, v in tensors.items():
            setattr(s, k, v.data_ptr() if v.numel() else None)
        self.struct = s
        self.L = s.n_lines


class DeviceCells:
    def __init__(self, cells, S, device, tensors=None):
        if tensors is None:
            tensors = dict(Ttr=_t(cells.Ttr, np.float64, device), Tve=_t(cells.Tve, np.float64, device),
                           n=_t(cells.n, np.float64, device))
        self.t = tensors
        C = int(tensors["Ttr"].shape[0])
        self.lnpref = torch.empty((C, S), dtype=torch.float64, device=device)
        s = Cells()
        s.n_cells = C
        s.Ttr, s.Tve, s.n = tensors["Ttr"].data_ptr(), tensors["Tve"].data_ptr(), tensors["n"].data_ptr()
        s.n_cols = int(tensors["n"].shape[1])
        s.ne_col = int(getattr(cells, "ne_col", 10)) if cells is not None else 10
        s.lnpref = self.lnpref.data_ptr()
        self.struct = s
        self.C = C


def grid_struct(g):
    s = Grid()
    s.lam_min, s.lam_max, s.n = float(g.lam_min), float(g.lam_max), int(g.n)
    return s


# ----------------------------------------------------------------------------
# the C-ABI calls
# ----------------------------------------------------------------------------

def _row_stride(kappa, emis, nk):
    ld = kappa.stride(0) if kappa.dim() == 2 and kappa.shape[0] > 1 else max(int(nk), kappa.shape[-1])
    if kappa.dim() != 2 or kappa.stride(1) != 1 or emis.shape != kappa.shape or emis.stride() != kappa.stride() \
            or kappa.shape[1] < nk:
        raise ValueError("kappa / emis must be equal [C, >= nk] row-major tensors or column views")
    return ld


def populations(ctx, dsp, dcells):
    ctx.check(ctx.lib.rapral_populations(ctx.h, ct.byref(dsp.struct), ct.byref(dcells.struct),
                                         _ptr(dcells.lnpref)))
    return dcells.lnpref


def spectral_coeffs(ctx, dsp, dlines, dcells, grid, k0, nk, precision, kappa, emis):
    """kappa, emis: [C, >= nk] tensors (or column views of them) of the precision's dtype,
    rows ld = stride(0) elements apart; columns 0..nk-1 are written."""
    ld = _row_stride(kappa, emis, nk)
    g = grid_struct(grid)
    ctx.check(ctx.lib.rapral_spectral_coeffs(ctx.h, ct.byref(dsp.struct), ct.byref(dlines.struct),
                                             ct.byref(dcells.struct), ct.byref(g), int(k0), int(nk),
                                             int(precision), _ptr(kappa), _ptr(emis), int(ld)))


def trace_rays(ctx, rays, n_cells, kappa, emis, grid, k0, nk, precision, q_lambda, I_out=None):
    """kappa, emis as for spectral_coeffs (columns 0..nk-1 are read); q_lambda [P, nk] and
    I_out [n_dirs, nk] contiguous."""
    ld = _row_stride(kappa, emis, nk)
    g = grid_struct(grid)
    ctx.check(ctx.lib.rapral_trace_rays(ctx.h, ct.byref(rays.struct), int(n_cells), _ptr(kappa), _ptr(emis),
                                        int(ld), ct.byref(g), int(k0), int(nk), int(precision),
                                        _ptr(q_lambda), _ptr(I_out)))


def wall_flux(ctx, q_lambda, precision, grid, k0, nk, n_points, q):
    g = grid_struct(grid)
    ctx.check(ctx.lib.rapral_wall_flux(ctx.h, _ptr(q_lambda), int(precision), ct.byref(g), int(k0), int(nk),
                                       int(n_points), _ptr(q)))


class DeviceRays:
    """Caller-owned ray arrays (torch tensors) and their rapral_rays struct."""

    def __init__(self):
        self.t = {}
        self.struct = Rays()

    @property
    def n_points(self):
        return self.struct.n_points

    @property
    def n_dirs(self):
        return self.struct.n_dirs


def rays_from_arrays(point_off, seg_off, seg_cell, seg_ds, dir_off, dir_scale, dir_weight, bundle_wall,
                     T_wall, device, node_values=False):
    """A caller-built ray set (host arrays in the rapral_rays layout) copied
    to the device; the maxima of directions per bundle and bundles per point
    are taken from the offsets."""
    r = DeviceRays()
    t = r.t
    point_off = np.asarray(point_off, np.int64); dir_off = np.asarray(dir_off, np.int64)
    t["point_off"] = _t(point_off, np.int64, device)
    t["seg_off"] = _t(seg_off, np.int64, device)
    t["seg_cell"] = _t(np.asarray(seg_cell).reshape(-1) if len(seg_cell) else np.zeros(1), np.int32, device)
    t["seg_ds"] = _t(np.asarray(seg_ds).reshape(-1) if len(seg_ds) else np.zeros(1), np.float64, device)
    t["dir_off"] = _t(dir_off, np.int64, device)
    t["dir_scale"] = _t(dir_scale, np.float64, device)
    t["dir_weight"] = _t(dir_weight, np.float64, device)
    t["bundle_wall"] = _t(bundle_wall, np.int32, device)
    s = r.struct
    s.n_points, s.n_bundles = len(point_off) - 1, len(dir_off) - 1
    s.n_segments, s.n_dirs = len(seg_cell), len(dir_scale)
    s.max_dirs = int(np.diff(dir_off).max()) if len(dir_off) > 1 else 0
    s.max_bundles_per_point = int(np.diff(point_off).max()) if len(point_off) > 1 else 0
    for k in ("point_off", "seg_off", "seg_cell", "seg_ds", "dir_off", "dir_scale", "dir_weight", "bundle_wall"):
        setattr(s, k, t[k].data_ptr())
    s.T_wall = float(T_wall)
    s.node_values = int(bool(node_values))
    return r


def slab_rays(ctx, geo, device):
    """Tangent-slab bundle (rapral_slab_rays) from a SlabGeometry."""
    r = DeviceRays()
    m = int(len(geo.cell_order))
    n_mu = int(len(geo.mu))
    nd = n_mu + (1 if geo.normal_ray else 0)
    nb = (nd + SLAB_DIRS - 1) // SLAB_DIRS
    i32, i64, f8 = torch.int32, torch.int64, torch.float64
    t = r.t
    t["cell_order"] = _t(geo.cell_order, np.int32, device)
    t["dx"] = _t(geo.dx, np.float64, device)
    t["mu"] = _t(geo.mu, np.float64, device)
    t["wmu"] = _t(geo.wmu, np.float64, device)
    t["point_off"] = torch.empty(2, dtype=i64, device=device)
    t["seg_off"] = torch.empty(nb + 1, dtype=i64, device=device)
    t["seg_cell"] = torch.empty(max(m * nb, 1), dtype=i32, device=device)
    t["seg_ds"] = torch.empty(max(m * nb, 1), dtype=f8, device=device)
    t["dir_off"] = torch.empty(nb + 1, dtype=i64, device=device)
    t["dir_scale"] = torch.empty(nd, dtype=f8, device=device)
    t["dir_weight"] = torch.empty(nd, dtype=f8, device=device)
    t["bundle_wall"] = torch.empty(nb, dtype=i32, device=device)
    ctx.check(ctx.lib.rapral_slab_rays(ctx.h, _ptr(t["cell_order"]), _ptr(t["dx"]), m, _ptr(t["mu"]),
                                       _ptr(t["wmu"]), n_mu, int(bool(geo.normal_ray)), int(bool(geo.wall_start)),
                                       float(geo.T_wall), _ptr(t["point_off"]), _ptr(t["seg_off"]),
                                       _ptr(t["seg_cell"]), _ptr(t["seg_ds"]), _ptr(t["dir_off"]),
                                       _ptr(t["dir_scale"]), _ptr(t["dir_weight"]), _ptr(t["bundle_wall"]),
                                       ct.byref(r.struct)))
    return r


class DeviceCrModel:
    """A level model (a dict of host arrays as made by synth.cr_model) on the
    device, with its rapral_cr_model struct."""

    def __init__(self, model, device):
        m = model
        t = {k: _t(m[k], np.float64, device) for k in ("E", "g", "hp_C", "hp_n", "e_C", "e_n", "A", "lam", "ii_C",
                                                          "ii_n")}
        t["lo"] = _t(m["lo"], np.int32, device)
        t["up"] = _t(m["up"], np.int32, device)
        self.t = t
        s = CrModel()
        s.n_levels, s.n_levels_all = int(m["l"]), int(len(m["E"]))
        s.n_trans = int(len(m["lo"]))
        for k, v in t.items():
            setattr(s, k, v.data_ptr())
        s.E_ionize, s.g_ion = float(m["E_ion"]), float(m["g_ion"])
        s.col, s.ion_col = int(m["col"]), int(m["ion_col"])
        self.struct = s
        self.l = s.n_levels


class DeviceContinuum:
    """Atomic continuum models (dicts of host arrays as made by
    synth.continuum_model) on the device, with their rapral_continuum array."""

    def __init__(self, models, device):
        self.t = []
        self.structs = (Continuum * len(models))()
        for k, m in enumerate(models):
            t = {n: _t(m[n], np.float64, device) for n in ("E", "g", "node_lam", "node_sigma", "ion_E", "ion_g",
                                                             "D_sigma", "D_T", "D")}
            t["node_off"] = _t(m["node_off"], np.int64, device)
            self.t.append(t)
            s = self.structs[k]
            s.species, s.atom_col, s.ion_col = int(m["species"]), int(m["atom_col"]), int(m["ion_col"])
            s.E_ionize = float(m["E_ion"])
            s.n_levels = int(len(m["E"]))
            s.n_nodes = int(m["node_off"][-1])
            s.n_ion_terms = int(len(m["ion_E"]))
            for n in ("E", "g", "node_off", "node_lam", "node_sigma", "ion_E", "ion_g"):
                setattr(s, n, t[n].data_ptr())
            for j in range(8):
                s.ff_c[j] = float(m["ff_c"][j])
            if m.get("D") is not None:
                s.n_D_sigma, s.n_D_T = int(len(m["D_sigma"])), int(len(m["D_T"]))
                s.D_sigma, s.D_T, s.D = t["D_sigma"].data_ptr(), t["D_T"].data_ptr(), t["D"].data_ptr()
        self.n = len(models)


def continuum_coeffs(ctx, dcont, n_species, dcells, grid, k0, nk, precision, kappa, emis):
    """Adds the atomic continuum (rapral_continuum_coeffs) to kappa, emis
    ([C, >= nk] of the precision's dtype, rows stride(0) apart)."""
    ld = _row_stride(kappa, emis, nk)
    g = grid_struct(grid)
    ctx.check(ctx.lib.rapral_continuum_coeffs(ctx.h, ct.byref(dcont.structs), dcont.n, int(n_species),
                                              ct.byref(dcells.struct), ct.byref(g), int(k0), int(nk),
                                              int(precision), _ptr(kappa), _ptr(emis), int(ld)))


def qss_populations(ctx, dmodel, dcells, out):
    """QSS level populations [C, l] (rapral_qss_populations) into `out`."""
    ctx.check(ctx.lib.rapral_qss_populations(ctx.h, ct.byref(dmodel.struct), ct.byref(dcells.struct), _ptr(out)))
    return out


def saha_populations(ctx, dcells, species, n_species, E_ionize, ion_col, ion_E, ion_g):
    """Saha-Boltzmann prefactor of radiator `species` into dcells.lnpref
    (rapral_saha_populations); ion_E, ion_g: device float64 tensors."""
    ctx.check(ctx.lib.rapral_saha_populations(ctx.h, ct.byref(dcells.struct), int(species), int(n_species),
                                              float(E_ionize), int(ion_col), int(ion_E.numel()), _ptr(ion_E),
                                              _ptr(ion_g), _ptr(dcells.lnpref)))


def qss_departures(ctx, dmodel, dcells, species, n_qss, ln_b):
    """ln b of the model's levels for radiator `species` (rapral_qss_departures)
    into the device table ln_b [C, S, n_lev]."""
    C, S, n = ln_b.shape
    ctx.check(ctx.lib.rapral_qss_departures(ctx.h, ct.byref(dmodel.struct), ct.byref(dcells.struct), int(species),
                                            int(S), _ptr(n_qss), _ptr(ln_b), int(n)))
    return ln_b


def fibonacci_rays(ctx, geo, n_los, device, points=None):
    """The paper's Fibonacci lines of sight (rapral_fibonacci_rays) from an
    AxisymGeometry's surface points (or the selected ones): node-valued rays
    with per-line los_index and the (x, r) of every node in t["node_x"],
    t["node_r"]."""
    r = DeviceRays()
    t = r.t
    sx = np.asarray(geo.surf_x) if points is None else np.asarray(geo.surf_x)[np.asarray(points)]
    P = int(len(sx)); V = int(n_los) // 2
    B = P * V
    nx, nr = len(geo.xf) - 1, len(geo.rf) - 1
    t["xf"] = _t(geo.xf, np.float64, device); t["rf"] = _t(geo.rf, np.float64, device)
    t["surf_x"] = _t(sx, np.float64, device)
    t["seg_off"] = torch.empty(B + 1, dtype=torch.int64, device=device)
    nseg = ct.c_int64()
    args0 = [ctx.h, _ptr(t["xf"]), nx, _ptr(t["rf"]), nr, _ptr(t["surf_x"]), P, int(n_los), _ptr(t["seg_off"]),
             ct.byref(nseg)]
    ctx.check(ctx.lib.rapral_fibonacci_rays(*args0, *([None] * 10), None))
    n = int(nseg.value)
    t["seg_cell"] = torch.empty(max(n, 1), dtype=torch.int32, device=device)
    t["seg_ds"] = torch.empty(max(n, 1), dtype=torch.float64, device=device)
    t["point_off"] = torch.empty(P + 1, dtype=torch.int64, device=device)
    t["dir_off"] = torch.empty(B + 1, dtype=torch.int64, device=device)
    for k in ("dir_scale", "dir_weight"):
        t[k] = torch.empty(max(B, 1), dtype=torch.float64, device=device)
    t["bundle_wall"] = torch.empty(max(B, 1), dtype=torch.int32, device=device)
    t["los_index"] = torch.empty(max(B, 1), dtype=torch.int32, device=device)
    t["node_x"] = torch.empty(max(n + B, 1), dtype=torch.float64, device=device)
    t["node_r"] = torch.empty(max(n + B, 1), dtype=torch.float64, device=device)
    ctx.check(ctx.lib.rapral_fibonacci_rays(*args0, _ptr(t["seg_cell"]), _ptr(t["seg_ds"]), _ptr(t["point_off"]),
                                            _ptr(t["dir_off"]), _ptr(t["dir_scale"]), _ptr(t["dir_weight"]),
                                            _ptr(t["bundle_wall"]), _ptr(t["los_index"]), _ptr(t["node_x"]),
                                            _ptr(t["node_r"]), ct.byref(r.struct)))
    r.n_los = int(n_los)
    r.n_nodes = n + B
    return r


def los_node_states(ctx, geo, dgrid_cells, rays, S, device):
    """Flow variables at the rays' nodes (rapral_los_node_states) from the
    grid's DeviceCells; returns DeviceCells of the nodes (S species columns
    of ln(N_s / Z_s) to be filled by populations)."""
    nx, nr = len(geo.xf) - 1, len(geo.rf) - 1
    N = rays.n_nodes
    nc = dgrid_cells.struct.n_cols
    tens = dict(Ttr=torch.empty(max(N, 1), dtype=torch.float64, device=device),
                Tve=torch.empty(max(N, 1), dtype=torch.float64, device=device),
                n=torch.empty((max(N, 1), nc), dtype=torch.float64, device=device))
    ctx.check(ctx.lib.rapral_los_node_states(ctx.h, _ptr(rays.t["xf"]), nx, _ptr(rays.t["rf"]), nr,
                                             ct.byref(dgrid_cells.struct), int(N), _ptr(rays.t["node_x"]),
                                             _ptr(rays.t["node_r"]), _ptr(tens["Ttr"]), _ptr(tens["Tve"]),
                                             _ptr(tens["n"])))
    if N == 0:
        tens = {k: v[:0] for k, v in tens.items()}
    dc = DeviceCells(None, S, device, tensors=tens)
    dc.struct.ne_col = dgrid_cells.struct.ne_col
    return dc


def fibonacci_flux(ctx, rays, S_los, n_phi, n_theta, q):
    """q[p] from the per-line wavelength integrals S_los (rapral_fibonacci_flux)."""
    ctx.check(ctx.lib.rapral_fibonacci_flux(ctx.h, int(rays.n_points), _ptr(rays.t["point_off"]),
                                            _ptr(rays.t["los_index"]), int(rays.n_los), _ptr(S_los), int(n_phi),
                                            int(n_theta), _ptr(q)))


def axisym_rays(ctx, geo, device, points=None):
    """Axisymmetric lines of sight (rapral_axisym_rays) from an AxisymGeometry;
    `points` selects a subset of the surface points."""
    r = DeviceRays()
    t = r.t
    sx = np.asarray(geo.surf_x) if points is None else np.asarray(geo.surf_x)[np.asarray(points)]
    P = int(len(sx)); n_mu = int(len(geo.mu)); n_phi = int(geo.n_phi)
    B = P * n_mu * n_phi
    nx, nr = len(geo.xf) - 1, len(geo.rf) - 1
    t["xf"] = _t(geo.xf, np.float64, device); t["rf"] = _t(geo.rf, np.float64, device)
    t["surf_x"] = _t(sx, np.float64, device)
    t["mu"] = _t(geo.mu, np.float64, device); t["wmu"] = _t(geo.wmu, np.float64, device)
    t["seg_off"] = torch.empty(B + 1, dtype=torch.int64, device=device)
    nseg = ct.c_int64()
    args0 = [ctx.h, _ptr(t["xf"]), nx, _ptr(t["rf"]), nr, _ptr(t["surf_x"]), P, _ptr(t["mu"]), _ptr(t["wmu"]),
             n_mu, n_phi, _ptr(t["seg_off"]), ct.byref(nseg)]
    ctx.check(ctx.lib.rapral_axisym_rays(*args0, None, None, None, None, None, None, None, None))
    n = int(nseg.value)
    t["seg_cell"] = torch.empty(max(n, 1), dtype=torch.int32, device=device)
    t["seg_ds"] = torch.empty(max(n, 1), dtype=torch.float64, device=device)
    t["point_off"] = torch.empty(P + 1, dtype=torch.int64, device=device)
    t["dir_off"] = torch.empty(B + 1, dtype=torch.int64, device=device)
    t["dir_scale"] = torch.empty(B, dtype=torch.float64, device=device)
    t["dir_weight"] = torch.empty(B, dtype=torch.float64, device=device)
    t["bundle_wall"] = torch.empty(B, dtype=torch.int32, device=device)
    ctx.check(ctx.lib.rapral_axisym_rays(*args0, _ptr(t["seg_cell"]), _ptr(t["seg_ds"]), _ptr(t["point_off"]),
                                         _ptr(t["dir_off"]), _ptr(t["dir_scale"]), _ptr(t["dir_weight"]),
                                         _ptr(t["bundle_wall"]), ct.byref(r.struct)))
    return r
