"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point include/rapral.h declares and nothing else, and the
Python binding refuses to run without a CUDA device (no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import pytest
import torch

from paper_2604_11856_gb300 import build as B
from paper_2604_11856_gb300 import rapral as R

HEADER = os.path.join(B.ROOT, "include", "rapral.h")


def declared():
    return sorted(set(re.findall(r"RAPRAL_API\s+[\w\s\*]+?\b(rapral_\w+)\s*\(", open(HEADER).read())))


def test_header_declares_the_boundary():
    names = declared()
    for n in ["rapral_populations", "rapral_spectral_coeffs", "rapral_trace_rays", "rapral_wall_flux",
              "rapral_create", "rapral_destroy", "rapral_sync"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for n in declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert exported == declared()


def test_workspace_query_is_host_only():
    b = R.workspace_bytes(320_000, 200, 1_000_000)
    assert b > 320_000 * 96


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU behaviour")
def test_no_cpu_fallback():
    with pytest.raises(RuntimeError, match="CUDA"):
        R.Context(0)


def test_noalloc_entry_point_rejects_bad_arguments_before_any_cuda_call():
    """The allocation-free entry point checks its host arguments first: null
    arrays and impossible sizes come back as RAPRAL_EINVAL with a message,
    without touching a device (this runs on a machine with none)."""
    lib = R.load()
    f = lib.rapral_spectral_coeffs_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(R.Species), ctypes.POINTER(R.Lines), ctypes.POINTER(R.Cells),
                  ctypes.POINTER(R.Grid), ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_char_p, ctypes.c_size_t]
    err = ctypes.create_string_buffer(256)
    sp, ln, ce = R.Species(), R.Lines(), R.Cells()
    fake = ctypes.c_void_p(16)   # never dereferenced: every case below fails a host check first
    assert f(None, None, None, None, None, 0, 1, R.FP32, None, None, 1, err, 256) == 1
    assert b"null" in err.value
    sp.n_species, ce.n_cells, ce.n_cols, ce.ne_col, ce.lnpref = 11, 4, 11, 10, 16

    def call(grid, k0=0, nk=10, precision=R.FP32, ld=10):
        err.value = b""
        return f(None, ctypes.byref(sp), ctypes.byref(ln), ctypes.byref(ce), ctypes.byref(grid), k0, nk, precision,
                 fake, fake, ld, err, 256)

    bad = [dict(grid=R.Grid(50.0, 100.0, 1)),                     # fewer than two grid points
           dict(grid=R.Grid(100.0, 50.0, 100)),                   # empty wavelength range
           dict(grid=R.Grid(50.0, float("inf"), 100)),            # infinite upper wavelength
           dict(grid=R.Grid(50.0, 100.0, 100), k0=95, nk=10),     # range past the grid's end
           dict(grid=R.Grid(50.0, 100.0, 100), ld=5),             # row stride below the range
           dict(grid=R.Grid(50.0, 100.0, 100), precision=7)]      # unknown precision
    for case in bad:
        assert call(**case) == 1, case
        assert err.value, case
