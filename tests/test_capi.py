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
