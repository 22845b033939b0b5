"""rapral_spectral_coeffs_noalloc: the coefficients for callers that cannot
allocate device memory (allocator-free real-time loops, plug-ins whose
device memory belongs to the host program's pool).  Its output must equal the regular entry point's on two
calls in a row with different problems (the shared static scratch keeps the
previous call's contents), a failed input check must not leak into the next
call through that shared scratch, and a problem larger than the 64 MiB
scratch (in its fixed part or in its tile lists) must be refused with ENOMEM
and a message.  Collected last (file name) so that a failure here does not
hide the other tests."""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _noalloc_fn():
    lib = R.load()
    f = lib.rapral_spectral_coeffs_noalloc
    f.restype = ct.c_int
    f.argtypes = [ct.c_void_p, ct.POINTER(R.Species), ct.POINTER(R.Lines), ct.POINTER(R.Cells),
                  ct.POINTER(R.Grid), ct.c_int64, ct.c_int64, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int64,
                  ct.c_char_p, ct.c_size_t]
    return f


def _call(ctx, dp, grid, k0, nk, precision, k, j, err):
    g = R.grid_struct(grid)
    return _noalloc_fn()(ct.c_void_p(ctx.stream.cuda_stream), ct.byref(dp.species.struct), ct.byref(dp.lines.struct),
                         ct.byref(dp.cells.struct), ct.byref(g), k0, nk, precision, ct.c_void_p(k.data_ptr()),
                         ct.c_void_p(j.data_ptr()), k.shape[1], err, 256)


def _both(ctx, p, precision, k0=0, nk=None):
    """Coefficients from the regular entry point and from the no-allocation one."""
    nk = p.grid.n - k0 if nk is None else nk
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    dt = torch.float64 if precision == R.FP64 else torch.float32
    ref_k = torch.empty((dp.C, nk), dtype=dt, device=ctx.device)
    ref_j = torch.empty_like(ref_k)
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, k0, nk, precision, ref_k, ref_j)
    ctx.sync()
    k = torch.full_like(ref_k, float("nan"))
    j = torch.full_like(ref_j, float("nan"))
    err = ct.create_string_buffer(256)
    g = R.grid_struct(p.grid)
    rc = _noalloc_fn()(ct.c_void_p(ctx.stream.cuda_stream), ct.byref(dp.species.struct), ct.byref(dp.lines.struct),
                       ct.byref(dp.cells.struct), ct.byref(g), k0, nk, precision, ct.c_void_p(k.data_ptr()),
                       ct.c_void_p(j.data_ptr()), nk, err, 256)
    assert rc == R.OK, err.value.decode()
    ctx.sync()
    return ref_k.double().cpu().numpy(), ref_j.double().cpu().numpy(), k.double().cpu().numpy(), j.double().cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice():
    ctx = R.Context(0)
    # first call: two-temperature cells, atoms and diatomics, FP64, a range inside the grid
    p1 = synth.stagnation_line(n_cells=10, n_atomic=2000, n_molecular=20000, n_grid=40001)
    rk, rj, k, j = _both(ctx, p1, R.FP64, k0=777, nk=30000)
    np.testing.assert_allclose(k, rk, rtol=TOL, atol=1e-300)
    np.testing.assert_allclose(j, rj, rtol=TOL, atol=1e-300)
    # second call right after: a different, smaller problem in FP32
    p2 = synth.uniform_slab(n_lines=300, n_cells=3, n_grid=20001)
    rk, rj, k, j = _both(ctx, p2, R.FP32)
    np.testing.assert_allclose(k, rk, rtol=TOL, atol=0)
    np.testing.assert_allclose(j, rj, rtol=TOL, atol=0)
    assert np.isfinite(k).all() and np.isfinite(j).all()


def test_noalloc_refuses_problems_beyond_its_scratch():
    ctx = R.Context(0)
    p = synth.uniform_slab(n_lines=20, n_cells=2, n_grid=2000)
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    big = 600_000
    t = {k: torch.full((big,), 500.0, dtype=torch.float64, device=ctx.device) for k in R.LINE_KEYS}
    t["species"] = torch.zeros(big, dtype=torch.int32, device=ctx.device)
    lines = R.DeviceLines(None, ctx.device, tensors=t)
    k = torch.empty((2, 2000), dtype=torch.float64, device=ctx.device)
    err = ct.create_string_buffer(256)
    g = R.grid_struct(p.grid)
    rc = _noalloc_fn()(ct.c_void_p(ctx.stream.cuda_stream), ct.byref(dp.species.struct), ct.byref(lines.struct),
                       ct.byref(dp.cells.struct), ct.byref(g), 0, 2000, R.FP64, ct.c_void_p(k.data_ptr()),
                       ct.c_void_p(k.data_ptr()), 2000, err, 256)
    assert rc == R.ENOMEM
    assert b"scratch" in err.value


def test_noalloc_failed_check_does_not_leak_into_the_next_call():
    """A call whose cells fail the device-side check (negative temperature)
    leaves its status word in the shared scratch; the next valid call must
    clear it and match the regular entry point."""
    ctx = R.Context(0)
    bad = synth.uniform_slab(n_lines=50, n_cells=3, n_grid=5001)
    bad.cells.Ttr[1] = -100.0
    dp = solver.DeviceProblem(bad, ctx)
    k = torch.empty((dp.C, bad.grid.n), dtype=torch.float64, device=ctx.device)
    err = ct.create_string_buffer(256)
    rc = _call(ctx, dp, bad.grid, 0, bad.grid.n, R.FP64, k, k.clone(), err)
    assert rc == R.EINVAL and b"check" in err.value
    good = synth.uniform_slab(n_lines=200, n_cells=3, n_grid=20001)
    rk, rj, k2, j2 = _both(ctx, good, R.FP64)
    np.testing.assert_allclose(k2, rk, rtol=TOL, atol=1e-300)
    np.testing.assert_allclose(j2, rj, rtol=TOL, atol=1e-300)


def test_noalloc_refuses_tile_lists_beyond_its_scratch():
    """Few lines, but every window spans the whole grid of 65,535 FP32 tiles:
    300 x 65,535 tile-list entries (79 MB) do not fit the 64 MiB scratch."""
    ctx = R.Context(0)
    p = synth.uniform_slab(n_lines=300, n_cells=2, n_grid=65535 * 128)
    p.lines.lamS0[:] = 1e3
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    ctx.sync()
    k = torch.empty((dp.C, p.grid.n), dtype=torch.float32, device=ctx.device)
    err = ct.create_string_buffer(256)
    rc = _call(ctx, dp, p.grid, 0, p.grid.n, R.FP32, k, torch.empty_like(k), err)
    assert rc == R.ENOMEM and b"tile lists" in err.value, err.value
