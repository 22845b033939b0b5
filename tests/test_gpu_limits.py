"""Size limits and input checks of the planning steps, through the C ABI.

The tile lists of the line sum are indexed by int32 offsets: a request whose
line windows give more than 2^31 - 1 (line, tile) entries must be refused
before anything is filled (EINVAL), and the context must stay usable.  The
batch planner must report a failed device-side input check as EINVAL before
it sizes anything from the tile counts."""
import numpy as np
import pytest
import torch

from paper_2604_11856_gb300 import batch, rapral as R, solver, synth

pytestmark = pytest.mark.gpu

N_TILES = 65535          # the most tiles one call may have
TILE_FP32 = 128          # default FP32 tile width


def wide_window_problem(n_lines, n_cells=2):
    """Lines whose Lorentz width (Stark HWHM 1e3 nm at the reference state)
    puts the whole grid inside every window, on a grid of exactly N_TILES
    FP32 tiles: every line lands in every tile."""
    n_grid = N_TILES * TILE_FP32
    p = synth.uniform_slab(n_lines=n_lines, n_cells=n_cells, n_grid=n_grid)
    p.lines.lamS0[:] = 1e3
    return p


def test_tile_list_entries_beyond_int32_are_refused():
    ctx = R.Context(0)
    L = 40_000            # 40,000 x 65,535 = 2.62e9 > 2^31 - 1
    p = wide_window_problem(L)
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    nk = p.grid.n
    kap = torch.empty((dp.C, nk), dtype=torch.float32, device=ctx.device)
    em = torch.empty_like(kap)
    with pytest.raises(R.RapralError) as e:
        R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, nk, R.FP32, kap, em)
    assert e.value.code == R.EINVAL and "2^31" in str(e.value)
    ctx.sync()   # nothing failed on the device; the context is usable
    # the same lines over a few tiles fit
    nk2 = 10 * TILE_FP32
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, nk2, R.FP32, kap[:, :nk2], em[:, :nk2])
    ctx.sync()
    assert torch.isfinite(kap[:, :nk2]).all() and (em[:, :nk2] > 0).all()


def test_batch_planning_reports_a_failed_device_check():
    ctx = R.Context(0)
    pool = synth._air_lines(np.random.default_rng(1001), 200, 2000)
    probs = synth.batch_slabs(n_solves=3, pool=pool, scale=0.002)
    probs[1].cells.Ttr[0] = -5.0
    with pytest.raises(R.RapralError) as e:
        batch.BatchSolver(probs, ctx, chunk=2000)
    assert e.value.code == R.EINVAL and "temperature" in str(e.value)
    ctx.clear_status()
    ctx.sync()
