"""The FP32-chosen path against the FP64 oracle, at the stated tolerances:
at most 1e-3 relative per spectral point where the quantity exceeds 1e-6 of
its maximum, at most 1e-4 on the integrated heat flux.  The measured errors
are printed (pytest -s) for the design notes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu

TOL_POINT = 1e-3
TOL_Q = 1e-4
MASK = 1e-6


@pytest.fixture(scope="module")
def ctx():
    return R.Context(0)


def point_error(gpu, ref, scale=None, what=""):
    """Largest relative error over points where |ref| >= 1e-6 max|ref|;
    `scale` (sum of term magnitudes) replaces |ref| as denominator for
    quantities whose terms can cancel."""
    gpu = np.asarray(gpu, np.float64); ref = np.asarray(ref, np.float64)
    den = np.abs(ref) if scale is None else np.maximum(np.abs(ref), np.asarray(scale))
    m = np.abs(ref) >= MASK * np.abs(ref).max()
    err = np.abs(gpu - ref)[m] / den[m]
    print(f"  {what}: max rel err {err.max():.3e} (p99 {np.quantile(err, 0.99):.3e}) over {m.sum()} points")
    return err.max()


def _coeffs(ctx, p, precision, tile=None):
    if tile:
        ctx.set_tiling(tile_width=tile)
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    dt = torch.float64 if precision == R.FP64 else torch.float32
    kap = torch.empty((dp.C, p.grid.n), dtype=dt, device=ctx.device)
    em = torch.empty_like(kap)
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, p.grid.n, precision, kap, em)
    ctx.sync()
    ctx.set_tiling(tile_width=-1)
    return kap.double().cpu().numpy(), em.double().cpu().numpy()


@pytest.mark.parametrize("tile", [128, 256, 512])
def test_coeffs_fp32_uniform_slab(ctx, tile):
    p = synth.uniform_slab(n_cells=2)
    kap, em = _coeffs(ctx, p, R.FP32, tile)
    rk, re, ra = oracle.spectral_coeffs(p, with_abs=True)
    assert point_error(em, re, what="j") <= TOL_POINT
    assert point_error(kap, rk, ra, what="kappa") <= TOL_POINT


def test_coeffs_fp32_stagnation(ctx):
    p = synth.stagnation_line(n_cells=16, n_atomic=4000, n_molecular=60000, n_grid=100001)
    kap, em = _coeffs(ctx, p, R.FP32)
    rk, re, ra = oracle.spectral_coeffs(p, with_abs=True)
    assert point_error(em, re, what="j") <= TOL_POINT
    assert point_error(kap, rk, ra, what="kappa") <= TOL_POINT


@pytest.mark.parametrize("tile,cpb,pb", [(128, 2, 32), (128, 4, 32), (128, 8, 32), (256, 4, 32), (512, 4, 32),
                                         (128, 4, 64), (256, 2, 64)])
def test_line_sum_launch_forms_are_bitwise_equal(ctx, tile, cpb, pb):
    """The FP32 line sum launched persistently (as many blocks as fit, or one
    block a SM, taking the units from a counter) and as one block per unit:
    the same coefficients to the bit and the same work counts, on a ragged
    cell count and a range that starts and ends inside a tile."""
    p = synth.stagnation_line(n_cells=19, n_atomic=3000, n_molecular=40000, n_grid=60001)
    dp = solver.DeviceProblem(p, ctx)
    k0, nk = 1234, 50000
    out = {}
    ctx.set_tiling(tile_width=tile, cells_per_block=cpb)
    ctx.set_line_batch(pb)
    try:
        for blocks in (-1, 1, 0):
            ctx.set_line_sum_blocks(blocks)
            R.populations(ctx, dp.species, dp.cells)
            kap = torch.empty((dp.C, nk), dtype=torch.float32, device=ctx.device)
            em = torch.empty_like(kap)
            ctx.reset_stats()
            R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, k0, nk, R.FP32, kap, em)
            ctx.sync()
            out[blocks] = (kap.cpu().numpy(), em.cpu().numpy(), ctx.get_stats())
    finally:
        ctx.set_line_sum_blocks(-1)
        ctx.set_line_batch(32)
        ctx.set_tiling(tile_width=-1, cells_per_block=4)
    for blocks in (1, 0):
        assert np.array_equal(out[blocks][0], out[-1][0]) and np.array_equal(out[blocks][1], out[-1][1]), blocks
        assert out[blocks][2] == out[-1][2]
    assert np.isfinite(out[-1][0]).all() and out[-1][2]["evaluations"] > 0


def test_line_sum_blocks_checked(ctx):
    for bad in (-2, 33):
        with pytest.raises(R.RapralError):
            ctx.set_line_sum_blocks(bad)
    ctx.set_line_sum_blocks(-1)
    for bad in (0, 16, 48, 128):
        with pytest.raises(R.RapralError):
            ctx.set_line_batch(bad)
    ctx.set_line_batch(32)


@pytest.mark.parametrize("pb", [32, 64])
def test_coeffs_fp32_pairs_per_pass(ctx, pb):
    """64 pairs a sweep pass against the oracle at the FP32 tolerance, on the
    two-temperature case with atoms and diatomics, and the same to the
    tolerance as 32 a pass (only the order of the terms in a point's sum
    differs)."""
    p = synth.stagnation_line(n_cells=8, n_atomic=3000, n_molecular=40000, n_grid=60001)
    ctx.set_line_batch(pb)
    try:
        kap, em = _coeffs(ctx, p, R.FP32)
    finally:
        ctx.set_line_batch(32)
    rk, re, ra = oracle.spectral_coeffs(p, with_abs=True)
    assert point_error(em, re, what=f"j, {pb} a pass") <= TOL_POINT
    assert point_error(kap, rk, ra, what=f"kappa, {pb} a pass") <= TOL_POINT


@pytest.mark.parametrize("tile", [None, 256])
def test_fp32_window_decisions_match_fp64(ctx, tile):
    """The FP32 path includes exactly the (line, point) pairs the FP64 path
    does, and both exactly those of the oracle's literal window test: the
    library's evaluation counter (the numerator of the line sum's roofline)
    equals the oracle's count of in-window (line, cell, point) triples on a
    two-temperature case."""
    p = synth.stagnation_line(n_cells=8, n_atomic=4000, n_molecular=20000, n_grid=80001)
    counts = {}
    for prec in (R.FP64, R.FP32):
        ctx.reset_stats()
        _coeffs(ctx, p, prec, tile)
        counts[prec] = ctx.get_stats()["evaluations"]
    oracle.spectral_coeffs(p)
    ref = oracle.last_evaluations()
    print(f"  evaluations: oracle {ref}, FP64 {counts[R.FP64]}, FP32 {counts[R.FP32]}")
    assert counts[R.FP64] == counts[R.FP32] == ref > 0


def test_slab_solve_fp32(ctx):
    p = synth.stagnation_line(n_cells=24, n_atomic=2000, n_molecular=30000, n_grid=50001)
    ref = oracle.solve_slab(p)
    dp = solver.DeviceProblem(p, ctx)
    out = solver.solve(dp, ctx, R.FP32, keep_intensity=True)
    ctx.sync()
    I = out["I"].double().cpu().numpy()
    for d in range(len(p.geometry.mu)):
        assert point_error(I[1 + d], ref["I_mu"][d], what=f"I mu{d}") <= TOL_POINT
    assert point_error(out["q_lambda"].double().cpu().numpy()[0], ref["q_lambda"], what="q_lambda") <= TOL_POINT
    q = out["q"].cpu().numpy()[0]
    print(f"  q: gpu {q!r} oracle {ref['q']!r} rel {abs(q / ref['q'] - 1):.3e}")
    assert abs(q / ref["q"] - 1) <= TOL_Q


def test_uniform_slab_fp32_flux(ctx):
    p = synth.uniform_slab()
    ref = oracle.solve_slab(p)
    dp = solver.DeviceProblem(p, ctx)
    out = solver.solve(dp, ctx, R.FP32)
    ctx.sync()
    q = out["q"].cpu().numpy()[0]
    print(f"  q: gpu {q!r} oracle {ref['q']!r} rel {abs(q / ref['q'] - 1):.3e}")
    assert abs(q / ref["q"] - 1) <= TOL_Q


@pytest.mark.parametrize("rays", [dict(), dict(n_points=2, n_mu=8, n_phi=16)], ids=["32rays", "128rays"])
def test_afterbody_small_fp32(ctx, rays):
    from test_gpu_parity import small_afterbody
    p = small_afterbody(**rays)
    dp = solver.DeviceProblem(p, ctx)
    out = solver.solve(dp, ctx, R.FP32)
    ctx.sync()
    rk, re = oracle.spectral_coeffs(p)
    qlam, q = oracle.solve_axisym_points(p, range(len(p.geometry.surf_x)), rk, re)
    assert point_error(out["q_lambda"].double().cpu().numpy(), qlam, what="q_lambda") <= TOL_POINT
    rel = np.abs(out["q"].cpu().numpy() / q - 1)
    print(f"  q rel err per point {rel}")
    assert rel.max() <= TOL_Q


def test_stagnation_full_size_sampled_fp32():
    """The benchmark's configuration (200 cells, 320k lines, 1e6 points,
    autotuned tiling): FP32 kappa and j at 600 sampled (cell, point) pairs
    against the oracle computed point by point, where the value is >= 1e-6
    of its row's maximum; q against the FP64 plain solve."""
    from paper_2604_11856_gb300 import autotune
    c = R.Context(0)
    p = synth.stagnation_line()
    autotune.tune(c, p)
    dp = solver.DeviceProblem(p, c)
    out = solver.solve(dp, c, R.FP32, keep_coeffs=True)
    c.sync()
    kap, em = out["kappa"], out["emis"]
    jmax = em.abs().amax(dim=1).double().cpu().numpy()
    kmax = kap.abs().amax(dim=1).double().cpu().numpy()
    rng = np.random.default_rng(12)
    # half uniform, half at line centres, where the spectrum is large
    h = (p.grid.lam_max - p.grid.lam_min) / (p.grid.n - 1)
    centres = np.rint((p.lines.lam0[rng.integers(0, len(p.lines), 300)] - p.grid.lam_min) / h).astype(np.int64)
    cells = rng.integers(0, 200, 600)
    ks = np.concatenate([rng.integers(0, p.grid.n, 300), np.clip(centres, 0, p.grid.n - 1)])
    lnp = oracle.lnpref(p)
    rk, re, ra = oracle.coeffs_at(p, cells, ks, lnp)
    ci = torch.as_tensor(cells, device=c.device); ki = torch.as_tensor(ks, device=c.device)
    gk = kap[ci, ki].double().cpu().numpy(); gj = em[ci, ki].double().cpu().numpy()
    mj = re >= MASK * jmax[cells]
    mk = np.maximum(np.abs(rk), ra) >= MASK * kmax[cells]
    ej = np.max(np.abs(gj - re)[mj] / re[mj])
    ek = np.max(np.abs(gk - rk)[mk] / np.maximum(np.abs(rk), ra)[mk])
    print(f"  j: {ej:.3e} over {mj.sum()} points, kappa: {ek:.3e} over {mk.sum()} points")
    assert mj.sum() > 100 and ej <= TOL_POINT and ek <= TOL_POINT
    q32 = float(out["q"].item())
    q64 = float(solver.solve(dp, c, R.FP64)["q"].item())
    c.sync()
    print(f"  q fp32 {q32:.8e} fp64 {q64:.8e}")
    assert abs(q32 / q64 - 1) <= 1e-4
    c.close()
