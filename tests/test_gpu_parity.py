"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 path: every kappa, j, intensity, spectral flux and flux agrees with the
oracle to 1e-10 relative.  For kappa the scale of the comparison is the sum
of the magnitudes of the terms (the sum can cancel where stimulated emission
exceeds absorption); j, I, q_lambda and q are sums of non-negative terms and
are compared against their own magnitude.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def ctx():
    return R.Context(0)


def _close(gpu, ref, scale, tol, what):
    gpu = np.asarray(gpu, np.float64); ref = np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(np.asarray(scale, np.float64)), np.abs(ref))
    err = np.abs(gpu - ref)
    bad = err > tol * scale + 1e-300
    if np.any(bad):
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} beyond {tol}; first at {tuple(i)}: "
                             f"gpu={gpu[tuple(i)]!r} ref={ref[tuple(i)]!r} scale={scale[tuple(i)]!r}")
    return float(np.max(err / np.where(scale > 0, scale, 1.0)))


def small_stagnation(n_cells=24, n_atomic=2000, n_molecular=30000, n_grid=60001):
    return synth.stagnation_line(n_cells=n_cells, n_atomic=n_atomic, n_molecular=n_molecular, n_grid=n_grid)


# ---------------------------------------------------------------- populations

@pytest.mark.parametrize("make", [lambda: synth.uniform_slab(), lambda: small_stagnation(n_cells=50)])
def test_populations_fp64(ctx, make):
    p = make()
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    ctx.sync()
    g = dp.cells.lnpref.cpu().numpy()
    ref = oracle.lnpref(p)
    assert np.array_equal(np.isneginf(g), np.isneginf(ref))
    f = np.isfinite(ref)
    np.testing.assert_allclose(g[f], ref[f], rtol=1e-13, atol=1e-12)


# ------------------------------------------------------------- coefficients

def _coeffs(ctx, p, precision=R.FP64, k0=0, nk=None, tile=None):
    if tile:
        ctx.set_tiling(tile_width=tile)
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    nk = p.grid.n - k0 if nk is None else nk
    dt = torch.float64 if precision == R.FP64 else torch.float32
    kap = torch.empty((dp.C, nk), dtype=dt, device=ctx.device)
    em = torch.empty((dp.C, nk), dtype=dt, device=ctx.device)
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, k0, nk, precision, kap, em)
    ctx.sync()
    if tile:
        ctx.set_tiling(tile_width=-1)
    return kap.cpu().numpy(), em.cpu().numpy()


def test_coeffs_fp64_uniform_slab(ctx):
    p = synth.uniform_slab(n_cells=3)
    kap, em = _coeffs(ctx, p)
    rk, re, ra = oracle.spectral_coeffs(p, with_abs=True)
    _close(em, re, re, TOL64, "j")
    _close(kap, rk, ra, TOL64, "kappa")


@pytest.mark.parametrize("tile", [128, 256, 512])
def test_coeffs_fp64_stagnation_ranges(ctx, tile):
    """Two-temperature cells with atoms and diatomics, a range that starts
    inside the grid and ends in a ragged last tile."""
    p = small_stagnation(n_cells=12, n_grid=40001)
    k0, nk = 1234, 30001
    kap, em = _coeffs(ctx, p, k0=k0, nk=nk, tile=tile)
    rk, re, ra = oracle.spectral_coeffs(p, k0=k0, nk=nk, with_abs=True)
    _close(em, re, re, TOL64, "j")
    _close(kap, rk, ra, TOL64, "kappa")


def test_coeffs_unsorted_lines_same_result(ctx):
    p = small_stagnation(n_cells=4, n_atomic=400, n_molecular=3000, n_grid=20001)
    kap, em = _coeffs(ctx, p)
    perm = np.random.default_rng(0).permutation(len(p.lines))
    q = synth.Problem(p.name, p.species, synth.Lines(**{k: getattr(p.lines, k)[perm] for k in synth.Lines.__dataclass_fields__}),
                      p.cells, p.grid, p.geometry)
    kap2, em2 = _coeffs(ctx, q)
    np.testing.assert_allclose(kap2, kap, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(em2, em, rtol=1e-12, atol=1e-300)


def test_coeffs_empty_lines_and_single_cell(ctx):
    p = small_stagnation(n_cells=1, n_atomic=4, n_molecular=0, n_grid=2000)
    kap, em = _coeffs(ctx, p)
    rk, re, ra = oracle.spectral_coeffs(p, with_abs=True)
    _close(em, re, re, TOL64, "j")
    empty = synth.Problem(p.name, p.species, synth.subset_lines(p.lines, []), p.cells, p.grid, p.geometry)
    kap0, em0 = _coeffs(ctx, empty)
    assert not kap0.any() and not em0.any()


# --------------------------------------------------------------- whole solve

def test_uniform_slab_solve_fp64(ctx):
    p = synth.uniform_slab()
    dp = solver.DeviceProblem(p, ctx)
    out = solver.solve(dp, ctx, R.FP64, keep_coeffs=True, keep_intensity=True)
    ctx.sync()
    ref = oracle.solve_slab(p)
    I = out["I"].cpu().numpy()
    _close(I[0], ref["I_normal"], ref["I_normal"], TOL64, "I normal")
    _close(I[1:], ref["I_mu"], ref["I_mu"], TOL64, "I mu")
    _close(out["q_lambda"].cpu().numpy()[0], ref["q_lambda"], ref["q_lambda"], TOL64, "q_lambda")
    _close(out["q"].cpu().numpy(), [ref["q"]], [ref["q"]], TOL64, "q")


def test_stagnation_solve_fp64_chunked(ctx):
    """Reduced stagnation line: full comparison of q_lambda and q, solved
    whole and in uneven spectral chunks (one stream and two streams)."""
    p = small_stagnation(n_cells=24, n_grid=50001)
    ref = oracle.solve_slab(p)
    dp = solver.DeviceProblem(p, ctx)
    whole = solver.solve(dp, ctx, R.FP64)
    ctx.sync()
    _close(whole["q_lambda"].cpu().numpy()[0], ref["q_lambda"], ref["q_lambda"], TOL64, "q_lambda")
    _close(whole["q"].cpu().numpy(), [ref["q"]], [ref["q"]], TOL64, "q")
    parts = solver.solve(dp, ctx, R.FP64, chunk=12345)
    ctx.sync()
    _close(parts["q"].cpu().numpy(), [ref["q"]], [ref["q"]], TOL64, "q chunked")
    s2 = torch.cuda.Stream()
    ctx2 = R.Context(0, stream=s2)
    two = solver.solve(dp, ctx, R.FP64, chunk=9999, ctx2=ctx2)
    ctx.sync(); ctx2.sync()
    _close(two["q"].cpu().numpy(), [ref["q"]], [ref["q"]], TOL64, "q two streams")


def test_stagnation_full_size_sampled_fp64(ctx):
    """The full stagnation line (200 cells, 320k lines, 1e6 points):
    kappa and j at 200 sampled (cell, point) pairs and the whole march at
    sampled wavelengths, against the oracle computed point by point."""
    p = synth.stagnation_line()
    dp = solver.DeviceProblem(p, ctx)
    out = solver.solve(dp, ctx, R.FP64, keep_coeffs=True, keep_intensity=True)
    ctx.sync()
    rng = np.random.default_rng(11)
    lnp = oracle.lnpref(p)
    cells = rng.integers(0, 200, 200); ks = rng.integers(0, p.grid.n, 200)
    rk, re, ra = oracle.coeffs_at(p, cells, ks, lnp)
    kap = out["kappa"][torch.as_tensor(cells, device=ctx.device), torch.as_tensor(ks, device=ctx.device)].cpu().numpy()
    em = out["emis"][torch.as_tensor(cells, device=ctx.device), torch.as_tensor(ks, device=ctx.device)].cpu().numpy()
    _close(em, re, re, TOL64, "j sampled")
    _close(kap, rk, ra, TOL64, "kappa sampled")
    # whole columns at a few wavelengths, marched by the oracle
    cols = np.sort(rng.integers(0, p.grid.n, 6))
    cc = np.repeat(np.arange(200), len(cols)); kk = np.tile(cols, 200)
    ck, ce, _ = oracle.coeffs_at(p, cc, kk, lnp)
    K = ck.reshape(200, len(cols)); E = ce.reshape(200, len(cols))
    I = out["I"][:, torch.as_tensor(cols, device=ctx.device)].cpu().numpy()
    geo = p.geometry
    for j, k in enumerate(cols):
        sub = synth.Grid(p.grid.lam_min, p.grid.lam_max, p.grid.n)
        for d, mu in enumerate(geo.mu):
            ref = oracle.march(geo.cell_order, geo.dx, 1.0 / mu, K[:, j:j + 1], E[:, j:j + 1], sub, k0=int(k))[0]
            _close(I[1 + d, j], ref, ref, TOL64, f"I(mu={mu:.3f}, k={k})")


# ------------------------------------------------------------------ geometry

def small_afterbody(nx=40, nr=20, n_points=3, n_mu=4, n_phi=8, n_atomic=400, n_molecular=3000, n_grid=8001):
    base = synth.stagnation_line(n_cells=2, n_atomic=n_atomic, n_molecular=n_molecular, n_grid=n_grid)
    return synth.afterbody(nx=nx, nr=nr, x_len=20.0, r_body=3.35, r_len=15.0, n_points=n_points, n_mu=n_mu,
                           n_phi=n_phi, n_grid=n_grid, lines_from=base, chunk=0)


def test_axisym_segments_match_oracle(ctx):
    p = small_afterbody(n_points=5, n_mu=6, n_phi=12)
    dp = solver.DeviceProblem(p, ctx)
    ctx.sync()
    t = dp.rays.t
    off = t["seg_off"].cpu().numpy(); cell = t["seg_cell"].cpu().numpy(); ds = t["seg_ds"].cpu().numpy()
    dirs, wts = oracle.hemisphere_directions(p.geometry)
    np.testing.assert_allclose(t["dir_weight"].cpu().numpy(), np.tile(wts, 5), rtol=1e-14)
    b = 0
    for ip in range(5):
        for d in dirs:
            rc, rds = oracle.axisym_segments(p.geometry, p.geometry.surf_x[ip], d)
            gc, gds = cell[off[b]:off[b + 1]], ds[off[b]:off[b + 1]]
            assert np.array_equal(gc, rc), f"ray {b}"
            np.testing.assert_allclose(gds, rds, rtol=1e-9, atol=1e-12)
            b += 1


@pytest.mark.parametrize("rays", [dict(), dict(n_points=2, n_mu=8, n_phi=16)], ids=["32rays", "128rays"])
def test_afterbody_small_solve_fp64(ctx, rays):
    """32 rays a point: one block per (point, wavelength tile); 128 rays a
    point: the point's rays split over several blocks, whose partial
    spectral fluxes are added in a fixed order."""
    p = small_afterbody(**rays)
    dp = solver.DeviceProblem(p, ctx)
    out = solver.solve(dp, ctx, R.FP64, keep_coeffs=True)
    ctx.sync()
    rk, re = oracle.spectral_coeffs(p)
    qlam, q = oracle.solve_axisym_points(p, range(len(p.geometry.surf_x)), rk, re)
    _close(out["q_lambda"].cpu().numpy(), qlam, qlam, TOL64, "q_lambda")
    _close(out["q"].cpu().numpy(), q, q, TOL64, "q")


@pytest.mark.parametrize("precision", [R.FP64, R.FP32])
def test_march_wavelength_ranges_match_whole(ctx, precision):
    """Marching a range of columns (views into the coefficient rows) gives
    each column what the march of the whole grid gives it: the ranges cover
    a single-lane tile (nk < 32), a partial second tile and the grid's last
    columns, so the wavelength tiling and the shifted last tile change no
    result."""
    p = small_afterbody(n_points=4, n_mu=8, n_phi=16)
    dp = solver.DeviceProblem(p, ctx)
    n = p.grid.n
    out = solver.solve(dp, ctx, precision, keep_coeffs=True, keep_intensity=True)
    ctx.sync()
    kap, em = out["kappa"], out["emis"]
    ql_all = out["q_lambda"].double().cpu().numpy()
    I_all = out["I"].double().cpu().numpy()
    dt = kap.dtype
    tol = 0.0 if precision == R.FP64 else 2.4e-7
    for a, nk in [(0, 5), (13, 71), (4000, 1), (n - 70, 70), (777, 2500)]:
        ql = torch.empty((dp.P, nk), dtype=dt, device=ctx.device)
        I = torch.empty((dp.rays.n_dirs, nk), dtype=dt, device=ctx.device)
        R.trace_rays(ctx, dp.rays, dp.C, kap[:, a:a + nk], em[:, a:a + nk], p.grid, a, nk, precision, ql, I)
        ctx.sync()
        for got, ref, what in ((ql, ql_all, "q_lambda"), (I, I_all, "I")):
            g = got.double().cpu().numpy()
            r = ref[:, a:a + nk]
            err = np.max(np.abs(g - r) / np.maximum(np.abs(r), 1e-300))
            assert err <= tol, (a, nk, what, err)


@pytest.mark.parametrize("n_mu", [16, 64])
@pytest.mark.parametrize("precision", [R.FP64, R.FP32])
def test_single_direction_bundles_from_wall(ctx, n_mu, precision):
    """A slab with a hot wall at its far end, every direction its own bundle
    (as a caller-built ray set): the single-direction march, starting from
    the wall's Planck intensity, agrees with the oracle's slab solve; with
    64 bundles the point's bundles are split over two blocks."""
    base = small_stagnation(n_cells=12, n_atomic=500, n_molecular=5000, n_grid=9001)
    mu, w = synth.gauss_legendre_01(n_mu)
    geo = synth.SlabGeometry(cell_order=base.geometry.cell_order, dx=base.geometry.dx, mu=mu, wmu=w,
                             normal_ray=False, wall_start=True, T_wall=3000.0)
    p = synth.Problem("wall slab", base.species, base.lines, base.cells, base.grid, geo)
    ref = oracle.solve_slab(p)
    m = len(geo.cell_order)
    rays = R.rays_from_arrays(point_off=[0, n_mu], seg_off=np.arange(n_mu + 1) * m,
                              seg_cell=np.tile(geo.cell_order, n_mu), seg_ds=np.tile(geo.dx, n_mu),
                              dir_off=np.arange(n_mu + 1), dir_scale=1.0 / mu, dir_weight=2 * np.pi * w * mu,
                              bundle_wall=np.ones(n_mu), T_wall=geo.T_wall, device=ctx.device)
    dp = solver.DeviceProblem(p, ctx)
    dt = torch.float64 if precision == R.FP64 else torch.float32
    n = p.grid.n
    kap = torch.empty((dp.C, n), dtype=dt, device=ctx.device); em = torch.empty_like(kap)
    R.populations(ctx, dp.species, dp.cells)
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, n, precision, kap, em)
    ql = torch.empty((1, n), dtype=dt, device=ctx.device)
    I = torch.empty((n_mu, n), dtype=dt, device=ctx.device)
    R.trace_rays(ctx, rays, dp.C, kap, em, p.grid, 0, n, precision, ql, I)
    ctx.sync()
    if precision == R.FP64:
        _close(I.cpu().numpy(), ref["I_mu"], ref["I_mu"], TOL64, "I")
        _close(ql.cpu().numpy()[0], ref["q_lambda"], ref["q_lambda"], TOL64, "q_lambda")
    else:
        g = ql.double().cpu().numpy()[0]
        big = ref["q_lambda"] >= 1e-6 * ref["q_lambda"].max()
        assert np.max(np.abs(g - ref["q_lambda"])[big] / ref["q_lambda"][big]) <= 1e-3


# ------------------------------------------------------------------- errors

def test_device_checks_report_einval(ctx):
    p = synth.uniform_slab(n_lines=10, n_cells=2, n_grid=1000)
    p.cells.Ttr[1] = np.nan
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    with pytest.raises(R.RapralError) as e:
        ctx.sync()
    assert e.value.code == R.EINVAL and "temperature" in str(e.value)
    ctx.clear_status()
    ctx.sync()


def test_host_checks_report_einval(ctx):
    p = synth.uniform_slab(n_lines=10, n_cells=2, n_grid=1000)
    dp = solver.DeviceProblem(p, ctx)
    kap = torch.empty((2, 100), dtype=torch.float64, device=ctx.device)
    with pytest.raises(R.RapralError) as e:
        R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 950, 100, R.FP64, kap, kap.clone())
    assert e.value.code == R.EINVAL
    ctx.sync()


def test_bad_segment_cell_reports_einval(ctx):
    p = synth.uniform_slab(n_lines=10, n_cells=2, n_grid=1000)
    p.geometry.cell_order[1] = 7
    dp = solver.DeviceProblem(p, ctx)
    kap = torch.zeros((2, 10), dtype=torch.float64, device=ctx.device)
    ql = torch.zeros((1, 10), dtype=torch.float64, device=ctx.device)
    R.trace_rays(ctx, dp.rays, 2, kap, kap, p.grid, 0, 10, R.FP64, ql)
    with pytest.raises(R.RapralError) as e:
        ctx.sync()
    assert e.value.code == R.EINVAL and "segment cell" in str(e.value)
    ctx.clear_status()
    ctx.sync()


def test_slab_many_directions_fp64(ctx):
    """More directions than one bundle holds: the slab is split into bundles
    that repeat the cell path; results still match the oracle."""
    p = synth.uniform_slab(n_lines=300, n_cells=8, n_grid=20001, n_mu=40)
    dp = solver.DeviceProblem(p, ctx)
    out = solver.solve(dp, ctx, R.FP64, keep_intensity=True)
    ctx.sync()
    ref = oracle.solve_slab(p)
    I = out["I"].cpu().numpy()
    _close(I[1:], ref["I_mu"], ref["I_mu"], TOL64, "I mu")
    _close(out["q"].cpu().numpy(), [ref["q"]], [ref["q"]], TOL64, "q")


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("dealt", [False, True])
def test_spectral_shards_sum_to_whole(ctx, world, dealt):
    """The multi-GPU path's spectral sharding (solver.solve_sharded) run for
    every rank one after another on one GPU, its all-reduce skipped and the
    partial fluxes summed on the host, equals the unsharded flux: contiguous
    shards whose edges fall inside the unsharded solve's chunks, and chunks
    dealt round-robin, each on the two-stream pipeline."""
    import torch
    p = small_stagnation(n_cells=10, n_grid=30001)
    dp = solver.DeviceProblem(p, ctx)
    chunk = 7000
    whole = solver.solve(dp, ctx, R.FP64, chunk=chunk)["q"].cpu().numpy()
    ctx2 = R.Context(0, stream=torch.cuda.Stream())
    parts = np.zeros_like(whole)
    for rank in range(world):
        q = solver.solve_sharded(dp, ctx, rank, world, R.FP64, chunk=chunk, ctx2=ctx2, dealt=dealt, reduce=False)
        parts += q.cpu().numpy()
    ctx.sync(); ctx2.sync()
    if not dealt:   # a shard edge inside a chunk of the unsharded solve
        assert any(solver.shard_range(p.grid.n, r, world)[0] % chunk for r in range(1, world))
    _close(parts, whole, whole, 1e-13, f"q over {world} shards")