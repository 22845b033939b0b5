"""The axisymmetric afterbody at full size (400 x 200 cells, 320k lines, a
1e6-point grid in 65,536-point chunks, 200 surface points x 512 rays).

1. The whole FP32 solve (two-stream chunk pipeline) gives 200 finite,
   positive wall fluxes.
2. On a 8,192-point range across a seam of that chunking, cut into two
   4,096-point chunks, every one of the 200 FP32 fluxes equals the FP64 GPU
   path's within 1e-4 (the FP64 path itself is held to the oracle at 1e-10).
3. The oracle on a subsample: 4 surface points x all 512 rays, the cells
   those rays cross, a 2,048-point range at the same seam.  It computes
   kappa / j of the crossed cells from the lines that can reach the range
   (a line farther from the range than 1.5 times the widest window any line
   has in any cell contributes nothing, and that width is checked), marches
   every ray and sums q_lambda and q.  FP64: q_lambda and q within 1e-10,
   and the 512 intensities of one point within 1e-10; FP32: q_lambda within
   1e-3 (where above 1e-6 of its maximum) and q within 1e-4.
Sampled kappa / j of one whole chunk are also checked against the oracle's
point evaluation."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu

POINTS = [0, 66, 133, 199]
TOL64, TOL_POINT, TOL_Q, MASK = 1e-10, 1e-3, 1e-4, 1e-6


@pytest.fixture(scope="module")
def setup():
    p = synth.afterbody()
    ctx = R.Context(0)
    ctx2 = R.Context(0, stream=torch.cuda.Stream())
    dp = solver.DeviceProblem(p, ctx)
    ctx.sync()
    return p, ctx, ctx2, dp


def test_afterbody_whole_solve_and_sampled_coefficients(setup):
    p, ctx, ctx2, dp = setup
    out = solver.solve(dp, ctx, R.FP32, chunk=p.chunk, ctx2=ctx2)
    ctx.sync(); ctx2.sync()
    q = out["q"].cpu().numpy()
    assert q.shape == (200,) and np.all(np.isfinite(q)) and np.all(q > 0)

    # one chunk again, with its coefficients kept, to check sampled outputs
    k0, nk = 4 * p.chunk, p.chunk
    kap = torch.empty((dp.C, nk), dtype=torch.float32, device=ctx.device)
    em = torch.empty_like(kap)
    R.populations(ctx, dp.species, dp.cells)
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, k0, nk, R.FP32, kap, em)
    ctx.sync()
    rng = np.random.default_rng(3)
    lnp = oracle.lnpref(p)
    cells = rng.integers(0, dp.C, 60)
    ks = rng.integers(k0, k0 + nk, 60)
    rk, re, ra = oracle.coeffs_at(p, cells, ks, lnp)
    idx = (torch.as_tensor(cells, device=ctx.device), torch.as_tensor(ks - k0, device=ctx.device))
    gk = kap[idx].double().cpu().numpy()
    gj = em[idx].double().cpu().numpy()
    big = re >= 1e-6 * re.max()
    assert np.all(np.abs(gj - re)[big] <= 1e-3 * re[big])
    bigk = np.abs(rk) >= 1e-6 * np.abs(rk).max()
    assert np.all(np.abs(gk - rk)[bigk] <= 1e-3 * np.maximum(np.abs(rk), ra)[bigk])


def test_afterbody_fp32_fluxes_equal_fp64_across_a_seam(setup):
    p, ctx, ctx2, dp = setup
    seam = p.chunk
    ka, kb = seam - 4096, seam + 4096
    q32 = solver.solve(dp, ctx, R.FP32, chunk=4096, k_start=ka, k_stop=kb)["q"].cpu().numpy()
    q64 = solver.solve(dp, ctx, R.FP64, chunk=4096, k_start=ka, k_stop=kb)["q"].cpu().numpy()
    ctx.sync()
    assert np.all(q64 > 0)
    err = np.abs(q32 / q64 - 1)
    print(f"  200 points, {kb - ka} grid points: max |q32/q64 - 1| = {err.max():.3e} (median {np.median(err):.2e})")
    assert err.max() <= TOL_Q


def _reachable_lines(p, lnp, lo_nm, hi_nm):
    """Indices of the lines that can reach [lo_nm, hi_nm] in some cell, and
    the widest window half-width found.  Every line's Doppler width grows
    with T_tr and its Lorentz width with one cell factor (the Stark factor),
    so the cells where the single line of largest Stark coefficient is
    widest give every line's largest widths."""
    ln = p.lines
    probe = int(np.argmax(ln.lamS0))
    one = synth.Problem(p.name, p.species, synth.subset_lines(ln, [probe]), p.cells, p.grid, p.geometry)
    w = oracle.line_widths_all_cells(one, lnp)
    G, L = w["lamG"][:, 0], w["lamL"][:, 0]
    sG = oracle.line_states(p, lnp, int(np.argmax(G)))
    sL = oracle.line_states(p, lnp, int(np.argmax(L)))
    half = 100.0 * (sG["lamG"] + sL["lamL"])   # lamV <= lamL + lamG for Whiting's fit
    wmax = float(half.max())
    margin = 1.5 * wmax
    keep = np.nonzero((ln.lam0 >= lo_nm - margin) & (ln.lam0 <= hi_nm + margin))[0]
    return keep, wmax


SUB_K0_OFFSET, SUB_NK = -1024, 2048   # the subsample's range, relative to the seam at one chunk


@pytest.fixture(scope="module")
def oracle_subsample(setup):
    """The oracle's q_lambda and q of the 4 points over the subsample range,
    with the compact kappa / j tables of the crossed cells."""
    p = setup[0]
    geo, g = p.geometry, p.grid
    k0, nk = p.chunk + SUB_K0_OFFSET, SUB_NK
    h = (g.lam_max - g.lam_min) / (g.n - 1)
    lo, hi = g.lam_min + k0 * h, g.lam_min + (k0 + nk - 1) * h
    dirs, _w = oracle.hemisphere_directions(geo)
    crossed = sorted({int(c) for pt in POINTS for d in dirs for c in oracle.axisym_segments(geo, geo.surf_x[pt], d)[0]})
    crossed = np.asarray(crossed, np.int64)
    rows = np.full(len(p.cells), -1, np.int64)
    rows[crossed] = np.arange(len(crossed))
    lnp = oracle.lnpref(p)
    keep, wmax = _reachable_lines(p, lnp, lo, hi)
    assert 1.5 * wmax < 0.5 * (g.lam_max - g.lam_min)
    cells = synth.Cells(Ttr=p.cells.Ttr[crossed], Tve=p.cells.Tve[crossed], n=p.cells.n[crossed])
    small = synth.Problem(p.name, p.species, synth.subset_lines(p.lines, keep), cells, g, geo)
    kap, em = oracle.spectral_coeffs(small, lnp[crossed], k0, nk)
    rql, rq = oracle.solve_axisym_points(p, POINTS, kap, em, k0, rows=rows)
    print(f"  {len(crossed)} crossed cells, {len(keep)} of {len(p.lines)} lines reach [{lo:.2f}, {hi:.2f}] nm "
          f"(widest window {wmax:.3f} nm)")
    return dict(k0=k0, nk=nk, rows=rows, kap=kap, em=em, q_lambda=rql, q=rq, dirs=dirs)


@pytest.mark.parametrize("precision", [R.FP64, R.FP32])
def test_afterbody_subsample_matches_oracle(setup, oracle_subsample, precision):
    p, ctx, ctx2, dp = setup
    o = oracle_subsample
    geo, g, k0, nk = p.geometry, p.grid, o["k0"], o["nk"]
    # GPU: the 4 points' 512 rays each, one chunk, intensities kept
    sub = solver.DeviceProblem(p, ctx, points=POINTS, lines=dp.lines, species=dp.species)
    out = solver.solve(sub, ctx, precision, k_start=k0, k_stop=k0 + nk, keep_intensity=True)
    ctx.sync()
    gq = out["q"].cpu().numpy()
    gql = out["q_lambda"].double().cpu().numpy()
    rql, rq = o["q_lambda"], o["q"]
    err_q = np.abs(gq / rq - 1)
    m = rql >= MASK * rql.max(axis=1, keepdims=True)
    err_ql = (np.abs(gql - rql) / np.where(m, rql, 1.0))[m]
    print(f"  q: max rel err {err_q.max():.3e}; q_lambda: max rel err {err_ql.max():.3e} over {m.sum()} points")
    if precision == R.FP64:
        assert err_q.max() <= TOL64
        assert np.all(np.abs(gql - rql) <= TOL64 * np.abs(rql) + 1e-300)
        # the 512 intensities of the first point, ray by ray (bundles are the point's rays in order)
        gI = out["I"].double().cpu().numpy()
        for b, d in enumerate(o["dirs"]):
            cl, ds = oracle.axisym_segments(geo, geo.surf_x[POINTS[0]], d)
            ref = oracle.march(o["rows"][cl], ds, 1.0, o["kap"], o["em"], g, k0)
            assert np.all(np.abs(gI[b] - ref) <= TOL64 * np.abs(ref) + 1e-300), b
    else:
        assert err_q.max() <= TOL_Q
        assert err_ql.max() <= TOL_POINT
