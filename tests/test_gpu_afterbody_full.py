"""The axisymmetric afterbody at full size (400 x 200 cells, 320k lines, a
1e6-point grid in 65,536-point chunks, 200 surface points x 512 rays), FP32
chunk pipeline on two streams.  The oracle cannot march it whole; it checks
sampled outputs: kappa and j at sampled (cell, point) pairs, and the
intensity along sampled rays at sampled wavelengths, marched by the oracle
through the cells those rays cross."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu


def test_afterbody_full_size_fp32():
    p = synth.afterbody()
    ctx = R.Context(0)
    ctx2 = R.Context(0, stream=torch.cuda.Stream())
    dp = solver.DeviceProblem(p, ctx)
    out = solver.solve(dp, ctx, R.FP32, chunk=p.chunk, ctx2=ctx2)
    ctx.sync(); ctx2.sync()
    q = out["q"].cpu().numpy()
    assert q.shape == (200,) and np.all(np.isfinite(q)) and np.all(q > 0)

    # one chunk again, with its coefficients kept, to check sampled outputs
    k0, nk = 4 * p.chunk, p.chunk
    kap = torch.empty((dp.C, nk), dtype=torch.float32, device=ctx.device)
    em = torch.empty_like(kap)
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, k0, nk, R.FP32, kap, em)
    ctx.sync()
    rng = np.random.default_rng(3)
    lnp = oracle.lnpref(p)
    cells = rng.integers(0, dp.C, 60)
    ks = rng.integers(k0, k0 + nk, 60)
    rk, re, ra = oracle.coeffs_at(p, cells, ks, lnp)
    gk = kap[torch.as_tensor(cells, device=ctx.device), torch.as_tensor(ks - k0, device=ctx.device)].double().cpu().numpy()
    gj = em[torch.as_tensor(cells, device=ctx.device), torch.as_tensor(ks - k0, device=ctx.device)].double().cpu().numpy()
    big = re >= 1e-6 * re.max()
    assert np.all(np.abs(gj - re)[big] <= 1e-3 * re[big])
    bigk = np.abs(rk) >= 1e-6 * np.abs(rk).max()
    assert np.all(np.abs(gk - rk)[bigk] <= 1e-3 * np.maximum(np.abs(rk), ra)[bigk])

    # rays of one surface point, intensities at three wavelengths of the chunk
    point = 57
    sub = solver.DeviceProblem(p, ctx, points=[point], lines=dp.lines, species=dp.species)
    R.populations(ctx, sub.species, sub.cells)
    ql = torch.empty((1, nk), dtype=torch.float32, device=ctx.device)
    I = torch.empty((sub.rays.n_dirs, nk), dtype=torch.float32, device=ctx.device)
    R.trace_rays(ctx, sub.rays, sub.C, kap, em, p.grid, k0, nk, R.FP32, ql, I)
    ctx.sync()
    dirs, _w = oracle.hemisphere_directions(p.geometry)
    cols = np.sort(rng.integers(0, nk, 3))
    for b in rng.choice(len(dirs), 6, replace=False):
        cl, ds = oracle.axisym_segments(p.geometry, p.geometry.surf_x[point], dirs[b])
        cc = np.repeat(cl, len(cols)); kk = np.tile(k0 + cols, len(cl))
        ck, ce, _ = oracle.coeffs_at(p, cc, kk, lnp)
        K = np.zeros((dp.C, len(cols))); E = np.zeros((dp.C, len(cols)))
        K[cl] = ck.reshape(len(cl), len(cols)); E[cl] = ce.reshape(len(cl), len(cols))
        for j, kcol in enumerate(cols):
            ref = oracle.march(cl, ds, 1.0, K[:, j:j + 1], E[:, j:j + 1], p.grid, k0=k0 + int(kcol))[0]
            got = float(I[b, kcol].item())
            assert abs(got - ref) <= 1e-3 * abs(ref) + 1e-30, (b, kcol, got, ref)
