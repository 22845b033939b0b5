"""The paper's own angular path on the GPU (Fibonacci lines of sight, node
states, node march, per-line wavelength integral, angular interpolation and
four-point sum) against the oracle of oracle/los.py.  FP64: 1e-10 relative
on every per-line intensity, S and q; FP32: the FP32 tolerances."""
import numpy as np
import pytest
import torch

import oracle
from oracle import los
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def ctx():
    return R.Context(0)


def small_problem(n_points=2, n_grid=8001, nx=40, nr=20):
    base = synth.stagnation_line(n_cells=2, n_atomic=400, n_molecular=3000, n_grid=n_grid)
    return synth.afterbody(nx=nx, nr=nr, x_len=20.0, r_body=3.35, r_len=15.0, n_points=n_points, n_mu=4,
                           n_phi=8, n_grid=n_grid, lines_from=base, chunk=0)


def test_fibonacci_rays_and_nodes_match_oracle(ctx):
    p = small_problem()
    geo = p.geometry
    rays = R.fibonacci_rays(ctx, geo, 64, ctx.device)
    ctx.sync()
    t = rays.t
    off = t["seg_off"].cpu().numpy(); ds = t["seg_ds"].cpu().numpy()
    nxp = t["node_x"].cpu().numpy(); nrp = t["node_r"].cpu().numpy()
    li = t["los_index"].cpu().numpy()
    dirs = los.fibonacci_directions(64)
    keep = los.valid_los(64)
    assert rays.n_dirs == 2 * len(keep)
    b = 0
    for ip in range(2):
        for i in keep:
            assert li[b] == i
            rds, rx, rr = los.los_nodes(geo, geo.surf_x[ip], dirs[i])
            s0, s1 = off[b], off[b + 1]
            np.testing.assert_allclose(ds[s0:s1], rds, rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(nxp[s0 + b:s1 + b + 1], rx, rtol=0, atol=1e-11)
            np.testing.assert_allclose(nrp[s0 + b:s1 + b + 1], rr, rtol=0, atol=1e-11)
            b += 1


def test_node_states_match_oracle(ctx):
    p = small_problem()
    geo = p.geometry
    rays = R.fibonacci_rays(ctx, geo, 64, ctx.device)
    sp = R.DeviceSpecies(p.species, ctx.device)
    gcells = R.DeviceCells(p.cells, sp.S, ctx.device)
    nc = R.los_node_states(ctx, geo, gcells, rays, sp.S, ctx.device)
    ctx.sync()
    x = rays.t["node_x"].cpu().numpy(); r = rays.t["node_r"].cpu().numpy()
    T = nc.t["Ttr"].cpu().numpy(); Tv = nc.t["Tve"].cpu().numpy(); n = nc.t["n"].cpu().numpy()
    for k in range(0, rays.n_nodes, 7):
        a, b, c = los.idw_state(geo, p.cells, x[k], r[k])
        assert abs(T[k] - a) <= 1e-13 * a and abs(Tv[k] - b) <= 1e-13 * b
        np.testing.assert_allclose(n[k], c, rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("n_los,n_phi,n_theta", [(64, 9, 17), (200, 5, 9)])
def test_fibonacci_solve_fp64(ctx, n_los, n_phi, n_theta):
    p = small_problem()
    out = solver.solve_fibonacci(p, ctx, n_los, n_phi, n_theta, R.FP64)
    ctx.sync()
    ref = los.solve_fibonacci(p, [0, 1], n_los, n_phi, n_theta)
    I = out["I"].cpu().numpy()
    err = np.abs(I - ref["I"]) / np.maximum(np.abs(ref["I"]), 1e-300)
    m = np.abs(ref["I"]) > 0
    print(f"  I: max rel err {err[m].max():.3e}")
    assert err[m].max() <= TOL64
    S = out["S"].cpu().numpy()
    assert np.max(np.abs(S / ref["S"] - 1)) <= TOL64
    q = out["q"].cpu().numpy()
    print(f"  q gpu {q} oracle {ref['q']}")
    assert np.max(np.abs(q / ref["q"] - 1)) <= TOL64


def test_fibonacci_solve_fp32(ctx):
    p = small_problem()
    out = solver.solve_fibonacci(p, ctx, 64, 9, 17, R.FP32)
    ctx.sync()
    ref = los.solve_fibonacci(p, [0, 1], 64, 9, 17)
    I = out["I"].double().cpu().numpy()
    big = np.abs(ref["I"]) >= 1e-6 * np.abs(ref["I"]).max(axis=1, keepdims=True)
    err = (np.abs(I - ref["I"]) / np.maximum(np.abs(ref["I"]), 1e-300))[big]
    print(f"  I: max rel err {err.max():.3e} (p99 {np.quantile(err, 0.99):.3e})")
    assert err.max() <= 1e-3
    q = out["q"].cpu().numpy()
    rel = np.abs(q / ref["q"] - 1)
    print(f"  q rel err {rel}")
    assert rel.max() <= 1e-4


def test_fibonacci_chunks_sum_to_whole(ctx):
    p = small_problem()
    whole = solver.solve_fibonacci(p, ctx, 64, 9, 17, R.FP64)["q"].cpu().numpy()
    parts = solver.solve_fibonacci(p, ctx, 64, 9, 17, R.FP64, chunk=2500)["q"].cpu().numpy()
    ctx.sync()
    assert np.max(np.abs(parts / whole - 1)) <= 1e-13


def test_fibonacci_host_checks(ctx):
    p = small_problem()
    geo = p.geometry
    with pytest.raises(R.RapralError):
        R.fibonacci_rays(ctx, geo, 1, ctx.device)
    rays = R.fibonacci_rays(ctx, geo, 16, ctx.device)
    S = torch.zeros(rays.n_dirs, dtype=torch.float64, device=ctx.device)
    q = torch.zeros(rays.n_points, dtype=torch.float64, device=ctx.device)
    with pytest.raises(R.RapralError):
        R.fibonacci_flux(ctx, rays, S, 1, 9, q)
    # node-valued rays need a row per node
    kap = torch.zeros((rays.n_nodes - 1, 10), dtype=torch.float64, device=ctx.device)
    ql = torch.zeros((rays.n_points, 10), dtype=torch.float64, device=ctx.device)
    with pytest.raises(R.RapralError):
        R.trace_rays(ctx, rays, rays.n_nodes - 1, kap, kap, p.grid, 0, 10, R.FP64, ql)
    ctx.sync()
