"""The atomic continuum of Sec. 2.2.1 on the GPU (rapral_continuum_coeffs:
bound-free with Kirchhoff / Saha-Boltzmann emission, free-free from the
Table 3 fit with D) against the oracle of oracle/continuum.py: FP64 to
1e-10 relative per point, FP32 to 1e-3 on values >= 1e-6 of the row's
maximum; added on top of the line sum; ragged ranges, cold cells, checks."""
import numpy as np
import pytest
import torch

import oracle
from oracle import continuum as ct
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import solver, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return R.Context(0)


def _models(n_levels=100):
    return [synth.continuum_model(species="N", n_levels=n_levels, seed=1007),
            synth.continuum_model(species="O", n_levels=n_levels, seed=1008)]


def _problem(n_cells=24, n_grid=60001, cold=False):
    p = synth.stagnation_line(n_cells=n_cells, n_atomic=2000, n_molecular=5000, n_grid=n_grid)
    if cold:   # frozen ions in cold gas: the Saha factor and the Planck function over- / underflow alone
        p.cells.Tve[:4] = [300.0, 800.0, 1500.0, 3000.0]
        p.cells.Ttr[:4] = p.cells.Tve[:4]
    return p


def _gpu(ctx, p, models, precision, k0=0, nk=None, lines=False):
    nk = p.grid.n - k0 if nk is None else nk
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    dt = torch.float64 if precision == R.FP64 else torch.float32
    kap = torch.zeros((dp.C, nk), dtype=dt, device=ctx.device)
    em = torch.zeros_like(kap)
    if lines:
        R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, k0, nk, precision, kap, em)
    dc = R.DeviceContinuum(models, ctx.device)
    R.continuum_coeffs(ctx, dc, dp.species.S, dp.cells, p.grid, k0, nk, precision, kap, em)
    ctx.sync()
    return kap.double().cpu().numpy(), em.double().cpu().numpy()


def _rel(got, ref):
    return np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300))


@pytest.mark.parametrize("k0,nk", [(0, None), (12345, 20011)])
def test_continuum_fp64_matches_oracle(ctx, k0, nk):
    p = _problem()
    ms = _models()
    kap, em = _gpu(ctx, p, ms, R.FP64, k0, nk)
    rk, re = ct.continuum(ms, p.cells, oracle.lnpref(p), p.grid, k0, nk)
    ek, ej = _rel(kap, rk), _rel(em, re)
    print(f"  kappa {ek:.3e}  j {ej:.3e}")
    assert ek <= 1e-10 and ej <= 1e-10


def test_continuum_fp32_within_tolerance(ctx):
    p = _problem()
    ms = _models()
    kap, em = _gpu(ctx, p, ms, R.FP32)
    rk, re = ct.continuum(ms, p.cells, oracle.lnpref(p), p.grid)
    for name, g, r in (("kappa", kap, rk), ("j", em, re)):
        big = r >= 1e-6 * r.max(axis=1, keepdims=True)
        err = (np.abs(g - r) / np.maximum(r, 1e-300))[big]
        print(f"  {name}: max rel err {err.max():.3e} (p99 {np.quantile(err, 0.99):.3e})")
        assert err.max() <= 1e-3


@pytest.mark.parametrize("precision", [R.FP64, R.FP32])
def test_continuum_in_cold_cells(ctx, precision):
    p = _problem(n_cells=8, n_grid=20001, cold=True)
    ms = _models(40)
    kap, em = _gpu(ctx, p, ms, precision)
    rk, re = ct.continuum(ms, p.cells, oracle.lnpref(p), p.grid)
    assert np.all(np.isfinite(kap)) and np.all(np.isfinite(em))
    if precision == R.FP64:
        assert _rel(kap, rk) <= 1e-10 and _rel(em, re) <= 1e-10
    else:
        big = re >= 1e-6 * re.max(axis=1, keepdims=True)
        assert np.max((np.abs(em - re) / np.maximum(re, 1e-300))[big]) <= 1e-3


def test_continuum_adds_to_the_line_sum(ctx):
    p = _problem(n_cells=6, n_grid=30001)
    ms = _models(60)
    kap, em = _gpu(ctx, p, ms, R.FP64, lines=True)
    lk, lj = oracle.spectral_coeffs(p)
    ck, cj = ct.continuum(ms, p.cells, oracle.lnpref(p), p.grid)
    assert _rel(kap, lk + ck) <= 1e-10 and _rel(em, lj + cj) <= 1e-10


def test_continuum_checks(ctx):
    p = _problem(n_cells=3, n_grid=4001)
    m = synth.continuum_model(species="N", n_levels=10)
    bad = dict(m, node_off=m["node_off"].copy())
    bad["node_off"][5] = bad["node_off"][4] + 1          # a level with one node: caught on the device
    with pytest.raises(R.RapralError):
        _gpu(ctx, p, [bad], R.FP64)
    ctx.clear_status()
    bad = dict(m, node_lam=m["node_lam"].copy())
    bad["node_lam"][[30, 31]] = bad["node_lam"][[31, 30]]  # not increasing
    with pytest.raises(R.RapralError):
        _gpu(ctx, p, [bad], R.FP64)
    ctx.clear_status()
    bad = dict(m, ion_col=99)                              # host-side check
    with pytest.raises(R.RapralError):
        _gpu(ctx, p, [bad], R.FP64)
    ctx.sync()


@pytest.mark.parametrize("precision", [R.FP64, R.FP32])
def test_saha_boltzmann_populations(ctx, precision):
    """rapral_saha_populations replaces the N and O prefactors; the line sum
    and the continuum then follow the oracle fed the same prefactors."""
    p = _problem(n_cells=12, n_grid=30001)
    p.cells.n[0, synth.FLOW_SPECIES.index("N+")] = 0.0          # no ions: no N population in cell 0
    ms = _models(40)
    dp = solver.DeviceProblem(p, ctx)
    R.populations(ctx, dp.species, dp.cells)
    lnp = oracle.lnpref(p)
    for m in ms:
        ie = torch.tensor(m["ion_E"], dtype=torch.float64, device=ctx.device)
        ig = torch.tensor(m["ion_g"], dtype=torch.float64, device=ctx.device)
        R.saha_populations(ctx, dp.cells, m["species"], dp.species.S, m["E_ion"], m["ion_col"], ie, ig)
        lnp[:, m["species"]] = ct.saha_lnpref(p.cells, m["ion_col"], m["E_ion"], m["ion_E"], m["ion_g"])
    got = dp.cells.lnpref.cpu().numpy()
    fin = np.isfinite(lnp)
    assert np.array_equal(np.isfinite(got), fin)
    assert np.max(np.abs(got[fin] - lnp[fin])) <= 1e-12 * np.max(np.abs(lnp[fin]))
    dt = torch.float64 if precision == R.FP64 else torch.float32
    kap = torch.zeros((dp.C, p.grid.n), dtype=dt, device=ctx.device)
    em = torch.zeros_like(kap)
    R.spectral_coeffs(ctx, dp.species, dp.lines, dp.cells, p.grid, 0, p.grid.n, precision, kap, em)
    R.continuum_coeffs(ctx, R.DeviceContinuum(ms, ctx.device), dp.species.S, dp.cells, p.grid, 0, p.grid.n,
                       precision, kap, em)
    ctx.sync()
    lk, lj = oracle.spectral_coeffs(p, lnp=lnp)
    ck, cj = ct.continuum(ms, p.cells, lnp, p.grid)
    rk, rj = lk + ck, lj + cj
    k, j = kap.double().cpu().numpy(), em.double().cpu().numpy()
    if precision == R.FP64:
        assert _rel(k, rk) <= 1e-10 and _rel(j, rj) <= 1e-10
    else:
        big = rj >= 1e-6 * rj.max(axis=1, keepdims=True)
        assert np.max((np.abs(j - rj) / np.maximum(rj, 1e-300))[big]) <= 1e-3


def test_continuum_edge_cases(ctx):
    """One grid point; a range below every edge; a table wholly outside the
    range; no cells."""
    p = _problem(n_cells=5, n_grid=20001)
    ms = _models(30)
    lnp = oracle.lnpref(p)
    for k0, nk in ((0, 1), (20000, 1), (7777, 129), (19900, 101)):
        kap, em = _gpu(ctx, p, ms, R.FP64, k0, nk)
        rk, re = ct.continuum(ms, p.cells, lnp, p.grid, k0, nk)
        assert _rel(kap, rk) <= 1e-10 and _rel(em, re) <= 1e-10, (k0, nk)
    far = dict(ms[0], node_lam=ms[0]["node_lam"] * 1e-3)        # tables at 0.01 .. 10 nm: no bound-free
    kap, em = _gpu(ctx, p, [far], R.FP32)
    rk, re = ct.continuum([far], p.cells, lnp, p.grid)
    big = re >= 1e-6 * re.max(axis=1, keepdims=True)
    assert np.max((np.abs(em - re) / np.maximum(re, 1e-300))[big]) <= 1e-3
    dp = solver.DeviceProblem(p, ctx)
    empty = R.Cells()
    empty.n_cells, empty.n_cols, empty.ne_col = 0, dp.cells.struct.n_cols, dp.cells.struct.ne_col
    kap = torch.zeros((1, 8), dtype=torch.float64, device=ctx.device)
    dc = R.DeviceContinuum(ms, ctx.device)
    g = R.grid_struct(p.grid)
    ctx.check(ctx.lib.rapral_continuum_coeffs(ctx.h, R.ct.byref(dc.structs), dc.n, dp.species.S, R.ct.byref(empty),
                                              R.ct.byref(g), 0, 8, R.FP64, R._ptr(kap), R._ptr(kap), 8))
    ctx.sync()
    assert float(kap.abs().sum()) == 0.0


@pytest.mark.parametrize("precision,chunk", [(R.FP64, None), (R.FP64, 7001), (R.FP32, None)])
def test_solve_with_continuum(ctx, precision, chunk):
    """The whole slab solve with the continuum added to every chunk's
    coefficients: q against the oracle's march of lines + continuum."""
    p = _problem(n_cells=10, n_grid=20001)
    ms = _models(40)
    dp = solver.DeviceProblem(p, ctx)
    out = solver.solve(dp, ctx, precision, chunk=chunk, continuum=R.DeviceContinuum(ms, ctx.device))
    ctx.sync()
    q = float(out["q"].cpu().numpy()[0])
    lk, lj = oracle.spectral_coeffs(p)
    ck, cj = ct.continuum(ms, p.cells, oracle.lnpref(p), p.grid)
    ref = oracle.solve_slab(p, coeffs=(lk + ck, lj + cj))["q"]
    ref_lines = oracle.solve_slab(p, coeffs=(lk, lj))["q"]
    print(f"  q {q:.6e} oracle {ref:.6e} (lines only {ref_lines:.6e})")
    assert abs(q / ref - 1) <= (1e-10 if precision == R.FP64 else 1e-4)
    assert abs(ref / ref_lines - 1) > 1e-6      # the continuum does change q
