"""QSS collisional-radiative populations on the GPU (rapral_qss_populations)
against the oracle of oracle/qss.py: FP64 within 1e-10 relative per level.
The rate matrices are well conditioned componentwise (a relative 1e-15
change of every entry moves the solution by < 2e-14), so a different
pivoted elimination order stays far inside that bar."""
import numpy as np
import pytest
import torch

from oracle import qss
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return R.Context(0)


def _gpu(ctx, model, cells):
    dm = R.DeviceCrModel(model, ctx.device)
    dc = R.DeviceCells(cells, 8, ctx.device)
    out = torch.empty((len(cells.Ttr), dm.l), dtype=torch.float64, device=ctx.device)
    R.qss_populations(ctx, dm, dc, out)
    ctx.sync()
    return out.cpu().numpy()


@pytest.mark.parametrize("species,lumped", [("N", 0), ("N", 4), ("O", 3)])
def test_qss_matches_oracle(ctx, species, lumped):
    m = synth.cr_model(species=species, n_levels=20, n_lumped=lumped, seed=1005 + lumped)
    p = synth.stagnation_line(n_cells=60, n_atomic=10, n_molecular=10, n_grid=11)
    got = _gpu(ctx, m, p.cells)
    ref = qss.solve_cells(m, p.cells, ion_col=m["ion_col"])
    err = np.max(np.abs(got - ref) / np.abs(ref))
    print(f"  {species}: max rel err {err:.3e}")
    assert err <= 1e-10


def test_qss_afterbody_cells_sampled(ctx):
    m = synth.cr_model(species="O", n_levels=32, seed=1009)
    p = synth.afterbody(nx=100, nr=50, n_points=2, n_grid=11)
    got = _gpu(ctx, m, p.cells)
    idx = np.random.default_rng(5).integers(0, len(p.cells.Ttr), 40)
    sub = synth.Cells(Ttr=p.cells.Ttr[idx], Tve=p.cells.Tve[idx], n=p.cells.n[idx])
    ref = qss.solve_cells(m, sub, ion_col=m["ion_col"])
    err = np.max(np.abs(got[idx] - ref) / np.abs(ref))
    print(f"  32 levels: max rel err {err:.3e}")
    assert err <= 1e-10


def test_qss_boltzmann_limit_on_gpu(ctx):
    m = synth.cr_model(species="N", n_levels=16, n_lumped=2)
    m["A"][:] = 0.0
    m["ii_C"][:] = 0.0
    p = synth.stagnation_line(n_cells=8, n_atomic=10, n_molecular=10, n_grid=11)
    cells = synth.Cells(Ttr=p.cells.Tve.copy(), Tve=p.cells.Tve.copy(), n=p.cells.n)
    got = _gpu(ctx, m, cells)
    for c in range(8):
        Q = qss.level_Q(m, cells.Tve[c])
        np.testing.assert_allclose(got[c], cells.n[c, m["col"]] * Q[:16] / Q.sum(), rtol=1e-10)


def test_qss_checks(ctx):
    p = synth.stagnation_line(n_cells=3, n_atomic=10, n_molecular=10, n_grid=11)
    m = synth.cr_model(n_levels=6)
    bad = dict(m)
    bad["up"] = m["up"].copy()
    bad["up"][3] = 6                                  # a level past n_levels: caught on the device
    with pytest.raises(R.RapralError):
        _gpu(ctx, bad, p.cells)
    ctx.clear_status()
    big = synth.cr_model(n_levels=33)
    with pytest.raises(R.RapralError):
        _gpu(ctx, big, p.cells)
    ctx.sync()
