"""The single-direction march over a ragged, caller-built ray set, against the
oracle's march of every bundle (Sec. 2.2.3: face-averaged nodes, kappa at the
far node, j linear, angular sum with the directions' weights).

Besides full bundle lists the set holds what the march kernels must also get
right:
- bundles of 0, 1 and 2 segments;
- bundles with no direction (skipped);
- a point with no bundles (q_lambda zero);
- points with an odd number of bundles and one with more than eight (its bundles
  split over block groups);
- far ends at a hot wall and in cold space;
- per-direction scales and weights that differ.

Both sides march the oracle's kappa / j tables (FP64; the FP32 path gets them
rounded to FP32). FP64: q_lambda and every intensity within 1e-10 of the
oracle. FP32: q_lambda within 1e-3 per column where it is above 1e-6 of the
point's maximum, over an aligned, even range and over an odd, unaligned one.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_11856_gb300 import rapral as R
from paper_2604_11856_gb300 import synth

pytestmark = pytest.mark.gpu

TOL64, TOL32, MASK = 1e-10, 1e-3, 1e-6
T_WALL = 4000.0
BUNDLES_PER_POINT = [3, 0, 9, 1, 40]


def ragged_rays(n_cells, seed=11):
    """Host arrays of a ray set: segment counts include 0, 1 and 2, every
    seventh bundle has no direction, walls on about half of the bundles."""
    rng = np.random.default_rng(seed)
    seg_off, seg_cell, seg_ds = [0], [], []
    dir_off, scale, weight, wall = [0], [], [], []
    special = [0, 1, 2]
    b = 0
    for nb in BUNDLES_PER_POINT:
        for _ in range(nb):
            m = special[b] if b < len(special) else int(rng.integers(3, 300))
            seg_cell.extend(rng.integers(0, n_cells, m).tolist())
            seg_ds.extend(rng.uniform(0.01, 0.5, m).tolist())
            seg_off.append(seg_off[-1] + m)
            has_dir = b % 7 != 6
            if has_dir:
                scale.append(float(rng.uniform(1.0, 3.0)))
                weight.append(float(rng.uniform(0.1, 1.0)))
            dir_off.append(dir_off[-1] + int(has_dir))
            wall.append(int(rng.integers(0, 2)))
            b += 1
    point_off = np.concatenate([[0], np.cumsum(BUNDLES_PER_POINT)])
    return dict(point_off=point_off, seg_off=np.asarray(seg_off), seg_cell=np.asarray(seg_cell, np.int64),
                seg_ds=np.asarray(seg_ds), dir_off=np.asarray(dir_off), dir_scale=np.asarray(scale),
                dir_weight=np.asarray(weight), bundle_wall=np.asarray(wall))


def oracle_march(h, kap, em, grid, k0):
    """Intensity of every direction and q_lambda of every point, by the
    oracle's march of each bundle."""
    nk = kap.shape[1]
    P = len(h["point_off"]) - 1
    I = np.zeros((len(h["dir_scale"]), nk))
    ql = np.zeros((P, nk))
    for p in range(P):
        for b in range(h["point_off"][p], h["point_off"][p + 1]):
            d0, d1 = h["dir_off"][b], h["dir_off"][b + 1]
            if d1 == d0:
                continue
            s0, s1 = h["seg_off"][b], h["seg_off"][b + 1]
            I[d0] = oracle.march(h["seg_cell"][s0:s1], h["seg_ds"][s0:s1], h["dir_scale"][d0], kap, em, grid, k0,
                                 wall_start=bool(h["bundle_wall"][b]), T_wall=T_WALL)
            ql[p] += h["dir_weight"][d0] * I[d0]
    return I, ql


@pytest.fixture(scope="module")
def case():
    p = synth.stagnation_line(n_cells=30, n_atomic=500, n_molecular=5000, n_grid=4001)
    kap, em = oracle.spectral_coeffs(p)
    h = ragged_rays(len(p.cells))
    return p, kap, em, h


@pytest.mark.parametrize("precision", [R.FP64, R.FP32])
@pytest.mark.parametrize("rng_cols", [(0, 4000), (33, 1001)])
def test_ragged_single_direction_march(case, precision, rng_cols):
    p, kap, em, h = case
    k0, nk = rng_cols
    kr, er = kap[:, k0:k0 + nk], em[:, k0:k0 + nk]
    I_ref, ql_ref = oracle_march(h, kr, er, p.grid, k0)
    dev = torch.device("cuda", 0)
    ctx = R.Context(0)
    rays = R.rays_from_arrays(h["point_off"], h["seg_off"], h["seg_cell"], h["seg_ds"], h["dir_off"], h["dir_scale"],
                              h["dir_weight"], h["bundle_wall"], T_WALL, dev)
    dt = torch.float64 if precision == R.FP64 else torch.float32
    dk = torch.as_tensor(np.ascontiguousarray(kr), dtype=dt, device=dev)
    de = torch.as_tensor(np.ascontiguousarray(er), dtype=dt, device=dev)
    P = len(BUNDLES_PER_POINT)
    ql = torch.full((P, nk), float("nan"), dtype=dt, device=dev)
    I = torch.full((len(h["dir_scale"]), nk), float("nan"), dtype=dt, device=dev)
    R.trace_rays(ctx, rays, len(p.cells), dk, de, p.grid, k0, nk, precision, ql, I)
    ctx.sync()
    g_ql = ql.double().cpu().numpy()
    g_I = I.double().cpu().numpy()
    assert np.all(g_ql[1] == 0.0)                      # the point without bundles
    if precision == R.FP64:
        assert np.all(np.abs(g_I - I_ref) <= TOL64 * np.abs(I_ref) + 1e-300)
        assert np.all(np.abs(g_ql - ql_ref) <= TOL64 * np.abs(ql_ref) + 1e-300)
    else:
        worst = 0.0
        for pt in range(P):
            ref = ql_ref[pt]
            if not np.any(ref > 0):
                continue
            m = ref >= MASK * ref.max()
            err = np.abs(g_ql[pt] - ref)[m] / ref[m]
            worst = max(worst, float(err.max()))
        print(f"  q_lambda: max rel err {worst:.3e}")
        assert worst <= TOL32
