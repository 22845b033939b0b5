"""Pins of the oracle of the paper's own angular path (Sec. 2.2.3: Fibonacci
LOS, nodes with interpolated flow variables, node march, angular
interpolation and four-point sum).  Each pin checks a property the paper or
the mathematics fixes, not a retyped formula."""
import numpy as np
import pytest

import oracle
from oracle import los
from paper_2604_11856_gb300 import synth


def small_geo(nx=12, nr=8):
    xf = np.linspace(0.0, 12.0, nx + 1)
    rf = np.linspace(2.0, 10.0, nr + 1)
    return synth.AxisymGeometry(xf=xf, rf=rf, surf_x=np.array([3.0, 6.5]), r_body=2.0,
                                mu=np.array([0.5]), wmu=np.array([1.0]), n_phi=4)


# ------------------------------------------------------------ directions ----

def test_fibonacci_set_is_nearly_uniform_on_the_sphere():
    d = los.fibonacci_directions(400)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    # sphere averages of x^2, y^2, z^2 are 1/3, of x, y, z and xy, yz, zx are 0
    for k in range(3):
        assert abs(np.mean(d[:, k] ** 2) - 1.0 / 3.0) < 4e-3
        assert abs(np.mean(d[:, k])) < 4e-3
    assert abs(np.mean(d[:, 0] * d[:, 2])) < 4e-3
    # the poles are the first and last LOS; w runs evenly from 1 to -1
    assert np.allclose(d[0], [0, 1, 0]) and np.allclose(d[-1], [0, -1, 0])
    assert np.allclose(np.diff(d[:, 1]), -2.0 / 399.0)


def test_fibonacci_neighbours_are_evenly_spaced():
    """Nearest-neighbour angular distances of a near-uniform set of n points
    cluster around sqrt(4 pi / n) (each point owns an equal area)."""
    n = 1000
    d = los.fibonacci_directions(n)
    cos = d @ d.T
    np.fill_diagonal(cos, -2.0)
    nn = np.arccos(np.clip(cos.max(axis=1), -1, 1))
    spacing = np.sqrt(4 * np.pi / n)
    assert 0.7 * spacing < np.median(nn) < 1.2 * spacing
    assert nn.min() > 0.3 * spacing


def test_fibonacci_azimuths_turn_by_the_golden_angle():
    """A Fibonacci sphere lattice turns each point by the golden angle
    2 pi / phi^2 (phi = (1 + sqrt 5) / 2) about the pole axis and steps the
    polar coordinate w uniformly from 1 to -1; the azimuth of direction i is
    atan2(dt, dx) here (Sec. 2.2.3)."""
    n = 257
    d = los.fibonacci_directions(n)
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    golden = 2.0 * np.pi / phi ** 2
    az = np.arctan2(d[:, 2], d[:, 0])
    inner = slice(1, n - 1)                     # the poles have no azimuth
    turn = np.diff(az[inner])
    off = np.minimum(np.abs((turn - golden + np.pi) % (2 * np.pi) - np.pi),
                     np.abs((turn + golden + np.pi) % (2 * np.pi) - np.pi))
    assert np.max(off) < 1e-9
    np.testing.assert_allclose(d[:, 1], np.linspace(1.0, -1.0, n), rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [64, 400, 401])
def test_valid_los_leave_the_body(n):
    keep = los.valid_los(n)
    d = los.fibonacci_directions(n)
    assert np.all(d[keep, 1] > 0)
    assert len(keep) == (n - 1) // 2 if n % 2 else n // 2


# ----------------------------------------------------------------- nodes ----

def test_los_nodes_lie_on_faces_and_end_on_the_boundary():
    geo = small_geo()
    d = los.fibonacci_directions(64)
    for i in los.valid_los(64)[::5]:
        ds, x, r = los.los_nodes(geo, 3.0, d[i])
        assert x[-1] == 3.0 and abs(r[-1] - geo.r_body) < 1e-14          # node m is O
        assert np.all(ds > 0)
        # the far node is on the domain boundary
        assert (min(abs(x[0] - geo.xf[0]), abs(x[0] - geo.xf[-1]), abs(r[0] - geo.rf[-1])) < 1e-9)
        # every interior node lies on an x face or an r face of the grid
        for xx, rr in zip(x[1:-1], r[1:-1]):
            assert (np.min(np.abs(geo.xf - xx)) < 1e-9) or (np.min(np.abs(geo.rf - rr)) < 1e-9)
        # consecutive nodes are ds apart in 3D: the projected positions give the
        # same chord when lifted back onto the straight LOS
        L = np.concatenate([np.cumsum(ds[::-1])[::-1], [0.0]])
        assert np.allclose(-np.diff(L), ds)


def test_idw_exact_at_centres_constant_fields_and_mean_at_equal_distances():
    geo = small_geo()
    nx, nr = len(geo.xf) - 1, len(geo.rf) - 1
    rng = np.random.default_rng(7)
    cells = synth.Cells(Ttr=rng.uniform(3e3, 9e3, nx * nr), Tve=rng.uniform(3e3, 9e3, nx * nr),
                        n=rng.uniform(1e14, 1e16, (nx * nr, 11)))
    xc, rc = 0.5 * (geo.xf[1:] + geo.xf[:-1]), 0.5 * (geo.rf[1:] + geo.rf[:-1])
    # at a centre: that cell
    a, b, c = los.idw_state(geo, cells, xc[4], rc[3])
    assert a == cells.Ttr[4 * nr + 3] and b == cells.Tve[4 * nr + 3] and np.array_equal(c, cells.n[4 * nr + 3])
    # equidistant from a 2 x 2 block of centres: the plain mean
    a, b, c = los.idw_state(geo, cells, 0.5 * (xc[4] + xc[5]), 0.5 * (rc[3] + rc[4]))
    ids = [4 * nr + 3, 4 * nr + 4, 5 * nr + 3, 5 * nr + 4]
    assert abs(a - np.mean(cells.Ttr[ids])) < 1e-9 * a
    assert np.allclose(c, np.mean(cells.n[ids], axis=0), rtol=1e-12)
    # anywhere: inside the range of the stencil; constant fields stay constant
    const = synth.Cells(Ttr=np.full(nx * nr, 5e3), Tve=np.full(nx * nr, 6e3), n=np.full((nx * nr, 11), 1e15))
    for x, r in rng.uniform([0, 2], [12, 10], (50, 2)):
        a, b, c = los.idw_state(geo, const, x, r)
        assert abs(a - 5e3) < 1e-9 and abs(b - 6e3) < 1e-9 and np.allclose(c, 1e15, rtol=1e-14)
        a, _, _ = los.idw_state(geo, cells, x, r)
        assert cells.Ttr.min() <= a <= cells.Ttr.max()


# ----------------------------------------------------------------- march ----

def _grid(n=5):
    return synth.Grid(500.0, 600.0, n)


def test_node_march_uniform_slab_closed_form():
    m, L = 7, 3.0
    kap = np.full((m + 1, 5), 0.8)
    em = np.full((m + 1, 5), 2.5)
    ds = np.full(m, L / m)
    I = oracle.march_nodes(np.arange(m + 1), ds, kap, em, _grid())
    assert np.allclose(I, 2.5 / 0.8 * (1 - np.exp(-0.8 * L)), rtol=1e-13)


def test_node_march_exact_for_linear_emission_at_constant_kappa():
    """With kappa constant and j linear in s along the LOS the segment scheme
    is exact: I = int_0^L j(s) e^{-kappa (L - s)} ds."""
    m, L, k = 9, 2.0, 1.3
    ds = np.random.default_rng(3).uniform(0.5, 1.5, m)
    ds *= L / ds.sum()
    s = np.concatenate([[0.0], np.cumsum(ds)])
    j0, j1 = 0.4, 3.1
    em = np.repeat((j0 + (j1 - j0) * s / L)[:, None], 3, axis=1)
    kap = np.full_like(em, k)
    I = oracle.march_nodes(np.arange(m + 1), ds, kap, em, _grid(3))
    e = np.exp(-k * L)
    exact = j1 / k - (j1 - j0) / (k * k * L) * (1 - e) - j0 * e / k
    assert np.allclose(I, exact, rtol=1e-12)


def test_node_march_equals_cell_march_with_face_averaged_nodes():
    rng = np.random.default_rng(11)
    m = 6
    cells = rng.integers(0, 5, m)
    ds = rng.uniform(0.1, 1.0, m)
    kc = rng.uniform(0.01, 2.0, (5, 4)); jc = rng.uniform(0.1, 3.0, (5, 4))
    kn = np.zeros((m + 1, 4)); jn = np.zeros((m + 1, 4))
    kn[0], jn[0] = kc[cells[0]], jc[cells[0]]
    kn[m], jn[m] = kc[cells[-1]], jc[cells[-1]]
    for i in range(1, m):
        kn[i] = 0.5 * (kc[cells[i - 1]] + kc[cells[i]])
        jn[i] = 0.5 * (jc[cells[i - 1]] + jc[cells[i]])
    a = oracle.march(cells, ds, 1.0, kc, jc, _grid(4))
    b = oracle.march_nodes(np.arange(m + 1), ds, kn, jn, _grid(4))
    assert np.allclose(a, b, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- angular ----

@pytest.mark.parametrize("n_phi,n_theta", [(2, 3), (9, 17), (16, 33)])
def test_isotropic_S_gives_pi_S(n_phi, n_theta):
    d = los.fibonacci_directions(200)[los.valid_los(200)]
    q = los.angular_flux(d, np.full(len(d), 2.7), n_phi, n_theta)
    assert abs(q - np.pi * 2.7) < 1e-12


def test_S_equal_cos_phi_converges_to_two_pi_over_three():
    errs = []
    for n_los, n_phi, n_theta in [(100, 9, 17), (400, 17, 33), (1600, 33, 65)]:
        d = los.fibonacci_directions(n_los)[los.valid_los(n_los)]
        q = los.angular_flux(d, d[:, 1], n_phi, n_theta)
        errs.append(abs(q - 2.0 * np.pi / 3.0))
    assert errs[-1] < 5e-3 and errs[2] < errs[1] < errs[0]


def test_azimuthally_odd_S_integrates_to_zero():
    d = los.fibonacci_directions(800)[los.valid_los(800)]
    q = los.angular_flux(d, d[:, 0], 17, 33)     # S = sin(phi) cos(theta)
    assert abs(q) < 1e-2


# ----------------------------------------------------------------- whole ----

def test_uniform_field_gives_slab_intensity_per_los():
    """All cells alike: every node has the cell's state, so each LOS gives
    (j / kappa)(1 - e^{-kappa L}) with L its length inside the domain."""
    base = synth.stagnation_line(n_cells=2, n_atomic=200, n_molecular=500, n_grid=401)
    geo = small_geo(6, 4)
    C = 6 * 4
    c0 = 1
    cells = synth.Cells(Ttr=np.full(C, base.cells.Ttr[c0]), Tve=np.full(C, base.cells.Tve[c0]),
                        n=np.repeat(base.cells.n[c0:c0 + 1], C, axis=0))
    p = synth.Problem("uniform", base.species, base.lines, cells, base.grid, geo, chunk=0)
    out = los.solve_fibonacci(p, [0], 32, 5, 9)
    one = synth.Problem("one", base.species, base.lines, synth.Cells(Ttr=cells.Ttr[:1], Tve=cells.Tve[:1],
                                                                      n=cells.n[:1]), base.grid, geo, chunk=0)
    k1, j1 = oracle.spectral_coeffs(one)
    k1, j1 = k1[0], j1[0]
    for b, (_p, _i, nodes, ds) in enumerate(out["los"]):
        L = ds.sum()
        ref = np.where(k1 > 0, j1 / np.where(k1 > 0, k1, 1) * -np.expm1(-k1 * L), j1 * L)
        assert np.allclose(out["I"][b], ref, rtol=1e-9, atol=1e-300)
