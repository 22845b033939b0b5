"""CPU oracle of the paper's own angular path (Sec. 2.2.3) -- test
infrastructure only, like the rest of this package.

Steps, in the paper's order, for a surface point O of an axisymmetric body:

1. Fibonacci-sphere LOS directions (Sec. 2.2.3, the Fibonacci sphere and its
   w, r, a formulas), in the frame x along the axis, y the outward normal at
   O, z completing it; only directions leaving the body (w > 0) are kept.
2. LOS nodes where the LOS, projected onto the (x, r) plane, crosses the
   grid's cell faces, plus its two ends (the far boundary and O).
3. Flow variables at a node by inverse-distance weighting (power 2) over the
   2 x 2 block of cell centres around the node's projected position.
4. kappa and j at the nodes (the line-by-line sum of the main oracle applied
   to the node states), the Johnston-Mazaheri march node to node, and the
   wavelength integral S of the intensity at O, per LOS.
5. S on a uniform (polar phi, azimuth theta) grid by inverse-distance
   weighting over the four nearest LOS directions, then the four-point
   average sum with the weight (cos^2 phi_p - cos^2 phi_{p+1}) / 2 times the
   azimuth step (the integral of sin phi cos phi over the cell).

Pinned in tests/test_oracle_los_pins.py: the Fibonacci formulas and their
symmetry, the node geometry against the segment walk, the interpolations'
exactness for constants and sample points, the node march against the slab
closed form and linear emission, the angular sum's exact value pi S for
isotropic S and its convergence for S = cos phi.
"""
from __future__ import annotations

import numpy as np

from . import axisym_segments, march_nodes, spectral_coeffs, spectral_integral, lnpref


def fibonacci_directions(n_los):
    """Unit directions (dx, dn, dt) of LOS i = 1..n_los (Sec. 2.2.3):
    w = 1 - 2 (i - 1) / (n_los - 1), r = sqrt(1 - w^2),
    a = (i - 1)(sqrt 5 - 1) pi, direction (r cos a, w, r sin a)."""
    i = np.arange(1, n_los + 1, dtype=np.float64)
    w = 1.0 - 2.0 * (i - 1.0) / (n_los - 1.0)
    r = np.sqrt(np.maximum(0.0, 1.0 - w * w))
    a = (i - 1.0) * (np.sqrt(5.0) - 1.0) * np.pi
    return np.stack([r * np.cos(a), w, r * np.sin(a)], axis=1)


def valid_los(n_los):
    """Indices (0-based) of the LOS that leave the body: w > 0."""
    d = fibonacci_directions(n_los)
    return np.nonzero(d[:, 1] > 0.0)[0]


def los_nodes(geo, x0, d):
    """Nodes of one LOS from the far boundary to O: segment lengths ds [m]
    (far first) and node positions (x, r) [m + 1] projected onto the
    axisymmetric plane, node m being O itself."""
    _cells, ds = axisym_segments(geo, x0, d)
    m = ds.shape[0]
    L = np.zeros(m + 1)                       # distance of node j from O
    for j in range(m - 1, -1, -1):
        L[j] = L[j + 1] + ds[j]
    dx, dn, dt = d
    x = x0 + dx * L
    r = np.sqrt((geo.r_body + dn * L) ** 2 + (dt * L) ** 2)
    return ds, x, r


def idw_state(geo, cells, x, r):
    """Flow variables at (x, r): inverse-distance weights 1/d^2 over the
    2 x 2 block of cell centres around the point (clamped to the grid); a
    point on a centre takes that cell's values.  Returns (Ttr, Tve, n[S])."""
    xf, rf = np.asarray(geo.xf), np.asarray(geo.rf)
    xc, rc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (rf[1:] + rf[:-1])
    nx, nr = xc.shape[0], rc.shape[0]
    i0 = int(np.clip(np.searchsorted(xc, x, side="right") - 1, 0, max(0, nx - 2)))
    j0 = int(np.clip(np.searchsorted(rc, r, side="right") - 1, 0, max(0, nr - 2)))
    idx, wts = [], []
    for i in range(i0, min(i0 + 2, nx)):
        for j in range(j0, min(j0 + 2, nr)):
            d2 = (x - xc[i]) ** 2 + (r - rc[j]) ** 2
            c = i * nr + j                     # cells are (x, r) row-major, r fastest
            if d2 == 0.0:
                return cells.Ttr[c], cells.Tve[c], np.array(cells.n[c], dtype=np.float64)
            idx.append(c)
            wts.append(1.0 / d2)
    w = np.asarray(wts) / np.sum(wts)
    idx = np.asarray(idx)
    return (float(np.dot(w, cells.Ttr[idx])), float(np.dot(w, cells.Tve[idx])),
            np.asarray(w @ np.asarray(cells.n)[idx], dtype=np.float64))


def node_problem(problem, points, n_los):
    """The LOS of the given surface points with their nodes: returns
    (node_problem, los) where node_problem has one 'cell' per node and los is
    a list of (point, los_index, node_ids far -> near, ds)."""
    from paper_2604_11856_gb300 import synth   # dataclasses only
    geo = problem.geometry
    dirs = fibonacci_directions(n_los)
    keep = valid_los(n_los)
    Ttr, Tve, n, los = [], [], [], []
    for p in points:
        x0 = geo.surf_x[p]
        for i in keep:
            ds, x, r = los_nodes(geo, x0, dirs[i])
            first = len(Ttr)
            for xx, rr in zip(x, r):
                a, b, c = idw_state(geo, problem.cells, xx, rr)
                Ttr.append(a); Tve.append(b); n.append(c)
            los.append((p, int(i), np.arange(first, len(Ttr), dtype=np.int64), ds))
    cells = synth.Cells(Ttr=np.asarray(Ttr), Tve=np.asarray(Tve), n=np.asarray(n))
    return synth.Problem(problem.name + " LOS nodes", problem.species, problem.lines, cells, problem.grid,
                         geo, chunk=0), los


def angular_flux(dirs, S, n_phi, n_theta, k_nn=4):
    """Flux at a point from LOS results S at unit directions dirs [n, 3]
    (frame x, normal, z): S on the grid phi_p = (pi/2) p / (n_phi - 1),
    theta_t = 2 pi t / (n_theta - 1) by inverse-distance weighting (chord
    distance squared) over the k_nn nearest directions, then the four-point
    average sum with weight (cos^2 phi_p - cos^2 phi_{p+1}) / 2 (theta_{t+1} - theta_t)."""
    dirs = np.asarray(dirs, np.float64)
    S = np.asarray(S, np.float64)
    phi = 0.5 * np.pi * np.arange(n_phi) / (n_phi - 1)
    theta = 2.0 * np.pi * np.arange(n_theta) / (n_theta - 1)
    G = np.zeros((n_phi, n_theta))
    for p in range(n_phi):
        for t in range(n_theta):
            g = np.array([np.sin(phi[p]) * np.cos(theta[t]), np.cos(phi[p]), np.sin(phi[p]) * np.sin(theta[t])])
            d2 = np.sum((dirs - g) ** 2, axis=1)
            near = np.argsort(d2, kind="stable")[:k_nn]
            if d2[near[0]] == 0.0:
                G[p, t] = S[near[0]]
                continue
            w = 1.0 / d2[near]
            G[p, t] = np.dot(w, S[near]) / np.sum(w)
    q = 0.0
    for t in range(n_theta - 1):
        for p in range(n_phi - 1):
            avg = 0.25 * (G[p, t] + G[p + 1, t] + G[p, t + 1] + G[p + 1, t + 1])
            q += avg * 0.5 * (np.cos(phi[p]) ** 2 - np.cos(phi[p + 1]) ** 2) * (theta[t + 1] - theta[t])
    return q


def solve_fibonacci(problem, points, n_los, n_phi, n_theta, k0=0, nk=None):
    """The whole angular path for the given surface points over grid points
    [k0, k0 + nk): per-LOS intensity I [n_valid_los_total, nk] at O, per-LOS
    S (this range's part of the wavelength integral, whole-grid trapezoid
    weights) and the flux q [points]."""
    nk = problem.grid.n - k0 if nk is None else nk
    npb, los = node_problem(problem, points, n_los)
    kap, em = spectral_coeffs(npb, lnpref(npb), k0, nk)
    dirs = fibonacci_directions(n_los)
    I = np.zeros((len(los), nk))
    S = np.zeros(len(los))
    for b, (_p, _i, nodes, ds) in enumerate(los):
        I[b] = march_nodes(nodes, ds, kap, em, problem.grid, k0)
        S[b] = spectral_integral(I[b], problem.grid, k0)
    q = np.zeros(len(points))
    for ip, p in enumerate(points):
        sel = [b for b, l in enumerate(los) if l[0] == p]
        q[ip] = angular_flux(dirs[[los[b][1] for b in sel]], S[sel], n_phi, n_theta)
    return dict(I=I, S=S, q=q, los=los, node_problem=npb, kappa=kap, emis=em)
