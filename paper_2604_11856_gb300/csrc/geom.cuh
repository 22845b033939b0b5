// Ray geometry on the rectilinear (x, r) grid of an axisymmetric body,
// shared by the ray builders.
#pragma once

#include <cstdint>

// Ray from the surface point (x0, rb): position x = x0 + t dx, radius
// sqrt((rb + t dn)^2 + (t dt)^2) (non-decreasing for dn > 0).  Walks the
// rectilinear (x, r) cells from the point outward, stepping to whichever face
// (x or r) comes first; emits (cell, length) for every piece of positive
// length.  With out_cell != nullptr the pieces are written backwards from
// out_end - 1 (so the list runs from the far boundary to the point).
__device__ inline int64_t walk_ray(const double* xf, int nx, const double* rf, int nr, double x0, double rb, double dx,
                            double dn, double dt, int32_t* out_cell, double* out_ds, int64_t out_end) {
    if (!(x0 >= xf[0] && x0 <= xf[nx])) return 0;
    int lo = 0, hi = nx;   // largest ix with xf[ix] <= x0
    while (hi - lo > 1) { int m = (lo + hi) >> 1; if (xf[m] <= x0) lo = m; else hi = m; }
    int ix = lo;
    if (x0 == xf[ix] && dx < 0.0) ix -= 1;
    if (ix >= nx) ix = nx - 1;
    int jr = 0;
    const double A = dn * dn + dt * dt, B = 2.0 * rb * dn;
    double t = 0.0;
    int64_t n = 0;
    const int guard = 2 * (nx + nr) + 8;
    for (int it = 0; it < guard && ix >= 0 && ix < nx && jr < nr; ++it) {
        double tx = INFINITY;
        if (dx > 0.0) tx = (xf[ix + 1] - x0) / dx;
        else if (dx < 0.0) tx = (xf[ix] - x0) / dx;
        double tr = INFINITY;
        if (A > 0.0) {
            const double rr = rf[jr + 1];
            const double cq = rb * rb - rr * rr;                 // <= 0
            tr = (-2.0 * cq) / (B + sqrt(B * B - 4.0 * A * cq));  // cancellation-free root
        }
        const double tn = fmin(tx, tr);
        const double len = tn - t;
        if (len > 0.0) {
            if (out_cell) { out_cell[out_end - 1 - n] = ix * nr + jr; out_ds[out_end - 1 - n] = len; }
            ++n;
            t = tn;
        }
        if (tx <= tr) ix += (dx > 0.0) ? 1 : -1;
        if (tr <= tx) jr += 1;
    }
    return n;
}

