// The paper's own angular path (Sec. 2.2.3): Fibonacci-sphere lines of
// sight from the surface points, their nodes on the (x, r) grid's faces,
// flow variables at the nodes by inverse-distance weighting, and the flux
// from per-line results carried to a uniform (phi, theta) grid and summed
// with the four-point average.  The march of node-valued lines is k_march
// in k_rays.cu (node_values = 1).
#include <algorithm>

#include "geom.cuh"
#include "rapral_internal.cuh"

namespace {

// Direction of LOS i (0-based; the paper's i_LOS - 1) of n_los:
// w = 1 - 2 i/(n_los - 1), r = sqrt(1 - w^2), a = i (sqrt 5 - 1) pi,
// (dx, dn, dt) = (r cos a, w, r sin a) with dn along the outward normal.
__device__ __forceinline__ void fib_dir(int i, int n_los, double* dx, double* dn, double* dt) {
    const double w = 1.0 - 2.0 * (double)i / (double)(n_los - 1);
    const double r = sqrt(fmax(0.0, 1.0 - w * w));
    const double a = (double)i * (sqrt(5.0) - 1.0) * M_PI;
    *dx = r * cos(a);
    *dn = w;
    *dt = r * sin(a);
}

__global__ void k_fib_count(const double* xf, int32_t nx, const double* rf, int32_t nr, const double* surf_x,
                            int32_t P, int32_t n_los, int32_t V, int64_t* counts) {
    const int64_t B = (int64_t)P * V;
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int64_t p = b / V;
    double dx, dn, dt;
    fib_dir((int)(b - p * V), n_los, &dx, &dn, &dt);
    counts[b] = walk_ray(xf, nx, rf, nr, surf_x[p], rf[0], dx, dn, dt, nullptr, nullptr, 0);
}

// Segments (far first), then the nodes: node s1 + b is the surface point,
// node s + b the far end of segment s; its distance L from the point sums the
// lengths from the near end, and its (x, r) is the projection
// (x0 + dx L, sqrt((r_b + dn L)^2 + (dt L)^2)), rounded step by step.
__global__ void k_fib_fill(const double* xf, int32_t nx, const double* rf, int32_t nr, const double* surf_x,
                           int32_t P, int32_t n_los, int32_t V, const int64_t* seg_off, int32_t* seg_cell,
                           double* seg_ds, int64_t* point_off, int64_t* dir_off, double* dir_scale,
                           double* dir_weight, int32_t* bundle_wall, int32_t* los_index, double* node_x,
                           double* node_r) {
    const int64_t B = (int64_t)P * V;
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b > B) return;
    dir_off[b] = b;
    if (b <= P) point_off[b] = b * (int64_t)V;
    if (b == B) return;
    const int64_t p = b / V;
    const int i = (int)(b - p * V);
    double dx, dn, dt;
    fib_dir(i, n_los, &dx, &dn, &dt);
    const double x0 = surf_x[p], rb = rf[0];
    const int64_t s0 = seg_off[b], s1 = seg_off[b + 1];
    walk_ray(xf, nx, rf, nr, x0, rb, dx, dn, dt, seg_cell, seg_ds, s1);
    dir_scale[b] = 1.0;
    dir_weight[b] = 1.0;
    bundle_wall[b] = 0;
    los_index[b] = i;
    double L = 0.0;
    node_x[s1 + b] = x0;
    node_r[s1 + b] = rb;
    for (int64_t s = s1 - 1; s >= s0; --s) {
        L = __dadd_rn(L, seg_ds[s]);
        const double y = __dadd_rn(rb, __dmul_rn(dn, L)), z = __dmul_rn(dt, L);
        node_x[s + b] = __dadd_rn(x0, __dmul_rn(dx, L));
        node_r[s + b] = __dsqrt_rn(__dadd_rn(__dmul_rn(y, y), __dmul_rn(z, z)));
        seg_cell[s] = (int32_t)(s + b);
    }
}

// Largest i in [0, n - 2] with c(i) <= v (0 when n == 1), c(i) the centre of
// cell i between faces f[i], f[i + 1].
__device__ __forceinline__ int centre_floor(const double* f, int n, double v) {
    int lo = 0, hi = n;   // c(lo) <= v < c(hi), c(n) = +inf
    if (!(0.5 * (f[0] + f[1]) <= v)) return 0;
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (0.5 * (f[m] + f[m + 1]) <= v) lo = m; else hi = m;
    }
    return min(lo, max(0, n - 2));
}

__global__ void k_node_idw(const double* xf, int32_t nx, const double* rf, int32_t nr, rapral_cells cells,
                           int64_t n_nodes, const double* node_x, const double* node_r, double* Ttr, double* Tve,
                           double* n_out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_nodes) return;
    const double x = node_x[k], r = node_r[k];
    const int i0 = centre_floor(xf, nx, x), j0 = centre_floor(rf, nr, r);
    const int i1 = min(i0 + 2, (int)nx), j1 = min(j0 + 2, (int)nr);
    int64_t id[4];
    double w[4];
    int m = 0;
    int64_t hit = -1;
    for (int i = i0; i < i1 && hit < 0; ++i) {
        const double xc = 0.5 * (xf[i + 1] + xf[i]);
        for (int j = j0; j < j1; ++j) {
            const double rc = 0.5 * (rf[j + 1] + rf[j]);
            const double ddx = __dadd_rn(x, -xc), ddr = __dadd_rn(r, -rc);
            const double d2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddr, ddr));
            const int64_t c = (int64_t)i * nr + j;
            if (d2 == 0.0) { hit = c; break; }
            id[m] = c;
            w[m] = 1.0 / d2;
            ++m;
        }
    }
    const int nc = cells.n_cols;
    if (hit >= 0) {
        Ttr[k] = cells.Ttr[hit];
        Tve[k] = cells.Tve[hit];
        for (int s = 0; s < nc; ++s) n_out[k * nc + s] = cells.n[hit * nc + s];
        return;
    }
    double ws = 0.0;
    for (int q = 0; q < m; ++q) ws = __dadd_rn(ws, w[q]);
    for (int q = 0; q < m; ++q) w[q] = w[q] / ws;
    double a = 0.0, c = 0.0;
    for (int q = 0; q < m; ++q) {
        a = __dadd_rn(a, __dmul_rn(w[q], cells.Ttr[id[q]]));
        c = __dadd_rn(c, __dmul_rn(w[q], cells.Tve[id[q]]));
    }
    Ttr[k] = a;
    Tve[k] = c;
    for (int s = 0; s < nc; ++s) {
        double v = 0.0;
        for (int q = 0; q < m; ++q) v = __dadd_rn(v, __dmul_rn(w[q], cells.n[id[q] * nc + s]));
        n_out[k * nc + s] = v;
    }
}

__global__ void k_fib_dirs(int32_t n_los, double* dirs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_los) return;
    fib_dir(i, n_los, &dirs[3 * i], &dirs[3 * i + 1], &dirs[3 * i + 2]);
}

// S at the grid direction (phi_q, theta_t) of point p: inverse-distance
// weights 1/|v - g|^2 over the point's four nearest line directions (ties:
// the earlier line), or the line's own S where a grid direction is one.
__global__ void k_fib_grid(int64_t P, const int64_t* point_off, const int32_t* los_index, int32_t n_los,
                           const double* dirs, const double* S, int32_t n_phi, int32_t n_theta, double* G,
                           int* status) {
    if (*status) return;
    const int64_t ng = (int64_t)n_phi * n_theta;
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= P * ng) return;
    const int64_t p = id / ng;
    const int g = (int)(id - p * ng);
    const int q = g / n_theta, t = g - q * n_theta;
    const double phi = 0.5 * M_PI * (double)q / (double)(n_phi - 1);
    const double theta = 2.0 * M_PI * (double)t / (double)(n_theta - 1);
    const double gx = sin(phi) * cos(theta), gy = cos(phi), gz = sin(phi) * sin(theta);
    double bd[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
    int64_t bi[4] = {-1, -1, -1, -1};
    for (int64_t b = point_off[p]; b < point_off[p + 1]; ++b) {
        const int li = los_index[b];
        if (li < 0 || li >= n_los) {   // checked: never read outside the direction table
            fail(status, CHK_LOS_INDEX, b);
            return;
        }
        const double* v = dirs + 3 * (int64_t)li;
        const double ex = __dadd_rn(v[0], -gx), ey = __dadd_rn(v[1], -gy), ez = __dadd_rn(v[2], -gz);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
        if (!(d2 < bd[3])) continue;
        int k = 3;
        while (k > 0 && d2 < bd[k - 1]) { bd[k] = bd[k - 1]; bi[k] = bi[k - 1]; --k; }
        bd[k] = d2;
        bi[k] = b;
    }
    double out = 0.0;
    if (bi[0] >= 0) {
        if (bd[0] == 0.0) {
            out = S[bi[0]];
        } else {
            double ws = 0.0, wsum = 0.0;
            for (int k = 0; k < 4 && bi[k] >= 0; ++k) {
                const double w = 1.0 / bd[k];
                ws = __dadd_rn(ws, __dmul_rn(w, S[bi[k]]));
                wsum = __dadd_rn(wsum, w);
            }
            out = ws / wsum;
        }
    }
    G[id] = out;
}

// Four-point average sum over the grid cells of point p, theta outer, phi
// inner, in one thread (a fixed order).
__global__ void k_fib_sum(int64_t P, int32_t n_phi, int32_t n_theta, const double* G, double* q, const int* status) {
    if (*status) return;
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double* g = G + p * (int64_t)n_phi * n_theta;
    double s = 0.0;
    for (int t = 0; t + 1 < n_theta; ++t) {
        const double th0 = 2.0 * M_PI * (double)t / (double)(n_theta - 1);
        const double th1 = 2.0 * M_PI * (double)(t + 1) / (double)(n_theta - 1);
        for (int a = 0; a + 1 < n_phi; ++a) {
            const double c0 = cos(0.5 * M_PI * (double)a / (double)(n_phi - 1));
            const double c1 = cos(0.5 * M_PI * (double)(a + 1) / (double)(n_phi - 1));
            const double avg = 0.25 * (((g[a * n_theta + t] + g[(a + 1) * n_theta + t]) + g[a * n_theta + t + 1]) +
                                       g[(a + 1) * n_theta + t + 1]);
            s = __dadd_rn(s, __dmul_rn(__dmul_rn(__dmul_rn(avg, 0.5), __dadd_rn(__dmul_rn(c0, c0), -__dmul_rn(c1, c1))),
                                       __dadd_rn(th1, -th0)));
        }
    }
    q[p] = s;
}

}  // namespace

cudaError_t launch_fib_count(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                             const double* surf_x, int32_t P, int32_t n_los, int64_t* seg_off) {
    const int32_t V = n_los / 2;
    const int64_t B = (int64_t)P * V;
    if (B == 0) return cudaMemsetAsync(seg_off, 0, sizeof(int64_t), ctx->stream);
    k_fib_count<<<div_up(B, 128), 128, 0, ctx->stream>>>(xf, nx, rf, nr, surf_x, P, n_los, V, seg_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_scan_i64(ctx, seg_off, B);
}

cudaError_t launch_fib_fill(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                            const double* surf_x, int32_t P, int32_t n_los, const int64_t* seg_off,
                            int32_t* seg_cell, double* seg_ds, int64_t* point_off, int64_t* dir_off,
                            double* dir_scale, double* dir_weight, int32_t* bundle_wall, int32_t* los_index,
                            double* node_x, double* node_r) {
    const int32_t V = n_los / 2;
    const int64_t B = (int64_t)P * V;
    k_fib_fill<<<div_up(B + 1, 128), 128, 0, ctx->stream>>>(xf, nx, rf, nr, surf_x, P, n_los, V, seg_off, seg_cell,
                                                            seg_ds, point_off, dir_off, dir_scale, dir_weight,
                                                            bundle_wall, los_index, node_x, node_r);
    return cudaGetLastError();
}

cudaError_t launch_node_idw(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                            const rapral_cells* cells, int64_t n_nodes, const double* node_x, const double* node_r,
                            double* Ttr, double* Tve, double* n) {
    if (n_nodes == 0) return cudaSuccess;
    k_node_idw<<<div_up(n_nodes, 128), 128, 0, ctx->stream>>>(xf, nx, rf, nr, *cells, n_nodes, node_x, node_r, Ttr,
                                                              Tve, n);
    return cudaGetLastError();
}

size_t fib_flux_scratch_bytes(int64_t P, int32_t n_los, int32_t n_phi, int32_t n_theta) {
    return (size_t)(3 * (int64_t)n_los + P * (int64_t)n_phi * n_theta) * sizeof(double) + 256;
}

cudaError_t launch_fib_flux(rapral_ctx* ctx, int64_t P, const int64_t* point_off, const int32_t* los_index,
                            int32_t n_los, const double* S, int32_t n_phi, int32_t n_theta, double* q,
                            void* scratch) {
    if (P == 0) return cudaSuccess;
    double* dirs = reinterpret_cast<double*>(scratch);
    double* G = dirs + 3 * (int64_t)n_los;
    k_fib_dirs<<<div_up(n_los, 128), 128, 0, ctx->stream>>>(n_los, dirs);
    const int64_t n = P * (int64_t)n_phi * n_theta;
    k_fib_grid<<<div_up(n, 128), 128, 0, ctx->stream>>>(P, point_off, los_index, n_los, dirs, S, n_phi, n_theta, G,
                                                        ctx->d_status);
    k_fib_sum<<<div_up(P, 64), 64, 0, ctx->stream>>>(P, n_phi, n_theta, G, q, ctx->d_status);
    return cudaGetLastError();
}
