// Quasi-steady-state collisional-radiative populations (Sec. 2.1): per cell
// and atomic radiator, the rate matrix R and source b of the QSS master
// equation, solved by LU with partial pivoting.  One warp per cell: lanes
// compute the transitions' up / down rates into shared memory, then lane i
// assembles row i in transition order (losses on the diagonal, gains off
// it), pivots and eliminates its row, and lane 0 substitutes back.  FP64
// throughout: the systems span many orders of magnitude in their rates.
#include "rapral_internal.cuh"

namespace {

constexpr int QW = 2;          // warps (cells) per block
constexpr int QMAXL = 32;      // levels solved
constexpr int QMAXT = QMAXL * (QMAXL - 1) / 2;
constexpr double N_AVOGADRO = 6.022e23;

__global__ void __launch_bounds__(32 * QW) k_qss(rapral_cr_model m, rapral_cells cells, Phys ph, double* n_out,
                                                 int* status) {
    if (*status) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * QW + w;
    if (c >= cells.n_cells) return;   // whole warp
    __shared__ double Rs[QW][QMAXL][QMAXL + 1];
    __shared__ double bs[QW][QMAXL];
    __shared__ double rate_up[QW][QMAXT], rate_dn[QW][QMAXT];
    __shared__ double Qh[QW][QMAXL], Qv[QW][QMAXL];
    double (*R)[QMAXL + 1] = Rs[w];
    double* b = bs[w];
    const int l = m.n_levels, T = m.n_trans, nc = cells.n_cols;
    const double Ttr = cells.Ttr[c], Tve = cells.Tve[c];
    const double* dens = cells.n + c * nc;
    double nM = 0.0;
    for (int k = 0; k < nc; ++k)
        if (k != cells.ne_col) nM += dens[k];
    const double ne = dens[cells.ne_col];
    const double nion = m.ion_col >= 0 ? dens[m.ion_col] : 0.0;
    // level weights Q_i = g_i e^{-c2 E_i / T} at both temperatures
    if (lane < l) {
        Qh[w][lane] = m.g[lane] * exp(-ph.c2 * m.E[lane] / Ttr);
        Qv[w][lane] = m.g[lane] * exp(-ph.c2 * m.E[lane] / Tve);
    }
    __syncwarp();
    const double lnTtr = log(Ttr), lnTve = log(Tve), iTtr = 1.0 / Ttr, iTve = 1.0 / Tve;
    // transition rates per particle of the lower (up) / upper (down) level;
    // every warp checks every transition before any indexed use
    bool bad = false;
    for (int t = lane; t < T; t += 32) {
        const int i = m.lo[t], j = m.up[t];
        if (i < 0 || j <= i || j >= l) {
            fail(status, CHK_CR_TRANS, t);
            bad = true;
            continue;
        }
        // C T^n e^{-theta/T} as C e^{n ln T - theta/T}: one exp a rate
        const double theta = ph.c2 * (m.E[j] - m.E[i]);
        const double kh_up = m.hp_C[t] * exp(m.hp_n[t] * lnTtr - theta * iTtr);
        const double kh_dn = kh_up * Qh[w][i] / Qh[w][j];
        const double ke_up = m.e_C[t] * exp(m.e_n[t] * lnTve - theta * iTve);
        const double ke_dn = ke_up * Qv[w][i] / Qv[w][j];
        const double rad = m.A[t] * (m.lam[t] >= 200.0 ? 1.0 : 0.0);
        rate_up[w][t] = (kh_up * nM + ke_up * ne) / N_AVOGADRO;
        rate_dn[w][t] = (kh_dn * nM + ke_dn * ne) / N_AVOGADRO + rad;
    }
    if (__any_sync(0xffffffffu, bad)) return;
    __syncwarp();
    // row assembly: lane r owns row r
    if (lane < l) {
        for (int j = 0; j < l; ++j) R[lane][j] = 0.0;
        b[lane] = 0.0;
        if (lane > 0) {
            for (int t = 0; t < T; ++t) {
                const int i = m.lo[t], j = m.up[t];
                if (lane == i) { R[i][i] -= rate_up[w][t]; R[i][j] += rate_dn[w][t]; }
                if (lane == j) { R[j][j] -= rate_dn[w][t]; R[j][i] += rate_up[w][t]; }
            }
            // electron-impact ionisation and three-body recombination
            const double Qp = m.g_ion * exp(-ph.c2 * m.E_ionize / Tve);
            const double Qe = 2.0 * pow(2.0 * M_PI * ph.me * ph.kB * Tve / (ph.h * ph.h), 1.5);
            const double kf = m.ii_C[lane] * pow(Tve, m.ii_n[lane]) * exp(-ph.c2 * (m.E_ionize - m.E[lane]) / Tve);
            const double kr = kf * Qv[w][lane] / (Qp * Qe);
            R[lane][lane] -= kf * ne / N_AVOGADRO;
            b[lane] = -kr * nion * ne * ne / N_AVOGADRO;
        } else {   // closure: the levels and the lumped ones above sum to the density
            for (int j = 0; j < l; ++j) R[0][j] = 1.0;
            if (m.n_levels_all > l) {
                double s = 0.0;
                for (int p = l; p < m.n_levels_all; ++p) s += m.g[p] * exp(-ph.c2 * m.E[p] / Tve);
                R[0][l - 1] = 1.0 + s / Qv[w][l - 1];
            }
            b[0] = dens[m.col];
        }
    }
    __syncwarp();
    // LU with partial pivoting (the first largest |R[r][k]| of rows r >= k)
    for (int k = 0; k < l - 1; ++k) {
        double v = (lane >= k && lane < l) ? fabs(R[lane][k]) : -1.0;
        int idx = lane;
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, v, off);
            const int oi = __shfl_down_sync(0xffffffffu, idx, off);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
        }
        const int p = __shfl_sync(0xffffffffu, idx, 0);
        const double pv = __shfl_sync(0xffffffffu, v, 0);
        if (!(pv > 0.0)) {
            if (lane == 0) fail(status, CHK_CR_SINGULAR, c);
            return;
        }
        if (p != k) {
            if (lane < l) { const double x = R[k][lane]; R[k][lane] = R[p][lane]; R[p][lane] = x; }
            if (lane == 0) { const double x = b[k]; b[k] = b[p]; b[p] = x; }
        }
        __syncwarp();
        if (lane > k && lane < l) {
            const double f = R[lane][k] / R[k][k];
            R[lane][k] = f;
            for (int j = k + 1; j < l; ++j) R[lane][j] -= f * R[k][j];
            b[lane] -= f * b[k];
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (!(fabs(R[l - 1][l - 1]) > 0.0)) {
            fail(status, CHK_CR_SINGULAR, c);
        } else {
            for (int i = l - 1; i >= 0; --i) {
                double s = b[i];
                for (int j = i + 1; j < l; ++j) s -= R[i][j] * b[j];
                b[i] = s / R[i][i];
            }
        }
    }
    __syncwarp();
    if (lane < l) n_out[c * l + lane] = b[lane];
}

// Departure coefficients of the model's levels (Sec. 2.1): ln b_i = ln N_i -
// ln N_i^B with the Boltzmann population of the main path, ln N_i^B =
// lnpref + ln g_i - c2 E_i / T_ve.  One thread per (cell, level slot); slots
// past the model's levels hold 0 (b = 1).
__global__ void k_qss_departures(const double* __restrict__ E, const double* __restrict__ g, int l,
                                 const double* __restrict__ Tve, const double* __restrict__ lnpref,
                                 const double* __restrict__ n_qss, int64_t C, int s, int S, int n_lev, double c2,
                                 double* __restrict__ ln_b, int* status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C * n_lev) return;
    const int64_t c = i / n_lev;
    const int k = (int)(i - c * n_lev);
    double v = 0.0;
    if (k < l) {
        const double N = n_qss[c * l + k];
        if (!(N > 0.0)) {
            fail(status, CHK_CR_POP, c);
            v = 0.0;
        } else {
            v = log(N) - (lnpref[c * S + s] + log(g[k]) - c2 * E[k] / Tve[c]);
        }
    }
    ln_b[(c * S + s) * n_lev + k] = v;
}

__global__ void k_check_levels(const int32_t* __restrict__ u, const int32_t* __restrict__ lo, int64_t L, int n_lev,
                               int* status) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    const int a = u[l], b = lo[l];
    if (a < -1 || a >= n_lev || b < -1 || b >= n_lev) fail(status, CHK_DEP_LEVEL, l);
}

}  // namespace

cudaError_t launch_qss(rapral_ctx* ctx, const rapral_cr_model* m, const rapral_cells* cells, double* n_out,
                       const Phys& ph) {
    if (cells->n_cells == 0) return cudaSuccess;
    if (m->n_trans > QMAXT || m->n_levels > QMAXL) return cudaErrorInvalidValue;
    k_qss<<<div_up(cells->n_cells, QW), 32 * QW, 0, ctx->stream>>>(*m, *cells, ph, n_out, ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_qss_departures(rapral_ctx* ctx, const rapral_cr_model* m, const rapral_cells* cells, int32_t s,
                                  int32_t S, const double* n_qss, double* ln_b, int32_t n_lev, const Phys& ph) {
    const int64_t n = cells->n_cells * n_lev;
    if (n == 0) return cudaSuccess;
    k_qss_departures<<<div_up(n, 256), 256, 0, ctx->stream>>>(m->E, m->g, m->n_levels, cells->Tve, cells->lnpref,
                                                             n_qss, cells->n_cells, s, S, n_lev, ph.c2, ln_b,
                                                             ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_check_levels(rapral_ctx* ctx, const int32_t* lev_u, const int32_t* lev_l, int64_t L,
                                int32_t n_lev) {
    if (L == 0) return cudaSuccess;
    k_check_levels<<<div_up(L, 256), 256, 0, ctx->stream>>>(lev_u, lev_l, L, n_lev, ctx->d_status);
    return cudaGetLastError();
}
