// Populations (Sec. 2.1) and per-cell preparation.
//
// k_populations: one warp per (cell, species).  Atoms: lanes stride over the
// level list and sum g exp(-c2 E / T_ve).  Diatomics: lanes stride over the
// rotational ladder of each (state, V) and add
//   g_i exp(-c2 E_i / T_ve) exp(-c2 E_V / T_ve) / sigma (2J+1) L_alter exp(-c2 E_J / T_tr),
// which is the product form of g_i exp(-c2E_i/T_ee) Q_vr,i.  One fixed-order
// warp reduction per (cell, species) keeps the result deterministic.  FP64
// throughout (partition sums are FP64 in both precisions).
#include "rapral_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_validate_cells(const double* Ttr, const double* Tve, const double* n, int64_t C,
                                 int32_t ncol, int* status) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= C) return;
    const double a = Ttr[i], b = Tve[i];
    if (!(a > 0.0) || !(b > 0.0) || !isfinite(a) || !isfinite(b)) fail(status, CHK_CELL_T, i);
    for (int j = 0; j < ncol; ++j) {
        const double v = n[i * ncol + j];
        if (!(v >= 0.0) || !isfinite(v)) { fail(status, CHK_CELL_N, i); break; }
    }
}

__global__ void __launch_bounds__(256) k_populations(rapral_species sp, const double* __restrict__ Ttr,
                                                     const double* __restrict__ Tve, const double* __restrict__ n,
                                                     int32_t ncol, int64_t C, double c2, double* __restrict__ lnpref,
                                                     const int* status) {
    if (*status) return;
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int S = sp.n_species;
    if (w >= C * S) return;
    const int64_t c = w / S;
    const int s = (int)(w - c * S);
    const double bve = c2 / Tve[c], btr = c2 / Ttr[c];
    const double N = n[c * ncol + sp.density_col[s]];
    double z = 0.0;
    if (sp.kind[s] == RAPRAL_ATOM) {
        const int64_t a = sp.atom_off[s], b = sp.atom_off[s + 1];
        for (int64_t l = a + lane; l < b; l += 32) z += sp.atom_g[l] * exp(-bve * sp.atom_E[l]);
    } else {
        const int64_t a = sp.st_off[s], b = sp.st_off[s + 1];
        for (int64_t i = a; i < b; ++i) {
            const double pre = sp.st_g[i] * exp(-bve * sp.st_E[i]) / sp.st_sigma[i];
            const int nv = sp.st_nv[i], nj = sp.st_nj[i];
            const double La = sp.st_Lalt[2 * i], Lb = sp.st_Lalt[2 * i + 1];
            const double* rot = sp.rot_E + sp.st_rot_off[i];
            const double* vib = sp.vib_E + sp.st_vib_off[i];
            for (int v = 0; v < nv; ++v) {
                const double pv = pre * exp(-bve * vib[v]);
                for (int J = lane; J < nj; J += 32)
                    z += pv * ((2.0 * J + 1.0) * ((J & 1) ? Lb : La) * exp(-btr * rot[(int64_t)v * nj + J]));
            }
        }
    }
    z = warp_sum(z);
    if (lane == 0) lnpref[c * S + s] = (N > 0.0) ? log(N) - log(z) : -INFINITY;
}

__global__ void k_cell_prep(const double* __restrict__ Ttr, const double* __restrict__ Tve,
                            const double* __restrict__ n, int32_t ncol, int32_t ne_col, int64_t C, double c2,
                            CellPrep* __restrict__ out, unsigned long long* dmax, const int* status) {
    if (*status) return;
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= C) return;
    CellPrep p;
    const double tt = Ttr[c], tv = Tve[c];
    p.bve = c2 / tv;
    p.btr = c2 / tt;
    p.sqrtT = sqrt(tt);
    p.stc = pow(tv / 10000.0, 0.33) * (n[c * ncol + ne_col] / 1e16);
    p.bve_f = (float)p.bve;
    p.btr_f = (float)p.btr;
    p.sqrtT_f = (float)p.sqrtT;
    p.stc_f = (float)p.stc;
    p.bve_ff = ff_from(p.bve);
    p.btr_ff = ff_from(p.btr);
    out[c] = p;
    // positive doubles order like their bit patterns
    atomicMax(&dmax[0], (unsigned long long)__double_as_longlong(p.sqrtT));
    atomicMax(&dmax[1], (unsigned long long)__double_as_longlong(p.stc));
}

// Ground-level weight of each atomic species: the summed g of its levels at
// E = 0 (0 for molecules).
__global__ void k_ground_weights(rapral_species sp, double* g0) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= sp.n_species) return;
    double g = 0.0;
    if (sp.kind[s] == RAPRAL_ATOM)
        for (int64_t k = sp.atom_off[s]; k < sp.atom_off[s + 1]; ++k)
            if (sp.atom_E[k] == 0.0) g += sp.atom_g[k];
    g0[s] = g;
}

// Per (cell, atomic species): ground-level density N_0 = n_s g_0 / Z_s and
// the van der Waals factor W = 6.65e-29 N (2T/M)^0.5 + 2.925e-29 N_o (2T/M_o)^0.5
// (the other heavy particles in column order); zeros for molecules or for
// terms that are off.  Largest values over the cells per species in dmax.
__global__ void k_cell_broad(rapral_species sp, rapral_cells cells, BroadArgs br, const double* __restrict__ g0,
                             double2* __restrict__ cb, float2* __restrict__ cb32, unsigned long long* dmax,
                             const int* status) {
    if (*status) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= cells.n_cells) return;
    const int S = sp.n_species, nc = cells.n_cols;
    const double T = cells.Ttr[c];
    const double* n = cells.n + c * nc;
    for (int s = 0; s < S; ++s) {
        double N0 = 0.0, W = 0.0;
        if (sp.kind[s] == RAPRAL_ATOM) {
            if ((br.flags & RAPRAL_BROAD_RESONANCE) && g0[s] > 0.0)
                N0 = exp(cells.lnpref[c * S + s] + log(g0[s]));
            if (br.flags & RAPRAL_BROAD_VDW) {
                const int col = sp.density_col[s];
                double No = 0.0, NoM = 0.0;
                for (int k = 0; k < nc && k < br.ncol; ++k) {
                    if (k == col || !(br.colmass[k] > 0.0)) continue;
                    No += n[k];
                    NoM += n[k] * br.colmass[k];
                }
                W = 6.65e-29 * n[col] * sqrt(2.0 * T / sp.mass[s]);
                if (No > 0.0) W += 2.925e-29 * No * sqrt(2.0 * T / (NoM / No));
            }
        }
        cb[c * S + s] = make_double2(N0, W);
        cb32[c * S + s] = make_float2((float)N0, (float)W);
        atomicMax(&dmax[2 + 2 * s], (unsigned long long)__double_as_longlong(N0));
        atomicMax(&dmax[3 + 2 * s], (unsigned long long)__double_as_longlong(W));
    }
}

}  // namespace

cudaError_t launch_broad_cells(rapral_ctx* ctx, const rapral_species* sp, const rapral_cells* cells,
                               const BroadArgs& br, double* g0, double2* cb, float2* cb32, unsigned long long* d_max) {
    const int S = sp->n_species;
    cudaError_t e = cudaMemsetAsync(d_max + 2, 0, 2 * (size_t)S * sizeof(unsigned long long), ctx->stream);
    if (e != cudaSuccess) return e;
    k_ground_weights<<<1, 32, 0, ctx->stream>>>(*sp, g0);
    if (cells->n_cells == 0) return cudaGetLastError();
    k_cell_broad<<<div_up(cells->n_cells, 128), 128, 0, ctx->stream>>>(*sp, *cells, br, g0, cb, cb32, d_max,
                                                                       ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_validate_cells(rapral_ctx* ctx, const rapral_cells* cells) {
    k_validate_cells<<<div_up(cells->n_cells, 256), 256, 0, ctx->stream>>>(
        cells->Ttr, cells->Tve, cells->n, cells->n_cells, cells->n_cols, ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_populations(rapral_ctx* ctx, const rapral_species* sp, const rapral_cells* cells,
                               double* lnpref, const Phys& ph) {
    const int64_t warps = cells->n_cells * sp->n_species;
    k_populations<<<div_up(warps * 32, 256), 256, 0, ctx->stream>>>(
        *sp, cells->Ttr, cells->Tve, cells->n, cells->n_cols, cells->n_cells, ph.c2, lnpref, ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_cell_prep(rapral_ctx* ctx, const rapral_cells* cells, const Phys& ph, CellPrep* out,
                             unsigned long long* d_max) {
    cudaError_t e = cudaMemsetAsync(d_max, 0, 2 * sizeof(unsigned long long), ctx->stream);
    if (e != cudaSuccess) return e;
    k_cell_prep<<<div_up(cells->n_cells, 256), 256, 0, ctx->stream>>>(
        cells->Ttr, cells->Tve, cells->n, cells->n_cols, cells->ne_col, cells->n_cells, ph.c2, out, d_max,
        ctx->d_status);
    return cudaGetLastError();
}

// Saha-Boltzmann populations of an atomic radiator (Sec. 2.1): N_i =
// N_+ N_e (h^2 / (2 pi m_e k T))^1.5 g_i e^{hc (E_ion - E_i) / kT} / (2 Q_+),
// that is the prefactor ln(N / Z) of the Boltzmann form replaced by
// ln(N_+ N_e) + 1.5 ln(h^2 / (2 pi m_e k T)) + c2 E_ion / T - ln(2 Q_+), T = T_ve.
// No ions or electrons: -inf (no population).
__global__ void k_saha_prefactor(const double* __restrict__ Tve, const double* __restrict__ n, int ncol, int ne_col,
                                 int64_t C, int s, int S, double E_ion, int ion_col, int n_terms,
                                 const double* __restrict__ ion_E, const double* __restrict__ ion_g, Phys ph,
                                 double* __restrict__ lnpref, const int* status) {
    if (*status) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double T = Tve[c];
    double Qp = 0.0;
    for (int k = 0; k < n_terms; ++k) Qp += ion_g[k] * exp(-ph.c2 * ion_E[k] / T);
    const double pe = n[c * ncol + ion_col] * n[c * ncol + ne_col];
    lnpref[c * S + s] = pe > 0.0 && Qp > 0.0
                            ? log(n[c * ncol + ion_col]) + log(n[c * ncol + ne_col]) +
                                  1.5 * log(ph.h * ph.h / (2.0 * M_PI * ph.me * ph.kB * T)) + ph.c2 * E_ion / T -
                                  log(2.0 * Qp)
                            : -INFINITY;
}

cudaError_t launch_saha_prefactor(rapral_ctx* ctx, const rapral_cells* cells, int s, int S, double E_ion,
                                  int ion_col, int n_terms, const double* ion_E, const double* ion_g,
                                  const Phys& ph, double* lnpref) {
    if (cells->n_cells == 0) return cudaSuccess;
    k_saha_prefactor<<<div_up(cells->n_cells, 256), 256, 0, ctx->stream>>>(
        cells->Tve, cells->n, cells->n_cols, cells->ne_col, cells->n_cells, s, S, E_ion, ion_col, n_terms, ion_E,
        ion_g, ph, lnpref, ctx->d_status);
    return cudaGetLastError();
}
