// Atomic continuum of Sec. 2.2.1: bound-free absorption N_i sigma_i and its
// Kirchhoff / Saha-Boltzmann emission, and the hydrogenic free-free fit of
// Table 3 with the D(sigma, T) correction, added to the coefficients of the
// line sum.
//
//   k_cont_validate  per model: node offsets, increasing tables, levels
//   k_cont_levels    one block: all models' levels in one list sorted by the
//                    last node of their tables, descending
//   k_cont_tiles     per tile of W grid points: the levels whose table
//                    reaches the tile (a prefix of the sorted list)
//   k_cont_sigma     the tables resampled at the tiles' points, FP64
//                    interpolation, stored [tile][level][W] in the path's type
//   k_cont_coef      per (level, cell): N_i and N_+ N_e S_i e^{...}; per cell
//                    and model: the free-free factors and the T-row of D
//   k_continuum      per (cell group, tile): the level sums from shared
//                    memory, then free-free and the Planck factor, added to
//                    kappa and j
//
// Emission without overflow: with v_i = (E_ion - E_i) / 1e7 and u = 1 / lam
// (nm^-1), theta = c2 1e7 / T, the bound-free term is
//   j_i = P(lam) / (1 - e^{-theta u}) * sigma_i * A_i e^{-theta (u - v_i)},
//   A_i = N_+ N_e (h^2 / (2 pi m_e k T))^1.5 g_i / (2 Q_+),
// where P(lam) = 2 h c^2 / lam^5 in the Planck function's units.  The
// exponent is <= 0 wherever sigma_i != 0 (lam below the edge), whereas the
// Saha factor and the Planck function alone over- and underflow at low T.
#include "rapral_internal.cuh"

namespace {

constexpr double LAM_H = 91.1267;   // nm, hydrogen's edge: sigma = LAM_H / lam
constexpr int CONT_DMAX = 64;       // D table nodes per axis
constexpr int CONT_LCH = 32;        // levels staged per chunk

struct ContLevel {
    double last;   // last table node, nm
    double v;      // (E_ion - E_i) / 1e7, nm^-1
    int m, i;      // model, level in the model
    int pad0, pad1;
};

struct ContModels {
    int M, I;                          // models, levels in all
    int lev0[RAPRAL_MAX_CONT_MODELS + 1];
    rapral_continuum m[RAPRAL_MAX_CONT_MODELS];
};

__device__ __forceinline__ float cont_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// exponential of the per-term factor: FP32 takes theta pre-scaled by log2(e)
__device__ __forceinline__ float cont_exp(float x) { return cont_ex2(x); }
__device__ __forceinline__ double cont_exp(double x) { return exp(x); }

__global__ void k_cont_validate(ContModels M, int* status) {
    const rapral_continuum& m = M.m[blockIdx.x];
    for (int i = threadIdx.x; i < m.n_levels; i += blockDim.x) {
        const int64_t a = m.node_off[i], b = m.node_off[i + 1];
        if ((i == 0 && a != 0) || (i == m.n_levels - 1 && b != m.n_nodes) || a < 0 || b < a + 2 ||
            b > m.n_nodes) {
            fail(status, CHK_CONT_TABLE, i);
            continue;
        }
        if (!(m.E[i] >= 0.0 && m.E[i] < m.E_ionize) || !(m.g[i] > 0.0) || !isfinite(m.g[i]))
            fail(status, CHK_CONT_TABLE, i);
        for (int64_t j = a; j < b; ++j) {
            if (!(m.node_sigma[j] >= 0.0) || !isfinite(m.node_sigma[j]) || !(m.node_lam[j] > 0.0) ||
                !isfinite(m.node_lam[j]) || (j + 1 < b && !(m.node_lam[j + 1] > m.node_lam[j]))) {
                fail(status, CHK_CONT_TABLE, j);
                break;
            }
        }
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < m.n_ion_terms; ++k)
            if (!(m.ion_g[k] >= 0.0) || !isfinite(m.ion_E[k])) fail(status, CHK_CONT_TABLE, k);
        if (m.D) {
            for (int k = 0; k + 1 < m.n_D_sigma; ++k)
                if (!(m.D_sigma[k + 1] > m.D_sigma[k])) fail(status, CHK_CONT_TABLE, k);
            for (int k = 0; k + 1 < m.n_D_T; ++k)
                if (!(m.D_T[k + 1] > m.D_T[k])) fail(status, CHK_CONT_TABLE, k);
        }
    }
}

// rank sort of at most 1024 levels by the last node of their tables
__global__ void __launch_bounds__(1024) k_cont_levels(ContModels M, ContLevel* out, const int* status) {
    if (*status) return;
    __shared__ double key[RAPRAL_MAX_CONT_LEVELS];
    const int r = threadIdx.x;
    int m = 0, i = 0;
    double last = 0.0;
    if (r < M.I) {
        while (r >= M.lev0[m + 1]) ++m;
        i = r - M.lev0[m];
        last = M.m[m].node_lam[M.m[m].node_off[i + 1] - 1];
        key[r] = last;
    }
    __syncthreads();
    if (r < M.I) {
        int rank = 0;
        for (int q = 0; q < M.I; ++q) rank += (key[q] > last || (key[q] == last && q < r)) ? 1 : 0;
        ContLevel L;
        L.last = last;
        L.v = (M.m[m].E_ionize - M.m[m].E[i]) * 1e-7;
        L.m = m; L.i = i; L.pad0 = L.pad1 = 0;
        out[rank] = L;
    }
}

// levels reaching each tile: the prefix of the sorted list with last >= the
// tile's first wavelength
__global__ void k_cont_tiles(const ContLevel* lev, int I, int64_t T, int W, double lam_min, double h, int64_t k0,
                             int* n_lev, int64_t* cnt, const int* status) {
    if (*status) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const double lam0 = lam_min + (double)(k0 + t * W) * h;
    int lo = 0, hi = I;   // first index with last < lam0
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (lev[mid].last >= lam0) lo = mid + 1;
        else hi = mid;
    }
    n_lev[t] = lo;
    cnt[t] = (int64_t)lo * W;
}

// linear interpolation in one level's table, zero outside it (FP64)
__device__ double cont_sigma(const rapral_continuum& m, int i, double lam) {
    int64_t a = m.node_off[i], b = m.node_off[i + 1] - 1;
    const double* x = m.node_lam;
    const double* y = m.node_sigma;
    if (!(lam >= x[a]) || lam > x[b]) return 0.0;
    if (lam == x[b]) return y[b];
    while (b - a > 1) {   // x[a] <= lam < x[b]
        const int64_t mid = (a + b) >> 1;
        if (x[mid] <= lam) a = mid;
        else b = mid;
    }
    const double slope = (y[a + 1] - y[a]) / (x[a + 1] - x[a]);
    return slope * (lam - x[a]) + y[a];
}

template <typename Tp>
__global__ void __launch_bounds__(128) k_cont_sigma(ContModels M, const ContLevel* lev, const int* n_lev,
                                                     const int64_t* tab_off, int W, double lam_min, double h,
                                                     int64_t k0, int64_t nk, Tp* tab, const int* status) {
    if (*status) return;
    const int64_t t = blockIdx.x;
    const int nl = n_lev[t];
    Tp* out = tab + tab_off[t];
    for (int r = 0; r < nl; ++r) {
        const ContLevel L = lev[r];
        const rapral_continuum& m = M.m[L.m];
        for (int p = threadIdx.x; p < W; p += blockDim.x) {
            const int64_t k = t * W + p;
            double s = 0.0;
            if (k < nk) s = cont_sigma(m, L.i, lam_min + (double)(k0 + k) * h);
            out[(int64_t)r * W + p] = (Tp)s;
        }
    }
}

// Per (level, cell): N_i (absorption) and A_i (emission, see the file head);
// per cell: theta; per (cell, model): F A1, F A2 of the free-free fit (F =
// N_a (N_+ N_e / N_a)_Saha 1e-40) and D interpolated to the cell's T.
template <typename Tp>
__global__ void k_cont_coef(ContModels M, const ContLevel* lev, rapral_cells cells, int S, Phys ph,
                            Tp* coefN, Tp* coefA, Tp* theta, Tp* ff, Tp* Drow, const int* status) {
    if (*status) return;
    const int64_t c = blockIdx.x;
    const int64_t C = cells.n_cells;
    const double T = cells.Tve[c];
    const double* n = cells.n + c * cells.n_cols;
    const double ne = n[cells.ne_col];
    const double lnS = 1.5 * log(ph.h * ph.h / (2.0 * M_PI * ph.me * ph.kB * T));
    for (int r = threadIdx.x; r < M.I; r += blockDim.x) {
        const ContLevel L = lev[r];
        const rapral_continuum& m = M.m[L.m];
        double Qp = 0.0;
        for (int k = 0; k < m.n_ion_terms; ++k) Qp += m.ion_g[k] * exp(-ph.c2 * m.ion_E[k] / T);
        const double lg = log(m.g[L.i]);
        const double N = exp(cells.lnpref[c * S + m.species] + lg - ph.c2 * m.E[L.i] / T);
        const double A = exp(log(n[m.ion_col]) + log(ne) + lnS - log(2.0 * Qp) + lg);
        coefN[r * C + c] = (Tp)N;
        coefA[r * C + c] = (Tp)A;
    }
    if (threadIdx.x == 0) {
        const double th = ph.c2 * 1e7 / T;
        theta[c] = (Tp)(sizeof(Tp) == 4 ? th * 1.4426950408889634 : th);
    }
    for (int mi = threadIdx.x; mi < M.M; mi += blockDim.x) {
        const rapral_continuum& m = M.m[mi];
        double Qp = 0.0;
        for (int k = 0; k < m.n_ion_terms; ++k) Qp += m.ion_g[k] * exp(-ph.c2 * m.ion_E[k] / T);
        const double F = exp(cells.lnpref[c * S + m.species] + log(2.0 * Qp) - lnS - ph.c2 * m.E_ionize / T) * 1e-40;
        const double* cc = m.ff_c;
        const double A1 = cc[0] + cc[1] * exp(-cc[2] * T);
        const double A2 = cc[3] + cc[4] * exp(-cc[5] * T) + cc[6] * exp(-cc[7] * T);
        ff[(c * M.M + mi) * 2] = (Tp)(F * A1);
        ff[(c * M.M + mi) * 2 + 1] = (Tp)(F * A2);
        Tp* row = Drow + (c * M.M + mi) * CONT_DMAX;
        if (m.D) {
            const int nT = m.n_D_T;
            const double Tc = fmin(fmax(T, m.D_T[0]), m.D_T[nT - 1]);
            int it = 0;
            while (it < nT - 2 && m.D_T[it + 1] <= Tc) ++it;
            const double w = (Tc - m.D_T[it]) / (m.D_T[it + 1] - m.D_T[it]);
            for (int j = 0; j < m.n_D_sigma; ++j)
                row[j] = (Tp)((1.0 - w) * m.D[it * m.n_D_sigma + j] + w * m.D[(it + 1) * m.n_D_sigma + j]);
        }
    }
}

struct ContMain {
    int M, I, S;
    int64_t C, nk, k0, ld;
    double lam_min, h;
    Phys ph;
    const ContLevel* lev;
    const int* n_lev;
    const int64_t* tab_off;
    const void* tab;
    const void *coefN, *coefA, *theta, *ff, *Drow;
    int nDs[RAPRAL_MAX_CONT_MODELS];           // D sigma nodes (0: no D)
    const double* Dsig[RAPRAL_MAX_CONT_MODELS];
    void *kappa, *emis;
    const int* status;
};

template <typename Tp, int PP>
struct VecOf;
template <>
struct VecOf<float, 4> { using type = float4; };
template <>
struct VecOf<double, 2> { using type = double2; };

template <typename Tp, int PP>
__device__ __forceinline__ void load_pts(const Tp* p, Tp (&o)[PP]) {
    using V = typename VecOf<Tp, PP>::type;
    const V x = *reinterpret_cast<const V*>(p);
    const Tp* e = reinterpret_cast<const Tp*>(&x);
#pragma unroll
    for (int q = 0; q < PP; ++q) o[q] = e[q];
}

// One block: 4 warps x RC cells, one tile of W = 32 PP points (lane l owns
// points PP l .. PP l + PP - 1).  Level chunks of the tile's prefix are
// staged in shared memory (table rows, N and A of the block's cells, v).
template <typename Tp, int RC, int PP>
__global__ void __launch_bounds__(128) k_continuum(ContMain a) {
    if (*a.status) return;
    constexpr int W = 32 * PP, CB = 4 * RC;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t t = blockIdx.y;
    const int64_t cb0 = (int64_t)blockIdx.x * CB;
    __shared__ __align__(16) Tp sg[CONT_LCH][W];
    __shared__ Tp sN[CONT_LCH][CB], sA[CONT_LCH][CB];
    __shared__ Tp sv[CONT_LCH];
    const Tp* tab = static_cast<const Tp*>(a.tab) + a.tab_off[t];
    const Tp* cN = static_cast<const Tp*>(a.coefN);
    const Tp* cA = static_cast<const Tp*>(a.coefA);
    const int nl = a.n_lev[t];
    double lam[PP];
    Tp u[PP];
#pragma unroll
    for (int q = 0; q < PP; ++q) {
        lam[q] = a.lam_min + (double)(a.k0 + t * W + lane * PP + q) * a.h;
        u[q] = (Tp)(1.0 / lam[q]);
    }
    Tp th[RC];
#pragma unroll
    for (int rc = 0; rc < RC; ++rc) {
        const int64_t c = cb0 + w * RC + rc;
        th[rc] = c < a.C ? static_cast<const Tp*>(a.theta)[c] : Tp(0);
    }
    Tp kap[RC][PP], jac[RC][PP];
#pragma unroll
    for (int rc = 0; rc < RC; ++rc)
#pragma unroll
        for (int q = 0; q < PP; ++q) kap[rc][q] = jac[rc][q] = Tp(0);

    for (int r0 = 0; r0 < nl; r0 += CONT_LCH) {
        const int nr = min(CONT_LCH, nl - r0);
        __syncthreads();
        for (int x = threadIdx.x; x < nr * W; x += blockDim.x) sg[x / W][x % W] = tab[(int64_t)r0 * W + x];
        for (int x = threadIdx.x; x < nr * CB; x += blockDim.x) {
            const int rr = x / CB, cc = x % CB;
            const int64_t c = cb0 + cc;
            const bool in = c < a.C;
            sN[rr][cc] = in ? cN[(int64_t)(r0 + rr) * a.C + c] : Tp(0);
            sA[rr][cc] = in ? cA[(int64_t)(r0 + rr) * a.C + c] : Tp(0);
        }
        if (threadIdx.x < nr) sv[threadIdx.x] = (Tp)a.lev[r0 + threadIdx.x].v;
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr) {
            Tp s[PP], d[PP];
            load_pts<Tp, PP>(&sg[rr][lane * PP], s);
            const Tp v = sv[rr];
#pragma unroll
            for (int q = 0; q < PP; ++q) d[q] = u[q] - v;
#pragma unroll
            for (int rc = 0; rc < RC; ++rc) {
                const Tp N = sN[rr][w * RC + rc], A = sA[rr][w * RC + rc];
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    kap[rc][q] = fma(N, s[q], kap[rc][q]);
                    jac[rc][q] = fma(A * s[q], cont_exp(-th[rc] * d[q]), jac[rc][q]);
                }
            }
        }
    }

    // free-free, the Planck factor, and the update of kappa and j
    Tp P[PP], s3[PP], s4[PP];
    const double lcm_pref = 1e-7 * 2.0 * a.ph.h * a.ph.c * a.ph.c / 1e4;
#pragma unroll
    for (int q = 0; q < PP; ++q) {
        const double lcm = lam[q] * 1e-7;
        P[q] = (Tp)(lcm_pref / (lcm * lcm * lcm * lcm * lcm));
        const double ir = lam[q] / LAM_H;   // 1 / sigma
        s3[q] = (Tp)(ir * ir * ir);
        s4[q] = (Tp)(ir * ir * ir * ir);
    }
    // D(sigma) intervals of the tile's points, per model (cell independent)
    __shared__ int sDj[RAPRAL_MAX_CONT_MODELS][W];
    __shared__ Tp sDw[RAPRAL_MAX_CONT_MODELS][W];
    __syncthreads();
    for (int x = threadIdx.x; x < a.M * W; x += blockDim.x) {
        const int m = x / W, p = x % W;
        const int nD = a.nDs[m];
        int j = 0;
        Tp wq = Tp(0);
        if (nD) {
            const double* xs = a.Dsig[m];
            const double lp = a.lam_min + (double)(a.k0 + t * W + p) * a.h;
            const double sg_ = fmin(fmax(LAM_H / lp, xs[0]), xs[nD - 1]);
            while (j < nD - 2 && xs[j + 1] <= sg_) ++j;
            wq = (Tp)((sg_ - xs[j]) / (xs[j + 1] - xs[j]));
        }
        sDj[m][p] = j;
        sDw[m][p] = wq;
    }
    __syncthreads();
    const Tp* ffp = static_cast<const Tp*>(a.ff);
    const Tp* Dr = static_cast<const Tp*>(a.Drow);
    Tp* kout = static_cast<Tp*>(a.kappa);
    Tp* jout = static_cast<Tp*>(a.emis);
#pragma unroll
    for (int rc = 0; rc < RC; ++rc) {
        const int64_t c = cb0 + w * RC + rc;
        if (c >= a.C) continue;
        Tp kff[PP];
#pragma unroll
        for (int q = 0; q < PP; ++q) kff[q] = Tp(0);
        for (int m = 0; m < a.M; ++m) {
            const Tp FA1 = ffp[(c * a.M + m) * 2], FA2 = ffp[(c * a.M + m) * 2 + 1];
            const int nD = a.nDs[m];
            const Tp* row = Dr + (c * a.M + m) * CONT_DMAX;
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                Tp D = Tp(0);
                if (nD) {
                    const int j = sDj[m][lane * PP + q];
                    const Tp wq = sDw[m][lane * PP + q];
                    D = (Tp(1) - wq) * row[j] + wq * row[j + 1];
                }
                kff[q] = fma(fma(FA1, s4[q], FA2 * s3[q]), Tp(1) + D, kff[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < PP; ++q) {
            const int64_t k = t * W + lane * PP + q;
            if (k >= a.nk) continue;
            const Tp x = th[rc] * u[q];
            Tp em, den;
            if (sizeof(Tp) == 4) {
                em = cont_exp(-x);
                den = Tp(1) - em;
            } else {
                em = exp(-(double)x);
                den = (Tp)(-expm1(-(double)x));
            }
            const int64_t o = c * a.ld + k;
            kout[o] += kap[rc][q] + kff[q];
            jout[o] += P[q] / den * (jac[rc][q] + em * kff[q]);
        }
    }
}

}  // namespace

static size_t cont_need(size_t need, int64_t I, int64_t T, int64_t C, int M, size_t esz) {
    need = arena_need(need, (size_t)I * sizeof(ContLevel));
    need = arena_need(need, (size_t)T * sizeof(int));
    need = arena_need(need, (size_t)(T + 1) * sizeof(int64_t));
    need = arena_need(need, (size_t)I * C * esz);
    need = arena_need(need, (size_t)I * C * esz);
    need = arena_need(need, (size_t)C * esz);
    need = arena_need(need, (size_t)C * M * 2 * esz);
    need = arena_need(need, (size_t)C * M * CONT_DMAX * esz);
    return need;
}

template <typename Tp, int RC, int PP>
static int cont_run(rapral_ctx* ctx, const ContModels& Mh, int S, const rapral_cells* cells, const rapral_grid* g,
                    double h, int64_t k0, int64_t nk, void* kappa, void* emis, int64_t ld, const Phys& ph) {
    constexpr int W = 32 * PP, CB = 4 * RC;
    const int64_t T = (nk + W - 1) / W, C = cells->n_cells;
    const int I = Mh.I, M = Mh.M;
    const size_t esz = sizeof(Tp);
    if (T > 65535) return set_error(ctx, RAPRAL_EINVAL, "continuum range of %lld points is too long", (long long)nk);
    if ((C + CB - 1) / CB > 2147483647LL) return set_error(ctx, RAPRAL_EINVAL, "too many cells");
    const size_t phase1 = cont_need(0, I, T, C, M, esz);
    int st = ws_reserve(ctx, phase1 + 256);
    if (st) return st;
    Arena ar{ctx->ws, ctx->ws_bytes};
    ContLevel* lev = ar.take<ContLevel>(I);
    int* n_lev = ar.take<int>(T);
    int64_t* tab_off = ar.take<int64_t>(T + 1);
    Tp* coefN = ar.take<Tp>((size_t)I * C);
    Tp* coefA = ar.take<Tp>((size_t)I * C);
    Tp* theta = ar.take<Tp>(C);
    Tp* ff = ar.take<Tp>((size_t)C * M * 2);
    Tp* Drow = ar.take<Tp>((size_t)C * M * CONT_DMAX);
    cudaStream_t s = ctx->stream;
    cudaError_t e = launch_validate_cells(ctx, cells);
    if (e == cudaSuccess) {
        k_cont_validate<<<M, 128, 0, s>>>(Mh, ctx->d_status);
        k_cont_levels<<<1, RAPRAL_MAX_CONT_LEVELS, 0, s>>>(Mh, lev, ctx->d_status);
        k_cont_tiles<<<div_up(T, 256), 256, 0, s>>>(lev, I, T, W, g->lam_min, h, k0, n_lev, tab_off, ctx->d_status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_scan_i64(ctx, tab_off, T);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned, tab_off + T, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->h_pinned + 4, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(ctx, e, "continuum tables");
    if (ctx->h_pinned[4 + ST_CODE]) return read_status(ctx);
    const int64_t total = *reinterpret_cast<const int64_t*>(ctx->h_pinned);
    const size_t need = arena_need(phase1, (size_t)total * esz);
    if (need + 256 > ctx->ws_bytes) {   // the arena moves: start again in the larger one
        st = ws_reserve(ctx, need + 256);
        if (st) return st;
        return cont_run<Tp, RC, PP>(ctx, Mh, S, cells, g, h, k0, nk, kappa, emis, ld, ph);
    }
    Tp* tab = ar.take<Tp>((size_t)total);
    k_cont_sigma<Tp><<<(unsigned)T, 128, 0, s>>>(Mh, lev, n_lev, tab_off, W, g->lam_min, h, k0, nk, tab,
                                                ctx->d_status);
    k_cont_coef<Tp><<<(unsigned)C, 128, 0, s>>>(Mh, lev, *cells, S, ph, coefN, coefA, theta, ff, Drow,
                                               ctx->d_status);
    ContMain a;
    a.M = M; a.I = I; a.S = S; a.C = C; a.nk = nk; a.k0 = k0; a.ld = ld;
    a.lam_min = g->lam_min; a.h = h; a.ph = ph;
    a.lev = lev; a.n_lev = n_lev; a.tab_off = tab_off; a.tab = tab;
    a.coefN = coefN; a.coefA = coefA; a.theta = theta; a.ff = ff; a.Drow = Drow;
    for (int m = 0; m < RAPRAL_MAX_CONT_MODELS; ++m) {
        a.nDs[m] = (m < M && Mh.m[m].D) ? Mh.m[m].n_D_sigma : 0;
        a.Dsig[m] = m < M ? Mh.m[m].D_sigma : nullptr;
    }
    a.kappa = kappa; a.emis = emis; a.status = ctx->d_status;
    dim3 grid((unsigned)((C + CB - 1) / CB), (unsigned)T);
    k_continuum<Tp, RC, PP><<<grid, 128, 0, s>>>(a);
    return cuda_status(ctx, cudaGetLastError(), "continuum");
}

int rapral_continuum_coeffs(rapral_ctx* ctx, const rapral_continuum* models, int32_t n_models, int32_t n_species,
                            const rapral_cells* cells, const rapral_grid* g, int64_t k0, int64_t nk, int precision,
                            void* kappa, void* emis, int64_t ld) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!models || !cells || !g || !kappa || !emis) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (n_models < 1 || n_models > RAPRAL_MAX_CONT_MODELS)
        return set_error(ctx, RAPRAL_EINVAL, "1 .. %d continuum models", RAPRAL_MAX_CONT_MODELS);
    if (precision != RAPRAL_FP64 && precision != RAPRAL_FP32)
        return set_error(ctx, RAPRAL_EINVAL, "precision %d", precision);
    if (g->n < 2 || !(g->lam_max > g->lam_min) || !(g->lam_min > 0.0) || k0 < 0 || nk < 1 || k0 + nk > g->n)
        return set_error(ctx, RAPRAL_EINVAL, "grid or range");
    if (ld < nk) return set_error(ctx, RAPRAL_EINVAL, "ld < nk");
    if (n_species < 1 || n_species > RAPRAL_MAX_SPECIES) return set_error(ctx, RAPRAL_EINVAL, "species count");
    if (cells->n_cells < 0 || cells->n_cols < 1 || cells->ne_col < 0 || cells->ne_col >= cells->n_cols)
        return set_error(ctx, RAPRAL_EINVAL, "cell array sizes");
    if (cells->n_cells == 0) return RAPRAL_OK;
    if (!cells->lnpref || !cells->Tve || !cells->n) return set_error(ctx, RAPRAL_EINVAL, "cells need Tve, n, lnpref");
    ContModels Mh{};
    Mh.M = n_models;
    Mh.lev0[0] = 0;
    for (int m = 0; m < n_models; ++m) {
        const rapral_continuum& c = models[m];
        if (c.species < 0 || c.species >= n_species || c.atom_col < 0 || c.atom_col >= cells->n_cols ||
            c.ion_col < 0 || c.ion_col >= cells->n_cols)
            return set_error(ctx, RAPRAL_EINVAL, "continuum model %d: species or density columns", m);
        if (c.n_levels < 1 || c.n_nodes < 2 || !c.E || !c.g || !c.node_off || !c.node_lam || !c.node_sigma)
            return set_error(ctx, RAPRAL_EINVAL, "continuum model %d: levels or tables", m);
        if (c.n_ion_terms < 1 || !c.ion_E || !c.ion_g)
            return set_error(ctx, RAPRAL_EINVAL, "continuum model %d: ion terms", m);
        if (!(c.E_ionize > 0.0) || !std::isfinite(c.E_ionize))
            return set_error(ctx, RAPRAL_EINVAL, "continuum model %d: ionisation energy", m);
        for (int k = 0; k < 8; ++k)
            if (!std::isfinite(c.ff_c[k])) return set_error(ctx, RAPRAL_EINVAL, "continuum model %d: ff_c", m);
        if (c.D && (c.n_D_sigma < 2 || c.n_D_T < 2 || c.n_D_sigma > CONT_DMAX || c.n_D_T > CONT_DMAX ||
                    !c.D_sigma || !c.D_T))
            return set_error(ctx, RAPRAL_EINVAL, "continuum model %d: D table sizes 2 .. %d", m, CONT_DMAX);
        Mh.m[m] = c;
        Mh.lev0[m + 1] = Mh.lev0[m] + c.n_levels;
        if (Mh.lev0[m + 1] > RAPRAL_MAX_CONT_LEVELS)
            return set_error(ctx, RAPRAL_EINVAL, "more than %d continuum levels", RAPRAL_MAX_CONT_LEVELS);
    }
    Mh.I = Mh.lev0[n_models];
    cudaSetDevice(ctx->device);
    const double h = (g->lam_max - g->lam_min) / (double)(g->n - 1);
    const Phys ph = make_phys(ctx->codata);
    if (precision == RAPRAL_FP64)
        return cont_run<double, 4, 2>(ctx, Mh, n_species, cells, g, h, k0, nk, kappa, emis, ld, ph);
    return cont_run<float, 8, 4>(ctx, Mh, n_species, cells, g, h, k0, nk, kappa, emis, ld, ph);
}
