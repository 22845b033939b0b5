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
    double last;        // last table node, nm
    double v;           // (E_ion - E_i) / 1e7, nm^-1
    int m, i;           // model, level in the model
    int64_t klo, khi;   // grid indices with x_first <= lam_k <= x_last (FP64, the grid's formula)
};

struct ContModels {
    int M, I;                          // models, levels in all
    int lev0[RAPRAL_MAX_CONT_MODELS + 1];
    int64_t node0[RAPRAL_MAX_CONT_MODELS + 1];   // first node of each model in the FP32 node copies
    rapral_continuum m[RAPRAL_MAX_CONT_MODELS];
};

// grid wavelength lam_min + k h with a rounded product and a rounded sum (no
// contraction into an FMA): the same bits as the host-side definition
__device__ __forceinline__ double grid_lam(double lam_min, double h, int64_t k) {
    return __dadd_rn(lam_min, __dmul_rn((double)k, h));
}

__device__ __forceinline__ float cont_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// exponential of the per-term factor: FP32 takes theta pre-scaled by log2(e)
__device__ __forceinline__ float cont_exp(float x) { return cont_ex2(x); }
__device__ __forceinline__ double cont_exp(double x) { return exp(x); }
// P / (1 - e^{-x}): FP32 to the approximate reciprocal's ~1 ulp, FP64 exact
__device__ __forceinline__ float cont_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double cont_div(double a, double b) { return a / b; }

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
__global__ void __launch_bounds__(1024) k_cont_levels(ContModels M, double lam_min, double h, ContLevel* out,
                                                      const int* status) {
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
        L.m = m; L.i = i;
        const double x0 = M.m[m].node_lam[M.m[m].node_off[i]];
        int64_t klo = (int64_t)ceil((x0 - lam_min) / h), khi = (int64_t)floor((last - lam_min) / h);
        while (grid_lam(lam_min, h, klo) < x0) ++klo;
        while (grid_lam(lam_min, h, klo - 1) >= x0) --klo;
        while (grid_lam(lam_min, h, khi) > last) --khi;
        while (grid_lam(lam_min, h, khi + 1) <= last) ++khi;
        L.klo = klo; L.khi = khi;
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
    const double lam0 = grid_lam(lam_min, h, k0 + t * W);
    int lo = 0, hi = I;   // first index with last < lam0
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (lev[mid].last >= lam0) lo = mid + 1;
        else hi = mid;
    }
    n_lev[t] = lo;
    cnt[t] = (int64_t)lo * W;
}

// Linear interpolation in one level's table, zero outside it (FP64).  j is a
// node index with x[j] <= lam on entry (or the first node); it moves forward
// only, so that increasing wavelengths walk the table once.
__device__ __forceinline__ double cont_sigma_walk(const double* x, const double* y, int64_t a, int64_t b,
                                                  int64_t& j, double lam) {
    if (!(lam >= x[a]) || lam > x[b]) return 0.0;
    if (lam == x[b]) return y[b];
    while (j + 1 < b && x[j + 1] <= lam) ++j;   // x[j] <= lam < x[j + 1]
    const double slope = (y[j + 1] - y[j]) / (x[j + 1] - x[j]);
    return slope * (lam - x[j]) + y[j];
}

// one warp per (tile, level): a binary search for the lane's first point,
// then a forward walk over its later points
template <typename Tp>
__global__ void __launch_bounds__(128) k_cont_sigma(ContModels M, const ContLevel* lev, const int* n_lev,
                                                     const int64_t* tab_off, int W, double lam_min, double h,
                                                     int64_t k0, int64_t nk, Tp* tab, const int* status) {
    if (*status) return;
    const int64_t t = blockIdx.x;
    const int nl = n_lev[t];
    const int lane = threadIdx.x & 31;
    Tp* out = tab + tab_off[t];
    for (int r = threadIdx.x >> 5; r < nl; r += blockDim.x >> 5) {
        const ContLevel L = lev[r];
        const rapral_continuum& m = M.m[L.m];
        const int64_t a = m.node_off[L.i], b = m.node_off[L.i + 1] - 1;
        const double* x = m.node_lam;
        const double* y = m.node_sigma;
        const double lam_first = grid_lam(lam_min, h, k0 + t * W + lane);
        int64_t lo = a, hi = b;   // last node <= lam_first (or a)
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (x[mid] <= lam_first) lo = mid;
            else hi = mid;
        }
        int64_t j = lo;
        for (int p = lane; p < W; p += 32) {
            const int64_t k = t * W + p;
            double sg = 0.0;
            if (k < nk) sg = cont_sigma_walk(x, y, a, b, j, grid_lam(lam_min, h, k0 + k));
            out[(int64_t)r * W + p] = (Tp)sg;
        }
    }
}

// Per (level, cell): N_i (absorption) and A_i (emission, see the file head);
// per cell: theta; per (cell, model): F A1, F A2 of the free-free fit (F =
// N_a (N_+ N_e / N_a)_Saha 1e-40) and D interpolated to the cell's T.
// FP32 copies of the tables for the FP32 resampling: per node the value, the
// slope to the next node and the gap to it (FP64 differences, rounded once).
__global__ void k_cont_nodes32(ContModels M, float* yf, float* sf, float* dxf, const int* status) {
    if (*status) return;
    const int m = blockIdx.y;
    if (m >= M.M) return;
    const rapral_continuum& md = M.m[m];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= md.n_nodes) return;
    const int64_t o = M.node0[m] + j;
    yf[o] = (float)md.node_sigma[j];
    const bool next = j + 1 < md.n_nodes;   // the slope of a level's last node is never read
    const double dx = next ? md.node_lam[j + 1] - md.node_lam[j] : 1.0;
    sf[o] = next ? (float)((md.node_sigma[j + 1] - md.node_sigma[j]) / dx) : 0.0f;
    dxf[o] = (float)dx;
}

// FP32 resampling, one warp per (tile, level): the window of grid indices
// inside the table is found in FP64 with the grid's own wavelength formula
// (so that zero / non-zero is decided as in FP64), the interpolation is FP32
// from the tile's first wavelength: lam - x_j = (lam_t - x_j) + p h.
__global__ void __launch_bounds__(128) k_cont_sigma32(ContModels M, const ContLevel* lev, const int* n_lev,
                                                       const int64_t* tab_off, int W, double lam_min, double h,
                                                       int64_t k0, int64_t nk, const float* yf, const float* sf,
                                                       const float* dxf, float* tab, const int* status) {
    if (*status) return;
    const int64_t t = blockIdx.x;
    const int nl = n_lev[t];
    const int lane = threadIdx.x & 31;
    float* out = tab + tab_off[t];
    const int64_t kt = k0 + t * W;   // absolute grid index of the tile's first point
    const double lam_t = grid_lam(lam_min, h, kt);
    const float hf = (float)h;
    for (int r = threadIdx.x >> 5; r < nl; r += blockDim.x >> 5) {
        const ContLevel L = lev[r];
        const rapral_continuum& m = M.m[L.m];
        const int64_t a = m.node_off[L.i], b = m.node_off[L.i + 1] - 1;
        const double* x = m.node_lam;
        const int64_t nb = M.node0[L.m];
        const int64_t klo = L.klo, khi = L.khi;
        // the lane's first point: last node <= its wavelength (or a)
        const double lam_first = grid_lam(lam_min, h, kt + lane);
        int64_t lo = a, hi = b;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (x[mid] <= lam_first) lo = mid;
            else hi = mid;
        }
        int64_t j = lo;
        float base = (float)(lam_t - x[j]);
        for (int p = lane; p < W; p += 32) {
            const int64_t k = kt + p;
            float sg = 0.0f;
            if (k - k0 < nk && k >= klo && k <= khi) {
                float d = fmaf((float)p, hf, base);
                while (j + 1 < b && d >= dxf[nb + j]) {
                    ++j;
                    base = (float)(lam_t - x[j]);
                    d = fmaf((float)p, hf, base);
                }
                sg = fmaf(sf[nb + j], d, yf[nb + j]);
            }
            out[(int64_t)r * W + p] = sg;
        }
    }
}

// Per grid point of the padded range (cell independent): u = 1 / lam, the
// Planck prefactor P = 2 h c^2 / lam^5 (in the Planck function's units),
// 1 / sigma^3 and 1 / sigma^4 of the free-free fit, and per model the D(sigma)
// interval and weight.  FP64 arithmetic, stored in the path's type.
template <typename Tp>
__global__ void k_cont_points(ContModels M, int64_t n_pad, double lam_min, double h, int64_t k0, Phys ph, Tp* pts,
                              int* Dj, Tp* Dw, const int* status) {
    if (*status) return;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pad) return;
    const double lam = grid_lam(lam_min, h, k0 + k);
    const double lcm = lam * 1e-7;
    const double ir = lam / LAM_H;   // 1 / sigma
    pts[k * 4 + 0] = (Tp)(1.0 / lam);
    pts[k * 4 + 1] = (Tp)(1e-7 * 2.0 * ph.h * ph.c * ph.c / (1e4 * lcm * lcm * lcm * lcm * lcm));
    pts[k * 4 + 2] = (Tp)(ir * ir * ir);
    pts[k * 4 + 3] = (Tp)(ir * ir * ir * ir);
    for (int m = 0; m < M.M; ++m) {
        const rapral_continuum& md = M.m[m];
        int j = 0;
        double w = 0.0;
        if (md.D) {
            const double* xs = md.D_sigma;
            const int nD = md.n_D_sigma;
            const double sg = fmin(fmax(LAM_H / lam, xs[0]), xs[nD - 1]);
            int lo = 0, hi = nD - 1;   // last node <= sg, at most nD - 2
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (xs[mid] <= sg) lo = mid;
                else hi = mid;
            }
            j = lo;
            w = (sg - xs[j]) / (xs[j + 1] - xs[j]);
        }
        Dj[m * n_pad + k] = j;
        Dw[m * n_pad + k] = (Tp)w;
    }
}

// A cell is "warm" when the emission factors can be split into a level part
// A_i e^{theta v_i} and the Planck function without leaving the type's range:
// theta u_max <= lim and ln(A_i e^{theta v_i}) <= lim for every level.
template <typename Tp>
__global__ void k_cont_coef(ContModels M, const ContLevel* lev, rapral_cells cells, int S, Phys ph, double u_max,
                            double lim, Tp* coefN, Tp* coefA, Tp* coefA2, int* warm, Tp* theta, Tp* ff, Tp* Drow,
                            const int* status) {
    if (*status) return;
    const int64_t c = blockIdx.x;
    const int64_t C = cells.n_cells;
    const double T = cells.Tve[c];
    const double* n = cells.n + c * cells.n_cols;
    const double ne = n[cells.ne_col];
    const double lnS = 1.5 * log(ph.h * ph.h / (2.0 * M_PI * ph.me * ph.kB * T));
    const double th = ph.c2 * 1e7 / T;
    int hot = th * u_max > lim;
    for (int r = threadIdx.x; r < M.I; r += blockDim.x) {
        const ContLevel L = lev[r];
        const rapral_continuum& m = M.m[L.m];
        double Qp = 0.0;
        for (int k = 0; k < m.n_ion_terms; ++k) Qp += m.ion_g[k] * exp(-ph.c2 * m.ion_E[k] / T);
        const double lg = log(m.g[L.i]);
        const double N = exp(cells.lnpref[c * S + m.species] + lg - ph.c2 * m.E[L.i] / T);
        const double lnA = log(n[m.ion_col]) + log(ne) + lnS - log(2.0 * Qp) + lg;
        const double lnA2 = lnA + th * L.v;
        if (lnA2 > lim) hot = 1;
        coefN[r * C + c] = (Tp)N;
        coefA[r * C + c] = (Tp)exp(lnA);
        coefA2[r * C + c] = (Tp)exp(lnA2);
    }
    hot = __syncthreads_or(hot);
    if (threadIdx.x == 0) {
        theta[c] = (Tp)(sizeof(Tp) == 4 ? th * 1.4426950408889634 : th);
        warm[c] = !hot;
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
    const void *coefN, *coefA, *coefA2, *theta, *ff, *Drow;
    const int* warm;
    int nDs[RAPRAL_MAX_CONT_MODELS];           // D sigma nodes (0: no D)
    int64_t n_pad;                             // T W points
    const void* pts;                           // [n_pad][4]: u, P, 1/sigma^3, 1/sigma^4
    const int* Dj;                             // [M][n_pad]
    const void* Dw;                            // [M][n_pad]
    void *kappa, *emis;
    const int* status;
};

template <typename Tp, int PP>
struct VecOf;
template <>
struct VecOf<float, 4> { using type = float4; };
template <>
struct VecOf<double, 2> { using type = double2; };

// pairs of accumulators: packed FP32 FMA (two lanes an instruction) or two FP64 FMAs
template <typename Tp>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
    static __device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
};
template <>
struct Pair<double> {
    using type = double2;
    static __device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
        return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
    }
};
template <typename V>
__device__ __forceinline__ auto& comp(V& v, int e) { return e ? v.y : v.x; }

// asynchronous global -> shared copies (cp.async): 16-byte pieces, and
// single 4- or 8-byte elements with zero fill when `in` is false
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
template <typename Tp>
__device__ __forceinline__ void cp_async_elem(unsigned dst, const Tp* src, bool in) {
    const unsigned n = in ? (unsigned)sizeof(Tp) : 0u;
    if (sizeof(Tp) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

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
// staged in shared memory (table rows, the level factors of the block's
// cells, v).  SPLIT (every cell of the block warm): j_i = B sigma_i A_i
// e^{theta v_i}, two FMAs a term; otherwise the exponent is taken per term.
template <typename Tp, int RC, int PP, bool SPLIT>
__device__ __forceinline__ void cont_block(const ContMain& a, int64_t t, int64_t cb0, int lane, int w,
                                           Tp (*sg)[32 * PP], Tp (*sN)[4 * RC], Tp (*sA)[4 * RC], Tp* sv) {
    constexpr int W = 32 * PP, CB = 4 * RC;
    const Tp* tab = static_cast<const Tp*>(a.tab) + a.tab_off[t];
    const Tp* cN = static_cast<const Tp*>(a.coefN);
    const Tp* cA = static_cast<const Tp*>(SPLIT ? a.coefA2 : a.coefA);
    const int nl = a.n_lev[t];
    const int64_t kq = t * W + lane * PP;   // the lane's first point in the padded range
    const Tp* pts = static_cast<const Tp*>(a.pts) + kq * 4;
    Tp u[PP];
#pragma unroll
    for (int q = 0; q < PP; ++q) u[q] = pts[q * 4];   // the other three per-point values are read at the end
    Tp th[RC];
#pragma unroll
    for (int rc = 0; rc < RC; ++rc) {
        const int64_t c = cb0 + w * RC + rc;
        th[rc] = c < a.C ? static_cast<const Tp*>(a.theta)[c] : Tp(0);
    }
    using V2 = typename Pair<Tp>::type;
    constexpr int P2 = PP / 2;
    V2 kap[RC][P2], jac[RC][P2];   // point q of cell rc: component q & 1 of entry q / 2
#pragma unroll
    for (int rc = 0; rc < RC; ++rc)
#pragma unroll
        for (int q = 0; q < P2; ++q) kap[rc][q] = jac[rc][q] = V2{Tp(0), Tp(0)};

    for (int r0 = 0; r0 < nl; r0 += CONT_LCH) {
        const int nr = min(CONT_LCH, nl - r0);
        __syncthreads();
        if (sizeof(Tp) == 4) {   // the chunk's table rows and level factors, copied asynchronously
            constexpr int NV = CONT_LCH * W * (int)sizeof(Tp) / 16 / 128;   // 16-byte pieces a thread
            constexpr int NC = CONT_LCH * CB / 128;                        // factors a thread
            const int nv = nr * W * (int)sizeof(Tp) / 16;
            const char* src = reinterpret_cast<const char*>(tab + (int64_t)r0 * W);
            const unsigned dst = (unsigned)__cvta_generic_to_shared(&sg[0][0]);
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int x = threadIdx.x + i * 128;
                if (x < nv) cp_async16(dst + 16u * x, src + 16 * (int64_t)x);
            }
            const unsigned dN = (unsigned)__cvta_generic_to_shared(&sN[0][0]);
            const unsigned dA = (unsigned)__cvta_generic_to_shared(&sA[0][0]);
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const int x = threadIdx.x + i * 128, rr = x / CB;
                const int64_t c = cb0 + x % CB;
                const bool in = rr < nr && c < a.C;
                const int64_t o = in ? (int64_t)(r0 + rr) * a.C + c : 0;   // a valid address; nothing is read when out
                cp_async_elem<Tp>(dN + sizeof(Tp) * x, cN + o, in);
                cp_async_elem<Tp>(dA + sizeof(Tp) * x, cA + o, in);
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        } else {   // FP64: every load of the chunk in flight before the first shared-memory store
            using V = typename VecOf<Tp, 16 / sizeof(Tp)>::type;
            constexpr int NV = CONT_LCH * W * (int)sizeof(Tp) / 16 / 128;
            constexpr int NC = CONT_LCH * CB / 128;
            const int nv = nr * W * (int)sizeof(Tp) / 16;
            const V* src = reinterpret_cast<const V*>(tab + (int64_t)r0 * W);
            V* dst = reinterpret_cast<V*>(&sg[0][0]);
            constexpr int HV = NV / 2;
#pragma unroll
            for (int hv = 0; hv < NV; hv += HV) {
                V rv[HV];
#pragma unroll
                for (int i = 0; i < HV; ++i) {
                    const int x = threadIdx.x + (hv + i) * 128;
                    if (x < nv) rv[i] = src[x];
                }
#pragma unroll
                for (int i = 0; i < HV; ++i) {
                    const int x = threadIdx.x + (hv + i) * 128;
                    if (x < nv) dst[x] = rv[i];
                }
            }
            Tp rn[NC], ra[NC];
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const int x = threadIdx.x + i * 128, rr = x / CB;
                const int64_t c = cb0 + x % CB;
                const bool in = rr < nr && c < a.C;
                rn[i] = in ? cN[(int64_t)(r0 + rr) * a.C + c] : Tp(0);
                ra[i] = in ? cA[(int64_t)(r0 + rr) * a.C + c] : Tp(0);
            }
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const int x = threadIdx.x + i * 128;
                sN[x / CB][x % CB] = rn[i];
                sA[x / CB][x % CB] = ra[i];
            }
        }
        if (!SPLIT && threadIdx.x < nr) sv[threadIdx.x] = (Tp)a.lev[r0 + threadIdx.x].v;
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr) {
            Tp sgp[PP], d[PP];
            load_pts<Tp, PP>(&sg[rr][lane * PP], sgp);
            if (!SPLIT) {
                const Tp v = sv[rr];
#pragma unroll
                for (int q = 0; q < PP; ++q) d[q] = u[q] - v;
            }
            // the warp's RC coefficients as 16-byte broadcast loads
            Tp Nw[RC], Aw[RC];
            {
                using V = typename VecOf<Tp, 16 / sizeof(Tp)>::type;
                constexpr int E = 16 / sizeof(Tp);
#pragma unroll
                for (int v0 = 0; v0 < RC; v0 += E) {
                    const V nv = *reinterpret_cast<const V*>(&sN[rr][w * RC + v0]);
                    const V av = *reinterpret_cast<const V*>(&sA[rr][w * RC + v0]);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        Nw[v0 + e] = reinterpret_cast<const Tp*>(&nv)[e];
                        Aw[v0 + e] = reinterpret_cast<const Tp*>(&av)[e];
                    }
                }
            }
#pragma unroll
            for (int rc = 0; rc < RC; ++rc) {
                const Tp N = Nw[rc], A = Aw[rc];
#pragma unroll
                for (int q2 = 0; q2 < P2; ++q2) {
                    const V2 s2{sgp[2 * q2], sgp[2 * q2 + 1]};
                    kap[rc][q2] = Pair<Tp>::fma2(V2{N, N}, s2, kap[rc][q2]);
                    if (SPLIT) {
                        jac[rc][q2] = Pair<Tp>::fma2(V2{A, A}, s2, jac[rc][q2]);
                    } else {
                        jac[rc][q2].x = fma(A * s2.x, cont_exp(-th[rc] * d[2 * q2]), jac[rc][q2].x);
                        jac[rc][q2].y = fma(A * s2.y, cont_exp(-th[rc] * d[2 * q2 + 1]), jac[rc][q2].y);
                    }
                }
            }
        }
    }

    // free-free, the Planck factor, and the update of kappa and j
    Tp s3[PP], s4[PP];
#pragma unroll
    for (int q = 0; q < PP; ++q) {
        s3[q] = pts[q * 4 + 2];
        s4[q] = pts[q * 4 + 3];
    }
    // per model: the block's D rows, the tile's D intervals and the free-free
    // factors staged in shared memory; kappa_ff joins the level sums
    Tp* sD = &sg[0][0];                                   // [CB][CONT_DMAX], the table rows are consumed
    Tp* sDw = sD + CB * CONT_DMAX;                        // [W]
    Tp* sF = sDw + W;                                     // [CB][2]
    int* sDj = reinterpret_cast<int*>(sF + 2 * CB);       // [W]
    const Tp* ffp = static_cast<const Tp*>(a.ff);
    const Tp* Dr = static_cast<const Tp*>(a.Drow);
    const Tp* Dw = static_cast<const Tp*>(a.Dw);
    const int64_t kt = t * W;
    for (int m = 0; m < a.M; ++m) {
        const int nD = a.nDs[m];
        __syncthreads();
        for (int x = threadIdx.x; x < CB * 2; x += blockDim.x) {
            const int64_t c = cb0 + x / 2;
            sF[x] = c < a.C ? ffp[(c * a.M + m) * 2 + (x & 1)] : Tp(0);
        }
        if (nD) {
            for (int x = threadIdx.x; x < CB * nD; x += blockDim.x) {
                const int cc = x / nD, j = x % nD;
                const int64_t c = cb0 + cc;
                sD[cc * CONT_DMAX + j] = c < a.C ? Dr[(c * a.M + m) * CONT_DMAX + j] : Tp(0);
            }
            for (int x = threadIdx.x; x < W; x += blockDim.x) {
                sDj[x] = a.Dj[m * a.n_pad + kt + x];
                sDw[x] = Dw[m * a.n_pad + kt + x];
            }
        }
        __syncthreads();
#pragma unroll
        for (int rc = 0; rc < RC; ++rc) {
            const int cc = w * RC + rc;
            const Tp FA1 = sF[cc * 2], FA2 = sF[cc * 2 + 1];
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                Tp D = Tp(0);
                if (nD) {
                    const int j = sDj[lane * PP + q];
                    const Tp wq = sDw[lane * PP + q];
                    D = (Tp(1) - wq) * sD[cc * CONT_DMAX + j] + wq * sD[cc * CONT_DMAX + j + 1];
                }
                const Tp kf = fma(FA1, s4[q], FA2 * s3[q]) * (Tp(1) + D);
                comp(kap[rc][q / 2], q & 1) += kf;
                // split sums carry e^{-x} at the end; per-term sums already hold it
                Tp& jq = comp(jac[rc][q / 2], q & 1);
                jq = SPLIT ? jq + kf : fma(cont_exp(-th[rc] * u[q]), kf, jq);
            }
        }
    }
    Tp P[PP];
#pragma unroll
    for (int q = 0; q < PP; ++q) P[q] = pts[q * 4 + 1];
    Tp* kout = static_cast<Tp*>(a.kappa);
    Tp* jout = static_cast<Tp*>(a.emis);
    // j = P / (1 - e^{-x}) (split: e^{-x}) sum.  Rows whose lane span is
    // 16-byte aligned and inside the range move as PP-wide vectors; every old
    // value of the warp's cells is loaded before the first store.
    using VP = typename VecOf<Tp, PP>::type;
    const int64_t k0l = kt + lane * PP;
    const bool vec = k0l + PP <= a.nk && (a.ld % PP) == 0 &&
                     ((reinterpret_cast<uintptr_t>(kout) | reinterpret_cast<uintptr_t>(jout)) & 15) == 0;
    Tp ko[RC][PP], jo[RC][PP];
#pragma unroll
    for (int rc = 0; rc < RC; ++rc) {
        const int64_t c = cb0 + w * RC + rc;
        if (vec && c < a.C) {
            const VP kv = *reinterpret_cast<const VP*>(kout + c * a.ld + k0l);
            const VP jv = *reinterpret_cast<const VP*>(jout + c * a.ld + k0l);
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                ko[rc][q] = reinterpret_cast<const Tp*>(&kv)[q];
                jo[rc][q] = reinterpret_cast<const Tp*>(&jv)[q];
            }
        } else {
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                const bool in = c < a.C && k0l + q < a.nk;
                ko[rc][q] = in ? kout[c * a.ld + k0l + q] : Tp(0);
                jo[rc][q] = in ? jout[c * a.ld + k0l + q] : Tp(0);
            }
        }
    }
#pragma unroll
    for (int rc = 0; rc < RC; ++rc) {
        const int64_t c = cb0 + w * RC + rc;
        if (c >= a.C) continue;
#pragma unroll
        for (int q = 0; q < PP; ++q) {
            const Tp e = cont_exp(-th[rc] * u[q]);   // e^{-x}, x = theta u
            Tp den;
            if (sizeof(Tp) == 4) den = Tp(1) - e;
            else den = (Tp)(-expm1(-(double)(th[rc] * u[q])));
            const Tp jq = comp(jac[rc][q / 2], q & 1);
            ko[rc][q] += comp(kap[rc][q / 2], q & 1);
            jo[rc][q] += cont_div(P[q], den) * (SPLIT ? e * jq : jq);
        }
        if (vec) {
            VP kv, jv;
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                reinterpret_cast<Tp*>(&kv)[q] = ko[rc][q];
                reinterpret_cast<Tp*>(&jv)[q] = jo[rc][q];
            }
            *reinterpret_cast<VP*>(kout + c * a.ld + k0l) = kv;
            *reinterpret_cast<VP*>(jout + c * a.ld + k0l) = jv;
        } else {
#pragma unroll
            for (int q = 0; q < PP; ++q)
                if (k0l + q < a.nk) {
                    kout[c * a.ld + k0l + q] = ko[rc][q];
                    jout[c * a.ld + k0l + q] = jo[rc][q];
                }
        }
    }
}

template <typename Tp, int RC, int PP>
__global__ void __launch_bounds__(128, sizeof(Tp) == 4 ? 4 : 3) k_continuum(ContMain a) {
    if (*a.status) return;
    constexpr int W = 32 * PP, CB = 4 * RC;
    __shared__ __align__(16) Tp sg[CONT_LCH][W];
    __shared__ __align__(16) Tp sN[CONT_LCH][CB];
    __shared__ __align__(16) Tp sA[CONT_LCH][CB];
    __shared__ Tp sv[CONT_LCH];
    const int64_t cb0 = (int64_t)blockIdx.x * CB;
    const int ok = threadIdx.x < CB && cb0 + threadIdx.x < a.C ? a.warm[cb0 + threadIdx.x] : 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    {   // the rows read back at the end: toward L2 while the level sums run
        const int64_t k = (int64_t)blockIdx.y * W + lane * PP;
        for (int rc = 0; rc < RC; ++rc) {
            const int64_t c = cb0 + w * RC + rc;
            if (c < a.C && k < a.nk && (lane & 7) == 0) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const Tp*>(a.kappa) + c * a.ld + k));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const Tp*>(a.emis) + c * a.ld + k));
            }
        }
    }
    if (__syncthreads_and(ok))
        cont_block<Tp, RC, PP, true>(a, blockIdx.y, cb0, lane, w, sg, sN, sA, sv);
    else
        cont_block<Tp, RC, PP, false>(a, blockIdx.y, cb0, lane, w, sg, sN, sA, sv);
}

}  // namespace

static size_t cont_need(size_t need, int64_t I, int64_t T, int64_t C, int M, size_t esz) {
    need = arena_need(need, (size_t)I * sizeof(ContLevel));
    need = arena_need(need, (size_t)T * sizeof(int));
    need = arena_need(need, (size_t)(T + 1) * sizeof(int64_t));
    need = arena_need(need, (size_t)I * C * esz);
    need = arena_need(need, (size_t)I * C * esz);
    need = arena_need(need, (size_t)I * C * esz);
    need = arena_need(need, (size_t)C * sizeof(int));
    need = arena_need(need, (size_t)C * esz);
    need = arena_need(need, (size_t)C * M * 2 * esz);
    need = arena_need(need, (size_t)C * M * CONT_DMAX * esz);
    need = arena_need(need, (size_t)T * 128 * 4 * esz);             // pts (W <= 128)
    need = arena_need(need, (size_t)T * 128 * M * sizeof(int));     // Dj
    need = arena_need(need, (size_t)T * 128 * M * esz);             // Dw
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
    Tp* coefA2 = ar.take<Tp>((size_t)I * C);
    int* warm = ar.take<int>(C);
    Tp* theta = ar.take<Tp>(C);
    Tp* ff = ar.take<Tp>((size_t)C * M * 2);
    Tp* Drow = ar.take<Tp>((size_t)C * M * CONT_DMAX);
    const int64_t n_pad = T * W;
    Tp* pts = ar.take<Tp>((size_t)n_pad * 4);
    int* Dj = ar.take<int>((size_t)n_pad * M);
    Tp* Dw = ar.take<Tp>((size_t)n_pad * M);
    cudaStream_t s = ctx->stream;
    cudaError_t e = launch_validate_cells(ctx, cells);
    if (e == cudaSuccess) {
        k_cont_validate<<<M, 128, 0, s>>>(Mh, ctx->d_status);
        k_cont_levels<<<1, RAPRAL_MAX_CONT_LEVELS, 0, s>>>(Mh, g->lam_min, h, lev, ctx->d_status);
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
    size_t need = arena_need(phase1, (size_t)total * esz);
    if (sizeof(Tp) == 4)
        for (int k = 0; k < 3; ++k) need = arena_need(need, (size_t)Mh.node0[M] * sizeof(float));
    if (need + 256 > ctx->ws_bytes) {   // the arena moves: start again in the larger one
        st = ws_reserve(ctx, need + 256);
        if (st) return st;
        return cont_run<Tp, RC, PP>(ctx, Mh, S, cells, g, h, k0, nk, kappa, emis, ld, ph);
    }
    Tp* tab = ar.take<Tp>((size_t)total);
    if (sizeof(Tp) == 4) {
        const int64_t NN = Mh.node0[M];
        float* yf = ar.take<float>(NN);
        float* sf = ar.take<float>(NN);
        float* dxf = ar.take<float>(NN);
        int64_t mx = 0;
        for (int m = 0; m < M; ++m) mx = std::max<int64_t>(mx, Mh.m[m].n_nodes);
        k_cont_nodes32<<<dim3(div_up(mx, 256), M), 256, 0, s>>>(Mh, yf, sf, dxf, ctx->d_status);
        k_cont_sigma32<<<(unsigned)T, 128, 0, s>>>(Mh, lev, n_lev, tab_off, W, g->lam_min, h, k0, nk, yf, sf, dxf,
                                                  reinterpret_cast<float*>(tab), ctx->d_status);
    } else {
        k_cont_sigma<Tp><<<(unsigned)T, 128, 0, s>>>(Mh, lev, n_lev, tab_off, W, g->lam_min, h, k0, nk, tab,
                                                    ctx->d_status);
    }
    k_cont_points<Tp><<<div_up(n_pad, 256), 256, 0, s>>>(Mh, n_pad, g->lam_min, h, k0, ph, pts, Dj, Dw,
                                                         ctx->d_status);
    // split-form limits: |exponents| well inside the type's range (e^88 FP32, e^709 FP64)
    const double lim = sizeof(Tp) == 4 ? 60.0 : 600.0;
    k_cont_coef<Tp><<<(unsigned)C, 128, 0, s>>>(Mh, lev, *cells, S, ph, 1.0 / g->lam_min, lim, coefN, coefA, coefA2,
                                               warm, theta, ff, Drow, ctx->d_status);
    ContMain a;
    a.M = M; a.I = I; a.S = S; a.C = C; a.nk = nk; a.k0 = k0; a.ld = ld;
    a.lam_min = g->lam_min; a.h = h; a.ph = ph;
    a.lev = lev; a.n_lev = n_lev; a.tab_off = tab_off; a.tab = tab;
    a.coefN = coefN; a.coefA = coefA; a.coefA2 = coefA2; a.warm = warm; a.theta = theta; a.ff = ff; a.Drow = Drow;
    for (int m = 0; m < RAPRAL_MAX_CONT_MODELS; ++m) {
        a.nDs[m] = (m < M && Mh.m[m].D) ? Mh.m[m].n_D_sigma : 0;
    }
    a.n_pad = n_pad; a.pts = pts; a.Dj = Dj; a.Dw = Dw;
    a.kappa = kappa; a.emis = emis; a.status = ctx->d_status;
    dim3 grid((unsigned)((C + CB - 1) / CB), (unsigned)T);
    if (ctx->ev_before) cudaEventRecord(ctx->ev_before, s);
    k_continuum<Tp, RC, PP><<<grid, 128, 0, s>>>(a);
    if (ctx->ev_after) cudaEventRecord(ctx->ev_after, s);
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
    if (const char* why = grid_problem(g)) return set_error(ctx, RAPRAL_EINVAL, "%s", why);
    if (!range_in_grid(g, k0, nk)) return set_error(ctx, RAPRAL_EINVAL, "range outside the grid");
    if (ld < nk) return set_error(ctx, RAPRAL_EINVAL, "ld < nk");
    if (n_species < 1 || n_species > RAPRAL_MAX_SPECIES) return set_error(ctx, RAPRAL_EINVAL, "species count");
    if (cells->n_cells < 0 || cells->n_cols < 1 || cells->ne_col < 0 || cells->ne_col >= cells->n_cols)
        return set_error(ctx, RAPRAL_EINVAL, "cell array sizes");
    if (cells->n_cells == 0) return RAPRAL_OK;
    if (!cells->lnpref || !cells->Tve || !cells->n) return set_error(ctx, RAPRAL_EINVAL, "cells need Tve, n, lnpref");
    ContModels Mh{};
    Mh.M = n_models;
    Mh.lev0[0] = 0;
    Mh.node0[0] = 0;
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
        Mh.node0[m + 1] = Mh.node0[m] + c.n_nodes;
        if (Mh.lev0[m + 1] > RAPRAL_MAX_CONT_LEVELS)
            return set_error(ctx, RAPRAL_EINVAL, "more than %d continuum levels", RAPRAL_MAX_CONT_LEVELS);
    }
    Mh.I = Mh.lev0[n_models];
    cudaSetDevice(ctx->device);
    const double h = (g->lam_max - g->lam_min) / (double)(g->n - 1);
    const Phys ph = make_phys(ctx->codata);
    if (precision == RAPRAL_FP64)
        return cont_run<double, 4, 2>(ctx, Mh, n_species, cells, g, h, k0, nk, kappa, emis, ld, ph);
    return cont_run<float, 4, 4>(ctx, Mh, n_species, cells, g, h, k0, nk, kappa, emis, ld, ph);
}
