// Line preparation, spectral-tile binning and the line-by-line sum
// (Sec. 2.2.1 atoms, Sec. 2.2.2 diatomics).
//
// Binning (deterministic, ordered by line index):
//   k_bin_bounds   per line, the tiles its window can touch in any cell of the
//                  request, from a conservative width: lamV <= lamL + lamG
//                  with both widths at their largest over the cells
//   k_bin_count    one block per tile: scan the lines whose centre lies within
//                  the widest window of the tile, count those that reach it
//   scan           exclusive prefix of the counts -> CSR offsets
//   k_bin_fill     same scan, ordered compaction of the line indices
//
// Line sum, FP64: one block per (tile, cell).  Threads own consecutive grid
// points of the tile.  Lines of the tile are processed in batches of
// blockDim: each thread sets up one (line, cell) pair -- populations in log
// space, strengths, Doppler / Stark / Voigt widths, profile normalisation and
// the window -- into shared memory; then every thread evaluates the profile
// of each staged pair at its own points inside that pair's window and
// accumulates kappa and j.  Results are written once, coalesced.  FP32: one
// warp per (tile, cell), described with its kernel below.
//
// Optional per-context parts, each a template flag of the kernels so that the
// default path is unchanged: the full Lorentz width (Stark from the
// ionisation gap, resonance, van der Waals), departure coefficients of
// collisional-radiative levels, and the exact Voigt shape (voigt.cuh) in
// place of Whiting's fit.
#include "rapral_internal.cuh"

// the rational Faddeeva expansion's coefficients (exact Voigt line shape)
__constant__ VoigtCoef c_voigt;

namespace {

__device__ __forceinline__ double voigt_hwhm(double lamL, double lamG) {
    const double d = (lamL - lamG) / (lamL + lamG);
    return (1.0 - 0.18121 * (1.0 - d * d) - (0.023665 * exp(0.6 * d) + 0.00418 * exp(-1.9 * d)) * sin(M_PI * d)) *
           (lamL + lamG);
}

__global__ void k_validate_lines(rapral_lines ln, int32_t S, int* status) {
    int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= ln.n_lines) return;
    const int s = ln.species[l];
    if (s < 0 || s >= S) fail(status, CHK_LINE_SPECIES, l);
    const double lam = ln.lam0[l];
    if (!(lam > 0.0) || !isfinite(lam) || !(ln.lamS0[l] >= 0.0) || !isfinite(ln.lamS0[l]))
        fail(status, CHK_LINE_LAM, l);
    if (!(ln.gu[l] > 0.0) || !(ln.gl[l] > 0.0) || !isfinite(ln.gu[l]) || !isfinite(ln.gl[l]))
        fail(status, CHK_LINE_G, l);
    if (!(ln.A[l] >= 0.0) || !isfinite(ln.A[l])) fail(status, CHK_LINE_A, l);
}

__global__ void k_line_prep(rapral_lines ln, const double* __restrict__ mass, const int32_t* __restrict__ kind,
                            double lam_min, double h, Phys ph, LinePrep* __restrict__ out,
                            LineF32* __restrict__ out32, int* sorted_flag, BroadArgs br, double2* lb,
                            float2* lb32, const int* status) {
    if (*status) return;
    int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= ln.n_lines) return;
    LinePrep p;
    const double lam0 = ln.lam0[l];
    const double lcm = lam0 * 1e-7;
    const double A = ln.A[l];
    const int s = ln.species[l];
    p.lam0 = lam0;
    p.lnAj = log(1e-7 * (ph.h * ph.c / (4.0 * M_PI)) * A / lcm);
    p.lnAk = log(1e4 * A * (lcm * lcm) * (lcm * lcm) / (8.0 * M_PI * ph.c));
    p.lngu = log(ln.gu[l]);
    p.lnAjg = p.lnAj + p.lngu;
    p.lnAkg = p.lnAk + p.lngu;
    p.Eve_u = ln.Eu_el[l] + ln.Eu_v[l];
    p.Er_u = ln.Eu_j[l];
    p.Eve_l = ln.El_el[l] + ln.El_v[l];
    p.Er_l = ln.El_j[l];
    p.dEve = p.Eve_u - p.Eve_l;
    p.dEr = p.Er_u - p.Er_l;
    p.cD = RAPRAL_DOPPLER_HALF * lam0 / sqrt(mass[s]);
    p.lamS0 = ln.lamS0[l];
    const bool atom = kind[s] == 0;
    if ((br.flags & RAPRAL_BROAD_STARK_IONIZE) && atom) {   // Stark coefficient from the ionisation gap
        const double dE = fmax(br.Eion[s] - ln.Eu_el[l], RAPRAL_E_IONIZE_H / 25.0);
        p.lamS0 = 1.69e3 * lam0 * lam0 / pow(dE, 2.623);
    }
    if (lb) {   // per-line factors of the resonance and van der Waals widths
        double cR = 0.0, cW = 0.0;
        if ((br.flags & RAPRAL_BROAD_RESONANCE) && atom && ln.El_el[l] == 0.0 && ln.El_v[l] == 0.0 &&
            ln.El_j[l] == 0.0) {
            const double f = ph.me * ph.c * lcm * lcm / (8.0 * M_PI * M_PI * ph.e * ph.e) * ln.gu[l] / ln.gl[l] * A;
            cR = 4.3e-28 * lam0 * f * sqrt(ln.gl[l] / ln.gu[l]) * lam0 * lam0;
        }
        if ((br.flags & RAPRAL_BROAD_VDW) && atom) cW = lam0 * lam0;
        lb[l] = make_double2(cR, cW);
        lb32[l] = make_float2((float)cR, (float)cW);
    }
    p.tpos = (lam0 - lam_min) / h;
    p.dEve_f = (float)p.dEve;
    p.dEr_f = (float)p.dEr;
    p.cD_f = (float)p.cD;
    p.lamS0_f = (float)p.lamS0;
    const double kcd = rint(p.tpos);
    p.kc = (int32_t)fmin(fmax(kcd, -1e9), 2e9);
    p.delta_f = (float)(p.tpos - (double)p.kc);
    p.species = s;
    p.pad = 0;
    out[l] = p;
    if (out32) {
        LineF32 f;
        f.lnAjg = ff_from(p.lnAjg);
        f.dAkj = ff_from(p.lnAk - p.lnAj);
        f.Eve_u = ff_from(p.Eve_u);
        f.Er_u = ff_from(p.Er_u);
        f.dEve = ff_from(p.dEve);
        f.dEr = ff_from(p.dEr);
        f.cD = p.cD_f;
        f.lamS0 = p.lamS0_f;
        f.delta = p.delta_f;
        f.kc = p.kc;
        f.species = s;
        f.kcf = (float)p.kc;
        out32[l] = f;
    }
    if (l + 1 < ln.n_lines && ln.lam0[l + 1] < lam0) *sorted_flag = 0;
}

// Conservative window per line: lamV <= lamL + lamG (the Voigt fit's factor
// never exceeds 1), both at their largest over the request's cells.
__global__ void k_bin_bounds(const LinePrep* __restrict__ lp, int64_t L, const unsigned long long* __restrict__ dmax,
                             double h, int64_t k0, int64_t nk, int tile_w, int2* __restrict__ line_tiles,
                             unsigned long long* wmax, const double2* lb, const int* status) {
    if (*status) return;
    int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= L) return;
    const double sqrtTmax = __longlong_as_double((long long)dmax[0]);
    const double stcmax = __longlong_as_double((long long)dmax[1]);
    const LinePrep p = lp[l];
    const double lamG = p.cD * sqrtTmax;
    double lamL = RAPRAL_LAM_NATURAL + p.lamS0 * stcmax;
    if (lb) {   // resonance / van der Waals terms at their largest over the cells
        const double2 c = lb[l];
        lamL += c.x * __longlong_as_double((long long)dmax[2 + 2 * p.species]) +
                c.y * __longlong_as_double((long long)dmax[3 + 2 * p.species]);
    }
    const double w = RAPRAL_WINDOW * (lamL + lamG) * (1.0 + 1e-9) / h + 2.0;   // grid points
    atomicMax(wmax, (unsigned long long)__double_as_longlong(w));
    const double lo = fmax(ceil(p.tpos - w), (double)k0);
    const double hi = fmin(floor(p.tpos + w), (double)(k0 + nk - 1));
    int2 t;
    if (lo > hi) {
        t.x = 1; t.y = 0;
    } else {
        t.x = (int)(((int64_t)lo - k0) / tile_w);
        t.y = (int)(((int64_t)hi - k0) / tile_w);
    }
    line_tiles[l] = t;
}

// Lines whose centre can reach tile t: lam0 within the widest window of the
// tile's wavelength span (binary search when lam0 is sorted, else all).
__device__ void tile_candidates(const double* lam0, int64_t L, int sorted, double wmax, double lam_min, double h,
                                int64_t kt0, int64_t kt1, int64_t* b0, int64_t* b1) {
    if (!sorted) { *b0 = 0; *b1 = L; return; }
    const double lo = lam_min + ((double)kt0 - wmax - 2.0) * h;
    const double hi = lam_min + ((double)kt1 + wmax + 2.0) * h;
    int64_t a = 0, b = L;
    while (a < b) { int64_t m = (a + b) >> 1; if (lam0[m] < lo) a = m + 1; else b = m; }
    *b0 = a;
    b = L;
    while (a < b) { int64_t m = (a + b) >> 1; if (lam0[m] <= hi) a = m + 1; else b = m; }
    *b1 = a;
}

__global__ void __launch_bounds__(256) k_bin_count(const double* __restrict__ lam0, int64_t L,
                                                   const int2* __restrict__ line_tiles, const int* sorted_flag,
                                                   const unsigned long long* wmaxp, double lam_min, double h,
                                                   int64_t k0, int64_t nk, int tile_w, int* __restrict__ counts,
                                                   const int* status) {
    if (*status) return;
    const int t = blockIdx.x;
    const int64_t kt0 = k0 + (int64_t)t * tile_w;
    const int64_t kt1 = min(kt0 + tile_w, k0 + nk) - 1;
    int64_t b0, b1;
    tile_candidates(lam0, L, *sorted_flag, __longlong_as_double((long long)*wmaxp), lam_min, h, kt0, kt1, &b0, &b1);
    int cnt = 0;
    for (int64_t l = b0 + threadIdx.x; l < b1; l += blockDim.x) {
        const int2 r = line_tiles[l];
        cnt += (r.x <= t && t <= r.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    __shared__ int ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i];
        counts[t] = s;
    }
}

__global__ void __launch_bounds__(256) k_bin_fill(const double* __restrict__ lam0, int64_t L,
                                                  const int2* __restrict__ line_tiles, const int* sorted_flag,
                                                  const unsigned long long* wmaxp, double lam_min, double h,
                                                  int64_t k0, int64_t nk, int tile_w, const int* __restrict__ off,
                                                  int* __restrict__ out, const int* status) {
    if (*status) return;
    const int t = blockIdx.x;
    const int64_t kt0 = k0 + (int64_t)t * tile_w;
    const int64_t kt1 = min(kt0 + tile_w, k0 + nk) - 1;
    int64_t b0, b1;
    tile_candidates(lam0, L, *sorted_flag, __longlong_as_double((long long)*wmaxp), lam_min, h, kt0, kt1, &b0, &b1);
    __shared__ int wsum[8];
    __shared__ int base_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int base = off[t];
    for (int64_t r0 = b0; r0 < b1; r0 += blockDim.x) {
        const int64_t l = r0 + threadIdx.x;
        bool in = false;
        if (l < b1) { const int2 r = line_tiles[l]; in = (r.x <= t && t <= r.y); }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int i = 0; i < nw; ++i) { int v = wsum[i]; wsum[i] = s; s += v; }
            base_s = s;
        }
        __syncthreads();
        if (in) out[base + wsum[warp] + __popc(m & ((1u << lane) - 1u))] = (int)l;
        base += base_s;
        __syncthreads();
    }
}

// Exclusive scan of the per-tile line counts into the int32 offsets of the
// tile lists, carried in int64 so that a total beyond 2^31 - 1 is seen:
// total[0] receives the exact sum (offsets past 2^31 - 1 wrap, and the
// callers refuse such a plan before the lists are filled).  Single block.
__global__ void __launch_bounds__(1024) k_scan_counts(int* data, int64_t n, long long* total) {
    __shared__ long long part[32];
    __shared__ long long carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c0 = 0; c0 < n; c0 += blockDim.x) {
        const int64_t i = c0 + threadIdx.x;
        const long long v = (i < n) ? (long long)data[i] : 0LL;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) part[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long p = (lane < (int)(blockDim.x >> 5)) ? part[lane] : 0LL;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p += y;
            }
            part[lane] = p;
        }
        __syncthreads();
        const long long carry = carry_s;
        const long long incl = x + (warp > 0 ? part[warp - 1] : 0LL);
        if (i < n) data[i] = (int)(unsigned)(unsigned long long)(carry + incl - v);
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_s = carry + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        data[n] = (int)(unsigned)(unsigned long long)carry_s;
        *total = carry_s;
    }
}

// Single-block exclusive scan over n entries; data[n] receives the total.
template <class T>
__global__ void __launch_bounds__(1024) k_scan(T* data, int64_t n) {
    __shared__ T part[32];
    __shared__ T carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c0 = 0; c0 < n; c0 += blockDim.x) {
        const int64_t i = c0 + threadIdx.x;
        T v = (i < n) ? data[i] : T(0);
        T x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) part[warp] = x;
        __syncthreads();
        if (warp == 0) {
            T p = (lane < (int)(blockDim.x >> 5)) ? part[lane] : T(0);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                T y = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p += y;
            }
            part[lane] = p;
        }
        __syncthreads();
        const T carry = carry_s;
        const T incl = x + (warp > 0 ? part[warp - 1] : T(0));
        if (i < n) data[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_s = carry + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) data[n] = carry_s;
}

// ------------------------------------------------------------ line sum FP64

// Block-wide sum of the per-thread work counters, one atomic per counter.
__device__ void block_count(unsigned long long* stats, int64_t ev, int64_t g, int64_t c, int64_t p) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
        g += __shfl_xor_sync(0xffffffffu, g, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
        p += __shfl_xor_sync(0xffffffffu, p, o);
    }
    if ((threadIdx.x & 31) == 0 && p > 0) {   // one atomic set per warp
        atomicAdd(&stats[0], (unsigned long long)ev);
        atomicAdd(&stats[1], (unsigned long long)g);
        atomicAdd(&stats[2], (unsigned long long)c);
        atomicAdd(&stats[3], (unsigned long long)p);
    }
}

struct __align__(16) PairF64 {
    double lam0, w100, inv2V, r, omr, c16, aj, ak;
    double ug2, ue2;   // u^2 past which the Gaussian / correction exponential is left out
    int klo, khi, pad0, pad1;
};

// Exponentials of the Whiting bracket left out where they are below 1e-17 of
// its Lorentz part (at least r / (2 (1 + 4u^2)); the part is positive for
// every u), far below the FP64 rounding of the sum:
//   Gaussian (1 - r) e^{-2.772 x}, x = u^2: from the x with
//     2.772 x - ln(1 + 4x) = ln(2e17 (1 - r) / r), by fixed-point iteration
//     from below plus a margin, capped at the FP64 underflow (2.772 x = 745.5);
//   correction c16 e^{-0.4 x^1.125}: c16 / r <= 0.016 for every r, so one
//     bound serves all pairs, x = 65.14 (0.4 x^1.125 - ln(1 + 4x) = ln(3.2e15)).
constexpr double SKIP_CORR_U2 = 65.14;
__device__ double skip_gauss_u2(double omr, double r) {
    const double under = 745.5 / 2.772;
    if (!(omr > 0.0)) return 0.0;
    if (!(r > 0.0)) return under;
    const double K = log(2e17 * omr / r);
    double x = fmax(K, 0.0) / 2.772;
    for (int i = 0; i < 4; ++i) x = fmax(K + log1p(4.0 * x), 0.0) / 2.772;
    return fmin(1.05 * x + 0.5, under);
}

// Lorentz HWHM of line l in cell c in FP64: natural + Stark, plus the
// optional resonance and van der Waals terms.
__device__ __forceinline__ double lorentz64(const LineSumArgs& a, const LinePrep& L, const CellPrep& cp, int64_t l,
                                            int64_t c) {
    double lamL = RAPRAL_LAM_NATURAL + L.lamS0 * cp.stc;
    if (a.lb) {
        const double2 x = a.lb[l], y = a.cb[c * a.S + L.species];
        lamL += x.x * y.x;
        lamL += x.y * y.y;
    }
    return lamL;
}

template <int PPT, bool VG = false>
__global__ void __launch_bounds__(128) k_line_sum_f64(LineSumArgs a) {
    if (*a.status) return;
    const int W = 128 * PPT;
    const int t = blockIdx.y;
    const int64_t c = blockIdx.x;
    const int64_t kt0 = a.k0 + (int64_t)t * W;
    const int64_t kend = min(kt0 + W, a.k0 + a.nk);   // exclusive
    const int64_t kp = kt0 + (int64_t)threadIdx.x * PPT;
    __shared__ PairF64 pr[128];
    int64_t n_ev = 0, n_g = 0, n_c = 0, n_pairs = 0;
    double acck[PPT], accj[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) { acck[i] = 0.0; accj[i] = 0.0; }
    const CellPrep cp = a.cp[c];
    const int beg = a.tile_off[t], end = a.tile_off[t + 1];
    for (int b = beg; b < end; b += 128) {
        const int nb = min(128, end - b);
        if ((int)threadIdx.x < nb) {
            const int l = a.tile_lines[b + threadIdx.x];
            const LinePrep L = a.lp[l];
            PairF64 P;
            P.klo = 1; P.khi = 0;
            double du = 0.0, dl = 0.0;   // departure coefficients (ln b) of the line's levels
            if (a.dep_lnb) {
                const double* row = a.dep_lnb + (c * a.S + L.species) * a.dep_nlev;
                const int iu = a.dep_u[l], il = a.dep_l[l];
                if (iu >= 0) du = row[iu];
                if (il >= 0) dl = row[il];
            }
            const double lnNu = a.lnpref[c * a.S + L.species] + L.lngu - (L.Eve_u * cp.bve + L.Er_u * cp.btr) + du;
            const double Sj = exp(L.lnAj + lnNu);
            if (Sj > 0.0) {
                const double x = L.dEve * cp.bve + L.dEr * cp.btr + (dl - du);
                const double Sk = exp(L.lnAk + lnNu) * expm1(x);
                const double lamG = L.cD * cp.sqrtT;
                const double lamL = lorentz64(a, L, cp, l, c);
                const double lamV = voigt_hwhm(lamL, lamG);
                double r = lamL / lamV;
                double pre = 1e3 / (2.0 * lamV * (1.065 + 0.447 * r + 0.058 * r * r));
                P.lam0 = L.lam0;
                P.w100 = RAPRAL_WINDOW * lamV;
                P.inv2V = 0.5 / lamV;
                if (VG) {   // exact Voigt: x = dlam / (sigma sqrt 2) = dlam sqrt(ln 2) / lamG, y = lamL sqrt(ln 2) / lamG
                    P.inv2V = 0.83255461115769775635 / lamG;
                    r = lamL * P.inv2V;
                    pre = 1e3 * 0.46971863934982566689 / lamG;   // 1e3 / (sigma sqrt(2 pi))
                }
                P.r = r;
                P.omr = 1.0 - r;
                P.c16 = 0.016 * r * (1.0 - r);
                if (!VG) {
                    P.ug2 = skip_gauss_u2(P.omr, r);
                    P.ue2 = P.c16 > 0.0 ? SKIP_CORR_U2 : 0.0;
                }
                P.aj = Sj * pre;
                P.ak = Sk * pre;
                const double lo = ceil((L.lam0 - P.w100 - a.lam_min) / a.h) - 1.0;
                const double hi = floor((L.lam0 + P.w100 - a.lam_min) / a.h) + 1.0;
                P.klo = (int)fmax(lo, (double)kt0);
                P.khi = (int)fmin(hi, (double)(kend - 1));
                if (P.klo <= P.khi) {
                    // counters: candidate points (the exact window is tested per point), and
                    // those where the two exponentials are above the FP64 underflow limit
                    const double kcen = L.tpos;
                    const double hg = 16.4 * 2.0 * lamV / a.h, hc = 28.4 * 2.0 * lamV / a.h;   // 2.772u^2, 0.4u^2.25 < 745.5
                    n_ev += min((int64_t)P.khi, (int64_t)floor(kcen + RAPRAL_WINDOW * lamV / a.h)) -
                            max((int64_t)P.klo, (int64_t)ceil(kcen - RAPRAL_WINDOW * lamV / a.h)) + 1;
                    n_g += max((int64_t)0, min((int64_t)P.khi, (int64_t)floor(kcen + hg)) -
                                               max((int64_t)P.klo, (int64_t)ceil(kcen - hg)) + 1);
                    n_c += max((int64_t)0, min((int64_t)P.khi, (int64_t)floor(kcen + hc)) -
                                               max((int64_t)P.klo, (int64_t)ceil(kcen - hc)) + 1);
                    ++n_pairs;
                }
            }
            pr[threadIdx.x] = P;
        }
        __syncthreads();
        for (int q = 0; q < nb; ++q) {
            const int klo = pr[q].klo, khi = pr[q].khi;
            if (khi < kp || klo > kp + PPT - 1) continue;
            const PairF64 P = pr[q];
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                const int64_t k = kp + i;
                if (k < klo || k > khi) continue;
                const double lk = __dadd_rn(a.lam_min, __dmul_rn((double)k, a.h));
                const double dl = fabs(lk - P.lam0);
                if (!(dl <= P.w100)) continue;
                if (VG) {
                    const double br = voigt_re<double>(c_voigt, dl * P.inv2V, P.r);
                    accj[i] += P.aj * br;
                    acck[i] += P.ak * br;
                    continue;
                }
                const double u = dl * P.inv2V;
                const double u2 = u * u;
                const double g = u2 < P.ug2 ? exp(-2.772 * u2) : 0.0;
                const double v = u2 * sqrt(sqrt(u));
                const double e2 = u2 < P.ue2 ? exp(-0.4 * v) : 0.0;
                const double qd = 1.0 + 4.0 * u2;
                const double pd = 1.0 + 0.1 * v;
                const double br = P.omr * g + (P.r * pd - P.c16 * qd) / (qd * pd) + P.c16 * e2;
                accj[i] += P.aj * br;
                acck[i] += P.ak * br;
            }
        }
        __syncthreads();
    }
    block_count(a.stats, n_ev, n_g, n_c, n_pairs);
    double* K = reinterpret_cast<double*>(a.kappa) + c * a.ld - a.k0;
    double* J = reinterpret_cast<double*>(a.emis) + c * a.ld - a.k0;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int64_t k = kp + i;
        if (k < kend) { __stcs(K + k, acck[i]); __stcs(J + k, accj[i]); }   // streaming, as the FP32 path
    }
}


// ------------------------------------------------------ line sum FP32 (chosen)
//
// Set-up per (line, cell): log-space populations and strengths in FP64,
// exponentials of the reduced log (integer power of two times 2^f, f in
// [0, 1)) in FP32; widths, Voigt HWHM and profile constants in FP32.  The
// window [klo, khi] is found in grid units in FP32 and certified: when an edge
// lies within the FP32 error bound of a grid point, both edges are decided
// again with the FP64 Voigt width and the literal test |lam_k - lam0| <=
// 100 lamV, so every (line, point) inclusion matches the FP64 decision.
// Per point: u = |(k - kc) s - u0| (s = h / 2lamV), the Whiting bracket with
// MUFU ex2 / rsqrt / rcp, terms that underflow FP32 skipped, and Kahan
// compensated sums of kappa and j over the tile's lines.

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ bool in_window64(int64_t k, double lam_min, double h, double lam0, double w100) {
    const double lk = __dadd_rn(lam_min, __dmul_rn((double)k, h));
    return fabs(lk - lam0) <= w100;
}

// Exact edges near the FP32 estimates (the estimate is within a fraction of a
// grid point of the truth).
__device__ __noinline__ void exact_edges(const LinePrep* __restrict__ Lp, const CellPrep* __restrict__ cpp,
                                         const double2* lb, const double2* cbrow, double lam_min, double h,
                                         int64_t* klo, int64_t* khi) {
    const LinePrep& L = *Lp;
    const CellPrep& cp = *cpp;
    const double lamG = L.cD * cp.sqrtT;
    double lamL = RAPRAL_LAM_NATURAL + L.lamS0 * cp.stc;
    if (lb) {   // the optional resonance / van der Waals terms, as lorentz64
        const double2 x = *lb, y = cbrow[L.species];
        lamL += x.x * y.x;
        lamL += x.y * y.y;
    }
    const double w100 = RAPRAL_WINDOW * voigt_hwhm(lamL, lamG);
    int64_t k = *khi + 2;
    while (k > *khi - 3 && !in_window64(k, lam_min, h, L.lam0, w100)) --k;
    const int64_t hi = k;
    k = *klo - 2;
    while (k < *klo + 3 && !in_window64(k, lam_min, h, L.lam0, w100)) ++k;
    *klo = k;
    *khi = hi;
}

// Conversion-free helpers for the FP32 set-up.  On GB300 float/integer
// conversions and roundings share the narrow FP64 pipe, so the set-up keeps
// to FMA-pipe arithmetic and MUFU ex2 / rcp.

// Nearest integer of |x| < 2^22 (adding and removing 1.5 * 2^23).
__device__ __forceinline__ float round_near(float x) { return (x + 12582912.0f) - 12582912.0f; }
__device__ __forceinline__ float floor_f(float x) { const float n = round_near(x); return n > x ? n - 1.0f : n; }
__device__ __forceinline__ float ceil_f(float x) { const float n = round_near(x); return n < x ? n + 1.0f : n; }

// e^y for y = hi + lo: t = y log2(e) (float-float), t = n + f with n the
// nearest integer, 2^f and 2^n by MUFU ex2.
__device__ __forceinline__ float exp_ff(float2 y) {
    const float2 t = ff_mul(y, make_float2(1.4426950216293335f, 1.925963033500011e-08f));
    const float n = round_near(t.x);
    return ex2_approx((t.x - n) + t.y) * ex2_approx(n);
}

// e^z - 1 for z <= 0: Taylor series through z^9 for z > -1/2 (error below
// 3e-10 relative), else 2^(z log2 e) - 1 (|result| >= 0.39).
__device__ __forceinline__ float expm1_neg(float z) {
    if (z > -0.5f) {
        float p = 1.0f / 362880.0f;
        p = fmaf(p, z, 1.0f / 40320.0f);
        p = fmaf(p, z, 1.0f / 5040.0f);
        p = fmaf(p, z, 1.0f / 720.0f);
        p = fmaf(p, z, 1.0f / 120.0f);
        p = fmaf(p, z, 1.0f / 24.0f);
        p = fmaf(p, z, 1.0f / 6.0f);
        p = fmaf(p, z, 0.5f);
        p = fmaf(p, z, 1.0f);
        return p * z;
    }
    return ex2_approx(z * 1.44269504f) - 1.0f;
}

// sin(pi d) for |d| <= 1: sin(pi a) = sin(pi (1 - a)) maps |d| to [0, 1/2],
// then the Taylor series of sin(pi x) through x^13 (error below 1e-9).
__device__ __forceinline__ float sinpi_series(float d) {
    const float a = fabsf(d);
    const float x = a > 0.5f ? 1.0f - a : a;
    const float z = x * x;
    float p = 4.663027939386666e-4f;
    p = fmaf(p, z, -7.37043097615242e-3f);
    p = fmaf(p, z, 8.214588463306427e-2f);
    p = fmaf(p, z, -0.5992645025253296f);
    p = fmaf(p, z, 2.550163984298706f);
    p = fmaf(p, z, -5.167712688446045f);
    p = fmaf(p, z, 3.1415927410125732f);
    return copysignf(x * p, d);
}

// One (line, cell) pair set up for a warp's tile [kt0, kt0 + TW): window
// offsets inside the tile (as floats), u at the tile's first point, profile
// constants, and whether every point of the window part in the tile lies in
// the far wings (|u| > 11, where both exponentials are zero in FP32) or past
// the Gaussian core (|u| > 5.62).  Everything a warp needs per pair is
// computed here, by one lane per pair.
// Bracket modes: both exponentials; the Gaussian core zero in FP32 over the
// span (|u| > 5.62, 2.772 u^2 log2(e) > 126); both zero (|u| > 11, also
// 0.4 u^2.25 log2(e) > 126).  Dropping a term that ex2 flushes to zero does
// not change a sum.
enum { BR_NEAR = 0, BR_MID = 1, BR_FAR = 2 };

struct PairF32 {
    float lo, hi;     // window part inside the tile, offsets from kt0
    float ub, ub_lo;  // signed u at kt0, (kt0 - kc) s - u0, as a float-float pair
    float s;          // h / (2 lamV): step of u per grid point
    float r, aj, ak;
    int mode;         // BR_NEAR, BR_MID or BR_FAR over the window part in the tile
};

// FL: bit 0 the optional Lorentz terms, bit 1 the departure coefficients.
template <int FL>
__device__ __forceinline__ bool setup_pair_f32(const LineSumArgs& a, const LineF32& L, const CellPrep& cp, float2 lp,
                                               float2 cb, int line, int64_t c, float hf, float inv_hf, int kt0,
                                               float kt0f, float kt1f, bool count, PairF32* P, int64_t* cnt) {
    constexpr bool BR = (FL & 1) != 0, DEP = (FL & 2) != 0, VG = (FL & 4) != 0;
    if (!(lp.x > -INFINITY)) return false;
    // widths first: most candidates of a tile list miss the tile in a given cell
    const float lamG = L.cD * cp.sqrtT_f;
    float lamL = (float)RAPRAL_LAM_NATURAL + L.lamS0 * cp.stc_f;
    if (BR) {   // resonance / van der Waals terms: c_R N_0 + c_W W
        const float2 x = a.lb32[line];
        lamL = fmaf(x.y, cb.y, fmaf(x.x, cb.x, lamL));
    }
    const float sum = lamL + lamG;
    {   // lamV <= lamL + lamG: cheap rejection before the Voigt fit
        const float wmax = (float)RAPRAL_WINDOW * sum * inv_hf * 1.0001f + 1.0f;
        if (kt1f - L.kcf < L.delta - wmax || kt0f - L.kcf > L.delta + wmax) return false;
    }
    const float d = (lamL - lamG) * rcp_approx(sum);
    const float F = 1.0f - 0.18121f * (1.0f - d * d) -
                    (0.023665f * ex2_approx(0.6f * 1.44269504f * d) + 0.00418f * ex2_approx(-1.9f * 1.44269504f * d)) *
                        sinpi_series(d);
    const float lamV = F * sum;
    const float wpts = (float)RAPRAL_WINDOW * lamV * inv_hf;
    const float hi = L.delta + wpts, lo = L.delta - wpts;
    const float fhi = floor_f(hi), clo = ceil_f(lo);
    // window in offsets from kt0 (exact: integers below 2^24)
    float lo_rel = L.kcf + clo - kt0f, hi_rel = L.kcf + fhi - kt0f;
    // Certification.  The FP32 edge positions are within 1.2e-6 wpts + 6e-8
    // grid units of the exact ones (lamV to 9e-7 relative through widths,
    // the Voigt fit, ex2 and the sin series; wpts and the sums to a few more
    // roundings).  Only an edge that lies inside this tile and within m of a
    // grid point is decided again in FP64.
    // (with the optional terms lamL carries two more roundings: a wider margin)
    const float m = (BR ? 2e-6f : 1.5e-6f) * wpts + 1e-6f;
    const float span = kt1f - kt0f;
    const bool lo_in = lo_rel >= -1.0f && lo_rel <= span + 1.0f;
    const bool hi_in = hi_rel >= -1.0f && hi_rel <= span + 1.0f;
    if ((hi_in && (hi - fhi < m || fhi + 1.0f - hi < m)) || (lo_in && (clo - lo < m || lo - (clo - 1.0f) < m))) {
        int64_t klo = (int64_t)L.kc + (int64_t)clo, khi = (int64_t)L.kc + (int64_t)fhi;
        exact_edges(a.lp + line, a.cp + c, BR ? a.lb + line : nullptr, BR ? a.cb + c * a.S : nullptr, a.lam_min, a.h,
                    &klo, &khi);
        lo_rel = (float)(klo - kt0);
        hi_rel = (float)(khi - kt0);
    }
    lo_rel = fmaxf(lo_rel, 0.0f);
    hi_rel = fminf(hi_rel, kt1f - kt0f);
    if (lo_rel > hi_rel) return false;
    // strengths: ln S_j = lnAj + ln g_u + ln(N_s/Z_s) - (E_el + E_V)_u c2/T_ve - E_J,u c2/T_tr
    // and x = ln(N_l g_u / (N_u g_l)) = dE_ve c2/T_ve + dE_J c2/T_tr, in float-float
    float2 yj = ff_add(ff_add(L.lnAjg, lp), ff_neg(ff_add(ff_mul(L.Eve_u, cp.bve_ff), ff_mul(L.Er_u, cp.btr_ff))));
    float2 x = ff_add(ff_mul(L.dEve, cp.bve_ff), ff_mul(L.dEr, cp.btr_ff));
    if (DEP) {   // departure coefficients: ln N_u += ln b_u, x += ln b_l - ln b_u
        const int iu = a.dep_u[line], il = a.dep_l[line];
        if (iu >= 0 || il >= 0) {
            const double* row = a.dep_lnb + ((int64_t)c * a.S + L.species) * a.dep_nlev;
            const double du = iu >= 0 ? row[iu] : 0.0, dl = il >= 0 ? row[il] : 0.0;
            yj = ff_add(yj, ff_from(du));
            x = ff_add(x, ff_from(dl - du));
        }
    }
    const float Sj = exp_ff(yj);
    float2 yk = ff_add(yj, L.dAkj);
    float fk;
    if (x.x >= 0.0f) {           // kappa0 = e^{lnAk + ln N_l g_u/g_l} (1 - e^{-x})
        yk = ff_add(yk, x);
        fk = -expm1_neg(-x.x);
    } else {                     // kappa0 = e^{lnAk + ln N_u} (e^{x} - 1)
        fk = expm1_neg(x.x);
    }
    const float Sk = exp_ff(yk) * fk;
    if (!(Sj > 0.0f) && Sk == 0.0f) return false;
    const float iv = rcp_approx(lamV);
    float r = lamL * iv;
    float pre = 1e3f * 0.5f * iv * rcp_approx(1.065f + 0.447f * r + 0.058f * r * r);
    float s = 0.5f * hf * iv;
    if (VG) {   // exact Voigt: u is x = dlam sqrt(ln 2) / lamG, r is y, pre 1e3 / (sigma sqrt(2 pi))
        const float ig = rcp_approx(lamG);
        r = 0.83255461f * lamL * ig;
        pre = 1e3f * 0.46971864f * ig;
        s = 0.83255461f * hf * ig;
    }
    const float u0 = L.delta * s;                    // u of the centre's offset from kc
    {   // signed u at kt0 without rounding loss: (kt0 - kc) is exact, its
        // product with s and the sum with -u0 are split into hi + lo
        const float dk = kt0f - L.kcf;
        const float p = dk * s;
        const float pe = fmaf(dk, s, -p);
        const float uh = p - u0;
        const float bb = uh - p;
        const float e = (p - (uh - bb)) + (-u0 - bb);
        P->ub = uh;
        P->ub_lo = e + pe;
    }
    // smallest |u| over the evaluated part of the tile
    const float ua = fmaf(lo_rel, s, P->ub), ue = fmaf(hi_rel, s, P->ub);
    const float umin = (ua > 0.0f) ? ua : (ue < 0.0f ? -ue : 0.0f);
    P->lo = lo_rel;
    P->hi = hi_rel;
    P->s = s;
    P->r = r;
    P->mode = umin > 11.0f ? BR_FAR : ((!VG && umin > 5.62f) ? BR_MID : BR_NEAR);
    P->aj = Sj * pre;
    P->ak = Sk * pre;
    if (count) {
        // work counters: points in the window; those where the Gaussian core and
        // the exponential correction are above the FP32 underflow limits
        const int64_t klo = kt0 + (int64_t)lo_rel, khi = kt0 + (int64_t)hi_rel;
        cnt[0] += khi - klo + 1;
        const float kcen = L.kcf + L.delta;
        const float hg = 5.6125f / s, hc = 10.95f / s;   // u^2 < 31.5, u^2.25 < 218
        cnt[1] += max((int64_t)0, min(khi, (int64_t)floorf(kcen + hg)) - max(klo, (int64_t)ceilf(kcen - hg)) + 1);
        cnt[2] += max((int64_t)0, min(khi, (int64_t)floorf(kcen + hc)) - max(klo, (int64_t)ceilf(kcen - hc)) + 1);
        cnt[3] += 1;
    }
    return true;
}

// One Whiting evaluation, bracket only (the factor 1e3 / (2 lamV (1.065 +
// 0.447 r + 0.058 r^2)) is folded into aj, ak).  Near the line centre both
// exponentials are kept; BR_MID drops the Gaussian core and BR_FAR both
// where they are zero in FP32 over the whole span being evaluated.
template <int M>
__device__ __forceinline__ float whiting_bracket(float u, float r, float omr, float c16) {
    const float u2 = u * u;
    const float v = u2 * rsqrt_approx(rsqrt_approx(u));                      // u^2.25
    const float q4 = fmaf(4.0f, u2, 1.0f);
    const float p1 = fmaf(0.1f, v, 1.0f);
    const float rd = rcp_approx(q4 * p1);
    const float num = fmaf(r, p1, -c16 * q4);                                // r(1+0.1v) - c16(1+4u^2)
    if (M == BR_FAR) return num * rd;
    // past u^2 = 31.5 and v = 218 the approximate ex2 returns 0 (flushed) or
    // below 1.5e-38, so neither exponential needs a guard
    const float e2 = ex2_approx(-0.5770780f * v);    // e^{-0.4 v}
    if (M == BR_MID) return fmaf(num, rd, c16 * e2);
    const float g = ex2_approx(-3.99915f * u2);      // e^{-2.772 u^2}
    return fmaf(omr, g, fmaf(num, rd, c16 * e2));
}

// Kahan step: (s, c) += x.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// One pair over the lane's points k = lane + 32 i of the tile: runs of 32
// points outside the window part [lo, hi] are skipped (the test is the same
// for the whole warp); in the others each lane adds its point if it lies in
// the window.
template <int PPT, int M>
__device__ __forceinline__ void sweep_pair(float lo, float hi, float lanef, float s, float ub, float ub_lo, float r,
                                           float omr, float c16, float aj, float ak, float (&bj)[PPT],
                                           float (&bk)[PPT]) {
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const float p0 = 32.0f * i;
        if (p0 + 31.0f < lo || p0 > hi) continue;
        const float k = lanef + p0;
        // signed u at point k: one rounding of k s + ub (exact product), then
        // the low part; relative to u itself, so the Gaussian core keeps FP32
        // accuracy however far the tile start lies from the line centre
        const float br = whiting_bracket<M>(fabsf(fmaf(k, s, ub) + ub_lo), r, omr, c16);
        if (k >= lo && k <= hi) {   // predicated update: lanes outside the window part add nothing
            bj[i] = fmaf(aj, br, bj[i]);
            bk[i] = fmaf(ak, br, bk[i]);
        }
    }
}

// One pair whose window covers every point of the tile: no point needs the
// window test, so the brackets of runs i and i + 1 are evaluated together in
// packed FP32 (two results per instruction; the MUFU operations stay
// scalar).  Operations and roundings are those of whiting_bracket and of the
// predicated update, so the sums are bitwise the same as sweep_pair's.
template <int PPT, int M>
__device__ __forceinline__ void sweep_pair_full(float lanef, float s, float ub, float ub_lo, float r, float omr,
                                                float c16, float aj, float ak, float (&bj)[PPT], float (&bk)[PPT]) {
    static_assert(PPT % 2 == 0, "runs are taken two at a time");
    const float2 s2 = make_float2(s, s), ub2 = make_float2(ub, ub), ubl2 = make_float2(ub_lo, ub_lo);
    const float2 one = make_float2(1.0f, 1.0f), four = make_float2(4.0f, 4.0f), tenth = make_float2(0.1f, 0.1f);
    const float2 r2 = make_float2(r, r), nc16 = make_float2(-c16, -c16);
    const float2 aj2 = make_float2(aj, aj), ak2 = make_float2(ak, ak);
#pragma unroll
    for (int i = 0; i < PPT; i += 2) {
        const float2 k = make_float2(lanef + 32.0f * i, lanef + 32.0f * (i + 1));
        const float2 u = __fadd2_rn(__ffma2_rn(k, s2, ub2), ubl2);     // signed u; only |u| and u^2 are used
        const float2 u2 = __fmul2_rn(u, u);
        const float2 q = make_float2(rsqrt_approx(rsqrt_approx(fabsf(u.x))), rsqrt_approx(rsqrt_approx(fabsf(u.y))));
        const float2 v = __fmul2_rn(u2, q);                            // u^2.25
        const float2 q4 = __ffma2_rn(four, u2, one);
        const float2 p1 = __ffma2_rn(tenth, v, one);
        const float2 qp = __fmul2_rn(q4, p1);
        const float2 rd = make_float2(rcp_approx(qp.x), rcp_approx(qp.y));
        const float2 num = __ffma2_rn(r2, p1, __fmul2_rn(nc16, q4));   // r(1+0.1v) - c16(1+4u^2)
        float2 br;
        if (M == BR_FAR) {
            br = __fmul2_rn(num, rd);
        } else {
            const float2 xc = __fmul2_rn(make_float2(-0.5770780f, -0.5770780f), v);
            const float2 e2 = make_float2(ex2_approx(xc.x), ex2_approx(xc.y));    // e^{-0.4 v}
            br = __ffma2_rn(num, rd, __fmul2_rn(make_float2(c16, c16), e2));
            if (M == BR_NEAR) {
                const float2 xg = __fmul2_rn(make_float2(-3.99915f, -3.99915f), u2);
                const float2 g = make_float2(ex2_approx(xg.x), ex2_approx(xg.y));     // e^{-2.772 u^2}
                br = __ffma2_rn(make_float2(omr, omr), g, br);
            }
        }
        const float2 j2 = __ffma2_rn(aj2, br, make_float2(bj[i], bj[i + 1]));
        const float2 k2 = __ffma2_rn(ak2, br, make_float2(bk[i], bk[i + 1]));
        bj[i] = j2.x; bj[i + 1] = j2.y;
        bk[i] = k2.x; bk[i + 1] = k2.y;
    }
}

// The staged pairs q0 .. q1 - 1 of one class: bracket mode M, and whether
// their windows cover the whole tile.
template <int PPT, int M, bool WHOLE>
__device__ __forceinline__ void sweep_class(const float4* sm0, const float4* sm1, int q0, int q1, float lanef,
                                            float (&bj)[PPT], float (&bk)[PPT]) {
    for (int q = q0; q < q1; ++q) {
        const float4 A = sm0[q];   // lo, hi, ub, s
        const float4 B = sm1[q];   // r, ub_lo, aj, ak
        const float r = B.x, omr = 1.0f - r, c16 = 0.016f * r * omr;
        if (WHOLE) sweep_pair_full<PPT, M>(lanef, A.w, A.z, B.y, r, omr, c16, B.z, B.w, bj, bk);
        else sweep_pair<PPT, M>(A.x, A.y, lanef, A.w, A.z, B.y, r, omr, c16, B.z, B.w, bj, bk);
    }
}

// The same sweep with the exact Voigt shape: r is y, u is x.
template <int PPT>
__device__ __forceinline__ void sweep_pair_voigt(const VoigtCoef& vc, float lo, float hi, float lanef, float s, float ub,
                                                 float ub_lo, float y, float aj, float ak, float (&bj)[PPT],
                                                 float (&bk)[PPT]) {
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const float p0 = 32.0f * i;
        if (p0 + 31.0f < lo || p0 > hi) continue;
        const float k = lanef + p0;
        const float br = voigt_re<float>(vc, fmaf(k, s, ub) + ub_lo, y);
        if (k >= lo && k <= hi) {
            bj[i] = fmaf(aj, br, bj[i]);
            bk[i] = fmaf(ak, br, bk[i]);
        }
    }
}

// Warp-level line sum: a warp owns one cell and the TW = 32 PPT points of
// tile t, lane l the points l, l + 32, ..., l + 32 (PPT - 1); it stages 32
// (line, cell) pairs at a time in its own shared-memory slice (one per lane),
// then sweeps them over its points.  With the points interleaved, whether a
// pair's window reaches the i-th run of 32 points is the same for the whole
// warp, so runs outside the window are skipped without a masked evaluation.
// The staged pairs are grouped by class (bracket mode, and whether the
// window covers the whole tile, where two points go per packed FP32
// instruction), one loop per class.  Warps never wait for each other.
template <int PPT, int FL, int PB = 32>
__device__ __forceinline__ void warp_tile_f32(const LineSumArgs& a, int t, int64_t c, float4* sm0, float4* sm1,
                                              float2* smlp, float2* smcb, float4* acc, int lane, int64_t* cnt) {
    constexpr int TW = 32 * PPT;
    const int kt0 = (int)(a.k0 + (int64_t)t * TW);
    const int kt1 = (int)min(a.k0 + (int64_t)(t + 1) * TW, a.k0 + a.nk) - 1;   // inclusive
    const float kt0f = (float)kt0, kt1f = (float)kt1;
    const float lanef = (float)lane;       // lane's first point, relative to kt0
    // compensated sums (Kahan) of the per-batch partial sums, kept in shared
    // memory (acc[i * 32 + lane] = (s_j, c_j, s_k, c_k)); inside a batch of at
    // most PB lines the terms are added plainly in registers (error <= (PB - 1) u
    // of the batch's magnitude, u = 2^-24)
    float bk[PPT], bj[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        bk[i] = bj[i] = 0.0f;
        acc[i * 32 + lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    const CellPrep cp = a.cp[c];
    const float hf = (float)a.h;
    const float inv_hf = (float)(1.0 / a.h);
    const bool count = a.count != 0;
    if (lane < a.S) {   // the cell's ln(N_s / Z_s) as float-float pairs
        const double v = a.lnpref[c * a.S + lane];
        smlp[lane] = v > -INFINITY ? ff_from(v) : make_float2(-INFINITY, 0.0f);
        if (FL & 1) smcb[lane] = a.cb32[c * a.S + lane];   // (N_0, W) of the optional terms
    }
    __syncwarp();
    const int beg = a.tile_off[t], end = a.tile_off[t + 1];
    constexpr int NH = PB / 32;   // staged halves of 32 pairs (one pair a lane each)
    constexpr int NCLS = (FL & 4) ? 1 : 6;
    for (int b = beg; b < end; b += PB) {
        // stage the pairs that reach the tile grouped by class (bracket mode,
        // plus 3 where the window covers the whole tile; one class with the
        // exact Voigt shape), in lane order within a class, so the sweeps
        // below run one loop per class with no test per pair; with PB = 64
        // the second 32 pairs are staged in their own half the same way
        int base[NH][NCLS + 1];
#pragma unroll
        for (int hh = 0; hh < NH; ++hh) {
            const int nb = min(32, end - (b + 32 * hh));
            PairF32 P;
            bool valid = false;
            if (lane < nb) {
                const int l = a.tile_lines[b + 32 * hh + lane];
                const LineF32 L = a.lf[l];
                valid = setup_pair_f32<FL>(a, L, cp, smlp[L.species], (FL & 1) ? smcb[L.species] : make_float2(0.f, 0.f),
                                           l, c, hf, inv_hf, kt0, kt0f, kt1f, count, &P, cnt);
            }
            int cls = -1;
            if (valid) cls = (FL & 4) ? 0 : P.mode + ((P.lo <= 0.0f && P.hi >= (float)(TW - 1)) ? 3 : 0);
            const unsigned lt = (1u << lane) - 1u;
            int pos = 0;
            base[hh][0] = 32 * hh;
#pragma unroll
            for (int k = 0; k < NCLS; ++k) {
                const unsigned m = __ballot_sync(0xffffffffu, cls == k);
                if (cls == k) pos = base[hh][k] + __popc(m & lt);
                base[hh][k + 1] = base[hh][k] + __popc(m);
            }
            if (cls >= 0) {
                sm0[pos] = make_float4(P.lo, P.hi, P.ub, P.s);
                sm1[pos] = make_float4(P.r, P.ub_lo, P.aj, P.ak);
            }
        }
        __syncwarp();
#pragma unroll
        for (int hh = 0; hh < NH; ++hh) {
            if (FL & 4) {
                for (int q = base[hh][0]; q < base[hh][NCLS]; ++q) {
                    const float4 A = sm0[q];
                    const float4 B = sm1[q];
                    sweep_pair_voigt<PPT>(c_voigt, A.x, A.y, lanef, A.w, A.z, B.y, B.x, B.z, B.w, bj, bk);
                }
            } else {
                sweep_class<PPT, BR_NEAR, false>(sm0, sm1, base[hh][0], base[hh][1], lanef, bj, bk);
                sweep_class<PPT, BR_MID, false>(sm0, sm1, base[hh][1], base[hh][2], lanef, bj, bk);
                sweep_class<PPT, BR_FAR, false>(sm0, sm1, base[hh][2], base[hh][3], lanef, bj, bk);
                sweep_class<PPT, BR_NEAR, true>(sm0, sm1, base[hh][3], base[hh][4], lanef, bj, bk);
                sweep_class<PPT, BR_MID, true>(sm0, sm1, base[hh][4], base[hh][5], lanef, bj, bk);
                sweep_class<PPT, BR_FAR, true>(sm0, sm1, base[hh][5], base[hh][6], lanef, bj, bk);
            }
        }
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            float4 v = acc[i * 32 + lane];
            kahan_add(v.x, v.y, bj[i]);
            kahan_add(v.z, v.w, bk[i]);
            acc[i * 32 + lane] = v;
            bj[i] = bk[i] = 0.0f;
        }
        __syncwarp();
    }
    float* K = reinterpret_cast<float*>(a.kappa) + c * a.ld - a.k0;
    float* J = reinterpret_cast<float*>(a.emis) + c * a.ld - a.k0;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int k = kt0 + lane + 32 * i;
        const float4 v = acc[i * 32 + lane];
        // streaming stores: the rows are read back by the march of a later
        // chunk, long after they would have left L2, so they are marked
        // evict-first and leave L2 to the gathers running beside them
        if (k <= kt1) { __stcs(K + k, v.z); __stcs(J + k, v.x); }
    }
}

// Resident blocks per SM asked of the compiler: 24 warps per SM, so at most
// 80 registers per thread (measured best against 32, 28 and 20 warps).
#ifndef RAPRAL_LS_WARPS
#define RAPRAL_LS_WARPS 24
#endif
#define RAPRAL_LS_BLOCKS(WPB) (RAPRAL_LS_WARPS / (WPB))

template <int PPT, int WPB, int FL = 0, int PB = 32>
__global__ void __launch_bounds__(32 * WPB, RAPRAL_LS_BLOCKS(WPB)) k_line_sum_f32(LineSumArgs a) {
    if (*a.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * WPB + warp;
    if (c >= a.C) return;
    __shared__ float4 sm0[WPB][PB];   // lo, hi, ub, s of each staged pair
    __shared__ float4 sm1[WPB][PB];   // r, ub_lo, aj, ak
    __shared__ float2 smlp[WPB][RAPRAL_MAX_SPECIES];
    __shared__ float2 smcb[WPB][RAPRAL_MAX_SPECIES];
    __shared__ float4 acc[WPB][32 * PPT];
    int64_t cnt[4] = {0, 0, 0, 0};
    warp_tile_f32<PPT, FL, PB>(a, blockIdx.y, c, sm0[warp], sm1[warp], smlp[warp], smcb[warp], acc[warp], lane, cnt);
    if (a.count) block_count(a.stats, cnt[0], cnt[1], cnt[2], cnt[3]);
}

// The same line sum as a persistent launch: a fixed number of blocks pull
// the units (tile, group of WPB cells) of k_line_sum_f32's grid, in its
// order (tile by tile), from an atomic counter; each warp does the same
// work as there, so the sums are bitwise the same.
template <int PPT, int WPB, int PB = 32>
__global__ void __launch_bounds__(32 * WPB, RAPRAL_LS_BLOCKS(WPB)) k_line_sum_f32_persist(LineSumArgs a, int64_t n_groups,
                                                                            int64_t total,
                                                                            unsigned long long* counter) {
    if (*a.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ float4 sm0[WPB][PB];
    __shared__ float4 sm1[WPB][PB];
    __shared__ float2 smlp[WPB][RAPRAL_MAX_SPECIES];
    __shared__ float2 smcb[WPB][RAPRAL_MAX_SPECIES];
    __shared__ float4 acc[WPB][32 * PPT];
    __shared__ long long unit_s;
    int64_t cnt[4] = {0, 0, 0, 0};
    for (;;) {
        if (threadIdx.x == 0) unit_s = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const int64_t u = unit_s;
        __syncthreads();
        if (u >= total) break;
        const int t = (int)(u / n_groups);
        const int64_t c = (u - (int64_t)t * n_groups) * WPB + warp;
        if (c < a.C) warp_tile_f32<PPT, 0, PB>(a, t, c, sm0[warp], sm1[warp], smlp[warp], smcb[warp], acc[warp], lane, cnt);
        __syncwarp();
    }
    if (a.count) block_count(a.stats, cnt[0], cnt[1], cnt[2], cnt[3]);
}

// Launches k_line_sum_f32_persist over the units of grid g: ctx->ls_persist
// blocks a SM, or as many as fit (-1); the unit counter (ctx->d_unit) is
// cleared on the stream first.
template <int PPT, int WPB, int PB>
static cudaError_t launch_persist(rapral_ctx* ctx, const LineSumArgs& a, dim3 g) {
    int dev = 0, sms = 0, per_sm = ctx->ls_persist;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && per_sm < 0)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_line_sum_f32_persist<PPT, WPB, PB>, 32 * WPB, 0);
    unsigned long long* counter = ctx->d_unit;
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), ctx->stream);
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)g.x * g.y;
    const int64_t blocks = std::min<int64_t>(total, (int64_t)sms * std::max(1, per_sm));
    k_line_sum_f32_persist<PPT, WPB, PB><<<(unsigned)blocks, 32 * WPB, 0, ctx->stream>>>(a, (int64_t)g.x, total, counter);
    return cudaGetLastError();
}

// Persistent line sum over many independent requests: blocks pull work
// units (request, tile, group of WPB cells) from one atomic counter until the
// list is exhausted; units of a request are ordered tile by tile so blocks
// working at the same time share a tile's line list in L2.
template <int PPT, int WPB, bool BR = false, int PB = 32>
__global__ void __launch_bounds__(32 * WPB, RAPRAL_LS_BLOCKS(WPB)) k_line_sum_batch(const BatchItem* __restrict__ items,
                                                                       int n_items, int64_t total,
                                                                       unsigned long long* counter,
                                                                       unsigned long long* stats, const int* status) {
    if (*status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ float4 sm0[WPB][PB];
    __shared__ float4 sm1[WPB][PB];
    __shared__ float2 smlp[WPB][RAPRAL_MAX_SPECIES];
    __shared__ float2 smcb[WPB][RAPRAL_MAX_SPECIES];
    __shared__ float4 acc[WPB][32 * PPT];
    __shared__ long long unit_s;
    int64_t cnt[4] = {0, 0, 0, 0};
    for (;;) {
        if (threadIdx.x == 0) unit_s = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const int64_t u = unit_s;
        __syncthreads();
        if (u >= total) break;
        int lo = 0, hi = n_items;     // last item whose first unit is <= u
        while (hi - lo > 1) {
            const int m = (lo + hi) >> 1;
            if (items[m].unit_off <= u) lo = m; else hi = m;
        }
        const BatchItem& it = items[lo];
        const int64_t local = u - it.unit_off;
        const int t = (int)(local / it.n_groups);
        const int64_t c = (local - (int64_t)t * it.n_groups) * WPB + warp;
        if (c < it.a.C)
            warp_tile_f32<PPT, BR ? 1 : 0, PB>(it.a, t, c, sm0[warp], sm1[warp], smlp[warp], smcb[warp], acc[warp],
                                               lane, cnt);
        __syncwarp();
    }
    if (items[0].a.count) block_count(stats, cnt[0], cnt[1], cnt[2], cnt[3]);
}

}  // namespace

cudaError_t launch_validate_lines(rapral_ctx* ctx, const rapral_lines* ln, int32_t n_species) {
    if (ln->n_lines == 0) return cudaSuccess;
    k_validate_lines<<<div_up(ln->n_lines, 256), 256, 0, ctx->stream>>>(*ln, n_species, ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_line_prep(rapral_ctx* ctx, const rapral_species* sp, const rapral_lines* ln,
                             double lam_min, double h, const Phys& ph, LinePrep* out, LineF32* out32,
                             int* sorted_flag, const BroadArgs* br, double2* lb, float2* lb32) {
    if (ln->n_lines == 0) return cudaSuccess;
    BroadArgs b = br ? *br : BroadArgs{};
    if (!broad_terms(br)) lb = nullptr, lb32 = nullptr;
    k_line_prep<<<div_up(ln->n_lines, 256), 256, 0, ctx->stream>>>(*ln, sp->mass, sp->kind, lam_min, h, ph, out,
                                                                   out32, sorted_flag, b, lb, lb32, ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_bin_bounds(rapral_ctx* ctx, const rapral_lines* ln, const LinePrep* lp, const CellPrep* cp,
                              const unsigned long long* d_max, double h, BinPlan* plan, const double2* lb) {
    (void)cp;
    if (ln->n_lines == 0) return cudaSuccess;
    k_bin_bounds<<<div_up(ln->n_lines, 256), 256, 0, ctx->stream>>>(lp, ln->n_lines, d_max, h, plan->k0, plan->nk,
                                                                    plan->tile_w, plan->line_tiles, plan->wmax,
                                                                    lb, ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_bin_count(rapral_ctx* ctx, const rapral_lines* ln, const rapral_grid* g, double h,
                             BinPlan* plan) {
    k_bin_count<<<(unsigned)plan->n_tiles, 256, 0, ctx->stream>>>(ln->lam0, ln->n_lines, plan->line_tiles,
                                                                  plan->sorted_flag, plan->wmax, g->lam_min, h,
                                                                  plan->k0, plan->nk, plan->tile_w, plan->tile_off,
                                                                  ctx->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan_counts<<<1, 1024, 0, ctx->stream>>>(plan->tile_off, plan->n_tiles, plan->total);
    return cudaGetLastError();
}

cudaError_t launch_bin_fill(rapral_ctx* ctx, const rapral_lines* ln, const rapral_grid* g, double h,
                            BinPlan* plan) {
    k_bin_fill<<<(unsigned)plan->n_tiles, 256, 0, ctx->stream>>>(ln->lam0, ln->n_lines, plan->line_tiles,
                                                                 plan->sorted_flag, plan->wmax, g->lam_min, h,
                                                                 plan->k0, plan->nk, plan->tile_w, plan->tile_off,
                                                                 plan->tile_lines, ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_scan_i64(rapral_ctx* ctx, int64_t* data, int64_t n) {
    k_scan<long long><<<1, 1024, 0, ctx->stream>>>(reinterpret_cast<long long*>(data), n);
    return cudaGetLastError();
}

static cudaError_t launch_line_sum_grid(rapral_ctx* ctx, const LineSumArgs& a, int precision, dim3 grid);

cudaError_t launch_line_sum(rapral_ctx* ctx, const LineSumArgs& a, int precision, int64_t n_tiles) {
    if (n_tiles == 0 || a.C == 0) return cudaSuccess;
    // cells along x (up to 2^31 - 1), tiles along y (<= 65535): consecutive
    // blocks share a tile's line list in L2
    dim3 grid((unsigned)a.C, (unsigned)n_tiles);
    if (ctx->ev_before) cudaEventRecord(ctx->ev_before, ctx->stream);
    cudaError_t e = launch_line_sum_grid(ctx, a, precision, grid);
    if (ctx->ev_after) cudaEventRecord(ctx->ev_after, ctx->stream);
    return e;
}

static cudaError_t launch_line_sum_grid(rapral_ctx* ctx, const LineSumArgs& a, int precision, dim3 grid) {
    if (precision == RAPRAL_FP64) {
        if (a.voigt) {   // one tiling with the exact line shape
            if (a.tile_w != 512) return cudaErrorInvalidValue;
            k_line_sum_f64<4, true><<<grid, 128, 0, ctx->stream>>>(a);
            return cudaGetLastError();
        }
        switch (a.tile_w) {
            case 128: k_line_sum_f64<1><<<grid, 128, 0, ctx->stream>>>(a); break;
            case 256: k_line_sum_f64<2><<<grid, 128, 0, ctx->stream>>>(a); break;
            case 512: k_line_sum_f64<4><<<grid, 128, 0, ctx->stream>>>(a); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    // FP32: warp-level kernel, WPB cells per block; with the optional
    // resonance / van der Waals terms four cells a block
    const int fl = (a.lb32 ? 1 : 0) | (a.dep_lnb ? 2 : 0) | (a.voigt ? 4 : 0);
    if (fl & 4) {   // exact Voigt shape: one tiling, 128 x 4
        if (a.tile_w != 128) return cudaErrorInvalidValue;
        dim3 gb(div_up(a.C, 4), grid.y);
        switch (fl) {
            case 4: k_line_sum_f32<4, 4, 4><<<gb, 128, 0, ctx->stream>>>(a); break;
            case 5: k_line_sum_f32<4, 4, 5><<<gb, 128, 0, ctx->stream>>>(a); break;
            case 6: k_line_sum_f32<4, 4, 6><<<gb, 128, 0, ctx->stream>>>(a); break;
            default: k_line_sum_f32<4, 4, 7><<<gb, 128, 0, ctx->stream>>>(a); break;
        }
        return cudaGetLastError();
    }
    if (fl) {
        dim3 gb(div_up(a.C, 4), grid.y);
#define RAPRAL_LSF(FL)                                                                   \
    switch (a.tile_w) {                                                                  \
        case 128: k_line_sum_f32<4, 4, FL><<<gb, 128, 0, ctx->stream>>>(a); break;      \
        case 256: k_line_sum_f32<8, 4, FL><<<gb, 128, 0, ctx->stream>>>(a); break;      \
        case 512: k_line_sum_f32<16, 4, FL><<<gb, 128, 0, ctx->stream>>>(a); break;     \
        default: return cudaErrorInvalidValue;                                           \
    }
        if (fl == 1) { RAPRAL_LSF(1) } else if (fl == 2) { RAPRAL_LSF(2) } else { RAPRAL_LSF(3) }
#undef RAPRAL_LSF
        return cudaGetLastError();
    }
    const int wpb = a.tile_w == 512 ? 4 : ctx->cells_per_block;
    dim3 g32(div_up(a.C, wpb), grid.y);
#define RAPRAL_LS32_PB(PPT, WPB, PB)                                                          \
    do {                                                                                      \
        if (ctx->ls_persist != 0 && ctx->d_unit) return launch_persist<PPT, WPB, PB>(ctx, a, g32); \
        k_line_sum_f32<PPT, WPB, 0, PB><<<g32, 32 * WPB, 0, ctx->stream>>>(a);                 \
    } while (0)
#define RAPRAL_LS32(PPT, WPB)                                  \
    do {                                                       \
        if (ctx->pairs_per_batch == 64) RAPRAL_LS32_PB(PPT, WPB, 64); \
        else RAPRAL_LS32_PB(PPT, WPB, 32);                     \
    } while (0)
    if (a.tile_w == 128 && wpb == 2) RAPRAL_LS32(4, 2);
    else if (a.tile_w == 128 && wpb == 4) RAPRAL_LS32(4, 4);
    else if (a.tile_w == 128 && wpb == 8) RAPRAL_LS32(4, 8);
    else if (a.tile_w == 256 && wpb == 2) RAPRAL_LS32(8, 2);
    else if (a.tile_w == 256 && wpb == 4) RAPRAL_LS32(8, 4);
    else if (a.tile_w == 256 && wpb == 8) RAPRAL_LS32(8, 8);
    else if (a.tile_w == 512) RAPRAL_LS32(16, 4);
    else return cudaErrorInvalidValue;
#undef RAPRAL_LS32
#undef RAPRAL_LS32_PB
    return cudaGetLastError();
}

template <int PPT, int WPB, bool BR = false, int PB = 32>
static cudaError_t batch_launch(rapral_ctx* ctx, const BatchItem* items, int n, int64_t total,
                                unsigned long long* counter, int* blocks_out, bool launch) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_line_sum_batch<PPT, WPB, BR, PB>, 32 * WPB, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = max(1, per_sm) * sms;
    if (blocks_out) *blocks_out = blocks;
    if (!launch) return cudaSuccess;
    k_line_sum_batch<PPT, WPB, BR, PB><<<blocks, 32 * WPB, 0, ctx->stream>>>(items, n, total, counter, ctx->d_stats,
                                                                             ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_line_sum_batch(rapral_ctx* ctx, int tile_w, int wpb, int pb, const BatchItem* items, int n,
                                  int64_t total, unsigned long long* counter, int* blocks_out, bool launch, bool broad) {
    if (broad) {   // the optional Lorentz terms: four cells a block (the plan's group size), 32 pairs a pass
        if (wpb != 4 || pb != 32) return cudaErrorInvalidValue;
        if (tile_w == 128) return batch_launch<4, 4, true>(ctx, items, n, total, counter, blocks_out, launch);
        if (tile_w == 256) return batch_launch<8, 4, true>(ctx, items, n, total, counter, blocks_out, launch);
        if (tile_w == 512) return batch_launch<16, 4, true>(ctx, items, n, total, counter, blocks_out, launch);
        return cudaErrorInvalidValue;
    }
#define RAPRAL_BL(PPT, WPB)                                                                          \
    return pb == 64 ? batch_launch<PPT, WPB, false, 64>(ctx, items, n, total, counter, blocks_out, launch) \
                    : batch_launch<PPT, WPB, false, 32>(ctx, items, n, total, counter, blocks_out, launch)
    if (pb != 32 && pb != 64) return cudaErrorInvalidValue;
    if (tile_w == 128 && wpb == 2) RAPRAL_BL(4, 2);
    if (tile_w == 128 && wpb == 4) RAPRAL_BL(4, 4);
    if (tile_w == 128 && wpb == 8) RAPRAL_BL(4, 8);
    if (tile_w == 256 && wpb == 2) RAPRAL_BL(8, 2);
    if (tile_w == 256 && wpb == 4) RAPRAL_BL(8, 4);
    if (tile_w == 256 && wpb == 8) RAPRAL_BL(8, 8);
    if (tile_w == 512) RAPRAL_BL(16, 4);
#undef RAPRAL_BL
    return cudaErrorInvalidValue;
}

// Fourier coefficients a_1 .. a_N of f(t) = L^2 sec^2(t/2) e^{-L^2 tan^2(t/2)},
// L = (N / sqrt 2)^{1/2}, by the trapezoid rule on 4N points of [-pi, pi)
// (f vanishes at -pi): the coefficients of Weideman's rational expansion.
static void weideman(int N, double* a, double* L) {
    const int M = 2 * N, M2 = 2 * M;
    const double l = std::sqrt(N / std::sqrt(2.0));
    *L = l;
    for (int n = 1; n <= N; ++n) {
        double acc = 0.0;
        for (int j = -M + 1; j <= M - 1; ++j) {
            const double th = j * M_PI / M;
            const double t = l * std::tan(0.5 * th);
            acc += std::exp(-t * t) * (l * l + t * t) * std::cos(n * th);
        }
        a[n - 1] = acc / M2;
    }
}

const VoigtCoef& voigt_coefficients() {
    static const VoigtCoef vc = [] {
        VoigtCoef v{};
        weideman(RAPRAL_VOIGT_NW64, v.a64, &v.L64);
        double a32[RAPRAL_VOIGT_NW32], L32;
        weideman(RAPRAL_VOIGT_NW32, a32, &L32);
        for (int n = 0; n < RAPRAL_VOIGT_NW32; ++n) v.a32[n] = (float)a32[n];
        v.L32 = (float)L32;
        return v;
    }();
    return vc;
}

cudaError_t voigt_upload() {
    return cudaMemcpyToSymbol(c_voigt, &voigt_coefficients(), sizeof(VoigtCoef));
}
