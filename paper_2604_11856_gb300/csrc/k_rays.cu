// Rays: builders (tangent slab, axisymmetric lines of sight), the segment
// march with the angular reduction, and the spectral flux integral
// (Sec. 2.2.3).
//
// k_march (below) marches the bundles of every surface point over a range of
// wavelength columns and reduces them to the spectral flux at the point;
// k_wall_flux_part / _sum integrate that over the range.
#include <algorithm>

#include "rapral_internal.cuh"
#include "geom.cuh"

namespace {

// Segment coefficients: e = e^{-dtau}, far-node coefficient ca = (f - e)/kappa
// and near-node coefficient cb = (1 - f)/kappa, f = (1 - e)/dtau, with their
// series for small |dtau|.
//   FP64: |dtau| < 4e-4 takes three terms of each series; e from expm1.
//   FP32: |dtau| < 0.5 takes seven terms (truncation <= 4e-7 relative), so
//   the closed form is used only where 1 - e >= 0.39 and an approximate ex2
//   for e keeps FP32 accuracy without expm1f.
__device__ __forceinline__ void seg_coeffs(double kap, double s, double inv_k, double /*inv_s*/, double* e,
                                           double* ca, double* cb) {
    const double dtau = kap * s;
    const double em1 = expm1(-dtau);   // e^{-dtau} - 1
    *e = 1.0 + em1;
    if (fabs(dtau) < RAPRAL_THIN_F64) {
        *ca = s * (0.5 - dtau * (1.0 / 3.0) + dtau * dtau * 0.125);
        *cb = s * (0.5 - dtau * (1.0 / 6.0) + dtau * dtau * (1.0 / 24.0));
    } else {
        const double f = -em1 / dtau;
        *ca = (f - *e) * inv_k;
        *cb = (1.0 - f) * inv_k;
    }
}

__device__ __forceinline__ float ex2f_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float recip(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The same coefficients for one direction per segment: the closed form takes
// a single reciprocal, of dtau, inside its branch (1/kappa = s / dtau).
__device__ __forceinline__ void seg_coeffs1(double kap, double s, double* e, double* ca, double* cb) {
    seg_coeffs(kap, s, 1.0 / kap, 0.0, e, ca, cb);
}
// One segment of the march for one direction: I <- I e + ca j_far + cb j_near.
// FP32 folds the common factor of ca and cb (s, or s / dtau) into one
// multiply: I e + m (a j_far + b j_near).
__device__ __forceinline__ void seg_step(double& I, double kf, double s, double jf, double jn) {
    double e, ca, cb;
    seg_coeffs1(kf, s, &e, &ca, &cb);
    I = I * e + ca * jf + cb * jn;
}
// FP32, thin (|dtau| < 0.5): with p = (1 - f)/dtau from its series
// p = sum_n (-dtau)^n / (n + 2)!, n = 0..6 (truncation below 4e-8 relative)
// and f = 1 - dtau p, the step I e + ca j_far + cb j_near is
// I + s f (j_far - kappa I) + s p (j_near - j_far): one series and no
// exponential (e = 1 - dtau f >= 0.6 keeps the subtraction within a factor
// 1/e of FP32 rounding).  Thick: e from ex2, f from one reciprocal.
__device__ __forceinline__ float thin_series(float t) {
    float p = fmaf(t, 1.0f / 40320.0f, -1.0f / 5040.0f);
    p = fmaf(t, p, 1.0f / 720.0f);
    p = fmaf(t, p, -1.0f / 120.0f);
    p = fmaf(t, p, 1.0f / 24.0f);
    p = fmaf(t, p, -1.0f / 6.0f);
    return fmaf(t, p, 0.5f);
}
__device__ __forceinline__ void seg_step(float& I, float kf, float s, float jf, float jn) {
    const float dtau = kf * s;
    if (fabsf(dtau) < (float)RAPRAL_THIN_F32) {
        const float p = thin_series(dtau);
        const float f = fmaf(-dtau, p, 1.0f);
        I = fmaf(s, fmaf(f, fmaf(-kf, I, jf), p * (jn - jf)), I);
        return;
    }
    const float e = ex2f_approx(-1.44269504f * dtau);
    const float r = recip(dtau);
    const float f = (1.0f - e) * r;
    I = fmaf(s * r, fmaf(f - e, jf, (1.0f - f) * jn), I * e);
}

// Two steps at once in FP32 (two wavelength columns, or two directions of a
// bundle): where both are optically thin the series and the update run as
// packed pairs (one instruction for both, each with the scalar step's IEEE
// result); otherwise each takes the scalar step.
__device__ __forceinline__ void seg_step2(float& I0, float& I1, float k0, float k1, float s0, float s1, float jf0,
                                          float jf1, float jn0, float jn1) {
    const float2 k = make_float2(k0, k1), s = make_float2(s0, s1);
    const float2 dt = __fmul2_rn(k, s);
    if (fabsf(dt.x) < (float)RAPRAL_THIN_F32 && fabsf(dt.y) < (float)RAPRAL_THIN_F32) {
        const auto c2 = [](float c) { return make_float2(c, c); };
        float2 p = __ffma2_rn(dt, c2(1.0f / 40320.0f), c2(-1.0f / 5040.0f));
        p = __ffma2_rn(dt, p, c2(1.0f / 720.0f));
        p = __ffma2_rn(dt, p, c2(-1.0f / 120.0f));
        p = __ffma2_rn(dt, p, c2(1.0f / 24.0f));
        p = __ffma2_rn(dt, p, c2(-1.0f / 6.0f));
        p = __ffma2_rn(dt, p, c2(0.5f));
        const float2 f = __ffma2_rn(make_float2(-dt.x, -dt.y), p, c2(1.0f));
        const float2 I = make_float2(I0, I1);
        const float2 A = __ffma2_rn(make_float2(-k0, -k1), I, make_float2(jf0, jf1));
        const float2 dJ = make_float2(jn0 - jf0, jn1 - jf1);
        const float2 r = __ffma2_rn(s, __ffma2_rn(f, A, __fmul2_rn(p, dJ)), I);
        I0 = r.x;
        I1 = r.y;
    } else {
        seg_step(I0, k0, s0, jf0, jn0);
        seg_step(I1, k1, s1, jf1, jn1);
    }
}

// the MAXD directions of one column: packed in pairs in FP32
template <class T, int MAXD>
__device__ __forceinline__ void dir_steps(T (&I)[MAXD], T kf, T ds, const T* sc, T jf, T jn) {
    if constexpr (sizeof(T) == 4 && MAXD > 1) {
#pragma unroll
        for (int d = 0; d + 1 < MAXD; d += 2)
            seg_step2(I[d], I[d + 1], kf, kf, ds * sc[d], ds * sc[d + 1], jf, jf, jn, jn);
        if (MAXD & 1) seg_step(I[MAXD - 1], kf, ds * sc[MAXD - 1], jf, jn);
    } else {
#pragma unroll
        for (int d = 0; d < MAXD; ++d) seg_step(I[d], kf, MAXD == 1 ? ds : ds * sc[d], jf, jn);
    }
}

__global__ void k_validate_rays(const int32_t* seg_cell, const double* seg_ds, int64_t nseg, int64_t C,
                                const double* dir_scale, int64_t ndir, int* status) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nseg) {
        const int c = seg_cell[i];
        if (c < 0 || c >= C) fail(status, CHK_SEG_CELL, i);
        const double d = seg_ds[i];
        if (!(d >= 0.0) || !isfinite(d)) fail(status, CHK_SEG_DS, i);
    }
    if (i < ndir) {
        const double s = dir_scale[i];
        if (!(s > 0.0) || !isfinite(s)) fail(status, CHK_DIR, i);
    }
}

struct MarchArgs {
    const int64_t* point_off;
    const int64_t* seg_off;
    const int32_t* seg_cell;
    const double* seg_ds;
    const int64_t* dir_off;
    const double* dir_scale;
    const double* dir_weight;
    const float* seg_ds_f;       // FP32 copies (FP32 march only): no conversion per
    const float* dir_scale_f;    // (segment, direction, wavelength)
    const float* dir_weight_f;
    const int32_t* bundle_wall;
    double T_wall;
    const void* wall_row;        // Planck intensity at T_wall per column (null: T_wall = 0)
    const void* kappa;
    const void* emis;
    int64_t ld;
    double lam_min, h;
    int64_t k0, nk;
    void* q_lambda;
    void* I_out;
    Phys ph;
    const int* status;
};

template <class T> __device__ __forceinline__ T seg_len(const MarchArgs& a, int64_t i);
template <> __device__ __forceinline__ double seg_len<double>(const MarchArgs& a, int64_t i) { return a.seg_ds[i]; }
template <> __device__ __forceinline__ float seg_len<float>(const MarchArgs& a, int64_t i) { return a.seg_ds_f[i]; }
template <class T> __device__ __forceinline__ T dir_val(const double* d, const float* f, int64_t i);
template <> __device__ __forceinline__ double dir_val<double>(const double* d, const float*, int64_t i) { return d[i]; }
template <> __device__ __forceinline__ float dir_val<float>(const double*, const float* f, int64_t i) { return f[i]; }

__global__ void k_to_float(const double* __restrict__ x, int64_t n, float* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

// Planck intensity, temperature form (Sec. 2.2), W/cm^2/sr/um.
__device__ __forceinline__ double planck(double lam_nm, double T, const Phys& ph) {
    const double lcm = lam_nm * 1e-7;
    const double l2 = lcm * lcm;
    return 1e-7 * 2.0 * ph.h * ph.c * ph.c / (1e4 * l2 * l2 * lcm * expm1(ph.h * ph.c / (lcm * ph.kB * T)));
}

// The march of one bundle over the lane's V columns: staged segment list,
// next-cell gathers one step ahead, all MAXD directions per segment.  A
// bundle with nd < MAXD directions marches the others with scale 0, which
// leaves their intensity at its start value (e = 1, zero source): no
// per-direction check in the loop.  Returns the intensities in I[v][d].
template <class T> struct __align__(16) SegStage {
    const char* row;   // kappa row of the segment's next cell
    T ds;              // path length (x the direction scale for one-direction bundles)
};

#ifndef RAPRAL_MARCH_UNROLL
#define RAPRAL_MARCH_UNROLL 3
#endif
constexpr int kUnroll = RAPRAL_MARCH_UNROLL;

// Node-valued rays (one direction): rows are the LOS nodes, segment s of
// bundle b runs from node s + b to node s + b + 1, kappa held at the far
// node, j linear between the nodes (the same coefficients).
template <class T, int V>
__device__ __forceinline__ void march_nodes(const MarchArgs& a, int64_t b, T sc, SegStage<T>* stage, int lane,
                                            const char* kbase, int64_t ldb, int64_t offK, int64_t offJ,
                                            T (&I)[V][1]) {
    const int64_t s0 = a.seg_off[b], s1 = a.seg_off[b + 1];
    if (s1 <= s0) return;
    T kf[V], jf[V];
    {
        const char* row = kbase + (s0 + b) * ldb;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            kf[v] = *reinterpret_cast<const T*>(row + offK + 32 * v * sizeof(T));
            jf[v] = *reinterpret_cast<const T*>(row + offJ + 32 * v * sizeof(T));
        }
    }
    for (int64_t g = s0; g < s1; g += 32) {
        const int64_t mine = g + lane;
        __syncwarp();
        const bool in = mine < s1;
        stage[lane].row = in ? kbase + (mine + 1 + b) * ldb : kbase;
        stage[lane].ds = in ? seg_len<T>(a, mine) * sc : T(0);
        if (lane == 0) stage[32].row = kbase;
        __syncwarp();
        const int n = s1 - g < 32 ? (int)(s1 - g) : 32;
        T kx[V], jx[V];
        {
            const char* r0 = stage[0].row;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                kx[v] = *reinterpret_cast<const T*>(r0 + offK + 32 * v * sizeof(T));
                jx[v] = *reinterpret_cast<const T*>(r0 + offJ + 32 * v * sizeof(T));
            }
        }
        for (int j = 0; j < n; ++j) {
            const T ds = stage[j].ds;
            const char* rn = stage[j + 1].row;
            T ky[V], jy[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                ky[v] = *reinterpret_cast<const T*>(rn + offK + 32 * v * sizeof(T));
                jy[v] = *reinterpret_cast<const T*>(rn + offJ + 32 * v * sizeof(T));
            }
            if constexpr (V == 2 && sizeof(T) == 4) {
                seg_step2(I[0][0], I[1][0], kf[0], kf[1], ds, ds, jf[0], jf[1], jx[0], jx[1]);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) seg_step(I[v][0], kf[v], ds, jf[v], jx[v]);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                kf[v] = kx[v]; jf[v] = jx[v];
                kx[v] = ky[v]; jx[v] = jy[v];
            }
        }
    }
}

template <class T, int V, int MAXD>
__device__ __forceinline__ void march_bundle(const MarchArgs& a, int64_t b, int64_t d0, int nd, SegStage<T>* stage,
                                             int lane, const char* kbase, int64_t ldb, int64_t offK, int64_t offJ,
                                             int col0, T (&I)[V][MAXD]) {
    T sc[MAXD];
#pragma unroll
    for (int d = 0; d < MAXD; ++d) sc[d] = d < nd ? dir_val<T>(a.dir_scale, a.dir_scale_f, d0 + d) : T(0);
    // one direction: its scale goes into the staged length
    const T stage_scale = MAXD == 1 ? sc[0] : T(1);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const T I0 = (a.wall_row && a.bundle_wall[b]) ? reinterpret_cast<const T*>(a.wall_row)[col0 + 32 * v] : T(0);
#pragma unroll
        for (int d = 0; d < MAXD; ++d) I[v][d] = I0;
    }
    const int64_t s0 = a.seg_off[b], s1 = a.seg_off[b + 1];
    if (s1 <= s0) return;
    T kc[V], jc[V], kf[V], jf[V];
    {
        const char* row = kbase + (int64_t)a.seg_cell[s0] * ldb;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            kc[v] = kf[v] = *reinterpret_cast<const T*>(row + offK + 32 * v * sizeof(T));
            jc[v] = jf[v] = *reinterpret_cast<const T*>(row + offJ + 32 * v * sizeof(T));
        }
    }
    // every segment but the last has a next cell: stage (row of the next
    // cell, length) for 32 segments, read back by all lanes
    for (int64_t g = s0; g < s1 - 1; g += 32) {
        const int64_t mine = g + lane;
        __syncwarp();
        // entries past the chunk point at row 0 (a valid row), so the
        // prefetch of entry j + 1 below never leaves the arrays
        const bool in = mine < s1 - 1;
        stage[lane].row = in ? kbase + (int64_t)a.seg_cell[mine + 1] * ldb : kbase;
        stage[lane].ds = in ? seg_len<T>(a, mine) * stage_scale : T(0);
        if (lane == 0) stage[32].row = kbase;
        __syncwarp();
        const int n = s1 - 1 - g < 32 ? (int)(s1 - 1 - g) : 32;
        T kx[V], jx[V];
        {
            const char* r0 = stage[0].row;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                kx[v] = *reinterpret_cast<const T*>(r0 + offK + 32 * v * sizeof(T));
                jx[v] = *reinterpret_cast<const T*>(r0 + offJ + 32 * v * sizeof(T));
            }
        }
        constexpr int U = MAXD == 1 ? kUnroll : 1;   // bundles of many directions: registers go to I
#pragma unroll U
        for (int j = 0; j < n; ++j) {
            const T ds = stage[j].ds;
            const char* rn = stage[j + 1].row;
            T ky[V], jy[V];   // next segment's next cell, loaded a step ahead
#pragma unroll
            for (int v = 0; v < V; ++v) {
                ky[v] = *reinterpret_cast<const T*>(rn + offK + 32 * v * sizeof(T));
                jy[v] = *reinterpret_cast<const T*>(rn + offJ + 32 * v * sizeof(T));
            }
            T kn[V], jn[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                kn[v] = T(0.5) * (kc[v] + kx[v]);
                jn[v] = T(0.5) * (jc[v] + jx[v]);
            }
            if constexpr (V == 2 && MAXD == 1 && sizeof(T) == 4) {
                seg_step2(I[0][0], I[1][0], kf[0], kf[1], ds, ds, jf[0], jf[1], jn[0], jn[1]);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) dir_steps<T, MAXD>(I[v], kf[v], ds, sc, jf[v], jn[v]);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                kf[v] = kn[v]; jf[v] = jn[v];
                kc[v] = kx[v]; jc[v] = jx[v];
                kx[v] = ky[v]; jx[v] = jy[v];
            }
        }
    }
    {   // last segment: its near node is the cell's own value
        const T ds = seg_len<T>(a, s1 - 1) * stage_scale;
        if constexpr (V == 2 && MAXD == 1 && sizeof(T) == 4) {
            seg_step2(I[0][0], I[1][0], kf[0], kf[1], ds, ds, jf[0], jf[1], jc[0], jc[1]);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) dir_steps<T, MAXD>(I[v], kf[v], ds, sc, jf[v], jc[v]);
        }
    }
}

// k_march: the segment march with the angular reduction.  A block of eight
// warps covers one (surface point, bundle group) and a tile of wavelength
// columns; its warps are SL bundle slices x CW = 8 / SL column groups, and
// lane l of a column group takes columns l, l + 32, ..., l + 32 (V - 1) of
// the group's 32 V.  Each gather of a segment is then V coalesced row
// reads, and the per-segment work (next cell, length, row address) is
// shared by the V columns and the bundle's directions.  SL = 8 (many bundles
// a point, as the axisymmetric rays): the eight warps take the bundles of
// the group round-robin; SL = 1 (a few bundles of many directions, as the
// tangent slab): all warps march every bundle over eight column groups.
// A warp stages the next cell's row address and the length of 32 segments at
// a time in shared memory (one coalesced read of the segment list), so no
// kappa / j gather waits on a dependent load of the list, and loads the next
// segment's values one step ahead; the last segment of a bundle, whose near
// node is its own cell, is taken after the loop.  A point's bundles are
// split over 2^lgG blocks (groups) so that enough blocks share a wavelength
// tile for its kappa / j rows to stay in L2.  Each slice Kahan-sums its
// bundles' weighted intensities, the slices are added in a fixed order, and
// the groups' partial spectral fluxes are added in group order by
// k_group_sum: results do not depend on timing.  The last wavelength tile is
// shifted back to end at nk (columns below the tile are computed again and
// not written), so every load is in bounds; with V = 1 and nk below the
// tile a lane past nk reads column nk - 1 and writes nothing.
#ifndef RAPRAL_MARCH_MINB
#define RAPRAL_MARCH_MINB 4
#endif
#ifndef RAPRAL_MARCH_MINB17
#define RAPRAL_MARCH_MINB17 3
#endif
template <class T, int V, int MAXD, int SL, bool NODES = false>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && MAXD == 1 && V > 1)  ? RAPRAL_MARCH_MINB
                                       : (sizeof(T) == 4 && MAXD == 17) ? RAPRAL_MARCH_MINB17
                                                                        : 1)
    k_march(MarchArgs a, int lgG, T* __restrict__ part) {
    static_assert(!NODES || MAXD == 1, "node-valued rays have one direction a bundle");
    if (*a.status) return;
    constexpr int W = 8, CW = W / SL, TW = CW * 32 * V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slice = warp / CW, cgrp = warp % CW;
    // columns fit in int: nk <= 32 x 65535 (checked by the caller)
    const int nk = (int)a.nk;
    const int tile0 = (int)blockIdx.y * TW;
    const int base = (tile0 + TW > nk && nk >= TW) ? nk - TW : tile0;
    const int colu = base + cgrp * 32 * V + lane;   // unclamped first column
    const int col0 = colu < nk ? colu : nk - 1;     // only when V = 1 and nk < TW
    // byte addressing: row of cell c at kbase + c ldb; this lane's kappa and
    // j columns at offK, offJ from it
    const char* kbase = reinterpret_cast<const char*>(a.kappa);
    const int64_t ldb = a.ld * (int64_t)sizeof(T);
    const int64_t offK = (int64_t)col0 * sizeof(T);
    const int64_t offJ = (reinterpret_cast<const char*>(a.emis) - kbase) + offK;
    __shared__ SegStage<T> stage_all[W][33];
    SegStage<T>* stage = stage_all[warp];
    T acc[V], comp[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = comp[v] = T(0);
    // G = 2^lgG groups of point p = blockIdx.x >> lgG; group g takes every
    // G-th run of SL bundles, slice s the s-th bundle of each run
    const unsigned p = blockIdx.x >> lgG, grp = blockIdx.x & ((1u << lgG) - 1u);
    const int64_t b1 = a.point_off[p + 1];
    for (int64_t b = a.point_off[p] + (int64_t)grp * SL + slice; b < b1; b += (int64_t)SL << lgG) {
        const int64_t d0 = a.dir_off[b];
        const int nd = (int)(a.dir_off[b + 1] - d0);
        if (nd == 0) continue;
        T I[V][MAXD];
        if constexpr (NODES) {
            const bool wall = a.wall_row && a.bundle_wall[b];
#pragma unroll
            for (int v = 0; v < V; ++v) I[v][0] = wall ? reinterpret_cast<const T*>(a.wall_row)[col0 + 32 * v] : T(0);
            march_nodes<T, V>(a, b, dir_val<T>(a.dir_scale, a.dir_scale_f, d0), stage, lane, kbase, ldb, offK, offJ,
                              I);
        } else {
            march_bundle<T, V, MAXD>(a, b, d0, nd, stage, lane, kbase, ldb, offK, offJ, col0, I);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int kk = colu + 32 * v;
            const bool own = kk >= tile0 && kk < nk;
            T part_v = T(0);
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                if (d < nd) {
                    part_v += dir_val<T>(a.dir_weight, a.dir_weight_f, d0 + d) * I[v][d];
                    if (a.I_out && own) reinterpret_cast<T*>(a.I_out)[(d0 + d) * a.nk + kk] = I[v][d];
                }
            }
            // compensated sum over the slice's bundles
            const T y = part_v - comp[v];
            const T tt = acc[v] + y;
            comp[v] = (tt - acc[v]) - y;
            acc[v] = tt;
        }
    }
    __shared__ T red[SL][TW];
#pragma unroll
    for (int v = 0; v < V; ++v) red[slice][cgrp * 32 * V + lane + 32 * v] = acc[v];
    __syncthreads();
    T* dst = (lgG == 0 ? reinterpret_cast<T*>(a.q_lambda) : part) + (int64_t)blockIdx.x * a.nk;
    for (int i = threadIdx.x; i < TW; i += 256) {
        const int kk = base + i;
        if (kk < tile0 || kk >= nk) continue;
        T s = red[0][i];
        for (int q = 1; q < SL; ++q) s += red[q][i];
        dst[kk] = s;
    }
}

// ---------------------------------------------------------------------------
// k_march1: the FP32 march of single-direction, cell-valued bundles (the
// axisymmetric lines of sight), the hot kernel of the afterbody.
//
// Same work and results contract as k_march<float, 2, 1, 8>, organised for
// fewer instructions per segment-wavelength:
//  * lane l owns two ADJACENT columns (base + 2l, base + 2l + 1): one 8-byte
//    load fetches both, for kappa and for j (a warp reads 256 contiguous
//    bytes of a row);
//  * node values are carried doubled (K = kappa_a + kappa_b, the sum of the
//    two cells at a face), with the segment length halved to match, which
//    removes the averaging multiplies;
//  * optically thin steps (|dtau| < 0.5) use I' = I + s f (j_f - kappa_f I)
//    + s p (j_n - j_f), with p = (1 - f)/dtau from one degree-6 series and
//    f = 1 - dtau p: one polynomial instead of two and no exponential.  With
//    e = 1 - dtau f >= 0.6 the subtraction inside costs at most a factor
//    1/e of relative rounding, so it stays in FP32 accuracy.  Thick steps use
//    the exponential form I' = I e + s f j_f + s p (j_n - j_f) with
//    f = (1 - e)/dtau, p = (1 - f)/dtau;
//  * the staged list holds, for step j, the segment's halved length (as the
//    packed pair the step multiplies by) and the byte offset of the row of the
//    cell PF steps ahead (row x ld, computed once by the staging lane), so a
//    step does no address arithmetic beyond adding that offset to its lane's
//    base; each step issues the loads it will use PF steps later and no load
//    is exposed at the 32-segment staging seams;
//  * the bundles of a block are dealt to its eight warps longest first
//    (k_march_plan), so the warps finish together at the block's reduction.
// Every slice still Kahan-sums its bundles in a fixed order and the slices
// and groups are added in fixed order: results do not depend on timing.
// Conditions (checked by the launcher): kappa, emis and the wall row 8-byte
// aligned, ld and nk even, nk >= 64.

#ifndef RAPRAL_M1_PF
#define RAPRAL_M1_PF 2
#endif
#ifndef RAPRAL_M1_UNROLL
#define RAPRAL_M1_UNROLL 4
#endif
constexpr int M1_PF = RAPRAL_M1_PF;            // steps between a load and its use
constexpr int kM1Unroll = RAPRAL_M1_UNROLL;    // segment steps unrolled
constexpr int M1_SLICES = 8;    // warps (bundle slices) per block

struct __align__(16) M1Stage {
    float2 sh;      // half the segment length (x the direction scale), twice: a packed pair
    int64_t off;    // byte offset of the row of the cell step j + M1_PF needs (its next cell); 0 past the end
};

// The thin-step series p(t) = (1 - f)/t = sum_n (-t)^n / (n + 2)!, n = 0..6
// (truncation below 4e-8 relative at |t| = 0.5), on a packed pair.
__device__ __forceinline__ float2 m1_series(float2 t) {
    const auto c2 = [](float c) { return make_float2(c, c); };
    float2 p = __ffma2_rn(t, c2(1.0f / 40320.0f), c2(-1.0f / 5040.0f));
    p = __ffma2_rn(t, p, c2(1.0f / 720.0f));
    p = __ffma2_rn(t, p, c2(-1.0f / 120.0f));
    p = __ffma2_rn(t, p, c2(1.0f / 24.0f));
    p = __ffma2_rn(t, p, c2(-1.0f / 6.0f));
    return __ffma2_rn(t, p, c2(0.5f));
}

// One step of one column with doubled node values Kf, Jf (far), Jn (near) and
// half length sh: the thin or the thick form by |t|.
__device__ __forceinline__ float m1_step1(float I, float Kf, float Jf, float Jn, float sh) {
    const float t = Kf * sh;   // kappa_far x length
    if (fabsf(t) < (float)RAPRAL_THIN_F32) {
        float p = fmaf(t, 1.0f / 40320.0f, -1.0f / 5040.0f);
        p = fmaf(t, p, 1.0f / 720.0f);
        p = fmaf(t, p, -1.0f / 120.0f);
        p = fmaf(t, p, 1.0f / 24.0f);
        p = fmaf(t, p, -1.0f / 6.0f);
        p = fmaf(t, p, 0.5f);
        const float f = fmaf(-t, p, 1.0f);
        const float A = fmaf(-Kf, I, Jf);
        return fmaf(sh, fmaf(f, A, p * (Jn - Jf)), I);
    }
    const float e = ex2f_approx(-1.44269504f * t);
    const float r = recip(t);
    const float f = (1.0f - e) * r;
    const float p = (1.0f - f) * r;
    return fmaf(sh, fmaf(f, Jf, p * (Jn - Jf)), I * e);
}

// One step of both columns: packed when both are thin.
__device__ __forceinline__ void m1_step(float2& I, float2 Kf, float2 Jf, float2 Jn, float2 sh2) {
    const float sh = sh2.x;
    const float2 t = __fmul2_rn(Kf, sh2);
    if (fmaxf(fabsf(t.x), fabsf(t.y)) < (float)RAPRAL_THIN_F32) {
        const float2 p = m1_series(t);
        const float2 f = __ffma2_rn(make_float2(-t.x, -t.y), p, make_float2(1.0f, 1.0f));
        const float2 A = __ffma2_rn(make_float2(-Kf.x, -Kf.y), I, Jf);
        const float2 dJ = __fadd2_rn(Jn, make_float2(-Jf.x, -Jf.y));
        const float2 B = __ffma2_rn(f, A, __fmul2_rn(p, dJ));
        I = __ffma2_rn(sh2, B, I);
    } else {
        I.x = m1_step1(I.x, Kf.x, Jf.x, Jn.x, sh);
        I.y = m1_step1(I.y, Kf.y, Jf.y, Jn.y, sh);
    }
}

// Bundle plan: for each (point p, group g) the group's bundles (a contiguous
// run of the point's bundles: with the rays of a point in angular order, the
// neighbours a block marches cross the same cells near the point, which L1
// then serves) dealt to M1_SLICES slices longest first (greedy to the
// least-loaded slice, ties to the lower slice; equal lengths in index order).  plan[] lists each group's bundles slice by slice, starting at the
// group's base; soff[(p G + g)(M1_SLICES + 1) + s] is where slice s starts.
// Groups of more than 1024 bundles are dealt round-robin in index order.
__global__ void __launch_bounds__(128) k_march_plan(const int64_t* __restrict__ point_off,
                                                    const int64_t* __restrict__ seg_off, int G,
                                                    int32_t* __restrict__ plan, int32_t* __restrict__ soff) {
    const int64_t p = blockIdx.x / G;
    const int g = (int)(blockIdx.x % G);
    const int64_t pb0 = point_off[p];
    const int64_t nb = point_off[p + 1] - pb0;
    const int64_t m = nb > g ? (nb - g + G - 1) / G : 0;                     // bundles of this group
    const int64_t base = pb0 + (int64_t)g * (nb / G) + (g < nb % G ? g : nb % G);   // the group's first bundle
    int32_t* so = soff + blockIdx.x * (M1_SLICES + 1);
    __shared__ int64_t len[1024];
    __shared__ int16_t order[1024];
    __shared__ int8_t slice_of[1024];
    __shared__ int32_t cnt[M1_SLICES + 1];
    if (m > 1024) {   // round-robin in index order
        for (int64_t k = threadIdx.x; k < m; k += blockDim.x) {
            const int s = (int)(k % M1_SLICES);
            const int64_t per = m / M1_SLICES, extra = m % M1_SLICES;
            const int64_t start = s * per + (s < extra ? s : extra);
            plan[base + start + k / M1_SLICES] = (int32_t)(base + k);
        }
        if (threadIdx.x <= M1_SLICES) {
            const int s = threadIdx.x;
            const int64_t per = m / M1_SLICES, extra = m % M1_SLICES;
            so[s] = (int32_t)(base + s * per + (s < extra ? s : extra));
        }
        return;
    }
    const int mm = (int)m;
    for (int k = threadIdx.x; k < mm; k += blockDim.x) {
        const int64_t b = base + k;
        len[k] = seg_off[b + 1] - seg_off[b];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < mm; k += blockDim.x) {   // rank: longer first, then lower index
        const int64_t lk = len[k];
        int r = 0;
        for (int q = 0; q < mm; ++q) r += (len[q] > lk) || (len[q] == lk && q < k);
        order[r] = (int16_t)k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t load[M1_SLICES];
        for (int s = 0; s < M1_SLICES; ++s) { load[s] = 0; cnt[s] = 0; }
        for (int r = 0; r < mm; ++r) {
            const int k = order[r];
            int best = 0;
            for (int s = 1; s < M1_SLICES; ++s) best = load[s] < load[best] ? s : best;
            slice_of[k] = (int8_t)best;
            load[best] += len[k] + 1;
            ++cnt[best];
        }
        int acc = 0;
        for (int s = 0; s < M1_SLICES; ++s) { const int c = cnt[s]; cnt[s] = acc; acc += c; }
        cnt[M1_SLICES] = acc;
        for (int s = 0; s <= M1_SLICES; ++s) so[s] = (int32_t)(base + cnt[s]);
        // each slice's bundles, longest first
        int fill[M1_SLICES];
        for (int s = 0; s < M1_SLICES; ++s) fill[s] = cnt[s];
        for (int r = 0; r < mm; ++r) {
            const int k = order[r];
            plan[base + fill[slice_of[k]]++] = (int32_t)(base + k);
        }
    }
}

// A lane's 2 NP adjacent columns of one row, as NP packed pairs.
template <int NP> struct M1V { float2 v[NP]; };

// The lane's columns of one row: one 8-byte (NP = 1) or 16-byte (NP = 2)
// load when the columns are aligned (VEC), else one 4-byte load a column at
// the offsets dq[] from the first (columns past the range repeat the last).
template <int NP, bool VEC>
__device__ __forceinline__ M1V<NP> m1_load(const float* __restrict__ p, const int (&dq)[2 * NP]) {
    M1V<NP> r;
    if constexpr (VEC && NP == 1) {
        r.v[0] = *reinterpret_cast<const float2*>(p);
    } else if constexpr (VEC) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        r.v[0] = make_float2(x.x, x.y);
        r.v[1] = make_float2(x.z, x.w);
    } else {
#pragma unroll
        for (int q = 0; q < NP; ++q) r.v[q] = make_float2(p[dq[2 * q]], p[dq[2 * q + 1]]);
    }
    return r;
}

template <int NP>
__device__ __forceinline__ M1V<NP> m1_sum(const M1V<NP>& x, const M1V<NP>& y) {
    M1V<NP> r;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.v[q] = __fadd2_rn(x.v[q], y.v[q]);
    return r;
}

// The lane's columns of one row of kappa and of emis: kb, jb point at the
// lane's first column in row 0, off is the row's byte offset.
template <int NP, bool VEC>
__device__ __forceinline__ M1V<NP> m1_rowload(const char* kb, const char* jb, int64_t off, const int (&dq)[2 * NP],
                                              M1V<NP>& j) {
    j = m1_load<NP, VEC>(reinterpret_cast<const float*>(jb + off), dq);
    return m1_load<NP, VEC>(reinterpret_cast<const float*>(kb + off), dq);
}

// The march of bundle b over the lane's columns (doubled node values).
template <int NP, bool VEC>
__device__ __forceinline__ M1V<NP> m1_bundle(const MarchArgs& a, int64_t b, float sc, M1Stage* st, int lane,
                                             const char* __restrict__ kb, const char* __restrict__ jb,
                                             const int (&dq)[2 * NP], int64_t ldb, M1V<NP> I) {
    const int64_t s0 = a.seg_off[b], s1 = a.seg_off[b + 1];
    if (s1 <= s0) return I;
    M1V<NP> kc, jc;
    kc = m1_rowload<NP, VEC>(kb, jb, (int64_t)a.seg_cell[s0] * ldb, dq, jc);
    M1V<NP> Kf = m1_sum(kc, kc), Jf = m1_sum(jc, jc);
    const float hs = 0.5f * sc;
    // ring of loads in flight: values of the next cells of the following PF segments
    M1V<NP> rk[M1_PF], rj[M1_PF];
#pragma unroll
    for (int q = 0; q < M1_PF; ++q) {
        const int64_t i = s0 + q;   // segment i's next cell is cell i + 1
        const int c = (i < s1 - 1) ? a.seg_cell[i + 1] : 0;
        rk[q] = m1_rowload<NP, VEC>(kb, jb, (int64_t)c * ldb, dq, rj[q]);
    }
    for (int64_t g = s0; g < s1 - 1; g += 32) {
        const int64_t mine = g + lane;
        __syncwarp();
        const int64_t ahead = mine + M1_PF;   // the segment whose next cell this entry fetches
        const float shl = mine < s1 - 1 ? seg_len<float>(a, mine) * hs : 0.0f;
        st[lane].sh = make_float2(shl, shl);
        st[lane].off = ahead < s1 - 1 ? (int64_t)a.seg_cell[ahead + 1] * ldb : 0;
        __syncwarp();
        const int n = s1 - 1 - g < 32 ? (int)(s1 - 1 - g) : 32;
#pragma unroll kM1Unroll
        for (int j = 0; j < n; ++j) {
            const M1Stage e = st[j];
            const M1V<NP> kx = rk[0], jx = rj[0];
#pragma unroll
            for (int q = 0; q + 1 < M1_PF; ++q) { rk[q] = rk[q + 1]; rj[q] = rj[q + 1]; }
            rk[M1_PF - 1] = m1_rowload<NP, VEC>(kb, jb, e.off, dq, rj[M1_PF - 1]);
            const M1V<NP> Kn = m1_sum(kc, kx), Jn = m1_sum(jc, jx);
#pragma unroll
            for (int q = 0; q < NP; ++q) m1_step(I.v[q], Kf.v[q], Jf.v[q], Jn.v[q], e.sh);
            Kf = Kn; Jf = Jn; kc = kx; jc = jx;
        }
    }
    {   // last segment: its near node is its own cell's value
        const float hl = seg_len<float>(a, s1 - 1) * hs;
        const M1V<NP> Jn = m1_sum(jc, jc);
#pragma unroll
        for (int q = 0; q < NP; ++q) m1_step(I.v[q], Kf.v[q], Jf.v[q], Jn.v[q], make_float2(hl, hl));
    }
    return I;
}

// Stores of a lane's columns: one vector store when aligned and owned, else
// one 4-byte store a column it owns.
template <int NP, bool VEC>
__device__ __forceinline__ void m1_store(float* __restrict__ p, const M1V<NP>& x, const bool (&own)[2 * NP]) {
    if constexpr (VEC && NP == 1) {
        if (own[0]) *reinterpret_cast<float2*>(p) = x.v[0];
    } else if constexpr (VEC) {
        if (own[0]) *reinterpret_cast<float4*>(p) = make_float4(x.v[0].x, x.v[0].y, x.v[1].x, x.v[1].y);
    } else {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            if (own[2 * q]) p[2 * q] = x.v[q].x;
            if (own[2 * q + 1]) p[2 * q + 1] = x.v[q].y;
        }
    }
}

// Block (point, bundle group) x tile of 64 NP columns; warp w is slice w of
// the group's plan; lane l owns the 2 NP adjacent columns from 2 NP l.  The
// last tile is shifted back to end at nk when nk >= the tile (columns below
// the tile are computed again and not written); a range shorter than a tile
// clamps the reads of lanes past it and writes nothing there.
template <int NP, bool VEC>
__global__ void __launch_bounds__(256, RAPRAL_MARCH_MINB) k_march1(MarchArgs a, int lgG, const int32_t* __restrict__ plan,
                                                                   const int32_t* __restrict__ soff,
                                                                   float* __restrict__ part) {
    if (*a.status) return;
    constexpr int TW = 64 * NP, SLC = M1_SLICES, NC = 2 * NP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nk = (int)a.nk;
    const int tile0 = (int)blockIdx.y * TW;
    const int base = (tile0 + TW > nk && nk >= TW) ? nk - TW : tile0;
    const int col = base + NC * lane;                 // the lane's columns: col .. col + NC - 1
    const int c0 = col < nk ? col : nk - 1;           // clamped reads (VEC: never clamped)
    int dq[NC];
    bool own[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        dq[q] = (col + q < nk ? col + q : nk - 1) - c0;
        own[q] = col + q >= tile0 && col + q < nk;
    }
    const char* kb = reinterpret_cast<const char*>(reinterpret_cast<const float*>(a.kappa) + c0);
    const char* jb = reinterpret_cast<const char*>(reinterpret_cast<const float*>(a.emis) + c0);
    __shared__ M1Stage stage_all[SLC][32];
    M1Stage* st = stage_all[warp];
    M1V<NP> acc, comp;
#pragma unroll
    for (int q = 0; q < NP; ++q) acc.v[q] = comp.v[q] = make_float2(0.f, 0.f);
    const int32_t* so = soff + (int64_t)blockIdx.x * (SLC + 1);
    const int k1 = so[warp + 1];
    for (int k = so[warp]; k < k1; ++k) {
        const int64_t b = plan[k];
        const int64_t d0 = a.dir_off[b];
        if (a.dir_off[b + 1] == d0) continue;
        M1V<NP> I0;
#pragma unroll
        for (int q = 0; q < NP; ++q) I0.v[q] = make_float2(0.f, 0.f);
        if (a.wall_row && a.bundle_wall[b]) I0 = m1_load<NP, VEC>(reinterpret_cast<const float*>(a.wall_row) + c0, dq);
        const M1V<NP> I = m1_bundle<NP, VEC>(a, b, a.dir_scale_f[d0], st, lane, kb, jb, dq, a.ld * 4, I0);
        if (a.I_out) m1_store<NP, VEC>(reinterpret_cast<float*>(a.I_out) + d0 * a.nk + col, I, own);
        const float w = a.dir_weight_f[d0];
#pragma unroll
        for (int q = 0; q < NP; ++q) {   // compensated sum over the slice's bundles
            const float2 y = make_float2(w * I.v[q].x - comp.v[q].x, w * I.v[q].y - comp.v[q].y);
            const float2 tt = make_float2(acc.v[q].x + y.x, acc.v[q].y + y.y);
            comp.v[q] = make_float2((tt.x - acc.v[q].x) - y.x, (tt.y - acc.v[q].y) - y.y);
            acc.v[q] = tt;
        }
    }
    __shared__ M1V<NP> red[SLC][32];
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        M1V<NP> sum = red[0][lane];
        for (int w = 1; w < SLC; ++w) {
#pragma unroll
            for (int q = 0; q < NP; ++q)
                sum.v[q] = make_float2(sum.v[q].x + red[w][lane].v[q].x, sum.v[q].y + red[w][lane].v[q].y);
        }
        float* dst = (lgG == 0 ? reinterpret_cast<float*>(a.q_lambda) : part) + (int64_t)blockIdx.x * a.nk + col;
        m1_store<NP, VEC>(dst, sum, own);
    }
}

// Planck intensity at the wall temperature for the columns of a range.
template <class T>
__global__ void k_planck_row(double lam_min, double h, int64_t k0, int64_t nk, double T_wall, Phys ph, T* row) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nk; k += (int64_t)gridDim.x * blockDim.x)
        row[k] = (T)planck(lam_min + (double)(k0 + k) * h, T_wall, ph);
}

// q_lambda[p][k] = sum of the G bundle-group partials of point p, in group order.
template <class T>
__global__ void k_group_sum(const T* __restrict__ part, int G, int64_t P, int64_t nk, T* __restrict__ q,
                            const int* status) {
    if (*status) return;
    const int64_t n = P * nk;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / nk, k = i - p * nk;
        const T* src = part + p * G * nk + k;
        T s = src[0];
        for (int g = 1; g < G; ++g) s += src[g * nk];
        q[i] = s;
    }
}

// Spectral integral in two deterministic stages: blocks (point, slice)
// Neumaier-sum a slice of FLUX_SPAN grid points each, then one block per
// point adds the slices in order.
constexpr int FLUX_SPAN = 4096;

template <class T>
__global__ void __launch_bounds__(256) k_wall_flux_part(const T* __restrict__ qlam, int64_t nk, int64_t k0,
                                                        int64_t n, double h_um, double2* __restrict__ part,
                                                        const int* status) {
    if (*status) return;
    const int64_t p = blockIdx.x;
    const int64_t a = (int64_t)blockIdx.y * FLUX_SPAN, b = min(a + FLUX_SPAN, nk);
    double s = 0.0, c = 0.0;
    for (int64_t k = a + threadIdx.x; k < b; k += blockDim.x) {
        const int64_t kg = k0 + k;
        const double w = (kg == 0 || kg == n - 1) ? 0.5 : 1.0;
        const double x = w * (double)qlam[p * nk + k] * h_um;
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
        s = t;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s + c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[p * gridDim.y + blockIdx.y] = make_double2(red[0], 0.0);
}

__global__ void __launch_bounds__(32) k_wall_flux_sum(const double2* __restrict__ part, int nparts,
                                                      double* __restrict__ q, const int* status) {
    if (*status) return;
    const int64_t p = blockIdx.x;
    if (threadIdx.x == 0) {
        double s = 0.0, c = 0.0;
        for (int i = 0; i < nparts; ++i) {
            const double x = part[p * nparts + i].x;
            const double t = s + x;
            if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
            s = t;
        }
        q[p] += s + c;
    }
}

// Tangent slab: directions are split into bundles of at most SLAB_DIRS
// (the normal ray first); every bundle repeats the cell path.
__global__ void k_slab_rays(const int32_t* cell_order, const double* dx, int32_t m, const double* mu,
                            const double* wmu, int32_t n_mu, int32_t normal_ray, int32_t wall_start,
                            int64_t* point_off, int64_t* seg_off, int32_t* seg_cell, double* seg_ds,
                            int64_t* dir_off, double* dir_scale, double* dir_weight, int32_t* bundle_wall) {
    const int nd = n_mu + (normal_ray ? 1 : 0);
    const int nb = (nd + RAPRAL_SLAB_DIRS - 1) / RAPRAL_SLAB_DIRS;
    for (int64_t i = threadIdx.x; i < (int64_t)m * nb; i += blockDim.x) {
        const int64_t j = i % m;
        seg_cell[i] = cell_order[j];
        seg_ds[i] = dx[j];
    }
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        if (normal_ray && d == 0) { dir_scale[0] = 1.0; dir_weight[0] = 0.0; continue; }
        const int mm = d - (normal_ray ? 1 : 0);
        dir_scale[d] = 1.0 / mu[mm];
        dir_weight[d] = 2.0 * M_PI * wmu[mm] * mu[mm];
    }
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) {
        seg_off[b] = (int64_t)b * m;
        dir_off[b] = min(b * RAPRAL_SLAB_DIRS, nd);
        if (b < nb) bundle_wall[b] = wall_start;
    }
    if (threadIdx.x == 0) { point_off[0] = 0; point_off[1] = nb; }
}

__device__ __forceinline__ void ray_dir(int64_t b, int32_t n_mu, int32_t n_phi, const double* mu, int64_t* p,
                                        int* m, double* dx, double* dn, double* dt) {
    const int64_t per = (int64_t)n_mu * n_phi;
    *p = b / per;
    const int64_t rem = b - *p * per;
    *m = (int)(rem / n_phi);
    const int a = (int)(rem - (int64_t)(*m) * n_phi);
    const double mm = mu[*m];
    const double st = sqrt(1.0 - mm * mm);
    const double psi = (a + 0.5) * (2.0 * M_PI / n_phi);
    *dx = st * cos(psi);
    *dn = mm;
    *dt = st * sin(psi);
}

__global__ void k_axisym_count(const double* xf, int32_t nx, const double* rf, int32_t nr, const double* surf_x,
                               int32_t P, const double* mu, int32_t n_mu, int32_t n_phi, int64_t* counts) {
    const int64_t B = (int64_t)P * n_mu * n_phi;
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B) return;
    int64_t p; int m; double dx, dn, dt;
    ray_dir(b, n_mu, n_phi, mu, &p, &m, &dx, &dn, &dt);
    counts[b] = walk_ray(xf, nx, rf, nr, surf_x[p], rf[0], dx, dn, dt, nullptr, nullptr, 0);
}

__global__ void k_axisym_fill(const double* xf, int32_t nx, const double* rf, int32_t nr, const double* surf_x,
                              int32_t P, const double* mu, const double* wmu, int32_t n_mu, int32_t n_phi,
                              const int64_t* seg_off, int32_t* seg_cell, double* seg_ds, int64_t* point_off,
                              int64_t* dir_off, double* dir_scale, double* dir_weight, int32_t* bundle_wall) {
    const int64_t B = (int64_t)P * n_mu * n_phi;
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b > B) return;
    dir_off[b] = b;
    if (b <= P) point_off[b] = b * (int64_t)n_mu * n_phi;
    if (b == B) return;
    int64_t p; int m; double dx, dn, dt;
    ray_dir(b, n_mu, n_phi, mu, &p, &m, &dx, &dn, &dt);
    walk_ray(xf, nx, rf, nr, surf_x[p], rf[0], dx, dn, dt, seg_cell, seg_ds, seg_off[b + 1]);
    dir_scale[b] = 1.0;
    dir_weight[b] = wmu[m] * mu[m] * (2.0 * M_PI / n_phi);
    bundle_wall[b] = 0;
}

#ifndef RAPRAL_MARCH_V
#define RAPRAL_MARCH_V 2
#endif

template <class T, int V, int MAXD, int SL, bool NODES = false>
cudaError_t march_launch(rapral_ctx* ctx, const MarchArgs& a, int64_t P, int64_t nk, int G, void* part) {
    constexpr int TW = (8 / SL) * 32 * V;
    int lgG = 0;
    while ((1 << lgG) < G) ++lgG;
    MarchArgs b = a;
    b.wall_row = nullptr;
    if (a.T_wall > 0.0) {   // the wall row follows the group partials in the scratch
        T* row = reinterpret_cast<T*>(part) + (G > 1 ? P * G * nk : 0);
        k_planck_row<T><<<(unsigned)std::min<int64_t>(div_up(nk, 256), 1024), 256, 0, ctx->stream>>>(
            a.lam_min, a.h, a.k0, nk, a.T_wall, a.ph, row);
        b.wall_row = row;
    }
    dim3 g((unsigned)(P << lgG), div_up(nk, TW));
    k_march<T, V, MAXD, SL, NODES><<<g, 256, 0, ctx->stream>>>(b, lgG, reinterpret_cast<T*>(part));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || G == 1) return e;
    k_group_sum<T><<<(unsigned)std::min<int64_t>(div_up(P * nk, 256), 152 * 16), 256, 0, ctx->stream>>>(
        reinterpret_cast<const T*>(part), G, P, nk, reinterpret_cast<T*>(a.q_lambda), a.status);
    return cudaGetLastError();
}

// k_march1 applies: FP32 cell-valued single-direction bundles, eight or more
// a point, and the 8-byte alignment and even sizes of its paired columns.
static bool march1_applies(const MarchArgs& a, int maxd, int maxb, bool nodes) {
    return !nodes && maxd <= 1 && maxb >= 8 && a.ld <= 2147483647LL;
}

// Columns a lane owns in k_march1 (2 NP) and the tile width (64 NP).
#ifndef RAPRAL_M1_NP
#define RAPRAL_M1_NP 1
#endif
constexpr int kM1NP = RAPRAL_M1_NP;

// Vector loads and stores of 2 NP floats: every row of kappa / emis,
// q_lambda, I_out and the wall row starts aligned to 8 NP bytes, and the
// range is whole tiles or ends on a multiple of 2 NP columns past the first
// tile.
static bool march1_vec(const MarchArgs& a, int64_t nk, const void* part) {
    const unsigned al = 8u * kM1NP - 1u;
    const auto ok = [al](const void* q) { return (reinterpret_cast<uintptr_t>(q) & al) == 0; };
    const int64_t nc = 2 * kM1NP;
    return nk >= 64 * kM1NP && nk % nc == 0 && a.ld % nc == 0 && ok(a.kappa) && ok(a.emis) && ok(a.q_lambda) &&
           ok(part) && (a.I_out == nullptr || ok(a.I_out));
}

static cudaError_t march1_launch(rapral_ctx* ctx, const MarchArgs& a, int64_t P, int64_t nk, int G, void* part,
                                 int32_t* plan, int32_t* soff) {
    int lgG = 0;
    while ((1 << lgG) < G) ++lgG;
    k_march_plan<<<(unsigned)(P * G), 128, 0, ctx->stream>>>(a.point_off, a.seg_off, G, plan, soff);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    MarchArgs b = a;
    b.wall_row = nullptr;
    if (a.T_wall > 0.0) {   // the wall row follows the group partials in the scratch
        float* row = reinterpret_cast<float*>(part) + (G > 1 ? P * G * nk : 0);
        k_planck_row<float><<<(unsigned)std::min<int64_t>(div_up(nk, 256), 1024), 256, 0, ctx->stream>>>(
            a.lam_min, a.h, a.k0, nk, a.T_wall, a.ph, row);
        b.wall_row = row;
    }
    dim3 g((unsigned)(P << lgG), div_up(nk, 64 * kM1NP));
    if (march1_vec(a, nk, part))
        k_march1<kM1NP, true><<<g, 32 * M1_SLICES, 0, ctx->stream>>>(b, lgG, plan, soff, reinterpret_cast<float*>(part));
    else
        k_march1<kM1NP, false><<<g, 32 * M1_SLICES, 0, ctx->stream>>>(b, lgG, plan, soff, reinterpret_cast<float*>(part));
    e = cudaGetLastError();
    if (e != cudaSuccess || G == 1) return e;
    k_group_sum<float><<<(unsigned)std::min<int64_t>(div_up(P * nk, 256), 152 * 16), 256, 0, ctx->stream>>>(
        reinterpret_cast<const float*>(part), G, P, nk, reinterpret_cast<float*>(a.q_lambda), a.status);
    return cudaGetLastError();
}

// Eight bundle slices for eight or more bundles a point, else one; V > 1
// columns a lane only for one-direction bundles in FP32 and ranges of at
// least one tile.
template <class T>
cudaError_t march_t(rapral_ctx* ctx, const MarchArgs& a, int64_t P, int64_t nk, int maxd, int maxb, int G,
                    void* part, bool nodes) {
    constexpr int VR = sizeof(T) == 4 ? RAPRAL_MARCH_V : 1;
    if (nodes) {   // node-valued lines of sight: one direction a bundle (checked by the caller)
        if (maxb < 8) return march_launch<T, 1, 1, 1, true>(ctx, a, P, nk, G, part);
        if (VR > 1 && nk >= 32 * VR) return march_launch<T, VR, 1, 8, true>(ctx, a, P, nk, G, part);
        return march_launch<T, 1, 1, 8, true>(ctx, a, P, nk, G, part);
    }
    if (maxb >= 8) {
        if (maxd <= 1) {
            if (VR > 1 && nk >= 32 * VR) return march_launch<T, VR, 1, 8>(ctx, a, P, nk, G, part);
            return march_launch<T, 1, 1, 8>(ctx, a, P, nk, G, part);
        }
        if (maxd <= 17) return march_launch<T, 1, 17, 8>(ctx, a, P, nk, G, part);
        return march_launch<T, 1, RAPRAL_MAX_DIRS, 8>(ctx, a, P, nk, G, part);
    }
    if (maxd <= 1) return march_launch<T, 1, 1, 1>(ctx, a, P, nk, G, part);
    if (maxd <= 17) return march_launch<T, 1, 17, 1>(ctx, a, P, nk, G, part);
    return march_launch<T, 1, RAPRAL_MAX_DIRS, 1>(ctx, a, P, nk, G, part);
}

}  // namespace

cudaError_t launch_validate_rays(rapral_ctx* ctx, const rapral_rays* r, int64_t n_cells) {
    const int64_t n = r->n_segments > r->n_dirs ? r->n_segments : r->n_dirs;
    if (n == 0) return cudaSuccess;
    k_validate_rays<<<div_up(n, 256), 256, 0, ctx->stream>>>(r->seg_cell, r->seg_ds, r->n_segments, n_cells,
                                                            r->dir_scale, r->n_dirs, ctx->d_status);
    return cudaGetLastError();
}

// Bundle groups per point where a point has eight or more bundles (a power of two):
// enough blocks share a wavelength tile (points x groups >= 1536, about two
// waves of resident blocks) that the tiles in flight, and so the kappa / j
// rows they gather, stay few enough for L2; each group keeps at least 32
// bundles, and points x groups stays below 2^31.
#ifndef RAPRAL_MARCH_TILE_BLOCKS
#define RAPRAL_MARCH_TILE_BLOCKS 1536
#endif
static int march_groups(const rapral_rays* r) {
    if (r->max_bundles_per_point < 8 || r->n_points <= 0) return 1;
    int G = 1;
    while (G * r->n_points < RAPRAL_MARCH_TILE_BLOCKS && 2 * G * 32 <= r->max_bundles_per_point && G < 1024 &&
           2 * G * r->n_points < (int64_t)1 << 31)
        G *= 2;
    return G;
}

static size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// FP32 scratch: the FP32 copies, then k_march1's bundle plan and slice starts.
static size_t march_plan_bytes(const rapral_rays* r) {
    return round256((size_t)(r->n_bundles + (int64_t)r->n_points * march_groups(r) * (M1_SLICES + 1) + 64) *
                    sizeof(int32_t));
}

size_t march_scratch_bytes(const rapral_rays* r, int64_t nk, int precision) {
    size_t bytes = 0;
    if (precision == RAPRAL_FP32)
        bytes = round256((size_t)(r->n_segments + 2 * r->n_dirs + 128) * sizeof(float)) + march_plan_bytes(r);
    const int G = march_groups(r);
    const size_t el = precision == RAPRAL_FP64 ? sizeof(double) : sizeof(float);
    if (G > 1) bytes += (size_t)r->n_points * G * nk * el;
    return bytes + nk * el + 256;   // + the wall's Planck row
}

cudaError_t launch_march(rapral_ctx* ctx, const rapral_rays* r, const void* kappa, const void* emis, int64_t ld,
                         const rapral_grid* g, double h, int64_t k0, int64_t nk, int precision, void* q_lambda,
                         void* I_out, const Phys& ph, void* scratch) {
    MarchArgs a;
    a.point_off = r->point_off; a.seg_off = r->seg_off; a.seg_cell = r->seg_cell; a.seg_ds = r->seg_ds;
    a.dir_off = r->dir_off; a.dir_scale = r->dir_scale; a.dir_weight = r->dir_weight;
    a.seg_ds_f = nullptr; a.dir_scale_f = nullptr; a.dir_weight_f = nullptr;
    a.bundle_wall = r->bundle_wall; a.T_wall = r->T_wall; a.wall_row = nullptr;
    a.kappa = kappa; a.emis = emis; a.ld = ld;
    a.lam_min = g->lam_min; a.h = h; a.k0 = k0; a.nk = nk;
    a.q_lambda = q_lambda; a.I_out = I_out; a.ph = ph; a.status = ctx->d_status;
    const int G = march_groups(r);
    if (precision == RAPRAL_FP64)
        return march_t<double>(ctx, a, r->n_points, nk, r->max_dirs, r->max_bundles_per_point, G, scratch,
                               r->node_values != 0);
    // FP32 copies of the path lengths, direction scales and weights, then the group partials
    float* f = reinterpret_cast<float*>(scratch);
    const size_t copies = round256((size_t)(r->n_segments + 2 * r->n_dirs + 128) * sizeof(float));
    int32_t* plan = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(scratch) + copies);
    int32_t* soff = plan + ((r->n_bundles + 63) / 64) * 64;
    void* part = reinterpret_cast<char*>(scratch) + copies + march_plan_bytes(r);
    float* fd = f + ((r->n_segments + 63) / 64) * 64;
    float* fw = fd + ((r->n_dirs + 63) / 64) * 64;
    if (r->n_segments > 0)
        k_to_float<<<(unsigned)std::min<int64_t>(div_up(r->n_segments, 256), 4096), 256, 0, ctx->stream>>>(
            r->seg_ds, r->n_segments, f);
    if (r->n_dirs > 0) {
        k_to_float<<<(unsigned)std::min<int64_t>(div_up(r->n_dirs, 256), 4096), 256, 0, ctx->stream>>>(
            r->dir_scale, r->n_dirs, fd);
        k_to_float<<<(unsigned)std::min<int64_t>(div_up(r->n_dirs, 256), 4096), 256, 0, ctx->stream>>>(
            r->dir_weight, r->n_dirs, fw);
    }
    a.seg_ds_f = f; a.dir_scale_f = fd; a.dir_weight_f = fw;
    if (march1_applies(a, r->max_dirs, r->max_bundles_per_point, r->node_values != 0))
        return march1_launch(ctx, a, r->n_points, nk, G, part, plan, soff);
    return march_t<float>(ctx, a, r->n_points, nk, r->max_dirs, r->max_bundles_per_point, G, part,
                          r->node_values != 0);
}

int64_t wall_flux_parts(int64_t nk) { return (nk + FLUX_SPAN - 1) / FLUX_SPAN; }

cudaError_t launch_wall_flux(rapral_ctx* ctx, const void* q_lambda, int precision, const rapral_grid* g, double h,
                             int64_t k0, int64_t nk, int64_t n_points, double* q, void* partials) {
    if (n_points == 0) return cudaSuccess;
    const double h_um = h * 1e-3;
    const int64_t np = wall_flux_parts(nk);
    double2* part = reinterpret_cast<double2*>(partials);
    dim3 grid((unsigned)n_points, (unsigned)np);
    if (precision == RAPRAL_FP64)
        k_wall_flux_part<double><<<grid, 256, 0, ctx->stream>>>(reinterpret_cast<const double*>(q_lambda), nk, k0,
                                                                g->n, h_um, part, ctx->d_status);
    else
        k_wall_flux_part<float><<<grid, 256, 0, ctx->stream>>>(reinterpret_cast<const float*>(q_lambda), nk, k0,
                                                               g->n, h_um, part, ctx->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_wall_flux_sum<<<(unsigned)n_points, 32, 0, ctx->stream>>>(part, (int)np, q, ctx->d_status);
    return cudaGetLastError();
}

cudaError_t launch_slab_rays(rapral_ctx* ctx, const int32_t* cell_order, const double* dx, int32_t m,
                             const double* mu, const double* wmu, int32_t n_mu, int32_t normal_ray,
                             int32_t wall_start, int64_t* point_off, int64_t* seg_off, int32_t* seg_cell,
                             double* seg_ds, int64_t* dir_off, double* dir_scale, double* dir_weight,
                             int32_t* bundle_wall) {
    k_slab_rays<<<1, 256, 0, ctx->stream>>>(cell_order, dx, m, mu, wmu, n_mu, normal_ray, wall_start, point_off,
                                           seg_off, seg_cell, seg_ds, dir_off, dir_scale, dir_weight, bundle_wall);
    return cudaGetLastError();
}

cudaError_t launch_axisym_count(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                                const double* surf_x, int32_t P, const double* mu, int32_t n_mu, int32_t n_phi,
                                int64_t* seg_off, int64_t* scan_tmp) {
    (void)scan_tmp;
    const int64_t B = (int64_t)P * n_mu * n_phi;
    if (B == 0) return cudaSuccess;
    k_axisym_count<<<div_up(B, 128), 128, 0, ctx->stream>>>(xf, nx, rf, nr, surf_x, P, mu, n_mu, n_phi, seg_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_scan_i64(ctx, seg_off, B);
}

cudaError_t launch_axisym_fill(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                               const double* surf_x, int32_t P, const double* mu, const double* wmu, int32_t n_mu,
                               int32_t n_phi, const int64_t* seg_off, int32_t* seg_cell, double* seg_ds,
                               int64_t* point_off, int64_t* dir_off, double* dir_scale, double* dir_weight,
                               int32_t* bundle_wall) {
    const int64_t B = (int64_t)P * n_mu * n_phi;
    k_axisym_fill<<<div_up(B + 1, 128), 128, 0, ctx->stream>>>(xf, nx, rf, nr, surf_x, P, mu, wmu, n_mu, n_phi,
                                                               seg_off, seg_cell, seg_ds, point_off, dir_off,
                                                               dir_scale, dir_weight, bundle_wall);
    return cudaGetLastError();
}
