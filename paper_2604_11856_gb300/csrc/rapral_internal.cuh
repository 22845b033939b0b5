// Internal declarations of librapral: context, workspace arena, status word,
// per-line and per-cell preparation records, and kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "rapral.h"
#include "voigt.cuh"

// ------------------------------------------------------------- constants ----

// Physical constants in cgs (Sec. 2.1 prints k, c, h with four digits).
struct Phys {
    double kB, c, h;
    double c2;        // h c / k, cm K
    double me, e;     // electron mass (g) and charge (esu), for oscillator strengths
};

inline Phys make_phys(int codata) {
    Phys p;
    if (codata) {
        p.kB = 1.380649e-16; p.c = 2.99792458e10; p.h = 6.62607015e-27; p.me = 9.1093837e-28; p.e = 4.80320471e-10;
    } else {
        p.kB = 1.380e-16; p.c = 2.998e10; p.h = 6.626e-27; p.me = 9.109e-28; p.e = 4.803e-10;
    }
    p.c2 = p.h * p.c / p.kB;
    return p;
}

// Optional Lorentz terms of Sec. 2.2.1 (rapral_set_broadening): flags
// RAPRAL_BROAD_*, per-species ionisation energies and per-column molar masses.
#define RAPRAL_MAX_COLS 32
#define RAPRAL_E_IONIZE_H 109678.77      // hydrogen ionisation energy, cm^-1
struct BroadArgs {
    int flags;
    int S, ncol;
    double Eion[RAPRAL_MAX_SPECIES];
    double colmass[RAPRAL_MAX_COLS];
};

// Sec. 2.2.1 constants.
#define RAPRAL_LAM_NATURAL 5.9e-6        // natural HWHM, nm
#define RAPRAL_DOPPLER_HALF (7.16233e-7 / 2.0)
#define RAPRAL_WINDOW 100.0              // lines reach |dlam| <= 100 lamV
#define RAPRAL_THIN_F64 4e-4             // |dtau| below which the series is used
#define RAPRAL_THIN_F32 0.5               // with seven-term series in FP32
#define RAPRAL_SLAB_DIRS 17              // directions per tangent-slab bundle

// Status word layout (device int[8]).
enum { ST_CODE = 0, ST_CHECK = 1, ST_INDEX = 2 };
enum {
    CHK_NONE = 0, CHK_CELL_T, CHK_CELL_N, CHK_LINE_SPECIES, CHK_LINE_LAM, CHK_LINE_G,
    CHK_LINE_A, CHK_SEG_CELL, CHK_SEG_DS, CHK_DIR, CHK_TIMEOUT, CHK_LOS_INDEX, CHK_CR_TRANS, CHK_CR_SINGULAR,
    CHK_CR_POP, CHK_DEP_LEVEL, CHK_CONT_TABLE
};

// ------------------------------------------------------------- records ----

// Per-line constants, independent of the cell.
struct __align__(16) LinePrep {
    double lam0;     // nm
    double tpos;     // (lam0 - lam_min) / h, grid units
    double lnAj;     // ln(1e-7 (hc/4pi) A / (lam0 1e-7))       ln S_j = lnAj + ln N_u
    double lnAk;     // ln(1e4 A (lam0 1e-7)^4 / (8 pi c))        S_k = e^{lnAk + ln N_u} expm1(x)
    double lngu;     // ln g_u
    double Eve_u;    // E_el + E_V of the upper level (at T_ve)
    double Er_u;     // E_J of the upper level (at T_tr)
    double Eve_l;    // E_el + E_V of the lower level
    double Er_l;     // E_J of the lower level
    double dEve;     // Eve_u - Eve_l
    double dEr;      // Er_u - Er_l
    double cD;       // Doppler: lamG = cD sqrt(T_tr)
    double lamS0;    // Stark HWHM at the reference state
    double lnAjg;    // lnAj + ln g_u
    double lnAkg;    // lnAk + ln g_u
    // FP32 copies for the chosen-precision path
    float dEve_f, dEr_f, cD_f, lamS0_f;
    float delta_f;   // tpos - kc
    int32_t kc;      // nearest grid index to lam0 (may lie outside the grid)
    int32_t species;
    int32_t pad;
};

// Compact per-line record of the FP32-chosen path.  The log-space terms are
// float-float pairs (hi + lo, about 44 significant bits): GB300's FP64 pipe
// is too narrow to run the per-(line, cell, tile) set-up in FP64, and pair
// arithmetic in the FP32 pipe keeps the same accuracy.
struct __align__(16) LineF32 {
    float2 lnAjg;    // lnAj + ln g_u
    float2 dAkj;     // lnAk - lnAj
    float2 Eve_u;    // E_el + E_V of the upper level
    float2 Er_u;     // E_J of the upper level
    float2 dEve;     // Eve_u - Eve_l
    float2 dEr;      // Er_u - Er_l
    float cD, lamS0, delta;
    int32_t kc, species;
    float kcf;       // kc as a float (exact for |kc| < 2^24)
};

// Per-cell constants.
struct __align__(16) CellPrep {
    double bve;      // c2 / T_ve
    double btr;      // c2 / T_tr
    double sqrtT;    // sqrt(T_tr)
    double stc;      // (T_ve/1e4)^0.33 (N_e/1e16)
    float bve_f, btr_f, sqrtT_f, stc_f;
    float2 bve_ff, btr_ff;   // float-float copies of bve, btr
};

// Float-float arithmetic (a value is hi + lo with |lo| <= ulp(hi)/2).
__host__ __device__ __forceinline__ float2 ff_from(double x) {
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb) + a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}
__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    const float e = fmaf(a.x, b.x, -p) + (a.x * b.y + a.y * b.x);
    const float hi = p + e;
    return make_float2(hi, e - (hi - p));
}

// ---------------------------------------------------------------- context ----

struct rapral_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int codata = 0;
    int tile_w = 0;            // grid points per line-sum tile (0: 512 for FP64, 128 for FP32)
    int cells_per_block = 4;   // warps (cells) per FP32 line-sum block
    int pairs_per_batch = 32;  // (line, cell) pairs a warp of the FP32 line sum stages per sweep pass (32 or 64)
    int ls_persist = -1;       // FP32 line sum: persistent with this many blocks a SM (-1: as many as fit; 0: a block a unit)
    // workspace arena (grown on demand; all users are stream-ordered)
    char* ws = nullptr;
    size_t ws_bytes = 0;
    // status word (device) and a pinned host mirror
    int* d_status = nullptr;
    int* h_pinned = nullptr;    // [16] pinned scratch for small read-backs
    unsigned long long* d_stats = nullptr;   // [4] line-sum work counters
    unsigned long long* d_unit = nullptr;    // the persistent line sum's unit counter (null: no persistent launch)
    int count_work = 1;                      // counters on (rapral_set_counters)
    cudaEvent_t ev_before = nullptr, ev_after = nullptr;   // optional timing events
    BroadArgs broad = {};                    // optional Lorentz terms (flags 0: off)
    // departure coefficients (rapral_set_departures; ln_b null: off)
    const double* dep_lnb = nullptr;
    const int32_t* dep_u = nullptr;
    const int32_t* dep_l = nullptr;
    int32_t dep_nlev = 0, dep_S = 0;
    int64_t dep_C = 0, dep_L = 0;
    int profile = 0;          // RAPRAL_PROFILE_WHITING or RAPRAL_PROFILE_VOIGT
    bool voigt_ready = false; // the expansion's coefficients are on this context's device
    char err[512] = {0};
};

// Records `msg` as the context's last error and returns `code`.
int set_error(rapral_ctx* ctx, int code, const char* fmt, ...);
// Wraps a CUDA call result.
int cuda_status(rapral_ctx* ctx, cudaError_t e, const char* what);
int read_status(rapral_ctx* ctx);   // sync, then the device status as an error code
// Ensures the arena holds `bytes`; may synchronise the stream.
int ws_reserve(rapral_ctx* ctx, size_t bytes);

// Bump allocator over the arena (256-byte aligned slices).
struct Arena {
    char* base;
    size_t cap, used = 0;
    template <class T>
    T* take(size_t n) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + n * sizeof(T);
        return reinterpret_cast<T*>(base + off);
    }
};
inline size_t arena_need(size_t cur, size_t bytes) { return ((cur + 255) & ~size_t(255)) + bytes; }

// Host-side check of a spectral grid and a range [k0, k0 + nk) of it: null
// when they are valid, else a message (static storage).  Every entry point
// that takes a grid uses this one check.
inline const char* grid_problem(const rapral_grid* g) {
    if (!g) return "null grid";
    if (g->n < 2 || !(g->lam_max > g->lam_min) || !(g->lam_min > 0.0) || !std::isfinite(g->lam_max))
        return "grid needs n >= 2 and 0 < lam_min < lam_max (finite)";
    return nullptr;
}
inline bool range_in_grid(const rapral_grid* g, int64_t k0, int64_t nk) {
    return k0 >= 0 && nk >= 1 && k0 <= g->n - nk;
}

// Grid launch helper.
inline unsigned div_up(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Device-side failure: first check wins.
__device__ __forceinline__ void fail(int* status, int check, long long index) {
    if (atomicCAS(&status[ST_CODE], 0, RAPRAL_EINVAL) == 0) {
        status[ST_CHECK] = check;
        status[ST_INDEX] = (int)(index > 2147483647LL ? 2147483647LL : index);
    }
}

// ------------------------------------------------------ kernel launchers ----
// (defined in the .cu files; all enqueue on ctx->stream)

cudaError_t launch_validate_cells(rapral_ctx* ctx, const rapral_cells* cells);
cudaError_t launch_populations(rapral_ctx* ctx, const rapral_species* sp, const rapral_cells* cells,
                               double* lnpref, const Phys& ph);
cudaError_t launch_validate_lines(rapral_ctx* ctx, const rapral_lines* ln, int32_t n_species);
// br: optional Lorentz terms (nullptr or flags 0: none); with resonance or van
// der Waals terms, lb / lb32 [L] receive per-line (c_R, c_W), the width
// gaining c_R N_0 + c_W W over the (cell, species) values of launch_broad_cells.
cudaError_t launch_line_prep(rapral_ctx* ctx, const rapral_species* sp, const rapral_lines* ln,
                             double lam_min, double h, const Phys& ph, LinePrep* out, LineF32* out32,
                             int* sorted_flag, const BroadArgs* br = nullptr, double2* lb = nullptr,
                             float2* lb32 = nullptr);
cudaError_t launch_cell_prep(rapral_ctx* ctx, const rapral_cells* cells, const Phys& ph, CellPrep* out,
                             unsigned long long* d_max /*[2 + 2 S]*/);
// Per (cell, species): ground-level density N_0 and van der Waals factor W
// (cb / cb32 [C][S]); their largest values over the cells go to
// d_max[2 + 2 s], d_max[3 + 2 s].  Needs the cells' lnpref.  g0: scratch [S].
cudaError_t launch_broad_cells(rapral_ctx* ctx, const rapral_species* sp, const rapral_cells* cells,
                               const BroadArgs& br, double* g0, double2* cb, float2* cb32,
                               unsigned long long* d_max);
// Whether the resonance or van der Waals terms are on.
inline bool broad_terms(const BroadArgs* br) { return br && (br->flags & (RAPRAL_BROAD_RESONANCE | RAPRAL_BROAD_VDW)); }

// Binning of lines into spectral tiles of the range [k0, k0 + nk).
struct BinPlan {
    int64_t k0, nk;
    int tile_w;
    int64_t n_tiles;
    int2* line_tiles;            // [L] first / last tile a line may touch (first > last: none)
    int* tile_off;               // [T+1]
    int* tile_lines;             // [tile_off[T]]
    long long* total;            // [1] exact number of (line, tile) entries (int64: may exceed the
                                 // int32 offsets; a plan with more than 2^31 - 1 is refused)
    int* sorted_flag;            // [1] 1 while lam0 is non-decreasing
    unsigned long long* wmax;    // [1] largest window half-width, grid points (double bits)
};
cudaError_t launch_bin_bounds(rapral_ctx* ctx, const rapral_lines* ln, const LinePrep* lp, const CellPrep* cp,
                              const unsigned long long* d_max, double h, BinPlan* plan,
                              const double2* lb = nullptr);
// Counts each tile's lines and scans the counts into plan->tile_off; the
// exact total goes to plan->total (device).
cudaError_t launch_bin_count(rapral_ctx* ctx, const rapral_lines* ln, const rapral_grid* g, double h,
                             BinPlan* plan);
// Largest number of (line, tile) entries a plan may hold: the tile lists are
// indexed by int32 offsets.
constexpr long long RAPRAL_MAX_TILE_ENTRIES = 2147483647LL;
cudaError_t launch_bin_fill(rapral_ctx* ctx, const rapral_lines* ln, const rapral_grid* g, double h,
                            BinPlan* plan);

struct LineSumArgs {
    const LinePrep* lp;
    const LineF32* lf;        // compact records (FP32 path)
    const CellPrep* cp;
    const double* lnpref;     // [C][S]
    int32_t S;
    int64_t C;
    const int* tile_off;
    const int* tile_lines;
    double lam_min, h;
    int64_t k0, nk, ld;
    int tile_w;
    void* kappa;
    void* emis;
    const int* status;
    unsigned long long* stats;   // [4] evaluations, gauss, correction, pairs
    int count;                   // accumulate the work counters (costs conversions per pair)
    // optional resonance / van der Waals terms (null: none): per line (c_R, c_W),
    // per (cell, species) (N_0, W)
    const double2* lb = nullptr;
    const float2* lb32 = nullptr;
    const double2* cb = nullptr;
    const float2* cb32 = nullptr;
    // optional departure coefficients (null: Boltzmann): ln b [C][S][dep_nlev],
    // level index of every line's upper / lower level (-1: none)
    const double* dep_lnb = nullptr;
    const int32_t* dep_u = nullptr;
    const int32_t* dep_l = nullptr;
    int32_t dep_nlev = 0;
    // exact Voigt line shape instead of Whiting's (rapral_set_profile; the
    // expansion's coefficients are in constant memory, see voigt_upload)
    int voigt = 0;
};

// Workspace of the optional resonance / van der Waals terms of one request:
// per-line factors, per-(cell, species) values, ground weights, and the
// maxima (after sqrt(T_tr) and the Stark factor) for the binning bound.
#define RAPRAL_DMAX_SLOTS (2 + 2 * RAPRAL_MAX_SPECIES)
inline size_t broad_need(size_t need, int64_t L, int64_t C, int S) {
    need = arena_need(need, (size_t)L * sizeof(double2));
    need = arena_need(need, (size_t)L * sizeof(float2));
    need = arena_need(need, (size_t)C * S * sizeof(double2));
    need = arena_need(need, (size_t)C * S * sizeof(float2));
    return arena_need(need, RAPRAL_MAX_SPECIES * sizeof(double));
}
cudaError_t launch_line_sum(rapral_ctx* ctx, const LineSumArgs& a, int precision, int64_t n_tiles);

// One request of a batched (persistent) line sum: its arguments and the
// first of its work units (tile-major, groups of WPB cells).
struct BatchItem {
    LineSumArgs a;
    int64_t unit_off;
    int64_t n_groups;   // cell groups per tile
};
// Launches the persistent FP32 line sum over all units (or only reports the
// grid size when `launch` is false).
cudaError_t launch_line_sum_batch(rapral_ctx* ctx, int tile_w, int wpb, int pb, const BatchItem* items, int n,
                                  int64_t total, unsigned long long* counter, int* blocks_out, bool launch, bool broad);

// Rays
cudaError_t launch_validate_rays(rapral_ctx* ctx, const rapral_rays* r, int64_t n_cells);
// The march needs march_scratch_bytes(r, nk, precision) of scratch (256-byte
// aligned): FP32 copies of the ray lengths, direction scales and weights
// (FP32 only), then per-group partial spectral fluxes where a point's
// bundles are split over several blocks.
size_t march_scratch_bytes(const rapral_rays* r, int64_t nk, int precision);
cudaError_t launch_march(rapral_ctx* ctx, const rapral_rays* r, const void* kappa, const void* emis,
                         int64_t ld, const rapral_grid* g, double h, int64_t k0, int64_t nk, int precision,
                         void* q_lambda, void* I_out, const Phys& ph, void* scratch);
// Spectral flux: needs `partials` of wall_flux_parts(nk) * n_points * 16 bytes.
int64_t wall_flux_parts(int64_t nk);
cudaError_t launch_wall_flux(rapral_ctx* ctx, const void* q_lambda, int precision, const rapral_grid* g,
                             double h, int64_t k0, int64_t nk, int64_t n_points, double* q, void* partials);
cudaError_t launch_slab_rays(rapral_ctx* ctx, const int32_t* cell_order, const double* dx, int32_t m,
                             const double* mu, const double* wmu, int32_t n_mu, int32_t normal_ray,
                             int32_t wall_start, int64_t* point_off, int64_t* seg_off, int32_t* seg_cell,
                             double* seg_ds, int64_t* dir_off, double* dir_scale, double* dir_weight,
                             int32_t* bundle_wall);
cudaError_t launch_axisym_count(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                                const double* surf_x, int32_t P, const double* mu, int32_t n_mu,
                                int32_t n_phi, int64_t* seg_off, int64_t* scan_tmp);
cudaError_t launch_axisym_fill(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                               const double* surf_x, int32_t P, const double* mu, const double* wmu,
                               int32_t n_mu, int32_t n_phi, const int64_t* seg_off, int32_t* seg_cell,
                               double* seg_ds, int64_t* point_off, int64_t* dir_off, double* dir_scale,
                               double* dir_weight, int32_t* bundle_wall);

// Exclusive scan of int64 counts in place over [0, n] (n + 1 entries; the
// last entry receives the total); single block.
cudaError_t launch_scan_i64(rapral_ctx* ctx, int64_t* data, int64_t n);

// Saha-Boltzmann prefactor of one atomic radiator into cells->lnpref (k_populations.cu).
cudaError_t launch_saha_prefactor(rapral_ctx* ctx, const rapral_cells* cells, int s, int S, double E_ion,
                                  int ion_col, int n_terms, const double* ion_E, const double* ion_g,
                                  const Phys& ph, double* lnpref);
// QSS collisional-radiative populations (k_qss.cu).
cudaError_t launch_qss(rapral_ctx* ctx, const rapral_cr_model* m, const rapral_cells* cells, double* n_out,
                       const Phys& ph);
// ln b of the model's levels for one species, and the check of a departure table's level indices.
cudaError_t launch_qss_departures(rapral_ctx* ctx, const rapral_cr_model* m, const rapral_cells* cells, int32_t s,
                                  int32_t S, const double* n_qss, double* ln_b, int32_t n_lev, const Phys& ph);
cudaError_t launch_check_levels(rapral_ctx* ctx, const int32_t* lev_u, const int32_t* lev_l, int64_t L,
                                int32_t n_lev);

// Fibonacci lines of sight, node states and the angular flux (k_los.cu).
cudaError_t launch_fib_count(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                             const double* surf_x, int32_t P, int32_t n_los, int64_t* seg_off);
cudaError_t launch_fib_fill(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                            const double* surf_x, int32_t P, int32_t n_los, const int64_t* seg_off,
                            int32_t* seg_cell, double* seg_ds, int64_t* point_off, int64_t* dir_off,
                            double* dir_scale, double* dir_weight, int32_t* bundle_wall, int32_t* los_index,
                            double* node_x, double* node_r);
cudaError_t launch_node_idw(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                            const rapral_cells* cells, int64_t n_nodes, const double* node_x, const double* node_r,
                            double* Ttr, double* Tve, double* n);
size_t fib_flux_scratch_bytes(int64_t P, int32_t n_los, int32_t n_phi, int32_t n_theta);
cudaError_t launch_fib_flux(rapral_ctx* ctx, int64_t P, const int64_t* point_off, const int32_t* los_index,
                            int32_t n_los, const double* S, int32_t n_phi, int32_t n_theta, double* q,
                            void* scratch);

// Coefficients of the rational Faddeeva expansion: computed once on the host,
// copied to the current device's constant memory by the first exact-Voigt
// call of each context.
const VoigtCoef& voigt_coefficients();
cudaError_t voigt_upload();
