/*
 * rapral.h -- C ABI of the GB300 (sm_103a) implementation of the RAPRAL hot
 * path (arXiv 2604.11856): two-temperature populations, line-by-line spectral
 * coefficients, the segment-wise RTE march and the wall radiative heat flux;
 * batched and allocation-free variants; and the optional parts of the method:
 * the Fibonacci lines of sight, the full Lorentz width and the exact Voigt
 * shape, quasi-steady-state collisional-radiative and Saha-Boltzmann
 * populations with departure coefficients, and the atomic continuum.
 *
 * Conventions (every entry point):
 *  - Returns an int status: RAPRAL_OK or one of the codes below.  No call
 *    aborts, traps or prints.  rapral_last_error() holds a message for the
 *    last failure of a context.
 *  - Array arguments are CALLER-OWNED DEVICE pointers (for example the
 *    data_ptr() of CUDA tensors) unless a comment says "host".  The library
 *    owns only the opaque context and its workspace (per-line constants, the
 *    line-binning tables and a status word); it never frees caller memory.
 *  - Work is enqueued asynchronously on the context's stream; outputs are
 *    valid once that stream has synchronised (rapral_sync()).  Arguments that
 *    can be checked on the host (sizes, ranges, null pointers) are checked
 *    before anything is enqueued and fail with RAPRAL_EINVAL at once.
 *    Checks of array CONTENTS (non-positive or non-finite temperatures,
 *    negative densities, out-of-range cell or species indices, negative path
 *    lengths) run on the device; a failure sets the context's sticky status,
 *    turns every later kernel of the context into a no-op, and is reported
 *    by rapral_sync() (and by the next call) as RAPRAL_EINVAL.
 *  - Units: T in K; number densities in cm^-3; energies in cm^-1;
 *    wavelengths in nm; path lengths in cm; kappa in cm^-1; j in
 *    W/cm^3/sr/um; intensity in W/cm^2/sr/um; q_lambda in W/cm^2/um;
 *    q in W/cm^2.  Physical constants are the paper's cgs values (Sec. 2.1).
 *  - Row-major layouts; "[a][b]" means b varies fastest.
 */
#ifndef RAPRAL_H
#define RAPRAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status -- */
enum {
    RAPRAL_OK = 0,
    RAPRAL_EINVAL = 1,     /* bad argument or out-of-range value            */
    RAPRAL_ENOMEM = 2,     /* workspace or budget exceeded                  */
    RAPRAL_ECUDA = 3,      /* a CUDA runtime call failed                    */
    RAPRAL_ETIMEOUT = 4,   /* a bounded device wait gave up                 */
    RAPRAL_ECANCELED = 5   /* work was cancelled                            */
};

/* Arithmetic of the spectral and transport steps.
 * RAPRAL_FP64: every step in FP64 ("plain").
 * RAPRAL_FP32: FP64 for the partition sums, the log-space part of the line
 *   set-up and the wavelength-integrated flux; FP32 with compensated (Kahan)
 *   sums for the line profiles and the march ("chosen"). */
enum { RAPRAL_FP64 = 0, RAPRAL_FP32 = 1 };

/* Kinds of radiating species. */
enum { RAPRAL_ATOM = 0, RAPRAL_DIATOMIC = 1 };

typedef struct rapral_ctx rapral_ctx;

#if defined(__GNUC__)
#define RAPRAL_API __attribute__((visibility("default")))
#else
#define RAPRAL_API
#endif

/* ------------------------------------------------------------ data model -- */

/* Radiating-species database (Sec. 2.1; the paper's first layer).
 * Atoms: a level list (E, g) per species.  Diatomics: electronic states
 * (term energy E_i, degeneracy g_i, symmetry factor sigma, line-alternation
 * factor for even / odd J) with a vibrational ladder E_V[V] and rotational
 * ladders E_J[V][J] (J = 0 .. nj-1) per state. */
typedef struct {
    int32_t n_species;            /* S (<= RAPRAL_MAX_SPECIES)                */
    const int32_t* kind;          /* [S] RAPRAL_ATOM / RAPRAL_DIATOMIC         */
    const int32_t* density_col;   /* [S] column of the species in cells.n      */
    const double* mass;           /* [S] molar mass, g/mol                     */
    const int64_t* atom_off;      /* [S+1] level ranges into atom_E / atom_g   */
    const double* atom_E;         /* [n_atom_levels] cm^-1                     */
    const double* atom_g;         /* [n_atom_levels]                           */
    const int64_t* st_off;        /* [S+1] state ranges                        */
    const double* st_E;           /* [n_states] electronic term energy, cm^-1  */
    const double* st_g;           /* [n_states]                                */
    const double* st_sigma;       /* [n_states]                                */
    const double* st_Lalt;        /* [n_states][2] even J, odd J               */
    const int32_t* st_nv;         /* [n_states] vibrational levels             */
    const int32_t* st_nj;         /* [n_states] rotational levels per V        */
    const int64_t* st_vib_off;    /* [n_states] offset into vib_E              */
    const int64_t* st_rot_off;    /* [n_states] offset into rot_E              */
    const double* vib_E;          /* [n_vib] E_V, cm^-1                        */
    const double* rot_E;          /* [n_rot] E_J(V), cm^-1, [V][J] per state   */
    int64_t n_atom_levels, n_states, n_vib, n_rot;  /* sizes (bounds checks)  */
} rapral_species;

/* Line list (Sec. 2.2.1 atoms, Sec. 2.2.2 diatomics), sorted by lam0
 * (ascending; an unsorted list still gives correct results, more slowly).
 * Level energies are split into electronic, vibrational (both at T_ve) and
 * rotational (at T_tr) parts; g is the statistical weight multiplying the
 * level's Boltzmann factor (g_i S_multi (2J+1) L_alter / sigma for a
 * rovibronic level). */
typedef struct {
    int64_t n_lines;
    const double* lam0;     /* [L] centre, nm                                 */
    const double* A;        /* [L] Einstein coefficient, s^-1                  */
    const double* lamS0;    /* [L] Stark HWHM at N_e = 1e16, T = 1e4 K, nm     */
    const int32_t* species; /* [L] radiating-species index                     */
    const double *Eu_el, *Eu_v, *Eu_j, *gu;   /* [L] upper level               */
    const double *El_el, *El_v, *El_j, *gl;   /* [L] lower level               */
} rapral_lines;

/* Cell states (cell-centred flowfield values, Sec. 2.3 first layer). */
typedef struct {
    int64_t n_cells;        /* C                                              */
    const double* Ttr;      /* [C] translational-rotational temperature, K    */
    const double* Tve;      /* [C] vibrational-electron-electronic temp., K   */
    const double* n;        /* [C][n_cols] number densities, cm^-3            */
    int32_t n_cols;
    int32_t ne_col;         /* column of the electron density                 */
    const double* lnpref;   /* [C][S] ln N_s - ln Z_s from rapral_populations  */
} rapral_cells;

/* Uniform wavelength grid: lam_k = lam_min + k h, h = (lam_max - lam_min) /
 * (n - 1), k = 0 .. n-1 (end points included). */
typedef struct {
    double lam_min, lam_max;
    int64_t n;
} rapral_grid;

/* Ray set.  A BUNDLE is a path through cells (segments listed from the far
 * boundary to the surface point) shared by one or more DIRECTIONS; a
 * direction scales every segment length (1/mu for a tangent-slab direction,
 * 1 for a single line of sight) and carries its weight in the angular sum
 * q_lambda[p] = sum_dir weight * I_dir (Sec. 2.2.3).  Bundles of surface
 * point p are [point_off[p], point_off[p+1]).  The caller owns every array;
 * rapral_slab_rays / rapral_axisym_rays / rapral_fibonacci_rays fill them. */
typedef struct {
    int64_t n_bundles;          /* B                                          */
    int64_t n_points;           /* P                                          */
    int64_t n_segments;         /* seg_off[B]                                 */
    int64_t n_dirs;             /* dir_off[B]                                 */
    int32_t max_dirs;           /* max directions of a bundle (<= RAPRAL_MAX_DIRS) */
    int32_t max_bundles_per_point;
    const int64_t* point_off;   /* [P+1]                                      */
    const int64_t* seg_off;     /* [B+1]                                      */
    const int32_t* seg_cell;    /* [n_segments] cell index, far -> near       */
    const double* seg_ds;       /* [n_segments] length, cm                    */
    const int64_t* dir_off;     /* [B+1]                                      */
    const double* dir_scale;    /* [n_dirs]                                   */
    const double* dir_weight;   /* [n_dirs]                                   */
    const int32_t* bundle_wall; /* [B] 1: the far end is a wall at T_wall     */
    double T_wall;              /* K                                          */
    /* 0: kappa / emis rows are cells, seg_cell names the cell of each
     *    segment and node values are face averages of adjacent cells;
     * 1: rows are LOS nodes (Sec. 2.2.3: flow variables interpolated to
     *    the nodes, coefficients evaluated there): segment s of bundle b
     *    runs from node s + b (far) to node s + b + 1 (near), kappa held at
     *    the far node and j linear between the two; bundles of one
     *    direction only. */
    int32_t node_values;
} rapral_rays;

#define RAPRAL_MAX_SPECIES 32
#define RAPRAL_MAX_DIRS 65

/* ---------------------------------------------------------------- context -- */

/* Creates a context on `device` that enqueues on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The caller owns the
 * stream.  Errors: RAPRAL_EINVAL (bad device), RAPRAL_ECUDA. */
RAPRAL_API int rapral_create(rapral_ctx** out, int device, void* cuda_stream);

/* Frees the context and its workspace (after synchronising its stream). */
RAPRAL_API void rapral_destroy(rapral_ctx* ctx);

/* Message of the last failure of `ctx` (static storage of the context). */
RAPRAL_API const char* rapral_last_error(const rapral_ctx* ctx);

/* Re-targets the context to another stream (for example a worker's). */
RAPRAL_API int rapral_set_stream(rapral_ctx* ctx, void* cuda_stream);

/* Synchronises the context's stream and reports the sticky device status:
 * RAPRAL_EINVAL if a device-side check failed since the last
 * rapral_clear_status(), RAPRAL_ECUDA on a CUDA error, else RAPRAL_OK. */
RAPRAL_API int rapral_sync(rapral_ctx* ctx);
RAPRAL_API int rapral_clear_status(rapral_ctx* ctx);

/* Physical constants: 0 = the paper's 4-digit cgs values (default),
 * 1 = CODATA 2018. */
RAPRAL_API int rapral_set_constants(rapral_ctx* ctx, int codata);

/* Spectral tile width (grid points per line-sum tile: 128, 256 or 512;
 * default 512 for FP64 and 128 for FP32) and cells per FP32 line-sum
 * block (2, 4 or 8; default 4).  0 keeps the current value; a tile width of -1 restores the
 * default.  Used by the autotuner. */
RAPRAL_API int rapral_set_tiling(rapral_ctx* ctx, int tile_width, int cells_per_block);

/* How the FP32 line sum (Sec. 2.2.1: the sum over lines of strength times
 * profile at every cell and grid point) is launched, for the default line
 * shape without the optional Lorentz terms or departure coefficients.  Its
 * work units are (spectral tile, group of cells_per_block cells).
 * blocks_per_sm = -1 (the default): a persistent launch of as many blocks
 * as fit on every SM, which take the units in tile order from an atomic
 * counter (cleared on the context's stream before each launch); n in
 * 1 .. 32: the same with n blocks a SM; 0: one block per unit.  Every unit
 * is computed the same way in all three, so the results are bitwise the
 * same.  Errors: EINVAL (blocks_per_sm outside -1 .. 32). */
RAPRAL_API int rapral_set_line_sum_blocks(rapral_ctx* ctx, int blocks_per_sm);

/* Lines a warp of the FP32 line sum stages per sweep pass (Sec. 2.2.1: a
 * cell's coefficients over a spectral tile are the sum over the tile's line
 * list): 32 (the default, one (line, cell) pair set up by each lane) or 64
 * (two passes of set-up, then one sweep over all 64).  Terms are added
 * plainly inside a pass and with compensation across passes, so the plain
 * part's error bound is (pairs - 1) u of a point's term magnitudes
 * (u = 2^-24).  Used by the autotuner with rapral_set_tiling; batches take
 * the value current at rapral_batch_create (32 with the optional Lorentz
 * terms); the exact Voigt shape, the optional terms and the allocation-free
 * entry point use 32.
 * Errors: EINVAL (not 32 or 64). */
RAPRAL_API int rapral_set_line_batch(rapral_ctx* ctx, int pairs);

/* Work counters of the line sum, accumulated over rapral_spectral_coeffs
 * calls since the last reset: in-window (line, cell, grid point) profile
 * evaluations, how many of them needed the Gaussian core term and the
 * exponential correction term in the chosen arithmetic (the others underflow
 * to zero), and (line, cell, tile) pairs set up. */
typedef struct {
    int64_t evaluations;
    int64_t gauss_terms;
    int64_t correction_terms;
    int64_t pairs;
} rapral_stats;

/* Turns the FP32 line sum's work counters on (default) or off; counting
 * costs a few conversions per (line, cell, tile) pair.  The FP64 path
 * always counts. */
RAPRAL_API int rapral_set_counters(rapral_ctx* ctx, int on);

/* Reads the counters (synchronises the stream). */
RAPRAL_API int rapral_get_stats(rapral_ctx* ctx, rapral_stats* out);
RAPRAL_API int rapral_reset_stats(rapral_ctx* ctx);

/* Records the CUDA events `before` / `after` (cudaEvent_t, caller-owned) on
 * the context's stream immediately around every line-sum kernel launch and
 * every continuum level-sum kernel launch, so a caller can time that kernel
 * alone.  NULL, NULL turns it off. */
RAPRAL_API int rapral_set_profile_events(rapral_ctx* ctx, void* before, void* after);

/* Device bytes the context's workspace needs for a solve of this size
 * (lines L, spectral range nk); for admission control.  Host-only. */
RAPRAL_API int rapral_workspace_bytes(int64_t n_lines, int64_t n_cells, int64_t nk, size_t* bytes);

/* ---------------------------------------------------------- hot-path steps -- */

/* Partition functions and log population prefactors (Sec. 2.1, Boltzmann
 * distribution of atoms; molecular Boltzmann distribution with the
 * rovibrational partition function Q_vr):
 *   atoms:      Z_s = sum_levels g exp(-hcE / k T_ve)
 *   diatomics:  Z_s = sum_i g_i exp(-hcE_i / k T_ve) Q_vr,i,
 *               Q_vr,i = sum_V exp(-hcE_V / k T_ve) (1/sigma)
 *                        sum_J (2J+1) L_alter exp(-hcE_J / k T_tr)
 *   lnpref[c][s] = ln n_{c, density_col[s]} - ln Z_s   (-inf when n = 0).
 * In: sp, cells (Ttr, Tve, n).  Out: lnpref [C][S] FP64 (device).
 * Errors: EINVAL (sizes, S > RAPRAL_MAX_SPECIES; device: T <= 0 or not
 * finite, n < 0). */
RAPRAL_API int rapral_populations(rapral_ctx* ctx, const rapral_species* sp,
                       const rapral_cells* cells, double* lnpref);

/* Line-by-line emission and absorption coefficients (Sec. 2.2.1 / 2.2.2):
 *   j(lam_k)     = sum_lines j0 phi(|lam_k - lam0|),
 *   kappa(lam_k) = sum_lines kappa0 phi(|lam_k - lam0|),
 *   j0 = 1e-7 (hc/4pi) N_u A / (lam0 1e-7), kappa0 = j0 / B(lam0) with B in
 *   population form (Sec. 2.2), N from lnpref and the level data, phi the
 *   Whiting Voigt shape with HWHMs Doppler(T_tr), Lorentz = natural +
 *   Stark(T_ve, N_e) and the Voigt fit; a line adds to point k only when
 *   |lam_k - lam0| <= 100 lamV.
 * Computes grid points [k0, k0 + nk) for every cell.
 * Out: kappa, emis [C][ld] (columns 0 .. nk-1 written), FP64 or FP32 per
 * `precision`.  ld >= nk.  Lines are binned into spectral tiles on the
 * device first (workspace).  Errors: EINVAL (k0 + nk > n, nk < 1, ld < nk,
 * n < 2, lam_max <= lam_min or not finite; line windows that give more than
 * 2^31 - 1 (line, tile) entries, the limit of the tile lists' int32 offsets,
 * before anything is filled: split the range; device: species index out of
 * range, lam0 <= 0, g <= 0), ENOMEM (workspace), ECUDA. */
RAPRAL_API int rapral_spectral_coeffs(rapral_ctx* ctx, const rapral_species* sp,
                           const rapral_lines* lines, const rapral_cells* cells,
                           const rapral_grid* grid, int64_t k0, int64_t nk,
                           int precision, void* kappa, void* emis, int64_t ld);

/* Ray march and angular reduction (Sec. 2.2.3).  For each bundle and grid
 * point, nodes sit on cell faces (end nodes take the adjacent cell's value,
 * interior nodes the mean of the two adjacent cells); over each segment
 * kappa is the far node's value and j is linear:
 *   I <- I e^{-dtau} + a j_far + b j_near,  dtau = kappa_far ds scale,
 *   a = (f - e^{-dtau}) / kappa_far,  b = (1 - f) / kappa_far,
 *   f = (1 - e^{-dtau}) / dtau,
 * with the series of a and b when |dtau| < 4e-4 (FP64, three terms) or
 * |dtau| < 0.5 (FP32, seven terms).
 * The march starts from 0 (far field) or the Planck intensity at T_wall.
 * Then q_lambda[p][k] = sum over the point's directions of weight * I.
 * In: kappa, emis [C][ld] for grid points [k0, k0+nk) (as written by
 * rapral_spectral_coeffs with the same precision).  Out: q_lambda [P][nk]
 * (FP64 or FP32); I_out [n_dirs][nk] or NULL.  Errors: EINVAL (sizes,
 * max_dirs > RAPRAL_MAX_DIRS; device: seg_cell not in [0, n_cells),
 * seg_ds < 0). */
RAPRAL_API int rapral_trace_rays(rapral_ctx* ctx, const rapral_rays* rays, int64_t n_cells,
                      const void* kappa, const void* emis, int64_t ld,
                      const rapral_grid* grid, int64_t k0, int64_t nk, int precision,
                      void* q_lambda, void* I_out);

/* Spectral integral of the wall flux (Sec. 2.2.3): q[p] += sum_k w_k
 * q_lambda[p][k] h 1e-3 (lam in um), w_k the trapezoid weights of the whole
 * grid (1/2 at k = 0 and k = n-1), so the chunks of one grid add up.  FP64
 * accumulation.  The caller zeroes q before the first chunk.
 * In: q_lambda [P][nk] FP64/FP32.  In/out: q [P] FP64. */
RAPRAL_API int rapral_wall_flux(rapral_ctx* ctx, const void* q_lambda, int precision,
                     const rapral_grid* grid, int64_t k0, int64_t nk, int64_t n_points,
                     double* q);

/* ------------------------------------------------------------------ batch -- */

/* One request of a batch: a whole solve over the grid points [k0, k0+nk)
 * (the steps of rapral_spectral_coeffs, rapral_trace_rays and
 * rapral_wall_flux).  Host pointers to the descriptors; the arrays inside
 * are device arrays.  cells->lnpref must hold rapral_populations' output
 * when the batch runs.  kappa / emis [C][ld] and q_lambda [P][nk] are FP32
 * scratch of the request; q [P] FP64 accumulates. */
typedef struct {
    const rapral_species* species;
    const rapral_lines* lines;
    const rapral_cells* cells;
    const rapral_grid* grid;
    const rapral_rays* rays;
    int64_t k0, nk;
    void* kappa;
    void* emis;
    int64_t ld;
    void* q_lambda;
    double* q;
} rapral_batch_item;

typedef struct rapral_batch rapral_batch;

/* Plans a batch of independent, uneven requests (the batching the paper's
 * per-LOS loop suggests; Sec. 2.2.3 runs one LBL + RTE per line of sight):
 * checks every request, builds its line records and spectral-tile line lists
 * with the context's tiling, and lays their work units end to end.  Copies
 * the descriptors (not the arrays).  Allocates the batch's own device memory
 * and synchronises the stream.  The plan stays valid while the arrays keep
 * their addresses and the cells' temperatures and electron densities do not
 * rise above the planned values (window bounds).  FP32 only.  Errors:
 * EINVAL (a request, with its index in the message; failed device checks),
 * ENOMEM, ECUDA. */
RAPRAL_API int rapral_batch_create(rapral_ctx* ctx, int n_items, const rapral_batch_item* items, int precision,
                                   rapral_batch** out);

/* Enqueues the batch: one persistent line-sum launch over every request's
 * (tile, cell group) units, pulled from an atomic counter, then each
 * request's march and flux.  No allocation, no host synchronisation: the
 * call can be captured in a CUDA graph on the context's stream. */
RAPRAL_API int rapral_batch_run(rapral_ctx* ctx, rapral_batch* batch);

/* Work units and persistent grid size of a planned batch (host only). */
RAPRAL_API int rapral_batch_units(const rapral_batch* batch, int64_t* units, int* blocks);

RAPRAL_API void rapral_batch_destroy(rapral_batch* batch);

/* rapral_spectral_coeffs without any device allocation.  (No counterpart in
 * the paper: it exists for callers that cannot allocate.)  Real-time loops
 * that must stay off the allocator (an allocation can block on the driver),
 * and plug-ins whose device memory belongs to the host program's own pool,
 * cannot call cudaMalloc; this entry point needs neither a context nor a
 * workspace.  Its scratch is one static device array
 * of 64 MiB inside the library, held by every GPU that loads the library
 * until the process exits.  The call runs on the device that owns
 * `cuda_stream` (for the legacy default stream, the current device): it makes
 * that device current while it runs and restores the caller's current device
 * before it returns.  The first call on a device, and the first after that
 * device's context was reset, looks the array's address up
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the array and clears what must start at zero;
 * calls that overlap on the GPU (other streams, unordered host threads) race
 * on it, so serialise them.  The call synchronises `cuda_stream` once (to
 * read the input checks and the tile-list length) and then enqueues the line
 * sum; outputs are valid once the stream synchronises.  Default tile
 * widths (512 FP64, 128 FP32), paper constants.  Arguments as rapral_spectral_coeffs, plus an optional
 * caller buffer `err` (err_len bytes) for a message.  Errors: EINVAL (sizes,
 * ranges, failed device-side input checks), ENOMEM (the problem needs more
 * than the 64 MiB scratch: about 230 bytes per line plus 64 per cell and 4
 * per (line, tile) entry of the tile lists), ECUDA. */
RAPRAL_API int rapral_spectral_coeffs_noalloc(void* cuda_stream, const rapral_species* sp,
                                              const rapral_lines* lines, const rapral_cells* cells,
                                              const rapral_grid* grid, int64_t k0, int64_t nk,
                                              int precision, void* kappa, void* emis, int64_t ld,
                                              char* err, size_t err_len);

/* ------------------------------------------------------------ ray builders -- */

/* Tangent slab (plane-parallel layers, Sec. 2.2.3 with the slab reading of
 * the solid-angle integral): `n_layers` cells cell_order[0] (far boundary)
 * .. cell_order[m-1] (wall), thickness dx[i]; directions mu[m] with weight
 * 2 pi wmu[m] mu[m] and path scale 1/mu[m]; with `normal_ray` a first
 * direction mu = 1 of weight 0 (intensity output only).  The nd = n_mu +
 * normal_ray directions (1 .. 4096) are split into nb = ceil(nd / 17)
 * bundles that each repeat the cell path.  Inputs are device arrays;
 * outputs are caller-owned device arrays sized point_off[2], seg_off[nb+1],
 * seg_cell / seg_ds[n_layers * nb], dir_off[nb+1], dir_scale /
 * dir_weight[nd], bundle_wall[nb].  Fills `rays` (host struct) with those
 * pointers and sizes. */
RAPRAL_API int rapral_slab_rays(rapral_ctx* ctx, const int32_t* cell_order, const double* dx,
                     int32_t n_layers, const double* mu, const double* wmu, int32_t n_mu,
                     int32_t normal_ray, int32_t wall_start, double T_wall,
                     int64_t* point_off, int64_t* seg_off, int32_t* seg_cell, double* seg_ds,
                     int64_t* dir_off, double* dir_scale, double* dir_weight,
                     int32_t* bundle_wall, rapral_rays* rays);

/* Axisymmetric rays (Sec. 2.2.3 lines of sight, on a rectilinear (x, r) grid
 * around a body of radius r_body = rf[0]): from each surface point
 * (surf_x[p], r_body) a ray per (mu_m, azimuth a) with mu = cos of the angle
 * to the outward normal and azimuths at (a + 1/2) 2 pi / n_phi; each ray is a
 * bundle of one direction (scale 1, weight wmu[m] mu_m 2 pi / n_phi).
 * Cells are numbered ix * nr + jr.  Segments run from the far boundary to
 * the point; zero-length pieces are dropped.
 * Two calls: with seg_cell == NULL the call counts segments, writes seg_off
 * [B+1] (B = P n_mu n_phi) and returns the total in *n_segments (host; the
 * call synchronises the stream); a second call with seg_cell / seg_ds
 * (device, n_segments entries) fills them and the remaining arrays
 * (point_off[P+1], dir_off[B+1], dir_scale[B], dir_weight[B],
 * bundle_wall[B]) and `rays`.  Geometry arrays (xf[nx+1], rf[nr+1],
 * surf_x[P], mu, wmu) are device arrays. */
RAPRAL_API int rapral_axisym_rays(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf,
                       int32_t nr, const double* surf_x, int32_t n_points,
                       const double* mu, const double* wmu, int32_t n_mu, int32_t n_phi,
                       int64_t* seg_off, int64_t* n_segments, int32_t* seg_cell, double* seg_ds,
                       int64_t* point_off, int64_t* dir_off, double* dir_scale,
                       double* dir_weight, int32_t* bundle_wall, rapral_rays* rays);

/* ------------------------------------------------ optional Lorentz terms -- */

#define RAPRAL_BROAD_STARK_IONIZE 1   /* atomic Stark coefficient from the ionisation gap */
#define RAPRAL_BROAD_RESONANCE 2      /* resonance broadening of atomic ground-level lines */
#define RAPRAL_BROAD_VDW 4            /* van der Waals broadening of atomic lines         */

/* The full Lorentz width of Sec. 2.2.1 for later rapral_spectral_coeffs /
 * rapral_batch_create calls of this context (flags 0, the default: natural +
 * Stark with the lines' own Stark coefficients).  For atomic lines:
 *   RAPRAL_BROAD_STARK_IONIZE: lamS0 = 1.69e3 lam0^2 / dE^2.623 (nm) with
 *     dE = max(E_ionize - E_u, 109678.77 / 25) cm^-1, replacing lines.lamS0;
 *   RAPRAL_BROAD_RESONANCE: lines whose lower level is at E = 0 gain
 *     lamR = 4.3e-28 lam0 f N_0 (g_l/g_u)^0.5 lam0^2, f = m_e c (lam0 1e-7)^2
 *     g_u A / (8 pi^2 e^2 g_l), N_0 = n_s g_0 / Z_s the ground-level density
 *     (g_0: the summed weight of the species' levels at E = 0);
 *   RAPRAL_BROAD_VDW: lamW = lam0^2 (6.65e-29 N (2 T_tr / M)^0.5 +
 *     2.925e-29 N_o (2 T_tr / M_o)^0.5), N, M the species' density and molar
 *     mass, N_o the summed density of every other density column of positive
 *     molar mass and M_o their density-weighted mean molar mass.
 * E_ionize [n_species] (cm^-1) and column_mass [n_cols] (g/mol, 0 for
 * electrons) are host arrays, copied; n_species <= 32, n_cols <= 32.  The
 * allocation-free coefficient call does not use these terms. */
RAPRAL_API int rapral_set_broadening(rapral_ctx* ctx, int32_t flags, int32_t n_species, const double* E_ionize,
                       int32_t n_cols, const double* column_mass);

/* ---------------------------------------------------------- line shape -- */

#define RAPRAL_PROFILE_WHITING 0   /* Whiting's pseudo-Voigt (Sec. 2.2.1), the default */
#define RAPRAL_PROFILE_VOIGT 1     /* the exact Voigt shape                            */

/* Line shape of later rapral_spectral_coeffs calls of this context
 * (Sec. 2.2.1).  RAPRAL_PROFILE_VOIGT: phi = 1e3 Re w(z) / (sigma sqrt(2 pi))
 * um^-1, z = (lam - lam0 + i lamL) / (sigma sqrt 2), sigma = lamG /
 * sqrt(2 ln 2), w the Faddeeva function (to ~5e-13 relative in FP64, ~1e-5
 * in FP32); the line windows (100 Olivero HWHMs) do not change.  The exact
 * shape uses 512-point tiles in FP64 and 128-point tiles in FP32 whatever
 * rapral_set_tiling chose.  The batch and allocation-free paths use
 * Whiting's shape.  Errors: EINVAL (unknown profile). */
RAPRAL_API int rapral_set_profile(rapral_ctx* ctx, int32_t profile);

/* ------------------------------------- QSS collisional-radiative populations -- */

/* Level model of one atomic radiator for the quasi-steady-state populations
 * of Sec. 2.1 (all arrays device, caller-owned).  Levels 0 .. n_levels-1 are
 * solved (0: ground); levels n_levels .. n_levels_all-1 only enter the
 * closure, in Boltzmann equilibrium with level n_levels-1 at T_ve.
 * Transition t joins levels lo[t] < up[t] < n_levels with upward Arrhenius
 * rates C T^n e^{-theta/T} (cm^3/mol/s; theta the level gap in K) for heavy-
 * particle impact (hp_C, hp_n; at T_tr) and electron impact (e_C, e_n; at
 * T_ve), downward rates by detailed balance k_down = k_up Q_lo / Q_up with
 * Q_i = g_i e^{-hc E_i / k T}, and spontaneous emission A (s^-1) at lam (nm),
 * which escapes (factor 1) at lam >= 200 nm and is trapped (0) below.  Level
 * i is ionised by electrons at ii_C[i] T_ve^{ii_n[i]} e^{-hc (E_ionize - E_i)/kT_ve}
 * and refilled by three-body recombination k_up Q_i / (Q_+ Q_e),
 * Q_+ = g_ion e^{-hc E_ionize / k T_ve}, Q_e = 2 (2 pi m_e k T_ve / h^2)^1.5. */
typedef struct {
    int32_t n_levels;            /* l, 2 .. 32                                 */
    int32_t n_levels_all;        /* l* >= l                                    */
    const double* E;             /* [l*] cm^-1                                 */
    const double* g;             /* [l*]                                       */
    int32_t n_trans;             /* <= 496                                     */
    const int32_t* lo;           /* [n_trans]                                  */
    const int32_t* up;           /* [n_trans]                                  */
    const double *hp_C, *hp_n;   /* [n_trans]                                  */
    const double *e_C, *e_n;     /* [n_trans]                                  */
    const double* A;             /* [n_trans] s^-1                             */
    const double* lam;           /* [n_trans] nm                               */
    const double *ii_C, *ii_n;   /* [l] (entry 0 unused)                       */
    double E_ionize;             /* cm^-1                                      */
    double g_ion;                /* ground weight of the ion                  */
    int32_t col;                 /* density column of the atom                */
    int32_t ion_col;             /* density column of its ion, -1: none       */
} rapral_cr_model;

/* Quasi-steady-state level populations (Sec. 2.1): per cell, 0 = gains -
 * losses for levels 1 .. l-1 (heavy-particle and electron impact excitation
 * and de-excitation, radiative decay, ionisation and recombination; N_M the
 * summed density of every column but the electrons') and the closure
 * sum_i N_i (with the lumped levels) = the atom's density, solved by LU with
 * partial pivoting.  Writes n_out [C][l] (device, cm^-3).  Transition
 * indices out of range or a singular system: RAPRAL_EINVAL at the next sync. */
RAPRAL_API int rapral_qss_populations(rapral_ctx* ctx, const rapral_cr_model* model, const rapral_cells* cells,
                       double* n_out);

/* Saha-Boltzmann populations of one atomic radiator (Sec. 2.1): overwrites
 * lnpref[c][species] (device, row length n_species: the output of
 * rapral_populations, normally the array cells->lnpref points to) with ln(N_+ N_e) + 1.5 ln(h^2 / (2 pi m_e k T_ve))
 * + hc E_ionize / (k T_ve) - ln(2 Q_+), Q_+ = sum_k ion_g[k] e^{-hc ion_E[k] / kT_ve},
 * so that every level of the species takes N_i = N_+ N_e (h^2/(2 pi m_e k T))^1.5
 * g_i e^{hc (E_ionize - E_i)/kT} / (2 Q_+) in later coefficient calls.  N_+ is
 * density column ion_col, N_e column ne_col; a cell without ions or electrons
 * gets -inf (no population).  ion_E, ion_g: device arrays [n_ion_terms].
 * Errors: EINVAL (sizes, columns, E_ionize <= 0). */
RAPRAL_API int rapral_saha_populations(rapral_ctx* ctx, const rapral_cells* cells, int32_t species,
                                       int32_t n_species, double E_ionize, int32_t ion_col, int32_t n_ion_terms,
                                       const double* ion_E, const double* ion_g, double* lnpref);

/* Departure coefficients b = N / N^B of the model's levels (Sec. 2.1: the
 * QSS populations replace the Boltzmann populations of the main path for the
 * levels they solve).  For radiator `species` of n_species, writes
 * ln_b[(c n_species + species) n_lev + i] = ln n_qss[c][i] - (lnpref[c][species]
 * + ln g_i - hc E_i / k T_ve) for i < n_levels and 0 for n_levels <= i < n_lev;
 * other species' rows are left as they are.  n_qss [C][n_levels] is
 * rapral_qss_populations' output, cells->lnpref rapral_populations'; all
 * arrays device.  Errors: EINVAL (sizes; device: a population <= 0, at the
 * next sync). */
RAPRAL_API int rapral_qss_departures(rapral_ctx* ctx, const rapral_cr_model* model, const rapral_cells* cells,
                                     int32_t species, int32_t n_species, const double* n_qss, double* ln_b,
                                     int32_t n_lev);

/* Non-Boltzmann level populations in later rapral_spectral_coeffs calls of
 * this context (Sec. 2.1): a line whose upper (lower) level has index
 * lev_u[l] >= 0 (lev_l[l] >= 0) takes N_u b_u (N_l b_l), with ln b read from
 * ln_b [n_cells][n_species][n_lev]; -1 keeps the Boltzmann population.  The
 * emission scales by b_u, the absorption by b_u (N_l b_l g_u / (N_u b_u g_l)
 * - 1) (stimulated emission from the departed populations).  All arrays are
 * device and caller-owned; they must stay valid while set.  A coefficient
 * call whose cell, species or line counts differ from these returns EINVAL;
 * an index outside [-1, n_lev) fails that call at its sync.  ln_b NULL turns
 * the departures off.  The batch and allocation-free paths do not use them. */
RAPRAL_API int rapral_set_departures(rapral_ctx* ctx, int32_t n_lev, const double* ln_b, int64_t n_cells,
                                     int32_t n_species, const int32_t* lev_u, const int32_t* lev_l,
                                     int64_t n_lines);

/* ------------------------------------------------------ atomic continuum -- */

#define RAPRAL_MAX_CONT_MODELS 8
#define RAPRAL_MAX_CONT_LEVELS 1024

/* One atomic radiator's continuum data for rapral_continuum_coeffs (all
 * arrays device, caller-owned).  Bound-free: levels i (E_i < E_ionize, g_i)
 * each with a photoionisation table of >= 2 nodes (node_lam increasing,
 * node_sigma >= 0), linear between nodes and zero outside them.  Free-free:
 * the hydrogenic fit of Table 3 (ff_c = c1..c8) and an optional D(sigma, T)
 * table, bilinear and clamped to its range (D NULL: D = 0).  Q_+ sums the
 * ion terms (ion_E, ion_g). */
typedef struct {
    int32_t species;            /* radiator index: column of cells->lnpref      */
    int32_t atom_col, ion_col;  /* density columns of the atom and of its ion   */
    double E_ionize;            /* cm^-1                                        */
    int32_t n_levels;           /* >= 1                                         */
    const double* E;            /* [n_levels] cm^-1                             */
    const double* g;            /* [n_levels]                                   */
    int64_t n_nodes;            /* node_off[n_levels]                           */
    const int64_t* node_off;    /* [n_levels + 1], node_off[0] = 0              */
    const double* node_lam;     /* [n_nodes] nm                                 */
    const double* node_sigma;   /* [n_nodes] cm^2                               */
    int32_t n_ion_terms;        /* >= 1                                         */
    const double* ion_E;        /* [n_ion_terms] cm^-1                          */
    const double* ion_g;        /* [n_ion_terms]                                */
    double ff_c[8];             /* free-free fit coefficients                   */
    int32_t n_D_sigma, n_D_T;   /* >= 2 each when D is given, <= 64             */
    const double* D_sigma;      /* [n_D_sigma] increasing                       */
    const double* D_T;          /* [n_D_T] increasing, K                        */
    const double* D;            /* [n_D_T][n_D_sigma] or NULL                   */
} rapral_continuum;

/* Atomic continuum of Sec. 2.2.1, ADDED to kappa and emis [C][ld] (FP64 or
 * FP32 by precision, e.g. the output of rapral_spectral_coeffs) over grid
 * points [k0, k0+nk).  Per cell (T = T_ve) and model:
 *   kappa_bf = sum_i N_i sigma_i,  N_i = exp(lnpref[species]) g_i e^{-c2 E_i/T};
 *   j_bf     = sum_i N_+ N_e S_i(T) B_lam(T) sigma_i (Kirchhoff with the
 *              Saha-Boltzmann N_i,eq = N_+ N_e S_i, S_i = (h^2/(2 pi m_e k T))^1.5
 *              g_i e^{c2 (E_ionize - E_i)/T} / (2 Q_+));
 *   kappa_ff = exp(lnpref[species]) 2 Q_+ (2 pi m_e k T/h^2)^1.5 e^{-c2 E_ionize/T}
 *              sigma^H (1 + D),  sigma^3 sigma^H 1e40 = A1/sigma + A2,
 *              sigma = 91.1267 / lam;  j_ff = B_lam kappa_ff.
 * cells->lnpref must hold rapral_populations' output; n_species is its row
 * length.  Errors: EINVAL (sizes, columns; device: tables not increasing,
 * node offsets, E_i >= E_ionize, g <= 0, at the call's sync). */
RAPRAL_API int rapral_continuum_coeffs(rapral_ctx* ctx, const rapral_continuum* models, int32_t n_models,
                                       int32_t n_species, const rapral_cells* cells, const rapral_grid* grid,
                                       int64_t k0, int64_t nk, int precision, void* kappa, void* emis,
                                       int64_t ld);

/* ----------------------------------------------- Fibonacci lines of sight -- */

/* Lines of sight of the paper's own angular path (Sec. 2.2.3, Fibonacci
 * sphere): from each surface point (surf_x[p], r_body = rf[0]) the n_los
 * directions (r cos a, w, r sin a) with w = 1 - 2 (i - 1)/(n_los - 1),
 * r = sqrt(1 - w^2), a = (i - 1)(sqrt(5) - 1) pi, i = 1 .. n_los, in the
 * frame x along the axis, y the outward normal at the point, z completing
 * it.  Only the V directions with w > 0 (leaving the body) are kept,
 * V = floor(n_los / 2); point p owns bundles [p V, (p + 1) V), each one
 * direction (scale 1, weight 1), los_index[b] = i - 1.  A line's nodes are
 * where its projection onto the (x, r) plane crosses a cell face, plus its
 * two ends: bundle b has seg_off[b+1] - seg_off[b] segments between nodes
 * seg_off[b] + b (far boundary) .. seg_off[b+1] + b (the surface point),
 * whose (x, r) go to node_x / node_r; seg_cell[s] = s + b (the far node)
 * and the set has node_values = 1.  n_los in 2 .. 65536.
 * Two calls as rapral_axisym_rays: with seg_cell == NULL it writes seg_off
 * [B+1] (B = P V) and *n_segments (host; synchronises); the second call
 * fills seg_cell / seg_ds [n_segments], point_off [P+1], dir_off [B+1],
 * dir_scale / dir_weight / bundle_wall / los_index [B] and node_x / node_r
 * [n_segments + B] (all device, caller-owned) and `rays`. */
RAPRAL_API int rapral_fibonacci_rays(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf,
                       int32_t nr, const double* surf_x, int32_t n_points, int32_t n_los,
                       int64_t* seg_off, int64_t* n_segments, int32_t* seg_cell, double* seg_ds,
                       int64_t* point_off, int64_t* dir_off, double* dir_scale, double* dir_weight,
                       int32_t* bundle_wall, int32_t* los_index, double* node_x, double* node_r,
                       rapral_rays* rays);

/* Flow variables at LOS nodes (Sec. 2.2.3, interpolation of the cell-centred
 * flowfield to the nodes): inverse-distance weights 1/d^2 over the 2 x 2
 * block of cell centres around (node_x, node_r), the block clamped to the
 * grid; a node on a centre takes that cell's values.  `cells` are the
 * grid's nx * nr cells numbered ix * nr + jr (lnpref not used).  Writes
 * Ttr, Tve [n_nodes] and n [n_nodes][cells->n_cols] (device). */
RAPRAL_API int rapral_los_node_states(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                       const rapral_cells* cells, int64_t n_nodes, const double* node_x,
                       const double* node_r, double* Ttr, double* Tve, double* n);

/* Wall flux from per-LOS results (Sec. 2.2.3 angular integral): for each
 * point, S (the wavelength integral of a line's intensity, e.g. from
 * rapral_wall_flux over the lines' intensities) is carried to the grid
 * phi_q = (pi/2) q / (n_phi - 1), theta_t = 2 pi t / (n_theta - 1) (phi
 * from the outward normal) by inverse-distance weights 1/|v - g|^2 over the
 * point's 4 nearest line directions v (a grid direction on a line takes its
 * S), then q[p] = sum_t sum_q (1/4)(S_{q,t} + S_{q+1,t} + S_{q,t+1} +
 * S_{q+1,t+1}) (cos^2 phi_q - cos^2 phi_{q+1}) / 2 (theta_{t+1} - theta_t).
 * point_off [P+1] (bundles of each point), los_index [B] and S [B] as from
 * rapral_fibonacci_rays; q [P] FP64 is written (device).  n_phi, n_theta
 * >= 2, n_phi n_theta <= 2^20. */
RAPRAL_API int rapral_fibonacci_flux(rapral_ctx* ctx, int64_t n_points, const int64_t* point_off,
                       const int32_t* los_index, int32_t n_los, const double* S, int32_t n_phi,
                       int32_t n_theta, double* q);

#ifdef __cplusplus
}
#endif

#endif /* RAPRAL_H */
