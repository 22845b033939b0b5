// C ABI of librapral: context, errors, host-side checks, workspace, and the
// orchestration of the hot-path kernels on the context's stream.
#include <cstdarg>
#include <new>

#include "rapral_internal.cuh"

int set_error(rapral_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_status(rapral_ctx* ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return RAPRAL_OK;
    return set_error(ctx, RAPRAL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ws_reserve(rapral_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return RAPRAL_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_status(ctx, e, "workspace sync");
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    size_t grow = bytes + bytes / 4 + (1u << 20);
    e = cudaMalloc(&ctx->ws, grow);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, RAPRAL_ENOMEM, "workspace of %zu bytes: %s", grow, cudaGetErrorString(e));
    }
    ctx->ws_bytes = grow;
    return RAPRAL_OK;
}

static const char* check_name(int c) {
    switch (c) {
        case CHK_CELL_T: return "cell temperature not positive and finite";
        case CHK_CELL_N: return "cell number density negative or not finite";
        case CHK_LINE_SPECIES: return "line species index out of range";
        case CHK_LINE_LAM: return "line centre or Stark width invalid";
        case CHK_LINE_G: return "line level weight not positive";
        case CHK_LINE_A: return "Einstein coefficient negative or not finite";
        case CHK_SEG_CELL: return "segment cell index out of range";
        case CHK_SEG_DS: return "segment length negative or not finite";
        case CHK_DIR: return "direction scale not positive";
        case CHK_TIMEOUT: return "bounded device wait expired";
        case CHK_LOS_INDEX: return "line-of-sight index out of range";
        case CHK_CR_TRANS: return "level-model transition indices out of range";
        case CHK_CR_SINGULAR: return "singular QSS rate matrix";
        case CHK_CR_POP: return "QSS population not positive: no departure coefficient";
        case CHK_DEP_LEVEL: return "line level index outside the departure table";
        case CHK_CONT_TABLE: return "continuum model: node offsets, tables, levels or D grid invalid";
        default: return "device check";
    }
}

// Reads the sticky status (synchronises the stream).
int read_status(rapral_ctx* ctx) {
    cudaError_t e = cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_status(ctx, e, "status read-back");
    const int code = ctx->h_pinned[ST_CODE];
    if (code != RAPRAL_OK)
        return set_error(ctx, code, "%s (index %d)", check_name(ctx->h_pinned[ST_CHECK]), ctx->h_pinned[ST_INDEX]);
    return RAPRAL_OK;
}

extern "C" {

int rapral_create(rapral_ctx** out, int device, void* cuda_stream) {
    if (!out) return RAPRAL_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return RAPRAL_EINVAL;
    }
    rapral_ctx* ctx = new (std::nothrow) rapral_ctx();
    if (!ctx) return RAPRAL_ENOMEM;
    ctx->device = device;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, 8 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, 8 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pinned, 16 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stats, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_stats, 0, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) ctx->d_unit = ctx->d_stats + 4;
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_status) cudaFree(ctx->d_status);
        delete ctx;
        return RAPRAL_ECUDA;
    }
    *out = ctx;
    return RAPRAL_OK;
}

void rapral_destroy(rapral_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_stats) cudaFree(ctx->d_stats);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    delete ctx;
}

int rapral_get_stats(rapral_ctx* ctx, rapral_stats* out) {
    if (!ctx || !out) return RAPRAL_EINVAL;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpyAsync(ctx->h_pinned, ctx->d_stats, 4 * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_status(ctx, e, "stats read-back");
    const unsigned long long* v = reinterpret_cast<const unsigned long long*>(ctx->h_pinned);
    out->evaluations = (int64_t)v[0];
    out->gauss_terms = (int64_t)v[1];
    out->correction_terms = (int64_t)v[2];
    out->pairs = (int64_t)v[3];
    return RAPRAL_OK;
}

int rapral_reset_stats(rapral_ctx* ctx) {
    if (!ctx) return RAPRAL_EINVAL;
    cudaSetDevice(ctx->device);
    return cuda_status(ctx, cudaMemsetAsync(ctx->d_stats, 0, 4 * sizeof(unsigned long long), ctx->stream),
                       "stats reset");
}

int rapral_set_counters(rapral_ctx* ctx, int on) {
    if (!ctx) return RAPRAL_EINVAL;
    ctx->count_work = on ? 1 : 0;
    return RAPRAL_OK;
}

int rapral_set_profile_events(rapral_ctx* ctx, void* before, void* after) {
    if (!ctx || ((before == nullptr) != (after == nullptr))) return RAPRAL_EINVAL;
    ctx->ev_before = reinterpret_cast<cudaEvent_t>(before);
    ctx->ev_after = reinterpret_cast<cudaEvent_t>(after);
    return RAPRAL_OK;
}

const char* rapral_last_error(const rapral_ctx* ctx) { return ctx ? ctx->err : "no context"; }

int rapral_set_stream(rapral_ctx* ctx, void* cuda_stream) {
    if (!ctx) return RAPRAL_EINVAL;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    return RAPRAL_OK;
}

int rapral_sync(rapral_ctx* ctx) {
    if (!ctx) return RAPRAL_EINVAL;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(ctx, e, "pending CUDA error");
    return read_status(ctx);
}

int rapral_clear_status(rapral_ctx* ctx) {
    if (!ctx) return RAPRAL_EINVAL;
    return cuda_status(ctx, cudaMemsetAsync(ctx->d_status, 0, 8 * sizeof(int), ctx->stream), "status clear");
}

int rapral_set_constants(rapral_ctx* ctx, int codata) {
    if (!ctx || (codata != 0 && codata != 1)) return RAPRAL_EINVAL;
    ctx->codata = codata;
    return RAPRAL_OK;
}

int rapral_set_tiling(rapral_ctx* ctx, int tile_width, int cells_per_block) {
    if (!ctx) return RAPRAL_EINVAL;
    if (tile_width == -1) {
        ctx->tile_w = 0;   // back to the per-precision default
    } else if (tile_width != 0) {
        if (tile_width != 128 && tile_width != 256 && tile_width != 512)
            return set_error(ctx, RAPRAL_EINVAL, "tile width %d not one of 128, 256, 512", tile_width);
        ctx->tile_w = tile_width;
    }
    if (cells_per_block != 0) {
        if (cells_per_block != 2 && cells_per_block != 4 && cells_per_block != 8)
            return set_error(ctx, RAPRAL_EINVAL, "cells per block %d not 2, 4 or 8", cells_per_block);
        ctx->cells_per_block = cells_per_block;
    }
    return RAPRAL_OK;
}

int rapral_set_line_batch(rapral_ctx* ctx, int pairs) {
    if (!ctx) return RAPRAL_EINVAL;
    if (pairs != 32 && pairs != 64)
        return set_error(ctx, RAPRAL_EINVAL, "line-sum pairs per pass %d not 32 or 64", pairs);
    ctx->pairs_per_batch = pairs;
    return RAPRAL_OK;
}

int rapral_set_line_sum_blocks(rapral_ctx* ctx, int blocks_per_sm) {
    if (!ctx) return RAPRAL_EINVAL;
    if (blocks_per_sm < -1 || blocks_per_sm > 32)
        return set_error(ctx, RAPRAL_EINVAL, "line-sum blocks per SM %d not in -1 .. 32", blocks_per_sm);
    ctx->ls_persist = blocks_per_sm;
    return RAPRAL_OK;
}

int rapral_workspace_bytes(int64_t n_lines, int64_t n_cells, int64_t nk, size_t* bytes) {
    if (!bytes || n_lines < 0 || n_cells < 0 || nk < 0) return RAPRAL_EINVAL;
    // per-line records + tile ranges, per-cell records, tile offsets, and a
    // tile-list estimate of three tiles per line
    const int64_t tiles = nk / 128 + 2;
    size_t b = 0;
    b = arena_need(b, (size_t)n_lines * sizeof(LinePrep));
    b = arena_need(b, (size_t)n_lines * sizeof(LineF32));
    b = arena_need(b, (size_t)n_lines * sizeof(int2));
    b = arena_need(b, (size_t)n_cells * sizeof(CellPrep));
    b = arena_need(b, (size_t)(tiles + 1) * sizeof(int));
    b = arena_need(b, (RAPRAL_DMAX_SLOTS + 2) * sizeof(unsigned long long) + 64);
    b = arena_need(b, (size_t)(3 * n_lines + tiles) * sizeof(int));
    *bytes = b + b / 4 + (1u << 20);
    return RAPRAL_OK;
}

int rapral_populations(rapral_ctx* ctx, const rapral_species* sp, const rapral_cells* cells, double* lnpref) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!sp || !cells || !lnpref) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (sp->n_species < 1 || sp->n_species > RAPRAL_MAX_SPECIES)
        return set_error(ctx, RAPRAL_EINVAL, "species count %d not in 1..%d", sp->n_species, RAPRAL_MAX_SPECIES);
    if (cells->n_cells < 0 || cells->n_cols < 1 || cells->ne_col < 0 || cells->ne_col >= cells->n_cols)
        return set_error(ctx, RAPRAL_EINVAL, "cell array sizes");
    if (cells->n_cells == 0) return RAPRAL_OK;
    if (!cells->Ttr || !cells->Tve || !cells->n || !sp->kind || !sp->density_col)
        return set_error(ctx, RAPRAL_EINVAL, "null cell or species array");
    cudaSetDevice(ctx->device);
    const Phys ph = make_phys(ctx->codata);
    cudaError_t e = launch_validate_cells(ctx, cells);
    if (e == cudaSuccess) e = launch_populations(ctx, sp, cells, lnpref, ph);
    return cuda_status(ctx, e, "populations");
}

static int check_grid(rapral_ctx* ctx, const rapral_grid* g, int64_t k0, int64_t nk) {
    const char* why = grid_problem(g);
    if (why) return set_error(ctx, RAPRAL_EINVAL, "%s", why);
    if (!range_in_grid(g, k0, nk))
        return set_error(ctx, RAPRAL_EINVAL, "range [%lld, %lld) outside the grid of %lld points", (long long)k0,
                         (long long)k0 + (long long)nk, (long long)g->n);
    return RAPRAL_OK;
}

static double grid_h(const rapral_grid* g) { return (g->lam_max - g->lam_min) / (double)(g->n - 1); }

int rapral_spectral_coeffs(rapral_ctx* ctx, const rapral_species* sp, const rapral_lines* ln,
                           const rapral_cells* cells, const rapral_grid* g, int64_t k0, int64_t nk, int precision,
                           void* kappa, void* emis, int64_t ld) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!sp || !ln || !cells || !kappa || !emis) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    int st = check_grid(ctx, g, k0, nk);
    if (st) return st;
    if (precision != RAPRAL_FP64 && precision != RAPRAL_FP32)
        return set_error(ctx, RAPRAL_EINVAL, "precision %d", precision);
    if (ld < nk) return set_error(ctx, RAPRAL_EINVAL, "ld %lld < nk %lld", (long long)ld, (long long)nk);
    if (ln->n_lines < 0 || ln->n_lines > 2147483647LL) return set_error(ctx, RAPRAL_EINVAL, "line count");
    if (cells->n_cells < 0 || cells->n_cols < 1 || cells->ne_col < 0 || cells->ne_col >= cells->n_cols)
        return set_error(ctx, RAPRAL_EINVAL, "cell array sizes");
    if (sp->n_species < 1 || sp->n_species > RAPRAL_MAX_SPECIES) return set_error(ctx, RAPRAL_EINVAL, "species count");
    if (cells->n_cells > 0 && !cells->lnpref) return set_error(ctx, RAPRAL_EINVAL, "cells.lnpref is null");
    if (ctx->dep_lnb && (ctx->dep_C != cells->n_cells || ctx->dep_S != sp->n_species || ctx->dep_L != ln->n_lines))
        return set_error(ctx, RAPRAL_EINVAL,
                         "departure table of %lld cells, %d species, %lld lines; call has %lld, %d, %lld",
                         (long long)ctx->dep_C, ctx->dep_S, (long long)ctx->dep_L, (long long)cells->n_cells,
                         sp->n_species, (long long)ln->n_lines);
    cudaSetDevice(ctx->device);
    const int64_t C = cells->n_cells, L = ln->n_lines;
    const size_t esz = precision == RAPRAL_FP64 ? 8 : 4;
    cudaError_t e = cudaSuccess;
    if (C == 0) return RAPRAL_OK;
    if (L == 0) {
        e = cudaMemset2DAsync(kappa, ld * esz, 0, nk * esz, C, ctx->stream);
        if (e == cudaSuccess) e = cudaMemset2DAsync(emis, ld * esz, 0, nk * esz, C, ctx->stream);
        return cuda_status(ctx, e, "zero coefficients");
    }
    // the exact Voigt shape runs in one tiling per precision
    const int W = (ctx->tile_w && ctx->profile == RAPRAL_PROFILE_WHITING) ? ctx->tile_w
                                                                          : (precision == RAPRAL_FP64 ? 512 : 128);
    if (W != 128 && W != 256 && W != 512)
        return set_error(ctx, RAPRAL_EINVAL, "line sum supports tile widths 128, 256, 512 (got %d)", W);
    const int64_t T = (nk + W - 1) / W;
    if (T > 65535) return set_error(ctx, RAPRAL_EINVAL, "range of %lld points needs more than 65535 tiles", (long long)nk);
    const double h = grid_h(g);
    const Phys ph = make_phys(ctx->codata);

    // phase 1: per-line and per-cell records, tile ranges, tile counts
    size_t need = 0;
    need = arena_need(need, L * sizeof(LinePrep));
    need = arena_need(need, L * sizeof(LineF32));
    need = arena_need(need, C * sizeof(CellPrep));
    need = arena_need(need, L * sizeof(int2));
    need = arena_need(need, (T + 1) * sizeof(int));
    need = arena_need(need, (RAPRAL_DMAX_SLOTS + 2) * sizeof(unsigned long long));
    need = arena_need(need, 4 * sizeof(int));
    const bool bt = broad_terms(&ctx->broad);
    if (bt) need = broad_need(need, L, C, sp->n_species);
    const size_t phase1 = need;
    need = arena_need(need, (size_t)(3 * L + T) * sizeof(int));   // first guess of the tile lists
    st = ws_reserve(ctx, need);
    if (st) return st;
    Arena ar{ctx->ws, ctx->ws_bytes};
    LinePrep* lp = ar.take<LinePrep>(L);
    LineF32* lf = ar.take<LineF32>(L);
    CellPrep* cp = ar.take<CellPrep>(C);
    BinPlan plan;
    plan.k0 = k0; plan.nk = nk; plan.tile_w = W; plan.n_tiles = T;
    plan.line_tiles = ar.take<int2>(L);
    plan.tile_off = ar.take<int>(T + 1);
    unsigned long long* dmax = ar.take<unsigned long long>(RAPRAL_DMAX_SLOTS + 2);
    plan.wmax = dmax + RAPRAL_DMAX_SLOTS;
    plan.total = reinterpret_cast<long long*>(dmax + RAPRAL_DMAX_SLOTS + 1);
    plan.sorted_flag = ar.take<int>(4);
    double2* lb = nullptr; float2* lb32 = nullptr; double2* cb = nullptr; float2* cb32 = nullptr;
    double* g0 = nullptr;
    if (bt) {
        lb = ar.take<double2>(L); lb32 = ar.take<float2>(L);
        cb = ar.take<double2>((size_t)C * sp->n_species); cb32 = ar.take<float2>((size_t)C * sp->n_species);
        g0 = ar.take<double>(RAPRAL_MAX_SPECIES);
    }
    const int one = 1;
    e = cudaMemcpyAsync(plan.sorted_flag, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan.wmax, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) e = launch_validate_cells(ctx, cells);
    if (e == cudaSuccess) e = launch_validate_lines(ctx, ln, sp->n_species);
    if (e == cudaSuccess && ctx->dep_lnb) e = launch_check_levels(ctx, ctx->dep_u, ctx->dep_l, L, ctx->dep_nlev);
    if (e == cudaSuccess)
        e = launch_line_prep(ctx, sp, ln, g->lam_min, h, ph, lp, lf, plan.sorted_flag, &ctx->broad, lb, lb32);
    if (e == cudaSuccess) e = launch_cell_prep(ctx, cells, ph, cp, dmax);
    if (e == cudaSuccess && bt) e = launch_broad_cells(ctx, sp, cells, ctx->broad, g0, cb, cb32, dmax);
    if (e == cudaSuccess) e = launch_bin_bounds(ctx, ln, lp, cp, dmax, h, &plan, lb);
    if (e == cudaSuccess) e = launch_bin_count(ctx, ln, g, h, &plan);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->h_pinned, plan.total, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream);
    // the device checks ran before: on a failed one the counts were never written
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->h_pinned + 4, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_status(ctx, e, "line binning");
    if (ctx->h_pinned[4 + ST_CODE]) return read_status(ctx);
    const int64_t total = reinterpret_cast<const long long*>(ctx->h_pinned)[0];
    if (total > RAPRAL_MAX_TILE_ENTRIES)
        return set_error(ctx, RAPRAL_EINVAL,
                         "the line windows give %lld (line, tile) entries, more than the 2^31 - 1 the tile lists "
                         "index; split the spectral range into smaller calls",
                         (long long)total);
    // phase 2: tile lists
    need = arena_need(phase1, (size_t)(total + 1) * sizeof(int));
    if (need > ctx->ws_bytes) {
        // the arena moves: records must be rebuilt in the new one
        st = ws_reserve(ctx, need + (size_t)(3 * L + T) * sizeof(int));
        if (st) return st;
        return rapral_spectral_coeffs(ctx, sp, ln, cells, g, k0, nk, precision, kappa, emis, ld);
    }
    ar.used = phase1;
    plan.tile_lines = ar.take<int>(total + 1);
    e = launch_bin_fill(ctx, ln, g, h, &plan);
    if (e != cudaSuccess) return cuda_status(ctx, e, "line binning");

    LineSumArgs a;
    a.lp = lp; a.lf = lf; a.cp = cp; a.lnpref = cells->lnpref; a.S = sp->n_species; a.C = C;
    a.tile_off = plan.tile_off; a.tile_lines = plan.tile_lines;
    a.lam_min = g->lam_min; a.h = h; a.k0 = k0; a.nk = nk; a.ld = ld; a.tile_w = W;
    a.kappa = kappa; a.emis = emis; a.status = ctx->d_status; a.stats = ctx->d_stats; a.count = ctx->count_work;
    a.lb = lb; a.lb32 = lb32; a.cb = cb; a.cb32 = cb32;
    if (ctx->dep_lnb) {
        a.dep_lnb = ctx->dep_lnb; a.dep_u = ctx->dep_u; a.dep_l = ctx->dep_l; a.dep_nlev = ctx->dep_nlev;
    }
    if (ctx->profile == RAPRAL_PROFILE_VOIGT) {
        a.voigt = 1;
        if (!ctx->voigt_ready) {
            e = voigt_upload();
            if (e != cudaSuccess) return cuda_status(ctx, e, "Voigt coefficients");
            ctx->voigt_ready = true;
        }
    }
    e = launch_line_sum(ctx, a, precision, T);
    return cuda_status(ctx, e, "line sum");
}

int rapral_trace_rays(rapral_ctx* ctx, const rapral_rays* rays, int64_t n_cells, const void* kappa, const void* emis,
                      int64_t ld, const rapral_grid* g, int64_t k0, int64_t nk, int precision, void* q_lambda,
                      void* I_out) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!rays || !kappa || !emis || !q_lambda) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    int st = check_grid(ctx, g, k0, nk);
    if (st) return st;
    if (precision != RAPRAL_FP64 && precision != RAPRAL_FP32)
        return set_error(ctx, RAPRAL_EINVAL, "precision %d", precision);
    if (ld < nk) return set_error(ctx, RAPRAL_EINVAL, "ld < nk");
    if (rays->n_points < 0 || rays->n_bundles < 0 || rays->n_segments < 0 || rays->n_dirs < 0)
        return set_error(ctx, RAPRAL_EINVAL, "ray set sizes");
    if (rays->max_dirs < 0 || rays->max_dirs > RAPRAL_MAX_DIRS)
        return set_error(ctx, RAPRAL_EINVAL, "max_dirs %d not in 0..%d", rays->max_dirs, RAPRAL_MAX_DIRS);
    if (rays->n_points > 2147483647LL) return set_error(ctx, RAPRAL_EINVAL, "too many surface points");
    if ((nk + 31) / 32 > 65535) return set_error(ctx, RAPRAL_EINVAL, "range of %lld points too long for one march call", (long long)nk);
    if (rays->n_points == 0) return RAPRAL_OK;
    if (!rays->point_off || !rays->seg_off || !rays->dir_off || !rays->dir_scale || !rays->dir_weight ||
        !rays->bundle_wall || (rays->n_segments > 0 && (!rays->seg_cell || !rays->seg_ds)))
        return set_error(ctx, RAPRAL_EINVAL, "null ray array");
    if (rays->bundle_wall && !(rays->T_wall >= 0.0)) return set_error(ctx, RAPRAL_EINVAL, "T_wall");
    if (rays->node_values != 0 && rays->node_values != 1) return set_error(ctx, RAPRAL_EINVAL, "node_values");
    if (rays->node_values && rays->max_dirs > 1)
        return set_error(ctx, RAPRAL_EINVAL, "node-valued rays need bundles of one direction");
    if (rays->node_values && n_cells < rays->n_segments + rays->n_bundles)
        return set_error(ctx, RAPRAL_EINVAL, "node-valued rays need n_segments + n_bundles rows");
    cudaSetDevice(ctx->device);
    const Phys ph = make_phys(ctx->codata);
    st = ws_reserve(ctx, march_scratch_bytes(rays, nk, precision));
    if (st) return st;
    cudaError_t e = launch_validate_rays(ctx, rays, n_cells);
    if (e == cudaSuccess)
        e = launch_march(ctx, rays, kappa, emis, ld, g, grid_h(g), k0, nk, precision, q_lambda, I_out, ph, ctx->ws);
    return cuda_status(ctx, e, "ray march");
}

int rapral_wall_flux(rapral_ctx* ctx, const void* q_lambda, int precision, const rapral_grid* g, int64_t k0,
                     int64_t nk, int64_t n_points, double* q) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!q_lambda || !q) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    int st = check_grid(ctx, g, k0, nk);
    if (st) return st;
    if (precision != RAPRAL_FP64 && precision != RAPRAL_FP32)
        return set_error(ctx, RAPRAL_EINVAL, "precision %d", precision);
    if (n_points < 0 || n_points > 2147483647LL) return set_error(ctx, RAPRAL_EINVAL, "n_points");
    cudaSetDevice(ctx->device);
    // the partial sums live at the start of the workspace: every earlier user
    // of the workspace on this stream has been enqueued before
    st = ws_reserve(ctx, (size_t)wall_flux_parts(nk) * (size_t)n_points * 16 + 256);
    if (st) return st;
    return cuda_status(ctx, launch_wall_flux(ctx, q_lambda, precision, g, grid_h(g), k0, nk, n_points, q, ctx->ws),
                       "wall flux");
}

int rapral_slab_rays(rapral_ctx* ctx, const int32_t* cell_order, const double* dx, int32_t n_layers, const double* mu,
                     const double* wmu, int32_t n_mu, int32_t normal_ray, int32_t wall_start, double T_wall,
                     int64_t* point_off, int64_t* seg_off, int32_t* seg_cell, double* seg_ds, int64_t* dir_off,
                     double* dir_scale, double* dir_weight, int32_t* bundle_wall, rapral_rays* rays) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!rays || !point_off || !seg_off || !dir_off || !dir_scale || !dir_weight || !bundle_wall)
        return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (n_layers < 0 || (n_layers > 0 && (!cell_order || !dx || !seg_cell || !seg_ds)))
        return set_error(ctx, RAPRAL_EINVAL, "layers");
    const int nd = n_mu + (normal_ray ? 1 : 0);
    if (n_mu < 0 || nd < 1 || nd > 4096 || (n_mu > 0 && (!mu || !wmu)))
        return set_error(ctx, RAPRAL_EINVAL, "direction count %d not in 1..4096", nd);
    const int nb = (nd + RAPRAL_SLAB_DIRS - 1) / RAPRAL_SLAB_DIRS;
    if (wall_start && !(T_wall > 0.0)) return set_error(ctx, RAPRAL_EINVAL, "T_wall must be positive for a wall start");
    cudaSetDevice(ctx->device);
    cudaError_t e = launch_slab_rays(ctx, cell_order, dx, n_layers, mu, wmu, n_mu, normal_ray, wall_start, point_off,
                                     seg_off, seg_cell, seg_ds, dir_off, dir_scale, dir_weight, bundle_wall);
    if (e != cudaSuccess) return cuda_status(ctx, e, "slab rays");
    rays->n_bundles = nb; rays->n_points = 1; rays->n_segments = (int64_t)n_layers * nb; rays->n_dirs = nd;
    rays->max_dirs = nd < RAPRAL_SLAB_DIRS ? nd : RAPRAL_SLAB_DIRS; rays->max_bundles_per_point = nb;
    rays->point_off = point_off; rays->seg_off = seg_off; rays->seg_cell = seg_cell; rays->seg_ds = seg_ds;
    rays->dir_off = dir_off; rays->dir_scale = dir_scale; rays->dir_weight = dir_weight;
    rays->bundle_wall = bundle_wall; rays->T_wall = T_wall; rays->node_values = 0;
    return RAPRAL_OK;
}

int rapral_axisym_rays(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                       const double* surf_x, int32_t n_points, const double* mu, const double* wmu, int32_t n_mu,
                       int32_t n_phi, int64_t* seg_off, int64_t* n_segments, int32_t* seg_cell, double* seg_ds,
                       int64_t* point_off, int64_t* dir_off, double* dir_scale, double* dir_weight,
                       int32_t* bundle_wall, rapral_rays* rays) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!xf || !rf || !surf_x || !mu || !wmu || !seg_off || !n_segments)
        return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (nx < 1 || nr < 1 || n_points < 0 || n_mu < 1 || n_phi < 1)
        return set_error(ctx, RAPRAL_EINVAL, "grid or direction counts");
    if ((int64_t)nx * nr > 2147483647LL) return set_error(ctx, RAPRAL_EINVAL, "too many cells");
    cudaSetDevice(ctx->device);
    const int64_t B = (int64_t)n_points * n_mu * n_phi;
    cudaError_t e;
    if (!seg_cell) {
        e = launch_axisym_count(ctx, xf, nx, rf, nr, surf_x, n_points, mu, n_mu, n_phi, seg_off, nullptr);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->h_pinned, seg_off + B, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_status(ctx, e, "axisymmetric ray count");
        *n_segments = reinterpret_cast<int64_t*>(ctx->h_pinned)[0];
        return RAPRAL_OK;
    }
    if (!seg_ds || !point_off || !dir_off || !dir_scale || !dir_weight || !bundle_wall || !rays)
        return set_error(ctx, RAPRAL_EINVAL, "null output array");
    e = launch_axisym_fill(ctx, xf, nx, rf, nr, surf_x, n_points, mu, wmu, n_mu, n_phi, seg_off, seg_cell, seg_ds,
                           point_off, dir_off, dir_scale, dir_weight, bundle_wall);
    if (e != cudaSuccess) return cuda_status(ctx, e, "axisymmetric rays");
    rays->n_bundles = B; rays->n_points = n_points; rays->n_segments = *n_segments; rays->n_dirs = B;
    rays->max_dirs = 1;
    rays->max_bundles_per_point = n_mu * n_phi;
    rays->point_off = point_off; rays->seg_off = seg_off; rays->seg_cell = seg_cell; rays->seg_ds = seg_ds;
    rays->dir_off = dir_off; rays->dir_scale = dir_scale; rays->dir_weight = dir_weight;
    rays->bundle_wall = bundle_wall; rays->T_wall = 0.0; rays->node_values = 0;
    return RAPRAL_OK;
}

int rapral_qss_populations(rapral_ctx* ctx, const rapral_cr_model* m, const rapral_cells* cells, double* n_out) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!m || !cells || !n_out) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (m->n_levels < 2 || m->n_levels > 32 || m->n_levels_all < m->n_levels || m->n_trans < 0 ||
        m->n_trans > 32 * 31 / 2)
        return set_error(ctx, RAPRAL_EINVAL,
                         "level model needs 2 <= n_levels <= 32, n_levels_all >= n_levels, n_trans <= 496");
    if (!m->E || !m->g || !m->ii_C || !m->ii_n ||
        (m->n_trans > 0 && (!m->lo || !m->up || !m->hp_C || !m->hp_n || !m->e_C || !m->e_n || !m->A || !m->lam)))
        return set_error(ctx, RAPRAL_EINVAL, "null level-model array");
    if (cells->n_cells < 0 || cells->n_cols < 1 || cells->ne_col < 0 || cells->ne_col >= cells->n_cols ||
        m->col < 0 || m->col >= cells->n_cols || m->ion_col >= cells->n_cols)
        return set_error(ctx, RAPRAL_EINVAL, "density columns");
    if (!(m->E_ionize > 0.0) || !(m->g_ion > 0.0)) return set_error(ctx, RAPRAL_EINVAL, "ionisation energy or ion weight");
    if (cells->n_cells == 0) return RAPRAL_OK;
    cudaSetDevice(ctx->device);
    cudaError_t e = launch_validate_cells(ctx, cells);
    if (e == cudaSuccess) e = launch_qss(ctx, m, cells, n_out, make_phys(ctx->codata));
    return cuda_status(ctx, e, "QSS populations");
}

int rapral_saha_populations(rapral_ctx* ctx, const rapral_cells* cells, int32_t species, int32_t n_species,
                            double E_ionize, int32_t ion_col, int32_t n_ion_terms, const double* ion_E,
                            const double* ion_g, double* lnpref) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!cells || !ion_E || !ion_g || !lnpref) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (n_species < 1 || n_species > RAPRAL_MAX_SPECIES || species < 0 || species >= n_species)
        return set_error(ctx, RAPRAL_EINVAL, "species %d of %d", species, n_species);
    if (cells->n_cells < 0 || cells->n_cols < 1 || cells->ne_col < 0 || cells->ne_col >= cells->n_cols ||
        ion_col < 0 || ion_col >= cells->n_cols)
        return set_error(ctx, RAPRAL_EINVAL, "density columns");
    if (!(E_ionize > 0.0) || !std::isfinite(E_ionize) || n_ion_terms < 1)
        return set_error(ctx, RAPRAL_EINVAL, "ionisation energy or ion terms");
    if (cells->n_cells == 0) return RAPRAL_OK;
    if (!cells->Tve || !cells->n) return set_error(ctx, RAPRAL_EINVAL, "cells need Tve and n");
    cudaSetDevice(ctx->device);
    cudaError_t e = launch_validate_cells(ctx, cells);
    if (e == cudaSuccess)
        e = launch_saha_prefactor(ctx, cells, species, n_species, E_ionize, ion_col, n_ion_terms, ion_E, ion_g,
                                  make_phys(ctx->codata), lnpref);
    return cuda_status(ctx, e, "Saha-Boltzmann populations");
}

int rapral_qss_departures(rapral_ctx* ctx, const rapral_cr_model* m, const rapral_cells* cells, int32_t species,
                          int32_t n_species, const double* n_qss, double* ln_b, int32_t n_lev) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!m || !cells || !n_qss || !ln_b) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (m->n_levels < 1 || m->n_levels > 32 || !m->E || !m->g) return set_error(ctx, RAPRAL_EINVAL, "level model");
    if (n_species < 1 || n_species > RAPRAL_MAX_SPECIES || species < 0 || species >= n_species)
        return set_error(ctx, RAPRAL_EINVAL, "species %d of %d", species, n_species);
    if (n_lev < m->n_levels) return set_error(ctx, RAPRAL_EINVAL, "n_lev %d < n_levels %d", n_lev, m->n_levels);
    if (cells->n_cells < 0) return set_error(ctx, RAPRAL_EINVAL, "cell count");
    if (cells->n_cells == 0) return RAPRAL_OK;
    if (!cells->Tve || !cells->lnpref) return set_error(ctx, RAPRAL_EINVAL, "cells need Tve and lnpref");
    cudaSetDevice(ctx->device);
    return cuda_status(ctx, launch_qss_departures(ctx, m, cells, species, n_species, n_qss, ln_b, n_lev,
                                                  make_phys(ctx->codata)),
                       "departure coefficients");
}

int rapral_set_departures(rapral_ctx* ctx, int32_t n_lev, const double* ln_b, int64_t n_cells, int32_t n_species,
                          const int32_t* lev_u, const int32_t* lev_l, int64_t n_lines) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!ln_b) {
        ctx->dep_lnb = nullptr; ctx->dep_u = ctx->dep_l = nullptr;
        ctx->dep_nlev = ctx->dep_S = 0; ctx->dep_C = ctx->dep_L = 0;
        return RAPRAL_OK;
    }
    if (!lev_u || !lev_l) return set_error(ctx, RAPRAL_EINVAL, "null level index array");
    if (n_lev < 1 || n_cells < 0 || n_lines < 0 || n_species < 1 || n_species > RAPRAL_MAX_SPECIES)
        return set_error(ctx, RAPRAL_EINVAL, "departure table sizes");
    ctx->dep_lnb = ln_b; ctx->dep_u = lev_u; ctx->dep_l = lev_l;
    ctx->dep_nlev = n_lev; ctx->dep_S = n_species; ctx->dep_C = n_cells; ctx->dep_L = n_lines;
    return RAPRAL_OK;
}

int rapral_set_profile(rapral_ctx* ctx, int32_t profile) {
    if (!ctx) return RAPRAL_EINVAL;
    if (profile != RAPRAL_PROFILE_WHITING && profile != RAPRAL_PROFILE_VOIGT)
        return set_error(ctx, RAPRAL_EINVAL, "line shape %d", profile);
    ctx->profile = profile;
    return RAPRAL_OK;
}

int rapral_set_broadening(rapral_ctx* ctx, int32_t flags, int32_t n_species, const double* E_ionize,
                          int32_t n_cols, const double* column_mass) {
    if (!ctx) return RAPRAL_EINVAL;
    const int all = RAPRAL_BROAD_STARK_IONIZE | RAPRAL_BROAD_RESONANCE | RAPRAL_BROAD_VDW;
    if (flags & ~all) return set_error(ctx, RAPRAL_EINVAL, "unknown broadening flags %d", flags);
    if (n_species < 0 || n_species > RAPRAL_MAX_SPECIES || n_cols < 0 || n_cols > RAPRAL_MAX_COLS)
        return set_error(ctx, RAPRAL_EINVAL, "at most %d species and %d density columns", RAPRAL_MAX_SPECIES,
                         RAPRAL_MAX_COLS);
    if ((flags & RAPRAL_BROAD_STARK_IONIZE) && (!E_ionize || n_species == 0))
        return set_error(ctx, RAPRAL_EINVAL, "the Stark option needs the species' ionisation energies");
    if ((flags & RAPRAL_BROAD_VDW) && (!column_mass || n_cols == 0))
        return set_error(ctx, RAPRAL_EINVAL, "the van der Waals option needs the columns' molar masses");
    BroadArgs b{};
    b.flags = flags;
    b.S = n_species;
    b.ncol = n_cols;
    for (int s = 0; s < n_species; ++s) {
        if (E_ionize && !(E_ionize[s] >= 0.0 && std::isfinite(E_ionize[s])))
            return set_error(ctx, RAPRAL_EINVAL, "ionisation energy of species %d", s);
        b.Eion[s] = E_ionize ? E_ionize[s] : 0.0;
    }
    for (int c = 0; c < n_cols; ++c) {
        if (column_mass && !(column_mass[c] >= 0.0 && std::isfinite(column_mass[c])))
            return set_error(ctx, RAPRAL_EINVAL, "molar mass of column %d", c);
        b.colmass[c] = column_mass ? column_mass[c] : 0.0;
    }
    ctx->broad = b;
    return RAPRAL_OK;
}

int rapral_fibonacci_rays(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                          const double* surf_x, int32_t n_points, int32_t n_los, int64_t* seg_off,
                          int64_t* n_segments, int32_t* seg_cell, double* seg_ds, int64_t* point_off,
                          int64_t* dir_off, double* dir_scale, double* dir_weight, int32_t* bundle_wall,
                          int32_t* los_index, double* node_x, double* node_r, rapral_rays* rays) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!xf || !rf || !surf_x || !seg_off || !n_segments) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (nx < 1 || nr < 1 || n_points < 0 || n_los < 2 || n_los > 65536)
        return set_error(ctx, RAPRAL_EINVAL, "grid counts, or n_los not in 2 .. 65536");
    if ((int64_t)nx * nr > 2147483647LL) return set_error(ctx, RAPRAL_EINVAL, "too many cells");
    cudaSetDevice(ctx->device);
    const int64_t B = (int64_t)n_points * (n_los / 2);
    cudaError_t e;
    if (!seg_cell) {
        e = launch_fib_count(ctx, xf, nx, rf, nr, surf_x, n_points, n_los, seg_off);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->h_pinned, seg_off + B, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_status(ctx, e, "Fibonacci ray count");
        *n_segments = reinterpret_cast<int64_t*>(ctx->h_pinned)[0];
        if (*n_segments + B > 2147483647LL) return set_error(ctx, RAPRAL_EINVAL, "more than 2^31 LOS nodes");
        return RAPRAL_OK;
    }
    if (!seg_ds || !point_off || !dir_off || !dir_scale || !dir_weight || !bundle_wall || !los_index || !node_x ||
        !node_r || !rays)
        return set_error(ctx, RAPRAL_EINVAL, "null output array");
    e = launch_fib_fill(ctx, xf, nx, rf, nr, surf_x, n_points, n_los, seg_off, seg_cell, seg_ds, point_off, dir_off,
                        dir_scale, dir_weight, bundle_wall, los_index, node_x, node_r);
    if (e != cudaSuccess) return cuda_status(ctx, e, "Fibonacci rays");
    rays->n_bundles = B; rays->n_points = n_points; rays->n_segments = *n_segments; rays->n_dirs = B;
    rays->max_dirs = 1;
    rays->max_bundles_per_point = n_los / 2;
    rays->point_off = point_off; rays->seg_off = seg_off; rays->seg_cell = seg_cell; rays->seg_ds = seg_ds;
    rays->dir_off = dir_off; rays->dir_scale = dir_scale; rays->dir_weight = dir_weight;
    rays->bundle_wall = bundle_wall; rays->T_wall = 0.0; rays->node_values = 1;
    return RAPRAL_OK;
}

int rapral_los_node_states(rapral_ctx* ctx, const double* xf, int32_t nx, const double* rf, int32_t nr,
                           const rapral_cells* cells, int64_t n_nodes, const double* node_x, const double* node_r,
                           double* Ttr, double* Tve, double* n) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!xf || !rf || !cells || (n_nodes > 0 && (!node_x || !node_r || !Ttr || !Tve || !n)))
        return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (nx < 1 || nr < 1 || n_nodes < 0) return set_error(ctx, RAPRAL_EINVAL, "grid or node counts");
    if (cells->n_cells != (int64_t)nx * nr) return set_error(ctx, RAPRAL_EINVAL, "cells != nx * nr");
    if (cells->n_cols < 1 || !cells->Ttr || !cells->Tve || !cells->n)
        return set_error(ctx, RAPRAL_EINVAL, "cell arrays");
    cudaSetDevice(ctx->device);
    return cuda_status(ctx, launch_node_idw(ctx, xf, nx, rf, nr, cells, n_nodes, node_x, node_r, Ttr, Tve, n),
                       "LOS node states");
}

int rapral_fibonacci_flux(rapral_ctx* ctx, int64_t n_points, const int64_t* point_off, const int32_t* los_index,
                          int32_t n_los, const double* S, int32_t n_phi, int32_t n_theta, double* q) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!point_off || !los_index || !S || !q) return set_error(ctx, RAPRAL_EINVAL, "null argument");
    if (n_points < 0 || n_los < 2 || n_los > 65536 || n_phi < 2 || n_theta < 2 ||
        (int64_t)n_phi * n_theta > (1 << 20))
        return set_error(ctx, RAPRAL_EINVAL, "counts out of range");
    cudaSetDevice(ctx->device);
    int st = ws_reserve(ctx, fib_flux_scratch_bytes(n_points, n_los, n_phi, n_theta));
    if (st) return st;
    return cuda_status(ctx, launch_fib_flux(ctx, n_points, point_off, los_index, n_los, S, n_phi, n_theta, q, ctx->ws),
                       "Fibonacci flux");
}

}  // extern "C"
