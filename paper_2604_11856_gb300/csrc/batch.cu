// Batched solves: many independent, uneven requests planned once and run
// with one persistent line-sum launch (rapral_batch_*).
//
// rapral_batch_create validates every request, builds its per-line and
// per-cell records and its spectral-tile line lists (one synchronisation for
// all tile-list lengths) in memory the batch owns, and lays the requests'
// work units end to end.  rapral_batch_run then only enqueues kernels -- the
// persistent line sum over all units, and each request's march and flux --
// with no allocation and no host synchronisation, so it can be captured in a
// CUDA graph and replayed.
#include <algorithm>
#include <new>
#include <vector>

#include "rapral_internal.cuh"

struct BatchReq {
    rapral_species sp;
    rapral_lines ln;
    rapral_cells cells;
    rapral_grid grid;
    rapral_rays rays;
    int64_t k0, nk, ld;
    void *kappa, *emis, *q_lambda;
    double* q;
    double h;
};

struct rapral_batch {
    int n = 0;
    int tile_w = 128, wpb = 4, pb = 32;   // tiling, cells a block, pairs a sweep pass
    bool broad = false;           // the optional Lorentz terms were planned in
    std::vector<BatchReq> req;
    char* ws = nullptr;           // records, tile ranges, offsets of every request
    int* csr = nullptr;           // tile lists of every request
    BatchItem* d_items = nullptr;
    unsigned long long* d_counter = nullptr;
    void* d_flux = nullptr;       // partial sums of the spectral integral (largest request)
    std::vector<void*> d_march;   // FP32 copies of each request's ray data
    int64_t total_units = 0;
    int blocks = 0;
};

static int check_item(rapral_ctx* ctx, const rapral_batch_item& it, int i) {
    if (!it.species || !it.lines || !it.cells || !it.grid || !it.rays || !it.kappa || !it.emis || !it.q_lambda || !it.q)
        return set_error(ctx, RAPRAL_EINVAL, "request %d: null argument", i);
    const rapral_grid* g = it.grid;
    if (grid_problem(g) || !range_in_grid(g, it.k0, it.nk) || it.ld < it.nk)
        return set_error(ctx, RAPRAL_EINVAL, "request %d: grid, range or ld", i);
    if (it.lines->n_lines < 1 || it.lines->n_lines > 2147483647LL || it.cells->n_cells < 1 || !it.cells->lnpref ||
        it.cells->n_cols < 1 || it.cells->ne_col < 0 || it.cells->ne_col >= it.cells->n_cols ||
        it.species->n_species < 1 || it.species->n_species > RAPRAL_MAX_SPECIES)
        return set_error(ctx, RAPRAL_EINVAL, "request %d: lines, cells or species", i);
    if (it.rays->n_points < 1 || it.rays->max_dirs < 1 || it.rays->max_dirs > RAPRAL_MAX_DIRS ||
        (it.nk + 31) / 32 > 65535)
        return set_error(ctx, RAPRAL_EINVAL, "request %d: rays", i);
    return RAPRAL_OK;
}

extern "C" {

int rapral_batch_create(rapral_ctx* ctx, int n_items, const rapral_batch_item* items, int precision,
                        rapral_batch** out) {
    if (!ctx) return RAPRAL_EINVAL;
    if (!out || !items || n_items < 1) return set_error(ctx, RAPRAL_EINVAL, "batch: no requests");
    if (precision != RAPRAL_FP32) return set_error(ctx, RAPRAL_EINVAL, "batch: only RAPRAL_FP32 is batched");
    *out = nullptr;
    for (int i = 0; i < n_items; ++i) {
        int st = check_item(ctx, items[i], i);
        if (st) return st;
    }
    cudaSetDevice(ctx->device);
    rapral_batch* B = new (std::nothrow) rapral_batch();
    if (!B) return RAPRAL_ENOMEM;
    B->n = n_items;
    B->tile_w = ctx->tile_w ? ctx->tile_w : 128;
    B->wpb = (B->tile_w == 512 || broad_terms(&ctx->broad)) ? 4 : ctx->cells_per_block;
    B->broad = broad_terms(&ctx->broad);
    B->pb = B->broad ? 32 : ctx->pairs_per_batch;
    const int W = B->tile_w;
    B->req.resize(n_items);
    // phase 1 sizes
    std::vector<size_t> base(n_items);
    size_t need = 0;
    for (int i = 0; i < n_items; ++i) {
        BatchReq& r = B->req[i];
        r.sp = *items[i].species; r.ln = *items[i].lines; r.cells = *items[i].cells; r.grid = *items[i].grid;
        r.rays = *items[i].rays;
        r.k0 = items[i].k0; r.nk = items[i].nk; r.ld = items[i].ld;
        r.kappa = items[i].kappa; r.emis = items[i].emis; r.q_lambda = items[i].q_lambda; r.q = items[i].q;
        r.h = (r.grid.lam_max - r.grid.lam_min) / (double)(r.grid.n - 1);
        const int64_t L = r.ln.n_lines, C = r.cells.n_cells, T = (r.nk + W - 1) / W;
        if (T > 65535) { delete B; return set_error(ctx, RAPRAL_EINVAL, "request %d: too many tiles", i); }
        base[i] = need;
        need = arena_need(need, L * sizeof(LinePrep));
        need = arena_need(need, L * sizeof(LineF32));
        need = arena_need(need, C * sizeof(CellPrep));
        need = arena_need(need, L * sizeof(int2));
        need = arena_need(need, (T + 1) * sizeof(int));
        need = arena_need(need, (RAPRAL_DMAX_SLOTS + 2) * sizeof(unsigned long long));
        need = arena_need(need, 4 * sizeof(int));
        if (broad_terms(&ctx->broad)) need = broad_need(need, L, C, r.sp.n_species);
        need = arena_need(need, 0);
    }
    cudaError_t e = cudaMalloc(&B->ws, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete B;
        return set_error(ctx, RAPRAL_ENOMEM, "batch records of %zu bytes", need);
    }
    std::vector<BinPlan> plans(n_items);
    std::vector<LinePrep*> lps(n_items);
    std::vector<LineF32*> lfs(n_items);
    std::vector<CellPrep*> cps(n_items);
    struct BroadTabs { double2* lb = nullptr; float2* lb32 = nullptr; double2* cb = nullptr; float2* cb32 = nullptr;
                       double* g0 = nullptr; };
    std::vector<BroadTabs> btabs(n_items);
    const Phys ph = make_phys(ctx->codata);
    static const int one = 1;
    long long* h_tot = nullptr;   // [n_items] tile-list lengths, then the status word
    e = cudaMallocHost(&h_tot, sizeof(long long) * (n_items + 1));
    for (int i = 0; i < n_items && e == cudaSuccess; ++i) {
        BatchReq& r = B->req[i];
        const int64_t L = r.ln.n_lines, C = r.cells.n_cells, T = (r.nk + W - 1) / W;
        Arena ar{B->ws, need, base[i]};
        lps[i] = ar.take<LinePrep>(L);
        lfs[i] = ar.take<LineF32>(L);
        cps[i] = ar.take<CellPrep>(C);
        BinPlan& pl = plans[i];
        pl.k0 = r.k0; pl.nk = r.nk; pl.tile_w = W; pl.n_tiles = T;
        pl.line_tiles = ar.take<int2>(L);
        pl.tile_off = ar.take<int>(T + 1);
        unsigned long long* dmax = ar.take<unsigned long long>(RAPRAL_DMAX_SLOTS + 2);
        pl.wmax = dmax + RAPRAL_DMAX_SLOTS;
        pl.total = reinterpret_cast<long long*>(dmax + RAPRAL_DMAX_SLOTS + 1);
        pl.sorted_flag = ar.take<int>(4);
        const bool bt = broad_terms(&ctx->broad);
        BroadTabs& bb = btabs[i];
        if (bt) {
            bb.lb = ar.take<double2>(L); bb.lb32 = ar.take<float2>(L);
            bb.cb = ar.take<double2>((size_t)C * r.sp.n_species); bb.cb32 = ar.take<float2>((size_t)C * r.sp.n_species);
            bb.g0 = ar.take<double>(RAPRAL_MAX_SPECIES);
        }
        e = cudaMemcpyAsync(pl.sorted_flag, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(pl.wmax, 0, sizeof(unsigned long long), ctx->stream);
        if (e == cudaSuccess) e = launch_validate_cells(ctx, &r.cells);
        if (e == cudaSuccess) e = launch_validate_lines(ctx, &r.ln, r.sp.n_species);
        if (e == cudaSuccess) e = launch_validate_rays(ctx, &r.rays, C);
        if (e == cudaSuccess) e = launch_line_prep(ctx, &r.sp, &r.ln, r.grid.lam_min, r.h, ph, lps[i], lfs[i],
                                                  pl.sorted_flag, &ctx->broad, bb.lb, bb.lb32);
        if (e == cudaSuccess) e = launch_cell_prep(ctx, &r.cells, ph, cps[i], dmax);
        if (e == cudaSuccess && bt) e = launch_broad_cells(ctx, &r.sp, &r.cells, ctx->broad, bb.g0, bb.cb, bb.cb32, dmax);
        if (e == cudaSuccess) e = launch_bin_bounds(ctx, &r.ln, lps[i], cps[i], dmax, r.h, &pl, bb.lb);
        if (e == cudaSuccess) e = launch_bin_count(ctx, &r.ln, &r.grid, r.h, &pl);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_tot + i, pl.total, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream);
    }
    // the device checks ran before the counts: on a failed one the counts were never written
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_tot + n_items, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && reinterpret_cast<const int*>(h_tot + n_items)[ST_CODE] != RAPRAL_OK) {
        cudaFreeHost(h_tot);
        rapral_batch_destroy(B);
        return read_status(ctx);
    }
    size_t csr_need = 0;
    std::vector<size_t> csr_base(n_items);
    for (int i = 0; i < n_items && e == cudaSuccess; ++i) {
        if (h_tot[i] > RAPRAL_MAX_TILE_ENTRIES) {
            cudaFreeHost(h_tot);
            rapral_batch_destroy(B);
            return set_error(ctx, RAPRAL_EINVAL,
                             "request %d: the line windows give %lld (line, tile) entries, more than the 2^31 - 1 "
                             "the tile lists index", i, h_tot[i]);
        }
        csr_base[i] = csr_need;
        csr_need += (size_t)h_tot[i] + 1;
    }
    if (e == cudaSuccess) e = cudaMalloc(&B->csr, csr_need * sizeof(int));
    std::vector<BatchItem> hitems(n_items);
    int64_t units = 0;
    for (int i = 0; i < n_items && e == cudaSuccess; ++i) {
        BatchReq& r = B->req[i];
        plans[i].tile_lines = B->csr + csr_base[i];
        e = launch_bin_fill(ctx, &r.ln, &r.grid, r.h, &plans[i]);
        LineSumArgs& a = hitems[i].a;
        a.lp = lps[i]; a.lf = lfs[i]; a.cp = cps[i]; a.lnpref = r.cells.lnpref; a.S = r.sp.n_species; a.C = r.cells.n_cells;
        a.tile_off = plans[i].tile_off; a.tile_lines = plans[i].tile_lines;
        a.lam_min = r.grid.lam_min; a.h = r.h; a.k0 = r.k0; a.nk = r.nk; a.ld = r.ld; a.tile_w = W;
        a.lb = btabs[i].lb; a.lb32 = btabs[i].lb32; a.cb = btabs[i].cb; a.cb32 = btabs[i].cb32;
        a.kappa = r.kappa; a.emis = r.emis; a.status = ctx->d_status; a.stats = ctx->d_stats; a.count = ctx->count_work;
        hitems[i].unit_off = units;
        hitems[i].n_groups = (r.cells.n_cells + B->wpb - 1) / B->wpb;
        units += plans[i].n_tiles * hitems[i].n_groups;
    }
    B->total_units = units;
    if (e == cudaSuccess) e = cudaMalloc(&B->d_items, sizeof(BatchItem) * n_items);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_counter, sizeof(unsigned long long));
    size_t flux_bytes = 256;
    for (int i = 0; i < n_items; ++i)
        flux_bytes = std::max(flux_bytes, (size_t)wall_flux_parts(B->req[i].nk) * (size_t)B->req[i].rays.n_points * 16);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_flux, flux_bytes);
    B->d_march.assign(n_items, nullptr);
    for (int i = 0; i < n_items && e == cudaSuccess; ++i) e = cudaMalloc(&B->d_march[i], march_scratch_bytes(&B->req[i].rays, B->req[i].nk, RAPRAL_FP32));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_items, hitems.data(), sizeof(BatchItem) * n_items, cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e == cudaSuccess)
        e = launch_line_sum_batch(ctx, W, B->wpb, B->pb, nullptr, 0, 0, nullptr, &B->blocks, false, B->broad);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (h_tot) cudaFreeHost(h_tot);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rapral_batch_destroy(B);
        return cuda_status(ctx, e, "batch planning");
    }
    int st = rapral_sync(ctx);
    if (st) {
        rapral_batch_destroy(B);
        return st;
    }
    *out = B;
    return RAPRAL_OK;
}

int rapral_batch_run(rapral_ctx* ctx, rapral_batch* B) {
    if (!ctx || !B) return RAPRAL_EINVAL;
    cudaSetDevice(ctx->device);
    const Phys ph = make_phys(ctx->codata);
    cudaError_t e = cudaMemsetAsync(B->d_counter, 0, sizeof(unsigned long long), ctx->stream);
    if (ctx->ev_before && e == cudaSuccess) e = cudaEventRecord(ctx->ev_before, ctx->stream);
    if (e == cudaSuccess)
        e = launch_line_sum_batch(ctx, B->tile_w, B->wpb, B->pb, B->d_items, B->n, B->total_units, B->d_counter, nullptr,
                                  true, B->broad);
    if (ctx->ev_after && e == cudaSuccess) e = cudaEventRecord(ctx->ev_after, ctx->stream);
    for (int i = 0; i < B->n && e == cudaSuccess; ++i) {
        const BatchReq& r = B->req[i];
        e = launch_march(ctx, &r.rays, r.kappa, r.emis, r.ld, &r.grid, r.h, r.k0, r.nk, RAPRAL_FP32, r.q_lambda,
                         nullptr, ph, B->d_march[i]);
        if (e == cudaSuccess)
            e = launch_wall_flux(ctx, r.q_lambda, RAPRAL_FP32, &r.grid, r.h, r.k0, r.nk, r.rays.n_points, r.q,
                                 B->d_flux);
    }
    return cuda_status(ctx, e, "batch run");
}

void rapral_batch_destroy(rapral_batch* B) {
    if (!B) return;
    if (B->ws) cudaFree(B->ws);
    if (B->csr) cudaFree(B->csr);
    if (B->d_items) cudaFree(B->d_items);
    if (B->d_counter) cudaFree(B->d_counter);
    if (B->d_flux) cudaFree(B->d_flux);
    for (void* p : B->d_march)
        if (p) cudaFree(p);
    delete B;
}

int rapral_batch_units(const rapral_batch* B, int64_t* units, int* blocks) {
    if (!B) return RAPRAL_EINVAL;
    if (units) *units = B->total_units;
    if (blocks) *blocks = B->blocks;
    return RAPRAL_OK;
}

}  // extern "C"
