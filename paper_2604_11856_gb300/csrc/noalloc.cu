// rapral_spectral_coeffs_noalloc: the line-by-line coefficients for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: real-time loops that must not touch
// the allocator (an allocation can block on the driver for an unbounded
// time), and plug-ins running inside a host program that owns all device
// memory through its own pool, which must not be fragmented or exceeded.  This entry point
// runs the same kernels as rapral_spectral_coeffs (its FP32 line sum as one
// block per work unit, which gives bitwise the same sums as the regular
// entry point's persistent launch), but every scratch buffer
// (per-line and per-cell records, the tile ranges, the tile lists, the
// status and counter words) lives in one file-scope __device__ array of
// SCRATCH_BYTES.  The caller passes inputs and outputs; nothing is allocated
// or freed here.
//
// The array exists once per GPU that loads this library and stays allocated
// until the process exits.  All calls on a device share it and it keeps the
// last call's contents, so each call clears the words that must start at
// zero.  Calls that overlap on the GPU (different streams, or host threads
// without ordering) race on the array: serialise them.
//
// The call runs on the device that owns `cuda_stream` (the current device
// for the legacy default stream): it makes that device current for its
// duration and restores the caller's current device before it returns.
#include <cuda.h>

#include <mutex>

#include "rapral_internal.cuh"

namespace {

constexpr size_t SCRATCH_BYTES = size_t(64) << 20;   // 64 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Per device: the scratch array's device address and the identity of the
// CUDA context it was looked up in.  A device reset destroys that context and
// the next one loads the array afresh, possibly elsewhere, so the address is
// looked up again whenever the current context's identity differs.
struct ScratchAddr {
    void* ptr = nullptr;
    unsigned long long ctx_id = 0;
    bool have_id = false;
};
std::mutex g_mu;
ScratchAddr g_addr[MAX_DEVICES];

void put_err(char* err, size_t len, const char* msg) {
    if (err && len) {
        strncpy(err, msg, len - 1);
        err[len - 1] = 0;
    }
}

// Unique identity of the calling thread's current CUDA context (driver API,
// reached through the runtime's entry-point table, so no link to libcuda).
// False when no context is current or the driver cannot tell.
bool current_ctx_id(unsigned long long* id) {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return false;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the scratch array on device `dev`, which must be current.
// This is the set-up of the first call on a device (and the first call after
// a reset of it): cudaGetSymbolAddress, with its return code checked.
int scratch_ptr(int dev, void** out, char* err, size_t len) {
    if (dev < 0 || dev >= MAX_DEVICES) {
        put_err(err, len, "device index beyond the scratch table");
        return RAPRAL_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAddr& a = g_addr[dev];
    unsigned long long id = 0;
    const bool have_id = current_ctx_id(&id);
    if (!a.ptr || !have_id || !a.have_id || a.ctx_id != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            a = ScratchAddr{};
            put_err(err, len, "cudaGetSymbolAddress of the scratch array failed");
            return RAPRAL_ECUDA;
        }
        a.ptr = p;
        a.have_id = current_ctx_id(&a.ctx_id);   // the lookup made the context current if none was
    }
    *out = a.ptr;
    return RAPRAL_OK;
}

// Makes `dev` current for the lifetime of the guard and restores the
// caller's current device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    cudaError_t enter(int dev) {
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if (prev == dev) return cudaSuccess;
        e = cudaSetDevice(dev);
        switched = e == cudaSuccess;
        return e;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

int noalloc_impl(int dev, cudaStream_t stream, const rapral_species* sp, const rapral_lines* ln,
                 const rapral_cells* cells, const rapral_grid* g, int64_t k0, int64_t nk, int precision,
                 void* kappa, void* emis, int64_t ld, char* err, size_t err_len);

}  // namespace

extern "C" int rapral_spectral_coeffs_noalloc(void* cuda_stream, const rapral_species* sp, const rapral_lines* ln,
                                              const rapral_cells* cells, const rapral_grid* g, int64_t k0,
                                              int64_t nk, int precision, void* kappa, void* emis, int64_t ld,
                                              char* err, size_t err_len) {
    if (!sp || !ln || !cells || !g || !kappa || !emis) {
        put_err(err, err_len, "null argument");
        return RAPRAL_EINVAL;
    }
    if (const char* why = grid_problem(g)) {
        put_err(err, err_len, why);
        return RAPRAL_EINVAL;
    }
    if (!range_in_grid(g, k0, nk) || ld < nk || (precision != RAPRAL_FP64 && precision != RAPRAL_FP32) ||
        ln->n_lines < 0 || ln->n_lines > 2147483647LL || cells->n_cells < 0 || cells->n_cols < 1 ||
        cells->ne_col < 0 || cells->ne_col >= cells->n_cols || sp->n_species < 1 ||
        sp->n_species > RAPRAL_MAX_SPECIES || (cells->n_cells > 0 && !cells->lnpref)) {
        put_err(err, err_len, "invalid size, range, precision or null array");
        return RAPRAL_EINVAL;
    }
    const cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    if (cudaStreamGetDevice(stream, &dev) != cudaSuccess) {
        cudaGetLastError();
        put_err(err, err_len, "cannot tell the device of the stream");
        return RAPRAL_ECUDA;
    }
    DeviceGuard guard;
    if (guard.enter(dev) != cudaSuccess) {
        cudaGetLastError();
        put_err(err, err_len, "cannot make the stream's device current");
        return RAPRAL_ECUDA;
    }
    return noalloc_impl(dev, stream, sp, ln, cells, g, k0, nk, precision, kappa, emis, ld, err, err_len);
}

namespace {

int noalloc_impl(int dev, cudaStream_t stream, const rapral_species* sp, const rapral_lines* ln,
                 const rapral_cells* cells, const rapral_grid* g, int64_t k0, int64_t nk, int precision,
                 void* kappa, void* emis, int64_t ld, char* err, size_t err_len) {
    const int64_t C = cells->n_cells, L = ln->n_lines;
    if (C == 0) return RAPRAL_OK;
    const int W = precision == RAPRAL_FP64 ? 512 : 128;   // the regular entry point's defaults
    const int64_t T = (nk + W - 1) / W;
    if (T > 65535) {
        put_err(err, err_len, "range needs more than 65535 tiles");
        return RAPRAL_EINVAL;
    }
    // fixed part of the scratch: records, ranges, offsets, status and counters
    size_t need = 0;
    need = arena_need(need, 8 * sizeof(int));                      // status word
    need = arena_need(need, 4 * sizeof(unsigned long long));       // counters
    need = arena_need(need, 4 * sizeof(unsigned long long));       // maxima
    need = arena_need(need, 4 * sizeof(int));                      // sorted flag
    need = arena_need(need, (size_t)L * sizeof(LinePrep));
    need = arena_need(need, (size_t)L * sizeof(LineF32));
    need = arena_need(need, (size_t)C * sizeof(CellPrep));
    need = arena_need(need, (size_t)L * sizeof(int2));
    need = arena_need(need, (size_t)(T + 1) * sizeof(int));
    const size_t fixed = need;
    if (fixed + 256 > SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof(msg), "problem needs %zu bytes of scratch before the tile lists; the limit is %zu",
                 fixed, SCRATCH_BYTES);
        put_err(err, err_len, msg);
        return RAPRAL_ENOMEM;
    }
    void* base = nullptr;
    int st = scratch_ptr(dev, &base, err, err_len);
    if (st) return st;

    // a context on the caller's stack: the stream, the status word and the
    // counters in the scratch array; no workspace of its own
    rapral_ctx ctx;
    ctx.device = dev;
    ctx.stream = stream;
    Arena ar{reinterpret_cast<char*>(base), SCRATCH_BYTES};
    ctx.d_status = ar.take<int>(8);
    ctx.d_stats = ar.take<unsigned long long>(4);
    unsigned long long* dmax = ar.take<unsigned long long>(4);
    int* sorted_flag = ar.take<int>(4);
    LinePrep* lp = ar.take<LinePrep>(L);
    LineF32* lf = ar.take<LineF32>(L);
    CellPrep* cp = ar.take<CellPrep>(C);
    BinPlan plan;
    plan.k0 = k0; plan.nk = nk; plan.tile_w = W; plan.n_tiles = T;
    plan.line_tiles = ar.take<int2>(L);
    plan.tile_off = ar.take<int>(T + 1);
    plan.sorted_flag = sorted_flag;
    plan.wmax = dmax + 2;
    plan.total = reinterpret_cast<long long*>(dmax + 3);
    const size_t csr_at = ar.used;

    const double h = (g->lam_max - g->lam_min) / (double)(g->n - 1);
    const Phys ph = make_phys(0);
    cudaError_t e = cudaSuccess;
    if (L == 0) {
        const size_t esz = precision == RAPRAL_FP64 ? 8 : 4;
        e = cudaMemset2DAsync(kappa, ld * esz, 0, nk * esz, C, ctx.stream);
        if (e == cudaSuccess) e = cudaMemset2DAsync(emis, ld * esz, 0, nk * esz, C, ctx.stream);
        if (e != cudaSuccess) put_err(err, err_len, cudaGetErrorString(e));
        return e == cudaSuccess ? RAPRAL_OK : RAPRAL_ECUDA;
    }
    // words that must start at zero (the array keeps the previous call's values)
    e = cudaMemsetAsync(ctx.d_status, 0, 8 * sizeof(int), ctx.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx.d_stats, 0, 4 * sizeof(unsigned long long), ctx.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan.wmax, 0, sizeof(unsigned long long), ctx.stream);
    static const int one = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(sorted_flag, &one, sizeof(int), cudaMemcpyHostToDevice, ctx.stream);
    if (e == cudaSuccess) e = launch_validate_cells(&ctx, cells);
    if (e == cudaSuccess) e = launch_validate_lines(&ctx, ln, sp->n_species);
    if (e == cudaSuccess) e = launch_line_prep(&ctx, sp, ln, g->lam_min, h, ph, lp, lf, sorted_flag);
    if (e == cudaSuccess) e = launch_cell_prep(&ctx, cells, ph, cp, dmax);
    if (e == cudaSuccess) e = launch_bin_bounds(&ctx, ln, lp, cp, dmax, h, &plan);
    if (e == cudaSuccess) e = launch_bin_count(&ctx, ln, g, h, &plan);
    // read the status word and the tile-list length (host stack, no pinned buffer)
    int status_words[3] = {0, 0, 0};
    long long total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(status_words, ctx.d_status, sizeof(status_words), cudaMemcpyDeviceToHost, ctx.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, plan.total, sizeof(long long), cudaMemcpyDeviceToHost, ctx.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        put_err(err, err_len, cudaGetErrorString(e));
        return RAPRAL_ECUDA;
    }
    if (status_words[ST_CODE] != RAPRAL_OK) {
        put_err(err, err_len, "a device-side input check failed (temperatures, densities, species, centres, "
                              "weights or Einstein coefficients)");
        return status_words[ST_CODE];
    }
    if (total > (long long)(SCRATCH_BYTES / sizeof(int)) ||
        arena_need(csr_at, (size_t)(total + 1) * sizeof(int)) > SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof(msg), "tile lists of %lld entries exceed the %zu-byte scratch", total, SCRATCH_BYTES);
        put_err(err, err_len, msg);
        return RAPRAL_ENOMEM;
    }
    ar.used = csr_at;
    plan.tile_lines = ar.take<int>((size_t)total + 1);
    e = launch_bin_fill(&ctx, ln, g, h, &plan);
    if (e == cudaSuccess) {
        LineSumArgs a;
        a.lp = lp; a.lf = lf; a.cp = cp; a.lnpref = cells->lnpref; a.S = sp->n_species; a.C = C;
        a.tile_off = plan.tile_off; a.tile_lines = plan.tile_lines;
        a.lam_min = g->lam_min; a.h = h; a.k0 = k0; a.nk = nk; a.ld = ld; a.tile_w = W;
        a.kappa = kappa; a.emis = emis; a.status = ctx.d_status; a.stats = ctx.d_stats; a.count = 0;
        e = launch_line_sum(&ctx, a, precision, T);
    }
    if (e != cudaSuccess) {
        put_err(err, err_len, cudaGetErrorString(e));
        return RAPRAL_ECUDA;
    }
    return RAPRAL_OK;
}

}  // namespace
