// soc_api.cu -- host side of libsoc: context, validated uploads, batch
// preparation and the iteration driver (the C-ABI of include/soc.h).
#include <cuda_runtime.h>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <exception>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <vector>
#include "soc_internal.h"

using namespace soc;

namespace soc {
// Read-bandwidth probe (measurement only, soc_temperature.cu): `reps` passes
// of 16-byte loads over buf.
cudaError_t launch_probe_read(const void *buf, uint64_t bytes, int reps, int sms, unsigned long long *sink,
                              cudaStream_t s);
}

namespace {

constexpr double kPi = 3.141592653589793;
constexpr double kHc = 6.62607015e-27, kKc = 1.380649e-16, kCc = 2.99792458e10;

template <class T>
struct DevBuf {                     // owning device buffer
    T *p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count)
    {
        if (count <= n && p) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) { p = nullptr; n = 0; return e; }
        n = count;
        return cudaSuccess;
    }
    void release() { if (p) cudaFree(p); p = nullptr; n = 0; }
};

struct CloudHost {
    int nx = 0, ny = 0, nz = 0, n_levels = 0;
    int64_t n_cells = 0, n_root = 0, n_leaf = 0;
    std::vector<int64_t> level_start;
    double ell = 1.0;
    DevBuf<uint32_t> cell;
    DevBuf<int32_t> parent, leaf;
    DevBuf<float> rho;
    DevBuf<double> volume;
    DevBuf<float2> kappa;
    DevBuf<float> ps_pos, ps_cdf;
    int n_ps = 0;
    bool freed = false;
    bool has_const = false;            // A_const holds an iteration-0 result
    std::vector<double> bg_I;                  // [n_freq] or empty
    std::vector<double> ps_L_total;            // [n_freq]
    // iteration scratch (library owned)
    DevBuf<int64_t> tally, self_tally;
    DevBuf<double> A_const, A, A_self;
    DevBuf<uint64_t> dust_w, dust_wp;
    DevBuf<double> e_unit, e_unit_w;
    DevBuf<int64_t> stats;
    // reference field
    DevBuf<double> L, L_ref, A_ref, A_d, e_unit_n;
    DevBuf<uint8_t> neg;
    DevBuf<uint64_t> dust_wn;
};

}  // namespace

struct BatchHost {
    int n_items = 0;
    uint64_t total = 0;
    HotCloud hot{};
    int32_t regular = 0;
    DevBuf<DevItem> items;
    DevBuf<uint64_t> prefix;
    DevBuf<unsigned long long> counter;
};

struct soc_ctx {
    int device = 0;
    uint64_t seed = 1;
    std::string err = "no error";
    std::vector<CloudHost *> clouds;
    DevBuf<DevCloud> d_clouds;
    bool clouds_dirty = true;
    // dust
    int n_freq = 0;
    std::vector<double> nu, kabs, ksca, g, w;
    DevBuf<float> d_g;
    DevBuf<double> d_w, d_w_kabs, d_nu, d_kabs, d_lnE, d_lnT;
    // batch scratch
    DevBuf<DevItem> d_items;
    DevBuf<uint64_t> d_prefix;
    DevBuf<unsigned long long> d_counter;
    DevBuf<unsigned long long> d_lmax;
    DevBuf<unsigned long long> d_wscratch;
    DevBuf<double> d_maxdT;
    DevBuf<int64_t> d_level_start;
    DevBuf<double> d_map_S;       // per-cell source function of the last map
    // pinned staging of grid uploads (grows to the largest grid)
    uint32_t *h_stage = nullptr;
    size_t h_stage_n = 0;
    // prepared batches and graphs
    std::vector<struct BatchHost *> batches;
    std::vector<cudaGraphExec_t> graphs;
    // abort flag (host-mapped pinned memory, 2 ints): [0] nonzero = tracer
    // launches take no more work; [1] set by a launch that left work untraced
    volatile int *h_abort = nullptr;
    int *d_abort = nullptr;
    double timeout_s = 0.0;       // soc_iterate watchdog (0 = none)
    // soc_iterate_batch scratch: counters of every item of a launch, self
    // counters (ALI), statistics and per-cloud max |dT|
    DevBuf<int64_t> b_tally, b_self, b_stats;
    DevBuf<double> b_maxdT;
    // launch
    int tpb = 256, bps = 4, chunk = 16, refill_min = 8, scatter_min = 8;   // autotuned on the 128^3 x 64 nu workload
    uint32_t max_steps = 10000000u;
    int sms = 0;
    int occ[2][2][8] = {};        // resident blocks/SM per (regular grid, build, threads/32), from soc_create
};

namespace {

soc_status fail(soc_ctx *c, soc_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

soc_status cuda_fail(soc_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, e == cudaErrorMemoryAllocation ? SOC_ERR_NOMEM : SOC_ERR_CUDA, "%s: %s", where,
                cudaGetErrorString(e));
}

// Runs the body of an entry point: an exception (a failed host allocation,
// host threads that could not start) becomes a status and never crosses the
// C ABI.
template <class F>
soc_status guarded(soc_ctx *ctx, F &&body)
{
    try {
        return body();
    } catch (const std::bad_alloc &) {
        return fail(ctx, SOC_ERR_NOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(ctx, SOC_ERR_NOMEM, "host resources: %s", e.what());
    } catch (...) {
        return fail(ctx, SOC_ERR_NOMEM, "host resources: unknown exception");
    }
}

#define CK(expr, where)                                          \
    do {                                                         \
        cudaError_t e_ = (expr);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

double planck_host(double nu, double T)
{
    const double x = kHc * nu / (kKc * T);
    return (2.0 * kHc * nu * nu * nu / (kCc * kCc)) / std::expm1(x);
}

std::vector<double> trapezoid(const std::vector<double> &nu)
{
    std::vector<double> w(nu.size(), 0.0);
    if (nu.size() == 1) { w[0] = 1.0; return w; }
    for (size_t i = 0; i + 1 < nu.size(); ++i) {
        const double d = 0.5 * (nu[i + 1] - nu[i]);
        w[i] += d;
        w[i + 1] += d;
    }
    return w;
}

// Per-cloud kappa table (kabs * ell, ksca * ell as FP32) and per-frequency
// point-source CDF need both the grid and the dust.
soc_status build_cloud_tables(soc_ctx *ctx, CloudHost &cl)
{
    if (ctx->n_freq == 0) return SOC_OK;
    std::vector<float2> k(ctx->n_freq);
    for (int f = 0; f < ctx->n_freq; ++f)
        k[f] = make_float2((float)(ctx->kabs[f] * cl.ell), (float)(ctx->ksca[f] * cl.ell));
    CK(cl.kappa.alloc(ctx->n_freq), "alloc kappa");
    CK(cudaMemcpy(cl.kappa.p, k.data(), sizeof(float2) * ctx->n_freq, cudaMemcpyHostToDevice), "copy kappa");
    ctx->clouds_dirty = true;
    return SOC_OK;
}

// The device form of one grid (no heap use: also called by the
// allocation-free tracer entry).  A freed grid gets an all-zero entry.
void fill_dev_cloud(const CloudHost &c, DevCloud &d)
{
    memset(&d, 0, sizeof d);
    if (c.freed) return;
    d.cell = c.cell.p; d.parent = c.parent.p; d.leaf = c.leaf.p; d.rho = c.rho.p;
    d.volume = c.volume.p; d.kappa = c.kappa.p; d.ps_pos = c.ps_pos.p; d.ps_cdf = c.ps_cdf.p;
    d.nx = c.nx; d.ny = c.ny; d.nz = c.nz; d.n_levels = c.n_levels; d.n_ps = c.n_ps;
    d.n_cells = c.n_cells; d.n_root = c.n_root; d.n_leaf = c.n_leaf;
    for (int L = 0; L <= c.n_levels; ++L) d.level_start[L] = c.level_start[L];
    for (int L = c.n_levels + 1; L <= SOC_MAX_LEVELS; ++L) d.level_start[L] = c.n_cells;
}

soc_status sync_clouds(soc_ctx *ctx)
{
    if (!ctx->clouds_dirty) return SOC_OK;
    std::vector<DevCloud> v(ctx->clouds.size());
    for (size_t i = 0; i < ctx->clouds.size(); ++i) fill_dev_cloud(*ctx->clouds[i], v[i]);
    CK(ctx->d_clouds.alloc(v.size()), "alloc cloud table");
    CK(cudaMemcpy(ctx->d_clouds.p, v.data(), sizeof(DevCloud) * v.size(), cudaMemcpyHostToDevice),
       "copy cloud table");
    ctx->clouds_dirty = false;
    return SOC_OK;
}

soc_status check_cloud(soc_ctx *ctx, int id)
{
    if (!ctx) return SOC_ERR_ARG;
    if (id < 0 || id >= (int)ctx->clouds.size()) return fail(ctx, SOC_ERR_ARG, "cloud id %d out of range", id);
    if (ctx->clouds[id]->freed) return fail(ctx, SOC_ERR_ARG, "cloud id %d was freed", id);
    return SOC_OK;
}

}  // namespace

extern "C" {

soc_status soc_create(soc_ctx **out, int device, uint64_t seed)
{
    return guarded(nullptr, [&]() -> soc_status {
        if (!out) return SOC_ERR_ARG;
        *out = nullptr;
        int n = 0;
        if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return SOC_ERR_CUDA;
        if (cudaSetDevice(device) != cudaSuccess) return SOC_ERR_CUDA;
        soc_ctx *ctx = new (std::nothrow) soc_ctx();
        if (!ctx) return SOC_ERR_NOMEM;
        ctx->device = device;
        ctx->seed = seed;
        cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
        for (int g = 0; g < 2; ++g)
            for (int v = 3; v <= 4; ++v)
                for (int t = 32; t <= 256; t += 32) ctx->occ[g][v - 3][t / 32 - 1] = trace_block_limit(t, v, g == 1);
        void *hab = nullptr;
        if (ctx->d_counter.alloc(1) != cudaSuccess || ctx->d_maxdT.alloc(1) != cudaSuccess ||
            cudaHostAlloc(&hab, 2 * sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
            ctx->d_counter.release(); ctx->d_maxdT.release();
            delete ctx;
            return SOC_ERR_NOMEM;
        }
        ctx->h_abort = static_cast<volatile int *>(hab);
        ctx->h_abort[0] = 0;
        ctx->h_abort[1] = 0;
        if (cudaHostGetDevicePointer((void **)&ctx->d_abort, hab, 0) != cudaSuccess) {
            cudaFreeHost(hab);
            ctx->d_counter.release(); ctx->d_maxdT.release();
            delete ctx;
            return SOC_ERR_CUDA;
        }
        *out = ctx;
        return SOC_OK;
    });
}

static void release_cloud(CloudHost *c)
{
    c->cell.release(); c->parent.release(); c->leaf.release(); c->rho.release();
    c->volume.release(); c->kappa.release(); c->ps_pos.release(); c->ps_cdf.release();
    c->tally.release(); c->A_const.release(); c->A.release(); c->dust_w.release(); c->dust_wp.release();
    c->self_tally.release(); c->A_self.release();
    c->e_unit.release(); c->e_unit_w.release(); c->stats.release();
    c->L.release(); c->L_ref.release(); c->A_ref.release(); c->A_d.release(); c->e_unit_n.release();
    c->neg.release(); c->dust_wn.release();
    c->freed = true;
}

soc_status soc_grid_free(soc_ctx *ctx, int cloud_id)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        CK(cudaDeviceSynchronize(), "synchronize before free");
        release_cloud(ctx->clouds[cloud_id]);
        ctx->clouds_dirty = true;
        return SOC_OK;
    });
}

void soc_destroy(soc_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    for (CloudHost *c : ctx->clouds) {
        release_cloud(c);
        delete c;
    }
    ctx->d_clouds.release(); ctx->d_g.release(); ctx->d_w.release(); ctx->d_w_kabs.release();
    ctx->d_nu.release(); ctx->d_kabs.release(); ctx->d_lnE.release(); ctx->d_lnT.release();
    ctx->d_items.release(); ctx->d_prefix.release(); ctx->d_counter.release(); ctx->d_lmax.release();
    ctx->d_maxdT.release();
    ctx->d_wscratch.release();
    ctx->d_level_start.release();
    ctx->d_map_S.release();
    ctx->b_tally.release(); ctx->b_self.release(); ctx->b_stats.release(); ctx->b_maxdT.release();
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->h_abort) cudaFreeHost((void *)ctx->h_abort);
    for (BatchHost *b : ctx->batches)
        if (b) { b->items.release(); b->prefix.release(); b->counter.release(); delete b; }
    for (cudaGraphExec_t g : ctx->graphs)
        if (g) cudaGraphExecDestroy(g);
    delete ctx;
}

const char *soc_last_error(const soc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

soc_status soc_set_launch(soc_ctx *ctx, int threads_per_block, int blocks_per_sm, int chunk)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx) return SOC_ERR_ARG;
        if (threads_per_block < 32 || threads_per_block > 256 || threads_per_block % 32)
            return fail(ctx, SOC_ERR_ARG, "threads_per_block must be a multiple of 32 in [32, 256]");
        if (blocks_per_sm < 0 || chunk < 1 || chunk > 1024) return fail(ctx, SOC_ERR_ARG, "bad blocks_per_sm/chunk");
        ctx->tpb = threads_per_block;
        ctx->bps = blocks_per_sm;
        ctx->chunk = chunk;
        return SOC_OK;
    });
}

soc_status soc_set_refill(soc_ctx *ctx, int min_idle_lanes)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx) return SOC_ERR_ARG;
        if (min_idle_lanes < 1 || min_idle_lanes > 32) return fail(ctx, SOC_ERR_ARG, "min_idle_lanes must be in [1, 32]");
        ctx->refill_min = min_idle_lanes;
        return SOC_OK;
    });
}

soc_status soc_set_scatter_batch(soc_ctx *ctx, int min_lanes)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx) return SOC_ERR_ARG;
        if (min_lanes < 1 || min_lanes > 32) return fail(ctx, SOC_ERR_ARG, "min_lanes must be in [1, 32]");
        ctx->scatter_min = min_lanes;
        return SOC_OK;
    });
}

soc_status soc_probe_read(soc_ctx *ctx, const void *d_buf, uint64_t bytes, int32_t reps, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx) return SOC_ERR_ARG;
        if (!d_buf || bytes == 0 || bytes % 16 || reinterpret_cast<uintptr_t>(d_buf) % 16 || reps < 1)
            return fail(ctx, SOC_ERR_ARG, "probe buffer must be 16-byte aligned, a positive multiple of 16 bytes");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        CK(launch_probe_read(d_buf, bytes, reps, ctx->sms, nullptr, static_cast<cudaStream_t>(stream)), "probe launch");
        return SOC_OK;
    });
}

soc_status soc_set_max_steps(soc_ctx *ctx, uint32_t max_steps)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || max_steps == 0) return SOC_ERR_ARG;
        ctx->max_steps = max_steps;
        return SOC_OK;
    });
}

soc_status soc_abort(soc_ctx *ctx)
{
    if (!ctx || !ctx->h_abort) return SOC_ERR_ARG;
    __atomic_store_n(const_cast<int *>(&ctx->h_abort[0]), 1, __ATOMIC_SEQ_CST);
    return SOC_OK;
}

soc_status soc_abort_clear(soc_ctx *ctx)
{
    if (!ctx || !ctx->h_abort) return SOC_ERR_ARG;
    __atomic_store_n(const_cast<int *>(&ctx->h_abort[1]), 0, __ATOMIC_SEQ_CST);
    __atomic_store_n(const_cast<int *>(&ctx->h_abort[0]), 0, __ATOMIC_SEQ_CST);
    return SOC_OK;
}

soc_status soc_abort_status(soc_ctx *ctx, int *requested, int *cut)
{
    if (!ctx || !ctx->h_abort) return SOC_ERR_ARG;
    if (requested) *requested = __atomic_load_n(const_cast<int *>(&ctx->h_abort[0]), __ATOMIC_SEQ_CST) != 0;
    if (cut) *cut = __atomic_load_n(const_cast<int *>(&ctx->h_abort[1]), __ATOMIC_SEQ_CST) != 0;
    return SOC_OK;
}

soc_status soc_set_timeout(soc_ctx *ctx, double seconds)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx) return SOC_ERR_ARG;
        if (!(seconds >= 0.0) || seconds > 1e9) return fail(ctx, SOC_ERR_ARG, "timeout must be in [0, 1e9] s");
        ctx->timeout_s = seconds;
        return SOC_OK;
    });
}

namespace {

struct GridCheck {
    std::vector<int64_t> start;
    std::vector<int32_t> parent;
    int64_t n = 0, n_root = 0, n_leaf = 0;
};

// One pass of the cell checks over cells [c0, c1): child links (from the
// child array, or the paper's negative-density encoding), leaf densities,
// link targets (the next level, octet-aligned) and one parent per octet
// (claimed by compare-and-swap, so chunks can run concurrently).  With `word`
// the cell words are written too.  Stops at the chunk's first bad cell.
struct CellPass {
    int64_t bad_cell = INT64_MAX;     // first bad cell of the chunk
    std::string msg;
    int64_t dup_octet = INT64_MAX;    // lowest octet claimed twice
    int64_t leaves = 0;
};

void cell_pass(const soc_grid_desc *d, const std::vector<int64_t> &start, int64_t n_root, int64_t c0,
               int64_t c1, int32_t *parent, uint32_t *word, CellPass &r)
{
    if (c0 >= c1) return;
    int lv = 0;
    while (c0 >= start[lv + 1]) ++lv;
    char buf[160];
    for (int64_t c = c0; c < c1; ++c) {
        while (c >= start[lv + 1]) ++lv;
        const float rho = d->rho[c];
        int32_t fc = -1;
        if (d->first_child) {
            fc = d->first_child[c] < 0 ? -1 : d->first_child[c];
        } else if (rho < 0.0f) {
            const float v = -rho;
            if (!(v < 16777216.0f) || v != std::floor(v)) {
                snprintf(buf, sizeof buf, "cell %lld: negative-density link %g not an exact index", (long long)c,
                         (double)rho);
                r.bad_cell = c; r.msg = buf;
                return;
            }
            fc = (int32_t)v;
        }
        if (fc < 0) {
            if (!std::isfinite(rho) || rho < 0.0f) {
                snprintf(buf, sizeof buf, "leaf %lld has invalid density %g", (long long)c, (double)rho);
                r.bad_cell = c; r.msg = buf;
                return;
            }
            if (word) {
                const float v = rho == 0.0f ? 0.0f : rho;          // no -0
                memcpy(&word[c], &v, 4);
            }
            ++r.leaves;
            continue;
        }
        if (lv + 1 >= d->n_levels || fc < start[lv + 1] || fc + 8 > start[lv + 2] || (fc - n_root) % 8 != 0) {
            snprintf(buf, sizeof buf, "cell %lld (level %d): child link %d out of range", (long long)c, lv + 1, fc);
            r.bad_cell = c; r.msg = buf;
            return;
        }
        const int64_t k = (fc - n_root) / 8;
        int32_t expect = -1;
        if (!__atomic_compare_exchange_n(parent + k, &expect, (int32_t)c, false, __ATOMIC_RELAXED,
                                         __ATOMIC_RELAXED))
            r.dup_octet = std::min(r.dup_octet, k);
        if (word) word[c] = kLinkBit | (uint32_t)fc;
    }
}

// Checks of a grid description that need no pass over its cells; fills the
// level starts (with a sentinel entry n at the end).
soc_status grid_header(soc_ctx *ctx, const soc_grid_desc *d, std::vector<int64_t> &start, int64_t &n_root)
{
    if (!d || !d->rho || !d->cells_per_level) return fail(ctx, SOC_ERR_ARG, "null argument");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(ctx, SOC_ERR_ARG, "root grid must be >= 1 cell per axis");
    if (d->n_levels < 1 || d->n_levels > SOC_MAX_LEVELS) return fail(ctx, SOC_ERR_ARG, "n_levels out of [1, 16]");
    if (!(d->root_cell_size > 0.0) || !std::isfinite(d->root_cell_size))
        return fail(ctx, SOC_ERR_ARG, "root_cell_size must be positive");
    n_root = (int64_t)d->nx * d->ny * d->nz;
    if (n_root >= (int64_t)1 << 31) return fail(ctx, SOC_ERR_GRID, "more than 2^31 - 1 root cells");
    start.assign(d->n_levels + 2, 0);
    for (int L = 0; L < d->n_levels; ++L) {
        const int64_t c = d->cells_per_level[L];
        if (c < 0 || (L == 0 && c != n_root) || (L > 0 && c % 8 != 0))
            return fail(ctx, SOC_ERR_GRID, "cells_per_level[%d] = %lld is inconsistent", L, (long long)c);
        start[L + 1] = start[L] + c;
        if (start[L + 1] >= (int64_t)1 << 31) return fail(ctx, SOC_ERR_GRID, "more than 2^31 - 1 cells");
    }
    start[d->n_levels + 1] = start[d->n_levels];
    return SOC_OK;
}

// Host validation of a grid description (paper Sect. 2.1.1 layout) after
// grid_header; with `word` and `leaf` (room for every cell) it also writes
// the cell words and the leaf list.  Large grids are split over host
// threads; the error reported is the one at the lowest cell index, then at
// the lowest octet.
soc_status grid_cells(soc_ctx *ctx, const soc_grid_desc *d, std::vector<int64_t> &start, int64_t n_root,
                      GridCheck &g, uint32_t *word = nullptr, int32_t *leaf = nullptr)
{
    const int64_t n = start[d->n_levels];
    const int64_t n_oct = (n - n_root) / 8;
    std::vector<int32_t> parent(n_oct, -1);
    unsigned hw = std::thread::hardware_concurrency();
    const int n_thr = n >= ((int64_t)1 << 18) ? (int)std::max(1u, std::min(hw, 16u)) : 1;
    std::vector<CellPass> part(n_thr);
    auto bounds = [&](int t) { return std::make_pair(n * t / n_thr, n * (t + 1) / n_thr); };
    auto run = [&](auto &&fn) {
        if (n_thr == 1) { fn(0); return; }
        std::vector<std::thread> th;
        th.reserve(n_thr);
        int t = 0;
        try {
            for (; t < n_thr; ++t) th.emplace_back(fn, t);
        } catch (const std::system_error &) {
            // fewer threads than chunks could start: the rest run on this one
        }
        for (int u = t; u < n_thr; ++u) fn(u);
        for (auto &x : th) x.join();
    };
    run([&](int t) {
        const auto b = bounds(t);
        cell_pass(d, start, n_root, b.first, b.second, parent.data(), word, part[t]);
    });
    int64_t dup = INT64_MAX;
    for (const CellPass &r : part) {
        if (r.bad_cell != INT64_MAX) return fail(ctx, SOC_ERR_GRID, "%s", r.msg.c_str());
        dup = std::min(dup, r.dup_octet);
    }
    if (dup != INT64_MAX) return fail(ctx, SOC_ERR_GRID, "octet %lld has two parents", (long long)dup);
    for (int64_t k = 0; k < n_oct; ++k) {
        if (parent[k] < 0) return fail(ctx, SOC_ERR_GRID, "octet %lld has no parent", (long long)k);
        if (d->parent && d->parent[k] != parent[k])
            return fail(ctx, SOC_ERR_GRID, "parent[%lld] = %d, links say %d", (long long)k, d->parent[k], parent[k]);
    }
    int64_t n_leaf = 0;
    for (const CellPass &r : part) n_leaf += r.leaves;
    if (word && leaf) {                    // leaf list: each chunk from its offset, in cell order
        std::vector<int64_t> off(n_thr, 0);
        for (int t = 1; t < n_thr; ++t) off[t] = off[t - 1] + part[t - 1].leaves;
        run([&](int t) {
            const auto b = bounds(t);
            int32_t *out = leaf + off[t];
            for (int64_t c = b.first; c < b.second; ++c)
                if (!(word[c] & kLinkBit)) *out++ = (int32_t)c;
        });
    }
    start.pop_back();
    g.start.swap(start);
    g.parent.swap(parent);
    g.n = n;
    g.n_root = n_root;
    g.n_leaf = n_leaf;
    return SOC_OK;
}

thread_local std::string g_validate_msg;

}  // namespace

extern "C" soc_status soc_grid_validate(const soc_grid_desc *desc, char *msg, int msg_len)
{
    return guarded(nullptr, [&]() -> soc_status {
        soc_ctx tmp;
        GridCheck g;
        std::vector<int64_t> start;
        int64_t n_root = 0;
        soc_status st = grid_header(&tmp, desc, start, n_root);
        if (st == SOC_OK) st = grid_cells(&tmp, desc, start, n_root, g);
        if (msg && msg_len > 0) {
            strncpy(msg, st == SOC_OK ? "ok" : tmp.err.c_str(), (size_t)msg_len - 1);
            msg[msg_len - 1] = '\0';
        }
        return st;
    });
}

extern "C" soc_status soc_grid_upload(soc_ctx *ctx, const soc_grid_desc *d, int *cloud_id)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || !cloud_id) return fail(ctx, SOC_ERR_ARG, "null argument");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        std::vector<int64_t> lstart;
        int64_t n_root0 = 0;
        soc_status hs = grid_header(ctx, d, lstart, n_root0);
        if (hs != SOC_OK) return hs;
        // cell words (tagged links or FP32 densities, -0 stored as +0) and the
        // leaf list are written in pinned memory by the validating pass and
        // copied once each; densities and volumes are derived on the device
        const int64_t n_max = lstart[d->n_levels];
        if (ctx->h_stage_n < (size_t)n_max) {
            if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
            ctx->h_stage = nullptr;
            ctx->h_stage_n = 0;
            CK(cudaMallocHost(&ctx->h_stage, 2 * sizeof(uint32_t) * (size_t)std::max<int64_t>(n_max, 1)),
               "pinned staging");
            ctx->h_stage_n = (size_t)n_max;
        }
        uint32_t *word = ctx->h_stage;
        int32_t *leaf = reinterpret_cast<int32_t *>(ctx->h_stage + ctx->h_stage_n);
        GridCheck g;
        soc_status vs = grid_cells(ctx, d, lstart, n_root0, g, word, leaf);
        if (vs != SOC_OK) return vs;
        const int64_t n = g.n, n_root = g.n_root, n_oct = (int64_t)g.parent.size(), n_leaf = g.n_leaf;
        std::vector<int64_t> &start = g.start;
        CloudHost *cl = new (std::nothrow) CloudHost();
        if (!cl) return fail(ctx, SOC_ERR_NOMEM, "host allocation");
        cl->nx = d->nx; cl->ny = d->ny; cl->nz = d->nz; cl->n_levels = d->n_levels;
        cl->n_cells = n; cl->n_root = n_root; cl->n_leaf = n_leaf; cl->level_start = start;
        cl->ell = d->root_cell_size;
        const double ell3 = (d->root_cell_size * d->root_cell_size) * d->root_cell_size;
        cudaError_t e = cudaSuccess;
        if ((e = cl->cell.alloc(n)) == cudaSuccess && (e = cl->parent.alloc(n_oct)) == cudaSuccess &&
            (e = cl->leaf.alloc(n_leaf)) == cudaSuccess && (e = cl->rho.alloc(n)) == cudaSuccess &&
            (e = cl->volume.alloc(n)) == cudaSuccess && (e = ctx->d_level_start.alloc(start.size())) == cudaSuccess &&
            (e = cudaMemcpy(cl->cell.p, word, 4 * n, cudaMemcpyHostToDevice)) == cudaSuccess &&
            (n_oct == 0 ||
             (e = cudaMemcpy(cl->parent.p, g.parent.data(), 4 * n_oct, cudaMemcpyHostToDevice)) == cudaSuccess) &&
            (e = cudaMemcpy(cl->leaf.p, leaf, 4 * n_leaf, cudaMemcpyHostToDevice)) == cudaSuccess &&
            (e = cudaMemcpy(ctx->d_level_start.p, start.data(), 8 * start.size(), cudaMemcpyHostToDevice)) ==
                cudaSuccess &&
            (e = launch_cell_init(cl->cell.p, n, ctx->d_level_start.p, d->n_levels, ell3, cl->rho.p, cl->volume.p, 0)) ==
                cudaSuccess &&
            (e = cudaStreamSynchronize(0)) == cudaSuccess) {
        }
        if (e != cudaSuccess) {
            cl->cell.release(); cl->parent.release(); cl->leaf.release(); cl->rho.release(); cl->volume.release();
            delete cl;
            return cuda_fail(ctx, e, "grid upload");
        }
        ctx->clouds.push_back(cl);
        ctx->clouds_dirty = true;
        soc_status st = build_cloud_tables(ctx, *cl);
        if (st != SOC_OK) return st;
        *cloud_id = (int)ctx->clouds.size() - 1;
        return SOC_OK;
    });
}

soc_status soc_dust_upload(soc_ctx *ctx, int n_freq, const double *nu, const double *kabs, const double *ksca,
                           const double *g)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || n_freq < 1 || n_freq > 65535 || !nu || !kabs || !ksca || !g)
            return fail(ctx, SOC_ERR_ARG, "bad dust arguments");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        for (int f = 0; f < n_freq; ++f) {
            if (!(nu[f] > 0) || (f && !(nu[f] > nu[f - 1])) || !(kabs[f] >= 0) || !(ksca[f] >= 0) ||
                !std::isfinite(kabs[f]) || !std::isfinite(ksca[f]) || !(std::fabs(g[f]) < 1.0))
                return fail(ctx, SOC_ERR_ARG, "dust table entry %d invalid", f);
        }
        ctx->n_freq = n_freq;
        ctx->nu.assign(nu, nu + n_freq);
        ctx->kabs.assign(kabs, kabs + n_freq);
        ctx->ksca.assign(ksca, ksca + n_freq);
        ctx->g.assign(g, g + n_freq);
        ctx->w = trapezoid(ctx->nu);
        std::vector<float> gf(n_freq);
        std::vector<double> wk(n_freq);
        for (int f = 0; f < n_freq; ++f) {
            gf[f] = (float)g[f];
            wk[f] = 4.0 * kPi * ctx->w[f] * kabs[f];
        }
        // emission table E(T_k), T_k log-spaced in [kTMin, kTMax]
        std::vector<double> lnE(kTableN), lnT(kTableN);
        const double l0 = std::log(kTMin), l1 = std::log(kTMax);
        for (int k = 0; k < kTableN; ++k) {
            lnT[k] = l0 + (l1 - l0) * k / (kTableN - 1);
            const double T = std::exp(lnT[k]);
            double E = 0.0;
            for (int f = 0; f < n_freq; ++f) E += wk[f] * planck_host(ctx->nu[f], T);
            lnE[k] = std::log(std::max(E, 1e-300));
        }
        CK(ctx->d_g.alloc(n_freq), "alloc");
        CK(ctx->d_w.alloc(n_freq), "alloc");
        CK(ctx->d_w_kabs.alloc(n_freq), "alloc");
        CK(ctx->d_nu.alloc(n_freq), "alloc");
        CK(ctx->d_kabs.alloc(n_freq), "alloc");
        CK(ctx->d_lnE.alloc(kTableN), "alloc");
        CK(ctx->d_lnT.alloc(kTableN), "alloc");
        CK(ctx->d_lmax.alloc(n_freq), "alloc");
        CK(cudaMemcpy(ctx->d_g.p, gf.data(), 4 * n_freq, cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(ctx->d_w.p, ctx->w.data(), 8 * n_freq, cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(ctx->d_w_kabs.p, wk.data(), 8 * n_freq, cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(ctx->d_nu.p, nu, 8 * n_freq, cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(ctx->d_kabs.p, kabs, 8 * n_freq, cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(ctx->d_lnE.p, lnE.data(), 8 * kTableN, cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(ctx->d_lnT.p, lnT.data(), 8 * kTableN, cudaMemcpyHostToDevice), "copy");
        for (CloudHost *c : ctx->clouds) {
            soc_status st = build_cloud_tables(ctx, *c);
            if (st != SOC_OK) return st;
            if (c->n_ps && c->ps_cdf.n != (size_t)c->n_ps * n_freq)
                return fail(ctx, SOC_ERR_STATE, "sources were uploaded for another frequency grid");
        }
        return SOC_OK;
    });
}

soc_status soc_sources_upload(soc_ctx *ctx, int cloud_id, const double *bg_I_nu, int n_ps, const double *ps_pos,
                              const double *ps_L_nu)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (ctx->n_freq == 0) return fail(ctx, SOC_ERR_STATE, "soc_dust_upload must come first");
        if (n_ps < 0 || (n_ps > 0 && (!ps_pos || !ps_L_nu))) return fail(ctx, SOC_ERR_ARG, "bad point sources");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        CloudHost &cl = *ctx->clouds[cloud_id];
        const int nf = ctx->n_freq;
        cl.bg_I.clear();
        if (bg_I_nu) {
            for (int f = 0; f < nf; ++f)
                if (!(bg_I_nu[f] >= 0) || !std::isfinite(bg_I_nu[f])) return fail(ctx, SOC_ERR_ARG, "bad bg_I_nu[%d]", f);
            cl.bg_I.assign(bg_I_nu, bg_I_nu + nf);
        }
        cl.n_ps = n_ps;
        cl.ps_L_total.assign(nf, 0.0);
        if (n_ps > 0) {
            const int nr[3] = {cl.nx, cl.ny, cl.nz};
            std::vector<float> pos(3 * n_ps);
            for (int k = 0; k < n_ps; ++k)
                for (int a = 0; a < 3; ++a) {
                    const double v = ps_pos[3 * k + a];
                    if (!(v > 0.0 && v < nr[a])) return fail(ctx, SOC_ERR_ARG, "point source %d outside the grid", k);
                    pos[3 * k + a] = (float)v;
                }
            std::vector<float> cdf((size_t)nf * n_ps);
            for (int f = 0; f < nf; ++f) {
                double tot = 0.0;
                for (int k = 0; k < n_ps; ++k) {
                    const double L = ps_L_nu[(size_t)k * nf + f];
                    if (!(L >= 0) || !std::isfinite(L)) return fail(ctx, SOC_ERR_ARG, "bad ps_L_nu");
                    tot += L;
                }
                cl.ps_L_total[f] = tot;
                double run = 0.0;
                for (int k = 0; k < n_ps; ++k) {
                    run += ps_L_nu[(size_t)k * nf + f];
                    cdf[(size_t)f * n_ps + k] = (float)(run / (tot > 0 ? tot : 1.0));
                }
                cdf[(size_t)f * n_ps + n_ps - 1] = 1.0f;
            }
            CK(cl.ps_pos.alloc(pos.size()), "alloc");
            CK(cl.ps_cdf.alloc(cdf.size()), "alloc");
            CK(cudaMemcpy(cl.ps_pos.p, pos.data(), 4 * pos.size(), cudaMemcpyHostToDevice), "copy");
            CK(cudaMemcpy(cl.ps_cdf.p, cdf.data(), 4 * cdf.size(), cudaMemcpyHostToDevice), "copy");
        }
        ctx->clouds_dirty = true;
        return SOC_OK;
    });
}

soc_status soc_package_energy(soc_ctx *ctx, int cloud_id, int source, uint64_t n_packages, double *e_unit)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!e_unit || n_packages == 0) return fail(ctx, SOC_ERR_ARG, "bad arguments");
        const CloudHost &cl = *ctx->clouds[cloud_id];
        const int nf = ctx->n_freq;
        if (source == SOC_SRC_BACKGROUND) {
            if (cl.bg_I.empty()) return fail(ctx, SOC_ERR_STATE, "no background uploaded");
            const double S = 2.0 * ((double)cl.nx * cl.ny + (double)cl.ny * cl.nz + (double)cl.nz * cl.nx) * cl.ell * cl.ell;
            for (int f = 0; f < nf; ++f) e_unit[f] = kPi * cl.bg_I[f] * S / (double)n_packages / kWUnit;
            return SOC_OK;
        }
        if (source == SOC_SRC_POINT) {
            if (cl.n_ps == 0) return fail(ctx, SOC_ERR_STATE, "no point sources uploaded");
            for (int f = 0; f < nf; ++f) e_unit[f] = cl.ps_L_total[f] / (double)n_packages / kWUnit;
            return SOC_OK;
        }
        return fail(ctx, SOC_ERR_ARG, "source must be background or point");
    });
}

// Check batch item i against the context and write its device form into d
// (no heap use: also called by the allocation-free tracer entry).
static soc_status check_item(soc_ctx *ctx, const soc_batch_item &it, int i, DevItem &d)
{
    if (it.cloud < 0 || it.cloud >= (int)ctx->clouds.size() || ctx->clouds[it.cloud]->freed)
        return fail(ctx, SOC_ERR_ARG, "item %d: bad or freed cloud", i);
    const CloudHost &cl = *ctx->clouds[it.cloud];
    if (it.freq < 0 || it.freq >= ctx->n_freq) return fail(ctx, SOC_ERR_ARG, "item %d: bad freq", i);
    if (it.iteration < 0 || it.iteration > 65535) return fail(ctx, SOC_ERR_ARG, "item %d: bad iteration", i);
    if (it.pid_offset + it.n_packages > 0xFFFFFFFFull || it.pid_offset > 0xFFFFFFFFull)
        return fail(ctx, SOC_ERR_ARG, "item %d: package ids exceed 2^32", i);
    if (it.tally_offset < 0) return fail(ctx, SOC_ERR_ARG, "item %d: negative tally offset", i);
    if (it.source == SOC_SRC_BACKGROUND || it.source == SOC_SRC_POINT) {
        if (it.w0 == 0 || it.w0 > SOC_W_UNIT) return fail(ctx, SOC_ERR_ARG, "item %d: w0 out of [1, 2^31]", i);
        if (it.source == SOC_SRC_POINT && cl.n_ps == 0)
            return fail(ctx, SOC_ERR_STATE, "item %d: cloud has no point sources", i);
    } else if (it.source == SOC_SRC_DUST) {
        if (!it.d_dust_w || it.n_per_cell == 0) return fail(ctx, SOC_ERR_ARG, "item %d: dust weights missing", i);
        if (!(it.reserved & SOC_ITEM_WEIGHTED) && it.pid_offset + it.n_packages > (uint64_t)cl.n_leaf * it.n_per_cell)
            return fail(ctx, SOC_ERR_ARG, "item %d: more dust packages than n_leaf*n_per_cell", i);
    } else {
        return fail(ctx, SOC_ERR_ARG, "item %d: unknown source %d", i, it.source);
    }
    memset(&d, 0, sizeof d);
    d.cloud = it.cloud; d.freq = it.freq; d.source = it.source; d.iteration = it.iteration;
    d.pid_offset = (uint32_t)it.pid_offset; d.n_per_cell = it.n_per_cell ? it.n_per_cell : 1;
    d.flags = (it.source == SOC_SRC_DUST && (it.reserved & SOC_ITEM_WEIGHTED)) ? kItemWeighted : 0u;
    d.w0 = it.w0; d.tally_offset = it.tally_offset; d.dust_w = it.d_dust_w;
    return SOC_OK;
}

// Check every item and write the device forms and the exclusive prefix of
// package counts into caller-given arrays dv[n_items], prefix[n_items + 1].
static soc_status prepare_items_into(soc_ctx *ctx, const soc_batch_item *items, int n_items, DevItem *dv,
                                     uint64_t *prefix)
{
    prefix[0] = 0;
    for (int i = 0; i < n_items; ++i) {
        const soc_status st = check_item(ctx, items[i], i, dv[i]);
        if (st != SOC_OK) return st;
        prefix[i + 1] = prefix[i] + items[i].n_packages;
    }
    return SOC_OK;
}

// Check the batch items and convert them to the device form (host vectors).
static soc_status prepare_items(soc_ctx *ctx, const soc_batch_item *items, int n_items, std::vector<DevItem> &dv,
                                std::vector<uint64_t> &prefix)
{
    dv.assign(n_items, DevItem{});
    prefix.assign(n_items + 1, 0);
    return prepare_items_into(ctx, items, n_items, dv.data(), prefix.data());
}

// The step fields of the one cloud all items use; cell = nullptr when they
// use several (the tracer then reads them through each lane's cloud).
static HotCloud one_cloud(const soc_ctx *ctx, const soc_batch_item *items, int n_items)
{
    HotCloud h{};
    for (int i = 1; i < n_items; ++i)
        if (items[i].cloud != items[0].cloud) return h;
    const CloudHost &c = *ctx->clouds[items[0].cloud];
    h.cell = c.cell.p;
    h.parent = c.parent.p;
    h.nx = c.nx; h.ny = c.ny; h.nz = c.nz;
    h.n_root = (int32_t)c.n_root;
    return h;
}

// 1 when every item's cloud is a regular grid (one level).
static int32_t all_regular(const soc_ctx *ctx, const soc_batch_item *items, int n_items)
{
    for (int i = 0; i < n_items; ++i)
        if (ctx->clouds[items[i].cloud]->n_levels != 1) return 0;
    return 1;
}

// Launch shape of the tracer for `total` work indices.
static void launch_geometry(soc_ctx *ctx, uint64_t total, bool regular, int &grid_out, int &variant)
{
    variant = ctx->bps >= 4 ? 4 : 3;
    const int limit = std::max(1, ctx->occ[regular ? 1 : 0][variant - 3][ctx->tpb / 32 - 1]);
    const int per_sm = ctx->bps > 0 ? std::min(ctx->bps, limit) : limit;
    const uint64_t warps_needed = (total + 31) / 32;
    int64_t grid = (int64_t)ctx->sms * per_sm;
    const int64_t grid_need = (int64_t)((warps_needed * 32 + ctx->tpb - 1) / ctx->tpb);
    if (grid_need < grid) grid = grid_need < 1 ? 1 : grid_need;
    grid_out = (int)grid;
}

// SOC_ERR_STATE when `s` is being captured into a CUDA graph: the direct
// tracer entries copy their tables from pageable host memory, which a
// capture cannot hold (prepared batches, soc_batch_launch, can be captured).
static soc_status refuse_capture(soc_ctx *ctx, cudaStream_t s, const char *who)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();            // not sticky: leave no error for the next launch check
        return fail(ctx, SOC_ERR_STATE, "%s: stream capture state unavailable (%s); use soc_batch_launch in graphs",
                    who, cudaGetErrorString(e));
    }
    if (cs != cudaStreamCaptureStatusNone)
        return fail(ctx, SOC_ERR_STATE, "%s copies from host memory and cannot be captured; "
                    "capture soc_batch_launch instead", who);
    return SOC_OK;
}

soc_status soc_simulate_frequency_batch(soc_ctx *ctx, const soc_batch_item *items, int n_items, int64_t *d_tally,
                                        int64_t *d_stats, uint32_t *d_pkg_steps, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        return soc_simulate_frequency_batch_ex(ctx, items, n_items, d_tally, nullptr, d_stats, d_pkg_steps, stream);
    });
}

soc_status soc_simulate_frequency_batch_ex(soc_ctx *ctx, const soc_batch_item *items, int n_items, int64_t *d_tally,
                                           int64_t *d_self, int64_t *d_stats, uint32_t *d_pkg_steps, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || !items || n_items < 1 || !d_tally || !d_stats) return fail(ctx, SOC_ERR_ARG, "null argument");
        if (ctx->n_freq == 0) return fail(ctx, SOC_ERR_STATE, "soc_dust_upload must come first");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        cudaStream_t s = (cudaStream_t)stream;
        if (soc_status cst = refuse_capture(ctx, s, "soc_simulate_frequency_batch")) return cst;
        std::vector<DevItem> dv;
        std::vector<uint64_t> prefix;
        soc_status pst = prepare_items(ctx, items, n_items, dv, prefix);
        if (pst != SOC_OK) return pst;
        const uint64_t total = prefix[n_items];
        soc_status st = sync_clouds(ctx);
        if (st) return st;
        if (total == 0) return SOC_OK;
        CK(ctx->d_items.alloc(n_items), "alloc items");
        CK(ctx->d_prefix.alloc(n_items + 1), "alloc prefix");
        CK(cudaMemcpyAsync(ctx->d_items.p, dv.data(), sizeof(DevItem) * n_items, cudaMemcpyHostToDevice, s), "copy items");
        CK(cudaMemcpyAsync(ctx->d_prefix.p, prefix.data(), 8 * (n_items + 1), cudaMemcpyHostToDevice, s), "copy prefix");
        CK(cudaMemsetAsync(ctx->d_counter.p, 0, sizeof(unsigned long long), s), "zero counter");
        TraceParams P;
        P.clouds = ctx->d_clouds.p;
        P.items = ctx->d_items.p;
        P.prefix = ctx->d_prefix.p;
        P.g_hg = ctx->d_g.p;
        P.tally = reinterpret_cast<unsigned long long *>(d_tally);
        P.self = reinterpret_cast<unsigned long long *>(d_self);
        P.stats = reinterpret_cast<unsigned long long *>(d_stats);
        P.pkg_steps = d_pkg_steps;
        P.counter = ctx->d_counter.p;
        P.abort_flag = ctx->d_abort;
        P.cut = ctx->d_abort + 1;
        P.total = total;
        P.seed = ctx->seed;
        P.n_items = n_items;
        P.max_steps = ctx->max_steps;
        P.chunk = ctx->chunk;
        P.refill_min = ctx->refill_min;
        P.scatter_min = ctx->scatter_min;
        P.hot = one_cloud(ctx, items, n_items);
        P.regular = all_regular(ctx, items, n_items);
        int grid = 1, variant = 3;
        launch_geometry(ctx, total, P.regular != 0, grid, variant);
        CK(launch_trace(P, grid, ctx->tpb, variant, s), "trace launch");
        // the host copies above used pageable buffers: they are staged before return
        return SOC_OK;
    });
}

soc_status soc_batch_create(soc_ctx *ctx, const soc_batch_item *items, int n_items, int *batch_id)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || !items || n_items < 1 || !batch_id) return fail(ctx, SOC_ERR_ARG, "null argument");
        if (ctx->n_freq == 0) return fail(ctx, SOC_ERR_STATE, "soc_dust_upload must come first");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        std::vector<DevItem> dv;
        std::vector<uint64_t> prefix;
        soc_status st = prepare_items(ctx, items, n_items, dv, prefix);
        if (st != SOC_OK) return st;
        BatchHost *b = new (std::nothrow) BatchHost();
        if (!b) return fail(ctx, SOC_ERR_NOMEM, "host allocation");
        b->n_items = n_items;
        b->total = prefix[n_items];
        b->hot = one_cloud(ctx, items, n_items);
        b->regular = all_regular(ctx, items, n_items);
        cudaError_t e = cudaSuccess;
        if ((e = b->items.alloc(n_items)) != cudaSuccess || (e = b->prefix.alloc(n_items + 1)) != cudaSuccess ||
            (e = b->counter.alloc(1)) != cudaSuccess ||
            (e = cudaMemcpy(b->items.p, dv.data(), sizeof(DevItem) * n_items, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(b->prefix.p, prefix.data(), 8 * (n_items + 1), cudaMemcpyHostToDevice)) != cudaSuccess) {
            b->items.release(); b->prefix.release(); b->counter.release();
            delete b;
            return cuda_fail(ctx, e, "batch upload");
        }
        ctx->batches.push_back(b);
        *batch_id = (int)ctx->batches.size() - 1;
        return sync_clouds(ctx);                 // the launch must not need to upload the grid table
    });
}

soc_status soc_batch_launch(soc_ctx *ctx, int batch_id, int64_t *d_tally, int64_t tally_len, int64_t *d_stats,
                            uint32_t *d_pkg_steps, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || batch_id < 0 || batch_id >= (int)ctx->batches.size() || !ctx->batches[batch_id])
            return fail(ctx, SOC_ERR_ARG, "bad batch id");
        if (!d_tally || !d_stats || tally_len < 0) return fail(ctx, SOC_ERR_ARG, "null argument");
        if (ctx->clouds_dirty) return fail(ctx, SOC_ERR_STATE, "grids changed after soc_batch_create");
        const BatchHost &b = *ctx->batches[batch_id];
        cudaStream_t s = (cudaStream_t)stream;
        if (tally_len) CK(cudaMemsetAsync(d_tally, 0, sizeof(int64_t) * tally_len, s), "zero tally");
        CK(cudaMemsetAsync(d_stats, 0, sizeof(int64_t) * 4 * b.n_items, s), "zero stats");
        if (b.total == 0) return SOC_OK;
        CK(cudaMemsetAsync(b.counter.p, 0, sizeof(unsigned long long), s), "zero counter");
        TraceParams P;
        P.clouds = ctx->d_clouds.p;
        P.items = b.items.p;
        P.prefix = b.prefix.p;
        P.g_hg = ctx->d_g.p;
        P.tally = reinterpret_cast<unsigned long long *>(d_tally);
        P.self = nullptr;
        P.stats = reinterpret_cast<unsigned long long *>(d_stats);
        P.pkg_steps = d_pkg_steps;
        P.counter = b.counter.p;
        P.abort_flag = ctx->d_abort;
        P.cut = ctx->d_abort + 1;
        P.total = b.total;
        P.seed = ctx->seed;
        P.n_items = b.n_items;
        P.max_steps = ctx->max_steps;
        P.chunk = ctx->chunk;
        P.refill_min = ctx->refill_min;
        P.scatter_min = ctx->scatter_min;
        P.hot = b.hot;
        P.regular = b.regular;
        int grid = 1, variant = 3;
        launch_geometry(ctx, b.total, P.regular != 0, grid, variant);
        CK(launch_trace(P, grid, ctx->tpb, variant, s), "trace launch");
        return SOC_OK;
    });
}

soc_status soc_batch_destroy(soc_ctx *ctx, int batch_id)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || batch_id < 0 || batch_id >= (int)ctx->batches.size() || !ctx->batches[batch_id])
            return fail(ctx, SOC_ERR_ARG, "bad batch id");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        CK(cudaDeviceSynchronize(), "synchronize before free");
        BatchHost *b = ctx->batches[batch_id];
        b->items.release(); b->prefix.release(); b->counter.release();
        delete b;
        ctx->batches[batch_id] = nullptr;
        return SOC_OK;
    });
}

soc_status soc_capture_begin(soc_ctx *ctx, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || !stream) return fail(ctx, SOC_ERR_ARG, "capture needs a non-default stream");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        soc_status st = sync_clouds(ctx);
        if (st) return st;
        CK(cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        return SOC_OK;
    });
}

soc_status soc_capture_end(soc_ctx *ctx, void *stream, int *graph_id)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || !stream || !graph_id) return fail(ctx, SOC_ERR_ARG, "null argument");
        cudaGraph_t g = nullptr;
        CK(cudaStreamEndCapture((cudaStream_t)stream, &g), "end capture");
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
        ctx->graphs.push_back(ex);
        *graph_id = (int)ctx->graphs.size() - 1;
        return SOC_OK;
    });
}

soc_status soc_graph_launch(soc_ctx *ctx, int graph_id, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || graph_id < 0 || graph_id >= (int)ctx->graphs.size() || !ctx->graphs[graph_id])
            return fail(ctx, SOC_ERR_ARG, "bad graph id");
        CK(cudaGraphLaunch(ctx->graphs[graph_id], (cudaStream_t)stream), "graph launch");
        return SOC_OK;
    });
}

soc_status soc_graph_destroy(soc_ctx *ctx, int graph_id)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || graph_id < 0 || graph_id >= (int)ctx->graphs.size() || !ctx->graphs[graph_id])
            return fail(ctx, SOC_ERR_ARG, "bad graph id");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        CK(cudaDeviceSynchronize(), "synchronize before free");
        cudaGraphExecDestroy(ctx->graphs[graph_id]);
        ctx->graphs[graph_id] = nullptr;
        return SOC_OK;
    });
}

soc_status soc_dust_emission(soc_ctx *ctx, int cloud_id, const float *d_T, int freq_lo, int n_freq,
                             uint32_t n_per_cell, uint64_t *d_w, double *d_e_unit, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_T || !d_w || !d_e_unit || n_per_cell == 0 || freq_lo < 0 || n_freq < 1 || freq_lo + n_freq > ctx->n_freq)
            return fail(ctx, SOC_ERR_ARG, "bad dust-emission arguments");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        if ((st = sync_clouds(ctx))) return st;
        const CloudHost &cl = *ctx->clouds[cloud_id];
        TempTables tt{ctx->n_freq, ctx->d_w_kabs.p, ctx->d_w.p, ctx->d_nu.p, ctx->d_kabs.p, ctx->d_lnE.p, ctx->d_lnT.p};
        CK(launch_dust_emission(ctx->d_clouds.p + cloud_id, cl.n_leaf, tt, d_T, freq_lo, n_freq, n_per_cell, d_w,
                                d_e_unit, ctx->d_lmax.p, (cudaStream_t)stream),
           "dust emission");
        return SOC_OK;
    });
}

soc_status soc_dust_weighted(soc_ctx *ctx, int cloud_id, const uint64_t *d_u, const double *d_e_unit_uniform,
                             int n_freq, uint64_t n_total, uint32_t cap, uint64_t *d_out, double *d_e_unit, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_u || !d_e_unit_uniform || !d_out || !d_e_unit || n_freq < 1 || n_total < 1 || cap < 1)
            return fail(ctx, SOC_ERR_ARG, "bad weighted-sampling arguments");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        const CloudHost &cl = *ctx->clouds[cloud_id];
        const int64_t n_chunks = (cl.n_leaf + 1023) / 1024;
        CK(ctx->d_wscratch.alloc((size_t)n_freq * (1 + n_chunks)), "alloc weighted-sampling scratch");
        CK(launch_dust_weighted(cl.n_leaf, n_freq, d_u, d_e_unit_uniform, n_total, cap, d_out, d_e_unit,
                                ctx->d_wscratch.p, (cudaStream_t)stream),
           "weighted sampling");
        return SOC_OK;
    });
}

soc_status soc_dust_reweight(soc_ctx *ctx, int cloud_id, const uint64_t *d_u, const double *d_e_unit_uniform,
                             int n_freq, uint64_t *d_inout, double *d_e_unit, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_u || !d_e_unit_uniform || !d_inout || !d_e_unit || n_freq < 1)
            return fail(ctx, SOC_ERR_ARG, "bad re-weighting arguments");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        const CloudHost &cl = *ctx->clouds[cloud_id];
        CK(ctx->d_wscratch.alloc((size_t)n_freq), "alloc weighted-sampling scratch");
        CK(launch_dust_reweight(cl.n_leaf, n_freq, d_u, d_e_unit_uniform, d_inout, d_e_unit, ctx->d_wscratch.p,
                                (cudaStream_t)stream),
           "dust re-weighting");
        return SOC_OK;
    });
}

soc_status soc_dust_luminosity(soc_ctx *ctx, int cloud_id, const float *d_T, int freq_lo, int n_freq, double *d_L,
                               void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_T || !d_L || n_freq < 1 || freq_lo < 0 || freq_lo + n_freq > ctx->n_freq)
            return fail(ctx, SOC_ERR_ARG, "bad dust-luminosity arguments");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        if ((st = sync_clouds(ctx))) return st;
        const CloudHost &cl = *ctx->clouds[cloud_id];
        TempTables tt{ctx->n_freq, ctx->d_w_kabs.p, ctx->d_w.p, ctx->d_nu.p, ctx->d_kabs.p, ctx->d_lnE.p, ctx->d_lnT.p};
        CK(launch_dust_luminosity(ctx->d_clouds.p + cloud_id, cl.n_leaf, tt, d_T, freq_lo, n_freq, d_L,
                                  (cudaStream_t)stream),
           "dust luminosity");
        return SOC_OK;
    });
}

soc_status soc_reference_delta(soc_ctx *ctx, int cloud_id, int n_freq, const double *d_L, double *d_L_ref,
                               double w, uint64_t *d_u, uint8_t *d_neg, double *d_e_unit_uniform, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_L || !d_L_ref || !d_u || !d_neg || !d_e_unit_uniform || n_freq < 1 || !(w >= 0.0 && w <= 1.0))
            return fail(ctx, SOC_ERR_ARG, "bad reference-delta arguments");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        const CloudHost &cl = *ctx->clouds[cloud_id];
        CK(ctx->d_wscratch.alloc((size_t)n_freq), "alloc scratch");
        CK(launch_reference_delta(cl.n_leaf, n_freq, d_L, d_L_ref, w, d_u, d_neg, d_e_unit_uniform, ctx->d_wscratch.p,
                                  (cudaStream_t)stream),
           "reference delta");
        return SOC_OK;
    });
}

soc_status soc_dust_split(soc_ctx *ctx, int cloud_id, int n_freq, const uint8_t *d_neg, uint64_t *d_alloc,
                          uint64_t *d_alloc_neg, const double *d_e_unit, double *d_e_unit_neg, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_neg || !d_alloc || !d_alloc_neg || !d_e_unit || !d_e_unit_neg || n_freq < 1 || d_alloc == d_alloc_neg)
            return fail(ctx, SOC_ERR_ARG, "bad split arguments");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        const CloudHost &cl = *ctx->clouds[cloud_id];
        CK(launch_dust_split(cl.n_leaf, n_freq, d_neg, d_alloc, d_alloc_neg, d_e_unit, d_e_unit_neg,
                             (cudaStream_t)stream),
           "dust split");
        return SOC_OK;
    });
}

soc_status soc_reference_update(soc_ctx *ctx, int cloud_id, double *d_A_ref, const double *d_A_d, double w,
                                const double *d_A_const, double *d_A_out, int out_mean, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_A_ref || !d_A_d || !(w >= 0.0 && w <= 1.0)) return fail(ctx, SOC_ERR_ARG, "bad reference-update arguments");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        const CloudHost &cl = *ctx->clouds[cloud_id];
        CK(launch_reference_update(cl.n_cells, d_A_ref, d_A_d, w, d_A_const, d_A_out, out_mean != 0,
                                   (cudaStream_t)stream),
           "reference update");
        return SOC_OK;
    });
}

soc_status soc_absorbed_power(soc_ctx *ctx, int cloud_id, const int64_t *d_tally, int64_t tally_stride,
                              const double *d_e_unit, const double *d_A_in, double *d_A_out, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        const CloudHost &cl = *ctx->clouds[cloud_id];
        if (!d_tally || !d_e_unit || !d_A_out || tally_stride < cl.n_cells)
            return fail(ctx, SOC_ERR_ARG, "bad absorbed-power arguments");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        if ((st = sync_clouds(ctx))) return st;
        CK(launch_absorbed_power(ctx->d_clouds.p + cloud_id, cl.n_cells, d_tally, tally_stride, d_e_unit, ctx->d_w.p,
                                 ctx->n_freq, d_A_in, d_A_out, (cudaStream_t)stream),
           "absorbed power");
        return SOC_OK;
    });
}

soc_status soc_update_temperature(soc_ctx *ctx, int cloud_id, const double *d_A, float *d_T, double *d_max_dT,
                                  void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_A || !d_T) return fail(ctx, SOC_ERR_ARG, "null argument");
        if (ctx->n_freq == 0) return fail(ctx, SOC_ERR_STATE, "soc_dust_upload must come first");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        if ((st = sync_clouds(ctx))) return st;
        const CloudHost &cl = *ctx->clouds[cloud_id];
        TempTables tt{ctx->n_freq, ctx->d_w_kabs.p, ctx->d_w.p, ctx->d_nu.p, ctx->d_kabs.p, ctx->d_lnE.p, ctx->d_lnT.p};
        CK(launch_update_temperature(ctx->d_clouds.p + cloud_id, cl.n_cells, tt, d_A, d_T, d_max_dT,
                                     (cudaStream_t)stream),
           "temperature");
        return SOC_OK;
    });
}

soc_status soc_update_temperature_ali(soc_ctx *ctx, int cloud_id, const double *d_A, const double *d_A_self, float *d_T,
                                      double *d_max_dT, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_A || !d_A_self || !d_T) return fail(ctx, SOC_ERR_ARG, "null argument");
        if (ctx->n_freq == 0) return fail(ctx, SOC_ERR_STATE, "soc_dust_upload must come first");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        if ((st = sync_clouds(ctx))) return st;
        const CloudHost &cl = *ctx->clouds[cloud_id];
        TempTables tt{ctx->n_freq, ctx->d_w_kabs.p, ctx->d_w.p, ctx->d_nu.p, ctx->d_kabs.p, ctx->d_lnE.p, ctx->d_lnT.p};
        CK(launch_update_temperature_ali(ctx->d_clouds.p + cloud_id, cl.n_cells, tt, d_A, d_A_self, d_T, d_max_dT,
                                         (cudaStream_t)stream),
           "temperature (ALI)");
        return SOC_OK;
    });
}

soc_status soc_seed_features(soc_ctx *ctx, int cloud_id, const float *d_T, const float *d_T_prev,
                             const float *d_T_prev2, const double *norm, int n_features, float *d_x, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_T || !norm || !d_x) return fail(ctx, SOC_ERR_ARG, "null argument");
        if (n_features < 2 || n_features > 4) return fail(ctx, SOC_ERR_ARG, "n_features must be 2, 3 or 4");
        if (n_features >= 3 && !d_T_prev) return fail(ctx, SOC_ERR_ARG, "3 or 4 features need d_T_prev");
        if (n_features == 4 && !d_T_prev2) return fail(ctx, SOC_ERR_ARG, "4 features need d_T_prev2");
        for (int k = 1; k < 2 * n_features; k += 2)
            if (!(norm[k] > 0.0)) return fail(ctx, SOC_ERR_ARG, "normalisation widths must be > 0");
        const CloudHost &cl = *ctx->clouds[cloud_id];
        if (cl.n_levels != 1 || cl.nx != cl.ny || cl.nx != cl.nz || cl.nx % 8)
            return fail(ctx, SOC_ERR_ARG, "the network takes regular cubic grids with a side that is a multiple of 8");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        CK(launch_seed_features(d_T, d_T_prev, d_T_prev2, cl.rho.p, cl.n_cells, n_features, norm, d_x,
                                (cudaStream_t)stream),
           "seed features");
        return SOC_OK;
    });
}

soc_status soc_seed_transform(soc_ctx *ctx, int cloud_id, const float *d_T1, const float *d_pred,
                              const soc_seed_map *map, float *d_T_seed, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_T1 || !d_pred || !map || !d_T_seed) return fail(ctx, SOC_ERR_ARG, "null argument");
        if (!std::isfinite(map->y_mean) || !std::isfinite(map->y_std) || !(map->shrink > 0.0) ||
            !std::isfinite(map->shrink))
            return fail(ctx, SOC_ERR_ARG, "y_mean, y_std must be finite and shrink > 0");
        if (map->n_bins < 0 || map->n_bins > SOC_SEED_MAX_BINS ||
            (map->n_bins > 0 && !(map->lnT1_hi > map->lnT1_lo)))
            return fail(ctx, SOC_ERR_ARG, "envelope: n_bins in [0, %d] and lnT1_lo < lnT1_hi", SOC_SEED_MAX_BINS);
        for (int b = 0; b < map->n_bins; ++b)
            if (!(map->y_lo[b] <= map->y_hi[b])) return fail(ctx, SOC_ERR_ARG, "envelope bin %d: y_lo > y_hi", b);
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        CK(launch_seed_transform(d_T1, d_pred, ctx->clouds[cloud_id]->n_cells, *map, d_T_seed, (cudaStream_t)stream),
           "seed transform");
        return SOC_OK;
    });
}

soc_status soc_map(soc_ctx *ctx, int cloud_id, const float *d_T, int freq, const double *dir, const double *up, int npx,
                   int npy, double pix_size, const double *center, double I_bg, float *d_map, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!d_T || !dir || !up || !center || !d_map || npx < 1 || npy < 1 || !(pix_size > 0.0))
            return fail(ctx, SOC_ERR_ARG, "bad map arguments");
        if (freq < 0 || freq >= ctx->n_freq) return fail(ctx, SOC_ERR_ARG, "bad frequency index");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        if ((st = sync_clouds(ctx))) return st;
        const CloudHost &cl = *ctx->clouds[cloud_id];
        MapParams M;
        memset(&M, 0, sizeof M);
        const double dn = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        if (!(dn > 0.0)) return fail(ctx, SOC_ERR_ARG, "zero view direction");
        for (int a = 0; a < 3; ++a) M.d[a] = dir[a] / dn;
        // e1 = up x d (normalised), e2 = d x e1
        double e1[3] = {up[1] * M.d[2] - up[2] * M.d[1], up[2] * M.d[0] - up[0] * M.d[2], up[0] * M.d[1] - up[1] * M.d[0]};
        const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        if (!(n1 > 1e-12)) return fail(ctx, SOC_ERR_ARG, "up vector parallel to the view direction");
        for (int a = 0; a < 3; ++a) M.e1[a] = e1[a] / n1;
        M.e2[0] = M.d[1] * M.e1[2] - M.d[2] * M.e1[1];
        M.e2[1] = M.d[2] * M.e1[0] - M.d[0] * M.e1[2];
        M.e2[2] = M.d[0] * M.e1[1] - M.d[1] * M.e1[0];
        for (int a = 0; a < 3; ++a) M.c[a] = center[a];
        M.cloud = ctx->d_clouds.p + cloud_id;
        M.T = d_T;
        M.map = d_map;
        M.pix = pix_size;
        M.nu = ctx->nu[freq];
        const double kext = ctx->kabs[freq] + ctx->ksca[freq];
        M.kext_root = kext * cl.ell;
        M.kabs_over_kext = kext > 0.0 ? ctx->kabs[freq] / kext : 0.0;
        M.I_bg = I_bg;
        M.npx = npx;
        M.npy = npy;
        M.max_cells = 100000000u;
        CK(ctx->d_map_S.alloc(cl.n_cells), "map source scratch");
        M.S = ctx->d_map_S.p;
        CK(launch_map(M, cl.n_cells, ctx->sms, (cudaStream_t)stream), "map");
        return SOC_OK;
    });
}

}  // extern "C"

namespace {
// Host watchdog of one soc_iterate call: sets the context's abort flag once
// `seconds` have passed, unless the call ends first (the destructor stops it).
struct Watchdog {
    std::mutex m;
    std::condition_variable cv;
    bool done = false;
    std::thread t;
    void start(volatile int *flag, double seconds)
    {
        t = std::thread([this, flag, seconds] {
            std::unique_lock<std::mutex> lk(m);
            if (!cv.wait_for(lk, std::chrono::duration<double>(seconds), [this] { return done; }))
                __atomic_store_n(const_cast<int *>(flag), 1, __ATOMIC_SEQ_CST);
        });
    }
    ~Watchdog()
    {
        if (!t.joinable()) return;
        {
            std::lock_guard<std::mutex> lk(m);
            done = true;
        }
        cv.notify_all();
        t.join();
    }
};
}  // namespace

extern "C" {

soc_status soc_iterate(soc_ctx *ctx, int cloud_id, const soc_iterate_params *prm, const float *d_T_seed,
                       float *d_T_out, soc_iterate_result *res, double *dT_history, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        soc_status st = check_cloud(ctx, cloud_id);
        if (st) return st;
        if (!prm || !d_T_out || prm->max_iter < 0) return fail(ctx, SOC_ERR_ARG, "bad iterate arguments");
        if (ctx->n_freq == 0) return fail(ctx, SOC_ERR_STATE, "soc_dust_upload must come first");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        CloudHost &cl = *ctx->clouds[cloud_id];
        cudaStream_t s = (cudaStream_t)stream;
        const int nf = ctx->n_freq;
        const int64_t n = cl.n_cells;
        if (prm->n_background && cl.bg_I.empty()) return fail(ctx, SOC_ERR_STATE, "no background uploaded");
        if (prm->n_point && cl.n_ps == 0) return fail(ctx, SOC_ERR_STATE, "no point sources uploaded");
        CK(cl.tally.alloc((size_t)nf * n), "alloc tally");
        CK(cl.A_const.alloc(n), "alloc A");
        CK(cl.A.alloc(n), "alloc A");
        CK(cl.e_unit.alloc(nf), "alloc e_unit");
        CK(cl.stats.alloc((size_t)4 * nf), "alloc stats");
        if (prm->max_iter > 0) CK(cl.dust_w.alloc((size_t)nf * cl.n_leaf), "alloc dust weights");
        const bool weighted = prm->n_weighted > 0;
        if (weighted && prm->weighted_cap == 0) return fail(ctx, SOC_ERR_ARG, "weighted_cap must be >= 1");
        if (weighted && prm->max_iter > 0) {
            CK(cl.dust_wp.alloc((size_t)nf * (2 * cl.n_leaf + 1)), "alloc weighted sampling");
            CK(cl.e_unit_w.alloc(nf), "alloc e_unit");
        }
        const int refmode = prm->reference_field;
        if (refmode < 0 || refmode > 2) return fail(ctx, SOC_ERR_ARG, "reference_field must be 0, 1 or 2");
        const bool reffield = refmode != 0;
        if (reffield) {
            if (prm->ali) return fail(ctx, SOC_ERR_ARG, "reference_field and ali together are not supported");
            if (prm->weighted_cap == 0) return fail(ctx, SOC_ERR_ARG, "weighted_cap must be >= 1");
            if (prm->n_dust_first == 0 && prm->n_weighted == 0)
                return fail(ctx, SOC_ERR_ARG, "reference_field needs n_dust_first/n_dust_last or n_weighted");
            if (prm->n_dust_first && prm->n_dust_last == 0)
                return fail(ctx, SOC_ERR_ARG, "n_dust_last must be >= 1");
        }
        if (reffield && prm->max_iter > 0) {
            CK(cl.A_ref.alloc(n), "alloc A_ref");
            CK(cl.A_d.alloc(n), "alloc A_d");
            CK(cl.dust_wp.alloc((size_t)nf * (2 * cl.n_leaf + 1)), "alloc weighted sampling");
            CK(cl.e_unit_w.alloc(nf), "alloc e_unit");
            CK(cudaMemsetAsync(cl.A_ref.p, 0, sizeof(double) * n, s), "zero A_ref");
            if (refmode == 2) {
                const size_t fl = (size_t)nf * cl.n_leaf;
                CK(cl.L.alloc(fl), "alloc L");
                CK(cl.L_ref.alloc(fl), "alloc L_ref");
                CK(cl.neg.alloc(fl), "alloc signs");
                CK(cl.dust_wn.alloc((size_t)nf * (2 * cl.n_leaf + 1)), "alloc weighted sampling");
                CK(cl.e_unit_n.alloc(nf), "alloc e_unit");
                CK(cudaMemsetAsync(cl.L_ref.p, 0, sizeof(double) * fl, s), "zero L_ref");
            }
        }
        const bool ali = prm->ali != 0;
        if (ali && prm->max_iter > 0) {
            CK(cl.self_tally.alloc((size_t)nf * n), "alloc self counters");
            CK(cl.A_self.alloc(n), "alloc A_self");
        }
        int64_t steps = 0, capped = 0;
        int it_done = 0, conv = 0;
        double dT = 0.0;
        Watchdog watchdog;
        if (ctx->timeout_s > 0.0) watchdog.start(ctx->h_abort, ctx->timeout_s);
        auto aborted = [&]() { return __atomic_load_n(const_cast<int *>(&ctx->h_abort[0]), __ATOMIC_SEQ_CST) != 0; };
        const soc_status run_st = [&]() -> soc_status {
        std::vector<int64_t> hstats(4 * nf);
        std::vector<soc_batch_item> items(nf);
        std::vector<double> e(nf);
        std::vector<uint64_t> wcount(nf, 0);
        auto run_items = [&](int source, uint64_t npk, int iteration, const uint64_t *dw, uint32_t npc,
                             int64_t *self, bool wsampled) -> soc_status {
            if (aborted()) return fail(ctx, SOC_ERR_TIMEOUT, "aborted (soc_abort or the soc_set_timeout deadline)");
            for (int f = 0; f < nf; ++f) {
                soc_batch_item &it = items[f];
                memset(&it, 0, sizeof it);
                it.cloud = cloud_id; it.freq = f; it.source = source; it.iteration = iteration;
                it.pid_offset = 0; it.n_packages = wsampled ? wcount[f] : npk; it.w0 = SOC_W_UNIT;
                it.tally_offset = (int64_t)f * n;
                it.d_dust_w = dw ? dw + (size_t)f * (wsampled ? 2 * cl.n_leaf + 1 : cl.n_leaf) : nullptr;
                it.n_per_cell = npc;
                it.reserved = wsampled ? SOC_ITEM_WEIGHTED : 0u;
            }
            CK(cudaMemsetAsync(cl.tally.p, 0, sizeof(int64_t) * nf * n, s), "zero tally");
            CK(cudaMemsetAsync(cl.stats.p, 0, sizeof(int64_t) * 4 * nf, s), "zero stats");
            if (self) CK(cudaMemsetAsync(self, 0, sizeof(int64_t) * nf * n, s), "zero self counters");
            soc_status r = soc_simulate_frequency_batch_ex(ctx, items.data(), nf, cl.tally.p, self, cl.stats.p, nullptr,
                                                           stream);
            if (r) return r;
            CK(cudaMemcpyAsync(hstats.data(), cl.stats.p, sizeof(int64_t) * 4 * nf, cudaMemcpyDeviceToHost, s), "stats");
            CK(cudaStreamSynchronize(s), "sync");
            for (int f = 0; f < nf; ++f) { capped += hstats[4 * f + 1]; steps += hstats[4 * f + 2]; }
            if (aborted()) return fail(ctx, SOC_ERR_TIMEOUT, "aborted (soc_abort or the soc_set_timeout deadline)");
            return SOC_OK;
        };
        // iteration 0: constant sources, kept as A_const
        if (prm->reuse_constant && !cl.has_const)
            return fail(ctx, SOC_ERR_STATE, "reuse_constant: no earlier iteration 0 on this cloud");
        if (!prm->reuse_constant) CK(cudaMemsetAsync(cl.A_const.p, 0, sizeof(double) * n, s), "zero A");
        const uint64_t nsrc[2] = {prm->reuse_constant ? 0 : prm->n_background, prm->reuse_constant ? 0 : prm->n_point};
        for (int k = 0; k < 2; ++k) {
            if (!nsrc[k]) continue;
            const int source = k == 0 ? SOC_SRC_BACKGROUND : SOC_SRC_POINT;
            if ((st = run_items(source, nsrc[k], 0, nullptr, 1, nullptr, false))) return st;
            if ((st = soc_package_energy(ctx, cloud_id, source, nsrc[k], e.data()))) return st;
            CK(cudaMemcpyAsync(cl.e_unit.p, e.data(), 8 * nf, cudaMemcpyHostToDevice, s), "copy e_unit");
            if ((st = soc_absorbed_power(ctx, cloud_id, cl.tally.p, n, cl.e_unit.p, cl.A_const.p, cl.A_const.p, stream)))
                return st;
        }
        cl.has_const = true;
        if (d_T_seed) {
            CK(cudaMemcpyAsync(d_T_out, d_T_seed, sizeof(float) * n, cudaMemcpyDeviceToDevice, s), "copy seed");
        } else {
            if ((st = soc_update_temperature(ctx, cloud_id, cl.A_const.p, d_T_out, nullptr, stream))) return st;
        }
        double n_cum = 0.0;
        for (int k = 1; k <= prm->max_iter; ++k) {
            if (reffield) {
                // packages of this iteration: log n linear from n_dust_first to n_dust_last
                uint64_t nk = prm->n_weighted;
                if (prm->n_dust_first) {
                    const double t = prm->max_iter > 1 ? (double)(k - 1) / (double)(prm->max_iter - 1) : 1.0;
                    const double ratio = (double)prm->n_dust_last / (double)prm->n_dust_first;
                    nk = (uint64_t)std::max(1.0, rint((double)prm->n_dust_first * pow(ratio, t)));
                    if (prm->max_iter == 1) nk = prm->n_dust_last;
                }
                n_cum += (double)nk;
                const double wk = (double)nk / n_cum;
                if (refmode == 1) {
                    // full dust emission, fresh random numbers; A_ref = running mean of the estimates
                    if ((st = soc_dust_emission(ctx, cloud_id, d_T_out, 0, nf, 1u, cl.dust_w.p, cl.e_unit.p, stream)))
                        return st;
                    if ((st = soc_dust_weighted(ctx, cloud_id, cl.dust_w.p, cl.e_unit.p, nf, nk, prm->weighted_cap,
                                                cl.dust_wp.p, cl.e_unit_w.p, stream)))
                        return st;
                    for (int f = 0; f < nf; ++f)
                        CK(cudaMemcpyAsync(&wcount[f], cl.dust_wp.p + (size_t)f * (2 * cl.n_leaf + 1) + 2 * cl.n_leaf,
                                           sizeof(uint64_t), cudaMemcpyDeviceToHost, s), "read package counts");
                    CK(cudaStreamSynchronize(s), "sync");
                    if ((st = run_items(SOC_SRC_DUST, 0, k, cl.dust_wp.p, 1, nullptr, true))) return st;
                    if ((st = soc_absorbed_power(ctx, cloud_id, cl.tally.p, n, cl.e_unit_w.p, nullptr, cl.A_d.p, stream)))
                        return st;
                    if ((st = soc_reference_update(ctx, cloud_id, cl.A_ref.p, cl.A_d.p, wk, cl.A_const.p, cl.A.p, 1,
                                                   stream)))
                        return st;
                    if ((st = soc_update_temperature(ctx, cloud_id, cl.A.p, d_T_out, ctx->d_maxdT.p, stream))) return st;
                    CK(cudaMemcpyAsync(&dT, ctx->d_maxdT.p, sizeof(double), cudaMemcpyDeviceToHost, s), "read max dT");
                    CK(cudaStreamSynchronize(s), "sync");
                    if (dT_history) dT_history[k - 1] = dT;
                    it_done = k;
                    if (dT < prm->dT_tol) { conv = 1; break; }
                    continue;
                }
                if ((st = soc_dust_luminosity(ctx, cloud_id, d_T_out, 0, nf, cl.L.p, stream))) return st;
                if ((st = soc_reference_delta(ctx, cloud_id, nf, cl.L.p, cl.L_ref.p, wk, cl.dust_w.p, cl.neg.p,
                                              cl.e_unit.p, stream)))
                    return st;
                if ((st = soc_dust_weighted(ctx, cloud_id, cl.dust_w.p, cl.e_unit.p, nf, nk, prm->weighted_cap,
                                            cl.dust_wp.p, cl.e_unit_w.p, stream)))
                    return st;
                if ((st = soc_dust_split(ctx, cloud_id, nf, cl.neg.p, cl.dust_wp.p, cl.dust_wn.p, cl.e_unit_w.p,
                                         cl.e_unit_n.p, stream)))
                    return st;
                for (int f = 0; f < nf; ++f)
                    CK(cudaMemcpyAsync(&wcount[f], cl.dust_wp.p + (size_t)f * (2 * cl.n_leaf + 1) + 2 * cl.n_leaf,
                                       sizeof(uint64_t), cudaMemcpyDeviceToHost, s), "read package counts");
                CK(cudaStreamSynchronize(s), "sync");
                // rising cells, then falling cells (same packages ids, weights of the other sign are 0)
                if ((st = run_items(SOC_SRC_DUST, 0, k, cl.dust_wp.p, 1, nullptr, true))) return st;
                if ((st = soc_absorbed_power(ctx, cloud_id, cl.tally.p, n, cl.e_unit_w.p, cl.A_ref.p, cl.A_d.p, stream)))
                    return st;
                if ((st = run_items(SOC_SRC_DUST, 0, k, cl.dust_wn.p, 1, nullptr, true))) return st;
                if ((st = soc_absorbed_power(ctx, cloud_id, cl.tally.p, n, cl.e_unit_n.p, cl.A_d.p, cl.A_d.p, stream)))
                    return st;
                if ((st = soc_reference_update(ctx, cloud_id, cl.A_ref.p, cl.A_d.p, wk, cl.A_const.p, cl.A.p, 0, stream)))
                    return st;
                if ((st = soc_update_temperature(ctx, cloud_id, cl.A.p, d_T_out, ctx->d_maxdT.p, stream))) return st;
                CK(cudaMemcpyAsync(&dT, ctx->d_maxdT.p, sizeof(double), cudaMemcpyDeviceToHost, s), "read max dT");
                CK(cudaStreamSynchronize(s), "sync");
                if (dT_history) dT_history[k - 1] = dT;
                it_done = k;
                if (dT < prm->dT_tol) { conv = 1; break; }
                continue;
            }
            if ((st = soc_dust_emission(ctx, cloud_id, d_T_out, 0, nf, weighted ? 1u : prm->n_per_cell, cl.dust_w.p,
                                        cl.e_unit.p, stream)))
                return st;
            const double *e_dust = cl.e_unit.p;
            if (weighted && k == 1) {
                // the allocation is made once, from the first dust temperatures,
                // and then frozen (only the weights follow T)
                if ((st = soc_dust_weighted(ctx, cloud_id, cl.dust_w.p, cl.e_unit.p, nf, prm->n_weighted,
                                            prm->weighted_cap, cl.dust_wp.p, cl.e_unit_w.p, stream)))
                    return st;
                for (int f = 0; f < nf; ++f)        // packages to trace = last prefix entry of each frequency
                    CK(cudaMemcpyAsync(&wcount[f], cl.dust_wp.p + (size_t)f * (2 * cl.n_leaf + 1) + 2 * cl.n_leaf,
                                       sizeof(uint64_t), cudaMemcpyDeviceToHost, s), "read package counts");
                CK(cudaStreamSynchronize(s), "sync");
            } else if (weighted) {
                if ((st = soc_dust_reweight(ctx, cloud_id, cl.dust_w.p, cl.e_unit.p, nf, cl.dust_wp.p, cl.e_unit_w.p,
                                            stream)))
                    return st;
            }
            if (weighted) e_dust = cl.e_unit_w.p;
            // frozen dust random numbers: the same RNG stream (iteration 1) every time
            if ((st = run_items(SOC_SRC_DUST, (uint64_t)cl.n_leaf * prm->n_per_cell, 1,
                                weighted ? cl.dust_wp.p : cl.dust_w.p, prm->n_per_cell, ali ? cl.self_tally.p : nullptr,
                                weighted)))
                return st;
            if ((st = soc_absorbed_power(ctx, cloud_id, cl.tally.p, n, e_dust, cl.A_const.p, cl.A.p, stream)))
                return st;
            if (ali) {
                if ((st = soc_absorbed_power(ctx, cloud_id, cl.self_tally.p, n, e_dust, nullptr, cl.A_self.p, stream)))
                    return st;
                if ((st = soc_update_temperature_ali(ctx, cloud_id, cl.A.p, cl.A_self.p, d_T_out, ctx->d_maxdT.p, stream)))
                    return st;
            } else if ((st = soc_update_temperature(ctx, cloud_id, cl.A.p, d_T_out, ctx->d_maxdT.p, stream))) {
                return st;
            }
            CK(cudaMemcpyAsync(&dT, ctx->d_maxdT.p, sizeof(double), cudaMemcpyDeviceToHost, s), "read max dT");
            CK(cudaStreamSynchronize(s), "sync");
            if (dT_history) dT_history[k - 1] = dT;
            it_done = k;
            if (dT < prm->dT_tol) { conv = 1; break; }
        }
        return SOC_OK;
        }();
        if (res) {
            res->iterations = it_done;
            res->converged = conv;
            res->final_max_dT = dT;
            res->steps = steps;
            res->capped = capped;
        }
        if (run_st != SOC_OK) return run_st;
        return capped ? fail(ctx, SOC_ERR_STEP_LIMIT, "%lld packages hit the step cap", (long long)capped) : SOC_OK;
    });
}

soc_status soc_iterate_batch(soc_ctx *ctx, int n_clouds, const int *cloud_ids, const soc_iterate_params *prm,
                             const float *const *d_T_seed, float *const *d_T_out, soc_iterate_result *res,
                             double *dT_history, void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || n_clouds < 1 || !cloud_ids || !prm || !d_T_out || prm->max_iter < 0)
            return fail(ctx, SOC_ERR_ARG, "bad iterate_batch arguments");
        if (prm->n_weighted || prm->reference_field)
            return fail(ctx, SOC_ERR_ARG, "iterate_batch: weighted sampling and the reference field are per-cloud "
                        "options (soc_iterate)");
        if (ctx->n_freq == 0) return fail(ctx, SOC_ERR_STATE, "soc_dust_upload must come first");
        if (prm->max_iter > 0 && prm->n_per_cell == 0) return fail(ctx, SOC_ERR_ARG, "n_per_cell must be >= 1");
        for (int k = 0; k < n_clouds; ++k) {
            soc_status st = check_cloud(ctx, cloud_ids[k]);
            if (st) return st;
            if (!d_T_out[k]) return fail(ctx, SOC_ERR_ARG, "d_T_out[%d] is NULL", k);
            for (int j = 0; j < k; ++j)
                if (cloud_ids[j] == cloud_ids[k]) return fail(ctx, SOC_ERR_ARG, "cloud %d listed twice", cloud_ids[k]);
            const CloudHost &cl = *ctx->clouds[cloud_ids[k]];
            if (prm->reuse_constant && !cl.has_const)
                return fail(ctx, SOC_ERR_STATE, "reuse_constant: no earlier iteration 0 on cloud %d", cloud_ids[k]);
            if (!prm->reuse_constant && prm->n_background && cl.bg_I.empty())
                return fail(ctx, SOC_ERR_STATE, "cloud %d: no background uploaded", cloud_ids[k]);
            if (!prm->reuse_constant && prm->n_point && cl.n_ps == 0)
                return fail(ctx, SOC_ERR_STATE, "cloud %d: no point sources uploaded", cloud_ids[k]);
        }
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        cudaStream_t s = (cudaStream_t)stream;
        const int nf = ctx->n_freq;
        const bool ali = prm->ali != 0;
        // per-cloud buffers (as soc_iterate) and the batch's shared scratch
        int64_t cells_all = 0;
        for (int k = 0; k < n_clouds; ++k) {
            CloudHost &cl = *ctx->clouds[cloud_ids[k]];
            CK(cl.A_const.alloc(cl.n_cells), "alloc A");
            CK(cl.A.alloc(cl.n_cells), "alloc A");
            CK(cl.e_unit.alloc(nf), "alloc e_unit");
            if (prm->max_iter > 0) CK(cl.dust_w.alloc((size_t)nf * cl.n_leaf), "alloc dust weights");
            if (ali && prm->max_iter > 0) CK(cl.A_self.alloc(cl.n_cells), "alloc A_self");
            cells_all += cl.n_cells;
        }
        const int n_src = (prm->reuse_constant ? 0 : (prm->n_background ? 1 : 0) + (prm->n_point ? 1 : 0));
        const int per_cloud_items = std::max(n_src, prm->max_iter > 0 ? 1 : 0) * nf;
        CK(ctx->b_tally.alloc((size_t)std::max(n_src, 1) * nf * cells_all), "alloc batch counters");
        if (ali && prm->max_iter > 0) CK(ctx->b_self.alloc((size_t)nf * cells_all), "alloc batch self counters");
        CK(ctx->b_stats.alloc((size_t)4 * std::max(per_cloud_items, 1) * n_clouds), "alloc batch stats");
        CK(ctx->b_maxdT.alloc(n_clouds), "alloc max dT");
        std::vector<int64_t> hstats(4 * (size_t)std::max(per_cloud_items, 1) * n_clouds);
        std::vector<double> hdT(n_clouds, 0.0);
        std::vector<int64_t> steps(n_clouds, 0), capped(n_clouds, 0);
        std::vector<int> it_done(n_clouds, 0), conv(n_clouds, 0);
        std::vector<soc_batch_item> items;
        std::vector<int> item_cloud;          // batch position of each item's cloud
        std::vector<int64_t> base(n_clouds);  // element offset of each cloud's slices in b_tally
        Watchdog watchdog;
        if (ctx->timeout_s > 0.0) watchdog.start(ctx->h_abort, ctx->timeout_s);
        auto aborted = [&]() { return __atomic_load_n(const_cast<int *>(&ctx->h_abort[0]), __ATOMIC_SEQ_CST) != 0; };
        // one tracer launch over `items`, then per-cloud statistics
        auto launch = [&](int64_t *self) -> soc_status {
            if (aborted()) return fail(ctx, SOC_ERR_TIMEOUT, "aborted (soc_abort or the soc_set_timeout deadline)");
            const int n_items = (int)items.size();
            CK(cudaMemsetAsync(ctx->b_stats.p, 0, sizeof(int64_t) * 4 * n_items, s), "zero stats");
            soc_status r = soc_simulate_frequency_batch_ex(ctx, items.data(), n_items, ctx->b_tally.p, self,
                                                           ctx->b_stats.p, nullptr, stream);
            if (r) return r;
            CK(cudaMemcpyAsync(hstats.data(), ctx->b_stats.p, sizeof(int64_t) * 4 * n_items, cudaMemcpyDeviceToHost, s),
               "stats");
            CK(cudaStreamSynchronize(s), "sync");
            for (int i = 0; i < n_items; ++i) {
                capped[item_cloud[i]] += hstats[4 * i + 1];
                steps[item_cloud[i]] += hstats[4 * i + 2];
            }
            if (aborted()) return fail(ctx, SOC_ERR_TIMEOUT, "aborted (soc_abort or the soc_set_timeout deadline)");
            return SOC_OK;
        };
        const soc_status run_st = [&]() -> soc_status {
            soc_status st;
            // iteration 0: background and point sources of every cloud in one launch
            if (!prm->reuse_constant) {
                items.clear(); item_cloud.clear();
                int64_t off = 0;
                for (int k = 0; k < n_clouds; ++k) {
                    const CloudHost &cl = *ctx->clouds[cloud_ids[k]];
                    base[k] = off;
                    for (int c = 0; c < 2; ++c) {
                        const uint64_t npk = c == 0 ? prm->n_background : prm->n_point;
                        if (!npk) continue;
                        for (int f = 0; f < nf; ++f) {
                            soc_batch_item it;
                            memset(&it, 0, sizeof it);
                            it.cloud = cloud_ids[k]; it.freq = f;
                            it.source = c == 0 ? SOC_SRC_BACKGROUND : SOC_SRC_POINT;
                            it.n_packages = npk; it.w0 = SOC_W_UNIT; it.tally_offset = off; it.n_per_cell = 1;
                            items.push_back(it);
                            item_cloud.push_back(k);
                            off += cl.n_cells;
                        }
                    }
                }
                if (!items.empty()) {
                    CK(cudaMemsetAsync(ctx->b_tally.p, 0, sizeof(int64_t) * off, s), "zero counters");
                    if ((st = launch(nullptr))) return st;
                }
                std::vector<double> e(nf);
                for (int k = 0; k < n_clouds; ++k) {
                    CloudHost &cl = *ctx->clouds[cloud_ids[k]];
                    CK(cudaMemsetAsync(cl.A_const.p, 0, sizeof(double) * cl.n_cells, s), "zero A");
                    int64_t o = base[k];
                    for (int c = 0; c < 2; ++c) {
                        const uint64_t npk = c == 0 ? prm->n_background : prm->n_point;
                        if (!npk) continue;
                        const int source = c == 0 ? SOC_SRC_BACKGROUND : SOC_SRC_POINT;
                        if ((st = soc_package_energy(ctx, cloud_ids[k], source, npk, e.data()))) return st;
                        CK(cudaMemcpyAsync(cl.e_unit.p, e.data(), 8 * nf, cudaMemcpyHostToDevice, s), "copy e_unit");
                        if ((st = soc_absorbed_power(ctx, cloud_ids[k], ctx->b_tally.p + o, cl.n_cells, cl.e_unit.p,
                                                     cl.A_const.p, cl.A_const.p, stream)))
                            return st;
                        o += (int64_t)nf * cl.n_cells;
                    }
                    cl.has_const = true;
                }
            }
            // start temperatures
            for (int k = 0; k < n_clouds; ++k) {
                CloudHost &cl = *ctx->clouds[cloud_ids[k]];
                const float *seed = d_T_seed ? d_T_seed[k] : nullptr;
                if (seed) {
                    CK(cudaMemcpyAsync(d_T_out[k], seed, sizeof(float) * cl.n_cells, cudaMemcpyDeviceToDevice, s),
                       "copy seed");
                } else if ((st = soc_update_temperature(ctx, cloud_ids[k], cl.A_const.p, d_T_out[k], nullptr, stream))) {
                    return st;
                }
            }
            // dust iterations: every unconverged cloud's re-emission in one launch
            for (int it_k = 1; it_k <= prm->max_iter; ++it_k) {
                items.clear(); item_cloud.clear();
                int64_t off = 0;
                std::vector<int> active;
                for (int k = 0; k < n_clouds; ++k) {
                    if (conv[k]) continue;
                    CloudHost &cl = *ctx->clouds[cloud_ids[k]];
                    if ((st = soc_dust_emission(ctx, cloud_ids[k], d_T_out[k], 0, nf, prm->n_per_cell, cl.dust_w.p,
                                                cl.e_unit.p, stream)))
                        return st;
                    base[k] = off;
                    for (int f = 0; f < nf; ++f) {
                        soc_batch_item it;
                        memset(&it, 0, sizeof it);
                        it.cloud = cloud_ids[k]; it.freq = f; it.source = SOC_SRC_DUST;
                        it.iteration = 1;      // frozen dust random numbers, as soc_iterate
                        it.n_packages = (uint64_t)cl.n_leaf * prm->n_per_cell; it.w0 = SOC_W_UNIT;
                        it.tally_offset = off; it.d_dust_w = cl.dust_w.p + (size_t)f * cl.n_leaf;
                        it.n_per_cell = prm->n_per_cell;
                        items.push_back(it);
                        item_cloud.push_back(k);
                        off += cl.n_cells;
                    }
                    active.push_back(k);
                }
                if (active.empty()) break;
                CK(cudaMemsetAsync(ctx->b_tally.p, 0, sizeof(int64_t) * off, s), "zero counters");
                if (ali) CK(cudaMemsetAsync(ctx->b_self.p, 0, sizeof(int64_t) * off, s), "zero self counters");
                if ((st = launch(ali ? ctx->b_self.p : nullptr))) return st;
                for (int k : active) {
                    CloudHost &cl = *ctx->clouds[cloud_ids[k]];
                    if ((st = soc_absorbed_power(ctx, cloud_ids[k], ctx->b_tally.p + base[k], cl.n_cells, cl.e_unit.p,
                                                 cl.A_const.p, cl.A.p, stream)))
                        return st;
                    if (ali) {
                        if ((st = soc_absorbed_power(ctx, cloud_ids[k], ctx->b_self.p + base[k], cl.n_cells,
                                                     cl.e_unit.p, nullptr, cl.A_self.p, stream)))
                            return st;
                        if ((st = soc_update_temperature_ali(ctx, cloud_ids[k], cl.A.p, cl.A_self.p, d_T_out[k],
                                                             ctx->b_maxdT.p + k, stream)))
                            return st;
                    } else if ((st = soc_update_temperature(ctx, cloud_ids[k], cl.A.p, d_T_out[k], ctx->b_maxdT.p + k,
                                                            stream))) {
                        return st;
                    }
                }
                CK(cudaMemcpyAsync(hdT.data(), ctx->b_maxdT.p, sizeof(double) * n_clouds, cudaMemcpyDeviceToHost, s),
                   "read max dT");
                CK(cudaStreamSynchronize(s), "sync");
                for (int k : active) {
                    if (dT_history) dT_history[(size_t)k * prm->max_iter + (it_k - 1)] = hdT[k];
                    it_done[k] = it_k;
                    if (hdT[k] < prm->dT_tol) conv[k] = 1;
                }
            }
            return SOC_OK;
        }();
        int64_t capped_all = 0;
        for (int k = 0; k < n_clouds; ++k) {
            capped_all += capped[k];
            if (res) {
                res[k].iterations = it_done[k];
                res[k].converged = conv[k];
                res[k].final_max_dT = it_done[k] ? hdT[k] : 0.0;
                res[k].steps = steps[k];
                res[k].capped = capped[k];
            }
        }
        if (run_st != SOC_OK) return run_st;
        return capped_all ? fail(ctx, SOC_ERR_STEP_LIMIT, "%lld packages hit the step cap", (long long)capped_all)
                          : SOC_OK;
    });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of soc_simulate_frequency_batch.
//
// Some callers cannot allocate device memory while they trace: code that runs
// under a framework's caching allocator or memory budget (where a cudaMalloc
// outside the pool breaks its accounting or fails at the limit), real-time
// loops where cudaMalloc/cudaFree would synchronise the device, and embedders
// that hand the library fixed buffers only.  This entry point keeps all of its
// per-call scratch -- the work counter, the item table and its prefix sums,
// and the grid table -- in one file-scope device array of fixed size, so it
// never calls cudaMalloc, cudaFree or any allocating library routine.  The
// caller still passes the counters and statistics buffers.  The item checks
// and the device forms of items and grids are the ones the ordinary entry
// uses (check_item, fill_dev_cloud), written into static host arrays.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxItems = SOC_NOALLOC_MAX_ITEMS;
constexpr int kNoAllocMaxClouds = SOC_NOALLOC_MAX_CLOUDS;

struct NoAllocLayout {
    unsigned long long counter;
    unsigned long long pad[31];              // keeps the tables 256-byte aligned
    uint64_t prefix[kNoAllocMaxItems + 1];
    DevItem items[kNoAllocMaxItems];
    DevCloud clouds[kNoAllocMaxClouds];
};

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocLayout)];

constexpr int kMaxDevices = 64;
// Device address of g_noalloc_scratch, per device.  Host threads making their
// first call on one device at the same time may both look it up; they store
// the same address, and the atomics make that race well defined.
std::atomic<void *> g_noalloc_addr[kMaxDevices];

// Host staging for the tables (static storage: no heap use either).
thread_local uint64_t t_prefix[kNoAllocMaxItems + 1];
thread_local DevItem t_items[kNoAllocMaxItems];
thread_local DevCloud t_clouds[kNoAllocMaxClouds];

}  // namespace

extern "C" soc_status soc_simulate_frequency_batch_noalloc(soc_ctx *ctx, const soc_batch_item *items, int n_items,
                                                           int64_t *d_tally, int64_t *d_stats, uint32_t *d_pkg_steps,
                                                           void *stream)
{
    return guarded(ctx, [&]() -> soc_status {
        if (!ctx || !items || n_items < 1 || !d_tally || !d_stats) return fail(ctx, SOC_ERR_ARG, "null argument");
        if (n_items > kNoAllocMaxItems)
            return fail(ctx, SOC_ERR_ARG, "n_items %d exceeds the allocation-free limit of %d items", n_items,
                        kNoAllocMaxItems);
        if ((int)ctx->clouds.size() > kNoAllocMaxClouds)
            return fail(ctx, SOC_ERR_ARG, "%d grids uploaded (freed ones included) exceed the allocation-free "
                        "limit of %d grids", (int)ctx->clouds.size(), kNoAllocMaxClouds);
        if (ctx->n_freq == 0) return fail(ctx, SOC_ERR_STATE, "soc_dust_upload must come first");
        if (ctx->device < 0 || ctx->device >= kMaxDevices) return fail(ctx, SOC_ERR_ARG, "device index too large");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        cudaStream_t s = (cudaStream_t)stream;
        if (soc_status cst = refuse_capture(ctx, s, "soc_simulate_frequency_batch_noalloc")) return cst;
        // set-up, once per device, with that device current: the host-side name
        // g_noalloc_scratch is only a stand-in, the kernel needs the device address
        void *addr = g_noalloc_addr[ctx->device].load(std::memory_order_acquire);
        if (!addr) {
            CK(cudaGetSymbolAddress(&addr, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
            g_noalloc_addr[ctx->device].store(addr, std::memory_order_release);
        }
        NoAllocLayout *S = static_cast<NoAllocLayout *>(addr);
        if (soc_status pst = prepare_items_into(ctx, items, n_items, t_items, t_prefix)) return pst;
        const uint64_t total = t_prefix[n_items];
        if (total == 0) return SOC_OK;
        const int nc = (int)ctx->clouds.size();
        for (int i = 0; i < nc; ++i) fill_dev_cloud(*ctx->clouds[i], t_clouds[i]);
        CK(cudaMemcpyAsync(S->clouds, t_clouds, sizeof(DevCloud) * nc, cudaMemcpyHostToDevice, s), "copy grid table");
        CK(cudaMemcpyAsync(S->items, t_items, sizeof(DevItem) * n_items, cudaMemcpyHostToDevice, s), "copy items");
        CK(cudaMemcpyAsync(S->prefix, t_prefix, sizeof(uint64_t) * (n_items + 1), cudaMemcpyHostToDevice, s),
           "copy prefix");
        CK(cudaMemsetAsync(&S->counter, 0, sizeof(unsigned long long), s), "zero counter");   // must start at 0
        TraceParams P;
        P.clouds = S->clouds;
        P.items = S->items;
        P.prefix = S->prefix;
        P.g_hg = ctx->d_g.p;
        P.tally = reinterpret_cast<unsigned long long *>(d_tally);
        P.self = nullptr;
        P.stats = reinterpret_cast<unsigned long long *>(d_stats);
        P.pkg_steps = d_pkg_steps;
        P.counter = &S->counter;
        P.abort_flag = ctx->d_abort;
        P.cut = ctx->d_abort + 1;
        P.total = total;
        P.seed = ctx->seed;
        P.n_items = n_items;
        P.max_steps = ctx->max_steps;
        P.chunk = ctx->chunk;
        P.refill_min = ctx->refill_min;
        P.scatter_min = ctx->scatter_min;
        P.hot = one_cloud(ctx, items, n_items);
        P.regular = all_regular(ctx, items, n_items);
        int grid = 1, variant = 3;
        launch_geometry(ctx, total, P.regular != 0, grid, variant);     // occupancy cached at soc_create
        CK(launch_trace(P, grid, ctx->tpb, variant, s), "trace launch");
        return SOC_OK;
    });
}
