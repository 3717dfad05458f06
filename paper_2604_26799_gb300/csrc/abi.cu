// C-ABI entry points of include/mgs.h: context, scenes, cost tables, codes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace mgs {

static thread_local char g_err[1024];
static std::atomic<int64_t> g_launches{0};
static std::atomic<int64_t> g_allocs{0};          // dev_malloc_async calls so far
static std::atomic<int64_t> g_fail_alloc_in{0};   // > 0: that many calls from now, the last one fails

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    int64_t c = g_fail_alloc_in.load();
    while (c > 0) {
        if (g_fail_alloc_in.compare_exchange_weak(c, c - 1)) {
            if (c == 1) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;   // injected: nothing is allocated
            }
            break;
        }
    }
    return cudaMallocAsync(p, bytes, st);
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int64_t n_groups_of(int64_t keep, int32_t G) { return (keep + G - 1) / G; }

mgs_status check_grid(const mgs_grid *grid, int64_t n) {
    if (!grid || !grid->keep || !grid->bits) {
        set_error("grid, grid->keep and grid->bits must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (grid->n_ratios < 1 || grid->n_ratios > MGS_MAX_RATIOS) {
        set_error("n_ratios %d outside 1..%d", grid->n_ratios, MGS_MAX_RATIOS);
        return MGS_ERR_INVALID_ARG;
    }
    if (grid->n_bits < 1 || grid->n_bits > MGS_MAX_OPTIONS) {
        set_error("n_bits %d outside 1..%d", grid->n_bits, MGS_MAX_OPTIONS);
        return MGS_ERR_INVALID_ARG;
    }
    if (grid->group_size < 1 || grid->group_size > MGS_MAX_GROUP) {
        set_error("group_size %d outside 1..%d", grid->group_size, MGS_MAX_GROUP);
        return MGS_ERR_INVALID_ARG;
    }
    for (int r = 0; r < grid->n_ratios; r++) {
        int64_t k = grid->keep[r];
        if (k < 1 || k > n || (r > 0 && k <= grid->keep[r - 1])) {
            set_error("keep[%d] = %lld: kept-set sizes must increase strictly within 1..%lld", r,
                      (long long)k, (long long)n);
            return MGS_ERR_INVALID_ARG;
        }
    }
    for (int k = 0; k < grid->n_bits; k++) {
        int b = grid->bits[k];
        if (b < 1 || b > MGS_MAX_BITS || (k > 0 && b <= grid->bits[k - 1])) {
            set_error("bits[%d] = %d: bit-widths must increase strictly within 1..%d", k, b,
                      MGS_MAX_BITS);
            return MGS_ERR_INVALID_ARG;
        }
    }
    return MGS_OK;
}

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Table sub-array pointers for a buffer laid out by `L`.
void table_ptrs(void *base, const mgs_table_layout &L, CostSeg *s) {
    char *b = static_cast<char *>(base);
    s->sse = reinterpret_cast<double *>(b + L.off_sse);
    s->l1 = reinterpret_cast<double *>(b + L.off_l1);
    s->hbits = reinterpret_cast<double *>(b + L.off_hbits);
    s->linf = reinterpret_cast<float *>(b + L.off_linf);
    s->cnt = reinterpret_cast<int32_t *>(b + L.off_count);
    s->vmin = reinterpret_cast<float *>(b + L.off_vmin);
    s->vmax = reinterpret_cast<float *>(b + L.off_vmax);
}

int pick_config(mgs_ctx *ctx, int G, int n_bits) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto &t : ctx->tiles)
        if (t.group_size == G && t.n_bits == n_bits) return t.config;
    return cost_default_config(G);
}

// Segments of one scene for all ratios of the grid.
mgs_status scene_segments(mgs_scene *sc, const mgs_grid *grid, void *table, cudaStream_t st,
                          std::vector<CostSeg> *segs) {
    mgs_table_layout L;
    MGS_TRY(mgs_table_layout_for(sc->n, sc->C, grid, &L));
    const int32_t *pos = nullptr;
    std::vector<int64_t> off;
    {
        std::lock_guard<std::mutex> lk(sc->mu);
        MGS_TRY(scene_kept(sc, grid->keep, grid->n_ratios, st, &pos, &off));
    }
    for (int r = 0; r < grid->n_ratios; r++) {
        CostSeg s{};
        s.slabs = sc->d_slabs;
        s.kept = pos + off[r];
        s.n = sc->n;
        s.K = grid->keep[r];
        s.item_base = L.item_begin[r];
        s.n_groups = (int32_t)L.n_groups[r];
        s.C = sc->C;
        table_ptrs(table, L, &s);
        segs->push_back(s);
    }
    return MGS_OK;
}

mgs_status run_cost(mgs_ctx *ctx, CostLaunch &launch, cudaStream_t st) {
    int cfg = pick_config(ctx, launch.group_size, launch.n_bits);
    CostSeg *d_segs = nullptr;
    unsigned int *d_counter = nullptr;
    size_t seg_bytes = align256(sizeof(CostSeg) * std::max<size_t>(launch.segs.size(), 1) * kMaxSpatialBuckets);
    void *scratch = nullptr;
    MGS_CUDA_TRY(dev_malloc_async(&scratch, seg_bytes + 256, st));
    d_segs = static_cast<CostSeg *>(scratch);
    d_counter = reinterpret_cast<unsigned int *>(static_cast<char *>(scratch) + seg_bytes);
    mgs_status s = cost_launch(ctx, launch, cfg, d_segs, d_counter, st);
    cudaFreeAsync(scratch, st);
    return s;
}

// [m][C] row-major coefficients into [n_slabs][m][8] slabs (padded channels 0).
__global__ void k_coeff_slabs(const float *__restrict__ in, int64_t m, int C, int n_slabs,
                              float *__restrict__ slabs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * n_slabs * kSlabWidth) return;
    const int j = (int)(t % kSlabWidth);
    const int64_t row = (t / kSlabWidth) % m;
    const int slab = (int)(t / ((int64_t)kSlabWidth * m));
    const int c = slab * kSlabWidth + j;
    slabs[t] = c < C ? in[row * C + c] : 0.0f;
}

// Finiteness and per-channel range of a [m][C] coefficient array: block (b, c)
// reduces rows [b * 4096, (b + 1) * 4096) of channel c, one atomic per block.
__device__ __forceinline__ unsigned int ord_u32(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
constexpr int kCheckRows = 4096;
__global__ void k_coeff_check(const float *__restrict__ in, int64_t m, int C, unsigned int *__restrict__ flag,
                              unsigned int *__restrict__ mn, unsigned int *__restrict__ mx) {
    __shared__ unsigned int s_mn[8], s_mx[8], s_bad;
    const int c = blockIdx.y;
    const int64_t r0 = (int64_t)blockIdx.x * kCheckRows;
    const int64_t r1 = r0 + kCheckRows < m ? r0 + kCheckRows : m;
    unsigned int lo = 0xFFFFFFFFu, hi = 0u, bad = 0u;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const float v = in[r * C + c];
        if (!isfinite(v)) {
            bad = 1u;
        } else {
            lo = min(lo, ord_u32(v));
            hi = max(hi, ord_u32(v));
        }
    }
    lo = __reduce_min_sync(0xFFFFFFFFu, lo);
    hi = __reduce_max_sync(0xFFFFFFFFu, hi);
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    if (threadIdx.x == 0) s_bad = 0u;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        s_mn[threadIdx.x >> 5] = lo;
        s_mx[threadIdx.x >> 5] = hi;
        if (bad) atomicOr(&s_bad, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) {
            lo = min(lo, s_mn[k]);
            hi = max(hi, s_mx[k]);
        }
        lo = min(lo, s_mn[0]);
        hi = max(hi, s_mx[0]);
        if (s_bad) atomicOr(flag, 1u);
        atomicMin(&mn[c], lo);
        atomicMax(&mx[c], hi);
    }
}

float from_ord_u32(unsigned int o) {
    const unsigned int u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Host-or-device table: run `fn` on a device table and copy back when needed.
template <typename F>
mgs_status with_device_table(void *table, size_t bytes, cudaStream_t st, F fn) {
    if (is_device_pointer(table)) return fn(table);
    void *d = nullptr;
    MGS_CUDA_TRY(dev_malloc_async(&d, bytes, st));
    mgs_status s = fn(d);
    if (s == MGS_OK) {
        cudaError_t e = cudaMemcpyAsync(table, d, bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("table copy-back failed: %s", cudaGetErrorString(e));
            s = MGS_ERR_CUDA;
        }
    }
    cudaFreeAsync(d, st);
    return s;
}

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" {

const char *mgs_last_error(void) { return g_err; }
const char *mgs_version(void) { return "mgs 0.1 (sm_103a)"; }
int64_t mgs_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

mgs_status mgs_debug_fail_allocation(int64_t nth) {
    clear_error();
    if (nth < 0) {
        set_error("nth = %lld must be >= 0", (long long)nth);
        return MGS_ERR_INVALID_ARG;
    }
    g_fail_alloc_in.store(nth);
    return MGS_OK;
}

int64_t mgs_debug_allocations(void) { return g_allocs.load(std::memory_order_relaxed); }

mgs_status mgs_create(int32_t device, mgs_ctx **out) {
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return MGS_ERR_INVALID_ARG;
    }
    int count = 0;
    MGS_CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) {
        set_error("device %d outside 0..%d", device, count - 1);
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard g(device);
    mgs_ctx *ctx = new (std::nothrow) mgs_ctx();
    if (!ctx) return MGS_ERR_OUT_OF_MEMORY;
    ctx->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete ctx;
        set_error("cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
        return MGS_ERR_CUDA;
    }
    // stream-ordered allocations (scenes, kept lists, staging, solver workspace) are
    // recycled from the device's default pool instead of being returned to the
    // driver at every synchronisation
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    // L(h) = h log2 h in units of 2^-22 bits, h = 0..MGS_MAX_GROUP (L(0) = L(1) = 0), and
    // its increments L(h) - L(h - 1) (< 2^26), which telescope exactly back to L.
    std::vector<unsigned long long> lt(MGS_MAX_GROUP + 1, 0ull);
    std::vector<uint32_t> dt(MGS_MAX_GROUP + 1, 0u);
    for (int h = 2; h <= MGS_MAX_GROUP; h++)
        lt[h] = (unsigned long long)std::llround((double)h * std::log2((double)h) * 4194304.0);
    for (int h = 1; h <= MGS_MAX_GROUP; h++) dt[h] = (uint32_t)(lt[h] - lt[h - 1]);
    const size_t lb = sizeof(unsigned long long) * lt.size(), db = sizeof(uint32_t) * dt.size();
    e = cudaMalloc(&ctx->d_ltab, lb + db);
    if (e == cudaSuccess) {
        ctx->d_dtab = reinterpret_cast<uint32_t *>(ctx->d_ltab + lt.size());
        e = cudaMemcpy(ctx->d_ltab, lt.data(), lb, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_dtab, dt.data(), db, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(ctx->d_ltab);
        delete ctx;
        set_error("entropy table upload: %s", cudaGetErrorString(e));
        return MGS_ERR_CUDA;
    }
    *out = ctx;
    return MGS_OK;
}

mgs_status mgs_destroy(mgs_ctx *ctx) {
    clear_error();
    if (!ctx) return MGS_OK;
    if (ctx->n_scenes != 0) {
        set_error("%d scenes still alive", ctx->n_scenes);
        return MGS_ERR_BUSY;
    }
    DeviceGuard g(ctx->device);
    cudaFree(ctx->d_ltab);
    delete ctx;
    return MGS_OK;
}

mgs_status mgs_scene_create(mgs_ctx *ctx, const float *attrs, const float *importance, int64_t n,
                            int32_t n_channels, void *stream, mgs_scene **out) {
    clear_error();
    if (!ctx || !attrs || !importance || !out) {
        set_error("ctx, attrs, importance and out must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (n < 1 || n >= ((int64_t)1 << 31) || n_channels < 3 || n_channels > MGS_MAX_CHANNELS) {
        set_error("n = %lld must be in 1..2^31-1 and n_channels = %d in 3..%d", (long long)n,
                  n_channels, MGS_MAX_CHANNELS);
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *d_attrs = attrs, *d_imp = importance;
    float *stage = nullptr;
    size_t abytes = sizeof(float) * (size_t)n * n_channels, ibytes = sizeof(float) * (size_t)n;
    bool host_a = !is_device_pointer(attrs), host_i = !is_device_pointer(importance);
    if (host_a || host_i) {
        size_t bytes = align256(host_a ? abytes : 0) + (host_i ? ibytes : 0);
        if (dev_malloc_async((void **)&stage, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            set_error("staging allocation of %zu bytes failed", bytes);
            return MGS_ERR_OUT_OF_MEMORY;
        }
        char *p = reinterpret_cast<char *>(stage);
        if (host_a) {
            MGS_CUDA_TRY(cudaMemcpyAsync(p, attrs, abytes, cudaMemcpyHostToDevice, st));
            d_attrs = reinterpret_cast<const float *>(p);
            p += align256(abytes);
        }
        if (host_i) {
            MGS_CUDA_TRY(cudaMemcpyAsync(p, importance, ibytes, cudaMemcpyHostToDevice, st));
            d_imp = reinterpret_cast<const float *>(p);
        }
    }
    mgs_scene *sc = new (std::nothrow) mgs_scene();
    if (!sc) return MGS_ERR_OUT_OF_MEMORY;
    mgs_status s = scene_build(ctx, d_attrs, d_imp, n, n_channels, st, sc);
    if (stage) cudaFreeAsync(stage, st);
    if (s != MGS_OK) {
        for (void *p : {(void *)sc->d_slabs, (void *)sc->d_rank_m, (void *)sc->d_order, (void *)sc->d_codes})
            if (p) cudaFreeAsync(p, st);
        cudaStreamSynchronize(st);
        cudaGetLastError();
        delete sc;
        return s;
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->n_scenes++;
    }
    *out = sc;
    return MGS_OK;
}

mgs_status mgs_scene_destroy(mgs_scene *sc) {
    clear_error();
    if (!sc) return MGS_OK;
    DeviceGuard g(sc->ctx->device);
    MGS_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(sc->d_slabs);
    cudaFree(sc->d_rank_m);
    cudaFree(sc->d_order);
    cudaFree(sc->d_codes);
    if (sc->kept.pos) cudaFree(sc->kept.pos);
    {
        std::lock_guard<std::mutex> lk(sc->ctx->mu);
        sc->ctx->n_scenes--;
    }
    delete sc;
    return MGS_OK;
}

mgs_status mgs_scene_info(const mgs_scene *sc, int64_t *n, int32_t *n_channels, int64_t *bytes) {
    clear_error();
    if (!sc) {
        set_error("scene is NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (n) *n = sc->n;
    if (n_channels) *n_channels = sc->C;
    if (bytes) *bytes = sc->device_bytes + (int64_t)sc->kept.bytes;
    return MGS_OK;
}

mgs_status mgs_scene_morton(const mgs_scene *sc, uint64_t *codes, int32_t *order, void *stream) {
    clear_error();
    if (!sc) {
        set_error("scene is NULL");
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard g(sc->ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (codes)
        MGS_CUDA_TRY(cudaMemcpyAsync(codes, sc->d_codes, sizeof(uint64_t) * sc->n,
                                     cudaMemcpyDefault, st));
    if (order)
        MGS_CUDA_TRY(cudaMemcpyAsync(order, sc->d_order, sizeof(int32_t) * sc->n, cudaMemcpyDefault,
                                     st));
    return MGS_OK;
}

mgs_status mgs_table_layout_for(int64_t n, int32_t n_channels, const mgs_grid *grid,
                                mgs_table_layout *out) {
    if (!out) {
        set_error("out is NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (n_channels < 1 || n_channels > MGS_MAX_CHANNELS) {
        set_error("n_channels %d outside 1..%d", n_channels, MGS_MAX_CHANNELS);
        return MGS_ERR_INVALID_ARG;
    }
    MGS_TRY(check_grid(grid, n));
    mgs_table_layout L;
    std::memset(&L, 0, sizeof(L));
    L.n_bits = grid->n_bits;
    L.n_ratios = grid->n_ratios;
    L.n_channels = n_channels;
    L.group_size = grid->group_size;
    int64_t items = 0;
    for (int r = 0; r < grid->n_ratios; r++) {
        L.item_begin[r] = items;
        L.n_groups[r] = n_groups_of(grid->keep[r], grid->group_size);
        items += (int64_t)n_channels * L.n_groups[r];
    }
    L.item_begin[grid->n_ratios] = items;
    L.n_items = items;
    size_t e = (size_t)items * grid->n_bits;
    size_t off = 0;
    L.off_sse = (int64_t)off;
    off = align256(off + 8 * e);
    L.off_l1 = (int64_t)off;
    off = align256(off + 8 * e);
    L.off_hbits = (int64_t)off;
    off = align256(off + 8 * e);
    L.off_linf = (int64_t)off;
    off = align256(off + 4 * e);
    L.off_count = (int64_t)off;
    off = align256(off + 4 * (size_t)items);
    L.off_vmin = (int64_t)off;
    off = align256(off + 4 * (size_t)items);
    L.off_vmax = (int64_t)off;
    off = align256(off + 4 * (size_t)items);
    L.total_bytes = (int64_t)off;
    *out = L;
    return MGS_OK;
}

static mgs_status build_table(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid,
                              void *table, void *stream, bool plain) {
    clear_error();
    if (!ctx || !scene || !table) {
        set_error("ctx, scene and table must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    mgs_scene *sc = const_cast<mgs_scene *>(scene);
    mgs_table_layout L;
    MGS_TRY(mgs_table_layout_for(sc->n, sc->C, grid, &L));
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return with_device_table(table, (size_t)L.total_bytes, st, [&](void *dt) -> mgs_status {
        std::vector<CostSeg> segs;
        MGS_TRY(scene_segments(sc, grid, dt, st, &segs));
        CostLaunch launch;
        launch.group_size = grid->group_size;
        launch.n_bits = grid->n_bits;
        for (int k = 0; k < grid->n_bits; k++) launch.bits[k] = grid->bits[k];
        if (!plain) {
            launch.segs = segs;
            launch.opt_lo = 0;
            launch.opt_hi = grid->n_bits;
            return run_cost(ctx, launch, st);
        }
        // plain per-configuration loop: one launch per (ratio, bit-width)
        for (size_t r = 0; r < segs.size(); r++) {
            for (int k = 0; k < grid->n_bits; k++) {
                launch.segs.assign(1, segs[r]);
                launch.opt_lo = k;
                launch.opt_hi = k + 1;
                MGS_TRY(run_cost(ctx, launch, st));
            }
        }
        return MGS_OK;
    });
}

mgs_status mgs_build_cost_table(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid,
                                void *table, void *stream) {
    return build_table(ctx, scene, grid, table, stream, false);
}

mgs_status mgs_build_cost_table_plain(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid,
                                      void *table, void *stream) {
    return build_table(ctx, scene, grid, table, stream, true);
}

mgs_status mgs_build_cost_table_probe(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid,
                                      void *table, uint32_t *hist, int64_t hist_capacity,
                                      uint16_t *codes, int64_t codes_capacity, void *stream) {
    clear_error();
    if (!ctx || !scene || !table) {
        set_error("ctx, scene and table must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    mgs_scene *sc = const_cast<mgs_scene *>(scene);
    mgs_table_layout L;
    MGS_TRY(mgs_table_layout_for(sc->n, sc->C, grid, &L));
    int64_t bins = 0, ncodes = 0;
    for (int k = 0; k < grid->n_bits; k++) bins += (int64_t)1 << grid->bits[k];
    for (int r = 0; r < grid->n_ratios; r++) ncodes += (int64_t)sc->C * grid->n_bits * grid->keep[r];
    if (hist && (hist_capacity < L.n_items * bins || !is_device_pointer(hist))) {
        set_error("hist must be device memory of at least %lld entries",
                  (long long)(L.n_items * bins));
        return MGS_ERR_INVALID_ARG;
    }
    if (codes && (codes_capacity < ncodes || !is_device_pointer(codes))) {
        set_error("codes must be device memory of at least %lld entries", (long long)ncodes);
        return MGS_ERR_INVALID_ARG;
    }
    const int cfg = cost_default_config(grid->group_size);
    if (!cost_config_has_probe(cfg)) {
        set_error("no probe kernel for group size %d", grid->group_size);
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return with_device_table(table, (size_t)L.total_bytes, st, [&](void *dt) -> mgs_status {
        std::vector<CostSeg> segs;
        MGS_TRY(scene_segments(sc, grid, dt, st, &segs));
        int64_t off = 0;
        for (int r = 0; r < grid->n_ratios; r++) {
            segs[r].code_off = off;
            off += (int64_t)sc->C * grid->n_bits * grid->keep[r];
        }
        CostLaunch launch;
        launch.group_size = grid->group_size;
        launch.n_bits = grid->n_bits;
        for (int k = 0; k < grid->n_bits; k++) launch.bits[k] = grid->bits[k];
        launch.segs = segs;
        launch.opt_lo = 0;
        launch.opt_hi = grid->n_bits;
        launch.probe_hist = hist;
        launch.probe_codes = codes;
        CostSeg *d_segs = nullptr;
        size_t seg_bytes = align256(sizeof(CostSeg) * std::max<size_t>(launch.segs.size(), 1) * kMaxSpatialBuckets);
        void *scratch = nullptr;
        MGS_CUDA_TRY(dev_malloc_async(&scratch, seg_bytes + 256, st));
        d_segs = static_cast<CostSeg *>(scratch);
        unsigned int *d_counter = reinterpret_cast<unsigned int *>(static_cast<char *>(scratch) + seg_bytes);
        mgs_status s = cost_launch(ctx, launch, cfg, d_segs, d_counter, st);
        cudaFreeAsync(scratch, st);
        return s;
    });
}

mgs_status mgs_build_cost_table_coeffs(mgs_ctx *ctx, const float *coeffs, int64_t m, int32_t n_channels,
                                       const mgs_grid *grid, void *table, void *stream) {
    clear_error();
    if (!ctx || !coeffs || !grid || !table) {
        set_error("ctx, coeffs, grid and table must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    mgs_table_layout L;
    MGS_TRY(mgs_table_layout_for(m, n_channels, grid, &L));
    if (m > ((int64_t)1 << 31) - 1) {
        set_error("%lld coefficients exceed 2^31 - 1", (long long)m);
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // validation: finite values and a finite FP32 range per channel (as for scenes)
    {
        unsigned int *chk = nullptr;
        MGS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&chk), sizeof(unsigned int) * (1 + 2 * (size_t)n_channels),
                                     st));
        std::vector<unsigned int> h(1 + 2 * (size_t)n_channels, 0u);
        for (int c = 0; c < n_channels; c++) h[1 + c] = 0xFFFFFFFFu;
        cudaError_t e = cudaMemcpyAsync(chk, h.data(), sizeof(unsigned int) * h.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            const dim3 grid((unsigned int)((m + kCheckRows - 1) / kCheckRows), (unsigned int)n_channels);
            k_coeff_check<<<grid, 256, 0, st>>>(coeffs, m, n_channels, chk, chk + 1, chk + 1 + n_channels);
            count_launches(1);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), chk, sizeof(unsigned int) * h.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFreeAsync(chk, st);
        if (e != cudaSuccess) {
            set_error("coefficient check failed: %s", cudaGetErrorString(e));
            return MGS_ERR_CUDA;
        }
        if (h[0]) {
            set_error("a coefficient is NaN or infinite");
            return MGS_ERR_NONFINITE;
        }
        for (int c = 0; c < n_channels; c++) {
            const float r = from_ord_u32(h[1 + n_channels + c]) - from_ord_u32(h[1 + c]);
            if (!std::isfinite(r)) {
                set_error("channel %d: max - min overflows FP32", c);
                return MGS_ERR_RANGE;
            }
        }
    }
    const int n_slabs = (n_channels + kSlabWidth - 1) / kSlabWidth;
    float *slabs = nullptr;
    MGS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&slabs), sizeof(float) * (size_t)m * n_slabs * kSlabWidth,
                                 st));
    const int64_t work = m * n_slabs * kSlabWidth;
    k_coeff_slabs<<<(unsigned int)((work + 255) / 256), 256, 0, st>>>(coeffs, m, n_channels, n_slabs, slabs);
    count_launches(1);
    mgs_status s = with_device_table(table, (size_t)L.total_bytes, st, [&](void *dt) -> mgs_status {
        CostLaunch launch;
        for (int r = 0; r < grid->n_ratios; r++) {
            CostSeg c{};
            c.slabs = slabs;
            c.kept = nullptr;   // the first K coefficients, in order
            c.n = m;
            c.K = grid->keep[r];
            c.item_base = L.item_begin[r];
            c.n_groups = (int32_t)L.n_groups[r];
            c.C = n_channels;
            table_ptrs(dt, L, &c);
            launch.segs.push_back(c);
        }
        launch.group_size = grid->group_size;
        launch.n_bits = grid->n_bits;
        for (int k = 0; k < grid->n_bits; k++) launch.bits[k] = grid->bits[k];
        launch.opt_lo = 0;
        launch.opt_hi = grid->n_bits;
        return run_cost(ctx, launch, st);
    });
    cudaFreeAsync(slabs, st);
    return s;
}

static mgs_status same_shape(int32_t n, const mgs_grid *grids) {
    for (int s = 1; s < n; s++) {
        if (grids[s].group_size != grids[0].group_size || grids[s].n_bits != grids[0].n_bits ||
            !grids[s].bits || !grids[0].bits ||
            std::memcmp(grids[s].bits, grids[0].bits, sizeof(int32_t) * grids[0].n_bits) != 0) {
            set_error("grid %d differs from grid 0 in group size or bit-widths", s);
            return MGS_ERR_INVALID_ARG;
        }
    }
    return MGS_OK;
}

mgs_status mgs_build_cost_tables_batched(mgs_ctx *ctx, int32_t n_scenes,
                                         const mgs_scene *const *scenes, const mgs_grid *grids,
                                         void *const *tables, void *stream) {
    clear_error();
    if (!ctx || n_scenes < 1 || !scenes || !tables || !grids) {
        set_error("ctx, scenes, grids and tables must be non-NULL and n_scenes >= 1");
        return MGS_ERR_INVALID_ARG;
    }
    MGS_TRY(same_shape(n_scenes, grids));
    int64_t n_segs = 0;
    for (int s = 0; s < n_scenes; s++) n_segs += grids[s].n_ratios;
    if (n_segs > kMaxSegments) {
        set_error("%lld (scene, ratio) segments exceed %d", (long long)n_segs, kMaxSegments);
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CostLaunch launch;
    launch.group_size = grids[0].group_size;
    launch.n_bits = grids[0].n_bits;
    for (int k = 0; k < grids[0].n_bits; k++) launch.bits[k] = grids[0].bits[k];
    launch.opt_lo = 0;
    launch.opt_hi = grids[0].n_bits;
    launch.persistent = true;
    for (int s = 0; s < n_scenes; s++) {
        if (!scenes[s] || !tables[s] || !is_device_pointer(tables[s])) {
            set_error("scene %d or its table is NULL or not device memory", s);
            return MGS_ERR_INVALID_ARG;
        }
        MGS_TRY(scene_segments(const_cast<mgs_scene *>(scenes[s]), &grids[s], tables[s], st,
                               &launch.segs));
    }
    return run_cost(ctx, launch, st);
}

int32_t mgs_tile_config_count(void) { return cost_config_count(); }

int32_t mgs_debug_cost_plan(int32_t config, int32_t n_bits, const int32_t *bits, int32_t *out, int32_t capacity) {
    clear_error();
    const int n = mgs::cost_plan_export(config, bits, n_bits, out, capacity);
    if (n < 0) set_error("no tile configuration %d or bad bit-widths", config);
    return n;
}

const char *mgs_tile_config_name(int32_t config) {
    if (config < 0 || config >= cost_config_count()) return "";
    return cost_config(config).name;
}

mgs_status mgs_set_tile_config(mgs_ctx *ctx, int32_t group_size, int32_t n_bits, int32_t config) {
    clear_error();
    if (!ctx || group_size < 1 || group_size > MGS_MAX_GROUP || n_bits < 1 ||
        n_bits > MGS_MAX_OPTIONS || config < -1 || config >= cost_config_count()) {
        set_error("bad tile request (G %d, %d bit-widths, config %d)", group_size, n_bits, config);
        return MGS_ERR_INVALID_ARG;
    }
    if (config >= 0 && !cost_config_fits(config, group_size, n_bits, nullptr)) {
        set_error("tile %s cannot run G=%d with %d bit-widths", cost_config(config).name,
                  group_size, n_bits);
        return MGS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto &v = ctx->tiles;
    v.erase(std::remove_if(v.begin(), v.end(),
                           [&](const TileChoice &t) {
                               return t.group_size == group_size && t.n_bits == n_bits;
                           }),
            v.end());
    if (config >= 0) v.push_back(TileChoice{group_size, n_bits, config});
    return MGS_OK;
}

mgs_status mgs_autotune(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid, void *stream,
                        int32_t *chosen, float *ms_per_config) {
    clear_error();
    if (!ctx || !scene) {
        set_error("ctx and scene must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    mgs_scene *sc = const_cast<mgs_scene *>(scene);
    mgs_table_layout L;
    MGS_TRY(mgs_table_layout_for(sc->n, sc->C, grid, &L));
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *table = nullptr, *scratch = nullptr;
    MGS_CUDA_TRY(dev_malloc_async(&table, (size_t)L.total_bytes, st));
    std::vector<CostSeg> segs;
    mgs_status s = scene_segments(sc, grid, table, st, &segs);
    const int nc = cost_config_count();
    size_t seg_bytes = align256(sizeof(CostSeg) * std::max<size_t>(segs.size(), 1) * kMaxSpatialBuckets);
    if (s == MGS_OK && dev_malloc_async(&scratch, seg_bytes + 256, st) != cudaSuccess) {
        set_error("autotune scratch allocation failed");
        s = MGS_ERR_OUT_OF_MEMORY;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = -1;
    float best_ms = 0;
    for (int c = 0; c < nc && s == MGS_OK; c++) {
        if (ms_per_config) ms_per_config[c] = -1.0f;
        if (!cost_config_fits(c, grid->group_size, grid->n_bits, grid->bits)) continue;
        CostLaunch launch;
        launch.segs = segs;
        launch.group_size = grid->group_size;
        launch.n_bits = grid->n_bits;
        for (int k = 0; k < grid->n_bits; k++) launch.bits[k] = grid->bits[k];
        launch.opt_hi = grid->n_bits;
        CostExec *X = nullptr;
        std::vector<CostSeg> prepared;
        int64_t n_work = 0;
        s = cost_exec_create(ctx, launch, c, &X, &prepared, &n_work);
        if (s != MGS_OK) break;
        cudaMemcpyAsync(scratch, prepared.data(), sizeof(CostSeg) * prepared.size(),
                        cudaMemcpyHostToDevice, st);
        cost_exec_bind(X, static_cast<CostSeg *>(scratch),
                       reinterpret_cast<unsigned int *>(static_cast<char *>(scratch) + seg_bytes));
        s = cost_exec_run(X, st);   // warm-up
        float ms = 0;
        if (s == MGS_OK) {
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < 2 && s == MGS_OK; rep++) s = cost_exec_run(X, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            ms *= 0.5f;
        }
        cost_exec_destroy(X);
        if (s != MGS_OK) break;
        if (ms_per_config) ms_per_config[c] = ms;
        if (best < 0 || ms < best_ms) {
            best = c;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (scratch) cudaFreeAsync(scratch, st);
    cudaFreeAsync(table, st);
    cudaStreamSynchronize(st);
    if (s != MGS_OK) return s;
    if (best < 0) {
        set_error("no tile shape holds G=%d", grid->group_size);
        return MGS_ERR_INVALID_ARG;
    }
    if (chosen) *chosen = best;
    return mgs_set_tile_config(ctx, grid->group_size, grid->n_bits, best);
}

}  // extern "C"

struct mgs_plan {
    mgs_ctx *ctx = nullptr;
    CostExec *exec = nullptr;
    void *scratch = nullptr;
    int64_t n_work = 0;
    int config = -1;
    bool use_graph = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
};

extern "C" {

mgs_status mgs_plan_create(mgs_ctx *ctx, int32_t n_scenes, const mgs_scene *const *scenes,
                           const mgs_grid *grids, void *const *tables, int32_t use_graph,
                           void *stream, mgs_plan **out) {
    clear_error();
    if (!ctx || n_scenes < 1 || !scenes || !tables || !grids || !out) {
        set_error("ctx, scenes, grids, tables and out must be non-NULL and n_scenes >= 1");
        return MGS_ERR_INVALID_ARG;
    }
    MGS_TRY(same_shape(n_scenes, grids));
    int64_t n_segs = 0;
    for (int s = 0; s < n_scenes; s++) n_segs += grids[s].n_ratios;
    if (n_segs > kMaxSegments) {
        set_error("%lld (scene, ratio) segments exceed %d", (long long)n_segs, kMaxSegments);
        return MGS_ERR_INVALID_ARG;
    }
    const mgs_grid *grid = &grids[0];
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CostLaunch launch;
    launch.group_size = grid->group_size;
    launch.n_bits = grid->n_bits;
    for (int k = 0; k < grid->n_bits; k++) launch.bits[k] = grid->bits[k];
    launch.opt_hi = grid->n_bits;
    launch.persistent = true;
    for (int s = 0; s < n_scenes; s++) {
        if (!scenes[s] || !tables[s] || !is_device_pointer(tables[s])) {
            set_error("scene %d or its table is NULL or not device memory", s);
            return MGS_ERR_INVALID_ARG;
        }
        MGS_TRY(scene_segments(const_cast<mgs_scene *>(scenes[s]), &grids[s], tables[s], st,
                               &launch.segs));
    }
    mgs_plan *P = new (std::nothrow) mgs_plan();
    if (!P) return MGS_ERR_OUT_OF_MEMORY;
    P->ctx = ctx;
    P->use_graph = use_graph != 0;
    P->config = pick_config(ctx, grid->group_size, grid->n_bits);
    std::vector<CostSeg> prepared;
    mgs_status s = cost_exec_create(ctx, launch, P->config, &P->exec, &prepared, &P->n_work);
    size_t seg_bytes = align256(sizeof(CostSeg) * std::max<size_t>(prepared.size(), 1));
    if (s == MGS_OK && cudaMalloc(&P->scratch, seg_bytes + 256) != cudaSuccess) {
        cudaGetLastError();
        set_error("plan scratch allocation failed");
        s = MGS_ERR_OUT_OF_MEMORY;
    }
    if (s == MGS_OK) {
        cudaError_t e = cudaMemcpyAsync(P->scratch, prepared.data(),
                                        sizeof(CostSeg) * prepared.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("plan upload: %s", cudaGetErrorString(e));
            s = MGS_ERR_CUDA;
        }
    }
    if (s != MGS_OK) {
        if (P->exec) cost_exec_destroy(P->exec);
        if (P->scratch) cudaFree(P->scratch);
        delete P;
        return s;
    }
    cost_exec_bind(P->exec, static_cast<CostSeg *>(P->scratch),
                   reinterpret_cast<unsigned int *>(static_cast<char *>(P->scratch) + seg_bytes));
    *out = P;
    return MGS_OK;
}

mgs_status mgs_plan_launch(mgs_plan *P, void *stream) {
    clear_error();
    if (!P) {
        set_error("plan is NULL");
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard g(P->ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!P->use_graph) return cost_exec_run(P->exec, st);
    if (!P->gexec) {
        if (st == nullptr) {
            set_error("graph capture needs a non-default stream");
            return MGS_ERR_INVALID_ARG;
        }
        MGS_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        mgs_status s = cost_exec_run(P->exec, st);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (s != MGS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        MGS_CUDA_TRY(e);
        P->graph = graph;
        MGS_CUDA_TRY(cudaGraphInstantiate(&P->gexec, graph, 0));
        count_launches(-1);   // the captured launch did not run; the replay below does
    }
    MGS_CUDA_TRY(cudaGraphLaunch(P->gexec, st));
    count_launches(1);
    return MGS_OK;
}

mgs_status mgs_plan_info(const mgs_plan *P, int64_t *work_items, int32_t *launches,
                         int32_t *tile_config) {
    if (!P) {
        set_error("plan is NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (work_items) *work_items = P->n_work;
    if (launches) *launches = P->n_work > 0 ? 1 : 0;
    if (tile_config) *tile_config = P->config;
    return MGS_OK;
}

mgs_status mgs_plan_destroy(mgs_plan *P) {
    clear_error();
    if (!P) return MGS_OK;
    DeviceGuard g(P->ctx->device);
    cudaDeviceSynchronize();
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->exec) cost_exec_destroy(P->exec);
    if (P->scratch) cudaFree(P->scratch);
    delete P;
    return MGS_OK;
}

mgs_status mgs_quantize_groups(mgs_ctx *ctx, const mgs_scene *scene, int64_t keep,
                               int32_t group_size, const uint8_t *bits, uint16_t *codes,
                               float *minmax, void *stream) {
    clear_error();
    if (!ctx || !scene || !bits || !codes || !minmax) {
        set_error("ctx, scene, bits, codes and minmax must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (keep < 1 || keep > scene->n || group_size < 1 || group_size > MGS_MAX_GROUP) {
        set_error("keep %lld or group_size %d out of range", (long long)keep, group_size);
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mgs_scene *sc = const_cast<mgs_scene *>(scene);
    // A one-ratio kept list; the scene's cached lists are left alone.
    mgs_scene tmp_owner;
    tmp_owner.ctx = sc->ctx;
    tmp_owner.n = sc->n;
    tmp_owner.C = sc->C;
    tmp_owner.d_rank_m = sc->d_rank_m;
    const int32_t *pos = nullptr;
    std::vector<int64_t> off;
    mgs_status s = scene_kept(&tmp_owner, &keep, 1, st, &pos, &off);
    if (s == MGS_OK) s = quantize_launch(ctx, sc, pos, keep, group_size, bits, codes, minmax, st);
    if (tmp_owner.kept.pos) cudaFreeAsync(tmp_owner.kept.pos, st);
    tmp_owner.kept.pos = nullptr;
    tmp_owner.d_rank_m = nullptr;
    return s;
}

}  // extern "C"
