// Scene pipeline: validation, importance rank (Sec. III-A), Morton order
// (Sec. III-G), relayout into channel slabs, kept lists per reserve ratio.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace mgs {
namespace {

constexpr int kTileThreads = 256;
constexpr int kTileItems = 16;                       // per thread
constexpr int kTile = kTileThreads * kTileItems;     // 4096 items per tile
constexpr int kWarps = kTileThreads / 32;

// Monotone map float -> uint32 (total order of finite floats; -0 < +0).
__device__ __forceinline__ uint32_t ordered_u32(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// ---------------------------------------------------------------------------
// Validation: per-channel min/max over all Gaussians, finiteness flags.
// The grid-stride step is a multiple of C, so each thread always reads the
// same channel of the row-major [n][C] array.
// ---------------------------------------------------------------------------
__global__ void k_validate(const float *__restrict__ attrs, int64_t total, int32_t C,
                           const float *__restrict__ imp, int64_t n, uint32_t *chan_min,
                           uint32_t *chan_max, uint32_t *flags) {
    __shared__ uint32_t smin[MGS_MAX_CHANNELS], smax[MGS_MAX_CHANNELS];
    __shared__ uint32_t sflag;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        smin[c] = 0xFFFFFFFFu;
        smax[c] = 0u;
    }
    if (threadIdx.x == 0) sflag = 0;
    __syncthreads();
    int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;   // multiple of C
    uint32_t mn = 0xFFFFFFFFu, mx = 0u, bad = 0u;
    // eight independent loads in flight per thread (the same channel: the
    // stride is a multiple of C); min, max and the flag do not depend on order
    int64_t e = gtid;
    for (; e + 7 * stride < total; e += 8 * stride) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = __ldg(attrs + e + u * stride);
#pragma unroll
        for (int u = 0; u < 8; u++) {
            if (!isfinite(v[u])) bad = 1u;
            const uint32_t o = ordered_u32(v[u]);
            mn = min(mn, o);
            mx = max(mx, o);
        }
    }
    for (; e < total; e += stride) {
        float v = __ldg(attrs + e);
        if (!isfinite(v)) bad = 1u;
        uint32_t o = ordered_u32(v);
        mn = min(mn, o);
        mx = max(mx, o);
    }
    for (int64_t i = gtid; i < n; i += stride)
        if (!isfinite(imp[i])) bad |= 2u;
    if (gtid < total) {
        int c = (int)(gtid % C);
        atomicMin(&smin[c], mn);
        atomicMax(&smax[c], mx);
    }
    if (bad) atomicOr(&sflag, bad);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        if (smin[c] != 0xFFFFFFFFu) atomicMin(&chan_min[c], smin[c]);
        if (smax[c] != 0u) atomicMax(&chan_max[c], smax[c]);
    }
    if (threadIdx.x == 0 && sflag) atomicOr(flags, sflag);
}

// ---------------------------------------------------------------------------
// LSD radix sort of (key, value) pairs, 8-bit digits, stable.
// ---------------------------------------------------------------------------
template <typename K>
__global__ void k_digit_hist(const K *__restrict__ keys, int64_t n, int shift,
                             uint32_t *__restrict__ hist, int n_tiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int j = 0; j < kTileItems; j++) {
        int64_t i = base + j * kTileThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of `total` uint32 entries in place, one block of 1024 threads.
__global__ void k_scan_u32(uint32_t *data, int64_t total) {
    __shared__ uint32_t part[1024];
    int t = threadIdx.x;
    int64_t chunk = (total + 1023) / 1024;
    int64_t lo = t * chunk, hi = min(total, lo + chunk);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; i++) s += data[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = t ? part[t - 1] : 0u;
    for (int64_t i = lo; i < hi; i++) {
        uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
}

// Exclusive scan of a long uint32 array in two launches: every block scans
// its chunk in place and records the chunk total; then every block adds the
// totals of the chunks before it.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanChunk = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads)
    k_scan_chunks(uint32_t *__restrict__ data, int64_t total, uint32_t *__restrict__ totals) {
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer], s = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        v[j] = base + j < total ? data[base + j] : 0u;
        s += v[j];
    }
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_tot[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_tot[lane] = wi - w;   // exclusive prefix of the warp totals
        if (lane == 31) totals[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + inc - s;
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        if (base + j < total) data[base + j] = run;
        run += v[j];
    }
}

__global__ void __launch_bounds__(kScanThreads)
    k_scan_add(uint32_t *__restrict__ data, int64_t total, const uint32_t *__restrict__ totals) {
    __shared__ uint32_t off;
    if (threadIdx.x < 32) {
        uint32_t s = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += 32) s += totals[b];
        s = __reduce_add_sync(0xFFFFFFFFu, s);
        if (threadIdx.x == 0) off = s;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    for (int j = threadIdx.x; j < kScanChunk; j += kScanThreads)
        if (base + j < total) data[base + j] += off;
}

// The tile's pairs are first placed in shared memory in (digit, tile order)
// order -- the same stable ranks as before -- and then written out from there,
// so consecutive threads store consecutive positions of a digit's bucket.
template <typename K>
__global__ void __launch_bounds__(kTileThreads) k_scatter(const K *__restrict__ kin,
                                                          const uint32_t *__restrict__ vin,
                                                          K *__restrict__ kout,
                                                          uint32_t *__restrict__ vout, int64_t n,
                                                          int shift,
                                                          const uint32_t *__restrict__ offs,
                                                          int n_tiles) {
    extern __shared__ __align__(16) unsigned char s_pairs[];   // K[kTile], then uint32[kTile]
    K *skey = reinterpret_cast<K *>(s_pairs);
    uint32_t *sval = reinterpret_cast<uint32_t *>(s_pairs + sizeof(K) * kTile);
    __shared__ uint32_t wcnt[kWarps][257];
    __shared__ uint32_t tdo[256];         // first tile slot of each digit
    __shared__ uint32_t wtot[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * 257; i += kTileThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * kTile;
    const int64_t base = tile0 + warp * (kTile / kWarps);
    K key[kTileItems];
    uint32_t val[kTileItems], local[kTileItems], dig[kTileItems];
#pragma unroll
    for (int c = 0; c < kTileItems; c++) {
        int64_t i = base + c * 32 + lane;
        bool valid = i < n;
        key[c] = valid ? kin[i] : K(0);
        val[c] = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((uint32_t)(key[c] >> shift) & 255u) : 256u;
        dig[c] = d;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        uint32_t before = wcnt[warp][d];
        local[c] = before + __popc(peers & lt);
        __syncwarp();
        if (lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive scan over warps, per digit (thread = digit), then over the
    // digits' tile totals
    uint32_t cnt = 0;
    {
        const int d = threadIdx.x;   // 256 threads = 256 digits
        for (int w = 0; w < kWarps; w++) {
            uint32_t v = wcnt[w][d];
            wcnt[w][d] = cnt;
            cnt += v;
        }
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += wtot[w];
    tdo[threadIdx.x] = wpre + inc - cnt;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kTileItems; c++) {
        if (dig[c] < 256u) {
            const uint32_t sp = tdo[dig[c]] + wcnt[warp][dig[c]] + local[c];
            skey[sp] = key[c];
            sval[sp] = val[c];
        }
    }
    __syncthreads();
    const int nv = n - tile0 < (int64_t)kTile ? (int)(n - tile0) : kTile;
#pragma unroll 4
    for (int j = threadIdx.x; j < nv; j += kTileThreads) {
        const K kk = skey[j];
        const uint32_t d = (uint32_t)(kk >> shift) & 255u;
        const uint64_t pos = (uint64_t)offs[(int64_t)d * n_tiles + blockIdx.x] + (uint32_t)(j - tdo[d]);
        kout[pos] = kk;
        vout[pos] = sval[j];
    }
}

template <typename K>
mgs_status radix_sort_pairs(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt,
                            uint32_t *hist, int64_t n, int key_bits, cudaStream_t st,
                            bool *result_in_alt) {
    int n_tiles = (int)((n + kTile - 1) / kTile);
    K *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    bool alt = false;
    const int64_t entries = (int64_t)256 * n_tiles;
    const int scan_blocks = (int)((entries + kScanChunk - 1) / kScanChunk);
    uint32_t *totals = hist + entries;   // hist holds 256 * n_tiles + scan_blocks entries
    const int kScatterSmem = (int)((sizeof(K) + sizeof(uint32_t)) * kTile);   // the tile's pairs
    MGS_CUDA_TRY(cudaFuncSetAttribute(k_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kScatterSmem));
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_digit_hist<K><<<n_tiles, kTileThreads, 0, st>>>(ki, n, shift, hist, n_tiles);
        k_scan_chunks<<<scan_blocks, kScanThreads, 0, st>>>(hist, entries, totals);
        k_scan_add<<<scan_blocks, kScanThreads, 0, st>>>(hist, entries, totals);
        k_scatter<K><<<n_tiles, kTileThreads, kScatterSmem, st>>>(ki, vi, ko, vo, n, shift, hist, n_tiles);
        count_launches(4);
        std::swap(ki, ko);
        std::swap(vi, vo);
        alt = !alt;
    }
    MGS_CUDA_TRY(cudaGetLastError());
    *result_in_alt = alt;
    return MGS_OK;
}

// ---------------------------------------------------------------------------
// Importance keys: descending importance, ties by index (stable sort on
// the complement of the ordered bits; -0 is folded onto +0 first).
// ---------------------------------------------------------------------------
__global__ void k_importance_keys(const float *__restrict__ imp, int64_t n, uint32_t *keys,
                                  uint32_t *vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f = imp[i];
    if (f == 0.0f) f = 0.0f;
    keys[i] = ~ordered_u32(f);
    vals[i] = (uint32_t)i;
}

__global__ void k_rank_scatter(const uint32_t *__restrict__ sorted_idx, int64_t n,
                               int32_t *__restrict__ rank) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) rank[sorted_idx[j]] = (int32_t)j;
}

// ---------------------------------------------------------------------------
// Morton codes: t = (p - lo) / (hi - lo) in FP32, axis code floor(t * 2^21)
// clamped to 2^21 - 1 (0 when hi == lo); bit k of x/y/z -> bit 3k/3k+1/3k+2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t axis_code(float p, float lo, float hi) {
    float d = __fsub_rn(hi, lo);
    if (d == 0.0f) return 0u;
    float t = __fdiv_rn(__fsub_rn(p, lo), d);
    float s = floorf(__fmul_rn(t, 2097152.0f));
    s = fminf(fmaxf(s, 0.0f), 2097151.0f);
    return (uint32_t)s;
}
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
__global__ void k_morton(const float *__restrict__ attrs, int64_t n, int32_t C, float lo0, float hi0,
                         float lo1, float hi1, float lo2, float hi2, uint64_t *codes,
                         uint64_t *keys, uint32_t *vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *row = attrs + i * C;
    uint32_t x = axis_code(row[0], lo0, hi0);
    uint32_t y = axis_code(row[1], lo1, hi1);
    uint32_t z = axis_code(row[2], lo2, hi2);
    uint64_t code = spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
    codes[i] = code;
    keys[i] = code;
    vals[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// Relayout: slabs[s][p][j] = attrs[order[p]][8 s + j] (0 past the last channel),
// rank_m[p] = rank[order[p]].  One warp per 32 consecutive positions: the
// warp reads each source row with coalesced loads (lane = channel) and writes
// channel c to slab c / 8, so one store fills four whole 32-byte slab rows.
// ---------------------------------------------------------------------------
__global__ void k_relayout(const float *__restrict__ attrs, int64_t n, int32_t C, int32_t n_slabs,
                           const uint32_t *__restrict__ order, const int32_t *__restrict__ rank,
                           float *__restrict__ slabs, int32_t *__restrict__ rank_m,
                           int32_t *__restrict__ order_out) {
    const int lane = threadIdx.x & 31;
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane;   // the warp's first position
    if (p0 >= n) return;   // whole warps
    const int nr = n - p0 < 32 ? (int)(n - p0) : 32;
    uint32_t my_i = 0;
    if (lane < nr) {
        my_i = order[p0 + lane];
        rank_m[p0 + lane] = rank[my_i];
        order_out[p0 + lane] = (int32_t)my_i;
    }
    const int width = 8 * n_slabs;   // channels including the zero padding
    for (int cb = 0; cb < width; cb += 32) {
        const int c = cb + lane;
        float *dst = slabs + (int64_t)(c >> 3) * n * 8 + (c & 7);
#pragma unroll 8
        for (int r = 0; r < 32; r++) {
            const uint32_t i = __shfl_sync(0xFFFFFFFFu, my_i, r);
            if (r < nr && c < width) dst[(p0 + r) * 8] = c < C ? __ldg(attrs + (int64_t)i * C + c) : 0.0f;
        }
    }
}

// ---------------------------------------------------------------------------
// Kept lists: for every ratio r, the Morton positions p with rank_m[p] < K_r,
// ascending.  r0(p) = #{r : K_r <= rank_m[p]}: position p is in lists r >= r0.
// ---------------------------------------------------------------------------
struct KeepArg {
    int64_t k[MGS_MAX_RATIOS];
    int32_t n_r;
};

__device__ __forceinline__ int first_ratio(int32_t rank, const KeepArg &ka) {
    int r0 = 0;
    for (int r = 0; r < ka.n_r; r++) r0 += (ka.k[r] <= (int64_t)rank) ? 1 : 0;
    return r0;
}

__global__ void __launch_bounds__(kTileThreads) k_kept_count(const int32_t *__restrict__ rank_m,
                                                             int64_t n, KeepArg ka,
                                                             uint32_t *__restrict__ cnt,
                                                             int n_tiles) {
    __shared__ uint32_t h[MGS_MAX_RATIOS + 1];
    for (int i = threadIdx.x; i <= ka.n_r; i += kTileThreads) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kTile;
    for (int j = 0; j < kTileItems; j++) {
        int64_t p = base + j * kTileThreads + threadIdx.x;
        if (p < n) atomicAdd(&h[first_ratio(rank_m[p], ka)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int r = 0; r < ka.n_r; r++) {
            run += h[r];
            cnt[(int64_t)r * n_tiles + blockIdx.x] = run;   // positions of this tile in list r
        }
    }
}

__global__ void __launch_bounds__(kTileThreads) k_kept_scatter(const int32_t *__restrict__ rank_m,
                                                               int64_t n, KeepArg ka,
                                                               const uint32_t *__restrict__ base_r,
                                                               int n_tiles,
                                                               int32_t *__restrict__ out) {
    __shared__ uint32_t wc[kWarps][MGS_MAX_RATIOS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t wbase = (int64_t)blockIdx.x * kTile + warp * (kTile / kWarps);
    int r0v[kTileItems];
    for (int c = 0; c < kTileItems; c++) {
        int64_t p = wbase + c * 32 + lane;
        r0v[c] = p < n ? first_ratio(rank_m[p], ka) : MGS_MAX_RATIOS + 1;
    }
    // per-warp counts per ratio
    for (int r = 0; r < ka.n_r; r++) {
        uint32_t tot = 0;
        for (int c = 0; c < kTileItems; c++) tot += __popc(__ballot_sync(0xFFFFFFFFu, r0v[c] <= r));
        if (lane == 0) wc[warp][r] = tot;
    }
    __syncthreads();
    if (threadIdx.x < ka.n_r) {
        int r = threadIdx.x;
        uint32_t run = base_r[(int64_t)r * n_tiles + blockIdx.x];
        for (int w = 0; w < kWarps; w++) {
            uint32_t v = wc[w][r];
            wc[w][r] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int r = 0; r < ka.n_r; r++) {
        uint32_t at = wc[warp][r];
        for (int c = 0; c < kTileItems; c++) {
            bool in = r0v[c] <= r;
            uint32_t m = __ballot_sync(0xFFFFFFFFu, in);
            if (in) out[at + __popc(m & lt)] = (int32_t)(wbase + c * 32 + lane);
            at += __popc(m);
        }
    }
}

template <typename T>
mgs_status dalloc(T **p, size_t count, cudaStream_t st) {
    cudaError_t e = dev_malloc_async((void **)p, std::max<size_t>(count, 1) * sizeof(T), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return MGS_ERR_OUT_OF_MEMORY;
    }
    return MGS_OK;
}

float host_from_ordered(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

mgs_status scene_build(mgs_ctx *ctx, const float *d_attrs, const float *d_imp, int64_t n, int32_t C,
                       cudaStream_t st, mgs_scene *sc) {
    sc->ctx = ctx;
    sc->n = n;
    sc->C = C;
    sc->n_slabs = (C + kSlabWidth - 1) / kSlabWidth;

    // 1. validation
    uint32_t *d_stat = nullptr;   // [C] min, [C] max, flags
    MGS_TRY(dalloc(&d_stat, 2 * (size_t)C + 1, st));
    MGS_CUDA_TRY(cudaMemsetAsync(d_stat, 0xFF, sizeof(uint32_t) * C, st));
    MGS_CUDA_TRY(cudaMemsetAsync(d_stat + C, 0, sizeof(uint32_t) * (C + 1), st));
    int vblocks = ctx->sm_count * 4;
    vblocks = std::max(C, (vblocks / C) * C);   // stride multiple of C
    k_validate<<<vblocks, 256, 0, st>>>(d_attrs, n * C, C, d_imp, n, d_stat, d_stat + C,
                                        d_stat + 2 * C);
    count_launches(1);
    MGS_CUDA_TRY(cudaGetLastError());
    std::vector<uint32_t> h_stat(2 * (size_t)C + 1);
    MGS_CUDA_TRY(cudaMemcpyAsync(h_stat.data(), d_stat, sizeof(uint32_t) * h_stat.size(),
                                 cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(d_stat, st);
    if (h_stat[2 * C] != 0) {
        set_error("scene has non-finite %s", (h_stat[2 * C] & 1u) ? "attributes" : "importance");
        return MGS_ERR_NONFINITE;
    }
    float lo[3], hi[3];
    for (int c = 0; c < C; c++) {
        float mn = host_from_ordered(h_stat[c]);
        float mx = host_from_ordered(h_stat[C + c]);
        volatile float range = mx - mn;
        if (!std::isfinite((float)range)) {
            set_error("channel %d range %g - %g overflows FP32", c, (double)mx, (double)mn);
            return MGS_ERR_RANGE;
        }
        if (c < 3) {
            lo[c] = mn;
            hi[c] = mx;
        }
    }

    // 2. scratch for the sorts (freed on every return from here on)
    uint64_t *k64 = nullptr, *k64b = nullptr;
    uint32_t *v = nullptr, *vb = nullptr, *hist = nullptr;
    int32_t *rank = nullptr;
    struct Scratch {
        void **p[6];
        cudaStream_t st;
        ~Scratch() {
            for (void **q : p)
                if (*q) cudaFreeAsync(*q, st);
        }
    } guard{{(void **)&k64, (void **)&k64b, (void **)&v, (void **)&vb, (void **)&hist, (void **)&rank}, st};
    int n_tiles = (int)((n + kTile - 1) / kTile);
    MGS_TRY(dalloc(&k64, n, st));
    MGS_TRY(dalloc(&k64b, n, st));
    MGS_TRY(dalloc(&v, n, st));
    MGS_TRY(dalloc(&vb, n, st));
    MGS_TRY(dalloc(&hist, (size_t)256 * n_tiles + (256 * (size_t)n_tiles + 8191) / 8192, st));
    uint32_t *k32 = reinterpret_cast<uint32_t *>(k64);
    uint32_t *k32b = reinterpret_cast<uint32_t *>(k64b);

    MGS_TRY(dalloc(&sc->d_rank_m, n, st));
    MGS_TRY(dalloc(&sc->d_order, n, st));
    MGS_TRY(dalloc(&sc->d_codes, n, st));
    MGS_TRY(dalloc(&sc->d_slabs, (size_t)sc->n_slabs * n * kSlabWidth, st));
    MGS_TRY(dalloc(&rank, n, st));

    int blocks = (int)((n + 255) / 256);
    // 3. importance rank
    k_importance_keys<<<blocks, 256, 0, st>>>(d_imp, n, k32, v);
    bool alt = false;
    MGS_TRY(radix_sort_pairs<uint32_t>(k32, v, k32b, vb, hist, n, 32, st, &alt));
    k_rank_scatter<<<blocks, 256, 0, st>>>(alt ? vb : v, n, rank);

    // 4. Morton order
    k_morton<<<blocks, 256, 0, st>>>(d_attrs, n, C, lo[0], hi[0], lo[1], hi[1], lo[2], hi[2],
                                     sc->d_codes, k64, v);
    MGS_TRY(radix_sort_pairs<uint64_t>(k64, v, k64b, vb, hist, n, 63, st, &alt));

    // 5. relayout
    k_relayout<<<blocks, 256, 0, st>>>(d_attrs, n, C, sc->n_slabs, alt ? vb : v, rank, sc->d_slabs,
                                       sc->d_rank_m, sc->d_order);
    count_launches(4);   // importance keys, rank scatter, Morton codes, relayout
    MGS_CUDA_TRY(cudaGetLastError());
    sc->device_bytes = (int64_t)sc->n_slabs * n * kSlabWidth * 4 + n * (4 + 4 + 8);
    return MGS_OK;
}

mgs_status scene_kept(mgs_scene *sc, const int64_t *keep, int32_t n_r, cudaStream_t st,
                      const int32_t **pos_out, std::vector<int64_t> *offset_out) {
    std::vector<int64_t> want(keep, keep + n_r);
    if (sc->kept.pos && sc->kept.keep == want) {
        *pos_out = sc->kept.pos;
        *offset_out = sc->kept.offset;
        return MGS_OK;
    }
    std::vector<int64_t> off(n_r + 1, 0);
    for (int r = 0; r < n_r; r++) off[r + 1] = off[r] + keep[r];
    int64_t total = off[n_r];
    if (total >= (int64_t)1 << 32) {
        set_error("kept lists of %lld entries exceed 2^32", (long long)total);
        return MGS_ERR_INVALID_ARG;
    }
    if (sc->kept.pos) {
        cudaFreeAsync(sc->kept.pos, st);
        sc->kept.pos = nullptr;
    }
    int32_t *pos = nullptr;
    MGS_TRY(dalloc(&pos, (size_t)total, st));
    int n_tiles = (int)((sc->n + kTile - 1) / kTile);
    uint32_t *cnt = nullptr;
    if (mgs_status s = dalloc(&cnt, (size_t)n_r * n_tiles, st); s != MGS_OK) {
        cudaFreeAsync(pos, st);
        return s;
    }
    KeepArg ka{};
    ka.n_r = n_r;
    for (int r = 0; r < n_r; r++) ka.k[r] = keep[r];
    k_kept_count<<<n_tiles, kTileThreads, 0, st>>>(sc->d_rank_m, sc->n, ka, cnt, n_tiles);
    // The per-tile counts are inclusive over ratios; turn them into per-ratio
    // counts of this tile, then an exclusive scan over [r][tile] gives each
    // tile's start in the concatenated lists.
    k_scan_u32<<<1, 1024, 0, st>>>(cnt, (int64_t)n_r * n_tiles);
    k_kept_scatter<<<n_tiles, kTileThreads, 0, st>>>(sc->d_rank_m, sc->n, ka, cnt, n_tiles, pos);
    count_launches(3);
    MGS_CUDA_TRY(cudaGetLastError());
    cudaFreeAsync(cnt, st);
    sc->kept.keep = want;
    sc->kept.offset = off;
    sc->kept.pos = pos;
    sc->kept.bytes = sizeof(int32_t) * (size_t)total;
    *pos_out = pos;
    *offset_out = off;
    return MGS_OK;
}

mgs_status kept_list_into(const mgs_scene *sc, int64_t keep, int32_t *pos, uint32_t *tile_cnt,
                          cudaStream_t st) {
    const int n_tiles = (int)((sc->n + kTile - 1) / kTile);
    KeepArg ka{};
    ka.n_r = 1;
    ka.k[0] = keep;
    k_kept_count<<<n_tiles, kTileThreads, 0, st>>>(sc->d_rank_m, sc->n, ka, tile_cnt, n_tiles);
    k_scan_u32<<<1, 1024, 0, st>>>(tile_cnt, (int64_t)n_tiles);
    k_kept_scatter<<<n_tiles, kTileThreads, 0, st>>>(sc->d_rank_m, sc->n, ka, tile_cnt, n_tiles, pos);
    count_launches(3);
    MGS_CUDA_TRY(cudaGetLastError());
    return MGS_OK;
}

static_assert(kTile == kKeptTile, "kept-list tiles are sized by kKeptTile");

}  // namespace mgs
