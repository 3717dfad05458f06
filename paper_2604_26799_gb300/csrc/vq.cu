// Vector quantisation of the 1+D SH coefficients (Sec. III-D "Clustering 1+D
// SH Coefficients"): nearest-codebook assignment and the batched (mini-batch)
// k-means the paper cites, in a form whose every decision is reproducible:
//
//   score(x, k) = fl(|c_k|^2 - 2 x.c_k)   (|x|^2 dropped: the argmin is the same)
//   both sums accumulated with fmaf over the dimensions in ascending order;
//   the smallest score wins, ties to the lower k.
//
//   batch update: every centre moves to the running mean of all vectors
//   assigned to it so far, c = (v c + sum x) / (v + m), the batch's sum taken
//   in FP64 in batch order and the result rounded once to FP32.
//
// k_vq_assign: 128 threads x 2 vectors per thread in registers (the dimension
// padded with zeros to DP, a multiple of 8; adding 0 * 0 leaves an fmaf chain
// unchanged), codebook tiles of 64 centres staged in shared memory and read
// as float4 broadcasts.  The update is a one-warp stable counting sort of the
// batch by centre (match_any ranks, centre cursors in shared memory), then one
// thread per (centre, dimension) summing its vectors in batch order.
#include <cuda_runtime.h>

#include <cfloat>
#include <mutex>

#include "internal.h"

namespace mgs {
namespace {

constexpr int kVqThreads = 128;
constexpr int kVqTile = 64;     // centres per shared-memory tile
constexpr int kVqMaxTrainK = 49152;      // centres whose sort counters fit in shared memory
constexpr int kVqMaxK = 1 << 20;

__global__ void k_vq_norms(const float *__restrict__ cb, int32_t K, int32_t D, float *__restrict__ cc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const float *c = cb + (int64_t)k * D;
    float s = 0.0f;
    for (int d = 0; d < D; d++) s = __fmaf_rn(c[d], c[d], s);
    cc[k] = s;
}

template <int DP, int kVqPts>
__global__ void __launch_bounds__(kVqThreads)
    k_vq_assign(const float *__restrict__ x, int64_t n, int32_t D, const int32_t *__restrict__ rows,
                const float *__restrict__ cb, const float *__restrict__ cc, int32_t K,
                int32_t *__restrict__ idx_out, float *__restrict__ score_out) {
    __shared__ __align__(16) float s_c[kVqTile * DP];
    __shared__ float s_cc[kVqTile];
    const int64_t base = ((int64_t)blockIdx.x * kVqThreads + threadIdx.x) * kVqPts;
    float xv[kVqPts][DP];
    int64_t row[kVqPts];
#pragma unroll
    for (int p = 0; p < kVqPts; p++) {
        const int64_t i = base + p;
        row[p] = i < n ? (rows ? (int64_t)rows[i] : i) : -1;
#pragma unroll
        for (int d = 0; d < DP; d++) xv[p][d] = (row[p] >= 0 && d < D) ? x[row[p] * D + d] : 0.0f;
    }
    float best[kVqPts];
    int32_t bi[kVqPts];
#pragma unroll
    for (int p = 0; p < kVqPts; p++) {
        best[p] = FLT_MAX;
        bi[p] = 0;
    }
    bool first = true;
    for (int k0 = 0; k0 < K; k0 += kVqTile) {
        const int nk = min(kVqTile, K - k0);
        __syncthreads();
        for (int e = threadIdx.x; e < kVqTile * DP; e += kVqThreads) {
            const int kk = e / DP, d = e - kk * DP;
            s_c[e] = (kk < nk && d < D) ? cb[(int64_t)(k0 + kk) * D + d] : 0.0f;
        }
        if (threadIdx.x < kVqTile) s_cc[threadIdx.x] = threadIdx.x < nk ? cc[k0 + threadIdx.x] : 0.0f;
        __syncthreads();
        for (int kk = 0; kk < nk; kk++) {
            const float4 *c4 = reinterpret_cast<const float4 *>(s_c + kk * DP);
            float dot[kVqPts];
#pragma unroll
            for (int p = 0; p < kVqPts; p++) dot[p] = 0.0f;
#pragma unroll
            for (int q = 0; q < DP / 4; q++) {
                const float4 c = c4[q];
#pragma unroll
                for (int p = 0; p < kVqPts; p++) {
                    dot[p] = __fmaf_rn(xv[p][4 * q + 0], c.x, dot[p]);
                    dot[p] = __fmaf_rn(xv[p][4 * q + 1], c.y, dot[p]);
                    dot[p] = __fmaf_rn(xv[p][4 * q + 2], c.z, dot[p]);
                    dot[p] = __fmaf_rn(xv[p][4 * q + 3], c.w, dot[p]);
                }
            }
            const float ck = s_cc[kk];
#pragma unroll
            for (int p = 0; p < kVqPts; p++) {
                const float score = __fmaf_rn(-2.0f, dot[p], ck);
                // the first centre is taken whatever its score (as a sequential scan would)
                if ((first && kk == 0) || score < best[p]) {
                    best[p] = score;
                    bi[p] = k0 + kk;
                }
            }
        }
        first = false;
    }
#pragma unroll
    for (int p = 0; p < kVqPts; p++) {
        const int64_t i = base + p;
        if (i < n) {
            idx_out[i] = bi[p];
            if (score_out) score_out[i] = best[p];
        }
    }
}

// Stable counting sort of the batch by assigned centre, in three steps over
// chunks of kVqChunk batch positions: per-chunk counts of every centre; the
// first slot of every (chunk, centre), the centre's first slot plus the
// counts of the earlier chunks; then each chunk places its positions, ranked among equal
// centres by the warps in order (match_any within a warp, running counts in
// shared memory across the warps), so positions stay in batch order.
constexpr int kVqChunk = 256;

__global__ void __launch_bounds__(kVqChunk)
    k_vq_chunk_counts(const int32_t *__restrict__ a, int32_t b, int32_t K, int32_t *__restrict__ cnt) {
    extern __shared__ int32_t s_cnt[];   // [K]
    for (int k = threadIdx.x; k < K; k += kVqChunk) s_cnt[k] = 0;
    __syncthreads();
    const int j = blockIdx.x * kVqChunk + threadIdx.x;
    if (j < b) atomicAdd(&s_cnt[a[j]], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += kVqChunk) cnt[(int64_t)blockIdx.x * K + k] = s_cnt[k];
}

// First slot of every (chunk, centre): the centre's first slot off[k] plus
// the counts of the earlier chunks (the counts are [chunk][centre], so a
// warp's loads are contiguous).
// One CTA per 32 entries (a lane each); its warps split the chunks into
// contiguous ranges: each warp sums its range (independent loads), the warps'
// sums give each range's start, then each warp writes its range's prefixes.
constexpr int kSlotWarps = 8;
__global__ void __launch_bounds__(32 * kSlotWarps)
    k_vq_slots(int32_t *__restrict__ cnt, int32_t nch, const int32_t *__restrict__ off, int32_t K) {
    __shared__ int32_t part[kSlotWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    const int per = (nch + kSlotWarps - 1) / kSlotWarps;
    const int c0 = warp * per, c1 = min(nch, c0 + per);
    int32_t sum = 0;
    if (k < K) {
#pragma unroll 8
        for (int c = c0; c < c1; c++) sum += cnt[(int64_t)c * K + k];
    }
    part[warp][lane] = sum;
    __syncthreads();
    if (k >= K) return;
    int32_t run = off[k];
    for (int w = 0; w < warp; w++) run += part[w][lane];
    for (int cb = c0; cb < c1; cb += 8) {
        int32_t t[8];
#pragma unroll
        for (int u = 0; u < 8; u++) t[u] = cb + u < c1 ? cnt[(int64_t)(cb + u) * K + k] : 0;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            if (cb + u < c1) cnt[(int64_t)(cb + u) * K + k] = run;
            run += t[u];
        }
    }
}

__global__ void __launch_bounds__(kVqChunk)
    k_vq_chunk_place(const int32_t *__restrict__ a, int32_t b, int32_t K,
                     const int32_t *__restrict__ slot, int32_t *__restrict__ perm) {
    extern __shared__ int32_t s_run[];   // [K]: positions of each centre placed by earlier warps
    for (int k = threadIdx.x; k < K; k += kVqChunk) s_run[k] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * kVqChunk + threadIdx.x;
    const bool act = j < b;
    const int k = act ? a[j] : -1 - lane;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, k);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    for (int w = 0; w < kVqChunk / 32; w++) {
        if (warp == w && act) {
            perm[slot[(int64_t)blockIdx.x * K + k] + s_run[k] + rank] = j;
        }
        __syncthreads();
        if (warp == w && act && rank == 0) s_run[k] += __popc(peers);
        __syncthreads();
    }
}

// Batch rows outside [0, n): *bad gets 1 (the update is then not run).
__global__ void k_vq_check_rows(const int32_t *__restrict__ rows, int64_t total, int64_t n,
                                unsigned int *__restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool out = i < total && (rows[i] < 0 || (int64_t)rows[i] >= n);
    if (__any_sync(0xFFFFFFFFu, out) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

__global__ void k_vq_count(const int32_t *__restrict__ a, int32_t b, int32_t *__restrict__ m) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < b) atomicAdd(&m[a[j]], 1);
}

// Exclusive scan of K counts (one CTA of 1024 threads, chunks in order).
__global__ void __launch_bounds__(1024)
    k_vq_scan(const int32_t *__restrict__ m, int32_t K, int32_t *__restrict__ off) {
    __shared__ int32_t s[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < K; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < K ? m[i] : 0;
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s[w] = inc;
        __syncthreads();
        int wb = 0, all = 0;
        for (int q = 0; q < 32; q++) {
            if (q < w) wb += s[q];
            all += s[q];
        }
        if (i < K) off[i] = carry + wb + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += all;
        __syncthreads();
    }
}

// One thread per (centre, dimension): the running mean over its batch vectors.
__global__ void k_vq_move(const float *__restrict__ x, int32_t D, const int32_t *__restrict__ rows,
                          const int32_t *__restrict__ perm, const int32_t *__restrict__ off,
                          const int32_t *__restrict__ m, float *__restrict__ cb, int32_t K,
                          const int64_t *__restrict__ counts) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)K * D) return;
    const int k = (int)(t / D), d = (int)(t - (int64_t)k * D);
    const int mk = m[k];
    if (!mk) return;
    double sum = 0.0;
    const int o = off[k];
    // eight vectors at a time: their row indices, then their values, are
    // loaded together; the sum still runs in batch order
    int r = 0;
    for (; r + 8 <= mk; r += 8) {
        int64_t ri[8];
        float xv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) ri[u] = rows[perm[o + r + u]];
#pragma unroll
        for (int u = 0; u < 8; u++) xv[u] = x[ri[u] * D + d];
#pragma unroll
        for (int u = 0; u < 8; u++) sum = __dadd_rn(sum, (double)xv[u]);
    }
    for (; r < mk; r++) sum = __dadd_rn(sum, (double)x[(int64_t)rows[perm[o + r]] * D + d]);
    const double v = (double)counts[k];
    const double num = __dadd_rn(__dmul_rn(v, (double)cb[t]), sum);
    cb[t] = __double2float_rn(__ddiv_rn(num, __dadd_rn(v, (double)mk)));
}

__global__ void k_vq_counts(int64_t *__restrict__ counts, const int32_t *__restrict__ m, int32_t K) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) counts[k] += m[k];
}

__global__ void k_vq_retain(const int32_t *__restrict__ rows, int64_t n_retain, int32_t K,
                            int32_t *__restrict__ idx) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_retain) idx[rows[j]] = K + (int32_t)j;
}

using AssignFn = void (*)(const float *, int64_t, int32_t, const int32_t *, const float *,
                          const float *, int32_t, int32_t *, float *);

template <int P>
AssignFn pick_assign(int D) {
    if (D <= 8) return k_vq_assign<8, P>;
    if (D <= 16) return k_vq_assign<16, P>;
    if (D <= 24) return k_vq_assign<24, P>;
    if (D <= 32) return k_vq_assign<32, P>;
    if (D <= 48) return k_vq_assign<48, P>;
    return k_vq_assign<64, P>;
}

// Two vectors per thread: each float4 broadcast of the codebook then feeds
// eight fused multiply-adds (one vector per thread measured 2.8x slower per score).
mgs_status assign_launch(const float *x, int64_t n, int32_t D, const int32_t *rows, const float *cb,
                         const float *cc, int32_t K, int32_t *idx, float *score, cudaStream_t st) {
    if (n == 0) return MGS_OK;
    const int P = 2;
    const int64_t per_cta = (int64_t)kVqThreads * P;
    const int64_t grid = (n + per_cta - 1) / per_cta;
    AssignFn f = pick_assign<2>(D);
    f<<<(unsigned)grid, kVqThreads, 0, st>>>(x, n, D, rows, cb, cc, K, idx, score);
    count_launches(1);
    MGS_CUDA_TRY(cudaGetLastError());
    return MGS_OK;
}

mgs_status check_vq_args(const void *x, int64_t n, int32_t D, const void *cb, int32_t K) {
    if (!x || !cb || n < 0 || D < 1 || D > 64 || K < 1 || K > kVqMaxK) {
        set_error("vq: x and codebook must be non-NULL, 1 <= D <= 64, 1 <= K <= %d", kVqMaxK);
        return MGS_ERR_INVALID_ARG;
    }
    if (!is_device_pointer(x) || !is_device_pointer(cb)) {
        set_error("vq: x and codebook must be device memory");
        return MGS_ERR_INVALID_ARG;
    }
    if (n > ((int64_t)1 << 31) - 1) {
        set_error("vq: n = %lld exceeds 2^31 - 1", (long long)n);
        return MGS_ERR_INVALID_ARG;
    }
    return MGS_OK;
}

}  // namespace
}  // namespace mgs

using namespace mgs;

// Per-call scratch of the tensor path: codebook tiles, then max |c|^2,
// the re-score count and the error flag.
struct TcScratch {
    unsigned char *tiles = nullptr;
    unsigned int *cmax2 = nullptr;
    unsigned long long *stats = nullptr;
    unsigned int *err = nullptr;
};

static mgs_status tc_scratch(int32_t K, int32_t D, cudaStream_t st, void **base, TcScratch *T) {
    const size_t tb = (vq_tc_workspace(K, D) + 255) & ~(size_t)255;
    MGS_CUDA_TRY(cudaMallocAsync(base, tb + 32, st));
    unsigned char *p = static_cast<unsigned char *>(*base);
    T->tiles = p;
    T->stats = reinterpret_cast<unsigned long long *>(p + tb);
    T->cmax2 = reinterpret_cast<unsigned int *>(p + tb + 8);
    T->err = reinterpret_cast<unsigned int *>(p + tb + 12);
    MGS_CUDA_TRY(cudaMemsetAsync(p + tb, 0, 32, st));
    return MGS_OK;
}

// Reads the re-score count and the error flag (synchronises `st`).
static mgs_status tc_finish(mgs_ctx *ctx, const TcScratch &T, int64_t scores, cudaStream_t st) {
    unsigned long long h[2] = {0, 0};
    MGS_CUDA_TRY(cudaMemcpyAsync(h, T.stats, 16, cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->vq_scores += scores;
        ctx->vq_rescored += (int64_t)h[0];
    }
    if ((h[1] >> 32) & 1u) {   // err: the upper half of the second word
        set_error("vq: a tensor-core wait ran out; the outputs are incomplete");
        return MGS_ERR_TIMEOUT;
    }
    return MGS_OK;
}

extern "C" mgs_status mgs_vq_assign(mgs_ctx *ctx, const float *x, int64_t n, int32_t D,
                                    const float *codebook, int32_t K, int32_t *index_out,
                                    float *score_out, void *stream) {
    clear_error();
    if (!ctx || !index_out) {
        set_error("ctx and index_out must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    MGS_TRY(check_vq_args(x, n, D, codebook, K));
    DeviceGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ctx->vq_tensor) {
        void *base = nullptr;
        TcScratch T;
        MGS_TRY(tc_scratch(K, D, st, &base, &T));
        mgs_status s = vq_assign_tc(x, n, D, nullptr, codebook, K, index_out, score_out, T.tiles, T.cmax2,
                                    T.stats, T.err, ctx->vq_wait_cycles, st);
        if (s == MGS_OK) s = tc_finish(ctx, T, n * (int64_t)K, st);
        cudaFreeAsync(base, st);
        return s;
    }
    float *cc = nullptr;
    MGS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&cc), sizeof(float) * (size_t)K, st));
    k_vq_norms<<<(K + 255) / 256, 256, 0, st>>>(codebook, K, D, cc);
    count_launches(1);
    mgs_status s = MGS_OK;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("vq norms: %s", cudaGetErrorString(e));
        s = MGS_ERR_CUDA;
    }
    if (s == MGS_OK) s = assign_launch(x, n, D, nullptr, codebook, cc, K, index_out, score_out, st);
    cudaFreeAsync(cc, st);
    return s;
}

extern "C" mgs_status mgs_vq_set_wait_limit(mgs_ctx *ctx, int64_t cycles) {
    clear_error();
    if (!ctx || cycles < 0) {
        set_error("ctx must be non-NULL and cycles >= 0");
        return MGS_ERR_INVALID_ARG;
    }
    ctx->vq_wait_cycles = (long long)cycles;
    return MGS_OK;
}

extern "C" mgs_status mgs_vq_set_tensor_cores(mgs_ctx *ctx, int32_t enable) {
    clear_error();
    if (!ctx) {
        set_error("ctx must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    ctx->vq_tensor = enable ? 1 : 0;
    return MGS_OK;
}

extern "C" mgs_status mgs_vq_stats(mgs_ctx *ctx, int64_t *scores, int64_t *rescored) {
    clear_error();
    if (!ctx || !scores || !rescored) {
        set_error("ctx, scores and rescored must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    *scores = ctx->vq_scores;
    *rescored = ctx->vq_rescored;
    ctx->vq_scores = ctx->vq_rescored = 0;
    return MGS_OK;
}

extern "C" mgs_status mgs_vq_train(mgs_ctx *ctx, const float *x, int64_t n, int32_t D,
                                   float *codebook, int32_t K, int64_t *counts,
                                   const int32_t *batches, int32_t iters, int32_t batch,
                                   int32_t *assign_out, void *stream) {
    clear_error();
    if (!ctx || !counts || !batches || iters < 0 || batch < 0 || n < 1) {
        set_error("ctx, counts and batches must be non-NULL; iters, batch >= 0; n >= 1");
        return MGS_ERR_INVALID_ARG;
    }
    MGS_TRY(check_vq_args(x, n, D, codebook, K));
    if (!is_device_pointer(counts) || !is_device_pointer(batches)) {
        set_error("vq: counts and batches must be device memory");
        return MGS_ERR_INVALID_ARG;
    }
    if (K > kVqMaxTrainK) {
        set_error("vq train: K = %d exceeds %d", K, kVqMaxTrainK);
        return MGS_ERR_INVALID_ARG;
    }
    if (iters == 0 || batch == 0) return MGS_OK;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // every batch row must index x: checked on the device, one flag read back
    {
        unsigned int *bad = nullptr, hbad = 0;
        const int64_t tot = (int64_t)iters * batch;
        MGS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&bad), sizeof(unsigned int), st));
        cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), st);
        if (e == cudaSuccess) {
            k_vq_check_rows<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(batches, tot, n, bad);
            count_launches(1);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFreeAsync(bad, st);
        if (e != cudaSuccess) {
            set_error("vq: batch check: %s", cudaGetErrorString(e));
            return MGS_ERR_CUDA;
        }
        if (hbad) {
            set_error("vq: a batch entry is not a row of x");
            return MGS_ERR_INVALID_ARG;
        }
    }
    const size_t b_cc = 4 * (size_t)K, b_m = 4 * (size_t)K, b_off = 4 * (size_t)K,
                 b_cur = 4 * (size_t)K * (size_t)((batch + kVqChunk - 1) / kVqChunk),
                 b_a = 4 * (size_t)batch, b_perm = 4 * (size_t)batch;
    unsigned char *ws = nullptr;
    const size_t ws_bytes = b_cc + b_m + b_off + b_cur + b_a + b_perm + 64;
    if (cudaMallocAsync(reinterpret_cast<void **>(&ws), ws_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("vq workspace of %zu bytes", ws_bytes);
        return MGS_ERR_OUT_OF_MEMORY;
    }
    const int smem_k = (int)(sizeof(int32_t) * (size_t)K);
    if (smem_k > 48 * 1024) {
        cudaFuncSetAttribute(k_vq_chunk_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_k);
        cudaFuncSetAttribute(k_vq_chunk_place, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_k);
    }
    float *cc = reinterpret_cast<float *>(ws);
    int32_t *m = reinterpret_cast<int32_t *>(ws + b_cc);
    int32_t *off = m + K;
    int32_t *ccnt = off + K;
    int32_t *a_ws = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(ccnt) + b_cur);
    int32_t *perm = a_ws + batch;
    mgs_status s = MGS_OK;
    void *tc_base = nullptr;
    TcScratch T;
    if (ctx->vq_tensor) s = tc_scratch(K, D, st, &tc_base, &T);
    for (int t = 0; t < iters && s == MGS_OK; t++) {
        const int32_t *rows = batches + (int64_t)t * batch;
        int32_t *a = assign_out ? assign_out + (int64_t)t * batch : a_ws;
        if (ctx->vq_tensor) {
            s = vq_assign_tc(x, batch, D, rows, codebook, K, a, nullptr, T.tiles, T.cmax2, T.stats, T.err, ctx->vq_wait_cycles, st);
        } else {
            k_vq_norms<<<(K + 255) / 256, 256, 0, st>>>(codebook, K, D, cc);
            count_launches(1);
            s = assign_launch(x, batch, D, rows, codebook, cc, K, a, nullptr, st);
        }
        if (s != MGS_OK) break;
        cudaError_t e = cudaMemsetAsync(m, 0, b_m, st);
        if (e == cudaSuccess) {
            k_vq_count<<<(batch + 255) / 256, 256, 0, st>>>(a, batch, m);
            k_vq_scan<<<1, 1024, 0, st>>>(m, K, off);
            const unsigned nch = (unsigned)((batch + kVqChunk - 1) / kVqChunk);
            const size_t ks = sizeof(int32_t) * (size_t)K;
            k_vq_chunk_counts<<<nch, kVqChunk, ks, st>>>(a, batch, K, ccnt);
            k_vq_slots<<<(K + 31) / 32, 32 * kSlotWarps, 0, st>>>(ccnt, (int32_t)nch, off, K);
            k_vq_chunk_place<<<nch, kVqChunk, ks, st>>>(a, batch, K, ccnt, perm);
            const int64_t kd = (int64_t)K * D;
            k_vq_move<<<(unsigned)((kd + 255) / 256), 256, 0, st>>>(x, D, rows, perm, off, m, codebook,
                                                                      K, counts);
            k_vq_counts<<<(K + 255) / 256, 256, 0, st>>>(counts, m, K);
            count_launches(7);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            set_error("vq update: %s", cudaGetErrorString(e));
            s = MGS_ERR_CUDA;
        }
    }
    if (s == MGS_OK && ctx->vq_tensor) s = tc_finish(ctx, T, (int64_t)iters * batch * K, st);
    if (tc_base) cudaFreeAsync(tc_base, st);
    cudaFreeAsync(ws, st);
    return s;
}

extern "C" mgs_status mgs_vq_retain(mgs_ctx *ctx, const int32_t *rows, int64_t n_retain, int32_t K,
                                    int32_t *index, void *stream) {
    clear_error();
    if (!ctx || (n_retain > 0 && (!rows || !index)) || n_retain < 0 || K < 0 ||
        (int64_t)K + n_retain > ((int64_t)1 << 31) - 1) {
        set_error("vq retain: bad arguments");
        return MGS_ERR_INVALID_ARG;
    }
    if (n_retain == 0) return MGS_OK;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_vq_retain<<<(unsigned)((n_retain + 255) / 256), 256, 0, st>>>(rows, n_retain, K, index);
    count_launches(1);
    MGS_CUDA_TRY(cudaGetLastError());
    return MGS_OK;
}
