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
// k_vq_assign: 128 threads x 1 or 2 vectors per thread in registers (the dimension
// padded with zeros to DP, a multiple of 8; adding 0 * 0 leaves an fmaf chain
// unchanged), codebook tiles of 64 centres staged in shared memory and read
// as float4 broadcasts.  The update is a one-warp stable counting sort of the
// batch by centre (match_any ranks, centre cursors in shared memory), then one
// thread per (centre, dimension) summing its vectors in batch order.
#include <cuda_runtime.h>

#include <cfloat>

#include "internal.h"

namespace mgs {
namespace {

constexpr int kVqThreads = 128;
constexpr int kVqTile = 64;     // centres per shared-memory tile
constexpr int kVqSmemCursors = 12288;   // centres whose sort cursors fit in shared memory
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

// One warp: stable counting sort of the batch by assigned centre.
// off[k] (exclusive scan of the counts) is read; perm[off[k] + r] = j for the
// r-th batch position j assigned to k, in batch order.  The cursors live in
// shared memory when K fits, else in `gcursor`; the next 32 centre ids are
// loaded while the current ones are placed.
template <bool SMEM>
__global__ void k_vq_perm(const int32_t *__restrict__ a, int32_t b, const int32_t *__restrict__ off,
                          int32_t K, int32_t *__restrict__ gcursor, int32_t *__restrict__ perm) {
    __shared__ int32_t s_cur[SMEM ? kVqSmemCursors : 1];
    int32_t *cursor = SMEM ? s_cur : gcursor;
    const int lane = threadIdx.x;
    for (int k = lane; k < K; k += 32) cursor[k] = 0;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    int next = lane < b ? a[lane] : -1 - lane;
    for (int j0 = 0; j0 < b; j0 += 32) {
        const int j = j0 + lane;
        const bool act = j < b;
        const int k = next;                     // inactive lanes hold distinct negatives
        next = j + 32 < b ? a[j + 32] : -1 - lane;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, k);
        int rank = 0, basec = 0;
        if (act) {
            rank = __popc(peers & lt);
            basec = cursor[k];
        }
        __syncwarp();
        if (act) {
            perm[off[k] + basec + rank] = j;
            if (rank == 0) cursor[k] = basec + __popc(peers);
        }
        __syncwarp();
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
    for (int r = 0; r < mk; r++) sum = __dadd_rn(sum, (double)x[(int64_t)rows[perm[o + r]] * D + d]);
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

// Two vectors per thread when there are enough CTAs to fill the GPU with
// them; one per thread (twice the CTAs) for batch-sized calls.
mgs_status assign_launch(const float *x, int64_t n, int32_t D, const int32_t *rows, const float *cb,
                         const float *cc, int32_t K, int32_t *idx, float *score, cudaStream_t st) {
    if (n == 0) return MGS_OK;
    const int P = n >= (int64_t)1 << 20 ? 2 : 1;
    const int64_t per_cta = (int64_t)kVqThreads * P;
    const int64_t grid = (n + per_cta - 1) / per_cta;
    AssignFn f = P == 2 ? pick_assign<2>(D) : pick_assign<1>(D);
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
                 b_cur = 4 * (size_t)K, b_a = 4 * (size_t)batch, b_perm = 4 * (size_t)batch;
    unsigned char *ws = nullptr;
    const size_t ws_bytes = b_cc + b_m + b_off + b_cur + b_a + b_perm + 64;
    if (cudaMallocAsync(reinterpret_cast<void **>(&ws), ws_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("vq workspace of %zu bytes", ws_bytes);
        return MGS_ERR_OUT_OF_MEMORY;
    }
    float *cc = reinterpret_cast<float *>(ws);
    int32_t *m = reinterpret_cast<int32_t *>(ws + b_cc);
    int32_t *off = m + K;
    int32_t *cur = off + K;
    int32_t *a_ws = cur + K;
    int32_t *perm = a_ws + batch;
    mgs_status s = MGS_OK;
    for (int t = 0; t < iters && s == MGS_OK; t++) {
        const int32_t *rows = batches + (int64_t)t * batch;
        int32_t *a = assign_out ? assign_out + (int64_t)t * batch : a_ws;
        k_vq_norms<<<(K + 255) / 256, 256, 0, st>>>(codebook, K, D, cc);
        count_launches(1);
        s = assign_launch(x, batch, D, rows, codebook, cc, K, a, nullptr, st);
        if (s != MGS_OK) break;
        cudaError_t e = cudaMemsetAsync(m, 0, b_m, st);
        if (e == cudaSuccess) {
            k_vq_count<<<(batch + 255) / 256, 256, 0, st>>>(a, batch, m);
            k_vq_scan<<<1, 1024, 0, st>>>(m, K, off);
            if (K <= kVqSmemCursors)
                k_vq_perm<true><<<1, 32, 0, st>>>(a, batch, off, K, cur, perm);
            else
                k_vq_perm<false><<<1, 32, 0, st>>>(a, batch, off, K, cur, perm);
            const int64_t kd = (int64_t)K * D;
            k_vq_move<<<(unsigned)((kd + 255) / 256), 256, 0, st>>>(x, D, rows, perm, off, m, codebook,
                                                                      K, counts);
            k_vq_counts<<<(K + 255) / 256, 256, 0, st>>>(counts, m, K);
            count_launches(5);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            set_error("vq update: %s", cudaGetErrorString(e));
            s = MGS_ERR_CUDA;
        }
    }
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
