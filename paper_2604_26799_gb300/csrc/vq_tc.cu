// Nearest-codebook assignment of the SH vectors (Sec. III-D) on the tensor
// cores, with the same decisions as the exact FP32 scores.
//
// A score fl(|c|^2 - 2 x.c) is a dense contraction (vectors x codebook), so
// x.c is first computed approximately by tcgen05.mma (kind::tf32, FP32
// accumulators in tensor memory).  The approximation error of every score of
// vector x is bounded by a margin m(x) (inputs rounded to TF32 lose at most
// 2^-10 relative each, and |x.c| <= |x| max|c|); an entry can be the exact
// argmin only if its approximate score is within 2 m(x) of the smallest
// approximate score seen, so exactly those entries are re-scored with the
// FP32 fmaf chain of mgs_vq_assign (dimensions in ascending order), and the
// smallest exact score wins, ties to the lower index.  Entry 0 and any entry
// whose approximate score is NaN are always re-scored, so the result is the
// exact path's for every input.
//
// Per CTA: 128 vectors (the MMA's M, one TMEM lane each) against the
// codebook in tiles of 128 entries (N).  The codebook is laid out once by
// k_vq_tc_prep in the no-swizzle K-major core-matrix layout the MMA reads
// (8 rows x 16 bytes per core matrix, LBO = 128 B between core matrices
// along K, SBO = 32 DP bytes between 8-row groups), each tile followed by its
// 128 exact norms, so a tile is one bulk copy (cp.async.bulk, completion on
// an mbarrier) into the CTA's one tile buffer, refilled as soon as the four
// warps have read it; four CTAs per SM overlap one another's copies, MMAs and
// candidate tests.  One thread issues DP / 8 MMAs per
// tile and commits them to an mbarrier; the four warps read their 32 TMEM
// lanes with tcgen05.ld and run the candidate test.  Every wait is bounded:
// on expiry the CTA records an error flag, drains what it issued, frees its
// tensor memory and returns.
#include <cuda_runtime.h>

#include <cfloat>

#include "internal.h"

namespace mgs {
namespace {

constexpr int kTcM = 128;            // vectors per CTA (MMA M, TMEM lanes)
constexpr int kTcN = 128;            // codebook entries per tile (MMA N, TMEM columns)
constexpr int kTcThreads = 128;
constexpr int kTcBufs = 1;           // codebook tile buffers per CTA
constexpr int kTcCtasPerSm = 4;      // resident CTAs: 4 x 128 TMEM columns = all 512
constexpr long long kWaitCycles = 1ll << 31;    // ~1 s at 2 GHz: a wait that long is a failure
constexpr long long kDrainCycles = 1ll << 28;   // draining one's own copies and MMAs

__host__ __device__ constexpr int tile_bytes(int DP) { return kTcN * DP * 4; }
// tile: core matrices, then |c|^2 [128] and upper bounds of |c| [128]
__host__ __device__ constexpr int tile_stride(int DP) { return tile_bytes(DP) + 2 * kTcN * 4; }

// Byte offset of element (row r, column k) in a core-matrix tile.
__host__ __device__ inline int cm_offset(int r, int k, int DP) {
    return (r >> 3) * (32 * DP) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// try_wait suspends the thread until the phase completes or `ns` nanoseconds
// have passed, whichever comes first.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Whether the phase with the given parity has completed (does not wait).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity: false once `limit` clock
// cycles have passed, or at once when another CTA has raised *err (if err).
// The thread suspends (up to 1 us at a time) only while more than 4096 cycles
// of the limit remain; closer to the limit it polls, so that a limit of a few
// cycles runs out however fast a suspended wait would have been woken.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const unsigned int *err,
                                          long long limit) {
    const long long t0 = clock64();
    for (;;) {
        if (mbar_test_wait(bar, parity)) return true;
        if (err && *(const volatile unsigned int *)err) return false;
        const long long el = clock64() - t0;
        if (el > limit) return false;
        if (limit - el > 4096 && mbar_try_wait(bar, parity, 1000u)) return true;
    }
}
// One bulk copy global -> this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {   // one whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {   // the same warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// Shared-memory matrix descriptor: no swizzle, K-major core matrices.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture
    return d;
}
// Instruction descriptor: FP32 accumulators, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; j++) v[j] = __uint_as_float(r[j]);
}

// Exact score of vector row v of the A tile against entry kk of a codebook
// tile: the FP32 fmaf chain of the plain search (dimensions ascending), then
// |c|^2 - 2 x.c in one fmaf.
template <int DP>
__device__ __forceinline__ float exact_score(const unsigned char *sA, int v, const unsigned char *tileB,
                                             int kk, int D, const float *ccs) {
    float dot = 0.0f;
#pragma unroll
    for (int k4 = 0; k4 < DP / 4; k4++) {
        if (4 * k4 < D) {
            const float4 a = *reinterpret_cast<const float4 *>(sA + cm_offset(v, 4 * k4, DP));
            const float4 b = *reinterpret_cast<const float4 *>(tileB + cm_offset(kk, 4 * k4, DP));
            dot = __fmaf_rn(a.x, b.x, dot);
            if (4 * k4 + 1 < D) dot = __fmaf_rn(a.y, b.y, dot);
            if (4 * k4 + 2 < D) dot = __fmaf_rn(a.z, b.z, dot);
            if (4 * k4 + 3 < D) dot = __fmaf_rn(a.w, b.w, dot);
        }
    }
    return __fmaf_rn(-2.0f, dot, ccs[kk]);
}

// The codebook in MMA tiles: tile t holds entries 128 t .. 128 t + 127 in the
// core-matrix layout (zeros beyond K and beyond D), then their exact squared
// norms |c|^2 (the fmaf chain of the exact path), then upper bounds of their
// norms |c|.  *cmax2 gets max |c|^2 (as bits).
template <int DP>
__global__ void k_vq_tc_prep(const float *__restrict__ cb, int32_t K, int32_t D,
                             unsigned char *__restrict__ tiles, unsigned int *__restrict__ cmax2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // padded entry
    const int64_t ntiles = ((int64_t)K + kTcN - 1) / kTcN;
    if (e >= ntiles * kTcN) return;
    const int t = (int)(e / kTcN), r = (int)(e % kTcN);
    unsigned char *tile = tiles + (int64_t)t * tile_stride(DP);
    float cc = 0.0f;
#pragma unroll 4
    for (int k = 0; k < DP; k++) {
        float v = 0.0f;
        if (e < K && k < D) {
            v = cb[e * D + k];
            cc = __fmaf_rn(v, v, cc);
        }
        *reinterpret_cast<float *>(tile + cm_offset(r, k, DP)) = v;
    }
    float *tail = reinterpret_cast<float *>(tile + tile_bytes(DP));
    const float nr = sqrtf(cc) * 1.001f;
    tail[r] = cc;
    tail[kTcN + r] = nr;
    if (e < K) atomicMax(cmax2, __float_as_uint(cc));   // non-negative floats order as integers
}

template <int DP>
__global__ void __launch_bounds__(kTcThreads, kTcCtasPerSm)
    k_vq_assign_tc(const float *__restrict__ x, int64_t n, int32_t D, const int32_t *__restrict__ rows,
                   const unsigned char *__restrict__ tiles, int32_t K, const float *__restrict__ cb,
                   const unsigned int *__restrict__ cmax2, int32_t *__restrict__ idx_out,
                   float *__restrict__ score_out, unsigned long long *__restrict__ stats,
                   unsigned int *__restrict__ err, long long wait_cycles) {
    constexpr int TB = tile_bytes(DP), TS = tile_stride(DP);
    constexpr int SBO = 32 * DP, LBO = 128;
    constexpr uint32_t IDESC = idesc_tf32(kTcM, kTcN);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                 // TB bytes (the same layout, 128 vectors)
    unsigned char *sB = smem + TB;            // kTcBufs tile buffers of TS bytes
    __shared__ __align__(8) uint64_t bar_full[kTcBufs];
    __shared__ __align__(8) uint64_t bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int t = threadIdx.x, warp = t >> 5;
    const int64_t i = (int64_t)blockIdx.x * kTcM + t;
    const int ntiles = (K + kTcN - 1) / kTcN;

    // ---- this thread's vector: registers (for exact re-scores) and the A tile
    float xr[DP];
    const int64_t row = i < n ? (rows ? (int64_t)rows[i] : i) : -1;
#pragma unroll
    for (int d = 0; d < DP; d++) xr[d] = (row >= 0 && d < D) ? x[row * D + d] : 0.0f;
#pragma unroll
    for (int k4 = 0; k4 < DP / 4; k4++)
        *reinterpret_cast<float4 *>(sA + cm_offset(t, 4 * k4, DP)) =
            make_float4(xr[4 * k4], xr[4 * k4 + 1], xr[4 * k4 + 2], xr[4 * k4 + 3]);
    float xx = 0.0f;
#pragma unroll
    for (int d = 0; d < DP; d++) xx = __fmaf_rn(xr[d], xr[d], xx);
    // Error bound of entry k's approximate score: TF32 keeps 10 of the 23
    // fraction bits of each operand, so each product x_d c_d is off by less
    // than 2^-9 |x_d c_d|, the score by less than 2^-8 |x| |c_k|; with 5 %
    // allowance for the FP32 accumulation and rounding terms of both scores,
    // m_k = a |c_k|, a = 1.05 2^-8 |x| + 2^-21 |x| + 2^-22 max|c| (norms
    // rounded up).  Entry k can be the exact argmin only if
    // approx_k - m_k <= min_j (approx_j + m_j).
    const float cm2 = __uint_as_float(__ldg(cmax2));
    const float xn = sqrtf(xx) * 1.001f, cn = sqrtf(cm2) * 1.001f;
    const float am = xn * (0.00410156250f + 4.76837158e-7f) + 2.38418579e-7f * cn + 1e-30f;
    const bool rescore_all = !(am * cn < 1e30f);   // a non-finite bound: test every entry exactly

    if (warp == 0) tmem_alloc(&s_tmem, kTcN);
    if (t == 0) {
        for (int b = 0; b < kTcBufs; b++) mbar_init(&bar_full[b], 1);
        mbar_init(&bar_mma, 1);
        s_abort = 0;
    }
    fence_proxy_async();   // the A tile and the barriers, for the async proxy
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    int issued[kTcBufs] = {};   // bulk copies issued into each buffer (thread 0)
    if (t == 0) {
        for (int b = 0; b < kTcBufs && b < ntiles; b++) {
            mbar_expect_tx(&bar_full[b], TS);
            bulk_load(sB + b * TS, tiles + (int64_t)b * TS, TS, &bar_full[b]);
            issued[b]++;
        }
    }

    float best_up = FLT_MAX;   // min over the entries seen of approx + m
    float best_s = 0.0f;
    int best_k = -1;
    unsigned long long rescored = 0;
    int mma_pending = -1;   // tile whose MMAs thread 0 committed and nobody has waited for
    const uint32_t a_base = smem_u32(sA);

    for (int tt = 0; tt < ntiles; tt++) {
        const int buf = tt % kTcBufs;
        unsigned char *tileB = sB + buf * TS;
        if (!mbar_wait(&bar_full[buf], (uint32_t)((tt / kTcBufs) & 1), err, wait_cycles)) s_abort = 1;
        if (t == 0 && !s_abort) {
            tc_fence_after();
            const uint32_t b_base = smem_u32(tileB);
#pragma unroll
            for (int s = 0; s < DP / 8; s++)
                mma_tf32(tmem, smem_desc(a_base + 256 * s, LBO, SBO), smem_desc(b_base + 256 * s, LBO, SBO),
                         IDESC, s > 0 ? 1u : 0u);
            mma_commit(&bar_mma);
            mma_pending = tt;
        }
        __syncthreads();
        if (s_abort) break;
        if (!mbar_wait(&bar_mma, (uint32_t)(tt & 1), err, wait_cycles)) s_abort = 1;
        if (t == 0 && !s_abort) mma_pending = -1;
        __syncthreads();
        if (s_abort) break;
        tc_fence_after();

        // ---- candidates of this tile (this thread's vector = TMEM lane t).  A
        // chunk of 32 entries whose smallest approximate score is above the
        // threshold holds no candidate (with a finite margin every approximate
        // score is finite); the others are tested entry by entry and their
        // candidates re-scored exactly, in ascending k.
        const float *ccs = reinterpret_cast<const float *>(tileB + TB);
        const float *nrs = ccs + kTcN;
#pragma unroll 1
        for (int q = 0; q < kTcN / 32; q++) {
            float acc[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * 32), acc);
            const int k0 = tt * kTcN + q * 32;
            const float4 *cc4 = reinterpret_cast<const float4 *>(ccs + q * 32);
            const float4 *nr4 = reinterpret_cast<const float4 *>(nrs + q * 32);
            float ap[32], lo[32];
            float mlo = FLT_MAX;
#pragma unroll
            for (int j4 = 0; j4 < 8; j4++) {
                const float4 c = cc4[j4], nr = nr4[j4];
                const float cj[4] = {c.x, c.y, c.z, c.w}, nj[4] = {nr.x, nr.y, nr.z, nr.w};
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int j = 4 * j4 + u;
                    ap[j] = __fmaf_rn(-2.0f, acc[j], cj[u]);
                    lo[j] = __fmaf_rn(-am, nj[u], ap[j]);
                    mlo = fminf(mlo, lo[j]);
                }
            }
            // no entry of this chunk qualifies when its smallest lower bound exceeds
            // the threshold (with a finite margin every bound is finite)
            const bool whole = k0 + 32 <= K;
            if (whole && !rescore_all && mlo > best_up) continue;
#pragma unroll
            for (int j4 = 0; j4 < 8; j4++) {
                const float4 nr = nr4[j4];
                const float nj[4] = {nr.x, nr.y, nr.z, nr.w};
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int j = 4 * j4 + u;
                    if (k0 + j < K) best_up = fminf(best_up, __fmaf_rn(am, nj[u], ap[j]));
                }
            }
            uint32_t cand = 0;
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const bool c = k0 + j < K && (rescore_all || k0 + j == 0 || !(lo[j] > best_up));
                cand |= (uint32_t)c << j;
            }
            if (row < 0) cand = 0;
            while (cand) {
                const int j = __ffs(cand) - 1;
                cand &= cand - 1u;
                const float sc = exact_score<DP>(sA, t, tileB, q * 32 + j, D, ccs);
                if (best_k < 0 || sc < best_s) {
                    best_s = sc;
                    best_k = k0 + j;
                }
                rescored++;
            }
        }
        tc_fence_before();
        __syncthreads();   // every lane read the accumulators and the norms of this buffer
        if (t == 0 && tt + kTcBufs < ntiles) {
            mbar_expect_tx(&bar_full[buf], TS);
            bulk_load(tileB, tiles + (int64_t)(tt + kTcBufs) * TS, TS, &bar_full[buf]);
            issued[buf]++;
        }
    }

    if (s_abort) {
        if (t == 0) {
            atomicOr(err, 1u);
            // drain: the last MMA and every bulk copy issued but not consumed
            if (mma_pending >= 0) mbar_wait(&bar_mma, (uint32_t)(mma_pending & 1), nullptr, kDrainCycles);
            for (int b = 0; b < kTcBufs; b++)
                if (issued[b] > 0) mbar_wait(&bar_full[b], (uint32_t)((issued[b] - 1) & 1), nullptr, kDrainCycles);
        }
    } else if (row >= 0) {
        idx_out[i] = best_k;
        if (score_out) score_out[i] = best_s;
    }
    // statistics: re-scored entries, warp-aggregated
    unsigned long long r = rescored;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xFFFFFFFFu, r, o);
    if ((t & 31) == 0 && r) atomicAdd(stats, r);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTcN);
}

template <int DP>
mgs_status launch_tc(const float *x, int64_t n, int32_t D, const int32_t *rows, const float *cb,
                     int32_t K, int32_t *idx, float *score, unsigned char *tiles, unsigned int *cmax2,
                     unsigned long long *stats, unsigned int *err, long long wait_cycles, cudaStream_t st) {
    const int64_t ntiles = ((int64_t)K + kTcN - 1) / kTcN;
    MGS_CUDA_TRY(cudaMemsetAsync(cmax2, 0, sizeof(unsigned int), st));
    k_vq_tc_prep<DP><<<(unsigned)((ntiles * kTcN + 255) / 256), 256, 0, st>>>(cb, K, D, tiles, cmax2);
    // the A tile and the codebook buffers, padded with unused shared memory
    // until at most kTcCtasPerSm CTAs are resident, so that tcgen05.alloc
    // never has to wait for tensor-memory columns
    int dev = 0, optin = 0;
    MGS_CUDA_TRY(cudaGetDevice(&dev));
    MGS_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    MGS_CUDA_TRY(cudaFuncGetAttributes(&fa, k_vq_assign_tc<DP>));
    const size_t limit = (size_t)optin - fa.sharedSizeBytes;   // dynamic bytes a CTA may have
    const size_t need = (size_t)tile_bytes(DP) + (size_t)kTcBufs * tile_stride(DP);
    if (need > limit) {
        set_error("vq tensor path: %zu bytes of shared memory needed, %zu available", need, limit);
        return MGS_ERR_CUDA;
    }
    MGS_CUDA_TRY(cudaFuncSetAttribute(k_vq_assign_tc<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)limit));
    size_t smem = need;
    for (;;) {
        int resident = 0;
        MGS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_vq_assign_tc<DP>, kTcThreads,
                                                                   smem));
        if (resident <= kTcCtasPerSm || smem + 1024 > limit) break;
        smem += 1024;
    }
    const int64_t grid = (n + kTcM - 1) / kTcM;
    if (grid > 0)
        k_vq_assign_tc<DP><<<(unsigned)grid, kTcThreads, smem, st>>>(x, n, D, rows, tiles, K, cb, cmax2, idx,
                                                                     score, stats, err,
                                                                     wait_cycles > 0 ? wait_cycles : kWaitCycles);
    count_launches(grid > 0 ? 2 : 1);
    MGS_CUDA_TRY(cudaGetLastError());
    return MGS_OK;
}

}  // namespace

size_t vq_tc_workspace(int32_t K, int32_t D) {
    const int DP = D <= 16 ? 16 : D <= 32 ? 32 : D <= 48 ? 48 : 64;
    const int64_t ntiles = ((int64_t)K + kTcN - 1) / kTcN;
    return (size_t)(ntiles * tile_stride(DP));
}

mgs_status vq_assign_tc(const float *x, int64_t n, int32_t D, const int32_t *rows, const float *cb,
                        int32_t K, int32_t *idx, float *score, unsigned char *tiles, unsigned int *cmax2,
                        unsigned long long *stats, unsigned int *err, long long wait_cycles, cudaStream_t st) {
    if (D <= 16) return launch_tc<16>(x, n, D, rows, cb, K, idx, score, tiles, cmax2, stats, err, wait_cycles, st);
    if (D <= 32) return launch_tc<32>(x, n, D, rows, cb, K, idx, score, tiles, cmax2, stats, err, wait_cycles, st);
    if (D <= 48) return launch_tc<48>(x, n, D, rows, cb, K, idx, score, tiles, cmax2, stats, err, wait_cycles, st);
    return launch_tc<64>(x, n, D, rows, cb, K, idx, score, tiles, cmax2, stats, err, wait_cycles, st);
}

}  // namespace mgs
