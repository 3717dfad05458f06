// Scene preprocessing: Sec. III-A's view-independent importance and Sec. III-D's
// quaternion -> Euler replacement, ahead of the cost tables.
//
//   k_pre_tile    128 rows per CTA staged in shared memory: channels 0..54 copied
//                 into [n][58]; per row the volume V = exp(s0 + s1 + s2) of the stored
//                 log-scales (FP32), the finiteness of the inputs it reads, a count
//                 histogram of V's top 16 bits (V >= 0, so its bits order like V), and
//                 the Euler angles of the normalised quaternion [w, x, y, z] (channels
//                 55..57) in FP32 where |sin(theta)| <= 0.95
//   k_pre_euler64 the other rows' angles in FP64 (the printed formula is
//                 ill-conditioned near theta = +-pi/2), rounded once to FP32
//   k_pre_select  one CTA: the bucket holding the k-th smallest V, k = floor(9(n-1)/10)
//   k_pre_hist_lo histogram of the low 16 bits inside that bucket
//   (k_pre_select again: V_q exactly, the lower 0.9-quantile of the volumes)
//   k_pre_imp     I_g = I_d * min(V / V_q, 1)^beta (V_norm = 1 when V_q = 0)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace mgs {
namespace {

constexpr int kInC = 59, kOutC = 58, kScale0 = 52, kQuat0 = 55;
constexpr int kBins = 1 << 16;
constexpr int kSelThreads = 1024;

struct PreState {
    unsigned int nonfinite;   // an input the preprocessing reads is NaN or infinite
    unsigned int bucket;      // top 16 bits of V_q (after the first selection)
    unsigned int rank_left;   // rank of V_q inside that bucket
    float vq;                 // the normaliser
    unsigned int n_slow;      // rows whose Euler angles are redone in FP64
};

constexpr int kTileRows = 128, kTileThreads = 128;   // one row per thread
// |sin(theta)| above which the FP32 evaluation of the printed formula loses
// accuracy (cos(theta) < 0.31): those rows are redone in FP64
constexpr float kSlowSin = 0.95f;

// Euler angles of one quaternion in FP64 (the printed formula, rounded once).
__device__ void euler64(double w, double x, double y, double z, float *e) {
    double phi = 0.0, theta = 0.0, psi = 0.0;
    const double nrm = sqrt(w * w + x * x + y * y + z * z);
    if (nrm > 0.0) {
        w /= nrm;
        x /= nrm;
        y /= nrm;
        z /= nrm;
        phi = atan2(2.0 * (w * x + y * z), 1.0 - 2.0 * (x * x + y * y));
        const double t = w * y - x * z;
        const double a = fmax(1.0 + 2.0 * t, 0.0), b = fmax(1.0 - 2.0 * t, 0.0);
        theta = -1.5707963267948966 + 2.0 * atan2(sqrt(a), sqrt(b));
        psi = atan2(2.0 * (w * z + x * y), 1.0 - 2.0 * (y * y + z * z));
    }
    e[0] = (float)phi;
    e[1] = (float)theta;
    e[2] = (float)psi;
}

// 128 rows per CTA: the [128][59] input tile is staged in shared memory
// (16-byte loads when the arrays are 16-byte aligned), one thread per row does
// the per-row work, and the [128][58] output tile is written back (16-byte
// stores).
template <bool VEC>
__global__ void __launch_bounds__(kTileThreads) k_pre_tile(const float *__restrict__ in,
                                                           const float *__restrict__ view_imp, int64_t n,
                                                           float *__restrict__ out, float *__restrict__ vol,
                                                           unsigned int *__restrict__ hist, PreState *st,
                                                           int64_t *__restrict__ slow, unsigned int *n_slow) {
    __shared__ __align__(16) float s_in[kTileRows * kInC];
    __shared__ float s_e[kTileRows][3];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kTileRows;
    const int rows = (int)(n - r0 < kTileRows ? n - r0 : kTileRows);
    const float *src = in + r0 * kInC;
    if (VEC && rows == kTileRows) {
        for (int j = tid; j < kTileRows * kInC / 4; j += kTileThreads)
            reinterpret_cast<float4 *>(s_in)[j] = __ldg(reinterpret_cast<const float4 *>(src) + j);
    } else {
        for (int j = tid; j < rows * kInC; j += kTileThreads) s_in[j] = __ldg(src + j);
    }
    __syncthreads();
    if (tid < rows) {
        const int64_t i = r0 + tid;
        const float *r = s_in + tid * kInC;
        const float s0 = r[kScale0], s1 = r[kScale0 + 1], s2 = r[kScale0 + 2];
        float w = r[kQuat0], x = r[kQuat0 + 1], y = r[kQuat0 + 2], z = r[kQuat0 + 3];
        const bool finite = isfinite(s0) && isfinite(s1) && isfinite(s2) && isfinite(w) && isfinite(x) &&
                            isfinite(y) && isfinite(z) && isfinite(view_imp[i]);
        if (!finite) atomicOr(&st->nonfinite, 1u);
        const float v = finite ? expf(s0 + s1 + s2) : 0.0f;
        vol[i] = v;
        // one atomic per distinct bucket in the warp (volumes cluster in few buckets)
        const unsigned int bucket = __float_as_uint(v) >> 16;
        const unsigned int peers = __match_any_sync(__activemask(), bucket);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bucket], (unsigned int)__popc(peers));
        float phi = 0.0f, theta = 0.0f, psi = 0.0f;
        const float nrm = sqrtf(w * w + x * x + y * y + z * z);
        if (finite && nrm > 0.0f) {
            w /= nrm;
            x /= nrm;
            y /= nrm;
            z /= nrm;
            const float t = w * y - x * z;
            if (fabsf(2.0f * t) > kSlowSin) {
                slow[atomicAdd(n_slow, 1u)] = i;   // redone in FP64 by k_pre_euler64
            } else {
                phi = atan2f(2.0f * (w * x + y * z), 1.0f - 2.0f * (x * x + y * y));
                theta = -1.57079632679489662f + 2.0f * atan2f(sqrtf(1.0f + 2.0f * t), sqrtf(1.0f - 2.0f * t));
                psi = atan2f(2.0f * (w * z + x * y), 1.0f - 2.0f * (y * y + z * z));
            }
        }
        s_e[tid][0] = phi;
        s_e[tid][1] = theta;
        s_e[tid][2] = psi;
    }
    __syncthreads();
    float *dst = out + r0 * kOutC;
    auto value = [&](int idx) {
        const int rr = idx / kOutC, c = idx - rr * kOutC;
        return c < kQuat0 ? s_in[rr * kInC + c] : s_e[rr][c - kQuat0];
    };
    if (VEC && rows == kTileRows) {
        for (int j = tid; j < kTileRows * kOutC / 4; j += kTileThreads)
            reinterpret_cast<float4 *>(dst)[j] =
                make_float4(value(4 * j), value(4 * j + 1), value(4 * j + 2), value(4 * j + 3));
    } else {
        for (int j = tid; j < rows * kOutC; j += kTileThreads) dst[j] = value(j);
    }
}

// The rows near gimbal lock, in FP64.
__global__ void k_pre_euler64(const float *__restrict__ in, const int64_t *__restrict__ slow,
                              const unsigned int *n_slow, float *__restrict__ out) {
    const unsigned int m = *n_slow;
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const int64_t i = slow[k];
        const float *r = in + i * kInC;
        float e[3];
        euler64(r[kQuat0], r[kQuat0 + 1], r[kQuat0 + 2], r[kQuat0 + 3], e);
        out[i * kOutC + kQuat0] = e[0];
        out[i * kOutC + kQuat0 + 1] = e[1];
        out[i * kOutC + kQuat0 + 2] = e[2];
    }
}

// One CTA: the bucket of a 2^16-bin count histogram holding the element of
// rank `want` (0-based, ascending).  Thread t owns 64 consecutive buckets.
__global__ void __launch_bounds__(kSelThreads) k_pre_select(const unsigned int *__restrict__ hist,
                                                            int64_t want_in, PreState *st, int stage) {
    __shared__ unsigned long long s_warp[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long want = stage == 0 ? want_in : (long long)st->rank_left;
    constexpr int per = kBins / kSelThreads;
    unsigned long long sum = 0;
    for (int j = 0; j < per; j++) sum += hist[tid * per + j];
    unsigned long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned long long v = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if (lane >= o) v += u;
        }
        s_warp[lane] = v;
    }
    __syncthreads();
    const unsigned long long before = (wid > 0 ? s_warp[wid - 1] : 0ull) + incl - sum;
    if ((long long)before <= want && want < (long long)(before + sum)) {
        unsigned long long c = before;
        for (int j = 0; j < per; j++) {
            const unsigned int h = hist[tid * per + j];
            if ((long long)(c + h) > want) {
                if (stage == 0) {
                    st->bucket = (unsigned int)(tid * per + j);
                    st->rank_left = (unsigned int)(want - (long long)c);
                } else {
                    st->vq = __uint_as_float((st->bucket << 16) | (unsigned int)(tid * per + j));
                }
                break;
            }
            c += h;
        }
    }
}

__global__ void k_pre_hist_lo(const float *__restrict__ vol, int64_t n, const PreState *st,
                              unsigned int *__restrict__ hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned int b = __float_as_uint(vol[i]);
    if ((b >> 16) == st->bucket) atomicAdd(&hist[b & 0xFFFFu], 1u);
}

__global__ void k_pre_imp(const float *__restrict__ vol, const float *__restrict__ view_imp, int64_t n,
                          float beta, const PreState *st, float *__restrict__ imp_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float vq = st->vq;
    const float vn = vq > 0.0f ? fminf(vol[i] / vq, 1.0f) : 1.0f;
    imp_out[i] = view_imp[i] * powf(vn, beta);
}

unsigned int blocks_for(int64_t work, int threads) { return (unsigned int)((work + threads - 1) / threads); }

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" mgs_status mgs_preprocess(mgs_ctx *ctx, const float *attrs, const float *view_importance,
                                     int64_t n, double beta, float *attrs_out, float *importance_out,
                                     float *vq_out, void *stream) {
    clear_error();
    if (!ctx || !attrs || !view_importance || !attrs_out || !importance_out || n < 1) {
        set_error("ctx, attrs, view_importance, attrs_out and importance_out must be non-NULL; n >= 1");
        return MGS_ERR_INVALID_ARG;
    }
    if (!(beta >= 0.0) || !std::isfinite(beta)) {
        set_error("beta = %g: the exponent must be finite and >= 0", beta);
        return MGS_ERR_INVALID_ARG;
    }
    if (n > (int64_t)1 << 32) {
        set_error("n = %lld Gaussians exceeds 2^32", (long long)n);
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t vol_bytes = (sizeof(float) * (size_t)n + 255) & ~(size_t)255;
    const size_t slow_bytes = (sizeof(int64_t) * (size_t)n + 255) & ~(size_t)255;
    const size_t hist_bytes = sizeof(unsigned int) * kBins;
    char *ws = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&ws), vol_bytes + slow_bytes + 2 * hist_bytes + 256, st) !=
        cudaSuccess) {
        cudaGetLastError();
        set_error("preprocessing workspace of %zu bytes could not be allocated", vol_bytes + 2 * hist_bytes);
        return MGS_ERR_OUT_OF_MEMORY;
    }
    struct Free {
        char *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } free_ws{ws, st};
    float *vol = reinterpret_cast<float *>(ws);
    int64_t *slow = reinterpret_cast<int64_t *>(ws + vol_bytes);
    unsigned int *hist_hi = reinterpret_cast<unsigned int *>(ws + vol_bytes + slow_bytes);
    unsigned int *hist_lo = hist_hi + kBins;
    PreState *pst = reinterpret_cast<PreState *>(ws + vol_bytes + slow_bytes + 2 * hist_bytes);
    unsigned int *n_slow = &pst->n_slow;
    MGS_CUDA_TRY(cudaMemsetAsync(hist_hi, 0, 2 * hist_bytes + sizeof(PreState), st));
    const int64_t want = (9 * (n - 1)) / 10;
    const bool vec = (reinterpret_cast<uintptr_t>(attrs) % 16 == 0) && (reinterpret_cast<uintptr_t>(attrs_out) % 16 == 0);
    const unsigned int tiles = blocks_for(n, kTileRows);
    if (vec)
        k_pre_tile<true><<<tiles, kTileThreads, 0, st>>>(attrs, view_importance, n, attrs_out, vol, hist_hi, pst,
                                                          slow, n_slow);
    else
        k_pre_tile<false><<<tiles, kTileThreads, 0, st>>>(attrs, view_importance, n, attrs_out, vol, hist_hi, pst,
                                                           slow, n_slow);
    const unsigned int slow_blocks = (unsigned int)std::min<int64_t>((int64_t)ctx->sm_count * 4, blocks_for(n, 256));
    k_pre_euler64<<<slow_blocks, 256, 0, st>>>(attrs, slow, n_slow, attrs_out);
    k_pre_select<<<1, kSelThreads, 0, st>>>(hist_hi, want, pst, 0);
    k_pre_hist_lo<<<blocks_for(n, 256), 256, 0, st>>>(vol, n, pst, hist_lo);
    k_pre_select<<<1, kSelThreads, 0, st>>>(hist_lo, 0, pst, 1);
    k_pre_imp<<<blocks_for(n, 256), 256, 0, st>>>(vol, view_importance, n, (float)beta, pst, importance_out);
    MGS_CUDA_TRY(cudaGetLastError());
    count_launches(6);
    PreState h{};
    MGS_CUDA_TRY(cudaMemcpyAsync(&h, pst, sizeof(PreState), cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.nonfinite) {
        set_error("a log-scale, quaternion or view-dependent importance value is NaN or infinite");
        return MGS_ERR_NONFINITE;
    }
    if (vq_out) *vq_out = h.vq;
    return MGS_OK;
}
