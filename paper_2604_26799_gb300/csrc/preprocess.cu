// Scene preprocessing: Sec. III-A's view-independent importance and Sec. III-D's
// quaternion -> Euler replacement, ahead of the cost tables.
//
//   k_pre_copy    channels 0..54 of [n][59] into [n][58] (one thread per output value)
//   k_pre_rows    per Gaussian: volume V = exp(s0 + s1 + s2) of the stored log-scales
//                 (FP32), Euler angles of the normalised quaternion [w, x, y, z] (FP64,
//                 rounded to FP32; channels 55..57 of the output), finiteness of the
//                 inputs it reads, and a histogram of V's top 16 bits (V >= 0, so its
//                 bits order like V)
//   k_pre_select  one CTA: the bucket holding the k-th smallest V, k = floor(9(n-1)/10)
//   k_pre_hist_lo histogram of the low 16 bits inside that bucket
//   (k_pre_select again: V_q exactly, the lower 0.9-quantile of the volumes)
//   k_pre_imp     I_g = I_d * min(V / V_q, 1)^beta (V_norm = 1 when V_q = 0)
#include <cuda_runtime.h>

#include <cmath>

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
};

__global__ void k_pre_copy(const float *__restrict__ in, float *__restrict__ out, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * kQuat0) return;
    const int64_t i = t / kQuat0;
    const int c = (int)(t - i * kQuat0);
    out[i * kOutC + c] = in[i * kInC + c];
}

__global__ void k_pre_rows(const float *__restrict__ in, const float *__restrict__ view_imp, int64_t n,
                           float *__restrict__ out, float *__restrict__ vol, unsigned int *__restrict__ hist,
                           PreState *st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *r = in + i * kInC;
    const float s0 = r[kScale0], s1 = r[kScale0 + 1], s2 = r[kScale0 + 2];
    double w = r[kQuat0], x = r[kQuat0 + 1], y = r[kQuat0 + 2], z = r[kQuat0 + 3];
    const bool finite = isfinite(s0) && isfinite(s1) && isfinite(s2) && isfinite(w) && isfinite(x) &&
                        isfinite(y) && isfinite(z) && isfinite(view_imp[i]);
    if (!finite) atomicOr(&st->nonfinite, 1u);
    const float v = finite ? expf(s0 + s1 + s2) : 0.0f;
    vol[i] = v;
    atomicAdd(&hist[__float_as_uint(v) >> 16], 1u);
    // The printed Euler formula is ill-conditioned near theta = +-pi/2 (through
    // sqrt(1 -+ 2t) and the small atan2 arguments of phi and psi), so it is
    // evaluated in FP64 and rounded once to FP32.
    double phi = 0.0, theta = 0.0, psi = 0.0;
    const double nrm = sqrt(w * w + x * x + y * y + z * z);
    if (finite && nrm > 0.0) {
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
    float *o = out + i * kOutC;
    o[kQuat0] = (float)phi;
    o[kQuat0 + 1] = (float)theta;
    o[kQuat0 + 2] = (float)psi;
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
    const size_t hist_bytes = sizeof(unsigned int) * kBins;
    char *ws = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&ws), vol_bytes + 2 * hist_bytes + 256, st) != cudaSuccess) {
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
    unsigned int *hist_hi = reinterpret_cast<unsigned int *>(ws + vol_bytes);
    unsigned int *hist_lo = hist_hi + kBins;
    PreState *pst = reinterpret_cast<PreState *>(ws + vol_bytes + 2 * hist_bytes);
    MGS_CUDA_TRY(cudaMemsetAsync(hist_hi, 0, 2 * hist_bytes + sizeof(PreState), st));
    const int64_t want = (9 * (n - 1)) / 10;
    k_pre_copy<<<blocks_for(n * kQuat0, 256), 256, 0, st>>>(attrs, attrs_out, n);
    k_pre_rows<<<blocks_for(n, 256), 256, 0, st>>>(attrs, view_importance, n, attrs_out, vol, hist_hi, pst);
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
