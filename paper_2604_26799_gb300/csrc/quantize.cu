// Codes of one chosen configuration (Sec. III-D): for every (channel, group)
// of one kept set, the group min/max and the b-bit codes
//   q = rint(min(max(fl(fl(v / S) + Z), 0), 2^b - 1)),  S = fl((max - min) / 2^b),
//   Z = rint(fl(2^b - fl(max / S))).
// One CTA per (group, channel); the group's values are staged in shared memory.
#include <cuda_runtime.h>

#include <cfloat>

#include "internal.h"

namespace mgs {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
    k_quantize(const float *__restrict__ slabs, int64_t n, const int32_t *__restrict__ kept,
               int64_t keep, int32_t G, int32_t n_groups, const uint8_t *__restrict__ bits,
               uint16_t *__restrict__ codes, float *__restrict__ minmax) {
    extern __shared__ float vals[];
    __shared__ float red[2][kThreads / 32];
    const int g = blockIdx.x % n_groups;
    const int c = blockIdx.x / n_groups;
    const int64_t start = (int64_t)g * G;
    const int nvalid = (int)((keep - start) < (int64_t)G ? (keep - start) : (int64_t)G);
    const float *base = slabs + (int64_t)(c / kSlabWidth) * n * kSlabWidth + (c % kSlabWidth);
    float mn = FLT_MAX, mx = -FLT_MAX;
    for (int i = threadIdx.x; i < nvalid; i += kThreads) {
        float v = __ldg(base + (int64_t)__ldg(&kept[start + i]) * kSlabWidth);
        vals[i] = v;
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = mn;
        red[1][threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    float m = red[0][0], M = red[1][0];
    for (int k = 1; k < kThreads / 32; k++) {
        m = fminf(m, red[0][k]);
        M = fmaxf(M, red[1][k]);
    }
    const int b = bits[(int64_t)c * n_groups + g];
    const float twob = (float)(1u << b);
    const float top = twob - 1.0f;
    const float R = __fsub_rn(M, m);
    const float S = __fdiv_rn(R, twob);
    uint16_t *out = codes + (int64_t)c * keep + start;
    if (threadIdx.x == 0) {
        minmax[((int64_t)c * n_groups + g) * 2] = m;
        minmax[((int64_t)c * n_groups + g) * 2 + 1] = M;
    }
    if (S == 0.0f) {
        for (int i = threadIdx.x; i < nvalid; i += kThreads) out[i] = 0;
        return;
    }
    const float Z = rintf(__fsub_rn(twob, __fdiv_rn(M, S)));
    for (int i = threadIdx.x; i < nvalid; i += kThreads) {
        float x = __fadd_rn(__fdiv_rn(vals[i], S), Z);
        float xc = fminf(fmaxf(x, 0.0f), top);
        out[i] = (uint16_t)__float2int_rn(xc);
    }
}

}  // namespace

mgs_status quantize_launch(mgs_ctx *ctx, const mgs_scene *sc, const int32_t *kept, int64_t keep,
                           int32_t G, const uint8_t *bits, uint16_t *codes, float *minmax,
                           cudaStream_t st) {
    (void)ctx;
    int64_t ng = n_groups_of(keep, G);
    int64_t blocks = ng * sc->C;
    if (blocks == 0) return MGS_OK;
    size_t smem = sizeof(float) * (size_t)G;
    MGS_CUDA_TRY(cudaFuncSetAttribute(k_quantize, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_quantize<<<(unsigned)blocks, kThreads, smem, st>>>(sc->d_slabs, sc->n, kept, keep, G,
                                                          (int32_t)ng, bits, codes, minmax);
    count_launches(1);
    MGS_CUDA_TRY(cudaGetLastError());
    return MGS_OK;
}

}  // namespace mgs
