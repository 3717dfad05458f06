// Codes of one chosen configuration (Sec. III-D): for every (channel, group)
// of one kept set, the group min/max and the b-bit codes
//   q = rint(min(max(fl(fl(v / S) + Z), 0), 2^b - 1)),  S = fl((max - min) / 2^b),
//   Z = rint(fl(2^b - fl(max / S))).
// One CTA per (group, 8-channel slab): each kept row's 32-byte slab row is
// read twice (the group min/max of the 8 channels, then their codes; the
// second read hits L2), instead of once per channel.
#include <cuda_runtime.h>

#include <cfloat>

#include "internal.h"

namespace mgs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__global__ void __launch_bounds__(kThreads)
    k_quantize(const float *__restrict__ slabs, int64_t n, const int32_t *__restrict__ kept,
               int64_t keep, int32_t G, int32_t n_groups, int32_t C, const uint8_t *__restrict__ bits,
               uint16_t *__restrict__ codes, float *__restrict__ minmax) {
    __shared__ float red[2][kSlabWidth][kWarps];
    __shared__ float s_S[kSlabWidth], s_Z[kSlabWidth], s_top[kSlabWidth];
    const int g = blockIdx.x % n_groups;
    const int slab = blockIdx.x / n_groups;
    const int64_t start = (int64_t)g * G;
    const int nvalid = (int)((keep - start) < (int64_t)G ? (keep - start) : (int64_t)G);
    const float *base = slabs + (int64_t)slab * n * kSlabWidth;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float mn[kSlabWidth], mx[kSlabWidth];
#pragma unroll
    for (int c = 0; c < kSlabWidth; c++) {
        mn[c] = FLT_MAX;
        mx[c] = -FLT_MAX;
    }
    for (int i = threadIdx.x; i < nvalid; i += kThreads) {
        const int64_t row = kept ? (int64_t)__ldg(&kept[start + i]) : start + i;
        const float4 a = __ldg(reinterpret_cast<const float4 *>(base + row * kSlabWidth));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(base + row * kSlabWidth) + 1);
        const float v[kSlabWidth] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < kSlabWidth; c++) {
            mn[c] = fminf(mn[c], v[c]);
            mx[c] = fmaxf(mx[c], v[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < kSlabWidth; c++) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xFFFFFFFFu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xFFFFFFFFu, mx[c], o));
        }
        if (lane == 0) {
            red[0][c][warp] = mn[c];
            red[1][c][warp] = mx[c];
        }
    }
    __syncthreads();
    if (threadIdx.x < kSlabWidth) {
        const int cc = threadIdx.x, c = slab * kSlabWidth + cc;
        float m = red[0][cc][0], M = red[1][cc][0];
        for (int k = 1; k < kWarps; k++) {
            m = fminf(m, red[0][cc][k]);
            M = fmaxf(M, red[1][cc][k]);
        }
        float S = 0.0f, Z = 0.0f, top = 0.0f;
        if (c < C) {
            const int b = bits[(int64_t)c * n_groups + g];
            const float twob = (float)(1u << b);
            top = twob - 1.0f;
            const float R = __fsub_rn(M, m);
            S = __fdiv_rn(R, twob);
            if (S != 0.0f) Z = rintf(__fsub_rn(twob, __fdiv_rn(M, S)));
            minmax[((int64_t)c * n_groups + g) * 2] = m;
            minmax[((int64_t)c * n_groups + g) * 2 + 1] = M;
        }
        s_S[cc] = S;
        s_Z[cc] = Z;
        s_top[cc] = top;
    }
    __syncthreads();
    const int cend = C - slab * kSlabWidth < kSlabWidth ? C - slab * kSlabWidth : kSlabWidth;
    float S[kSlabWidth], Z[kSlabWidth], top[kSlabWidth];
#pragma unroll
    for (int c = 0; c < kSlabWidth; c++) {
        S[c] = s_S[c];
        Z[c] = s_Z[c];
        top[c] = s_top[c];
    }
    for (int i = threadIdx.x; i < nvalid; i += kThreads) {
        const int64_t row = kept ? (int64_t)__ldg(&kept[start + i]) : start + i;
        const float4 a = __ldg(reinterpret_cast<const float4 *>(base + row * kSlabWidth));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(base + row * kSlabWidth) + 1);
        const float v[kSlabWidth] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < kSlabWidth; c++) {
            if (c >= cend) break;
            uint16_t q = 0;
            if (S[c] != 0.0f) {
                const float x = __fadd_rn(__fdiv_rn(v[c], S[c]), Z[c]);
                q = (uint16_t)__float2int_rn(fminf(fmaxf(x, 0.0f), top[c]));
            }
            codes[(int64_t)(slab * kSlabWidth + c) * keep + start + i] = q;
        }
    }
}

}  // namespace

mgs_status quantize_launch(mgs_ctx *ctx, const mgs_scene *sc, const int32_t *kept, int64_t keep,
                           int32_t G, const uint8_t *bits, uint16_t *codes, float *minmax,
                           cudaStream_t st) {
    (void)ctx;
    int64_t ng = n_groups_of(keep, G);
    int64_t blocks = ng * sc->n_slabs;
    if (blocks == 0) return MGS_OK;
    k_quantize<<<(unsigned)blocks, kThreads, 0, st>>>(sc->d_slabs, sc->n, kept, keep, G, (int32_t)ng,
                                                       sc->C, bits, codes, minmax);
    count_launches(1);
    MGS_CUDA_TRY(cudaGetLastError());
    return MGS_OK;
}

}  // namespace mgs
