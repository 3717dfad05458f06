// RAHT (Sec. III-D "Region Adaptive Hierarchical Transform") of a resident
// scene's channels at octree depth d.
//
//   k_rh_heads   voxel code of every Morton position (Morton code >> 3(21 - d))
//                and a flag where a new voxel starts
//   scan         voxel index of every position (exclusive prefix sum)
//   k_rh_starts  first Morton position and code of every voxel
//   k_rh_means   one thread per voxel: mean of its Gaussians, summed in
//                Morton order (weight 1)
//   per step s = 0 .. 3d - 1 (the node count, the AC offset, the current list
//   and the pending level live in device memory; the host reads them once per
//   octree level to size the grids):
//     k_rh_scan_pairs  flag i when nodes i, i + 1 agree above bit 1 of their
//                 codes, fused with the block-local scan; k_scan_sums: the block
//                 offsets and the number of pairs
//     k_rh_merge  the parent list (code >> 1, slot): a pair merges in place into
//                 the lower node's slot by the printed T, with its entries
//                 t1 = sqrt(w1) / sqrt(w1 + w2), t2 = sqrt(w2) / sqrt(w1 + w2) formed
//                 once per pair: DC = t1 x1 + t2 x2, weight w1 + w2, and it emits
//                 AC = t1 x2 - t2 x1 at the next AC slot; an unpaired node moves up.
//                 Attribute vectors stay in their voxel slots: only pairs touch them.
//     k_rh_advance  node count -= pairs, AC offset += pairs, swap the lists; a
//                 step without pairs only raises the pending level
// FP32 arithmetic with integer weights.  (An FP64 version matched the FP64
// oracle bit for bit, but GB300's FP64 pipe ran 73-87% busy and bounded it:
// 11.4 ms for 5.27 M voxels.)  Every merge is an orthonormal rotation, so the
// FP32 error of a coefficient stays within a few ulp per level of the size
// sqrt(w) * |x| of the node it comes from.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace mgs {
namespace {

constexpr int kScanBlock = 1024;
constexpr int kMaxRahtChannels = 64;

// t runs over the transformed Gaussians in Morton order: Morton position
// pos[t] (the kept list), or t itself when pos is NULL.
__global__ void k_rh_heads(const uint64_t *__restrict__ codes, const int32_t *__restrict__ order,
                           const int32_t *__restrict__ pos, int64_t K, int shift, uint64_t *__restrict__ vcode,
                           unsigned int *__restrict__ head) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    const int64_t p = pos ? pos[t] : t;
    const uint64_t v = codes[order[p]] >> shift;
    vcode[t] = v;
    head[t] = (t == 0 || (codes[order[pos ? pos[t - 1] : t - 1]] >> shift) != v) ? 1u : 0u;
}

// ---- exclusive scan of n uint32 flags (three phases) ----
__global__ void __launch_bounds__(kScanBlock) k_scan_local(const unsigned int *__restrict__ in, int64_t n,
                                                           unsigned int *__restrict__ out,
                                                           unsigned int *__restrict__ block_sum) {
    __shared__ unsigned int s_w[32];
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const unsigned int v = i < n ? in[i] : 0u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned int y = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, y, o);
            if (lane >= o) y += t;
        }
        s_w[lane] = y;
    }
    __syncthreads();
    const unsigned int incl = x + (wid > 0 ? s_w[wid - 1] : 0u);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == kScanBlock - 1) block_sum[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_sums(unsigned int *__restrict__ block_sum, int64_t nb,
                                                          unsigned long long *__restrict__ total) {
    __shared__ unsigned int s_w[32];
    __shared__ unsigned int s_carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const unsigned int v = i < nb ? block_sum[i] : 0u;
        unsigned int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned int y = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, y, o);
                if (lane >= o) y += t;
            }
            s_w[lane] = y;
        }
        __syncthreads();
        const unsigned int incl = x + (wid > 0 ? s_w[wid - 1] : 0u);
        const unsigned int carry = s_carry;
        if (i < nb) block_sum[i] = carry + incl - v;   // exclusive offset of block i
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) s_carry = carry + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s_carry;
}

__global__ void k_scan_add(unsigned int *__restrict__ out, int64_t n, const unsigned int *__restrict__ block_off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += block_off[i / kScanBlock];
}

__global__ void k_rh_starts(const unsigned int *__restrict__ head, const unsigned int *__restrict__ vidx,
                            const uint64_t *__restrict__ vcode, int64_t n, int64_t *__restrict__ start,
                            uint64_t *__restrict__ key) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !head[p]) return;
    start[vidx[p]] = p;
    key[vidx[p]] = vcode[p];
}

__global__ void k_rh_means(const float *__restrict__ slabs, int64_t n, const int32_t *__restrict__ pos,
                           int64_t K, const int64_t *__restrict__ start, int64_t V,
                           const int32_t *__restrict__ chan, int n_c, float *__restrict__ x,
                           unsigned int *__restrict__ w) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int64_t t0 = start[v], t1 = v + 1 < V ? start[v + 1] : K;
    for (int k = 0; k < n_c; k++) {
        const int c = chan[k];
        const float *col = slabs + (int64_t)(c / kSlabWidth) * n * kSlabWidth + (c % kSlabWidth);
        float sum = 0.0f;
        for (int64_t t = t0; t < t1; t++) sum = __fadd_rn(sum, col[(int64_t)(pos ? pos[t] : t) * kSlabWidth]);
        x[v * n_c + k] = t1 - t0 > 1 ? __fdiv_rn(sum, (float)(t1 - t0)) : sum;
    }
    w[v] = 1u;
}

struct RahtState {
    long long m;         // nodes in the current list
    long long ac_base;   // ACs emitted so far
    int cur;             // which of the two lists is current
    int pending;         // levels not yet applied to the current list's codes
};

// Steps whose list has no pair change nothing but the level: they only raise
// `pending`, and the codes are compared (and shifted when the list is next
// rewritten) by pending + 1 bits.
// Pair flags of the current list fused with the block-local exclusive scan
// (the flags are recomputed from the codes by k_rh_merge; no flag array).
__device__ __forceinline__ unsigned int pair_flag(const uint64_t *key, int64_t i, int64_t m, int sh) {
    return (i + 1 < m && (key[i] >> sh) == (key[i + 1] >> sh)) ? 1u : 0u;
}

__global__ void __launch_bounds__(kScanBlock) k_rh_scan_pairs(const uint64_t *__restrict__ key0,
                                                              const uint64_t *__restrict__ key1,
                                                              const RahtState *st, int64_t cap,
                                                              unsigned int *__restrict__ out,
                                                              unsigned int *__restrict__ block_sum) {
    __shared__ unsigned int s_w[32];
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const int64_t m = st->m;
    const uint64_t *key = st->cur ? key1 : key0;
    const unsigned int v = i < cap ? pair_flag(key, i, m, st->pending + 1) : 0u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned int y = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, y, o);
            if (lane >= o) y += t;
        }
        s_w[lane] = y;
    }
    __syncthreads();
    const unsigned int incl = x + (wid > 0 ? s_w[wid - 1] : 0u);
    if (i < cap) out[i] = incl - v;
    if (threadIdx.x == kScanBlock - 1) block_sum[blockIdx.x] = incl;
}

__global__ void k_rh_merge(uint64_t *__restrict__ key0, uint64_t *__restrict__ key1,
                           unsigned int *__restrict__ slot0, unsigned int *__restrict__ slot1,
                           const RahtState *st, const unsigned long long *pairs, int n_c,
                           const unsigned int *__restrict__ local, const unsigned int *__restrict__ block_off,
                           float *__restrict__ x, unsigned int *__restrict__ w, float *__restrict__ ac) {
    if (*pairs == 0) return;   // nothing to merge at this level
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = st->m;
    if (i >= m) return;
    const int sh = st->pending + 1;
    const uint64_t *kc = st->cur ? key1 : key0;
    if (i > 0 && pair_flag(kc, i - 1, m, sh)) return;   // the upper node of a pair: merged by its partner
    const unsigned int pf_i = pair_flag(kc, i, m, sh);
    const unsigned int pidx_i = local[i] + block_off[i / kScanBlock];
    const bool c = st->cur;
    const uint64_t *key = c ? key1 : key0;
    const unsigned int *slot = c ? slot1 : slot0;
    uint64_t *key2 = c ? key0 : key1;
    unsigned int *slot2 = c ? slot0 : slot1;
    const int64_t j = i - (int64_t)pidx_i;
    key2[j] = key[i] >> sh;
    const unsigned int sa = slot[i];
    slot2[j] = sa;
    if (!pf_i) return;
    const unsigned int sb = slot[i + 1];
    const unsigned int wa = w[sa], wb = w[sb];
    // the entries of T, once per pair
    const float sw = __fsqrt_rn((float)(wa + wb));
    const float t1 = __fdiv_rn(__fsqrt_rn((float)wa), sw), t2 = __fdiv_rn(__fsqrt_rn((float)wb), sw);
    const int64_t out = st->ac_base + (int64_t)pidx_i;
    float *xa = x + (int64_t)sa * n_c;
    const float *xbp = x + (int64_t)sb * n_c;
    float *acp = ac + out * n_c;
    int k = 0;
    for (; k + 4 <= n_c; k += 4) {   // four channels at a time: independent loads in flight
        float x1[4], x2[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            x1[u] = xa[k + u];
            x2[u] = xbp[k + u];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            xa[k + u] = __fadd_rn(__fmul_rn(t1, x1[u]), __fmul_rn(t2, x2[u]));
            acp[k + u] = __fsub_rn(__fmul_rn(t1, x2[u]), __fmul_rn(t2, x1[u]));
        }
    }
    for (; k < n_c; k++) {
        const float x1 = xa[k], x2 = xbp[k];
        xa[k] = __fadd_rn(__fmul_rn(t1, x1), __fmul_rn(t2, x2));
        acp[k] = __fsub_rn(__fmul_rn(t1, x2), __fmul_rn(t2, x1));
    }
    w[sa] = wa + wb;
}

__global__ void k_rh_advance(RahtState *st, const unsigned long long *pairs) {
    const long long p = (long long)*pairs;
    if (p == 0) {
        st->pending++;
        return;
    }
    st->m -= p;
    st->ac_base += p;
    st->cur ^= 1;
    st->pending = 0;
}

__global__ void k_rh_init(RahtState *st, const unsigned long long *V, unsigned int *__restrict__ slot, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) slot[i] = (unsigned int)i;
    if (i == 0) {
        st->m = (long long)*V;
        st->ac_base = 0;
        st->cur = 0;
        st->pending = 0;
    }
}

unsigned int blocks_of(int64_t n, int t) { return (unsigned int)((n + t - 1) / t); }

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" mgs_status mgs_raht(mgs_ctx *ctx, const mgs_scene *scene, const int32_t *channels, int32_t n_c,
                               int32_t depth, int64_t keep, float *dc_out, float *ac_out, int64_t *n_voxels_out,
                               void *stream) {
    clear_error();
    if (!ctx || !scene || !channels || !dc_out || !ac_out || !n_voxels_out) {
        set_error("ctx, scene, channels, dc_out, ac_out and n_voxels_out must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (n_c < 1 || n_c > kMaxRahtChannels || depth < 1 || depth > 21) {
        set_error("n_channels = %d (1..%d) or depth = %d (1..21) out of range", n_c, kMaxRahtChannels, depth);
        return MGS_ERR_INVALID_ARG;
    }
    for (int k = 0; k < n_c; k++)
        if (channels[k] < 0 || channels[k] >= scene->C) {
            set_error("channel %d outside the scene's %d channels", channels[k], scene->C);
            return MGS_ERR_INVALID_ARG;
        }
    const int64_t n = scene->n;
    if (keep < 0 || keep > n) {
        set_error("keep = %lld outside 0..%lld", (long long)keep, (long long)n);
        return MGS_ERR_INVALID_ARG;
    }
    const bool subset = keep > 0 && keep < n;
    const int64_t K = subset ? keep : n;   // Gaussians transformed
    if (n > ((int64_t)1 << 31)) {
        set_error("scene of %lld Gaussians exceeds 2^31", (long long)n);
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off += al(b); return o; };
    const size_t o_vcode = take(8 * (size_t)n), o_head = take(4 * (size_t)n), o_idx = take(4 * (size_t)n);
    const size_t o_bsum = take(4 * (size_t)nb), o_total = take(8), o_start = take(8 * (size_t)n);
    const size_t o_key0 = take(8 * (size_t)n), o_key1 = take(8 * (size_t)n);
    const size_t o_slot0 = take(4 * (size_t)n), o_slot1 = take(4 * (size_t)n);
    const size_t o_w = take(4 * (size_t)n), o_x = take(4 * (size_t)n * n_c);
    const size_t o_chan = take(4 * (size_t)n_c), o_state = take(sizeof(RahtState));
    const size_t o_pos = take(subset ? 4 * (size_t)K : 0), o_tiles = take(subset ? 4 * (size_t)kept_tiles_for(n) : 0);
    char *ws = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&ws), off, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("RAHT workspace of %zu bytes could not be allocated", off);
        return MGS_ERR_OUT_OF_MEMORY;
    }
    struct Free {
        char *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } free_ws{ws, st};
    uint64_t *vcode = reinterpret_cast<uint64_t *>(ws + o_vcode);
    unsigned int *head = reinterpret_cast<unsigned int *>(ws + o_head);
    unsigned int *idx = reinterpret_cast<unsigned int *>(ws + o_idx);
    unsigned int *bsum = reinterpret_cast<unsigned int *>(ws + o_bsum);
    unsigned long long *total = reinterpret_cast<unsigned long long *>(ws + o_total);
    int64_t *start = reinterpret_cast<int64_t *>(ws + o_start);
    uint64_t *key[2] = {reinterpret_cast<uint64_t *>(ws + o_key0), reinterpret_cast<uint64_t *>(ws + o_key1)};
    unsigned int *slot[2] = {reinterpret_cast<unsigned int *>(ws + o_slot0),
                             reinterpret_cast<unsigned int *>(ws + o_slot1)};
    unsigned int *w = reinterpret_cast<unsigned int *>(ws + o_w);
    float *x = reinterpret_cast<float *>(ws + o_x);
    int32_t *d_chan = reinterpret_cast<int32_t *>(ws + o_chan);
    RahtState *rst = reinterpret_cast<RahtState *>(ws + o_state);
    int32_t *pos = nullptr;
    if (subset) {
        pos = reinterpret_cast<int32_t *>(ws + o_pos);
        MGS_TRY(kept_list_into(scene, keep, pos, reinterpret_cast<uint32_t *>(ws + o_tiles), st));
    }
    MGS_CUDA_TRY(cudaMemcpyAsync(d_chan, channels, 4 * (size_t)n_c, cudaMemcpyHostToDevice, st));
    int64_t launches = 0;
    // exclusive scan of `len` flags into `out`; the total goes to `total` (device)
    auto scan = [&](const unsigned int *in, int64_t len, unsigned int *out) {
        const int64_t blocks = (len + kScanBlock - 1) / kScanBlock;
        k_scan_local<<<(unsigned int)blocks, kScanBlock, 0, st>>>(in, len, out, bsum);
        k_scan_sums<<<1, kScanBlock, 0, st>>>(bsum, blocks, total);
        k_scan_add<<<blocks_of(len, 256), 256, 0, st>>>(out, len, bsum);
        launches += 3;
    };
    // voxels and their means
    k_rh_heads<<<blocks_of(K, 256), 256, 0, st>>>(scene->d_codes, scene->d_order, pos, K, 3 * (21 - depth),
                                                  vcode, head);
    launches++;
    scan(head, K, idx);
    unsigned long long V = 0;
    MGS_CUDA_TRY(cudaMemcpyAsync(&V, total, 8, cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    k_rh_starts<<<blocks_of(K, 256), 256, 0, st>>>(head, idx, vcode, K, start, key[0]);
    k_rh_means<<<blocks_of((int64_t)V, 256), 256, 0, st>>>(scene->d_slabs, n, pos, K, start, (int64_t)V, d_chan,
                                                           n_c, x, w);
    k_rh_init<<<blocks_of((int64_t)V, 256), 256, 0, st>>>(rst, total, slot[0], (int64_t)V);
    launches += 3;
    MGS_CUDA_TRY(cudaGetLastError());
    // merges, finest level first, on the device-resident node list; once per
    // octree level (three steps) the host reads the node count to size the grids
    int64_t cap = (int64_t)V;
    for (int s = 0; s < 3 * depth && V > 1 && cap > 1; s++) {
        const int64_t blocks = (cap + kScanBlock - 1) / kScanBlock;
        k_rh_scan_pairs<<<(unsigned int)blocks, kScanBlock, 0, st>>>(key[0], key[1], rst, cap, idx, bsum);
        k_scan_sums<<<1, kScanBlock, 0, st>>>(bsum, blocks, total);
        k_rh_merge<<<blocks_of(cap, 256), 256, 0, st>>>(key[0], key[1], slot[0], slot[1], rst, total, n_c, idx,
                                                        bsum, x, w, ac_out);
        k_rh_advance<<<1, 1, 0, st>>>(rst, total);
        launches += 4;
        if (s % 3 == 2) {
            RahtState h{};
            MGS_CUDA_TRY(cudaMemcpyAsync(&h, rst, sizeof(RahtState), cudaMemcpyDeviceToHost, st));
            MGS_CUDA_TRY(cudaStreamSynchronize(st));
            cap = h.m;
        }
    }
    MGS_CUDA_TRY(cudaGetLastError());
    count_launches(launches);
    RahtState h{};
    MGS_CUDA_TRY(cudaMemcpyAsync(&h, rst, sizeof(RahtState), cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    unsigned int root = 0;
    MGS_CUDA_TRY(cudaMemcpyAsync(&root, slot[h.cur], 4, cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    if (V > 1 && (h.m != 1 || h.ac_base != (long long)V - 1)) {
        set_error("RAHT ended with %lld nodes and %lld ACs for %llu voxels", h.m, h.ac_base, V);
        return MGS_ERR_CUDA;
    }
    MGS_CUDA_TRY(cudaMemcpyAsync(dc_out, x + (size_t)(V > 1 ? root : 0) * n_c, 4 * (size_t)n_c,
                                 cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    *n_voxels_out = (int64_t)V;
    return MGS_OK;
}
