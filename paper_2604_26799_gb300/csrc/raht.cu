// RAHT (Sec. III-D "Region Adaptive Hierarchical Transform") of a resident
// scene's channels at octree depth d.
//
//   k_rh_heads   voxel code of every Morton position (Morton code >> 3(21 - d))
//                and a flag where a new voxel starts
//   scan         voxel index of every position (exclusive prefix sum)
//   k_rh_starts  first Morton position and code of every voxel
//   k_rh_means   one thread per voxel: mean of its Gaussians, summed in
//                Morton order (weight 1)
//   the merge tree: RAHT step s merges the nodes that are siblings at bit s
//   of the binary trie over the sorted voxel codes, so the internal node
//   between voxels g and g + 1 merges at step delta(g) = the highest bit in
//   which their codes differ, and every merge of the transform is one
//   internal node:
//     k_rh_delta, k_rh_delta_slots, k_rh_delta_place  delta of every internal
//                 node and its AC slot: ACs listed step by step, ascending
//                 code within a step (a stable counting sort on delta); the
//                 slots of one step are contiguous
//     k_rh_step   one launch per step that has merges: its merges join
//                 disjoint segments (a node's children have smaller deltas,
//                 so they were formed by earlier launches), one thread each,
//                 by the printed T with its entries t1 = sqrt(w1) / sqrt(w1 + w2),
//                 t2 = sqrt(w2) / sqrt(w1 + w2) formed once per pair:
//                 DC = t1 x1 + t2 x2 (into the left segment's first slot),
//                 weight w1 + w2, AC = t1 x2 - t2 x1 at the node's AC slot;
//                 each segment keeps its endpoints at its two ends.
//   (An earlier version ran the 3d steps as 4 launches each over the whole
//   node list; with sparse fine levels most of its ~20 heavy steps moved every
//   node for a handful of pairs.  A version that walked the tree up with one
//   thread per voxel and arrival counters spent 1.9 ms in grid-wide fences.)
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

// ---- the merge tree ----
// The nodes RAHT merges at step s are siblings at bit s of a binary trie over
// the sorted voxel codes: the internal node between voxels g and g + 1 merges
// at step delta(g), the highest bit in which their codes differ.
constexpr int kDeltaKeys = 64;
constexpr int kDeltaChunk = 1024;

// delta of every internal node, and per chunk of 1024 nodes the count of each delta
__global__ void __launch_bounds__(kDeltaChunk)
    k_rh_delta(const uint64_t *__restrict__ vc, int64_t V, unsigned char *__restrict__ delta,
               unsigned int *__restrict__ cnt) {
    __shared__ unsigned int s_cnt[kDeltaKeys];
    if (threadIdx.x < kDeltaKeys) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * kDeltaChunk + threadIdx.x;
    if (g < V - 1) {
        const int d = 63 - __clzll((long long)(vc[g] ^ vc[g + 1]));
        delta[g] = (unsigned char)d;
        atomicAdd(&s_cnt[d], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kDeltaKeys) cnt[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = s_cnt[threadIdx.x];
}

// Per delta value (one CTA each): the exclusive prefix over chunks of its
// counts, in place, and its total.
__global__ void __launch_bounds__(1024)
    k_rh_delta_slots(unsigned int *__restrict__ cnt, int64_t nchunks, unsigned int *__restrict__ total) {
    __shared__ unsigned int s_w[32];
    __shared__ unsigned int s_carry;
    unsigned int *row = cnt + (int64_t)blockIdx.x * nchunks;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nchunks; base += 1024) {
        const int64_t c = base + threadIdx.x;
        const unsigned int v = c < nchunks ? row[c] : 0u;
        unsigned int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        unsigned int wb = 0, all = 0;
        for (int q = 0; q < 32; q++) {
            if (q < wid) wb += s_w[q];
            all += s_w[q];
        }
        if (c < nchunks) row[c] = s_carry + wb + x - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) total[blockIdx.x] = s_carry;
}

// The AC slot of every internal node (ACs step by step, ascending code within
// a step): the totals of the smaller deltas, plus its (delta, chunk) prefix,
// plus its rank among the chunk's nodes of equal delta, the warps in order.
// node[slot] is the inverse map.
__global__ void __launch_bounds__(kDeltaChunk)
    k_rh_delta_place(const unsigned char *__restrict__ delta, int64_t V, const unsigned int *__restrict__ prefix,
                     const unsigned int *__restrict__ total, unsigned int *__restrict__ node) {
    __shared__ unsigned int s_run[kDeltaKeys], s_base[kDeltaKeys];
    if (threadIdx.x < kDeltaKeys) {
        s_run[threadIdx.x] = 0;
        unsigned int b = 0;
        for (int q = 0; q < (int)threadIdx.x; q++) b += total[q];
        s_base[threadIdx.x] = b;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * kDeltaChunk + threadIdx.x;
    const bool act = g < V - 1;
    const int k = act ? (int)delta[g] : kDeltaKeys + lane;   // inactive lanes never match
    const unsigned int peers = __match_any_sync(0xFFFFFFFFu, k);
    const unsigned int rank = __popc(peers & ((1u << lane) - 1u));
    for (int w = 0; w < kDeltaChunk / 32; w++) {
        if (warp == w && act)
            node[s_base[k] + prefix[(int64_t)k * gridDim.x + blockIdx.x] + s_run[k] + rank] = (unsigned int)g;
        __syncthreads();
        if (warp == w && act && rank == 0) s_run[k] += __popc(peers);
        __syncthreads();
    }
}

// One RAHT step: the m merges of AC slots [a0, a0 + m), all at the same bit,
// so they touch disjoint segments.  A segment [l, r] keeps its value in slot
// l and its endpoints at its two ends (endL[r] = l, endR[l] = r).  The node
// between voxels g and g + 1 merges the segment ending at g with the one
// starting at g + 1 by the printed T, with its entries t1 = sqrt(w1) /
// sqrt(w1 + w2), t2 = sqrt(w2) / sqrt(w1 + w2) formed once per pair:
// DC = t1 x1 + t2 x2, weight w1 + w2, AC = t1 x2 - t2 x1.
__global__ void k_rh_step(const unsigned int *__restrict__ node, int64_t a0, int64_t m, int n_c,
                          float *__restrict__ x, unsigned int *__restrict__ w, unsigned int *__restrict__ endL,
                          unsigned int *__restrict__ endR, float *__restrict__ ac) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int64_t a = a0 + t;
    const unsigned int g = node[a];
    const unsigned int l = endL[g], r = endR[g + 1];
    const int64_t sa = l, sb = (int64_t)g + 1;
    const unsigned int wa = w[sa], wb = w[sb];
    const float sw = __fsqrt_rn((float)(wa + wb));
    const float t1 = __fdiv_rn(__fsqrt_rn((float)wa), sw), t2 = __fdiv_rn(__fsqrt_rn((float)wb), sw);
    float *xa = x + sa * n_c;
    const float *xb = x + sb * n_c;
    float *acp = ac + a * n_c;
    int k = 0;
    for (; k + 4 <= n_c; k += 4) {   // four channels at a time: independent loads in flight
        float x1[4], x2[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            x1[u] = xa[k + u];
            x2[u] = xb[k + u];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            xa[k + u] = __fadd_rn(__fmul_rn(t1, x1[u]), __fmul_rn(t2, x2[u]));
            acp[k + u] = __fsub_rn(__fmul_rn(t1, x2[u]), __fmul_rn(t2, x1[u]));
        }
    }
    for (; k < n_c; k++) {
        const float x1 = xa[k], x2 = xb[k];
        xa[k] = __fadd_rn(__fmul_rn(t1, x1), __fmul_rn(t2, x2));
        acp[k] = __fsub_rn(__fmul_rn(t1, x2), __fmul_rn(t2, x1));
    }
    w[sa] = wa + wb;
    endL[r] = l;
    endR[l] = r;
}

__global__ void k_rh_ends(unsigned int *__restrict__ endL, unsigned int *__restrict__ endR, int64_t V) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < V) endL[i] = endR[i] = (unsigned int)i;
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
    const int64_t nchunks = (n + kDeltaChunk - 1) / kDeltaChunk;
    const size_t o_key0 = take(8 * (size_t)n), o_delta = take((size_t)n), o_acpos = take(4 * (size_t)n);
    const size_t o_dcnt = take(4 * (size_t)kDeltaKeys * (size_t)nchunks), o_dtot = take(4 * kDeltaKeys);
    const size_t o_endl = take(4 * (size_t)n), o_endr = take(4 * (size_t)n);
    const size_t o_w = take(4 * (size_t)n), o_x = take(4 * (size_t)n * n_c);
    const size_t o_chan = take(4 * (size_t)n_c);
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
    uint64_t *vc = reinterpret_cast<uint64_t *>(ws + o_key0);
    unsigned char *delta = reinterpret_cast<unsigned char *>(ws + o_delta);
    unsigned int *node = reinterpret_cast<unsigned int *>(ws + o_acpos);
    unsigned int *dcnt = reinterpret_cast<unsigned int *>(ws + o_dcnt);
    unsigned int *dtot = reinterpret_cast<unsigned int *>(ws + o_dtot);
    unsigned int *endL = reinterpret_cast<unsigned int *>(ws + o_endl);
    unsigned int *endR = reinterpret_cast<unsigned int *>(ws + o_endr);
    unsigned int *w = reinterpret_cast<unsigned int *>(ws + o_w);
    float *x = reinterpret_cast<float *>(ws + o_x);
    int32_t *d_chan = reinterpret_cast<int32_t *>(ws + o_chan);
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
    k_rh_starts<<<blocks_of(K, 256), 256, 0, st>>>(head, idx, vcode, K, start, vc);
    k_rh_means<<<blocks_of((int64_t)V, 256), 256, 0, st>>>(scene->d_slabs, n, pos, K, start, (int64_t)V, d_chan,
                                                           n_c, x, w);
    launches += 2;
    if (V > 1) {
        // the merge tree: AC slots by (step, code); then one launch per step
        // that has merges, over that step's slots
        const int64_t ch = ((int64_t)V - 1 + kDeltaChunk - 1) / kDeltaChunk;
        k_rh_delta<<<(unsigned int)ch, kDeltaChunk, 0, st>>>(vc, (int64_t)V, delta, dcnt);
        k_rh_delta_slots<<<kDeltaKeys, 1024, 0, st>>>(dcnt, ch, dtot);
        k_rh_delta_place<<<(unsigned int)ch, kDeltaChunk, 0, st>>>(delta, (int64_t)V, dcnt, dtot, node);
        k_rh_ends<<<blocks_of((int64_t)V, 256), 256, 0, st>>>(endL, endR, (int64_t)V);
        launches += 4;
        unsigned int h_tot[kDeltaKeys];
        MGS_CUDA_TRY(cudaMemcpyAsync(h_tot, dtot, sizeof(h_tot), cudaMemcpyDeviceToHost, st));
        MGS_CUDA_TRY(cudaStreamSynchronize(st));
        int64_t a0 = 0;
        for (int b = 0; b < kDeltaKeys; b++) {
            if (!h_tot[b]) continue;
            k_rh_step<<<blocks_of((int64_t)h_tot[b], 256), 256, 0, st>>>(node, a0, (int64_t)h_tot[b], n_c, x, w,
                                                                        endL, endR, ac_out);
            launches++;
            a0 += h_tot[b];
        }
        if (a0 != (int64_t)V - 1) {
            set_error("RAHT: %lld merges for %llu voxels", (long long)a0, V);
            return MGS_ERR_CUDA;
        }
    }
    MGS_CUDA_TRY(cudaGetLastError());
    count_launches(launches);
    MGS_CUDA_TRY(cudaMemcpyAsync(dc_out, x, 4 * (size_t)n_c, cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    *n_voxels_out = (int64_t)V;
    return MGS_OK;
}
