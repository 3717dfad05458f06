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
//                 code within a step (a stable counting sort on delta)
//     k_rh_tree   one thread per voxel walks up; a node [l, r] merges next with
//                 the neighbour across the split of smaller delta; the first
//                 child to arrive stops, the second merges both by the printed
//                 T, with its entries t1 = sqrt(w1) / sqrt(w1 + w2),
//                 t2 = sqrt(w2) / sqrt(w1 + w2) formed once per pair:
//                 DC = t1 x1 + t2 x2 (into the left child's slot), weight
//                 w1 + w2, AC = t1 x2 - t2 x1 at the node's AC slot.
//   (An earlier version ran the 3d steps as 4 launches each over the whole
//   node list; with sparse fine levels most of its ~20 heavy steps moved every
//   node for a handful of pairs.)
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
// at step delta(g), the highest bit in which their codes differ.  A node
// covering voxels [l, r] merges next with the neighbour across the split of
// smaller delta (l - 1 or r; the two are never equal for distinct codes).
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

// First AC slot of every (delta, chunk): ACs are listed step by step (delta
// ascending), in ascending code within a step.  One thread per delta value.
__global__ void k_rh_delta_slots(unsigned int *__restrict__ cnt, int64_t nchunks) {
    __shared__ unsigned long long s_tot[kDeltaKeys];
    const int k = threadIdx.x;
    unsigned int *row = cnt + (int64_t)k * nchunks;
    unsigned long long tot = 0;
    for (int64_t c = 0; c < nchunks; c++) tot += row[c];
    s_tot[k] = tot;
    __syncthreads();
    unsigned long long run = 0;
    for (int q = 0; q < k; q++) run += s_tot[q];
    for (int64_t c = 0; c < nchunks; c++) {
        const unsigned int t = row[c];
        row[c] = (unsigned int)run;
        run += t;
    }
}

// The AC slot of every internal node: its (delta, chunk) slot plus its rank
// among the chunk's nodes of equal delta, the warps in order.
__global__ void __launch_bounds__(kDeltaChunk)
    k_rh_delta_place(const unsigned char *__restrict__ delta, int64_t V, const unsigned int *__restrict__ slot,
                     unsigned int *__restrict__ acpos) {
    __shared__ unsigned int s_run[kDeltaKeys];
    if (threadIdx.x < kDeltaKeys) s_run[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * kDeltaChunk + threadIdx.x;
    const bool act = g < V - 1;
    const int k = act ? (int)delta[g] : kDeltaKeys + lane;   // inactive lanes never match
    const unsigned int peers = __match_any_sync(0xFFFFFFFFu, k);
    const unsigned int rank = __popc(peers & ((1u << lane) - 1u));
    for (int w = 0; w < kDeltaChunk / 32; w++) {
        if (warp == w && act) acpos[g] = slot[(int64_t)k * gridDim.x + blockIdx.x] + s_run[k] + rank;
        __syncthreads();
        if (warp == w && act && rank == 0) s_run[k] += __popc(peers);
        __syncthreads();
    }
}

__device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }

// One thread per voxel, walking up: the first child to reach a node records
// its extent and stops; the second merges both children by the printed T
// (entries t1 = sqrt(w1) / sqrt(w1 + w2), t2 = sqrt(w2) / sqrt(w1 + w2), once
// per pair: DC = t1 x1 + t2 x2 into the left child's slot, AC = t1 x2 - t2 x1
// at the node's AC slot, weight w1 + w2) and goes on.  A node's value lives in
// the slot of its leftmost voxel.
__global__ void k_rh_tree(const unsigned char *__restrict__ delta, const unsigned int *__restrict__ acpos,
                          int64_t V, int n_c, float *__restrict__ x, unsigned int *__restrict__ w,
                          int64_t *__restrict__ ext, unsigned int *__restrict__ arrive,
                          float *__restrict__ ac) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    int64_t l = v, r = v;
    while (!(l == 0 && r == V - 1)) {
        // the parent: the split of smaller delta next to [l, r]
        const bool left_child = l == 0 || (r < V - 1 && delta[r] < delta[l - 1]);
        const int64_t g = left_child ? r : l - 1;
        ext[2 * g + (left_child ? 0 : 1)] = left_child ? l : r;   // my extent, for my sibling
        __threadfence();
        if (atomicAdd(&arrive[g], 1u) == 0u) return;   // the sibling merges this node
        __threadfence();
        const long long *e2 = reinterpret_cast<const long long *>(ext) + 2 * g;
        const int64_t ll = left_child ? l : (int64_t)__ldcg(e2);
        const int64_t rr = left_child ? (int64_t)__ldcg(e2 + 1) : r;
        const int64_t sa = ll, sb = g + 1;   // the left and right children's slots
        const unsigned int wa = __ldcg(&w[sa]), wb = __ldcg(&w[sb]);
        const float sw = __fsqrt_rn((float)(wa + wb));
        const float t1 = __fdiv_rn(__fsqrt_rn((float)wa), sw), t2 = __fdiv_rn(__fsqrt_rn((float)wb), sw);
        float *xa = x + sa * n_c;
        const float *xb = x + sb * n_c;
        float *acp = ac + (int64_t)acpos[g] * n_c;
        for (int k = 0; k < n_c; k++) {
            const float x1 = ld_cg(xa + k), x2 = ld_cg(xb + k);
            xa[k] = __fadd_rn(__fmul_rn(t1, x1), __fmul_rn(t2, x2));
            acp[k] = __fsub_rn(__fmul_rn(t1, x2), __fmul_rn(t2, x1));
        }
        w[sa] = wa + wb;
        l = ll;
        r = rr;
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
    const int64_t nchunks = (n + kDeltaChunk - 1) / kDeltaChunk;
    const size_t o_key0 = take(8 * (size_t)n), o_delta = take((size_t)n), o_acpos = take(4 * (size_t)n);
    const size_t o_dcnt = take(4 * (size_t)kDeltaKeys * (size_t)nchunks), o_ext = take(16 * (size_t)n);
    const size_t o_arrive = take(4 * (size_t)n);
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
    unsigned int *acpos = reinterpret_cast<unsigned int *>(ws + o_acpos);
    unsigned int *dcnt = reinterpret_cast<unsigned int *>(ws + o_dcnt);
    int64_t *ext = reinterpret_cast<int64_t *>(ws + o_ext);
    unsigned int *arrive = reinterpret_cast<unsigned int *>(ws + o_arrive);
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
        // the merge tree: AC slots by (step, code), then every voxel walks up
        const int64_t ch = ((int64_t)V - 1 + kDeltaChunk - 1) / kDeltaChunk;
        MGS_CUDA_TRY(cudaMemsetAsync(arrive, 0, 4 * (size_t)V, st));
        k_rh_delta<<<(unsigned int)ch, kDeltaChunk, 0, st>>>(vc, (int64_t)V, delta, dcnt);
        k_rh_delta_slots<<<1, kDeltaKeys, 0, st>>>(dcnt, ch);
        k_rh_delta_place<<<(unsigned int)ch, kDeltaChunk, 0, st>>>(delta, (int64_t)V, dcnt, acpos);
        k_rh_tree<<<blocks_of((int64_t)V, 256), 256, 0, st>>>(delta, acpos, (int64_t)V, n_c, x, w, ext, arrive,
                                                              ac_out);
        launches += 4;
    }
    MGS_CUDA_TRY(cudaGetLastError());
    count_launches(launches);
    MGS_CUDA_TRY(cudaMemcpyAsync(dc_out, x, 4 * (size_t)n_c, cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    *n_voxels_out = (int64_t)V;
    return MGS_OK;
}
