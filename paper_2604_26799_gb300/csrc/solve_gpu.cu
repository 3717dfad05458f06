// Budget solve on the device: Eq. (eq:ilp), Sec. III-F, one multiple-choice
// knapsack per (budget, reserve ratio), then Alg. 1's tau pick on the host.
// The arithmetic is solve_def.h's, so the answers equal the host solver's bit
// for bit.
//
//   k_hull           one thread per (channel, group) item: rates in 2^-22-bit
//                    units, losses, lower convex hull, increment keys
//                    (level-major arrays), per-ratio rate totals and a
//                    2^16-bucket histogram of increment rates by the top 16
//                    key bits.
// Then every (budget, ratio) problem at once; a problem's items are cut into
// chunks of 1024, passes over items run one CTA per chunk of every problem,
// the steps that need a whole problem one CTA per problem:
//   k_split_coarse   the bucket holding the LP split, from the histogram;
//   k_split_fine /   the split key K*, 12 key bits per pass: a histogram of the
//   k_split_select   bucket's increments over every chunk, then the bucket of
//                    the split (a bucket with a single increment: its key);
//   k_order_ties /   the ordered pass: increments above K* are taken whole,
//   k_order_scan /   those equal to K* in (item, level) order while they fit
//   k_order_apply    (tie rates per chunk, their prefix over the chunks, the
//                    decisions); the first that does not fit is the split;
//   k_greedy         the loss at the split and the LP bound, then the greedy
//                    completion, one block-wide arg-min per take: the next
//                    increment is the first one in solve order, after the last
//                    one taken, that is its item's next increment and fits the
//                    remaining capacity (every increment before it in that
//                    order has already been passed over for good);
//   k_final_chunks / the chosen options and the final loss.
//   k_final_sum
// Loss totals are tree sums over chunks of 1024 items added in chunk order,
// as the host solver adds them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "solve_def.h"

namespace mgs {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSolveThreads = 1024;
constexpr int kCoarseBins = 1 << 16;
constexpr int kFineBits = 12;
constexpr int kFineBins = 1 << kFineBits;

struct TableDev {
    const double *sse, *l1, *hbits;
    const float *linf;
    const int32_t *cnt;
};

// Hulls of every item, level-major: array[v * NI + item].
struct HullDev {
    int64_t NI;
    int nb;
    uint8_t *nv;     // vertices per item
    int8_t *opt;     // [nb][NI] option index of vertex v
    int64_t *w;      // [nb][NI] rate of vertex v
    double *d;       // [nb][NI] loss of vertex v
    uint64_t *key;   // [nb - 1][NI] key of increment l
};

struct ProblemIn {
    int64_t cap;    // capacity in rate units (solve_def.h), -1 if the fixed bytes exceed the budget
    double fixed;   // fixed bytes of the ratio
    int32_t ratio;
    int32_t budget;
};

struct ProblemOut {
    int32_t status;   // 0 solved, -1 infeasible
    int32_t takes;    // increments added by the greedy completion
    double objective, bytes, lp, bytes_min, bytes_top;
};

__device__ __forceinline__ double item_loss(int norm, const TableDev &T, int64_t idx) {
    switch (norm) {
        case MGS_NORM_L2: return sqrt(T.sse[idx]);
        case MGS_NORM_L1: return T.l1[idx];
        case MGS_NORM_LINF: return (double)T.linf[idx];
        default: return T.sse[idx];
    }
}

__global__ void k_hull(TableDev T, HullDev H, int rate_model, int norm, const int32_t *__restrict__ bits,
                       const int64_t *__restrict__ item_begin, int nr,
                       unsigned long long *__restrict__ ratio_sums,
                       unsigned long long *__restrict__ hist_w, unsigned *__restrict__ hist_n) {
    __shared__ unsigned long long s_sum[2 * 64];
    // the block's share of the coarse histograms, gathered in a small open-
    // addressing table of (ratio, bucket) slots and added to the global
    // histograms once per distinct slot (integer sums: the order does not matter)
    constexpr int kSlots = 1024;
    constexpr unsigned kEmpty = 0xFFFFFFFFu;
    __shared__ unsigned s_key[kSlots];
    __shared__ unsigned long long s_w[kSlots];
    __shared__ unsigned s_n[kSlots];
    for (int k = threadIdx.x; k < 2 * nr; k += blockDim.x) s_sum[k] = 0ull;
    for (int j = threadIdx.x; j < kSlots; j += blockDim.x) {
        s_key[j] = kEmpty;
        s_w[j] = 0ull;
        s_n[j] = 0u;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < H.NI) {
        const int nb = H.nb;
        int64_t w[kMaxVerts];
        double d[kMaxVerts];
        for (int k = 0; k < nb; k++) {
            w[k] = rate_units(rate_model, T.hbits[i * nb + k], T.cnt[i], bits[k]);
            d[k] = item_loss(norm, T, i * nb + k);
        }
        int8_t opt[kMaxVerts];
        int64_t hw[kMaxVerts];
        double hd[kMaxVerts];
        const int n = build_hull(w, d, nb, opt, hw, hd);
        int lo = 0, hi = nr - 1;   // ratio of item i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_begin[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const int r = lo;
        H.nv[i] = (uint8_t)n;
        for (int v = 0; v < n; v++) {
            H.opt[v * H.NI + i] = opt[v];
            H.w[v * H.NI + i] = hw[v];
            H.d[v * H.NI + i] = hd[v];
        }
        for (int l = 0; l + 1 < n; l++) {
            const int64_t dw = hw[l + 1] - hw[l];
            const uint64_t k = inc_key(hd[l] - hd[l + 1], dw);
            H.key[l * H.NI + i] = k;
            const unsigned key = (unsigned)r * kCoarseBins + (unsigned)(k >> 48);
            unsigned h = (key * 2654435761u) >> 22;   // 10 bits
            bool done = false;
            for (int probe = 0; probe < 32 && !done; probe++, h = (h + 1) & (kSlots - 1)) {
                const unsigned prev = atomicCAS(&s_key[h], kEmpty, key);
                if (prev == kEmpty || prev == key) {
                    atomicAdd(&s_w[h], (unsigned long long)dw);
                    atomicAdd(&s_n[h], 1u);
                    done = true;
                }
            }
            if (!done) {   // a crowded table: straight to the global histogram
                atomicAdd(&hist_w[(size_t)key], (unsigned long long)dw);
                atomicAdd(&hist_n[(size_t)key], 1u);
            }
        }
        atomicAdd(&s_sum[2 * r], (unsigned long long)hw[0]);
        atomicAdd(&s_sum[2 * r + 1], (unsigned long long)w[nb - 1]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * nr; k += blockDim.x)
        if (s_sum[k]) atomicAdd(&ratio_sums[k], s_sum[k]);
    for (int j = threadIdx.x; j < kSlots; j += blockDim.x)
        if (s_key[j] != kEmpty) {
            atomicAdd(&hist_w[(size_t)s_key[j]], s_w[j]);
            atomicAdd(&hist_n[(size_t)s_key[j]], s_n[j]);
        }
}

// ---- block-wide helpers (blockDim.x == kSolveThreads) ----------------------

struct BlockScratch {
    int64_t i64[32];
    double f64[32];
};

// Inclusive prefix sum over the block; `total` receives the block's sum.
__device__ int64_t block_incl_scan(int64_t v, BlockScratch &sc, int64_t &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sc.i64[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int64_t s = sc.i64[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += t;
        }
        sc.i64[lane] = s;
    }
    __syncthreads();
    const int64_t pre = wid > 0 ? sc.i64[wid - 1] : 0;
    total = sc.i64[31];
    __syncthreads();
    return v + pre;
}

__device__ int64_t block_sum_i64(int64_t v, BlockScratch &sc) {
    int64_t total;
    block_incl_scan(v, sc, total);
    return total;
}

// The 32 x 32 pairwise tree of solve_def.h over one chunk of 1024 values;
// the result is valid in thread 0.
__device__ double block_tree_sum(double v, BlockScratch &sc) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = __dadd_rn(v, __shfl_down_sync(kFull, v, off));
    if (lane == 0) sc.f64[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = sc.f64[lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t = __dadd_rn(t, __shfl_down_sync(kFull, t, off));
    }
    __syncthreads();
    return t;
}

// Find the bucket of a descending walk over `nbins` weights where the running
// sum first exceeds `target`.  Thread t owns nbins / kSolveThreads consecutive
// buckets from the top.  Returns true (in every thread) if the total exceeds
// target; then *bin and *above (weight of the buckets above it) are set.
template <typename WFn>
__device__ bool block_find_crossing(int nbins, int64_t target, WFn weight, BlockScratch &sc,
                                    int *s_bin, int64_t *s_above, int64_t *s_total) {
    const int per = nbins / kSolveThreads;
    const int top = nbins - 1 - per * (int)threadIdx.x;
    if (threadIdx.x == 0) {   // overwritten by the crossing thread (after the scan's barriers)
        *s_bin = 0;
        *s_above = 0;
    }
    int64_t s = 0;
    for (int j = 0; j < per; j++) s += weight(top - j);
    int64_t total;
    const int64_t incl = block_incl_scan(s, sc, total);
    const int64_t excl = incl - s;
    if (total > target && excl <= target && target < incl) {
        int64_t c = excl;
        for (int j = 0; j < per; j++) {
            const int64_t hb = weight(top - j);
            if (c + hb > target) {
                *s_bin = top - j;
                *s_above = c;
                break;
            }
            c += hb;
        }
    }
    if (threadIdx.x == 0) *s_total = total;
    __syncthreads();
    return total > target;
}

// Solve order of increments (key, item, level): larger key first, then item, then level.
struct IncPos {
    uint64_t key;
    int64_t item;   // -1: none
    int level;
};
__device__ __forceinline__ bool inc_first(const IncPos &a, const IncPos &b) {
    if (a.item < 0) return false;
    if (b.item < 0) return true;
    if (a.key != b.key) return a.key > b.key;
    if (a.item != b.item) return a.item < b.item;
    return a.level < b.level;
}

// The first increment in solve order over the block; valid in every thread.
__device__ IncPos block_first(IncPos v, IncPos *s_warp, IncPos *s_out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        IncPos o;
        o.key = __shfl_down_sync(kFull, v.key, off);
        o.item = __shfl_down_sync(kFull, v.item, off);
        o.level = __shfl_down_sync(kFull, v.level, off);
        if (lane + off < 32 && inc_first(o, v)) v = o;
    }
    if (lane == 0) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = s_warp[lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            IncPos o;
            o.key = __shfl_down_sync(kFull, v.key, off);
            o.item = __shfl_down_sync(kFull, v.item, off);
            o.level = __shfl_down_sync(kFull, v.level, off);
            if (lane + off < 32 && inc_first(o, v)) v = o;
        }
        if (lane == 0) *s_out = v;
    }
    __syncthreads();
    const IncPos r = *s_out;
    __syncthreads();
    return r;
}

// ---- the solve of every (budget, ratio) problem, spread over the GPU --------
//
// A problem's items are cut into chunks of kTreeChunk (1024) items; the passes
// over items run one CTA per chunk of every problem at once, and the steps
// that need a whole problem (bucket selections, scans of chunk totals, the
// greedy completion) run one CTA per problem.  Chunk totals are combined in
// chunk order, so every sum and decision is the one-CTA-per-problem solve's.

struct Chunk {
    int32_t p;   // problem
    int32_t c;   // chunk index within the problem
};

// Per-problem state carried between the launches.
struct ProbState {
    int64_t target;      // capacity for increments (cap - W0), -1 when infeasible
    int64_t res;         // capacity left at and below the current key prefix
    int64_t total;       // rate of every increment of the ratio
    int64_t rem;         // capacity left after the ordered pass, then after the greedy takes
    uint64_t prefix;     // split-key prefix (pbits bits); the split key K* once refined
    uint64_t kfound;     // the key of a one-increment bucket
    int64_t split_item;  // the LP split increment (-1: none)
    double lp;
    int32_t pbits;
    uint32_t count;      // increments in the current bucket
    int32_t has_split;   // 0: every increment fits
    int32_t active;      // the split key is still being refined
    int32_t split_level;
    int32_t takes;
};

struct SolveArgs {
    HullDev H;
    const ProblemIn *pin;
    ProblemOut *pout;
    ProbState *state;
    const int64_t *item_begin;
    const unsigned long long *ratio_sums;
    const unsigned long long *hist_w;   // coarse histograms [ratio][2^16]
    const unsigned *hist_n;
    unsigned long long *fine_w;         // fine histograms [problem][4096], zero between passes
    unsigned *fine_n;
    const Chunk *chunks;
    const int32_t *chunk0;              // first chunk of each problem (n_problems + 1)
    int64_t *chunk_i64;                 // per chunk: tie rates, then their exclusive prefix
    int64_t *chunk_taken;               // per chunk: tie rates taken
    double *chunk_sum;                  // per chunk: tree sum of the losses
    uint8_t *level_all;                 // [budget][NI]
    uint8_t *choice_all;                // [budget][NI]
    uint64_t *next_key_all;             // [budget][NI] key of each item's next increment
    int64_t *next_dw_all;               // [budget][NI] its rate (kNoIncrement: none left)
};

constexpr int64_t kNoIncrement = INT64_MAX;   // never fits a capacity

struct ProbView {
    int64_t i0, M;
    const uint8_t *nv;
};
__device__ __forceinline__ ProbView prob_view(const SolveArgs &A, int p) {
    const int r = A.pin[p].ratio;
    ProbView v;
    v.i0 = A.item_begin[r];
    v.M = A.item_begin[r + 1] - v.i0;
    v.nv = A.H.nv + v.i0;
    return v;
}
__device__ __forceinline__ uint64_t key_of(const HullDev &H, int64_t i0, int64_t i, int l) {
    return H.key[l * H.NI + i0 + i];
}
__device__ __forceinline__ int64_t dw_of(const HullDev &H, int64_t i0, int64_t i, int l) {
    return H.w[(l + 1) * H.NI + i0 + i] - H.w[l * H.NI + i0 + i];
}

// 1. One CTA per problem: feasibility, and the coarse bucket of the LP split.
__global__ void __launch_bounds__(kSolveThreads, 1) k_split_coarse(SolveArgs A) {
    __shared__ BlockScratch sc;
    __shared__ int s_bin;
    __shared__ int64_t s_above, s_total;
    const int p = blockIdx.x;
    const ProblemIn P = A.pin[p];
    const int r = P.ratio;
    const int64_t W0 = (int64_t)A.ratio_sums[2 * r], Wtop = (int64_t)A.ratio_sums[2 * r + 1];
    ProbState st{};
    st.split_item = -1;
    if (P.cap < 0 || W0 > P.cap) {
        st.target = -1;
    } else {
        st.target = P.cap - W0;
        const unsigned long long *hw0 = A.hist_w + (size_t)r * kCoarseBins;
        const bool has_split = block_find_crossing(
            kCoarseBins, st.target, [&](int b) { return (int64_t)hw0[b]; }, sc, &s_bin, &s_above, &s_total);
        st.total = s_total;
        st.has_split = has_split ? 1 : 0;
        if (has_split) {
            st.prefix = (uint64_t)s_bin;
            st.pbits = 16;
            st.res = st.target - s_above;
            st.count = A.hist_n[(size_t)r * kCoarseBins + s_bin];
            st.active = 1;
        } else {
            st.res = st.target - s_total;   // every increment fits
        }
    }
    if (threadIdx.x == 0) {
        A.state[p] = st;
        ProblemOut out{};
        out.status = -1;
        out.bytes_min = units_to_bytes(W0, P.fixed);
        out.bytes_top = units_to_bytes(Wtop, P.fixed);
        A.pout[p] = out;
    }
}

// 2a. One CTA per chunk: the fine histogram of the increments in the current
// bucket (kFineBits more key bits), or, when the bucket holds one increment,
// its key.
__global__ void __launch_bounds__(256) k_split_fine(SolveArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Chunk ch = A.chunks[blockIdx.x];
    const ProbState st = A.state[ch.p];
    if (!st.active) return;
    const ProbView v = prob_view(A, ch.p);
    const int64_t lo = (int64_t)ch.c * kTreeChunk, hi = min(v.M, lo + kTreeChunk);
    if (st.count == 1) {
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const int n = v.nv[i];
            for (int l = 0; l + 1 < n; l++) {
                const uint64_t k = key_of(A.H, v.i0, i, l);
                if ((k >> (64 - st.pbits)) == st.prefix) A.state[ch.p].kfound = k;   // the only one
            }
        }
        return;
    }
    uint64_t *fw = reinterpret_cast<uint64_t *>(smem);
    unsigned *fc = reinterpret_cast<unsigned *>(smem + kFineBins * sizeof(uint64_t));
    for (int b = threadIdx.x; b < kFineBins; b += blockDim.x) {
        fw[b] = 0ull;
        fc[b] = 0u;
    }
    __syncthreads();
    const int shift = 64 - st.pbits - kFineBits;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int n = v.nv[i];
        for (int l = 0; l + 1 < n; l++) {
            const uint64_t k = key_of(A.H, v.i0, i, l);
            if ((k >> (shift + kFineBits)) == st.prefix) {
                const int b = (int)((k >> shift) & (kFineBins - 1));
                atomicAdd(reinterpret_cast<unsigned long long *>(&fw[b]), (unsigned long long)dw_of(A.H, v.i0, i, l));
                atomicAdd(&fc[b], 1u);
            }
        }
    }
    __syncthreads();
    unsigned long long *gw = A.fine_w + (size_t)ch.p * kFineBins;
    unsigned *gc = A.fine_n + (size_t)ch.p * kFineBins;
    for (int b = threadIdx.x; b < kFineBins; b += blockDim.x)
        if (fc[b]) {
            atomicAdd(&gw[b], (unsigned long long)fw[b]);
            atomicAdd(&gc[b], fc[b]);
        }
}

// 2b. One CTA per problem: the fine bucket of the split (or the key found),
// and a clean fine histogram for the next pass.
__global__ void __launch_bounds__(kSolveThreads, 1) k_split_select(SolveArgs A) {
    __shared__ BlockScratch sc;
    __shared__ int s_bin;
    __shared__ int64_t s_above, s_total;
    const int p = blockIdx.x;
    ProbState st = A.state[p];
    if (!st.active) return;
    unsigned long long *gw = A.fine_w + (size_t)p * kFineBins;
    unsigned *gc = A.fine_n + (size_t)p * kFineBins;
    if (st.count == 1) {
        st.prefix = st.kfound;
        st.pbits = 64;
        st.active = 0;
    } else {
        block_find_crossing(kFineBins, st.res, [&](int b) { return (int64_t)gw[b]; }, sc, &s_bin, &s_above,
                            &s_total);
        st.prefix = (st.prefix << kFineBits) | (uint64_t)s_bin;
        st.pbits += kFineBits;
        st.res -= s_above;
        st.count = gc[s_bin];
        if (st.pbits >= 64) st.active = 0;
        __syncthreads();   // every thread has read the histogram
        for (int b = threadIdx.x; b < kFineBins; b += kSolveThreads) {
            gw[b] = 0ull;
            gc[b] = 0u;
        }
    }
    if (threadIdx.x == 0) A.state[p] = st;
}

// Per item of the ordered pass: the level reached by the increments above K*,
// and the increments equal to K* (the ties), which are taken in (item, level)
// order while they fit.
struct ItemTies {
    int lvl, tfirst, tcount, n;
    int64_t tsum;
};
__device__ __forceinline__ ItemTies item_ties(const SolveArgs &A, const ProbView &v, int64_t i,
                                              const ProbState &st) {
    ItemTies t{0, -1, 0, 0, 0};
    if (i >= v.M) return t;
    t.n = v.nv[i];
    if (!st.has_split) {
        t.lvl = t.n - 1;
        return t;
    }
    const uint64_t kstar = st.prefix;
#pragma unroll
    for (int l = 0; l < kMaxVerts - 1; l++) {
        if (l + 1 >= t.n) break;
        const uint64_t k = key_of(A.H, v.i0, i, l);
        if (k > kstar) {
            t.lvl = l + 1;
        } else if (k == kstar) {
            if (t.tfirst < 0) t.tfirst = l;
            t.tcount++;
            t.tsum += dw_of(A.H, v.i0, i, l);
        }
    }
    return t;
}

// 3a. One CTA per chunk: the tie rate of the chunk.
__global__ void __launch_bounds__(kSolveThreads, 1) k_order_ties(SolveArgs A) {
    __shared__ BlockScratch sc;
    const Chunk ch = A.chunks[blockIdx.x];
    const ProbState st = A.state[ch.p];
    if (st.target < 0) return;
    const ProbView v = prob_view(A, ch.p);
    const ItemTies t = item_ties(A, v, (int64_t)ch.c * kTreeChunk + threadIdx.x, st);
    const int64_t total = block_sum_i64(t.tsum, sc);
    if (threadIdx.x == 0) A.chunk_i64[blockIdx.x] = total;
}

// 3b. One CTA per problem: exclusive prefix of the chunks' tie rates.
__global__ void __launch_bounds__(kSolveThreads, 1) k_order_scan(SolveArgs A) {
    __shared__ BlockScratch sc;
    const int p = blockIdx.x;
    if (A.state[p].target < 0) return;
    const int c0 = A.chunk0[p], c1 = A.chunk0[p + 1];
    int64_t carry = 0;
    for (int b = c0; b < c1; b += kSolveThreads) {
        const int c = b + threadIdx.x;
        const int64_t x = c < c1 ? A.chunk_i64[c] : 0;
        int64_t tot;
        const int64_t incl = block_incl_scan(x, sc, tot);
        if (c < c1) A.chunk_i64[c] = carry + incl - x;
        carry += tot;
    }
}

// 3c. One CTA per chunk: whole increments above K*, ties in order while they
// fit, the split; the levels and the chunk's loss tree sum.
__global__ void __launch_bounds__(kSolveThreads, 1) k_order_apply(SolveArgs A) {
    __shared__ BlockScratch sc;
    const Chunk ch = A.chunks[blockIdx.x];
    const ProbState st = A.state[ch.p];
    if (st.target < 0) return;
    const ProbView v = prob_view(A, ch.p);
    const int64_t i = (int64_t)ch.c * kTreeChunk + threadIdx.x;
    ItemTies t = item_ties(A, v, i, st);
    int64_t ctot;
    const int64_t incl = block_incl_scan(t.tsum, sc, ctot);
    int64_t pb = A.chunk_i64[blockIdx.x] + (incl - t.tsum);   // tie rate before this item's first tie
    int64_t my_taken = 0;
    for (int q = 0; q < t.tcount; q++) {
        const int l = t.tfirst + q;
        const int64_t dw = dw_of(A.H, v.i0, i, l);
        if (pb + dw <= st.res) {
            t.lvl = l + 1;
            my_taken += dw;
        } else if (pb <= st.res) {
            A.state[ch.p].split_item = i;   // the one tie that straddles the capacity
            A.state[ch.p].split_level = l;
        }
        pb += dw;
    }
    double d = 0.0;
    if (i < v.M) {
        const int64_t o = (int64_t)A.pin[ch.p].budget * A.H.NI + v.i0 + i;
        A.level_all[o] = (uint8_t)t.lvl;
        d = A.H.d[t.lvl * A.H.NI + v.i0 + i];
        // the item's next increment, for the greedy completion's passes
        const bool more = t.lvl + 1 < t.n;
        A.next_key_all[o] = more ? key_of(A.H, v.i0, i, t.lvl) : 0ull;
        A.next_dw_all[o] = more ? dw_of(A.H, v.i0, i, t.lvl) : kNoIncrement;
    }
    const double tsum = block_tree_sum(d, sc);
    const int64_t taken = block_sum_i64(my_taken, sc);
    if (threadIdx.x == 0) {
        A.chunk_sum[blockIdx.x] = tsum;
        A.chunk_taken[blockIdx.x] = taken;
    }
}

// 3d + 4. One CTA per problem: the loss at the split and the LP bound (chunk
// sums in chunk order), then the greedy completion, one block-wide arg-min per
// take: the next increment is the first one in solve order, after the last
// one taken, that is its item's next increment and fits the capacity left.
__global__ void __launch_bounds__(kSolveThreads, 1) k_greedy(SolveArgs A) {
    __shared__ IncPos s_warp[32];
    __shared__ IncPos s_first;
    const int p = blockIdx.x;
    ProbState st = A.state[p];
    if (st.target < 0) return;
    const ProbView v = prob_view(A, p);
    const int c0 = A.chunk0[p], c1 = A.chunk0[p + 1];
    // the chunks' sums, added in chunk order by one thread (the loads in parallel)
    __shared__ double s_cs[kSolveThreads];
    __shared__ int64_t s_ct[kSolveThreads];
    __shared__ double s_dsplit;
    __shared__ int64_t s_taken;
    double d_split = 0.0;
    int64_t taken = 0;
    for (int b = c0; b < c1; b += kSolveThreads) {
        const int c = b + threadIdx.x;
        if (c < c1) {
            s_cs[threadIdx.x] = A.chunk_sum[c];
            s_ct[threadIdx.x] = A.chunk_taken[c];
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int j = 0; j < min(kSolveThreads, c1 - b); j++) {
                d_split = d_split + s_cs[j];
                taken += s_ct[j];
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s_dsplit = d_split;
        s_taken = taken;
    }
    __syncthreads();
    d_split = s_dsplit;
    taken = s_taken;
    int64_t rem = st.res - taken;
    double lp = d_split;
    if (st.split_item >= 0) {
        const int64_t si = st.split_item;
        const int sl = st.split_level;
        const double frac = (double)rem / (double)dw_of(A.H, v.i0, si, sl);
        const double dd = A.H.d[sl * A.H.NI + v.i0 + si] - A.H.d[(sl + 1) * A.H.NI + v.i0 + si];
        if (frac > 0) lp = lp - frac * dd;
    }
    const int64_t ob = (int64_t)A.pin[p].budget * A.H.NI + v.i0;
    uint8_t *level = A.level_all + ob;
    uint64_t *nkey = A.next_key_all + ob;
    int64_t *ndw = A.next_dw_all + ob;
    IncPos last;
    last.key = 0;
    last.item = -1;
    last.level = 0;
    int takes = 0;
    while (true) {
        IncPos best;
        best.key = 0;
        best.item = -1;
        best.level = 0;
#pragma unroll 4
        for (int64_t i = threadIdx.x; i < v.M; i += kSolveThreads) {
            const int64_t dw = ndw[i];
            if (dw > rem) continue;   // none left, or it does not fit
            IncPos c;
            c.key = nkey[i];
            c.item = i;
            c.level = level[i];
            if (last.item >= 0 && !inc_first(last, c)) continue;   // passed over already
            if (inc_first(c, best)) best = c;
        }
        const IncPos f = block_first(best, s_warp, &s_first);
        if (f.item < 0) break;
        rem -= dw_of(A.H, v.i0, f.item, f.level);
        if (threadIdx.x == 0) {
            const int nl = f.level + 1;
            level[f.item] = (uint8_t)nl;
            const bool more = nl + 1 < v.nv[f.item];
            nkey[f.item] = more ? key_of(A.H, v.i0, f.item, nl) : 0ull;
            ndw[f.item] = more ? dw_of(A.H, v.i0, f.item, nl) : kNoIncrement;
        }
        last = f;
        takes++;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A.state[p].rem = rem;
        A.state[p].lp = lp;
        A.state[p].takes = takes;
    }
}

// 5a. One CTA per chunk: the chosen options and the chunk's final loss.
__global__ void __launch_bounds__(kSolveThreads, 1) k_final_chunks(SolveArgs A) {
    __shared__ BlockScratch sc;
    const Chunk ch = A.chunks[blockIdx.x];
    if (A.state[ch.p].target < 0) return;
    const ProbView v = prob_view(A, ch.p);
    const int64_t i = (int64_t)ch.c * kTreeChunk + threadIdx.x;
    const int64_t off = (int64_t)A.pin[ch.p].budget * A.H.NI + v.i0;
    double d = 0.0;
    if (i < v.M) {
        const int lvl = A.level_all[off + i];
        A.choice_all[off + i] = (uint8_t)A.H.opt[lvl * A.H.NI + v.i0 + i];
        d = A.H.d[lvl * A.H.NI + v.i0 + i];
    }
    const double tsum = block_tree_sum(d, sc);
    if (threadIdx.x == 0) A.chunk_sum[blockIdx.x] = tsum;
}

// 5b. One thread per problem: the final loss (chunk sums in chunk order).
__global__ void k_final_sum(SolveArgs A, int n_problems) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_problems) return;
    const ProbState st = A.state[p];
    if (st.target < 0) return;
    double obj = 0.0;
    for (int c = A.chunk0[p]; c < A.chunk0[p + 1]; c++) obj = obj + A.chunk_sum[c];
    const int r = A.pin[p].ratio;
    const int64_t W0 = (int64_t)A.ratio_sums[2 * r];
    ProblemOut out = A.pout[p];
    out.status = 0;
    out.takes = st.takes;
    out.objective = obj;
    out.bytes = units_to_bytes(W0 + (st.target - st.rem), A.pin[p].fixed);
    out.lp = st.lp;
    A.pout[p] = out;
}

constexpr size_t kFineSmem = kFineBins * (sizeof(uint64_t) + sizeof(unsigned));   // fine histogram

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" mgs_status mgs_solve_budgets_device(mgs_ctx *ctx, const void *table,
                                               const mgs_table_layout *layout, const mgs_grid *grid,
                                               int32_t n_budgets, const double *budgets,
                                               const mgs_solve_opts *opts, mgs_solution *out,
                                               void *stream) {
    clear_error();
    if (!ctx || !table || !layout || !grid || !opts || !out || !budgets || n_budgets < 1) {
        set_error("ctx, table, layout, grid, budgets, opts and out must be non-NULL; n_budgets >= 1");
        return MGS_ERR_INVALID_ARG;
    }
    if (grid->n_bits != layout->n_bits || grid->n_ratios != layout->n_ratios || !grid->bits ||
        opts->rate_model < 0 || opts->rate_model > 1 || opts->norm < 0 || opts->norm > 3 ||
        layout->n_bits < 1 || layout->n_bits > MGS_MAX_OPTIONS || layout->n_ratios < 1 ||
        layout->n_ratios > 64) {
        set_error("grid/layout mismatch or bad options");
        return MGS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n_budgets; i++)
        if (!(budgets[i] >= 0)) {
            set_error("budget %d is negative or NaN", i);
            return MGS_ERR_INVALID_ARG;
        }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nr = layout->n_ratios, nb = layout->n_bits;
    const int64_t NI = layout->item_begin[nr];
    const int P = n_budgets * nr;

    // a host table is copied in first
    cudaPointerAttributes pa{};
    const bool on_device = cudaPointerGetAttributes(&pa, table) == cudaSuccess &&
                           (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    cudaGetLastError();

    std::vector<ProblemIn> pin(P);
    for (int b = 0; b < n_budgets; b++)
        for (int r = 0; r < nr; r++) {
            const int64_t M = layout->item_begin[r + 1] - layout->item_begin[r];
            ProblemIn &p = pin[b * nr + r];
            p.fixed = opts->meta_bytes_per_group * (double)M + opts->const_bytes + opts->delta_bytes;
            p.cap = capacity_units(budgets[b], p.fixed);
            p.ratio = r;
            p.budget = b;
        }

    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += a256(bytes);
        return o;
    };
    const size_t o_tab = on_device ? 0 : take(layout->total_bytes);
    const size_t o_nv = take(NI);
    const size_t o_opt = take((size_t)nb * NI);
    const size_t o_w = take(sizeof(int64_t) * nb * NI);
    const size_t o_d = take(sizeof(double) * nb * NI);
    const size_t o_key = take(sizeof(uint64_t) * std::max(1, nb - 1) * NI);
    const size_t o_zero = off;   // zeroed region: ratio sums and histograms
    const size_t o_sums = take(sizeof(unsigned long long) * 2 * nr);
    const size_t o_hw = take(sizeof(unsigned long long) * kCoarseBins * nr);
    const size_t o_hn = take(sizeof(unsigned) * kCoarseBins * nr);
    const size_t zero_bytes = off - o_zero;
    const size_t o_bits = take(sizeof(int32_t) * nb);
    const size_t o_ib = take(sizeof(int64_t) * (nr + 1));
    // chunks of kTreeChunk items of every problem
    std::vector<Chunk> chunks;
    std::vector<int32_t> chunk0(P + 1, 0);
    for (int p = 0; p < P; p++) {
        const int r = pin[p].ratio;
        const int64_t M = layout->item_begin[r + 1] - layout->item_begin[r];
        chunk0[p] = (int32_t)chunks.size();
        for (int64_t c = 0; c * kTreeChunk < M; c++) chunks.push_back(Chunk{p, (int32_t)c});
    }
    chunk0[P] = (int32_t)chunks.size();
    const int64_t NC = std::max<int64_t>((int64_t)chunks.size(), 1);
    const size_t o_pin = take(sizeof(ProblemIn) * P);
    const size_t o_pout = take(sizeof(ProblemOut) * P);
    const size_t o_state = take(sizeof(ProbState) * P);
    const size_t o_chunks = take(sizeof(Chunk) * NC);
    const size_t o_chunk0 = take(sizeof(int32_t) * (P + 1));
    const size_t o_ci64 = take(sizeof(int64_t) * NC);
    const size_t o_ctaken = take(sizeof(int64_t) * NC);
    const size_t o_csum = take(sizeof(double) * NC);
    const size_t o_fz = off;   // zeroed: fine histograms
    const size_t o_fw = take(sizeof(unsigned long long) * kFineBins * P);
    const size_t o_fn = take(sizeof(unsigned) * kFineBins * P);
    const size_t fine_bytes = off - o_fz;
    const size_t o_level = take((size_t)n_budgets * NI);
    const size_t o_choice = take((size_t)n_budgets * NI);
    const size_t o_nkey = take(sizeof(uint64_t) * n_budgets * NI);
    const size_t o_ndw = take(sizeof(int64_t) * n_budgets * NI);
    char *ws = nullptr;
    cudaError_t e = dev_malloc_async(reinterpret_cast<void **>(&ws), off, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device workspace of %zu bytes: %s", off, cudaGetErrorString(e));
        return MGS_ERR_OUT_OF_MEMORY;
    }
    struct Free {
        char *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } free_ws{ws, st};

    const char *tab = on_device ? static_cast<const char *>(table) : ws + o_tab;
    if (!on_device) MGS_CUDA_TRY(cudaMemcpyAsync(ws + o_tab, table, layout->total_bytes, cudaMemcpyHostToDevice, st));
    MGS_CUDA_TRY(cudaMemsetAsync(ws + o_zero, 0, zero_bytes, st));
    MGS_CUDA_TRY(cudaMemsetAsync(ws + o_fz, 0, fine_bytes, st));
    MGS_CUDA_TRY(cudaMemcpyAsync(ws + o_bits, grid->bits, sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st));
    MGS_CUDA_TRY(cudaMemcpyAsync(ws + o_ib, layout->item_begin, sizeof(int64_t) * (nr + 1),
                                 cudaMemcpyHostToDevice, st));
    MGS_CUDA_TRY(cudaMemcpyAsync(ws + o_pin, pin.data(), sizeof(ProblemIn) * P, cudaMemcpyHostToDevice, st));
    MGS_CUDA_TRY(cudaMemcpyAsync(ws + o_chunks, chunks.data(), sizeof(Chunk) * chunks.size(),
                                 cudaMemcpyHostToDevice, st));
    MGS_CUDA_TRY(cudaMemcpyAsync(ws + o_chunk0, chunk0.data(), sizeof(int32_t) * (P + 1), cudaMemcpyHostToDevice,
                                 st));

    TableDev T;
    T.sse = reinterpret_cast<const double *>(tab + layout->off_sse);
    T.l1 = reinterpret_cast<const double *>(tab + layout->off_l1);
    T.hbits = reinterpret_cast<const double *>(tab + layout->off_hbits);
    T.linf = reinterpret_cast<const float *>(tab + layout->off_linf);
    T.cnt = reinterpret_cast<const int32_t *>(tab + layout->off_count);
    HullDev H;
    H.NI = NI;
    H.nb = nb;
    H.nv = reinterpret_cast<uint8_t *>(ws + o_nv);
    H.opt = reinterpret_cast<int8_t *>(ws + o_opt);
    H.w = reinterpret_cast<int64_t *>(ws + o_w);
    H.d = reinterpret_cast<double *>(ws + o_d);
    H.key = reinterpret_cast<uint64_t *>(ws + o_key);
    auto *sums = reinterpret_cast<unsigned long long *>(ws + o_sums);
    auto *hw = reinterpret_cast<unsigned long long *>(ws + o_hw);
    auto *hn = reinterpret_cast<unsigned *>(ws + o_hn);
    const int64_t *d_ib = reinterpret_cast<const int64_t *>(ws + o_ib);

    k_hull<<<(unsigned)((NI + 255) / 256), 256, 0, st>>>(T, H, opts->rate_model, opts->norm,
                                                        reinterpret_cast<const int32_t *>(ws + o_bits),
                                                        d_ib, nr, sums, hw, hn);
    MGS_CUDA_TRY(cudaGetLastError());
    SolveArgs A;
    A.H = H;
    A.pin = reinterpret_cast<const ProblemIn *>(ws + o_pin);
    A.pout = reinterpret_cast<ProblemOut *>(ws + o_pout);
    A.state = reinterpret_cast<ProbState *>(ws + o_state);
    A.item_begin = d_ib;
    A.ratio_sums = sums;
    A.hist_w = hw;
    A.hist_n = hn;
    A.fine_w = reinterpret_cast<unsigned long long *>(ws + o_fw);
    A.fine_n = reinterpret_cast<unsigned *>(ws + o_fn);
    A.chunks = reinterpret_cast<const Chunk *>(ws + o_chunks);
    A.chunk0 = reinterpret_cast<const int32_t *>(ws + o_chunk0);
    A.chunk_i64 = reinterpret_cast<int64_t *>(ws + o_ci64);
    A.chunk_taken = reinterpret_cast<int64_t *>(ws + o_ctaken);
    A.chunk_sum = reinterpret_cast<double *>(ws + o_csum);
    A.level_all = reinterpret_cast<uint8_t *>(ws + o_level);
    A.choice_all = reinterpret_cast<uint8_t *>(ws + o_choice);
    A.next_key_all = reinterpret_cast<uint64_t *>(ws + o_nkey);
    A.next_dw_all = reinterpret_cast<int64_t *>(ws + o_ndw);
    const unsigned nc = (unsigned)chunks.size();
    int launches = 1;
    k_split_coarse<<<P, kSolveThreads, 0, st>>>(A);
    launches++;
    // the split key: 16 bits from the coarse histogram, kFineBits per pass after
    for (int pass = 0; pass < (64 - 16 + kFineBits - 1) / kFineBits && nc > 0; pass++) {
        k_split_fine<<<nc, 256, kFineSmem, st>>>(A);
        k_split_select<<<P, kSolveThreads, 0, st>>>(A);
        launches += 2;
    }
    if (nc > 0) {
        k_order_ties<<<nc, kSolveThreads, 0, st>>>(A);
        k_order_scan<<<P, kSolveThreads, 0, st>>>(A);
        k_order_apply<<<nc, kSolveThreads, 0, st>>>(A);
        launches += 3;
    }
    k_greedy<<<P, kSolveThreads, 0, st>>>(A);
    launches++;
    if (nc > 0) {
        k_final_chunks<<<nc, kSolveThreads, 0, st>>>(A);
        launches++;
    }
    k_final_sum<<<(P + 127) / 128, 128, 0, st>>>(A, P);
    launches++;
    MGS_CUDA_TRY(cudaGetLastError());
    count_launches(launches);
    std::vector<ProblemOut> po(P);
    MGS_CUDA_TRY(cudaMemcpyAsync(po.data(), ws + o_pout, sizeof(ProblemOut) * P, cudaMemcpyDeviceToHost, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));

    // tau rule (Alg. 1), as in mgs_solve_budgets
    mgs_status worst = MGS_OK;
    for (int b = 0; b < n_budgets; b++) {
        ProblemOut *pr = &po[(size_t)b * nr];
        mgs_solution *o = &out[b];
        int best = -1, largest_feasible = -1;
        std::vector<int> status(nr);
        for (int r = 0; r < nr; r++) {
            status[r] = pr[r].status;
            if (status[r] < 0) continue;
            largest_feasible = r;
            if (pr[r].bytes_top < budgets[b]) {
                status[r] = 1;
                continue;
            }
            if (best < 0 || pr[r].objective <= pr[best].objective) best = r;
        }
        if (best < 0) best = largest_feasible;
        for (int r = 0; r < nr; r++) {
            if (o->ratio_status) o->ratio_status[r] = status[r];
            if (o->ratio_objective) o->ratio_objective[r] = pr[r].status < 0 ? 0.0 : pr[r].objective;
            if (o->ratio_bytes) o->ratio_bytes[r] = pr[r].status < 0 ? 0.0 : pr[r].bytes;
            if (o->ratio_lp_bound) o->ratio_lp_bound[r] = pr[r].status < 0 ? 0.0 : pr[r].lp;
        }
        o->r_index = best;
        if (best < 0) {
            o->est_bytes = o->objective = o->lp_bound = 0;
            set_error("no ratio fits a budget of %.0f bytes", budgets[b]);
            worst = MGS_ERR_INFEASIBLE;
            continue;
        }
        o->est_bytes = pr[best].bytes;
        o->objective = pr[best].objective;
        o->lp_bound = pr[best].lp;
        if (o->choice) {
            const int64_t i0 = layout->item_begin[best], M = layout->item_begin[best + 1] - i0;
            MGS_CUDA_TRY(cudaMemcpyAsync(o->choice, ws + o_choice + (size_t)b * NI + i0, M,
                                         cudaMemcpyDeviceToHost, st));
        }
    }
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    return worst;
}
