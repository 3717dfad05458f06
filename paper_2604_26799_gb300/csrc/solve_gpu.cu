// Budget solve on the device: Eq. (eq:ilp), Sec. III-F, one multiple-choice
// knapsack per (budget, reserve ratio), then Alg. 1's tau pick on the host.
// The arithmetic is solve_def.h's, so the answers equal the host solver's bit
// for bit.
//
//   k_hull   one thread per (channel, group) item: rates in 2^-22-bit units,
//            losses, lower convex hull, increment keys (level-major arrays),
//            per-ratio rate totals and a 2^16-bucket histogram of increment
//            rates by the top 16 key bits.
//   k_solve  one 1024-thread CTA per (budget, ratio) problem:
//            1. the bucket holding the LP split, from the histogram;
//            2. the split key K*, 12 key bits per pass over the ratio's
//               increments (shared-memory histogram; a bucket with a single
//               increment ends the search early);
//            3. one ordered pass over the items: increments above K* are
//               taken whole, those equal to K* in (item, level) order while
//               they fit (block prefix sums); the first that does not fit is
//               the split; the loss at the split and the LP bound;
//            4. greedy completion, one block-wide arg-min per take: the next
//               increment to take is the first one in solve order, after
//               the last one taken, that is its item's next increment and
//               fits the remaining capacity (every increment before it in
//               that order has already been passed over for good);
//            5. the chosen options and the final loss (tree sum).
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
    for (int k = threadIdx.x; k < 2 * nr; k += blockDim.x) s_sum[k] = 0ull;
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
            atomicAdd(&hist_w[(size_t)r * kCoarseBins + (k >> 48)], (unsigned long long)dw);
            atomicAdd(&hist_n[(size_t)r * kCoarseBins + (k >> 48)], 1u);
        }
        atomicAdd(&s_sum[2 * r], (unsigned long long)hw[0]);
        atomicAdd(&s_sum[2 * r + 1], (unsigned long long)w[nb - 1]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * nr; k += blockDim.x)
        if (s_sum[k]) atomicAdd(&ratio_sums[k], s_sum[k]);
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

__global__ void __launch_bounds__(kSolveThreads, 1)
    k_solve(HullDev H, const ProblemIn *__restrict__ pin, ProblemOut *__restrict__ pout,
            const int64_t *__restrict__ item_begin, const unsigned long long *__restrict__ ratio_sums,
            const unsigned long long *__restrict__ hist_w, const unsigned *__restrict__ hist_n,
            uint8_t *__restrict__ level_all, uint8_t *__restrict__ choice_all) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockScratch sc;
    __shared__ int s_bin;
    __shared__ int64_t s_above, s_total;
    __shared__ uint64_t s_kstar;
    __shared__ int64_t s_split_item;
    __shared__ int s_split_level;
    __shared__ IncPos s_warp[32];
    __shared__ IncPos s_first;

    const int tid = threadIdx.x;
    const ProblemIn P = pin[blockIdx.x];
    const int r = P.ratio;
    const int64_t i0 = item_begin[r], M = item_begin[r + 1] - i0;
    const int64_t NI = H.NI;
    const int64_t W0 = (int64_t)ratio_sums[2 * r], Wtop = (int64_t)ratio_sums[2 * r + 1];
    ProblemOut out;
    out.status = -1;
    out.takes = 0;
    out.objective = out.bytes = out.lp = 0.0;
    out.bytes_min = units_to_bytes(W0, P.fixed);
    out.bytes_top = units_to_bytes(Wtop, P.fixed);
    if (P.cap < 0 || W0 > P.cap) {
        if (tid == 0) pout[blockIdx.x] = out;
        return;
    }
    const int64_t target = P.cap - W0;
    uint8_t *level = level_all + (int64_t)P.budget * NI + i0;
    const uint8_t *nv = H.nv + i0;
    auto key_at = [&](int64_t i, int l) { return H.key[l * NI + i0 + i]; };
    auto dw_at = [&](int64_t i, int l) { return H.w[(l + 1) * NI + i0 + i] - H.w[l * NI + i0 + i]; };

    // ---- 1. coarse bucket of the split
    const unsigned long long *hw0 = hist_w + (size_t)r * kCoarseBins;
    const bool has_split = block_find_crossing(
        kCoarseBins, target, [&](int b) { return (int64_t)hw0[b]; }, sc, &s_bin, &s_above, &s_total);
    int64_t res = 0;   // capacity left for the increments at or below the current prefix
    if (has_split) {
        uint64_t prefix = (uint64_t)s_bin;
        int pbits = 16;
        res = target - s_above;
        unsigned count = hist_n[(size_t)r * kCoarseBins + s_bin];
        uint64_t *fw = reinterpret_cast<uint64_t *>(smem);
        unsigned *fc = reinterpret_cast<unsigned *>(smem + kFineBins * sizeof(uint64_t));
        // ---- 2. the split key, kFineBits per pass
        while (pbits < 64) {
            __syncthreads();
            if (count == 1) {
                for (int64_t i = tid; i < M; i += kSolveThreads) {
                    const int n = nv[i];
#pragma unroll
                    for (int l = 0; l < kMaxVerts - 1; l++) {
                        if (l + 1 >= n) break;
                        const uint64_t k = key_at(i, l);
                        if ((k >> (64 - pbits)) == prefix) s_kstar = k;
                    }
                }
                __syncthreads();
                prefix = s_kstar;
                pbits = 64;
                break;
            }
            const int shift = 64 - pbits - kFineBits;
            for (int b = tid; b < kFineBins; b += kSolveThreads) {
                fw[b] = 0ull;
                fc[b] = 0u;
            }
            __syncthreads();
            for (int64_t i = tid; i < M; i += kSolveThreads) {
                const int n = nv[i];
#pragma unroll
                for (int l = 0; l < kMaxVerts - 1; l++) {
                    if (l + 1 >= n) break;
                    const uint64_t k = key_at(i, l);
                    if ((k >> (shift + kFineBits)) == prefix) {
                        const int b = (int)((k >> shift) & (kFineBins - 1));
                        atomicAdd(reinterpret_cast<unsigned long long *>(&fw[b]),
                                  (unsigned long long)dw_at(i, l));
                        atomicAdd(&fc[b], 1u);
                    }
                }
            }
            __syncthreads();
            block_find_crossing(
                kFineBins, res, [&](int b) { return (int64_t)fw[b]; }, sc, &s_bin, &s_above, &s_total);
            prefix = (prefix << kFineBits) | (uint64_t)s_bin;
            pbits += kFineBits;
            res -= s_above;
            count = fc[s_bin];
        }
        if (tid == 0) s_kstar = prefix;
    }
    if (tid == 0) {
        s_split_item = -1;
        s_split_level = 0;
    }
    __syncthreads();
    const uint64_t kstar = has_split ? s_kstar : 0ull;
    if (!has_split) res = target - s_total;   // every increment fits

    // ---- 3. ordered pass: whole increments above K*, ties in order, the split
    int64_t carry = 0, my_taken = 0;
    double d_split = 0.0;
    for (int64_t c0 = 0; c0 < M; c0 += kSolveThreads) {
        const int64_t i = c0 + tid;
        int lvl = 0, tfirst = -1, tcount = 0, n = 0;
        int64_t tsum = 0;
        if (i < M) {
            n = nv[i];
            if (!has_split) {
                lvl = n - 1;
            } else {
#pragma unroll
                for (int l = 0; l < kMaxVerts - 1; l++) {
                    if (l + 1 >= n) break;
                    const uint64_t k = key_at(i, l);
                    if (k > kstar) {
                        lvl = l + 1;
                    } else if (k == kstar) {
                        if (tfirst < 0) tfirst = l;
                        tcount++;
                        tsum += dw_at(i, l);
                    }
                }
            }
        }
        int64_t ctot;
        const int64_t incl = block_incl_scan(tsum, sc, ctot);
        int64_t pb = carry + (incl - tsum);   // tie rate before this item's first tie
        for (int q = 0; q < tcount; q++) {
            const int l = tfirst + q;
            const int64_t dw = dw_at(i, l);
            if (pb + dw <= res) {
                lvl = l + 1;
                my_taken += dw;
            } else if (pb <= res) {
                s_split_item = i;
                s_split_level = l;
            }
            pb += dw;
        }
        carry += ctot;
        double v = 0.0;
        if (i < M) {
            level[i] = (uint8_t)lvl;
            v = H.d[lvl * NI + i0 + i];
        }
        const double t = block_tree_sum(v, sc);
        if (tid == 0) d_split = d_split + t;
    }
    const int64_t taken_ties = block_sum_i64(my_taken, sc);
    int64_t rem = res - taken_ties;
    double lp = d_split;
    const int64_t si = s_split_item;
    if (si >= 0) {
        const int sl = s_split_level;
        const double frac = (double)rem / (double)dw_at(si, sl);
        const double dd = H.d[sl * NI + i0 + si] - H.d[(sl + 1) * NI + i0 + si];
        if (frac > 0) lp = lp - frac * dd;
    }

    // ---- 4. greedy completion
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
        for (int64_t i = tid; i < M; i += kSolveThreads) {
            const int lvl = level[i];
            if (lvl + 1 >= nv[i]) continue;
            IncPos c;
            c.key = key_at(i, lvl);
            c.item = i;
            c.level = lvl;
            if (last.item >= 0 && !inc_first(last, c)) continue;   // passed over already
            if (dw_at(i, lvl) > rem) continue;
            if (inc_first(c, best)) best = c;
        }
        const IncPos f = block_first(best, s_warp, &s_first);
        if (f.item < 0) break;
        if (tid == 0) level[f.item] = (uint8_t)(f.level + 1);
        rem -= dw_at(f.item, f.level);
        last = f;
        takes++;
        __syncthreads();
    }

    // ---- 5. choice and final loss
    double obj = 0.0;
    uint8_t *choice = choice_all + (int64_t)P.budget * NI + i0;
    for (int64_t c0 = 0; c0 < M; c0 += kSolveThreads) {
        const int64_t i = c0 + tid;
        double v = 0.0;
        if (i < M) {
            const int lvl = level[i];
            choice[i] = (uint8_t)H.opt[lvl * NI + i0 + i];
            v = H.d[lvl * NI + i0 + i];
        }
        const double t = block_tree_sum(v, sc);
        if (tid == 0) obj = obj + t;
    }
    if (tid == 0) {
        out.status = 0;
        out.takes = takes;
        out.objective = obj;
        out.bytes = units_to_bytes(W0 + (target - rem), P.fixed);
        out.lp = lp;
        pout[blockIdx.x] = out;
    }
}

constexpr size_t kSolveSmem = kFineBins * (sizeof(uint64_t) + sizeof(unsigned));   // fine histogram

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
    const size_t o_pin = take(sizeof(ProblemIn) * P);
    const size_t o_pout = take(sizeof(ProblemOut) * P);
    const size_t o_level = take((size_t)n_budgets * NI);
    const size_t o_choice = take((size_t)n_budgets * NI);
    char *ws = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&ws), off, st);
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
    MGS_CUDA_TRY(cudaMemcpyAsync(ws + o_bits, grid->bits, sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st));
    MGS_CUDA_TRY(cudaMemcpyAsync(ws + o_ib, layout->item_begin, sizeof(int64_t) * (nr + 1),
                                 cudaMemcpyHostToDevice, st));
    MGS_CUDA_TRY(cudaMemcpyAsync(ws + o_pin, pin.data(), sizeof(ProblemIn) * P, cudaMemcpyHostToDevice, st));

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
    MGS_CUDA_TRY(cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveSmem));
    k_solve<<<P, kSolveThreads, kSolveSmem, st>>>(H, reinterpret_cast<const ProblemIn *>(ws + o_pin),
                                                  reinterpret_cast<ProblemOut *>(ws + o_pout), d_ib, sums,
                                                  hw, hn, reinterpret_cast<uint8_t *>(ws + o_level),
                                                  reinterpret_cast<uint8_t *>(ws + o_choice));
    MGS_CUDA_TRY(cudaGetLastError());
    count_launches(2);
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
