// Size estimate and bit-width 0-1 ILP over a cost table (host C++).
//
// Eq. (eq:ilp), Sec. III-F: per (channel, block) item pick one bit-width,
// minimise sum of the loss Omega subject to the estimated size <= budget.
// That is a multiple-choice knapsack.  Per ratio:
//   1. every item's options are reduced to their lower convex hull in the
//      (rate, distortion) plane; the LP relaxation takes hull increments in
//      order of decreasing efficiency -dD/dRate until the capacity is used
//      (a weighted radix selection on the efficiency's bit pattern: one
//      histogram pass, then a full sort of the boundary bucket only);
//   2. the integral answer keeps the increments that fit completely and then
//      greedily adds further whole increments that still fit;
//   3. the LP value (with the fractional split increment) is a lower bound.
// Alg. 1 then picks tau from the per-ratio results (see mgs_solve_budget).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <queue>
#include <thread>
#include <vector>

#include "internal.h"

namespace mgs {
namespace {

struct View {
    const double *sse, *l1, *hbits;
    const float *linf;
    const int32_t *cnt;
    int n_b;
    const int32_t *bits;
    int rate_model, norm;
};

View make_view(const void *table, const mgs_table_layout *L, const mgs_grid *grid,
               const mgs_solve_opts *o) {
    const char *b = static_cast<const char *>(table);
    View v;
    v.sse = reinterpret_cast<const double *>(b + L->off_sse);
    v.l1 = reinterpret_cast<const double *>(b + L->off_l1);
    v.hbits = reinterpret_cast<const double *>(b + L->off_hbits);
    v.linf = reinterpret_cast<const float *>(b + L->off_linf);
    v.cnt = reinterpret_cast<const int32_t *>(b + L->off_count);
    v.n_b = L->n_bits;
    v.bits = grid->bits;
    v.rate_model = o->rate_model;
    v.norm = o->norm;
    return v;
}

inline double rate_bits(const View &v, int64_t item, int k) {
    if (v.rate_model == MGS_RATE_FIXED) return (double)v.cnt[item] * v.bits[k];
    return v.hbits[item * v.n_b + k];
}
inline double dist(const View &v, int64_t item, int k) {
    int64_t i = item * v.n_b + k;
    switch (v.norm) {
        case MGS_NORM_L2: return std::sqrt(v.sse[i]);
        case MGS_NORM_L1: return v.l1[i];
        case MGS_NORM_LINF: return (double)v.linf[i];
        default: return v.sse[i];
    }
}

// Hull increments of every item, at a fixed stride of (n_b - 1) slots per item.
struct Hulls {
    int stride = 0;
    std::vector<double> eff, dw, dd;   // [item * stride + level]
    std::vector<int8_t> to;            // option reached by the increment
    std::vector<int8_t> len;           // increments per item
    std::vector<int8_t> start;         // first hull option per item
    std::vector<double> w0, d0, wtop;  // per item: start rate/distortion, top-bit-width rate
};

// Lower convex hull of one item's (rate, distortion) options.
void build_hull(const View &v, int64_t item, int64_t slot, Hulls &H) {
    const int nb = v.n_b;
    double w[MGS_MAX_OPTIONS], d[MGS_MAX_OPTIONS];
    int ord[MGS_MAX_OPTIONS], hull[MGS_MAX_OPTIONS];
    for (int k = 0; k < nb; k++) {
        w[k] = rate_bits(v, item, k);
        d[k] = dist(v, item, k);
        ord[k] = k;
    }
    // insertion sort by (rate, distortion, index): the options usually arrive sorted
    for (int i = 1; i < nb; i++) {
        int x = ord[i], j = i - 1;
        while (j >= 0 && (w[ord[j]] > w[x] || (w[ord[j]] == w[x] && (d[ord[j]] > d[x] ||
                                                                     (d[ord[j]] == d[x] && ord[j] > x))))) {
            ord[j + 1] = ord[j];
            j--;
        }
        ord[j + 1] = x;
    }
    int h = 0;
    for (int t = 0; t < nb; t++) {
        const int k = ord[t];
        if (h > 0 && (d[k] >= d[hull[h - 1]] || w[k] == w[hull[h - 1]])) continue;   // dominated
        while (h >= 2) {
            const int a = hull[h - 2], b = hull[h - 1];
            if ((d[b] - d[a]) * (w[k] - w[a]) >= (d[k] - d[a]) * (w[b] - w[a])) h--;
            else break;
        }
        hull[h++] = k;
    }
    H.start[slot] = (int8_t)hull[0];
    H.w0[slot] = w[hull[0]];
    H.d0[slot] = d[hull[0]];
    H.wtop[slot] = w[nb - 1];
    H.len[slot] = (int8_t)(h - 1);
    const int64_t base = slot * H.stride;
    for (int i = 0; i + 1 < h; i++) {
        const int a = hull[i], b = hull[i + 1];
        H.dw[base + i] = w[b] - w[a];
        H.dd[base + i] = d[a] - d[b];
        H.eff[base + i] = H.dd[base + i] / H.dw[base + i];
        H.to[base + i] = (int8_t)b;
    }
}

struct RatioResult {
    int status = -1;   // 0 solved, 1 skipped, -1 infeasible
    double objective = 0, bytes = 0, lp = 0, bytes_min = 0, bytes_top = 0;
    std::vector<uint8_t> choice;
};

// Order of increments: larger efficiency first, then item, then hull level.
struct IncRef {
    double eff;
    int32_t item;
    int32_t level;
};
inline bool inc_before(const IncRef &a, const IncRef &b) {
    if (a.eff != b.eff) return a.eff > b.eff;
    if (a.item != b.item) return a.item < b.item;
    return a.level < b.level;
}

// Non-negative doubles order like their bit patterns.
inline uint64_t eff_key(double e) {
    uint64_t u;
    std::memcpy(&u, &e, 8);
    return u;
}

void solve_ratio(const Hulls &H, int64_t slot0, int64_t M, double budget, const mgs_solve_opts *o,
                 RatioResult *res) {
    const int S = H.stride;
    const double fixed_bytes = o->meta_bytes_per_group * (double)M + o->const_bytes + o->delta_bytes;
    const double cap = 8.0 * (budget - fixed_bytes);   // capacity in bits
    double w0 = 0, d0 = 0, wtop = 0;
    for (int64_t i = 0; i < M; i++) {
        w0 += H.w0[slot0 + i];
        d0 += H.d0[slot0 + i];
        wtop += H.wtop[slot0 + i];
    }
    res->bytes_min = w0 / 8.0 + fixed_bytes;
    res->bytes_top = wtop / 8.0 + fixed_bytes;
    if (cap < 0 || w0 > cap) {
        res->status = -1;
        return;
    }
    const double target = cap - w0;
    // pass 1: rate histogram over the top 16 bits of the efficiency key
    static thread_local std::vector<double> hist;
    hist.assign(1 << 16, 0.0);
    for (int64_t i = 0; i < M; i++) {
        const int64_t base = (slot0 + i) * S;
        for (int l = 0; l < H.len[slot0 + i]; l++) hist[eff_key(H.eff[base + l]) >> 48] += H.dw[base + l];
    }
    // buckets above the boundary are taken whole
    double taken = 0;
    int boundary = -1;
    for (int bk = (1 << 16) - 1; bk >= 0; bk--) {
        if (taken + hist[bk] <= target) {
            taken += hist[bk];
        } else {
            boundary = bk;
            break;
        }
    }
    std::vector<int16_t> level(M, 0);
    std::vector<uint8_t> cur(M);
    double D = d0, W = w0, lp;
    for (int64_t i = 0; i < M; i++) cur[i] = (uint8_t)H.start[slot0 + i];
    std::vector<IncRef> edge;
    for (int64_t i = 0; i < M; i++) {
        const int64_t base = (slot0 + i) * S;
        for (int l = 0; l < H.len[slot0 + i]; l++) {
            const int bk = (int)(eff_key(H.eff[base + l]) >> 48);
            if (bk > boundary) {
                // whole bucket taken: the item's earlier levels are in higher buckets too
                level[i] = (int16_t)(l + 1);
                cur[i] = (uint8_t)H.to[base + l];
                D -= H.dd[base + l];
                W += H.dw[base + l];
            } else if (bk == boundary) {
                edge.push_back(IncRef{H.eff[base + l], (int32_t)i, l});
            }
        }
    }
    // pass 2: the boundary bucket in full order
    std::sort(edge.begin(), edge.end(), inc_before);
    size_t split = 0;
    while (split < edge.size()) {
        const IncRef &e = edge[split];
        const int64_t at = (slot0 + e.item) * S + e.level;
        if (taken + H.dw[at] > target) break;
        taken += H.dw[at];
        level[e.item] = (int16_t)(e.level + 1);
        cur[e.item] = (uint8_t)H.to[at];
        D -= H.dd[at];
        W += H.dw[at];
        split++;
    }
    lp = D;
    if (split < edge.size()) {
        const int64_t at = (slot0 + edge[split].item) * S + edge[split].level;
        const double frac = (target - taken) / H.dw[at];
        if (frac > 0) lp -= frac * H.dd[at];
    }
    // greedy completion: whole next increments that still fit, best first
    struct Cand {
        double eff;
        int32_t item, level;
        bool operator<(const Cand &b) const {   // max-heap on the increment order
            return inc_before(IncRef{b.eff, b.item, b.level}, IncRef{eff, item, level});
        }
    };
    std::priority_queue<Cand> pq;
    double rem = cap - W;
    for (int64_t i = 0; i < M; i++) {
        const int l = level[i];
        if (l < H.len[slot0 + i]) {
            const int64_t at = (slot0 + i) * S + l;
            if (H.dw[at] <= rem) pq.push(Cand{H.eff[at], (int32_t)i, l});
        }
    }
    while (!pq.empty()) {
        const Cand c = pq.top();
        pq.pop();
        const int64_t at = (slot0 + c.item) * S + c.level;
        if (H.dw[at] > rem || level[c.item] != c.level) continue;
        cur[c.item] = (uint8_t)H.to[at];
        level[c.item]++;
        rem -= H.dw[at];
        W += H.dw[at];
        D -= H.dd[at];
        const int l = level[c.item];
        if (l < H.len[slot0 + c.item]) {
            const int64_t nx = (slot0 + c.item) * S + l;
            if (H.dw[nx] <= rem) pq.push(Cand{H.eff[nx], c.item, l});
        }
    }
    res->status = 0;
    res->objective = D;
    res->bytes = W / 8.0 + fixed_bytes;
    res->lp = lp;
    res->choice.assign(cur.begin(), cur.end());
}

template <typename F>
void parallel_for(int64_t n, int64_t grain, F fn) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t chunks = (n + grain - 1) / grain;
    const unsigned nt = (unsigned)std::min<int64_t>(hw, chunks);
    if (nt <= 1) {
        fn(0, n);
        return;
    }
    std::atomic<int64_t> next{0};
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; t++)
        th.emplace_back([&] {
            for (int64_t c; (c = next.fetch_add(1)) < chunks;) fn(c * grain, std::min(n, (c + 1) * grain));
        });
    for (auto &x : th) x.join();
}

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" {

mgs_status mgs_estimate_size(const void *table, const mgs_table_layout *layout,
                             const mgs_grid *grid, int32_t r_index, const uint8_t *choice,
                             const mgs_solve_opts *opts, double *bytes_out) {
    clear_error();
    if (!table || !layout || !grid || !choice || !opts || !bytes_out) {
        set_error("table, layout, grid, choice, opts and bytes_out must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (r_index < 0 || r_index >= layout->n_ratios || grid->n_bits != layout->n_bits) {
        set_error("r_index %d or grid does not match the layout", r_index);
        return MGS_ERR_INVALID_ARG;
    }
    View v = make_view(table, layout, grid, opts);
    int64_t b = layout->item_begin[r_index], e = layout->item_begin[r_index + 1];
    double bits = 0;
    for (int64_t i = b; i < e; i++) {
        int k = choice[i - b];
        if (k >= v.n_b) {
            set_error("choice[%lld] = %d outside the %d options", (long long)(i - b), k, v.n_b);
            return MGS_ERR_INVALID_ARG;
        }
        bits += rate_bits(v, i, k);
    }
    *bytes_out = bits / 8.0 + opts->meta_bytes_per_group * (double)(e - b) + opts->const_bytes +
                 opts->delta_bytes;
    return MGS_OK;
}

mgs_status mgs_solve_budgets(const void *table, const mgs_table_layout *layout,
                             const mgs_grid *grid, int32_t n_budgets, const double *budgets,
                             const mgs_solve_opts *opts, mgs_solution *out) {
    clear_error();
    if (!table || !layout || !grid || !opts || !out || !budgets || n_budgets < 1) {
        set_error("table, layout, grid, budgets, opts and out must be non-NULL; n_budgets >= 1");
        return MGS_ERR_INVALID_ARG;
    }
    if (grid->n_bits != layout->n_bits || grid->n_ratios != layout->n_ratios ||
        opts->rate_model < 0 || opts->rate_model > 1 || opts->norm < 0 || opts->norm > 3) {
        set_error("grid/layout mismatch or bad options");
        return MGS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n_budgets; i++)
        if (!(budgets[i] >= 0)) {
            set_error("budget %d is negative or NaN", i);
            return MGS_ERR_INVALID_ARG;
        }
    View v = make_view(table, layout, grid, opts);
    const int nr = layout->n_ratios;
    const int64_t n_items = layout->item_begin[nr];
    static thread_local Hulls H_tls;   // capacity persists across calls (no page faults per solve)
    Hulls &H = H_tls;                  // the caller's instance, shared with the worker threads
    H.stride = std::max(1, v.n_b - 1);
    H.eff.resize((size_t)n_items * H.stride);
    H.dw.resize((size_t)n_items * H.stride);
    H.dd.resize((size_t)n_items * H.stride);
    H.to.resize((size_t)n_items * H.stride);
    H.len.resize(n_items);
    H.start.resize(n_items);
    H.w0.resize(n_items);
    H.d0.resize(n_items);
    H.wtop.resize(n_items);
    parallel_for(n_items, 4096, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; i++) build_hull(v, i, i, H);
    });
    // every (budget, ratio) pair is independent once the hulls exist
    std::vector<RatioResult> res((size_t)n_budgets * nr);
    parallel_for((int64_t)n_budgets * nr, 1, [&](int64_t lo, int64_t hi) {
        for (int64_t t = lo; t < hi; t++) {
            const int bi = (int)(t / nr), r = (int)(t % nr);
            solve_ratio(H, layout->item_begin[r], layout->item_begin[r + 1] - layout->item_begin[r],
                        budgets[bi], opts, &res[t]);
        }
    });
    mgs_status worst = MGS_OK;
    for (int bi = 0; bi < n_budgets; bi++) {
        RatioResult *rr = &res[(size_t)bi * nr];
        mgs_solution *o = &out[bi];
        // tau rule (Alg. 1): skip ratios whose all-top size stays under the budget
        int best = -1, largest_feasible = -1;
        for (int r = 0; r < nr; r++) {
            if (rr[r].status < 0) continue;
            largest_feasible = r;
            if (rr[r].bytes_top < budgets[bi]) {
                rr[r].status = 1;
                continue;
            }
            if (best < 0 || rr[r].objective <= rr[best].objective) best = r;
        }
        if (best < 0) best = largest_feasible;
        for (int r = 0; r < nr; r++) {
            if (o->ratio_status) o->ratio_status[r] = rr[r].status;
            if (o->ratio_objective) o->ratio_objective[r] = rr[r].objective;
            if (o->ratio_bytes) o->ratio_bytes[r] = rr[r].bytes;
            if (o->ratio_lp_bound) o->ratio_lp_bound[r] = rr[r].lp;
        }
        o->r_index = best;
        if (best < 0) {
            o->est_bytes = 0;
            o->objective = 0;
            o->lp_bound = 0;
            set_error("no ratio fits a budget of %.0f bytes", budgets[bi]);
            worst = MGS_ERR_INFEASIBLE;
            continue;
        }
        o->est_bytes = rr[best].bytes;
        o->objective = rr[best].objective;
        o->lp_bound = rr[best].lp;
        if (o->choice) std::memcpy(o->choice, rr[best].choice.data(), rr[best].choice.size());
    }
    return worst;
}

mgs_status mgs_solve_budget(const void *table, const mgs_table_layout *layout,
                            const mgs_grid *grid, double budget_bytes, const mgs_solve_opts *opts,
                            mgs_solution *out) {
    return mgs_solve_budgets(table, layout, grid, 1, &budget_bytes, opts, out);
}

}  // extern "C"
