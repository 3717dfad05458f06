// Size estimate and bit-width 0-1 ILP over a cost table (host C++).
//
// Eq. (eq:ilp), Sec. III-F: per (channel, block) item pick one bit-width,
// minimise sum of the loss Omega subject to the estimated size <= budget.
// That is a multiple-choice knapsack.  Per ratio:
//   1. every item's options are reduced to their lower convex hull in the
//      (rate, distortion) plane; the LP relaxation takes hull increments in
//      order of decreasing efficiency -dD/dRate until the capacity is used
//      (a weighted selection, expected linear time);
//   2. the integral answer keeps the increments that fit completely and then
//      greedily adds further whole increments that still fit;
//   3. the LP value (with the fractional split increment) is a lower bound.
// Alg. 1 then picks tau from the per-ratio results (see mgs_solve_budget).
#include <algorithm>
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

struct Inc {
    double eff;    // -dD / dW
    double dw;     // rate increase (bits)
    double dd;     // distortion decrease (>= 0)
    int32_t item;  // item index within the ratio
    int16_t level; // position on the item's hull (increment from level to level + 1)
    int16_t to;    // option index reached
};

inline bool before(const Inc &a, const Inc &b) {   // strict total order, best first
    if (a.eff != b.eff) return a.eff > b.eff;
    if (a.item != b.item) return a.item < b.item;
    return a.level < b.level;
}

struct RatioResult {
    int status = -1;   // 0 solved, 1 skipped, -1 infeasible
    double objective = 0, bytes = 0, lp = 0, bytes_min = 0, bytes_top = 0;
    std::vector<uint8_t> choice;
};

void solve_ratio(const View &v, int64_t begin, int64_t end, double budget, const mgs_solve_opts *o,
                 RatioResult *res) {
    const int64_t M = end - begin;
    const int nb = v.n_b;
    const double fixed_bytes = o->meta_bytes_per_group * (double)M + o->const_bytes + o->delta_bytes;
    const double cap = 8.0 * (budget - fixed_bytes);   // capacity in bits
    std::vector<int16_t> start(M);
    std::vector<Inc> incs;
    incs.reserve((size_t)M * (nb > 1 ? nb - 1 : 1));
    double w0 = 0, d0 = 0, wtop = 0;
    std::vector<int> hull;
    hull.reserve(nb);
    std::vector<int> ord(nb);
    for (int64_t i = 0; i < M; i++) {
        const int64_t item = begin + i;
        wtop += rate_bits(v, item, nb - 1);
        // options sorted by (rate, distortion)
        for (int k = 0; k < nb; k++) ord[k] = k;
        std::sort(ord.begin(), ord.end(), [&](int a, int b) {
            double wa = rate_bits(v, item, a), wb = rate_bits(v, item, b);
            if (wa != wb) return wa < wb;
            double da = dist(v, item, a), db = dist(v, item, b);
            if (da != db) return da < db;
            return a < b;
        });
        // lower convex hull of the non-dominated options
        hull.clear();
        for (int t = 0; t < nb; t++) {
            int k = ord[t];
            double wk = rate_bits(v, item, k), dk = dist(v, item, k);
            if (!hull.empty() && dk >= dist(v, item, hull.back())) continue;   // dominated
            if (!hull.empty() && wk == rate_bits(v, item, hull.back())) continue;
            while (hull.size() >= 2) {
                int a = hull[hull.size() - 2], b = hull.back();
                double wa = rate_bits(v, item, a), da = dist(v, item, a);
                double wb = rate_bits(v, item, b), db = dist(v, item, b);
                // b is above or on segment a-k: remove
                double lhs = (db - da) * (wk - wa), rhs = (dk - da) * (wb - wa);
                if (lhs >= rhs) hull.pop_back(); else break;
            }
            hull.push_back(k);
        }
        start[i] = (int16_t)hull[0];
        w0 += rate_bits(v, item, hull[0]);
        d0 += dist(v, item, hull[0]);
        for (size_t h = 0; h + 1 < hull.size(); h++) {
            int a = hull[h], b = hull[h + 1];
            Inc in;
            in.dw = rate_bits(v, item, b) - rate_bits(v, item, a);
            in.dd = dist(v, item, a) - dist(v, item, b);
            in.eff = in.dd / in.dw;
            in.item = (int32_t)i;
            in.level = (int16_t)h;
            in.to = (int16_t)b;
            incs.push_back(in);
        }
    }
    res->bytes_min = w0 / 8.0 + fixed_bytes;
    res->bytes_top = wtop / 8.0 + fixed_bytes;
    if (cap < 0 || w0 > cap) {
        res->status = -1;
        return;
    }
    // weighted selection: the longest best-first prefix with total dw <= cap - w0
    const double target = cap - w0;
    size_t a = 0, b = incs.size();
    double taken = 0;
    while (b - a > 32) {
        // median-of-three pivot on the total order
        const Inc &x = incs[a], &y = incs[(a + b) / 2], &z = incs[b - 1];
        Inc piv = before(x, y) ? (before(y, z) ? y : (before(x, z) ? z : x))
                               : (before(x, z) ? x : (before(y, z) ? z : y));
        auto mid = std::partition(incs.begin() + a, incs.begin() + b,
                                  [&](const Inc &q) { return before(q, piv); });
        size_t m = (size_t)(mid - incs.begin());
        if (m == a) {   // pivot is the best of the range: take it alone
            auto it = std::min_element(incs.begin() + a, incs.begin() + b, before);
            std::iter_swap(incs.begin() + a, it);
            if (taken + incs[a].dw <= target) {
                taken += incs[a].dw;
                a++;
                continue;
            }
            b = a;
            break;
        }
        double wsum = 0;
        for (size_t t = a; t < m; t++) wsum += incs[t].dw;
        if (taken + wsum <= target) {
            taken += wsum;
            a = m;
        } else {
            b = m;
        }
    }
    std::sort(incs.begin() + a, incs.begin() + b, before);
    size_t split = a;
    while (split < b && taken + incs[split].dw <= target) taken += incs[split++].dw;
    // [0, split) are the taken increments; split (if < size) is the fractional one
    std::vector<int16_t> level(M, 0), cur(start);
    double D = d0, W = w0;
    for (size_t t = 0; t < split; t++) {
        // the taken increments of an item are its first levels, in any order here
        const Inc &in = incs[t];
        if (in.level + 1 > level[in.item]) {
            level[in.item] = (int16_t)(in.level + 1);
            cur[in.item] = in.to;
        }
        D -= in.dd;
        W += in.dw;
    }
    double lp = D;
    if (split < incs.size()) {
        // the split increment is the best remaining one in the total order
        size_t best = split;
        for (size_t t = split + 1; t < incs.size() && t < b; t++)
            if (before(incs[t], incs[best])) best = t;
        if (b < incs.size())
            for (size_t t = b; t < incs.size(); t++)
                if (before(incs[t], incs[best])) best = t;
        std::iter_swap(incs.begin() + split, incs.begin() + best);
        const Inc &in = incs[split];
        double frac = (target - taken) / in.dw;
        if (frac > 0) lp -= frac * in.dd;
    }
    // greedy completion: whole next-increments that still fit, best first
    {
        // the next increment of every item, keyed by (item, level)
        std::vector<int32_t> first_inc(M + 1, 0);
        std::vector<const Inc *> flat(incs.size());
        {
            std::vector<int32_t> count(M + 1, 0);
            for (const Inc &in : incs) count[in.item + 1]++;
            for (int64_t i = 0; i < M; i++) count[i + 1] += count[i];
            first_inc = count;
            std::vector<int32_t> fill(count.begin(), count.end() - 1);
            for (const Inc &in : incs) flat[fill[in.item]++] = &in;
            for (int64_t i = 0; i < M; i++)
                std::sort(flat.begin() + first_inc[i], flat.begin() + first_inc[i + 1],
                          [](const Inc *p, const Inc *q) { return p->level < q->level; });
        }
        auto next_of = [&](int64_t i) -> const Inc * {
            int32_t at = first_inc[i] + level[i];
            return at < first_inc[i + 1] ? flat[at] : nullptr;
        };
        auto cmp = [](const Inc *p, const Inc *q) { return before(*q, *p); };
        std::priority_queue<const Inc *, std::vector<const Inc *>, decltype(cmp)> pq(cmp);
        double rem = cap - W;
        for (int64_t i = 0; i < M; i++) {
            const Inc *nx = next_of(i);
            if (nx && nx->dw <= rem) pq.push(nx);
        }
        while (!pq.empty()) {
            const Inc *in = pq.top();
            pq.pop();
            if (in->dw > rem || level[in->item] != in->level) continue;
            cur[in->item] = in->to;
            level[in->item]++;
            rem -= in->dw;
            W += in->dw;
            D -= in->dd;
            const Inc *nx = next_of(in->item);
            if (nx && nx->dw <= rem) pq.push(nx);
        }
    }
    res->status = 0;
    res->objective = D;
    res->bytes = W / 8.0 + fixed_bytes;
    res->lp = lp;
    res->choice.assign(cur.begin(), cur.end());
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

mgs_status mgs_solve_budget(const void *table, const mgs_table_layout *layout,
                            const mgs_grid *grid, double budget_bytes, const mgs_solve_opts *opts,
                            mgs_solution *out) {
    clear_error();
    if (!table || !layout || !grid || !opts || !out) {
        set_error("table, layout, grid, opts and out must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (grid->n_bits != layout->n_bits || grid->n_ratios != layout->n_ratios ||
        opts->rate_model < 0 || opts->rate_model > 1 || opts->norm < 0 || opts->norm > 3 ||
        !(budget_bytes >= 0)) {
        set_error("grid/layout mismatch or bad options");
        return MGS_ERR_INVALID_ARG;
    }
    View v = make_view(table, layout, grid, opts);
    const int nr = layout->n_ratios;
    std::vector<RatioResult> res(nr);
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    unsigned nt = std::min<unsigned>(hw, (unsigned)nr);
    if (nt <= 1) {
        for (int r = 0; r < nr; r++)
            solve_ratio(v, layout->item_begin[r], layout->item_begin[r + 1], budget_bytes, opts,
                        &res[r]);
    } else {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; t++)
            th.emplace_back([&, t] {
                for (int r = (int)t; r < nr; r += (int)nt)
                    solve_ratio(v, layout->item_begin[r], layout->item_begin[r + 1], budget_bytes,
                                opts, &res[r]);
            });
        for (auto &x : th) x.join();
    }
    // tau rule (Alg. 1): skip ratios whose all-top size stays under the budget
    int best = -1, largest_feasible = -1;
    for (int r = 0; r < nr; r++) {
        if (res[r].status < 0) continue;
        largest_feasible = r;
        if (res[r].bytes_top < budget_bytes) {
            res[r].status = 1;
            continue;
        }
        if (best < 0 || res[r].objective <= res[best].objective) best = r;
    }
    if (best < 0) best = largest_feasible;
    for (int r = 0; r < nr; r++) {
        if (out->ratio_status) out->ratio_status[r] = res[r].status;
        if (out->ratio_objective) out->ratio_objective[r] = res[r].objective;
        if (out->ratio_bytes) out->ratio_bytes[r] = res[r].bytes;
        if (out->ratio_lp_bound) out->ratio_lp_bound[r] = res[r].lp;
    }
    out->r_index = best;
    if (best < 0) {
        out->est_bytes = 0;
        out->objective = 0;
        out->lp_bound = 0;
        set_error("no ratio fits a budget of %.0f bytes", budget_bytes);
        return MGS_ERR_INFEASIBLE;
    }
    out->est_bytes = res[best].bytes;
    out->objective = res[best].objective;
    out->lp_bound = res[best].lp;
    if (out->choice)
        std::memcpy(out->choice, res[best].choice.data(), res[best].choice.size());
    return MGS_OK;
}

}  // extern "C"
