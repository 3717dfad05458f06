// Size estimate and bit-width 0-1 ILP over a host cost table (host C++).
//
// Eq. (eq:ilp), Sec. III-F: per (channel, block) item pick one bit-width,
// minimise the summed loss Omega subject to the estimated size <= budget, a
// multiple-choice knapsack per reserve ratio.  The arithmetic (integer rates,
// hulls, increment order, LP split, greedy completion, tree sums) is defined
// in solve_def.h and shared with the device solver.  Here the LP split is
// found by a weighted radix selection on the increment keys: one histogram
// pass over the top 16 bits, then a sort of the boundary bucket only.
// Alg. 1 then picks tau from the per-ratio results (see mgs_solve_budgets).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <queue>
#include <thread>
#include <vector>

#include "internal.h"
#include "solve_def.h"

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

inline double dist(const View &v, int64_t item, int k) {
    int64_t i = item * v.n_b + k;
    switch (v.norm) {
        case MGS_NORM_L2: return std::sqrt(v.sse[i]);
        case MGS_NORM_L1: return v.l1[i];
        case MGS_NORM_LINF: return (double)v.linf[i];
        default: return v.sse[i];
    }
}

// Lower convex hulls of every item, item-major at a stride of n_b vertices.
struct Hulls {
    int nb = 0;
    std::vector<uint8_t> nv;     // vertices per item
    std::vector<int8_t> opt;     // option index of each vertex
    std::vector<int64_t> w;      // rate of each vertex (2^-22 bit units)
    std::vector<double> d;       // loss of each vertex
    std::vector<uint64_t> key;   // key of increment l (vertex l -> l + 1)
    std::vector<int64_t> wtop;   // rate of the top bit-width option
};

void hull_item(const View &v, int64_t item, Hulls &H) {
    const int nb = v.n_b;
    int64_t w[MGS_MAX_OPTIONS] = {};
    double d[MGS_MAX_OPTIONS] = {};
    for (int k = 0; k < nb; k++) {
        w[k] = rate_units(v.rate_model, v.hbits[item * nb + k], v.cnt[item], v.bits[k]);
        d[k] = dist(v, item, k);
    }
    const int64_t b = item * nb;
    const int n = build_hull(w, d, nb, &H.opt[b], &H.w[b], &H.d[b]);
    H.nv[item] = (uint8_t)n;
    H.wtop[item] = w[nb - 1];
    for (int l = 0; l + 1 < n; l++) H.key[b + l] = inc_key(H.d[b + l] - H.d[b + l + 1], H.w[b + l + 1] - H.w[b + l]);
}

// Chunked pairwise sum in item order (the tree of solve_def.h).
inline double tree32(double *v) {
    for (int off = 16; off > 0; off >>= 1)
        for (int l = 0; l < off; l++) v[l] = v[l] + v[l + off];
    return v[0];
}
template <typename F>
double tree_sum(int64_t n, F x) {
    double s = 0.0;
    for (int64_t c0 = 0; c0 < n; c0 += kTreeChunk) {
        double part[32];
        for (int wp = 0; wp < 32; wp++) {
            double v[32];
            for (int l = 0; l < 32; l++) {
                const int64_t i = c0 + wp * 32 + l;
                v[l] = i < n ? x(i) : 0.0;
            }
            part[wp] = tree32(v);
        }
        s = s + tree32(part);
    }
    return s;
}

struct RatioResult {
    int status = -1;   // 0 solved, 1 skipped, -1 infeasible
    double objective = 0, bytes = 0, lp = 0, bytes_min = 0, bytes_top = 0;
    std::vector<uint8_t> choice;
};

// An increment in the solve order: larger key first, then item, then level.
struct IncRef {
    uint64_t key;
    int32_t item;
    int32_t level;
};
inline bool inc_before(const IncRef &a, const IncRef &b) {
    if (a.key != b.key) return a.key > b.key;
    if (a.item != b.item) return a.item < b.item;
    return a.level < b.level;
}

void solve_ratio(const Hulls &H, int64_t i0, int64_t M, double budget, const mgs_solve_opts *o,
                 RatioResult *res) {
    const int nb = H.nb;
    const double fixed = o->meta_bytes_per_group * (double)M + o->const_bytes + o->delta_bytes;
    int64_t W0 = 0, Wtop = 0;
    for (int64_t i = 0; i < M; i++) {
        W0 += H.w[(i0 + i) * nb];
        Wtop += H.wtop[i0 + i];
    }
    res->bytes_min = units_to_bytes(W0, fixed);
    res->bytes_top = units_to_bytes(Wtop, fixed);
    const int64_t cap = capacity_units(budget, fixed);
    if (cap < 0 || W0 > cap) {
        res->status = -1;
        return;
    }
    const int64_t target = cap - W0;
    auto dw_of = [&](int64_t i, int l) { return H.w[(i0 + i) * nb + l + 1] - H.w[(i0 + i) * nb + l]; };
    // LP split.  Pass 1: rate per bucket of the top 16 key bits; buckets above
    // the boundary are taken whole.
    static thread_local std::vector<int64_t> hist;
    hist.assign(1 << 16, 0);
    for (int64_t i = 0; i < M; i++) {
        const int64_t b = (i0 + i) * nb;
        for (int l = 0; l + 1 < H.nv[i0 + i]; l++) hist[H.key[b + l] >> 48] += dw_of(i, l);
    }
    int64_t taken = 0;
    int boundary = -1;
    for (int bk = (1 << 16) - 1; bk >= 0; bk--) {
        if (taken + hist[bk] <= target) {
            taken += hist[bk];
        } else {
            boundary = bk;
            break;
        }
    }
    static thread_local std::vector<int32_t> level;
    static thread_local std::vector<IncRef> edge;
    level.assign(M, 0);
    edge.clear();
    for (int64_t i = 0; i < M; i++) {
        const int64_t b = (i0 + i) * nb;
        for (int l = 0; l + 1 < H.nv[i0 + i]; l++) {
            const int bk = (int)(H.key[b + l] >> 48);
            if (bk > boundary) level[i] = l + 1;   // keys fall along an item's levels
            else if (bk == boundary) edge.push_back(IncRef{H.key[b + l], (int32_t)i, l});
        }
    }
    // pass 2: the boundary bucket in full order, up to the split
    std::sort(edge.begin(), edge.end(), inc_before);
    int64_t split_item = -1;
    int split_level = 0;
    for (const IncRef &e : edge) {
        const int64_t dw = dw_of(e.item, e.level);
        if (taken + dw > target) {
            split_item = e.item;
            split_level = e.level;
            break;
        }
        taken += dw;
        level[e.item] = e.level + 1;
    }
    const double d_split = tree_sum(M, [&](int64_t i) { return H.d[(i0 + i) * nb + level[i]]; });
    double lp = d_split;
    if (split_item >= 0) {
        const int64_t b = (i0 + split_item) * nb + split_level;
        const double frac = (double)(target - taken) / (double)(H.w[b + 1] - H.w[b]);
        if (frac > 0) lp = lp - frac * (H.d[b] - H.d[b + 1]);
    }
    // greedy completion, one take at a time: the first increment in solve order
    // after the last one taken that is its item's next increment and fits
    int64_t rem = target - taken;
    IncRef last{0, -1, 0};
    while (true) {
        IncRef best{0, -1, 0};
        for (int64_t i = 0; i < M; i++) {
            const int l = level[i];
            if (l + 1 >= H.nv[i0 + i]) continue;
            const IncRef c{H.key[(i0 + i) * nb + l], (int32_t)i, l};
            if (last.item >= 0 && !inc_before(last, c)) continue;   // passed over already
            if (dw_of(i, l) > rem) continue;
            if (best.item < 0 || inc_before(c, best)) best = c;
        }
        if (best.item < 0) break;
        rem -= dw_of(best.item, best.level);
        level[best.item]++;
        last = best;
    }
    res->status = 0;
    res->objective = tree_sum(M, [&](int64_t i) { return H.d[(i0 + i) * nb + level[i]]; });
    res->bytes = units_to_bytes(W0 + (target - rem), fixed);
    res->lp = lp;
    res->choice.resize(M);
    for (int64_t i = 0; i < M; i++) res->choice[i] = (uint8_t)H.opt[(i0 + i) * nb + level[i]];
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
    int64_t units = 0;
    for (int64_t i = b; i < e; i++) {
        int k = choice[i - b];
        if (k >= v.n_b) {
            set_error("choice[%lld] = %d outside the %d options", (long long)(i - b), k, v.n_b);
            return MGS_ERR_INVALID_ARG;
        }
        units += rate_units(v.rate_model, v.hbits[i * v.n_b + k], v.cnt[i], v.bits[k]);
    }
    *bytes_out = units_to_bytes(units, opts->meta_bytes_per_group * (double)(e - b) +
                                           opts->const_bytes + opts->delta_bytes);
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
    H.nb = v.n_b;
    H.nv.resize(n_items);
    H.opt.resize((size_t)n_items * H.nb);
    H.w.resize((size_t)n_items * H.nb);
    H.d.resize((size_t)n_items * H.nb);
    H.key.resize((size_t)n_items * H.nb);
    H.wtop.resize(n_items);
    parallel_for(n_items, 4096, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; i++) hull_item(v, i, H);
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

// Sec. III-F "Hierarchical Solver": per ratio, (1) one width per channel from
// the MCKP over channels (each channel an item whose options sum its groups'
// loss and rate), (2) the channel budgets S_c = A Q_c / sum Q_c of the bytes A
// left after C and S_Delta, (3) per channel the MCKP over its groups within
// S_c.  Every sub-problem is the flat solver's.  tau as in mgs_solve_budgets.
mgs_status mgs_solve_hierarchical(const void *table, const mgs_table_layout *layout,
                                  const mgs_grid *grid, double budget_bytes,
                                  const mgs_solve_opts *opts, mgs_solution *out) {
    clear_error();
    if (!table || !layout || !grid || !opts || !out) {
        set_error("table, layout, grid, opts and out must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (grid->n_bits != layout->n_bits || grid->n_ratios != layout->n_ratios ||
        opts->rate_model < 0 || opts->rate_model > 1 || opts->norm < 0 || opts->norm > 3 ||
        !(budget_bytes >= 0) || layout->n_channels < 1) {
        set_error("grid/layout mismatch, bad options or budget");
        return MGS_ERR_INVALID_ARG;
    }
    const View v = make_view(table, layout, grid, opts);
    const int nr = layout->n_ratios, nb = layout->n_bits, C = layout->n_channels;
    struct Res {
        int status = -1;
        double objective = 0, bytes = 0, lp = 0, bytes_top = 0;
        std::vector<uint8_t> choice;
    };
    std::vector<Res> res(nr);
    for (int r = 0; r < nr; r++) {
        const int64_t ng = layout->n_groups[r], ib = layout->item_begin[r];
        Res &R = res[r];
        // all-top size, for the tau rule
        int64_t top_units = 0;
        for (int64_t i = ib; i < ib + C * ng; i++)
            top_units += rate_units(v.rate_model, v.hbits[i * nb + nb - 1], v.cnt[i], v.bits[nb - 1]);
        R.bytes_top = units_to_bytes(top_units, opts->meta_bytes_per_group * (double)(C * ng) +
                                                    opts->const_bytes + opts->delta_bytes);
        // (1) channel level: a table of C items
        int64_t one = 1;
        mgs_grid g1 = *grid;
        g1.n_ratios = 1;
        g1.keep = &one;
        g1.group_size = 1;
        mgs_table_layout l1;
        MGS_TRY(mgs_table_layout_for(1, C, &g1, &l1));
        std::vector<unsigned char> buf((size_t)l1.total_bytes, 0);
        double *csse = reinterpret_cast<double *>(buf.data() + l1.off_sse);
        double *chb = reinterpret_cast<double *>(buf.data() + l1.off_hbits);
        int32_t *ccnt = reinterpret_cast<int32_t *>(buf.data() + l1.off_count);
        for (int c = 0; c < C; c++) {
            int64_t n_c = 0;
            for (int64_t g = 0; g < ng; g++) {
                const int64_t it = ib + c * ng + g;
                n_c += v.cnt[it];
                for (int k = 0; k < nb; k++) {
                    csse[c * nb + k] += dist(v, it, k);
                    chb[c * nb + k] += v.hbits[it * nb + k];
                }
            }
            ccnt[c] = (int32_t)n_c;
        }
        mgs_solve_opts o1 = *opts;
        o1.norm = MGS_NORM_SSE;   // the channel items carry the chosen norm's sums
        o1.meta_bytes_per_group = opts->meta_bytes_per_group * (double)ng;
        std::vector<uint8_t> qc((size_t)C);
        mgs_solution s1{};
        s1.choice = qc.data();
        mgs_status st = mgs_solve_budgets(buf.data(), &l1, &g1, 1, &budget_bytes, &o1, &s1);
        if (st == MGS_ERR_INFEASIBLE || s1.r_index < 0) continue;
        MGS_TRY(st);
        // (2) channel budgets
        double qsum = 0;
        for (int c = 0; c < C; c++) qsum += grid->bits[qc[c]];
        const double A = budget_bytes - opts->const_bytes - opts->delta_bytes;
        // (3) group level per channel
        R.choice.assign((size_t)(C * ng), 0);
        bool ok = true;
        int64_t keep_r = grid->keep[r];
        for (int c = 0; c < C && ok; c++) {
            mgs_table_layout lv = *layout;
            const int64_t base = ib + c * ng;
            lv.n_ratios = 1;
            lv.n_channels = 1;
            lv.n_items = ng;
            lv.item_begin[0] = 0;
            lv.item_begin[1] = ng;
            lv.n_groups[0] = ng;
            lv.off_sse += 8 * base * nb;
            lv.off_l1 += 8 * base * nb;
            lv.off_hbits += 8 * base * nb;
            lv.off_linf += 4 * base * nb;
            lv.off_count += 4 * base;
            lv.off_vmin += 4 * base;
            lv.off_vmax += 4 * base;
            mgs_grid gv = *grid;
            gv.n_ratios = 1;
            gv.keep = &keep_r;
            mgs_solve_opts o2 = *opts;
            o2.const_bytes = 0;
            o2.delta_bytes = 0;
            const double S_c = A * (double)grid->bits[qc[c]] / qsum;
            mgs_solution s2{};
            s2.choice = R.choice.data() + c * ng;
            st = mgs_solve_budgets(table, &lv, &gv, 1, &S_c, &o2, &s2);
            if (st == MGS_ERR_INFEASIBLE || s2.r_index < 0) {
                ok = false;
                break;
            }
            MGS_TRY(st);
            R.objective += s2.objective;
            R.bytes += s2.est_bytes;
            R.lp += s2.lp_bound;
        }
        clear_error();
        if (!ok) {
            R.choice.clear();
            R.objective = R.bytes = R.lp = 0;
            continue;
        }
        R.bytes += opts->const_bytes + opts->delta_bytes;
        R.status = 0;
    }
    // tau rule (Alg. 1), as in mgs_solve_budgets
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
        out->est_bytes = out->objective = out->lp_bound = 0;
        set_error("no ratio fits a budget of %.0f bytes", budget_bytes);
        return MGS_ERR_INFEASIBLE;
    }
    out->est_bytes = res[best].bytes;
    out->objective = res[best].objective;
    out->lp_bound = res[best].lp;
    if (out->choice) std::memcpy(out->choice, res[best].choice.data(), res[best].choice.size());
    return MGS_OK;
}

}  // extern "C"
