// Alg. 1 with real compression: for every reserve ratio, compress at the
// initial width, skip the ratio when twice that size is still under the
// budget, then alternate the 0-1 ILP of Eq. (eq:ilp) -- sizes from the linear
// estimate of Eq. (eq:size_estim), S(Q) = sum P Q + C + S_Delta -- with a real
// compression of the chosen widths (mgs_encode_config's block coder), until
// the actual size S_a is within the tolerance of the budget.  S_Delta is the
// calibration offset that makes the estimate exact at the configuration just
// compressed: S_Delta = S_a - (estimate of that configuration without it).
// Among the ratios that converge, the smallest Omega wins (ties: larger ratio).
//
// Each ILP is the device solver on a one-ratio view of the cost table (same
// buffer, offsets moved to that ratio's items); each compression runs the
// quantiser and the block coder on the GPU with the scene's kept lists.  The
// ratios do not depend on one another until the final pick, so each runs its
// loop on a host thread with its own stream and buffers; every ratio's rounds
// are the same as when they run one after another.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using namespace mgs;

// The one-ratio view of a cost table.
void ratio_view(const mgs_table_layout &L, const mgs_grid &G, int r, mgs_table_layout *V,
                mgs_grid *VG, int64_t *keep_r) {
    *V = L;
    const int64_t ib = L.item_begin[r];
    const int64_t items = L.item_begin[r + 1] - ib;
    V->n_ratios = 1;
    V->n_items = items;
    V->item_begin[0] = 0;
    V->item_begin[1] = items;
    V->n_groups[0] = L.n_groups[r];
    const int64_t e = ib * L.n_bits;
    V->off_sse += 8 * e;
    V->off_l1 += 8 * e;
    V->off_hbits += 8 * e;
    V->off_linf += 4 * e;
    V->off_count += 4 * ib;
    V->off_vmin += 4 * ib;
    V->off_vmax += 4 * ib;
    *keep_r = G.keep[r];
    *VG = G;
    VG->n_ratios = 1;
    VG->keep = keep_r;
}

// What one ratio's loop produced.
struct RatioRun {
    int32_t status = -1, rounds = 0;
    double actual = 0.0, delta = 0.0, obj = 0.0, est = 0.0;
    std::vector<uint8_t> bits;   // the widths of its last compression
    mgs_status err = MGS_OK;
    std::string msg;
};

// Alg. 1's loop for ratio r on stream st: compress at init_bits; skip when
// twice that is still under the budget; then S_Delta, one-ratio ILP,
// compression, until the actual size is within the tolerance.
mgs_status run_ratio(mgs_ctx *ctx, mgs_scene *sc, const mgs_grid *grid, const void *table,
                     const mgs_table_layout *layout, const mgs_calib_opts *opts, int k0,
                     const int32_t *kept, int r, cudaStream_t st, RatioRun *R) {
    const int nb = grid->n_bits;
    const int32_t G = grid->group_size;
    const double S_T = opts->budget_bytes;
    const double cst = opts->solve.const_bytes, meta = opts->solve.meta_bytes_per_group;
    const int64_t m = layout->item_begin[r + 1] - layout->item_begin[r];
    const int64_t ib = layout->item_begin[r];
    const unsigned char *tb = static_cast<const unsigned char *>(table);
    std::vector<uint8_t> choice((size_t)m), qbits((size_t)m);
    uint8_t *d_bits = nullptr;
    MGS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&d_bits), (size_t)std::max<int64_t>(m, 1), st));
    struct Free {
        uint8_t *p;
        cudaStream_t st;
        ~Free() { cudaFreeAsync(p, st); }
    } free_bits{d_bits, st};

    auto compress = [&](double *S_a) -> mgs_status {
        int64_t coded = 0;
        MGS_TRY(encode_launch(ctx, sc, kept, grid->keep[r], G, d_bits, nullptr, 0, nullptr, &coded, st));
        *S_a = (double)coded + cst;
        R->rounds++;
        return MGS_OK;
    };

    // Q = {init_bits}: compress, and its estimate without S_Delta
    MGS_CUDA_TRY(cudaMemsetAsync(d_bits, opts->init_bits, (size_t)m, st));
    double S_a = 0;
    MGS_TRY(compress(&S_a));
    double est0 = meta * (double)m + cst;
    if (opts->solve.rate_model == MGS_RATE_ENTROPY) {
        std::vector<double> col((size_t)m);
        MGS_CUDA_TRY(cudaMemcpy2DAsync(col.data(), sizeof(double), tb + layout->off_hbits + 8 * (ib * nb + k0),
                                       8 * (size_t)nb, sizeof(double), (size_t)m, cudaMemcpyDeviceToHost,
                                       st));
        MGS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < m; i++) est0 += col[i] / 8.0;
    } else {
        std::vector<int32_t> cnt((size_t)m);
        MGS_CUDA_TRY(cudaMemcpyAsync(cnt.data(), tb + layout->off_count + 4 * ib, 4 * (size_t)m,
                                     cudaMemcpyDeviceToHost, st));
        MGS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < m; i++) est0 += (double)cnt[i] * opts->init_bits / 8.0;
    }
    R->actual = S_a;
    if (2.0 * S_a < S_T) {   // even twice the widths stay under the budget: tau too small
        R->status = 1;
        return MGS_OK;
    }
    mgs_table_layout V;
    mgs_grid VG;
    int64_t keep_r;
    ratio_view(*layout, *grid, r, &V, &VG, &keep_r);
    R->status = 2;
    for (int round = 0; round < opts->max_rounds; round++) {
        const double delta = S_a - est0;
        mgs_solve_opts so = opts->solve;
        so.delta_bytes = delta;
        mgs_solution sol{};
        int32_t st1 = 0;
        double ob = 0, by = 0, lp = 0;
        sol.choice = choice.data();
        sol.ratio_status = &st1;
        sol.ratio_objective = &ob;
        sol.ratio_bytes = &by;
        sol.ratio_lp_bound = &lp;
        mgs_status e = mgs_solve_budgets_device(ctx, table, &V, &VG, 1, &S_T, &so, &sol, st);
        if (e == MGS_ERR_INFEASIBLE || sol.r_index < 0) {
            clear_error();
            R->status = -1;
            return MGS_OK;
        }
        if (e != MGS_OK) return e;
        for (int64_t i = 0; i < m; i++) qbits[i] = (uint8_t)grid->bits[choice[i]];
        MGS_CUDA_TRY(cudaMemcpyAsync(d_bits, qbits.data(), (size_t)m, cudaMemcpyHostToDevice, st));
        est0 = sol.est_bytes - delta;
        R->delta = delta;
        R->obj = sol.objective;
        R->est = sol.est_bytes;
        MGS_TRY(compress(&S_a));
        R->actual = S_a;
        R->bits.assign(qbits.begin(), qbits.begin() + m);
        if (std::fabs(S_a - S_T) / S_T < opts->tolerance) {
            R->status = 0;
            return MGS_OK;
        }
    }
    return MGS_OK;
}

}  // namespace

extern "C" mgs_status mgs_search_calibrated(mgs_ctx *ctx, const mgs_scene *scene,
                                            const mgs_grid *grid, const void *table,
                                            const mgs_table_layout *layout,
                                            const mgs_calib_opts *opts, mgs_calib_result *out,
                                            void *stream) {
    clear_error();
    if (!ctx || !scene || !grid || !table || !layout || !opts || !out) {
        set_error("ctx, scene, grid, table, layout, opts and out must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    const int nr = grid->n_ratios, nb = grid->n_bits;
    if (nr != layout->n_ratios || nb != layout->n_bits || layout->n_channels != scene->C ||
        grid->group_size != layout->group_size || !(opts->budget_bytes > 0) ||
        !(opts->tolerance > 0) || opts->max_rounds < 1 || opts->init_bits < 1 ||
        opts->init_bits > 16 || opts->solve.rate_model < 0 || opts->solve.rate_model > 1) {
        set_error("grid/layout/scene mismatch or bad options");
        return MGS_ERR_INVALID_ARG;
    }
    int k0 = -1;   // the initial width's option (the entropy estimate needs its column)
    for (int k = 0; k < nb; k++)
        if (grid->bits[k] == opts->init_bits) k0 = k;
    if (opts->solve.rate_model == MGS_RATE_ENTROPY && k0 < 0) {
        set_error("init_bits %d is not one of the grid's widths", opts->init_bits);
        return MGS_ERR_INVALID_ARG;
    }
    cudaPointerAttributes pa{};
    const bool on_device = cudaPointerGetAttributes(&pa, table) == cudaSuccess &&
                           (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (!on_device) {
        set_error("the cost table must be in device memory");
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mgs_scene *sc = const_cast<mgs_scene *>(scene);

    const int32_t *pos = nullptr;
    std::vector<int64_t> off;
    {
        std::lock_guard<std::mutex> lk(sc->mu);
        MGS_TRY(scene_kept(sc, grid->keep, nr, st, &pos, &off));
    }
    // every ratio's stream starts after the caller's work and the kept lists
    cudaEvent_t ready = nullptr;
    MGS_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    if (cudaEventRecord(ready, st) != cudaSuccess) {
        cudaEventDestroy(ready);
        set_error("event record failed");
        return MGS_ERR_CUDA;
    }

    std::vector<RatioRun> runs(nr);
    std::atomic<int> next{0};
    auto worker = [&]() {
        DeviceGuard g(ctx->device);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamWaitEvent(ws, ready, 0) != cudaSuccess) {
            for (int r; (r = next.fetch_add(1)) < nr;) {
                runs[r].err = MGS_ERR_CUDA;
                runs[r].msg = "stream creation failed";
            }
            if (ws) cudaStreamDestroy(ws);
            return;
        }
        for (int r; (r = next.fetch_add(1)) < nr;) {
            clear_error();
            const mgs_status e = run_ratio(ctx, sc, grid, table, layout, opts, k0, pos + off[r], r, ws, &runs[r]);
            if (e != MGS_OK) {
                runs[r].err = e;
                runs[r].msg = mgs_last_error();
            }
        }
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    };
    const int n_workers = std::min(nr, 16);
    std::vector<std::thread> pool;
    for (int w = 1; w < n_workers; w++) pool.emplace_back(worker);
    worker();
    for (auto &th : pool) th.join();
    cudaEventDestroy(ready);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("calibrated search: stream error");
        return MGS_ERR_CUDA;
    }
    for (int r = 0; r < nr; r++)
        if (runs[r].err != MGS_OK) {
            set_error("%s", runs[r].msg.c_str());
            return runs[r].err;
        }

    int best = -1;
    int32_t total_rounds = 0;
    for (int r = 0; r < nr; r++) {
        total_rounds += runs[r].rounds;
        if (runs[r].status != 0) continue;
        if (best < 0 || runs[r].obj <= runs[best].obj) best = r;   // ties: the larger ratio
    }
    out->r_index = best;
    out->rounds = total_rounds;
    out->actual_bytes = best >= 0 ? runs[best].actual : 0.0;
    out->est_bytes = best >= 0 ? runs[best].est : 0.0;
    out->objective = best >= 0 ? runs[best].obj : 0.0;
    if (out->bits && best >= 0) std::copy(runs[best].bits.begin(), runs[best].bits.end(), out->bits);
    for (int r = 0; r < nr; r++) {
        if (out->ratio_status) out->ratio_status[r] = runs[r].status;
        if (out->ratio_rounds) out->ratio_rounds[r] = runs[r].rounds;
        if (out->ratio_actual) out->ratio_actual[r] = runs[r].actual;
        if (out->ratio_delta) out->ratio_delta[r] = runs[r].delta;
        if (out->ratio_objective) out->ratio_objective[r] = runs[r].obj;
    }
    if (best < 0) {
        set_error("no ratio reached the budget within the tolerance");
        return MGS_ERR_INFEASIBLE;
    }
    return MGS_OK;
}
