// Serving loop: (scene, byte budget) search jobs arrive at any time; scenes are
// made resident, their cost-table work is run in shared batched launches, and
// each finished table is solved on the device (mgs_solve_budgets_device) by a
// solver thread with its own stream, while the next launches run.
//
// Continuous batching: jobs are admitted while a slot is free and their
// device footprint fits the HBM budget.  The compute thread repeatedly builds
// one persistent launch over a slice of the remaining work items of EVERY
// admitted job (round-robin shares), so a job that arrives while others run
// joins the next launch and its work overlaps theirs on the device.  Results
// do not depend on the mix: every (ratio, group, channel) work item is
// computed by the same kernel with the same tile shape whichever launch it
// lands in, and each item's reductions are fixed-order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace mgs {
namespace {

using Clock = std::chrono::steady_clock;

enum JobState { kPending, kIngesting, kReady, kSolving, kDone };

struct Job {
    int64_t id = 0;
    // request
    const float *attrs = nullptr;
    const float *importance = nullptr;
    int64_t n = 0;
    int32_t C = 0;
    std::vector<int64_t> keep;
    std::vector<int32_t> bits;
    int32_t G = 0;
    double budget = 0;
    mgs_solve_opts opts{};
    void *table_out = nullptr;       // caller's host copy of the finished table (optional)
    // resources
    mgs_scene *scene = nullptr;
    void *d_table = nullptr;
    mgs_table_layout layout{};
    std::vector<CostSeg> segs;       // one per ratio, whole ratio
    std::vector<int32_t> cursor;     // next group per ratio
    int64_t groups_left = 0;
    int64_t footprint = 0;
    // result
    JobState state = kPending;
    mgs_status status = MGS_OK;
    std::string error;
    int32_t r_index = -1;
    double est_bytes = 0, objective = 0, lp_bound = 0;
    std::vector<uint8_t> choice;
    double t_submit = 0, t_admit = 0, t_ready = 0, t_table = 0, t_done = 0;
};

}  // namespace
}  // namespace mgs

struct mgs_server {
    mgs_ctx *ctx = nullptr;
    mgs_server_opts opts{};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;        // state changes
    bool stopping = false;
    int64_t next_id = 1;
    std::deque<mgs::Job *> pending;    // FIFO, not yet admitted
    std::vector<mgs::Job *> active;    // admitted, work not finished (admission order)
    std::deque<mgs::Job *> to_solve;
    std::map<int64_t, std::unique_ptr<mgs::Job>> jobs;
    int in_flight = 0;
    int64_t used_bytes = 0;
    std::atomic<int> ingesting{0};   // scene builds in flight: cost launches are shortened
    cudaStream_t ingest_stream = nullptr, compute_stream = nullptr, copy_stream = nullptr;   // copy: frees
    std::thread ingest_thread, compute_thread;
    std::vector<std::thread> solvers;
    // compute-launch scratch
    mgs::CostSeg *h_segs = nullptr;    // pinned
    void *d_scratch = nullptr;
    size_t seg_capacity = 0;
    int64_t launches = 0;
    int64_t work_items = 0;
};

namespace mgs {
namespace {

double now_s(const mgs_server *S) {
    return std::chrono::duration<double>(Clock::now() - S->t0).count();
}

int64_t job_footprint(const Job &j, const mgs_table_layout &L) {
    const int64_t slabs = (int64_t)((j.C + 7) / 8) * j.n * 32;
    int64_t kept = 0;
    for (auto k : j.keep) kept += k * 4;
    // resident scene + kept lists + table, plus the transient staging and sort
    // scratch of scene creation and the device solver's hulls and histograms
    const int64_t nb = (int64_t)j.bits.size(), ni = L.item_begin[L.n_ratios];
    const int64_t solver = ni * (3 + 17 * nb + 8 * std::max<int64_t>(1, nb - 1)) +
                           (int64_t)L.n_ratios * 65536 * 12;
    return slabs + j.n * 16 + kept + L.total_bytes + (int64_t)j.n * j.C * 4 + j.n * 28 + solver;
}

void fail_job(mgs_server *S, Job *j, mgs_status s, const char *what) {
    j->status = s;
    j->error = std::string(what) + ": " + mgs_last_error();
    j->state = kDone;
    j->t_done = now_s(S);
}

// Free a job's device and pinned memory (stream-ordered on the copy stream).
void release_job(mgs_server *S, Job *j) {
    if (j->scene) {
        mgs_scene *sc = j->scene;
        cudaFreeAsync(sc->d_slabs, S->copy_stream);
        cudaFreeAsync(sc->d_rank_m, S->copy_stream);
        cudaFreeAsync(sc->d_order, S->copy_stream);
        cudaFreeAsync(sc->d_codes, S->copy_stream);
        if (sc->kept.pos) cudaFreeAsync(sc->kept.pos, S->copy_stream);
        {
            std::lock_guard<std::mutex> lk(S->ctx->mu);
            S->ctx->n_scenes--;
        }
        delete sc;
        j->scene = nullptr;
    }
    if (j->d_table) {
        cudaFreeAsync(j->d_table, S->copy_stream);
        j->d_table = nullptr;
    }
    cudaStreamSynchronize(S->copy_stream);
}

// Admit pending jobs (FIFO) while slots and memory allow; make scenes resident.
void ingest_loop(mgs_server *S) {
    cudaSetDevice(S->ctx->device);
    while (true) {
        Job *j = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] {
                if (S->stopping) return true;
                if (S->pending.empty()) return false;
                Job *h = S->pending.front();
                return S->in_flight < S->opts.max_jobs &&
                       (S->used_bytes + h->footprint <= S->opts.hbm_budget_bytes || S->in_flight == 0);
            });
            if (S->stopping && S->pending.empty()) return;
            if (S->stopping) {
                // drain: fail what was never admitted
                while (!S->pending.empty()) {
                    Job *p = S->pending.front();
                    S->pending.pop_front();
                    p->status = MGS_ERR_BUSY;
                    p->error = "server stopped before the job was admitted";
                    p->state = kDone;
                }
                S->cv.notify_all();
                return;
            }
            j = S->pending.front();
            S->pending.pop_front();
            S->in_flight++;
            S->used_bytes += j->footprint;
            j->state = kIngesting;
            j->t_admit = now_s(S);
            S->ingesting++;
        }
        mgs_status s = mgs_scene_create(S->ctx, j->attrs, j->importance, j->n, j->C,
                                        S->ingest_stream, &j->scene);
        if (s == MGS_OK) {
            mgs_grid g{(int32_t)j->keep.size(), j->keep.data(), (int32_t)j->bits.size(),
                       j->bits.data(), j->G};
            s = mgs_table_layout_for(j->n, j->C, &g, &j->layout);
            if (s == MGS_OK &&
                dev_malloc_async(&j->d_table, j->layout.total_bytes, S->ingest_stream) != cudaSuccess) {
                cudaGetLastError();
                set_error("table allocation failed");
                s = MGS_ERR_OUT_OF_MEMORY;
            }
            if (s == MGS_OK) {
                const int32_t *pos = nullptr;
                std::vector<int64_t> off;
                {
                    std::lock_guard<std::mutex> lk(j->scene->mu);
                    s = scene_kept(j->scene, j->keep.data(), (int32_t)j->keep.size(),
                                   S->ingest_stream, &pos, &off);
                }
                if (s == MGS_OK) {
                    char *b = static_cast<char *>(j->d_table);
                    for (size_t r = 0; r < j->keep.size(); r++) {
                        CostSeg c{};
                        c.slabs = j->scene->d_slabs;
                        c.kept = pos + off[r];
                        c.n = j->n;
                        c.K = j->keep[r];
                        c.item_base = j->layout.item_begin[r];
                        c.n_groups = (int32_t)j->layout.n_groups[r];
                        c.C = j->C;
                        c.sse = reinterpret_cast<double *>(b + j->layout.off_sse);
                        c.l1 = reinterpret_cast<double *>(b + j->layout.off_l1);
                        c.hbits = reinterpret_cast<double *>(b + j->layout.off_hbits);
                        c.linf = reinterpret_cast<float *>(b + j->layout.off_linf);
                        c.cnt = reinterpret_cast<int32_t *>(b + j->layout.off_count);
                        c.vmin = reinterpret_cast<float *>(b + j->layout.off_vmin);
                        c.vmax = reinterpret_cast<float *>(b + j->layout.off_vmax);
                        j->segs.push_back(c);
                        j->groups_left += c.n_groups;
                    }
                    j->cursor.assign(j->keep.size(), 0);
                }
            }
            if (s == MGS_OK && cudaStreamSynchronize(S->ingest_stream) != cudaSuccess) {
                set_error("ingest stream failed: %s", cudaGetErrorString(cudaGetLastError()));
                s = MGS_ERR_CUDA;
            }
        }
        S->ingesting--;
        std::lock_guard<std::mutex> lk(S->mu);
        if (s != MGS_OK) {
            fail_job(S, j, s, "ingest");
            release_job(S, j);
            S->in_flight--;
            S->used_bytes -= j->footprint;
        } else {
            j->state = kReady;
            j->t_ready = now_s(S);
            S->active.push_back(j);
        }
        S->cv.notify_all();
    }
}

// One batched launch per iteration over slices of every active job's remaining work.
void compute_loop(mgs_server *S) {
    cudaSetDevice(S->ctx->device);
    while (true) {
        std::vector<CostSeg> slice;
        std::vector<Job *> finished;
        int32_t G = 0, n_bits = 0;
        int32_t bits[MGS_MAX_OPTIONS] = {};
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stopping || !S->active.empty(); });
            if (S->active.empty()) return;
            // jobs sharing a launch must share the grid shape (G and bit-widths)
            Job *lead = S->active.front();
            G = lead->G;
            n_bits = (int32_t)lead->bits.size();
            for (int k = 0; k < n_bits; k++) bits[k] = lead->bits[k];
            std::vector<Job *> batch;
            for (Job *j : S->active)
                if (j->G == G && j->bits == lead->bits) batch.push_back(j);
            const int width = cost_config(std::max(0, cost_default_config(G))).width;
            const int chunks_per_group = (lead->C + width - 1) / width;
            int64_t budget_groups =
                S->opts.slice_items > 0 ? std::max<int64_t>(1, S->opts.slice_items / chunks_per_group)
                                        : INT64_MAX;
            // a launch holds every SM until its slice is done, so while a new job's
            // scene is being built the slices are an eighth as long
            if (S->ingesting.load() > 0 && budget_groups != INT64_MAX)
                budget_groups = std::max<int64_t>(1, budget_groups / 8);
            int64_t share = std::max<int64_t>(1, budget_groups / (int64_t)batch.size());
            for (Job *j : batch) {
                int64_t take = std::min<int64_t>(share, j->groups_left);
                for (size_t r = 0; r < j->segs.size() && take > 0; r++) {
                    int32_t left = j->segs[r].n_groups - j->cursor[r];
                    if (left <= 0) continue;
                    int32_t t = (int32_t)std::min<int64_t>(left, take);
                    CostSeg c = j->segs[r];
                    c.g_first = j->cursor[r];
                    c.g_count = t;
                    slice.push_back(c);
                    j->cursor[r] += t;
                    j->groups_left -= t;
                    take -= t;
                }
                if (j->groups_left == 0) finished.push_back(j);
            }
        }
        if (!slice.empty()) {
            CostLaunch L;
            L.segs = slice;
            L.group_size = G;
            L.n_bits = n_bits;
            for (int k = 0; k < n_bits; k++) L.bits[k] = bits[k];
            L.opt_hi = n_bits;
            L.persistent = true;
            int config = -1;
            {
                std::lock_guard<std::mutex> lk(S->ctx->mu);
                for (auto &t : S->ctx->tiles)
                    if (t.group_size == G && t.n_bits == n_bits) config = t.config;
            }
            if (config < 0) config = cost_default_config(G);
            CostExec *X = nullptr;
            std::vector<CostSeg> prepared;
            int64_t n_work = 0;
            mgs_status s = cost_exec_create(S->ctx, L, config, &X, &prepared, &n_work);
            if (s == MGS_OK) {
                if (prepared.size() > S->seg_capacity) {
                    cudaFreeHost(S->h_segs);
                    cudaFree(S->d_scratch);
                    S->seg_capacity = prepared.size() * 2;
                    cudaMallocHost(&S->h_segs, sizeof(CostSeg) * S->seg_capacity);
                    cudaMalloc(&S->d_scratch, sizeof(CostSeg) * S->seg_capacity + 256);
                }
                std::memcpy(S->h_segs, prepared.data(), sizeof(CostSeg) * prepared.size());
                cudaMemcpyAsync(S->d_scratch, S->h_segs, sizeof(CostSeg) * prepared.size(),
                                cudaMemcpyHostToDevice, S->compute_stream);
                cost_exec_bind(X, static_cast<CostSeg *>(S->d_scratch),
                               reinterpret_cast<unsigned int *>(static_cast<char *>(S->d_scratch) +
                                                                sizeof(CostSeg) * S->seg_capacity));
                s = cost_exec_run(X, S->compute_stream);
                cost_exec_destroy(X);
            }
            if (s == MGS_OK && cudaStreamSynchronize(S->compute_stream) != cudaSuccess) {
                set_error("compute stream failed: %s", cudaGetErrorString(cudaGetLastError()));
                s = MGS_ERR_CUDA;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            S->launches++;
            S->work_items += n_work;
            if (s != MGS_OK) {
                // every job in this slice fails
                for (Job *j : S->active) {
                    if (j->state == kReady) fail_job(S, j, s, "compute");
                }
            }
        }
        std::lock_guard<std::mutex> lk(S->mu);
        for (Job *j : finished) {
            S->active.erase(std::find(S->active.begin(), S->active.end(), j));
            if (j->state == kDone) {   // failed above
                release_job(S, j);
                S->in_flight--;
                S->used_bytes -= j->footprint;
                continue;
            }
            j->t_table = now_s(S);   // the compute stream has been synchronised: the table is complete
            j->state = kSolving;
            S->to_solve.push_back(j);
        }
        S->cv.notify_all();
    }
}

void solve_loop(mgs_server *S) {
    cudaSetDevice(S->ctx->device);
    cudaStream_t st = nullptr;
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_high) != cudaSuccess) st = nullptr;
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() {
            if (s) cudaStreamDestroy(s);
        }
    } guard{st};
    while (true) {
        Job *j = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return !S->to_solve.empty() || (S->stopping && S->in_flight == 0); });
            if (S->to_solve.empty()) return;
            j = S->to_solve.front();
            S->to_solve.pop_front();
        }
        mgs_status s = MGS_OK;
        if (!st) {
            set_error("solver stream creation failed");
            s = MGS_ERR_CUDA;
        }
        mgs_solution sol{};
        std::vector<uint8_t> choice;
        if (s == MGS_OK) {
            int64_t max_items = 0;
            for (int r = 0; r < j->layout.n_ratios; r++)
                max_items = std::max(max_items, j->layout.item_begin[r + 1] - j->layout.item_begin[r]);
            choice.assign((size_t)std::max<int64_t>(max_items, 1), 0);
            sol.choice = choice.data();
            mgs_grid g{(int32_t)j->keep.size(), j->keep.data(), (int32_t)j->bits.size(),
                       j->bits.data(), j->G};
            if (j->table_out) {
                cudaError_t e = cudaMemcpyAsync(j->table_out, j->d_table, (size_t)j->layout.total_bytes,
                                                cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) {
                    set_error("table copy: %s", cudaGetErrorString(e));
                    s = MGS_ERR_CUDA;
                }
            }
            if (s == MGS_OK)
                s = mgs_solve_budgets_device(S->ctx, j->d_table, &j->layout, &g, 1, &j->budget, &j->opts, &sol, st);
        }
        release_job(S, j);   // outside the lock: it waits for the copy stream
        std::lock_guard<std::mutex> lk(S->mu);
        if (s != MGS_OK) {
            fail_job(S, j, s, "solve");
        } else {
            j->r_index = sol.r_index;
            j->est_bytes = sol.est_bytes;
            j->objective = sol.objective;
            j->lp_bound = sol.lp_bound;
            int64_t m = j->layout.item_begin[sol.r_index + 1] - j->layout.item_begin[sol.r_index];
            j->choice.assign(choice.begin(), choice.begin() + m);
            j->state = kDone;
            j->t_done = now_s(S);
        }
        S->in_flight--;
        S->used_bytes -= j->footprint;
        S->cv.notify_all();
    }
}

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" {

mgs_status mgs_server_create(mgs_ctx *ctx, const mgs_server_opts *opts, mgs_server **out) {
    clear_error();
    if (!ctx || !opts || !out || opts->max_jobs < 1 || opts->hbm_budget_bytes <= 0 ||
        opts->solver_threads < 1 || opts->slice_items < 0) {
        set_error("ctx, opts and out must be non-NULL; max_jobs, solver_threads >= 1, "
                  "hbm_budget_bytes > 0, slice_items >= 0");
        return MGS_ERR_INVALID_ARG;
    }
    mgs_server *S = new (std::nothrow) mgs_server();
    if (!S) return MGS_ERR_OUT_OF_MEMORY;
    S->ctx = ctx;
    S->opts = *opts;
    S->t0 = Clock::now();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    // ingest and solves ahead of the batched cost launches: a new job's scene
    // build and a finished job's solve are short and on every job's critical
    // path, while the persistent cost kernel would otherwise hold every SM
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    cudaError_t e = cudaStreamCreateWithPriority(&S->ingest_stream, cudaStreamNonBlocking, prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&S->compute_stream, cudaStreamNonBlocking, prio_low);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        set_error("stream creation: %s", cudaGetErrorString(e));
        delete S;
        return MGS_ERR_CUDA;
    }
    S->ingest_thread = std::thread(ingest_loop, S);
    S->compute_thread = std::thread(compute_loop, S);
    for (int i = 0; i < opts->solver_threads; i++) S->solvers.emplace_back(solve_loop, S);
    *out = S;
    return MGS_OK;
}

mgs_status mgs_server_submit(mgs_server *S, const mgs_job *job, int64_t *id_out) {
    clear_error();
    if (!S || !job || !id_out || !job->attrs || !job->importance) {
        set_error("server, job, id_out, attrs and importance must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    MGS_TRY(check_grid(&job->grid, job->n));
    if (job->n_channels < 3 || job->n_channels > MGS_MAX_CHANNELS || !(job->budget_bytes >= 0)) {
        set_error("bad channel count or budget");
        return MGS_ERR_INVALID_ARG;
    }
    auto j = std::make_unique<Job>();
    j->attrs = job->attrs;
    j->importance = job->importance;
    j->n = job->n;
    j->C = job->n_channels;
    j->keep.assign(job->grid.keep, job->grid.keep + job->grid.n_ratios);
    j->bits.assign(job->grid.bits, job->grid.bits + job->grid.n_bits);
    j->G = job->grid.group_size;
    j->budget = job->budget_bytes;
    j->opts = job->opts;
    j->table_out = job->table_out;
    mgs_table_layout L;
    MGS_TRY(mgs_table_layout_for(j->n, j->C, &job->grid, &L));
    j->footprint = job_footprint(*j, L);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) {
        set_error("server is stopping");
        return MGS_ERR_BUSY;
    }
    j->id = S->next_id++;
    j->t_submit = now_s(S);
    *id_out = j->id;
    S->pending.push_back(j.get());
    S->jobs[j->id] = std::move(j);
    S->cv.notify_all();
    return MGS_OK;
}

mgs_status mgs_server_wait(mgs_server *S, int64_t id, int32_t timeout_ms, mgs_job_result *out,
                           uint8_t *choice, int64_t choice_capacity) {
    clear_error();
    if (!S || !out) {
        set_error("server and out must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) {
        set_error("unknown job %lld", (long long)id);
        return MGS_ERR_INVALID_ARG;
    }
    Job *j = it->second.get();
    bool done = S->cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                               [&] { return j->state == kDone; });
    if (!done) {
        set_error("job %lld not finished within %d ms", (long long)id, timeout_ms);
        return MGS_ERR_TIMEOUT;
    }
    out->status = j->status;
    out->r_index = j->r_index;
    out->est_bytes = j->est_bytes;
    out->objective = j->objective;
    out->lp_bound = j->lp_bound;
    out->n_choice = (int64_t)j->choice.size();
    out->t_submit = j->t_submit;
    out->t_admit = j->t_admit;
    out->t_ready = j->t_ready;
    out->t_table = j->t_table;
    out->t_done = j->t_done;
    if (choice && choice_capacity > 0)
        std::memcpy(choice, j->choice.data(),
                    (size_t)std::min<int64_t>(choice_capacity, (int64_t)j->choice.size()));
    if (j->status != MGS_OK) set_error("%s", j->error.c_str());
    return MGS_OK;
}

mgs_status mgs_server_stats(mgs_server *S, int64_t *launches, int64_t *work_items,
                            int32_t *in_flight, int64_t *used_bytes) {
    if (!S) {
        set_error("server is NULL");
        return MGS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (launches) *launches = S->launches;
    if (work_items) *work_items = S->work_items;
    if (in_flight) *in_flight = S->in_flight;
    if (used_bytes) *used_bytes = S->used_bytes;
    return MGS_OK;
}

mgs_status mgs_server_destroy(mgs_server *S) {
    clear_error();
    if (!S) return MGS_OK;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        // let admitted work finish; never-admitted jobs are dropped
        S->cv.wait(lk, [&] { return S->in_flight == 0 && S->pending.empty(); });
        S->stopping = true;
        S->cv.notify_all();
    }
    S->ingest_thread.join();
    S->compute_thread.join();
    for (auto &t : S->solvers) t.join();
    cudaSetDevice(S->ctx->device);
    if (S->h_segs) cudaFreeHost(S->h_segs);
    if (S->d_scratch) cudaFree(S->d_scratch);
    cudaStreamDestroy(S->ingest_stream);
    cudaStreamDestroy(S->compute_stream);
    cudaStreamDestroy(S->copy_stream);
    delete S;
    return MGS_OK;
}

}  // extern "C"
