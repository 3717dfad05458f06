// Internal declarations of the mgs library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mgs.h"

namespace mgs {

// Thread-local error message behind mgs_last_error().
void set_error(const char *fmt, ...);
void clear_error();

#define MGS_CUDA_TRY(expr)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            mgs::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                           __LINE__);                                                         \
            return MGS_ERR_CUDA;                                                              \
        }                                                                                     \
    } while (0)

#define MGS_TRY(expr)                  \
    do {                               \
        mgs_status s_ = (expr);        \
        if (s_ != MGS_OK) return s_;   \
    } while (0)

constexpr int kSlabWidth = 8;         // channels per slab row (32 bytes)
constexpr int kLtabFracBits = 22;     // fixed point of L(n) = n log2 n
constexpr int kMaxSegments = 4096;    // (scene, ratio) pairs in one batched launch

// Makes `dev` current for a scope and restores the caller's device after.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Device buffer owned by the library (stream-ordered allocation).
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Kept lists of one keep-array, cached on the scene.
struct KeptLists {
    std::vector<int64_t> keep;     // the K_r they were built for
    std::vector<int64_t> offset;   // start of list r in `pos`
    int32_t *pos = nullptr;        // concatenated Morton positions, sum_r K_r entries
    size_t bytes = 0;
};

// Per-context tile configuration chosen for a group size.
struct TileChoice {
    int group_size;
    int n_bits;
    int config;   // index into the cost kernel's configuration table
};

}  // namespace mgs

struct mgs_ctx {
    int device = 0;
    int sm_count = 0;
    unsigned long long *d_ltab = nullptr;   // L(n) = n log2 n for n in [0, MGS_MAX_GROUP], 2^-22 bits
    uint32_t *d_dtab = nullptr;             // L(n) - L(n - 1), same range and unit (0 at n = 0)
    std::mutex mu;
    std::vector<mgs::TileChoice> tiles;     // autotuned choices
    int forced_config = -1;                 // testing hook: force a tile configuration
    int n_scenes = 0;
    int vq_tensor = 1;                      // SH assignment on the tensor cores (else CUDA cores)
    long long vq_wait_cycles = 0;           // bounded-wait limit of the tensor path (0: default)
    int64_t vq_scores = 0, vq_rescored = 0; // since the last mgs_vq_stats
};

struct mgs_scene {
    mgs_ctx *ctx = nullptr;
    int64_t n = 0;
    int32_t C = 0;
    int32_t n_slabs = 0;
    float *d_slabs = nullptr;     // [n_slabs][n][8] FP32, Morton order, padded channels = 0
    int32_t *d_rank_m = nullptr;  // importance rank of the Gaussian at Morton position p
    int32_t *d_order = nullptr;   // Gaussian index at Morton position p
    uint64_t *d_codes = nullptr;  // Morton code of Gaussian i (index order)
    int64_t device_bytes = 0;
    std::mutex mu;
    mgs::KeptLists kept;
};

namespace mgs {

// ---- scene pipeline (scene.cu) ----
mgs_status scene_build(mgs_ctx *ctx, const float *d_attrs, const float *d_imp, int64_t n, int32_t C,
                       cudaStream_t st, mgs_scene *scene);
// Build (or reuse) the kept lists of `keep` for the scene.
mgs_status scene_kept(mgs_scene *scene, const int64_t *keep, int32_t n_r, cudaStream_t st,
                      const int32_t **pos_out, std::vector<int64_t> *offset_out);

// Kept list of one kept-set size into caller memory: pos[keep] and
// tile_cnt[kept_tiles_for(n)] (fully overwritten; nothing needs clearing).
mgs_status kept_list_into(const mgs_scene *scene, int64_t keep, int32_t *pos, uint32_t *tile_cnt,
                          cudaStream_t st);
constexpr int kKeptTile = 4096;       // positions counted per tile by the kept-list kernels
constexpr int64_t kept_tiles_for(int64_t n) { return (n + kKeptTile - 1) / kKeptTile; }

// ---- cost kernels (cost.cu) ----
struct CostSeg {
    const float *slabs;
    const int32_t *kept;   // Morton positions of this ratio's kept set (NULL: positions 0..K-1)
    int64_t n;             // scene size (slab stride)
    int64_t K;             // kept-set size
    int64_t work_begin;    // first work item of this segment
    int64_t item_base;     // table item of (r, c = 0, g = 0)
    int32_t n_groups;      // groups of this ratio (table stride)
    int32_t n_chunks;
    int32_t C;
    int32_t g_first;       // first group computed by this segment
    int32_t g_count;       // groups computed (0 = all n_groups)
    int32_t pad_;
    int64_t code_off;      // probe launches: codes of this segment start here ([C][n_bits][K])
    double *sse;
    double *l1;
    double *hbits;
    float *linf;
    int32_t *cnt;
    float *vmin;
    float *vmax;
};

// A launch's segments are cut into at most this many runs of groups each
// (Morton-range buckets; see cost_exec_create): size segment scratch for it.
constexpr int kMaxSpatialBuckets = 64;

struct CostLaunch {
    std::vector<CostSeg> segs;
    int32_t group_size = 0;
    int32_t n_bits = 0;          // options in the table
    int32_t bits[MGS_MAX_OPTIONS] = {};
    int32_t opt_lo = 0;          // options computed by this launch: [opt_lo, opt_hi)
    int32_t opt_hi = 0;
    bool persistent = false;
    // probe launches (test and inspection): every bin of every histogram,
    // [item][sum of 2^b over the grid's options], and every code
    uint32_t *probe_hist = nullptr;
    uint16_t *probe_codes = nullptr;
};

// Tile configurations of the cost kernel.
struct CostConfig {
    int threads;
    int ept;      // elements per thread: threads * ept >= group size
    int width;    // channels per work item
    const char *name;
};
int cost_config_count();
const CostConfig &cost_config(int i);
// Default configuration for a group size (or -1).
int cost_default_config(int group_size);

// Launch the cost kernel over all segments of `L`.  d_segs is scratch for the
// segment array (at least segs.size() entries); counter is a device uint (persistent mode).
mgs_status cost_launch(mgs_ctx *ctx, const CostLaunch &L, int config, CostSeg *d_segs,
                       unsigned int *d_counter, cudaStream_t st);
size_t cost_smem_bytes(int config, int group_size, int n_opts, const int32_t *bits);
bool cost_config_fits(int config, int group_size, int n_opts, const int32_t *bits);
// The configuration has a probe instantiation.
bool cost_config_has_probe(int config);
// The histogram plan of a launch, flattened for inspection (mgs_debug_cost_plan).
int cost_plan_export(int config, const int32_t *bits, int n_opts, int32_t *out, int cap);

// A prepared launch: work layout, kernel arguments and shape, reusable and
// capturable (cost_exec_run issues only a memset and a kernel launch).
struct CostExec;
mgs_status cost_exec_create(mgs_ctx *ctx, const CostLaunch &L, int config, CostExec **out,
                            std::vector<CostSeg> *segs, int64_t *n_work);
void cost_exec_bind(CostExec *X, const CostSeg *d_segs, unsigned int *d_counter);
mgs_status cost_exec_run(const CostExec *X, cudaStream_t st);
void cost_exec_destroy(CostExec *X);

// ---- quantise one configuration (quantize.cu) ----
mgs_status quantize_launch(mgs_ctx *ctx, const mgs_scene *scene, const int32_t *kept, int64_t keep,
                           int32_t G, const uint8_t *bits, uint16_t *codes, float *minmax,
                           cudaStream_t st);

// ---- block coder (encode.cu) ----
// Upper bound of a configuration's stream: C * (10 * n_groups + 2 * keep) bytes.
int64_t encode_bound(int64_t keep, int32_t G, int32_t C);
// Quantise with d_bits (device, [C][n_groups], each in 1..16) and encode every
// block; writes the stream when `stream` is non-NULL (capacity checked), the
// block sizes when d_sizes_out is non-NULL, and the total into *total_out.
// Synchronises `st`.
mgs_status encode_launch(mgs_ctx *ctx, const mgs_scene *sc, const int32_t *kept, int64_t keep,
                         int32_t G, const uint8_t *d_bits, uint8_t *stream, int64_t capacity,
                         int32_t *d_sizes_out, int64_t *total_out, cudaStream_t st);

// ---- SH vector quantisation on the tensor cores (vq_tc.cu) ----
// Bytes of the codebook's MMA tiles for K entries of D dimensions.
size_t vq_tc_workspace(int32_t K, int32_t D);
// Lay out the codebook in `tiles` and assign x[rows[i]] (rows may be NULL)
// with the exact path's decisions; *stats += entries re-scored exactly,
// *err |= 1 if a bounded wait ran out (cmax2: 4 bytes of scratch).
// wait_cycles: clock-cycle limit of each bounded wait (0: the default, about one second).
mgs_status vq_assign_tc(const float *x, int64_t n, int32_t D, const int32_t *rows, const float *cb,
                        int32_t K, int32_t *idx, float *score, unsigned char *tiles, unsigned int *cmax2,
                        unsigned long long *stats, unsigned int *err, long long wait_cycles, cudaStream_t st);

// ---- helpers (abi.cu) ----
// Stream-ordered device allocation of the library's scenes, tables and
// workspaces; fails on purpose when a test armed mgs_debug_fail_allocation.
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);
// Count kernels enqueued by this library (mgs_kernel_launches()).
void count_launches(int64_t k);
bool is_device_pointer(const void *p);
int64_t n_groups_of(int64_t keep, int32_t G);
mgs_status check_grid(const mgs_grid *grid, int64_t n);

}  // namespace mgs
