/*
 * mgs.h -- C ABI of a GB300 (sm_103a) library that builds the candidate cost
 * table of MesonGS++'s size-aware configuration search and solves the bit-width
 * 0-1 ILP over it.
 *
 * The problem (Eq. (eq:nilp), Sec. III-E): choose the reserve ratio tau and a
 * bit-width per (channel, block) to minimise the quality loss subject to the
 * estimated size <= budget.  Alg. 1 (Sec. III-E/F) samples tau on a grid and
 * solves a 0-1 ILP (Eq. (eq:ilp)) per tau over a precomputed loss matrix
 * Omega[C][B][Q] (Sec. III-F "Acceleration") and a size estimate (Sec. III-F
 * "Size Estimator").  This library computes that matrix for every tau at once
 * (mgs_build_cost_table), estimates sizes (mgs_estimate_size), solves the ILP
 * and picks tau (mgs_solve_budget), and emits the codes of a chosen
 * configuration (mgs_quantize_groups).
 *
 * Conventions.
 *   - Every function returns an mgs_status; MGS_OK is 0, errors are negative.
 *     mgs_last_error() gives a message for the last failing call on the
 *     calling thread.  No C++ exception crosses this interface.
 *   - "device" pointers are CUDA device memory of the context's GPU; "host"
 *     pointers are CPU memory.  Where a pointer may be either, the library
 *     asks the CUDA driver which it is.
 *   - The caller owns every buffer it passes; inputs are never modified.  The
 *     library owns its handles (mgs_ctx, mgs_scene) and the device memory
 *     behind them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls that take a stream are ordered on it; a call that writes
 *     host memory synchronises that stream before returning.
 *   - Budgets and sizes are bytes (1 MB = 10^6 B).
 *
 * Channel layout of a scene (Sec. II "Preliminary"): attrs[i][c] is channel c
 * of Gaussian i, FP32, row-major; channels 0..2 must be the position (they
 * define the Morton order, Sec. III-G).  The synthetic scenes of this project
 * use 59 channels: position(3), SH DC(3), SH rest(45), opacity(1), log-scale(3),
 * rotation(4).
 */
#ifndef MGS_H
#define MGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mgs_status;

#define MGS_OK 0
#define MGS_ERR_INVALID_ARG (-1)   /* a size, pointer or option is out of range */
#define MGS_ERR_NONFINITE (-2)     /* an attribute or importance is NaN or +-inf */
#define MGS_ERR_RANGE (-3)         /* a channel's max - min overflows FP32 */
#define MGS_ERR_OUT_OF_MEMORY (-4) /* device or host allocation failed */
#define MGS_ERR_CUDA (-5)          /* a CUDA call failed (message has the CUDA error) */
#define MGS_ERR_INFEASIBLE (-6)    /* no ratio fits the budget even at the lowest bit-widths */
#define MGS_ERR_TIMEOUT (-7)       /* a bounded wait ran out */
#define MGS_ERR_BUSY (-8)          /* the resource is in use (e.g. a server at capacity) */

#define MGS_MAX_RATIOS 64      /* kept-set sizes per grid */
#define MGS_MAX_OPTIONS 16     /* candidate bit-widths per grid */
#define MGS_MAX_BITS 16        /* largest bit-width */
#define MGS_MAX_GROUP 16384    /* largest group size G */
#define MGS_MAX_CHANNELS 256

typedef struct mgs_ctx mgs_ctx;
typedef struct mgs_scene mgs_scene;

/*
 * The search grid (Alg. 1's tau loop x Eq. (eq:ilp)'s Q options; Sec. III-D
 * groups of fixed length G, Tab. tab:robust / Sec. IV "block quantisation").
 *   keep[r]  kept-set size K_r for reserve ratio r: the K_r most important
 *            Gaussians are kept (Sec. III-A).  Strictly increasing, 1 <= K_r <= n.
 *   bits[k]  candidate bit-width b_k, strictly increasing, each in 1..16.
 *   group_size  G: the kept set, in Morton order (Sec. III-G), is cut into
 *            consecutive groups of G; the last group holds the remainder.
 * Both arrays are host memory, read during the call only.
 */
typedef struct {
    int32_t n_ratios;
    const int64_t *keep;
    int32_t n_bits;
    const int32_t *bits;
    int32_t group_size;
} mgs_grid;

/*
 * Layout of one cost table in a single caller-allocated buffer (256-byte
 * aligned, `total_bytes` long).  Items are the (ratio r, channel c, group g)
 * triples, enumerated r-major, then c, then g:
 *     item(r, c, g) = item_begin[r] + c * n_groups[r] + g
 *     item_begin[r] = n_channels * sum_{r' < r} n_groups[r'],  n_groups[r] = ceil(K_r / G)
 * Per item and option k (index item * n_bits + k):
 *     sse   f64  sum of squared dequantisation errors        (Omega, 2-norm squared)
 *     l1    f64  sum of absolute errors                        (Omega, 1-norm)
 *     hbits f64  entropy bound -sum_s h_s log2(h_s / n) in bits (Sec. III-F)
 *     linf  f32  largest absolute error                        (Omega, inf-norm)
 * Per item: count (i32, group size n), vmin and vmax (f32, the stored
 * metadata of Sec. III-D).  Offsets are byte offsets from the buffer start.
 */
typedef struct {
    int64_t n_items;
    int32_t n_bits;
    int32_t n_ratios;
    int32_t n_channels;
    int32_t group_size;
    int64_t item_begin[MGS_MAX_RATIOS + 1];
    int64_t n_groups[MGS_MAX_RATIOS];
    int64_t off_sse;
    int64_t off_l1;
    int64_t off_hbits;
    int64_t off_linf;
    int64_t off_count;
    int64_t off_vmin;
    int64_t off_vmax;
    int64_t total_bytes;
} mgs_table_layout;

/* Rate and distortion models of the solver. */
#define MGS_RATE_ENTROPY 0 /* rate = hbits (entropy bound, Sec. III-F) */
#define MGS_RATE_FIXED 1   /* rate = n * b bits (Eq. (eq:size_estim), P_ij * Q_ij) */
#define MGS_NORM_SSE 0     /* Omega = sum of squared errors */
#define MGS_NORM_L2 1      /* Omega = sum over groups of sqrt(SSE) */
#define MGS_NORM_L1 2      /* Omega = sum of absolute errors */
#define MGS_NORM_LINF 3    /* Omega = sum over groups of the largest error */

typedef struct {
    int32_t rate_model;          /* MGS_RATE_* */
    int32_t norm;                /* MGS_NORM_* */
    double const_bytes;          /* C of Eq. (eq:size_estim): exact bytes of coordinates etc. */
    double meta_bytes_per_group; /* per (channel, group) metadata; 9 = FP32 min + max + 1 B width */
    double delta_bytes;          /* S_Delta of Eq. (eq:size_estim): calibration offset, usually 0 */
} mgs_solve_opts;

/*
 * Result of a budget solve.  The arrays are caller-provided and may be NULL:
 *   choice[n_channels * n_groups[r]]  option index per (c, g) of the chosen ratio
 *   ratio_status[n_ratios]   0 = solved, 1 = skipped (top bit-widths stay under
 *                            the budget: tau too small, Alg. 1), -1 = infeasible
 *   ratio_objective, ratio_bytes, ratio_lp_bound [n_ratios]
 */
typedef struct {
    int32_t r_index;     /* chosen ratio; -1 if no ratio is feasible */
    double est_bytes;    /* estimated size of the chosen configuration */
    double objective;    /* its total distortion */
    double lp_bound;     /* LP-relaxation lower bound of that ratio's optimum */
    uint8_t *choice;
    int32_t *ratio_status;
    double *ratio_objective;
    double *ratio_bytes;
    double *ratio_lp_bound;
} mgs_solution;

/* ---- context --------------------------------------------------------- */

/* Create a context on CUDA device `device`.  Allocates the entropy tables
 * (L(n) = n log2 n and L(n) - L(n - 1) in units of 2^-22 bits, n <= MGS_MAX_GROUP).
 * Sets the release threshold of the device's default memory pool to keep freed
 * memory (the library's stream-ordered allocations are then recycled; memory
 * freed into that pool is not returned to the driver until the process ends
 * or the pool is trimmed). */
mgs_status mgs_create(int32_t device, mgs_ctx **out);
/* Destroy a context; its scenes must have been destroyed first. */
mgs_status mgs_destroy(mgs_ctx *ctx);
/* Message of the last failing call on this thread ("" if none).  Static
 * thread-local storage: valid until the next call on the same thread. */
const char *mgs_last_error(void);
/* Library version string. */
const char *mgs_version(void);
/* Number of CUDA kernels this library has enqueued in this process so far
 * (a CUDA-graph replay counts the kernels it runs). */
int64_t mgs_kernel_launches(void);

/*
 * Failure injection for tests of error handling (no counterpart in the
 * paper).  After mgs_debug_fail_allocation(nth), the nth stream-ordered device
 * allocation the library makes from then on (1 = the next one; scenes, their
 * staging and sort scratch, kept lists, cost tables, launch scratch, solver
 * workspaces, served jobs' tables) fails as if the device were out of memory:
 * nothing is allocated and the call that needed it returns its usual error
 * (MGS_ERR_OUT_OF_MEMORY or MGS_ERR_CUDA) after releasing what it holds.
 * nth = 0 disarms.  Process-wide, for every context and thread.
 * mgs_debug_allocations returns how many such allocations have been made.
 */
mgs_status mgs_debug_fail_allocation(int64_t nth);
int64_t mgs_debug_allocations(void);

/*
 * Inspection of the cost kernel's shared-memory histogram plan for tile
 * configuration `config` (mgs_tile_config_name) and the bit-widths bits[n_bits]
 * (ascending, 1..16), for tests of the host logic; host only, no device needed.
 * Writes at most `capacity` int32 to `out` (may be NULL) and returns how many
 * the plan has (negative on a bad argument):
 *   [0] shared memory of a CTA (bytes), [1] the budget for the configuration's
 *   CTAs per SM, [2] 1 if every large option has its own table, [3] region A
 *   words, [4] region B words, [5] small options, [6] of them lane tables,
 *   [7] direct tables, [8] finishing units U;
 *   then per option k: mode (0 lane, 1 direct, 2 16-bit pairs, 3 8-bit
 *   counters), word offset (region A for small options, region B for large
 *   ones when [2] = 1), words, byte-counter windows, 16-bit-pair windows;
 *   then per unit: option, first bin, end bin.
 */
int32_t mgs_debug_cost_plan(int32_t config, int32_t n_bits, const int32_t *bits, int32_t *out, int32_t capacity);

/* ---- scenes ----------------------------------------------------------- */

/*
 * Make a scene resident on the device: validate (finite values, finite
 * per-channel range), rank by importance (Sec. III-A: descending importance,
 * ties by ascending index), order by Morton code of the position (Sec. III-G:
 * 21-bit axis codes over the scene's bounding box, ties by index), and copy
 * the attributes into Morton order in 8-channel slabs.
 *   attrs       [n][n_channels] FP32 row-major, host or device
 *   importance  [n] FP32 (joint importance I_g), host or device
 * Synchronous on `stream`: returns after validation.  Errors:
 * INVALID_ARG (n < 1, n >= 2^31, n_channels < 3 or > MGS_MAX_CHANNELS),
 * NONFINITE, RANGE, OUT_OF_MEMORY, CUDA.
 */
mgs_status mgs_scene_create(mgs_ctx *ctx, const float *attrs, const float *importance, int64_t n,
                            int32_t n_channels, void *stream, mgs_scene **out);

/*
 * Preprocessing ahead of mgs_scene_create (Sec. III-A "Gaussians Pruning",
 * view-independent importance; Sec. III-D "Attribute Transformation",
 * Replacement).  For a 3D-GS scene in the 59-channel layout (channels 52..54
 * log-scales, 55..58 the rotation quaternion [w, x, y, z]):
 *   attrs_out [n][58]   channels 0..54 copied; 55..57 = Euler angles
 *                       [phi, theta, psi] of the normalised quaternion (radians;
 *                       a zero quaternion gives zeros)
 *   importance_out [n]  I_g = I_d * V_norm^beta with I_d = view_importance,
 *                       V = exp(s0 + s1 + s2) the product of the scales,
 *                       V_norm = min(V / V_q, 1) (1 when V_q = 0), V_q the
 *                       lower 0.9-quantile of V (the element of ascending rank
 *                       floor(9 (n - 1) / 10), selected exactly)
 *   vq_out              (host, may be NULL) V_q
 * All arrays are device memory.  Volumes and importance in FP32 (CUDA's expf,
 * powf); Euler angles in FP64 (the printed formula is ill-conditioned near
 * theta = +-pi/2), rounded to FP32.
 * Synchronous on `stream` (it returns V_q and the input check); a temporary
 * device workspace of 4 n + 512 KiB bytes is allocated on `stream`.
 * Errors: INVALID_ARG (NULL, n < 1, beta < 0 or not finite),
 * NONFINITE (a log-scale, quaternion or I_d value is NaN or infinite).
 */
mgs_status mgs_preprocess(mgs_ctx *ctx, const float *attrs, const float *view_importance, int64_t n,
                          double beta, float *attrs_out, float *importance_out, float *vq_out,
                          void *stream);
mgs_status mgs_scene_destroy(mgs_scene *scene);
/* n, channel count and device bytes held by the scene (any may be NULL). */
mgs_status mgs_scene_info(const mgs_scene *scene, int64_t *n, int32_t *n_channels,
                          int64_t *device_bytes);
/* Copy the Morton code of each Gaussian (uint64 [n], index order) and the
 * Morton permutation (int32 [n]: Gaussian at Morton position p) to device
 * buffers; either may be NULL. */
mgs_status mgs_scene_morton(const mgs_scene *scene, uint64_t *codes, int32_t *order, void *stream);

/*
 * RAHT of a resident scene (Sec. III-D "Region Adaptive Hierarchical
 * Transform").  The Gaussians are voxelised at octree depth `depth` (1..21):
 * the voxel of a Gaussian is its Morton code >> 3 (21 - depth), with the
 * scene's Morton reading (per-axis bounding box, 21 bits per axis).  A voxel's
 * value is the mean of its Gaussians (summed in Morton order) and its weight 1.  Step s = 0 .. 3 depth - 1 merges the nodes whose voxel codes
 * agree above bit s + 1 -- along x, then y, then z, finest level first -- by
 * the transform T with entries t1 = sqrt(w1) / sqrt(w1 + w2) and
 * t2 = sqrt(w2) / sqrt(w1 + w2):
 *   DC = t1 x1 + t2 x2,  weight w1 + w2,     AC = t1 x2 - t2 x1,
 * with x1 the node of the lower code; an unpaired node moves up unchanged.
 *   channels [n_channels]      host: the scene channels to transform (1..64 of them)
 *   keep                       0 (or n): every Gaussian; otherwise the kept set of the
 *                              `keep` most important (Sec. III-A), as for the cost tables
 *   dc_out [n_channels]        host: the final DC coefficient of each channel
 *   ac_out [(n - 1)][n_channels] device (capacity for the scene's n Gaussians):
 *                              the V - 1 AC coefficients, step by step, in
 *                              ascending voxel code within a step
 *   n_voxels_out               host: V
 * FP32 arithmetic (each merge is an orthonormal rotation: a coefficient's
 * error stays within a few ulp per level of sqrt(w) |x| of its node).
 * Synchronous on `stream` (three host round trips: the voxel count, the
 * merges per step, the DC); allocates a device workspace of about
 * (54 + 4 n_channels) n bytes on `stream`.
 */
mgs_status mgs_raht(mgs_ctx *ctx, const mgs_scene *scene, const int32_t *channels, int32_t n_channels,
                    int32_t depth, int64_t keep, float *dc_out, float *ac_out, int64_t *n_voxels_out,
                    void *stream);

/* ---- cost table --------------------------------------------------------- */

/* Fill `out` for a scene of n Gaussians with n_channels channels. */
mgs_status mgs_table_layout_for(int64_t n, int32_t n_channels, const mgs_grid *grid,
                                mgs_table_layout *out);

/*
 * Build the candidate cost table (Sec. III-F: Omega[c][g][b] for every ratio,
 * plus the entropy bound per option).  For every ratio r, channel c, group g
 * and bit-width b: min m and max M of the group's values, S = (M - m) / 2^b,
 * Z = round(2^b - M / S), codes q = round(clamp(v / S + Z, 0, 2^b - 1))
 * (Sec. III-D; round = nearest, ties to even), reconstruction
 * (q - Z) * S, its errors, and the histogram of q.  A group whose S is 0 is
 * degenerate: all codes 0, no error, zero entropy.  Codes and histograms are
 * exact FP32 evaluations of those formulas; error sums are FP32 per thread and
 * tree-reduced (relative error below 1e-5 against FP64); the entropy bound is
 * an integer sum of L(h) = h log2 h rounded to 2^-22 bits (error at most
 * (bins + 1) * 2^-23 bits).
 *   table  layout.total_bytes bytes, device or host (host: copied back, the
 *          stream is synchronised).
 */
mgs_status mgs_build_cost_table(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid,
                                void *table, void *stream);

/*
 * The same table computed the way a plain per-configuration search does it:
 * one launch per (ratio, bit-width), each re-reading the group data.  Kept as
 * the comparator of the fused path; results equal mgs_build_cost_table's up to
 * the FP32 summation order.
 */
mgs_status mgs_build_cost_table_plain(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid,
                                      void *table, void *stream);

/*
 * The same table as mgs_build_cost_table, from the same fused kernel, which
 * also writes out what it counted (Sec. III-D codes; the histograms behind the
 * Sec. III-F entropy bound) so that they can be checked or inspected:
 *   hist  (device, or NULL): uint32 [n_items][sum_k 2^bits[k]]; row `item`
 *         (table order [r][c][g]) holds option k's 2^bits[k] bin counts at
 *         offset sum_{j<k} 2^bits[j]; every bin is written (zeros included).
 *   codes (device, or NULL): uint16; ratio r's block starts at
 *         sum_{r'<r} n_channels * n_bits * keep[r'] and holds
 *         [n_channels][n_bits][keep[r]] codes, group g of a channel at
 *         elements [g * G, g * G + n_g) in the group's (Morton) order.
 * hist_capacity / codes_capacity are the entries available; a smaller
 * buffer is MGS_ERR_INVALID_ARG.  Runs the default tile of the group size
 * (group sizes above 16384 are not supported).  Meant for test-sized scenes:
 * the histogram array grows with 2^16 per item at b = 16.
 */
mgs_status mgs_build_cost_table_probe(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid,
                                      void *table, uint32_t *hist, int64_t hist_capacity,
                                      uint16_t *codes, int64_t codes_capacity, void *stream);

/*
 * The cost table of an arbitrary coefficient array -- e.g. the RAHT AC
 * coefficients of mgs_raht (Sec. III-D: after RAHT the AC coefficients are
 * the quantised signal) -- with the same quantiser, errors and entropy bound
 * as mgs_build_cost_table.  coeffs [m][n_channels] row-major FP32, device.
 * Ratio r of `grid` takes the first keep[r] coefficients, in their order, cut
 * into consecutive groups of grid->group_size (no importance ranking and no
 * Morton reordering: the array's order is the group order).  `table` may be
 * device or host memory (layout from mgs_table_layout_for(m, n_channels, grid)).
 * Synchronous on `stream` (it validates the array first); allocates a slab
 * copy of the coefficients (4 m * ceil(n_channels / 8) * 8 bytes) on `stream`.
 * Errors: INVALID_ARG, NONFINITE (a NaN or infinite coefficient), RANGE (a
 * channel's max - min overflows FP32).
 */
mgs_status mgs_build_cost_table_coeffs(mgs_ctx *ctx, const float *coeffs, int64_t m, int32_t n_channels,
                                       const mgs_grid *grid, void *table, void *stream);

/*
 * Several scenes, one persistent launch over all their (scene, ratio, group,
 * channel-chunk) work items.  grids[s] is scene s's grid (its own kept-set
 * sizes); all grids share the group size and the bit-widths.  tables[s]
 * follows mgs_table_layout_for(n_s, C_s, &grids[s]) and must be device memory.
 */
mgs_status mgs_build_cost_tables_batched(mgs_ctx *ctx, int32_t n_scenes,
                                         const mgs_scene *const *scenes, const mgs_grid *grids,
                                         void *const *tables, void *stream);

/* ---- batched plans, CUDA graphs and tile shapes ------------------------- */

typedef struct mgs_plan mgs_plan;

/*
 * A reusable batched launch: the kept lists of every scene for the grid, the
 * (scene, ratio) segment table in device memory and the tile shape are built
 * once; mgs_plan_launch then enqueues one persistent kernel over every
 * (scene, ratio, group, channel-chunk) work item.  With use_graph != 0 the
 * first launch captures that work into a CUDA graph and later launches replay
 * it.  grids[s] is scene s's grid (all share the group size and bit-widths);
 * tables[s] follows mgs_table_layout_for(n_s, C_s, &grids[s]), device memory;
 * the scenes and tables must outlive the plan.
 */
mgs_status mgs_plan_create(mgs_ctx *ctx, int32_t n_scenes, const mgs_scene *const *scenes,
                           const mgs_grid *grids, void *const *tables, int32_t use_graph,
                           void *stream, mgs_plan **out);
mgs_status mgs_plan_launch(mgs_plan *plan, void *stream);
mgs_status mgs_plan_destroy(mgs_plan *plan);
/* Work items and kernel launches of one mgs_plan_launch. */
mgs_status mgs_plan_info(const mgs_plan *plan, int64_t *work_items, int32_t *launches,
                         int32_t *tile_config);

/*
 * Tile shapes of the cost kernel: threads per CTA x elements per thread
 * (>= G) x channels per work item.  mgs_set_tile_config pins one for a
 * (group size, bit-width count) pair on this context (-1 restores the
 * default); mgs_autotune times every shape that can hold the grid's group
 * size on this scene and pins the fastest.  ms_per_config[count] (may be
 * NULL) receives each shape's time, or -1 where it does not apply.
 */
int32_t mgs_tile_config_count(void);
const char *mgs_tile_config_name(int32_t config);
mgs_status mgs_set_tile_config(mgs_ctx *ctx, int32_t group_size, int32_t n_bits, int32_t config);
mgs_status mgs_autotune(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid, void *stream,
                        int32_t *chosen, float *ms_per_config);

/* ---- codes of one configuration ---------------------------------------- */

/*
 * Quantise one chosen configuration (Sec. III-D): kept-set size `keep`, group
 * size G, bit-width bits[c * n_groups + g] (uint8, 1..16) per (channel, group).
 *   codes   [n_channels][keep] uint16, device: code of the j-th kept Gaussian
 *           in Morton order
 *   minmax  [n_channels][n_groups][2] FP32, device: group min and max
 *   bits    device
 */
mgs_status mgs_quantize_groups(mgs_ctx *ctx, const mgs_scene *scene, int64_t keep,
                               int32_t group_size, const uint8_t *bits, uint16_t *codes,
                               float *minmax, void *stream);

/*
 * mgs_quantize_groups without any allocation.  The paper has no counterpart:
 * this is an interface for callers that must not allocate device memory
 * while they run -- processes whose device memory is owned and capped by
 * another framework's allocator (an allocation there can fail or steal the
 * other framework's headroom), and real-time encoder threads with a
 * no-allocation rule (an allocation can block or synchronise the device).
 * Same arguments, results and errors as mgs_quantize_groups, and the caller
 * still provides every input and output.
 *
 * The scratch it needs (the kept list and its per-tile counts) lives in
 * file-scope device arrays of fixed size that every GPU loading this library
 * holds until the process exits: at most MGS_NOALLOC_MAX_KEEP kept Gaussians
 * (16 MiB of indices) of a scene of at most MGS_NOALLOC_MAX_SCENE Gaussians;
 * larger requests return MGS_ERR_INVALID_ARG.  The first call on a device looks
 * up the arrays' device addresses (cudaGetSymbolAddress, once per device), and
 * with lazy module loading that lookup may load the library's device code and
 * block; make that first call during set-up, before any stream capture and
 * before entering a thread that must not block.  Later calls do not look up
 * anything.  Every call shares the arrays and
 * they keep the last call's contents (nothing in them needs clearing): calls
 * that overlap on the GPU (different streams, or different host threads with
 * no ordering between them) race on the scratch and must be serialised.
 */
#define MGS_NOALLOC_MAX_KEEP 4194304
#define MGS_NOALLOC_MAX_SCENE 16777216
mgs_status mgs_quantize_groups_noalloc(mgs_ctx *ctx, const mgs_scene *scene, int64_t keep,
                                       int32_t group_size, const uint8_t *bits, uint16_t *codes,
                                       float *minmax, void *stream);

/* ---- block coder: the actual size of a configuration -------------------- */

/*
 * Compress one configuration and measure it: Alg. 1's "compress the model
 * with the current hyperparameters, obtain its size S_a", with entropy coding
 * as in Sec. III-G (the paper codes with torchac + LZ77; this block format is
 * the library's own).  The kept set of `keep` Gaussians (Sec. III-A, Morton
 * order) is cut into groups of group_size, each (channel, group) is quantised
 * with bits[c * n_groups + g] (1..16, host or device memory) exactly as
 * mgs_quantize_groups does, and each block of n codes is written as
 *
 *   b:u8  min:f32  max:f32            metadata (9 bytes, little-endian)
 *   nothing more when max - min == 0  (R = 0: every code is 0), else
 *   mode:u8                           0 = raw, 1 = rANS (the shorter one; raw on ties)
 *   raw:  ceil(n b / 8) bytes: bit j of code i is stream bit i b + j, and
 *         stream bit t is bit t % 8 of byte t / 8
 *   rANS: the table's bits (same order), zero-padded to a byte:
 *           gamma(D), then per distinct code in ascending order gamma(gap)
 *           and gamma(f), gap = code - previous code (first: code + 1);
 *         lanes x u32: the encoder's final states, lane 0 first;
 *         the renormalisation bytes in the order a decoder reads them.
 *   gamma(x), x >= 1: floor(log2 x) zero bits, then x's bits from the top.
 *
 * Model: M = 2^ceil(log2 n); f = floor(count * M / n), and M - sum f is added
 * to the most frequent code (the lowest one on ties).  rANS: states in
 * [2^23, 2^31), byte renormalisation (emit the low byte while
 * x >= 2^(31 - log2 M) * f, then x = floor(x / f) M + x mod f + cum);
 * lanes = min(32, max(1, n / 512)) interleaved states, lane j coding the
 * symbols i = j (mod lanes); encoding runs from the last symbol to the first.
 *
 * Blocks are concatenated in (channel, group) order.  stream (device memory,
 * `capacity` bytes; may be NULL to measure only) receives them;
 * block_bytes[c * n_groups + g] (host or device, may be NULL) each block's
 * size; *total_bytes (host) the stream's length.  The call allocates its
 * workspace on `stream` and synchronises it.  Errors: INVALID_ARG (a width
 * outside 1..16, keep or group_size out of range, capacity too small: the
 * needed length is still returned in *total_bytes), OUT_OF_MEMORY, CUDA.
 */
mgs_status mgs_encode_config(mgs_ctx *ctx, const mgs_scene *scene, int64_t keep,
                             int32_t group_size, const uint8_t *bits, uint8_t *stream,
                             int64_t capacity, int32_t *block_bytes, int64_t *total_bytes,
                             void *cuda_stream);
/* Largest stream mgs_encode_config can write: C * (10 * n_groups + 2 * keep)
 * bytes (-1 for invalid arguments). */
int64_t mgs_encode_bound(int64_t keep, int32_t group_size, int32_t n_channels);

/* ---- Alg. 1 with real compression: the S_Delta calibration loop ---------- */

typedef struct {
    double budget_bytes;   /* S_T */
    double tolerance;      /* stop once |S_a - S_T| / S_T < tolerance (Alg. 1: 0.05) */
    int32_t max_rounds;    /* ILP + compression rounds per ratio after the first compression */
    int32_t init_bits;     /* Alg. 1's initial width (8); with MGS_RATE_ENTROPY it must be
                              one of the grid's widths */
    mgs_solve_opts solve;  /* rate model (MGS_RATE_FIXED: Eq. (eq:size_estim)'s sum P Q),
                              norm, const_bytes (C, added to every actual size too),
                              meta_bytes_per_group; delta_bytes is ignored (calibrated) */
} mgs_calib_opts;

/*
 * Result of mgs_search_calibrated.  Arrays are caller-provided and may be NULL:
 *   bits[n_channels * n_groups[r_index]]  the chosen widths (capacity: the
 *                          largest ratio's n_channels * n_groups)
 *   ratio_status[n_ratios] 0 converged, 1 skipped (twice the initial size is
 *                          under the budget: tau too small), 2 not converged in
 *                          max_rounds, -1 infeasible
 *   ratio_rounds           compressions run for the ratio
 *   ratio_actual           its last actual size S_a (bytes, coded + const_bytes)
 *   ratio_delta            its last S_Delta
 *   ratio_objective        Omega of its last ILP solution
 */
typedef struct {
    int32_t r_index;       /* chosen ratio; -1 if none converged */
    int32_t rounds;        /* compressions run in total */
    double actual_bytes;   /* S_a of the chosen configuration */
    double est_bytes;      /* its calibrated estimate (Eq. (eq:size_estim) with S_Delta) */
    double objective;      /* its Omega */
    uint8_t *bits;
    int32_t *ratio_status;
    int32_t *ratio_rounds;
    double *ratio_actual;
    double *ratio_delta;
    double *ratio_objective;
} mgs_calib_result;

/*
 * Alg. 1 with real compression.  For each ratio r (grid order): compress with
 * every width init_bits (mgs_encode_config's coder) to get S_a; skip r when
 * 2 S_a < S_T; otherwise repeat up to max_rounds times: S_Delta = S_a minus
 * the estimate (Eq. (eq:size_estim) without S_Delta) of the configuration just
 * compressed; solve Eq. (eq:ilp) for r alone with that S_Delta (the device
 * solver); compress the solution; stop once |S_a - S_T| / S_T < tolerance.
 * Among the converged ratios the smallest Omega wins (ties: the larger
 * ratio).  `table` is the scene's cost table for `grid` (device memory, laid
 * out by `layout`).  The ratios run concurrently, each on a host thread (at
 * most 16) with its own stream that starts after the work already queued on
 * `stream`; each ratio's rounds, and so the result, are the same as when they
 * run one after another.  Synchronises `stream`.  INFEASIBLE if no ratio
 * converged (the per-ratio arrays are still filled); INVALID_ARG for
 * mismatched grid, layout and scene or bad options.
 */
mgs_status mgs_search_calibrated(mgs_ctx *ctx, const mgs_scene *scene, const mgs_grid *grid,
                                 const void *table, const mgs_table_layout *layout,
                                 const mgs_calib_opts *opts, mgs_calib_result *out, void *stream);

/* ---- vector quantisation of the 1+D SH coefficients ----------------------- */

/*
 * Sec. III-D "Clustering 1+D SH Coefficients": each SH vector is replaced by
 * the index of a codebook entry.  Decisions are reproducible bit for bit: the
 * score of entry k for vector x is fl(|c_k|^2 - 2 x.c_k) (|x|^2 is dropped; it
 * does not change the argmin), both sums accumulated by fmaf over the D
 * dimensions in ascending order; the smallest score wins, ties to the lower
 * k.
 *   x         [n][D] FP32, device, row-major (1 <= D <= 64, n < 2^31)
 *   codebook  [K][D] FP32, device (1 <= K <= 2^20)
 *   index_out [n] int32, device: the chosen entry
 *   score_out [n] FP32, device, may be NULL: its score (add |x|^2 for the
 *             squared distance)
 * Stream-ordered; workspace is allocated on `stream`.
 */
mgs_status mgs_vq_assign(mgs_ctx *ctx, const float *x, int64_t n, int32_t D, const float *codebook,
                         int32_t K, int32_t *index_out, float *score_out, void *stream);

/*
 * The batched clustering the paper cites (Sculley's mini-batch k-means): for
 * t = 0 .. iters - 1, the vectors x[batches[t][j]] are assigned as by
 * mgs_vq_assign, then every entry with m > 0 of them moves to the running
 * mean of all vectors ever assigned to it: c = (v c + sum x) / (v + m), the
 * sum in FP64 in batch order, rounded once to FP32, and v += m.  This is the
 * per-vector update with learning rate 1 / count, carried out exactly over
 * each batch.  The random batches are the caller's (device int32
 * [iters][batch], each a row of x; checked on the device).  codebook and
 * counts ([K] int64, zero for a fresh codebook; K <= 49152 here) are updated
 * in place; assign_out ([iters][batch] int32, device, may be NULL) receives
 * every batch's assignment.  Stream-ordered apart from one 4-byte read-back
 * of the batch check.
 */
mgs_status mgs_vq_train(mgs_ctx *ctx, const float *x, int64_t n, int32_t D, float *codebook,
                        int32_t K, int64_t *counts, const int32_t *batches, int32_t iters,
                        int32_t batch, int32_t *assign_out, void *stream);

/*
 * Where the scores are computed.  By default (enable = 1) x.c is computed on
 * the tensor cores (tcgen05.mma, TF32 inputs, FP32 accumulators) and every
 * entry whose approximate score lies within twice the bound of the TF32
 * error of the best one is re-scored exactly as above, so the results are
 * the same; enable = 0 scores every entry on the CUDA cores.
 * mgs_vq_stats returns, and resets, the scores of the tensor path since the
 * last call and how many of them were re-scored exactly.  With the tensor
 * path, mgs_vq_assign and mgs_vq_train synchronise `stream` and return
 * MGS_ERR_TIMEOUT if a bounded wait of the tensor-core pipeline ran out.
 */
mgs_status mgs_vq_set_tensor_cores(mgs_ctx *ctx, int32_t enable);
mgs_status mgs_vq_stats(mgs_ctx *ctx, int64_t *scores, int64_t *rescored);
/*
 * Clock-cycle limit of each bounded wait of the tensor-core pipeline (a copy
 * or an MMA that has not completed by then is a failure: the CTA drains its
 * own copies and MMAs, frees its tensor memory, and the call returns
 * MGS_ERR_TIMEOUT).  0 restores the default, about one second.  No
 * counterpart in the paper: failure detection, and tests of it (a limit of a
 * few cycles makes the waits run out without any fault).
 */
mgs_status mgs_vq_set_wait_limit(mgs_ctx *ctx, int64_t cycles);

/*
 * Budget-first retention: the vectors of rows[0 .. n_retain) (the top-ranked
 * Gaussians, whose original SH the remaining budget keeps) are appended to
 * the codebook as entries K, K + 1, ...; their indices are rewritten to
 * index[rows[j]] = K + j (device memory; rows must be distinct rows of
 * index).  Appending the vectors themselves is the caller's copy.
 */
mgs_status mgs_vq_retain(mgs_ctx *ctx, const int32_t *rows, int64_t n_retain, int32_t K,
                         int32_t *index, void *stream);

/* ---- serving ------------------------------------------------------------ */

/*
 * A search server: jobs (a scene in host memory, a grid and a byte budget) are
 * submitted at any time and each is answered with Alg. 1's result (the chosen
 * ratio and bit-widths).  Continuous batching: a job is admitted while fewer
 * than max_jobs are in flight and its device footprint fits hbm_budget_bytes
 * (a lone job is always admitted); an ingest thread makes its scene resident;
 * a compute thread runs one persistent launch per iteration over a slice of
 * the remaining work items of every admitted job (about slice_items items per
 * launch, 0 = all; an eighth of that while a scene is being made resident, so
 * that its build is not held up by a long launch), so jobs that arrive while
 * others are on the GPU join the next launch; each finished table is solved on the device
 * (mgs_solve_budgets_device) by one of solver_threads host threads, each with
 * its own stream, while the next launches run.  A job's results are the same
 * whichever jobs it shares launches with.
 */
typedef struct mgs_server mgs_server;

typedef struct {
    int32_t max_jobs;          /* jobs admitted at once (>= 1) */
    int32_t solver_threads;    /* threads driving the device solve of finished tables (>= 1) */
    int64_t hbm_budget_bytes;  /* device memory the server may hold for jobs (scene, table,
                                  solver workspace) */
    int64_t slice_items;       /* work items per batched launch (0 = everything ready) */
} mgs_server_opts;

typedef struct {
    const float *attrs;        /* [n][n_channels] host memory, valid until the job is done */
    const float *importance;   /* [n] host memory, valid until the job is done */
    int64_t n;
    int32_t n_channels;
    mgs_grid grid;             /* copied at submission */
    double budget_bytes;
    mgs_solve_opts opts;
    void *table_out;           /* optional host buffer of mgs_table_layout_for(n, n_channels,
                                  grid).total_bytes bytes: when non-NULL the job's finished cost
                                  table is copied there before the solve (to check it, or to
                                  solve other budgets later); valid until the job is done */
} mgs_job;

typedef struct {
    mgs_status status;         /* the job's own status (MGS_OK or its error) */
    int32_t r_index;
    double est_bytes;
    double objective;
    double lp_bound;
    int64_t n_choice;          /* entries of the chosen ratio's option array */
    double t_submit, t_admit, t_ready, t_table, t_done;   /* seconds since server start */
} mgs_job_result;

mgs_status mgs_server_create(mgs_ctx *ctx, const mgs_server_opts *opts, mgs_server **out);
mgs_status mgs_server_submit(mgs_server *server, const mgs_job *job, int64_t *job_id);
/* Wait up to timeout_ms for a job; MGS_ERR_TIMEOUT if it is not done by then.
 * choice[choice_capacity] (may be NULL) receives the chosen options. */
mgs_status mgs_server_wait(mgs_server *server, int64_t job_id, int32_t timeout_ms,
                           mgs_job_result *out, uint8_t *choice, int64_t choice_capacity);
/* Batched launches and work items run so far, jobs in flight, bytes held. */
mgs_status mgs_server_stats(mgs_server *server, int64_t *launches, int64_t *work_items,
                            int32_t *in_flight, int64_t *used_bytes);
/* Finish every admitted job, then stop the threads and free the server. */
mgs_status mgs_server_destroy(mgs_server *server);

/* ---- size estimate and budget solve (host) ------------------------------ */

/*
 * Estimated size (Eq. (eq:size_estim)) of ratio r_index with option
 * choice[c * n_groups[r] + g]:
 *   bytes = sum rate / 8 + meta_bytes_per_group * n_items(r) + const_bytes + delta_bytes
 * `table` is host memory laid out by `layout`.
 */
mgs_status mgs_estimate_size(const void *table, const mgs_table_layout *layout,
                             const mgs_grid *grid, int32_t r_index, const uint8_t *choice,
                             const mgs_solve_opts *opts, double *bytes_out);

/*
 * Solve Eq. (eq:ilp) for every ratio (a multiple-choice knapsack over the
 * (channel, group) items) and pick tau per Alg. 1: ratios whose all-top-bit-
 * width size stays under the budget are skipped (tau too small); among the
 * others the smallest total distortion wins (ties: larger ratio); if all
 * feasible ratios are skipped the largest feasible one is taken.  Per ratio
 * the solver takes the LP relaxation over each item's lower convex hull and
 * rounds it to an integral choice by greedy upgrades; the LP value is returned
 * as a lower bound.  Rates are taken in integer units of 2^-22 bits (entropy
 * rates are rounded to that unit; a cost table's are exact multiples of it),
 * so size sums are exact.  `table` is host memory.  INFEASIBLE if no ratio
 * fits.
 */
mgs_status mgs_solve_budget(const void *table, const mgs_table_layout *layout,
                            const mgs_grid *grid, double budget_bytes, const mgs_solve_opts *opts,
                            mgs_solution *out);

/*
 * mgs_solve_budget for several budgets over the same table: the per-item hulls
 * are built once and every (budget, ratio) pair is solved in parallel.
 * out[i] answers budgets[i]; returns MGS_ERR_INFEASIBLE if any budget is
 * infeasible (that entry has r_index = -1; the others are filled).
 */
mgs_status mgs_solve_budgets(const void *table, const mgs_table_layout *layout,
                             const mgs_grid *grid, int32_t n_budgets, const double *budgets,
                             const mgs_solve_opts *opts, mgs_solution *out);

/*
 * The paper's hierarchical solve of Eq. (eq:ilp) (Sec. III-F "Hierarchical
 * Solver"), per ratio: (1) one width per channel, from the multiple-choice
 * knapsack whose items are the channels (a channel's option sums its groups'
 * losses, in the chosen norm, and rates; its metadata is its groups'); (2)
 * channel budgets S_c = A * Q_c / sum_c Q_c, A = budget - const_bytes -
 * delta_bytes; (3) per channel, the knapsack over its groups within S_c.
 * Every knapsack is the flat solver's (mgs_solve_budgets).  A ratio is
 * infeasible when step (1) or any channel's step (3) is.  tau is picked as by
 * mgs_solve_budget; out->choice and the per-ratio arrays are filled the same
 * way (ratio_lp_bound holds the sum of the channels' LP bounds).  `table` is
 * host memory.
 */
mgs_status mgs_solve_hierarchical(const void *table, const mgs_table_layout *layout,
                                  const mgs_grid *grid, double budget_bytes,
                                  const mgs_solve_opts *opts, mgs_solution *out);

/*
 * mgs_solve_budgets on the device: the same answers bit for bit (the
 * arithmetic is shared: rates in units of 2^-22 bits, hull increments in
 * (efficiency, item, level) order, LP split, greedy completion, chunked
 * pairwise loss sums), computed by two kernels -- one thread per item builds
 * the hulls, one CTA per (budget, ratio) finds the split key by radix
 * selection and completes the choice -- then Alg. 1's tau pick on the host.
 * `table` may be device or host memory (a host table is copied in first).
 * Device workspace is allocated and freed on `stream`; the call synchronises
 * `stream` before returning, and `out` (host memory) is filled as by
 * mgs_solve_budgets.  The greedy completion takes one block-wide arg-min
 * per increment, so any number of increments is completed on the device.
 */
mgs_status mgs_solve_budgets_device(mgs_ctx *ctx, const void *table, const mgs_table_layout *layout,
                                    const mgs_grid *grid, int32_t n_budgets, const double *budgets,
                                    const mgs_solve_opts *opts, mgs_solution *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MGS_H */
