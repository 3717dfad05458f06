/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for the candidate
 * cost table of MesonGS++'s size-aware configuration search.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code with the
 * CUDA path (no headers, helpers or tables in common).
 *
 * Arithmetic rules: every per-element quantity is computed in IEEE FP32,
 * one operation per C statement, compiled with -ffp-contract=off and no
 * fast-math, so that each "fl(.)" below is exactly one rounding.  Every
 * accumulation (squared error, absolute error, entropy) is FP64.
 *
 * What each function follows (section names of the paper):
 *   oracle_rank          Sec. III-A "Gaussians Pruning": keep the tau fraction
 *                        with the largest joint importance I_g.
 *   oracle_morton        Sec. III-G "Entropy Encoding", last paragraph: Morton
 *                        order of the coordinates builds the quantisation groups.
 *   oracle_kept          Sec. III-A + III-G: the kept set, in Morton order.
 *   oracle_group_cost    Sec. III-D "Group-wise Attribute Quantization" (the
 *                        quantiser c_q, S_c, Z_c), Sec. III-F "Acceleration"
 *                        (quality loss Omega with 1-, 2- and inf-norms) and
 *                        Sec. III-F "Size Estimator" (entropy lower bound
 *                        tau*N * (-sum p log2 p)).
 *   oracle_cost_table    the loops of Sec. III-F: every reserve ratio, every
 *                        (channel, block), every bit-width.
 *   oracle_cost_table_mt the same items spread over POSIX threads (same
 *                        entries; used to time the oracle on every core).
 *   oracle_quantize      Sec. III-D quantiser for one chosen configuration.
 *   oracle_euler         Sec. III-D "Attribute Transformation", Replacement:
 *                        the Euler angles of a rotation quaternion.
 *   oracle_raht          Sec. III-D "Region Adaptive Hierarchical Transform":
 *                        voxels at octree depth d (Gaussians sharing a voxel
 *                        averaged), merged pairwise along x, y, z from the
 *                        finest level up; one DC and V - 1 AC coefficients.
 *   oracle_encode_block  Alg. 1 ("compress the model, obtain its size S_a")
 *   oracle_decode_block  and Sec. III-G "Entropy Encoding": a lossless coder of
 *   oracle_encode_config one (channel, group) block of codes, and of a whole
 *                        configuration, whose byte count is the actual size
 *                        that calibrates S_Delta of Eq. (eq:size_estim).  The
 *                        paper codes with torchac + LZ77; the block format
 *                        here is this library's own (static-model rANS with a
 *                        raw fallback), written out below.
 *   oracle_vq_assign     Sec. III-D "Clustering 1+D SH Coefficients": the
 *   oracle_vq_update     nearest codebook entry of each vector, and one
 *                        batch of the batched (mini-batch) k-means the paper
 *                        cites: each centre moves to the running mean of
 *                        every vector ever assigned to it.
 *   oracle_preprocess    Sec. III-A (view-independent importance I_i =
 *                        V_norm^beta, joint score I_g = I_d * I_i) and the
 *                        quaternion -> Euler replacement of Sec. III-D, over
 *                        a whole scene; FP64 arithmetic, FP32 outputs.
 *
 * Readings where the paper is silent, fixed here as follows:
 *   - S_c = (max - min) / 2^b exactly as printed (not 2^b - 1); the element
 *     equal to max lands at x ~ 2^b and is clamped to 2^b - 1.
 *   - "rounding to nearest" is round-half-to-even (rintf) for Z_c and c_q.
 *   - dequantisation (never printed) is the inverse map c_hat = (c_q - Z_c) * S_c
 *     in FP32; the error is e = c_hat - c in FP32.
 *   - a group whose scale S underflows to 0 (max == min, or a range too small
 *     for 2^-b scaling) is degenerate: every code 0, c_hat = c, one symbol.
 *   - Morton: per-axis min/max over ALL Gaussians; t = (p - lo) / (hi - lo);
 *     21-bit axis codes floor(t * 2^21) clamped to 2^21 - 1; x bit k -> code
 *     bit 3k, y -> 3k+1, z -> 3k+2; order by (code, index).
 *   - importance order: descending importance, ties by ascending index.
 *   - preprocessing: V = exp(s0 + s1 + s2) from the stored log-scales (the
 *     product of the scale vector); the normaliser is the lower 0.9-quantile
 *     of the sorted volumes (index floor(9 (n - 1) / 10), ascending);
 *     V_norm = min(V / V_q, 1) (1 if V_q = 0); the quaternion [w, x, y, z]
 *     is normalised first (a zero quaternion gives zero angles) and the
 *     square roots' arguments are clamped at 0.
 *   - RAHT: the voxel of a Gaussian at depth d is its Morton code >> 3(21 - d)
 *     (so the x, y, z bits of the voxel code are those of the Morton code);
 *     a voxel's attribute is the FP64 mean of its Gaussians, summed in Morton
 *     order, and its weight is 1; step s = 0 .. 3d - 1 merges the nodes whose
 *     codes agree above bit s + 1 (the lower node first: x1, w1) by the
 *     printed T, whose entries t1 = sqrt(w1) / sqrt(w1 + w2) and
 *     t2 = sqrt(w2) / sqrt(w1 + w2) are formed once per pair:
 *     DC = t1 x1 + t2 x2, AC = t1 x2 - t2 x1, weight w1 + w2; an unpaired
 *     node passes up unchanged.  ACs are listed step by step, in
 *     ascending code within a step.
 *   - block coder (the paper names only torchac and LZ77): see the format
 *     comment above oracle_encode_block.
 *   - vector quantisation: the score of centre k for vector x is
 *     fl(|c_k|^2 - 2 x.c_k) (|x|^2 dropped: it does not change the argmin),
 *     both sums accumulated by fmaf over the dimensions in ascending order;
 *     the smallest score wins, ties to the lower k.  The mini-batch update
 *     of a centre with count v and the m batch vectors assigned to it is
 *     c = (v c + sum x) / (v + m), the sum taken in FP64 in batch order and
 *     the result rounded once to FP32; this is the per-vector update with
 *     learning rate 1/count carried out exactly over one batch.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG -1
#define ORACLE_ERR_NONFINITE -2
#define ORACLE_ERR_RANGE -3
#define ORACLE_ERR_NOMEM -4

/* ------------------------------------------------------------------------ */
/* Importance rank (Sec. III-A).                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    float key;
    int64_t idx;
} rank_item;

static int cmp_rank(const void *a, const void *b) {
    const rank_item *x = (const rank_item *)a;
    const rank_item *y = (const rank_item *)b;
    if (x->key > y->key) return -1; /* larger importance first */
    if (x->key < y->key) return 1;
    if (x->idx < y->idx) return -1; /* ties: smaller index first */
    if (x->idx > y->idx) return 1;
    return 0;
}

/* rank_out[i] = position of Gaussian i in the order of decreasing importance. */
int oracle_rank(const float *importance, int64_t n, int32_t *rank_out) {
    if (n < 0 || (n > 0 && (!importance || !rank_out))) return ORACLE_ERR_ARG;
    rank_item *items = (rank_item *)malloc(sizeof(rank_item) * (size_t)(n > 0 ? n : 1));
    if (!items) return ORACLE_ERR_NOMEM;
    for (int64_t i = 0; i < n; i++) {
        if (!isfinite(importance[i])) {
            free(items);
            return ORACLE_ERR_NONFINITE;
        }
        items[i].key = importance[i];
        items[i].idx = i;
    }
    qsort(items, (size_t)n, sizeof(rank_item), cmp_rank);
    for (int64_t j = 0; j < n; j++) rank_out[items[j].idx] = (int32_t)j;
    free(items);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Morton order of the coordinates (Sec. III-G, last paragraph).             */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t code;
    int64_t idx;
} morton_item;

static int cmp_morton(const void *a, const void *b) {
    const morton_item *x = (const morton_item *)a;
    const morton_item *y = (const morton_item *)b;
    if (x->code < y->code) return -1;
    if (x->code > y->code) return 1;
    if (x->idx < y->idx) return -1;
    if (x->idx > y->idx) return 1;
    return 0;
}

/* Quantised axis coordinate in [0, 2^21). */
static uint32_t axis_code(float p, float lo, float hi) {
    float d = hi - lo;
    if (d == 0.0f) return 0;
    float num = p - lo;
    float t = num / d;
    double s = floor((double)t * 2097152.0);
    if (s > 2097151.0) s = 2097151.0;
    if (s < 0.0) s = 0.0;
    return (uint32_t)s;
}

/* Bit k of x goes to bit 3k, of y to 3k+1, of z to 3k+2 (one bit at a time). */
static uint64_t interleave3(uint32_t x, uint32_t y, uint32_t z) {
    uint64_t code = 0;
    for (int k = 0; k < 21; k++) {
        code |= (uint64_t)((x >> k) & 1u) << (3 * k);
        code |= (uint64_t)((y >> k) & 1u) << (3 * k + 1);
        code |= (uint64_t)((z >> k) & 1u) << (3 * k + 2);
    }
    return code;
}

/*
 * attrs: [n][n_channels] row-major FP32, channels 0..2 are the position.
 * code_out[i]: 63-bit Morton code of Gaussian i (may be NULL).
 * order_out[p]: index of the Gaussian at Morton position p.
 */
int oracle_morton(const float *attrs, int64_t n, int32_t n_channels, uint64_t *code_out,
                  int64_t *order_out) {
    if (n < 0 || n_channels < 3 || (n > 0 && (!attrs || !order_out))) return ORACLE_ERR_ARG;
    float lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
    }
    for (int64_t i = 0; i < n; i++) {
        for (int a = 0; a < 3; a++) {
            float p = attrs[i * n_channels + a];
            if (!isfinite(p)) return ORACLE_ERR_NONFINITE;
            if (p < lo[a]) lo[a] = p;
            if (p > hi[a]) hi[a] = p;
        }
    }
    for (int a = 0; a < 3 && n > 0; a++) {
        float d = hi[a] - lo[a];
        if (!isfinite(d)) return ORACLE_ERR_RANGE;
    }
    morton_item *items = (morton_item *)malloc(sizeof(morton_item) * (size_t)(n > 0 ? n : 1));
    if (!items) return ORACLE_ERR_NOMEM;
    for (int64_t i = 0; i < n; i++) {
        uint32_t q[3];
        for (int a = 0; a < 3; a++) q[a] = axis_code(attrs[i * n_channels + a], lo[a], hi[a]);
        items[i].code = interleave3(q[0], q[1], q[2]);
        items[i].idx = i;
        if (code_out) code_out[i] = items[i].code;
    }
    qsort(items, (size_t)n, sizeof(morton_item), cmp_morton);
    for (int64_t p = 0; p < n; p++) order_out[p] = items[p].idx;
    free(items);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Kept set for one reserve ratio, in Morton order (Sec. III-A, III-G).      */
/* ------------------------------------------------------------------------ */

/*
 * kept_out[j] (j < keep) = the j-th Morton position p whose Gaussian
 * order[p] has rank < keep.  Returns the number written (must equal keep).
 */
int64_t oracle_kept(const int32_t *rank, const int64_t *order, int64_t n, int64_t keep,
                    int64_t *kept_out) {
    int64_t j = 0;
    for (int64_t p = 0; p < n; p++) {
        if ((int64_t)rank[order[p]] < keep) kept_out[j++] = p;
    }
    return j;
}

/* ------------------------------------------------------------------------ */
/* One quantisation group of one channel, all bit-widths (Sec. III-D, III-F). */
/* ------------------------------------------------------------------------ */

/*
 * vals: the n values of the group (n >= 1).
 * bits[k]: bit-width of option k, 1..16.
 * Per option k: sse[k] = sum e^2, l1[k] = sum |e|, linf[k] = max |e|,
 * hbits[k] = -sum_s h_s log2(h_s / n) (entropy lower bound in bits),
 * codes[k * n + i] (optional) = c_q of element i.
 * vmin/vmax: the group min and max stored as metadata.
 */
int oracle_group_cost(const float *vals, int64_t n, const int32_t *bits, int32_t n_b,
                      double *sse, double *l1, float *linf, double *hbits, float *vmin,
                      float *vmax, uint16_t *codes) {
    if (n < 1 || n_b < 1 || !vals || !bits) return ORACLE_ERR_ARG;
    float m = vals[0];
    float M = vals[0];
    for (int64_t i = 0; i < n; i++) {
        if (!isfinite(vals[i])) return ORACLE_ERR_NONFINITE;
        if (vals[i] < m) m = vals[i];
        if (vals[i] > M) M = vals[i];
    }
    float R = M - m;
    if (!isfinite(R)) return ORACLE_ERR_RANGE;
    if (vmin) *vmin = m;
    if (vmax) *vmax = M;

    for (int32_t k = 0; k < n_b; k++) {
        int b = bits[k];
        if (b < 1 || b > 16) return ORACLE_ERR_ARG;
        float twob = (float)(1u << b);  /* 2^b, exact */
        float top = twob - 1.0f;        /* 2^b - 1, exact */
        float S = R / twob;             /* S_c = (max - min) / 2^b */
        double s2 = 0.0, s1 = 0.0;
        float smax = 0.0f;
        double h_bits = 0.0;
        if (S == 0.0f) {
            /* degenerate group: one symbol, exact reconstruction */
            if (codes)
                for (int64_t i = 0; i < n; i++) codes[(int64_t)k * n + i] = 0;
        } else {
            float t = M / S;
            float zr = twob - t;
            float Z = rintf(zr); /* Z_c = round(2^b - max / S_c) */
            uint32_t *hist = (uint32_t *)calloc((size_t)1u << b, sizeof(uint32_t));
            if (!hist) return ORACLE_ERR_NOMEM;
            for (int64_t i = 0; i < n; i++) {
                float c = vals[i];
                float y = c / S;
                float x = y + Z;                       /* c / S_c + Z_c */
                float xc = fminf(fmaxf(x, 0.0f), top); /* clamp(., 0, 2^b - 1) */
                int q = (int)rintf(xc);                /* round to nearest */
                float qz = (float)q - Z;
                float chat = qz * S;                   /* dequantised value */
                float e = chat - c;
                s2 += (double)e * (double)e;
                s1 += fabs((double)e);
                if (fabsf(e) > smax) smax = fabsf(e);
                hist[q] += 1u;
                if (codes) codes[(int64_t)k * n + i] = (uint16_t)q;
            }
            for (uint32_t s = 0; s < (1u << b); s++) {
                if (hist[s] > 0) {
                    double p = (double)hist[s] / (double)n;
                    h_bits += -(double)hist[s] * log2(p);
                }
            }
            free(hist);
        }
        if (sse) sse[k] = s2;
        if (l1) l1[k] = s1;
        if (linf) linf[k] = smax;
        if (hbits) hbits[k] = h_bits;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Full cost table (Sec. III-F): every ratio, channel, group, bit-width.     */
/* ------------------------------------------------------------------------ */

/* Number of groups of size G over a kept set of size keep (last one partial). */
int64_t oracle_n_groups(int64_t keep, int32_t G) { return (keep + G - 1) / G; }

/*
 * Items are enumerated r-major, then channel, then group:
 *   item(r, c, g) = C * sum_{r' < r} n_groups(r') + c * n_groups(r) + g
 * Per item: cnt, vmin, vmax.  Per (item, option k): index item * n_b + k.
 * keep[r] must satisfy 0 <= keep[r] <= n.
 */
int oracle_cost_table(const float *attrs, const float *importance, int64_t n, int32_t n_channels,
                      const int64_t *keep, int32_t n_r, const int32_t *bits, int32_t n_b, int32_t G,
                      double *sse, double *l1, float *linf, double *hbits, int32_t *cnt,
                      float *vmin, float *vmax) {
    if (n < 0 || n_channels < 3 || n_r < 1 || n_b < 1 || G < 1) return ORACLE_ERR_ARG;
    for (int32_t r = 0; r < n_r; r++)
        if (keep[r] < 0 || keep[r] > n) return ORACLE_ERR_ARG;
    for (int64_t i = 0; i < n * n_channels; i++)
        if (!isfinite(attrs[i])) return ORACLE_ERR_NONFINITE;
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *kept = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    float *vals = (float *)malloc(sizeof(float) * (size_t)(G));
    int rc = ORACLE_OK;
    if (!rank || !order || !kept || !vals) {
        rc = ORACLE_ERR_NOMEM;
        goto done;
    }
    rc = oracle_rank(importance, n, rank);
    if (rc) goto done;
    rc = oracle_morton(attrs, n, n_channels, NULL, order);
    if (rc) goto done;
    int64_t item = 0;
    for (int32_t r = 0; r < n_r; r++) {
        int64_t K = oracle_kept(rank, order, n, keep[r], kept);
        int64_t ng = oracle_n_groups(K, G);
        for (int32_t c = 0; c < n_channels; c++) {
            for (int64_t g = 0; g < ng; g++, item++) {
                int64_t start = g * G;
                int64_t len = K - start < G ? K - start : G;
                for (int64_t i = 0; i < len; i++)
                    vals[i] = attrs[order[kept[start + i]] * n_channels + c];
                cnt[item] = (int32_t)len;
                rc = oracle_group_cost(vals, len, bits, n_b, sse + item * n_b, l1 + item * n_b,
                                       linf + item * n_b, hbits + item * n_b, vmin + item,
                                       vmax + item, NULL);
                if (rc) goto done;
            }
        }
    }
done:
    free(rank);
    free(order);
    free(kept);
    free(vals);
    return rc;
}

/*
 * The same table with its independent (ratio, channel, group) items handed
 * out to n_threads POSIX threads (the CPU baseline on every host core).  The
 * ranks, the Morton order and the kept sets are computed once, as above; each
 * item runs oracle_group_cost unchanged, so every entry equals the
 * single-threaded table's.  n_threads < 1 means 1.
 */
typedef struct {
    const float *attrs;
    int32_t n_channels, n_b, G, n_r;
    const int32_t *bits;
    const int64_t *order;
    int64_t **kept;          /* per ratio: kept set (Morton positions into order) */
    const int64_t *K, *ng, *item0;   /* per ratio; item0 has n_r + 1 entries */
    double *sse, *l1, *hbits;
    float *linf, *vmin, *vmax;
    int32_t *cnt;
    int64_t next;
    int rc;
    pthread_mutex_t mu;
} oracle_table_job;

static void *oracle_table_worker(void *arg) {
    oracle_table_job *J = (oracle_table_job *)arg;
    float *vals = (float *)malloc(sizeof(float) * (size_t)J->G);
    if (!vals) {
        pthread_mutex_lock(&J->mu);
        J->rc = ORACLE_ERR_NOMEM;
        pthread_mutex_unlock(&J->mu);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t item = J->next;
        int stop = J->rc != ORACLE_OK || item >= J->item0[J->n_r];
        if (!stop) J->next = item + 1;
        pthread_mutex_unlock(&J->mu);
        if (stop) break;
        int32_t r = 0;
        while (J->item0[r + 1] <= item) r++;
        int64_t local = item - J->item0[r];
        int64_t c = local / J->ng[r], g = local % J->ng[r];
        int64_t start = g * J->G;
        int64_t len = J->K[r] - start < J->G ? J->K[r] - start : J->G;
        for (int64_t i = 0; i < len; i++)
            vals[i] = J->attrs[J->order[J->kept[r][start + i]] * J->n_channels + c];
        J->cnt[item] = (int32_t)len;
        int rc = oracle_group_cost(vals, len, J->bits, J->n_b, J->sse + item * J->n_b,
                                   J->l1 + item * J->n_b, J->linf + item * J->n_b,
                                   J->hbits + item * J->n_b, J->vmin + item, J->vmax + item, NULL);
        if (rc) {
            pthread_mutex_lock(&J->mu);
            J->rc = rc;
            pthread_mutex_unlock(&J->mu);
        }
    }
    free(vals);
    return NULL;
}

int oracle_cost_table_mt(const float *attrs, const float *importance, int64_t n, int32_t n_channels,
                         const int64_t *keep, int32_t n_r, const int32_t *bits, int32_t n_b, int32_t G,
                         double *sse, double *l1, float *linf, double *hbits, int32_t *cnt,
                         float *vmin, float *vmax, int32_t n_threads) {
    if (n < 0 || n_channels < 3 || n_r < 1 || n_b < 1 || G < 1) return ORACLE_ERR_ARG;
    for (int32_t r = 0; r < n_r; r++)
        if (keep[r] < 0 || keep[r] > n) return ORACLE_ERR_ARG;
    for (int64_t i = 0; i < n * n_channels; i++)
        if (!isfinite(attrs[i])) return ORACLE_ERR_NONFINITE;
    if (n_threads < 1) n_threads = 1;
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t **kept = (int64_t **)calloc((size_t)n_r, sizeof(int64_t *));
    int64_t *K = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_r);
    int64_t *ng = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_r);
    int64_t *item0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_r + 1));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    int rc = ORACLE_OK;
    if (!rank || !order || !kept || !K || !ng || !item0 || !th) {
        rc = ORACLE_ERR_NOMEM;
        goto done;
    }
    rc = oracle_rank(importance, n, rank);
    if (rc) goto done;
    rc = oracle_morton(attrs, n, n_channels, NULL, order);
    if (rc) goto done;
    item0[0] = 0;
    for (int32_t r = 0; r < n_r; r++) {
        kept[r] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(keep[r] > 0 ? keep[r] : 1));
        if (!kept[r]) {
            rc = ORACLE_ERR_NOMEM;
            goto done;
        }
        K[r] = oracle_kept(rank, order, n, keep[r], kept[r]);
        ng[r] = oracle_n_groups(K[r], G);
        item0[r + 1] = item0[r] + ng[r] * n_channels;
    }
    {
        oracle_table_job J = {attrs, n_channels, n_b, G, n_r, bits, order, kept, K, ng, item0,
                              sse, l1, hbits, linf, vmin, vmax, cnt, 0, ORACLE_OK};
        pthread_mutex_init(&J.mu, NULL);
        int started = 0;
        for (; started < n_threads; started++)
            if (pthread_create(&th[started], NULL, oracle_table_worker, &J) != 0) break;
        if (started == 0) oracle_table_worker(&J);
        for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
        pthread_mutex_destroy(&J.mu);
        rc = J.rc;
    }
done:
    if (kept)
        for (int32_t r = 0; r < n_r; r++) free(kept[r]);
    free(kept);
    free(rank);
    free(order);
    free(K);
    free(ng);
    free(item0);
    free(th);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Quantise one chosen configuration (Sec. III-D).                            */
/* ------------------------------------------------------------------------ */

/*
 * For one kept-set size `keep` and group size G, quantise every (channel,
 * group) with its chosen bit-width q_bits[c * n_groups + g].
 * codes_out[c * keep + j]: code of the j-th kept Gaussian (Morton order).
 * minmax_out[(c * n_groups + g) * 2 + {0,1}]: group min and max.
 */
int oracle_quantize(const float *attrs, const float *importance, int64_t n, int32_t n_channels,
                    int64_t keep, int32_t G, const uint8_t *q_bits, uint16_t *codes_out,
                    float *minmax_out) {
    if (n < 0 || keep < 0 || keep > n || G < 1) return ORACLE_ERR_ARG;
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *kept = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    float *vals = (float *)malloc(sizeof(float) * (size_t)G);
    uint16_t *codes = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)G);
    int rc = ORACLE_OK;
    if (!rank || !order || !kept || !vals || !codes) {
        rc = ORACLE_ERR_NOMEM;
        goto done;
    }
    rc = oracle_rank(importance, n, rank);
    if (rc) goto done;
    rc = oracle_morton(attrs, n, n_channels, NULL, order);
    if (rc) goto done;
    int64_t K = oracle_kept(rank, order, n, keep, kept);
    int64_t ng = oracle_n_groups(K, G);
    for (int32_t c = 0; c < n_channels; c++) {
        for (int64_t g = 0; g < ng; g++) {
            int64_t start = g * G;
            int64_t len = K - start < G ? K - start : G;
            for (int64_t i = 0; i < len; i++) vals[i] = attrs[order[kept[start + i]] * n_channels + c];
            int32_t b = q_bits[c * ng + g];
            double d0;
            double d1;
            float d2;
            double d3;
            rc = oracle_group_cost(vals, len, &b, 1, &d0, &d1, &d2, &d3,
                                   &minmax_out[(c * ng + g) * 2], &minmax_out[(c * ng + g) * 2 + 1],
                                   codes);
            if (rc) goto done;
            memcpy(&codes_out[(int64_t)c * K + start], codes, sizeof(uint16_t) * (size_t)len);
        }
    }
done:
    free(rank);
    free(order);
    free(kept);
    free(vals);
    free(codes);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Preprocessing (Sec. III-A view-independent importance, Sec. III-D Euler).  */
/* ------------------------------------------------------------------------ */

#define ORACLE_PI 3.14159265358979323846
#define ORACLE_PRE_CHANNELS 59   /* input layout: 52..54 log-scale, 55..58 quaternion w, x, y, z */
#define ORACLE_PRE_SCALE0 52
#define ORACLE_PRE_QUAT0 55

/* Euler angles [phi, theta, psi] of the rotation quaternion q = [w, x, y, z]
 * with the formula of Sec. III-D, after normalising q. */
void oracle_euler(const double q_in[4], double e[3]) {
    double nrm = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    if (!(nrm > 0.0)) {
        e[0] = e[1] = e[2] = 0.0;
        return;
    }
    double w = q_in[0] / nrm, x = q_in[1] / nrm, y = q_in[2] / nrm, z = q_in[3] / nrm;
    /* roll: rotation about x */
    e[0] = atan2(2.0 * (w * x + y * z), 1.0 - 2.0 * (x * x + y * y));
    /* pitch: -pi/2 + 2 atan2(sqrt(1 + 2(wy - xz)), sqrt(1 - 2(wy - xz))) */
    double t = w * y - x * z;
    double a = 1.0 + 2.0 * t, b = 1.0 - 2.0 * t;
    if (a < 0.0) a = 0.0;
    if (b < 0.0) b = 0.0;
    e[1] = -ORACLE_PI / 2.0 + 2.0 * atan2(sqrt(a), sqrt(b));
    /* yaw: rotation about z */
    e[2] = atan2(2.0 * (w * z + x * y), 1.0 - 2.0 * (y * y + z * z));
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Scene preprocessing.  attrs [n][59] (FP32), view_imp [n] = I_d.  Outputs:
 * attrs_out [n][58] (channels 0..54 unchanged, 55..57 = phi, theta, psi),
 * imp_out [n] = I_g = I_d * V_norm^beta, and *vq_out = the volume normaliser. */
int oracle_preprocess(const float *attrs, int64_t n, int32_t n_channels, const float *view_imp,
                      double beta, float *attrs_out, float *imp_out, double *vq_out) {
    if (n < 1 || n_channels != ORACLE_PRE_CHANNELS || !(beta >= 0.0)) return ORACLE_ERR_ARG;
    double *vol = (double *)malloc(sizeof(double) * (size_t)n);
    double *sorted = (double *)malloc(sizeof(double) * (size_t)n);
    if (!vol || !sorted) {
        free(vol);
        free(sorted);
        return ORACLE_ERR_NOMEM;
    }
    for (int64_t i = 0; i < n; i++) {
        const float *r = attrs + i * n_channels;
        double ls = (double)r[ORACLE_PRE_SCALE0] + (double)r[ORACLE_PRE_SCALE0 + 1] +
                    (double)r[ORACLE_PRE_SCALE0 + 2];
        vol[i] = exp(ls);
        sorted[i] = vol[i];
        float *o = attrs_out + i * (n_channels - 1);
        for (int c = 0; c < ORACLE_PRE_QUAT0; c++) o[c] = r[c];
        double q[4] = {r[ORACLE_PRE_QUAT0], r[ORACLE_PRE_QUAT0 + 1], r[ORACLE_PRE_QUAT0 + 2],
                       r[ORACLE_PRE_QUAT0 + 3]};
        double e[3];
        oracle_euler(q, e);
        o[ORACLE_PRE_QUAT0] = (float)e[0];
        o[ORACLE_PRE_QUAT0 + 1] = (float)e[1];
        o[ORACLE_PRE_QUAT0 + 2] = (float)e[2];
    }
    qsort(sorted, (size_t)n, sizeof(double), cmp_double);
    double vq = sorted[(9 * (n - 1)) / 10];
    for (int64_t i = 0; i < n; i++) {
        double vn = vq > 0.0 ? fmin(vol[i] / vq, 1.0) : 1.0;
        imp_out[i] = (float)((double)view_imp[i] * pow(vn, beta));
    }
    if (vq_out) *vq_out = vq;
    free(vol);
    free(sorted);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* RAHT (Sec. III-D).                                                         */
/* ------------------------------------------------------------------------ */

/* attrs [n][n_channels]; chan [n_c] the transformed channels; depth 1..21.
 * keep = 0 (or n) transforms every Gaussian; otherwise the kept set of the
 * `keep` most important (importance [n]), with the whole scene's Morton
 * reading.  dc_out [n_c]; ac_out [(n - 1)][n_c] (capacity); ac_w_out
 * [(n - 1)] (may be NULL) the weight w1 + w2 of each AC's merge;
 * ac_range_out [(n - 1)][n_c] (may be NULL) the largest |value| of a Gaussian
 * under each AC's merged node, per channel (the scale its rounding errors
 * follow); *n_vox_out = V.  FP64. */
int oracle_raht(const float *attrs, int64_t n, int32_t n_channels, const int32_t *chan, int32_t n_c,
                int32_t depth, const float *importance, int64_t keep, double *dc_out, double *ac_out,
                int64_t *ac_w_out, double *ac_range_out, int64_t *n_vox_out) {
    if (n < 1 || n_c < 1 || depth < 1 || depth > 21 || keep < 0 || keep > n) return ORACLE_ERR_ARG;
    if (keep > 0 && keep < n && !importance) return ORACLE_ERR_ARG;
    for (int32_t k = 0; k < n_c; k++)
        if (chan[k] < 0 || chan[k] >= n_channels) return ORACLE_ERR_ARG;
    uint64_t *code = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int64_t *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n_c);
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *xr = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n_c);   /* node's largest |value| */
    if (!code || !order || !key || !w || !x || !pos || !rank || !xr) {
        free(code); free(order); free(key); free(w); free(x); free(pos); free(rank); free(xr);
        return ORACLE_ERR_NOMEM;
    }
    int rc = oracle_morton(attrs, n, n_channels, code, order);
    if (rc) goto done;
    /* the Morton positions taken: all, or the kept set of the `keep` most important */
    int64_t K = n;
    if (keep > 0 && keep < n) {
        rc = oracle_rank(importance, n, rank);
        if (rc) goto done;
        K = oracle_kept(rank, order, n, keep, pos);
    } else {
        for (int64_t t = 0; t < n; t++) pos[t] = t;
    }
    /* voxels: runs of equal code >> 3(21 - d) in Morton order, FP64 means */
    int shift = 3 * (21 - depth);
    int64_t m = 0;
    for (int64_t p = 0; p < K;) {
        uint64_t vc = code[order[pos[p]]] >> shift;
        int64_t q = p;
        while (q < K && (code[order[pos[q]]] >> shift) == vc) q++;
        for (int32_t k = 0; k < n_c; k++) {
            double sum = 0.0, big = 0.0;
            for (int64_t t = p; t < q; t++) {
                const double v = (double)attrs[order[pos[t]] * n_channels + chan[k]];
                sum += v;
                big = fabs(v) > big ? fabs(v) : big;
            }
            x[m * n_c + k] = q - p > 1 ? sum / (double)(q - p) : sum;
            xr[m * n_c + k] = big;
        }
        key[m] = vc;
        w[m] = 1;
        m++;
        p = q;
    }
    *n_vox_out = m;
    /* merges, finest level first: bit 0 of the voxel code is x, 1 y, 2 z, ... */
    int64_t n_ac = 0;
    for (int s = 0; s < 3 * depth; s++) {
        int64_t out = 0;
        for (int64_t i = 0; i < m;) {
            if (i + 1 < m && (key[i] >> 1) == (key[i + 1] >> 1)) {
                /* the entries of T: sqrt(w1) / sqrt(w1 + w2) and sqrt(w2) / sqrt(w1 + w2) */
                double w1 = (double)w[i], w2 = (double)w[i + 1];
                double sw = sqrt(w1 + w2);
                double t1 = sqrt(w1) / sw, t2 = sqrt(w2) / sw;
                for (int32_t k = 0; k < n_c; k++) {
                    double x1 = x[i * n_c + k], x2 = x[(i + 1) * n_c + k];
                    double dc = t1 * x1 + t2 * x2;
                    double ac = t1 * x2 - t2 * x1;
                    double r1 = xr[i * n_c + k], r2 = xr[(i + 1) * n_c + k];
                    double r = r1 > r2 ? r1 : r2;
                    ac_out[n_ac * n_c + k] = ac;
                    if (ac_range_out) ac_range_out[n_ac * n_c + k] = r;
                    x[out * n_c + k] = dc;
                    xr[out * n_c + k] = r;
                }
                if (ac_w_out) ac_w_out[n_ac] = w[i] + w[i + 1];
                n_ac++;
                w[out] = w[i] + w[i + 1];
                key[out] = key[i] >> 1;
                out++;
                i += 2;
            } else {
                for (int32_t k = 0; k < n_c; k++) {
                    x[out * n_c + k] = x[i * n_c + k];
                    xr[out * n_c + k] = xr[i * n_c + k];
                }
                w[out] = w[i];
                key[out] = key[i] >> 1;
                out++;
                i += 1;
            }
        }
        m = out;
    }
    if (m != 1) {
        rc = ORACLE_ERR_ARG;
        goto done;
    }
    for (int32_t k = 0; k < n_c; k++) dc_out[k] = x[k];
done:
    free(code); free(order); free(key); free(w); free(x); free(pos); free(rank); free(xr);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Block coder (Alg. 1: actual size S_a; Sec. III-G entropy encoding).        */
/* ------------------------------------------------------------------------ */
/*
 * Format of one (channel, group) block of n codes of b bits (little-endian):
 *   b:u8  min:f32  max:f32                       (9 bytes of metadata)
 *   nothing more when max - min == 0 (R = 0: every code is 0), else
 *   mode:u8  0 = raw, 1 = rANS
 *   raw   ceil(n b / 8) bytes; bit j of code i is stream bit i b + j, and
 *         stream bit t is bit t % 8 of byte t / 8
 *   rANS  table bits (same bit order), zero-padded to a whole byte:
 *           gamma(D), then for each of the D distinct codes in ascending
 *           order gamma(gap) and gamma(f): gap = code - previous code (the
 *           first: code + 1), f its normalised frequency;
 *         lanes x u32, the encoder's final states, lane 0 first;
 *         the renormalisation bytes in the order the decoder reads them.
 *   gamma(x), x >= 1: floor(log2 x) zero bits, then the bits of x from the
 *   most significant down.
 * Model: M = 2^k with k = ceil(log2 n) (so M >= n), f = floor(count M / n),
 * and the shortfall M - sum f added to the most frequent code (the lowest
 * such code on ties); with n a power of two f is the count itself.
 * rANS: states in [L, 256 L), L = 2^23, byte-wise renormalisation; lane j of
 * lanes = min(32, max(1, n / 512)) codes the symbols i = j (mod lanes).
 * Encoding runs from the last symbol to the first: renormalise (emit the low
 * byte while x >= 2^(31 - k) f), then x = floor(x / f) M + x mod f + cum.
 * Decoding runs forwards: slot = x mod M, x = f (x >> k) + slot - cum, then
 * read bytes while x < L.  The rANS payload is used when it is shorter than
 * the raw one.
 */
#define ORACLE_RANS_L (1u << 23)

typedef struct {
    uint8_t *p;
    int64_t bit;
} oracle_bitw;

static void put_bit(oracle_bitw *w, unsigned v) {
    if (v) w->p[w->bit >> 3] |= (uint8_t)(1u << (w->bit & 7));
    w->bit++;
}

static int floor_log2_u64(uint64_t x) {
    int k = -1;
    while (x) {
        x >>= 1;
        k++;
    }
    return k;
}

static void put_gamma(oracle_bitw *w, uint64_t x) {
    int N = floor_log2_u64(x);
    for (int i = 0; i < N; i++) put_bit(w, 0);
    for (int j = N; j >= 0; j--) put_bit(w, (unsigned)((x >> j) & 1u));
}

static int ceil_log2_i64(int64_t n) {
    int k = 0;
    while (((int64_t)1 << k) < n) k++;
    return k;
}

int32_t oracle_rans_lanes(int64_t n) {
    int64_t l = n / 512;
    if (l < 1) l = 1;
    if (l > 32) l = 32;
    return (int32_t)l;
}

int64_t oracle_block_bound(int64_t n, int32_t b) { return 10 + (n * (int64_t)b + 7) / 8; }

/* Encode one block into out (at least oracle_block_bound(n, b) bytes).
 * Returns the block's size in bytes, or a negative error. */
int64_t oracle_encode_block(const uint16_t *codes, int64_t n, int32_t b, float mn, float mx,
                            uint8_t *out, int64_t cap) {
    if (n < 1 || b < 1 || b > 16 || cap < oracle_block_bound(n, b)) return ORACLE_ERR_ARG;
    int64_t bound = oracle_block_bound(n, b);
    memset(out, 0, (size_t)bound);
    out[0] = (uint8_t)b;
    memcpy(out + 1, &mn, 4);
    memcpy(out + 5, &mx, 4);
    const uint32_t nsym = 1u << b;
    float R = mx - mn;
    if (R == 0.0f) {
        for (int64_t i = 0; i < n; i++)
            if (codes[i] != 0) return ORACLE_ERR_ARG;
        return 9;
    }
    for (int64_t i = 0; i < n; i++)
        if (codes[i] >= nsym) return ORACLE_ERR_ARG;

    int64_t raw_payload = 1 + (n * b + 7) / 8;
    uint32_t *hist = (uint32_t *)calloc(nsym, sizeof(uint32_t));
    uint32_t *f = (uint32_t *)calloc(nsym, sizeof(uint32_t));
    uint32_t *cum = (uint32_t *)calloc(nsym, sizeof(uint32_t));
    uint8_t *em = (uint8_t *)malloc((size_t)(2 * n + 8));
    uint8_t *tab = (uint8_t *)calloc((size_t)(8 * nsym + 8), 1);
    int64_t result;
    if (!hist || !f || !cum || !em || !tab) {
        result = ORACLE_ERR_NOMEM;
        goto done;
    }
    for (int64_t i = 0; i < n; i++) hist[codes[i]]++;

    /* normalised frequencies */
    int k = ceil_log2_i64(n);
    uint64_t M = (uint64_t)1 << k;
    uint64_t fsum = 0;
    uint32_t top = 0;
    for (uint32_t s = 0; s < nsym; s++) {
        f[s] = (uint32_t)(((uint64_t)hist[s] * M) / (uint64_t)n);
        fsum += f[s];
        if (hist[s] > hist[top]) top = s;
    }
    f[top] += (uint32_t)(M - fsum);
    uint32_t run = 0;
    for (uint32_t s = 0; s < nsym; s++) {
        cum[s] = run;
        run += f[s];
    }

    /* table */
    oracle_bitw tw = {tab, 0};
    uint64_t D = 0;
    for (uint32_t s = 0; s < nsym; s++) D += hist[s] > 0;
    put_gamma(&tw, D);
    int64_t prev = -1;
    for (uint32_t s = 0; s < nsym; s++) {
        if (!hist[s]) continue;
        put_gamma(&tw, (uint64_t)((int64_t)s - prev));
        put_gamma(&tw, f[s]);
        prev = s;
    }
    int64_t tab_bytes = (tw.bit + 7) / 8;

    /* interleaved rANS, last symbol first */
    int32_t lanes = oracle_rans_lanes(n);
    uint32_t x[32];
    for (int j = 0; j < 32; j++) x[j] = ORACLE_RANS_L;
    int64_t E = 0;
    for (int64_t i = n - 1; i >= 0; i--) {
        int lane = (int)(i % lanes);
        uint32_t s = codes[i];
        uint64_t xmax = ((uint64_t)(ORACLE_RANS_L >> k) << 8) * f[s];
        while ((uint64_t)x[lane] >= xmax) {
            em[E++] = (uint8_t)(x[lane] & 0xffu);
            x[lane] >>= 8;
        }
        x[lane] = (uint32_t)((x[lane] / f[s]) * M + x[lane] % f[s] + cum[s]);
    }
    int64_t rans_payload = 1 + tab_bytes + 4 * (int64_t)lanes + E;

    if (rans_payload < raw_payload) {
        uint8_t *p = out + 9;
        *p++ = 1;
        memcpy(p, tab, (size_t)tab_bytes);
        p += tab_bytes;
        for (int j = 0; j < lanes; j++) {
            for (int q = 0; q < 4; q++) *p++ = (uint8_t)(x[j] >> (8 * q));
        }
        for (int64_t e = E - 1; e >= 0; e--) *p++ = em[e];
        result = 9 + rans_payload;
    } else {
        out[9] = 0;
        oracle_bitw rw = {out + 10, 0};
        for (int64_t i = 0; i < n; i++)
            for (int j = 0; j < b; j++) put_bit(&rw, (codes[i] >> j) & 1u);
        result = 9 + raw_payload;
    }
done:
    free(hist);
    free(f);
    free(cum);
    free(em);
    free(tab);
    return result;
}

typedef struct {
    const uint8_t *p;
    int64_t bit;
    int64_t nbits;
} oracle_bitr;

static int get_bit(oracle_bitr *r, unsigned *v) {
    if (r->bit >= r->nbits) return 0;
    *v = (r->p[r->bit >> 3] >> (r->bit & 7)) & 1u;
    r->bit++;
    return 1;
}

static int get_gamma(oracle_bitr *r, uint64_t *x) {
    int N = 0;
    unsigned v;
    for (;;) {
        if (!get_bit(r, &v)) return 0;
        if (v) break;
        if (++N > 40) return 0;
    }
    uint64_t val = 1;
    for (int j = 0; j < N; j++) {
        if (!get_bit(r, &v)) return 0;
        val = (val << 1) | v;
    }
    *x = val;
    return 1;
}

/* Decode one block of n codes from in[0 .. avail).  Returns the bytes the
 * block occupies, or ORACLE_ERR_ARG if the block is malformed. */
int64_t oracle_decode_block(const uint8_t *in, int64_t avail, int64_t n, uint16_t *codes,
                            int32_t *b_out, float *mn_out, float *mx_out) {
    if (n < 1 || avail < 9) return ORACLE_ERR_ARG;
    int32_t b = in[0];
    float mn, mx;
    memcpy(&mn, in + 1, 4);
    memcpy(&mx, in + 5, 4);
    if (b < 1 || b > 16) return ORACLE_ERR_ARG;
    *b_out = b;
    *mn_out = mn;
    *mx_out = mx;
    float R = mx - mn;
    if (R == 0.0f) {
        for (int64_t i = 0; i < n; i++) codes[i] = 0;
        return 9;
    }
    if (avail < 10) return ORACLE_ERR_ARG;
    const uint32_t nsym = 1u << b;
    if (in[9] == 0) {
        int64_t bytes = (n * b + 7) / 8;
        if (avail < 10 + bytes) return ORACLE_ERR_ARG;
        oracle_bitr r = {in + 10, 0, 8 * bytes};
        for (int64_t i = 0; i < n; i++) {
            unsigned c = 0, v = 0;
            for (int j = 0; j < b; j++) {
                get_bit(&r, &v);
                c |= v << j;
            }
            codes[i] = (uint16_t)c;
        }
        return 10 + bytes;
    }
    if (in[9] != 1) return ORACLE_ERR_ARG;
    int k = ceil_log2_i64(n);
    uint32_t M = 1u << k;
    uint32_t *f = (uint32_t *)calloc(nsym, sizeof(uint32_t));
    uint32_t *cum = (uint32_t *)calloc(nsym, sizeof(uint32_t));
    uint16_t *lut = (uint16_t *)malloc(sizeof(uint16_t) * M);
    int64_t result = ORACLE_ERR_ARG;
    if (!f || !cum || !lut) {
        result = ORACLE_ERR_NOMEM;
        goto done;
    }
    oracle_bitr r = {in + 10, 0, 8 * (avail - 10)};
    uint64_t D, gap, fv;
    if (!get_gamma(&r, &D) || D < 1 || D > nsym) goto done;
    int64_t sym = -1;
    uint64_t total = 0;
    for (uint64_t e = 0; e < D; e++) {
        if (!get_gamma(&r, &gap) || !get_gamma(&r, &fv)) goto done;
        sym += (int64_t)gap;
        if (sym >= (int64_t)nsym || fv > M) goto done;
        f[sym] = (uint32_t)fv;
        total += fv;
    }
    if (total != M) goto done;
    uint32_t run = 0;
    for (uint32_t s = 0; s < nsym; s++) {
        cum[s] = run;
        for (uint32_t t = 0; t < f[s]; t++) lut[run + t] = (uint16_t)s;
        run += f[s];
    }
    int64_t pos = 10 + (r.bit + 7) / 8;
    int32_t lanes = oracle_rans_lanes(n);
    if (avail < pos + 4 * lanes) goto done;
    uint32_t x[32];
    for (int j = 0; j < lanes; j++) {
        x[j] = 0;
        for (int q = 0; q < 4; q++) x[j] |= (uint32_t)in[pos++] << (8 * q);
    }
    for (int64_t i = 0; i < n; i++) {
        int j = (int)(i % lanes);
        uint32_t slot = x[j] & (M - 1);
        uint32_t s = lut[slot];
        codes[i] = (uint16_t)s;
        x[j] = f[s] * (x[j] >> k) + slot - cum[s];
        while (x[j] < ORACLE_RANS_L) {
            if (pos >= avail) goto done;
            x[j] = (x[j] << 8) | in[pos++];
        }
    }
    for (int j = 0; j < lanes; j++)
        if (x[j] != ORACLE_RANS_L) goto done;
    result = pos;
done:
    free(f);
    free(cum);
    free(lut);
    return result;
}

/*
 * Compress one configuration: quantise (oracle_quantize) and encode every
 * (channel, group) block in (c, g) order, appended into out[0 .. cap).
 * block_bytes[c * n_groups + g] receives each block's size.  Returns the
 * total bytes, or a negative error.
 */
int64_t oracle_encode_config(const float *attrs, const float *importance, int64_t n,
                             int32_t n_channels, int64_t keep, int32_t G, const uint8_t *q_bits,
                             uint8_t *out, int64_t cap, int64_t *block_bytes) {
    if (n < 0 || keep < 1 || keep > n || G < 1 || n_channels < 1) return ORACLE_ERR_ARG;
    int64_t ng = oracle_n_groups(keep, G);
    uint16_t *codes = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(keep * n_channels));
    float *minmax = (float *)malloc(sizeof(float) * (size_t)(2 * ng * n_channels));
    int64_t total = 0;
    if (!codes || !minmax) {
        total = ORACLE_ERR_NOMEM;
        goto done;
    }
    int rc = oracle_quantize(attrs, importance, n, n_channels, keep, G, q_bits, codes, minmax);
    if (rc) {
        total = rc;
        goto done;
    }
    for (int32_t c = 0; c < n_channels; c++) {
        for (int64_t g = 0; g < ng; g++) {
            int64_t start = g * G;
            int64_t len = keep - start < G ? keep - start : G;
            int32_t b = q_bits[c * ng + g];
            if (total + oracle_block_bound(len, b) > cap) {
                total = ORACLE_ERR_ARG;
                goto done;
            }
            int64_t sz = oracle_encode_block(&codes[(int64_t)c * keep + start], len, b,
                                             minmax[(c * ng + g) * 2], minmax[(c * ng + g) * 2 + 1],
                                             out + total, cap - total);
            if (sz < 0) {
                total = sz;
                goto done;
            }
            block_bytes[c * ng + g] = sz;
            total += sz;
        }
    }
done:
    free(codes);
    free(minmax);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Vector quantisation of the 1+D SH coefficients (Sec. III-D).               */
/* ------------------------------------------------------------------------ */

/* Nearest codebook entry of each of the n vectors x[i][0..D).  idx_out[i]
 * gets the entry, score_out[i] (may be NULL) its score fl(|c|^2 - 2 x.c). */
int oracle_vq_assign(const float *x, int64_t n, int32_t D, const float *cb, int32_t K,
                     int32_t *idx_out, float *score_out) {
    if (n < 0 || D < 1 || K < 1) return ORACLE_ERR_ARG;
    float *cc = (float *)malloc(sizeof(float) * (size_t)K);
    if (!cc) return ORACLE_ERR_NOMEM;
    for (int32_t k = 0; k < K; k++) {
        float s = 0.0f;
        for (int32_t d = 0; d < D; d++) s = fmaf(cb[(int64_t)k * D + d], cb[(int64_t)k * D + d], s);
        cc[k] = s;
    }
    for (int64_t i = 0; i < n; i++) {
        const float *xi = x + i * D;
        int32_t best = 0;
        float best_s = 0.0f;
        for (int32_t k = 0; k < K; k++) {
            float dot = 0.0f;
            for (int32_t d = 0; d < D; d++) dot = fmaf(xi[d], cb[(int64_t)k * D + d], dot);
            float score = fmaf(-2.0f, dot, cc[k]);
            if (k == 0 || score < best_s) {
                best = k;
                best_s = score;
            }
        }
        idx_out[i] = best;
        if (score_out) score_out[i] = best_s;
    }
    free(cc);
    return ORACLE_OK;
}

/* One batch of the mini-batch k-means: the vectors x[rows[j]] (j = 0..b-1)
 * are assigned to their nearest centre, then every centre moves to the mean
 * of all vectors assigned to it so far: c = (v c + sum x) / (v + m), with the
 * count v updated to v + m.  cb [K][D] and counts [K] are updated in place;
 * assign_out[j] (may be NULL) gets the batch's assignment. */
int oracle_vq_update(const float *x, int64_t n, int32_t D, float *cb, int32_t K, int64_t *counts,
                     const int32_t *rows, int32_t b, int32_t *assign_out) {
    if (n < 1 || D < 1 || K < 1 || b < 0) return ORACLE_ERR_ARG;
    for (int32_t j = 0; j < b; j++)
        if (rows[j] < 0 || rows[j] >= n) return ORACLE_ERR_ARG;
    float *xb = (float *)calloc((size_t)(b > 0 ? b : 1) * D, sizeof(float));
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(b > 0 ? b : 1));
    double *sum = (double *)calloc((size_t)K * D, sizeof(double));
    int64_t *m = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int rc = ORACLE_OK;
    if (!xb || !a || !sum || !m) {
        rc = ORACLE_ERR_NOMEM;
        goto done;
    }
    for (int32_t j = 0; j < b; j++) memcpy(xb + (int64_t)j * D, x + (int64_t)rows[j] * D, sizeof(float) * D);
    rc = oracle_vq_assign(xb, b, D, cb, K, a, NULL);
    if (rc) goto done;
    for (int32_t j = 0; j < b; j++) {   /* batch order */
        m[a[j]]++;
        for (int32_t d = 0; d < D; d++) sum[(int64_t)a[j] * D + d] += (double)xb[(int64_t)j * D + d];
    }
    for (int32_t k = 0; k < K; k++) {
        if (!m[k]) continue;
        double v = (double)counts[k];
        for (int32_t d = 0; d < D; d++) {
            double num = v * (double)cb[(int64_t)k * D + d] + sum[(int64_t)k * D + d];
            cb[(int64_t)k * D + d] = (float)(num / (v + (double)m[k]));
        }
        counts[k] += m[k];
    }
    if (assign_out) memcpy(assign_out, a, sizeof(int32_t) * (size_t)b);
done:
    free(xb);
    free(a);
    free(sum);
    free(m);
    return rc;
}
