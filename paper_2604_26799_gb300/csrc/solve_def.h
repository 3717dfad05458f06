// The budget solve's arithmetic, shared by the host solver (solve.cpp) and the
// device solver (solve_gpu.cu) so that both give bit-identical answers.
//
// Eq. (eq:ilp), Sec. III-F, is a multiple-choice knapsack per reserve ratio:
// every (channel, group) item takes exactly one bit-width option, the summed
// loss Omega is minimised and the summed rate must fit the byte budget.
//
//  * Rates are integers in units of 2^-22 bits.  Entropy rates from a cost
//    table are exact multiples of that unit (the table is built that way);
//    fixed-length rates n * b are integers.  All rate sums are therefore exact
//    and do not depend on the order of summation.
//  * Every item's options are reduced to their lower convex hull in the
//    (rate, loss) plane.  Increment l of an item moves it from hull vertex l
//    to l + 1; its efficiency is (loss drop) / (rate rise), and its sort key is
//    the bit pattern of that positive double.
//  * Increment order: larger key first, then smaller item index, then smaller
//    level.  The LP relaxation takes increments in that order until the next
//    one (the split) does not fit; the LP value subtracts the fitting fraction
//    of the split.  The integral answer keeps the whole increments before the
//    split, then scans the rest in the same order and takes every increment
//    that is its item's next one and still fits (greedy completion).
//  * Loss totals are "tree sums" over items in item order: chunks of 1024
//    items, each reduced by a fixed 32 x 32 pairwise tree, the chunk totals
//    added one after another.
#pragma once

#include <stdint.h>
#include <math.h>
#include <string.h>

#ifdef __CUDACC__
#define MGS_HD __host__ __device__ __forceinline__
#else
#define MGS_HD inline
#endif

namespace mgs {

constexpr double kRateUnit = 4194304.0;                 // 2^22 units per bit
constexpr double kUnitsToBytes = 1.0 / (8.0 * 4194304.0);
constexpr int kTreeChunk = 1024;
constexpr int kMaxVerts = 16;

// Rate of one option in units of 2^-22 bits.
MGS_HD int64_t rate_units(int rate_model, double hbits, int32_t count, int32_t bits) {
    if (rate_model == 1) return (int64_t)count * (int64_t)bits * 4194304ll;
    return (int64_t)llrint(hbits * kRateUnit);
}

// Lower convex hull of one item's options.  w[k], d[k]: rate and loss of
// option k (k < nb).  Out: nv vertices opt[v] with rates hw[v] (increasing)
// and losses hd[v] (decreasing).  Options are visited in (rate, loss, index)
// order; an option that does not lower the loss, or has the rate of the last
// vertex, is dominated; a vertex that does not lie strictly below the chord of
// its neighbours is dropped.
MGS_HD int build_hull(const int64_t *w, const double *d, int nb, int8_t *opt, int64_t *hw,
                      double *hd) {
    int ord[kMaxVerts];
    for (int k = 0; k < nb; k++) ord[k] = k;
    for (int i = 1; i < nb; i++) {   // insertion sort; the options usually arrive sorted
        const int x = ord[i];
        int j = i - 1;
        while (j >= 0) {
            const int y = ord[j];
            const bool after = w[y] > w[x] || (w[y] == w[x] && (d[y] > d[x] || (d[y] == d[x] && y > x)));
            if (!after) break;
            ord[j + 1] = y;
            j--;
        }
        ord[j + 1] = x;
    }
    int h = 0;
    int hull[kMaxVerts];
    for (int t = 0; t < nb; t++) {
        const int k = ord[t];
        if (h > 0 && (d[k] >= d[hull[h - 1]] || w[k] == w[hull[h - 1]])) continue;
        while (h >= 2) {
            const int a = hull[h - 2], b = hull[h - 1];
            const double lhs = (d[b] - d[a]) * (double)(w[k] - w[a]);
            const double rhs = (d[k] - d[a]) * (double)(w[b] - w[a]);
            if (lhs >= rhs) h--;
            else break;
        }
        hull[h++] = k;
    }
    for (int v = 0; v < h; v++) {
        opt[v] = (int8_t)hull[v];
        hw[v] = w[hull[v]];
        hd[v] = d[hull[v]];
    }
    return h;
}

// Sort key of an increment: the bit pattern of its (positive) efficiency.
MGS_HD uint64_t inc_key(double dd, int64_t dw) {
    const double e = dd / (double)dw;
    uint64_t u;
    memcpy(&u, &e, 8);
    return u;
}

// Capacity in rate units for a byte budget after the fixed bytes; -1 if the
// fixed bytes alone exceed it.
MGS_HD int64_t capacity_units(double budget, double fixed_bytes) {
    const double c = 8.0 * (budget - fixed_bytes) * kRateUnit;
    if (!(c >= 0.0)) return -1;
    if (c >= 4.0e18) return (int64_t)4000000000000000000ll;
    return (int64_t)floor(c);
}

MGS_HD double units_to_bytes(int64_t units, double fixed_bytes) {
    return (double)units * kUnitsToBytes + fixed_bytes;
}

}  // namespace mgs
