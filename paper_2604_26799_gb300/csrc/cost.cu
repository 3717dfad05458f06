// Fused candidate-cost kernel (Sec. III-D quantiser, Sec. III-F loss matrix
// Omega and entropy bound) for every (ratio, group, channel, bit-width).
//
// One work item = (segment = (scene, ratio), group g, chunk of W channels).
// The CTA gathers the group's rows through the kept list once (W channels of
// each 32-byte slab row, vector loads) into registers, reduces min/max, and
// then evaluates every bit-width from those registers:
//
//   S = fl(R / 2^b), Z = rint(fl(2^b - fl(M / S))), R = fl(M - m)
//   x = fl(fl(c / S) + Z),  q = rint(min(max(x, 0), 2^b - 1))
//   c_hat = fl(fl(q - Z) * S),  e = fl(c_hat - c)
//
// Exact reformulations used on the fast path (each gives the same FP32 bits):
//  * When S is normal, S = R * 2^-b exactly, so fl(c / S) = fl(c / R) * 2^b
//    whenever u = fl(c / R) is normal or zero: one division per element serves
//    every bit-width, and x = fma(u, 2^b, Z) is the same single rounding.
//  * rint(x) for |x| < 2^22 is fl(x + 1.5 * 2^23) - 1.5 * 2^23; the code sits in
//    the low mantissa bits of y = fl(x + 1.5 * 2^23), which also address the
//    histogram.  Clamping y to [1.5 * 2^23, 1.5 * 2^23 + 2^b - 1] equals rounding
//    the clamped x (the bounds are integers), and fl(q - Z) = fl(y - (1.5 * 2^23 + Z))
//    when |Z| < 2^22 (the second operand is then an exact integer).
//  * x is monotone in c, so if the group minimum does not round below 0 no
//    element does, and the lower clamp is skipped.
//  * Packed f32x2 adds, subtracts and FMAs are used where no contraction can
//    arise; the reconstruction product stays a scalar multiply.
//  * Each channel is scaled by an exact power of two 2^k (R * 2^k in [1, 2)):
//    c' = c 2^k, S' = S 2^k give c'/S' = c/S and e' = e 2^k exactly, so squares
//    and sums stay in the normal FP32 range; the sums are rescaled in FP64.
// Groups where a precondition fails (subnormal S or u, |Z| >= 2^22) take the
// literal per-element formula.  Pairs of elements use packed f32x2 arithmetic.
//
// Histograms live in shared memory, in two buffers that consecutive
// bit-widths alternate between, so one barrier per bit-width suffices:
// per-lane columns for b <= 6 and a direct table for b <= 10 (summed after the
// pass); for larger b the atomic returns the old count j - 1 and the thread
// adds delta(j) = L(j) - L(j - 1), L(h) = h log2 h in units of 2^-22 bits, so
// sum_j delta telescopes to sum_bins L(h) with no scan (direct 32-bit counters
// or 16-bit counter pairs; a table larger than the big buffer is counted in
// windows, one pass over the elements per window).  Entropy sums are
// integers, so they do not depend on the reduction order.

#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>

#include "internal.h"

namespace mgs {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;   // its bit pattern
constexpr int kLaneMaxBits = 6;
constexpr int kDirectMaxBits = 10;

enum HistMode { kLane = 0, kDirect = 1, kDelta32 = 2, kDelta16 = 3 };
enum Path { kFast = 0, kFastBottom = 1, kGeneric = 2, kDegenerate = 3 };

struct BitParam {
    float S, Ss, Z, twob;
    float MZ;     // 1.5 * 2^23 + Z (exact when |Z| < 2^22)
    float ytop;   // 1.5 * 2^23 + 2^b - 1
    float top;    // 2^b - 1
    int b;
    int mode;
    int path;
    int buf;      // histogram buffer: 0, 1 (second small buffer) or 2 (big buffer)
    int sync;     // 1: barrier before the pass (the previous option used the same buffer)
    int windows;  // passes over the elements (16-bit pairs larger than the big buffer)
    int wwords;   // words counted per pass (16-bit-pair mode)
    int pad[2];
};

struct KernelArgs {
    const CostSeg *segs;
    int32_t n_segs;
    int32_t G;
    int64_t n_work;
    int32_t n_bits;
    int32_t opt_lo, opt_hi;
    int32_t bits[MGS_MAX_OPTIONS];
    const unsigned long long *ltab;   // L(h) in 2^-22 bits
    const uint32_t *dtab;             // L(h) - L(h - 1) in 2^-22 bits (< 2^26)
    unsigned int *counter;
    int32_t hist_words;               // words per small histogram buffer (power of two)
    int32_t n_small;                  // small buffers (1 or 2)
    int32_t big_words;                // words of the big buffer (0: none)
    // per option (index k = option - opt_lo), fixed for the launch: histogram mode,
    // buffer (0, 1: small; 2: big), barrier before the pass, windows, words per window
    int8_t opt_mode[MGS_MAX_OPTIONS], opt_buf[MGS_MAX_OPTIONS], opt_sync[MGS_MAX_OPTIONS];
    int8_t opt_windows[MGS_MAX_OPTIONS];
    int32_t opt_wwords[MGS_MAX_OPTIONS];
};

// ---- packed FP32 pairs ----------------------------------------------------
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
#define MGS_F2_BINOP(NAME, OP)                                                            \
    __device__ __forceinline__ float2 NAME(float2 a, float2 b) {                          \
        float2 d;                                                                         \
        asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t" \
            OP " rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"                                 \
            : "=f"(d.x), "=f"(d.y)                                                        \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                    \
        return d;                                                                         \
    }
MGS_F2_BINOP(fadd2, "add.rn.f32x2")
MGS_F2_BINOP(fsub2, "sub.rn.f32x2")
#undef MGS_F2_BINOP

// ---- global loads with L1 eviction hints: the gathered rows and kept
// positions are read once and must not evict the entropy tables, which every
// pass reads.  Read-only data: not volatile, so the compiler may schedule them
// freely around the (volatile) shared-memory atomics
__device__ __forceinline__ float4 ld_stream(const float4 *p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ float2 ld_stream(const float2 *p) {
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned long long ld_keep(const unsigned long long *p) {
    unsigned long long v;
    asm("ld.global.nc.L1::evict_last.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_keep(const uint32_t *p) {
    uint32_t v;
    asm("ld.global.nc.L1::evict_last.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// ---- shared-memory histogram operations ------------------------------------
__device__ __forceinline__ void red_add(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ uint32_t atom_add(uint32_t addr, uint32_t v) {
    uint32_t old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(v));
    return old;
}
// The same, executed only where `pred` holds (predicated, not branched: lanes
// of a warp taking different sides do not split the warp); 0 elsewhere.
__device__ __forceinline__ uint32_t atom_add_if(bool pred, uint32_t addr, uint32_t v) {
    uint32_t old = 0;
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q atom.shared.add.u32 %0, [%1], %2;\n\t}"
                 : "+r"(old)
                 : "r"(addr), "r"(v), "r"((uint32_t)pred));
    return old;
}

// One code into a table of 16-bit counter pairs, counted only if `valid` and
// its word lies in the current window [wlo, wlo + wn).  Branch-free.
__device__ __forceinline__ void pair_count(bool valid, uint32_t y, uint32_t hbase, uint32_t wlo,
                                           uint32_t wn, const uint32_t *dtab, uint32_t &dacc) {
    const uint32_t q = y - kMagicBits;
    const uint32_t word = (q >> 1) - wlo;
    const bool in = valid && word < wn;
    const uint32_t sh = (q & 1u) << 4;
    const uint32_t old = atom_add_if(in, hbase + (word << 2), 1u << sh);
    const uint32_t d = ld_keep(&dtab[((old >> sh) & 0xFFFFu) + 1u]);
    dacc += in ? d : 0u;
}

// Count one code.  y is the code's bit pattern kMagicBits + q.  For the delta
// modes the return is delta(new count) to be added to the entropy sum.
template <int MODE>
__device__ __forceinline__ void hist_op(uint32_t y, uint32_t hbase, uint32_t lane_base,
                                        uint32_t wlo, uint32_t wn, const uint32_t *dtab,
                                        uint32_t &dacc) {
    if (MODE == kLane) {
        red_add(lane_base + (y << 7), 1u);           // (q * 32 + lane) * 4, magic folded in
    } else if (MODE == kDirect) {
        red_add(hbase + (y << 2), 1u);               // q * 4, magic folded in
    } else if (MODE == kDelta32) {
        uint32_t old = atom_add(hbase + (y << 2), 1u);
        dacc += ld_keep(&dtab[old + 1u]);
    } else {
        // 16-bit counter pairs; only codes whose word lies in the current window
        // [wlo, wlo + wn) are counted by this pass
        pair_count(true, y, hbase, wlo, wn, dtab, dacc);
    }
}

// Fast path for one bit-width over this thread's elements (pairs, packed).
template <int T, int EPT, int MODE, bool BOTTOM, bool FULL>
__device__ __forceinline__ void eval_fast(const float (&c)[EPT], const float (&u)[EPT], int nvalid,
                                          const BitParam &p, uint32_t hbase, uint32_t lane_base,
                                          uint32_t wlo, uint32_t wn, const uint32_t *dtab,
                                          float &sse, float &l1, float &linf,
                                          unsigned long long &hacc) {
    const float2 tw = make_float2(p.twob, p.twob), zz = make_float2(p.Z, p.Z);
    const float2 mg = make_float2(kMagic, kMagic), mz = make_float2(p.MZ, p.MZ);
    float2 s2 = make_float2(0.0f, 0.0f);
    float la = 0.0f, lb = 0.0f, ma = 0.0f, mb = 0.0f;
    uint32_t dacc = 0;   // delta sums: at most EPT * 2^26 < 2^32
#pragma unroll
    for (int e = 0; e < EPT; e += 2) {
        const bool v1 = FULL || (e + 1) * T + (int)threadIdx.x < nvalid;
        const bool v0 = FULL || e * T + (int)threadIdx.x < nvalid;
        if (v1) {
            float2 x = ffma2(make_float2(u[e], u[e + 1]), tw, zz);
            float2 y = fadd2(x, mg);
            y.x = fminf(y.x, p.ytop);
            y.y = fminf(y.y, p.ytop);
            if (BOTTOM) {
                y.x = fmaxf(y.x, kMagic);
                y.y = fmaxf(y.y, kMagic);
            }
            // c_hat' = fl(fl(q - Z) * S'): scalar multiplies, so the product is rounded on
            // its own and never contracted with the subtraction that follows
            const float2 d = fsub2(y, mz);
            const float2 ch = make_float2(__fmul_rn(d.x, p.Ss), __fmul_rn(d.y, p.Ss));
            float2 er = fsub2(ch, make_float2(c[e], c[e + 1]));
            s2 = ffma2(er, er, s2);
            la = __fadd_rn(la, fabsf(er.x));
            lb = __fadd_rn(lb, fabsf(er.y));
            ma = fmaxf(ma, fabsf(er.x));
            mb = fmaxf(mb, fabsf(er.y));
            hist_op<MODE>(__float_as_uint(y.x), hbase, lane_base, wlo, wn, dtab, dacc);
            hist_op<MODE>(__float_as_uint(y.y), hbase, lane_base, wlo, wn, dtab, dacc);
        } else if (v0) {
            float x = __fmaf_rn(u[e], p.twob, p.Z);
            float y = __fadd_rn(x, kMagic);
            y = fminf(y, p.ytop);
            if (BOTTOM) y = fmaxf(y, kMagic);
            float er = __fsub_rn(__fmul_rn(__fsub_rn(y, p.MZ), p.Ss), c[e]);
            s2.x = __fmaf_rn(er, er, s2.x);
            la = __fadd_rn(la, fabsf(er));
            ma = fmaxf(ma, fabsf(er));
            hist_op<MODE>(__float_as_uint(y), hbase, lane_base, wlo, wn, dtab, dacc);
        }
    }
    sse = __fadd_rn(s2.x, s2.y);
    l1 = __fadd_rn(la, lb);
    linf = fmaxf(ma, mb);
    hacc += dacc;
}

// Literal per-element formula (divisions, both clamps); any group.
template <int T, int EPT, int MODE>
__device__ __forceinline__ void eval_generic(const float (&c)[EPT], int nvalid, const BitParam &p,
                                          uint32_t hbase, uint32_t lane_base, uint32_t wlo,
                                          uint32_t wn, const uint32_t *dtab, float &sse, float &l1,
                                          float &linf, unsigned long long &hacc) {
    float s = 0.0f, a = 0.0f, m = 0.0f;
    uint32_t dacc = 0;
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        if (e * T + (int)threadIdx.x >= nvalid) continue;
        float x = __fadd_rn(__fdiv_rn(c[e], p.Ss), p.Z);   // c'/S' == c/S exactly
        float xc = fminf(fmaxf(x, 0.0f), p.top);
        int q = __float2int_rn(xc);
        float qz = __fsub_rn(__int2float_rn(q), p.Z);
        float er = __fsub_rn(__fmul_rn(qz, p.Ss), c[e]);
        s = __fmaf_rn(er, er, s);
        a = __fadd_rn(a, fabsf(er));
        m = fmaxf(m, fabsf(er));
        hist_op<MODE>(kMagicBits + (uint32_t)q, hbase, lane_base, wlo, wn, dtab, dacc);
    }
    sse = s;
    l1 = a;
    linf = m;
    hacc += dacc;
}

// Count-only pass of one window of a 16-bit-pair table: the codes of
// eval_fast (same operations, packed), no error sums, no branches per element.
template <int T, int EPT>
__device__ __forceinline__ void count_window_fast(const float (&u)[EPT], int nvalid, const BitParam &p,
                                                  uint32_t hbase, uint32_t wlo, uint32_t wn,
                                                  const uint32_t *dtab, unsigned long long &hacc) {
    const float2 tw = make_float2(p.twob, p.twob), zz = make_float2(p.Z, p.Z);
    const float2 mg = make_float2(kMagic, kMagic);
    // the lower clamp is a no-op unless the group minimum rounds below code 0
    const float lo = p.path == kFastBottom ? kMagic : -FLT_MAX;
    uint32_t dacc = 0;
#pragma unroll
    for (int e = 0; e < EPT; e += 2) {
        float2 y = fadd2(ffma2(make_float2(u[e], u[e + 1]), tw, zz), mg);
        y.x = fmaxf(fminf(y.x, p.ytop), lo);
        y.y = fmaxf(fminf(y.y, p.ytop), lo);
        const bool v0 = e * T + (int)threadIdx.x < nvalid;
        const bool v1 = (e + 1) * T + (int)threadIdx.x < nvalid;
        pair_count(v0, __float_as_uint(y.x), hbase, wlo, wn, dtab, dacc);
        pair_count(v1, __float_as_uint(y.y), hbase, wlo, wn, dtab, dacc);
    }
    hacc += dacc;
}

// The same for groups on the literal-division path (codes as in eval_generic).
template <int T, int EPT>
__device__ __forceinline__ void count_window_generic(const float (&c)[EPT], int nvalid, const BitParam &p,
                                                     uint32_t hbase, uint32_t wlo, uint32_t wn,
                                                     const uint32_t *dtab, unsigned long long &hacc) {
    uint32_t dacc = 0;
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        const float x = __fadd_rn(__fdiv_rn(c[e], p.Ss), p.Z);
        const uint32_t y = kMagicBits + (uint32_t)__float2int_rn(fminf(fmaxf(x, 0.0f), p.top));
        pair_count(e * T + (int)threadIdx.x < nvalid, y, hbase, wlo, wn, dtab, dacc);
    }
    hacc += dacc;
}

template <int T, int EPT, int MODE>
__device__ __forceinline__ void eval_dispatch(const float (&c)[EPT], const float (&u)[EPT],
                                              int nvalid, bool full, bool generic,
                                              const BitParam &p, uint32_t hbase,
                                              uint32_t lane_base, uint32_t wlo, uint32_t wn,
                                              const uint32_t *dtab, float &sse,
                                              float &l1, float &linf, unsigned long long &hacc) {
    if (generic) {
        eval_generic<T, EPT, MODE>(c, nvalid, p, hbase, lane_base, wlo, wn, dtab, sse, l1, linf, hacc);
    } else if (p.path == kFast) {
        if (full) eval_fast<T, EPT, MODE, false, true>(c, u, nvalid, p, hbase, lane_base, wlo, wn, dtab, sse, l1, linf, hacc);
        else eval_fast<T, EPT, MODE, false, false>(c, u, nvalid, p, hbase, lane_base, wlo, wn, dtab, sse, l1, linf, hacc);
    } else {
        if (full) eval_fast<T, EPT, MODE, true, true>(c, u, nvalid, p, hbase, lane_base, wlo, wn, dtab, sse, l1, linf, hacc);
        else eval_fast<T, EPT, MODE, true, false>(c, u, nvalid, p, hbase, lane_base, wlo, wn, dtab, sse, l1, linf, hacc);
    }
}

// After a pass: add sum L(h) of a summed mode to hacc and clear the buffer
// (the first clear_words words for the delta modes).
template <int T>
__device__ __forceinline__ void hist_finish(uint32_t *hist, int mode, int b, int clear_words,
                                            const unsigned long long *__restrict__ ltab,
                                            unsigned long long &hacc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (mode == kLane) {
        // the warp's j-th bin count is kept by lane j (bins / warps <= 32 for
        // b <= 6), so the table lookups of all its bins go out together
        static_assert((1 << kLaneMaxBits) / (T / 32) <= 32, "one lane per bin of a warp");
        const int bins = 1 << b;
        uint32_t mine = 0;
        int j = 0;
#pragma unroll 4
        for (int k = warp; k < bins; k += T / 32, j++) {
            const uint32_t v = hist[k * 32 + lane];
            hist[k * 32 + lane] = 0u;
            const uint32_t s = __reduce_add_sync(kFull, v);
            mine = lane == j ? s : mine;
        }
        hacc += ld_keep(&ltab[mine]);   // L(0) = 0 for lanes without a bin
    } else if (mode == kDirect) {
        // branch-free: L(0) = 0, so an empty bin adds nothing
        const int bins = 1 << b;
#pragma unroll 4
        for (int k = threadIdx.x; k < bins; k += T) {
            const uint32_t v = hist[k];
            hist[k] = 0u;
            hacc += ld_keep(&ltab[v]);
        }
    } else {
        uint4 *h4 = reinterpret_cast<uint4 *>(hist);
        for (int k = threadIdx.x; k < clear_words / 4; k += T) h4[k] = make_uint4(0u, 0u, 0u, 0u);
    }
}

__device__ __forceinline__ unsigned long long warp_sum_u64_redux(unsigned long long v) {
    // v < 2^48 (entropy sums of one group in 2^-22 bits): two 24-bit slices, each
    // summed exactly with redux.sync (32 x 2^24 < 2^32)
    uint32_t lo = (uint32_t)(v & 0xFFFFFFull), hi = (uint32_t)(v >> 24);
    lo = __reduce_add_sync(kFull, lo);
    hi = __reduce_add_sync(kFull, hi);
    return (unsigned long long)lo + ((unsigned long long)hi << 24);
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

template <int W>
__device__ __forceinline__ void load_row(const float *p, float (&v)[W]) {
    if (W == 8) {
        float4 a = ld_stream(reinterpret_cast<const float4 *>(p));
        float4 b = ld_stream(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4 % W] = b.x; v[5 % W] = b.y; v[6 % W] = b.z; v[7 % W] = b.w;
    } else if (W == 4) {
        float4 a = ld_stream(reinterpret_cast<const float4 *>(p));
        v[0] = a.x; v[1 % W] = a.y; v[2 % W] = a.z; v[3 % W] = a.w;
    } else if (W == 2) {
        float2 a = ld_stream(reinterpret_cast<const float2 *>(p));
        v[0] = a.x; v[1 % W] = a.y;
    } else {
        v[0] = ld_stream(p);
    }
}

// Shared-memory layout (dynamic):
//   hist[n_small][hist_words] hist_big[big_words] | psse[n_opts][T] | pl1[n_opts][T] | hpart[n_opts][T/32] (u64)
//   | plinf[n_opts][T/32] | bp[n_opts] | mm[T/32][W][2]
struct Smem {
    uint32_t *hist;
    float *psse, *pl1, *plinf;
    unsigned long long *hpart;
    BitParam *bp;
    float *mm;
};

__host__ __device__ inline size_t smem_layout(int T, int W, int hist_words, int nbuf, int big_words,
                                              int n_opts, size_t *o) {
    size_t off = 0;
    o[0] = off; off += (size_t)nbuf * hist_words * 4 + (size_t)big_words * 4;
    o[1] = off; off += (size_t)n_opts * T * 4;
    o[2] = off; off += (size_t)n_opts * T * 4;
    off = (off + 15) & ~(size_t)15;
    o[3] = off; off += (size_t)n_opts * (T / 32) * 8;
    o[4] = off; off += (size_t)n_opts * (T / 32) * 4;
    off = (off + 15) & ~(size_t)15;
    o[5] = off; off += (size_t)n_opts * sizeof(BitParam);
    o[6] = off; off += (size_t)(T / 32) * W * 2 * 4;
    return off;
}

template <int T, int EPT, int W>
__device__ void process_item(const KernelArgs &A, const Smem &sm, int64_t work) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = T / 32;
    // ---- decode the work item
    __shared__ int s_seg;
    if (threadIdx.x == 0) {
        int lo = 0, hi = A.n_segs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (A.segs[mid].work_begin <= work) lo = mid; else hi = mid - 1;
        }
        s_seg = lo;
    }
    __syncthreads();
    const CostSeg &S = A.segs[s_seg];
    const int64_t local = work - S.work_begin;
    const int g = S.g_first + (int)(local / S.n_chunks);
    const int chunk = (int)(local % S.n_chunks);
    const int c0 = chunk * W;
    const int slab = c0 / kSlabWidth;
    const int j0 = c0 % kSlabWidth;
    const int64_t gstart = (int64_t)g * A.G;
    const int nvalid = (int)((S.K - gstart) < (int64_t)A.G ? (S.K - gstart) : (int64_t)A.G);
    const bool full = nvalid >= T * EPT;

    // ---- gather: each element's W channels from its slab row
    float v[W][EPT];
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        int i = e * T + threadIdx.x;
        float row[W];
        if (i < nvalid) {
            const int32_t pos = S.kept ? ld_stream(&S.kept[gstart + i]) : (int32_t)(gstart + i);
            load_row<W>(S.slabs + ((int64_t)slab * S.n + pos) * kSlabWidth + j0, row);
        } else {
#pragma unroll
            for (int w = 0; w < W; w++) row[w] = 0.0f;
        }
#pragma unroll
        for (int w = 0; w < W; w++) v[w][e] = row[w];
    }

    // ---- group min / max of every channel of the chunk
#pragma unroll
    for (int w = 0; w < W; w++) {
        float mn = FLT_MAX, mx = -FLT_MAX;
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            if (e * T + (int)threadIdx.x < nvalid) {
                mn = fminf(mn, v[w][e]);
                mx = fmaxf(mx, v[w][e]);
            }
        }
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0) {
            sm.mm[(warp * W + w) * 2] = mn;
            sm.mm[(warp * W + w) * 2 + 1] = mx;
        }
    }
    __syncthreads();
    if (threadIdx.x < W) {
        int w = threadIdx.x;
        float a = FLT_MAX, b = -FLT_MAX;
        for (int k = 0; k < NW; k++) {
            a = fminf(a, sm.mm[(k * W + w) * 2]);
            b = fmaxf(b, sm.mm[(k * W + w) * 2 + 1]);
        }
        sm.mm[w * 2] = a;
        sm.mm[w * 2 + 1] = b;
    }
    __syncthreads();

    const int n_opts = A.opt_hi - A.opt_lo;
    const int hw = A.hist_words;
    const uint32_t hist_addr = (uint32_t)__cvta_generic_to_shared(sm.hist);
#pragma unroll 1
    for (int w = 0; w < W; w++) {
        const int ch = c0 + w;
        if (ch >= S.C) break;
        const float m = sm.mm[w * 2], M = sm.mm[w * 2 + 1];
        const float R = __fsub_rn(M, m);
        const int64_t item = S.item_base + (int64_t)ch * S.n_groups + g;
        // exact power-of-two scale 2^k = s1 * s2 with R * 2^k in [1, 2)
        const int kexp = R > 0.0f ? -ilogbf(R) : 0;
        const int k1 = kexp / 2, k2 = kexp - k1;
        const float s1 = __int_as_float((k1 + 127) << 23), s2 = __int_as_float((k2 + 127) << 23);
        if (threadIdx.x < n_opts) {
            BitParam p;
            p.b = A.bits[A.opt_lo + threadIdx.x];
            p.twob = (float)(1u << p.b);
            p.top = p.twob - 1.0f;
            p.ytop = kMagic + p.top;
            p.S = __fdiv_rn(R, p.twob);
            p.Ss = __fmul_rn(__fmul_rn(p.S, s1), s2);
            p.mode = A.opt_mode[threadIdx.x];
            p.buf = A.opt_buf[threadIdx.x];
            p.sync = A.opt_sync[threadIdx.x];
            p.windows = A.opt_windows[threadIdx.x];
            p.wwords = A.opt_wwords[threadIdx.x];
            if (p.S == 0.0f) {
                p.path = kDegenerate;
                p.Z = 0.0f;
                p.MZ = kMagic;
            } else {
                p.Z = rintf(__fsub_rn(p.twob, __fdiv_rn(M, p.S)));
                p.MZ = __fadd_rn(kMagic, p.Z);
                if (p.S < FLT_MIN || fabsf(p.Z) >= 4194304.0f) {
                    p.path = kGeneric;
                } else {
                    // the group minimum gives the smallest x: lower clamp only if it rounds below 0
                    float um = __fdiv_rn(m, R);
                    float ym = __fadd_rn(__fmaf_rn(um, p.twob, p.Z), kMagic);
                    p.path = ym < kMagic ? kFastBottom : kFast;
                }
            }
            sm.bp[threadIdx.x] = p;
        }
        if (threadIdx.x == 0) {
            S.cnt[item] = nvalid;
            S.vmin[item] = m;
            S.vmax[item] = M;
        }
        // this channel's values (compile-time indices keep v in registers)
        float cw[EPT];
#pragma unroll
        for (int e = 0; e < EPT; e++) cw[e] = v[0][e];
#pragma unroll
        for (int ww = 1; ww < W; ww++)
            if (ww == w)
#pragma unroll
                for (int e = 0; e < EPT; e++) cw[e] = v[ww][e];
        // one division per element, shared by every bit-width; then scale by 2^k
        float u[EPT];
        int slow = 0;
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            u[e] = R > 0.0f ? __fdiv_rn(cw[e], R) : 0.0f;
            slow |= (u[e] != 0.0f && fabsf(u[e]) <= FLT_MIN && e * T + (int)threadIdx.x < nvalid);
            cw[e] = __fmul_rn(__fmul_rn(cw[e], s1), s2);
        }
        const int any_slow = __syncthreads_or(slow);   // also publishes bp

#pragma unroll 1
        for (int k = 0; k < n_opts; k++) {
            const BitParam p = sm.bp[k];
            if (p.sync) __syncthreads();
            const int slot = p.buf == 2 ? A.n_small : p.buf;   // the big buffer follows the small ones
            uint32_t *hist = sm.hist + (size_t)slot * hw;
            const uint32_t hbase_raw = hist_addr + (uint32_t)slot * hw * 4u;
            float sse = 0.0f, l1 = 0.0f, linf = 0.0f;
            unsigned long long hacc = 0ull;
            if (p.path == kDegenerate) {
                if (threadIdx.x == 0) hacc = __ldg(&A.ltab[nvalid]);
            } else {
                const bool generic = p.path == kGeneric || any_slow;
                // code bit patterns are kMagicBits + q: fold the offset into the bases
                const uint32_t lane_base = hbase_raw + lane * 4u - (kMagicBits << 7);
                const uint32_t dbase = hbase_raw - (kMagicBits << 2);
                const uint32_t wn = (uint32_t)p.wwords;   // window 0 (the whole table if one)
                switch (p.mode) {
                    case kLane:
                        eval_dispatch<T, EPT, kLane>(cw, u, nvalid, full, generic, p, dbase, lane_base, 0u, wn, A.dtab, sse, l1, linf, hacc);
                        break;
                    case kDirect:
                        eval_dispatch<T, EPT, kDirect>(cw, u, nvalid, full, generic, p, dbase, lane_base, 0u, wn, A.dtab, sse, l1, linf, hacc);
                        break;
                    case kDelta32:
                        eval_dispatch<T, EPT, kDelta32>(cw, u, nvalid, full, generic, p, dbase, lane_base, 0u, wn, A.dtab, sse, l1, linf, hacc);
                        break;
                    default:
                        eval_dispatch<T, EPT, kDelta16>(cw, u, nvalid, full, generic, p, hbase_raw, lane_base, 0u, wn, A.dtab, sse, l1, linf, hacc);
                        break;
                }
                // further windows of a 16-bit-pair table: wait for every count, clear,
                // wait, count the next range of codes (the errors are already summed)
#pragma unroll 1
                for (int win = 1; win < p.windows; win++) {
                    __syncthreads();
                    hist_finish<T>(hist, kDelta16, p.b, p.wwords, A.ltab, hacc);
                    __syncthreads();
                    const uint32_t wlo = (uint32_t)(win * p.wwords);
                    if (generic)
                        count_window_generic<T, EPT>(cw, nvalid, p, hbase_raw, wlo, wn, A.dtab, hacc);
                    else
                        count_window_fast<T, EPT>(u, nvalid, p, hbase_raw, wlo, wn, A.dtab, hacc);
                }
            }
            sm.psse[k * T + threadIdx.x] = sse;
            sm.pl1[k * T + threadIdx.x] = l1;
            const uint32_t lmax = __reduce_max_sync(kFull, __float_as_uint(linf));
            if (lane == 0) sm.plinf[k * NW + warp] = __uint_as_float(lmax);
            __syncthreads();   // every update of this buffer is done
            if (p.path != kDegenerate)
                hist_finish<T>(hist, p.mode, p.b, p.mode == kDelta32 ? (1 << p.b) : p.wwords, A.ltab, hacc);
            hacc = warp_sum_u64_redux(hacc);
            if (lane == 0) sm.hpart[k * NW + warp] = hacc;
        }
        __syncthreads();
        // ---- reduce the partials and write this channel's entries
        for (int k = warp; k < n_opts; k += NW) {
            float a = 0.0f, b = 0.0f;
#pragma unroll
            for (int j = 0; j < T / 32; j++) {
                a = __fadd_rn(a, sm.psse[k * T + j * 32 + lane]);
                b = __fadd_rn(b, sm.pl1[k * T + j * 32 + lane]);
            }
            a = warp_sum(a);
            b = warp_sum(b);
            float cmax = lane < NW ? sm.plinf[k * NW + lane] : 0.0f;
            cmax = warp_max(cmax);
            unsigned long long hs = 0;
            for (int j = lane; j < NW; j += 32) hs += sm.hpart[k * NW + j];
            hs = warp_sum_u64_redux(hs);
            if (lane == 0) {
                const int64_t o = item * A.n_bits + A.opt_lo + k;
                // undo the 2^k scale in FP64 (exact powers of two)
                const double inv = __longlong_as_double((long long)(1023 - kexp) << 52);
                const double inv2 = __longlong_as_double((long long)(1023 - 2 * kexp) << 52);
                S.sse[o] = (double)a * inv2;
                S.l1[o] = (double)b * inv;
                S.linf[o] = (float)((double)cmax * inv);
                unsigned long long ln = __ldg(&A.ltab[nvalid]);
                S.hbits[o] = (double)(long long)(ln - hs) * (1.0 / 4194304.0);   // 2^-22
            }
        }
        __syncthreads();
    }
}

template <int T, int EPT, int W>
__global__ void __launch_bounds__(T, (T >= 512 ? 1 : 512 / T))
    k_cost(const __grid_constant__ KernelArgs A, int unused) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n_opts = A.opt_hi - A.opt_lo;
    size_t o[7];
    smem_layout(T, W, A.hist_words, A.n_small, A.big_words, n_opts, o);
    static_assert(EPT % 2 == 0, "elements are processed in pairs");
    Smem sm;
    sm.hist = reinterpret_cast<uint32_t *>(smem_raw + o[0]);
    sm.psse = reinterpret_cast<float *>(smem_raw + o[1]);
    sm.pl1 = reinterpret_cast<float *>(smem_raw + o[2]);
    sm.hpart = reinterpret_cast<unsigned long long *>(smem_raw + o[3]);
    sm.plinf = reinterpret_cast<float *>(smem_raw + o[4]);
    sm.bp = reinterpret_cast<BitParam *>(smem_raw + o[5]);
    sm.mm = reinterpret_cast<float *>(smem_raw + o[6]);
    for (int i = threadIdx.x; i < A.n_small * A.hist_words + A.big_words; i += T) sm.hist[i] = 0u;
    __syncthreads();
    if (A.counter == nullptr) {
        process_item<T, EPT, W>(A, sm, blockIdx.x);
    } else {
        __shared__ int64_t s_work;
        while (true) {
            if (threadIdx.x == 0) s_work = (int64_t)atomicAdd(A.counter, 1u);
            __syncthreads();
            const int64_t work = s_work;
            if (work >= A.n_work) break;
            process_item<T, EPT, W>(A, sm, work);
            __syncthreads();
        }
    }
}

struct ConfigEntry {
    CostConfig cfg;
    void (*kernel)(KernelArgs, int);
};

#define MGS_CFG(T, E, W) {{T, E, W, "t" #T "_e" #E "_w" #W}, k_cost<T, E, W>}
const ConfigEntry kConfigs[] = {
    MGS_CFG(256, 16, 4),
    MGS_CFG(512, 8, 4),
    MGS_CFG(256, 16, 2),
    MGS_CFG(512, 8, 8),
    MGS_CFG(256, 8, 8),
    MGS_CFG(256, 8, 4),
    MGS_CFG(128, 8, 8),
    MGS_CFG(256, 4, 8),
    MGS_CFG(512, 32, 1),
    MGS_CFG(256, 16, 1),
    MGS_CFG(512, 8, 2),
    MGS_CFG(512, 4, 8),
    MGS_CFG(512, 4, 4),
};
#undef MGS_CFG
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

// Histogram buffers of a launch.  Small buffers hold the per-lane columns
// (b <= 6), the direct tables (b <= 10) and the delta tables that fit; a big
// buffer of 16384 words takes larger bit-widths (32-bit counters up to b = 14,
// 16-bit pairs for b = 15, and b = 16 in two windows).  With a big buffer there
// is one small buffer (options alternate between the two); otherwise two.
struct HistPlan {
    int hist_words, n_small, big_words;
};
constexpr int kBigWords = 16384;

// Histogram mode and buffer of every option (fixed for a launch).  Consecutive
// options alternate buffers so that one barrier per bit-width suffices; an
// option that must reuse the previous option's buffer waits for its clearing.
void option_plan(const HistPlan &h, const int32_t *bits, int n_opts, KernelArgs *A) {
    int last = -1;
    for (int k = 0; k < n_opts; k++) {
        const int b = bits[k];
        int mode, buf = 0, windows = 1, wwords = 1 << (b - 1);
        if (b <= kLaneMaxBits) mode = kLane;
        else if (b <= kDirectMaxBits) mode = kDirect;
        else if ((1 << b) <= h.hist_words) mode = kDelta32;
        else if ((1 << (b - 1)) <= h.hist_words) mode = kDelta16;
        else if ((1 << b) <= h.big_words) {
            mode = kDelta32;
            buf = 2;
        } else {
            // 16-bit pairs in the big buffer, in windows of big_words words
            mode = kDelta16;
            buf = 2;
            wwords = std::min(1 << (b - 1), h.big_words);
            windows = (1 << (b - 1)) / wwords;
        }
        if (buf != 2) {
            buf = -1;
            for (int c = 0; c < 3 && buf < 0; c++) {
                if (c == 1 && h.n_small < 2) continue;
                if (c == 2 && h.big_words == 0) continue;
                if (c != last) buf = c;
            }
            if (buf < 0) buf = 0;
        }
        A->opt_mode[k] = (int8_t)mode;
        A->opt_buf[k] = (int8_t)buf;
        A->opt_sync[k] = (int8_t)(buf == last);
        A->opt_windows[k] = (int8_t)windows;
        A->opt_wwords[k] = wwords;
        last = buf;
    }
}

size_t smem_for(const CostConfig &c, const HistPlan &h, int n_opts) {
    size_t o[7];
    return smem_layout(c.threads, c.width, h.hist_words, h.n_small, h.big_words, n_opts, o);
}

HistPlan hist_plan(const CostConfig &c, int G, const int32_t *bits, int n_opts) {
    (void)c;
    HistPlan h{G <= 2048 ? 2048 : 4096, 2, 0};
    int bmax = bits ? 0 : MGS_MAX_BITS;
    for (int k = 0; bits && k < n_opts; k++) bmax = std::max(bmax, (int)bits[k]);
    if ((1 << (bmax - 1)) > h.hist_words) {
        h.n_small = 1;
        h.big_words = kBigWords;
    }
    return h;
}

}  // namespace

int cost_config_count() { return kNumConfigs; }
const CostConfig &cost_config(int i) { return kConfigs[i].cfg; }

int cost_default_config(int G) {
    if (G <= 1024) return 7;    // 256 x 4, W 8
    if (G <= 2048) return 5;    // 256 x 8, W 4
    if (G <= 4096) return 0;    // 256 x 16, W 4
    if (G <= 16384) return 8;   // 512 x 32, W 1
    return -1;
}

size_t cost_smem_bytes(int config, int G, int n_opts, const int32_t *bits) {
    const CostConfig &c = kConfigs[config].cfg;
    return smem_for(c, hist_plan(c, G, bits, n_opts), n_opts);
}

struct CostExec {
    const ConfigEntry *entry = nullptr;
    KernelArgs args{};
    size_t smem = 0;
    int64_t grid = 0;
    bool persistent = false;
};

mgs_status cost_exec_create(mgs_ctx *ctx, const CostLaunch &L, int config, CostExec **out,
                            std::vector<CostSeg> *segs, int64_t *n_work_out) {
    if (config < 0 || config >= kNumConfigs) {
        set_error("no tile configuration for group size %d", L.group_size);
        return MGS_ERR_INVALID_ARG;
    }
    const ConfigEntry &E = kConfigs[config];
    if ((int64_t)E.cfg.threads * E.cfg.ept < L.group_size) {
        set_error("tile %s cannot hold a group of %d", E.cfg.name, L.group_size);
        return MGS_ERR_INVALID_ARG;
    }
    int64_t n_work = 0;
    *segs = L.segs;
    for (auto &s : *segs) {
        s.n_chunks = (s.C + E.cfg.width - 1) / E.cfg.width;
        s.work_begin = n_work;
        if (s.g_count <= 0) {
            s.g_first = 0;
            s.g_count = s.n_groups;
        }
        n_work += (int64_t)s.g_count * s.n_chunks;
    }
    CostExec *X = new CostExec();
    X->entry = &E;
    KernelArgs &A = X->args;
    A.n_segs = (int32_t)segs->size();
    A.G = L.group_size;
    A.n_work = n_work;
    A.n_bits = L.n_bits;
    A.opt_lo = L.opt_lo;
    A.opt_hi = L.opt_hi;
    for (int k = 0; k < L.n_bits; k++) A.bits[k] = L.bits[k];
    A.ltab = ctx->d_ltab;
    A.dtab = ctx->d_dtab;
    const HistPlan hp = hist_plan(E.cfg, L.group_size, L.bits + L.opt_lo, L.opt_hi - L.opt_lo);
    A.hist_words = hp.hist_words;
    A.n_small = hp.n_small;
    A.big_words = hp.big_words;
    option_plan(hp, L.bits + L.opt_lo, L.opt_hi - L.opt_lo, &A);
    X->smem = smem_for(E.cfg, hp, L.opt_hi - L.opt_lo);
    X->persistent = L.persistent;
    if (X->smem > 227 * 1024) {
        set_error("tile %s needs %zu bytes of shared memory for G=%d and %d options", E.cfg.name,
                  X->smem, L.group_size, L.opt_hi - L.opt_lo);
        delete X;
        return MGS_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaFuncSetAttribute(E.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)X->smem);
    X->grid = n_work;
    if (e == cudaSuccess && L.persistent) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, E.kernel, E.cfg.threads, X->smem);
        per_sm = std::max(per_sm, 1);
        X->grid = std::min<int64_t>(n_work, (int64_t)ctx->sm_count * per_sm);
    }
    if (e != cudaSuccess) {
        set_error("cost kernel set-up: %s", cudaGetErrorString(e));
        delete X;
        return MGS_ERR_CUDA;
    }
    if (X->grid > 0x7FFFFFFF) {
        set_error("too many work items (%lld)", (long long)X->grid);
        delete X;
        return MGS_ERR_INVALID_ARG;
    }
    *n_work_out = n_work;
    *out = X;
    return MGS_OK;
}

void cost_exec_bind(CostExec *X, const CostSeg *d_segs, unsigned int *d_counter) {
    X->args.segs = d_segs;
    X->args.counter = X->persistent ? d_counter : nullptr;
}

mgs_status cost_exec_run(const CostExec *X, cudaStream_t st) {
    if (X->grid == 0) return MGS_OK;
    if (X->persistent)
        MGS_CUDA_TRY(cudaMemsetAsync(X->args.counter, 0, sizeof(unsigned int), st));
    X->entry->kernel<<<(unsigned)X->grid, X->entry->cfg.threads, X->smem, st>>>(X->args, 0);
    count_launches(1);
    MGS_CUDA_TRY(cudaGetLastError());
    return MGS_OK;
}

void cost_exec_destroy(CostExec *X) { delete X; }

mgs_status cost_launch(mgs_ctx *ctx, const CostLaunch &L, int config, CostSeg *d_segs,
                       unsigned int *d_counter, cudaStream_t st) {
    CostExec *X = nullptr;
    std::vector<CostSeg> segs;
    int64_t n_work = 0;
    MGS_TRY(cost_exec_create(ctx, L, config, &X, &segs, &n_work));
    mgs_status s = MGS_OK;
    if (n_work > 0) {
        cudaError_t e = cudaMemcpyAsync(d_segs, segs.data(), sizeof(CostSeg) * segs.size(),
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            set_error("segment upload: %s", cudaGetErrorString(e));
            s = MGS_ERR_CUDA;
        } else {
            cost_exec_bind(X, d_segs, d_counter);
            s = cost_exec_run(X, st);
        }
    }
    cost_exec_destroy(X);
    return s;
}

bool cost_config_fits(int config, int group_size, int n_opts, const int32_t *bits) {
    if (config < 0 || config >= kNumConfigs) return false;
    const CostConfig &c = kConfigs[config].cfg;
    return (int64_t)c.threads * c.ept >= group_size &&
           cost_smem_bytes(config, group_size, n_opts, bits) <= 227 * 1024;
}

}  // namespace mgs
