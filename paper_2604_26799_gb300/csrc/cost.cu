// Fused candidate-cost kernel (Sec. III-D quantiser, Sec. III-F loss matrix
// Omega and entropy bound) for every (ratio, group, channel, bit-width).
//
// One work item = (segment = (scene, ratio), group g, chunk of W channels).
// The CTA gathers the group's rows through the kept list once (W channels of
// each 32-byte slab row, vector loads), reduces min/max, and then evaluates
// every bit-width of one channel after the other.  The gathered tile stays in
// registers, or (TM tile shapes) in tensor memory, one TMEM lane per thread,
// from which one channel at a time is loaded into registers:
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
//  * Each channel is scaled by an exact power of two 2^k (R * 2^k in [1, 2)):
//    c' = c 2^k, S' = S 2^k give c'/S' = c/S and e' = e 2^k exactly, so squares
//    and sums stay in the normal FP32 range; the sums are rescaled in FP64.
// Groups where a precondition fails (subnormal S or u, |Z| >= 2^22) take the
// literal per-element formula.
//
// Histograms live in shared memory, planned on the host per launch.  The
// bit-widths up to 12 of a channel are counted together, each in its own table
// of region A, with no barrier between them: per-lane columns for b <= 6 (a
// warp never hits one address twice) and a direct table for b <= 10 (both
// summed once every count is in, in per-warp units of bins), and 16-bit
// counter pairs for b = 11, 12, where the atomic returns the bin's old count
// h - 1 and the thread adds delta(h) = L(h) - L(h - 1), L(h) = h log2 h in units
// of 2^-22 bits, so the deltas telescope to sum_bins L(h) with no scan.  Larger
// bit-widths take region B with 8-bit counters (a quarter of the 16-bit table:
// b = 16 fits 64 KB), the same telescoping sum and a shared-memory delta table:
// each in its own table when they all fit (then a channel needs two barriers),
// else one at a time.  A counter that reaches 255 sets an overflow flag, and
// the bit-width is then counted again exactly with 16-bit pairs (in windows of
// region B).  Entropy sums are integers, so they do not depend on the order of
// the updates.  Parameters of every (channel, bit-width) are computed once per
// item, and the quotients u by one correctly rounded division per element.
//
// A probe instantiation of the kernel also writes every code and every bin of
// every histogram to caller memory (test and inspection only).

#include <cuda_runtime.h>

#include <algorithm>
#include <vector>
#include <cstring>
#include <cfloat>

#include "internal.h"

namespace mgs {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;   // its bit pattern (a multiple of 4)
constexpr int kLaneMaxBits = 6;
constexpr int kDirectMaxBits = 10;
constexpr int kPairMaxBits = 12;
constexpr int kByteDelta = 260;                // delta(h), h = 0..256, in shared memory (+ pad)

enum HistMode { kLane = 0, kDirect = 1, kPair = 2, kByte = 3 };
enum Path { kFast = 0, kFastBottom = 1, kGeneric = 2, kDegenerate = 3 };

struct __align__(16) BitParam {
    float twob, Z, ytop, Ss;   // 2^b, Z, 1.5 * 2^23 + 2^b - 1, S * 2^k
    float MZ, top;             // 1.5 * 2^23 + Z (exact when |Z| < 2^22), 2^b - 1
    int path, b;
};

// Per channel of a work item: the group's range and the exact power-of-two
// scale 2^k = s1 * s2 that brings R into [1, 2).
struct __align__(16) ChanParam {
    float m, M;      // group min, max
    float Rs, rcp;   // R * 2^k and RN(1 / (R * 2^k))
    float s1, s2;
    int kexp, pad;
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
    // histogram plan (index k = option - opt_lo), fixed for the launch
    int32_t n_small;                  // options [0, n_small) share region A
    int32_t n_lane, n_direct;         // of which [0, n_lane) lane tables, then n_direct direct ones
    int32_t concurrent;               // every large option has its own table in region B
    int32_t n_units;                  // finishing work of region A: unit u = bins [lo, hi) of option k
    int16_t unit_opt[MGS_MAX_OPTIONS], unit_lo[MGS_MAX_OPTIONS], unit_hi[MGS_MAX_OPTIONS];
    int32_t a_words, b_words;         // region sizes in 32-bit words
    int8_t opt_mode[MGS_MAX_OPTIONS];
    int8_t opt_windows[MGS_MAX_OPTIONS];    // byte-counter passes of a large option
    int8_t opt_rwindows[MGS_MAX_OPTIONS];   // 16-bit-pair passes of its exact recount
    int32_t opt_off[MGS_MAX_OPTIONS];       // word offset of an option's table in region A (small)
                                            // or, when concurrent, in region B (large)
    int32_t opt_words[MGS_MAX_OPTIONS];     // words of one pass's table
    // probe outputs (probe instantiation only)
    uint32_t *hist_out;               // [item][hist_stride]: every bin of every option
    uint16_t *codes_out;              // per segment at seg.code_off: [C][n_bits][K]
    int64_t hist_stride;
    int64_t hist_off[MGS_MAX_OPTIONS];  // bin offset of option j (global index) in an item's row
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
MGS_F2_BINOP(fmul2, "mul.rn.f32x2")
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

// ---- tensor memory: the gathered tile of a slab (8 channels) is kept in this
// CTA's TMEM, one lane per thread, channel-major columns, so that only the
// channel being evaluated occupies registers.
__device__ __forceinline__ void tm_alloc(uint32_t *dst, uint32_t ncols) {   // one whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {   // the same warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tm_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Four consecutive 32-bit columns of this thread's lane.
__device__ __forceinline__ void tm_st4(uint32_t taddr, float a, float b, float c, float d) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)),
                 "r"(__float_as_uint(d))
                 : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 16 or 8 consecutive columns of this thread's lane (no wait).
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tm_ld8(uint32_t taddr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
// N (8, 16 or 32) consecutive columns of this thread's lane into v.
template <int N>
__device__ __forceinline__ void tm_ld(uint32_t taddr, float (&v)[N]) {
    static_assert(N == 8 || N % 16 == 0, "8 or a multiple of 16 columns");
    uint32_t r[N];
    if constexpr (N == 8) {
        tm_ld8(taddr, r);
    } else {
#pragma unroll
        for (int j = 0; j < N; j += 16) tm_ld16(taddr + (uint32_t)j, r + j);
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < N; j++) v[j] = __uint_as_float(r[j]);
}
// TMEM columns of a CTA: T/128 column blocks (warps w and w + 4 share lanes) of
// EPT x W columns, rounded up to a power of two (at least 32).
__host__ __device__ constexpr int tm_cols(int T, int EPT, int W) {
    int c = (T / 128 > 0 ? T / 128 : 1) * EPT * W, p = 32;
    while (p < c) p <<= 1;
    return p;
}

// ---- shared-memory histogram operations ------------------------------------
// Predicated forms execute only where `pred` holds (predicated, not branched:
// lanes taking different sides do not split the warp); atom_if returns 0 elsewhere.
__device__ __forceinline__ void red_if(bool pred, uint32_t addr, uint32_t v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q red.shared.add.u32 [%0], %1;\n\t}"
                 ::"r"(addr), "r"(v), "r"((uint32_t)pred));
}
__device__ __forceinline__ uint32_t atom_if(bool pred, uint32_t addr, uint32_t v) {
    uint32_t old = 0;
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q atom.shared.add.u32 %0, [%1], %2;\n\t}"
                 : "+r"(old)
                 : "r"(addr), "r"(v), "r"((uint32_t)pred));
    return old;
}
__device__ __forceinline__ void red_add(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ uint32_t atom_add(uint32_t addr, uint32_t v) {
    uint32_t old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(v));
    return old;
}
// Shared-memory stores executed only where `pred` holds, as predicated
// instructions: lanes never take different branches around them.
__device__ __forceinline__ void sts_if(bool pred, uint32_t addr, uint32_t v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.u32 [%0], %1;\n\t}"
                 ::"r"(addr), "r"(v), "r"((uint32_t)pred) : "memory");
}
__device__ __forceinline__ void sts_if(bool pred, uint32_t addr, unsigned long long v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.u64 [%0], %1;\n\t}"
                 ::"r"(addr), "l"(v), "r"((uint32_t)pred) : "memory");
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// Byte permutes: b4e places byte 0 of a at byte position sel & 3 (the other
// bytes come from zeros); f4e brings byte sel & 3 of a down to byte 0.
__device__ __forceinline__ uint32_t byte_at(uint32_t a, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32.b4e %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(0u), "r"(sel));
    return d;
}
__device__ __forceinline__ uint32_t byte_from(uint32_t a, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32.f4e %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(0u), "r"(sel));
    return d & 0xFFu;
}

// Where one pass counts.  y is a code's bit pattern kMagicBits + q; the magic
// offset is folded into the bases.
struct HistPass {
    uint32_t lane_base;   // lane: table + lane * 4 - (kMagicBits << 7)
    uint32_t dbase;       // direct: table - (kMagicBits << 2)
    uint32_t base;        // pair / byte: table (shared address)
    uint32_t wlo, wn;     // pair / byte: words [wlo, wlo + wn) of the full table are counted
    uint32_t boff, wn4;   // byte: kMagicBits + 4 wlo, 4 wn
    const uint32_t *dtab; // pair: global delta table
    uint32_t dsm;         // byte: shared delta table (h = 0..256)
};

// Count one code.  PRED: `valid` may be false (partial groups, windows); WIN:
// only codes whose word lies in the pass's window are counted.  The delta modes
// add delta(new count) to dacc; byte mode keeps in ovf the largest count a
// counter had before its increment (255: it overflowed).
template <int MODE, bool PRED, bool WIN>
__device__ __forceinline__ void hist_count(bool valid, uint32_t y, const HistPass &h, uint32_t &dacc,
                                           uint32_t &ovf) {
    if (MODE == kLane) {
        const uint32_t a = h.lane_base + (y << 7);
        if (PRED) red_if(valid, a, 1u); else red_add(a, 1u);
    } else if (MODE == kDirect) {
        const uint32_t a = h.dbase + (y << 2);
        if (PRED) red_if(valid, a, 1u); else red_add(a, 1u);
    } else if (MODE == kPair) {
        const uint32_t q = y - kMagicBits;
        const uint32_t word = (q >> 1) - (WIN ? h.wlo : 0u);
        const uint32_t sh = (q & 1u) << 4;
        const bool in = (!PRED || valid) && (!WIN || word < h.wn);
        const uint32_t old = (PRED || WIN) ? atom_if(in, h.base + (word << 2), 1u << sh)
                                           : atom_add(h.base + (word << 2), 1u << sh);
        const uint32_t d = ld_keep(&h.dtab[((old >> sh) & 0xFFFFu) + 1u]);
        dacc += (PRED || WIN) ? (in ? d : 0u) : d;
    } else {
        // kMagicBits is a multiple of 4: the counter is byte y & 3 of the word at
        // byte offset (y & ~3) - kMagicBits of the full table
        const uint32_t off = (y & ~3u) - h.boff;
        const bool in = (!PRED || valid) && (!WIN || off < h.wn4);
        const uint32_t inc = byte_at(1u, y);
        const uint32_t old = (PRED || WIN) ? atom_if(in, h.base + off, inc) : atom_add(h.base + off, inc);
        const uint32_t cnt = byte_from(old, y);   // 0 where nothing was counted
        const uint32_t d = lds_u32(h.dsm + 4u + (cnt << 2));
        dacc += (PRED || WIN) ? (in ? d : 0u) : d;
        ovf = max(ovf, cnt);
    }
}

struct EvalOut {
    float sse, l1, linf;
    uint32_t dacc, ovf;
};

// Fast path for one bit-width over this thread's elements (pairs, packed
// f32x2 adds, subtracts and FMAs).  The reconstruction product (q - Z) S is an
// FMA with a zero addend: the same single rounding as the product, and an FMA
// result is never fused with the subtraction after it.
template <int T, int EPT, int MODE, bool BOTTOM, bool FULL, bool WIN, bool PROBE>
__device__ __forceinline__ void eval_fast(const float2 (&c)[EPT / 2], const float2 (&u)[EPT / 2], int nvalid,
                                          const BitParam &p, const HistPass &h, uint16_t *codes,
                                          EvalOut &o) {
    const float2 tw = make_float2(p.twob, p.twob), zz = make_float2(p.Z, p.Z);
    const float2 mg = make_float2(kMagic, kMagic), mz = make_float2(p.MZ, p.MZ);
    const float2 ss = make_float2(p.Ss, p.Ss), zero = make_float2(0.0f, 0.0f);
    float2 s2 = make_float2(0.0f, 0.0f);
    float la = 0.0f, lb = 0.0f, lm = 0.0f;
    uint32_t dacc = 0, ovf = 0;   // delta sums: at most EPT * 2^26 < 2^32
#pragma unroll
    for (int e = 0; e < EPT; e += 2) {
        const int i0 = e * T + (int)threadIdx.x, i1 = i0 + T;
        const bool v0 = FULL || i0 < nvalid, v1 = FULL || i1 < nvalid;
        const float2 x = ffma2(u[e / 2], tw, zz);
        float2 y = fadd2(x, mg);
        y.x = fminf(y.x, p.ytop);
        y.y = fminf(y.y, p.ytop);
        if (BOTTOM) {
            y.x = fmaxf(y.x, kMagic);
            y.y = fmaxf(y.y, kMagic);
        }
        const float2 d = fsub2(y, mz);
        const float2 ch = ffma2(d, ss, zero);   // d = q - Z is never -0
        float2 er = fsub2(ch, c[e / 2]);
        if (!FULL) {
            er.x = v0 ? er.x : 0.0f;
            er.y = v1 ? er.y : 0.0f;
        }
        s2 = ffma2(er, er, s2);
        la = __fadd_rn(la, fabsf(er.x));
        lb = __fadd_rn(lb, fabsf(er.y));
        lm = fmaxf(lm, fmaxf(fabsf(er.x), fabsf(er.y)));
        const uint32_t y0 = __float_as_uint(y.x), y1 = __float_as_uint(y.y);
        hist_count<MODE, !FULL, WIN>(v0, y0, h, dacc, ovf);
        hist_count<MODE, !FULL, WIN>(v1, y1, h, dacc, ovf);
        if (PROBE) {
            if (v0) codes[i0] = (uint16_t)(y0 - kMagicBits);
            if (v1) codes[i1] = (uint16_t)(y1 - kMagicBits);
        }
    }
    o.sse = __fadd_rn(s2.x, s2.y);
    o.l1 = __fadd_rn(la, lb);
    o.linf = lm;
    o.dacc = dacc;
    o.ovf = ovf >= 0xFFu;
}

// Literal per-element formula (divisions, both clamps); any group.
template <int T, int EPT, int MODE, bool WIN, bool PROBE>
__device__ __forceinline__ void eval_generic(const float2 (&c2)[EPT / 2], int nvalid, const BitParam &p,
                                             const HistPass &h, uint16_t *codes, EvalOut &o) {
    float s = 0.0f, a = 0.0f, m = 0.0f;
    uint32_t dacc = 0, ovf = 0;
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        const int i = e * T + (int)threadIdx.x;
        const bool valid = i < nvalid;
        const float ce = (e & 1) ? c2[e / 2].y : c2[e / 2].x;
        const float x = __fadd_rn(__fdiv_rn(ce, p.Ss), p.Z);   // c'/S' == c/S exactly
        const float xc = fminf(fmaxf(x, 0.0f), p.top);
        const int q = __float2int_rn(xc);
        const float qz = __fsub_rn(__int2float_rn(q), p.Z);
        float er = __fsub_rn(__fmul_rn(qz, p.Ss), ce);
        er = valid ? er : 0.0f;
        s = __fmaf_rn(er, er, s);
        a = __fadd_rn(a, fabsf(er));
        m = fmaxf(m, fabsf(er));
        hist_count<MODE, true, WIN>(valid, kMagicBits + (uint32_t)q, h, dacc, ovf);
        if (PROBE && valid) codes[i] = (uint16_t)q;
    }
    o.sse = s;
    o.l1 = a;
    o.linf = m;
    o.dacc = dacc;
    o.ovf = ovf >= 0xFFu;
}

// The fast path runs for warps whose elements are all valid, in groups whose
// minimum does not round below code 0; every other warp (the tail of a partial
// group) and every other group takes the literal formula, which gives the same
// codes and errors.  WIN: only the codes of the pass's window are counted (a
// table larger than its region).
template <int T, int EPT, int MODE, bool WIN, bool PROBE>
__device__ __forceinline__ void eval_dispatch(const float2 (&c)[EPT / 2], const float2 (&u)[EPT / 2], int nvalid,
                                              bool full, bool generic, const BitParam &p,
                                              const HistPass &h, uint16_t *codes, EvalOut &o) {
    if (!generic && full && p.path == kFast)
        eval_fast<T, EPT, MODE, false, true, WIN, PROBE>(c, u, nvalid, p, h, codes, o);
    else
        eval_generic<T, EPT, MODE, WIN, PROBE>(c, nvalid, p, h, codes, o);
}

// Count-only pass over one window of a pair or byte table: the codes of the
// evaluation pass (same operations), no error sums.
template <int T, int EPT, int MODE>
__device__ __forceinline__ void count_window(const float2 (&c)[EPT / 2], const float2 (&u)[EPT / 2],
                                             int nvalid, bool generic, const BitParam &p, const HistPass &h,
                                             uint32_t &dacc, uint32_t &ovf) {
    if (generic) {
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            const float ce = (e & 1) ? c[e / 2].y : c[e / 2].x;
            const float x = __fadd_rn(__fdiv_rn(ce, p.Ss), p.Z);
            const uint32_t y = kMagicBits + (uint32_t)__float2int_rn(fminf(fmaxf(x, 0.0f), p.top));
            hist_count<MODE, true, true>(e * T + (int)threadIdx.x < nvalid, y, h, dacc, ovf);
        }
    } else {
        // the lower clamp is a no-op unless the group minimum rounds below code 0
        const float lo = p.path == kFastBottom ? kMagic : -FLT_MAX;
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            const float ue = (e & 1) ? u[e / 2].y : u[e / 2].x;
            float y = __fadd_rn(__fmaf_rn(ue, p.twob, p.Z), kMagic);
            y = fmaxf(fminf(y, p.ytop), lo);
            hist_count<MODE, true, true>(e * T + (int)threadIdx.x < nvalid, __float_as_uint(y), h, dacc, ovf);
        }
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

// Shared-memory layout (dynamic).  The per-warp partials of a channel's
// options are double-buffered by channel parity, so that one warp reduces a
// channel while the others evaluate the next:
//   regionA[a_words] | regionB[b_words] | bdelta[kByteDelta]
//   | part2[2][n_opts][NW] (float2) | hpart[2][n_opts][NW] (u64) | plinf[2][n_opts][NW]
//   | bp[W][n_opts] | ch[W] | mm[NW][W][2] | flags[2][n_opts]
struct Smem {
    uint32_t *ra, *rb, *bdelta, *flags;
    float2 *part2;
    unsigned long long *hpart;
    float *plinf, *mm;
    BitParam *bp;
    ChanParam *ch;
};

__host__ __device__ inline size_t smem_layout(int T, int W, int a_words, int b_words, int n_opts,
                                              size_t *o) {
    const int NW = T / 32;
    size_t off = 0;
    o[0] = off; off += (size_t)a_words * 4;
    o[1] = off; off += (size_t)b_words * 4;
    o[2] = off; off += (size_t)kByteDelta * 4;
    off = (off + 15) & ~(size_t)15;
    o[3] = off; off += (size_t)2 * n_opts * NW * 8;
    o[4] = off; off += (size_t)2 * n_opts * NW * 8;
    o[5] = off; off += (size_t)2 * n_opts * NW * 4;
    off = (off + 15) & ~(size_t)15;
    o[6] = off; off += (size_t)W * n_opts * sizeof(BitParam);
    o[7] = off; off += (size_t)W * sizeof(ChanParam);
    o[8] = off; off += (size_t)NW * W * 2 * 4;
    o[9] = off; off += (size_t)2 * n_opts * 4;
    return (off + 15) & ~(size_t)15;
}

// Clear `words` words (a multiple of 4) of a table, 16 bytes per store.
template <int T>
__device__ __forceinline__ void clear_words(uint32_t *t, int words) {
    uint4 *t4 = reinterpret_cast<uint4 *>(t);
    for (int k = threadIdx.x; k < words / 4; k += T) t4[k] = make_uint4(0u, 0u, 0u, 0u);
}

// Probe readout of a table of `per_word` counters per word (2: 16-bit pairs,
// 4: 8-bit), holding bins [first, first + words * per_word) of an option; each
// thread clears the words it read (the readout replaces clear_words, whose
// thread-to-word mapping differs, so that no word is cleared before it is read).
template <int T>
__device__ void probe_packed_clear(uint32_t *t, int words, int per_word, int64_t first, int bins,
                                   uint32_t *out) {
    const int bits = 32 / per_word;
    const uint32_t mask = per_word == 2 ? 0xFFFFu : 0xFFu;
    for (int j = threadIdx.x; j < words; j += T) {
        const uint32_t v = t[j];
        t[j] = 0u;
        for (int s = 0; s < per_word; s++) {
            const int64_t bin = first + (int64_t)j * per_word + s;
            if (bin < bins) out[bin] = (v >> (s * bits)) & mask;
        }
    }
}

// Probe readout of a degenerate option (every code 0): bin 0 holds the group.
template <int T>
__device__ void probe_degenerate(uint32_t *out, int bins, int nvalid) {
    for (int j = threadIdx.x; j < bins; j += T) out[j] = j == 0 ? (uint32_t)nvalid : 0u;
}

// After every count of region A is in: sum L(h) of the scanned tables, clear
// every table, and add each option's sum to the finishing warp's hpart slot.
// The work is cut on the host into units (a range of one option's bins), one
// per warp when there are enough: lane l of a warp takes bins lo + l, lo + l +
// 32, ...; a lane table's bin is its 32 lane columns, read as 16-byte chunks
// in a rotated order so that eight lanes hit eight distinct bank groups.  The
// integer sums do not depend on which warp adds what.
template <int T, bool PROBE>
__device__ void finish_small(const KernelArgs &A, const Smem &sm, const BitParam *bpw, int par,
                             int nvalid, int64_t item) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = T / 32;
    const int n_opts = A.opt_hi - A.opt_lo;
    const int n_ld = A.n_lane + A.n_direct;
    for (int un = warp; un < A.n_units; un += NW) {
        const int k = A.unit_opt[un], lo = A.unit_lo[un], hi = A.unit_hi[un];
        const BitParam &bp = bpw[k];
        uint32_t *t = sm.ra + A.opt_off[k];
        uint32_t *pout = PROBE ? A.hist_out + item * A.hist_stride + A.hist_off[A.opt_lo + k] : nullptr;
        if (bp.path == kDegenerate) {
            if (PROBE)
                for (int j = lo + lane; j < hi; j += 32) pout[j] = j == 0 ? (uint32_t)nvalid : 0u;
            continue;   // table untouched; hpart written by the evaluation pass
        }
        unsigned long long hacc = 0ull;
        if (k < A.n_lane) {
            for (int r = lo + lane; r < hi; r += 32) {
                uint4 *row = reinterpret_cast<uint4 *>(t + r * 32);
                uint32_t s = 0;
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const uint4 v = row[(q + r) & 7];
                    s += v.x + v.y + v.z + v.w;
                }
#pragma unroll
                for (int q = 0; q < 8; q++) row[(q + r) & 7] = make_uint4(0u, 0u, 0u, 0u);
                hacc += ld_keep(&A.ltab[s]);
                if (PROBE) pout[r] = s;
            }
        } else if (k < n_ld) {
            // L(0) = 0, so an empty bin adds nothing
#pragma unroll 8
            for (int j = lo + lane; j < hi; j += 32) {
                const uint32_t v = t[j];
                t[j] = 0u;
                hacc += ld_keep(&A.ltab[v]);
                if (PROBE) pout[j] = v;
            }
        } else {
            // 16-bit pairs (two bins a word): the delta sums were added by the evaluation pass
            for (int j = lo / 2 + lane; j < hi / 2; j += 32) {
                const uint32_t v = t[j];
                t[j] = 0u;
                if (PROBE) {
                    pout[2 * j] = v & 0xFFFFu;
                    pout[2 * j + 1] = v >> 16;
                }
            }
            continue;
        }
        hacc = warp_sum_u64_redux(hacc);
        if (lane == 0) sm.hpart[(par * n_opts + k) * NW + warp] += hacc;
        __syncwarp();
    }
}

// One evaluation pass of option k: codes, errors and counts into table `t`;
// the warp's sums into its slot of the option's partials (parity `par`).
template <int T, int EPT, bool PROBE, int MODE, bool WIN>
__device__ __forceinline__ void run_option(const KernelArgs &A, const Smem &sm, int k, int par,
                                           const BitParam &pp, uint32_t *t, uint32_t wn,
                                           const float2 (&cw)[EPT / 2], const float2 (&u)[EPT / 2],
                                           int nvalid, unsigned long long lnv, bool full, bool any_slow,
                                           uint16_t *codes) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = T / 32;
    const int n_opts = A.opt_hi - A.opt_lo;
    const BitParam p = pp;
    EvalOut o{0.0f, 0.0f, 0.0f, 0u, 0u};
    unsigned long long hdeg = 0ull;
    if (p.path == kDegenerate) {
        if (threadIdx.x == 0) hdeg = lnv;
        if (PROBE)
            for (int e = 0; e < EPT; e++)
                if (e * T + (int)threadIdx.x < nvalid) codes[e * T + threadIdx.x] = 0;
    } else {
        const bool generic = p.path == kGeneric || any_slow;
        HistPass h;
        const uint32_t tb = (uint32_t)__cvta_generic_to_shared(t);
        h.lane_base = tb + lane * 4u - (kMagicBits << 7);
        h.dbase = tb - (kMagicBits << 2);
        h.base = tb;
        h.wlo = 0u;
        h.wn = wn;
        h.boff = kMagicBits;
        h.wn4 = wn * 4u;
        h.dtab = A.dtab;
        h.dsm = (uint32_t)__cvta_generic_to_shared(sm.bdelta);
        eval_dispatch<T, EPT, MODE, WIN, PROBE>(cw, u, nvalid, full, generic, p, h, codes, o);
    }
    // the warp's sums, in a fixed shuffle tree: the first step leaves the SSE
    // halves in lanes 0-15 and the L1 halves in lanes 16-31, so that one tree
    // of four more steps ends with the SSE in lane 0 and the L1 in lane 16
    const bool upper = (lane & 16) != 0;
    float sl = __fadd_rn(upper ? o.l1 : o.sse, __shfl_xor_sync(kFull, upper ? o.sse : o.l1, 16));
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) sl = __fadd_rn(sl, __shfl_xor_sync(kFull, sl, off));
    const uint32_t lmax = __reduce_max_sync(kFull, __float_as_uint(o.linf));
    constexpr bool kDelta = MODE == kPair || MODE == kByte;
    const unsigned long long hs = warp_sum_u64_redux((unsigned long long)o.dacc + hdeg);
    const uint32_t ovf = kDelta ? __any_sync(kFull, o.ovf != 0u) : 0u;
    // the stores are predicated, so that the warp stays converged into the
    // collectives of the next pass
    const int slot = (par * n_opts + k) * NW + warp;
    sts_if(lane == 0 || lane == 16, (uint32_t)__cvta_generic_to_shared(&sm.part2[slot]) + (lane ? 4u : 0u),
           __float_as_uint(sl));
    sts_if(lane == 0, (uint32_t)__cvta_generic_to_shared(&sm.plinf[slot]), lmax);
    sts_if(lane == 0, (uint32_t)__cvta_generic_to_shared(&sm.hpart[slot]), hs);
    sts_if(lane == 0 && ovf != 0u, (uint32_t)__cvta_generic_to_shared(&sm.flags[par * n_opts + k]), 1u);
    __syncwarp();
}

// Sums of one channel's options over the warps' slots (fixed order), written
// to the table; the slots' flags are reset for the channel after next.
template <int T>
__device__ __forceinline__ void reduce_channel(const KernelArgs &A, const Smem &sm, const CostSeg &S,
                                               int par, int64_t item, int kexp, unsigned long long lnv) {
    constexpr int NW = T / 32;
    const int n_opts = A.opt_hi - A.opt_lo;
    const int j = threadIdx.x & 31;
    if (j >= n_opts) return;
    float a = 0.0f, b = 0.0f, cmax = 0.0f;
    unsigned long long hs = 0ull;
    const int base = (par * n_opts + j) * NW;
#pragma unroll
    for (int q = 0; q < NW; q++) {
        const float2 v = sm.part2[base + q];
        a = __fadd_rn(a, v.x);
        b = __fadd_rn(b, v.y);
        cmax = fmaxf(cmax, sm.plinf[base + q]);
        hs += sm.hpart[base + q];
    }
    sm.flags[par * n_opts + j] = 0u;
    const int64_t o = item * A.n_bits + A.opt_lo + j;
    // undo the 2^k scale in FP64 (exact powers of two)
    const double inv = __longlong_as_double((long long)(1023 - kexp) << 52);
    const double inv2 = __longlong_as_double((long long)(1023 - 2 * kexp) << 52);
    S.sse[o] = (double)a * inv2;
    S.l1[o] = (double)b * inv;
    S.linf[o] = (float)((double)cmax * inv);
    S.hbits[o] = (double)(long long)(lnv - hs) * (1.0 / 4194304.0);   // 2^-22
}

// The parameters of option k (bit-width b) of a channel (Sec. III-D): S, Z, and
// which evaluation path the group takes.
__device__ __forceinline__ BitParam make_param(int b, float m, float M, float R, float s1, float s2) {
    BitParam p;
    p.b = b;
    p.twob = (float)(1u << b);
    p.top = p.twob - 1.0f;
    p.ytop = kMagic + p.top;
    const float S_ = __fdiv_rn(R, p.twob);
    p.Ss = __fmul_rn(__fmul_rn(S_, s1), s2);
    if (S_ == 0.0f) {
        p.path = kDegenerate;
        p.Z = 0.0f;
        p.MZ = kMagic;
    } else {
        p.Z = rintf(__fsub_rn(p.twob, __fdiv_rn(M, S_)));
        p.MZ = __fadd_rn(kMagic, p.Z);
        if (S_ < FLT_MIN || fabsf(p.Z) >= 4194304.0f) {
            p.path = kGeneric;
        } else {
            // the group minimum gives the smallest x: lower clamp only if it rounds below 0
            const float um = __fdiv_rn(m, R);
            const float ym = __fadd_rn(__fmaf_rn(um, p.twob, p.Z), kMagic);
            p.path = ym < kMagic ? kFastBottom : kFast;
        }
    }
    return p;
}

// A large option whose byte counters overflowed: count it again exactly with
// 16-bit pairs, in windows of region B (which this clears first), and replace
// the warps' entropy sums.
template <int T, int EPT, bool PROBE>
__device__ void recount_pairs(const KernelArgs &A, const Smem &sm, int k, int par, const BitParam &p,
                              const float2 (&cv)[EPT / 2], const float2 (&uv)[EPT / 2], int nvalid,
                              bool generic, uint32_t *pout) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = T / 32;
    const int n_opts = A.opt_hi - A.opt_lo;
    const int bins = 1 << p.b;
    HistPass h;
    h.base = (uint32_t)__cvta_generic_to_shared(sm.rb);
    h.dtab = A.dtab;
    h.dsm = (uint32_t)__cvta_generic_to_shared(sm.bdelta);
    h.lane_base = h.dbase = 0u;
    uint32_t dacc = 0, ovf = 0;
    clear_words<T>(sm.rb, A.b_words);
    const int rw = A.b_words;
#pragma unroll 1
    for (int win = 0; win < A.opt_rwindows[k]; win++) {
        __syncthreads();
        h.wlo = (uint32_t)win * rw;
        h.wn = (uint32_t)rw;
        count_window<T, EPT, kPair>(cv, uv, nvalid, generic, p, h, dacc, ovf);
        __syncthreads();
        if (PROBE) probe_packed_clear<T>(sm.rb, rw, 2, (int64_t)win * rw * 2, bins, pout);
        else clear_words<T>(sm.rb, rw);
    }
    const unsigned long long hs = warp_sum_u64_redux((unsigned long long)dacc);
    if (lane == 0) sm.hpart[(par * n_opts + k) * NW + warp] = hs;
}

// TM: the item is a whole slab (W = 8), staged in TMEM at column base `tm`
// (this thread's lane and column block); else the W channels stay in registers.
// `par` is the parity of the partials' buffers, carried from item to item.
template <int T, int EPT, int W, bool PROBE, bool TM>
__device__ void process_item(const KernelArgs &A, const Smem &sm, int64_t work, uint32_t tm, int &par,
                             int &seg_hint) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = T / 32;
    // ---- decode the work item: a persistent CTA's work indices rise, so its
    // segment is found by stepping on from the previous one
    __shared__ int s_seg;
    if (threadIdx.x == 0) {
        int lo;
        if (A.counter != nullptr && seg_hint >= 0 && A.segs[seg_hint].work_begin <= work) {
            lo = seg_hint;
            while (lo + 1 < A.n_segs && A.segs[lo + 1].work_begin <= work) lo++;
        } else {
            lo = 0;
            int hi = A.n_segs - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (A.segs[mid].work_begin <= work) lo = mid; else hi = mid - 1;
            }
        }
        s_seg = lo;
    }
    __syncthreads();
    seg_hint = s_seg;
    const CostSeg &S = A.segs[s_seg];
    const int64_t local = work - S.work_begin;
    const int g = S.g_first + (int)(local / S.n_chunks);
    const int chunk = (int)(local % S.n_chunks);
    const int c0 = chunk * W;
    const int slab = c0 / kSlabWidth;
    const int j0 = c0 % kSlabWidth;
    const int64_t gstart = (int64_t)g * A.G;
    const int nvalid = (int)((S.K - gstart) < (int64_t)A.G ? (S.K - gstart) : (int64_t)A.G);
    // every element of this warp is valid (warp-uniform)
    const bool full = __all_sync(kFull, (EPT - 1) * T + (int)threadIdx.x < nvalid);
    const unsigned long long lnv = __ldg(&A.ltab[nvalid]);   // L(n) of the group
    const int n_opts = A.opt_hi - A.opt_lo;

    // ---- gather: each element's W channels from its slab row, and the
    // per-thread min / max of every channel
    float v[TM ? 1 : W][EPT];   // TM: the channel being evaluated; else all W channels
    float tmn[W], tmx[W];
#pragma unroll
    for (int w = 0; w < W; w++) {
        tmn[w] = FLT_MAX;
        tmx[w] = -FLT_MAX;
    }
    if constexpr (TM) {
        static_assert(W == kSlabWidth && EPT % 8 == 0, "a TMEM tile holds whole slab rows, 8 elements per batch");
        int32_t pos[EPT];
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            const int i = e * T + threadIdx.x;
            pos[e] = i < nvalid ? (S.kept ? ld_stream(&S.kept[gstart + i]) : (int32_t)(gstart + i)) : -1;
        }
#pragma unroll
        for (int e0 = 0; e0 < EPT; e0 += 8) {
            float r[8][W];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (pos[e0 + j] >= 0) {
                    load_row<W>(S.slabs + ((int64_t)slab * S.n + pos[e0 + j]) * kSlabWidth, r[j]);
#pragma unroll
                    for (int w = 0; w < W; w++) {
                        tmn[w] = fminf(tmn[w], r[j][w]);
                        tmx[w] = fmaxf(tmx[w], r[j][w]);
                    }
                } else {
#pragma unroll
                    for (int w = 0; w < W; w++) r[j][w] = 0.0f;
                }
            }
            __syncwarp();   // the stores below are warp-collective
#pragma unroll
            for (int w = 0; w < W; w++) {
                tm_st4(tm + (uint32_t)(w * EPT + e0), r[0][w], r[1][w], r[2][w], r[3][w]);
                tm_st4(tm + (uint32_t)(w * EPT + e0 + 4), r[4][w], r[5][w], r[6][w], r[7][w]);
            }
        }
        tm_wait_st();
    } else {
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            int i = e * T + threadIdx.x;
            float row[W];
            if (i < nvalid) {
                const int32_t pos = S.kept ? ld_stream(&S.kept[gstart + i]) : (int32_t)(gstart + i);
                load_row<W>(S.slabs + ((int64_t)slab * S.n + pos) * kSlabWidth + j0, row);
#pragma unroll
                for (int w = 0; w < W; w++) {
                    tmn[w] = fminf(tmn[w], row[w]);
                    tmx[w] = fmaxf(tmx[w], row[w]);
                }
            } else {
#pragma unroll
                for (int w = 0; w < W; w++) row[w] = 0.0f;
            }
#pragma unroll
            for (int w = 0; w < W; w++) v[TM ? 0 : w][e] = row[w];
        }
    }

    // ---- warp min / max of every channel
#pragma unroll
    for (int w = 0; w < W; w++) {
        const float mn = warp_min(tmn[w]), mx = warp_max(tmx[w]);
        if (lane == 0) {
            sm.mm[(warp * W + w) * 2] = mn;
            sm.mm[(warp * W + w) * 2 + 1] = mx;
        }
    }
    __syncthreads();
    // ---- every (channel, option) parameter of the item at once
    for (int i = threadIdx.x; i < W * n_opts; i += T) {
        const int w = i / n_opts, k = i - w * n_opts;
        float m = FLT_MAX, M = -FLT_MAX;
        for (int q = 0; q < NW; q++) {
            m = fminf(m, sm.mm[(q * W + w) * 2]);
            M = fmaxf(M, sm.mm[(q * W + w) * 2 + 1]);
        }
        const float R = __fsub_rn(M, m);
        // exact power-of-two scale 2^k = s1 * s2 with R * 2^k in [1, 2)
        const int kexp = R > 0.0f ? -ilogbf(R) : 0;
        const int k1 = kexp / 2, k2 = kexp - k1;
        const float s1 = __int_as_float((k1 + 127) << 23), s2 = __int_as_float((k2 + 127) << 23);
        if (k == 0) {
            ChanParam c;
            c.m = m;
            c.M = M;
            c.Rs = __fmul_rn(__fmul_rn(R, s1), s2);
            c.rcp = R > 0.0f ? __frcp_rn(c.Rs) : 0.0f;
            c.s1 = s1;
            c.s2 = s2;
            c.kexp = kexp;
            c.pad = 0;
            sm.ch[w] = c;
            if (c0 + w < S.C) {
                const int64_t item = S.item_base + (int64_t)(c0 + w) * S.n_groups + g;
                S.cnt[item] = nvalid;
                S.vmin[item] = m;
                S.vmax[item] = M;
            }
        }
        sm.bp[w * n_opts + k] = make_param(A.bits[A.opt_lo + k], m, M, R, s1, s2);
    }
    __syncthreads();

    const int n_ld = A.n_lane + A.n_direct;
#pragma unroll 1
    for (int w = 0; w < W; w++) {
        const int ch = c0 + w;
        if (ch >= S.C) break;
        const ChanParam cp = sm.ch[w];
        const BitParam *bpw = sm.bp + w * n_opts;
        const int64_t item = S.item_base + (int64_t)ch * S.n_groups + g;
        if constexpr (TM) tm_ld<EPT>(tm + (uint32_t)(w * EPT), v[0]);   // this channel's values
        // scale by 2^k (exact), then one correctly rounded division per element,
        // u = c / R, shared by every bit-width: q0 = c * r with r = RN(1 / R),
        // and two corrections q' = q + RN(c - q R) r (Markstein's method; the
        // second remainder is exact because q is then within an ulp, and the
        // result rounds correctly because r is the correctly rounded reciprocal).
        // A warp with a nonzero scaled value below 2^-100 takes the literal
        // formula instead (its quotients may be subnormal, and the remainders of
        // such tiny values need not be exact); the two paths give the same codes.
        // (R = 0: r = 0 gives u = 0; such a group is degenerate at every width)
        float2 cv[EPT / 2], uv[EPT / 2];
        bool slow = false;
        const float2 ss1 = make_float2(cp.s1, cp.s1), ss2 = make_float2(cp.s2, cp.s2);
        const float2 rr = make_float2(cp.rcp, cp.rcp), nR = make_float2(-cp.Rs, -cp.Rs);
#pragma unroll
        for (int e = 0; e < EPT; e += 2) {
            const float2 c2 = fmul2(fmul2(make_float2(v[0][e], v[0][e + 1]), ss1), ss2);
            cv[e / 2] = c2;
            float2 q = fmul2(c2, rr);
            q = ffma2(ffma2(q, nR, c2), rr, q);
            uv[e / 2] = ffma2(ffma2(q, nR, c2), rr, q);
            slow |= (fabsf(c2.x) < 7.8886090522101181e-31f && c2.x != 0.0f) ||   // 2^-100
                    (fabsf(c2.y) < 7.8886090522101181e-31f && c2.y != 0.0f);
        }
        const bool any_slow = __any_sync(kFull, slow);

        uint16_t *codes = nullptr;
        if (PROBE && A.codes_out)
            codes = A.codes_out + S.code_off + (int64_t)ch * A.n_bits * S.K + gstart;
        const int64_t kstride = S.K;   // codes of consecutive options of a channel
#define MGS_CODES(k) (codes ? codes + (A.opt_lo + (k)) * kstride : nullptr)
        // ---- bit-widths up to 12: every table of region A, no barrier between them
        int k = 0;
#pragma unroll 1
        for (; k < A.n_lane; k++)
            run_option<T, EPT, PROBE, kLane, false>(A, sm, k, par, bpw[k], sm.ra + A.opt_off[k], 0u, cv, uv,
                                                    nvalid, lnv, full, any_slow, MGS_CODES(k));
#pragma unroll 1
        for (; k < n_ld; k++)
            run_option<T, EPT, PROBE, kDirect, false>(A, sm, k, par, bpw[k], sm.ra + A.opt_off[k], 0u, cv,
                                                      uv, nvalid, lnv, full, any_slow, MGS_CODES(k));
#pragma unroll 1
        for (; k < A.n_small; k++)
            run_option<T, EPT, PROBE, kPair, false>(A, sm, k, par, bpw[k], sm.ra + A.opt_off[k], 0u, cv, uv,
                                                    nvalid, lnv, full, any_slow, MGS_CODES(k));
        uint32_t *flags = sm.flags + par * n_opts;
        if (A.concurrent) {
            // ---- larger bit-widths, each in its own table of region B (byte
            // counters): no barrier until every count of the channel is in
#pragma unroll 1
            for (; k < n_opts; k++)
                run_option<T, EPT, PROBE, kByte, false>(A, sm, k, par, bpw[k], sm.rb + A.opt_off[k],
                                                        (uint32_t)A.opt_words[k], cv, uv, nvalid, lnv, full,
                                                        any_slow, MGS_CODES(k));
            __syncthreads();
            finish_small<T, PROBE>(A, sm, bpw, par, nvalid, item);
            bool any_ovf = false;
#pragma unroll 1
            for (int j = A.n_small; j < n_opts; j++) {
                const BitParam &p = bpw[j];
                uint32_t *pout = PROBE ? A.hist_out + item * A.hist_stride + A.hist_off[A.opt_lo + j] : nullptr;
                if (p.path == kDegenerate) {
                    if (PROBE) probe_degenerate<T>(pout, 1 << p.b, nvalid);
                    continue;
                }
                if (flags[j] != 0u) {
                    any_ovf = true;
                    continue;
                }
                if (PROBE) probe_packed_clear<T>(sm.rb + A.opt_off[j], A.opt_words[j], 4, 0, 1 << p.b, pout);
                else clear_words<T>(sm.rb + A.opt_off[j], A.opt_words[j]);
            }
            if (any_ovf) {   // flags are read after the barrier: the same for every thread
#pragma unroll 1
                for (int j = A.n_small; j < n_opts; j++) {
                    const BitParam &p = bpw[j];
                    if (p.path == kDegenerate || flags[j] == 0u) continue;
                    __syncthreads();   // the other tables' readouts are done
                    recount_pairs<T, EPT, PROBE>(
                        A, sm, j, par, p, cv, uv, nvalid, p.path == kGeneric || any_slow,
                        PROBE ? A.hist_out + item * A.hist_stride + A.hist_off[A.opt_lo + j] : nullptr);
                }
            }
            k = n_opts;
        }
        // ---- larger bit-widths one at a time in region B (byte counters)
#pragma unroll 1
        for (; k < n_opts; k++) {
            const BitParam &p = bpw[k];
            const uint32_t wn = (uint32_t)A.opt_words[k];
            if (A.opt_windows[k] > 1)
                run_option<T, EPT, PROBE, kByte, true>(A, sm, k, par, p, sm.rb, wn, cv, uv, nvalid, lnv, full,
                                                       any_slow, MGS_CODES(k));
            else
                run_option<T, EPT, PROBE, kByte, false>(A, sm, k, par, p, sm.rb, wn, cv, uv, nvalid, lnv, full,
                                                        any_slow, MGS_CODES(k));
            __syncthreads();   // every count of this pass (and of region A) is in
            if (k == A.n_small) finish_small<T, PROBE>(A, sm, bpw, par, nvalid, item);
            if (p.path != kDegenerate) {
                const bool generic = p.path == kGeneric || any_slow;
                const int bins = 1 << p.b;
                uint32_t *pout = PROBE ? A.hist_out + item * A.hist_stride + A.hist_off[A.opt_lo + k] : nullptr;
                unsigned long long *hslot = sm.hpart + (par * n_opts + k) * NW + warp;
                HistPass h;
                h.base = (uint32_t)__cvta_generic_to_shared(sm.rb);
                h.dtab = A.dtab;
                h.dsm = (uint32_t)__cvta_generic_to_shared(sm.bdelta);
                h.lane_base = h.dbase = 0u;
                uint32_t dacc = 0, ovf = 0;
                if (flags[k] == 0u) {
                    // byte counters held: the first window is complete
                    if (PROBE) probe_packed_clear<T>(sm.rb, (int)wn, 4, 0, bins, pout);
                    else clear_words<T>(sm.rb, (int)wn);
                    if (A.opt_windows[k] > 1) {
#pragma unroll 1
                        for (int win = 1; win < A.opt_windows[k]; win++) {
                            __syncthreads();
                            h.wlo = (uint32_t)win * wn;
                            h.wn = wn;
                            h.boff = kMagicBits + 4u * h.wlo;
                            h.wn4 = wn * 4u;
                            count_window<T, EPT, kByte>(cv, uv, nvalid, generic, p, h, dacc, ovf);
                            __syncthreads();
                            if (PROBE) probe_packed_clear<T>(sm.rb, (int)wn, 4, (int64_t)win * wn * 4, bins, pout);
                            else clear_words<T>(sm.rb, (int)wn);
                        }
                        // a counter of a later window may have overflowed too
                        const uint32_t any = __syncthreads_or(ovf >= 0xFFu);
                        if (any) {
                            if (threadIdx.x == 0) flags[k] = 1u;
                        } else {
                            const unsigned long long hs = warp_sum_u64_redux((unsigned long long)dacc);
                            if (lane == 0) *hslot += hs;
                        }
                        dacc = 0;
                        __syncthreads();   // the flag of the later windows is visible
                    }
                    // one window: the flag was set by the evaluation pass, before the
                    // barrier after it, and nothing has written it since
                }
                if (flags[k] != 0u)   // some counter reached 255: count again exactly
                    recount_pairs<T, EPT, PROBE>(A, sm, k, par, p, cv, uv, nvalid, generic, pout);
            } else if (PROBE) {
                probe_degenerate<T>(A.hist_out + item * A.hist_stride + A.hist_off[A.opt_lo + k],
                                    1 << p.b, nvalid);
            }
            if (k + 1 < n_opts) __syncthreads();   // region B is clear for the next option
        }
#undef MGS_CODES
        if (A.n_small == n_opts && !A.concurrent) {
            __syncthreads();
            finish_small<T, PROBE>(A, sm, bpw, par, nvalid, item);
        }
        // every table is clear and every partial of this channel is in; one warp
        // reduces them while the others go on with the next channel (its partials
        // take the other buffers)
        __syncthreads();
        if (warp == w % NW) reduce_channel<T>(A, sm, S, par, item, cp.kexp, lnv);
        __syncwarp();   // converged again before the next channel's collectives
        par ^= 1;
        // the next channel takes the values of the following one (compile-time
        // register indices)
        if constexpr (!TM) {
#pragma unroll
            for (int ww = 0; ww + 1 < (TM ? 1 : W); ww++)
#pragma unroll
                for (int e = 0; e < EPT; e++) v[ww][e] = v[ww + 1][e];
        }
    }
}

template <int T, int EPT, int W, bool PROBE, int MINB, bool TM>
__global__ void __launch_bounds__(T, MINB)
    k_cost(const __grid_constant__ KernelArgs A, int unused) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n_opts = A.opt_hi - A.opt_lo;
    size_t o[10];
    smem_layout(T, W, A.a_words, A.b_words, n_opts, o);
    static_assert(EPT % 2 == 0, "elements are processed in pairs");
    static_assert(T >= 64, "partials are read by whole warps");
    Smem sm;
    sm.ra = reinterpret_cast<uint32_t *>(smem_raw + o[0]);
    sm.rb = reinterpret_cast<uint32_t *>(smem_raw + o[1]);
    sm.bdelta = reinterpret_cast<uint32_t *>(smem_raw + o[2]);
    sm.part2 = reinterpret_cast<float2 *>(smem_raw + o[3]);
    sm.hpart = reinterpret_cast<unsigned long long *>(smem_raw + o[4]);
    sm.plinf = reinterpret_cast<float *>(smem_raw + o[5]);
    sm.bp = reinterpret_cast<BitParam *>(smem_raw + o[6]);
    sm.ch = reinterpret_cast<ChanParam *>(smem_raw + o[7]);
    sm.mm = reinterpret_cast<float *>(smem_raw + o[8]);
    sm.flags = reinterpret_cast<uint32_t *>(smem_raw + o[9]);
    for (int i = threadIdx.x; i < A.a_words + A.b_words; i += T) sm.ra[i] = 0u;
    for (int i = threadIdx.x; i < kByteDelta; i += T) sm.bdelta[i] = i <= 256 ? __ldg(&A.dtab[i]) : 0u;
    for (int i = threadIdx.x; i < 2 * n_opts; i += T) sm.flags[i] = 0u;
    int par = 0;        // parity of the partials' buffers
    int seg_hint = -1;  // segment of the previous item
    // TMEM for the gathered tile: at most 512 / tm_cols CTAs share an SM (the
    // launch pads shared memory so), so the allocation never waits on another
    // CTA of this kernel
    constexpr int kCols = tm_cols(T, EPT, W);
    __shared__ uint32_t s_tmem;
    if (TM && (threadIdx.x >> 5) == 0) tm_alloc(&s_tmem, kCols);
    if (TM) tm_fence_before();
    __syncthreads();
    uint32_t tm = 0;
    if (TM) {
        tm_fence_after();
        const int warp = threadIdx.x >> 5;
        tm = s_tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * EPT * W);
    }
    if (A.counter == nullptr) {
        process_item<T, EPT, W, PROBE, TM>(A, sm, blockIdx.x, tm, par, seg_hint);
    } else {
        __shared__ int64_t s_work;
        while (true) {
            if (threadIdx.x == 0) s_work = (int64_t)atomicAdd(A.counter, 1u);
            __syncthreads();
            const int64_t work = s_work;
            if (work >= A.n_work) break;
            process_item<T, EPT, W, PROBE, TM>(A, sm, work, tm, par, seg_hint);
            __syncthreads();
        }
    }
    if (TM) {
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        if ((threadIdx.x >> 5) == 0) tm_dealloc(s_tmem, kCols);
    }
}

struct ConfigEntry {
    CostConfig cfg;
    void (*kernel)(KernelArgs, int);
    void (*probe)(KernelArgs, int);   // probe instantiation (or NULL)
    int ctas;                         // resident CTAs per SM the shared-memory plan aims at
    int tm_cols;                      // TMEM columns of a CTA (0: the tile stays in registers)
};

// {threads, elements per thread, channels per item, name}, the kernel, its
// probe instantiation, the CTAs per SM that its registers (launch bounds) and
// shared-memory plan aim at, and its TMEM columns ("tm" shapes keep the whole
// slab's tile in tensor memory).
#define MGS_NAME(T, E, W, C, X) "t" #T "_e" #E "_w" #W "_c" #C X
#define MGS_CFG(T, E, W, C) \
    {{T, E, W, MGS_NAME(T, E, W, C, "")}, k_cost<T, E, W, false, C, false>, nullptr, C, 0}
#define MGS_CFGP(T, E, W, C) \
    {{T, E, W, MGS_NAME(T, E, W, C, "")}, k_cost<T, E, W, false, C, false>, k_cost<T, E, W, true, C, false>, C, 0}
#define MGS_CFGT(T, E, C)                                                                   \
    {{T, E, 8, MGS_NAME(T, E, 8, C, "_tm")}, k_cost<T, E, 8, false, C, true>, k_cost<T, E, 8, true, C, true>, C, \
     tm_cols(T, E, 8)}
const ConfigEntry kConfigs[] = {
    MGS_CFGP(256, 16, 4, 2),
    MGS_CFG(512, 8, 4, 1),
    MGS_CFG(256, 16, 2, 2),
    MGS_CFGP(256, 8, 4, 2),
    MGS_CFG(128, 8, 8, 4),
    MGS_CFGP(256, 4, 8, 2),
    MGS_CFGP(512, 32, 1, 1),
    MGS_CFG(256, 16, 1, 2),
    MGS_CFG(256, 16, 1, 3),
    MGS_CFGT(256, 16, 2),
    MGS_CFGT(256, 8, 2),
    MGS_CFGT(128, 8, 4),
};
#undef MGS_CFG
#undef MGS_CFGP
#undef MGS_CFGT
#undef MGS_NAME
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

// Histogram plan of a launch: region A holds a table per option up to 12 bits
// (lane columns, direct counters or 16-bit pairs), region B the byte counters
// of one larger option at a time, in windows when region B is smaller than the
// option's table.
struct HistPlan {
    int n_small = 0, n_lane = 0, n_direct = 0, a_words = 0, b_words = 0;
    bool concurrent = false;
    int n_units = 0;
    int16_t unit_opt[MGS_MAX_OPTIONS] = {}, unit_lo[MGS_MAX_OPTIONS] = {}, unit_hi[MGS_MAX_OPTIONS] = {};
    int8_t mode[MGS_MAX_OPTIONS] = {}, windows[MGS_MAX_OPTIONS] = {}, rwindows[MGS_MAX_OPTIONS] = {};
    int32_t off[MGS_MAX_OPTIONS] = {}, words[MGS_MAX_OPTIONS] = {};
    size_t smem = 0;
};

// Shared memory a CTA may use when `ctas` of them share an SM (228 KB per SM,
// 1 KB reserved per CTA, and up to 512 bytes of the kernel's static variables).
size_t smem_budget(int ctas) { return std::min<size_t>(227 * 1024 - 512, (228 * 1024) / ctas - 1024 - 512); }

// One layout: options up to `pair_max` bits take region A (lane columns, direct
// counters, 16-bit pairs), larger ones byte counters in region B, either each
// in its own table (concurrent) or one after another in the largest window that
// fits (sequential).
HistPlan plan_layout(const ConfigEntry &E, const int *bl, int n_opts, int pair_max, bool concurrent) {
    const CostConfig &c = E.cfg;
    HistPlan h;
    h.concurrent = concurrent;
    const int NW = c.threads / 32;
    int large_words = 0;
    for (int k = 0; k < n_opts; k++) {
        const int b = bl[k];
        int mode, words;
        if (b <= kLaneMaxBits && (1 << b) <= 32 * NW) {
            mode = kLane;
            words = 32 << b;
        } else if (b <= kDirectMaxBits) {
            mode = kDirect;
            words = 1 << b;
        } else if (b <= pair_max) {
            mode = kPair;
            words = 1 << (b - 1);
        } else {
            mode = kByte;
            words = std::max(4, 1 << (b - 2));
        }
        words = (words + 3) & ~3;
        h.mode[k] = (int8_t)mode;
        if (mode == kLane) h.n_lane++;
        if (mode == kDirect) h.n_direct++;
        h.words[k] = words;
        if (mode != kByte) {
            // bit-widths ascend, so the small options form a prefix (lane, direct, pair)
            h.off[k] = h.a_words;
            h.a_words += words;
            h.n_small = k + 1;
        } else if (concurrent) {
            h.off[k] = h.b_words;
            h.b_words += words;
        } else {
            large_words = std::max(large_words, words);
        }
    }
    size_t o[10];
    if (!concurrent) {
        const size_t fixed = smem_layout(c.threads, c.width, h.a_words, 0, n_opts, o);
        const size_t budget = smem_budget(E.ctas);
        int bw = large_words;
        if (bw > 0) {
            // region B: the largest table that fits, in whole power-of-two windows
            int cap = budget > fixed ? (int)((budget - fixed) / 4) : 0;
            while (bw > cap && bw > 1024) bw >>= 1;
            bw = std::max(bw, 1024);
        }
        h.b_words = bw;
    }
    for (int k = h.n_small; k < n_opts; k++) {
        const int b = bl[k];
        const int need = std::max(4, 1 << (b - 2)), need_pairs = 1 << (b - 1);
        if (!concurrent) h.words[k] = std::min(need, h.b_words);
        h.windows[k] = (int8_t)(concurrent ? 1 : (need + h.b_words - 1) / h.b_words);
        h.rwindows[k] = (int8_t)((need_pairs + h.b_words - 1) / h.b_words);
    }
    h.smem = smem_layout(c.threads, c.width, h.a_words, h.b_words, n_opts, o);
    // finishing units of region A: one per small option, then the costliest
    // split in two (at a multiple of 32 bins, 64 for 16-bit pairs) until every
    // warp has one; cost = the lanes' steps x the work of a step
    auto cost = [&](int u) {
        const int m = h.mode[h.unit_opt[u]], n = h.unit_hi[u] - h.unit_lo[u];
        return m == kLane ? (n + 31) / 32 * 24 : m == kDirect ? (n + 31) / 32 * 4 : (n / 2 + 31) / 32;
    };
    for (int k = 0; k < h.n_small; k++) {
        h.unit_opt[h.n_units] = (int16_t)k;
        h.unit_lo[h.n_units] = 0;
        h.unit_hi[h.n_units] = (int16_t)std::min(1 << bl[k], 32767);
        h.n_units++;
    }
    while (h.n_units < NW && h.n_units < MGS_MAX_OPTIONS) {
        int best = -1;
        for (int u = 0; u < h.n_units; u++) {
            const int step = h.mode[h.unit_opt[u]] == kPair ? 64 : 32;
            if (h.unit_hi[u] - h.unit_lo[u] >= 2 * step && (best < 0 || cost(u) > cost(best))) best = u;
        }
        if (best < 0) break;
        const int step = h.mode[h.unit_opt[best]] == kPair ? 64 : 32;
        const int lo = h.unit_lo[best], hi = h.unit_hi[best];
        const int mid = lo + (hi - lo) / 2 / step * step;
        h.unit_opt[h.n_units] = h.unit_opt[best];
        h.unit_lo[h.n_units] = (int16_t)mid;
        h.unit_hi[h.n_units] = (int16_t)hi;
        h.unit_hi[best] = (int16_t)mid;
        h.n_units++;
    }
    return h;
}

// The plan of a launch: every large option in its own table if that fits the
// shared memory of `ctas` CTAs per SM (first with 11 and 12 bits as 16-bit
// pairs in region A, then as byte counters in region B), else one large option
// after another.
HistPlan plan_hist(const ConfigEntry &E, const int32_t *bits, int n_opts) {
    int bl[MGS_MAX_OPTIONS];
    for (int k = 0; k < n_opts; k++) bl[k] = bits ? bits[k] : MGS_MAX_BITS - n_opts + 1 + k;
    const size_t budget = smem_budget(E.ctas);
    for (int pair_max : {kPairMaxBits, kDirectMaxBits}) {
        const HistPlan h = plan_layout(E, bl, n_opts, pair_max, true);
        if (h.smem <= budget) return h;
    }
    return plan_layout(E, bl, n_opts, kPairMaxBits, false);
}

}  // namespace

int cost_config_count() { return kNumConfigs; }
const CostConfig &cost_config(int i) { return kConfigs[i].cfg; }

int cost_default_config(int G) {
    if (G <= 1024) return 11;   // 128 x 8, slab tile in TMEM
    if (G <= 2048) return 10;   // 256 x 8, slab tile in TMEM
    if (G <= 4096) return 9;    // 256 x 16, slab tile in TMEM
    if (G <= 16384) return 6;   // 512 x 32, W 1
    return -1;
}

int cost_plan_export(int config, const int32_t *bits, int n_opts, int32_t *out, int cap) {
    if (config < 0 || config >= kNumConfigs || n_opts < 1 || n_opts > MGS_MAX_OPTIONS || !bits) return -1;
    const HistPlan h = plan_hist(kConfigs[config], bits, n_opts);
    std::vector<int32_t> v = {(int32_t)h.smem, (int32_t)smem_budget(kConfigs[config].ctas), h.concurrent ? 1 : 0,
                              h.a_words, h.b_words, h.n_small, h.n_lane, h.n_direct, h.n_units};
    for (int k = 0; k < n_opts; k++) {
        v.push_back(h.mode[k]);
        v.push_back(h.off[k]);
        v.push_back(h.words[k]);
        v.push_back(h.windows[k]);
        v.push_back(h.rwindows[k]);
    }
    for (int u = 0; u < h.n_units; u++) {
        v.push_back(h.unit_opt[u]);
        v.push_back(h.unit_lo[u]);
        v.push_back(h.unit_hi[u]);
    }
    if (out && cap > 0) std::memcpy(out, v.data(), sizeof(int32_t) * std::min<size_t>(v.size(), (size_t)cap));
    return (int)v.size();
}

bool cost_config_has_probe(int config) {
    return config >= 0 && config < kNumConfigs && kConfigs[config].probe != nullptr;
}

size_t cost_smem_bytes(int config, int G, int n_opts, const int32_t *bits) {
    (void)G;
    return plan_hist(kConfigs[config], bits, n_opts).smem;
}

struct CostExec {
    const ConfigEntry *entry = nullptr;
    void (*kernel)(KernelArgs, int) = nullptr;
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
    const bool probe = L.probe_hist != nullptr || L.probe_codes != nullptr;
    if (probe && !E.probe) {
        set_error("tile %s has no probe kernel", E.cfg.name);
        return MGS_ERR_INVALID_ARG;
    }
    // Work order.  The ratios of one scene read the same slab rows (their kept
    // sets are nested and Morton-ordered, so group g of a ratio with n_g groups
    // covers about the fraction [g / n_g, (g + 1) / n_g) of the scene).  The
    // segments of each scene (consecutive segments over the same slabs) are
    // cut into B Morton-range buckets, bucket t of a segment being its groups
    // [g_count t / B, g_count (t + 1) / B), and the launch takes bucket 0 of
    // every segment, then bucket 1, ...: the rows a bucket reads stay in L2
    // while all ratios use them (DRAM traffic falls to about a fifth of the
    // bytes the items read).  B gives a bucket a few waves of CTAs; results do
    // not depend on the order.
    std::vector<CostSeg> in = L.segs;
    for (auto &s : in) {
        s.n_chunks = (s.C + E.cfg.width - 1) / E.cfg.width;
        if (s.g_count <= 0) {
            s.g_first = 0;
            s.g_count = s.n_groups;
        }
    }
    segs->clear();
    const int64_t wave = (int64_t)std::max(ctx->sm_count, 1) * E.ctas;
    for (size_t a = 0; a < in.size();) {
        size_t b = a + 1;
        while (b < in.size() && in[b].slabs == in[a].slabs && in[b].n == in[a].n) b++;
        int64_t items = 0;
        int32_t max_groups = 1;
        for (size_t i = a; i < b; i++) {
            items += (int64_t)in[i].g_count * in[i].n_chunks;
            max_groups = std::max(max_groups, in[i].g_count);
        }
        const int64_t nb = std::min<int64_t>({(int64_t)kMaxSpatialBuckets, (int64_t)max_groups,
                                              std::max<int64_t>(1, (items + 4 * wave - 1) / (4 * wave))});
        for (int64_t t = 0; t < nb; t++) {
            for (size_t i = a; i < b; i++) {
                CostSeg s = in[i];
                const int64_t lo = (int64_t)in[i].g_count * t / nb, hi = (int64_t)in[i].g_count * (t + 1) / nb;
                if (hi <= lo) continue;
                s.g_first = in[i].g_first + (int32_t)lo;
                s.g_count = (int32_t)(hi - lo);
                segs->push_back(s);
            }
        }
        a = b;
    }
    int64_t n_work = 0;
    for (auto &s : *segs) {
        s.work_begin = n_work;
        n_work += (int64_t)s.g_count * s.n_chunks;
    }
    CostExec *X = new CostExec();
    X->entry = &E;
    X->kernel = probe ? E.probe : E.kernel;
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
    const int n_opts = L.opt_hi - L.opt_lo;
    const HistPlan hp = plan_hist(E, L.bits + L.opt_lo, n_opts);
    A.n_small = hp.n_small;
    A.n_lane = hp.n_lane;
    A.n_direct = hp.n_direct;
    A.concurrent = hp.concurrent ? 1 : 0;
    A.n_units = hp.n_units;
    for (int u = 0; u < hp.n_units; u++) {
        A.unit_opt[u] = hp.unit_opt[u];
        A.unit_lo[u] = hp.unit_lo[u];
        A.unit_hi[u] = hp.unit_hi[u];
    }
    A.a_words = hp.a_words;
    A.b_words = hp.b_words;
    for (int k = 0; k < n_opts; k++) {
        A.opt_mode[k] = hp.mode[k];
        A.opt_windows[k] = hp.windows[k];
        A.opt_rwindows[k] = hp.rwindows[k];
        A.opt_off[k] = hp.off[k];
        A.opt_words[k] = hp.words[k];
    }
    A.hist_out = L.probe_hist;
    A.codes_out = L.probe_codes;
    int64_t hs = 0;
    for (int k = 0; k < L.n_bits; k++) {
        A.hist_off[k] = hs;
        hs += (int64_t)1 << L.bits[k];
    }
    A.hist_stride = hs;
    X->smem = hp.smem;
    X->persistent = L.persistent;
    if (X->smem > 227 * 1024) {
        set_error("tile %s needs %zu bytes of shared memory for G=%d and %d options", E.cfg.name,
                  X->smem, L.group_size, n_opts);
        delete X;
        return MGS_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSuccess;
    if (E.tm_cols > 0) {
        // at most 512 / tm_cols CTAs of this kernel per SM, so tcgen05.alloc never waits
        // on a CTA of the same kernel: pad the shared memory until occupancy says so
        const int max_ctas = 512 / E.tm_cols;
        int optin = 0;
        cudaFuncAttributes fa{};
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, X->kernel);
        const size_t limit = e == cudaSuccess ? (size_t)optin - fa.sharedSizeBytes : 0;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(X->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
        for (; e == cudaSuccess;) {
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, X->kernel, E.cfg.threads, X->smem);
            if (e != cudaSuccess || per_sm <= max_ctas || X->smem + 1024 > limit) break;
            X->smem += 1024;
        }
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(X->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X->smem);
    X->grid = n_work;
    if (e == cudaSuccess && L.persistent) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, X->kernel, E.cfg.threads, X->smem);
        // the occupancy calculator reports one CTA per SM for any kernel that
        // allocates tensor memory (it cannot know how many columns a CTA takes);
        // these CTAs take tm_cols each and their registers and shared memory are
        // planned for `ctas` per SM.  Surplus CTAs of a persistent launch only find
        // the work counter exhausted.
        if (E.tm_cols > 0) per_sm = std::max(per_sm, std::min(E.ctas, 512 / E.tm_cols));
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
    X->kernel<<<(unsigned)X->grid, X->entry->cfg.threads, X->smem, st>>>(X->args, 0);
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
