// Block coder of one chosen configuration: the actual compressed size S_a of
// Alg. 1 ("compress the model with the current hyperparameters, obtain its
// size") and the entropy coding of Sec. III-G, with this library's own block
// format (static-model rANS with a raw fallback; the format is written out in
// include/mgs.h above mgs_encode_config).
//
// Pipeline (all on `stream`): kept list -> quantise (quantize.cu) ->
//   k_enc_model, one CTA per (channel, group) block: count the codes in windows
//     of 4096 (16 windows at b = 16, empty ones skipped), list the distinct
//     codes in ascending order, normalise the counts to M = 2^ceil(log2 n), lay
//     out the gamma-coded table by a block-wide scan of its bit lengths and
//     write it into the block's slot, and store (f << 16 | cum) for every code;
//   k_enc_rans, one sub-group of lanes per block (four 4096-code blocks per
//     warp): the interleaved rANS encoder (lane j owns
//     symbols i = j mod lanes; the bytes a step emits are ordered by two
//     ballots), which needs no shared memory, so many blocks are in flight;
//   block sizes -> exclusive scan -> k_enc_gather, which writes each block at
//     its offset (raw blocks bit-packed from the codes, rANS bytes reversed
//     into decoding order); skipped when only the size is wanted.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace mgs {
namespace {

constexpr int kEncThreads = 128;
constexpr int kEncWarps = kEncThreads / 32;
constexpr uint32_t kRansL = 1u << 23;   // states live in [L, 2^31)
constexpr int kWin = 4096;              // histogram window (codes)
constexpr int kScanChunk = 1024;        // sizes per CTA of the scan

__host__ __device__ inline int64_t a16(int64_t x) { return (x + 15) & ~(int64_t)15; }

// Shared-memory layout of k_enc_model for group size G.
struct EncSmem {
    int64_t hist, sym, f, cum, tab, total;
    __host__ __device__ explicit EncSmem(int G) {
        // uint16[kWin] counts as 16-bit pairs in 32-bit words (a count is at most
        // G <= 16384), then the code -> entry map; once the map has been read,
        // the same bytes hold the table's bits (uint32 words, < 2G + 16 bytes)
        hist = 0;
        tab = 0;
        const int64_t shared_bytes = 2 * (int64_t)G + 16 > 2 * kWin ? 2 * (int64_t)G + 16 : 2 * kWin;
        sym = a16(shared_bytes);              // uint16[G]: distinct codes, ascending
        f = sym + a16(2 * (int64_t)G);        // uint16[G]: normalised frequencies (counts first)
        cum = f + a16(2 * (int64_t)G);        // uint16[G]
        total = cum + a16(2 * (int64_t)G);
    }
};

__device__ __forceinline__ int glen(uint32_t x) { return 2 * (31 - __clz(x)) + 1; }

// Exclusive scan over the CTA of one 64-bit value per thread; *total gets the sum.
__device__ uint64_t block_excl_scan(uint64_t v, uint64_t *total, uint64_t *s_warp) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    uint64_t base = 0, all = 0;
    for (int k = 0; k < kEncWarps; k++) {
        if (k < w) base += s_warp[k];
        all += s_warp[k];
    }
    __syncthreads();
    *total = all;
    return base + inc - v;
}

// Writes gamma(x) at bit p of the zeroed word buffer (LSB-first bit order).
__device__ __forceinline__ void put_gamma(uint32_t *tab, int64_t p, uint32_t x) {
    const int N = 31 - __clz(x);
    p += N;   // N zero bits
    for (int u = 0; u <= N; u++, p++)
        if ((x >> (N - u)) & 1u) atomicOr(&tab[p >> 5], 1u << (p & 31));
}

// What k_enc_model leaves for the rANS and gather kernels, per block.
struct EncInfo {
    int32_t lanes;       // interleaved rANS states; 0: no rANS attempt (R = 0, or raw is shorter)
    int32_t k;           // log2 M
    int32_t tab_bytes;   // the gamma table, zero-padded to a byte
    int32_t e_cap;       // rANS is used iff its renormalisation byte count E < e_cap
    int32_t E;           // min(E, e_cap), from k_enc_rans
    int32_t pad_;
};

// Block geometry shared by the three kernels.
struct EncBlock {
    int c, g, n;
    int64_t start;
};
__device__ __forceinline__ EncBlock enc_block(int64_t blk, int64_t K, int32_t G, int32_t ng) {
    EncBlock B;
    B.c = (int)(blk / ng);
    B.g = (int)(blk % ng);
    B.start = (int64_t)B.g * G;
    B.n = (int)((K - B.start) < (int64_t)G ? (K - B.start) : (int64_t)G);
    return B;
}

// One CTA per (channel, group) block: metadata, the distinct codes and their
// normalised frequencies, the gamma table in the block's slot, and the packed
// (f << 16 | cum) of every code for the rANS kernel.
__global__ void __launch_bounds__(kEncThreads)
    k_enc_model(const uint16_t *__restrict__ codes, int64_t K, int32_t G, int32_t ng,
                const uint8_t *__restrict__ bits, const float *__restrict__ minmax,
                uint8_t *__restrict__ slots, int64_t slot_bytes, EncInfo *__restrict__ info,
                uint32_t *__restrict__ fcpos, int32_t *__restrict__ sizes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t s_warp[kEncWarps];
    __shared__ uint32_t s_wcnt[16];
    __shared__ int s_D;
    __shared__ uint32_t s_top;

    const EncSmem L(G);
    uint32_t *s_hw = reinterpret_cast<uint32_t *>(smem + L.hist);   // counter pairs
    uint16_t *s_hist = reinterpret_cast<uint16_t *>(smem + L.hist);
    uint16_t *s_sym = reinterpret_cast<uint16_t *>(smem + L.sym);
    uint16_t *s_f = reinterpret_cast<uint16_t *>(smem + L.f);
    uint16_t *s_cum = reinterpret_cast<uint16_t *>(smem + L.cum);
    uint32_t *s_tab = reinterpret_cast<uint32_t *>(smem + L.tab);

    const int64_t blk = blockIdx.x;
    const EncBlock B = enc_block(blk, K, G, ng);
    const int n = B.n;
    const int b = bits[blk];
    const float mn = minmax[2 * blk], mx = minmax[2 * blk + 1];
    uint8_t *out = slots + blk * slot_bytes;
    const int t = threadIdx.x;
    const uint16_t *src = codes + (int64_t)B.c * K + B.start;

    if (t < 9) {
        uint32_t v = t == 0 ? (uint32_t)b : __float_as_uint(t < 5 ? mn : mx) >> (8 * ((t - 1) & 3));
        out[t] = (uint8_t)v;
    }
    const int64_t raw_payload = 1 + ((int64_t)n * b + 7) / 8;
    if (__fsub_rn(mx, mn) == 0.0f) {   // R = 0: every code is 0, metadata only
        if (t == 0) {
            sizes[blk] = 9;
            info[blk] = EncInfo{0, 0, 0, 0, 0, 0};
        }
        return;
    }

    // ---- per-window counts when b > 12 ----
    const int logW = b < 12 ? b : 12;
    const int W = 1 << logW;
    const int nwin = 1 << (b - logW);
    if (t < 16) s_wcnt[t] = 0;
    if (t == 0) s_D = 0;
    __syncthreads();
    if (nwin > 1)
        for (int i = t; i < n; i += kEncThreads) atomicAdd(&s_wcnt[src[i] >> 12], 1u);
    __syncthreads();

    // ---- distinct codes (ascending) with their counts ----
    const int per = (W + kEncThreads - 1) / kEncThreads;
    for (int w = 0; w < nwin; w++) {
        if (nwin > 1 && s_wcnt[w] == 0) continue;   // uniform: s_wcnt is settled
        for (int i = t; i < W / 2; i += kEncThreads) s_hw[i] = 0;   // W >= 2
        __syncthreads();
        for (int i = t; i < n; i += kEncThreads) {
            uint32_t q = src[i];
            const uint32_t c = q & (W - 1);
            if ((int)(q >> logW) == w) atomicAdd(&s_hw[c >> 1], 1u << (16 * (c & 1)));
        }
        __syncthreads();
        const int lo = t * per, hi = min(W, lo + per);
        uint32_t mine = 0;
        for (int i = lo; i < hi; i++) mine += s_hist[i] != 0;
        uint64_t tot;
        uint64_t at = (uint64_t)s_D + block_excl_scan(mine, &tot, s_warp);
        for (int i = lo; i < hi; i++) {
            uint32_t h = s_hist[i];
            if (h) {
                s_sym[at] = (uint16_t)((w << logW) + i);
                s_f[at] = (uint16_t)h;   // count for now
                if (nwin == 1) s_hist[i] = (uint16_t)at;   // code -> entry map
                at++;
            }
        }
        __syncthreads();
        if (t == 0) s_D += (int)tot;
        __syncthreads();
    }
    const int D = s_D;

    // ---- normalised frequencies: floor(cnt M / n), shortfall to the most frequent ----
    const int k = 32 - __clz((unsigned)(n - 1));   // ceil(log2 n); n >= 2 here
    const uint32_t M = 1u << k;
    uint64_t fsum = 0;
    uint32_t best = 0;   // (count << 16) | (65535 - entry): max = most frequent, lowest code
    for (int e = t; e < D; e += kEncThreads) {
        uint32_t cnt = s_f[e];
        uint32_t fv = (uint32_t)(((uint64_t)cnt * M) / (uint32_t)n);
        fsum += fv;
        best = max(best, (cnt << 16) | (uint32_t)(65535 - e));
        s_f[e] = (uint16_t)fv;
    }
    if (t == 0) s_top = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) {
        fsum += __shfl_xor_sync(0xFFFFFFFFu, fsum, o);
        best = max(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
    }
    if ((t & 31) == 0) {
        s_warp[t >> 5] = fsum;
        atomicMax(&s_top, best);
    }
    __syncthreads();
    if (t == 0) {
        uint64_t all = 0;
        for (int w = 0; w < kEncWarps; w++) all += s_warp[w];
        const int top = 65535 - (int)(s_top & 0xFFFFu);
        s_f[top] = (uint16_t)(s_f[top] + (uint32_t)(M - all));
    }
    __syncthreads();

    // ---- cumulative frequencies and table bit offsets (one chunk of entries per thread) ----
    const int eper = (D + kEncThreads - 1) / kEncThreads;
    const int e0 = min(D, t * eper), e1 = min(D, e0 + eper);
    uint32_t fl = 0, bl = 0;
    for (int e = e0; e < e1; e++) {
        uint32_t gap = e == 0 ? (uint32_t)s_sym[0] + 1u : (uint32_t)(s_sym[e] - s_sym[e - 1]);
        fl += s_f[e];
        bl += glen(gap) + glen(s_f[e]);
    }
    uint64_t tot2;
    const uint64_t pre = block_excl_scan(((uint64_t)fl << 32) | bl, &tot2, s_warp);
    const int64_t tbits = glen((uint32_t)D) + (int64_t)(tot2 & 0xFFFFFFFFu);
    {
        uint32_t run = (uint32_t)(pre >> 32);
        for (int e = e0; e < e1; e++) {
            s_cum[e] = (uint16_t)run;
            run += s_f[e];
        }
    }

    // ---- can rANS beat the raw payload at all? ----
    const int lanes = min(32, max(1, n >> 9));
    const int64_t tab_bytes = (tbits + 7) / 8;
    const int64_t e_cap = raw_payload - 1 - tab_bytes - 4 * (int64_t)lanes;   // rANS iff E < e_cap
    if (e_cap <= 0) {
        if (t == 0) {
            sizes[blk] = (int32_t)(9 + raw_payload);
            info[blk] = EncInfo{0, k, 0, 0, 0, 0};
        }
        return;
    }
    __syncthreads();   // s_cum complete

    // ---- (f, cum) of every code, and the table in the slot ----
    uint32_t *fc = fcpos + (int64_t)B.c * K + B.start;
    for (int i = t; i < n; i += kEncThreads) {
        const uint32_t q = src[i];
        int e;
        if (nwin == 1) {
            e = (int)s_hist[q];
        } else {
            int lo = 0, hi = D - 1;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (s_sym[mid] < q) lo = mid + 1;
                else hi = mid;
            }
            e = lo;
        }
        fc[i] = ((uint32_t)s_f[e] << 16) | (uint32_t)s_cum[e];
    }
    __syncthreads();   // the map is read: its bytes now hold the table
    const int64_t words = (tab_bytes + 3) / 4;
    for (int64_t q = t; q < words; q += kEncThreads) s_tab[q] = 0;
    __syncthreads();
    if (t == 0) put_gamma(s_tab, 0, (uint32_t)D);
    int64_t p = glen((uint32_t)D) + (int64_t)(pre & 0xFFFFFFFFu);
    for (int e = e0; e < e1; e++) {
        uint32_t gap = e == 0 ? (uint32_t)s_sym[0] + 1u : (uint32_t)(s_sym[e] - s_sym[e - 1]);
        put_gamma(s_tab, p, gap);
        p += glen(gap);
        put_gamma(s_tab, p, s_f[e]);
        p += glen(s_f[e]);
    }
    __syncthreads();
    const uint8_t *tb = reinterpret_cast<const uint8_t *>(s_tab);
    for (int64_t q = t; q < tab_bytes; q += kEncThreads) out[10 + q] = tb[q];
    if (t == 0) info[blk] = EncInfo{lanes, k, (int32_t)tab_bytes, (int32_t)e_cap, 0, 0};
}

// The interleaved rANS encoder, last symbol first, one sub-group of GW lanes
// per block (GW = 32 / blocks per warp, at least the block's lane count; a
// 4096-code block has 8 lanes, so four blocks share a warp).  Lane j of a
// block owns its symbols i = j (mod lanes); each step emits 0-2 bytes per
// lane, placed by the sub-group's slices of two warp ballots in emission order
// (higher lanes first within a step); the bytes go into the slot after the
// table and the states, and the gather kernel writes them out in reverse,
// which is decoding order.
template <int GW>
__global__ void __launch_bounds__(kEncThreads)
    k_enc_rans(const uint32_t *__restrict__ fcpos, int64_t K, int32_t G, int32_t ng, int64_t m,
               const uint8_t *__restrict__ bits, uint8_t *__restrict__ slots, int64_t slot_bytes,
               EncInfo *__restrict__ info, int32_t *__restrict__ sizes) {
    constexpr int PER_WARP = 32 / GW;
    const int lane = threadIdx.x & 31;
    const int sub = lane / GW, j = lane % GW;
    const int64_t blk = ((int64_t)blockIdx.x * kEncWarps + (threadIdx.x >> 5)) * PER_WARP + sub;
    const bool have = blk < m;
    EncInfo I = {0, 0, 0, 0, 0, 0};
    if (have) I = info[blk];
    const bool live = have && I.lanes > 0;
    int n = 0;
    int64_t cstart = 0;
    if (live) {
        const EncBlock B = enc_block(blk, K, G, ng);
        n = B.n;
        cstart = (int64_t)B.c * K + B.start;
    }
    const int lanes = live ? I.lanes : 1, k = I.k;
    const uint32_t M = 1u << k;
    const uint32_t *fc = fcpos + cstart;
    uint8_t *out = live ? slots + blk * slot_bytes + 10 + I.tab_bytes : nullptr;
    uint8_t *em = live ? out + 4 * lanes : nullptr;
    const int64_t e_cap = I.e_cap;
    uint32_t x = kRansL;
    int64_t base = 0;
    const uint32_t gmask = GW == 32 ? 0xFFFFFFFFu : ((1u << GW) - 1u);
    const uint32_t above = ~((2u << j) - 1u) & gmask;   // lanes of this sub-group above j
    const uint32_t xunit = live ? 1u << (31 - k) : 0u;   // (L >> k) << 8
    const int steps = live ? (n + lanes - 1) / lanes : 0;
    int max_steps = steps;   // the warp runs as long as its longest block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) max_steps = max(max_steps, __shfl_xor_sync(0xFFFFFFFFu, max_steps, o));
    for (int st = max_steps - 1; st >= 0; st--) {
        const int i = st * lanes + j;
        int cnt = 0;
        uint32_t b1 = 0, b2 = 0;
        if (live && st < steps && j < lanes && i < n) {
            const uint32_t w = fc[i];
            const uint32_t fs = w >> 16, cs = w & 0xFFFFu;
            const uint64_t xmax = (uint64_t)xunit * fs;
            if (x >= xmax) {
                b1 = x & 0xFFu;
                x >>= 8;
                cnt = 1;
                if (x >= xmax) {
                    b2 = x & 0xFFu;
                    x >>= 8;
                    cnt = 2;
                }
            }
            x = (x / fs) * M + x % fs + cs;
        }
        const uint32_t m1 = (__ballot_sync(0xFFFFFFFFu, cnt >= 1) >> (sub * GW)) & gmask;
        const uint32_t m2 = (__ballot_sync(0xFFFFFFFFu, cnt == 2) >> (sub * GW)) & gmask;
        const int64_t idx = base + __popc(m1 & above) + __popc(m2 & above);
        if (cnt >= 1 && idx < e_cap) em[idx] = (uint8_t)b1;
        if (cnt == 2 && idx + 1 < e_cap) em[idx + 1] = (uint8_t)b2;
        base += __popc(m1) + __popc(m2);
    }
    if (live && j < lanes)
        for (int q = 0; q < 4; q++) out[4 * j + q] = (uint8_t)(x >> (8 * q));
    if (live && j == 0) {
        const int64_t E = base < e_cap ? base : e_cap;
        info[blk].E = (int32_t)E;
        sizes[blk] = E < e_cap ? (int32_t)(10 + I.tab_bytes + 4 * lanes + E)
                               : (int32_t)(10 + ((int64_t)n * bits[blk] + 7) / 8);
    }
}

// Exclusive scan of int32 sizes into int64 offsets: per-chunk sums, one CTA
// over the chunk sums, then the per-chunk scan with its base.
__global__ void __launch_bounds__(1024)
    k_enc_chunk_sums(const int32_t *__restrict__ sizes, int64_t m, int64_t *__restrict__ sums) {
    __shared__ int64_t s[32];
    const int64_t i = (int64_t)blockIdx.x * kScanChunk + threadIdx.x;
    int64_t v = i < m ? sizes[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t a = 0;
        for (int w = 0; w < 32; w++) a += s[w];
        sums[blockIdx.x] = a;
    }
}

__global__ void __launch_bounds__(1024)
    k_enc_scan_sums(int64_t *__restrict__ sums, int64_t nchunks, int64_t *__restrict__ total) {
    __shared__ int64_t s[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nchunks; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nchunks ? sums[i] : 0;
        int64_t inc = v;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s[w] = inc;
        __syncthreads();
        int64_t wb = 0, all = 0;
        for (int k = 0; k < 32; k++) {
            if (k < w) wb += s[k];
            all += s[k];
        }
        if (i < nchunks) sums[i] = carry + wb + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(1024)
    k_enc_offsets(const int32_t *__restrict__ sizes, int64_t m, const int64_t *__restrict__ sums,
                  int64_t *__restrict__ off) {
    __shared__ int64_t s[32];
    const int64_t i = (int64_t)blockIdx.x * kScanChunk + threadIdx.x;
    const int64_t v = i < m ? sizes[i] : 0;
    int64_t inc = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s[w] = inc;
    __syncthreads();
    int64_t wb = 0;
    for (int k = 0; k < w; k++) wb += s[k];
    if (i < m) off[i] = sums[blockIdx.x] + wb + inc - v;
}

// Writes each block at its offset: the metadata, then either the rANS
// payload (mode, table and states as they are in the slot, the
// renormalisation bytes reversed into decoding order) or the raw payload,
// bit-packed from the codes.
__global__ void __launch_bounds__(256)
    k_enc_gather(const uint16_t *__restrict__ codes, int64_t K, int32_t G, int32_t ng,
                 const uint8_t *__restrict__ bits, const uint8_t *__restrict__ slots,
                 int64_t slot_bytes, const EncInfo *__restrict__ info,
                 const int32_t *__restrict__ sizes, const int64_t *__restrict__ off,
                 uint8_t *__restrict__ stream) {
    const int64_t blk = blockIdx.x;
    const uint8_t *src = slots + blk * slot_bytes;
    uint8_t *dst = stream + off[blk];
    const int sz = sizes[blk];
    const int t = threadIdx.x;
    if (t < 9) dst[t] = src[t];
    if (sz == 9) return;
    const EncInfo I = info[blk];
    if (I.lanes > 0 && I.E < I.e_cap) {
        if (t == 0) dst[9] = 1;
        const int head = I.tab_bytes + 4 * I.lanes;
        for (int q = t; q < head; q += 256) dst[10 + q] = src[10 + q];
        const int E = I.E;
        for (int q = t; q < E; q += 256) dst[10 + head + q] = src[10 + head + E - 1 - q];
        return;
    }
    if (t == 0) dst[9] = 0;
    const EncBlock B = enc_block(blk, K, G, ng);
    const int n = B.n, b = bits[blk];
    const uint16_t *cs = codes + (int64_t)B.c * K + B.start;
    // 32 stream bits per step: the codes overlapping bits [32 wq, 32 wq + 32)
    const int nb = (int)(((int64_t)n * b + 7) / 8);
    const int nwords = (nb + 3) / 4;
    for (int wq = t; wq < nwords; wq += 256) {
        const int lo = 32 * wq;
        const int i0 = lo / b, i1 = min(n - 1, (lo + 31) / b);
        uint64_t v = 0;
        for (int i = i0; i <= i1; i++) {
            const int p = i * b - lo;
            const uint64_t q = cs[i];
            v |= p >= 0 ? q << p : q >> (-p);
        }
        for (int u = 0; u < 4 && 4 * wq + u < nb; u++) dst[10 + 4 * wq + u] = (uint8_t)(v >> (8 * u));
    }
}

}  // namespace

int64_t encode_bound(int64_t keep, int32_t G, int32_t C) {
    const int64_t ng = n_groups_of(keep, G);
    return (int64_t)C * (10 * ng + 2 * keep);
}

mgs_status encode_launch(mgs_ctx *ctx, const mgs_scene *sc, const int32_t *kept, int64_t keep,
                         int32_t G, const uint8_t *d_bits, uint8_t *stream, int64_t capacity,
                         int32_t *d_sizes_out, int64_t *total_out, cudaStream_t st) {
    const int64_t ng = n_groups_of(keep, G);
    const int64_t m = ng * sc->C;
    if (m > 0x7FFFFFFFLL) {
        set_error("%lld blocks exceed one launch", (long long)m);
        return MGS_ERR_INVALID_ARG;
    }
    const int64_t slot_bytes = a16(10 + 2 * (int64_t)G);
    const int64_t nchunks = (m + kScanChunk - 1) / kScanChunk;
    const size_t b_codes = (size_t)a16(2 * keep * sc->C), b_mm = (size_t)a16(8 * m);
    const size_t b_slots = (size_t)(m * slot_bytes), b_sizes = (size_t)a16(4 * m);
    const size_t b_off = (size_t)a16(8 * m), b_sums = (size_t)a16(8 * (nchunks + 1));
    const size_t b_info = (size_t)a16((int64_t)sizeof(EncInfo) * m), b_fc = (size_t)a16(4 * keep * sc->C);
    unsigned char *ws = nullptr;
    const size_t ws_bytes = b_codes + b_mm + b_slots + b_sizes + b_off + b_sums + b_info + b_fc;
    if (cudaMallocAsync(reinterpret_cast<void **>(&ws), ws_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("encoder workspace of %zu bytes", ws_bytes);
        return MGS_ERR_OUT_OF_MEMORY;
    }
    size_t o = 0;
    uint16_t *d_codes = reinterpret_cast<uint16_t *>(ws + o);
    o += b_codes;
    float *d_mm = reinterpret_cast<float *>(ws + o);
    o += b_mm;
    uint8_t *d_slots = ws + o;
    o += b_slots;
    int32_t *d_sizes = reinterpret_cast<int32_t *>(ws + o);
    o += b_sizes;
    int64_t *d_off = reinterpret_cast<int64_t *>(ws + o);
    o += b_off;
    int64_t *d_sums = reinterpret_cast<int64_t *>(ws + o);
    o += b_sums;
    EncInfo *d_info = reinterpret_cast<EncInfo *>(ws + o);
    o += b_info;
    uint32_t *d_fc = reinterpret_cast<uint32_t *>(ws + o);

    mgs_status s = quantize_launch(ctx, sc, kept, keep, G, d_bits, d_codes, d_mm, st);
    int64_t total = 0;
    if (s == MGS_OK && m > 0) {
        const EncSmem L(G);
        const size_t smem = (size_t)L.total;
        cudaError_t e = cudaFuncSetAttribute(k_enc_model, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess) {
            k_enc_model<<<(unsigned)m, kEncThreads, smem, st>>>(d_codes, keep, G, (int32_t)ng, d_bits,
                                                                d_mm, d_slots, slot_bytes, d_info,
                                                                d_fc, d_sizes);
            // sub-group width: the lanes of a full group, rounded up to a power of two
            const int full_lanes = std::min(32, std::max(1, G >> 9));
            const int gw = full_lanes <= 1 ? 1 : full_lanes <= 2 ? 2 : full_lanes <= 4 ? 4
                         : full_lanes <= 8 ? 8 : full_lanes <= 16 ? 16 : 32;
            const int64_t per_cta = (int64_t)kEncWarps * (32 / gw);
            const unsigned grid = (unsigned)((m + per_cta - 1) / per_cta);
            switch (gw) {
                case 1: k_enc_rans<1><<<grid, kEncThreads, 0, st>>>(d_fc, keep, G, (int32_t)ng, m, d_bits, d_slots, slot_bytes, d_info, d_sizes); break;
                case 2: k_enc_rans<2><<<grid, kEncThreads, 0, st>>>(d_fc, keep, G, (int32_t)ng, m, d_bits, d_slots, slot_bytes, d_info, d_sizes); break;
                case 4: k_enc_rans<4><<<grid, kEncThreads, 0, st>>>(d_fc, keep, G, (int32_t)ng, m, d_bits, d_slots, slot_bytes, d_info, d_sizes); break;
                case 8: k_enc_rans<8><<<grid, kEncThreads, 0, st>>>(d_fc, keep, G, (int32_t)ng, m, d_bits, d_slots, slot_bytes, d_info, d_sizes); break;
                case 16: k_enc_rans<16><<<grid, kEncThreads, 0, st>>>(d_fc, keep, G, (int32_t)ng, m, d_bits, d_slots, slot_bytes, d_info, d_sizes); break;
                default: k_enc_rans<32><<<grid, kEncThreads, 0, st>>>(d_fc, keep, G, (int32_t)ng, m, d_bits, d_slots, slot_bytes, d_info, d_sizes); break;
            }
            k_enc_chunk_sums<<<(unsigned)nchunks, 1024, 0, st>>>(d_sizes, m, d_sums);
            k_enc_scan_sums<<<1, 1024, 0, st>>>(d_sums, nchunks, d_sums + nchunks);
            k_enc_offsets<<<(unsigned)nchunks, 1024, 0, st>>>(d_sizes, m, d_sums, d_off);
            count_launches(5);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, d_sums + nchunks, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("block coder: %s", cudaGetErrorString(e));
            s = MGS_ERR_CUDA;
        }
        if (s == MGS_OK && stream) {
            if (capacity < total) {
                set_error("stream capacity %lld < %lld bytes", (long long)capacity, (long long)total);
                s = MGS_ERR_INVALID_ARG;
            } else {
                k_enc_gather<<<(unsigned)m, 256, 0, st>>>(d_codes, keep, G, (int32_t)ng, d_bits, d_slots,
                                                          slot_bytes, d_info, d_sizes, d_off, stream);
                count_launches(1);
                e = cudaGetLastError();
                if (e != cudaSuccess) {
                    set_error("block gather: %s", cudaGetErrorString(e));
                    s = MGS_ERR_CUDA;
                }
            }
        }
        if (s == MGS_OK && d_sizes_out) {
            e = cudaMemcpyAsync(d_sizes_out, d_sizes, 4 * (size_t)m, cudaMemcpyDefault, st);
            if (e != cudaSuccess) {
                set_error("block sizes copy: %s", cudaGetErrorString(e));
                s = MGS_ERR_CUDA;
            }
        }
    }
    cudaFreeAsync(ws, st);
    if (s == MGS_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("block coder: %s", cudaGetErrorString(e));
            s = MGS_ERR_CUDA;
        }
    }
    *total_out = total;
    return s;
}

}  // namespace mgs

extern "C" int64_t mgs_encode_bound(int64_t keep, int32_t group_size, int32_t n_channels) {
    if (keep < 1 || group_size < 1 || n_channels < 1) return -1;
    return mgs::encode_bound(keep, group_size, n_channels);
}

extern "C" mgs_status mgs_encode_config(mgs_ctx *ctx, const mgs_scene *scene, int64_t keep,
                                        int32_t group_size, const uint8_t *bits, uint8_t *stream,
                                        int64_t capacity, int32_t *block_bytes,
                                        int64_t *total_bytes, void *cuda_stream) {
    using namespace mgs;
    clear_error();
    if (!ctx || !scene || !bits || !total_bytes) {
        set_error("ctx, scene, bits and total_bytes must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (keep < 1 || keep > scene->n || group_size < 1 || group_size > MGS_MAX_GROUP) {
        set_error("keep %lld or group_size %d out of range", (long long)keep, group_size);
        return MGS_ERR_INVALID_ARG;
    }
    if (stream && !is_device_pointer(stream)) {
        set_error("stream must be device memory");
        return MGS_ERR_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t m = n_groups_of(keep, group_size) * scene->C;
    // the widths on the device, checked to lie in 1..16
    std::vector<uint8_t> hb((size_t)m);
    MGS_CUDA_TRY(cudaMemcpyAsync(hb.data(), bits, (size_t)m, cudaMemcpyDefault, st));
    MGS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < m; i++) {
        if (hb[i] < 1 || hb[i] > 16) {
            set_error("bits[%lld] = %d is not in 1..16", (long long)i, (int)hb[i]);
            return MGS_ERR_INVALID_ARG;
        }
    }
    uint8_t *d_bits = nullptr;
    MGS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&d_bits), (size_t)m, st));
    cudaError_t e = cudaMemcpyAsync(d_bits, hb.data(), (size_t)m, cudaMemcpyHostToDevice, st);
    mgs_scene *sc = const_cast<mgs_scene *>(scene);
    mgs_scene tmp_owner;   // a one-ratio kept list; the scene's cached lists are left alone
    tmp_owner.ctx = sc->ctx;
    tmp_owner.n = sc->n;
    tmp_owner.C = sc->C;
    tmp_owner.d_rank_m = sc->d_rank_m;
    mgs_status s = MGS_OK;
    if (e != cudaSuccess) {
        set_error("bits copy: %s", cudaGetErrorString(e));
        s = MGS_ERR_CUDA;
    }
    const int32_t *pos = nullptr;
    std::vector<int64_t> off;
    if (s == MGS_OK) s = scene_kept(&tmp_owner, &keep, 1, st, &pos, &off);
    if (s == MGS_OK)
        s = encode_launch(ctx, sc, pos, keep, group_size, d_bits, stream, capacity, block_bytes,
                          total_bytes, st);
    if (tmp_owner.kept.pos) cudaFreeAsync(tmp_owner.kept.pos, st);
    tmp_owner.kept.pos = nullptr;
    tmp_owner.d_rank_m = nullptr;
    cudaFreeAsync(d_bits, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (s == MGS_OK && e2 != cudaSuccess) {
        set_error("encode: %s", cudaGetErrorString(e2));
        s = MGS_ERR_CUDA;
    }
    return s;
}
