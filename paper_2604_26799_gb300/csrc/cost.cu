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
// When S is a normal float, S = R * 2^-b exactly, so fl(c / S) = fl(c / R) * 2^b
// whenever fl(c / R) is normal or zero; the kernel divides once per element
// (u = fl(c / R)) and forms x = fma(u, 2^b, Z), which is the same single
// rounding of the same exact sum.  Groups with a subnormal |u| or a subnormal S
// take the literal division per element and bit-width.
//
// Histograms live in shared memory: per-lane columns for b <= 6 (no
// same-address conflicts inside a warp), a direct table for 7 <= b <= 12, and
// an open-addressing hash of (code, count) for b >= 13.  The entropy bound is
// accumulated as L(n) - sum L(h) with L(h) = h log2 h in 32.32 fixed point, so
// it does not depend on the reduction order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>

#include "internal.h"

namespace mgs {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kDirectMaxBits = 12;
constexpr int kLaneMaxBits = 6;

struct BitParam {
    float S, Z, twob, top;
    float Ss;      // S * 2^k: the step in the group's scaled units (exact)
    int b;
    int literal;   // 1: divide per element and bit-width
    int degenerate;
};

struct KernelArgs {
    const CostSeg *segs;
    int32_t n_segs;
    int32_t G;
    int64_t n_work;
    int32_t n_bits;
    int32_t opt_lo, opt_hi;
    int32_t bits[MGS_MAX_OPTIONS];
    const unsigned long long *ltab;
    unsigned int *counter;
    uint32_t hash_log2;   // log2 of the hash capacity
};

__device__ __forceinline__ uint32_t hash_slot(uint32_t q, uint32_t log2cap) {
    return (q * 2654435769u) >> (32 - log2cap);
}

// Histogram update for one code.
template <int MODE>
__device__ __forceinline__ void hist_add(uint32_t *hist, uint32_t q, int lane, uint32_t log2cap) {
    if (MODE == 0) {
        atomicAdd(&hist[q * 32u + lane], 1u);
    } else if (MODE == 1) {
        atomicAdd(&hist[q], 1u);
    } else {
        // slot word: (q + 1) << 15 | count, count < 2^15
        const uint32_t key = (q + 1u) << 15;
        const uint32_t mask = (1u << log2cap) - 1u;
        uint32_t s = hash_slot(q, log2cap);
        volatile uint32_t *vh = hist;
        while (true) {
            uint32_t v = vh[s];
            if (v == 0u) {
                uint32_t old = atomicCAS(&hist[s], 0u, key | 1u);
                if (old == 0u) break;
                v = old;
            }
            if ((v & ~0x7FFFu) == key) {
                atomicAdd(&hist[s], 1u);
                break;
            }
            s = (s + 1u) & mask;
        }
    }
}

// Evaluate one bit-width for this thread's elements of one channel.  c holds
// the values scaled by 2^k (exact), so err, its square and sums stay in the
// normal FP32 range whatever the magnitude of the channel.
template <int T, int EPT, int MODE, bool LITERAL>
__device__ __forceinline__ void eval_bits(const float (&c)[EPT], const float (&u)[EPT], int nvalid,
                                          const BitParam &p, uint32_t *hist, uint32_t log2cap,
                                          float &sse, float &l1, float &linf) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        if (e * T + (int)threadIdx.x < nvalid) {
            float x;
            if (LITERAL) {
                x = __fadd_rn(__fdiv_rn(c[e], p.Ss), p.Z);   // c' / S' == c / S exactly
            } else {
                x = __fmaf_rn(u[e], p.twob, p.Z);
            }
            float xc = fminf(fmaxf(x, 0.0f), p.top);
            int q = __float2int_rn(xc);
            float qz = __fsub_rn(__int2float_rn(q), p.Z);
            float chat = __fmul_rn(qz, p.Ss);                 // c_hat * 2^k
            float err = __fsub_rn(chat, c[e]);                // e * 2^k
            sse = __fmaf_rn(err, err, sse);
            l1 = __fadd_rn(l1, fabsf(err));
            linf = fmaxf(linf, fabsf(err));
            hist_add<MODE>(hist, (uint32_t)q, lane, log2cap);
        }
    }
}

// Sum of L(h) over the histogram of one bit-width, clearing it.
template <int T, int MODE>
__device__ __forceinline__ unsigned long long hist_scan(uint32_t *hist, int b, uint32_t log2cap,
                                                        const unsigned long long *__restrict__ ltab) {
    unsigned long long acc = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (MODE == 0) {
        const int bins = 1 << b;
        for (int k = warp; k < bins; k += T / 32) {
            uint32_t v = hist[k * 32 + lane];
            hist[k * 32 + lane] = 0u;
            uint32_t s = __reduce_add_sync(kFull, v);
            if (lane == 0 && s) acc += __ldg(&ltab[s]);
        }
    } else if (MODE == 1) {
        const int bins = 1 << b;
        for (int k = threadIdx.x; k < bins; k += T) {
            uint32_t v = hist[k];
            if (v) {
                acc += __ldg(&ltab[v]);
                hist[k] = 0u;
            }
        }
    } else {
        const int cap = 1 << log2cap;
        for (int k = threadIdx.x; k < cap; k += T) {
            uint32_t v = hist[k];
            if (v) {
                acc += __ldg(&ltab[v & 0x7FFFu]);
                hist[k] = 0u;
            }
        }
    }
    return acc;
}

template <int T>
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
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <int W>
__device__ __forceinline__ void load_row(const float *p, float (&v)[W]) {
    if (W == 8) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4 % W] = b.x; v[5 % W] = b.y; v[6 % W] = b.z; v[7 % W] = b.w;
    } else if (W == 4) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = a.x; v[1 % W] = a.y; v[2 % W] = a.z; v[3 % W] = a.w;
    } else if (W == 2) {
        float2 a = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = a.x; v[1 % W] = a.y;
    } else {
        v[0] = __ldg(p);
    }
}

// Shared-memory layout (dynamic): hist | psse | pl1 | plinf | hpart | params | minmax
struct Smem {
    uint32_t *hist;
    float *psse, *pl1, *plinf;            // [n_opts][T]
    unsigned long long *hpart;            // [n_opts][T/32]
    BitParam *bp;                         // [n_opts]
    float *mm;                            // [T/32][W][2]
    int *misc;                            // [4]
};

template <int T, int W>
__device__ __forceinline__ Smem carve(unsigned char *base, int hist_words, int n_opts) {
    Smem s;
    size_t off = 0;
    s.hist = reinterpret_cast<uint32_t *>(base + off);
    off += (size_t)hist_words * 4;
    s.psse = reinterpret_cast<float *>(base + off);
    off += (size_t)n_opts * T * 4;
    s.pl1 = reinterpret_cast<float *>(base + off);
    off += (size_t)n_opts * T * 4;
    s.plinf = reinterpret_cast<float *>(base + off);
    off += (size_t)n_opts * T * 4;
    off = (off + 15) & ~(size_t)15;
    s.hpart = reinterpret_cast<unsigned long long *>(base + off);
    off += (size_t)n_opts * (T / 32) * 8;
    s.bp = reinterpret_cast<BitParam *>(base + off);
    off += (size_t)n_opts * sizeof(BitParam);
    s.mm = reinterpret_cast<float *>(base + off);
    off += (size_t)(T / 32) * W * 2 * 4;
    s.misc = reinterpret_cast<int *>(base + off);
    return s;
}

__host__ __device__ inline int hist_words_for(int G, int hash_log2) {
    int lane_words = (1 << kLaneMaxBits) * 32;
    int direct_words = 1 << kDirectMaxBits;
    int hash_words = 1 << hash_log2;
    int w = lane_words > direct_words ? lane_words : direct_words;
    return w > hash_words ? w : hash_words;
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
    const int g = (int)(local / S.n_chunks);
    const int chunk = (int)(local % S.n_chunks);
    const int c0 = chunk * W;
    const int slab = c0 / kSlabWidth;
    const int j0 = c0 % kSlabWidth;
    const int64_t gstart = (int64_t)g * A.G;
    const int nvalid = (int)((S.K - gstart) < (int64_t)A.G ? (S.K - gstart) : (int64_t)A.G);

    // ---- gather: each element's W channels from its slab row
    float v[W][EPT];
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        int i = e * T + threadIdx.x;
        float row[W];
        if (i < nvalid) {
            int32_t pos = __ldg(&S.kept[gstart + i]);
            load_row<W>(S.slabs + ((int64_t)slab * S.n + pos) * kSlabWidth + j0, row);
        } else {
#pragma unroll
            for (int w = 0; w < W; w++) row[w] = 0.0f;
        }
#pragma unroll
        for (int w = 0; w < W; w++) v[w][e] = row[w];
    }

    // ---- group min / max of every channel of the chunk
    {
        float mn[W], mx[W];
#pragma unroll
        for (int w = 0; w < W; w++) {
            mn[w] = FLT_MAX;
            mx[w] = -FLT_MAX;
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                if (e * T + (int)threadIdx.x < nvalid) {
                    mn[w] = fminf(mn[w], v[w][e]);
                    mx[w] = fmaxf(mx[w], v[w][e]);
                }
            }
            mn[w] = warp_min(mn[w]);
            mx[w] = warp_max(mx[w]);
            if (lane == 0) {
                sm.mm[(warp * W + w) * 2] = mn[w];
                sm.mm[(warp * W + w) * 2 + 1] = mx[w];
            }
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
            p.S = __fdiv_rn(R, p.twob);
            p.Ss = __fmul_rn(__fmul_rn(p.S, s1), s2);
            p.degenerate = p.S == 0.0f;
            if (!p.degenerate) {
                float t = __fdiv_rn(M, p.S);
                p.Z = rintf(__fsub_rn(p.twob, t));
            } else {
                p.Z = 0.0f;
            }
            p.literal = p.S < FLT_MIN;
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
        const int any_slow = __syncthreads_or(slow);

#pragma unroll 1
        for (int k = 0; k < n_opts; k++) {
            const BitParam p = sm.bp[k];
            float sse = 0.0f, l1 = 0.0f, linf = 0.0f;
            if (p.degenerate) {
                sm.psse[k * T + threadIdx.x] = 0.0f;
                sm.pl1[k * T + threadIdx.x] = 0.0f;
                sm.plinf[k * T + threadIdx.x] = 0.0f;
                if (lane == 0) sm.hpart[k * NW + warp] = warp == 0 ? __ldg(&A.ltab[nvalid]) : 0ull;
                continue;
            }
            const int mode = p.b <= kLaneMaxBits ? 0 : (p.b <= kDirectMaxBits ? 1 : 2);
            const bool lit = p.literal || any_slow;
            if (mode == 0) {
                if (lit) eval_bits<T, EPT, 0, true>(cw, u, nvalid, p, sm.hist, A.hash_log2, sse, l1, linf);
                else eval_bits<T, EPT, 0, false>(cw, u, nvalid, p, sm.hist, A.hash_log2, sse, l1, linf);
            } else if (mode == 1) {
                if (lit) eval_bits<T, EPT, 1, true>(cw, u, nvalid, p, sm.hist, A.hash_log2, sse, l1, linf);
                else eval_bits<T, EPT, 1, false>(cw, u, nvalid, p, sm.hist, A.hash_log2, sse, l1, linf);
            } else {
                if (lit) eval_bits<T, EPT, 2, true>(cw, u, nvalid, p, sm.hist, A.hash_log2, sse, l1, linf);
                else eval_bits<T, EPT, 2, false>(cw, u, nvalid, p, sm.hist, A.hash_log2, sse, l1, linf);
            }
            sm.psse[k * T + threadIdx.x] = sse;
            sm.pl1[k * T + threadIdx.x] = l1;
            sm.plinf[k * T + threadIdx.x] = linf;
            __syncthreads();
            unsigned long long acc;
            if (mode == 0) acc = hist_scan<T, 0>(sm.hist, p.b, A.hash_log2, A.ltab);
            else if (mode == 1) acc = hist_scan<T, 1>(sm.hist, p.b, A.hash_log2, A.ltab);
            else acc = hist_scan<T, 2>(sm.hist, p.b, A.hash_log2, A.ltab);
            acc = warp_sum_u64(acc);
            if (lane == 0) sm.hpart[k * NW + warp] = acc;
            __syncthreads();
        }
        __syncthreads();
        // ---- reduce the per-thread partials and write this channel's entries
        for (int k = warp; k < n_opts; k += NW) {
            float a = 0.0f, b = 0.0f, cmax = 0.0f;
#pragma unroll
            for (int j = 0; j < T / 32; j++) {
                a = __fadd_rn(a, sm.psse[k * T + j * 32 + lane]);
                b = __fadd_rn(b, sm.pl1[k * T + j * 32 + lane]);
                cmax = fmaxf(cmax, sm.plinf[k * T + j * 32 + lane]);
            }
            a = warp_sum<T>(a);
            b = warp_sum<T>(b);
            cmax = warp_max(cmax);
            unsigned long long hs = 0;
            for (int j = lane; j < NW; j += 32) hs += sm.hpart[k * NW + j];
            hs = warp_sum_u64(hs);
            if (lane == 0) {
                const int64_t o = item * A.n_bits + A.opt_lo + k;
                // undo the 2^k scale in FP64 (exact powers of two)
                const double inv = __longlong_as_double((long long)(1023 - kexp) << 52);
                const double inv2 = __longlong_as_double((long long)(1023 - 2 * kexp) << 52);
                S.sse[o] = (double)a * inv2;
                S.l1[o] = (double)b * inv;
                S.linf[o] = (float)((double)cmax * inv);
                unsigned long long ln = __ldg(&A.ltab[nvalid]);
                S.hbits[o] = (double)(long long)(ln - hs) * (1.0 / 4294967296.0);
            }
        }
        __syncthreads();
    }
}

template <int T, int EPT, int W>
__global__ void __launch_bounds__(T, (T >= 512 ? 1 : 512 / T)) k_cost(const __grid_constant__ KernelArgs A,
                                                                      int hist_words) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n_opts = A.opt_hi - A.opt_lo;
    Smem sm = carve<T, W>(smem_raw, hist_words, n_opts);
    for (int i = threadIdx.x; i < hist_words; i += T) sm.hist[i] = 0u;
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
};
#undef MGS_CFG
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

int hash_log2_for(int G) {
    int cap = 1;
    while (cap < 2 * G) cap <<= 1;
    int l = 0;
    while ((1 << l) < cap) l++;
    return std::max(l, 5);
}

}  // namespace

int cost_config_count() { return kNumConfigs; }
const CostConfig &cost_config(int i) { return kConfigs[i].cfg; }

int cost_default_config(int G) {
    if (G <= 1024) return 6;    // 128 x 8, W 8
    if (G <= 2048) return 4;    // 256 x 8, W 8
    if (G <= 4096) return 0;    // 256 x 16, W 4
    if (G <= 16384) return 8;   // 512 x 32, W 1
    return -1;
}

size_t cost_smem_bytes(int config, int G, int n_opts) {
    const CostConfig &c = kConfigs[config].cfg;
    int hw = hist_words_for(G, hash_log2_for(G));
    size_t off = (size_t)hw * 4 + (size_t)n_opts * c.threads * 4 * 3;
    off = (off + 15) & ~(size_t)15;
    off += (size_t)n_opts * (c.threads / 32) * 8 + (size_t)n_opts * sizeof(BitParam) +
           (size_t)(c.threads / 32) * c.width * 2 * 4 + 16;
    return off;
}

struct CostExec {
    const ConfigEntry *entry = nullptr;
    KernelArgs args{};
    int hist_words = 0;
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
        n_work += (int64_t)s.n_groups * s.n_chunks;
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
    A.hash_log2 = (uint32_t)hash_log2_for(L.group_size);
    X->hist_words = hist_words_for(L.group_size, (int)A.hash_log2);
    X->smem = cost_smem_bytes(config, L.group_size, L.opt_hi - L.opt_lo);
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
    X->entry->kernel<<<(unsigned)X->grid, X->entry->cfg.threads, X->smem, st>>>(X->args,
                                                                                   X->hist_words);
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

bool cost_config_fits(int config, int group_size, int n_opts) {
    if (config < 0 || config >= kNumConfigs) return false;
    const CostConfig &c = kConfigs[config].cfg;
    return (int64_t)c.threads * c.ept >= group_size &&
           cost_smem_bytes(config, group_size, n_opts) <= 227 * 1024;
}

}  // namespace mgs
