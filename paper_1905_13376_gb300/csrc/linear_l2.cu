// linear_l2.cu -- the linear 3-way join R(A,B) S(B,C) T(C,D) with shares
// I = J = 1 (Section 4, Algorithm 1, with one bucket on each side).
//
// Algorithm 1 partitions R by h(B) and T by g(C) so that one bucket of each
// fits the on-chip memory while the matching part of S streams past.  The
// shares are the smallest that make the held buckets fit; on this GPU the
// on-chip memory every SM reaches is the 129 MB L2, and the key tables of a
// relation with a few million distinct keys fit it whole.  Then I = J = 1:
// nothing is partitioned, and the aggregates become three streaming passes,
// each reading one relation once:
//
//   T pass   deg_T(c)                          (T's single table)
//   S pass   w(b)   += deg_T(c)     per (b, c) of S   (S's weight table)
//   R pass   cnt[a] += w(b), total += w(b)  per (a, b) of R
//
// which adds the terms of COUNT = sum over (b,c) in S of deg_R(b) deg_T(c)
// and of cnt(a) = sum over (a,b) in R, (b,c) in S of deg_T(c) in another
// order.  S is keyed by its own B column, so the table gets one insertion
// per distinct b, and runs of equal keys (edge lists sorted by source) are
// summed inside each warp before they reach the L2; the R pass only reads
// the table and adds each run of equal a once.
#include "internal.h"
#include "linear_l2.h"
#include "skew.h"
#include "warp_runs.cuh"

namespace mwj {
namespace {

constexpr int WT = 256;     // threads per CTA
constexpr int WQ = kRunQ;   // tuples per lane per warp round: one 128-bit load per column
constexpr uint32_t WCHUNK = 32 * WQ;   // tuples per warp round

// Tuples [i, i + WQ) of two int32 columns (fewer at the end); returns how
// many are valid.
__device__ __forceinline__ uint32_t load_pairs(const int32_t *__restrict__ X, const int32_t *__restrict__ Y,
                                               uint32_t n, uint32_t i, bool vec, uint64_t pol,
                                               int32_t (&x)[WQ], int32_t (&y)[WQ]) {
    if (i >= n) return 0;
    if (vec && i + WQ <= n) {
        const int4 a = ld_stream((const int4 *)(X + i), pol);
        const int4 b = ld_stream((const int4 *)(Y + i), pol);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        y[0] = b.x; y[1] = b.y; y[2] = b.z; y[3] = b.w;
        return WQ;
    }
    const uint32_t m = min((uint32_t)WQ, n - i);
#pragma unroll
    for (int q = 0; q < WQ; ++q) {
        if ((uint32_t)q < m) {
            x[q] = __ldg(X + i + q);
            y[q] = __ldg(Y + i + q);
        }
    }
    return m;
}

// deg_T(c) from the first probe (slot s, value v) of c in T's single table.
__device__ __forceinline__ unsigned long long t_deg(const uint64_t *__restrict__ img, uint32_t tmask,
                                                    uint32_t c, uint32_t s, unsigned long long v) {
    for (uint32_t it = 0; it < tmask && v != kEmpty64 && (uint32_t)v != c; ++it) {
        s = (s + 1) & tmask;
        v = __ldg((const unsigned long long *)(img + s));
    }
    return (v == kEmpty64 || (uint32_t)v != c) ? 0ull : (v >> 32);
}

// w(b) += x (x > 0).  The key is claimed with a CAS that also stores x's low
// word; later adds go to the upper word, and the carry out of it (read back
// from the add's old value) goes to hi[].
__device__ __forceinline__ void w_add(const WTable &w, uint32_t mask, uint32_t b, unsigned long long x,
                                      DevStatus *st) {
    if (b == kEmptyKey) {
        atomicAdd(w.W + mask + 1, x);
        return;
    }
    const unsigned long long lo = x & 0xFFFFFFFFull;
    const uint32_t hx = (uint32_t)(x >> 32);
    uint32_t s = slot_of(b, w.seed, mask);
    for (uint32_t it = 0; it <= mask; ++it) {
        unsigned long long v = __ldcg(w.W + s);
        if (v == kEmpty64) {
            const unsigned long long old = atomicCAS(w.W + s, kEmpty64, (lo << 32) | b);
            if (old == kEmpty64) {
                if (hx) {
                    atomicAdd(w.hi + s, hx);
                    atomicOr(w.meta + 2, 1u);
                }
                return;
            }
            v = old;
        }
        if ((uint32_t)v == b) {
            const unsigned long long old = atomicAdd(w.W + s, lo << 32);
            const uint32_t h = hx + (uint32_t)(((old >> 32) + lo) >> 32);
            if (h) {
                atomicAdd(w.hi + s, h);
                atomicOr(w.meta + 2, 1u);
            }
            return;
        }
        s = (s + 1) & mask;
    }
    set_status(st, MWJ_ERR_CHECK, 7);   // table full: the sizing step under-estimated
}

// Direct-address weights (the sizing pass chose that layout for S's B
// values): w(b) is the plain 64-bit word W[b - min], added to with 64-bit
// atomics whose results are not needed (exact modulo 2^64, no carry word).
__device__ __forceinline__ void w_add_direct(unsigned long long *__restrict__ W, uint32_t wmin, uint32_t wspan,
                                             uint32_t b, unsigned long long x, DevStatus *st) {
    if (b - wmin < wspan)
        atomicAdd(W + (b - wmin), x);
    else
        set_status(st, MWJ_ERR_CHECK, 9);   // a key outside the range the sizing pass saw
}

__global__ void k_w_clear(unsigned long long *__restrict__ W, uint32_t *__restrict__ hi,
                          uint32_t *__restrict__ meta) {
    const uint32_t stride = gridDim.x * blockDim.x;
    if (meta[kMetaDense]) {
        const uint32_t span = meta[kMetaSpan];
        for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < span; s += stride) W[s] = 0ull;
    } else {
        const uint32_t slots = meta[0] + 1;   // a power of two >= 16
        for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < slots / 2; s += stride) {
            ((ulonglong2 *)W)[s] = make_ulonglong2(kEmpty64, kEmpty64);
            ((uint2 *)hi)[s] = make_uint2(0u, 0u);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            W[slots] = 0ull;
            hi[slots] = 0u;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) meta[kMetaWide] = 0u;
}

// S pass.  Warp-uniform loop: a warp takes 128 consecutive tuples per round,
// four per lane, and loads its next round before it works on this one.
// Heavy keys (sampled, see heavy_detect) are summed per CTA in shared
// memory and added to the table once per CTA, so that a key holding a large
// share of S in no particular order does not funnel every warp's adds into
// one L2 word.  TD / WD: T's table / S's weight table in the direct-address
// layout (one load per T lookup, one fire-and-forget 64-bit add per run of
// equal B values) rather than hashed.
// One warp round of the S pass: lane l holds tuples (b[q], c[q]), q < m, of
// 128 consecutive ones.  x = deg_T(c); heavy B keys go to the CTA's sums;
// runs of equal b are summed in the warp and added to w(b) once.
template <bool TD, bool WD>
struct SPass {
    const TImg &t;
    const WTable &w;
    DevStatus *st;
    const uint32_t *hs;
    unsigned long long *hacc;
    uint32_t tmask, wmask, tmin, tspan, wmin, wspan;

    __device__ SPass(const TImg &t_, const WTable &w_, DevStatus *st_, const uint32_t *hs_,
                     unsigned long long *hacc_)
        : t(t_), w(w_), st(st_), hs(hs_), hacc(hacc_) {
        tmask = __ldg(t.meta);
        wmask = __ldg(w.meta);
        tmin = TD ? __ldg(t.meta + kMetaMin) : 0u;
        tspan = TD ? __ldg(t.meta + kMetaSpan) : 0u;
        wmin = WD ? __ldg(w.meta + kMetaMin) : 0u;
        wspan = WD ? __ldg(w.meta + kMetaSpan) : 0u;
    }

    __device__ __forceinline__ void round(const int32_t (&b)[WQ], const int32_t (&c)[WQ], uint32_t m) {
        unsigned long long x[WQ];
        if constexpr (TD) {
            const uint32_t *tdeg = (const uint32_t *)t.img;
#pragma unroll
            for (int q = 0; q < WQ; ++q) {
                const uint32_t k = (uint32_t)c[q] - tmin;
                x[q] = ((uint32_t)q < m && k < tspan) ? (unsigned long long)__ldg(tdeg + k) : 0ull;
            }
        } else {
            uint32_t ts[WQ];
            unsigned long long tv[WQ];
#pragma unroll
            for (int q = 0; q < WQ; ++q) {
                if ((uint32_t)q < m) {
                    ts[q] = slot_of((uint32_t)c[q], t.seed_slot, tmask);
                    tv[q] = __ldg((const unsigned long long *)(t.img + ts[q]));
                }
            }
#pragma unroll
            for (int q = 0; q < WQ; ++q)
                x[q] = ((uint32_t)q < m) ? t_deg(t.img, tmask, (uint32_t)c[q], ts[q], tv[q]) : 0ull;
        }
        if (hs) {
#pragma unroll
            for (int q = 0; q < WQ; ++q) {
                if (x[q] == 0) continue;
                const int hsl = heavy_slot(hs, (uint32_t)b[q]);
                if (hsl >= 0) {
                    atomicAdd(&hacc[hsl], x[q]);
                    x[q] = 0;
                }
            }
        }
        warp_runs(b, x, m, [&](int32_t key, unsigned long long sum) { add((uint32_t)key, sum); });
    }

    __device__ __forceinline__ void add(uint32_t b, unsigned long long x) {
        if constexpr (WD)
            w_add_direct(w.W, wmin, wspan, b, x, st);
        else
            w_add(w, wmask, b, x, st);
    }

    // the CTA's heavy-key sums into the table (every thread of the CTA calls this)
    __device__ __forceinline__ void flush_heavy(uint32_t nthreads) {
        if (!hs) return;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < kHeavySlots; i += nthreads)
            if (hacc[i]) add(hs[i], hacc[i]);
    }
};

// Tuples [lo, hi) of a column pair in warp rounds of 128 (warp `warp` of
// `warps` takes rounds warp, warp + warps, ...), each round's loads issued
// before the previous round is used; round(x, y, m) per round.
template <typename F>
__device__ __forceinline__ void rounds_plain(const int32_t *__restrict__ X, const int32_t *__restrict__ Y,
                                             uint32_t lo, uint32_t hi, uint32_t warp, uint32_t warps, F &&round) {
    const uint32_t lane = threadIdx.x & 31;
    const bool vec = (((uintptr_t)X | (uintptr_t)Y) & 15) == 0 && (lo & 3u) == 0;
    const uint64_t pol = l2_evict_first();
    const uint32_t n = hi;
    const uint32_t rounds = (hi - lo + WCHUNK - 1) / WCHUNK;
    int32_t x[WQ], y[WQ];
    uint32_t m = 0;
    uint32_t r = warp;
    if (r < rounds) m = load_pairs(X, Y, n, lo + r * WCHUNK + lane * WQ, vec, pol, x, y);
    while (r < rounds) {
        const uint32_t nr = r + warps;
        int32_t nx[WQ], ny[WQ];
        uint32_t nm = 0;
        if (nr < rounds) nm = load_pairs(X, Y, n, lo + nr * WCHUNK + lane * WQ, vec, pol, nx, ny);
        round(x, y, m);
#pragma unroll
        for (int q = 0; q < WQ; ++q) {
            x[q] = nx[q];
            y[q] = ny[q];
        }
        m = nm;
        r = nr;
    }
}

template <bool TD, bool WD>
__device__ __forceinline__ void w_build_pass(const int32_t *__restrict__ Sb, const int32_t *__restrict__ Sc,
                                             uint32_t n, const TImg &t, const WTable &w, DevStatus *st,
                                             const uint32_t *hs, unsigned long long *hacc) {
    SPass<TD, WD> P(t, w, st, hs, hacc);
    const uint32_t warp = (blockIdx.x * WT + threadIdx.x) >> 5, warps = (gridDim.x * WT) >> 5;
    rounds_plain(Sb, Sc, 0u, n, warp, warps,
                 [&](const int32_t (&b)[WQ], const int32_t (&c)[WQ], uint32_t m) { P.round(b, c, m); });
    P.flush_heavy(WT);
}

// Two kernels share the S pass: the direct-address one (both tables in that
// layout, few registers) and the general one; the call launches both and the
// one whose layout the sizing passes did not choose returns at once.
__global__ void __launch_bounds__(WT) k_w_build(const int32_t *__restrict__ Sb, const int32_t *__restrict__ Sc,
                                                uint32_t n, TImg t, WTable w, DevStatus *st) {
    const bool td = __ldg(t.meta + kMetaDense) != 0u, wd = __ldg(w.meta + kMetaDense) != 0u;
    if (td && wd) return;
    __shared__ uint32_t hbuf[kHeavySlots];
    __shared__ unsigned long long hacc[kHeavySlots];
    const uint32_t *hs = heavy_to_smem(w.heavy, hbuf);
    if (hs) {
        for (uint32_t i = threadIdx.x; i < kHeavySlots; i += WT) hacc[i] = 0ull;
        __syncthreads();
    }
    if (td)
        w_build_pass<true, false>(Sb, Sc, n, t, w, st, hs, hacc);
    else if (wd)
        w_build_pass<false, true>(Sb, Sc, n, t, w, st, hs, hacc);
    else
        w_build_pass<false, false>(Sb, Sc, n, t, w, st, hs, hacc);
}

__global__ void __launch_bounds__(WT) k_w_build_direct(const int32_t *__restrict__ Sb,
                                                       const int32_t *__restrict__ Sc, uint32_t n, TImg t,
                                                       WTable w, DevStatus *st) {
    if (!__ldg(t.meta + kMetaDense) || !__ldg(w.meta + kMetaDense)) return;
    __shared__ uint32_t hbuf[kHeavySlots];
    __shared__ unsigned long long hacc[kHeavySlots];
    const uint32_t *hs = heavy_to_smem(w.heavy, hbuf);
    if (hs) {
        for (uint32_t i = threadIdx.x; i < kHeavySlots; i += WT) hacc[i] = 0ull;
        __syncthreads();
    }
    w_build_pass<true, true>(Sb, Sc, n, t, w, st, hs, hacc);
}

// w(b) from the first probe (slot s, value v); 0 when b is not in S.
__device__ __forceinline__ unsigned long long w_get(const WTable &w, uint32_t mask, bool wide, uint32_t b,
                                                    uint32_t s, unsigned long long v) {
    if (b == kEmptyKey) return v;   // slot mask + 1: the plain sum of key -1
    for (uint32_t it = 0; it < mask && v != kEmpty64 && (uint32_t)v != b; ++it) {
        s = (s + 1) & mask;
        v = __ldg(w.W + s);
    }
    if (v == kEmpty64 || (uint32_t)v != b) return 0ull;
    unsigned long long r = v >> 32;
    if (wide) r += (unsigned long long)__ldg(w.hi + s) << 32;
    return r;
}

// R pass (MODE 0: COUNT, MODE 1: GROUP BY A); same loop as the S pass.
// WD: the weight table in the direct-address layout.
// One warp round of the R pass: x = w(b) for the lane's tuples (a[q], b[q]),
// q < m, added to the thread's total and (GROUP BY A) per run of equal a to
// cnt[a].
template <int MODE, bool WD>
struct RPass {
    const WTable &w;
    int32_t a_domain;
    unsigned long long *cnt;
    DevStatus *st;
    uint32_t wmask, wmin, wspan;
    bool wide;
    unsigned long long acc = 0;

    __device__ RPass(const WTable &w_, int32_t a_domain_, unsigned long long *cnt_, DevStatus *st_)
        : w(w_), a_domain(a_domain_), cnt(cnt_), st(st_) {
        wmask = __ldg(w.meta);
        wide = !WD && __ldg(w.meta + kMetaWide) != 0;
        wmin = WD ? __ldg(w.meta + kMetaMin) : 0u;
        wspan = WD ? __ldg(w.meta + kMetaSpan) : 0u;
    }

    __device__ __forceinline__ void round(const int32_t (&a)[WQ], const int32_t (&b)[WQ], uint32_t m) {
        unsigned long long x[WQ];
        if constexpr (WD) {
#pragma unroll
            for (int q = 0; q < WQ; ++q) {
                const uint32_t k = (uint32_t)b[q] - wmin;
                x[q] = ((uint32_t)q < m && k < wspan) ? __ldg(w.W + k) : 0ull;
                acc += x[q];
            }
        } else {
            uint32_t ws[WQ];
            unsigned long long wv[WQ];
#pragma unroll
            for (int q = 0; q < WQ; ++q) {
                if ((uint32_t)q < m) {
                    const uint32_t k = (uint32_t)b[q];
                    ws[q] = (k == kEmptyKey) ? wmask + 1 : slot_of(k, w.seed, wmask);
                    wv[q] = __ldg(w.W + ws[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < WQ; ++q) {
                x[q] = ((uint32_t)q < m) ? w_get(w, wmask, wide, (uint32_t)b[q], ws[q], wv[q]) : 0ull;
                acc += x[q];
            }
        }
        if (MODE == 1) {
#pragma unroll
            for (int q = 0; q < WQ; ++q)
                if ((uint32_t)q < m && (uint32_t)a[q] >= (uint32_t)a_domain) set_status(st, MWJ_ERR_DOMAIN, a[q]);
            warp_runs(a, x, m, [&](int32_t key, unsigned long long sum) {
                if ((uint32_t)key < (uint32_t)a_domain) atomicAdd(cnt + key, sum);
            });
        }
    }
};

template <int MODE, bool WD>
__device__ __forceinline__ void w_probe_pass(const int32_t *__restrict__ Ra, const int32_t *__restrict__ Rb,
                                             uint32_t n, const WTable &w, int32_t a_domain,
                                             unsigned long long *__restrict__ cnt,
                                             unsigned long long *__restrict__ total, DevStatus *st,
                                             unsigned long long *red) {
    RPass<MODE, WD> P(w, a_domain, cnt, st);
    const uint32_t warp = (blockIdx.x * WT + threadIdx.x) >> 5, warps = (gridDim.x * WT) >> 5;
    rounds_plain(Ra, Rb, 0u, n, warp, warps,
                 [&](const int32_t (&a)[WQ], const int32_t (&b)[WQ], uint32_t m) { P.round(a, b, m); });
    const unsigned long long acc = block_sum_u64(P.acc, red);
    if (threadIdx.x == 0 && acc) atomicAdd(total, acc);
}

// The R pass as two kernels in the same way: direct-address weights, hashed.
template <int MODE>
__global__ void __launch_bounds__(WT) k_w_probe(const int32_t *__restrict__ Ra, const int32_t *__restrict__ Rb,
                                                uint32_t n, WTable w, int32_t a_domain,
                                                unsigned long long *__restrict__ cnt,
                                                unsigned long long *__restrict__ total, DevStatus *st) {
    if (__ldg(w.meta + kMetaDense)) return;
    __shared__ unsigned long long red[32];
    w_probe_pass<MODE, false>(Ra, Rb, n, w, a_domain, cnt, total, st, red);
}

template <int MODE>
__global__ void __launch_bounds__(WT) k_w_probe_direct(const int32_t *__restrict__ Ra,
                                                       const int32_t *__restrict__ Rb, uint32_t n, WTable w,
                                                       int32_t a_domain, unsigned long long *__restrict__ cnt,
                                                       unsigned long long *__restrict__ total, DevStatus *st) {
    if (!__ldg(w.meta + kMetaDense)) return;
    __shared__ unsigned long long red[32];
    w_probe_pass<MODE, true>(Ra, Rb, n, w, a_domain, cnt, total, st, red);
}

// CTAs of a grid-stride pass: every SM filled, no more warps than rounds.
template <typename K>
uint32_t pass_grid(K kernel, uint32_t n, int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, WT, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const uint64_t want = ((uint64_t)n + WCHUNK * (WT / 32) - 1) / (WCHUNK * (WT / 32));
    const uint64_t full = (uint64_t)num_sms * (uint64_t)per_sm;
    return (uint32_t)(want < full ? (want ? want : 1) : full);
}

}  // namespace

size_t w_table_slots(int64_t nS) { return single_table_slots(nS); }

cudaError_t w_table_size(const int32_t *Sb, int64_t nS, const WTable &w, unsigned int *hll,
                         uint64_t reserve_slots, int num_sms, cudaStream_t st, uint32_t *tmeta,
                         uint64_t treserve) {
    return single_table_size(Sb, nS, w.seed, hll, w.meta, reserve_slots, num_sms, st, "w_hll", "w_size", true,
                             tmeta, treserve);
}

cudaError_t w_table_clear(const WTable &w, int num_sms, cudaStream_t st) {
    ProfScope ps_("w_clear", st);
    k_w_clear<<<num_sms * 4, 512, 0, st>>>(w.W, w.hi, w.meta);
    return cudaGetLastError();
}

cudaError_t w_table_prepare(const int32_t *Sb, int64_t nS, const WTable &w, unsigned int *hll,
                            uint64_t reserve_slots, int num_sms, cudaStream_t st) {
    cudaError_t e = w_table_size(Sb, nS, w, hll, reserve_slots, num_sms, st);
    if (e != cudaSuccess) return e;
    return w_table_clear(w, num_sms, st);
}

cudaError_t w_table_build(const int32_t *Sb, const int32_t *Sc, int64_t nS, const TImg &t,
                          const WTable &w, DevStatus *status, int num_sms, cudaStream_t st) {
    if (nS <= 0) return cudaSuccess;
    const uint32_t n = (uint32_t)nS;
    {
        ProfScope ps_("w_build", st);
        k_w_build_direct<<<pass_grid(k_w_build_direct, n, num_sms), WT, 0, st>>>(Sb, Sc, n, t, w, status);
    }
    ProfScope ps_("w_build_hashed", st);
    k_w_build<<<pass_grid(k_w_build, n, num_sms), WT, 0, st>>>(Sb, Sc, n, t, w, status);
    return cudaGetLastError();
}

cudaError_t w_table_probe(const int32_t *Ra, const int32_t *Rb, int64_t nR, const WTable &w, int mode,
                          int32_t a_domain, unsigned long long *cnt, unsigned long long *total,
                          DevStatus *status, int num_sms, cudaStream_t st) {
    if (nR <= 0) return cudaSuccess;
    const uint32_t n = (uint32_t)nR;
    if (mode == 1) {
        {
            ProfScope ps_("w_probe_groupby", st);
            k_w_probe_direct<1><<<pass_grid(k_w_probe_direct<1>, n, num_sms), WT, 0, st>>>(
                Ra, Rb, n, w, a_domain, cnt, total, status);
        }
        ProfScope ps_("w_probe_groupby_hashed", st);
        k_w_probe<1><<<pass_grid(k_w_probe<1>, n, num_sms), WT, 0, st>>>(Ra, Rb, n, w, a_domain, cnt, total,
                                                                         status);
    } else {
        {
            ProfScope ps_("w_probe_count", st);
            k_w_probe_direct<0><<<pass_grid(k_w_probe_direct<0>, n, num_sms), WT, 0, st>>>(
                Ra, Rb, n, w, a_domain, cnt, total, status);
        }
        ProfScope ps_("w_probe_count_hashed", st);
        k_w_probe<0><<<pass_grid(k_w_probe<0>, n, num_sms), WT, 0, st>>>(Ra, Rb, n, w, a_domain, cnt, total,
                                                                         status);
    }
    return cudaGetLastError();
}

}  // namespace mwj
