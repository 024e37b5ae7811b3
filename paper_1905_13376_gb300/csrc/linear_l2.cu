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

namespace mwj {
namespace {

constexpr int WT = 256;     // threads per CTA
constexpr int WQ = 4;       // tuples per lane per warp round: one 128-bit load per column
constexpr uint32_t WCHUNK = 32 * WQ;   // tuples per warp round

// Every run of equal keys in the warp's 128 tuples (lane l holds tuples
// 4l .. 4l+3, in order), summed exactly (modulo 2^64) and handed to
// emit(key, sum) once, by one lane; runs with sum 0 are skipped.  Runs that
// end inside a lane are emitted by it; a run that crosses lanes (through any
// number of lanes holding nothing else) is summed by a segmented inclusive
// scan over the lanes and emitted by the lane where it ends.  Only adjacent
// equal keys merge: sorted inputs get one emission per key and warp, any
// other order is still exact.  Every lane of the warp calls this.
template <typename F>
__device__ __forceinline__ void warp_runs(const int32_t (&k)[WQ], const unsigned long long (&x)[WQ],
                                          uint32_t m, F &&emit) {
    const uint32_t lane = threadIdx.x & 31;
    const bool has = m > 0;
    // the lane's first run (kf, sf) and last run (kl, run); runs between
    // them end inside the lane and are emitted here
    int32_t kf = k[0], kl = k[0];
    unsigned long long sf = 0, run = 0;
    uint32_t nruns = 0;
#pragma unroll
    for (int q = 0; q < WQ; ++q) {
        if ((uint32_t)q < m) {
            if (q > 0 && k[q] != kl) {
                if (nruns == 0)
                    sf = run;
                else if (run)
                    emit(kl, run);
                ++nruns;
                kl = k[q];
                run = 0;
            }
            run += x[q];
        }
    }
    const bool single = (nruns == 0);   // the lane holds one run (or nothing)
    if (single) sf = run;
    // the first run continues the previous lane's last run
    const int32_t pk = __shfl_up_sync(0xffffffffu, kl, 1);
    const int phas = __shfl_up_sync(0xffffffffu, (int)has, 1);
    const bool cont = has && lane > 0 && phas && pk == kf;
    // segmented inclusive scan: a chain starts at a lane that does not
    // continue its predecessor or holds more than one run (its last run
    // starts the chain); lanes of one run that continue it add their sum
    unsigned long long v = has ? run : 0ull;   // single: the lane's only run
    bool head = !(cont && single);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long pv = __shfl_up_sync(0xffffffffu, v, o);
        const int ph = __shfl_up_sync(0xffffffffu, (int)head, o);
        if (lane >= (uint32_t)o && !head) {
            v += pv;
            head = ph != 0;
        }
    }
    const unsigned long long prev = __shfl_up_sync(0xffffffffu, v, 1);   // chain through lane - 1
    const int next_cont = __shfl_down_sync(0xffffffffu, (int)cont, 1);
    if (!has) return;
    if (!single) {   // the first run ends inside this lane
        const unsigned long long s = cont ? prev + sf : sf;
        if (s) emit(kf, s);
    }
    if ((lane == 31 || !next_cont) && v) emit(kl, v);   // the chain ends here
}

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

__global__ void k_w_clear(unsigned long long *__restrict__ W, uint32_t *__restrict__ hi,
                          uint32_t *__restrict__ meta) {
    const uint32_t slots = meta[0] + 1;   // a power of two >= 16
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < slots / 2; s += stride) {
        ((ulonglong2 *)W)[s] = make_ulonglong2(kEmpty64, kEmpty64);
        ((uint2 *)hi)[s] = make_uint2(0u, 0u);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        W[slots] = 0ull;
        hi[slots] = 0u;
        meta[2] = 0u;
    }
}

// S pass.  Warp-uniform loop: a warp takes 128 consecutive tuples per round,
// four per lane, and loads its next round before it works on this one.
// Heavy keys (sampled, see heavy_detect) are summed per CTA in shared
// memory and added to the table once per CTA, so that a key holding a large
// share of S in no particular order does not funnel every warp's adds into
// one L2 word.
__global__ void __launch_bounds__(WT) k_w_build(const int32_t *__restrict__ Sb, const int32_t *__restrict__ Sc,
                                                uint32_t n, TImg t, WTable w, DevStatus *st) {
    __shared__ uint32_t hbuf[kHeavySlots];
    __shared__ unsigned long long hacc[kHeavySlots];
    const uint32_t *hs = heavy_to_smem(w.heavy, hbuf);
    if (hs) {
        for (uint32_t i = threadIdx.x; i < kHeavySlots; i += WT) hacc[i] = 0ull;
        __syncthreads();
    }
    const uint32_t tmask = __ldg(t.meta);
    const uint32_t wmask = __ldg(w.meta);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * WT + threadIdx.x) >> 5, warps = (gridDim.x * WT) >> 5;
    const bool vec = (((uintptr_t)Sb | (uintptr_t)Sc) & 15) == 0;
    const uint64_t pol = l2_evict_first();
    const uint32_t rounds = (n + WCHUNK - 1) / WCHUNK;
    int32_t b[WQ], c[WQ];
    uint32_t m = 0;
    uint32_t r = warp;
    if (r < rounds) m = load_pairs(Sb, Sc, n, r * WCHUNK + lane * WQ, vec, pol, b, c);
    while (r < rounds) {
        const uint32_t nr = r + warps;
        int32_t nb[WQ], nc[WQ];
        uint32_t nm = 0;
        if (nr < rounds) nm = load_pairs(Sb, Sc, n, nr * WCHUNK + lane * WQ, vec, pol, nb, nc);
        uint32_t ts[WQ];
        unsigned long long tv[WQ], x[WQ];
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
        warp_runs(b, x, m, [&](int32_t key, unsigned long long s) { w_add(w, wmask, (uint32_t)key, s, st); });
#pragma unroll
        for (int q = 0; q < WQ; ++q) {
            b[q] = nb[q];
            c[q] = nc[q];
        }
        m = nm;
        r = nr;
    }
    if (hs) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < kHeavySlots; i += WT)
            if (hacc[i]) w_add(w, wmask, hbuf[i], hacc[i], st);
    }
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
template <int MODE>
__global__ void __launch_bounds__(WT) k_w_probe(const int32_t *__restrict__ Ra, const int32_t *__restrict__ Rb,
                                                uint32_t n, WTable w, int32_t a_domain,
                                                unsigned long long *__restrict__ cnt,
                                                unsigned long long *__restrict__ total, DevStatus *st) {
    __shared__ unsigned long long red[32];
    const uint32_t wmask = __ldg(w.meta);
    const bool wide = __ldg(w.meta + 2) != 0;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * WT + threadIdx.x) >> 5, warps = (gridDim.x * WT) >> 5;
    const bool vec = (((uintptr_t)Ra | (uintptr_t)Rb) & 15) == 0;
    const uint64_t pol = l2_evict_first();
    const uint32_t rounds = (n + WCHUNK - 1) / WCHUNK;
    unsigned long long acc = 0;
    int32_t a[WQ], b[WQ];
    uint32_t m = 0;
    uint32_t r = warp;
    if (r < rounds) m = load_pairs(Ra, Rb, n, r * WCHUNK + lane * WQ, vec, pol, a, b);
    while (r < rounds) {
        const uint32_t nr = r + warps;
        int32_t na[WQ], nb[WQ];
        uint32_t nm = 0;
        if (nr < rounds) nm = load_pairs(Ra, Rb, n, nr * WCHUNK + lane * WQ, vec, pol, na, nb);
        uint32_t ws[WQ];
        unsigned long long wv[WQ], x[WQ];
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
        if (MODE == 1) {
#pragma unroll
            for (int q = 0; q < WQ; ++q)
                if ((uint32_t)q < m && (uint32_t)a[q] >= (uint32_t)a_domain)
                    set_status(st, MWJ_ERR_DOMAIN, a[q]);
            warp_runs(a, x, m, [&](int32_t key, unsigned long long s) {
                if ((uint32_t)key < (uint32_t)a_domain) atomicAdd(cnt + key, s);
            });
        }
#pragma unroll
        for (int q = 0; q < WQ; ++q) {
            a[q] = na[q];
            b[q] = nb[q];
        }
        m = nm;
        r = nr;
    }
    acc = block_sum_u64(acc, red);
    if (threadIdx.x == 0 && acc) atomicAdd(total, acc);
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

cudaError_t w_table_prepare(const int32_t *Sb, int64_t nS, const WTable &w, unsigned int *hll,
                            uint64_t reserve_slots, int num_sms, cudaStream_t st) {
    cudaError_t e = single_table_size(Sb, nS, w.seed, hll, w.meta, reserve_slots, num_sms, st, "w_hll",
                                      "w_size");
    if (e != cudaSuccess) return e;
    ProfScope ps_("w_clear", st);
    k_w_clear<<<num_sms * 4, 512, 0, st>>>(w.W, w.hi, w.meta);
    return cudaGetLastError();
}

cudaError_t w_table_build(const int32_t *Sb, const int32_t *Sc, int64_t nS, const TImg &t,
                          const WTable &w, DevStatus *status, int num_sms, cudaStream_t st) {
    if (nS <= 0) return cudaSuccess;
    ProfScope ps_("w_build", st);
    const uint32_t n = (uint32_t)nS;
    k_w_build<<<pass_grid(k_w_build, n, num_sms), WT, 0, st>>>(Sb, Sc, n, t, w, status);
    return cudaGetLastError();
}

cudaError_t w_table_probe(const int32_t *Ra, const int32_t *Rb, int64_t nR, const WTable &w, int mode,
                          int32_t a_domain, unsigned long long *cnt, unsigned long long *total,
                          DevStatus *status, int num_sms, cudaStream_t st) {
    if (nR <= 0) return cudaSuccess;
    const uint32_t n = (uint32_t)nR;
    if (mode == 1) {
        ProfScope ps_("w_probe_groupby", st);
        k_w_probe<1><<<pass_grid(k_w_probe<1>, n, num_sms), WT, 0, st>>>(Ra, Rb, n, w, a_domain, cnt, total,
                                                                         status);
    } else {
        ProfScope ps_("w_probe_count", st);
        k_w_probe<0><<<pass_grid(k_w_probe<0>, n, num_sms), WT, 0, st>>>(Ra, Rb, n, w, a_domain, cnt, total,
                                                                         status);
    }
    return cudaGetLastError();
}

}  // namespace mwj
