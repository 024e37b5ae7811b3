// tables.cu -- hash tables of T's C values (K4).
//
// After T is partitioned by g(C) (Algorithm 1, step 1) the probe needs, for
// each c, deg_T(c) = |{(c,d) in T}| (count modes) or c's group of D values
// (row output).  Two layouts:
//
//  * one table ("T held whole on chip", used when S is not split by C):
//    every bucket T_j is aggregated in shared memory (one CTA per bucket,
//    32-bit atomics), its (c, count) entries are appended to a compact list,
//    and the entries are then inserted into a single open-addressing table of
//    2^k >= 2 x (entries) packed (count << 32 | c) slots that stays resident
//    in L2.  A probe is one 8-byte load in the common case.
//  * bucket images (S split by (H(B), g(C)), and row output): bucket j's
//    table occupies slots [2*off[j], 2*off[j] + cap[j]) of one image array,
//    cap[j] = 2 x its distinct keys, 16-byte aligned so that it can be copied
//    into shared memory in one bulk copy.  With row output a parallel start[]
//    array gives the first position of c's D values in dlist.
//
// A bucket whose distinct keys overflow the shared-memory table is handled
// in pieces (the table is flushed and restarted), and the global insert adds
// the partial counts together, so any skew stays exact.
#include <climits>

#include "internal.h"
#include "tables.h"
#include "warp_runs.cuh"

namespace mwj {
namespace {

constexpr int BT = 512;
constexpr uint32_t kAggSlots = 8192;          // shared-memory aggregation table
// Slots of the single T table per estimated distinct C value: the power of
// two at or above 4 x the estimate keeps the load between 1/8 and 1/4 (a
// factor of 2 measured slower: longer probe runs in both insert and lookup).
constexpr double kSingleTableFactor = 4.0;
constexpr uint32_t kImgSmemSlots = 8192;      // 64 KB of packed slots (bucket images)

// insert into a global region of arbitrary capacity (fastrange start), adding `add`
__device__ __forceinline__ uint32_t gagg_insert(unsigned long long *tbl, uint32_t cap, uint32_t k,
                                                uint32_t seed, unsigned long long add,
                                                DevStatus *st) {
    uint32_t s = fastrange(mix32(k ^ seed), cap);
    const unsigned long long fresh = (add << 32) | (unsigned long long)k;
    for (uint32_t it = 0; it < cap; ++it) {
        unsigned long long v = tbl[s];
        if (v == kEmpty64) {
            unsigned long long old = atomicCAS(&tbl[s], kEmpty64, fresh);
            if (old == kEmpty64) return s;
            v = old;
        }
        if ((uint32_t)v == k) {
            atomicAdd(&tbl[s], add << 32);
            return s;
        }
        s = (s + 1 == cap) ? 0 : s + 1;
    }
    set_status(st, MWJ_ERR_CHECK, 2);   // sized to stay half empty: cannot happen
    return 0;
}

// insert into the power-of-two single table
__device__ __forceinline__ void single_insert(unsigned long long *tbl, uint32_t mask, uint32_t k,
                                              uint32_t seed, unsigned long long add,
                                              DevStatus *st) {
    uint32_t s = slot_of(k, seed, mask);
    const unsigned long long fresh = (add << 32) | (unsigned long long)k;
    for (uint32_t it = 0; it <= mask; ++it) {
        unsigned long long v = tbl[s];
        if (v == kEmpty64) {
            unsigned long long old = atomicCAS(&tbl[s], kEmpty64, fresh);
            if (old == kEmpty64) return;
            v = old;
        }
        if ((uint32_t)v == k) {
            atomicAdd(&tbl[s], add << 32);
            return;
        }
        s = (s + 1) & mask;
    }
    set_status(st, MWJ_ERR_CHECK, 3);
}

// ---------------------------------------------------------------------------
// single table
// ---------------------------------------------------------------------------

// One CTA per bucket: aggregate the bucket's keys in shared memory and append
// (key, count) entries to ekey/ecnt at the bucket's tuple offset.
__global__ void __launch_bounds__(BT) k_tagg(const uint32_t *__restrict__ keys,
                                             const uint32_t *__restrict__ off, uint32_t J,
                                             uint32_t seed, uint32_t *__restrict__ ekey,
                                             uint32_t *__restrict__ ecnt,
                                             uint32_t *__restrict__ ecount, DevStatus *st) {
    extern __shared__ uint32_t sm[];
    uint32_t *tk = sm;                         // kAggSlots + 1 keys
    uint32_t *tc = sm + kAggSlots + 1;         // kAggSlots + 1 counts
    __shared__ uint32_t nd, nout;
    const uint32_t mask = kAggSlots - 1;
    for (uint32_t j = blockIdx.x; j < J; j += gridDim.x) {
        const uint32_t o0 = off[j], o1 = off[j + 1];
        if (threadIdx.x == 0) nout = 0;
        uint32_t pos = o0;
        while (pos < o1) {
            for (uint32_t s = threadIdx.x; s <= kAggSlots; s += BT) {
                tk[s] = (s < kAggSlots) ? kEmptyKey : 0u;
                tc[s] = 0u;
            }
            if (threadIdx.x == 0) nd = 0;
            // rounds of rt keys while the table stays at most 3/4 full
            const uint32_t rt = round_tuples(kAggSlots, 4 * BT);
            for (;;) {
                __syncthreads();
                const uint32_t filled = nd;
                __syncthreads();
                if (pos >= o1 || filled + rt > kAggSlots - kAggSlots / 4) break;
                uint32_t fresh_n = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t li = threadIdx.x + k * BT;
                    uint32_t i = pos + li;
                    if (li < rt && i < o1) {
                        bool fresh;
                        int s = tbl_insert(tk, mask, __ldg(keys + i), seed, &fresh);
                        if (s < 0) {
                            set_status(st, MWJ_ERR_CHECK, 4);
                            continue;
                        }
                        fresh_n += fresh;
                        atomicAdd(&tc[s], 1u);
                    }
                }
                fresh_n = warp_sum(fresh_n);
                if ((threadIdx.x & 31) == 0 && fresh_n) atomicAdd(&nd, fresh_n);
                pos += rt;
            }
            // flush the table's entries
            for (uint32_t s = threadIdx.x; s <= kAggSlots; s += BT) {
                uint32_t c = tc[s];
                if (c) {
                    uint32_t k = (s < kAggSlots) ? tk[s] : kEmptyKey;
                    uint32_t p = atomicAdd(&nout, 1u);
                    ekey[o0 + p] = k;
                    ecnt[o0 + p] = c;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) ecount[j] = nout;
        __syncthreads();
    }
}

// Sum of the entry counts (one CTA) and the table's power-of-two mask.
__global__ void k_tsize(const uint32_t *__restrict__ ecount, uint32_t J, uint32_t *__restrict__ meta) {
    __shared__ unsigned long long red[32];
    unsigned long long s = 0;
    for (uint32_t j = threadIdx.x; j < J; j += blockDim.x) s += ecount[j];
    s = block_sum_u64(s, red);
    if (threadIdx.x == 0) {
        unsigned long long cap = 16;
        while (cap < 2 * s) cap <<= 1;
        meta[0] = (uint32_t)(cap - 1);   // mask
        meta[1] = (uint32_t)s;
        meta[kMetaDense] = 0u;           // hashed slots
    }
}

// Empty hashed slots, or zero degrees of the direct-address layout.
__global__ void k_tclear(unsigned long long *__restrict__ tbl, const uint32_t *__restrict__ meta) {
    const bool dense = meta[kMetaDense] != 0u;
    const uint64_t words = dense ? ((uint64_t)meta[kMetaSpan] + 1) / 2 : (uint64_t)meta[0] + 1;
    const unsigned long long fill = dense ? 0ull : kEmpty64;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < words;
         s += (uint64_t)gridDim.x * blockDim.x)
        tbl[s] = fill;
}

__global__ void __launch_bounds__(BT) k_tinsert(const uint32_t *__restrict__ ekey,
                                                const uint32_t *__restrict__ ecnt,
                                                const uint32_t *__restrict__ off,
                                                const uint32_t *__restrict__ ecount, uint32_t J,
                                                uint32_t seed, unsigned long long *__restrict__ tbl,
                                                const uint32_t *__restrict__ meta, DevStatus *st) {
    const uint32_t mask = meta[0];
    for (uint32_t j = blockIdx.x; j < J; j += gridDim.x) {
        const uint32_t o0 = off[j], e = ecount[j];
        for (uint32_t i = threadIdx.x; i < e; i += BT)
            single_insert(tbl, mask, ekey[o0 + i], seed, ecnt[o0 + i], st);
    }
}

// ---------------------------------------------------------------------------
// bucket images
// ---------------------------------------------------------------------------

__device__ __forceinline__ void img_agg_insert(unsigned long long *tbl, uint32_t mask, uint32_t k,
                                               uint32_t seed) {
    uint32_t s = mix32(k ^ seed) & mask;
    const unsigned long long fresh = (1ull << 32) | (unsigned long long)k;
    for (uint32_t it = 0; it <= mask; ++it) {   // sized >= 2x the bucket: never full
        unsigned long long v = tbl[s];
        if (v == kEmpty64) {
            unsigned long long old = atomicCAS(&tbl[s], kEmpty64, fresh);
            if (old == kEmpty64) return;
            v = old;
        }
        if ((uint32_t)v == k) {
            atomicAdd(&tbl[s], 1ull << 32);
            return;
        }
        s = (s + 1) & mask;
    }
}

__device__ __forceinline__ uint32_t key_of(const uint32_t *keys, const uint2 *pairs, uint32_t i) {
    return keys ? keys[i] : pairs[i].x;
}

// One CTA per bucket.  keys (count modes) or pairs (row mode, (c,d)).
template <bool CSR>
__global__ void __launch_bounds__(BT) k_tbuild(const uint32_t *__restrict__ keys,
                                               const uint2 *__restrict__ pairs,
                                               const uint32_t *__restrict__ off, uint32_t J,
                                               uint32_t seed, unsigned long long *__restrict__ img,
                                               uint32_t *__restrict__ capv,
                                               uint32_t *__restrict__ startv,
                                               int32_t *__restrict__ dlist, DevStatus *st) {
    extern __shared__ unsigned long long tbl[];   // kImgSmemSlots
    __shared__ unsigned long long red[32];
    for (uint32_t j = blockIdx.x; j < J; j += gridDim.x) {
        const uint32_t o0 = off[j], o1 = off[j + 1];
        const uint32_t n = o1 - o0;
        unsigned long long *reg = img + 2ull * o0;
        uint32_t cap;
        if (n == 0) {
            if (threadIdx.x == 0) capv[j] = 0;
            continue;
        }
        if (2u * n <= kImgSmemSlots) {
            uint32_t sc = 16;
            while (sc < 2u * n) sc <<= 1;
            const uint32_t mask = sc - 1;
            for (uint32_t s = threadIdx.x; s < sc; s += BT) tbl[s] = kEmpty64;
            __syncthreads();
            for (uint32_t i = o0 + threadIdx.x; i < o1; i += BT)
                img_agg_insert(tbl, mask, key_of(keys, pairs, i), seed);
            __syncthreads();
            unsigned long long mine = 0;
            for (uint32_t s = threadIdx.x; s < sc; s += BT) mine += (tbl[s] != kEmpty64);
            const uint32_t D = (uint32_t)block_sum_u64(mine, red);
            cap = 2u * D;
            for (uint32_t s = threadIdx.x; s < cap; s += BT) reg[s] = kEmpty64;
            __syncthreads();
            for (uint32_t s = threadIdx.x; s < sc; s += BT) {
                unsigned long long v = tbl[s];
                if (v != kEmpty64) gagg_insert(reg, cap, (uint32_t)v, seed, v >> 32, st);
            }
        } else {
            cap = 2u * n;
            for (uint32_t s = threadIdx.x; s < cap; s += BT) reg[s] = kEmpty64;
            __syncthreads();
            for (uint32_t i = o0 + threadIdx.x; i < o1; i += BT)
                gagg_insert(reg, cap, key_of(keys, pairs, i), seed, 1ull, st);
        }
        if (threadIdx.x == 0) capv[j] = cap;
        __syncthreads();
        if (CSR) {
            // starts: exclusive scan of the degrees over the image's slots, as
            // absolute positions in dlist, used first as fill cursors
            uint32_t *sv = startv + 2ull * o0;
            __shared__ uint32_t scan_scratch[33];
            __shared__ uint32_t carry;
            if (threadIdx.x == 0) carry = o0;
            __syncthreads();
            for (uint32_t b = 0; b < cap; b += BT) {
                uint32_t s = b + threadIdx.x;
                unsigned long long v = (s < cap) ? reg[s] : kEmpty64;
                uint32_t d = (v == kEmpty64) ? 0u : (uint32_t)(v >> 32);
                uint32_t tot;
                uint32_t ex = block_excl_scan_u32(d, scan_scratch, &tot);
                if (s < cap) sv[s] = carry + ex;
                __syncthreads();
                if (threadIdx.x == 0) carry += tot;
                __syncthreads();
            }
            for (uint32_t i = o0 + threadIdx.x; i < o1; i += BT) {
                uint2 t = pairs[i];
                // plain loads: the image was written earlier in this kernel
                uint32_t s = fastrange(mix32(t.x ^ seed), cap);
                bool found = false;
                for (uint32_t it = 0; it < cap; ++it) {
                    unsigned long long v = reg[s];
                    if (v != kEmpty64 && (uint32_t)v == t.x) { found = true; break; }
                    s = (s + 1 == cap) ? 0 : s + 1;
                }
                if (!found) {
                    set_status(st, MWJ_ERR_CHECK, 5);
                    continue;
                }
                uint32_t p = atomicAdd(&sv[s], 1u);
                if (p >= o0 && p < o1) dlist[p] = (int32_t)t.y;
                else set_status(st, MWJ_ERR_CHECK, 6);
            }
            __syncthreads();
            for (uint32_t s = threadIdx.x; s < cap; s += BT) {
                unsigned long long v = reg[s];
                if (v != kEmpty64) sv[s] -= (uint32_t)(v >> 32);
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t single_table_slots(int64_t nT) {
    uint64_t cap = 16;
    while (cap < 2 * (uint64_t)(nT > 0 ? nT : 1)) cap <<= 1;
    return cap;
}

cudaError_t single_table_build(const uint32_t *keys, const uint32_t *off, uint32_t J, uint32_t seed,
                               uint32_t *ekey, uint32_t *ecnt, uint32_t *ecount, uint32_t *meta,
                               uint64_t *tbl, DevStatus *status, int num_sms, cudaStream_t st) {
    unsigned grid = J < (uint32_t)num_sms * 4 ? J : (unsigned)num_sms * 4;
    if (grid == 0) grid = 1;
    const size_t smem = 2 * (kAggSlots + 1) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_tagg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (J > 0) {
        ProfScope ps_("t_aggregate", st);
        k_tagg<<<grid, BT, smem, st>>>(keys, off, J, seed, ekey, ecnt, ecount, status);
    }
    {
        ProfScope ps_("t_size", st);
        k_tsize<<<1, 1024, 0, st>>>(ecount, J, meta);
    }
    {
        ProfScope ps_("t_clear", st);
        k_tclear<<<num_sms * 4, 512, 0, st>>>((unsigned long long *)tbl, meta);
    }
    if (J > 0) {
        ProfScope ps_("t_insert", st);
        k_tinsert<<<grid, BT, 0, st>>>(ekey, ecnt, off, ecount, J, seed, (unsigned long long *)tbl,
                                       meta, status);
    }
    return cudaGetLastError();
}

cudaError_t tables_build(const uint32_t *keys, const uint2 *pairs, const uint32_t *off, uint32_t J,
                         uint32_t seed, uint64_t *img, uint32_t *capv, uint32_t *startv,
                         int32_t *dlist, DevStatus *status, int num_sms, cudaStream_t st) {
    if (J == 0) return cudaSuccess;
    unsigned grid = J < (uint32_t)num_sms * 8 ? J : (unsigned)num_sms * 8;
    const size_t smem = kImgSmemSlots * sizeof(unsigned long long);
    cudaError_t e;
    if (startv) {
        e = cudaFuncSetAttribute(k_tbuild<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ProfScope ps_("table_build_csr", st);
        k_tbuild<true><<<grid, BT, smem, st>>>(keys, pairs, off, J, seed,
                                               (unsigned long long *)img, capv, startv, dlist,
                                               status);
    } else {
        e = cudaFuncSetAttribute(k_tbuild<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ProfScope ps_("table_build", st);
        k_tbuild<false><<<grid, BT, smem, st>>>(keys, pairs, off, J, seed,
                                                (unsigned long long *)img, capv, nullptr, nullptr,
                                                status);
    }
    return cudaGetLastError();
}

}  // namespace mwj

// ---------------------------------------------------------------------------
// single table without partitioning T: size it from a HyperLogLog estimate
// of T's distinct C values, then insert T's C column directly
// ---------------------------------------------------------------------------
namespace mwj {
namespace {

constexpr int HLL_BITS = 12;
constexpr uint32_t HLL_M = 1u << HLL_BITS;
constexpr int HLL_CTAS_PER_SM = 2;   // resident CTAs of the sizing pass (its registers allow two)

// HyperLogLog registers (Flajolet, Fusy, Gandouet, Meunier 2007): register
// h >> (32 - HLL_BITS) keeps the largest rank (position of the first 1 bit)
// of the remaining bits.  mix32 is a bijection of 32-bit keys, so distinct
// keys have distinct hashes.
// With mm != null the CTA also leaves the smallest and largest key it saw in
// mm[2 b], mm[2 b + 1] (b = blockIdx.x; INT32_MAX, INT32_MIN when it saw none).
__global__ void __launch_bounds__(BT, HLL_CTAS_PER_SM) k_hll(const int32_t *__restrict__ keys, uint32_t n,
                                            uint32_t seed, unsigned int *__restrict__ regs,
                                            unsigned int *__restrict__ done, int32_t *__restrict__ mm) {
    __shared__ unsigned int r[HLL_M];
    __shared__ int32_t smin, smax;
    if (done && blockIdx.x == 0 && threadIdx.x == 0) *done = 0;   // for k_hll_merge_size
    for (uint32_t j = threadIdx.x; j < HLL_M; j += BT) r[j] = 0;
    if (threadIdx.x == 0) {
        smin = INT32_MAX;
        smax = INT32_MIN;
    }
    int32_t kmin = INT32_MAX, kmax = INT32_MIN;
    __syncthreads();
    const bool vec = ((uintptr_t)keys & 15) == 0;
    const uint64_t pol = l2_evict_first();
    // strips of 16 consecutive keys, one per thread and iteration (four
    // 16-byte loads), so that a run of equal keys (edge lists come sorted by
    // source) costs one register update per strip: a register only grows, so
    // a key equal to its predecessor changes nothing.  The next strip's loads
    // are issued before this one is used.
    const uint32_t nst = (n + 15) / 16;
    const uint32_t T = gridDim.x * BT;
    auto load = [&](uint32_t c, int32_t (&v)[16]) -> uint32_t {
        if (c >= nst) return 0u;
        const uint32_t i = c * 16;
        const uint32_t cnt = min(16u, n - i);
        if (cnt == 16 && vec) {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int4 q = ld_stream((const int4 *)(keys + i) + g, pol);
                v[4 * g] = q.x; v[4 * g + 1] = q.y; v[4 * g + 2] = q.z; v[4 * g + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = ((uint32_t)k < cnt) ? __ldg(keys + i + k) : 0;
        }
        return cnt;
    };
    int32_t v[16];
    uint32_t c = blockIdx.x * BT + threadIdx.x;
    uint32_t cnt = load(c, v);
    for (; c < nst; c += T) {
        int32_t nv[16];
        const uint32_t ncnt = load(c + T, nv);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if ((uint32_t)k >= cnt) break;
            if (k > 0 && v[k] == v[k - 1]) continue;   // nothing a repeat could change
            kmin = min(kmin, v[k]);
            kmax = max(kmax, v[k]);
            const uint32_t h = mix32((uint32_t)v[k] ^ seed);
            const uint32_t w = h << HLL_BITS;
            const uint32_t rank = (w == 0) ? (33u - HLL_BITS) : (uint32_t)__clz(w) + 1u;
            unsigned int *reg = &r[h >> (32 - HLL_BITS)];
            if (*(volatile unsigned int *)reg < rank) atomicMax(reg, rank);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = nv[k];
        cnt = ncnt;
    }
    if (mm) {
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&smin, kmin);
            atomicMax(&smax, kmax);
        }
    }
    __syncthreads();
    // this CTA's registers; the size kernel takes the maximum over CTAs
    for (uint32_t j = threadIdx.x; j < HLL_M; j += BT) regs[(size_t)blockIdx.x * HLL_M + j] = r[j];
    if (mm && threadIdx.x == 0) {
        mm[2 * blockIdx.x] = smin;
        mm[2 * blockIdx.x + 1] = smax;
    }
}

// regs[0..HLL_M) = max over the rows of regs[ctas][HLL_M]
__global__ void k_hll_merge(unsigned int *__restrict__ regs, uint32_t ctas) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= HLL_M) return;
    unsigned int m = 0;
    for (uint32_t c = 0; c < ctas; ++c) m = max(m, regs[(size_t)c * HLL_M + j]);
    regs[j] = m;
}

constexpr uint32_t HLL_MB = 32;                  // registers merged per CTA
constexpr uint32_t HLL_MCTAS = HLL_M / HLL_MB;   // merge CTAs
// after the per-CTA registers: per merge CTA its part of the estimator's sum
// (double) and of the empty-register count, then the finish counter
constexpr size_t HLL_TAIL = 2 * HLL_MCTAS + HLL_MCTAS + 8;

// Merge the per-CTA registers (maximum over `rows` rows) into row 0 and size
// the table: CTA b merges registers [32 b, 32 b + 32) and leaves its part of
// sum(2^-reg) and of the zero count; the last CTA to finish adds the parts
// in a fixed order (so the estimate does not depend on the finishing order)
// and writes meta: table of 2^k >= factor x estimate slots (at most
// `reserve`).  With per-CTA key ranges kr (rows pairs, or null) the keys may
// instead get the direct-address layout (slot = key - min, no key stored)
// when their span max - min + 1 is at most the hashed table's slot count:
// the keys then fill at least 1/(2 factor) of the span, the array is no
// larger than the hashed table and a lookup is one load with no probing.
constexpr int HLL_MW = 32;   // warps of a merge CTA, each over every HLL_MW-th row

__global__ void __launch_bounds__(HLL_MW * 32) k_hll_merge_size(unsigned int *__restrict__ regs, uint32_t rows,
                                                        unsigned int *__restrict__ tail, uint64_t reserve,
                                                        double factor, uint32_t *__restrict__ meta,
                                                        const int32_t *__restrict__ kr,
                                                        uint32_t *__restrict__ meta2, uint64_t reserve2) {
    __shared__ unsigned int m[HLL_MW][HLL_MB];
    __shared__ bool last;
    double *part_s = (double *)tail;
    unsigned int *part_z = tail + 2 * HLL_MCTAS;
    unsigned int *done = part_z + HLL_MCTAS;
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t j = blockIdx.x * HLL_MB + lane;
    // eight rows in flight per thread: the rows are independent loads
    unsigned int mx = 0;
    uint32_t r = w;
    for (; r + 7 * HLL_MW < rows; r += 8 * HLL_MW) {
        unsigned int v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(regs + (size_t)(r + HLL_MW * u) * HLL_M + j);
#pragma unroll
        for (int u = 0; u < 8; ++u) mx = max(mx, v[u]);
    }
    for (; r < rows; r += HLL_MW) mx = max(mx, __ldcg(regs + (size_t)r * HLL_M + j));
    m[w][lane] = mx;
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 1; q < HLL_MW; ++q) mx = max(mx, m[q][lane]);
        regs[j] = mx;
        double sum = 1.0 / (double)(1ull << mx);   // exact: ranks are at most 33 - HLL_BITS
        unsigned int z = (mx == 0);
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            z += __shfl_xor_sync(0xffffffffu, z, o);
        }
        if (lane == 0) {
            part_s[blockIdx.x] = sum;
            part_z[blockIdx.x] = z;
            __threadfence();
            last = atomicAdd(done, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last CTA: the parts in a fixed order (lane l adds parts l, l + 32,
    // ... in turn, then a fixed butterfly), and the key ranges with all threads
    __shared__ int32_t rlo[HLL_MW], rhi[HLL_MW];
    double S = 0.0;
    unsigned int Z = 0;
    if (w == 0) {
        for (uint32_t b = lane; b < gridDim.x; b += 32) {
            S += __ldcg(part_s + b);
            Z += __ldcg(part_z + b);
        }
        for (int o = 16; o > 0; o >>= 1) {
            S += __shfl_xor_sync(0xffffffffu, S, o);
            Z += __shfl_xor_sync(0xffffffffu, Z, o);
        }
    }
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    if (kr) {
        for (uint32_t b = threadIdx.x; b < rows; b += blockDim.x) {
            lo = min(lo, __ldcg(kr + 2 * b));
            hi = max(hi, __ldcg(kr + 2 * b + 1));
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            rlo[w] = lo;
            rhi[w] = hi;
        }
        __syncthreads();
        for (uint32_t q = 0; q < blockDim.x / 32; ++q) {
            lo = min(lo, rlo[q]);
            hi = max(hi, rhi[q]);
        }
    }
    if (threadIdx.x != 0) return;
    const double mm = (double)HLL_M;
    double E = (0.7213 / (1.0 + 1.079 / mm)) * mm * mm / S;
    if (E <= 2.5 * mm && Z > 0) E = mm * log(mm / (double)Z);   // small-range correction
    // meta2 (optional): a second table of the same keys, at most reserve2 slots
    for (int t = 0; t < 2; ++t) {
        uint32_t *mt = t ? meta2 : meta;
        const uint64_t res = t ? reserve2 : reserve;
        if (!mt) continue;
        uint64_t cap = 16;
        while ((double)cap < factor * E && cap < res) cap <<= 1;
        if (cap > res) cap = res;
        mt[0] = (uint32_t)(cap - 1);
        mt[1] = (uint32_t)E;
        uint32_t dense = 0u;
        if (kr) {
            const int64_t span = (int64_t)hi - (int64_t)lo + 1;
            if (lo <= hi && (uint64_t)span <= cap) {
                dense = 1u;
                mt[kMetaMin] = (uint32_t)lo;
                mt[kMetaSpan] = (uint32_t)span;
            }
        }
        mt[kMetaDense] = dense;
    }
    *done = 0;
}

// Insert T's C column.  A warp round is four blocks of 128 consecutive keys
// (four per lane), all loaded, with the next round's loads issued, before
// they are used; every run of equal keys in a block is measured once by
// warp_run_lengths and added to its entry once:
// hashed slots through single_insert, the direct-address layout as
// deg[c - min] += run with a 32-bit add whose result is not needed.
__global__ void __launch_bounds__(BT) k_tinsert_direct(const int32_t *__restrict__ keys, uint32_t n,
                                                       uint32_t seed, unsigned long long *__restrict__ tbl,
                                                       const uint32_t *__restrict__ meta, DevStatus *st) {
    const uint32_t mask = meta[0];
    const bool dense = meta[kMetaDense] != 0u;
    const uint32_t kmin = dense ? meta[kMetaMin] : 0u, span = dense ? meta[kMetaSpan] : 0u;
    uint32_t *deg = (uint32_t *)tbl;
    const bool vec = ((uintptr_t)keys & 15) == 0;
    const uint64_t pol = l2_evict_first();
    constexpr uint32_t CH = 32 * kRunQ;   // keys of one warp_runs block
    constexpr int G = 4;                  // blocks per warp round, loaded together
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * BT + threadIdx.x) >> 5, warps = (gridDim.x * BT) >> 5;
    const uint32_t blocks = (n + CH - 1) / CH;
    const uint32_t rounds = (blocks + G - 1) / G;
    auto load = [&](uint32_t blk, int32_t (&v)[kRunQ]) -> uint32_t {
        const uint32_t i = blk * CH + lane * kRunQ;
        if (blk >= blocks || i >= n) return 0u;
        if (vec && i + kRunQ <= n) {
            const int4 a = ld_stream((const int4 *)(keys + i), pol);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            return kRunQ;
        }
        const uint32_t m = min((uint32_t)kRunQ, n - i);
#pragma unroll
        for (int q = 0; q < kRunQ; ++q)
            if ((uint32_t)q < m) v[q] = __ldg(keys + i + q);
        return m;
    };
    auto emit = [&](int32_t key, uint32_t run) {
        const uint32_t k = (uint32_t)key;
        if (!dense)
            single_insert(tbl, mask, k, seed, (uint32_t)run, st);
        else if (k - kmin < span)
            atomicAdd(deg + (k - kmin), (uint32_t)run);
        else
            set_status(st, MWJ_ERR_CHECK, 8);   // a key outside the range the sizing pass saw
    };
    int32_t v[G][kRunQ];
    uint32_t m[G];
    uint32_t r = warp;
#pragma unroll
    for (int g = 0; g < G; ++g) m[g] = load(r * G + g, v[g]);
    while (r < rounds) {
        const uint32_t nr = r + warps;
        int32_t nv[G][kRunQ];
        uint32_t nm[G];
#pragma unroll
        for (int g = 0; g < G; ++g) nm[g] = load(nr * G + g, nv[g]);
#pragma unroll
        for (int g = 0; g < G; ++g) warp_run_lengths(v[g], m[g], emit);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            m[g] = nm[g];
#pragma unroll
            for (int q = 0; q < kRunQ; ++q) v[g][q] = nv[g][q];
        }
        r = nr;
    }
}

}  // namespace

cudaError_t single_table_size(const int32_t *keys, int64_t n, uint32_t seed, unsigned int *hll_regs,
                              uint32_t *meta, uint64_t reserve_slots, int num_sms, cudaStream_t st,
                              const char *hll_name, const char *size_name, bool allow_dense,
                              uint32_t *meta2, uint64_t reserve2) {
    cudaError_t e;
    const uint32_t nn = (uint32_t)n;
    const uint32_t ctas = (uint32_t)num_sms * HLL_CTAS_PER_SM;
    unsigned int *tail = hll_regs + (size_t)ctas * HLL_M;
    unsigned int *done = tail + 3 * HLL_MCTAS;
    int32_t *mm = (allow_dense && nn > 0) ? (int32_t *)(tail + HLL_TAIL) : nullptr;
    uint32_t rows = ctas;
    if (nn > 0) {
        ProfScope ps_(hll_name, st);
        k_hll<<<ctas, BT, 0, st>>>(keys, nn, seed, hll_regs, done, mm);
    } else {
        rows = 1;
        if ((e = cudaMemsetAsync(hll_regs, 0, HLL_M * sizeof(unsigned int), st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(done, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    }
    ProfScope ps_(size_name, st);
    k_hll_merge_size<<<HLL_MCTAS, HLL_MW * 32, 0, st>>>(hll_regs, rows, tail, reserve_slots, kSingleTableFactor,
                                                         meta, mm, meta2, reserve2);
    return cudaGetLastError();
}

cudaError_t single_table_direct(const int32_t *keys, int64_t n, uint32_t seed, unsigned int *hll_regs,
                                uint32_t *meta, uint64_t *tbl, uint64_t reserve_slots,
                                DevStatus *status, int num_sms, cudaStream_t st, bool allow_dense) {
    cudaError_t e;
    if ((e = single_table_size(keys, n, seed, hll_regs, meta, reserve_slots, num_sms, st, "t_hll", "t_size",
                               allow_dense)) != cudaSuccess)
        return e;
    return single_table_fill(keys, n, seed, meta, tbl, status, num_sms, st);
}

cudaError_t single_table_fill(const int32_t *keys, int64_t n, uint32_t seed, const uint32_t *meta,
                              uint64_t *tbl, DevStatus *status, int num_sms, cudaStream_t st) {
    const uint32_t nn = (uint32_t)n;
    {
        ProfScope ps_("t_clear", st);
        k_tclear<<<num_sms * 4, 512, 0, st>>>((unsigned long long *)tbl, meta);
    }
    if (nn > 0) {
        ProfScope ps_("t_insert", st);
        const uint32_t groups = (nn + 4 * kRunQ * BT - 1) / (4 * kRunQ * BT);
        const uint32_t grid = groups < (uint32_t)num_sms * 4 ? groups : (uint32_t)num_sms * 4;
        k_tinsert_direct<<<grid, BT, 0, st>>>(keys, nn, seed, (unsigned long long *)tbl, meta, status);
    }
    return cudaGetLastError();
}

uint32_t hll_registers() { return HLL_M; }

cudaError_t hll_regs(const int32_t *keys, int64_t n, uint32_t seed, unsigned int *regs, int num_sms,
                     cudaStream_t st) {
    cudaError_t e;
    if (n > 0) {
        const uint32_t ctas = (uint32_t)num_sms * HLL_CTAS_PER_SM;
        {
            ProfScope ps_("sketch_hll", st);
            k_hll<<<ctas, BT, 0, st>>>(keys, (uint32_t)n, seed, regs, nullptr, nullptr);
        }
        ProfScope ps_("sketch_hll_merge", st);
        k_hll_merge<<<(HLL_M + 255) / 256, 256, 0, st>>>(regs, ctas);
    } else if ((e = cudaMemsetAsync(regs, 0, HLL_M * sizeof(unsigned int), st)) != cudaSuccess) {
        return e;
    }
    return cudaGetLastError();
}

size_t hll_scratch_registers(int num_sms) {
    const size_t ctas = (size_t)num_sms * HLL_CTAS_PER_SM;
    return ctas * HLL_M + HLL_TAIL + 2 * ctas;   // registers, sizing tail, per-CTA key ranges
}

}  // namespace mwj
