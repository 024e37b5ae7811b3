// common.cuh -- shared device helpers of the multiway hash join library.
//
// Hashing (Section 4, "robust hash functions"; Fig. 2's two hash levels):
// every attribute has its own seed; the top-level bucket of a key is
// fastrange(mix32(key ^ seed), P) so that any bucket count P works, and the
// slot of a key inside a power-of-two table uses slot_of (Fibonacci hashing:
// one multiply, cheaper than mix32) with a different seed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mwj.h"

namespace mwj {

constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;   // empty slot marker of u32-key tables
constexpr uint64_t kEmpty64 = ~0ull;          // empty slot of packed (val<<32 | key) tables

// Device status word: first error wins.
struct DevStatus {
    int32_t code;
    int32_t pad;
    int64_t aux;
};

__device__ __forceinline__ void set_status(DevStatus *st, int code, int64_t aux = 0) {
    if (atomicCAS(&st->code, 0, code) == 0) st->aux = aux;
}

// "lowbias32" integer finaliser (Wellons' hash-prospector family): a
// bijection of uint32 with good avalanche.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Lemire's multiply-shift range reduction: uniform hash -> [0, n).
__host__ __device__ __forceinline__ uint32_t fastrange(uint32_t h, uint32_t n) {
    return (uint32_t)(((uint64_t)h * (uint64_t)n) >> 32);
}

// Home slot of key k in a table of mask + 1 = 2^L slots: Fibonacci hashing,
// the top L bits of (k ^ seed) * floor(2^32 / phi).  The top bits of the
// product depend on every bit of the key (the low bits only on the key's low
// bits), and a run of consecutive keys lands spread evenly over the table.
__host__ __device__ __forceinline__ uint32_t slot_of(uint32_t k, uint32_t seed, uint32_t mask) {
    return fastrange((k ^ seed) * 0x9E3779B1u, mask + 1u);
}

__host__ __device__ __forceinline__ uint32_t bucket_of(int32_t key, uint32_t seed, uint32_t P) {
    return fastrange(mix32((uint32_t)key ^ seed), P);
}

// Seeds of the per-attribute hash functions (top level) and of the slot hash
// used inside tables.  Derived from the context seed.
struct Seeds {
    uint32_t A, B, C, D, slot, slot2;
};

inline Seeds make_seeds(uint32_t s) {
    Seeds r;
    r.A = mix32(s ^ 0x1b873593u);
    r.B = mix32(s ^ 0x85ebca6bu);
    r.C = mix32(s ^ 0xc2b2ae35u);
    r.D = mix32(s ^ 0x27d4eb2fu);
    r.slot = mix32(s ^ 0x165667b1u);
    r.slot2 = mix32(s ^ 0x9e3779b9u);
    return r;
}

// ---------------------------------------------------------------------------
// Open-addressing table with u32 keys, power-of-two capacity `cap`
// (mask = cap-1), linear probing.  The key value 0xFFFFFFFF (int32 -1) is the
// empty marker, so that key is kept in the extra slot `cap`, whose keys[]
// entry is used as its presence flag.  Arrays are sized cap + 1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tbl_find(const uint32_t *keys, uint32_t mask, uint32_t k,
                                        uint32_t seed) {
    if (k == kEmptyKey) return keys[mask + 1] ? (int)(mask + 1) : -1;
    uint32_t s = slot_of(k, seed, mask);
    for (uint32_t it = 0; it <= mask; ++it) {   // bounded: a full table ends the search
        uint32_t q = keys[s];
        if (q == k) return (int)s;
        if (q == kEmptyKey) return -1;
        s = (s + 1) & mask;
    }
    return -1;
}

// Insert-or-find; returns the slot and sets *fresh when this call claimed it.
// Callers keep the fill below cap; should the table be full anyway the
// search stops after cap probes and returns -1.
__device__ __forceinline__ int tbl_insert(uint32_t *keys, uint32_t mask, uint32_t k,
                                          uint32_t seed, bool *fresh) {
    *fresh = false;
    if (k == kEmptyKey) {
        if (!keys[mask + 1]) {
            if (atomicExch(&keys[mask + 1], 1u) == 0u) *fresh = true;
        }
        return (int)(mask + 1);
    }
    uint32_t s = slot_of(k, seed, mask);
    for (uint32_t it = 0; it <= mask; ++it) {
        uint32_t q = keys[s];
        if (q == k) return (int)s;
        if (q == kEmptyKey) {
            uint32_t old = atomicCAS(&keys[s], kEmptyKey, k);
            if (old == kEmptyKey) { *fresh = true; return (int)s; }
            if (old == k) return (int)s;
        }
        s = (s + 1) & mask;
    }
    return -1;
}

// Tuples per build round for a table of cap slots: at most cap/4, so that a
// round started below 3/4 fill can never fill the table.
__host__ __device__ __forceinline__ uint32_t round_tuples(uint32_t cap, uint32_t max_round) {
    uint32_t r = cap / 4;
    return r < max_round ? r : max_round;
}

// ---------------------------------------------------------------------------
// Packed (count << 32 | key) slots, arbitrary capacity, used for the bucket
// tables of T kept in global memory (images).  kEmpty64 never equals an
// occupied slot because counts stay below 2^31.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t img_lookup(const uint64_t *img, uint32_t cap, uint32_t k,
                                               uint32_t seed) {
    if (cap == 0) return 0;
    uint32_t s = fastrange(mix32(k ^ seed), cap);
    for (uint32_t it = 0; it < cap; ++it) {
        uint64_t v = __ldg((const unsigned long long *)(img + s));
        if (v == kEmpty64) return 0;
        if ((uint32_t)v == k) return (uint32_t)(v >> 32);
        s = (s + 1 == cap) ? 0 : s + 1;
    }
    return 0;
}

// Same lookup returning the slot index (for parallel arrays), -1 if absent.
__device__ __forceinline__ int64_t img_slot(const uint64_t *img, uint32_t cap, uint32_t k,
                                            uint32_t seed) {
    if (cap == 0) return -1;
    uint32_t s = fastrange(mix32(k ^ seed), cap);
    for (uint32_t it = 0; it < cap; ++it) {
        uint64_t v = __ldg((const unsigned long long *)(img + s));
        if (v == kEmpty64) return -1;
        if ((uint32_t)v == k) return (int64_t)s;
        s = (s + 1 == cap) ? 0 : s + 1;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Read-once streams.  Relations and partitions pass through the L2 once; an
// L2 evict_first policy lets them leave before the lookup tables that many
// CTAs share (T's C table), and L1::no_allocate keeps them out of the L1,
// which then caches the hot part of those tables.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ int4 ld_stream(const int4 *ptr, uint64_t pol) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint4 ld_stream(const uint4 *ptr, uint64_t pol) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ void st_stream(uint2 *ptr, uint2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(ptr), "r"(v.x), "r"(v.y),
                 "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void st_stream(uint32_t *ptr, uint32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(ptr), "r"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) {
    atomicAdd(p, v);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies global -> shared (the copy engine of sm_90+), with
// an mbarrier counting the bytes that have landed.  Source and destination
// must be 16-byte aligned and the size a multiple of 16.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the barrier initialisation visible to the copy engine
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait for the phase `parity` of bar; gives up after `limit` polls and
// returns false (the caller records MWJ_ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity,
                                                  uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of a u64 (blockDim.x multiple of 32, <= 1024).  All threads
// receive the result.
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long *scratch32) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch32[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    unsigned long long t = (threadIdx.x < (unsigned)nw) ? scratch32[threadIdx.x] : 0ull;
    if (w == 0) t = warp_sum(t);
    if (threadIdx.x == 0) scratch32[0] = t;
    __syncthreads();
    t = scratch32[0];
    __syncthreads();
    return t;
}

// Block-wide exclusive scan of u32 values (one per thread); returns the
// exclusive prefix, *total gets the block total.  scratch: >= 33 u32.
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *scratch,
                                                        uint32_t *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) scratch[w] = x;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (w == 0) {
        uint32_t s = (lane < nw) ? scratch[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) scratch[lane] = s;   // inclusive warp totals
    }
    __syncthreads();
    uint32_t warp_base = (w > 0) ? scratch[w - 1] : 0u;
    uint32_t tot = scratch[nw - 1];
    __syncthreads();
    if (total) *total = tot;
    return warp_base + x - v;
}

}  // namespace mwj
