// tables.cu -- per-bucket hash-table images of a partitioned relation (K4).
//
// After T is partitioned by g(C) (Algorithm 1, step 1) every bucket T_j is
// aggregated into an open-addressing table image: key c -> deg_T(c) (the
// number of T tuples with that c), and for row output additionally the
// start of c's group in a D-list.  Bucket j's image occupies slots
// [2*off[j], 2*off[j] + cap[j]) of one image array, with cap[j] = 2 x the
// bucket's distinct keys (fill 1/2), so images are 16-byte aligned and can be
// copied into shared memory with one bulk copy.  The probe kernels hold these
// images on chip (in shared memory, or in L2 when T stays whole).
//
// A bucket is first aggregated in a shared-memory table (one CTA per
// bucket); a bucket with more tuples than that table can hold is aggregated
// directly in its global region instead (capacity 2 x its tuples), which
// keeps every input exact whatever its skew.
#include "internal.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr int BT = 512;
constexpr uint32_t kSmemSlots = 8192;   // 64 KB of packed slots

__device__ __forceinline__ void agg_insert(unsigned long long *tbl, uint32_t mask, uint32_t k,
                                           uint32_t seed) {
    uint32_t s = mix32(k ^ seed) & mask;
    const unsigned long long fresh = (1ull << 32) | (unsigned long long)k;
    for (;;) {
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

// insert into a global region of arbitrary capacity (fastrange start)
__device__ __forceinline__ uint32_t gagg_insert(unsigned long long *tbl, uint32_t cap, uint32_t k,
                                                uint32_t seed, unsigned long long add) {
    uint32_t s = fastrange(mix32(k ^ seed), cap);
    const unsigned long long fresh = (add << 32) | (unsigned long long)k;
    for (;;) {
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
                                               int32_t *__restrict__ dlist) {
    extern __shared__ unsigned long long tbl[];   // kSmemSlots
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
        if (2u * n <= kSmemSlots) {
            uint32_t sc = 16;
            while (sc < 2u * n) sc <<= 1;
            const uint32_t mask = sc - 1;
            for (uint32_t s = threadIdx.x; s < sc; s += BT) tbl[s] = kEmpty64;
            __syncthreads();
            for (uint32_t i = o0 + threadIdx.x; i < o1; i += BT)
                agg_insert(tbl, mask, key_of(keys, pairs, i), seed);
            __syncthreads();
            unsigned long long mine = 0;
            for (uint32_t s = threadIdx.x; s < sc; s += BT) mine += (tbl[s] != kEmpty64);
            const uint32_t D = (uint32_t)block_sum_u64(mine, red);
            cap = 2u * D;
            for (uint32_t s = threadIdx.x; s < cap; s += BT) reg[s] = kEmpty64;
            __syncthreads();
            for (uint32_t s = threadIdx.x; s < sc; s += BT) {
                unsigned long long v = tbl[s];
                if (v != kEmpty64) gagg_insert(reg, cap, (uint32_t)v, seed, v >> 32);
            }
        } else {
            cap = 2u * n;
            for (uint32_t s = threadIdx.x; s < cap; s += BT) reg[s] = kEmpty64;
            __syncthreads();
            for (uint32_t i = o0 + threadIdx.x; i < o1; i += BT)
                gagg_insert(reg, cap, key_of(keys, pairs, i), seed, 1ull);
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
                for (;;) {
                    unsigned long long v = reg[s];
                    if (v != kEmpty64 && (uint32_t)v == t.x) break;
                    s = (s + 1 == cap) ? 0 : s + 1;
                }
                uint32_t p = atomicAdd(&sv[s], 1u);
                dlist[p] = (int32_t)t.y;
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

cudaError_t tables_build(const uint32_t *keys, const uint2 *pairs, const uint32_t *off, uint32_t J,
                         uint32_t seed, uint64_t *img, uint32_t *capv, uint32_t *startv,
                         int32_t *dlist, int num_sms, cudaStream_t st) {
    if (J == 0) return cudaSuccess;
    unsigned grid = J < (uint32_t)num_sms * 8 ? J : (unsigned)num_sms * 8;
    const size_t smem = kSmemSlots * sizeof(unsigned long long);
    cudaError_t e;
    if (startv) {
        e = cudaFuncSetAttribute(k_tbuild<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tbuild<true><<<grid, BT, smem, st>>>(keys, pairs, off, J, seed,
                                               (unsigned long long *)img, capv, startv, dlist);
    } else {
        e = cudaFuncSetAttribute(k_tbuild<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tbuild<false><<<grid, BT, smem, st>>>(keys, pairs, off, J, seed,
                                                (unsigned long long *)img, capv, nullptr, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace mwj
