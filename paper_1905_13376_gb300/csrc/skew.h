// skew.h -- heavy join keys: detection, partition routing, and the
// aggregate kernels of the heavy bucket.
#pragma once

#include "tables.h"

namespace mwj {

// Heavy-key table: kHeavySlots keys (open addressing, home slot
// slot_of(key, kHeavySeed, kHeavySlots - 1), kEmptyKey = empty) followed by
// the number of keys; at most kHeavyMax keys.
constexpr uint32_t kHeavySlots = 512;
constexpr uint32_t kHeavyMax = 256;
constexpr uint32_t kHeavySeed = 0x2545F491u;
constexpr size_t kHeavyTableWords = kHeavySlots + 4;

// Slot of key k in the heavy table (a copy in shared memory), -1 if absent.
// Not inlined: the partition kernels call it only when the table holds keys,
// and an inlined probe loop at every bucket computation of their unrolled
// loops would crowd the instruction cache of the common, heavy-free case.
static __device__ __noinline__ int heavy_slot(const uint32_t *hs, uint32_t k) {
    if (k == kEmptyKey) return -1;
    uint32_t s = slot_of(k, kHeavySeed, kHeavySlots - 1);
    for (uint32_t it = 0; it < kHeavySlots; ++it) {
        const uint32_t q = hs[s];
        if (q == k) return (int)s;
        if (q == kEmptyKey) return -1;
        s = (s + 1) & (kHeavySlots - 1);
    }
    return -1;
}

// Copy a heavy table into shared memory (every thread of the CTA calls this;
// ends with a barrier when it copies).  Returns null when there is no table
// or it holds no key, so that callers skip the per-tuple check.
__device__ __forceinline__ const uint32_t *heavy_to_smem(const uint32_t *heavy, uint32_t *buf) {
    if (!heavy || __ldg(heavy + kHeavySlots) == 0) return nullptr;
    for (uint32_t i = threadIdx.x; i < kHeavySlots; i += blockDim.x) buf[i] = __ldg(heavy + i);
    __syncthreads();
    return buf;
}

// Heavy keys of the join column B from samples of R's and S's B columns: a
// key is heavy when its sampled share in either relation reaches half of an
// average H(B) bucket (1 / (2 I)).  Also zeroes hw (kHeavySlots u64).
cudaError_t heavy_detect(const int32_t *rb, int64_t nR, const int32_t *sb, int64_t nS, uint32_t I,
                         uint32_t *heavy, unsigned long long *hw, cudaStream_t st);

// The heavy bucket (index hb of the partitions) of the linear aggregates:
// hw[h] = sum of deg_T(c) over S tuples (h, c), then for R tuples (a, h):
// total += hw[h] and (GROUP BY A) cnt[a] += hw[h].
cudaError_t heavy_linear(const uint2 *Sp, const uint32_t *offS, uint32_t hbS, const uint2 *Rp,
                         const uint32_t *offR, uint32_t hbR, const uint32_t *heavy, const TImg &T,
                         unsigned long long *hw, int32_t a_domain, unsigned long long *cnt,
                         unsigned long long *total, int num_sms, cudaStream_t st);

}  // namespace mwj
