// tables.h -- bucket table images of a partitioned relation and their lookup.
#pragma once

#include "common.cuh"

namespace mwj {

// Images of T's g(C) buckets: bucket j = bucket_of(c, seed_bucket, J) lives
// at img[2*off[j] .. 2*off[j] + cap[j]) as packed (deg << 32 | c) slots.  With
// row output, start[2*off[j] + slot] is the first position of c's D values in
// dlist (dlist is grouped by bucket, then by key).
struct TImg {
    const uint64_t *img;
    const uint32_t *off;
    const uint32_t *cap;
    const uint32_t *start;
    const int32_t *dlist;
    uint32_t J;
    uint32_t seed_bucket;
    uint32_t seed_slot;
};

__device__ __forceinline__ uint32_t timg_deg(const TImg &t, int32_t c) {
    uint32_t j = (t.J == 1) ? 0u : bucket_of(c, t.seed_bucket, t.J);
    uint64_t base = 2ull * __ldg(t.off + j);
    return img_lookup(t.img + base, __ldg(t.cap + j), (uint32_t)c, t.seed_slot);
}

// deg and start of c (deg 0 when absent)
__device__ __forceinline__ uint32_t timg_deg_start(const TImg &t, int32_t c, uint32_t *start) {
    uint32_t j = (t.J == 1) ? 0u : bucket_of(c, t.seed_bucket, t.J);
    uint64_t base = 2ull * __ldg(t.off + j);
    int64_t s = img_slot(t.img + base, __ldg(t.cap + j), (uint32_t)c, t.seed_slot);
    if (s < 0) return 0;
    uint64_t v = __ldg((const unsigned long long *)(t.img + base + s));
    *start = __ldg(t.start + base + s);
    return (uint32_t)(v >> 32);
}

cudaError_t tables_build(const uint32_t *keys, const uint2 *pairs, const uint32_t *off, uint32_t J,
                         uint32_t seed, uint64_t *img, uint32_t *capv, uint32_t *startv,
                         int32_t *dlist, int num_sms, cudaStream_t st);

}  // namespace mwj
