// linear_l2.h -- the linear 3-way join with one bucket on each side: S's
// weight table w(b) = sum over (b, c) in S of deg_T(c), held in the L2.
#pragma once

#include "tables.h"

namespace mwj {

// Open-addressing table of 2^k slots (k from a HyperLogLog estimate of S's
// distinct B values), linear probing from slot_of(b, seed, mask).
//   W[s]        (w(b) mod 2^32) << 32 | b, or kEmpty64 when free; key -1,
//               which would make a full slot look free, lives in W[mask + 1]
//               as a plain 64-bit sum
//   hi[s]       w(b) >> 32 (touched only when some w(b) reaches 2^32)
//   meta[0]     mask; meta[1] the distinct-key estimate; meta[2] set to 1
//               when some hi[] entry is non-zero; meta[3..5] the
//               direct-address layout (tables.h): when the sizing pass chose
//               it, w(b) is the plain 64-bit word W[b - min] and hi[] is unused
struct WTable {
    unsigned long long *W;   // w_table_slots(nS) + 2 entries reserved
    uint32_t *hi;            // w_table_slots(nS) + 2 entries reserved
    uint32_t *meta;          // kMetaWords entries
    uint32_t seed;
    const uint32_t *heavy;   // heavy B keys of S (heavy_detect's table), or null
};

// Heavy keys of the S pass: a sampled share of at least 1 / (2 x this) of S
// (heavy_detect's bucket-count argument).
constexpr uint32_t kWHeavyBuckets = 128;

// Slots to reserve for S of nS tuples (the table never grows past this).
size_t w_table_slots(int64_t nS);

// Size the table from S's B column (hll: hll_scratch_registers(num_sms) u32)
// and clear it; or the two steps apart.
cudaError_t w_table_prepare(const int32_t *Sb, int64_t nS, const WTable &w, unsigned int *hll,
                            uint64_t reserve_slots, int num_sms, cudaStream_t st);
// tmeta (optional): T's single table when its C column is S's B column,
// sized from the same pass (at most treserve slots).
cudaError_t w_table_size(const int32_t *Sb, int64_t nS, const WTable &w, unsigned int *hll,
                         uint64_t reserve_slots, int num_sms, cudaStream_t st, uint32_t *tmeta = nullptr,
                         uint64_t treserve = 0);
cudaError_t w_table_clear(const WTable &w, int num_sms, cudaStream_t st);

// S pass: w(b) += deg_T(c) for every (b, c) of S, T's single table t
// (t.J == 0) already built.
cudaError_t w_table_build(const int32_t *Sb, const int32_t *Sc, int64_t nS, const TImg &t,
                          const WTable &w, DevStatus *status, int num_sms, cudaStream_t st);

// R pass: total += w(b) for every (a, b) of R and, with mode 1 (GROUP BY A),
// cnt[a] += w(b); a outside [0, a_domain) raises MWJ_ERR_DOMAIN.
cudaError_t w_table_probe(const int32_t *Ra, const int32_t *Rb, int64_t nR, const WTable &w, int mode,
                          int32_t a_domain, unsigned long long *cnt, unsigned long long *total,
                          DevStatus *status, int num_sms, cudaStream_t st);

}  // namespace mwj
