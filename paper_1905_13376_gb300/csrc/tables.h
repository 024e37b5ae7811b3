// tables.h -- T's tables (one L2-resident table, or per-bucket images) and their lookup.
#pragma once

#include "common.cuh"

namespace mwj {

// Words of a single table's meta array: mask of the hashed slots, distinct
// estimate, a flag of the weight table (see linear_l2.h), and, when the
// sizing pass chose the direct-address layout (kMetaDense = 1), the smallest
// key and the span of the keys: the entry of key k is then at k - min,
// nothing is hashed and no key is stored.
constexpr int kMetaMask = 0, kMetaEst = 1, kMetaWide = 2, kMetaDense = 3, kMetaMin = 4, kMetaSpan = 5;
constexpr int kMetaWords = 8;

// J == 0: one table of (meta[0] + 1) packed (deg << 32 | c) slots, home slot
//         slot_of(c, seed_slot, meta[0]); or, with meta[kMetaDense], a
//         uint32 deg[] over [min, min + span) (only the one-bucket plan of
//         linear_l2.cu asks for that layout).
// J >= 1: bucket j = bucket_of(c, seed_bucket, J) lives at
//         img[2*off[j] .. 2*off[j] + cap[j]); with row output start[2*off[j] + slot]
//         is the first position of c's D values in dlist.
struct TImg {
    const uint64_t *img;
    const uint32_t *off;
    const uint32_t *cap;
    const uint32_t *start;
    const int32_t *dlist;
    const uint32_t *meta;
    uint32_t J;
    uint32_t seed_bucket;
    uint32_t seed_slot;
};

__device__ __forceinline__ uint32_t timg_deg(const TImg &t, int32_t c) {
    if (t.J == 0) {
        const uint32_t mask = __ldg(t.meta);
        uint32_t s = slot_of((uint32_t)c, t.seed_slot, mask);
        for (uint32_t it = 0; it <= mask; ++it) {
            uint64_t v = __ldg((const unsigned long long *)(t.img + s));
            if (v == kEmpty64) return 0;
            if ((uint32_t)v == (uint32_t)c) return (uint32_t)(v >> 32);
            s = (s + 1) & mask;
        }
        return 0;
    }
    uint32_t j = (t.J == 1) ? 0u : bucket_of(c, t.seed_bucket, t.J);
    uint64_t base = 2ull * __ldg(t.off + j);
    return img_lookup(t.img + base, __ldg(t.cap + j), (uint32_t)c, t.seed_slot);
}

// deg and start of c (deg 0 when absent); bucket images only
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
                         int32_t *dlist, DevStatus *status, int num_sms, cudaStream_t st);

// slots to reserve for the single table of nT tuples (worst case)
size_t single_table_slots(int64_t nT);
// ekey/ecnt: nT entries each; ecount: J; meta: at least 4 words (the layout
// flag, kMetaDense, is written too).
cudaError_t single_table_build(const uint32_t *keys, const uint32_t *off, uint32_t J, uint32_t seed,
                               uint32_t *ekey, uint32_t *ecnt, uint32_t *ecount, uint32_t *meta,
                               uint64_t *tbl, DevStatus *status, int num_sms, cudaStream_t st);

// One table without partitioning T: a HyperLogLog pass over the keys sizes
// the table (2^k >= 4 x the estimate, at most reserve_slots), then the keys
// are inserted directly.  hll_regs: hll_scratch_registers(num_sms) u32 (per-CTA
// registers, then the sizing step's partial sums, then per-CTA key ranges);
// meta: at least 4 u32, kMetaWords when allow_dense.
// allow_dense: the keys may get the direct-address layout (meta words above);
// meta must then hold kMetaWords words.
cudaError_t single_table_direct(const int32_t *keys, int64_t n, uint32_t seed, unsigned int *hll_regs,
                                uint32_t *meta, uint64_t *tbl, uint64_t reserve_slots,
                                DevStatus *status, int num_sms, cudaStream_t st, bool allow_dense = false);
// The second step of single_table_direct: clear the table meta describes
// and insert the keys.
cudaError_t single_table_fill(const int32_t *keys, int64_t n, uint32_t seed, const uint32_t *meta,
                              uint64_t *tbl, DevStatus *status, int num_sms, cudaStream_t st);
// Only the sizing step of single_table_direct: meta[0] = mask of a table of
// 2^k >= 4 x (estimated distinct keys) slots (at most reserve_slots).
// hll_name, size_name: the two launches' names in the per-kernel profile.
// With meta2 != null a second table of the same keys (at most reserve2
// slots) is sized in the same launch.
cudaError_t single_table_size(const int32_t *keys, int64_t n, uint32_t seed, unsigned int *hll_regs,
                              uint32_t *meta, uint64_t reserve_slots, int num_sms, cudaStream_t st,
                              const char *hll_name = "t_hll", const char *size_name = "t_size",
                              bool allow_dense = false, uint32_t *meta2 = nullptr, uint64_t reserve2 = 0);
uint32_t hll_registers();
size_t hll_scratch_registers(int num_sms);
// HyperLogLog registers of keys[0, n) into regs[0, hll_registers()); regs must
// hold hll_scratch_registers(num_sms) u32 (per-CTA registers, then merged)
cudaError_t hll_regs(const int32_t *keys, int64_t n, uint32_t seed, unsigned int *regs, int num_sms,
                     cudaStream_t st);

}  // namespace mwj
