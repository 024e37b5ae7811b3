// cyclic.h -- launch interface of the cyclic 3-way join kernels.
#pragma once

#include "common.cuh"

namespace mwj {

struct CycArgs {
    const uint2 *Rp;            // R grouped by (H(a), G(b)): (a, b)
    const uint32_t *offR;       // x*y + 1
    const uint2 *Sp;            // S grouped by (G(b), F(c)): (b, c)
    const uint32_t *offS;       // y*z + 1
    const uint2 *Tp;            // T grouped by (F(c), H(a)): (c, a)
    const uint32_t *offT;       // z*x + 1
    uint32_t x, y, z;
    uint32_t seed_slot, seed_slot2;
    int32_t a_domain;
    unsigned long long *cnt;    // GROUP BY A, or null
    unsigned long long *total;
    DevStatus *st;
};

// ---- shares (1, 1, z): R whole, grouped by B; S and T split by F(c) ----
// R grouped by B: b -> [a] lists.  The sizing pass (tables.h) gives B the
// direct-address layout (entry b - min) or a hashed key table (slot mask + 1
// holds key -1); deg[e] is entry e's list length and, once built, end[e] the
// position after its list in alist.
struct RGroup {
    const uint32_t *meta;   // kMetaWords
    uint32_t *keys;         // hashed layout: mask + 2 entries
    uint32_t *deg;          // entries
    uint32_t *end;          // entries
    int32_t *alist;         // |R|
    uint32_t seed;
};

struct CycCArgs {
    RGroup r;
    const uint2 *Sp;            // S grouped by F(c): (b, c)
    const uint32_t *offS;       // z + 1
    const uint2 *Tp;            // T grouped by F(c): (c, a)
    const uint32_t *offT;       // z + 1
    uint32_t z;
    uint32_t schunk;            // S tuples of a work item at most (cyc_c_schunk)
    const unsigned long long *big_off;   // z + 1: big buckets' set regions (slots), scanned
    const unsigned long long *bigset;    // the regions: one slot per distinct (c, a) pair
    const uint32_t *bigcnt;              // the pairs' multiplicities, at the same indexes
    const uint32_t *big_neg;             // z: (-1, -1) pairs of a big bucket
    uint32_t seed;              // hash of the (c, a) sets
    int32_t a_domain;
    unsigned long long *cnt;    // GROUP BY A, or null
    unsigned long long *total;
    DevStatus *st;
};

// T tuples a bucket's on-chip set holds (larger buckets keep theirs in the L2).
uint32_t cyc_c_tcap();
// S tuples of a work item at most: S_k is split so that a join with few
// buckets (a small T) still gives every probe CTA work.
uint32_t cyc_c_schunk(int64_t nS, int num_sms);
// Slots of the probe CTAs' regions for chunks that repeat (c, a) pairs (the
// rep_set (u64) and rep_cnt (u32) arguments of cyc_c_run).
size_t cyc_c_rep_slots(int num_sms);
// Group R = (a, b) by b (sizing pass over R's B column first).  hll:
// hll_scratch_registers(num_sms) u32; reserve: the entries the arrays hold;
// a_domain > 0: every a must lie in [0, a_domain) (MWJ_ERR_DOMAIN).
cudaError_t rgroup_build(const int32_t *Ra, const int32_t *Rb, int64_t nR, const RGroup &r, unsigned int *hll,
                         uint64_t reserve, unsigned int *bump, int32_t a_domain, DevStatus *status, int num_sms,
                         cudaStream_t st);
// items: z + 1 u32; big_slots: z u64 (scanned into g.big_off, z + 2 u64,
// with scan_tmp64b); g.bigset: 4 |T| + 16 u64 slots, g.bigcnt as many u32;
// g.big_neg: z u32;
// bucket_rows: z + 1 u64, bucket_base: z + 2 u64 (row output); rep_set,
// rep_cnt: cyc_c_rep_slots(num_sms) u64 and u32.
cudaError_t cyc_c_run(const CycCArgs &g, uint32_t *items, void *scan_tmp, unsigned int *counter,
                      unsigned long long *big_slots, void *scan_tmp64b, unsigned long long *bucket_rows,
                      unsigned long long *bucket_base, void *scan_tmp64, int32_t *rows, long long capacity,
                      long long *n_rows, unsigned long long *rep_set, uint32_t *rep_cnt, int num_sms,
                      cudaStream_t st);

uint32_t cyc_rcap();
uint32_t cyc_tcap();
size_t cyc_probe_smem();
// items: x*y*z + 1 u32; counter: 1 u32; tile_rows: x*y*z + 1 u64; tile_base: x*y*z + 2 u64.
cudaError_t cyc_run(const CycArgs &g, uint32_t *items, void *scan_tmp, unsigned int *counter,
                    unsigned long long *tile_rows, unsigned long long *tile_base, void *scan_tmp64,
                    int32_t *rows, long long capacity, long long *n_rows, int num_sms,
                    cudaStream_t st);

}  // namespace mwj
