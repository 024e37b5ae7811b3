// linear.h -- launch interface of the linear 3-way join kernels.
#pragma once

#include "tables.h"

namespace mwj {

struct LinArgs {
    const uint2 *Rp;            // R grouped by H(b): (a, b)
    const uint32_t *offR;       // I + 1 offsets
    const uint2 *Sp;            // S grouped by (H(b), g(c)): (b, c)
    const uint32_t *offS;       // I * JS + 1 offsets
    uint32_t I, JS;
    TImg t;                     // T's g(C) bucket images
    uint32_t cap_log2;          // on-chip R table: 2^cap_log2 slots
    uint32_t seed_slot;         // slot hash seed of the R table
    int32_t a_domain;
    unsigned long long *cnt;    // GROUP BY A output
    unsigned long long *total;
    unsigned long long *rowcount;   // per R bucket (row output, pass 1), or null
    DevStatus *st;
    uint32_t spin_limit;        // polls of a bounded barrier wait before MWJ_ERR_TIMEOUT
    uint32_t build_s;           // aggregates: 1 = S_i is the on-chip side, 0 = R_i (Algorithm 1)
    // chain of four relations: T's weighted table (16-byte slots, see
    // k_lin_agg_s) instead of T's degrees; null for the 3-way join
    const unsigned long long *tw;
    const uint32_t *tw_meta;    // tw_meta[0] = slot mask
    uint32_t tw_seed;
};

// On-chip side of the aggregate kernels: S_i whenever |S| <= 2 |R|, so that
// every R tuple is read and hashed once; R_i (Algorithm 1's roles) when S is
// much larger than R, where the T lookups of S tuples that meet no R tuple
// would cost more than the second pass over R.
inline uint32_t lin_build_s(int64_t nR, int64_t nS) { return nS <= 2 * nR ? 1u : 0u; }

size_t lin_agg_smem(uint32_t cap_log2, int mode, bool build_s);
size_t lin_rows_smem(uint32_t cap_log2, uint32_t max_tuples);
cudaError_t lin_agg_launch(const LinArgs &g, int mode, cudaStream_t st);
cudaError_t lin_rows_launch(const LinArgs &g, const unsigned long long *base, int32_t *rows,
                            long long capacity, long long *n_rows, uint32_t max_tuples,
                            cudaStream_t st);

}  // namespace mwj
