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
};

size_t lin_agg_smem(uint32_t cap_log2, int mode);
size_t lin_rows_smem(uint32_t cap_log2, uint32_t max_tuples);
cudaError_t lin_agg_launch(const LinArgs &g, int mode, cudaStream_t st);
cudaError_t lin_rows_launch(const LinArgs &g, const unsigned long long *base, int32_t *rows,
                            long long capacity, long long *n_rows, uint32_t max_tuples,
                            cudaStream_t st);

}  // namespace mwj
