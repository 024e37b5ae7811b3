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

uint32_t cyc_rcap();
uint32_t cyc_tcap();
size_t cyc_probe_smem();
// items: x*y*z + 1 u32; counter: 1 u32; tile_rows: x*y*z + 1 u64; tile_base: x*y*z + 2 u64.
cudaError_t cyc_run(const CycArgs &g, uint32_t *items, void *scan_tmp, unsigned int *counter,
                    unsigned long long *tile_rows, unsigned long long *tile_base, void *scan_tmp64,
                    int32_t *rows, long long capacity, long long *n_rows, int num_sms,
                    cudaStream_t st);

}  // namespace mwj
