// warp_runs.cuh -- runs of equal keys summed inside a warp.
//
// Edge lists and other relations often arrive sorted by one column, so the
// keys a warp reads in one round come in runs.  Summing each run in
// registers and touching the L2 once per run (instead of once per tuple)
// is what lets the one-bucket passes and T's table build stream at close
// to memory speed on such inputs; any other order stays exact.
#pragma once

#include <cstdint>

namespace mwj {

constexpr int kRunQ = 4;   // keys per lane per warp round (lane l holds keys 4l .. 4l+3)

// Every run of equal keys in the warp's 128 tuples (lane l holds tuples
// 4l .. 4l+3, in order), summed exactly (modulo 2^64) and handed to
// emit(key, sum) once, by one lane; runs with sum 0 are skipped.  Runs that
// end inside a lane are emitted by it; a run that crosses lanes (through any
// number of lanes holding nothing else) is summed by a segmented inclusive
// scan over the lanes and emitted by the lane where it ends.  Only adjacent
// equal keys merge: sorted inputs get one emission per key and warp, any
// other order is still exact.  Every lane of the warp calls this.
template <typename F>
__device__ __forceinline__ void warp_runs(const int32_t (&k)[kRunQ], const unsigned long long (&x)[kRunQ],
                                          uint32_t m, F &&emit) {
    const uint32_t lane = threadIdx.x & 31;
    const bool has = m > 0;
    // the lane's first run (kf, sf) and last run (kl, run); runs between
    // them end inside the lane and are emitted here
    int32_t kf = k[0], kl = k[0];
    unsigned long long sf = 0, run = 0;
    uint32_t nruns = 0;
#pragma unroll
    for (int q = 0; q < kRunQ; ++q) {
        if ((uint32_t)q < m) {
            if (q > 0 && k[q] != kl) {
                if (nruns == 0)
                    sf = run;
                else if (run)
                    emit(kl, run);
                ++nruns;
                kl = k[q];
                run = 0;
            }
            run += x[q];
        }
    }
    const bool single = (nruns == 0);   // the lane holds one run (or nothing)
    if (single) sf = run;
    // the first run continues the previous lane's last run
    const int32_t pk = __shfl_up_sync(0xffffffffu, kl, 1);
    const int phas = __shfl_up_sync(0xffffffffu, (int)has, 1);
    const bool cont = has && lane > 0 && phas && pk == kf;
    // segmented inclusive scan: a chain starts at a lane that does not
    // continue its predecessor or holds more than one run (its last run
    // starts the chain); lanes of one run that continue it add their sum
    unsigned long long v = has ? run : 0ull;   // single: the lane's only run
    bool head = !(cont && single);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long pv = __shfl_up_sync(0xffffffffu, v, o);
        const int ph = __shfl_up_sync(0xffffffffu, (int)head, o);
        if (lane >= (uint32_t)o && !head) {
            v += pv;
            head = ph != 0;
        }
    }
    const unsigned long long prev = __shfl_up_sync(0xffffffffu, v, 1);   // chain through lane - 1
    const int next_cont = __shfl_down_sync(0xffffffffu, (int)cont, 1);
    if (!has) return;
    if (!single) {   // the first run ends inside this lane
        const unsigned long long s = cont ? prev + sf : sf;
        if (s) emit(kf, s);
    }
    if ((lane == 31 || !next_cont) && v) emit(kl, v);   // the chain ends here
}

}  // namespace mwj

namespace mwj {

// The lengths of the runs of equal keys in a warp's block of 128 keys (lane
// l holds positions 4l .. 4l+3, the first m of them valid; the valid
// positions of a block are a prefix).  A run starts where a key differs
// from the one before it (and at the block's first position); it ends at
// the next start or at the first invalid position.  Each lane finds the ends
// of its own runs from its four start flags, and the end of its last run
// from the first later lane that holds a start or an invalid position (one
// ballot, one shuffle).  emit(key, length) is called once per run by the lane
// where it starts.  Runs that continue into the next block are emitted in
// parts.  Every lane of the warp calls this.
template <typename F>
__device__ __forceinline__ void warp_run_lengths(const int32_t (&k)[kRunQ], uint32_t m, F &&emit) {
    const uint32_t lane = threadIdx.x & 31;
    const int32_t prev = __shfl_up_sync(0xffffffffu, k[kRunQ - 1], 1);
    uint32_t start = 0, endm = 0;   // bit q: a run starts / a run ends before position q
#pragma unroll
    for (int q = 0; q < kRunQ; ++q) {
        const bool valid = (uint32_t)q < m;
        const bool s = valid && (q == 0 ? (lane == 0 || k[0] != prev) : k[q] != k[q - 1]);
        start |= (uint32_t)s << q;
        endm |= (uint32_t)(s || !valid) << q;
    }
    const uint32_t any = __ballot_sync(0xffffffffu, endm != 0u);
    const uint32_t later = lane < 31 ? (any & (0xffffffffu << (lane + 1))) : 0u;
    const int nl = later ? __ffs(later) - 1 : -1;
    const uint32_t nnib = __shfl_sync(0xffffffffu, endm, nl < 0 ? 0 : nl);
    const uint32_t block_end = nl < 0 ? 32u * kRunQ : 4u * (uint32_t)nl + (uint32_t)(__ffs(nnib) - 1);
#pragma unroll
    for (int q = 0; q < kRunQ; ++q) {
        if (!((start >> q) & 1u)) continue;
        const uint32_t rest = endm & ~((2u << q) - 1u);   // ends after position q in this lane
        const uint32_t end = rest ? 4u * lane + (uint32_t)(__ffs(rest) - 1) : block_end;
        emit(k[q], end - (4u * lane + (uint32_t)q));
    }
}

}  // namespace mwj
