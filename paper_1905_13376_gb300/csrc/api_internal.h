// api_internal.h -- the context object and helpers shared by the C-ABI files.
#pragma once

#include <cstdarg>

#include "internal.h"
#include "prof.h"

struct mwj_ctx {
    mwj::DevInfo dev;
    uint32_t seed;
    mwj::Seeds seeds;
    int32_t smem_bytes;
    int32_t load_pct;
    int64_t spin_limit;
    uint32_t cap_log2;        // on-chip R table size (log2 slots)
    mwj::DevStatus *status;   // device status word
    // work of one call that shares no buffer with the rest (T's table while
    // R and S are partitioned) runs on `side`, forked from and joined back
    // to the caller's stream with these events
    cudaStream_t side, side2;
    cudaEvent_t fork, join, join2, heavy_ready;
    mwj::Profiler prof;
    // batch planning rules per kind and size class (mwj_batch_set_rules):
    // R tuples per linear bucket, T table slots per tuple, cyclic fit (%)
    int32_t batch_tpb[2][32], batch_tfac[2][32], batch_fit[2][32];
    int32_t batch_prep_cps, batch_join_cps;   // CTAs per SM (0: the library's choice)
    char err[512];
};

namespace mwj {

const char *status_text(int s);
mwj_status fail(mwj_ctx *ctx, mwj_status s, const char *fmt, ...);
mwj_status cuda_fail(mwj_ctx *ctx, cudaError_t e, const char *where);
bool rel_ok(const mwj_rel &r);
uint32_t pow2_at_least(uint64_t v);
mwj_status check_out(mwj_ctx *ctx, const mwj_out *out, int arity);

mwj_status plan_linear_default(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                               mwj_shares *sh);
mwj_status linear_default_shares(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                                 mwj_mode mode, mwj_shares *sh);
mwj_status plan_cyclic_default(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                               mwj_shares *sh);
mwj_status plan_cyclic_cube(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                            mwj_shares *sh);
mwj_status cyc_workspace(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                         const mwj_shares *shares, mwj_mode mode, size_t *bytes);
mwj_status star_workspace(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                          const mwj_shares *shares, mwj_mode mode, size_t *bytes);
mwj_status plan_star_default(const mwj_rel &R, const mwj_rel &T, mwj_shares *sh);
mwj_status cascade_workspace(mwj_ctx *ctx, int kind, const mwj_rel &R, const mwj_rel &S,
                             const mwj_rel &T, mwj_mode mode, size_t *bytes);

}  // namespace mwj
