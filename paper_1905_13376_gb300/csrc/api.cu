// api.cu -- the C ABI of include/mwj.h: argument checks, workspace layout and
// the order of the kernels of each join.
#include <cstdio>
#include <cstring>
#include <string>

#include "api_internal.h"
#include "linear.h"
#include "linear_l2.h"
#include "tables.h"
#include "skew.h"

using namespace mwj;

namespace mwj {

const char *status_text(int s) {
    switch (s) {
        case MWJ_OK: return "ok";
        case MWJ_ERR_INVALID_ARG: return "invalid argument";
        case MWJ_ERR_DOMAIN: return "a value of A lies outside [0, a_domain)";
        case MWJ_ERR_CAPACITY: return "more result rows than the output capacity";
        case MWJ_ERR_WORKSPACE: return "workspace too small";
        case MWJ_ERR_CUDA: return "CUDA error";
        case MWJ_ERR_TIMEOUT: return "a bounded device wait ran out";
        case MWJ_ERR_CHECK: return "device consistency check failed";
        case MWJ_ERR_UNIMPLEMENTED: return "not implemented";
        default: return "unknown status";
    }
}

mwj_status fail(mwj_ctx *ctx, mwj_status s, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

mwj_status cuda_fail(mwj_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, MWJ_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool rel_ok(const mwj_rel &r) {
    if (r.n < 0 || r.n > 0x7FFFFFFFll) return false;
    if (r.n > 0 && (!r.x || !r.y)) return false;
    return true;
}

uint32_t pow2_at_least(uint64_t v) {
    uint32_t p = 1;
    while (p < v && p < (1u << 30)) p <<= 1;
    return p;
}

}  // namespace mwj

// ---------------------------------------------------------------------------
// linear join: workspace layout
// ---------------------------------------------------------------------------
namespace {

struct LinPlan {
    uint32_t I, J, JT;
    bool rows;
    bool single;   // T in one L2-resident table (S not split by C, count modes)
    bool heavy;    // aggregates: heavy B keys split off into one extra bucket
    bool l2;       // aggregates with I = J = 1: S's weight table and T's table in the L2
};

// bucket count of T's tables: small buckets so that each is aggregated in
// one CTA's shared memory; equal to J when S is split by g(C) as well.
uint32_t t_buckets(int64_t nT, uint32_t J, bool single) {
    if (J > 1) return J;
    const uint64_t per = single ? 8192 : 2048;
    uint64_t want = (uint64_t)(nT + per - 1) / per;
    uint32_t p = pow2_at_least(want ? want : 1);
    return p > kMaxBuckets ? kMaxBuckets : p;
}

struct LinLayout {
    uint32_t *heavy; unsigned long long *hw;
    uint2 *Rp; uint32_t *offR;
    uint2 *Sp; uint32_t *offS;
    uint32_t *Tk; uint2 *Tp; uint32_t *offT;
    uint64_t *img; uint32_t *capT; uint32_t *startT; int32_t *dlist;
    uint32_t *ekey, *ecnt, *ecount, *meta;
    unsigned int *hll;
    void *pscratch; size_t pscratch_bytes;
    void *pscratchR;   // single mode: R's own partition scratch (R is partitioned on the side stream)
    unsigned long long *rowcount, *base; void *sscratch;
    WTable w; unsigned int *whll;   // one-bucket plan: S's weight table
};

size_t lin_layout(Arena &A, const LinPlan &p, const mwj_rel &R, const mwj_rel &S,
                  const mwj_rel &T, int num_sms, LinLayout &L) {
    L = LinLayout{};
    if (p.l2) {   // nothing is partitioned: T's table and S's weight table
        L.img = A.take<uint64_t>(single_table_slots(T.n));
        L.meta = A.take<uint32_t>(kMetaWords);
        L.hll = A.take<unsigned int>(hll_scratch_registers(num_sms));
        const size_t ws = w_table_slots(S.n) + 2;
        L.w.W = A.take<unsigned long long>(ws);
        L.w.hi = A.take<uint32_t>(ws);
        L.w.meta = A.take<uint32_t>(kMetaWords);
        L.whll = A.take<unsigned int>(hll_scratch_registers(num_sms));
        L.heavy = A.take<uint32_t>(kHeavyTableWords);
        L.hw = A.take<unsigned long long>(kHeavySlots);
        return A.used;
    }
    const uint32_t extra = p.heavy ? 1u : 0u;   // the heavy-key bucket
    L.heavy = p.heavy ? A.take<uint32_t>(kHeavyTableWords) : nullptr;
    L.hw = p.heavy ? A.take<unsigned long long>(kHeavySlots) : nullptr;
    L.Rp = A.take<uint2>(R.n + 2);
    L.offR = A.take<uint32_t>(p.I + extra + 1);
    L.Sp = A.take<uint2>(S.n + 2);
    L.offS = A.take<uint32_t>((size_t)p.I * p.J + extra + 1);
    if (p.single) {
        // T stays unpartitioned: one table sized from a HyperLogLog estimate
        L.Tk = nullptr;
        L.Tp = nullptr;
        L.offT = nullptr;
        L.img = A.take<uint64_t>(single_table_slots(T.n));
        L.capT = nullptr;
        L.ekey = L.ecnt = L.ecount = nullptr;
        L.meta = A.take<uint32_t>(kMetaWords);
        L.hll = A.take<unsigned int>(hll_scratch_registers(num_sms));
    } else {
        if (p.rows) {
            L.Tk = nullptr;
            L.Tp = A.take<uint2>(T.n + 2);
        } else {
            L.Tk = A.take<uint32_t>(T.n + 4);
            L.Tp = nullptr;
        }
        L.offT = A.take<uint32_t>(p.JT + 1);
        L.hll = nullptr;
        L.img = A.take<uint64_t>(2 * (size_t)T.n + 4);
        L.capT = A.take<uint32_t>(p.JT + 1);
        L.ekey = L.ecnt = L.ecount = L.meta = nullptr;
    }
    if (p.rows) {
        L.startT = A.take<uint32_t>(2 * (size_t)T.n + 4);
        L.dlist = A.take<int32_t>(T.n + 4);
        L.rowcount = A.take<unsigned long long>(p.I + 1);
        L.base = A.take<unsigned long long>(p.I + 2);
        L.sscratch = A.take<char>(scan_scratch_bytes(p.I + 1));
    } else {
        L.startT = nullptr;
        L.dlist = nullptr;
        L.rowcount = L.base = nullptr;
        L.sscratch = nullptr;
    }
    size_t ps = part_scratch_bytes(R.n, p.I + extra, num_sms);
    size_t ps2 = part_scratch_bytes(S.n, p.I * p.J + extra, num_sms);
    size_t ps3 = p.single ? 0 : part_scratch_bytes(T.n, p.JT, num_sms);
    if (ps2 > ps) ps = ps2;
    if (ps3 > ps) ps = ps3;
    L.pscratch = A.take<char>(ps);
    L.pscratch_bytes = ps;
    L.pscratchR = p.single ? A.take<char>(ps) : nullptr;
    return A.used;
}

}  // namespace

namespace mwj {

mwj_status plan_linear_default(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                               mwj_shares *sh) {
    (void)S;
    (void)T;
    // R bucket tables of 2^12 slots hold up to ~2K distinct B values; aim for
    // ~32K tuples of R per bucket and at least four buckets per SM.
    uint64_t want = (uint64_t)(R.n + 32767) / 32768;
    uint64_t minb = (uint64_t)ctx->dev.num_sms * 4;
    if (want < minb) want = minb;
    uint32_t I = pow2_at_least(want);
    if (I > 16384) I = 16384;
    sh->s[0] = (int32_t)I;
    sh->s[1] = 1;
    sh->s[2] = 1;
    return MWJ_OK;
}

// Default shares of mwj_join3_linear.  Aggregates: I = J = 1, the plan in
// which S's weight table and T's table are held whole in the L2 and nothing
// is partitioned.  Rows: the partitioned plan above (the row output needs the
// a-lists of R's buckets in shared memory).
mwj_status linear_default_shares(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                                 mwj_mode mode, mwj_shares *sh) {
    if (mode == MWJ_MATERIALIZE) return plan_linear_default(ctx, R, S, T, sh);
    sh->s[0] = 1;
    sh->s[1] = 1;
    sh->s[2] = 1;
    return MWJ_OK;
}

mwj_status lin_check_shares(mwj_ctx *ctx, const mwj_shares *sh, uint32_t *I, uint32_t *J) {
    if (sh->s[0] < 1 || sh->s[1] < 1) return fail(ctx, MWJ_ERR_INVALID_ARG, "shares must be >= 1");
    if (sh->s[2] > 1 && (sh->s[2] < 9 || sh->s[2] > 14))
        return fail(ctx, MWJ_ERR_INVALID_ARG, "linear shares: s[2] (log2 table slots) must be 9..14");
    uint64_t P = (uint64_t)sh->s[0] * (uint64_t)sh->s[1];
    if ((uint64_t)sh->s[0] > kMaxBuckets || P > kMaxBuckets)
        return fail(ctx, MWJ_ERR_INVALID_ARG, "linear shares: I*J must be <= %u", kMaxBuckets);
    *I = (uint32_t)sh->s[0];
    *J = (uint32_t)sh->s[1];
    return MWJ_OK;
}

}  // namespace mwj

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *mwj_version(void) { return "mwj 0.1 sm_103a"; }

mwj_status mwj_create(mwj_ctx **out, const mwj_config *cfg) {
    if (!out) return MWJ_ERR_INVALID_ARG;
    *out = nullptr;
    mwj_ctx *ctx = new mwj_ctx();
    std::memset(ctx->err, 0, sizeof(ctx->err));
    mwj_config c{};
    if (cfg) c = *cfg;
    int dev = c.device;
    cudaError_t e;
    if (dev < 0) {
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) { delete ctx; return MWJ_ERR_CUDA; }
    }
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) { delete ctx; return MWJ_ERR_CUDA; }
    ctx->dev.device = dev;
    cudaDeviceGetAttribute(&ctx->dev.num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&ctx->dev.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&ctx->dev.cc_major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&ctx->dev.cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
    ctx->seed = c.seed;
    ctx->seeds = make_seeds(c.seed);
    ctx->smem_bytes = c.smem_bytes;
    ctx->load_pct = c.load_pct > 0 ? c.load_pct : 50;
    ctx->spin_limit = c.spin_limit > 0 ? c.spin_limit : (1ll << 26);
    // on-chip R table: 2^cap_log2 slots of 12 bytes (GROUP BY A), default 4096
    ctx->cap_log2 = 12;
    if (c.smem_bytes > 0) {
        uint32_t l = 9;
        while (l < 14 && (12ull << (l + 1)) <= (unsigned long long)c.smem_bytes) ++l;
        ctx->cap_log2 = l;
    }
    e = cudaMalloc(&ctx->status, sizeof(DevStatus));
    if (e != cudaSuccess) { delete ctx; return MWJ_ERR_CUDA; }
    e = cudaMemset(ctx->status, 0, sizeof(DevStatus));
    if (e != cudaSuccess) { cudaFree(ctx->status); delete ctx; return MWJ_ERR_CUDA; }
    for (int k = 0; k < 2; ++k)
        for (int c = 0; c < 32; ++c) {
            ctx->batch_tpb[k][c] = 0;
            ctx->batch_tfac[k][c] = 0;
            ctx->batch_fit[k][c] = 0;
        }
    ctx->batch_prep_cps = ctx->batch_join_cps = 0;
    ctx->side = ctx->side2 = nullptr;
    ctx->fork = ctx->join = ctx->join2 = ctx->heavy_ready = nullptr;
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->side2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->join2, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->heavy_ready, cudaEventDisableTiming) != cudaSuccess) {
        mwj_destroy(ctx);
        return MWJ_ERR_CUDA;
    }
    *out = ctx;
    return MWJ_OK;
}

mwj_status mwj_destroy(mwj_ctx *ctx) {
    if (!ctx) return MWJ_ERR_INVALID_ARG;
    for (cudaStream_t s : {ctx->side, ctx->side2}) {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
    if (ctx->join2) cudaEventDestroy(ctx->join2);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->join) cudaEventDestroy(ctx->join);
    if (ctx->heavy_ready) cudaEventDestroy(ctx->heavy_ready);
    if (ctx->status) cudaFree(ctx->status);
    delete ctx;
    return MWJ_OK;
}

const char *mwj_last_error(mwj_ctx *ctx) { return ctx ? ctx->err : "no context"; }

mwj_status mwj_set_profiling(mwj_ctx *ctx, int enable) {
    if (!ctx) return MWJ_ERR_INVALID_ARG;
    ctx->prof.enable(enable != 0, 1 << 15);
    return MWJ_OK;
}

long long mwj_launch_count(mwj_ctx *ctx) { return ctx ? ctx->prof.launches : -1; }

int mwj_get_phase_times(mwj_ctx *ctx, const char **names, double *ms, long long *launches,
                        int max) {
    if (!ctx) return -1;
    ctx->prof.resolve();
    int i = 0;
    for (auto &kv : ctx->prof.acc) {
        if (i < max) {
            if (names) names[i] = kv.first.c_str();
            if (ms) ms[i] = kv.second.first;
            if (launches) launches[i] = kv.second.second;
        }
        ++i;
    }
    return i;
}

mwj_status mwj_reset_phase_times(mwj_ctx *ctx) {
    if (!ctx) return MWJ_ERR_INVALID_ARG;
    ctx->prof.resolve();
    ctx->prof.acc.clear();
    return MWJ_OK;
}

mwj_status mwj_stream_status(mwj_ctx *ctx, void *stream) {
    if (!ctx) return MWJ_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    DevStatus h{};
    e = cudaMemcpy(&h, ctx->status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
    if (h.code != 0) {
        DevStatus z{};
        cudaMemcpy(ctx->status, &z, sizeof(z), cudaMemcpyHostToDevice);
        return fail(ctx, (mwj_status)h.code, "%s (detail %lld)", status_text(h.code),
                    (long long)h.aux);
    }
    return MWJ_OK;
}

mwj_status mwj_workspace_size(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T,
                              const mwj_shares *shares, mwj_mode mode, size_t *bytes) {
    if (!ctx || !bytes) return MWJ_ERR_INVALID_ARG;
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    if (mode < MWJ_COUNT || mode > MWJ_MATERIALIZE) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad mode");
    mwj_shares sh;
    if (kind == MWJ_LINEAR) {
        if (shares) sh = *shares; else linear_default_shares(ctx, R, S, T, mode, &sh);
        LinPlan p;
        mwj_status s = lin_check_shares(ctx, &sh, &p.I, &p.J);
        if (s != MWJ_OK) return s;
        p.rows = (mode == MWJ_MATERIALIZE);
        p.single = (p.J == 1 && !p.rows);
        p.heavy = !p.rows;
        p.l2 = (p.I == 1 && p.J == 1 && !p.rows);
        p.JT = t_buckets(T.n, p.J, p.single);
        Arena A(nullptr, 0);
        LinLayout L;
        *bytes = lin_layout(A, p, R, S, T, ctx->dev.num_sms, L);
        return MWJ_OK;
    }
    if (kind == MWJ_CYCLIC) return cyc_workspace(ctx, R, S, T, shares, mode, bytes);
    if (kind == 2 + MWJ_LINEAR || kind == 2 + MWJ_CYCLIC)
        return cascade_workspace(ctx, kind - 2, R, S, T, mode, bytes);
    if (kind == MWJ_STAR) return star_workspace(ctx, R, S, T, shares, mode, bytes);
    return fail(ctx, MWJ_ERR_INVALID_ARG, "bad kind %d", kind);
}

mwj_status mwj_join3_linear(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T,
                            const mwj_shares *shares, const mwj_out *out, void *workspace,
                            size_t ws_bytes, void *stream) {
    if (!ctx || !out) return MWJ_ERR_INVALID_ARG;
    ApiScope api_scope(&ctx->prof);
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    mwj_status s = check_out(ctx, out, 4);
    if (s != MWJ_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    mwj_shares sh;
    if (shares) sh = *shares; else linear_default_shares(ctx, R, S, T, out->mode, &sh);
    LinPlan p;
    s = lin_check_shares(ctx, &sh, &p.I, &p.J);
    if (s != MWJ_OK) return s;
    p.rows = (out->mode == MWJ_MATERIALIZE);
    p.single = (p.J == 1 && !p.rows);
    p.heavy = !p.rows;
    p.l2 = (p.I == 1 && p.J == 1 && !p.rows);
    p.JT = t_buckets(T.n, p.J, p.single);
    Arena A(workspace, ws_bytes);
    LinLayout L;
    lin_layout(A, p, R, S, T, ctx->dev.num_sms, L);
    if (A.overflow || !workspace)
        return fail(ctx, MWJ_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, A.used);

    const Seeds &sd = ctx->seeds;
    cudaError_t e;
    if ((e = cudaMemsetAsync(out->total, 0, sizeof(int64_t), st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset total");
    if (out->mode == MWJ_COUNT_GROUP_BY_A &&
        (e = cudaMemsetAsync(out->group_counts, 0, sizeof(int64_t) * (size_t)out->a_domain, st)) !=
            cudaSuccess)
        return cuda_fail(ctx, e, "memset group_counts");
    // With one g(C) bucket T is not partitioned: its C table is built
    // directly, on a side stream, while S is partitioned here and R on a
    // second side stream.
    // On every return after the fork the caller's stream waits for the side
    // stream, so no work of this call outlives it on the caller's stream.
    struct JoinGuard {
        cudaStream_t st;
        cudaEvent_t ev;
        bool armed;
        ~JoinGuard() {
            if (armed) cudaStreamWaitEvent(st, ev, 0);
        }
    } join_guard{st, ctx->join, false}, join_guard2{st, ctx->join2, false};
    // with per-kernel profiling on, everything runs on the caller's stream so
    // that each kernel's event pair times that kernel alone
    cudaStream_t side = ctx->prof.on ? st : ctx->side;
    cudaStream_t side2 = ctx->prof.on ? st : ctx->side2;
    if (p.l2) {
        // T's table on the side stream while S's weight table is sized and
        // cleared here; then the S pass and the R pass.  T's C values and
        // S's B values may get the direct-address layout (only these passes
        // read the two tables).  When T's C column is S's B column (a
        // self-join such as friends of friends of friends) one pass over it
        // sizes both tables.
        L.w.seed = sd.slot;
        L.w.heavy = L.heavy;
        const bool same_keys = T.x == S.x && T.n == S.n;
        if (same_keys) {
            e = w_table_size(S.x, S.n, L.w, L.whll, w_table_slots(S.n), ctx->dev.num_sms, st, L.meta,
                             single_table_slots(T.n));
            if (e != cudaSuccess) return cuda_fail(ctx, e, "table sizes");
        }
        if ((e = cudaEventRecord(ctx->fork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(side, ctx->fork, 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "fork");
        if (same_keys)
            e = single_table_fill(T.x, T.n, sd.slot2, L.meta, L.img, ctx->status, ctx->dev.num_sms, side);
        else
            e = single_table_direct(T.x, T.n, sd.slot2, L.hll, L.meta, L.img, single_table_slots(T.n),
                                    ctx->status, ctx->dev.num_sms, side, true);
        const cudaError_t ej = cudaEventRecord(ctx->join, side);
        if (ej != cudaSuccess) return cuda_fail(ctx, ej, "join");
        join_guard.armed = true;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "T table");
        if ((e = heavy_detect(R.y, R.n, S.x, S.n, kWHeavyBuckets, L.heavy, L.hw, st)) != cudaSuccess)
            return cuda_fail(ctx, e, "heavy keys");
        e = same_keys ? w_table_clear(L.w, ctx->dev.num_sms, st)
                      : w_table_prepare(S.x, S.n, L.w, L.whll, w_table_slots(S.n), ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "S weight table");
        e = cudaStreamWaitEvent(st, ctx->join, 0);
        join_guard.armed = false;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "join");
        const TImg t{L.img, nullptr, nullptr, nullptr, nullptr, L.meta, 0u, sd.C, sd.slot2};
        e = w_table_build(S.x, S.y, S.n, t, L.w, ctx->status, ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "S pass");
        const int mode = out->mode == MWJ_COUNT_GROUP_BY_A ? 1 : 0;
        e = w_table_probe(R.x, R.y, R.n, L.w, mode, out->a_domain, (unsigned long long *)out->group_counts,
                          (unsigned long long *)out->total, ctx->status, ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "R pass");
        return MWJ_OK;
    }
    if (p.single) {
        if ((e = cudaEventRecord(ctx->fork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(side, ctx->fork, 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "fork");
        e = single_table_direct(T.x, T.n, sd.slot2, L.hll, L.meta, L.img, single_table_slots(T.n),
                                ctx->status, ctx->dev.num_sms, side);
        const cudaError_t ej = cudaEventRecord(ctx->join, side);   // whatever was queued
        if (ej != cudaSuccess) return cuda_fail(ctx, ej, "join");
        join_guard.armed = true;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "T tables");
    }
    // Algorithm 1, steps 1-3: T by g(C), S by (H(B), g(C)), R by H(B).
    if (!p.single) {
        PartSpec pt{0, sd.C, p.JT, -1, 0, 1};
        pt.st = ctx->status;
        e = part_run(T.x, T.y, T.n, pt, p.rows ? PAY_PAIR : PAY_X, p.rows ? (void *)L.Tp : (void *)L.Tk,
                     L.offT, L.pscratch, L.pscratch_bytes, ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "partition T");
    }
    // heavy B keys (aggregates): named from samples of R's and S's B columns
    if (p.heavy && (e = heavy_detect(R.y, R.n, S.x, S.n, p.I, L.heavy, L.hw, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "heavy keys");
    // single mode: R is partitioned on the second side stream (its own
    // scratch) once the heavy keys are known, while S is partitioned here
    PartSpec pr{1, sd.B, p.I, -1, 0, 1};
    pr.st = ctx->status;
    pr.heavy = L.heavy;
    if (out->mode == MWJ_COUNT_GROUP_BY_A) pr.dom = (uint32_t)out->a_domain;   // every a of R in the domain
    if (p.single) {
        if ((e = cudaEventRecord(ctx->heavy_ready, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(side2, ctx->heavy_ready, 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "fork");
        e = part_run(R.x, R.y, R.n, pr, PAY_PAIR, L.Rp, L.offR, L.pscratchR, L.pscratch_bytes,
                     ctx->dev.num_sms, side2);
        const cudaError_t ej = cudaEventRecord(ctx->join2, side2);
        if (ej != cudaSuccess) return cuda_fail(ctx, ej, "join");
        join_guard2.armed = true;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "partition R");
    }
    PartSpec ps{0, sd.B, p.I, p.J > 1 ? 1 : -1, sd.C, p.J};
    ps.st = ctx->status;
    ps.heavy = L.heavy;
    e = part_run(S.x, S.y, S.n, ps, PAY_PAIR, L.Sp, L.offS, L.pscratch, L.pscratch_bytes,
                 ctx->dev.num_sms, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "partition S");
    if (!p.single) {
        e = part_run(R.x, R.y, R.n, pr, PAY_PAIR, L.Rp, L.offR, L.pscratch, L.pscratch_bytes,
                     ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "partition R");
    }
    // T's tables
    if (p.single) {
        e = cudaStreamWaitEvent(st, ctx->join, 0);   // T's table is ready
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->join2, 0);   // and R's partitions
        join_guard.armed = join_guard2.armed = false;
    } else
        e = tables_build(L.Tk, L.Tp, L.offT, p.JT, sd.slot2, L.img, L.capT, L.startT, L.dlist,
                         ctx->status, ctx->dev.num_sms, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "T tables");

    LinArgs g{};
    g.Rp = L.Rp; g.offR = L.offR; g.Sp = L.Sp; g.offS = L.offS; g.I = p.I; g.JS = p.J;
    if (p.single)
        g.t = TImg{L.img, nullptr, nullptr, nullptr, nullptr, L.meta, 0u, sd.C, sd.slot2};
    else
        g.t = TImg{L.img, L.offT, L.capT, L.startT, L.dlist, nullptr, p.JT, sd.C, sd.slot2};
    // on-chip R table: 2^s[2] slots when given, else the context's default;
    // row output keeps it at most 2^13 (it also holds the a-lists)
    g.cap_log2 = (sh.s[2] >= 9) ? (uint32_t)sh.s[2] : ctx->cap_log2;
    if (p.rows && g.cap_log2 > 13) g.cap_log2 = 13;
    g.seed_slot = sd.slot;
    g.a_domain = out->a_domain;
    g.cnt = (unsigned long long *)out->group_counts;
    g.total = (unsigned long long *)out->total;
    g.rowcount = L.rowcount;
    g.st = ctx->status;
    g.spin_limit = (uint32_t)(ctx->spin_limit < (1ll << 24) ? ctx->spin_limit : (1ll << 24));
    g.build_s = lin_build_s(R.n, S.n);
    int mode = out->mode == MWJ_COUNT_GROUP_BY_A ? 1 : 0;
    if ((e = lin_agg_launch(g, mode, st)) != cudaSuccess) return cuda_fail(ctx, e, "linear probe");
    if (p.heavy) {   // the heavy-key bucket, after the I light ones
        e = heavy_linear(L.Sp, L.offS, p.I * p.J, L.Rp, L.offR, p.I, L.heavy, g.t, L.hw, out->a_domain,
                         mode == 1 ? (unsigned long long *)out->group_counts : nullptr,
                         (unsigned long long *)out->total, ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "heavy keys");
    }
    if (p.rows) {
        e = scan_excl_u64((const uint64_t *)L.rowcount, (uint64_t *)L.base, p.I, true, L.sscratch, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "row scan");
        e = lin_rows_launch(g, L.base, out->rows, out->capacity, (long long *)out->n_rows, 16384, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "linear rows");
    }
    return MWJ_OK;
}

mwj_status mwj_plan_shares_alt(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T, mwj_shares *shares) {
    if (!ctx || !shares) return MWJ_ERR_INVALID_ARG;
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    if (kind == MWJ_LINEAR) return plan_linear_default(ctx, R, S, T, shares);
    if (kind == MWJ_CYCLIC) return plan_cyclic_cube(ctx, R, S, T, shares);
    return fail(ctx, MWJ_ERR_INVALID_ARG, "bad kind");
}

mwj_status mwj_plan_shares(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T, mwj_mode mode,
                           mwj_shares *shares, void *stream) {
    (void)stream;
    if (!ctx || !shares) return MWJ_ERR_INVALID_ARG;
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    if (kind == MWJ_LINEAR) return linear_default_shares(ctx, R, S, T, mode, shares);
    if (kind == MWJ_CYCLIC) return plan_cyclic_default(ctx, R, S, T, shares);
    if (kind == MWJ_STAR) return plan_star_default(R, T, shares);
    return fail(ctx, MWJ_ERR_INVALID_ARG, "bad kind");
}

}  // extern "C"

namespace mwj {

mwj_status check_out(mwj_ctx *ctx, const mwj_out *out, int arity) {
    if (!out->total) return fail(ctx, MWJ_ERR_INVALID_ARG, "out.total is NULL");
    switch (out->mode) {
        case MWJ_COUNT: return MWJ_OK;
        case MWJ_COUNT_GROUP_BY_A:
            if (!out->group_counts || out->a_domain <= 0)
                return fail(ctx, MWJ_ERR_INVALID_ARG, "group_counts NULL or a_domain <= 0");
            return MWJ_OK;
        case MWJ_MATERIALIZE:
            if (!out->n_rows || out->capacity < 0 || (out->capacity > 0 && !out->rows))
                return fail(ctx, MWJ_ERR_INVALID_ARG, "rows/n_rows/capacity invalid");
            if (arity == 4 && ((uintptr_t)out->rows & 15) != 0)
                return fail(ctx, MWJ_ERR_INVALID_ARG, "linear rows must be 16-byte aligned");
            if (((uintptr_t)out->rows & 3) != 0)
                return fail(ctx, MWJ_ERR_INVALID_ARG, "rows must be 4-byte aligned");
            return MWJ_OK;
        default: return fail(ctx, MWJ_ERR_INVALID_ARG, "bad mode %d", (int)out->mode);
    }
}

}  // namespace mwj
