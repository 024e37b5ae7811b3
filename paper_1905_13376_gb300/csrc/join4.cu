// join4.cu -- the chain of four relations R(A,B) S(B,C) T(C,D) U(D,E),
// COUNT(*) and COUNT(*) GROUP BY A (Section 7: "additional levels of
// hashing beyond two levels").
//
// Algorithm 1 joins three relations with two hash levels: H(B) partitions R
// and S, and T's C side is held whole on chip.  A fourth relation adds one
// more level, on D: U becomes a table of deg_U(d) (L2-resident, sized from a
// HyperLogLog estimate), T a table of weights
//     w_T(c) = sum over T's (c, d) of deg_U(d)
// built by one pass over T against U's table, and the 3-way kernel then
// runs unchanged except that each S tuple (b, c) adds w_T(c) where it added
// deg_T(c):
//     COUNT          = sum over (b,c) in S of deg_R(b) * w_T(c)
//     GROUP BY A     cnt[a] += sum over (b,c) in S of w_T(c)   for (a,b) in R
// which is the definition of the chain's count summed level by level.  No
// intermediate relation is materialised; every relation is read once.
#include "api_internal.h"
#include "linear.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr int WB = 256;   // threads per CTA of the table kernels

__global__ void k_wt_clear(unsigned long long *__restrict__ tw, const uint32_t *__restrict__ meta) {
    const uint64_t words = 2ull * ((uint64_t)meta[0] + 1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x)
        tw[i] = 0ull;
}

// deg_U(d) from U's packed single table
__device__ __forceinline__ uint32_t udeg(const unsigned long long *tu, uint32_t mask, uint32_t seed,
                                         uint32_t d) {
    uint32_t s = slot_of(d, seed, mask);
    for (uint32_t it = 0; it <= mask; ++it) {
        const unsigned long long x = __ldg(tu + s);
        if (x == kEmpty64) return 0;
        if ((uint32_t)x == d) return (uint32_t)(x >> 32);
        s = (s + 1) & mask;
    }
    return 0;
}

// w_T(c) += v in T's weighted table (16-byte slots: word 0 = 1 << 32 | c,
// word 1 = weight).  The table has at least 4x the estimated distinct keys;
// should it be full anyway the insert is dropped and MWJ_ERR_CHECK recorded.
__device__ __forceinline__ void tw_add(unsigned long long *tw, uint32_t mask, uint32_t seed, uint32_t c,
                                       unsigned long long v, DevStatus *st) {
    const unsigned long long want = (1ull << 32) | c;
    uint32_t s = slot_of(c, seed, mask);
    for (uint32_t it = 0; it <= mask; ++it) {
        unsigned long long x = *(volatile unsigned long long *)(tw + 2 * (size_t)s);
        if (x == 0ull) {
            x = atomicCAS(tw + 2 * (size_t)s, 0ull, want);
            if (x == 0ull) x = want;
        }
        if (x == want) {
            atomicAdd(tw + 2 * (size_t)s + 1, v);
            return;
        }
        s = (s + 1) & mask;
    }
    set_status(st, MWJ_ERR_CHECK, 8);
}

// One pass over T: every (c, d) adds deg_U(d) to w_T(c); each thread takes 8
// consecutive tuples, looks up their 8 degrees together and merges runs of
// equal c before touching the table.
__global__ void __launch_bounds__(WB) k_wt_build(const int32_t *__restrict__ tc, const int32_t *__restrict__ td,
                                                 uint32_t n, const unsigned long long *__restrict__ tu,
                                                 const uint32_t *__restrict__ umeta, uint32_t useed,
                                                 unsigned long long *__restrict__ tw,
                                                 const uint32_t *__restrict__ wmeta, uint32_t wseed,
                                                 DevStatus *st) {
    const uint32_t umask = __ldg(umeta), wmask = __ldg(wmeta);
    constexpr uint32_t K = 8;
    const uint32_t stride = gridDim.x * WB * K;
    for (uint32_t i = (blockIdx.x * WB + threadIdx.x) * K; i < n; i += stride) {
        const uint32_t m = min(K, n - i);
        uint32_t c[K], dg[K];
#pragma unroll
        for (uint32_t k = 0; k < K; ++k) {
            c[k] = k < m ? (uint32_t)__ldg(tc + i + k) : 0u;
            dg[k] = k < m ? udeg(tu, umask, useed, (uint32_t)__ldg(td + i + k)) : 0u;
        }
        uint32_t cur = c[0];
        unsigned long long run = 0;
#pragma unroll
        for (uint32_t k = 0; k < K; ++k) {
            if (k >= m) break;
            if (c[k] != cur) {
                if (run) tw_add(tw, wmask, wseed, cur, run, st);
                cur = c[k];
                run = 0;
            }
            run += dg[k];
        }
        if (run) tw_add(tw, wmask, wseed, cur, run, st);
    }
}

struct J4Layout {
    uint2 *Rp, *Sp;
    uint32_t *offR, *offS;
    uint64_t *tu;
    uint32_t *umeta;
    unsigned long long *tw;
    uint32_t *wmeta;
    unsigned int *hll;
    void *pscratch;
    size_t pscratch_bytes;
};

size_t j4_layout(Arena &A, uint32_t I, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                 const mwj_rel &U, int num_sms, J4Layout &L) {
    L.Rp = A.take<uint2>(R.n + 2);
    L.offR = A.take<uint32_t>(I + 1);
    L.Sp = A.take<uint2>(S.n + 2);
    L.offS = A.take<uint32_t>(I + 1);
    L.tu = A.take<uint64_t>(single_table_slots(U.n));
    L.umeta = A.take<uint32_t>(4);
    L.tw = A.take<unsigned long long>(2 * single_table_slots(T.n));
    L.wmeta = A.take<uint32_t>(4);
    L.hll = A.take<unsigned int>(hll_scratch_registers(num_sms));
    size_t ps = part_scratch_bytes(R.n, I, num_sms);
    const size_t ps2 = part_scratch_bytes(S.n, I, num_sms);
    if (ps2 > ps) ps = ps2;
    L.pscratch = A.take<char>(ps);
    L.pscratch_bytes = ps;
    return A.used;
}

mwj_status j4_shares(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                     const mwj_shares *shares, uint32_t *I, uint32_t *cap_log2) {
    mwj_shares sh;
    if (shares) sh = *shares; else plan_linear_default(ctx, R, S, T, &sh);
    if (sh.s[0] < 1 || (uint32_t)sh.s[0] > kMaxBuckets)
        return fail(ctx, MWJ_ERR_INVALID_ARG, "4-relation chain: s[0] must be in [1, %u]", kMaxBuckets);
    if (sh.s[1] != 1) return fail(ctx, MWJ_ERR_INVALID_ARG, "4-relation chain: s[1] must be 1");
    if (sh.s[2] > 1 && (sh.s[2] < 9 || sh.s[2] > 14))
        return fail(ctx, MWJ_ERR_INVALID_ARG, "4-relation chain: s[2] (log2 table slots) must be 9..14");
    *I = (uint32_t)sh.s[0];
    *cap_log2 = sh.s[2] >= 9 ? (uint32_t)sh.s[2] : ctx->cap_log2;
    return MWJ_OK;
}

}  // namespace
}  // namespace mwj

using namespace mwj;

extern "C" mwj_status mwj_join4_workspace_size(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T, mwj_rel U,
                                               const mwj_shares *shares, mwj_mode mode, size_t *bytes) {
    if (!ctx || !bytes) return MWJ_ERR_INVALID_ARG;
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T) || !rel_ok(U))
        return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    if (mode != MWJ_COUNT && mode != MWJ_COUNT_GROUP_BY_A)
        return fail(ctx, MWJ_ERR_INVALID_ARG, "4-relation chain: COUNT or COUNT GROUP BY A only");
    uint32_t I, cl;
    mwj_status s = j4_shares(ctx, R, S, T, shares, &I, &cl);
    if (s != MWJ_OK) return s;
    Arena A(nullptr, 0);
    J4Layout L;
    *bytes = j4_layout(A, I, R, S, T, U, ctx->dev.num_sms, L);
    return MWJ_OK;
}

extern "C" mwj_status mwj_join4_linear(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T, mwj_rel U,
                                       const mwj_shares *shares, const mwj_out *out, void *workspace,
                                       size_t ws_bytes, void *stream) {
    if (!ctx || !out) return MWJ_ERR_INVALID_ARG;
    ApiScope api_scope(&ctx->prof);
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T) || !rel_ok(U))
        return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    mwj_status s = check_out(ctx, out, 4);
    if (s != MWJ_OK) return s;
    if (out->mode != MWJ_COUNT && out->mode != MWJ_COUNT_GROUP_BY_A)
        return fail(ctx, MWJ_ERR_INVALID_ARG, "4-relation chain: COUNT or COUNT GROUP BY A only");
    uint32_t I, cap_log2;
    if ((s = j4_shares(ctx, R, S, T, shares, &I, &cap_log2)) != MWJ_OK) return s;
    Arena A(workspace, ws_bytes);
    J4Layout L;
    j4_layout(A, I, R, S, T, U, ctx->dev.num_sms, L);
    if (A.overflow || !workspace)
        return fail(ctx, MWJ_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, A.used);

    cudaStream_t st = (cudaStream_t)stream;
    const Seeds &sd = ctx->seeds;
    const int sms = ctx->dev.num_sms;
    const uint32_t useed = sd.D ^ sd.slot2;
    cudaError_t e;
    if ((e = cudaMemsetAsync(out->total, 0, sizeof(int64_t), st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset total");
    if (out->mode == MWJ_COUNT_GROUP_BY_A &&
        (e = cudaMemsetAsync(out->group_counts, 0, sizeof(int64_t) * (size_t)out->a_domain, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset group_counts");
    // level D: U's degrees
    if ((e = single_table_direct(U.x, U.n, useed, L.hll, L.umeta, L.tu, single_table_slots(U.n), ctx->status,
                                 sms, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "U table");
    // level C: T's weights w_T(c) = sum of deg_U(d)
    if ((e = single_table_size(T.x, T.n, sd.slot2, L.hll, L.wmeta, single_table_slots(T.n), sms, st)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "T table size");
    {
        ProfScope ps_("t_clear", st);
        k_wt_clear<<<sms * 4, 512, 0, st>>>(L.tw, L.wmeta);
    }
    if (T.n > 0) {
        ProfScope ps_("t_weights", st);
        const uint64_t groups = ((uint64_t)T.n + 8 * WB - 1) / (8 * WB);
        const unsigned grid = (unsigned)(groups < (uint64_t)sms * 8 ? groups : (uint64_t)sms * 8);
        k_wt_build<<<grid, WB, 0, st>>>(T.x, T.y, (uint32_t)T.n, (const unsigned long long *)L.tu, L.umeta,
                                        useed, L.tw, L.wmeta, sd.slot2, ctx->status);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "T weights");
    // level B: R and S by H(B), as in the 3-way join
    PartSpec ps{0, sd.B, I, -1, 0, 1};
    ps.st = ctx->status;
    if ((e = part_run(S.x, S.y, S.n, ps, PAY_PAIR, L.Sp, L.offS, L.pscratch, L.pscratch_bytes, sms, st)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "partition S");
    PartSpec pr{1, sd.B, I, -1, 0, 1};
    pr.st = ctx->status;
    if (out->mode == MWJ_COUNT_GROUP_BY_A) pr.dom = (uint32_t)out->a_domain;
    if ((e = part_run(R.x, R.y, R.n, pr, PAY_PAIR, L.Rp, L.offR, L.pscratch, L.pscratch_bytes, sms, st)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "partition R");
    LinArgs g{};
    g.Rp = L.Rp; g.offR = L.offR; g.Sp = L.Sp; g.offS = L.offS; g.I = I; g.JS = 1;
    g.t = TImg{nullptr, nullptr, nullptr, nullptr, nullptr, L.wmeta, 0u, sd.C, sd.slot2};
    g.cap_log2 = cap_log2;
    g.seed_slot = sd.slot;
    g.a_domain = out->a_domain;
    g.cnt = (unsigned long long *)out->group_counts;
    g.total = (unsigned long long *)out->total;
    g.rowcount = nullptr;
    g.st = ctx->status;
    g.spin_limit = (uint32_t)(ctx->spin_limit < (1ll << 24) ? ctx->spin_limit : (1ll << 24));
    g.build_s = 1;   // S_i on chip: the weighted table is looked up per S tuple
    g.tw = L.tw;
    g.tw_meta = L.wmeta;
    g.tw_seed = sd.slot2;
    if ((e = lin_agg_launch(g, out->mode == MWJ_COUNT_GROUP_BY_A ? 1 : 0, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "chain probe");
    return MWJ_OK;
}
