// star.cu -- the star 3-way join R(A,B) S(B,C) T(C,D) (Section 6, "linear
// star 3-way join"): the dimension relations R and T are small enough to be
// held on chip, so one level of hashing suffices and the large fact relation
// S is streamed exactly once.
//
// The paper maps each (h(b), g(c)) pair of hash values to one memory unit,
// loads R and T into the units first and then routes every S tuple to the
// unit of its pair.  On this GPU the on-chip memory that every SM can reach
// is the L2 (with the L1 in front of it).  For the two aggregates R and T
// each become one table of their keys' degrees (b -> deg_R(b), c ->
// deg_T(c)), sized from a HyperLogLog estimate of the distinct keys and
// filled without partitioning; for row output R is grouped by h(B) and T by
// g(C) into bucket tables that also hold the lists b -> [a] and c -> [d].
// Either way the tables stay resident in the L2, and every CTA streams its
// own contiguous stretch of S straight from the input columns, looking each
// tuple up in both tables:
//
//   COUNT(*)             total += deg_R(b) * deg_T(c)            per S tuple
//   COUNT(*) GROUP BY A  w[b] += deg_T(c)  per S tuple, then
//                        cnt[a] += w[b]    per (a, b) of R       (flush)
//   rows                 (a,b,c,d) for a in R[b], d in T[c]      (two passes)
//
// S is never partitioned and never re-read (twice in total for rows).
#include "api_internal.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr int ST = 256;                 // threads per CTA (four CTAs per SM at up to 64 registers)
constexpr int SB = 4;                   // S tuples per thread per batch
constexpr int kStarCtasPerSm = 4;

// CTA c of G streams S tuples [c * chunk, (c + 1) * chunk), chunk a multiple
// of 4 * SB so that every chunk starts 16-byte aligned.
struct StarChunk {
    uint32_t begin, end;
};

__device__ __forceinline__ StarChunk star_chunk(uint32_t n, uint32_t chunk) {
    const uint64_t b = (uint64_t)blockIdx.x * chunk, e = b + chunk;
    return StarChunk{(uint32_t)(b < n ? b : n), (uint32_t)(e < n ? e : n)};
}

// Global image slot of key k in the bucket images of t (-1 when absent) and
// its degree; the first probes of all SB keys are issued before any is
// resolved.
__device__ __forceinline__ void img_find_batch(const TImg &t, const int32_t (&k)[SB],
                                               const bool (&use)[SB], long long (&gs)[SB],
                                               uint32_t (&deg)[SB]) {
    uint64_t base[SB];
    uint32_t cap[SB], s[SB];
    unsigned long long v[SB];
#pragma unroll
    for (int q = 0; q < SB; ++q) {
        gs[q] = -1;
        deg[q] = 0;
        cap[q] = 0;
        if (use[q]) {
            const uint32_t j = (t.J == 1) ? 0u : bucket_of(k[q], t.seed_bucket, t.J);
            base[q] = 2ull * __ldg(t.off + j);
            cap[q] = __ldg(t.cap + j);
        }
    }
#pragma unroll
    for (int q = 0; q < SB; ++q) {
        if (cap[q]) {
            s[q] = fastrange(mix32((uint32_t)k[q] ^ t.seed_slot), cap[q]);
            v[q] = __ldg((const unsigned long long *)(t.img + base[q] + s[q]));
        }
    }
#pragma unroll
    for (int q = 0; q < SB; ++q) {
        if (!cap[q]) continue;
        unsigned long long x = v[q];
        uint32_t sl = s[q];
        for (uint32_t it = 0; it < cap[q] && x != kEmpty64 && (uint32_t)x != (uint32_t)k[q]; ++it) {
            sl = (sl + 1 == cap[q]) ? 0u : sl + 1;
            x = __ldg((const unsigned long long *)(t.img + base[q] + sl));
        }
        if (x != kEmpty64 && (uint32_t)x == (uint32_t)k[q]) {
            gs[q] = (long long)(base[q] + sl);
            deg[q] = (uint32_t)(x >> 32);
        }
    }
}

// Lookups of a batch in the two single tables (packed deg << 32 | key,
// mask + 1 slots, home slot slot_of): R's slot (-1 when absent) and degree of
// every b, T's degree of every c.  All 2 * SB first probes are in flight
// before any is resolved.
struct Single {
    const unsigned long long *tbl;
    uint32_t mask, seed;
};

__device__ __forceinline__ uint32_t single_resolve(const Single &t, uint32_t k, uint32_t &s,
                                                   unsigned long long x) {
    for (uint32_t it = 0; it < t.mask && x != kEmpty64 && (uint32_t)x != k; ++it) {
        s = (s + 1) & t.mask;
        x = __ldg(t.tbl + s);
    }
    return (x == kEmpty64 || (uint32_t)x != k) ? 0u : (uint32_t)(x >> 32);
}

__device__ __forceinline__ void single_find2(const Single &r, const Single &t, const int32_t (&b)[SB],
                                             const int32_t (&c)[SB], const bool (&use)[SB],
                                             long long (&rs)[SB], uint32_t (&dR)[SB],
                                             uint32_t (&dT)[SB]) {
    uint32_t sr[SB], stt[SB];
    unsigned long long vr[SB], vt[SB];
#pragma unroll
    for (int q = 0; q < SB; ++q) {
        if (use[q]) {
            sr[q] = slot_of((uint32_t)b[q], r.seed, r.mask);
            stt[q] = slot_of((uint32_t)c[q], t.seed, t.mask);
            vr[q] = __ldg(r.tbl + sr[q]);
            vt[q] = __ldg(t.tbl + stt[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < SB; ++q) {
        rs[q] = -1;
        dR[q] = dT[q] = 0;
        if (!use[q]) continue;
        dR[q] = single_resolve(r, (uint32_t)b[q], sr[q], vr[q]);
        if (dR[q]) rs[q] = sr[q];
        dT[q] = single_resolve(t, (uint32_t)c[q], stt[q], vt[q]);
    }
}

// The S tuples [c.begin, c.end) of this CTA in batches of SB per thread
// (16-byte loads of both columns where aligned); f(b, c, n) per batch.
template <typename F>
__device__ __forceinline__ void star_stream(const int32_t *__restrict__ sx, const int32_t *__restrict__ sy,
                                            StarChunk c, bool vec, F &&f) {
    const uint64_t pol = l2_evict_first();
    auto load = [&](uint32_t i, int32_t (&b)[SB], int32_t (&cc)[SB]) {
        const uint32_t n = min((uint32_t)SB, c.end - i);
        if (vec && n == SB) {
            const int4 u = ld_stream((const int4 *)(sx + i), pol);
            const int4 w = ld_stream((const int4 *)(sy + i), pol);
            b[0] = u.x; b[1] = u.y; b[2] = u.z; b[3] = u.w;
            cc[0] = w.x; cc[1] = w.y; cc[2] = w.z; cc[3] = w.w;
        } else {
#pragma unroll
            for (int q = 0; q < SB; ++q) {
                b[q] = q < (int)n ? __ldg(sx + i + q) : 0;
                cc[q] = q < (int)n ? __ldg(sy + i + q) : 0;
            }
        }
    };
    // the next batch's loads are issued before the current one is looked up
    uint32_t i = c.begin + threadIdx.x * SB;
    int32_t b[SB], cc[SB];
    if (i < c.end) load(i, b, cc);
    while (i < c.end) {
        const uint32_t ni = i + ST * SB;
        int32_t nb[SB], nc[SB];
        if (ni < c.end) load(ni, nb, nc);
        f(b, cc, min((uint32_t)SB, c.end - i));
#pragma unroll
        for (int q = 0; q < SB; ++q) {
            b[q] = nb[q];
            cc[q] = nc[q];
        }
        i = ni;
    }
}

struct StarArgs {
    const int32_t *sx, *sy;     // S columns (b, c), unpartitioned
    uint32_t nS, chunk;
    const unsigned long long *tr, *tt;   // aggregates: R's b table, T's c table
    const uint32_t *metaR, *metaT;       // their masks (meta[0])
    uint32_t seedR, seedT;
    TImg r, t;                  // row output: R's b images (payload a), T's c images (payload d)
    unsigned long long *w;      // GROUP BY A: per slot of R's table
    unsigned long long *total;
    unsigned long long *rowcount;   // row output pass 1: per CTA
    DevStatus *st;
};

// MODE 0: COUNT; 1: GROUP BY A (w per R image slot); 2: per-CTA row counts.
template <int MODE>
__global__ void __launch_bounds__(ST, kStarCtasPerSm) k_star_agg(StarArgs g) {
    __shared__ unsigned long long red[32];
    const StarChunk c = star_chunk(g.nS, g.chunk);
    const bool vec = (((uintptr_t)g.sx | (uintptr_t)g.sy) & 15) == 0;
    unsigned long long acc = 0;
    const Single sr{g.tr, MODE == 2 ? 0u : __ldg(g.metaR), g.seedR};
    const Single stt{g.tt, MODE == 2 ? 0u : __ldg(g.metaT), g.seedT};
    star_stream(g.sx, g.sy, c, vec, [&](const int32_t (&b)[SB], const int32_t (&cc)[SB], uint32_t n) {
        bool use[SB];
#pragma unroll
        for (int q = 0; q < SB; ++q) use[q] = q < (int)n;
        long long rs[SB];
        uint32_t dR[SB], dT[SB];
        if (MODE == 2) {
            long long ts[SB];
            img_find_batch(g.r, b, use, rs, dR);
            img_find_batch(g.t, cc, use, ts, dT);
        } else {
            single_find2(sr, stt, b, cc, use, rs, dR, dT);
        }
#pragma unroll
        for (int q = 0; q < SB; ++q) acc += (unsigned long long)dR[q] * dT[q];
        if (MODE == 1) {
            // w[slot of b] += deg_T(c), runs of equal b merged
            long long cur = -1;
            unsigned long long run = 0;
#pragma unroll
            for (int q = 0; q < SB; ++q) {
                if (rs[q] < 0 || !dT[q]) continue;
                if (rs[q] == cur) {
                    run += dT[q];
                } else {
                    if (cur >= 0) atomicAdd(g.w + cur, run);
                    cur = rs[q];
                    run = dT[q];
                }
            }
            if (cur >= 0) atomicAdd(g.w + cur, run);
        }
    });
    const unsigned long long tot = block_sum_u64(acc, red);
    if (threadIdx.x == 0) {
        if (MODE == 2) g.rowcount[blockIdx.x] = tot;
        else if (tot) atomicAdd(g.total, tot);
    }
}

// GROUP BY A flush: cnt[a] += w[slot of b] for every (a, b) of R, read from
// its input columns; a outside [0, a_domain) is reported and skipped.
__global__ void __launch_bounds__(ST) k_star_flush(const int32_t *__restrict__ ra,
                                                   const int32_t *__restrict__ rb, uint32_t nR,
                                                   const unsigned long long *__restrict__ tr,
                                                   const uint32_t *__restrict__ metaR, uint32_t seedR,
                                                   const unsigned long long *__restrict__ w,
                                                   int32_t a_domain, unsigned long long *__restrict__ cnt,
                                                   DevStatus *st) {
    const Single r{tr, __ldg(metaR), seedR};
    for (uint32_t i0 = (blockIdx.x * ST + threadIdx.x) * SB; i0 < nR; i0 += gridDim.x * ST * SB) {
        int32_t b[SB], a[SB];
        bool use[SB];
        uint32_t s[SB];
        unsigned long long v[SB];
#pragma unroll
        for (int q = 0; q < SB; ++q) {
            use[q] = i0 + q < nR;
            a[q] = use[q] ? __ldg(ra + i0 + q) : 0;
            b[q] = use[q] ? __ldg(rb + i0 + q) : 0;
            if (use[q]) {
                s[q] = slot_of((uint32_t)b[q], r.seed, r.mask);
                v[q] = __ldg(r.tbl + s[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < SB; ++q) {
            if (!use[q]) continue;
            if ((uint32_t)a[q] >= (uint32_t)a_domain) {
                set_status(st, MWJ_ERR_DOMAIN, a[q]);
                continue;
            }
            if (!single_resolve(r, (uint32_t)b[q], s[q], v[q])) continue;   // cannot happen: b is in R
            const unsigned long long x = __ldg(w + s[q]);
            if (x) atomicAdd(cnt + a[q], x);
        }
    }
}

// Row output, pass 2: the same chunks as pass 1; lane l of a warp takes one S
// tuple, a warp scan places its rows after the CTA's cursor.
__global__ void __launch_bounds__(ST) k_star_rows(StarArgs g, const unsigned long long *__restrict__ base,
                                                  int4 *__restrict__ rows, long long capacity) {
    if (base[gridDim.x] > (unsigned long long)capacity) return;   // pass 1 recorded the overflow
    __shared__ unsigned long long cursor;
    if (threadIdx.x == 0) cursor = base[blockIdx.x];
    __syncthreads();
    const StarChunk c = star_chunk(g.nS, g.chunk);
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t b0 = c.begin + (threadIdx.x & ~31u); b0 < c.end; b0 += ST) {
        const uint32_t i = b0 + lane;
        uint32_t dR = 0, dT = 0, rst = 0, tst = 0;
        int32_t b = 0, cc = 0;
        if (i < c.end) {
            b = __ldg(g.sx + i);
            cc = __ldg(g.sy + i);
            dR = timg_deg_start(g.r, b, &rst);
            if (dR) dT = timg_deg_start(g.t, cc, &tst);
        }
        const unsigned long long k = (unsigned long long)dR * dT;
        unsigned long long incl = k;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += y;
        }
        const unsigned long long wtot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long wbase = 0;
        if (lane == 0 && wtot) wbase = atomicAdd(&cursor, wtot);
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (!k) continue;
        unsigned long long p = wbase + incl - k;
        for (uint32_t ia = 0; ia < dR; ++ia) {
            const int32_t a = __ldg(g.r.dlist + rst + ia);
            for (uint32_t id = 0; id < dT; ++id, ++p) {
                if (p < (unsigned long long)capacity)
                    rows[p] = make_int4(a, b, cc, __ldg(g.t.dlist + tst + id));
                else   // the two passes disagree: record it, write nothing
                    set_status(g.st, MWJ_ERR_CHECK, (long long)p);
            }
        }
    }
}

__global__ void k_star_rows_check(const unsigned long long *base, uint32_t G, long long capacity,
                                  long long *n_rows, DevStatus *st) {
    const unsigned long long tot = base[G];
    *n_rows = (long long)tot;
    if (tot > (unsigned long long)capacity) set_status(st, MWJ_ERR_CAPACITY, (long long)tot);
}

struct StarPlan {
    uint32_t JR, JT;
    bool rows, group;
    uint32_t G, chunk;
};

struct StarLayout {
    uint64_t *tblR, *tblT;          // aggregates: single tables
    uint32_t *metaR, *metaT;
    unsigned int *hll, *hllT;       // separate scratch: the two tables are built concurrently
    uint2 *Rp, *Tp;
    uint32_t *offR, *offT;
    uint64_t *imgR, *imgT;
    uint32_t *capR, *capT;
    uint32_t *startR, *startT;
    int32_t *alist, *dlist;
    unsigned long long *w;
    unsigned long long *rowcount, *base;
    void *sscratch;
    void *pscratch;
    size_t pscratch_bytes;
};

// h(B) / g(C) buckets of a dimension relation: ~2048 tuples each, so that
// each bucket's table is built in shared memory
uint32_t star_buckets(int64_t n, int32_t given) {
    if (given >= 1) return (uint32_t)given;
    uint64_t want = (uint64_t)(n + 2047) / 2048;
    uint32_t p = pow2_at_least(want ? want : 1);
    return p > kMaxBuckets ? kMaxBuckets : p;
}

mwj_status star_plan(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                     const mwj_shares *sh, mwj_mode mode, StarPlan *p) {
    for (int k = 0; sh && k < 2; ++k) {
        if (sh->s[k] < 0) return fail(ctx, MWJ_ERR_INVALID_ARG, "star shares must be >= 0 (0: default)");
        if ((uint32_t)sh->s[k] > kMaxBuckets)
            return fail(ctx, MWJ_ERR_INVALID_ARG, "star shares: at most %u buckets", kMaxBuckets);
    }
    p->JR = star_buckets(R.n, sh ? sh->s[0] : 0);
    p->JT = star_buckets(T.n, sh ? sh->s[1] : 0);
    p->rows = mode == MWJ_MATERIALIZE;
    p->group = mode == MWJ_COUNT_GROUP_BY_A;
    // one resident wave of CTAs, each a contiguous 16-byte aligned stretch of S
    const uint64_t ctas = (uint64_t)ctx->dev.num_sms * kStarCtasPerSm;
    uint64_t chunk = (uint64_t)(S.n + ctas - 1) / ctas;
    chunk = (chunk + 4 * SB - 1) / (4 * SB) * (4 * SB);
    if (chunk == 0) chunk = 4 * SB;
    p->chunk = (uint32_t)chunk;
    p->G = (uint32_t)((S.n + chunk - 1) / chunk);
    if (p->G == 0) p->G = 1;
    return MWJ_OK;
}

size_t star_layout(Arena &A, const StarPlan &p, const mwj_rel &R, const mwj_rel &T, int num_sms,
                   StarLayout &L) {
    if (!p.rows) {
        L.tblR = A.take<uint64_t>(single_table_slots(R.n));
        L.metaR = A.take<uint32_t>(4);
        L.tblT = A.take<uint64_t>(single_table_slots(T.n));
        L.metaT = A.take<uint32_t>(4);
        L.hll = A.take<unsigned int>(hll_scratch_registers(num_sms));
        L.hllT = A.take<unsigned int>(hll_scratch_registers(num_sms));
        L.w = p.group ? A.take<unsigned long long>(single_table_slots(R.n)) : nullptr;
        L.Rp = L.Tp = nullptr;
        L.offR = L.offT = L.capR = L.capT = L.startR = L.startT = nullptr;
        L.imgR = L.imgT = nullptr;
        L.alist = L.dlist = nullptr;
        L.rowcount = L.base = nullptr;
        L.sscratch = L.pscratch = nullptr;
        L.pscratch_bytes = 0;
        return A.used;
    }
    L.tblR = L.tblT = nullptr;
    L.metaR = L.metaT = nullptr;
    L.hll = L.hllT = nullptr;
    L.w = nullptr;
    L.Rp = A.take<uint2>(R.n + 2);
    L.offR = A.take<uint32_t>(p.JR + 1);
    L.Tp = A.take<uint2>(T.n + 2);
    L.offT = A.take<uint32_t>(p.JT + 1);
    L.imgR = A.take<uint64_t>(2 * (size_t)R.n + 4);
    L.capR = A.take<uint32_t>(p.JR + 1);
    L.imgT = A.take<uint64_t>(2 * (size_t)T.n + 4);
    L.capT = A.take<uint32_t>(p.JT + 1);
    L.startR = A.take<uint32_t>(2 * (size_t)R.n + 4);
    L.alist = A.take<int32_t>(R.n + 4);
    L.startT = A.take<uint32_t>(2 * (size_t)T.n + 4);
    L.dlist = A.take<int32_t>(T.n + 4);
    L.rowcount = A.take<unsigned long long>(p.G + 1);
    L.base = A.take<unsigned long long>(p.G + 2);
    L.sscratch = A.take<char>(scan_scratch_bytes(p.G + 1));
    size_t ps = part_scratch_bytes(R.n, p.JR, num_sms);
    const size_t ps2 = part_scratch_bytes(T.n, p.JT, num_sms);
    if (ps2 > ps) ps = ps2;
    L.pscratch = A.take<char>(ps);
    L.pscratch_bytes = ps;
    return A.used;
}

}  // namespace

mwj_status plan_star_default(const mwj_rel &R, const mwj_rel &T, mwj_shares *sh) {
    sh->s[0] = (int32_t)star_buckets(R.n, 0);
    sh->s[1] = (int32_t)star_buckets(T.n, 0);
    sh->s[2] = 0;
    return MWJ_OK;
}

mwj_status star_workspace(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                          const mwj_shares *shares, mwj_mode mode, size_t *bytes) {
    StarPlan p;
    mwj_status s = star_plan(ctx, R, S, T, shares, mode, &p);
    if (s != MWJ_OK) return s;
    Arena A(nullptr, 0);
    StarLayout L;
    *bytes = star_layout(A, p, R, T, ctx->dev.num_sms, L);
    return MWJ_OK;
}

}  // namespace mwj

using namespace mwj;

extern "C" mwj_status mwj_join3_star(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T,
                                     const mwj_shares *shares, const mwj_out *out, void *workspace,
                                     size_t ws_bytes, void *stream) {
    if (!ctx || !out) return MWJ_ERR_INVALID_ARG;
    ApiScope api_scope(&ctx->prof);
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    mwj_status s = check_out(ctx, out, 4);
    if (s != MWJ_OK) return s;
    StarPlan p;
    if ((s = star_plan(ctx, R, S, T, shares, out->mode, &p)) != MWJ_OK) return s;
    Arena A(workspace, ws_bytes);
    StarLayout L;
    star_layout(A, p, R, T, ctx->dev.num_sms, L);
    if (A.overflow || !workspace)
        return fail(ctx, MWJ_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, A.used);

    cudaStream_t st = (cudaStream_t)stream;
    const Seeds &sd = ctx->seeds;
    const int sms = ctx->dev.num_sms;
    cudaError_t e;
    if ((e = cudaMemsetAsync(out->total, 0, sizeof(int64_t), st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset total");
    if (p.group &&
        (e = cudaMemsetAsync(out->group_counts, 0, sizeof(int64_t) * (size_t)out->a_domain, st)) !=
            cudaSuccess)
        return cuda_fail(ctx, e, "memset group_counts");
    // the caller's stream waits for the side stream on every return after
    // the fork, so no work of this call outlives it
    struct JoinGuard {
        cudaStream_t st;
        cudaEvent_t ev;
        bool armed;
        ~JoinGuard() {
            if (armed) cudaStreamWaitEvent(st, ev, 0);
        }
    } join_guard{st, ctx->join, false};
    if (!p.rows) {
        // the aggregates: one degree table per dimension relation, T's on the
        // side stream while R's is built here
        // (with per-kernel profiling on, on the caller's stream: see the linear join)
        cudaStream_t side = ctx->prof.on ? st : ctx->side;
        if ((e = cudaEventRecord(ctx->fork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(side, ctx->fork, 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "fork");
        e = single_table_direct(T.x, T.n, sd.slot2, L.hllT, L.metaT, L.tblT, single_table_slots(T.n),
                                ctx->status, sms, side);
        const cudaError_t ej = cudaEventRecord(ctx->join, side);
        if (ej != cudaSuccess) return cuda_fail(ctx, ej, "join");
        join_guard.armed = true;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "T table");
        if ((e = single_table_direct(R.y, R.n, sd.slot, L.hll, L.metaR, L.tblR, single_table_slots(R.n),
                                     ctx->status, sms, st)) != cudaSuccess)
            return cuda_fail(ctx, e, "R table");
        if ((e = cudaStreamWaitEvent(st, ctx->join, 0)) != cudaSuccess) return cuda_fail(ctx, e, "join");
        join_guard.armed = false;
        if (p.group &&
            (e = cudaMemsetAsync(L.w, 0, sizeof(unsigned long long) * single_table_slots(R.n), st)) !=
                cudaSuccess)
            return cuda_fail(ctx, e, "memset w");
    } else {
        // row output: R as (b, a) pairs by h(B), T as (c, d) pairs by g(C),
        // each bucket a table of its keys' degrees and lists
        PartSpec pr{0, sd.B, p.JR, -1, 0, 1};
        pr.st = ctx->status;
        if ((e = part_run(R.y, R.x, R.n, pr, PAY_PAIR, L.Rp, L.offR, L.pscratch, L.pscratch_bytes, sms,
                          st)) != cudaSuccess)
            return cuda_fail(ctx, e, "partition R");
        PartSpec pt{0, sd.C, p.JT, -1, 0, 1};
        pt.st = ctx->status;
        if ((e = part_run(T.x, T.y, T.n, pt, PAY_PAIR, L.Tp, L.offT, L.pscratch, L.pscratch_bytes, sms,
                          st)) != cudaSuccess)
            return cuda_fail(ctx, e, "partition T");
        if ((e = tables_build(nullptr, L.Rp, L.offR, p.JR, sd.slot, L.imgR, L.capR, L.startR, L.alist,
                              ctx->status, sms, st)) != cudaSuccess)
            return cuda_fail(ctx, e, "R tables");
        if ((e = tables_build(nullptr, L.Tp, L.offT, p.JT, sd.slot2, L.imgT, L.capT, L.startT, L.dlist,
                              ctx->status, sms, st)) != cudaSuccess)
            return cuda_fail(ctx, e, "T tables");
    }

    StarArgs g{};
    g.sx = S.x;
    g.sy = S.y;
    g.nS = (uint32_t)S.n;
    g.chunk = p.chunk;
    g.tr = (const unsigned long long *)L.tblR;
    g.tt = (const unsigned long long *)L.tblT;
    g.metaR = L.metaR;
    g.metaT = L.metaT;
    g.seedR = sd.slot;
    g.seedT = sd.slot2;
    g.r = TImg{L.imgR, L.offR, L.capR, L.startR, L.alist, nullptr, p.JR, sd.B, sd.slot};
    g.t = TImg{L.imgT, L.offT, L.capT, L.startT, L.dlist, nullptr, p.JT, sd.C, sd.slot2};
    g.w = L.w;
    g.total = (unsigned long long *)out->total;
    g.rowcount = L.rowcount;
    g.st = ctx->status;
    if (S.n > 0) {
        if (p.rows) {
            ProfScope ps_("star_rowcount", st);
            k_star_agg<2><<<p.G, ST, 0, st>>>(g);
        } else if (p.group) {
            ProfScope ps_("star_probe_groupby", st);
            k_star_agg<1><<<p.G, ST, 0, st>>>(g);
        } else {
            ProfScope ps_("star_probe_count", st);
            k_star_agg<0><<<p.G, ST, 0, st>>>(g);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "star probe");
    }
    if (p.group && R.n > 0) {
        const uint64_t want = ((uint64_t)R.n + (uint64_t)ST * SB - 1) / ((uint64_t)ST * SB);
        const unsigned grid = (unsigned)(want < (uint64_t)sms * 4 ? want : (uint64_t)sms * 4);
        ProfScope ps_("star_flush", st);
        k_star_flush<<<grid, ST, 0, st>>>(R.x, R.y, (uint32_t)R.n, g.tr, L.metaR, sd.slot, L.w,
                                           out->a_domain, (unsigned long long *)out->group_counts,
                                           ctx->status);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "star flush");
    }
    if (p.rows) {
        if (S.n == 0 && (e = cudaMemsetAsync(L.rowcount, 0, sizeof(unsigned long long) * p.G, st)) != cudaSuccess)
            return cuda_fail(ctx, e, "memset row counts");
        e = scan_excl_u64((const uint64_t *)L.rowcount, (uint64_t *)L.base, p.G, true, L.sscratch, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "row scan");
        {
            ProfScope ps_("rows_check", st);
            k_star_rows_check<<<1, 1, 0, st>>>(L.base, p.G, out->capacity, (long long *)out->n_rows,
                                               ctx->status);
        }
        if (S.n > 0) {
            ProfScope ps_("star_rows", st);
            k_star_rows<<<p.G, ST, 0, st>>>(g, L.base, (int4 *)out->rows, out->capacity);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "star rows");
        // total = number of rows
        if ((e = cudaMemcpyAsync(out->total, L.base + p.G, sizeof(int64_t), cudaMemcpyDeviceToDevice, st)) !=
            cudaSuccess)
            return cuda_fail(ctx, e, "total");
    }
    return MWJ_OK;
}
