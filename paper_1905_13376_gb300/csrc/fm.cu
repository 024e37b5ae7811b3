// fm.cu -- Flajolet-Martin sketches of the distinct friends of friends of
// friends of every A (Section 4.1's footnote; the approximate variant of
// Example 1's query):
//
//     D(a) = { d : (a,b) in R, (b,c) in S, (c,d) in T }
//
// is summarised by a PCSA sketch (Flajolet and Martin, 1985): M = 16 bitmaps
// of 32 bits; a value d sets bit rho(h div M) of bitmap h mod M, with
// h = fmix32(d xor SEED) (MurmurHash3's 32-bit finaliser) and rho the index
// of the lowest 1 bit (27 when h div M is 0).  The sketch of a union is the
// OR of the sketches, so the linear join carries sketches along the chain the
// way it carries counts for COUNT(*) GROUP BY A, with OR in place of +:
//
//     skT(c) = OR of bit(d) over T's (c, d)                  (one pass over T)
//     w(b)   = OR of skT(c) over S_i's (b, c)                (on chip, per bucket)
//     sk(a) |= w(b) for every (a, b) of R_i                  (global, per bucket)
//
// R and S are partitioned by H(B) as in Algorithm 1; bucket i's on-chip table
// holds S_i's B values with their 64-byte sketches (the "~100 bytes per
// tuple" of the paper's footnote).  Four lanes handle one tuple, four
// bitmaps (16 bytes) per lane.  The estimate of |D(a)| is (M / PHI) * 2^(mean R_j),
// R_j the lowest 0 bit of bitmap j, PHI = 0.77351.
#include "api_internal.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr uint32_t FM_M = 16;                 // bitmaps per sketch
constexpr uint32_t FM_SEED = 0x5BD1E995u;
constexpr double FM_PHI = 0.77351;
constexpr int FT = 512;                        // threads per CTA
constexpr uint32_t kFmCapLog2 = 10;            // on-chip table: 1024 slots of 68 bytes

// MurmurHash3's 32-bit finalisation mix (Appleby's published constants).
__device__ __forceinline__ uint32_t fmix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

// (bitmap, bit) that value d sets
__device__ __forceinline__ void fm_bit(int32_t d, uint32_t *j, uint32_t *r) {
    const uint32_t h = fmix32((uint32_t)d ^ FM_SEED);
    *j = h & (FM_M - 1);
    const uint32_t q = h >> 4;
    *r = q ? (uint32_t)(__ffs((int)q) - 1) : 27u;
}

constexpr uint32_t kNoIndex = 0xFFFFFFFFu;

// dense sketch index of c from T's key table, whose entries hold
// (index << 32 | c) once k_fm_index has run (kNoIndex if c is absent)
__device__ __forceinline__ uint32_t tkey_index(const unsigned long long *tbl, uint32_t mask, uint32_t seed,
                                               uint32_t c) {
    uint32_t s = slot_of(c, seed, mask);
    for (uint32_t it = 0; it <= mask; ++it) {
        const unsigned long long x = __ldg(tbl + s);
        if (x == kEmpty64) return kNoIndex;
        if ((uint32_t)x == c) return (uint32_t)(x >> 32);
        s = (s + 1) & mask;
    }
    return kNoIndex;
}

// dense index of every occupied slot of T's key table (warp-aggregated
// counter; the order of the indices is immaterial), stored in the entry's
// upper half in place of the degree; count = their number.  An index is
// below 2^31, so an entry never becomes kEmpty64.
__global__ void k_fm_index(unsigned long long *__restrict__ tbl, const uint32_t *__restrict__ meta,
                           unsigned int *__restrict__ count) {
    const uint64_t slots = (uint64_t)meta[0] + 1;
    for (uint64_t s0 = (uint64_t)blockIdx.x * blockDim.x; s0 < slots; s0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = s0 + threadIdx.x;
        const unsigned long long x = s < slots ? tbl[s] : kEmpty64;
        const bool occ = x != kEmpty64;
        const unsigned m = __ballot_sync(0xffffffffu, occ);
        unsigned base = 0;
        if ((threadIdx.x & 31) == 0 && m) base = atomicAdd(count, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        const unsigned idx = base + __popc(m & ((1u << (threadIdx.x & 31)) - 1u));
        if (occ) tbl[s] = ((unsigned long long)idx << 32) | (uint32_t)x;
    }
}

__global__ void k_fm_zero(uint32_t *__restrict__ sk, const unsigned int *__restrict__ count) {
    const uint64_t words = (uint64_t)(*count) * FM_M;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x)
        sk[i] = 0u;
}

// skT(c) |= bit(d) for every (c, d) of T; each thread takes 8 consecutive
// tuples and ORs a run of equal c into a local sketch first
__global__ void __launch_bounds__(256) k_fm_tsketch(const int32_t *__restrict__ tc, const int32_t *__restrict__ td,
                                                    uint32_t n, const unsigned long long *__restrict__ tbl,
                                                    const uint32_t *__restrict__ meta, uint32_t seed,
                                                    uint32_t *__restrict__ skT) {
    const uint32_t mask = __ldg(meta);
    constexpr uint32_t K = 8;
    for (uint32_t i = (blockIdx.x * 256 + threadIdx.x) * K; i < n; i += gridDim.x * 256 * K) {
        const uint32_t m = min(K, n - i);
        uint32_t loc[FM_M];
#pragma unroll
        for (uint32_t j = 0; j < FM_M; ++j) loc[j] = 0;
        int32_t cur = __ldg(tc + i);
        auto flush = [&](int32_t c) {
            const uint32_t ix = tkey_index(tbl, mask, seed, (uint32_t)c);
            if (ix == kNoIndex) return;   // cannot happen: every c of T is in the table
            uint32_t *dst = skT + (size_t)ix * FM_M;
#pragma unroll
            for (uint32_t j = 0; j < FM_M; ++j)
                if (loc[j]) atomicOr(dst + j, loc[j]);
        };
        for (uint32_t k = 0; k < m; ++k) {
            const int32_t c = __ldg(tc + i + k);
            if (c != cur) {
                flush(cur);
#pragma unroll
                for (uint32_t j = 0; j < FM_M; ++j) loc[j] = 0;
                cur = c;
            }
            uint32_t j, r;
            fm_bit(__ldg(td + i + k), &j, &r);
#pragma unroll
            for (uint32_t q = 0; q < FM_M; ++q)
                if (q == j) loc[q] |= 1u << r;
        }
        flush(cur);
    }
}

struct FmArgs {
    const uint2 *Rp, *Sp;
    const uint32_t *offR, *offS;
    const unsigned long long *ttbl;   // T's key table, entries (dense index << 32 | c)
    const uint32_t *tmeta;
    uint32_t tseed;
    const uint32_t *skT;              // dense sketches of T's keys
    uint32_t seed_slot;
    int32_t a_domain;
    uint32_t *out;                    // a_domain x FM_M
    DevStatus *st;
};

// One CTA per H(B) bucket.  S_i's B values with their sketches on chip
// (optimistic pass with inserts of at most 32 probes; bounded rounds if that
// fails), then R_i streams past: sk(a) |= w(b).
__global__ void __launch_bounds__(FT) k_fm_probe(FmArgs g) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr uint32_t cap = 1u << kFmCapLog2, mask = cap - 1;
    uint32_t *keys = (uint32_t *)smem;                                    // cap + 1
    uint32_t *w = (uint32_t *)(smem + align256((cap + 1) * 4));          // (cap + 1) x FM_M
    __shared__ uint32_t nd, bad;
    const uint32_t i = blockIdx.x;
    const uint32_t r0 = g.offR[i], r1 = g.offR[i + 1], s0 = g.offS[i], s1 = g.offS[i + 1];
    if (r0 >= r1 || s0 >= s1) return;
    const uint32_t tmask = __ldg(g.tmeta);
    // four lanes per tuple, bitmaps 4 l4 .. 4 l4 + 3 on lane l4
    const uint32_t l4 = threadIdx.x & 3, grp = threadIdx.x >> 2, groups = FT / 4;

    auto tsk = [&](int32_t c) -> uint4 {   // this lane's bitmaps of skT(c) (0 if c not in T)
        const uint32_t ix = tkey_index(g.ttbl, tmask, g.tseed, (uint32_t)c);
        return ix == kNoIndex ? make_uint4(0u, 0u, 0u, 0u)
                              : __ldg((const uint4 *)(g.skT + (size_t)ix * FM_M) + l4);
    };
    auto or_in = [&](int slot, const uint4 &v) {   // w(b) |= skT(c), this lane's 4 bitmaps
        uint32_t *dst = w + (uint32_t)slot * FM_M + 4 * l4;
        if (v.x) atomicOr(dst, v.x);
        if (v.y) atomicOr(dst + 1, v.y);
        if (v.z) atomicOr(dst + 2, v.z);
        if (v.w) atomicOr(dst + 3, v.w);
    };
    auto clear = [&]() {   // ends with a barrier
        for (uint32_t s = threadIdx.x; s <= cap; s += FT) keys[s] = kEmptyKey;
        if (threadIdx.x == 0) keys[cap] = 0u;
        for (uint32_t s = threadIdx.x; s < (cap + 1) * FM_M; s += FT) w[s] = 0u;
        if (threadIdx.x == 0) {
            nd = 0;
            bad = 0;
        }
        __syncthreads();
    };

    for (uint32_t pos = s0; pos < s1;) {
        clear();
        uint32_t cend = s1;
        bool ok = false;
        if (pos == s0) {
            // optimistic pass: one tuple per four lanes; they insert the same
            // key (idempotent: the first CAS wins) and OR four bitmaps each
            uint32_t fresh_n = 0;
            for (uint32_t t = s0 + grp; t < s1; t += groups) {
                if (*(volatile uint32_t *)&bad) break;
                const uint2 st = __ldg(g.Sp + t);
                bool fresh;
                const int slot = tbl_insert(keys, mask, st.x, g.seed_slot, &fresh);
                fresh_n += fresh;
                if (slot < 0) {
                    atomicOr(&bad, 1u);
                    break;
                }
                or_in(slot, tsk((int32_t)st.y));
            }
            fresh_n = warp_sum(fresh_n);
            if ((threadIdx.x & 31) == 0 && fresh_n) atomicAdd(&nd, fresh_n);
            __syncthreads();
            ok = !bad && nd <= cap - cap / 4;
            __syncthreads();   // every thread has read nd and bad
            if (!ok) clear();
        }
        if (!ok) {
            // bounded rounds of at most cap / 4 tuples while the table stays at
            // most 3/4 full; one tuple per four lanes again
            const uint32_t rt = cap / 4;
            cend = pos;
            for (;;) {
                __syncthreads();
                const uint32_t filled = nd;
                __syncthreads();
                if (cend >= s1 || filled + rt > cap - cap / 4) break;
                const uint32_t e = min(s1, cend + rt);
                uint32_t fresh_n = 0;
                for (uint32_t t = cend + grp; t < e; t += groups) {
                    const uint2 st = __ldg(g.Sp + t);
                    bool fresh;
                    const int slot = tbl_insert(keys, mask, st.x, g.seed_slot, &fresh);
                    fresh_n += fresh;
                    if (slot < 0) {   // cannot happen: the table is never full
                        if (l4 == 0) set_status(g.st, MWJ_ERR_CHECK, 9);
                        continue;
                    }
                    or_in(slot, tsk((int32_t)st.y));
                }
                fresh_n = warp_sum(fresh_n);
                if ((threadIdx.x & 31) == 0 && fresh_n) atomicAdd(&nd, fresh_n);
                cend = e;
            }
        }
        // R_i streams past: sk(a) |= w(b), only bits that are new cost an atomic
        for (uint32_t t = r0 + grp; t < r1; t += groups) {
            const uint2 tr = __ldg(g.Rp + t);
            if ((uint32_t)tr.x >= (uint32_t)g.a_domain) continue;   // reported by the partitioner
            const int slot = tbl_find(keys, mask, tr.y, g.seed_slot);
            if (slot < 0) continue;
            const uint4 v = *(const uint4 *)(w + (uint32_t)slot * FM_M + 4 * l4);
            if (!(v.x | v.y | v.z | v.w)) continue;
            uint32_t *dst = g.out + (size_t)tr.x * FM_M + 4 * l4;
            const uint4 cur = __ldcg((const uint4 *)dst);
            if (v.x & ~cur.x) atomicOr(dst, v.x);
            if (v.y & ~cur.y) atomicOr(dst + 1, v.y);
            if (v.z & ~cur.z) atomicOr(dst + 2, v.z);
            if (v.w & ~cur.w) atomicOr(dst + 3, v.w);
        }
        __syncthreads();   // the table is rebuilt for the next chunk
        pos = cend;
    }
}

__global__ void k_fm_estimate(const uint32_t *__restrict__ sk, int32_t a_domain, float *__restrict__ est) {
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < (uint32_t)a_domain; a += gridDim.x * blockDim.x) {
        uint32_t tot = 0;
#pragma unroll
        for (uint32_t j = 0; j < FM_M; ++j) {   // index of the lowest 0 bit (32 when none)
            const uint32_t word = __ldg(sk + (size_t)a * FM_M + j);
            tot += word == 0xFFFFFFFFu ? 32u : (uint32_t)__ffs((int)~word) - 1u;
        }
        est[a] = (float)((FM_M / FM_PHI) * exp2((double)tot / FM_M));
    }
}

struct FmLayout {
    uint2 *Rp, *Sp;
    uint32_t *offR, *offS;
    uint64_t *ttbl;
    uint32_t *tmeta;
    unsigned int *hll;
    unsigned int *tcount;
    uint32_t *skT;
    void *pscratch;
    size_t pscratch_bytes;
};

size_t fm_layout(Arena &A, uint32_t I, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T, int num_sms,
                 FmLayout &L) {
    L.Rp = A.take<uint2>(R.n + 2);
    L.offR = A.take<uint32_t>(I + 1);
    L.Sp = A.take<uint2>(S.n + 2);
    L.offS = A.take<uint32_t>(I + 1);
    L.ttbl = A.take<uint64_t>(single_table_slots(T.n));
    L.tmeta = A.take<uint32_t>(4);
    L.hll = A.take<unsigned int>(hll_scratch_registers(num_sms));
    L.tcount = A.take<unsigned int>(4);
    L.skT = A.take<uint32_t>((size_t)(T.n + 1) * FM_M);
    size_t ps = part_scratch_bytes(R.n, I, num_sms);
    const size_t ps2 = part_scratch_bytes(S.n, I, num_sms);
    if (ps2 > ps) ps = ps2;
    L.pscratch = A.take<char>(ps);
    L.pscratch_bytes = ps;
    return A.used;
}

// H(B) buckets: ~16K S tuples each (about 500 distinct B values of a
// friends relation fit the 1024-slot table), at least four per SM
mwj_status fm_buckets(mwj_ctx *ctx, const mwj_rel &S, const mwj_shares *sh, uint32_t *I) {
    if (sh) {
        if (sh->s[0] < 1 || (uint32_t)sh->s[0] > kMaxBuckets)
            return fail(ctx, MWJ_ERR_INVALID_ARG, "FM sketches: s[0] must be in [1, %u]", kMaxBuckets);
        *I = (uint32_t)sh->s[0];
        return MWJ_OK;
    }
    uint64_t want = (uint64_t)(S.n + 16383) / 16384;
    const uint64_t minb = (uint64_t)ctx->dev.num_sms * 4;
    if (want < minb) want = minb;
    uint32_t p = pow2_at_least(want);
    *I = p > 16384 ? 16384u : p;
    return MWJ_OK;
}

}  // namespace
}  // namespace mwj

using namespace mwj;

extern "C" mwj_status mwj_fm_workspace_size(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T,
                                            const mwj_shares *shares, size_t *bytes) {
    if (!ctx || !bytes) return MWJ_ERR_INVALID_ARG;
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    uint32_t I;
    mwj_status s = fm_buckets(ctx, S, shares, &I);
    if (s != MWJ_OK) return s;
    Arena A(nullptr, 0);
    FmLayout L;
    *bytes = fm_layout(A, I, R, S, T, ctx->dev.num_sms, L);
    return MWJ_OK;
}

extern "C" mwj_status mwj_fm_linear(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T, const mwj_shares *shares,
                                    int32_t a_domain, uint32_t *sketches, float *estimates, void *workspace,
                                    size_t ws_bytes, void *stream) {
    if (!ctx || !sketches || a_domain <= 0 || ((uintptr_t)sketches & 15)) return MWJ_ERR_INVALID_ARG;
    ApiScope api_scope(&ctx->prof);
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    uint32_t I;
    mwj_status s = fm_buckets(ctx, S, shares, &I);
    if (s != MWJ_OK) return s;
    Arena A(workspace, ws_bytes);
    FmLayout L;
    fm_layout(A, I, R, S, T, ctx->dev.num_sms, L);
    if (A.overflow || !workspace)
        return fail(ctx, MWJ_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, A.used);

    cudaStream_t st = (cudaStream_t)stream;
    const Seeds &sd = ctx->seeds;
    const int sms = ctx->dev.num_sms;
    cudaError_t e;
    if ((e = cudaMemsetAsync(sketches, 0, sizeof(uint32_t) * FM_M * (size_t)a_domain, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset sketches");
    if ((e = cudaMemsetAsync(L.tcount, 0, sizeof(unsigned int), st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset count");
    // T's keys, their dense indices, and the sketch of every key's D values
    if ((e = single_table_direct(T.x, T.n, sd.slot2, L.hll, L.tmeta, L.ttbl, single_table_slots(T.n), ctx->status,
                                 sms, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "T keys");
    {
        ProfScope ps_("fm_index", st);
        k_fm_index<<<sms * 4, 256, 0, st>>>((unsigned long long *)L.ttbl, L.tmeta, L.tcount);
    }
    {
        ProfScope ps_("fm_zero", st);
        k_fm_zero<<<sms * 4, 256, 0, st>>>(L.skT, L.tcount);
    }
    if (T.n > 0) {
        ProfScope ps_("fm_tsketch", st);
        const uint64_t groups = ((uint64_t)T.n + 8 * 256 - 1) / (8 * 256);
        const unsigned grid = (unsigned)(groups < (uint64_t)sms * 8 ? groups : (uint64_t)sms * 8);
        k_fm_tsketch<<<grid, 256, 0, st>>>(T.x, T.y, (uint32_t)T.n, (const unsigned long long *)L.ttbl, L.tmeta,
                                          sd.slot2, L.skT);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "T sketches");
    // R and S by H(B) (Algorithm 1's first level)
    PartSpec ps{0, sd.B, I, -1, 0, 1};
    ps.st = ctx->status;
    if ((e = part_run(S.x, S.y, S.n, ps, PAY_PAIR, L.Sp, L.offS, L.pscratch, L.pscratch_bytes, sms, st)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "partition S");
    PartSpec pr{1, sd.B, I, -1, 0, 1};
    pr.st = ctx->status;
    pr.dom = (uint32_t)a_domain;
    if ((e = part_run(R.x, R.y, R.n, pr, PAY_PAIR, L.Rp, L.offR, L.pscratch, L.pscratch_bytes, sms, st)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "partition R");
    FmArgs g{};
    g.Rp = L.Rp; g.Sp = L.Sp; g.offR = L.offR; g.offS = L.offS;
    g.ttbl = (const unsigned long long *)L.ttbl;
    g.tmeta = L.tmeta;
    g.tseed = sd.slot2;
    g.skT = L.skT;
    g.seed_slot = sd.slot;
    g.a_domain = a_domain;
    g.out = sketches;
    g.st = ctx->status;
    const size_t smem = align256(((1u << kFmCapLog2) + 1) * 4) + ((1u << kFmCapLog2) + 1) * FM_M * 4;
    if ((e = cudaFuncSetAttribute(k_fm_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "fm probe attribute");
    {
        ProfScope ps_("fm_probe", st);
        k_fm_probe<<<I, FT, smem, st>>>(g);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "fm probe");
    if (estimates) {
        ProfScope ps_("fm_estimate", st);
        k_fm_estimate<<<sms * 4, 256, 0, st>>>(sketches, a_domain, estimates);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "fm estimate");
    }
    return MWJ_OK;
}
