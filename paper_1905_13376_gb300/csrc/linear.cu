// linear.cu -- the linear 3-way join R(A,B) S(B,C) T(C,D) (Section 4, Algorithm 1).
//
// After partitioning, CTA i takes R_i (H(b) = i) and mirrors the PMU grid of
// Algorithm 1: R_i is stored in a shared-memory open-addressing table keyed
// by h(b) (MemGrid[h(b)] <- r), the matching S partition S_i streams past
// it, and every S tuple (b, c) that meets R_i looks up c in T's bucket
// tables (the broadcast of T_j to every memory unit becomes every CTA reading
// the same T images, held on chip in L2 or staged in shared memory).  Results
// are aggregated on the fly (Section 4.1, step 4; Section 6):
//
//   COUNT(*)             total += deg_R(b) * deg_T(c)            per S tuple
//   COUNT(*) GROUP BY A  w[b] += deg_T(c)  per S tuple, then
//                        cnt[a] += w[b]    per (a, b) of R_i     (flush)
//   rows                 (a,b,c,d) for a in R_i[b], d in T[c]    (two passes)
//
// which are the definitions of the three outputs summed in a different
// order.  If R_i holds more distinct B values than the table can keep, the
// CTA processes R_i in chunks, each followed by its own pass over S_i; the
// join distributes over the union of the chunks, so the result is unchanged.
#include <type_traits>

#include "internal.h"
#include "linear.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr int LT = 512;          // threads per CTA
constexpr int ROUND = LT * 4;    // R tuples inserted per build round
constexpr uint32_t RCH = 2048;   // R tuples per bulk-copy buffer of the tile build (two buffers)

// Clear the table; values are cleared by the caller.
__device__ __forceinline__ void tbl_clear(uint32_t *keys, uint32_t cap) {
    for (uint32_t s = threadIdx.x; s < cap; s += LT) keys[s] = kEmptyKey;
    if (threadIdx.x == 0) keys[cap] = 0u;
}

// Insert tuples [pos, ...) of a bucket, keyed by their second column (R's
// b) or, with KEY_X, their first (S's b), in rounds of round_tuples(cap)
// tuples while the table stays at most 3/4 full (so it is never full) and
// the chunk stays within max_tuples; returns the chunk end, which is always
// past pos.  on_insert(slot, tuple) runs for every inserted tuple.  Ends
// with a barrier.
template <bool KEY_X = false, typename F>
__device__ __forceinline__ uint32_t build_chunk(const uint2 *__restrict__ Rp, uint32_t pos,
                                                uint32_t r1, uint32_t *keys, uint32_t cap,
                                                uint32_t seed, uint32_t max_tuples,
                                                uint32_t *nd, DevStatus *st, F &&on_insert) {
    const uint32_t mask = cap - 1;
    const uint32_t rt = round_tuples(cap, ROUND);
    uint32_t cend = pos;
    for (;;) {
        __syncthreads();
        const uint32_t filled = *nd;
        __syncthreads();   // every thread has read the count before this round adds to it
        if (cend >= r1 || filled + rt > cap - cap / 4 || cend - pos + rt > max_tuples) break;
        uint32_t fresh_n = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t li = threadIdx.x + k * LT;
            uint32_t idx = cend + li;
            if (li < rt && idx < r1) {
                uint2 t = __ldg(Rp + idx);
                bool fresh;
                int slot = tbl_insert(keys, mask, KEY_X ? t.x : t.y, seed, &fresh);
                if (slot < 0) {
                    set_status(st, MWJ_ERR_CHECK, 1);
                    continue;
                }
                fresh_n += fresh;
                on_insert(slot, t);
            }
        }
        fresh_n = warp_sum(fresh_n);
        if ((threadIdx.x & 31) == 0 && fresh_n) atomicAdd(nd, fresh_n);
        cend += rt;
    }
    return cend < r1 ? cend : r1;
}

// Insert-or-find with a probe sequence of at most 32 slots (optimistic
// passes); -1 when the sequence ran out, which the caller treats as a failed
// pass.  The key kEmptyKey lives in the extra slot mask + 1.
__device__ __forceinline__ int tbl_insert32(uint32_t *keys, uint32_t mask, uint32_t k, uint32_t seed,
                                            bool *fresh) {
    if (k == kEmptyKey) return tbl_insert(keys, mask, k, seed, fresh);
    *fresh = false;
    uint32_t s = slot_of(k, seed, mask);
    for (int it = 0; it < 32; ++it) {
        uint32_t q = keys[s];
        if (q == k) return (int)s;
        if (q == kEmptyKey) {
            uint32_t old = atomicCAS(&keys[s], kEmptyKey, k);
            if (old == kEmptyKey) { *fresh = true; return (int)s; }
            if (old == k) return (int)s;
        }
        s = (s + 1) & mask;
    }
    return -1;
}

// Bulk-copy pipeline of two shared-memory buffers, each with a "full"
// barrier: thread 0 refills a buffer after a CTA barrier has shown every
// thread done with it.  Used to stage an R bucket tile into shared memory.
// Polls a CTA spends, after a fill did not land within the context's wait
// limit, waiting for its copies in flight before it returns.
constexpr uint32_t kDrainLimit = 1u << 24;

struct Ring {
    uint2 *buf;                     // 2 x RCH tuples
    unsigned long long *full;       // 2 barriers
    uint32_t uses[2];               // completed fills of each buffer (same in every thread)
};

// One optimistic pass over R tuples [pos, r1), staged through the ring by
// bulk copies (16-byte aligned superset of the range, rows outside it are
// skipped): insert every tuple with probe sequences of at most 32 slots.
// Succeeds when no insert failed and the table ended at most 3/4 full;
// otherwise the caller clears the table and builds in bounded rounds.
// Returns -1 when a copy did not land within the wait limit.  Ends with a
// barrier.
template <typename F>
__device__ __forceinline__ int build_all(const uint2 *__restrict__ Rp, uint32_t pos, uint32_t r1,
                                         uint32_t *keys, uint32_t cap, uint32_t seed, uint32_t *nd,
                                         uint32_t *bad, Ring &ring, uint32_t spin_limit,
                                         F &&on_insert) {
    const uint32_t mask = cap - 1;
    const uint32_t a0 = pos & ~1u;
    const uint32_t total = ((r1 - a0) + 1u) & ~1u;
    const uint32_t nch = (total + RCH - 1) / RCH;
    auto issue = [&](uint32_t c) {
        const uint32_t b = c & 1u;
        const uint32_t len = min(RCH, total - c * RCH);
        fence_proxy_async();
        mbar_expect_tx(&ring.full[b], len * 8u);
        bulk_copy_g2s(ring.buf + b * RCH, Rp + a0 + c * RCH, len * 8u, &ring.full[b]);
    };
    if (threadIdx.x == 0) {
        if (nch > 0) issue(0);
        if (nch > 1) issue(1);
    }
    uint32_t fresh_n = 0;
    bool failed = false, late = false;
    uint32_t late_c = 0;   // the chunk whose fill did not land in time
    for (uint32_t c = 0; c < nch; ++c) {
        const uint32_t b = c & 1u;
        late |= !mbar_wait_bounded(&ring.full[b], ring.uses[b] & 1u, spin_limit);
        ++ring.uses[b];
        if (__syncthreads_or(late)) {
            late_c = c;
            break;
        }
        const uint32_t len = min(RCH, total - c * RCH);
        const uint32_t base = a0 + c * RCH;
        const uint2 *src = ring.buf + b * RCH;
        for (uint32_t j = threadIdx.x; j < len && !failed; j += LT) {
            const uint32_t gi = base + j;
            if (gi < pos || gi >= r1) continue;
            const uint2 t = src[j];
            bool fresh;
            const int slot = tbl_insert32(keys, mask, t.y, seed, &fresh);
            if (slot < 0) {
                failed = true;
                break;
            }
            fresh_n += fresh;
            on_insert(slot, t);
        }
        __syncthreads();   // every thread is done with buffer b
        if (threadIdx.x == 0 && c + 2 < nch) issue(c + 2);
    }
    if (late) {
        // Wait (bounded, with a fixed limit of its own) for the fills still
        // in flight before the CTA lets go of its shared memory: the fill of
        // chunk late_c, whose phase is the one before the increment above,
        // and the fill of chunk late_c + 1 in the other buffer when it was
        // issued (it was, before chunk late_c was waited on, if it exists).
        if (threadIdx.x == 0) {
            const uint32_t b = late_c & 1u;
            mbar_wait_bounded(&ring.full[b], (ring.uses[b] - 1u) & 1u, kDrainLimit);
            if (late_c + 1 < nch) mbar_wait_bounded(&ring.full[b ^ 1u], ring.uses[b ^ 1u] & 1u, kDrainLimit);
        }
        __syncthreads();
        return -1;
    }
    fresh_n = warp_sum(fresh_n);
    unsigned anyfail = __ballot_sync(0xffffffffu, failed);
    if ((threadIdx.x & 31) == 0) {
        if (fresh_n) atomicAdd(nd, fresh_n);
        if (anyfail) atomicOr(bad, 1u);
    }
    __syncthreads();
    return (!(*bad) && *nd <= cap - cap / 4) ? 1 : 0;
}

constexpr int NB = 4;   // tuples per thread per batch

// Tuples p[s0, s1) in batches of up to NB consecutive tuples per thread
// (thread t takes [b + NB t, b + NB (t+1)) of every NB*LT-tuple round), loaded
// with 128-bit loads; f(t, n) gets the batch and its length.
template <typename F>
__device__ __forceinline__ void stream_batches(const uint2 *__restrict__ p, uint32_t s0, uint32_t s1,
                                               F &&f) {
    if (s0 >= s1) return;
    const uint64_t pol = l2_evict_first();
    uint32_t a = s0;
    uint2 t[NB];
    if (a & 1u) {
        if (threadIdx.x == 0) {
            t[0] = __ldg(p + a);
            f(t, 1);
        }
        ++a;
    }
    // the next batch's loads are issued before the current batch is handed on
    auto load = [&](uint32_t b, uint2 (&t)[NB]) {
        if (b + NB <= s1) {
            const uint4 *q = (const uint4 *)(p + b);
#pragma unroll
            for (int k = 0; k < NB / 2; ++k) {
                uint4 u = ld_stream(q + k, pol);
                t[2 * k] = make_uint2(u.x, u.y);
                t[2 * k + 1] = make_uint2(u.z, u.w);
            }
        } else {
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (b + k < s1) t[k] = __ldg(p + b + k);
        }
    };
    uint32_t b = a + NB * threadIdx.x;
    if (b < s1) load(b, t);
    while (b < s1) {
        const uint32_t nb = b + NB * LT;
        uint2 nx[NB];
        if (nb < s1) load(nb, nx);
        f(t, min((uint32_t)NB, s1 - b));
#pragma unroll
        for (int k = 0; k < NB; ++k) t[k] = nx[k];
        b = nb;
    }
}

// First probes of T's single table (T.J == 0) for the C values of a batch,
// all issued before any is consumed: one L2 round trip for the batch in the
// common case.  use[k] selects the tuples that need deg_T.
__device__ __forceinline__ void t_issue(const TImg &T, uint32_t tmask, const uint2 (&t)[NB],
                                        const bool (&use)[NB], uint32_t (&ts)[NB],
                                        unsigned long long (&v)[NB]) {
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if (use[k]) {
            ts[k] = slot_of(t[k].y, T.seed_slot, tmask);
            v[k] = __ldg((const unsigned long long *)(T.img + ts[k]));
        }
    }
}

// deg_T(c) from the first probe (slot s, value x) of c in the single table.
__device__ __forceinline__ uint32_t t_resolve(const TImg &T, uint32_t tmask, uint32_t c, uint32_t s,
                                              unsigned long long x) {
    for (uint32_t it = 0; it < tmask && x != kEmpty64 && (uint32_t)x != c; ++it) {
        s = (s + 1) & tmask;
        x = __ldg((const unsigned long long *)(T.img + s));
    }
    return (x == kEmpty64 || (uint32_t)x != c) ? 0u : (uint32_t)(x >> 32);
}

// deg_T of the C values of the batch tuples with use[k] (0 for the others).
__device__ __forceinline__ void t_degrees(const TImg &T, uint32_t tmask, const uint2 (&t)[NB],
                                          const bool (&use)[NB], uint32_t (&dT)[NB]) {
    if (T.J == 0) {
        uint32_t ts[NB];
        unsigned long long v[NB];
        t_issue(T, tmask, t, use, ts, v);
#pragma unroll
        for (int k = 0; k < NB; ++k) dT[k] = use[k] ? t_resolve(T, tmask, t[k].y, ts[k], v[k]) : 0u;
    } else {
#pragma unroll
        for (int k = 0; k < NB; ++k) dT[k] = use[k] ? timg_deg(T, (int32_t)t[k].y) : 0u;
    }
}

// 64-bit add into (hi, lo) 32-bit shared counters, exact modulo 2^64.
__device__ __forceinline__ void add_u64_split(uint32_t *lo, uint32_t *hi, unsigned long long v) {
    uint32_t l = (uint32_t)v, h = (uint32_t)(v >> 32);
    uint32_t old = atomicAdd(lo, l);
    if (old + l < old) ++h;
    if (h) atomicAdd(hi, h);
}

// COUNT (MODE 0) and GROUP BY A (MODE 1).  One CTA per R bucket.
template <int MODE>
__global__ void __launch_bounds__(LT, 2) k_lin_agg(LinArgs g) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t cap = 1u << g.cap_log2;
    const size_t arr = align256((cap + 1) * sizeof(uint32_t));
    uint32_t *keys = (uint32_t *)smem;
    uint32_t *deg = (uint32_t *)(smem + arr);          // MODE 0
    uint32_t *wlo = (uint32_t *)(smem + arr);          // MODE 1
    uint32_t *whi = (uint32_t *)(smem + 2 * arr);      // MODE 1
    __shared__ uint32_t nd, bad;
    __shared__ unsigned long long red[32];
    __shared__ __align__(8) unsigned long long fullb[2];
    Ring ring{(uint2 *)(smem + (MODE == 0 ? 2 : 3) * arr), fullb, {0u, 0u}};
    if (threadIdx.x == 0) {
        mbar_init(&fullb[0], 1);
        mbar_init(&fullb[1], 1);
        fence_barrier_init();
    }
    __syncthreads();

    const uint32_t i = blockIdx.x;
    const uint32_t r0 = g.offR[i], r1 = g.offR[i + 1];
    const uint32_t s0 = g.offS[(size_t)i * g.JS], s1 = g.offS[(size_t)(i + 1) * g.JS];
    const uint32_t tmask = (g.t.J == 0) ? __ldg(g.t.meta) : 0u;
    unsigned long long acc = 0;
    const uint32_t mask = cap - 1;

    if (r0 < r1 && s0 < s1) {
        for (uint32_t pos = r0; pos < r1;) {
            tbl_clear(keys, cap);
            for (uint32_t s = threadIdx.x; s <= cap; s += LT) {
                if (MODE == 0) {
                    deg[s] = 0u;
                } else {
                    wlo[s] = 0u;
                    whi[s] = 0u;
                }
            }
            if (threadIdx.x == 0) {
                nd = 0;
                bad = 0;
            }
            // (A values were checked against the group-by domain while R was partitioned)
            auto on_insert = [&](int slot, uint2) {
                if (MODE == 0) atomicAdd(&deg[slot], 1u);
            };
            uint32_t cend;
            __syncthreads();
            int fast = (pos == r0) ? build_all(g.Rp, pos, r1, keys, cap, g.seed_slot, &nd, &bad, ring,
                                               g.spin_limit, on_insert)
                                   : 0;
            if (fast < 0) {   // a bulk copy did not arrive in time
                if (threadIdx.x == 0) set_status(g.st, MWJ_ERR_TIMEOUT, (long long)blockIdx.x);
                return;
            }
            if (fast) {
                cend = r1;
            } else {
                if (pos == r0) {   // the optimistic pass overflowed: start over in rounds
                    tbl_clear(keys, cap);
                    for (uint32_t s = threadIdx.x; s <= cap; s += LT) {
                        if (MODE == 0) {
                            deg[s] = 0u;
                        } else {
                            wlo[s] = 0u;
                            whi[s] = 0u;
                        }
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) nd = 0;
                }
                cend = build_chunk(g.Rp, pos, r1, keys, cap, g.seed_slot, 0xFFFFFFFFu, &nd, g.st,
                                   on_insert);
            }
            // stream S_i past the R chunk
            stream_batches(g.Sp, s0, s1, [&](const uint2 (&t)[NB], uint32_t n) {
                int sl[NB];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    sl[k] = (k < (int)n) ? tbl_find(keys, mask, t[k].x, g.seed_slot) : -1;
                bool use[NB];
#pragma unroll
                for (int k = 0; k < NB; ++k) use[k] = sl[k] >= 0;
                uint32_t dT[NB];
                t_degrees(g.t, tmask, t, use, dT);
                if (MODE == 0) {
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (dT[k]) acc += (unsigned long long)deg[sl[k]] * dT[k];
                } else {
                    // merge runs of equal B before touching shared memory
                    int cur = -1;
                    unsigned long long run = 0;
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        if (!dT[k]) continue;
                        if (sl[k] == cur) {
                            run += dT[k];
                        } else {
                            if (cur >= 0) add_u64_split(&wlo[cur], &whi[cur], run);
                            cur = sl[k];
                            run = dT[k];
                        }
                    }
                    if (cur >= 0) add_u64_split(&wlo[cur], &whi[cur], run);
                }
            });
            __syncthreads();
            if (MODE == 1) {
                // flush: cnt[a] += w[b] for the chunk's R tuples, runs of equal A merged
                stream_batches(g.Rp, pos, cend, [&](const uint2 (&t)[NB], uint32_t n) {
                    int32_t cur = 0;
                    unsigned long long run = 0;
                    bool have = false;
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        if (k >= (int)n) break;
                        int slot = tbl_find(keys, mask, t[k].y, g.seed_slot);
                        if (slot < 0) continue;   // only after a recorded insert failure
                        unsigned long long w =
                            ((unsigned long long)whi[slot] << 32) | (unsigned long long)wlo[slot];
                        if (!w || (uint32_t)t[k].x >= (uint32_t)g.a_domain) continue;
                        if (have && (int32_t)t[k].x == cur) {
                            run += w;
                        } else {
                            if (have) atomicAdd(g.cnt + cur, run);
                            cur = (int32_t)t[k].x;
                            run = w;
                            have = true;
                        }
                        acc += w;
                    }
                    if (have) atomicAdd(g.cnt + cur, run);
                });
            }
            __syncthreads();   // the table is rebuilt for the next chunk
            pos = cend;
        }
    }
    unsigned long long tot = block_sum_u64(acc, red);
    if (threadIdx.x == 0) {
        if (tot) atomicAdd(g.total, tot);
        if (g.rowcount) g.rowcount[i] = tot;
    }
}

// T's weighted table (4-relation chain): 16-byte slots, word 0 = (1 << 32 |
// c) when occupied (0 when empty), word 1 = the 64-bit weight of c.  The
// first probes of a batch read word 0 only; the weight is read from the
// found slot (same sector).
__device__ __forceinline__ void tw_issue(const unsigned long long *tw, uint32_t seed, uint32_t mask,
                                         const uint2 (&t)[NB], const bool (&use)[NB], uint32_t (&ts)[NB],
                                         unsigned long long (&v)[NB]) {
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if (use[k]) {
            ts[k] = slot_of(t[k].y, seed, mask);
            v[k] = __ldg(tw + 2 * (size_t)ts[k]);
        }
    }
}

__device__ __forceinline__ unsigned long long tw_resolve(const unsigned long long *tw, uint32_t mask,
                                                         uint32_t c, uint32_t s, unsigned long long x) {
    const unsigned long long want = (1ull << 32) | c;
    for (uint32_t it = 0; it < mask && x != 0ull && x != want; ++it) {
        s = (s + 1) & mask;
        x = __ldg(tw + 2 * (size_t)s);
    }
    return x == want ? __ldg(tw + 2 * (size_t)s + 1) : 0ull;
}

__device__ __forceinline__ unsigned long long tw_weight(const unsigned long long *tw, uint32_t seed,
                                                        uint32_t mask, uint32_t c) {
    const uint32_t s = slot_of(c, seed, mask);
    return tw_resolve(tw, mask, c, s, __ldg(tw + 2 * (size_t)s));
}

// The same two aggregates with S_i as the on-chip side.  The B-keyed table
// of CTA i gathers w(b) = sum of deg_T(c) over the tuples (b, c) of S_i while
// S_i streams in once; then R_i streams past it once, adding w(b) to total
// and to cnt[a] for every (a, b).  Each R tuple is read and hashed once
// (the R-side kernel above reads and hashes it twice, to build and to
// flush); in exchange every S tuple pays its T lookup whether or not its b
// occurs in R_i.  When S_i holds more distinct B values than the table
// keeps, S_i is taken in chunks, each followed by its own pass over R_i.
// WT: T's table holds 64-bit weights w_T(c) instead of degrees (the chain
// of four relations, where w_T(c) = sum of deg_U(d) over T's (c, d)).
template <int MODE, bool WT>
__global__ void __launch_bounds__(LT, 2) k_lin_agg_s(LinArgs g) {
    using TW = typename std::conditional<WT, unsigned long long, uint32_t>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t cap = 1u << g.cap_log2;
    const size_t arr = align256((cap + 1) * sizeof(uint32_t));
    uint32_t *keys = (uint32_t *)smem;
    uint32_t *wlo = (uint32_t *)(smem + arr);
    uint32_t *whi = (uint32_t *)(smem + 2 * arr);
    __shared__ uint32_t nd, bad;
    __shared__ unsigned long long red[32];

    const uint32_t i = blockIdx.x;
    const uint32_t r0 = g.offR[i], r1 = g.offR[i + 1];
    const uint32_t s0 = g.offS[(size_t)i * g.JS], s1 = g.offS[(size_t)(i + 1) * g.JS];
    const uint32_t tmask = WT ? __ldg(g.tw_meta) : (g.t.J == 0) ? __ldg(g.t.meta) : 0u;
    const uint32_t mask = cap - 1;
    unsigned long long acc = 0;

    auto clear = [&]() {   // ends with a barrier
        tbl_clear(keys, cap);
        for (uint32_t s = threadIdx.x; s <= cap; s += LT) {
            wlo[s] = 0u;
            whi[s] = 0u;
        }
        if (threadIdx.x == 0) {
            nd = 0;
            bad = 0;
        }
        __syncthreads();
    };
    // w[slot] += v for the batch's (slot, v), runs of equal slots merged
    auto add_w = [&](const int (&sl)[NB], const TW (&dT)[NB]) {
        int cur = -1;
        unsigned long long run = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (sl[k] < 0 || !dT[k]) continue;
            if (sl[k] == cur) {
                run += dT[k];
            } else {
                if (cur >= 0) add_u64_split(&wlo[cur], &whi[cur], run);
                cur = sl[k];
                run = dT[k];
            }
        }
        if (cur >= 0) add_u64_split(&wlo[cur], &whi[cur], run);
    };

    if (r0 < r1 && s0 < s1) {
        for (uint32_t pos = s0; pos < s1;) {
            clear();
            uint32_t cend = s1;
            bool ok = false;
            if (pos == s0) {
                // optimistic pass over all of S_i, inserts of at most 32 probes
                uint32_t fresh_n = 0;
                stream_batches(g.Sp, s0, s1, [&](const uint2 (&t)[NB], uint32_t n) {
                    if (*(volatile uint32_t *)&bad) return;   // the pass has failed already
                    bool use[NB];
#pragma unroll
                    for (int k = 0; k < NB; ++k) use[k] = k < (int)n;
                    uint32_t ts[NB];
                    unsigned long long v[NB];
                    // in flight during the inserts
                    if (WT) tw_issue(g.tw, g.tw_seed, tmask, t, use, ts, v);
                    else if (g.t.J == 0) t_issue(g.t, tmask, t, use, ts, v);
                    int sl[NB];
                    bool failed = false;
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        sl[k] = -1;
                        if (!use[k]) continue;
                        if (k > 0 && t[k].x == t[k - 1].x) {   // S arrives grouped by b
                            sl[k] = sl[k - 1];
                            continue;
                        }
                        bool fresh;
                        sl[k] = tbl_insert32(keys, mask, t[k].x, g.seed_slot, &fresh);
                        fresh_n += fresh;
                        failed |= sl[k] < 0;
                    }
                    if (failed) {
                        atomicOr(&bad, 1u);
                        return;
                    }
                    TW dT[NB];
                    if (WT) {
#pragma unroll
                        for (int k = 0; k < NB; ++k)
                            dT[k] = use[k] ? (TW)tw_resolve(g.tw, tmask, t[k].y, ts[k], v[k]) : (TW)0;
                    } else if (g.t.J == 0) {
#pragma unroll
                        for (int k = 0; k < NB; ++k)
                            dT[k] = use[k] ? (TW)t_resolve(g.t, tmask, t[k].y, ts[k], v[k]) : (TW)0;
                    } else {
#pragma unroll
                        for (int k = 0; k < NB; ++k)
                            dT[k] = use[k] ? (TW)timg_deg(g.t, (int32_t)t[k].y) : (TW)0;
                    }
                    add_w(sl, dT);
                });
                fresh_n = warp_sum(fresh_n);
                if ((threadIdx.x & 31) == 0 && fresh_n) atomicAdd(&nd, fresh_n);
                __syncthreads();
                ok = !bad && nd <= cap - cap / 4;
                __syncthreads();   // every thread has read nd and bad
                if (!ok) clear();
            }
            if (!ok)   // chunks built in bounded rounds, one T lookup per tuple
                cend = build_chunk<true>(g.Sp, pos, s1, keys, cap, g.seed_slot, 0xFFFFFFFFu, &nd, g.st,
                                         [&](int slot, uint2 t) {
                                             const unsigned long long d =
                                                 WT ? tw_weight(g.tw, g.tw_seed, tmask, t.y)
                                                    : (unsigned long long)timg_deg(g.t, (int32_t)t.y);
                                             if (d) add_u64_split(&wlo[slot], &whi[slot], d);
                                         });
            // R_i streams past w: total += w(b), cnt[a] += w(b), runs of equal A merged
            stream_batches(g.Rp, r0, r1, [&](const uint2 (&t)[NB], uint32_t n) {
                int32_t cur = 0;
                unsigned long long run = 0;
                bool have = false;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    if (k >= (int)n) break;
                    const int slot = tbl_find(keys, mask, t[k].y, g.seed_slot);
                    if (slot < 0) continue;
                    const unsigned long long w =
                        ((unsigned long long)whi[slot] << 32) | (unsigned long long)wlo[slot];
                    if (!w) continue;
                    if (MODE == 1) {
                        if ((uint32_t)t[k].x >= (uint32_t)g.a_domain) continue;
                        if (have && (int32_t)t[k].x == cur) {
                            run += w;
                        } else {
                            if (have) atomicAdd(g.cnt + cur, run);
                            cur = (int32_t)t[k].x;
                            run = w;
                            have = true;
                        }
                    }
                    acc += w;
                }
                if (MODE == 1 && have) atomicAdd(g.cnt + cur, run);
            });
            __syncthreads();   // the table is rebuilt for the next chunk
            pos = cend;
        }
    }
    unsigned long long tot = block_sum_u64(acc, red);
    if (threadIdx.x == 0) {
        if (tot) atomicAdd(g.total, tot);
        if (g.rowcount) g.rowcount[i] = tot;
    }
}

// Row output, pass 2: R chunk as b -> [a] lists in shared memory, T as
// c -> [d] lists in global memory; row positions from the per-bucket bases
// of pass 1 plus a per-CTA cursor.
__global__ void __launch_bounds__(LT) k_lin_rows(LinArgs g, const unsigned long long *base,
                                                 int4 *rows, long long capacity,
                                                 uint32_t max_tuples) {
    if (base[g.I] > (unsigned long long)capacity) return;   // pass 1 recorded the overflow
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t cap = 1u << g.cap_log2;
    uint32_t *keys = (uint32_t *)smem;
    uint32_t *deg = (uint32_t *)(smem + align256((cap + 1) * 4));
    uint32_t *start = (uint32_t *)((unsigned char *)deg + align256((cap + 1) * 4));
    int32_t *alist = (int32_t *)((unsigned char *)start + align256((cap + 1) * 4));
    __shared__ uint32_t nd;
    __shared__ unsigned long long cursor;
    __shared__ uint32_t scan_scratch[33];
    __shared__ uint32_t carry;

    const uint32_t i = blockIdx.x;
    const uint32_t r0 = g.offR[i], r1 = g.offR[i + 1];
    const uint32_t s0 = g.offS[(size_t)i * g.JS], s1 = g.offS[(size_t)(i + 1) * g.JS];
    const uint32_t mask = cap - 1;
    if (threadIdx.x == 0) cursor = base[i];
    if (r0 >= r1 || s0 >= s1) return;
    for (uint32_t pos = r0; pos < r1;) {
        tbl_clear(keys, cap);
        for (uint32_t s = threadIdx.x; s <= cap; s += LT) deg[s] = 0u;
        if (threadIdx.x == 0) nd = 0;
        uint32_t cend = build_chunk(g.Rp, pos, r1, keys, cap, g.seed_slot, max_tuples, &nd, g.st,
                                    [&](int slot, uint2) { atomicAdd(&deg[slot], 1u); });
        // starts of the a-lists: exclusive scan of deg over the slots
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (uint32_t b = 0; b <= cap; b += LT) {
            uint32_t s = b + threadIdx.x;
            uint32_t d = (s <= cap) ? deg[s] : 0u;
            uint32_t tot;
            uint32_t ex = block_excl_scan_u32(d, scan_scratch, &tot);
            if (s <= cap) start[s] = carry + ex;
            __syncthreads();
            if (threadIdx.x == 0) carry += tot;
            __syncthreads();
        }
        for (uint32_t idx = pos + threadIdx.x; idx < cend; idx += LT) {
            uint2 t = __ldg(g.Rp + idx);
            int slot = tbl_find(keys, mask, t.y, g.seed_slot);
            if (slot >= 0) alist[atomicAdd(&start[slot], 1u)] = (int32_t)t.x;
        }
        __syncthreads();
        for (uint32_t s = threadIdx.x; s <= cap; s += LT) start[s] -= deg[s];
        __syncthreads();
        const uint32_t lane = threadIdx.x & 31;
        // warp-uniform walk over S_i: lane l of a warp takes tuple b0 + l
        for (uint32_t b0 = s0 + (threadIdx.x & ~31u); b0 < s1; b0 += LT) {
            const uint32_t idx = b0 + lane;
            uint2 s = make_uint2(0u, 0u);
            int slot = -1;
            uint32_t dR = 0, dT = 0, tst = 0;
            if (idx < s1) {
                s = __ldg(g.Sp + idx);
                slot = tbl_find(keys, mask, s.x, g.seed_slot);
                if (slot >= 0) {
                    dR = deg[slot];
                    dT = timg_deg_start(g.t, (int32_t)s.y, &tst);
                }
            }
            const unsigned long long k = (unsigned long long)dR * dT;
            unsigned long long incl = k;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += y;
            }
            const unsigned long long wtot = __shfl_sync(0xffffffffu, incl, 31);
            unsigned long long wbase = 0;
            if (lane == 0 && wtot) wbase = atomicAdd(&cursor, wtot);
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
            if (k) {
                unsigned long long p = wbase + incl - k;
                const uint32_t as = start[slot];
                for (uint32_t ia = 0; ia < dR; ++ia) {
                    const int32_t a = alist[as + ia];
                    for (uint32_t id = 0; id < dT; ++id, ++p) {
                        if (p < (unsigned long long)capacity)
                            rows[p] = make_int4(a, (int32_t)s.x, (int32_t)s.y,
                                                __ldg(g.t.dlist + tst + id));
                        else   // the two passes disagree: record it, write nothing
                            set_status(g.st, MWJ_ERR_CHECK, (long long)p);
                    }
                }
            }
        }
        __syncthreads();
        pos = cend;
    }
}

__global__ void k_rows_check(const unsigned long long *base, uint32_t I, long long capacity,
                             long long *n_rows, DevStatus *st) {
    unsigned long long tot = base[I];
    *n_rows = (long long)tot;
    if (tot > (unsigned long long)capacity) set_status(st, MWJ_ERR_CAPACITY, (long long)tot);
}

}  // namespace

size_t lin_agg_smem(uint32_t cap_log2, int mode, bool build_s) {
    uint32_t cap = 1u << cap_log2;
    if (build_s) return align256((cap + 1) * 4) * 3;
    return align256((cap + 1) * 4) * (mode == 1 ? 3 : 2) + 2 * RCH * sizeof(uint2);
}

size_t lin_rows_smem(uint32_t cap_log2, uint32_t max_tuples) {
    uint32_t cap = 1u << cap_log2;
    return 3 * align256((cap + 1) * 4) + (size_t)max_tuples * 4;
}

template <typename K>
static cudaError_t launch_agg(K kernel, const LinArgs &g, size_t smem, const char *name,
                             cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ProfScope ps_(name, st);
    kernel<<<g.I, LT, smem, st>>>(g);
    return cudaGetLastError();
}

cudaError_t lin_agg_launch(const LinArgs &g, int mode, cudaStream_t st) {
    if (g.I == 0) return cudaSuccess;
    const size_t smem = lin_agg_smem(g.cap_log2, mode, g.build_s != 0);
    const char *name = mode == 1 ? "lin_probe_groupby" : "lin_probe_count";
    if (g.build_s)
        return g.tw ? (mode == 1 ? launch_agg(k_lin_agg_s<1, true>, g, smem, name, st)
                                 : launch_agg(k_lin_agg_s<0, true>, g, smem, name, st))
                    : (mode == 1 ? launch_agg(k_lin_agg_s<1, false>, g, smem, name, st)
                                 : launch_agg(k_lin_agg_s<0, false>, g, smem, name, st));
    return mode == 1 ? launch_agg(k_lin_agg<1>, g, smem, name, st)
                     : launch_agg(k_lin_agg<0>, g, smem, name, st);
}

cudaError_t lin_rows_launch(const LinArgs &g, const unsigned long long *base, int32_t *rows,
                            long long capacity, long long *n_rows, uint32_t max_tuples,
                            cudaStream_t st) {
    {
        ProfScope ps_("rows_check", st);
        k_rows_check<<<1, 1, 0, st>>>(base, g.I, capacity, n_rows, g.st);
    }
    if (g.I == 0) return cudaGetLastError();
    size_t smem = lin_rows_smem(g.cap_log2, max_tuples);
    cudaError_t e = cudaFuncSetAttribute(k_lin_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps_("lin_rows", st);
        k_lin_rows<<<g.I, LT, smem, st>>>(g, base, (int4 *)rows, capacity, max_tuples);
    }
    return cudaGetLastError();
}

}  // namespace mwj
