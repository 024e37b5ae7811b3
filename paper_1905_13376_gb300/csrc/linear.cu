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
#include "internal.h"
#include "linear.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr int LT = 512;          // threads per CTA
constexpr int ROUND = LT * 4;    // R tuples inserted per build round

// Calls f(tuple) for every tuple of p[s0, s1), two tuples per 128-bit load.
template <typename F>
__device__ __forceinline__ void stream_pairs(const uint2 *__restrict__ p, uint32_t s0, uint32_t s1,
                                             F &&f) {
    if (s0 >= s1) return;
    uint32_t a = s0;
    if (a & 1u) {
        if (threadIdx.x == 0) f(p[a]);
        ++a;
    }
    const uint32_t npair = (s1 - a) >> 1;
    const uint4 *p4 = (const uint4 *)(p + a);
    uint32_t q = threadIdx.x;
    for (; q + LT < npair; q += 2 * LT) {
        uint4 u = __ldg(p4 + q);
        uint4 v = __ldg(p4 + q + LT);
        f(make_uint2(u.x, u.y));
        f(make_uint2(u.z, u.w));
        f(make_uint2(v.x, v.y));
        f(make_uint2(v.z, v.w));
    }
    for (; q < npair; q += LT) {
        uint4 u = __ldg(p4 + q);
        f(make_uint2(u.x, u.y));
        f(make_uint2(u.z, u.w));
    }
    if ((s1 - a) & 1u) {
        if (threadIdx.x == LT - 1) f(p[s1 - 1]);
    }
}

struct SmemTbl {
    uint32_t *keys;   // cap + 1
    uint32_t mask;
};

// Clear the table; values are cleared by the caller.
__device__ __forceinline__ void tbl_clear(uint32_t *keys, uint32_t cap) {
    for (uint32_t s = threadIdx.x; s < cap; s += LT) keys[s] = kEmptyKey;
    if (threadIdx.x == 0) keys[cap] = 0u;
}

// Insert R tuples [pos, ...) in rounds until the table holds more than half
// of cap distinct keys or the chunk reaches max_tuples; returns the chunk end.
// on_insert(slot, tuple) runs for every inserted tuple.  Ends with a barrier.
template <typename F>
__device__ __forceinline__ uint32_t build_chunk(const uint2 *__restrict__ Rp, uint32_t pos,
                                                uint32_t r1, uint32_t *keys, uint32_t cap,
                                                uint32_t seed, uint32_t max_tuples,
                                                uint32_t *nd, F &&on_insert) {
    const uint32_t mask = cap - 1;
    uint32_t cend = pos;
    for (;;) {
        __syncthreads();
        const uint32_t filled = *nd;
        __syncthreads();   // every thread has read the count before this round adds to it
        if (cend >= r1 || filled > cap / 2 || cend - pos + ROUND > max_tuples) break;
        uint32_t fresh_n = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t idx = cend + threadIdx.x + k * LT;
            if (idx < r1) {
                uint2 t = __ldg(Rp + idx);
                bool fresh;
                int slot = tbl_insert(keys, mask, t.y, seed, &fresh);
                fresh_n += fresh;
                on_insert(slot, t);
            }
        }
        fresh_n = warp_sum(fresh_n);
        if ((threadIdx.x & 31) == 0 && fresh_n) atomicAdd(nd, fresh_n);
        cend += ROUND;
    }
    return cend < r1 ? cend : r1;
}

// COUNT (MODE 0) and GROUP BY A (MODE 1).  One CTA per R bucket.
template <int MODE>
__global__ void __launch_bounds__(LT) k_lin_agg(LinArgs g) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t cap = 1u << g.cap_log2;
    uint32_t *keys = (uint32_t *)smem;
    unsigned char *vbase = smem + align256((cap + 1) * sizeof(uint32_t));
    uint32_t *deg = (uint32_t *)vbase;                            // MODE 0
    unsigned long long *w = (unsigned long long *)vbase;          // MODE 1
    __shared__ uint32_t nd;
    __shared__ unsigned long long red[32];

    const uint32_t i = blockIdx.x;
    const uint32_t r0 = g.offR[i], r1 = g.offR[i + 1];
    const uint32_t s0 = g.offS[(size_t)i * g.JS], s1 = g.offS[(size_t)(i + 1) * g.JS];
    unsigned long long acc = 0;
    const uint32_t mask = cap - 1;

    if (r0 < r1 && s0 < s1) {
        for (uint32_t pos = r0; pos < r1;) {
            tbl_clear(keys, cap);
            for (uint32_t s = threadIdx.x; s <= cap; s += LT) {
                if (MODE == 0) deg[s] = 0u; else w[s] = 0ull;
            }
            if (threadIdx.x == 0) nd = 0;
            uint32_t cend = build_chunk(g.Rp, pos, r1, keys, cap, g.seed_slot, 0xFFFFFFFFu, &nd,
                                        [&](int slot, uint2 t) {
                                            if (MODE == 0) {
                                                atomicAdd(&deg[slot], 1u);
                                            } else if ((uint32_t)t.x >= (uint32_t)g.a_domain) {
                                                set_status(g.st, MWJ_ERR_DOMAIN, (int32_t)t.x);
                                            }
                                        });
            // stream S_i past the R chunk
            stream_pairs(g.Sp, s0, s1, [&](uint2 s) {
                int slot = tbl_find(keys, mask, s.x, g.seed_slot);
                if (slot < 0) return;
                uint32_t dT = timg_deg(g.t, (int32_t)s.y);
                if (dT == 0) return;
                if (MODE == 0) acc += (unsigned long long)deg[slot] * dT;
                else atomicAdd(&w[slot], (unsigned long long)dT);
            });
            __syncthreads();
            if (MODE == 1) {
                // flush: cnt[a] += w[b] for the chunk's R tuples
                for (uint32_t idx = pos + threadIdx.x; idx < cend; idx += LT) {
                    uint2 t = __ldg(g.Rp + idx);
                    int slot = tbl_find(keys, mask, t.y, g.seed_slot);
                    unsigned long long v = w[slot];
                    if (v && (uint32_t)t.x < (uint32_t)g.a_domain) {
                        atomicAdd(g.cnt + t.x, v);
                        acc += v;
                    }
                }
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
        uint32_t cend = build_chunk(g.Rp, pos, r1, keys, cap, g.seed_slot, max_tuples, &nd,
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
            alist[atomicAdd(&start[slot], 1u)] = (int32_t)t.x;
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

size_t lin_agg_smem(uint32_t cap_log2, int mode) {
    uint32_t cap = 1u << cap_log2;
    return align256((cap + 1) * 4) + (size_t)(cap + 1) * (mode == 1 ? 8 : 4);
}

size_t lin_rows_smem(uint32_t cap_log2, uint32_t max_tuples) {
    uint32_t cap = 1u << cap_log2;
    return 3 * align256((cap + 1) * 4) + (size_t)max_tuples * 4;
}

cudaError_t lin_agg_launch(const LinArgs &g, int mode, cudaStream_t st) {
    if (g.I == 0) return cudaSuccess;
    size_t smem = lin_agg_smem(g.cap_log2, mode);
    cudaError_t e;
    if (mode == 1) {
        e = cudaFuncSetAttribute(k_lin_agg<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_lin_agg<1><<<g.I, LT, smem, st>>>(g);
    } else {
        e = cudaFuncSetAttribute(k_lin_agg<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_lin_agg<0><<<g.I, LT, smem, st>>>(g);
    }
    return cudaGetLastError();
}

cudaError_t lin_rows_launch(const LinArgs &g, const unsigned long long *base, int32_t *rows,
                            long long capacity, long long *n_rows, uint32_t max_tuples,
                            cudaStream_t st) {
    k_rows_check<<<1, 1, 0, st>>>(base, g.I, capacity, n_rows, g.st);
    if (g.I == 0) return cudaGetLastError();
    size_t smem = lin_rows_smem(g.cap_log2, max_tuples);
    cudaError_t e = cudaFuncSetAttribute(k_lin_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_lin_rows<<<g.I, LT, smem, st>>>(g, base, (int4 *)rows, capacity, max_tuples);
    return cudaGetLastError();
}

}  // namespace mwj
