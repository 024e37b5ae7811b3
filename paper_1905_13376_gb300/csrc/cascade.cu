// cascade.cu -- the cascade of binary hash joins (Section 6.3).
//
// Join 1 computes I(A,B,C) = R(A,B) |x| S(B,C) and writes it to HBM; join 2
// computes I |x| T.  Both joins use the same machinery as the 3-way join, so
// the comparison isolates what the paper measures, the cost of materialising
// and re-reading the intermediate relation:
//
//   join 1   R and S partitioned by H(B); per work item (bucket, S chunk) the
//            S chunk is kept on chip as b -> [c] lists and R_i streams past
//            it; two passes (count, then write at scanned positions) emit I
//            as three int32 columns.  The rows of one R tuple are adjacent.
//   join 2   linear: I streams past T's C table (one L2-resident table for
//            the counts, bucket images with D lists for rows), the paper's
//            "load partitions of T on chip while streaming I".
//            cyclic: I and T are partitioned by the same hash of (C, A) and
//            each T bucket is kept on chip as a (c, a) multiset while the
//            matching I bucket streams past it.
//
// I is produced in chunks that fit the workspace (the paper spills it to
// SSD when it exceeds DRAM; here it stays in HBM, chunk by chunk).  The host
// reads the per-item row counts to size the chunks, so the call synchronises
// its stream.
#include <algorithm>
#include <vector>

#include "api_internal.h"
#include "prof.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr int KT = 512;
constexpr uint32_t SCAP = 4096;     // S tuples per join-1 chunk
constexpr uint32_t SSLOTS = 8192;   // b-table slots (2 x SCAP)
constexpr uint32_t TCAP2 = 2048;    // T tuples per join-2 (cyclic) chunk
constexpr uint32_t TSLOTS2 = 4096;

struct Item {
    uint32_t bucket, a0, a1;   // bucket and a [a0, a1) range of its build side
};

struct J1Smem {
    uint32_t keys[SSLOTS + 1];
    uint32_t deg[SSLOTS + 1];
    uint32_t start[SSLOTS + 1];
    int32_t clist[SCAP];
};

struct J1Args {
    const uint2 *Rp;
    const uint32_t *offR;
    const uint2 *Sp;
    const Item *items;
    uint32_t seed_slot;
    unsigned long long *item_rows;          // pass 0
    const unsigned long long *item_base;    // pass 1: chunk-relative first row of each item
    int32_t *Ia, *Ib, *Ic;
    unsigned long long room;
    DevStatus *st;
};

// One CTA per work item of join 1.  PASS 0 counts rows per item; PASS 1
// writes them.
template <int PASS>
__global__ void __launch_bounds__(KT) k_join1(J1Args g, uint32_t first) {
    extern __shared__ __align__(16) unsigned char smraw[];
    J1Smem &sm = *(J1Smem *)smraw;
    __shared__ uint32_t scan_scratch[33];
    __shared__ uint32_t carry;
    __shared__ unsigned long long red[32];
    __shared__ unsigned long long cursor;
    const uint32_t item = first + blockIdx.x;
    const Item it = g.items[item];
    const uint32_t r0 = g.offR[it.bucket], r1 = g.offR[it.bucket + 1];
    const uint32_t lane = threadIdx.x & 31;
    // S chunk as b -> [c]
    for (uint32_t q = threadIdx.x; q <= SSLOTS; q += KT) {
        sm.keys[q] = (q < SSLOTS) ? kEmptyKey : 0u;
        sm.deg[q] = 0u;
    }
    if (threadIdx.x == 0) {
        carry = 0;
        cursor = (PASS == 1) ? g.item_base[item] : 0ull;
    }
    __syncthreads();
    for (uint32_t s = it.a0 + threadIdx.x; s < it.a1; s += KT) {
        uint2 tu = __ldg(g.Sp + s);
        bool fresh;
        int slot = tbl_insert(sm.keys, SSLOTS - 1, tu.x, g.seed_slot, &fresh);
        if (slot >= 0) atomicAdd(&sm.deg[slot], 1u);
        else set_status(g.st, MWJ_ERR_CHECK, 21);
    }
    __syncthreads();
    for (uint32_t b0 = 0; b0 <= SSLOTS; b0 += KT) {
        uint32_t q = b0 + threadIdx.x;
        uint32_t d = (q <= SSLOTS) ? sm.deg[q] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan_u32(d, scan_scratch, &tot);
        if (q <= SSLOTS) sm.start[q] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    for (uint32_t s = it.a0 + threadIdx.x; s < it.a1; s += KT) {
        uint2 tu = __ldg(g.Sp + s);
        int slot = tbl_find(sm.keys, SSLOTS - 1, tu.x, g.seed_slot);
        if (slot >= 0) {
            uint32_t p = atomicAdd(&sm.start[slot], 1u);
            if (p < SCAP) sm.clist[p] = (int32_t)tu.y;
        }
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q <= SSLOTS; q += KT) sm.start[q] -= sm.deg[q];
    __syncthreads();

    unsigned long long acc = 0;
    for (uint32_t w0 = r0 + (threadIdx.x & ~31u); w0 < r1; w0 += KT) {
        const uint32_t idx = w0 + lane;
        uint32_t a = 0, b = 0, n = 0, stt = 0;
        if (idx < r1) {
            uint2 tu = __ldg(g.Rp + idx);
            a = tu.x;
            b = tu.y;
            int slot = tbl_find(sm.keys, SSLOTS - 1, b, g.seed_slot);
            if (slot >= 0) {
                n = sm.deg[slot];
                stt = sm.start[slot];
            }
        }
        if (PASS == 0) {
            acc += n;
            continue;
        }
        uint32_t incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += y;
        }
        const uint32_t W = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t excl = incl - n;
        unsigned long long wb = 0;
        if (lane == 0 && W) wb = atomicAdd(&cursor, (unsigned long long)W);
        wb = __shfl_sync(0xffffffffu, wb, 0);
        for (uint32_t base = 0; base < W; base += 32) {
            const uint32_t wi = base + lane;
            int olo = 0, ohi = 31;
            const uint32_t q = (wi < W) ? wi : 0u;
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                int mid = (olo + ohi) >> 1;
                uint32_t v = __shfl_sync(0xffffffffu, incl, mid);
                if (v > q) ohi = mid; else olo = mid + 1;
            }
            const uint32_t oa = __shfl_sync(0xffffffffu, a, olo);
            const uint32_t ob = __shfl_sync(0xffffffffu, b, olo);
            const uint32_t ost = __shfl_sync(0xffffffffu, stt, olo);
            const uint32_t oex = __shfl_sync(0xffffffffu, excl, olo);
            if (wi < W) {
                const uint32_t ci = ost + (wi - oex);
                const unsigned long long p = wb + wi;
                if (p < g.room && ci < SCAP) {
                    g.Ia[p] = (int32_t)oa;
                    g.Ib[p] = (int32_t)ob;
                    g.Ic[p] = sm.clist[ci];
                } else {
                    set_status(g.st, MWJ_ERR_CHECK, 22);
                }
            }
        }
    }
    if (PASS == 0) {
        unsigned long long tot = block_sum_u64(acc, red);
        if (threadIdx.x == 0) g.item_rows[item] = tot;
    }
}

// ---- join 2, linear, count modes: stream I past T's single table ---------
template <int MODE>
__global__ void __launch_bounds__(KT) k_join2_lin(const int32_t *__restrict__ Ia,
                                                  const int32_t *__restrict__ Ic, uint64_t n,
                                                  TImg T, int32_t a_domain,
                                                  unsigned long long *__restrict__ cnt,
                                                  unsigned long long *__restrict__ total) {
    __shared__ unsigned long long red[32];
    const uint32_t tmask = __ldg(T.meta);
    unsigned long long acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * KT * 4;
    for (uint64_t r = ((uint64_t)blockIdx.x * KT + threadIdx.x) * 4; r < n; r += stride) {
        int32_t av[4], cv[4];
        const uint32_t m = (uint32_t)min((uint64_t)4, n - r);
        if (m == 4) {
            int4 a4 = __ldg((const int4 *)(Ia + r));
            int4 c4 = __ldg((const int4 *)(Ic + r));
            av[0] = a4.x; av[1] = a4.y; av[2] = a4.z; av[3] = a4.w;
            cv[0] = c4.x; cv[1] = c4.y; cv[2] = c4.z; cv[3] = c4.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                av[k] = (k < (int)m) ? __ldg(Ia + r + k) : 0;
                cv[k] = (k < (int)m) ? __ldg(Ic + r + k) : 0;
            }
        }
        uint32_t ts[4];
        unsigned long long v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ts[k] = slot_of((uint32_t)cv[k], T.seed_slot, tmask);
            v[k] = (k < (int)m) ? __ldg((const unsigned long long *)(T.img + ts[k])) : kEmpty64;
        }
        int32_t cur = 0;
        unsigned long long run = 0;
        bool have = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k >= (int)m) break;
            unsigned long long x = v[k];
            uint32_t s = ts[k];
            for (uint32_t it = 0; it < tmask && x != kEmpty64 && (uint32_t)x != (uint32_t)cv[k]; ++it) {
                s = (s + 1) & tmask;
                x = __ldg((const unsigned long long *)(T.img + s));
            }
            const uint32_t d = (x != kEmpty64 && (uint32_t)x == (uint32_t)cv[k]) ? (uint32_t)(x >> 32) : 0u;
            if (!d) continue;
            acc += d;
            if (MODE == 1 && (uint32_t)av[k] < (uint32_t)a_domain) {
                if (have && av[k] == cur) {
                    run += d;
                } else {
                    if (have) atomicAdd(cnt + cur, run);
                    cur = av[k];
                    run = d;
                    have = true;
                }
            }
        }
        if (MODE == 1 && have) atomicAdd(cnt + cur, run);
    }
    unsigned long long tot = block_sum_u64(acc, red);
    if (threadIdx.x == 0 && tot) atomicAdd(total, tot);
}

// ---- join 2, linear, rows: two passes over contiguous row ranges ---------
// CTA q owns rows [q*per, (q+1)*per).  PASS 0 stores the range's output count,
// PASS 1 writes (a,b,c,d) from base[q].
template <int PASS>
__global__ void __launch_bounds__(KT) k_join2_lin_rows(const int32_t *__restrict__ Ia,
                                                       const int32_t *__restrict__ Ib,
                                                       const int32_t *__restrict__ Ic, uint64_t n,
                                                       uint64_t per, TImg T,
                                                       unsigned long long *__restrict__ cta_rows,
                                                       const unsigned long long *__restrict__ base,
                                                       unsigned long long out_off, int4 *rows,
                                                       long long capacity, DevStatus *st) {
    __shared__ unsigned long long red[32];
    __shared__ unsigned long long cursor;
    const uint64_t lo = (uint64_t)blockIdx.x * per, hi = min(n, lo + per);
    const uint32_t lane = threadIdx.x & 31;
    if (threadIdx.x == 0) cursor = (PASS == 1) ? out_off + base[blockIdx.x] : 0ull;
    __syncthreads();
    unsigned long long acc = 0;
    for (uint64_t w0 = lo + (threadIdx.x & ~31u); w0 < hi; w0 += KT) {
        const uint64_t r = w0 + lane;
        uint32_t d = 0, tst = 0;
        int32_t a = 0, b = 0, c = 0;
        if (r < hi) {
            a = __ldg(Ia + r);
            c = __ldg(Ic + r);
            d = timg_deg_start(T, c, &tst);
            if (PASS == 1) b = __ldg(Ib + r);
        }
        if (PASS == 0) {
            acc += d;
            continue;
        }
        unsigned long long incl = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += y;
        }
        const unsigned long long W = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long wb = 0;
        if (lane == 0 && W) wb = atomicAdd(&cursor, W);
        wb = __shfl_sync(0xffffffffu, wb, 0);
        unsigned long long p = wb + incl - d;
        for (uint32_t e = 0; e < d; ++e, ++p) {
            if (p < (unsigned long long)capacity)
                rows[p] = make_int4(a, b, c, __ldg(T.dlist + tst + e));
            else
                set_status(st, MWJ_ERR_CHECK, 23);
        }
    }
    if (PASS == 0) {
        unsigned long long tot = block_sum_u64(acc, red);
        if (threadIdx.x == 0) cta_rows[blockIdx.x] = tot;
    }
}

// ---- join 2, cyclic: T bucket as a (c,a) multiset, I bucket streamed ----
struct J2Smem {
    unsigned long long keys[TSLOTS2];
    uint32_t cntv[TSLOTS2 + 1];
};

__device__ __forceinline__ uint32_t h2(uint32_t c, uint32_t a, uint32_t seed) {
    return mix32(c ^ mix32(a ^ seed));
}

template <int PASS>
__global__ void __launch_bounds__(KT) k_join2_cyc(const uint2 *__restrict__ T2,   // (c,a) by bucket
                                                  const uint2 *__restrict__ I2,   // (c,a) by bucket
                                                  const int32_t *__restrict__ Ib2,
                                                  const uint32_t *__restrict__ offI2,
                                                  const Item *__restrict__ items, uint32_t seed,
                                                  int32_t a_domain, unsigned long long *cnt,
                                                  unsigned long long *total,
                                                  unsigned long long *item_rows,
                                                  const unsigned long long *item_base,
                                                  unsigned long long out_off, int32_t *rows,
                                                  long long capacity, DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smraw[];
    J2Smem &sm = *(J2Smem *)smraw;
    __shared__ unsigned long long red[32];
    __shared__ unsigned long long cursor;
    const Item it = items[blockIdx.x];
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t q = threadIdx.x; q <= TSLOTS2; q += KT) {
        if (q < TSLOTS2) sm.keys[q] = kEmpty64;
        sm.cntv[q] = 0u;
    }
    if (threadIdx.x == 0) cursor = (PASS == 1) ? out_off + item_base[blockIdx.x] : 0ull;
    __syncthreads();
    for (uint32_t q = it.a0 + threadIdx.x; q < it.a1; q += KT) {
        uint2 tu = __ldg(T2 + q);
        const unsigned long long key = ((unsigned long long)tu.x << 32) | tu.y;
        if (key == kEmpty64) {
            atomicAdd(&sm.cntv[TSLOTS2], 1u);
            continue;
        }
        uint32_t h = h2(tu.x, tu.y, seed) & (TSLOTS2 - 1);
        bool done = false;
        for (uint32_t k = 0; k < TSLOTS2; ++k) {
            unsigned long long v = sm.keys[h];
            if (v == kEmpty64) {
                unsigned long long old = atomicCAS(&sm.keys[h], kEmpty64, key);
                if (old == kEmpty64 || old == key) {
                    atomicAdd(&sm.cntv[h], 1u);
                    done = true;
                    break;
                }
                v = old;
            }
            if (v == key) {
                atomicAdd(&sm.cntv[h], 1u);
                done = true;
                break;
            }
            h = (h + 1) & (TSLOTS2 - 1);
        }
        if (!done) set_status(st, MWJ_ERR_CHECK, 24);
    }
    __syncthreads();
    const uint32_t i0 = offI2[it.bucket], i1 = offI2[it.bucket + 1];
    unsigned long long acc = 0;
    for (uint32_t w0 = i0 + (threadIdx.x & ~31u); w0 < i1; w0 += KT) {
        const uint32_t r = w0 + lane;
        uint32_t m = 0, c = 0, a = 0;
        if (r < i1) {
            uint2 tu = __ldg(I2 + r);
            c = tu.x;
            a = tu.y;
            const unsigned long long key = ((unsigned long long)c << 32) | a;
            if (key == kEmpty64) {
                m = sm.cntv[TSLOTS2];
            } else {
                uint32_t h = h2(c, a, seed) & (TSLOTS2 - 1);
                for (uint32_t k = 0; k < TSLOTS2; ++k) {
                    unsigned long long v = sm.keys[h];
                    if (v == key) { m = sm.cntv[h]; break; }
                    if (v == kEmpty64) break;
                    h = (h + 1) & (TSLOTS2 - 1);
                }
            }
        }
        if (PASS == 0) {
            acc += m;
            if (cnt && m && (uint32_t)a < (uint32_t)a_domain) atomicAdd(cnt + a, (unsigned long long)m);
            continue;
        }
        uint32_t incl = m;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += y;
        }
        const uint32_t W = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long wb = 0;
        if (lane == 0 && W) wb = atomicAdd(&cursor, (unsigned long long)W);
        wb = __shfl_sync(0xffffffffu, wb, 0);
        unsigned long long p = wb + incl - m;
        const int32_t b = (m && r < i1) ? __ldg(Ib2 + r) : 0;
        for (uint32_t e = 0; e < m; ++e, ++p) {
            if (p < (unsigned long long)capacity) {
                rows[3 * p] = (int32_t)a;
                rows[3 * p + 1] = b;
                rows[3 * p + 2] = (int32_t)c;
            } else {
                set_status(st, MWJ_ERR_CHECK, 25);
            }
        }
    }
    if (PASS == 0) {
        unsigned long long tot = block_sum_u64(acc, red);
        if (threadIdx.x == 0) {
            if (item_rows) item_rows[blockIdx.x] = tot;
            if (tot && total) atomicAdd(total, tot);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct CascPlan {
    uint32_t I1;        // H(B) buckets of join 1
    uint32_t JT;        // T buckets (linear)
    uint32_t P2a, P2b;  // (c, a) buckets of join 2 (cyclic)
    size_t max_items1, max_items2;
    size_t room;        // rows of I per chunk
    int kind;
    bool rows;
};

struct CascLayout {
    uint2 *Rp, *Sp;
    uint32_t *offR, *offS;
    // linear T
    uint32_t *Tk, *offT, *ekey, *ecnt, *ecount, *meta, *capT, *startT;
    uint2 *Tp;
    uint64_t *img;
    int32_t *dlist;
    // cyclic T and I partitions
    uint2 *T2, *I2;
    int32_t *Ib2;
    uint32_t *offT2, *offI2;
    // items
    Item *items1, *items2;
    unsigned long long *rows1, *base1, *rows2, *base2;
    void *scan_tmp;
    // I chunk
    int32_t *Ia, *Ib, *Ic;
    void *pscratch;
    size_t pscratch_bytes;
};

uint32_t pow2_le_sqrt(uint32_t P) {
    uint32_t r = 1;
    while ((uint64_t)(r * 2) * (r * 2) <= P) r *= 2;
    return r;
}

size_t casc_layout(Arena &A, const CascPlan &p, const mwj_rel &R, const mwj_rel &S,
                   const mwj_rel &T, int num_sms, CascLayout &L) {
    const size_t room = p.room;
    L.Rp = A.take<uint2>(R.n + 2);
    L.offR = A.take<uint32_t>(p.I1 + 1);
    L.Sp = A.take<uint2>(S.n + 2);
    L.offS = A.take<uint32_t>(p.I1 + 1);
    const uint32_t P2 = p.P2a * p.P2b;
    if (p.kind == MWJ_LINEAR) {
        L.offT = A.take<uint32_t>(p.JT + 1);
        if (p.rows) {
            L.Tk = nullptr;
            L.Tp = A.take<uint2>(T.n + 2);
            L.img = A.take<uint64_t>(2 * (size_t)T.n + 4);
            L.capT = A.take<uint32_t>(p.JT + 1);
            L.startT = A.take<uint32_t>(2 * (size_t)T.n + 4);
            L.dlist = A.take<int32_t>(T.n + 4);
            L.ekey = L.ecnt = L.ecount = L.meta = nullptr;
        } else {
            L.Tk = A.take<uint32_t>(T.n + 4);
            L.Tp = nullptr;
            L.img = A.take<uint64_t>(single_table_slots(T.n));
            L.ekey = A.take<uint32_t>(T.n + 4);
            L.ecnt = A.take<uint32_t>(T.n + 4);
            L.ecount = A.take<uint32_t>(p.JT + 1);
            L.meta = A.take<uint32_t>(4);
            L.capT = L.startT = nullptr;
            L.dlist = nullptr;
        }
        L.T2 = L.I2 = nullptr;
        L.Ib2 = nullptr;
        L.offT2 = L.offI2 = nullptr;
    } else {
        L.T2 = A.take<uint2>(T.n + 2);
        L.offT2 = A.take<uint32_t>(P2 + 1);
        L.I2 = A.take<uint2>(room + 2);
        L.Ib2 = p.rows ? A.take<int32_t>(room + 4) : nullptr;
        L.offI2 = A.take<uint32_t>(P2 + 1);
        L.Tk = L.offT = L.ekey = L.ecnt = L.ecount = L.meta = L.capT = L.startT = nullptr;
        L.Tp = nullptr;
        L.img = nullptr;
        L.dlist = nullptr;
    }
    L.items1 = A.take<Item>(p.max_items1);
    L.rows1 = A.take<unsigned long long>(p.max_items1 + 1);
    L.base1 = A.take<unsigned long long>(p.max_items1 + 2);
    L.items2 = A.take<Item>(p.max_items2);
    L.rows2 = A.take<unsigned long long>(p.max_items2 + 1);
    L.base2 = A.take<unsigned long long>(p.max_items2 + 2);
    size_t sc = p.max_items1 > p.max_items2 ? p.max_items1 : p.max_items2;
    L.scan_tmp = A.take<char>(scan_scratch_bytes(sc + 2));
    L.Ia = A.take<int32_t>(room + 4);
    L.Ib = A.take<int32_t>(room + 4);
    L.Ic = A.take<int32_t>(room + 4);
    size_t ps = part_scratch_bytes(R.n, p.I1, num_sms);
    ps = std::max(ps, part_scratch_bytes(S.n, p.I1, num_sms));
    if (p.kind == MWJ_LINEAR) ps = std::max(ps, part_scratch_bytes(T.n, p.JT, num_sms));
    else {
        ps = std::max(ps, part_scratch_bytes(T.n, P2, num_sms));
        ps = std::max(ps, part_scratch_bytes((int64_t)std::min<size_t>(room, 0x7FFFFFFF), P2, num_sms));
    }
    L.pscratch = A.take<char>(ps);
    L.pscratch_bytes = ps;
    return A.used;
}

CascPlan casc_plan(mwj_ctx *ctx, int kind, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                   mwj_mode mode, size_t room) {
    CascPlan p;
    p.kind = kind;
    p.rows = (mode == MWJ_MATERIALIZE);
    mwj_shares sh;
    plan_linear_default(ctx, R, S, T, &sh);
    p.I1 = (uint32_t)sh.s[0];
    uint64_t want = (uint64_t)(T.n + 8191) / 8192;
    p.JT = pow2_at_least(want ? want : 1);
    if (p.JT > kMaxBuckets) p.JT = kMaxBuckets;
    if (p.rows && kind == MWJ_LINEAR) {
        uint64_t w2 = (uint64_t)(T.n + 2047) / 2048;
        p.JT = pow2_at_least(w2 ? w2 : 1);
        if (p.JT > kMaxBuckets) p.JT = kMaxBuckets;
    }
    uint64_t P2 = pow2_at_least((uint64_t)(T.n + 1023) / 1024 + 1);
    if (P2 > kMaxBuckets) P2 = kMaxBuckets;
    p.P2a = pow2_le_sqrt((uint32_t)P2);
    p.P2b = (uint32_t)P2 / p.P2a;
    p.max_items1 = p.I1 + (size_t)S.n / SCAP + 1;
    // join 2: work items (cyclic) or one count per CTA of the row pass (linear)
    p.max_items2 = (kind == MWJ_CYCLIC) ? (size_t)P2 + (size_t)T.n / TCAP2 + 1
                                        : (size_t)ctx->dev.num_sms * 4;
    p.room = room;
    return p;
}

constexpr size_t kDefaultRoom = 1u << 24;   // rows of I per chunk in the default workspace

}  // namespace

mwj_status cascade_workspace(mwj_ctx *ctx, int kind, const mwj_rel &R, const mwj_rel &S,
                             const mwj_rel &T, mwj_mode mode, size_t *bytes) {
    if (kind != MWJ_LINEAR && kind != MWJ_CYCLIC) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad kind");
    CascPlan p = casc_plan(ctx, kind, R, S, T, mode, kDefaultRoom);
    Arena A(nullptr, 0);
    CascLayout L;
    *bytes = casc_layout(A, p, R, S, T, ctx->dev.num_sms, L);
    return MWJ_OK;
}

}  // namespace mwj

using namespace mwj;

namespace {

mwj_status sync_fail(mwj_ctx *ctx, cudaError_t e, const char *w) { return cuda_fail(ctx, e, w); }

}  // namespace

extern "C" mwj_status mwj_cascade_join(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T,
                                       const mwj_out *out, void *workspace, size_t ws_bytes,
                                       void *stream) {
    if (!ctx || !out) return MWJ_ERR_INVALID_ARG;
    ApiScope api_scope(&ctx->prof);
    if (kind != MWJ_LINEAR && kind != MWJ_CYCLIC) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad kind");
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    mwj_status s = check_out(ctx, out, kind == MWJ_LINEAR ? 4 : 3);
    if (s != MWJ_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const bool rows = out->mode == MWJ_MATERIALIZE;

    // room for I: whatever the workspace holds beyond the fixed part
    CascPlan p = casc_plan(ctx, kind, R, S, T, out->mode, 0);
    {
        Arena A0(nullptr, 0);
        CascLayout L0;
        size_t fixed = casc_layout(A0, p, R, S, T, ctx->dev.num_sms, L0);
        if (!workspace || ws_bytes <= fixed + 4096)
            return fail(ctx, MWJ_ERR_WORKSPACE, "workspace of %zu bytes, need more than %zu",
                        ws_bytes, fixed);
        const size_t per_row = (kind == MWJ_LINEAR) ? 12 : (rows ? 24 : 20);
        size_t room = (ws_bytes - fixed - 4096) / per_row;
        for (;;) {
            p.room = room;
            Arena A1(nullptr, 0);
            CascLayout L1;
            if (casc_layout(A1, p, R, S, T, ctx->dev.num_sms, L1) <= ws_bytes || room < 1024) break;
            room -= room / 64 + 64;
        }
        if (room > 0x7FFFFFFFull) room = 0x7FFFFFFF;
        p.room = room;
    }
    Arena A(workspace, ws_bytes);
    CascLayout L;
    casc_layout(A, p, R, S, T, ctx->dev.num_sms, L);
    if (A.overflow) return fail(ctx, MWJ_ERR_WORKSPACE, "workspace too small");

    const Seeds &sd = ctx->seeds;
    const int sms = ctx->dev.num_sms;
    cudaError_t e;
    if ((e = cudaMemsetAsync(out->total, 0, sizeof(int64_t), st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset total");
    if (out->mode == MWJ_COUNT_GROUP_BY_A &&
        (e = cudaMemsetAsync(out->group_counts, 0, sizeof(int64_t) * (size_t)out->a_domain, st)) !=
            cudaSuccess)
        return cuda_fail(ctx, e, "memset group_counts");

    // join 1 inputs: R and S by H(B)
    PartSpec pr{1, sd.B, p.I1, -1, 0, 1};
    pr.st = ctx->status;
    if (out->mode == MWJ_COUNT_GROUP_BY_A) pr.dom = (uint32_t)out->a_domain;
    if ((e = part_run(R.x, R.y, R.n, pr, PAY_PAIR, L.Rp, L.offR, L.pscratch, L.pscratch_bytes, sms,
                      st)) != cudaSuccess)
        return cuda_fail(ctx, e, "partition R");
    PartSpec ps{0, sd.B, p.I1, -1, 0, 1};
    ps.st = ctx->status;
    if ((e = part_run(S.x, S.y, S.n, ps, PAY_PAIR, L.Sp, L.offS, L.pscratch, L.pscratch_bytes, sms,
                      st)) != cudaSuccess)
        return cuda_fail(ctx, e, "partition S");
    // join 2's T side
    TImg timg{};
    PartSpec p2{0, sd.C ^ 0x5bd1e995u, p.P2a, 1, sd.A ^ 0x5bd1e995u, p.P2b};
    p2.st = ctx->status;
    if (kind == MWJ_LINEAR) {
        PartSpec pt{0, sd.C, p.JT, -1, 0, 1};
        pt.st = ctx->status;
        e = part_run(T.x, T.y, T.n, pt, rows ? PAY_PAIR : PAY_X, rows ? (void *)L.Tp : (void *)L.Tk,
                     L.offT, L.pscratch, L.pscratch_bytes, sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "partition T");
        if (rows) {
            e = tables_build(nullptr, L.Tp, L.offT, p.JT, sd.slot2, L.img, L.capT, L.startT, L.dlist,
                             ctx->status, sms, st);
            timg = TImg{L.img, L.offT, L.capT, L.startT, L.dlist, nullptr, p.JT, sd.C, sd.slot2};
        } else {
            e = single_table_build(L.Tk, L.offT, p.JT, sd.slot2, L.ekey, L.ecnt, L.ecount, L.meta,
                                   L.img, ctx->status, sms, st);
            timg = TImg{L.img, nullptr, nullptr, nullptr, nullptr, L.meta, 0u, sd.C, sd.slot2};
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "T tables");
    } else {
        e = part_run(T.x, T.y, T.n, p2, PAY_PAIR, L.T2, L.offT2, L.pscratch, L.pscratch_bytes, sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "partition T");
    }

    // ---- plan join 1's items (and join 2's for cyclic) on the host ----
    std::vector<uint32_t> offR(p.I1 + 1), offS(p.I1 + 1);
    cudaMemcpyAsync(offR.data(), L.offR, offR.size() * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(offS.data(), L.offS, offS.size() * 4, cudaMemcpyDeviceToHost, st);
    const uint32_t P2 = p.P2a * p.P2b;
    std::vector<uint32_t> offT2;
    if (kind == MWJ_CYCLIC) {
        offT2.resize(P2 + 1);
        cudaMemcpyAsync(offT2.data(), L.offT2, offT2.size() * 4, cudaMemcpyDeviceToHost, st);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return sync_fail(ctx, e, "plan sync");
    std::vector<Item> it1;
    for (uint32_t i = 0; i < p.I1; ++i) {
        if (offR[i] == offR[i + 1]) continue;
        for (uint32_t a = offS[i]; a < offS[i + 1]; a += SCAP)
            it1.push_back(Item{i, a, std::min(offS[i + 1], a + SCAP)});
    }
    std::vector<Item> it2;
    if (kind == MWJ_CYCLIC)
        for (uint32_t q = 0; q < P2; ++q)
            for (uint32_t a = offT2[q]; a < offT2[q + 1]; a += TCAP2)
                it2.push_back(Item{q, a, std::min(offT2[q + 1], a + TCAP2)});
    if (it1.size() > p.max_items1 || it2.size() > p.max_items2)
        return fail(ctx, MWJ_ERR_CHECK, "cascade item planning overflow");
    if (!it1.empty())
        cudaMemcpyAsync(L.items1, it1.data(), it1.size() * sizeof(Item), cudaMemcpyHostToDevice, st);
    if (!it2.empty())
        cudaMemcpyAsync(L.items2, it2.data(), it2.size() * sizeof(Item), cudaMemcpyHostToDevice, st);

    J1Args g1{};
    g1.Rp = L.Rp; g1.offR = L.offR; g1.Sp = L.Sp; g1.items = L.items1;
    g1.seed_slot = sd.slot; g1.item_rows = L.rows1; g1.item_base = L.base1;
    g1.Ia = L.Ia; g1.Ib = L.Ib; g1.Ic = L.Ic; g1.room = p.room; g1.st = ctx->status;
    const size_t sm1 = sizeof(J1Smem);
    cudaFuncSetAttribute(k_join1<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    cudaFuncSetAttribute(k_join1<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    const uint32_t n1 = (uint32_t)it1.size();
    if (n1) {
        ProfScope ps_("cascade_join1_count", st);
        k_join1<0><<<n1, KT, sm1, st>>>(g1, 0);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "join 1 count");
    std::vector<unsigned long long> r1(n1);
    if (n1) cudaMemcpyAsync(r1.data(), L.rows1, n1 * 8, cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return sync_fail(ctx, e, "join 1 sync");

    const size_t sm2 = sizeof(J2Smem);
    cudaFuncSetAttribute(k_join2_cyc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    cudaFuncSetAttribute(k_join2_cyc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    const uint32_t n2 = (uint32_t)it2.size();
    unsigned long long out_off = 0;       // rows emitted so far (row output)
    bool over = false;
    std::vector<unsigned long long> base(n1 + 1);
    const unsigned j2_grid = (unsigned)sms * 4;   // = p.max_items2 for the linear row pass

    // ---- chunks of consecutive items whose I fits the room ----
    for (uint32_t c0 = 0; c0 < n1;) {
        unsigned long long acc = 0;
        uint32_t c1 = c0;
        while (c1 < n1 && acc + r1[c1] <= p.room) acc += r1[c1++];
        if (c1 == c0) return fail(ctx, MWJ_ERR_WORKSPACE, "one join-1 item needs %llu rows of I, "
                                  "the workspace holds %zu", r1[c0], p.room);
        if (acc == 0) {
            c0 = c1;
            continue;
        }
        // chunk-relative bases of the items
        unsigned long long run = 0;
        for (uint32_t k = c0; k < c1; ++k) {
            base[k] = run;
            run += r1[k];
        }
        cudaMemcpyAsync(L.base1 + c0, base.data() + c0, (c1 - c0) * 8, cudaMemcpyHostToDevice, st);
        {
            ProfScope ps_("cascade_join1_write", st);
            k_join1<1><<<c1 - c0, KT, sm1, st>>>(g1, c0);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "join 1 write");
        const uint64_t nI = acc;

        if (kind == MWJ_LINEAR && !rows) {
            ProfScope ps_("cascade_join2", st);
            if (out->mode == MWJ_COUNT_GROUP_BY_A)
                k_join2_lin<1><<<j2_grid, KT, 0, st>>>(L.Ia, L.Ic, nI, timg, out->a_domain,
                                                       (unsigned long long *)out->group_counts,
                                                       (unsigned long long *)out->total);
            else
                k_join2_lin<0><<<j2_grid, KT, 0, st>>>(L.Ia, L.Ic, nI, timg, 0, nullptr,
                                                       (unsigned long long *)out->total);
        } else if (kind == MWJ_LINEAR) {
            const uint64_t per = (nI + j2_grid - 1) / j2_grid;
            {
                ProfScope ps_("cascade_join2_count", st);
                k_join2_lin_rows<0><<<j2_grid, KT, 0, st>>>(L.Ia, L.Ib, L.Ic, nI, per, timg, L.rows2,
                                                            nullptr, 0, nullptr, 0, ctx->status);
            }
            if ((e = scan_excl_u64((const uint64_t *)L.rows2, (uint64_t *)L.base2, j2_grid, true,
                                   L.scan_tmp, st)) != cudaSuccess)
                return cuda_fail(ctx, e, "join 2 scan");
            unsigned long long ctot = 0;
            cudaMemcpyAsync(&ctot, L.base2 + j2_grid, 8, cudaMemcpyDeviceToHost, st);
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return sync_fail(ctx, e, "join 2 sync");
            if (!over && out_off + ctot <= (unsigned long long)out->capacity) {
                ProfScope ps_("cascade_join2_write", st);
                k_join2_lin_rows<1><<<j2_grid, KT, 0, st>>>(L.Ia, L.Ib, L.Ic, nI, per, timg, nullptr,
                                                            L.base2, out_off, (int4 *)out->rows,
                                                            out->capacity, ctx->status);
            } else {
                over = true;
            }
            out_off += ctot;
        } else {
            // cyclic: I by the same hash of (C, A) as T, then bucket-wise probes
            e = part_run(L.Ic, L.Ia, (int64_t)nI, p2, PAY_PAIR, L.I2, L.offI2, L.pscratch,
                         L.pscratch_bytes, sms, st, rows ? L.Ib : nullptr, rows ? L.Ib2 : nullptr);
            if (e != cudaSuccess)
                return fail(ctx, MWJ_ERR_CUDA, "partition I: %s (%llu rows into %u x %u buckets, scratch %zu of %zu)",
                            cudaGetErrorString(e), (unsigned long long)nI, p.P2a, p.P2b, L.pscratch_bytes,
                            part_scratch_bytes((int64_t)nI, p.P2a * p.P2b, sms));
            if (n2 == 0) {
                c0 = c1;
                continue;
            }
            {
                ProfScope ps_("cascade_join2", st);
                k_join2_cyc<0><<<n2, KT, sm2, st>>>(
                    L.T2, L.I2, L.Ib2, L.offI2, L.items2, sd.slot2, out->a_domain,
                    out->mode == MWJ_COUNT_GROUP_BY_A ? (unsigned long long *)out->group_counts : nullptr,
                    rows ? nullptr : (unsigned long long *)out->total, rows ? L.rows2 : nullptr,
                    nullptr, 0, nullptr, 0, ctx->status);
            }
            if (rows) {
                if ((e = scan_excl_u64((const uint64_t *)L.rows2, (uint64_t *)L.base2, n2, true,
                                       L.scan_tmp, st)) != cudaSuccess)
                    return cuda_fail(ctx, e, "join 2 scan");
                unsigned long long ctot = 0;
                cudaMemcpyAsync(&ctot, L.base2 + n2, 8, cudaMemcpyDeviceToHost, st);
                if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
                    return sync_fail(ctx, e, "join 2 sync");
                if (!over && out_off + ctot <= (unsigned long long)out->capacity) {
                    ProfScope ps_("cascade_join2_write", st);
                    k_join2_cyc<1><<<n2, KT, sm2, st>>>(L.T2, L.I2, L.Ib2, L.offI2, L.items2, sd.slot2,
                                                        0, nullptr, nullptr, nullptr, L.base2, out_off,
                                                        out->rows, out->capacity, ctx->status);
                } else {
                    over = true;
                }
                out_off += ctot;
            }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "join 2");
        c0 = c1;
    }
    if (rows) {
        long long n = (long long)out_off;
        cudaMemcpyAsync(out->n_rows, &n, 8, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(out->total, &n, 8, cudaMemcpyHostToDevice, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return sync_fail(ctx, e, "rows sync");
        if (over)
            return fail(ctx, MWJ_ERR_CAPACITY, "%s (needed %lld rows)", status_text(MWJ_ERR_CAPACITY), n);
    }
    return MWJ_OK;
}
