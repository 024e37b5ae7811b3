// batch.cu -- many independent 3-way joins (linear and cyclic, COUNT(*)) in
// one persistent launch.
//
// The plan (mwj_batch_create) chooses every query's shares on the host from
// the relation sizes alone, lays all partitions and tables out in one
// workspace, and uploads per-query descriptors.  mwj_batch_launch then
// enqueues a fixed sequence of kernels with no host round trip, so the whole
// batch can be captured into a CUDA graph and replayed:
//
//   k_batch_prep   persistent over "segments", largest first: each CTA
//                  partitions one relation of one query entirely in shared
//                  memory (histogram, scan, scatter through shared cursors) --
//                  R by H(B) and S by H(B) for linear queries, R/S/T by the
//                  cube shares for cyclic ones -- or builds a linear query's
//                  T degree table (C -> deg_T(C)) in its own region, which
//                  stays in L2 while the query's items run
//   k_batch_plan   work items of the cyclic tiles (R chunks x T chunks)
//   scan           item offsets over all cyclic tiles of all queries
//   k_batch_join   persistent over one queue: linear items (query, R bucket)
//                  first (sorted by size on the host), then cyclic items
//                  (query, tile, R chunk, T chunk); counts[q] accumulates with
//                  one 64-bit atomic per item.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "api_internal.h"
#include "prof.h"

namespace mwj {
namespace {

constexpr int BTH = 512;
constexpr uint32_t kSegMaxP = 4096;        // buckets per partitioned relation
constexpr uint32_t LCAP = 4096;            // linear R table slots
constexpr uint32_t CRCAP = 2048, CRSLOTS = 4096, CTCAP = 2048, CTSLOTS = 4096;

enum SegKind : uint32_t { SEG_PART = 0, SEG_TTAB = 1 };

struct Seg {
    const int32_t *x, *y;
    uint32_t n;
    uint32_t kind;
    PartSpec sp;            // SEG_PART
    uint2 *out;             // SEG_PART
    uint32_t *off;          // SEG_PART: P + 1
    unsigned long long *tbl;   // SEG_TTAB
    uint32_t tmask;         // SEG_TTAB
};

struct LinQ {               // a linear query's device view
    const uint2 *Rp, *Sp;
    const uint32_t *offR, *offS;
    const unsigned long long *tbl;
    uint32_t tmask, I;
};

struct CycQ {
    const uint2 *Rp, *Sp, *Tp;
    const uint32_t *offR, *offS, *offT;
    uint32_t x, y, z;
    uint32_t tile0;         // first global tile index of this query
    uint32_t q;             // query index (output slot)
};

struct LinItem {
    uint32_t q, lq, i;      // output slot, linear-query index, R bucket
};

struct BatchDev {
    const Seg *segs;
    uint32_t nseg;
    const LinQ *lin;
    const LinItem *litems;
    uint32_t nlitems;
    const CycQ *cyc;
    uint32_t ncyc;
    uint32_t ntiles;        // cyclic tiles over all queries
    const uint32_t *tile_q; // cyclic tile -> CycQ index (searching tile0 is also possible)
    uint32_t seed_slot, seed_slot2;
};

__device__ __forceinline__ uint32_t seg_bucket(int32_t x, int32_t y, const PartSpec &sp) {
    int32_t k1 = sp.col1 ? y : x;
    uint32_t b = bucket_of(k1, sp.seed1, sp.P1);
    if (sp.col2 >= 0) {
        int32_t k2 = sp.col2 ? y : x;
        b = b * sp.P2 + bucket_of(k2, sp.seed2, sp.P2);
    }
    return b;
}

__device__ __forceinline__ void ttab_insert(unsigned long long *tbl, uint32_t mask, uint32_t k,
                                            uint32_t seed, DevStatus *st) {
    uint32_t s = slot_of(k, seed, mask);
    const unsigned long long fresh = (1ull << 32) | (unsigned long long)k;
    for (uint32_t it = 0; it <= mask; ++it) {
        unsigned long long v = tbl[s];
        if (v == kEmpty64) {
            unsigned long long old = atomicCAS(&tbl[s], kEmpty64, fresh);
            if (old == kEmpty64) return;
            v = old;
        }
        if ((uint32_t)v == k) {
            atomicAdd(&tbl[s], 1ull << 32);
            return;
        }
        s = (s + 1) & mask;
    }
    set_status(st, MWJ_ERR_CHECK, 31);
}

// ---- persistent segment kernel --------------------------------------------
__global__ void __launch_bounds__(BTH) k_batch_prep(BatchDev b, unsigned int *counter, DevStatus *st) {
    __shared__ uint32_t hist[kSegMaxP + 1];
    __shared__ uint32_t scan_scratch[33];
    __shared__ uint32_t seg_s, carry;
    for (;;) {
        if (threadIdx.x == 0) seg_s = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t si = seg_s;
        __syncthreads();
        if (si >= b.nseg) break;
        const Seg sg = b.segs[si];
        if (sg.kind == SEG_TTAB) {
            for (uint32_t s = threadIdx.x; s <= sg.tmask; s += BTH) sg.tbl[s] = kEmpty64;
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < sg.n; i += BTH)
                ttab_insert(sg.tbl, sg.tmask, (uint32_t)__ldg(sg.x + i), b.seed_slot2, st);
            __syncthreads();
            continue;
        }
        const uint32_t P = sg.sp.P();
        for (uint32_t k = threadIdx.x; k <= P; k += BTH) hist[k] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < sg.n; i += BTH)
            atomicAdd(&hist[seg_bucket(__ldg(sg.x + i), __ldg(sg.y + i), sg.sp)], 1u);
        __syncthreads();
        // exclusive scan of hist[0..P) -> off[] and cursors
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (uint32_t b0 = 0; b0 < P; b0 += BTH) {
            uint32_t k = b0 + threadIdx.x;
            uint32_t v = (k < P) ? hist[k] : 0u;
            uint32_t tot;
            uint32_t ex = block_excl_scan_u32(v, scan_scratch, &tot);
            if (k < P) {
                hist[k] = carry + ex;
                sg.off[k] = carry + ex;
            }
            __syncthreads();
            if (threadIdx.x == 0) carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) sg.off[P] = sg.n;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < sg.n; i += BTH) {
            int32_t xv = __ldg(sg.x + i), yv = __ldg(sg.y + i);
            uint32_t p = atomicAdd(&hist[seg_bucket(xv, yv, sg.sp)], 1u);
            if (p < sg.n) sg.out[p] = make_uint2((uint32_t)xv, (uint32_t)yv);
            else set_status(st, MWJ_ERR_CHECK, 32);
        }
        __syncthreads();
    }
}

// ---- cyclic tile planning ----------------------------------------------------
__host__ __device__ __forceinline__ uint32_t cdiv(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

struct TileIdx {
    uint32_t i, j, k;
};
__device__ __forceinline__ TileIdx tile_in(uint32_t t, const CycQ &c) {
    TileIdx id;
    id.i = t % c.x;
    uint32_t jk = t / c.x;
    id.k = jk % c.z;
    id.j = jk / c.z;
    return id;
}

__global__ void k_batch_plan(BatchDev b, uint32_t *items) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < b.ntiles; t += gridDim.x * blockDim.x) {
        const CycQ c = b.cyc[b.tile_q[t]];
        const TileIdx id = tile_in(t - c.tile0, c);
        uint32_t rb = id.i * c.y + id.j, sb = id.j * c.z + id.k, tb = id.k * c.x + id.i;
        uint32_t nr = c.offR[rb + 1] - c.offR[rb];
        uint32_t ns = c.offS[sb + 1] - c.offS[sb];
        uint32_t nt = c.offT[tb + 1] - c.offT[tb];
        items[t] = (nr && ns && nt) ? cdiv(nr, CRCAP) * cdiv(nt, CTCAP) : 0u;
    }
}

// ---- the persistent join kernel -------------------------------------------------
struct LinSmem {
    uint32_t keys[LCAP + 1];
    uint32_t deg[LCAP + 1];
};
struct CycSmem {
    uint32_t rkeys[CRSLOTS + 1];
    uint32_t rdeg[CRSLOTS + 1];
    uint32_t rstart[CRSLOTS + 1];
    int32_t alist[CRCAP];
    unsigned long long tkeys[CTSLOTS];
    uint32_t tcnt[CTSLOTS + 1];
};
union JoinSmem {
    LinSmem lin;
    CycSmem cyc;
};

__device__ __forceinline__ uint32_t t_deg(const unsigned long long *tbl, uint32_t mask, uint32_t c,
                                          uint32_t seed) {
    uint32_t s = slot_of(c, seed, mask);
    for (uint32_t it = 0; it <= mask; ++it) {
        unsigned long long v = __ldg(tbl + s);
        if (v == kEmpty64) return 0;
        if ((uint32_t)v == c) return (uint32_t)(v >> 32);
        s = (s + 1) & mask;
    }
    return 0;
}

__device__ __forceinline__ unsigned long long cpack(uint32_t c, uint32_t a) {
    return ((unsigned long long)c << 32) | a;
}
__device__ __forceinline__ uint32_t cpair_hash(uint32_t c, uint32_t a, uint32_t seed) {
    return mix32(c ^ mix32(a ^ seed));
}

// COUNT of one linear item (R bucket i of a query): R_i in shared memory as
// b -> deg_R(b), in chunks that keep the table at most 3/4 full.
__device__ unsigned long long lin_item(const LinQ &L, uint32_t i, LinSmem &sm, uint32_t seed,
                                       uint32_t seed2, uint32_t *nd, DevStatus *st) {
    const uint32_t r0 = L.offR[i], r1 = L.offR[i + 1];
    const uint32_t s0 = L.offS[i], s1 = L.offS[i + 1];
    unsigned long long acc = 0;
    if (r0 >= r1 || s0 >= s1) return 0;
    const uint32_t mask = LCAP - 1;
    const uint32_t rt = round_tuples(LCAP, 4 * BTH);
    for (uint32_t pos = r0; pos < r1;) {
        __syncthreads();
        for (uint32_t q = threadIdx.x; q <= LCAP; q += BTH) {
            sm.keys[q] = (q < LCAP) ? kEmptyKey : 0u;
            sm.deg[q] = 0u;
        }
        if (threadIdx.x == 0) *nd = 0;
        uint32_t cend = pos;
        for (;;) {
            __syncthreads();
            const uint32_t filled = *nd;
            __syncthreads();
            if (cend >= r1 || filled + rt > LCAP - LCAP / 4) break;
            uint32_t fresh_n = 0;
            for (uint32_t k = threadIdx.x; k < rt; k += BTH) {
                const uint32_t idx = cend + k;
                if (idx >= r1) break;
                bool fresh;
                int slot = tbl_insert(sm.keys, mask, __ldg(L.Rp + idx).y, seed, &fresh);
                if (slot < 0) {
                    set_status(st, MWJ_ERR_CHECK, 33);
                    continue;
                }
                fresh_n += fresh;
                atomicAdd(&sm.deg[slot], 1u);
            }
            fresh_n = warp_sum(fresh_n);
            if ((threadIdx.x & 31) == 0 && fresh_n) atomicAdd(nd, fresh_n);
            cend += rt;
        }
        cend = min(cend, r1);
        for (uint32_t s = s0 + threadIdx.x; s < s1; s += BTH) {
            const uint2 t = __ldg(L.Sp + s);
            const int slot = tbl_find(sm.keys, mask, t.x, seed);
            if (slot < 0) continue;
            const uint32_t d = t_deg(L.tbl, L.tmask, t.y, seed2);
            acc += (unsigned long long)sm.deg[slot] * d;
        }
        pos = cend;
    }
    return acc;
}

// COUNT of one cyclic item (tile, R chunk, T chunk).
__device__ unsigned long long cyc_item(const CycQ &c, uint32_t t_local, uint32_t local, CycSmem &sm,
                                       uint32_t seed, uint32_t seed2, uint32_t *carry,
                                       uint32_t *scan_scratch, DevStatus *st) {
    const TileIdx id = tile_in(t_local, c);
    const uint32_t rb = id.i * c.y + id.j, sb = id.j * c.z + id.k, tb = id.k * c.x + id.i;
    const uint32_t r0 = c.offR[rb], r1 = c.offR[rb + 1];
    const uint32_t s0 = c.offS[sb], s1 = c.offS[sb + 1];
    const uint32_t t0 = c.offT[tb], t1 = c.offT[tb + 1];
    const uint32_t ntc = cdiv(t1 - t0, CTCAP);
    const uint32_t rc = local / ntc, tc = local % ntc;
    const uint32_t ra = r0 + rc * CRCAP, rz = min(r1, ra + CRCAP);
    const uint32_t ta = t0 + tc * CTCAP, tz = min(t1, ta + CTCAP);
    const uint32_t lane = threadIdx.x & 31;
    __syncthreads();
    for (uint32_t q = threadIdx.x; q <= CRSLOTS; q += BTH) {
        sm.rkeys[q] = (q < CRSLOTS) ? kEmptyKey : 0u;
        sm.rdeg[q] = 0u;
    }
    for (uint32_t q = threadIdx.x; q <= CTSLOTS; q += BTH) {
        if (q < CTSLOTS) sm.tkeys[q] = kEmpty64;
        sm.tcnt[q] = 0u;
    }
    if (threadIdx.x == 0) *carry = 0;
    __syncthreads();
    for (uint32_t r = ra + threadIdx.x; r < rz; r += BTH) {
        bool fresh;
        int slot = tbl_insert(sm.rkeys, CRSLOTS - 1, __ldg(c.Rp + r).y, seed, &fresh);
        if (slot >= 0) atomicAdd(&sm.rdeg[slot], 1u);
        else set_status(st, MWJ_ERR_CHECK, 34);
    }
    for (uint32_t q = ta + threadIdx.x; q < tz; q += BTH) {
        const uint2 tu = __ldg(c.Tp + q);
        const unsigned long long key = cpack(tu.x, tu.y);
        if (key == kEmpty64) {
            atomicAdd(&sm.tcnt[CTSLOTS], 1u);
            continue;
        }
        uint32_t h = cpair_hash(tu.x, tu.y, seed2) & (CTSLOTS - 1);
        bool done = false;
        for (uint32_t it = 0; it < CTSLOTS; ++it) {
            unsigned long long v = sm.tkeys[h];
            if (v == kEmpty64) {
                unsigned long long old = atomicCAS(&sm.tkeys[h], kEmpty64, key);
                if (old == kEmpty64 || old == key) {
                    atomicAdd(&sm.tcnt[h], 1u);
                    done = true;
                    break;
                }
                v = old;
            }
            if (v == key) {
                atomicAdd(&sm.tcnt[h], 1u);
                done = true;
                break;
            }
            h = (h + 1) & (CTSLOTS - 1);
        }
        if (!done) set_status(st, MWJ_ERR_CHECK, 35);
    }
    __syncthreads();
    for (uint32_t b0 = 0; b0 <= CRSLOTS; b0 += BTH) {
        uint32_t q = b0 + threadIdx.x;
        uint32_t d = (q <= CRSLOTS) ? sm.rdeg[q] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan_u32(d, scan_scratch, &tot);
        if (q <= CRSLOTS) sm.rstart[q] = *carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) *carry += tot;
        __syncthreads();
    }
    for (uint32_t r = ra + threadIdx.x; r < rz; r += BTH) {
        const uint2 tu = __ldg(c.Rp + r);
        int slot = tbl_find(sm.rkeys, CRSLOTS - 1, tu.y, seed);
        if (slot >= 0) {
            uint32_t p = atomicAdd(&sm.rstart[slot], 1u);
            if (p < CRCAP) sm.alist[p] = (int32_t)tu.x;
        }
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q <= CRSLOTS; q += BTH) sm.rstart[q] -= sm.rdeg[q];
    __syncthreads();
    unsigned long long acc = 0;
    for (uint32_t w0 = s0 + (threadIdx.x & ~31u); w0 < s1; w0 += BTH) {
        const uint32_t idx = w0 + lane;
        uint32_t cc = 0, n = 0, stt = 0;
        if (idx < s1) {
            const uint2 tu = __ldg(c.Sp + idx);
            cc = tu.y;
            int slot = tbl_find(sm.rkeys, CRSLOTS - 1, tu.x, seed);
            if (slot >= 0) {
                n = sm.rdeg[slot];
                stt = sm.rstart[slot];
            }
        }
        uint32_t incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += y;
        }
        const uint32_t W = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t excl = incl - n;
        for (uint32_t base = 0; base < W; base += 32) {
            const uint32_t wi = base + lane;
            int olo = 0, ohi = 31;
            const uint32_t qq = (wi < W) ? wi : 0u;
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                int mid = (olo + ohi) >> 1;
                uint32_t v = __shfl_sync(0xffffffffu, incl, mid);
                if (v > qq) ohi = mid; else olo = mid + 1;
            }
            const uint32_t oc = __shfl_sync(0xffffffffu, cc, olo);
            const uint32_t ost = __shfl_sync(0xffffffffu, stt, olo);
            const uint32_t oex = __shfl_sync(0xffffffffu, excl, olo);
            if (wi < W) {
                const uint32_t ai = ost + (wi - oex);
                const uint32_t a = (ai < CRCAP) ? (uint32_t)sm.alist[ai] : 0u;
                const unsigned long long key = cpack(oc, a);
                uint32_t m = 0;
                if (key == kEmpty64) {
                    m = sm.tcnt[CTSLOTS];
                } else {
                    uint32_t h = cpair_hash(oc, a, seed2) & (CTSLOTS - 1);
                    for (uint32_t it = 0; it < CTSLOTS; ++it) {
                        unsigned long long v = sm.tkeys[h];
                        if (v == key) { m = sm.tcnt[h]; break; }
                        if (v == kEmpty64) break;
                        h = (h + 1) & (CTSLOTS - 1);
                    }
                }
                acc += m;
            }
        }
    }
    return acc;
}

__global__ void __launch_bounds__(BTH) k_batch_join(BatchDev b, const uint32_t *item_off,
                                                   unsigned int *counter,
                                                   unsigned long long *counts, DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smraw[];
    JoinSmem &sm = *(JoinSmem *)smraw;
    __shared__ uint32_t item_s, nd, carry;
    __shared__ uint32_t scan_scratch[33];
    __shared__ unsigned long long red[32];
    const uint32_t ncyc_items = (b.ntiles > 0) ? item_off[b.ntiles] : 0u;
    const uint32_t total = b.nlitems + ncyc_items;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t item = item_s;
        __syncthreads();
        if (item >= total) break;
        unsigned long long acc;
        uint32_t q;
        if (item < b.nlitems) {
            const LinItem li = b.litems[item];
            q = li.q;
            acc = lin_item(b.lin[li.lq], li.i, sm.lin, b.seed_slot, b.seed_slot2, &nd, st);
        } else {
            const uint32_t ci = item - b.nlitems;
            uint32_t lo = 0, hi = b.ntiles;   // last tile t with item_off[t] <= ci
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (item_off[mid] <= ci) lo = mid; else hi = mid;
            }
            const CycQ c = b.cyc[b.tile_q[lo]];
            q = c.q;
            acc = cyc_item(c, lo - c.tile0, ci - item_off[lo], sm.cyc, b.seed_slot, b.seed_slot2,
                           &carry, scan_scratch, st);
        }
        unsigned long long tot = block_sum_u64(acc, red);
        if (threadIdx.x == 0 && tot) atomicAdd(counts + q, tot);
    }
}

}  // namespace
}  // namespace mwj

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using namespace mwj;

struct mwj_batch {
    mwj_ctx *ctx;
    int32_t n;
    size_t ws_bytes;
    // device descriptor arrays (allocated at create time, not on the hot path)
    void *dmem;
    BatchDev dev;
    uint32_t nlin_q, ncyc_tiles;
    // workspace offsets of the per-query buffers are baked into the descriptors
    // relative to a workspace base; they are rebased when the workspace pointer
    // changes
    std::vector<Seg> segs;
    std::vector<LinQ> lin;
    std::vector<CycQ> cyc;
    std::vector<LinItem> litems;
    std::vector<uint32_t> tile_q;
    size_t off_items, off_scan, off_counter;
    void *bound_ws;
    std::vector<mwj_shares> shares;
    int32_t prep_cps, join_cps;   // launch shapes fixed at create time
};

namespace {

template <typename P>
P *rebase(P *p, char *old_base, char *new_base) {
    const uintptr_t off = reinterpret_cast<uintptr_t>(p) - reinterpret_cast<uintptr_t>(old_base);
    return reinterpret_cast<P *>(reinterpret_cast<uintptr_t>(new_base) + off);
}

uint32_t pow2_ge(uint64_t v) {
    uint32_t p = 1;
    while (p < v && p < (1u << 30)) p <<= 1;
    return p;
}

// The planning rule of one query: its kind's rule for the size class
// floor(log2(max(|R|, |S|, |T|))), the library's where the context has none.
struct Rule {
    uint32_t tpb;    // linear: R tuples per bucket
    uint32_t tfac;   // linear: T table slots per tuple
    double fit;      // cyclic: fraction of a tile's capacity R_ij and T_ki may fill
};

Rule batch_rule(const mwj_ctx *ctx, const mwj_query &q) {
    const int64_t m = std::max(std::max(q.R.n, q.S.n), std::max(q.T.n, (int64_t)1));
    int c = 0;
    while (c < 31 && (2ll << c) <= m) ++c;
    const int k = q.kind == MWJ_LINEAR ? 0 : 1;
    Rule r{8192u, 2u, 0.5};
    if (ctx->batch_tpb[k][c] > 0) r.tpb = (uint32_t)ctx->batch_tpb[k][c];
    if (ctx->batch_tfac[k][c] > 0) r.tfac = (uint32_t)ctx->batch_tfac[k][c];
    if (ctx->batch_fit[k][c] > 0) r.fit = ctx->batch_fit[k][c] / 100.0;
    return r;
}

// shares of one batched query from its sizes: linear: about rule.tpb R
// tuples per bucket; cyclic: the cost-model choice (z|R| + x|S| + y|T|)
// under the chunk fit, with every relation's bucket count at most kSegMaxP
void batch_shares(const mwj_query &q, const Rule &rule, mwj_shares *sh) {
    if (q.kind == MWJ_LINEAR) {
        uint64_t want = (uint64_t)(q.R.n + rule.tpb - 1) / rule.tpb;
        uint32_t I = pow2_ge(want ? want : 1);
        if (I > kSegMaxP) I = kSegMaxP;
        sh->s[0] = (int32_t)I;
        sh->s[1] = 1;
        sh->s[2] = 1;
        return;
    }
    const double nR = (double)q.R.n, nS = (double)q.S.n, nT = (double)q.T.n;
    double best = INFINITY;
    uint32_t bx = 1, by = 1, bz = 1;
    for (uint32_t x = 1; x <= 64; x <<= 1)
        for (uint32_t y = 1; y <= 64; y <<= 1)
            for (uint32_t z = 1; z <= 64; z <<= 1) {
                if (x * y > kSegMaxP || y * z > kSegMaxP || z * x > kSegMaxP) continue;
                if (nR / (x * y) > rule.fit * CRCAP || nT / (z * x) > rule.fit * CTCAP) continue;
                double cost = z * nR + x * nS + y * nT;
                if (cost < best) {
                    best = cost;
                    bx = x;
                    by = y;
                    bz = z;
                }
            }
    if (!std::isfinite(best)) {
        bx = 64;
        by = 64;
        bz = 64;
    }
    sh->s[0] = (int32_t)bx;
    sh->s[1] = (int32_t)by;
    sh->s[2] = (int32_t)bz;
}

}  // namespace

extern "C" {

mwj_status mwj_batch_create(mwj_ctx *ctx, const mwj_query *queries, int32_t n, mwj_batch **out) {
    if (!ctx || !out || n < 0 || (n > 0 && !queries)) return MWJ_ERR_INVALID_ARG;
    *out = nullptr;
    mwj_batch *b = new mwj_batch();
    b->ctx = ctx;
    b->n = n;
    b->dmem = nullptr;
    b->bound_ws = nullptr;
    b->prep_cps = ctx->batch_prep_cps;
    b->join_cps = ctx->batch_join_cps;
    const Seeds &sd = ctx->seeds;
    // workspace layout, with base 0 (rebased at launch)
    Arena A(nullptr, 0);
    // offsets from the workspace base, kept as pointers relative to address 0
    // until the first launch binds them to a workspace; the first 256 bytes
    // are reserved so that no buffer has offset 0 (a null pointer means "not
    // in the workspace")
    A.take<char>(1);
    auto take = [&](size_t bytes) -> char * {
        size_t off = A.used;
        A.take<char>(bytes);
        return reinterpret_cast<char *>(static_cast<uintptr_t>(off));
    };
    uint32_t tiles = 0;
    for (int32_t qi = 0; qi < n; ++qi) {
        const mwj_query &q = queries[qi];
        if ((q.kind != MWJ_LINEAR && q.kind != MWJ_CYCLIC) || !rel_ok(q.R) || !rel_ok(q.S) ||
            !rel_ok(q.T)) {
            delete b;
            return fail(ctx, MWJ_ERR_INVALID_ARG, "query %d: bad kind or relation", qi);
        }
        mwj_shares sh = q.shares;
        const Rule rule = batch_rule(ctx, q);
        if (sh.s[0] <= 0) batch_shares(q, rule, &sh);
        b->shares.push_back(sh);
        if (q.kind == MWJ_LINEAR) {
            const uint32_t I = (uint32_t)sh.s[0];
            if (I < 1 || I > kSegMaxP) {
                delete b;
                return fail(ctx, MWJ_ERR_INVALID_ARG, "query %d: linear share out of [1, %u]", qi, kSegMaxP);
            }
            LinQ L{};
            L.Rp = (uint2 *)take(sizeof(uint2) * (q.R.n + 2));
            L.offR = (uint32_t *)take(4 * (I + 1));
            L.Sp = (uint2 *)take(sizeof(uint2) * (q.S.n + 2));
            L.offS = (uint32_t *)take(4 * (I + 1));
            const uint32_t tcap = pow2_ge((uint64_t)rule.tfac * (uint64_t)(q.T.n > 0 ? q.T.n : 1) + 16);
            L.tbl = (unsigned long long *)take(8ull * tcap);
            L.tmask = tcap - 1;
            L.I = I;
            Seg sr{q.R.x, q.R.y, (uint32_t)q.R.n, SEG_PART, PartSpec{1, sd.B, I, -1, 0, 1},
                   (uint2 *)L.Rp, (uint32_t *)L.offR, nullptr, 0};
            Seg ss{q.S.x, q.S.y, (uint32_t)q.S.n, SEG_PART, PartSpec{0, sd.B, I, -1, 0, 1},
                   (uint2 *)L.Sp, (uint32_t *)L.offS, nullptr, 0};
            Seg stt{q.T.x, q.T.y, (uint32_t)q.T.n, SEG_TTAB, PartSpec{0, 0, 1, -1, 0, 1}, nullptr,
                    nullptr, (unsigned long long *)L.tbl, L.tmask};
            b->segs.push_back(sr);
            b->segs.push_back(ss);
            b->segs.push_back(stt);
            const uint32_t lq = (uint32_t)b->lin.size();
            b->lin.push_back(L);
            for (uint32_t i = 0; i < I; ++i) b->litems.push_back(LinItem{(uint32_t)qi, lq, i});
        } else {
            const uint32_t x = (uint32_t)sh.s[0], y = (uint32_t)sh.s[1], z = (uint32_t)sh.s[2];
            if (x < 1 || y < 1 || z < 1 || (uint64_t)x * y > kSegMaxP || (uint64_t)y * z > kSegMaxP ||
                (uint64_t)z * x > kSegMaxP) {
                delete b;
                return fail(ctx, MWJ_ERR_INVALID_ARG, "query %d: cyclic shares out of range", qi);
            }
            CycQ C{};
            C.Rp = (uint2 *)take(sizeof(uint2) * (q.R.n + 2));
            C.offR = (uint32_t *)take(4 * (x * y + 1));
            C.Sp = (uint2 *)take(sizeof(uint2) * (q.S.n + 2));
            C.offS = (uint32_t *)take(4 * (y * z + 1));
            C.Tp = (uint2 *)take(sizeof(uint2) * (q.T.n + 2));
            C.offT = (uint32_t *)take(4 * (z * x + 1));
            C.x = x;
            C.y = y;
            C.z = z;
            C.tile0 = tiles;
            C.q = (uint32_t)qi;
            b->segs.push_back(Seg{q.R.x, q.R.y, (uint32_t)q.R.n, SEG_PART, PartSpec{0, sd.A, x, 1, sd.B, y},
                                  (uint2 *)C.Rp, (uint32_t *)C.offR, nullptr, 0});
            b->segs.push_back(Seg{q.S.x, q.S.y, (uint32_t)q.S.n, SEG_PART, PartSpec{0, sd.B, y, 1, sd.C, z},
                                  (uint2 *)C.Sp, (uint32_t *)C.offS, nullptr, 0});
            b->segs.push_back(Seg{q.T.x, q.T.y, (uint32_t)q.T.n, SEG_PART, PartSpec{0, sd.C, z, 1, sd.A, x},
                                  (uint2 *)C.Tp, (uint32_t *)C.offT, nullptr, 0});
            const uint32_t nt = x * y * z;
            for (uint32_t t = 0; t < nt; ++t) b->tile_q.push_back((uint32_t)b->cyc.size());
            tiles += nt;
            b->cyc.push_back(C);
        }
    }
    b->ncyc_tiles = tiles;
    b->off_items = A.used;
    A.take<uint32_t>(tiles + 1);
    b->off_scan = A.used;
    A.take<char>(scan_scratch_bytes(tiles + 1));
    b->off_counter = A.used;
    A.take<unsigned int>(4);
    b->ws_bytes = A.used;
    // largest segments first; linear items by their expected S work, largest first
    std::stable_sort(b->segs.begin(), b->segs.end(), [](const Seg &a, const Seg &c) { return a.n > c.n; });
    std::stable_sort(b->litems.begin(), b->litems.end(), [&](const LinItem &a, const LinItem &c) {
        const mwj_query &qa = queries[a.q], &qc = queries[c.q];
        return (double)qa.S.n / b->lin[a.lq].I > (double)qc.S.n / b->lin[c.lq].I;
    });
    *out = b;
    return MWJ_OK;
}

mwj_status mwj_batch_workspace_size(mwj_batch *b, size_t *bytes) {
    if (!b || !bytes) return MWJ_ERR_INVALID_ARG;
    *bytes = b->ws_bytes;
    return MWJ_OK;
}

mwj_status mwj_batch_shares(mwj_batch *b, int32_t q, mwj_shares *sh) {
    if (!b || !sh || q < 0 || q >= b->n) return MWJ_ERR_INVALID_ARG;
    *sh = b->shares[q];
    return MWJ_OK;
}

mwj_status mwj_batch_launch(mwj_batch *b, int64_t *counts, void *workspace, size_t ws_bytes,
                            void *stream) {
    if (!b || (b->n > 0 && !counts)) return MWJ_ERR_INVALID_ARG;
    mwj_ctx *ctx = b->ctx;
    ApiScope api_scope(&ctx->prof);
    if (!workspace || ws_bytes < b->ws_bytes)
        return fail(ctx, MWJ_ERR_WORKSPACE, "batch workspace of %zu bytes, %zu needed", ws_bytes,
                    b->ws_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (b->bound_ws != workspace) {
        // bind the descriptors to this workspace and upload them (outside any
        // capture: the first launch on a workspace must not be captured)
        char *nb = (char *)workspace, *ob = (char *)b->bound_ws;
        if (!ob) ob = (char *)nullptr;
        for (Seg &s : b->segs) {
            if (s.out) s.out = rebase(s.out, ob, nb);
            if (s.off) s.off = rebase(s.off, ob, nb);
            if (s.tbl) s.tbl = rebase(s.tbl, ob, nb);
        }
        for (LinQ &L : b->lin) {
            L.Rp = rebase(L.Rp, ob, nb); L.Sp = rebase(L.Sp, ob, nb);
            L.offR = rebase(L.offR, ob, nb); L.offS = rebase(L.offS, ob, nb);
            L.tbl = rebase(L.tbl, ob, nb);
        }
        for (CycQ &C : b->cyc) {
            C.Rp = rebase(C.Rp, ob, nb); C.Sp = rebase(C.Sp, ob, nb); C.Tp = rebase(C.Tp, ob, nb);
            C.offR = rebase(C.offR, ob, nb); C.offS = rebase(C.offS, ob, nb);
            C.offT = rebase(C.offT, ob, nb);
        }
        b->bound_ws = workspace;
        if (b->dmem) cudaFree(b->dmem);
        size_t bytes = align256(sizeof(Seg) * (b->segs.size() + 1)) +
                       align256(sizeof(LinQ) * (b->lin.size() + 1)) +
                       align256(sizeof(LinItem) * (b->litems.size() + 1)) +
                       align256(sizeof(CycQ) * (b->cyc.size() + 1)) +
                       align256(sizeof(uint32_t) * (b->tile_q.size() + 1));
        if ((e = cudaMalloc(&b->dmem, bytes)) != cudaSuccess) return cuda_fail(ctx, e, "batch descriptors");
        char *p = (char *)b->dmem;
        auto put = [&](const void *src, size_t sz) -> const void * {
            if (sz) cudaMemcpy(p, src, sz, cudaMemcpyHostToDevice);
            const void *r = p;
            p += align256(sz + 1);
            return r;
        };
        b->dev.segs = (const Seg *)put(b->segs.data(), sizeof(Seg) * b->segs.size());
        b->dev.nseg = (uint32_t)b->segs.size();
        b->dev.lin = (const LinQ *)put(b->lin.data(), sizeof(LinQ) * b->lin.size());
        b->dev.litems = (const LinItem *)put(b->litems.data(), sizeof(LinItem) * b->litems.size());
        b->dev.nlitems = (uint32_t)b->litems.size();
        b->dev.cyc = (const CycQ *)put(b->cyc.data(), sizeof(CycQ) * b->cyc.size());
        b->dev.ncyc = (uint32_t)b->cyc.size();
        b->dev.tile_q = (const uint32_t *)put(b->tile_q.data(), sizeof(uint32_t) * b->tile_q.size());
        b->dev.ntiles = b->ncyc_tiles;
        b->dev.seed_slot = ctx->seeds.slot;
        b->dev.seed_slot2 = ctx->seeds.slot2;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "batch upload");
    }
    char *ws = (char *)workspace;
    uint32_t *items = (uint32_t *)(ws + b->off_items);
    void *scan_tmp = ws + b->off_scan;
    unsigned int *counter = (unsigned int *)(ws + b->off_counter);
    const int sms = ctx->dev.num_sms;
    if ((e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * (size_t)b->n, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset counts");
    if ((e = cudaMemsetAsync(counter, 0, 4 * sizeof(unsigned int), st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset counter");
    {
        ProfScope ps_("batch_prep", st);
        k_batch_prep<<<sms * (b->prep_cps > 0 ? b->prep_cps : 3), BTH, 0, st>>>(b->dev, counter, ctx->status);
    }
    if (b->ncyc_tiles) {
        {
            ProfScope ps_("batch_plan", st);
            k_batch_plan<<<(b->ncyc_tiles + 255) / 256, 256, 0, st>>>(b->dev, items);
        }
        if ((e = cudaMemsetAsync(items + b->ncyc_tiles, 0, 4, st)) != cudaSuccess)
            return cuda_fail(ctx, e, "memset items");
        if ((e = scan_excl_u32(items, b->ncyc_tiles + 1, scan_tmp, st)) != cudaSuccess)
            return cuda_fail(ctx, e, "batch scan");
    }
    const size_t smem = sizeof(JoinSmem);
    if ((e = cudaFuncSetAttribute(k_batch_join, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "batch smem");
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_join, BTH, smem);
    if (occ < 1) occ = 1;
    if (b->join_cps > 0 && b->join_cps < occ) occ = b->join_cps;
    {
        ProfScope ps_("batch_join", st);
        k_batch_join<<<sms * occ, BTH, smem, st>>>(b->dev, items, counter + 1,
                                                    (unsigned long long *)counts, ctx->status);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "batch launch");
    return MWJ_OK;
}

mwj_status mwj_batch_set_rules(mwj_ctx *ctx, const mwj_batch_rule *rules, int32_t n) {
    if (!ctx || n < 0 || (n > 0 && !rules)) return MWJ_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n; ++i) {
        const mwj_batch_rule &r = rules[i];
        if ((r.kind != MWJ_LINEAR && r.kind != MWJ_CYCLIC) || r.size_log2 < 0 || r.size_log2 > 31 ||
            r.tuples_per_bucket > (1 << 30) || r.table_factor > 8 || (r.table_factor > 0 && r.table_factor < 2) ||
            r.fit_pct > 100 || (r.fit_pct > 0 && r.fit_pct < 10))
            return fail(ctx, MWJ_ERR_INVALID_ARG, "batch rule %d out of range", i);
    }
    for (int k = 0; k < 2; ++k)
        for (int c = 0; c < 32; ++c) ctx->batch_tpb[k][c] = ctx->batch_tfac[k][c] = ctx->batch_fit[k][c] = 0;
    for (int32_t i = 0; i < n; ++i) {
        const mwj_batch_rule &r = rules[i];
        const int k = r.kind == MWJ_LINEAR ? 0 : 1;
        ctx->batch_tpb[k][r.size_log2] = r.tuples_per_bucket;
        ctx->batch_tfac[k][r.size_log2] = r.table_factor;
        ctx->batch_fit[k][r.size_log2] = r.fit_pct;
    }
    return MWJ_OK;
}

mwj_status mwj_batch_set_launch(mwj_ctx *ctx, int32_t prep_ctas_per_sm, int32_t join_ctas_per_sm) {
    if (!ctx || prep_ctas_per_sm < 0 || prep_ctas_per_sm > 8 || join_ctas_per_sm < 0 || join_ctas_per_sm > 8)
        return MWJ_ERR_INVALID_ARG;
    ctx->batch_prep_cps = prep_ctas_per_sm;
    ctx->batch_join_cps = join_ctas_per_sm;
    return MWJ_OK;
}

mwj_status mwj_batch_destroy(mwj_batch *b) {
    if (!b) return MWJ_ERR_INVALID_ARG;
    if (b->dmem) cudaFree(b->dmem);
    delete b;
    return MWJ_OK;
}

}  // extern "C"
