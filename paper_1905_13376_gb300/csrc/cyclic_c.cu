// cyclic_c.cu -- the cyclic 3-way join R(A,B) S(B,C) T(C,A) with R whole and
// C split into buckets: shares (1, 1, z) (Section 5).
//
// Section 5 keeps R's (H(a), G(b)) buckets on chip and streams S and T past
// them; with cube shares (x, y, z) a tile (i, j, k) holds R_ij and T_ki in a
// CTA's shared memory and streams S_jk (cyclic.cu).  On a large graph the
// tiles that fit shared memory are so small -- millions of them -- that
// rebuilding their tables costs far more than the wedge checks.  This plan
// follows the two levels of on-chip memory of the GPU instead: R stays whole,
// grouped by B (b -> [a], in global memory and read through the L2 by every
// SM), and only C is split: T by F(c) into z buckets whose (c, a) multiset
// fits one CTA's shared memory, S by F(c) into the same buckets.  A CTA takes
// bucket k, builds T_k's set on chip and streams S_k past it: per S tuple
// (b, c) it visits every a of R[b] and counts (c, a) in the set.  These are
// the cube tiling's wedge checks, each wedge of R |x| S once, without the
// per-tile rebuilds.  A bucket whose T_k exceeds a CTA's shared-memory set
// is taken in chunks of it, S_k streamed past each (every chunk checks the
// bucket's wedges again, against its part of T_k), up to kChunkMax chunks; a
// larger one (a C value with many T tuples: skewed or tiny C domains) keeps
// its set in an L2-resident region of the workspace instead, built before
// the probe, so that its wedges are checked once.  Results do not depend on
// z.
#include "api_internal.h"
#include "cyclic.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr int CC_T = 768;                // threads per probe CTA (two CTAs per SM)
constexpr uint32_t CC_TCAP = 4096;       // T tuples of an on-chip set: it is at most half full
constexpr uint32_t kChunkMax = 4;        // on-chip chunks of a bucket before its set moves to the L2
constexpr uint32_t CC_TSLOTS = 8192;     // slots of an on-chip (c, a) multiset (64 KB)
constexpr int RG_T = 512;                // threads of the grouping kernels
constexpr uint32_t CC_QCAP = 2048;       // long R lists queued per work item
constexpr uint32_t CC_CH = 256;          // wedges of a queued list per warp step
constexpr uint32_t kQueueMin = 128;      // lists this long go to the item's queue
constexpr uint32_t CC_SCHUNK_MIN = 32;   // S tuples of a bucket's work item, at least (a warp's batch)

__device__ __forceinline__ unsigned long long cpack(uint32_t c, uint32_t a) {
    return ((unsigned long long)c << 32) | a;
}

// An on-chip (c, a) set: CC_TSLOTS / 2 buckets of two 8-byte slots (16
// bytes, one shared-memory load), one slot per distinct pair.  An insert
// takes the first slot of its home bucket or of the buckets after it that is
// free or holds its pair, so the occupied slots of a bucket are a prefix and
// a lookup can stop at the first bucket with a free slot: with the set at
// most half full that is nearly always the home bucket.  T is a bag: a chunk
// that repeats a pair (rare) is rebuilt in the CTA's own region of the
// workspace with a multiplicity per slot and looked up there like a big
// bucket's set, so that the lookups of every other chunk stay as they are.
constexpr uint32_t CC_NB = CC_TSLOTS / 2;
constexpr int CC_MAX_CTAS_PER_SM = 2;   // probe CTAs per SM (shared memory); one region each
// two probe CTAs per SM: each keeps below half of the SM's 228 KB of shared
// memory less the 1 KB the hardware reserves per CTA and the static arrays
static_assert(CC_TSLOTS * 8 + CC_QCAP * 16 + (CC_QCAP + 1) * 4 + 1024 <= 228 * 1024 / 2 - 1024,
              "the probe's shared memory must leave room for two CTAs per SM");

__device__ __forceinline__ uint32_t cbucket(uint32_t c, uint32_t a, uint32_t seed) {
    uint32_t h = (c ^ seed) * 0x9E3779B1u ^ a * 0x85EBCA6Bu;
    h ^= h >> 16;
    h *= 0x7feb352dU;
    h ^= h >> 15;
    return h & (CC_NB - 1);
}

// 1: the pair took a free slot; 2: it was there already; 0: the set is full.
__device__ __forceinline__ int cset_insert(unsigned long long *tk, unsigned long long key, uint32_t bk) {
    for (uint32_t it = 0; it < CC_NB; ++it) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            unsigned long long *p = tk + 2 * bk + q;
            unsigned long long v = *p;
            if (v == kEmpty64) {
                v = atomicCAS(p, kEmpty64, key);
                if (v == kEmpty64) return 1;
            }
            if (v == key) return 2;
        }
        bk = (bk + 1) & (CC_NB - 1);
    }
    return 0;
}

// 1 when key is in the set, else 0 (key != kEmpty64)
__device__ __forceinline__ uint32_t cset_count(const unsigned long long *tk, unsigned long long key, uint32_t bk) {
    uint32_t m = 0;
    for (uint32_t it = 0; it < CC_NB; ++it) {
        const ulonglong2 v = *(const ulonglong2 *)(tk + 2 * bk);
        m += (v.x == key) + (v.y == key);
        if (v.y == kEmpty64) break;   // (v.x empty implies v.y empty)
        bk = (bk + 1) & (CC_NB - 1);
    }
    return m;
}

// Entries of R's grouping: the direct-address layout (key b at b - min) or
// the hashed key table's slot (slot mask + 1 holds key -1).
__device__ __forceinline__ uint32_t rg_entries(const uint32_t *meta) {
    return meta[kMetaDense] ? meta[kMetaSpan] : meta[kMetaMask] + 2u;
}

__device__ __forceinline__ int rg_find(const RGroup &r, const uint32_t *meta, uint32_t b) {
    if (meta[kMetaDense]) {
        const uint32_t k = b - meta[kMetaMin];
        return k < meta[kMetaSpan] ? (int)k : -1;
    }
    return tbl_find(r.keys, meta[kMetaMask], b, r.seed);
}

__global__ void k_rg_clear(RGroup r) {
    const uint32_t *meta = r.meta;
    const uint32_t n = rg_entries(meta);
    const bool hashed = meta[kMetaDense] == 0u;
    const uint32_t mask = meta[kMetaMask];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        r.deg[i] = 0u;
        if (hashed) r.keys[i] = (i <= mask) ? kEmptyKey : 0u;
    }
}

// deg[index(b)] += 1 for every (a, b) of R (the hashed layout inserts b);
// with a_domain > 0 every a must lie in [0, a_domain).
__global__ void __launch_bounds__(RG_T) k_rg_count(const int32_t *__restrict__ Ra, const int32_t *__restrict__ Rb,
                                                   uint32_t n, RGroup r, int32_t a_domain, DevStatus *st) {
    const uint32_t *meta = r.meta;
    const bool dense = meta[kMetaDense] != 0u;
    const uint32_t kmin = meta[kMetaMin], span = meta[kMetaSpan], mask = meta[kMetaMask];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t a = __ldg(Ra + i);
        const uint32_t b = (uint32_t)__ldg(Rb + i);
        if (a_domain > 0 && (uint32_t)a >= (uint32_t)a_domain) set_status(st, MWJ_ERR_DOMAIN, a);
        int idx;
        if (dense) {
            idx = (b - kmin < span) ? (int)(b - kmin) : -1;
        } else {
            bool fresh;
            idx = tbl_insert(r.keys, mask, b, r.seed, &fresh);
        }
        if (idx >= 0)
            atomicAdd(r.deg + idx, 1u);
        else
            set_status(st, MWJ_ERR_CHECK, 21);   // outside the sized range / table full
    }
}

// end[i] = start of entry i's list (block-aggregated bump allocation: the
// lists are contiguous per key, in no particular key order); the scatter
// advances end[i] to the list's end.
__global__ void __launch_bounds__(RG_T) k_rg_offsets(RGroup r, unsigned int *__restrict__ bump) {
    __shared__ uint32_t scratch[33];
    __shared__ uint32_t base;
    const uint32_t n = rg_entries(r.meta);
    for (uint32_t b0 = blockIdx.x * RG_T; b0 < n; b0 += gridDim.x * RG_T) {
        const uint32_t i = b0 + threadIdx.x;
        const uint32_t d = i < n ? r.deg[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan_u32(d, scratch, &tot);
        if (threadIdx.x == 0) base = tot ? atomicAdd(bump, tot) : 0u;
        __syncthreads();
        if (i < n) r.end[i] = base + ex;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(RG_T) k_rg_scatter(const int32_t *__restrict__ Ra,
                                                     const int32_t *__restrict__ Rb, uint32_t n, RGroup r,
                                                     uint32_t nR, DevStatus *st) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int idx = rg_find(r, r.meta, (uint32_t)__ldg(Rb + i));
        if (idx < 0) {
            set_status(st, MWJ_ERR_CHECK, 22);
            continue;
        }
        const uint32_t p = atomicAdd(r.end + idx, 1u);
        if (p < nR)
            r.alist[p] = __ldg(Ra + i);
        else
            set_status(st, MWJ_ERR_CHECK, 23);
    }
}

__host__ __device__ __forceinline__ bool cc_big(uint32_t nt) { return nt > kChunkMax * CC_TCAP; }

// S chunks of a bucket: S_k in pieces of at most schunk tuples
__host__ __device__ __forceinline__ uint32_t cc_schunks(uint32_t ns, uint32_t schunk) {
    return (ns + schunk - 1) / schunk;
}

// Work items of a bucket whose S_k and T_k are both non-empty: each of its
// T chunks (on-chip sets; one set when the bucket is big, cc_big) with each
// of its S chunks, item (t, s) at t * S chunks + s; a big bucket also gets a
// region of 2^k >= 2 |T_k| slots for its set in the workspace (big_slots[k],
// 0 for the others).
__global__ void k_cc_plan(const uint32_t *__restrict__ offS, const uint32_t *__restrict__ offT, uint32_t z,
                          uint32_t schunk, uint32_t *__restrict__ items,
                          unsigned long long *__restrict__ big_slots) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < z; k += gridDim.x * blockDim.x) {
        const uint32_t ns = offS[k + 1] - offS[k], nt = offT[k + 1] - offT[k];
        items[k] = (ns && nt) ? (cc_big(nt) ? 1u : (nt + CC_TCAP - 1) / CC_TCAP) * cc_schunks(ns, schunk) : 0u;
        unsigned long long slots = 0;
        if (ns && cc_big(nt)) {
            slots = 16;
            while (slots < 2ull * nt) slots <<= 1;
        }
        big_slots[k] = slots;
    }
}

// Empty every big bucket's region and zero its counts (the total is the
// scan's last entry).
__global__ void k_cc_bigclear(unsigned long long *__restrict__ gs, uint32_t *__restrict__ gc,
                              const unsigned long long *__restrict__ big_off, uint32_t z) {
    const unsigned long long total = big_off[z];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        gs[i] = kEmpty64;
        gc[i] = 0u;
    }
}

__device__ __forceinline__ uint32_t gslot(uint32_t c, uint32_t a, uint32_t seed) {
    uint32_t h = (c ^ seed) * 0x85EBCA6Bu ^ a * 0x9E3779B1u;
    h ^= h >> 15;
    h *= 0x846ca68bU;
    h ^= h >> 16;
    return h;
}

// Big buckets' sets: a CTA per bucket (buckets blockIdx.x, + gridDim.x, ...)
// inserts T_k's (c, a) pairs into the bucket's region, one slot per distinct
// pair (linear probing from gslot) and its multiplicity in gc at the same
// index; (-1, -1) pairs are counted in big_neg[k].
__global__ void k_cc_bigbuild(const uint2 *__restrict__ Tp, const uint32_t *__restrict__ offT, uint32_t z,
                              const unsigned long long *__restrict__ big_off, unsigned long long *__restrict__ gs,
                              uint32_t *__restrict__ gc, uint32_t *__restrict__ big_neg, uint32_t seed,
                              DevStatus *st) {
    __shared__ uint32_t negs;
    for (uint32_t k = blockIdx.x; k < z; k += gridDim.x) {
        const unsigned long long base = big_off[k], slots = big_off[k + 1] - base;
        if (slots == 0) continue;
        if (threadIdx.x == 0) negs = 0u;
        __syncthreads();
        const uint32_t mask = (uint32_t)(slots - 1);
        unsigned long long *reg = gs + base;
        uint32_t *cnt = gc + base;
        for (uint32_t q = offT[k] + threadIdx.x; q < offT[k + 1]; q += blockDim.x) {
            const uint2 tu = __ldg(Tp + q);
            const unsigned long long key = cpack(tu.x, tu.y);
            if (key == kEmpty64) {
                atomicAdd(&negs, 1u);
                continue;
            }
            uint32_t s = gslot(tu.x, tu.y, seed) & mask;
            bool done = false;
            for (uint32_t it = 0; it <= mask; ++it) {
                unsigned long long v = reg[s];
                if (v == kEmpty64) v = atomicCAS(reg + s, kEmpty64, key);   // kEmpty64: claimed here
                if (v == kEmpty64 || v == key) {
                    atomicAdd(cnt + s, 1u);
                    done = true;
                    break;
                }
                s = (s + 1) & mask;
            }
            if (!done) set_status(st, MWJ_ERR_CHECK, 26);
        }
        __syncthreads();
        if (threadIdx.x == 0) big_neg[k] = negs;
        __syncthreads();
    }
}

// Persistent kernel over the work items (bucket, chunk).  PASS 0 counts
// (COUNT, GROUP BY A, and the first pass of row output, which adds each
// item's count to its bucket's total); PASS 1 writes rows at positions taken
// from the bucket's cursor (its scanned total, advanced atomically).
template <int PASS>
__global__ void __launch_bounds__(CC_T, CC_MAX_CTAS_PER_SM) k_cc_probe(CycCArgs g, const uint32_t *__restrict__ item_off,
                                                      unsigned int *__restrict__ counter,
                                                      unsigned long long *__restrict__ bucket_rows,
                                                      int32_t *__restrict__ rows, long long capacity,
                                                      unsigned long long *__restrict__ rep_set,
                                                      uint32_t *__restrict__ rep_cnt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *tk = (unsigned long long *)smraw;                      // CC_TSLOTS
    uint4 *queue = (uint4 *)(tk + CC_TSLOTS);                                   // CC_QCAP x (b, c, start, n)
    uint32_t *cpre = (uint32_t *)(queue + CC_QCAP);                             // CC_QCAP + 1 chunk offsets
    __shared__ uint32_t item_s, tneg, batch_ctr, chunk_ctr, qn, carry, tdup;
    // this CTA's region for a chunk that repeats pairs
    unsigned long long *const my_set = rep_set + (size_t)blockIdx.x * CC_TSLOTS;
    uint32_t *const my_cnt = rep_cnt + (size_t)blockIdx.x * CC_TSLOTS;
    __shared__ uint32_t scan_scratch[33];
    __shared__ unsigned long long red[32];
    const uint32_t z = g.z;
    const uint32_t total_items = item_off[z];
    if (PASS == 1 && bucket_rows[z] > (unsigned long long)capacity) return;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t *meta = g.r.meta;
    unsigned long long acc_all = 0;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t item = item_s;
        if (item >= total_items) break;
        // bucket of this item: last k with item_off[k] <= item
        uint32_t lo = 0, hi = z;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (item_off[mid] <= item) lo = mid; else hi = mid;
        }
        const uint32_t k = lo;
        // (T chunk, S chunk) of this item
        const uint32_t sch = cc_schunks(g.offS[k + 1] - g.offS[k], g.schunk);
        const uint32_t li = item - item_off[k];
        const uint32_t tci = li / sch, sci = li - tci * sch;
        const uint32_t s0 = g.offS[k] + sci * g.schunk, s1 = min(g.offS[k + 1], s0 + g.schunk);
        // T_k's set: the item's chunk on chip, or for a big bucket its region
        // of the workspace, built before this kernel
        bool big = cc_big(g.offT[k + 1] - g.offT[k]);
        const uint32_t ta = g.offT[k] + tci * CC_TCAP;
        const uint32_t tz = big ? g.offT[k + 1] : min(g.offT[k + 1], ta + CC_TCAP);
        const unsigned long long gbase = g.big_off[k];
        uint32_t gmask = (uint32_t)(g.big_off[k + 1] - gbase) - 1u;
        const unsigned long long *gset = g.bigset + gbase;
        const uint32_t *gcnt = g.bigcnt + gbase;

        // ---- T_k as a (c, a) multiset: a slot per distinct pair ----
        if (!big)
            for (uint32_t q = threadIdx.x; q < CC_TSLOTS; q += CC_T) tk[q] = kEmpty64;
        if (threadIdx.x == 0) {
            tdup = 0u;
            tneg = big ? g.big_neg[k] : 0u;
            batch_ctr = 0u;
            chunk_ctr = 0u;
            qn = 0u;
            carry = 0u;
        }
        __syncthreads();
        for (uint32_t q = ta + threadIdx.x; !big && q < tz; q += CC_T) {
            const uint2 tu = __ldg(g.Tp + q);   // (c, a)
            const unsigned long long key = cpack(tu.x, tu.y);
            if (key == kEmpty64) {               // (-1, -1) is the empty marker: counted apart
                atomicAdd(&tneg, 1u);
                continue;
            }
            const int r = cset_insert(tk, key, cbucket(tu.x, tu.y, g.seed));
            if (r == 2 && !tdup) tdup = 1u;
            if (r == 0) set_status(g.st, MWJ_ERR_CHECK, 24);
        }
        __syncthreads();
        if (tdup) {
            // the chunk repeats pairs: its set with multiplicities in this
            // CTA's region, looked up through the L2 like a big bucket's
            for (uint32_t q = threadIdx.x; q < CC_TSLOTS; q += CC_T) {
                my_set[q] = kEmpty64;
                my_cnt[q] = 0u;
            }
            __syncthreads();
            for (uint32_t q = ta + threadIdx.x; q < tz; q += CC_T) {
                const uint2 tu = __ldg(g.Tp + q);
                const unsigned long long key = cpack(tu.x, tu.y);
                if (key == kEmpty64) continue;   // counted in tneg already
                uint32_t s = gslot(tu.x, tu.y, g.seed) & (CC_TSLOTS - 1);
                for (uint32_t it = 0; it < CC_TSLOTS; ++it) {
                    const unsigned long long v = atomicCAS(my_set + s, kEmpty64, key);
                    if (v == kEmpty64 || v == key) {
                        atomicAdd(my_cnt + s, 1u);
                        break;
                    }
                    s = (s + 1) & (CC_TSLOTS - 1);
                }
            }
            __syncthreads();
            big = true;
            gset = my_set;
            gcnt = my_cnt;
            gmask = CC_TSLOTS - 1;
        }
        const uint32_t negs = tneg;

        // ---- stream S_k past the set ----
        // One closed or open wedge per lane and call: m copies of (c, a) in
        // T_k close wedge (a, b, c).  PASS 0 adds them up (and into cnt[a]);
        // PASS 1 writes the rows, reserving the warp's positions at once.
        // Every lane of the warp calls this.
        unsigned long long acc = 0;
        auto emit = [&](uint32_t a, uint32_t b, uint32_t c, uint32_t m) {
            if (PASS == 0) {
                acc += m;
                if (g.cnt && m && a < (uint32_t)g.a_domain) atomicAdd(g.cnt + a, (unsigned long long)m);
                return;
            }
            if (!__any_sync(0xffffffffu, m != 0u)) return;
            uint32_t pincl = m;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, pincl, o);
                if ((int)lane >= o) pincl += y;
            }
            const uint32_t btot = __shfl_sync(0xffffffffu, pincl, 31);
            unsigned long long bb = 0;
            if (lane == 0) bb = atomicAdd(bucket_rows + k, (unsigned long long)btot);
            bb = __shfl_sync(0xffffffffu, bb, 0);
            unsigned long long p = bb + pincl - m;
            for (uint32_t e = 0; e < m; ++e, ++p) {
                if (p < (unsigned long long)capacity) {
                    int32_t *row = rows + 3 * p;
                    row[0] = (int32_t)a;
                    row[1] = (int32_t)b;
                    row[2] = (int32_t)c;
                } else {
                    set_status(g.st, MWJ_ERR_CHECK, 25);
                }
            }
        };
        auto count = [&](uint32_t c, uint32_t a) -> uint32_t {
            const unsigned long long key = cpack(c, a);
            if (key == kEmpty64) return negs;
            if (!big) return cset_count(tk, key, cbucket(c, a, g.seed));
            // a big bucket's set, or this CTA's for a chunk that repeats
            // pairs (written in this kernel: read through the L2)
            uint32_t s = gslot(c, a, g.seed) & gmask;
            for (uint32_t it = 0; it <= gmask; ++it) {
                const unsigned long long v = __ldcg(gset + s);
                if (v == key) return __ldcg(gcnt + s);
                if (v == kEmpty64) break;
                s = (s + 1) & gmask;
            }
            return 0u;
        };
        // walk one list of the warp's: entries [lo, hi) of (b, c)'s R list,
        // 32 a step, two steps in flight
        auto walk = [&](uint32_t jb, uint32_t jc, uint32_t jst, uint32_t lo, uint32_t hi) {
            for (uint32_t i0 = lo; i0 < hi; i0 += 64) {
                const uint32_t i = i0 + lane, i2 = i + 32;
                const uint32_t a = i < hi ? (uint32_t)__ldg(g.r.alist + jst + i) : 0u;
                const uint32_t a2 = i2 < hi ? (uint32_t)__ldg(g.r.alist + jst + i2) : 0u;
                const uint32_t m = i < hi ? count(jc, a) : 0u;
                const uint32_t m2 = i2 < hi ? count(jc, a2) : 0u;
                emit(a, jb, jc, m);
                emit(a2, jb, jc, m2);
            }
        };
        // phase 1: warps take batches of 32 S tuples as they come free;
        // lists of kQueueMin or more entries go to the item's queue (walked at
        // once when it is full), lists of 32 or more are walked by the warp,
        // shorter ones are spread over the warp's lanes, wedge wi going to
        // the first lane whose inclusive count exceeds it
        for (;;) {
            uint32_t bi = 0;
            if (lane == 0) bi = atomicAdd(&batch_ctr, 1u);
            bi = __shfl_sync(0xffffffffu, bi, 0);
            const uint32_t w0 = s0 + bi * 32u;
            if (w0 >= s1) break;
            const uint32_t idx = w0 + lane;
            uint32_t b = 0, c = 0, n = 0, st = 0;
            if (idx < s1) {
                const uint2 tu = __ldg(g.Sp + idx);
                b = tu.x;
                c = tu.y;
                const int e = rg_find(g.r, meta, b);
                if (e >= 0) {
                    n = __ldg(g.r.deg + e);
                    st = __ldg(g.r.end + e) - n;
                }
            }
            bool spill = false;
            if (n >= kQueueMin) {
                const uint32_t qs = atomicAdd(&qn, 1u);
                if (qs < CC_QCAP)
                    queue[qs] = make_uint4(b, c, st, n);
                else
                    spill = true;
            }
            unsigned sm_ = __ballot_sync(0xffffffffu, spill);
            while (sm_) {
                const int j = __ffs(sm_) - 1;
                sm_ &= sm_ - 1u;
                walk(__shfl_sync(0xffffffffu, b, j), __shfl_sync(0xffffffffu, c, j),
                     __shfl_sync(0xffffffffu, st, j), 0u, __shfl_sync(0xffffffffu, n, j));
            }
            // lists of 32 .. kQueueMin - 1 entries: the warp walks each one
            unsigned mid_ = __ballot_sync(0xffffffffu, n >= 32u && n < kQueueMin);
            while (mid_) {
                const int j = __ffs(mid_) - 1;
                mid_ &= mid_ - 1u;
                walk(__shfl_sync(0xffffffffu, b, j), __shfl_sync(0xffffffffu, c, j),
                     __shfl_sync(0xffffffffu, st, j), 0u, __shfl_sync(0xffffffffu, n, j));
            }
            const uint32_t ns = n < 32u ? n : 0u;
            uint32_t incl = ns;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += y;
            }
            const uint32_t W = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - ns;
            for (uint32_t base = 0; base < W; base += 32) {
                const uint32_t wi = base + lane;
                int olo = 0, ohi = 31;
                const uint32_t qv = (wi < W) ? wi : 0u;
#pragma unroll
                for (int step = 0; step < 5; ++step) {
                    const int mid = (olo + ohi) >> 1;
                    const uint32_t v = __shfl_sync(0xffffffffu, incl, mid);
                    if (v > qv) ohi = mid; else olo = mid + 1;
                }
                const uint32_t ob = __shfl_sync(0xffffffffu, b, olo);
                const uint32_t oc = __shfl_sync(0xffffffffu, c, olo);
                const uint32_t ost = __shfl_sync(0xffffffffu, st, olo);
                const uint32_t oex = __shfl_sync(0xffffffffu, excl, olo);
                uint32_t a = 0, m = 0;
                if (wi < W) {
                    a = (uint32_t)__ldg(g.r.alist + ost + (wi - oex));
                    m = count(oc, a);
                }
                emit(a, ob, oc, m);
            }
        }
        __syncthreads();
        // phase 2: the queued lists in chunks of CC_CH entries, taken by the
        // warps as they come free (a hub's long list is shared by all of them)
        const uint32_t nq = min(qn, CC_QCAP);
        for (uint32_t q0 = 0; q0 <= nq; q0 += CC_T) {
            const uint32_t q = q0 + threadIdx.x;
            const uint32_t d = q < nq ? (queue[q].w + CC_CH - 1) / CC_CH : 0u;
            uint32_t tot;
            const uint32_t ex = block_excl_scan_u32(d, scan_scratch, &tot);
            if (q <= nq) cpre[q] = carry + ex;
            __syncthreads();
            if (threadIdx.x == 0) carry += tot;
            __syncthreads();
        }
        const uint32_t nchunks = cpre[nq];
        for (;;) {
            uint32_t ci = 0;
            if (lane == 0) ci = atomicAdd(&chunk_ctr, 1u);
            ci = __shfl_sync(0xffffffffu, ci, 0);
            if (ci >= nchunks) break;
            uint32_t lo = 0, hi = nq;   // last list with cpre <= ci
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (cpre[mid] <= ci) lo = mid; else hi = mid;
            }
            const uint4 L = queue[lo];
            const uint32_t first = (ci - cpre[lo]) * CC_CH;
            walk(L.x, L.y, L.z, first, min(first + CC_CH, L.w));
        }
        if (PASS == 0) {
            const unsigned long long tot = block_sum_u64(acc, red);   // ends with a barrier
            if (threadIdx.x == 0 && bucket_rows && tot) atomicAdd(bucket_rows + k, tot);
            acc_all += acc;
        } else {
            __syncthreads();
        }
    }
    if (PASS == 0) {
        const unsigned long long tot = block_sum_u64(acc_all, red);
        if (threadIdx.x == 0 && tot) atomicAdd(g.total, tot);
    }
}

__global__ void k_cc_rows_check(const unsigned long long *base, uint32_t z, long long capacity, long long *n_rows,
                                DevStatus *st) {
    const unsigned long long tot = base[z];
    *n_rows = (long long)tot;
    if (tot > (unsigned long long)capacity) set_status(st, MWJ_ERR_CAPACITY, (long long)tot);
}

}  // namespace

uint32_t cyc_c_schunk(int64_t nS, int num_sms) {
    // about four items per probe CTA over the whole of S: a join with few
    // buckets (a small T, cheap to rebuild per item) is spread over the GPU,
    // one with many buckets (S_k below the piece) is not split at all
    const uint64_t want = ((uint64_t)(nS > 0 ? nS : 0) + 4ull * num_sms * CC_MAX_CTAS_PER_SM - 1) /
                          (4ull * num_sms * CC_MAX_CTAS_PER_SM);
    return (uint32_t)(want > CC_SCHUNK_MIN ? (want < 0x7FFFFFFFull ? want : 0x7FFFFFFFull) : CC_SCHUNK_MIN);
}

size_t cyc_c_rep_slots(int num_sms) { return (size_t)num_sms * CC_MAX_CTAS_PER_SM * CC_TSLOTS; }

uint32_t cyc_c_tcap() { return CC_TCAP; }

cudaError_t rgroup_build(const int32_t *Ra, const int32_t *Rb, int64_t nR, const RGroup &r, unsigned int *hll,
                         uint64_t reserve, unsigned int *bump, int32_t a_domain, DevStatus *status, int num_sms,
                         cudaStream_t st) {
    cudaError_t e = single_table_size(Rb, nR, r.seed, hll, (uint32_t *)r.meta, reserve, num_sms, st, "rg_hll",
                                      "rg_size", true);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bump, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    const uint32_t n = (uint32_t)nR;
    const unsigned grid = (unsigned)num_sms * 4;
    {
        ProfScope ps_("rg_clear", st);
        k_rg_clear<<<grid, RG_T, 0, st>>>(r);
    }
    if (n == 0) return cudaGetLastError();
    {
        ProfScope ps_("rg_count", st);
        k_rg_count<<<grid, RG_T, 0, st>>>(Ra, Rb, n, r, a_domain, status);
    }
    {
        ProfScope ps_("rg_offsets", st);
        k_rg_offsets<<<grid, RG_T, 0, st>>>(r, bump);
    }
    ProfScope ps_("rg_scatter", st);
    k_rg_scatter<<<grid, RG_T, 0, st>>>(Ra, Rb, n, r, n, status);
    return cudaGetLastError();
}

cudaError_t cyc_c_run(const CycCArgs &g, uint32_t *items, void *scan_tmp, unsigned int *counter,
                      unsigned long long *big_slots, void *scan_tmp64b, unsigned long long *bucket_rows,
                      unsigned long long *bucket_base, void *scan_tmp64, int32_t *rows, long long capacity,
                      long long *n_rows, unsigned long long *rep_set, uint32_t *rep_cnt, int num_sms,
                      cudaStream_t st) {
    const uint32_t z = g.z;
    const bool with_rows = (n_rows != nullptr);
    cudaError_t e;
    {
        ProfScope ps_("cyc_c_plan", st);
        k_cc_plan<<<(z + 255) / 256, 256, 0, st>>>(g.offS, g.offT, z, g.schunk, items, big_slots);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(items + z, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = scan_excl_u32(items, z + 1, scan_tmp, st)) != cudaSuccess) return e;
    // big buckets' sets in the workspace
    if ((e = scan_excl_u64((const uint64_t *)big_slots, (uint64_t *)g.big_off, z, true, scan_tmp64b, st)) !=
        cudaSuccess)
        return e;
    {
        ProfScope ps_("cyc_c_bigclear", st);
        k_cc_bigclear<<<num_sms * 4, 512, 0, st>>>((unsigned long long *)g.bigset, (uint32_t *)g.bigcnt,
                                                   g.big_off, z);
    }
    {
        ProfScope ps_("cyc_c_bigbuild", st);
        k_cc_bigbuild<<<num_sms * 2, 512, 0, st>>>(g.Tp, g.offT, z, g.big_off, (unsigned long long *)g.bigset,
                                                   (uint32_t *)g.bigcnt, (uint32_t *)g.big_neg, g.seed, g.st);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = CC_TSLOTS * sizeof(unsigned long long) + CC_QCAP * sizeof(uint4) +
                        (CC_QCAP + 1) * sizeof(uint32_t);
    if ((e = cudaFuncSetAttribute(k_cc_probe<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_cc_probe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cc_probe<0>, CC_T, smem) != cudaSuccess || occ < 1)
        occ = 1;
    if (occ > CC_MAX_CTAS_PER_SM) occ = CC_MAX_CTAS_PER_SM;   // one region per CTA for repeated pairs
    const unsigned grid = (unsigned)(num_sms * occ);
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    if (with_rows &&
        (e = cudaMemsetAsync(bucket_rows, 0, sizeof(unsigned long long) * (z + 1), st)) != cudaSuccess)
        return e;
    {
        ProfScope ps_("cyc_c_probe", st);
        k_cc_probe<0><<<grid, CC_T, smem, st>>>(g, items, counter, with_rows ? bucket_rows : nullptr, nullptr, 0,
                                                rep_set, rep_cnt);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!with_rows) return cudaSuccess;
    if ((e = scan_excl_u64((const uint64_t *)bucket_rows, (uint64_t *)bucket_base, z, true, scan_tmp64, st)) !=
        cudaSuccess)
        return e;
    {
        ProfScope ps_("rows_check", st);
        k_cc_rows_check<<<1, 1, 0, st>>>(bucket_base, z, capacity, n_rows, g.st);
    }
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    ProfScope ps_("cyc_c_rows", st);
    k_cc_probe<1><<<grid, CC_T, smem, st>>>(g, items, counter, bucket_base, rows, capacity, rep_set, rep_cnt);
    return cudaGetLastError();
}

}  // namespace mwj
