// cyclic.cu -- the cyclic 3-way join R(A,B) S(B,C) T(C,A) (Section 5).
//
// Shares (x, y, z) are the bucket counts of H(A), G(B) and F(C).  R is
// partitioned by (H(a), G(b)), S by (G(b), F(c)) and T by (F(c), H(a))
// (Fig. 3), so tile (i, j, k) joins R_ij, S_jk and T_ki.  The paper keeps
// R' on chip and streams S' and T' by f(c) through a sqrt(U) x sqrt(U) grid
// of memories; on the GPU a tile keeps both R_ij (as b -> [a] lists) and T_ki
// (as a multiset of (c, a) pairs) in one CTA's shared memory while S_jk
// streams past them, which generalises the paper's H, G partitioning with a
// third share on C (z = 1 is the paper's case).  Per S tuple (b, c) the CTA
// visits every a in R_ij[b] and counts (c, a) in T_ki.
//
// A tile whose R_ij or T_ki exceeds the on-chip capacity becomes several
// work items, one per (R chunk, T chunk) pair; the join distributes over the
// union of the chunks, so results do not change.  Work items are planned on
// the device (no host round trip) and a persistent grid takes them from an
// atomic counter.
#include "api_internal.h"
#include "cyclic.h"

namespace mwj {
namespace {

constexpr int CT = 512;              // threads per CTA
constexpr uint32_t RCAP = 2048;      // R tuples per chunk
constexpr uint32_t RSLOTS = 4096;    // b-table slots (>= 2 RCAP)
constexpr uint32_t TCAP = 2048;      // T tuples per chunk
constexpr uint32_t TSLOTS = 4096;    // (c,a)-set slots (>= 2 TCAP)

__host__ __device__ __forceinline__ uint32_t ceil_div(uint32_t a, uint32_t b) {
    return (a + b - 1) / b;
}

// tile index t = ((j * z + k) * x + i): consecutive items share S_jk
struct TileId {
    uint32_t i, j, k;
};
__device__ __forceinline__ TileId tile_of(uint32_t t, const CycArgs &g) {
    TileId id;
    id.i = t % g.x;
    uint32_t jk = t / g.x;
    id.k = jk % g.z;
    id.j = jk / g.z;
    return id;
}

// items per tile: R chunks x T chunks, 0 when any of the three is empty
__global__ void k_cyc_plan(CycArgs g, uint32_t *__restrict__ items) {
    const uint32_t ntiles = g.x * g.y * g.z;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        TileId id = tile_of(t, g);
        uint32_t rb = id.i * g.y + id.j, sb = id.j * g.z + id.k, tb = id.k * g.x + id.i;
        uint32_t nr = g.offR[rb + 1] - g.offR[rb];
        uint32_t ns = g.offS[sb + 1] - g.offS[sb];
        uint32_t nt = g.offT[tb + 1] - g.offT[tb];
        items[t] = (nr && ns && nt) ? ceil_div(nr, RCAP) * ceil_div(nt, TCAP) : 0u;
    }
}

__device__ __forceinline__ uint32_t pair_hash(uint32_t c, uint32_t a, uint32_t seed) {
    return mix32(c ^ mix32(a ^ seed));
}

__device__ __forceinline__ unsigned long long pack(uint32_t c, uint32_t a) {
    return ((unsigned long long)c << 32) | a;
}

// multiplicity of (c, a) in the T chunk set; slot TSLOTS holds (-1, -1)
__device__ __forceinline__ uint32_t tset_count(const unsigned long long *tk, const uint32_t *tc,
                                               uint32_t c, uint32_t a, uint32_t seed) {
    const unsigned long long key = pack(c, a);
    if (key == kEmpty64) return tc[TSLOTS];
    uint32_t s = pair_hash(c, a, seed) & (TSLOTS - 1);
    for (uint32_t it = 0; it < TSLOTS; ++it) {
        unsigned long long q = tk[s];
        if (q == key) return tc[s];
        if (q == kEmpty64) return 0;
        s = (s + 1) & (TSLOTS - 1);
    }
    return 0;
}

struct Smem {
    uint32_t rkeys[RSLOTS + 1];
    uint32_t rdeg[RSLOTS + 1];
    uint32_t rstart[RSLOTS + 1];
    int32_t alist[RCAP];
    unsigned long long tkeys[TSLOTS];
    uint32_t tcnt[TSLOTS + 1];
};

// Persistent kernel over the planned work items.  PASS 0 counts (COUNT,
// GROUP BY A, and pass 1 of row output, which adds each item's count to its
// tile's total); PASS 1 writes rows, taking positions from the tile's cursor
// (the scanned tile totals, advanced atomically).
template <int PASS>
__global__ void __launch_bounds__(CT) k_cyc_probe(CycArgs g, const uint32_t *__restrict__ item_off,
                                                  uint32_t ntiles, unsigned int *__restrict__ counter,
                                                  unsigned long long *__restrict__ tile_rows,
                                                  int32_t *__restrict__ rows, long long capacity) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem &sm = *(Smem *)smraw;
    __shared__ uint32_t item_s;
    __shared__ uint32_t scan_scratch[33];
    __shared__ uint32_t carry;
    __shared__ unsigned long long red[32];
    const uint32_t total_items = item_off[ntiles];
    if (PASS == 1 && tile_rows[ntiles] > (unsigned long long)capacity) return;
    const uint32_t lane = threadIdx.x & 31;
    unsigned long long acc_all = 0;

    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t item = item_s;
        __syncthreads();
        if (item >= total_items) break;
        // tile of this item: last t with item_off[t] <= item
        uint32_t lo = 0, hi = ntiles;
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (item_off[mid] <= item) lo = mid; else hi = mid;
        }
        const uint32_t t = lo;
        const TileId id = tile_of(t, g);
        const uint32_t rb = id.i * g.y + id.j, sb = id.j * g.z + id.k, tb = id.k * g.x + id.i;
        const uint32_t r0 = g.offR[rb], r1 = g.offR[rb + 1];
        const uint32_t s0 = g.offS[sb], s1 = g.offS[sb + 1];
        const uint32_t t0 = g.offT[tb], t1 = g.offT[tb + 1];
        const uint32_t ntc = ceil_div(t1 - t0, TCAP);
        const uint32_t local = item - item_off[t];
        const uint32_t rc = local / ntc, tc = local % ntc;
        const uint32_t ra = r0 + rc * RCAP, rz = min(r1, ra + RCAP);
        const uint32_t ta = t0 + tc * TCAP, tz = min(t1, ta + TCAP);

        // ---- build: R chunk as b -> [a], T chunk as a (c,a) multiset ----
        for (uint32_t q = threadIdx.x; q <= RSLOTS; q += CT) {
            sm.rkeys[q] = (q < RSLOTS) ? kEmptyKey : 0u;
            sm.rdeg[q] = 0u;
        }
        for (uint32_t q = threadIdx.x; q <= TSLOTS; q += CT) {
            if (q < TSLOTS) sm.tkeys[q] = kEmpty64;
            sm.tcnt[q] = 0u;
        }
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (uint32_t r = ra + threadIdx.x; r < rz; r += CT) {
            uint2 tu = __ldg(g.Rp + r);
            bool fresh;
            int slot = tbl_insert(sm.rkeys, RSLOTS - 1, tu.y, g.seed_slot, &fresh);
            if (slot >= 0) atomicAdd(&sm.rdeg[slot], 1u);
            else set_status(g.st, MWJ_ERR_CHECK, 11);
        }
        for (uint32_t q = ta + threadIdx.x; q < tz; q += CT) {
            uint2 tu = __ldg(g.Tp + q);   // (c, a)
            const unsigned long long key = pack(tu.x, tu.y);
            if (key == kEmpty64) {
                atomicAdd(&sm.tcnt[TSLOTS], 1u);
                continue;
            }
            uint32_t h = pair_hash(tu.x, tu.y, g.seed_slot2) & (TSLOTS - 1);
            bool done = false;
            for (uint32_t it = 0; it < TSLOTS; ++it) {
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
                h = (h + 1) & (TSLOTS - 1);
            }
            if (!done) set_status(g.st, MWJ_ERR_CHECK, 12);
        }
        __syncthreads();
        for (uint32_t b0 = 0; b0 <= RSLOTS; b0 += CT) {
            uint32_t q = b0 + threadIdx.x;
            uint32_t d = (q <= RSLOTS) ? sm.rdeg[q] : 0u;
            uint32_t tot;
            uint32_t ex = block_excl_scan_u32(d, scan_scratch, &tot);
            if (q <= RSLOTS) sm.rstart[q] = carry + ex;
            __syncthreads();
            if (threadIdx.x == 0) carry += tot;
            __syncthreads();
        }
        for (uint32_t r = ra + threadIdx.x; r < rz; r += CT) {
            uint2 tu = __ldg(g.Rp + r);
            int slot = tbl_find(sm.rkeys, RSLOTS - 1, tu.y, g.seed_slot);
            if (slot >= 0) {
                uint32_t p = atomicAdd(&sm.rstart[slot], 1u);
                if (p < RCAP) sm.alist[p] = (int32_t)tu.x;
            }
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q <= RSLOTS; q += CT) sm.rstart[q] -= sm.rdeg[q];
        __syncthreads();

        // ---- stream S_jk; each warp spreads its 32 tuples' a-lists evenly ----
        unsigned long long acc = 0;
        for (uint32_t w0 = s0 + (threadIdx.x & ~31u); w0 < s1; w0 += CT) {
            const uint32_t idx = w0 + lane;
            uint32_t b = 0, c = 0, n = 0, st = 0;
            if (idx < s1) {
                uint2 tu = __ldg(g.Sp + idx);
                b = tu.x;
                c = tu.y;
                int slot = tbl_find(sm.rkeys, RSLOTS - 1, b, g.seed_slot);
                if (slot >= 0) {
                    n = sm.rdeg[slot];
                    st = sm.rstart[slot];
                }
            }
            uint32_t incl = n;   // inclusive scan of the lanes' work counts
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += y;
            }
            const uint32_t W = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - n;
            for (uint32_t base = 0; base < W; base += 32) {
                const uint32_t wi = base + lane;
                // owner lane of work item wi: the first lane whose inclusive
                // count exceeds it (every lane runs the search)
                int olo = 0, ohi = 31;
                const uint32_t q = (wi < W) ? wi : 0u;
#pragma unroll
                for (int step = 0; step < 5; ++step) {
                    int mid = (olo + ohi) >> 1;
                    uint32_t v = __shfl_sync(0xffffffffu, incl, mid);
                    if (v > q) ohi = mid; else olo = mid + 1;
                }
                const int own = olo;
                const uint32_t ob = __shfl_sync(0xffffffffu, b, own);
                const uint32_t oc = __shfl_sync(0xffffffffu, c, own);
                const uint32_t ost = __shfl_sync(0xffffffffu, st, own);
                const uint32_t oex = __shfl_sync(0xffffffffu, excl, own);
                uint32_t m = 0, a = 0;
                if (wi < W) {
                    const uint32_t ai = ost + (wi - oex);
                    a = (ai < RCAP) ? (uint32_t)sm.alist[ai] : 0u;
                    m = tset_count(sm.tkeys, sm.tcnt, oc, a, g.seed_slot2);
                }
                if (PASS == 0) {
                    acc += m;
                    if (g.cnt && m && (uint32_t)a < (uint32_t)g.a_domain)
                        atomicAdd(g.cnt + a, (unsigned long long)m);
                } else {
                    uint32_t pincl = m;   // positions of this sweep's matches
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        uint32_t y = __shfl_up_sync(0xffffffffu, pincl, o);
                        if ((int)lane >= o) pincl += y;
                    }
                    const uint32_t btot = __shfl_sync(0xffffffffu, pincl, 31);
                    unsigned long long bb = 0;
                    if (lane == 0 && btot) bb = atomicAdd(tile_rows + t, (unsigned long long)btot);
                    bb = __shfl_sync(0xffffffffu, bb, 0);
                    unsigned long long p = bb + pincl - m;
                    for (uint32_t e = 0; e < m; ++e, ++p) {
                        if (p < (unsigned long long)capacity) {
                            int32_t *row = rows + 3 * p;
                            row[0] = (int32_t)a;
                            row[1] = (int32_t)ob;
                            row[2] = (int32_t)oc;
                        } else {
                            set_status(g.st, MWJ_ERR_CHECK, 13);
                        }
                    }
                }
            }
        }
        if (PASS == 0) {
            unsigned long long tot = block_sum_u64(acc, red);
            if (threadIdx.x == 0 && tile_rows && tot) atomicAdd(tile_rows + t, tot);
            acc_all += acc;
        }
        __syncthreads();
    }
    if (PASS == 0) {
        unsigned long long tot = block_sum_u64(acc_all, red);
        if (threadIdx.x == 0 && tot) atomicAdd(g.total, tot);
    }
}

__global__ void k_cyc_rows_check(const unsigned long long *base, uint32_t ntiles,
                                 long long capacity, long long *n_rows, DevStatus *st) {
    unsigned long long tot = base[ntiles];
    *n_rows = (long long)tot;
    if (tot > (unsigned long long)capacity) set_status(st, MWJ_ERR_CAPACITY, (long long)tot);
}

}  // namespace

uint32_t cyc_rcap() { return RCAP; }
uint32_t cyc_tcap() { return TCAP; }

size_t cyc_probe_smem() { return sizeof(Smem); }

cudaError_t cyc_run(const CycArgs &g, uint32_t *items, void *scan_tmp, unsigned int *counter,
                    unsigned long long *tile_rows, unsigned long long *tile_base, void *scan_tmp64,
                    int32_t *rows, long long capacity, long long *n_rows, int num_sms,
                    cudaStream_t st) {
    const uint32_t ntiles = g.x * g.y * g.z;
    const bool with_rows = (n_rows != nullptr);
    cudaError_t e;
    {
        ProfScope ps_("cyc_plan", st);
        k_cyc_plan<<<(ntiles + 255) / 256, 256, 0, st>>>(g, items);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // exclusive scan with the total at items[ntiles] (items[ntiles] = 0 on entry)
    if ((e = cudaMemsetAsync(items + ntiles, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = scan_excl_u32(items, ntiles + 1, scan_tmp, st)) != cudaSuccess) return e;
    const size_t smem = sizeof(Smem);
    e = cudaFuncSetAttribute(k_cyc_probe<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_cyc_probe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cyc_probe<0>, CT, smem);
    if (occ < 1) occ = 1;
    const unsigned grid = (unsigned)(num_sms * occ);
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    if (with_rows &&
        (e = cudaMemsetAsync(tile_rows, 0, sizeof(unsigned long long) * ntiles, st)) != cudaSuccess)
        return e;
    {
        ProfScope ps_("cyc_probe", st);
        k_cyc_probe<0><<<grid, CT, smem, st>>>(g, items, ntiles, counter,
                                               with_rows ? tile_rows : nullptr, nullptr, 0);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (with_rows) {
        if ((e = scan_excl_u64((const uint64_t *)tile_rows, (uint64_t *)tile_base, ntiles, true,
                               scan_tmp64, st)) != cudaSuccess)
            return e;
        {
            ProfScope ps_("rows_check", st);
            k_cyc_rows_check<<<1, 1, 0, st>>>(tile_base, ntiles, capacity, n_rows, g.st);
        }
        if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
        {
            ProfScope ps_("cyc_rows", st);
            k_cyc_probe<1><<<grid, CT, smem, st>>>(g, items, ntiles, counter, tile_base, rows,
                                                   capacity);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mwj
