// partition.cu -- radix hash partitioning of a relation (K1-K3).
//
// Algorithm 1's first three steps partition T by g(C), S by (H(B), g(C)) and
// R by H(B); Section 5 partitions R by (H(A), G(B)), S by (G(B), F(C)) and
// T by (F(C), H(A)) (Fig. 3).  All of these are one operation: bucket every
// tuple by one or two hashed columns and write the relation out grouped by
// bucket, with the bucket offsets.  The paper leaves the partitioner's
// design open (Section 4); this is the GB300 one:
//
//   K1 hist     every CTA owns a contiguous chunk of tiles and counts its
//               tuples per bucket in shared memory (one private histogram per
//               warp when they fit, so warps do not contend)
//   K2 scan     exclusive scan of the bucket-major (bucket, CTA) counts gives
//               every CTA its write cursor in every bucket
//   K3 scatter  every CTA re-reads its chunk tile by tile (128-bit loads),
//               counting-sorts each 4096-tuple tile by bucket in shared memory
//               and then writes each bucket's run with consecutive threads on
//               consecutive addresses, so the scattered output is written in
//               full sectors; for more than 4096 buckets the tile sort is
//               skipped and tuples go straight to their cursor.
//
// The order of tuples inside a bucket is not specified (atomics decide it);
// consumers never depend on it.
#include "internal.h"
#include "skew.h"

namespace mwj {
namespace {

constexpr int PT = 512;               // threads per CTA
constexpr int IPT = 8;                // tuples per thread per tile
constexpr int TILE = PT * IPT;        // 4096 tuples
constexpr uint32_t kStagedMaxP = 4096;
constexpr int kWarps = PT / 32;

// hs: the heavy-key table in shared memory, or null (no heavy keys)
__device__ __forceinline__ uint32_t bucket_tuple(int32_t x, int32_t y, const PartSpec &sp,
                                                 const uint32_t *hs) {
    int32_t k1 = sp.col1 ? y : x;
    if (hs && heavy_slot(hs, (uint32_t)k1) >= 0) return sp.Pbase();
    uint32_t b = bucket_of(k1, sp.seed1, sp.P1);
    if (sp.col2 >= 0) {
        int32_t k2 = sp.col2 ? y : x;
        b = b * sp.P2 + bucket_of(k2, sp.seed2, sp.P2);
    }
    return b;
}

struct Chunk {
    uint32_t begin, end;
};

__device__ __forceinline__ Chunk cta_chunk(uint32_t n, uint32_t tiles_per_cta) {
    uint64_t b = (uint64_t)blockIdx.x * tiles_per_cta * TILE;
    uint64_t e = b + (uint64_t)tiles_per_cta * TILE;
    Chunk c;
    c.begin = (uint32_t)(b < n ? b : n);
    c.end = (uint32_t)(e < n ? e : n);
    return c;
}

// K1: counts[b * G + cta] = number of this CTA's tuples in bucket b.  USE
// says which columns the bucket function reads (1 = x, 2 = y); only those
// are loaded.
template <bool WARP_PRIVATE, int USE>
__global__ void __launch_bounds__(PT) k_part_hist(const int32_t *__restrict__ x,
                                                  const int32_t *__restrict__ y, uint32_t n,
                                                  PartSpec sp, uint32_t tiles_per_cta,
                                                  uint32_t *__restrict__ counts) {
    __shared__ uint32_t hbuf[kHeavySlots];
    const uint32_t *hs = heavy_to_smem(sp.heavy, hbuf);
    extern __shared__ uint32_t hist[];
    const uint32_t P = sp.P();
    const uint32_t H = WARP_PRIVATE ? P * kWarps : P;
    for (uint32_t i = threadIdx.x; i < H; i += PT) hist[i] = 0;
    __syncthreads();
    uint32_t *my = WARP_PRIVATE ? hist + (threadIdx.x >> 5) * P : hist;
    Chunk c = cta_chunk(n, tiles_per_cta);
    const bool vec = (((uintptr_t)x | (uintptr_t)y) & 15) == 0;
    const uint64_t pol = l2_evict_first();
    uint32_t i = c.begin + threadIdx.x * 4;
    // one atomic per run of equal buckets among 4 consecutive tuples
    auto count4 = [&](const int4 &xv, const int4 &yv) {
        const uint32_t b0 = bucket_tuple(xv.x, yv.x, sp, hs), b1 = bucket_tuple(xv.y, yv.y, sp, hs),
                       b2 = bucket_tuple(xv.z, yv.z, sp, hs), b3 = bucket_tuple(xv.w, yv.w, sp, hs);
        uint32_t run = 1;
        if (b1 == b0) ++run; else { atomicAdd(&my[b0], run); run = 1; }
        if (b2 == b1) ++run; else { atomicAdd(&my[b1], run); run = 1; }
        if (b3 == b2) ++run; else { atomicAdd(&my[b2], run); run = 1; }
        atomicAdd(&my[b3], run);
    };
    if (vec) {
        // four 16-byte loads in flight per thread before any is consumed
        constexpr uint32_t U = 4;
        for (; i + (U - 1) * PT * 4 + 3 < c.end; i += U * PT * 4) {
            int4 xv[U], yv[U];
#pragma unroll
            for (uint32_t u = 0; u < U; ++u) {
                xv[u] = make_int4(0, 0, 0, 0);
                yv[u] = make_int4(0, 0, 0, 0);
                if (USE & 1) xv[u] = ld_stream((const int4 *)(x + i + u * PT * 4), pol);
                if (USE & 2) yv[u] = ld_stream((const int4 *)(y + i + u * PT * 4), pol);
            }
#pragma unroll
            for (uint32_t u = 0; u < U; ++u) count4(xv[u], yv[u]);
        }
        for (; i + 3 < c.end; i += PT * 4) {
            int4 xv = make_int4(0, 0, 0, 0), yv = make_int4(0, 0, 0, 0);
            if (USE & 1) xv = ld_stream((const int4 *)(x + i), pol);
            if (USE & 2) yv = ld_stream((const int4 *)(y + i), pol);
            count4(xv, yv);
        }
    }
    for (; i < c.end; i += PT * 4) {
        for (uint32_t k = i; k < i + 4 && k < c.end; ++k) {
            int32_t xv = (USE & 1) ? __ldg(x + k) : 0;
            int32_t yv = (USE & 2) ? __ldg(y + k) : 0;
            atomicAdd(&my[bucket_tuple(xv, yv, sp, hs)], 1u);
        }
    }
    __syncthreads();
    const uint32_t G = gridDim.x;
    for (uint32_t b = threadIdx.x; b < P; b += PT) {
        uint32_t s = 0;
        if (WARP_PRIVATE) {
#pragma unroll 4
            for (int w = 0; w < kWarps; ++w) s += hist[w * P + b];
        } else {
            s = hist[b];
        }
        counts[(size_t)b * G + blockIdx.x] = s;
    }
}

template <bool WP>
cudaError_t hist_launch(const int32_t *x, const int32_t *y, uint32_t n, const PartSpec &sp,
                        uint32_t G, uint32_t tpc, uint32_t *counts, size_t hs, cudaStream_t st) {
    int use = (sp.col1 ? 2 : 1) | (sp.col2 < 0 ? 0 : (sp.col2 ? 2 : 1));
    auto kern = use == 1 ? k_part_hist<WP, 1> : (use == 2 ? k_part_hist<WP, 2> : k_part_hist<WP, 3>);
    if (hs > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs);
        if (e != cudaSuccess) return e;
    }
    ProfScope ps_("part_hist", st);
    kern<<<G, PT, hs, st>>>(x, y, n, sp, tpc, counts);
    return cudaGetLastError();
}

// bucket_off[b] = scanned[b * G], bucket_off[P] = n.
__global__ void k_bucket_offsets(const uint32_t *__restrict__ scanned, uint32_t P, uint32_t G,
                                 uint32_t n, uint32_t *__restrict__ bucket_off) {
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < P) bucket_off[b] = scanned[(size_t)b * G];
    if (b == P) bucket_off[P] = n;
}

template <int PAY>
struct PayT {
    using T = uint32_t;
};
template <>
struct PayT<PAY_PAIR> {
    using T = uint2;
};

template <int PAY>
__device__ __forceinline__ typename PayT<PAY>::T make_pay(int32_t x, int32_t y) {
    if constexpr (PAY == PAY_PAIR) {
        return make_uint2((uint32_t)x, (uint32_t)y);
    } else if constexpr (PAY == PAY_X) {
        return (uint32_t)x;
    } else {
        return (uint32_t)y;
    }
}

// K3 (P <= 4096): tile-local counting sort in shared memory, coalesced runs.
template <int PAY>
__global__ void __launch_bounds__(PT) k_part_scatter_staged(
    const int32_t *__restrict__ x, const int32_t *__restrict__ y, uint32_t n, PartSpec sp,
    uint32_t tiles_per_cta, const uint32_t *__restrict__ scanned,
    typename PayT<PAY>::T *__restrict__ out) {
    __shared__ uint32_t hbuf[kHeavySlots];
    const uint32_t *hs = heavy_to_smem(sp.heavy, hbuf);
    using T = typename PayT<PAY>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t P = sp.P();
    uint32_t *cur = (uint32_t *)smem;                    // P: global write cursor
    uint32_t *cnt = cur + P;                             // P: tile counts
    uint32_t *off = cnt + P;                             // P: tile offsets
    T *stage = (T *)(smem + align256(3 * P * sizeof(uint32_t)));   // TILE
    uint32_t *gpos = (uint32_t *)(stage + TILE);         // TILE: output position of each staged tuple
    int32_t *xin = (int32_t *)(gpos + TILE);             // TILE: the tile's x column (bulk copy)
    int32_t *yin = xin + TILE;                           // TILE: its y column
    __shared__ uint32_t scan_scratch[33];
    __shared__ __align__(8) unsigned long long tile_bar;

    const uint32_t G = gridDim.x;
    for (uint32_t b = threadIdx.x; b < P; b += PT) cur[b] = scanned[(size_t)b * G + blockIdx.x];
    Chunk c = cta_chunk(n, tiles_per_cta);
    // tiles start at multiples of TILE, so with 16-byte aligned columns every
    // tile's first 4*floor(tn/4) values can be bulk-copied; the last few
    // values of a ragged final tile are read directly
    const bool vec = (((uintptr_t)x | (uintptr_t)y) & 15) == 0;
    const bool same = (x == y);
    // entries of the per-thread scan over P
    const uint32_t per = (P + PT - 1) / PT;
    auto issue = [&](uint32_t t0) {
        const uint32_t tn = min((uint32_t)TILE, c.end - t0);
        const uint32_t bulk = (tn & ~3u) * 4u;   // bytes, multiple of 16
        if (bulk == 0) return;
        fence_proxy_async();
        mbar_expect_tx(&tile_bar, same ? bulk : 2 * bulk);
        bulk_copy_g2s(xin, x + t0, bulk, &tile_bar);
        if (!same) bulk_copy_g2s(yin, y + t0, bulk, &tile_bar);
    };
    uint32_t fills = 0;   // completed phases of tile_bar (same in every thread)
    if (vec) {
        if (threadIdx.x == 0) {
            mbar_init(&tile_bar, 1);
            fence_barrier_init();
        }
        __syncthreads();
        if (threadIdx.x == 0 && c.begin < c.end) issue(c.begin);
    }

    for (uint32_t t0 = c.begin; t0 < c.end; t0 += TILE) {
        const uint32_t tn = min((uint32_t)TILE, c.end - t0);
        for (uint32_t b = threadIdx.x; b < P; b += PT) cnt[b] = 0;
        const bool staged_in = vec && (tn & ~3u) > 0;
        bool ok = true;
        if (staged_in) {
            ok = mbar_wait_bounded(&tile_bar, fills & 1u, 1u << 24);
            ++fills;
        }
        if (__syncthreads_or(!ok)) {
            // the tile's copy did not land in time: record it and stop (its
            // data would not match the histogram, so nothing may be written)
            if (threadIdx.x == 0) {
                if (sp.st) set_status(sp.st, MWJ_ERR_TIMEOUT, (long long)blockIdx.x);
                mbar_wait_bounded(&tile_bar, (fills - 1u) & 1u, 1u << 24);
            }
            __syncthreads();
            return;
        }
        uint32_t bk[IPT], rk[IPT];
        T pv[IPT];
        int32_t xs8[IPT], ys8[IPT];
        // thread t handles tuples t0 + 4*t + {0..3} and t0 + 2048 + 4*t + {0..3}
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t li = (uint32_t)h * (TILE / 2) + threadIdx.x * 4;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t l = li + k;
                int32_t xv = 0, yv = 0;
                if (l < tn) {
                    if (staged_in && l < (tn & ~3u)) {
                        xv = xin[l];
                        yv = same ? xv : yin[l];
                    } else {
                        xv = __ldg(x + t0 + l);
                        yv = __ldg(y + t0 + l);
                    }
                }
                xs8[h * 4 + k] = xv;
                ys8[h * 4 + k] = yv;
            }
        }
        if (staged_in) {
            __syncthreads();   // every thread has its values: the buffers are free
            if (threadIdx.x == 0 && t0 + TILE < c.end) issue(t0 + TILE);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t li = (uint32_t)h * (TILE / 2) + threadIdx.x * 4;
            int32_t xs[4], ys[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                xs[k] = xs8[h * 4 + k];
                ys[k] = ys8[h * 4 + k];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int j = h * 4 + k;
                if (li + k < tn) {
                    if (sp.dom && (uint32_t)xs[k] >= sp.dom && sp.st) set_status(sp.st, MWJ_ERR_DOMAIN, xs[k]);
                    bk[j] = bucket_tuple(xs[k], ys[k], sp, hs);
                    rk[j] = atomicAdd(&cnt[bk[j]], 1u);
                    pv[j] = make_pay<PAY>(xs[k], ys[k]);
                } else {
                    bk[j] = 0xFFFFFFFFu;
                }
            }
        }
        __syncthreads();
        // exclusive scan of cnt[0..P) into off[]
        {
            uint32_t b0 = threadIdx.x * per;
            uint32_t s = 0;
            for (uint32_t k = 0; k < per; ++k)
                if (b0 + k < P) s += cnt[b0 + k];
            uint32_t base = block_excl_scan_u32(s, scan_scratch, nullptr);
            for (uint32_t k = 0; k < per; ++k)
                if (b0 + k < P) {
                    off[b0 + k] = base;
                    base += cnt[b0 + k];
                }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            if (bk[j] != 0xFFFFFFFFu) {
                uint32_t p = off[bk[j]] + rk[j];
                stage[p] = pv[j];
                gpos[p] = cur[bk[j]] + rk[j];
            }
        }
        __syncthreads();
        // consecutive threads write consecutive positions of each bucket's run
        for (uint32_t e = threadIdx.x; e < tn; e += PT) out[gpos[e]] = stage[e];
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < P; b += PT) cur[b] += cnt[b];
        __syncthreads();
    }
}

// K3 (P <= kWcMaxP): tile-local counting sort with write combining.  The
// run of bucket b in a tile is the tuples the CTA carried over from its
// earlier tiles followed by the tile's own; only whole 32-byte sectors of
// the run are written and the remainder (less than a sector) is carried on.
// Apart from the first and the last sector of each CTA's range in a bucket,
// every output sector is thus written once and whole, within one phase of
// one tile, so the L2 never has to merge a partly written sector with its
// DRAM contents (a DRAM read each).
//
// Carried tuples always lie in one sector, [gs, gs + carried): either the
// run completes that sector (then all of them are written, W >= carried)
// or nothing of the run is written and they stay in their carry slots.
constexpr uint32_t kWcMaxP = 1152;   // 1024 hashed buckets + a heavy-key bucket fit two CTAs per SM
constexpr uint32_t kToCarry = 0x80000000u;   // gpos flag: carry slot, not an output position
constexpr uint32_t kNoBucket = 0xFFFFu;      // past the end of a ragged tile

template <int PAY>
__host__ __device__ constexpr uint32_t wc_carry() {
    return 32u / (uint32_t)sizeof(typename PayT<PAY>::T) - 1u;
}

template <int PAY>
size_t wc_smem(uint32_t P) {
    using T = typename PayT<PAY>::T;
    return align256((size_t)P * sizeof(uint4)) + align256((size_t)P * sizeof(uint32_t)) +
           align256((size_t)P * wc_carry<PAY>() * sizeof(T)) + TILE * sizeof(T) + TILE * sizeof(uint32_t);
}

template <int PAY>
__global__ void __launch_bounds__(PT, 2) k_part_scatter_wc(
    const int32_t *__restrict__ x, const int32_t *__restrict__ y, uint32_t n, PartSpec sp,
    uint32_t tiles_per_cta, const uint32_t *__restrict__ scanned,
    typename PayT<PAY>::T *__restrict__ out) {
    __shared__ uint32_t hbuf[kHeavySlots];
    const uint32_t *hs = heavy_to_smem(sp.heavy, hbuf);
    using T = typename PayT<PAY>::T;
    constexpr uint32_t CARRY = wc_carry<PAY>();
    constexpr uint32_t SECT = CARRY + 1;   // tuples per 32-byte sector
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t P = sp.P();
    // per bucket: x = the tile run's start in stage, y = tuples carried in,
    // z = tuples of the run to write (W), w = global position of the run
    uint4 *bs = (uint4 *)smem;
    uint32_t *cnt = (uint32_t *)(smem + align256((size_t)P * sizeof(uint4)));
    T *carry = (T *)((unsigned char *)cnt + align256((size_t)P * sizeof(uint32_t)));
    T *stage = (T *)((unsigned char *)carry + align256((size_t)P * CARRY * sizeof(T)));
    uint32_t *gpos = (uint32_t *)(stage + TILE);
    __shared__ uint32_t scan_scratch[33];

    const uint32_t G = gridDim.x;
    for (uint32_t b = threadIdx.x; b < P; b += PT) {
        bs[b] = make_uint4(0u, 0u, 0u, scanned[(size_t)b * G + blockIdx.x]);
        cnt[b] = 0;
    }
    const Chunk c = cta_chunk(n, tiles_per_cta);
    const bool vec = (((uintptr_t)x | (uintptr_t)y) & 15) == 0;
    const uint32_t per = (P + PT - 1) / PT;
    const uint64_t pol = l2_evict_first();
    // thread t holds tuples 4t + {0..3} and TILE/2 + 4t + {0..3} of a tile
    int32_t xs[IPT], ys[IPT];
    auto load = [&](uint32_t t0) {
        const uint32_t tn = min((uint32_t)TILE, c.end - t0);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t li = (uint32_t)h * (TILE / 2) + threadIdx.x * 4;
            if (vec && li + 3 < tn) {
                const int4 a = ld_stream((const int4 *)(x + t0 + li), pol);
                const int4 b = ld_stream((const int4 *)(y + t0 + li), pol);
                xs[4 * h] = a.x; xs[4 * h + 1] = a.y; xs[4 * h + 2] = a.z; xs[4 * h + 3] = a.w;
                ys[4 * h] = b.x; ys[4 * h + 1] = b.y; ys[4 * h + 2] = b.z; ys[4 * h + 3] = b.w;
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t l = li + k;
                    xs[4 * h + k] = l < tn ? __ldg(x + t0 + l) : 0;
                    ys[4 * h + k] = l < tn ? __ldg(y + t0 + l) : 0;
                }
            }
        }
    };
    if (c.begin < c.end) load(c.begin);
    __syncthreads();

    for (uint32_t t0 = c.begin; t0 < c.end; t0 += TILE) {
        const uint32_t tn = min((uint32_t)TILE, c.end - t0);
        const bool last = t0 + TILE >= c.end;
        // 1. bucket and rank of every tuple, packed (bucket << 16 | rank);
        //    a thread's runs of equal buckets among its 4 consecutive tuples
        //    take one atomic each
        uint32_t br[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t l = (uint32_t)(j >> 2) * (TILE / 2) + threadIdx.x * 4 + (j & 3);
            uint32_t b = kNoBucket;
            if (l < tn) {
                if (sp.dom && (uint32_t)xs[j] >= sp.dom && sp.st) set_status(sp.st, MWJ_ERR_DOMAIN, xs[j]);
                b = bucket_tuple(xs[j], ys[j], sp, hs);
            }
            const bool cont = (j & 3) && b == (br[j - 1 < 0 ? 0 : j - 1] >> 16);
            br[j] = (b << 16) | (cont ? (br[j - 1 < 0 ? 0 : j - 1] & 0xFFFFu) + 1u : 0u);   // place in its run
        }
        {
            uint32_t base = 0;   // of the run being walked back from its end
#pragma unroll
            for (int j = IPT - 1; j >= 0; --j) {
                const uint32_t b = br[j] >> 16;
                const bool run_end = (j & 3) == 3 || (br[j + 1 < IPT ? j + 1 : j] >> 16) != b;
                if (run_end && b != kNoBucket) base = atomicAdd(&cnt[b], (br[j] & 0xFFFFu) + 1u);
                br[j] += base;
            }
        }
        __syncthreads();
        // 2. the tile's counts scanned into run starts; W = whole sectors of
        //    carried + new (all of it in the CTA's last tile)
        {
            const uint32_t b0 = threadIdx.x * per;
            uint32_t sum = 0;
            for (uint32_t k = 0; k < per; ++k)
                if (b0 + k < P) sum += cnt[b0 + k];
            uint32_t base = block_excl_scan_u32(sum, scan_scratch, nullptr);
            for (uint32_t k = 0; k < per; ++k) {
                const uint32_t b = b0 + k;
                if (b >= P) break;
                uint4 v = bs[b];
                const uint32_t L = v.y + cnt[b];
                const uint32_t aligned = (v.w + L) & ~(SECT - 1u);
                v.x = base;
                v.z = last ? L : (aligned > v.w ? aligned - v.w : 0u);
                bs[b] = v;
                base += cnt[b];
            }
        }
        __syncthreads();
        // 3. stage the tile by bucket with each tuple's destination; write
        //    the carried tuples of the runs that complete their sector
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t b = br[j] >> 16, rk = br[j] & 0xFFFFu;
            if (b != kNoBucket) {
                const uint4 v = bs[b];
                const uint32_t p = v.x + rk, r = v.y + rk;
                stage[p] = make_pay<PAY>(xs[j], ys[j]);
                gpos[p] = r < v.z ? v.w + r : (kToCarry | (b * CARRY + (r - v.z)));
            }
        }
        for (uint32_t b = threadIdx.x; b < P; b += PT) {
            const uint4 v = bs[b];
            if (v.z)
                for (uint32_t q = 0; q < v.y; ++q) st_stream(out + v.w + q, carry[b * CARRY + q], pol);
        }
        if (!last) load(t0 + TILE);   // the next tile's loads fly during the write-out
        __syncthreads();
        // 4. write the tile: whole sectors out, the rest into the carry slots
        for (uint32_t e = threadIdx.x; e < tn; e += PT) {
            const uint32_t g = gpos[e];
            const T v = stage[e];
            if (g & kToCarry) carry[g & ~kToCarry] = v;
            else st_stream(out + g, v, pol);
        }
        __syncthreads();
        // 5. the next run starts where this one's writes ended
        for (uint32_t b = threadIdx.x; b < P; b += PT) {
            uint4 v = bs[b];
            const uint32_t L = v.y + cnt[b];
            v.w += v.z;
            v.y = L - v.z;
            bs[b] = v;
            cnt[b] = 0;
        }
        __syncthreads();
    }
}

// K3 (P > 4096): direct scatter through shared-memory cursors.
template <int PAY>
__global__ void __launch_bounds__(PT) k_part_scatter_direct(
    const int32_t *__restrict__ x, const int32_t *__restrict__ y, uint32_t n, PartSpec sp,
    uint32_t tiles_per_cta, const uint32_t *__restrict__ scanned,
    typename PayT<PAY>::T *__restrict__ out) {
    __shared__ uint32_t hbuf[kHeavySlots];
    const uint32_t *hs = heavy_to_smem(sp.heavy, hbuf);
    extern __shared__ uint32_t cur[];
    const uint32_t P = sp.P();
    const uint32_t G = gridDim.x;
    for (uint32_t b = threadIdx.x; b < P; b += PT) cur[b] = scanned[(size_t)b * G + blockIdx.x];
    __syncthreads();
    Chunk c = cta_chunk(n, tiles_per_cta);
    for (uint32_t i = c.begin + threadIdx.x; i < c.end; i += PT) {
        int32_t xv = __ldg(x + i), yv = __ldg(y + i);
        if (sp.dom && (uint32_t)xv >= sp.dom && sp.st) set_status(sp.st, MWJ_ERR_DOMAIN, xv);
        uint32_t b = bucket_tuple(xv, yv, sp, hs);
        uint32_t p = atomicAdd(&cur[b], 1u);
        out[p] = make_pay<PAY>(xv, yv);
    }
}

// K3 with a third carried column z (pairs + z, direct scatter): the cascade's
// second cyclic join partitions I(a,b,c) by (c,a) and carries b.
__global__ void __launch_bounds__(PT) k_part_scatter_z(
    const int32_t *__restrict__ x, const int32_t *__restrict__ y, const int32_t *__restrict__ z,
    uint32_t n, PartSpec sp, uint32_t tiles_per_cta, const uint32_t *__restrict__ scanned,
    uint2 *__restrict__ out, int32_t *__restrict__ outz) {
    __shared__ uint32_t hbuf[kHeavySlots];
    const uint32_t *hs = heavy_to_smem(sp.heavy, hbuf);
    extern __shared__ uint32_t cur[];
    const uint32_t P = sp.P();
    const uint32_t G = gridDim.x;
    for (uint32_t b = threadIdx.x; b < P; b += PT) cur[b] = scanned[(size_t)b * G + blockIdx.x];
    __syncthreads();
    Chunk c = cta_chunk(n, tiles_per_cta);
    for (uint32_t i = c.begin + threadIdx.x; i < c.end; i += PT) {
        int32_t xv = __ldg(x + i), yv = __ldg(y + i);
        uint32_t b = bucket_tuple(xv, yv, sp, hs);
        uint32_t p = atomicAdd(&cur[b], 1u);
        out[p] = make_uint2((uint32_t)xv, (uint32_t)yv);
        outz[p] = __ldg(z + i);
    }
}

struct Geometry {
    uint32_t G, tiles_per_cta;
};

// G CTAs (at most max_ctas, one resident wave) each own a contiguous run of
// tiles_per_cta tiles.
Geometry geometry(int64_t n, int max_ctas) {
    uint64_t tiles = ((uint64_t)n + TILE - 1) / TILE;
    if (tiles == 0) tiles = 1;
    uint64_t gmax = (uint64_t)(max_ctas > 0 ? max_ctas : 1);
    uint64_t G = tiles < gmax ? tiles : gmax;
    uint64_t tpc = (tiles + G - 1) / G;
    G = (tiles + tpc - 1) / tpc;
    return Geometry{(uint32_t)G, (uint32_t)tpc};
}

size_t hist_smem(uint32_t P, bool warp_private) {
    return (size_t)P * sizeof(uint32_t) * (warp_private ? kWarps : 1);
}

template <int PAY>
cudaError_t scatter_launch(const int32_t *x, const int32_t *y, uint32_t n, const PartSpec &sp,
                           Geometry g, const uint32_t *scanned, void *out, cudaStream_t st) {
    using T = typename PayT<PAY>::T;
    const uint32_t P = sp.P();
    if (P <= kWcMaxP) {
        const size_t smem = wc_smem<PAY>(P);
        auto kern = k_part_scatter_wc<PAY>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        ProfScope ps_("part_scatter", st);
        kern<<<g.G, PT, smem, st>>>(x, y, n, sp, g.tiles_per_cta, scanned, (T *)out);
    } else if (P <= kStagedMaxP) {
        size_t smem = align256(3 * P * sizeof(uint32_t)) + TILE * sizeof(T) + TILE * sizeof(uint32_t) +
                      2 * TILE * sizeof(int32_t);
        auto kern = k_part_scatter_staged<PAY>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        ProfScope ps_("part_scatter", st);
        kern<<<g.G, PT, smem, st>>>(x, y, n, sp, g.tiles_per_cta, scanned, (T *)out);
    } else {
        size_t smem = P * sizeof(uint32_t);
        auto kern = k_part_scatter_direct<PAY>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        ProfScope ps_("part_scatter_direct", st);
        kern<<<g.G, PT, smem, st>>>(x, y, n, sp, g.tiles_per_cta, scanned, (T *)out);
    }
    return cudaGetLastError();
}

}  // namespace

// Sized for the largest grid any n' <= n can get, min(tiles(n), max CTAs),
// so a workspace sized for n serves every smaller call (geometry()'s own G is
// not monotone in n: rounding tiles per CTA up can leave fewer CTAs).
size_t part_scratch_bytes(int64_t n, uint32_t P, int num_sms) {
    uint64_t tiles = ((uint64_t)(n > 0 ? n : 0) + TILE - 1) / TILE;
    if (tiles == 0) tiles = 1;
    const uint64_t gmax = (uint64_t)(num_sms > 0 ? num_sms : 1) * 4;
    const size_t cnt = (size_t)P * (size_t)(tiles < gmax ? tiles : gmax);
    return align256(cnt * sizeof(uint32_t)) + scan_scratch_bytes(cnt);
}

cudaError_t part_run(const int32_t *x, const int32_t *y, int64_t n64, const PartSpec &sp,
                     int payload, void *out, uint32_t *bucket_off, void *scratch,
                     size_t scratch_bytes, int num_sms, cudaStream_t st, const int32_t *z,
                     int32_t *outz) {
    const uint32_t P = sp.P();
    if (P == 0 || P > kMaxBuckets || n64 < 0 || n64 > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    if (scratch_bytes < part_scratch_bytes(n64, P, num_sms)) return cudaErrorInvalidValue;
    const uint32_t n = (uint32_t)n64;
    if (n == 0) {
        return cudaMemsetAsync(bucket_off, 0, (P + 1) * sizeof(uint32_t), st);
    }
    // one wave of the scatter kernel: its resident CTAs per SM x SMs
    int occ = 1;
    {
        const bool staged = P <= kStagedMaxP;
        const bool pair = payload == PAY_PAIR;
        size_t ssz = pair ? sizeof(uint2) : sizeof(uint32_t);
        size_t smem = staged ? align256(3 * P * sizeof(uint32_t)) + TILE * ssz + TILE * sizeof(uint32_t) +
                                   2 * TILE * sizeof(int32_t)
                             : P * sizeof(uint32_t);
        const void *kern = staged ? (pair ? (const void *)k_part_scatter_staged<PAY_PAIR>
                                          : (const void *)k_part_scatter_staged<PAY_X>)
                                  : (pair ? (const void *)k_part_scatter_direct<PAY_PAIR>
                                          : (const void *)k_part_scatter_direct<PAY_X>);
        if (P <= kWcMaxP && !z) {
            smem = pair ? wc_smem<PAY_PAIR>(P) : wc_smem<PAY_X>(P);
            kern = pair ? (const void *)k_part_scatter_wc<PAY_PAIR> : (const void *)k_part_scatter_wc<PAY_X>;
        }
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, PT, smem) != cudaSuccess || occ < 1)
            occ = 1;
        if (occ > 4) occ = 4;
    }
    Geometry g = geometry(n64, num_sms * occ);
    uint32_t *counts = (uint32_t *)scratch;
    size_t ncnt = (size_t)P * g.G;
    void *scan_tmp = (char *)scratch + align256(ncnt * sizeof(uint32_t));

    const bool warp_private = hist_smem(P, true) <= 48 * 1024;
    size_t hs = hist_smem(P, warp_private);
    cudaError_t e = warp_private ? hist_launch<true>(x, y, n, sp, g.G, g.tiles_per_cta, counts, hs, st)
                                 : hist_launch<false>(x, y, n, sp, g.G, g.tiles_per_cta, counts, hs, st);
    if (e != cudaSuccess) return e;
    if ((e = scan_excl_u32(counts, ncnt, scan_tmp, st)) != cudaSuccess) return e;
    {
        ProfScope ps_("part_offsets", st);
        k_bucket_offsets<<<(P + 1 + 255) / 256, 256, 0, st>>>(counts, P, g.G, n, bucket_off);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // a column that neither the bucket function nor the payload reads is
    // aliased to the other one, so the scatter's loads of it hit the same lines
    const bool need_x = sp.col1 == 0 || sp.col2 == 0 || payload == PAY_PAIR || payload == PAY_X ||
                        sp.dom > 0;
    const bool need_y = sp.col1 == 1 || sp.col2 == 1 || payload == PAY_PAIR || payload == PAY_Y;
    if (!need_y) y = x;
    if (!need_x) x = y;
    if (z) {
        size_t smem = P * sizeof(uint32_t);
        e = cudaFuncSetAttribute(k_part_scatter_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ProfScope ps_("part_scatter_z", st);
        k_part_scatter_z<<<g.G, PT, smem, st>>>(x, y, z, n, sp, g.tiles_per_cta, counts, (uint2 *)out,
                                                outz);
        return cudaGetLastError();
    }
    switch (payload) {
        case PAY_PAIR: return scatter_launch<PAY_PAIR>(x, y, n, sp, g, counts, out, st);
        case PAY_X: return scatter_launch<PAY_X>(x, y, n, sp, g, counts, out, st);
        default: return scatter_launch<PAY_Y>(x, y, n, sp, g, counts, out, st);
    }
}

}  // namespace mwj
