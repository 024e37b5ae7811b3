// skew.cu -- heavy join keys of the linear aggregates.
//
// Section 1.2 assumes no skew, and the paper names skewed inputs as future
// work.  Under a skewed B column (Zipf, a few keys holding a large share of
// R or S) hash partitioning by H(B) puts each heavy key, with all of its
// tuples, into one bucket, and the CTA that owns that bucket does a large
// share of the whole join alone.  Heavy keys are therefore split off (the
// heavy/light decomposition of skew-aware multiway joins):
//
//   1. a sample of R's and S's B columns names the heavy keys: those whose
//      sampled share in either relation reaches half an average bucket;
//   2. the partitioner sends every tuple whose B value is heavy to one extra
//      bucket (the light keys are partitioned as before);
//   3. the per-bucket join handles the light buckets; the heavy bucket is
//      aggregated by every CTA at once.  For a heavy key h,
//        w(h) = sum over S tuples (h, c) of deg_T(c)
//      is a plain reduction (per-CTA shared sums, one global add per key and
//      CTA), and every R tuple (a, h) then adds w(h) to cnt[a] and to the
//      total.
//
// The heavy and light parts are disjoint in B, so their results add up to
// the join's: the decomposition changes the work assignment only.
#include "skew.h"

#include "internal.h"

namespace mwj {
namespace {

constexpr int DT = 1024;                 // detection: one CTA
constexpr uint32_t kSample = 2048;       // sampled tuples per relation
constexpr uint32_t kCountSlots = 8192;   // sample count table (shared memory), at most half full
constexpr uint32_t kMinCount = 8;        // a heavy key is seen at least this often in its sample
constexpr uint32_t kPerThread = kSample / DT;
constexpr int HT = 512;                  // heavy-bucket kernels: threads per CTA

// One CTA: count a strided sample of each B column (kSample tuples, every
// thread's loads in flight together) in a shared table of (key, count in R,
// count in S, packed in one word); keys whose count reaches the threshold of
// their relation go into the heavy table.  The sample decides only which
// keys take the heavy path, never the join's result.  The threshold is half
// an average bucket and at least kMinCount sampled tuples (a 0.4% share): a
// key far below it -- a hub of a power-law graph holds ~1e-4 of the edges --
// is practically never sampled that often, so inputs without heavy keys keep
// an empty table and the partitioner skips the per-tuple check.
__global__ void __launch_bounds__(DT) k_heavy_detect(const int32_t *__restrict__ rb, uint32_t nR,
                                                     const int32_t *__restrict__ sb, uint32_t nS,
                                                     uint32_t I, uint32_t *__restrict__ heavy,
                                                     unsigned long long *__restrict__ hw) {
    extern __shared__ uint32_t sm[];
    uint32_t *key = sm;                      // kCountSlots
    uint32_t *cnt = key + kCountSlots;       // kCountSlots: count in R | count in S << 16
    uint32_t *ht = cnt + kCountSlots;        // kHeavySlots
    __shared__ uint32_t nh;
    for (uint32_t i = threadIdx.x; i < kCountSlots; i += DT) {
        key[i] = kEmptyKey;
        cnt[i] = 0;
    }
    for (uint32_t i = threadIdx.x; i < kHeavySlots; i += DT) {
        ht[i] = kEmptyKey;
        hw[i] = 0;
    }
    if (threadIdx.x == 0) nh = 0;
    __syncthreads();
    auto count = [&](const int32_t *col, uint32_t n, uint32_t one) {
        const uint32_t m = n < kSample ? n : kSample;
        uint32_t ks[kPerThread];
#pragma unroll
        for (uint32_t q = 0; q < kPerThread; ++q) {
            const uint32_t j = threadIdx.x + q * DT;
            ks[q] = j < m ? (uint32_t)__ldg(col + (uint32_t)(((uint64_t)j * n) / m)) : kEmptyKey;
        }
#pragma unroll
        for (uint32_t q = 0; q < kPerThread; ++q) {
            const uint32_t k = ks[q];
            if (k == kEmptyKey) continue;   // the table's empty marker is never heavy
            uint32_t s = slot_of(k, kHeavySeed, kCountSlots - 1);
            for (uint32_t it = 0; it < kCountSlots; ++it) {   // at most half full: ends early
                uint32_t held = key[s];
                if (held == kEmptyKey) {
                    held = atomicCAS(&key[s], kEmptyKey, k);
                    if (held == kEmptyKey) held = k;
                }
                if (held == k) {
                    atomicAdd(&cnt[s], one);
                    break;
                }
                s = (s + 1) & (kCountSlots - 1);
            }
        }
    };
    count(rb, nR, 1u);
    count(sb, nS, 1u << 16);
    __syncthreads();
    // share >= 1 / (2 I) of the sample, and at least kMinCount sampled tuples
    const uint32_t mR = nR < kSample ? nR : kSample, mS = nS < kSample ? nS : kSample;
    const uint32_t tR = max(kMinCount, mR / (2u * I)), tS = max(kMinCount, mS / (2u * I));
    for (uint32_t i = threadIdx.x; i < kCountSlots; i += DT) {
        const uint32_t k = key[i];
        if (k == kEmptyKey || ((cnt[i] & 0xFFFFu) < tR && (cnt[i] >> 16) < tS)) continue;
        if (atomicAdd(&nh, 1u) >= kHeavyMax) continue;
        // at most kHeavyMax = kHeavySlots / 2 keys: a free slot is always found
        uint32_t s = slot_of(k, kHeavySeed, kHeavySlots - 1);
        for (uint32_t it = 0; it < kHeavySlots && atomicCAS(&ht[s], kEmptyKey, k) != kEmptyKey; ++it)
            s = (s + 1) & (kHeavySlots - 1);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kHeavySlots; i += DT) heavy[i] = ht[i];
    if (threadIdx.x == 0) heavy[kHeavySlots] = nh < kHeavyMax ? nh : kHeavyMax;
}

// Sum of v over the lanes of the warp that hold the same key (key < 0: no
// value); the lowest such lane receives the sum, the others 0.  Every lane of
// the warp calls this.  v < 2^35: the parts summed in 32 bits cannot overflow.
__device__ __forceinline__ unsigned long long warp_key_sum(int key, unsigned long long v) {
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const unsigned lo = __reduce_add_sync(peers, (unsigned)(v & 0xFFFFu));
    const unsigned mid = __reduce_add_sync(peers, (unsigned)((v >> 16) & 0xFFFFu));
    const unsigned hi = __reduce_add_sync(peers, (unsigned)(v >> 32));
    if ((threadIdx.x & 31) != (unsigned)(__ffs(peers) - 1)) return 0;
    return (unsigned long long)lo + ((unsigned long long)mid << 16) + ((unsigned long long)hi << 32);
}

// S's heavy bucket: hw[slot of h] += deg_T(c).  Most tuples of this bucket
// share a few keys, so each warp first adds up its lanes' values per key;
// per-CTA shared sums; one global add per key and CTA.
__global__ void __launch_bounds__(HT) k_heavy_s(const uint2 *__restrict__ Sp, const uint32_t *__restrict__ offS,
                                                uint32_t hb, const uint32_t *__restrict__ heavy, TImg T,
                                                unsigned long long *__restrict__ hw) {
    __shared__ uint32_t hbuf[kHeavySlots];
    __shared__ unsigned long long acc[kHeavySlots];
    const uint32_t *hs = heavy_to_smem(heavy, hbuf);
    if (!hs) return;
    for (uint32_t i = threadIdx.x; i < kHeavySlots; i += HT) acc[i] = 0;
    __syncthreads();
    const uint32_t s0 = offS[hb], s1 = offS[hb + 1];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * HT + threadIdx.x) >> 5, warps = gridDim.x * (HT / 32);
    const uint32_t tmask = (T.J == 0) ? __ldg(T.meta) : 0u;
    // warp-uniform loop: a warp takes 128 consecutive tuples, 4 per lane
    for (uint64_t base = (uint64_t)s0 + (uint64_t)warp * 128; base < s1; base += (uint64_t)warps * 128) {
        const uint32_t i0 = (uint32_t)base + lane * 4;
        uint2 t[4];
        int h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            t[q] = i0 + q < s1 ? __ldg(Sp + i0 + q) : make_uint2(kEmptyKey, 0u);
            h[q] = heavy_slot(hs, t[q].x);
        }
        // deg_T(c): with T's single table the first probes of the four
        // tuples are all in flight before any is resolved
        uint32_t d[4];
        if (T.J == 0) {
            uint32_t sl[4];
            unsigned long long v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (h[q] >= 0) {
                    sl[q] = slot_of(t[q].y, T.seed_slot, tmask);
                    v[q] = __ldg((const unsigned long long *)(T.img + sl[q]));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                d[q] = 0;
                if (h[q] < 0) continue;
                unsigned long long x = v[q];
                uint32_t p = sl[q];
                for (uint32_t it = 0; it < tmask && x != kEmpty64 && (uint32_t)x != t[q].y; ++it) {
                    p = (p + 1) & tmask;
                    x = __ldg((const unsigned long long *)(T.img + p));
                }
                if (x != kEmpty64 && (uint32_t)x == t[q].y) d[q] = (uint32_t)(x >> 32);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = h[q] >= 0 ? timg_deg(T, (int32_t)t[q].y) : 0u;
        }
        // the lane's runs of equal keys first (at most 4 values), then per
        // key across the warp
        int key[4];
        unsigned long long val[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            key[q] = d[q] ? h[q] : -1;
            val[q] = d[q];
        }
#pragma unroll
        for (int q = 3; q > 0; --q) {
            if (key[q] >= 0 && key[q] == key[q - 1]) {
                val[q - 1] += val[q];
                key[q] = -1;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned long long sum = warp_key_sum(key[q], key[q] >= 0 ? val[q] : 0ull);
            if (sum) atomicAdd(&acc[key[q]], sum);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kHeavySlots; i += HT)
        if (acc[i]) atomicAdd(hw + i, acc[i]);
}

// R's heavy bucket: total += hw[slot of h] and (GROUP BY A) cnt[a] +=
// hw[slot of h] for every (a, h); runs of equal a merged.
template <int MODE>
__global__ void __launch_bounds__(HT) k_heavy_r(const uint2 *__restrict__ Rp, const uint32_t *__restrict__ offR,
                                                uint32_t hb, const uint32_t *__restrict__ heavy,
                                                const unsigned long long *__restrict__ hw, int32_t a_domain,
                                                unsigned long long *__restrict__ cnt,
                                                unsigned long long *__restrict__ total) {
    __shared__ uint32_t hbuf[kHeavySlots];
    __shared__ unsigned long long w[kHeavySlots];
    __shared__ unsigned long long red[32];
    const uint32_t *hs = heavy_to_smem(heavy, hbuf);
    if (!hs) return;
    for (uint32_t i = threadIdx.x; i < kHeavySlots; i += HT) w[i] = __ldcg(hw + i);
    __syncthreads();
    const uint32_t r0 = offR[hb], r1 = offR[hb + 1];
    const uint32_t stride = gridDim.x * HT * 4;
    unsigned long long tot = 0;
    for (uint32_t i0 = r0 + (blockIdx.x * HT + threadIdx.x) * 4; i0 < r1; i0 += stride) {
        int32_t cur = 0;
        unsigned long long run = 0;
        bool have = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (i0 + q >= r1) break;
            const uint2 t = __ldg(Rp + i0 + q);
            const int h = heavy_slot(hs, t.y);
            if (h < 0) continue;
            const unsigned long long v = w[h];
            if (!v) continue;
            if (MODE == 1) {
                if ((uint32_t)t.x >= (uint32_t)a_domain) continue;   // reported by the partitioner
                if (have && (int32_t)t.x == cur) {
                    run += v;
                } else {
                    if (have) atomicAdd(cnt + cur, run);
                    cur = (int32_t)t.x;
                    run = v;
                    have = true;
                }
            }
            tot += v;
        }
        if (MODE == 1 && have) atomicAdd(cnt + cur, run);
    }
    tot = block_sum_u64(tot, red);
    if (threadIdx.x == 0 && tot) atomicAdd(total, tot);
}

}  // namespace

cudaError_t heavy_detect(const int32_t *rb, int64_t nR, const int32_t *sb, int64_t nS, uint32_t I,
                         uint32_t *heavy, unsigned long long *hw, cudaStream_t st) {
    const size_t smem = (2 * (size_t)kCountSlots + kHeavySlots) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_heavy_detect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ProfScope ps_("heavy_detect", st);
    k_heavy_detect<<<1, DT, smem, st>>>(rb, (uint32_t)nR, sb, (uint32_t)nS, I ? I : 1u, heavy, hw);
    return cudaGetLastError();
}

cudaError_t heavy_linear(const uint2 *Sp, const uint32_t *offS, uint32_t hbS, const uint2 *Rp,
                         const uint32_t *offR, uint32_t hbR, const uint32_t *heavy, const TImg &T,
                         unsigned long long *hw, int32_t a_domain, unsigned long long *cnt,
                         unsigned long long *total, int num_sms, cudaStream_t st) {
    const unsigned grid = (unsigned)num_sms * 2;
    {
        ProfScope ps_("heavy_s", st);
        k_heavy_s<<<grid, HT, 0, st>>>(Sp, offS, hbS, heavy, T, hw);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ProfScope ps_("heavy_r", st);
    if (cnt)
        k_heavy_r<1><<<grid, HT, 0, st>>>(Rp, offR, hbR, heavy, hw, a_domain, cnt, total);
    else
        k_heavy_r<0><<<grid, HT, 0, st>>>(Rp, offR, hbR, heavy, hw, a_domain, cnt, total);
    return cudaGetLastError();
}

}  // namespace mwj
