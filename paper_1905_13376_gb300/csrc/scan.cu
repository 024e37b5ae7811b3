// scan.cu -- exclusive prefix sums (bucket offsets, output positions).
//
// Three launches, no inter-CTA waiting: per-tile totals, one CTA scanning the
// tile totals, per-tile scan plus the tile's base.
#include "internal.h"

namespace mwj {
namespace {

constexpr int SC_THREADS = 512;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

template <typename T>
__global__ void k_tile_sums(const T *in, size_t n, T *sums) {
    size_t base = (size_t)blockIdx.x * SC_TILE;
    T s = 0;
    for (int k = 0; k < SC_ITEMS; ++k) {
        size_t i = base + (size_t)k * SC_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    __shared__ unsigned long long red[32];
    unsigned long long t = block_sum_u64((unsigned long long)s, red);
    if (threadIdx.x == 0) sums[blockIdx.x] = (T)t;
}

// One CTA: exclusive scan of the tile totals, in place.
template <typename T>
__global__ void k_scan_sums(T *sums, size_t m) {
    __shared__ unsigned long long carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (size_t base = 0; base < m; base += SC_THREADS) {
        size_t i = base + threadIdx.x;
        T v = (i < m) ? sums[i] : (T)0;
        unsigned long long x = (unsigned long long)v;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ unsigned long long wt[32];
        if (lane == 31) wt[w] = x;
        __syncthreads();
        if (w == 0) {
            unsigned long long s = (lane < (SC_THREADS >> 5)) ? wt[lane] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wt[lane] = s;
        }
        __syncthreads();
        unsigned long long wb = (w > 0) ? wt[w - 1] : 0ull;
        unsigned long long excl = carry_s + wb + x - (unsigned long long)v;
        if (i < m) sums[i] = (T)excl;
        __syncthreads();
        if (threadIdx.x == SC_THREADS - 1) carry_s = excl + (unsigned long long)v;
        __syncthreads();
    }
}

template <typename T>
__global__ void k_tile_scan(const T *in, T *out, size_t n, const T *sums, bool with_total) {
    size_t base = (size_t)blockIdx.x * SC_TILE + (size_t)threadIdx.x * SC_ITEMS;
    T v[SC_ITEMS];
    T local = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        size_t i = base + k;
        v[k] = (i < n) ? in[i] : (T)0;
        local += v[k];
    }
    // block exclusive scan of `local` in 64-bit
    unsigned long long x = (unsigned long long)local;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __shared__ unsigned long long wt[32];
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = (lane < (SC_THREADS >> 5)) ? wt[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wt[lane] = s;
    }
    __syncthreads();
    unsigned long long wb = (w > 0) ? wt[w - 1] : 0ull;
    T run = (T)((unsigned long long)sums[blockIdx.x] + wb + x - (unsigned long long)local);
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        size_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (with_total && base < n && base + SC_ITEMS >= n) out[n] = run;
}

template <typename T>
cudaError_t scan_impl(const T *in, T *out, size_t n, bool with_total, void *scratch,
                      cudaStream_t st) {
    if (n == 0) {
        if (with_total) return cudaMemsetAsync(out, 0, sizeof(T), st);
        return cudaSuccess;
    }
    size_t tiles = (n + SC_TILE - 1) / SC_TILE;
    T *sums = (T *)scratch;
    {
        ProfScope ps_("scan_tile_sums", st);
        k_tile_sums<T><<<(unsigned)tiles, SC_THREADS, 0, st>>>(in, n, sums);
    }
    {
        ProfScope ps_("scan_sums", st);
        k_scan_sums<T><<<1, SC_THREADS, 0, st>>>(sums, tiles);
    }
    {
        ProfScope ps_("scan_tiles", st);
        k_tile_scan<T><<<(unsigned)tiles, SC_THREADS, 0, st>>>(in, out, n, sums, with_total);
    }
    return cudaGetLastError();
}

}  // namespace

size_t scan_scratch_bytes(size_t n) {
    size_t tiles = (n + SC_TILE - 1) / SC_TILE + 1;
    return align256(tiles * sizeof(uint64_t));
}

cudaError_t scan_excl_u32(uint32_t *data, size_t n, void *scratch, cudaStream_t st) {
    return scan_impl<uint32_t>(data, data, n, false, scratch, st);
}

cudaError_t scan_excl_u64(const uint64_t *in, uint64_t *out, size_t n, bool with_total,
                          void *scratch, cudaStream_t st) {
    return scan_impl<uint64_t>(in, out, n, with_total, scratch, st);
}

}  // namespace mwj
