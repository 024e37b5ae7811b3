// internal.h -- host-side launchers shared by the translation units of libmwj.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mwj {

// ---- partitioning (Algorithm 1's partition steps; Fig. 2 and Fig. 3) -------
// bucket(t) = fastrange(mix32(key1 ^ seed1), P1) * P2 + fastrange(mix32(key2 ^ seed2), P2)
// where key1/key2 are column col1/col2 (0 = x, 1 = y) of tuple t; col2 < 0
// means a single level (P2 = 1).
// With a heavy-key table (`heavy`, see skew.h), a tuple whose col1 value is a
// heavy key goes to one extra bucket after the hashed ones (index Pbase()).
struct PartSpec {
    int col1;
    uint32_t seed1, P1;
    int col2;
    uint32_t seed2, P2;
    uint32_t dom = 0;     // when > 0: every x must lie in [0, dom), else MWJ_ERR_DOMAIN
    DevStatus *st = nullptr;
    const uint32_t *heavy = nullptr;   // device heavy-key table, or null
    __host__ __device__ uint32_t Pbase() const { return P1 * (col2 >= 0 ? P2 : 1u); }
    __host__ __device__ uint32_t P() const { return Pbase() + (heavy ? 1u : 0u); }
};

enum Payload { PAY_PAIR = 0, PAY_X = 1, PAY_Y = 2 };

constexpr uint32_t kMaxBuckets = 32768;

// Scratch bytes for partitioning n tuples into P buckets.
size_t part_scratch_bytes(int64_t n, uint32_t P, int num_sms);

// Partition (x,y)[0,n) into `out` (uint2 pairs for PAY_PAIR, uint32 for
// PAY_X/PAY_Y) grouped by bucket; bucket_off[0..P] receives the offsets.
// Returns a cudaError_t of the launches.
// With z != null the pairs (x,y) carry a third column z, written to outz in
// the same order (PAY_PAIR only).
cudaError_t part_run(const int32_t *x, const int32_t *y, int64_t n, const PartSpec &spec,
                     int payload, void *out, uint32_t *bucket_off, void *scratch,
                     size_t scratch_bytes, int num_sms, cudaStream_t st,
                     const int32_t *z = nullptr, int32_t *outz = nullptr);

// ---- scans --------------------------------------------------------------
size_t scan_scratch_bytes(size_t n);
// In-place exclusive scan of n uint32 values.
cudaError_t scan_excl_u32(uint32_t *data, size_t n, void *scratch, cudaStream_t st);
// Exclusive scan of n uint64 values from `in` into `out` (may alias); out[n]
// receives the total when `with_total`.
cudaError_t scan_excl_u64(const uint64_t *in, uint64_t *out, size_t n, bool with_total,
                          void *scratch, cudaStream_t st);

// ---- device properties cached per context ---------------------------------
struct DevInfo {
    int device;
    int num_sms;
    int smem_optin;   // max dynamic shared memory per block (opt-in)
    int cc_major, cc_minor;
};

// Round up to a multiple of 256 bytes.
__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Bump allocator over a caller workspace.
struct Arena {
    char *base;
    size_t cap, used;
    bool overflow;
    Arena(void *b, size_t c) : base((char *)b), cap(c), used(0), overflow(false) {}
    template <typename T>
    T *take(size_t count) {
        size_t bytes = align256(count * sizeof(T) + 16);
        if (used + bytes > cap) {
            overflow = true;
            used += bytes;
            return nullptr;
        }
        T *p = (T *)(base ? base + used : nullptr);
        used += bytes;
        return p;
    }
};

}  // namespace mwj

// ---- launch accounting and optional per-kernel timing ----------------------
// Every kernel launch of the library sits inside a ProfScope.  The scope
// always counts the launch; when profiling is enabled on the calling
// context it also records a CUDA event pair on the launch stream, resolved
// later by mwj_get_phase_times().
namespace mwj {

struct Profiler;
Profiler *current_profiler();
void set_current_profiler(Profiler *p);

struct ProfScope {
    Profiler *p;
    int slot;
    ProfScope(const char *name, cudaStream_t st);
    ~ProfScope();
    cudaStream_t st;
};

}  // namespace mwj
