// noalloc.cu -- the linear 3-way join (COUNT / GROUP BY A) for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another runtime's
// memory pool or allocator hook, plug-ins loaded into a host process that
// owns all device allocations, or real-time paths where an allocation could
// block or fail at an unpredictable moment.  mwj_join3_linear_noalloc serves
// them: it needs neither a context (whose creation allocates a status word)
// nor a caller workspace.  Its scratch memory is one file-scope device array
// of kNoAllocBytes that the library image carries, so every GPU that loads
// the library holds that array until the process exits.
//
// Because all calls share the one array (and one status word), two calls
// whose work overlaps on the GPU -- on different streams, or from different
// host threads -- race and corrupt each other's results; callers must order
// them.  Every piece of scratch that has to start at zero is cleared by the
// call itself, so the contents a previous call left behind never matter.
//
// The first call on each device looks up the device addresses of the array
// and of the status word (cudaGetSymbolAddress, with that device current);
// make that first call before capturing the stream into a CUDA graph.  The
// addresses are kept until the process exits; cudaDeviceReset on a device
// reloads the library's device image elsewhere, so the entry point must not
// be called on that device after a reset.  The host never passes the
// array's name to a kernel: in host code that name is a stand-in, not a
// device address.
#include <mutex>

#include "api_internal.h"
#include "linear.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr int64_t kNoAllocMaxTuples = 1 << 18;     // per relation
constexpr uint32_t kNoAllocMaxBuckets = 1024;       // I * J
constexpr size_t kNoAllocBytes = 24u << 20;         // 24 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static __device__ __align__(256) DevStatus g_noalloc_status;

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch
    DevStatus *status = nullptr;        // device address of g_noalloc_status
    int num_sms = 0;
};

constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

mwj_status setup_device(int dev, DeviceSetup *out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MWJ_ERR_CUDA;
        s.scratch = (unsigned char *)p;
        p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_status) != cudaSuccess || !p) return MWJ_ERR_CUDA;
        s.status = (DevStatus *)p;
        if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return MWJ_ERR_CUDA;
        s.ready = true;
    }
    *out = s;
    return MWJ_OK;
}

}  // namespace
}  // namespace mwj

using namespace mwj;

extern "C" mwj_status mwj_join3_linear_noalloc(mwj_rel R, mwj_rel S, mwj_rel T,
                                               const mwj_shares *shares, const mwj_out *out,
                                               void *stream) {
    // ---- arguments (nothing touches the GPU before these pass) ----
    if (!out || !out->total) return MWJ_ERR_INVALID_ARG;
    if (out->mode != MWJ_COUNT && out->mode != MWJ_COUNT_GROUP_BY_A) return MWJ_ERR_INVALID_ARG;
    if (out->mode == MWJ_COUNT_GROUP_BY_A && (!out->group_counts || out->a_domain <= 0))
        return MWJ_ERR_INVALID_ARG;
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return MWJ_ERR_INVALID_ARG;
    if (R.n > kNoAllocMaxTuples || S.n > kNoAllocMaxTuples || T.n > kNoAllocMaxTuples)
        return MWJ_ERR_WORKSPACE;   // beyond the fixed scratch: use mwj_join3_linear
    uint32_t I = 0, J = 1;
    if (shares) {
        if (shares->s[0] < 1 || shares->s[1] < 1) return MWJ_ERR_INVALID_ARG;
        if ((uint64_t)shares->s[0] * (uint64_t)shares->s[1] > kNoAllocMaxBuckets)
            return MWJ_ERR_WORKSPACE;
        I = (uint32_t)shares->s[0];
        J = (uint32_t)shares->s[1];
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MWJ_ERR_CUDA;
    DeviceSetup ds;
    mwj_status s = setup_device(dev, &ds);
    if (s != MWJ_OK) return s;
    if (I == 0) {   // default: ~16K R tuples per bucket, at least one bucket per SM
        uint64_t want = (uint64_t)(R.n + 16383) / 16384;
        if (want < (uint64_t)ds.num_sms) want = (uint64_t)ds.num_sms;
        I = pow2_at_least(want);
        if (I > kNoAllocMaxBuckets) I = kNoAllocMaxBuckets;
    }

    // ---- layout inside the fixed array ----
    uint64_t want_t = (uint64_t)(T.n + 8191) / 8192;
    const uint32_t JT = (J > 1) ? J : pow2_at_least(want_t ? want_t : 1);
    const bool single = (J == 1);
    Arena A(ds.scratch, kNoAllocBytes);
    uint2 *Rp = A.take<uint2>(R.n + 2);
    uint32_t *offR = A.take<uint32_t>(I + 1);
    uint2 *Sp = A.take<uint2>(S.n + 2);
    uint32_t *offS = A.take<uint32_t>((size_t)I * J + 1);
    uint32_t *Tk = A.take<uint32_t>(T.n + 4);
    uint32_t *offT = A.take<uint32_t>(JT + 1);
    uint64_t *img = single ? A.take<uint64_t>(single_table_slots(T.n)) : A.take<uint64_t>(2 * (size_t)T.n + 4);
    uint32_t *capT = single ? nullptr : A.take<uint32_t>(JT + 1);
    uint32_t *ekey = single ? A.take<uint32_t>(T.n + 4) : nullptr;
    uint32_t *ecnt = single ? A.take<uint32_t>(T.n + 4) : nullptr;
    uint32_t *ecount = single ? A.take<uint32_t>(JT + 1) : nullptr;
    uint32_t *meta = single ? A.take<uint32_t>(4) : nullptr;
    size_t psb = part_scratch_bytes(R.n, I, ds.num_sms);
    size_t ps2 = part_scratch_bytes(S.n, I * J, ds.num_sms);
    size_t ps3 = part_scratch_bytes(T.n, JT, ds.num_sms);
    if (ps2 > psb) psb = ps2;
    if (ps3 > psb) psb = ps3;
    void *pscratch = A.take<char>(psb);
    if (A.overflow) return MWJ_ERR_WORKSPACE;

    // ---- the join (same kernels as mwj_join3_linear) ----
    cudaStream_t st = (cudaStream_t)stream;
    ApiScope no_profiler(nullptr);
    const Seeds sd = make_seeds(0);
    if (cudaMemsetAsync(ds.status, 0, sizeof(DevStatus), st) != cudaSuccess) return MWJ_ERR_CUDA;
    if (cudaMemsetAsync(out->total, 0, sizeof(int64_t), st) != cudaSuccess) return MWJ_ERR_CUDA;
    if (out->mode == MWJ_COUNT_GROUP_BY_A &&
        cudaMemsetAsync(out->group_counts, 0, sizeof(int64_t) * (size_t)out->a_domain, st) != cudaSuccess)
        return MWJ_ERR_CUDA;
    PartSpec pt{0, sd.C, JT, -1, 0, 1};
    pt.st = ds.status;
    if (part_run(T.x, T.y, T.n, pt, PAY_X, Tk, offT, pscratch, psb, ds.num_sms, st) != cudaSuccess)
        return MWJ_ERR_CUDA;
    PartSpec pS{0, sd.B, I, J > 1 ? 1 : -1, sd.C, J};
    pS.st = ds.status;
    if (part_run(S.x, S.y, S.n, pS, PAY_PAIR, Sp, offS, pscratch, psb, ds.num_sms, st) != cudaSuccess)
        return MWJ_ERR_CUDA;
    PartSpec pr{1, sd.B, I, -1, 0, 1};
    pr.st = ds.status;
    if (out->mode == MWJ_COUNT_GROUP_BY_A) pr.dom = (uint32_t)out->a_domain;
    if (part_run(R.x, R.y, R.n, pr, PAY_PAIR, Rp, offR, pscratch, psb, ds.num_sms, st) != cudaSuccess)
        return MWJ_ERR_CUDA;
    cudaError_t e = single ? single_table_build(Tk, offT, JT, sd.slot2, ekey, ecnt, ecount, meta, img,
                                                ds.status, ds.num_sms, st)
                           : tables_build(Tk, nullptr, offT, JT, sd.slot2, img, capT, nullptr, nullptr,
                                          ds.status, ds.num_sms, st);
    if (e != cudaSuccess) return MWJ_ERR_CUDA;
    LinArgs g{};
    g.Rp = Rp; g.offR = offR; g.Sp = Sp; g.offS = offS; g.I = I; g.JS = J;
    g.t = single ? TImg{img, nullptr, nullptr, nullptr, nullptr, meta, 0u, sd.C, sd.slot2}
                 : TImg{img, offT, capT, nullptr, nullptr, nullptr, JT, sd.C, sd.slot2};
    g.cap_log2 = 12;
    g.seed_slot = sd.slot;
    g.a_domain = out->a_domain;
    g.cnt = (unsigned long long *)out->group_counts;
    g.total = (unsigned long long *)out->total;
    g.rowcount = nullptr;
    g.st = ds.status;
    g.spin_limit = 1u << 24;
    g.build_s = lin_build_s(R.n, S.n);
    if (lin_agg_launch(g, out->mode == MWJ_COUNT_GROUP_BY_A ? 1 : 0, st) != cudaSuccess)
        return MWJ_ERR_CUDA;

    // ---- device-side errors: wait for the stream and read the status word ----
    DevStatus h{};
    if (cudaMemcpyAsync(&h, ds.status, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return MWJ_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MWJ_ERR_CUDA;
    return h.code == 0 ? MWJ_OK : (mwj_status)h.code;
}
