// waitcheck.cu -- a bounded device wait that is made to run out.
//
// Every wait of the library's kernels is a poll of an mbarrier phase with an
// iteration limit; when the limit is reached the CTA records MWJ_ERR_TIMEOUT
// in the context's status word, waits (bounded) for its own copies still in
// flight and returns, so that the context stays usable.  In the joins the
// phases always complete (they count bytes of copies that land), so this
// entry point exercises the give-up path on purpose: one CTA arms a
// barrier for a transfer that is never issued and waits on it.
#include "api_internal.h"

namespace mwj {
namespace {

__global__ void k_wait_nothing(uint32_t polls, DevStatus *st) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_barrier_init();
    mbar_expect_tx(&bar, 16);   // 16 bytes that no copy will deliver
    if (!mbar_wait_bounded(&bar, 0u, polls)) set_status(st, MWJ_ERR_TIMEOUT, -1);
}

}  // namespace
}  // namespace mwj

using namespace mwj;

extern "C" mwj_status mwj_check_bounded_wait(mwj_ctx *ctx, int64_t polls, void *stream) {
    if (!ctx || polls < 1 || polls > (1ll << 24)) return MWJ_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ProfScope ps_("wait_check", st);
    k_wait_nothing<<<1, 32, 0, st>>>((uint32_t)polls, ctx->status);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MWJ_OK : cuda_fail(ctx, e, "wait check");
}
