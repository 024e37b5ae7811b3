// cascade.cu -- the cascade of binary hash joins (Section 6.3).
#include "api_internal.h"

namespace mwj {

mwj_status cascade_workspace(mwj_ctx *ctx, int, const mwj_rel &, const mwj_rel &, const mwj_rel &,
                             mwj_mode, size_t *bytes) {
    *bytes = 0;
    return fail(ctx, MWJ_ERR_UNIMPLEMENTED, "cascade not built yet");
}

}  // namespace mwj

extern "C" mwj_status mwj_cascade_join(mwj_ctx *ctx, int, mwj_rel, mwj_rel, mwj_rel,
                                       const mwj_out *, void *, size_t, void *) {
    return mwj::fail(ctx, MWJ_ERR_UNIMPLEMENTED, "cascade not built yet");
}
