// cyclic.cu -- the cyclic 3-way join R(A,B) S(B,C) T(C,A) (Section 5).
#include "api_internal.h"

namespace mwj {

mwj_status plan_cyclic_default(mwj_ctx *ctx, const mwj_rel &, const mwj_rel &, const mwj_rel &,
                               mwj_shares *sh) {
    sh->s[0] = sh->s[1] = sh->s[2] = 1;
    return fail(ctx, MWJ_ERR_UNIMPLEMENTED, "cyclic join not built yet");
}

mwj_status cyc_workspace(mwj_ctx *ctx, const mwj_rel &, const mwj_rel &, const mwj_rel &,
                         const mwj_shares *, mwj_mode, size_t *bytes) {
    *bytes = 0;
    return fail(ctx, MWJ_ERR_UNIMPLEMENTED, "cyclic join not built yet");
}

}  // namespace mwj

extern "C" mwj_status mwj_join3_cyclic(mwj_ctx *ctx, mwj_rel, mwj_rel, mwj_rel, const mwj_shares *,
                                       const mwj_out *, void *, size_t, void *) {
    return mwj::fail(ctx, MWJ_ERR_UNIMPLEMENTED, "cyclic join not built yet");
}
