// Split-precision engine (BF16 slices on tcgen05 tensor cores).
#include "jk_internal.h"

namespace jk {

size_t split_build_workspace(const Problem &) { return 0; }
size_t split_adjoint_workspace(const Problem &, bool) { return 0; }

jk_status split_build(jk_ctx *h, const Problem &, cudaStream_t) {
    return set_error(h, JK_ERR_UNSUPPORTED, "split-precision build not built yet");
}

jk_status split_adjoint(jk_ctx *h, const Problem &, const double *, const double *,
                        double *, double *, double *, cudaStream_t) {
    return set_error(h, JK_ERR_UNSUPPORTED, "split-precision adjoint not built yet");
}

}  // namespace jk
