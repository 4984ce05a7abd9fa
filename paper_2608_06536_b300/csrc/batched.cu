// Batched builds over many independent molecules (uneven nbf, naux, nd).
// Split precision: grouped persistent GEMM launches over all molecules (split.cu).
// FP64: molecules one after another on the caller's stream.
#include "jk_internal.h"

namespace jk {

jk_status batched_build(jk_ctx *h, int nmol, const Problem *pbs, jk_precision p,
                        cudaStream_t st) {
    if (p == JK_SPLIT_BF16) {
        // All molecules' panels and rank updates as grouped persistent launches.
        h->arena.reset(align_up(sizeof(DeviceFlags)));
        return split_batched(h, nmol, pbs, st);
    }
    for (int m = 0; m < nmol; m++) {
        h->arena.reset(align_up(sizeof(DeviceFlags)));
        if (p == JK_FP64) {
            JK_TRY(fp64_build(h, pbs[m], st));
        } else {
            JK_TRY(split_build(h, pbs[m], st));
        }
    }
    return JK_OK;
}

}  // namespace jk
