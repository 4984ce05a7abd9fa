/*
 * jk_debug.h -- test hooks of libjk.so (not part of the J/K engine's API).
 *
 * They expose single building blocks of the split-precision engine so that
 * tests can check them in isolation against exact references.
 */
#ifndef JK_DEBUG_H
#define JK_DEBUG_H

#include "jk.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C[M][N] = A[M][K] * B[N][K]^T (all FP64, row-major, device) through the
 * split-precision path: each row of A and B is cut into six BF16 slices with
 * its own power-of-two scale, the 21 leading slice products run on tcgen05
 * tensor cores with exact FP32 accumulation windows, and the result is
 * recombined in integers and rounded once to FP64.  Uses the handle's arena
 * (size from jk_debug_sliced_gemm_workspace); JK_ERR_OOM if it is too small. */
jk_status jk_debug_sliced_gemm(jk_handle h, int32_t M, int32_t N, int32_t K,
                               const double *A, const double *B, double *C,
                               void *stream);
size_t jk_debug_sliced_gemm_workspace(int32_t M, int32_t N, int32_t K);

/* The same product with `slices` BF16 slices per operand: 6 (48-bit
 * fixed-point operands, 21 slice pairs) or 7 (56-bit operands, 28 slice
 * pairs, exact windows on one more diagonal, 128 x 64 tiles: the
 * configuration of the split adjoint).  JK_ERR_ARG for another count.  The
 * arena must hold jk_debug_sliced_gemm_workspace_slices(M, N, K, slices). */
jk_status jk_debug_sliced_gemm_slices(jk_handle h, int32_t M, int32_t N, int32_t K, const double *A,
                                      const double *B, double *C, int32_t slices, void *stream);
size_t jk_debug_sliced_gemm_workspace_slices(int32_t M, int32_t N, int32_t K, int32_t slices);

/* Exercises the engine's bounded waits: one thread waits on an mbarrier
 * phase that nothing completes, with the same helper and limit (4 s) the
 * tcgen05 pipeline uses; when the limit runs out it raises JK_ERR_TIMEOUT in
 * the handle's device status word and returns.  jk_sync_status(h, stream)
 * then reports JK_ERR_TIMEOUT and clears it; the CUDA context stays usable.
 * Nothing faults or hangs. */
jk_status jk_debug_wait_timeout(jk_handle h, void *stream);

/* Measures the device's FP64 FMA throughput, the ceiling of the plain FP64
 * engine and of the FP64 J kernels: one launch of blocks_per_sm x SMs blocks
 * of 256 threads, each thread running sixteen independent FMA chains for
 * `iters` steps (no memory traffic inside the loop).  *flops receives the
 * FP64 flops the launch performs (2 per FMA); time the launch on `stream`
 * with CUDA events.  sink: one device double the kernel may write (keeps the
 * chains live).  JK_ERR_ARG for a NULL handle, sink or flops pointer, or
 * blocks_per_sm or iters outside [1, 64] / [1, 2^24]. */
jk_status jk_debug_fp64_fma(jk_handle h, int32_t blocks_per_sm, int32_t iters, double *sink, double *flops,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif /* JK_DEBUG_H */
