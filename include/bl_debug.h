/*
 * bl_debug.h -- diagnostic entry points of libbl.so (not part of the tracking
 * API). The paper has no counterpart; they check the tensor-core operand
 * layouts that the surrogate kernel relies on, inject host-side failures for
 * the library's error-path tests, select the training kernel and expose the
 * host-side pooling of chunked moments.
 */
#ifndef BL_DEBUG_H
#define BL_DEBUG_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* One tcgen05 MMA D = A * B^T on the current device.
 * A: device, 128 x K BF16 row-major (placed in tensor memory, two values per
 * 32-bit column); B: device, N x K BF16 row-major, staged into shared memory
 * as 8x8 core matrices of 128 bytes, adjacent core matrices `ks` bytes apart
 * along K and `ns` bytes apart along N; the shared-memory descriptor gets
 * leading offset `lbo` and stride offset `sbo`. D: device, 128 x N FP32
 * row-major. N in {16,32,64,128}, K in {16,32,64,128}, 128 <= ks, ns <= 2048,
 * multiples of 16. Returns 0 on launch success, 1 for invalid sizes, 2 for a
 * launch error. Asynchronous on `stream` (a cudaStream_t). */
int bl_debug_umma_probe(const void *A, const void *B, float *D, int N, int K, uint32_t ks,
                        uint32_t ns, uint32_t lbo, uint32_t sbo, void *stream);

/* Host-side fault injection for failure-path tests: the next n workspace
 * allocations of the library fail with BL_ERR_OOM before reaching the
 * allocator (no device fault is involved). n = 0 turns it off. Returns 0. */
int bl_debug_fail_allocations(int n);

/* The FP64 pooling that bl_track_host applies to chunked moment reductions:
 * parts holds k moment vectors of disjoint particle sets, 28 doubles each
 * ([N, 6 means, 21 central second moments with 1/N], host); out (host, 28
 * doubles) receives the moments of their union: counts add, means pool with
 * weights N_c, and each central moment gains (mu_c - mu)(mu_c - mu)^T. Sets
 * with N_c = 0 contribute nothing. Host computation, no GPU involved.
 * Returns 0, or 1 for a NULL pointer or k < 1. */
int bl_debug_pool_moments(const double *parts, int32_t k, double *out);

/* Selects the kernel behind bl_surrogate_train_step and bl_surrogate_grad:
 * simt = 0 (the default) the tensor-core kernel (BF16 operands, FP32
 * accumulation, one partial row per 128-sample tile); simt != 0 the SIMT FP32
 * kernel, kept as an independent second evaluation of the same gradient for
 * cross-checks. Host-side switch for the whole process; call it with no
 * training call in flight. Returns the previous setting (0 or 1). */
int bl_debug_train_kernel(int simt);

#ifdef __cplusplus
}
#endif
#endif
