/*
 * bl_debug.h -- diagnostic entry points of libbl.so (not part of the tracking
 * API). The paper has no counterpart; they inject host-side failures for
 * the library's error-path tests, select the training kernel and expose the
 * host-side pooling of chunked moments.
 */
#ifndef BL_DEBUG_H
#define BL_DEBUG_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

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
