// Device helpers shared by the library's kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define BL_DEV __device__ __forceinline__

// Device-side error flags (bit mask) raised by bounded waits into a word the
// host passes to the kernel; read and cleared by bl_poll_device_errors.
enum : unsigned { BL_DEVERR_MMA_TIMEOUT = 1u, BL_DEVERR_TMA_TIMEOUT = 2u, BL_DEVERR_BARRIER_TIMEOUT = 4u };

// ---------------------------------------------------------------------------
// Float-float accumulation. A sum is held as an unevaluated pair hi + lo of
// FP32 numbers; TwoSum (Knuth) makes each addition exact up to the rounding
// of lo, and TwoProd (an fma residual) makes each product of two FP32 values
// exact. The relative error of a float-float accumulation is about 2^-44,
// enough for FP64-quality second moments without per-particle FP64 work.
// The additions and the product are written with the _rn intrinsics, which
// the compiler never contracts into an fma: a contracted hi + a*b would
// round the exact product away and break the error-free transformations.
BL_DEV void ff_add(float &hi, float &lo, float p) {
  const float s = __fadd_rn(hi, p);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

BL_DEV void ff_add_prod(float &hi, float &lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// Raw moment sums of one particle: 6 coordinates and their 21 products
// (a <= b, row-major), in float-float (FP32 particles) or FP64 (FP64 particles).
struct MomAccF {
  float hi[27];
  float lo[27];
  BL_DEV void zero() {
#pragma unroll
    for (int i = 0; i < 27; ++i) { hi[i] = 0.f; lo[i] = 0.f; }
  }
  BL_DEV void add(const float z[6]) {
#pragma unroll
    for (int a = 0; a < 6; ++a) ff_add(hi[a], lo[a], z[a]);
    int j = 6;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = a; b < 6; ++b) { ff_add_prod(hi[j], lo[j], z[a], z[b]); ++j; }
  }
  BL_DEV double get(int i) const { return (double)hi[i] + (double)lo[i]; }
};

struct MomAccD {
  double s[27];
  BL_DEV void zero() {
#pragma unroll
    for (int i = 0; i < 27; ++i) s[i] = 0.0;
  }
  BL_DEV void add(const double z[6]) {
#pragma unroll
    for (int a = 0; a < 6; ++a) s[a] += z[a];
    int j = 6;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = a; b < 6; ++b) { s[j] = fma(z[a], z[b], s[j]); ++j; }
  }
  BL_DEV double get(int i) const { return s[i]; }
};

template <typename T> struct MomAccOf;
template <> struct MomAccOf<float> { using type = MomAccF; };
template <> struct MomAccOf<double> { using type = MomAccD; };

BL_DEV double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NV doubles per thread; the result is valid in thread 0.
// smem must hold (blockDim.x/32) * NV doubles. Contains __syncthreads.
template <int NV>
BL_DEV void block_sum(double (&v)[NV], double *smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) smem[warp * NV + i] = v[i];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = lane < nw ? smem[lane * NV + i] : 0.0;
      v[i] = warp_sum(s);
    }
  }
}

// Bunch that contains particle p: largest b with offsets[b] <= p (offsets has
// n_bunch+1 entries, offsets[n_bunch] = n). NULL offsets mean one bunch.
BL_DEV int find_bunch(const int64_t *offsets, int n_bunch, int64_t p) {
  if (offsets == nullptr) return 0;
  int lo = 0, hi = n_bunch;  // invariant: offsets[lo] <= p < offsets[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(offsets + mid) <= p) lo = mid; else hi = mid;
  }
  return lo;
}

BL_DEV int64_t bunch_begin(const int64_t *offsets, int b) { return offsets ? __ldg(offsets + b) : 0; }
BL_DEV int64_t bunch_end(const int64_t *offsets, int b, int64_t n) { return offsets ? __ldg(offsets + b + 1) : n; }

template <typename T> BL_DEV bool finite6(const T z[6]) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 6; ++i) ok = ok && isfinite(z[i]);
  return ok;
}
