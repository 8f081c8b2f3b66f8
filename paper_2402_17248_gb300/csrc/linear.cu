// Particle-streaming kernels: linear segment maps (Sec. 1: elements as
// per-particle transfer maps, here linear, fused over a run of consecutive
// elements), beam-moment reductions (Sec. 4: count, means and second
// moments), the adjoint seed and the transposed segment map with its
// cross-moment reduction.
//
// Work decomposition: block k owns particles [k*CHUNK, (k+1)*CHUNK). A block
// walks the bunches that intersect its range; for each (bunch b, block k)
// piece it reduces one partial into slot b + k, which is unique because both
// bunches and blocks tile the particle line contiguously. A finalize kernel
// per bunch sums the slots of the blocks its range touches, in FP64.
#include "common.cuh"
#include "internal.h"

namespace bl {

template <typename T> BL_DEV T ldg_(const T *p) { return __ldg(p); }

template <typename T, bool APPLY, bool MOMENTS>
__global__ void __launch_bounds__(STREAM_THREADS)
stream_kernel(Soa<T> zin, Soa<T> zout, int64_t n, const int64_t *__restrict__ offsets,
              int n_bunch, const T *__restrict__ mats, int per_bunch,
              const T *__restrict__ centers, double *__restrict__ partials) {
  using Acc = typename MomAccOf<T>::type;
  __shared__ int s_b0;
  __shared__ double s_red[(STREAM_THREADS / 32) * 28];
  const int64_t start = (int64_t)blockIdx.x * STREAM_CHUNK;
  const int64_t end = min(n, start + STREAM_CHUNK);
  if (threadIdx.x == 0) s_b0 = find_bunch(offsets, n_bunch, start);
  __syncthreads();
  int b = s_b0;
  int64_t lo = start;
  while (lo < end) {
    const int64_t hi = min(end, bunch_end(offsets, b, n));
    if (hi > lo) {
      T M[36], c[6];
      if (APPLY) {
        const T *Mb = mats + (per_bunch ? (int64_t)b * 36 : 0);
#pragma unroll
        for (int i = 0; i < 36; ++i) M[i] = ldg_(Mb + i);
#pragma unroll
        for (int i = 0; i < 6; ++i) c[i] = centers ? ldg_(centers + (int64_t)b * 6 + i) : T(0);
      }
      Acc acc;
      double nonfin = 0.0;
      if (MOMENTS) acc.zero();
#pragma unroll 4
      for (int64_t p = lo + threadIdx.x; p < hi; p += STREAM_THREADS) {
        T v[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] = zin.c[i][p];
        if (MOMENTS) {
          acc.add(v);
          nonfin += finite6(v) ? 0.0 : 1.0;
        }
        if (APPLY) {
#pragma unroll
          for (int i = 0; i < 6; ++i) v[i] -= c[i];
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            T s = T(0);
#pragma unroll
            for (int j = 0; j < 6; ++j) s = fma(M[i * 6 + j], v[j], s);
            zout.c[i][p] = s;
          }
        }
      }
      if (MOMENTS) {
        double r[28];
#pragma unroll
        for (int i = 0; i < 27; ++i) r[i] = acc.get(i);
        r[27] = nonfin;
        block_sum<28>(r, s_red);
        if (threadIdx.x == 0) {
          double *dst = partials + ((int64_t)b + blockIdx.x) * 28;
#pragma unroll
          for (int i = 0; i < 28; ++i) dst[i] = r[i];
        }
      }
    }
    lo = max(lo, hi);
    ++b;
    if (b >= n_bunch) break;
  }
}

// FP32 particles with moments: two warps share each group of 32 particles. The
// even warp of a pair accumulates sums 0..13 (6 linear sums, 8 products) and
// writes output rows 0..2; the odd warp accumulates sums 14..26 and writes
// rows 3..5. Splitting the 27 float-float accumulators this way halves the
// registers per thread, so more warps keep loads in flight. Roles are
// warp-uniform, so no lane diverges. Because the update is in place and each
// warp reads all six coordinates, the pair meets at a 64-thread named barrier
// between its loads and its stores.
template <int J0, int J1>
BL_DEV void mom_subset(float (&hi)[J1 - J0], float (&lo)[J1 - J0], const float (&v)[6]) {
#pragma unroll
  for (int a = 0; a < 6; ++a)
    if (a >= J0 && a < J1) ff_add(hi[a - J0], lo[a - J0], v[a]);
  int j = 6;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int b = a; b < 6; ++b) {
      if (j >= J0 && j < J1) ff_add_prod(hi[j - J0], lo[j - J0], v[a], v[b]);
      ++j;
    }
}

// One role's share of a (bunch, block) piece: accumulate, then reduce the
// role's sums across its warp; lane 0 leaves them in red[warp][0..13].
template <bool APPLY, int ROLE>
BL_DEV void mom_piece(Soa<float> &zin, Soa<float> &zout, int64_t lo_p, int64_t hi_p, int plane,
                      const float *__restrict__ Mb, const float *__restrict__ cb,
                      double (*red)[15]) {
  constexpr int J0 = ROLE ? 14 : 0, J1 = ROLE ? 27 : 14;
  float M[18], c[6], shi[J1 - J0], slo[J1 - J0];
  if (APPLY) {
#pragma unroll
    for (int i = 0; i < 18; ++i) M[i] = __ldg(Mb + 18 * ROLE + i);
#pragma unroll
    for (int i = 0; i < 6; ++i) c[i] = cb ? __ldg(cb + i) : 0.0f;
  }
#pragma unroll
  for (int i = 0; i < J1 - J0; ++i) { shi[i] = 0.f; slo[i] = 0.f; }
  float nf = 0.f;
  const int pair = threadIdx.x >> 6;
  const int64_t last = (hi_p - lo_p - 1) / (STREAM_THREADS / 2) * (STREAM_THREADS / 2);
  // every warp of the pair runs the same trip count (the tail is masked, not
  // skipped) so the pair barrier is always matched
#pragma unroll 2
  for (int64_t q = 0; q <= last; q += STREAM_THREADS / 2) {
    const int64_t p = lo_p + q + plane;
    const bool in = p < hi_p;
    float v[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = in ? zin.c[i][p] : 0.0f;
    if (in) {
      mom_subset<J0, J1>(shi, slo, v);
      if (ROLE == 0) nf += finite6(v) ? 0.f : 1.f;
    }
    if (APPLY) asm volatile("bar.sync %0, 64;" ::"r"(1 + pair) : "memory");
    if (APPLY && in) {
#pragma unroll
      for (int i = 0; i < 6; ++i) v[i] -= c[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < 6; ++j) acc = fmaf(M[i * 6 + j], v[j], acc);
        zout.c[3 * ROLE + i][p] = acc;
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < J1 - J0; ++i) {
    const double t = warp_sum((double)shi[i] + (double)slo[i]);
    if (lane == 0) red[warp][i] = t;
  }
  if (ROLE == 0) {
    const double t = warp_sum((double)nf);
    if (lane == 0) red[warp][14] = t;
  }
}

template <bool APPLY>
__global__ void __launch_bounds__(STREAM_THREADS, 3)
stream_mom_f32_kernel(Soa<float> zin, Soa<float> zout, int64_t n,
                      const int64_t *__restrict__ offsets, int n_bunch,
                      const float *__restrict__ mats, int per_bunch,
                      const float *__restrict__ centers, double *__restrict__ partials) {
  __shared__ int s_b0;
  __shared__ double s_red[STREAM_THREADS / 32][15];
  const int64_t start = (int64_t)blockIdx.x * STREAM_CHUNK;
  const int64_t end = min(n, start + STREAM_CHUNK);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int role = warp & 1;
  const int plane = (warp >> 1) * 32 + lane;  // particle lane 0..127
  if (threadIdx.x == 0) s_b0 = find_bunch(offsets, n_bunch, start);
  __syncthreads();
  int b = s_b0;
  int64_t lo = start;
  while (lo < end) {
    const int64_t hi = min(end, bunch_end(offsets, b, n));
    if (hi > lo) {
      const float *Mb = APPLY ? mats + (per_bunch ? (int64_t)b * 36 : 0) : nullptr;
      const float *cb = (APPLY && centers) ? centers + (int64_t)b * 6 : nullptr;
      if (role == 0) mom_piece<APPLY, 0>(zin, zout, lo, hi, plane, Mb, cb, s_red);
      else mom_piece<APPLY, 1>(zin, zout, lo, hi, plane, Mb, cb, s_red);
      __syncthreads();
      if (threadIdx.x < 28) {
        // sum j: role-0 warps hold j < 14 (and the non-finite count at 14),
        // role-1 warps hold j >= 14 at j - 14
        const int j = threadIdx.x;
        const int r = (j >= 14 && j < 27) ? 1 : 0;
        const int k = (j == 27) ? 14 : (r ? j - 14 : j);
        double t = 0.0;
        for (int w = r; w < STREAM_THREADS / 32; w += 2) t += s_red[w][k];
        partials[((int64_t)b + blockIdx.x) * 28 + j] = t;
      }
      __syncthreads();
    }
    lo = max(lo, hi);
    ++b;
    if (b >= n_bunch) break;
  }
}

template <typename T>
cudaError_t launch_stream(Soa<T> zin, Soa<T> zout, int64_t n, const int64_t *offsets,
                          int n_bunch, const T *mats, int per_bunch, const T *centers,
                          bool apply, bool moments, double *partials, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = stream_blocks(n);
  dim3 grid((unsigned)nb), block(STREAM_THREADS);
  if constexpr (sizeof(T) == 4) {
    if (moments) {
      if (apply)
        stream_mom_f32_kernel<true><<<grid, block, 0, st>>>(zin, zout, n, offsets, n_bunch, mats, per_bunch, centers, partials);
      else
        stream_mom_f32_kernel<false><<<grid, block, 0, st>>>(zin, zout, n, offsets, n_bunch, mats, per_bunch, centers, partials);
      return cudaGetLastError();
    }
  }
  if (apply && moments)
    stream_kernel<T, true, true><<<grid, block, 0, st>>>(zin, zout, n, offsets, n_bunch, mats, per_bunch, centers, partials);
  else if (apply)
    stream_kernel<T, true, false><<<grid, block, 0, st>>>(zin, zout, n, offsets, n_bunch, mats, per_bunch, centers, partials);
  else if (moments)
    stream_kernel<T, false, true><<<grid, block, 0, st>>>(zin, zout, n, offsets, n_bunch, mats, per_bunch, centers, partials);
  return cudaGetLastError();
}

template cudaError_t launch_stream<float>(Soa<float>, Soa<float>, int64_t, const int64_t *, int,
                                          const float *, int, const float *, bool, bool, double *,
                                          cudaStream_t);
template cudaError_t launch_stream<double>(Soa<double>, Soa<double>, int64_t, const int64_t *, int,
                                           const double *, int, const double *, bool, bool,
                                           double *, cudaStream_t);

// Sum the partial slots of bunch b; out[b] = [N, means, central moments].
__global__ void __launch_bounds__(256)
moments_finalize_kernel(const double *__restrict__ partials, const int64_t *__restrict__ offsets,
                        int n_bunch, int64_t n, double *__restrict__ out,
                        unsigned long long *nonfinite) {
  __shared__ double s_red[8 * 28];
  const int b = blockIdx.x;
  const int64_t beg = bunch_begin(offsets, b), end = bunch_end(offsets, b, n);
  double r[28];
#pragma unroll
  for (int i = 0; i < 28; ++i) r[i] = 0.0;
  if (end > beg) {
    const int64_t k0 = beg / STREAM_CHUNK, k1 = (end - 1) / STREAM_CHUNK;
    for (int64_t k = k0 + threadIdx.x; k <= k1; k += blockDim.x) {
      const double *src = partials + ((int64_t)b + k) * 28;
#pragma unroll
      for (int i = 0; i < 28; ++i) r[i] += src[i];
    }
  }
  block_sum<28>(r, s_red);
  if (threadIdx.x == 0) {
    double *o = out + (int64_t)b * 28;
    const double N = (double)(end - beg);
    o[0] = N;
    if (end <= beg) {
      for (int i = 1; i < 28; ++i) o[i] = 0.0;
      return;
    }
    double m[6];
    for (int a = 0; a < 6; ++a) { m[a] = r[a] / N; o[1 + a] = m[a]; }
    int j = 6;
    for (int a = 0; a < 6; ++a)
      for (int c = a; c < 6; ++c) {
        o[1 + j] = r[j] / N - m[a] * m[c];
        ++j;
      }
    if (nonfinite && r[27] > 0.0) atomicAdd(nonfinite, (unsigned long long)r[27]);
  }
}

cudaError_t launch_moments_finalize(const double *partials, const int64_t *offsets, int n_bunch,
                                    int64_t n, double *out, unsigned long long *nonfinite,
                                    cudaStream_t st) {
  moments_finalize_kernel<<<n_bunch, 256, 0, st>>>(partials, offsets, n_bunch, n, out, nonfinite);
  return cudaGetLastError();
}

// ------------------------------------------------------------- adjoint ----
// lambda_in = M_b^T lambda_out in place; partial cross moments
// C_ab = sum_i lambda_out,i,a * z_in,i,b (36 values per slot).
template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS)
linear_adjoint_kernel(Soa<T> lam, Soa<T> zin, int64_t n, const int64_t *__restrict__ offsets,
                      int n_bunch, const T *__restrict__ mats, int per_bunch,
                      double *__restrict__ partials) {
  __shared__ int s_b0;
  __shared__ double s_red[(STREAM_THREADS / 32) * 36];
  const int64_t start = (int64_t)blockIdx.x * STREAM_CHUNK;
  const int64_t end = min(n, start + STREAM_CHUNK);
  if (threadIdx.x == 0) s_b0 = find_bunch(offsets, n_bunch, start);
  __syncthreads();
  int b = s_b0;
  int64_t lo = start;
  while (lo < end) {
    const int64_t hi = min(end, bunch_end(offsets, b, n));
    if (hi > lo) {
      T M[36];
      const T *Mb = mats + (per_bunch ? (int64_t)b * 36 : 0);
#pragma unroll
      for (int i = 0; i < 36; ++i) M[i] = ldg_(Mb + i);
      float chi[36], clo[36];
      double cd[36];
#pragma unroll
      for (int i = 0; i < 36; ++i) { chi[i] = 0.f; clo[i] = 0.f; cd[i] = 0.0; }
      for (int64_t p = lo + threadIdx.x; p < hi; p += STREAM_THREADS) {
        T l[6], z[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) { l[i] = lam.c[i][p]; z[i] = zin.c[i][p]; }
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            if constexpr (sizeof(T) == 4) ff_add_prod(chi[a * 6 + c], clo[a * 6 + c], l[a], z[c]);
            else cd[a * 6 + c] = fma((double)l[a], (double)z[c], cd[a * 6 + c]);
          }
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          T s = T(0);
#pragma unroll
          for (int i = 0; i < 6; ++i) s = fma(M[i * 6 + j], l[i], s);
          lam.c[j][p] = s;
        }
      }
      double r[36];
#pragma unroll
      for (int i = 0; i < 36; ++i)
        r[i] = (sizeof(T) == 4) ? (double)chi[i] + (double)clo[i] : cd[i];
      block_sum<36>(r, s_red);
      if (threadIdx.x == 0) {
        double *dst = partials + ((int64_t)b + blockIdx.x) * 36;
#pragma unroll
        for (int i = 0; i < 36; ++i) dst[i] = r[i];
      }
    }
    lo = max(lo, hi);
    ++b;
    if (b >= n_bunch) break;
  }
}

template <typename T>
cudaError_t launch_linear_adjoint(Soa<T> lam, Soa<T> zin, int64_t n, const int64_t *offsets,
                                  int n_bunch, const T *mats, int per_bunch, double *partials,
                                  cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  linear_adjoint_kernel<T><<<(unsigned)stream_blocks(n), STREAM_THREADS, 0, st>>>(
      lam, zin, n, offsets, n_bunch, mats, per_bunch, partials);
  return cudaGetLastError();
}
template cudaError_t launch_linear_adjoint<float>(Soa<float>, Soa<float>, int64_t, const int64_t *,
                                                  int, const float *, int, double *, cudaStream_t);
template cudaError_t launch_linear_adjoint<double>(Soa<double>, Soa<double>, int64_t,
                                                   const int64_t *, int, const double *, int,
                                                   double *, cudaStream_t);

__global__ void __launch_bounds__(256)
cross_finalize_kernel(const double *__restrict__ partials, const int64_t *__restrict__ offsets,
                      int n_bunch, int64_t n, double *__restrict__ out) {
  __shared__ double s_red[8 * 36];
  const int b = blockIdx.x;
  const int64_t beg = bunch_begin(offsets, b), end = bunch_end(offsets, b, n);
  double r[36];
#pragma unroll
  for (int i = 0; i < 36; ++i) r[i] = 0.0;
  if (end > beg) {
    const int64_t k0 = beg / STREAM_CHUNK, k1 = (end - 1) / STREAM_CHUNK;
    for (int64_t k = k0 + threadIdx.x; k <= k1; k += blockDim.x) {
      const double *src = partials + ((int64_t)b + k) * 36;
#pragma unroll
      for (int i = 0; i < 36; ++i) r[i] += src[i];
    }
  }
  block_sum<36>(r, s_red);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 36; ++i) out[(int64_t)b * 36 + i] = r[i];
  }
}

cudaError_t launch_cross_finalize(const double *partials, const int64_t *offsets, int n_bunch,
                                  int64_t n, double *out, cudaStream_t st) {
  cross_finalize_kernel<<<n_bunch, 256, 0, st>>>(partials, offsets, n_bunch, n, out);
  return cudaGetLastError();
}

}  // namespace bl
