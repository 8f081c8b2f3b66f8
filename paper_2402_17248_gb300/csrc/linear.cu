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
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "runtime.h"
#include "tc.cuh"

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

// ------------------------------------------------ FP32 segment streaming ----
// Persistent kernel for FP32 bunches whose six arrays are 16-byte aligned:
// z_out = M_b (z_in - c_b) and/or the raw moment sums of z_in, the two jobs
// of a segment pass (Sec. 1: a run of linear elements as one per-particle
// map; Sec. 4: beam moments at the segment entry).
//
// Each CTA owns a contiguous range of SUB-particle sub-chunks, its "unit";
// bunch b's partial sums of that range go to slot b + (CTA index), and the
// unit length is handed to the finalize step. The range streams through a
// STAGES-deep ring of shared-memory stages filled by bulk async copies (one
// per coordinate, completion counted in bytes on an mbarrier): the first
// STAGES are issued at the start, and each later one by the last warp to
// release the stage it reuses, so later sub-chunks are in flight while the
// warps compute and no warp is set aside for the copies. One CTA of eight
// warps runs per SM, so that each thread has the registers for four
// particles and its sums without spilling (two CTAs of 128 registers a
// thread ran 1.9x slower with these sums). The warps, in two roles, read a
// stage with 16-byte shared-memory loads, PPT particles per thread: the even
// warps accumulate sums 0..13 (6 linear sums, 8 products)
// and the non-finite count and write output rows 0..2; the odd warps take
// sums 14..26 and rows 3..5, with vector stores. The sums stay in per-thread
// registers across the whole range (biased sums, folded every FOLD_SUBS
// stages into float-float pairs) and are reduced across the block (float-float within a warp, FP64 across warps) only where a bunch or
// the range ends, so a CTA pays one block reduction per bunch piece rather
// than one per few thousand particles. Every wait is bounded; after a
// timeout the warps keep the same sequence of block barriers without
// waiting, and the CTA waits for its own copies before it exits.
namespace segk {
constexpr int WARPS = 8;
constexpr int THREADS = 32 * WARPS;
constexpr int PPT = 4;                  // particles per thread and pass
constexpr int PASS = (WARPS / 2) * 32 * PPT;  // particles per pass of the block over a stage
constexpr int PASSES = 4;               // passes per stage
constexpr int SUB = PASS * PASSES;      // particles per ring stage
constexpr int STAGES = 4;
constexpr int MIN_SUB_PER_CTA = 4;      // a unit spans >= 4096 particles: at most as many
                                        // partial slots as the generic kernel's blocks
static_assert(MIN_SUB_PER_CTA * SUB >= 4096, "unit");
constexpr int FOLD_SUBS = 1;            // stages between folds of the biased sums
constexpr int FOLD_TERMS = PPT * PASSES * FOLD_SUBS;  // terms a thread adds between folds
constexpr float BIAS_MUL = 2.0f * FOLD_TERMS;         // bias = BIAS_MUL * (bound of a term)
constexpr uint32_t COORD_BYTES = SUB * 4;
constexpr uint32_t STAGE_BYTES = 6 * COORD_BYTES;
constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES;
}  // namespace segk

BL_DEV void mbar_arrive_cta(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// hi + lo summed over the warp in float-float (TwoSum of the high parts, the
// low parts and the rounding errors added); the result is valid in lane 0.
BL_DEV void ff_warp_sum(float &hi, float &lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
    const float s = __fadd_rn(hi, h2);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(h2, bp));
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, l2), e);
  }
}

// Biased accumulation of the raw sums. Sum j keeps H = B_j + A, where A
// is the sum of the terms added since the last fold and B_j a power-of-two
// bias of at least twice the largest |A| possible, so that H stays in
// [B/2, 3B/2]. B_j comes from per-coordinate power-of-two bounds S_a >= |z_a|
// of the warp's particles: BIAS_MUL S_a for the coordinate sums and
// BIAS_MUL S_a S_b for the products. Then s = H + term and s - H are exact
// (Sterbenz' lemma), and the rounding error of s is the term minus (s - H):
// exact for a coordinate (Fast2Sum), and for a product one more FMA that
// rounds only that error (relative 2^-24 of it, at most 2^-48 B). The errors
// go to the low part OL of the sum's float-float pair (OH, OL): four
// instructions a term, against ten for TwoProd and TwoSum. Every FOLD_TERMS
// terms at most, H - B (exact, again by Sterbenz) is added to the pair, which
// is renormalised, and H restarts at B.
BL_DEV void fb_add(float &H, float &OL, float x) {
  const float s = __fadd_rn(H, x);
  const float z = __fsub_rn(s, H);
  OL = __fadd_rn(OL, __fsub_rn(x, z));
  H = s;
}

BL_DEV void fb_add_prod(float &H, float &OL, float a, float b) {
  const float s = __fmaf_rn(a, b, H);
  const float z = __fsub_rn(s, H);
  OL = __fadd_rn(OL, __fmaf_rn(a, b, -z));
  H = s;
}

// Move H - B into the float-float pair (OH, OL) (TwoSum of OH and H - B),
// renormalise the pair (Fast2Sum of OH and OL) and restart H at the bias B.
BL_DEV void fb_fold(float &H, float B, float &OH, float &OL) {
  const float d = __fsub_rn(H, B);
  const float s = __fadd_rn(OH, d);
  const float bp = __fsub_rn(s, OH);
  const float e = __fadd_rn(__fsub_rn(OH, __fsub_rn(s, bp)), __fsub_rn(d, bp));
  const float l = __fadd_rn(OL, e);
  const float s2 = __fadd_rn(s, l);
  OL = __fsub_rn(l, __fsub_rn(s2, s));
  OH = s2;
  H = B;
}

// Smallest power of two >= m (m finite, >= 0; 0 for 0), at most 2^127.
BL_DEV float pow2_at_least(float m) {
  const unsigned u = (__float_as_uint(m) + 0x007fffffu) & 0x7f800000u;
  return __uint_as_float(min(u, 0x7f000000u));
}

// The bias of raw sum j (j < 6: coordinate j; then the products z_a z_b,
// a <= b, row-major) from the coordinate bounds S.
BL_DEV float fb_bias(int j, int a, int b, const float (&S)[6]) {
  return j < 6 ? segk::BIAS_MUL * S[j] : segk::BIAS_MUL * S[a] * S[b];
}

// Fold sums J0 <= j < J1 into (OH, OL) and restart them at the biases of S.
template <int J0, int J1>
BL_DEV void fb_fold_subset(float (&H)[J1 - J0], float (&OH)[J1 - J0], float (&OL)[J1 - J0],
                           const float (&S)[6]) {
#pragma unroll
  for (int a = 0; a < 6; ++a)
    if (a >= J0 && a < J1) fb_fold(H[a - J0], fb_bias(a, 0, 0, S), OH[a - J0], OL[a - J0]);
  int j = 6;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int b = a; b < 6; ++b) {
      if (j >= J0 && j < J1) fb_fold(H[j - J0], fb_bias(j, a, b, S), OH[j - J0], OL[j - J0]);
      ++j;
    }
}

// Restart sums J0 <= j < J1 (already folded) at the biases of new bounds S.
template <int J0, int J1>
BL_DEV void fb_rebias_subset(float (&H)[J1 - J0], const float (&S)[6]) {
#pragma unroll
  for (int a = 0; a < 6; ++a)
    if (a >= J0 && a < J1) H[a - J0] = fb_bias(a, 0, 0, S);
  int j = 6;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int b = a; b < 6; ++b) {
      if (j >= J0 && j < J1) H[j - J0] = fb_bias(j, a, b, S);
      ++j;
    }
}

// Issue the bulk copies of sub-chunk j (particles [q0, q0 + cnt)) into ring
// stage s: the largest multiple of four particles of each coordinate (16-byte
// sizes); the rest are read from global memory by the threads.
BL_DEV void seg_issue(const Soa<float> &zin, int64_t q0, int64_t cnt, int s, uint32_t sb,
                      uint32_t full) {
  const uint32_t bytes = (uint32_t)(cnt & ~(int64_t)3) * 4u;
  tc::mbar_expect_tx(full, 6u * bytes);
  if (bytes) {
#pragma unroll
    for (int i = 0; i < 6; ++i)
      tc::bulk_g2s(sb + s * segk::STAGE_BYTES + i * segk::COORD_BYTES, zin.c[i] + q0, bytes,
                   full);
  }
}

// Biased accumulation of the raw sums with index J0 <= j < J1 of one
// particle (errors into the low parts L): j < 6 the coordinates, then the 21
// products z_a z_b (a <= b, row-major).
template <int J0, int J1>
BL_DEV void mom_subset(float (&H)[J1 - J0], float (&L)[J1 - J0], const float (&v)[6]) {
#pragma unroll
  for (int a = 0; a < 6; ++a)
    if (a >= J0 && a < J1) fb_add(H[a - J0], L[a - J0], v[a]);
  int j = 6;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int b = a; b < 6; ++b) {
      if (j >= J0 && j < J1) fb_add_prod(H[j - J0], L[j - J0], v[a], v[b]);
      ++j;
    }
}

// Vector of PPT floats for the 8- or 16-byte shared and global accesses.
template <int P> struct VecOf;
template <> struct VecOf<2> { using type = float2; };
template <> struct VecOf<4> { using type = float4; };
BL_DEV void vec_get(const float2 &w, float (&o)[2]) { o[0] = w.x; o[1] = w.y; }
BL_DEV void vec_get(const float4 &w, float (&o)[4]) { o[0] = w.x; o[1] = w.y; o[2] = w.z; o[3] = w.w; }
BL_DEV float2 vec_make(const float (&o)[2]) { return make_float2(o[0], o[1]); }
BL_DEV float4 vec_make(const float (&o)[4]) { return make_float4(o[0], o[1], o[2], o[3]); }

// One group of PPT particles of one role: moments of the inputs (masked to
// [lo, hi) when MASK) and the role's three output rows. When a particle of
// the warp exceeds the bounds S of a coordinate the role uses (or is not
// finite), the warp folds its sums, raises S to the next power of two of
// the warp's largest finite |z_a| and restarts the sums at the new biases.
template <int ROLE, bool APPLY, bool MOMENTS, bool MASK, bool HAS_C>
BL_DEV void seg_group(const float (&v)[segk::PPT][6], int64_t p0, int64_t lo, int64_t hi,
                      const float (&M)[18], const float (&c)[6],
                      float (&fH)[ROLE ? 13 : 14], float (&S)[6],
                      float (&shi)[ROLE ? 13 : 14], float (&slo)[ROLE ? 13 : 14], float &nf,
                      Soa<float> &zout) {
  constexpr int J0 = ROLE ? 14 : 0, J1 = ROLE ? 27 : 14;
  constexpr int A0 = ROLE ? 1 : 0;  // first coordinate the role's sums use
  constexpr int P = segk::PPT;
  bool act[P];
#pragma unroll
  for (int k = 0; k < P; ++k) act[k] = MASK ? (p0 + k >= lo && p0 + k < hi) : true;
  if (MOMENTS) {
    bool out = false;
#pragma unroll
    for (int k = 0; k < P; ++k)
#pragma unroll
      for (int a = A0; a < 6; ++a) out |= act[k] && !(fabsf(v[k][a]) <= S[a]);
    if (__any_sync(0xffffffffu, out)) {
      fb_fold_subset<J0, J1>(fH, shi, slo, S);
#pragma unroll
      for (int a = A0; a < 6; ++a) {
        float m = 0.0f;
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const float w = fabsf(v[k][a]);
          if (act[k] && w <= 3.4028235e38f) m = fmaxf(m, w);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        S[a] = fmaxf(S[a], pow2_at_least(m));
      }
      fb_rebias_subset<J0, J1>(fH, S);
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      if (!act[k]) continue;
      mom_subset<J0, J1>(fH, slo, v[k]);
      if (ROLE == 0) {
        // v * 0 is 0 for a finite value and NaN for an infinite or NaN one
        float t = 0.0f;
#pragma unroll
        for (int i = 0; i < 6; ++i) t = fmaf(v[k][i], 0.0f, t);
        nf += (t == 0.0f) ? 0.0f : 1.0f;
      }
    }
  }
  if (APPLY) {
    float o[3][P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      float d[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) d[i] = v[k][i];
      if (HAS_C) {
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] -= c[i];
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        float a = 0.0f;
#pragma unroll
        for (int j = 0; j < 6; ++j) a = fmaf(M[6 * r + j], d[j], a);
        o[r][k] = a;
      }
    }
    if (!MASK) {
      using V = typename VecOf<P>::type;
#pragma unroll
      for (int r = 0; r < 3; ++r) *reinterpret_cast<V *>(zout.c[3 * ROLE + r] + p0) = vec_make(o[r]);
    } else {
#pragma unroll
      for (int k = 0; k < P; ++k)
        if (act[k]) {
#pragma unroll
          for (int r = 0; r < 3; ++r) zout.c[3 * ROLE + r][p0 + k] = o[r][k];
        }
    }
  }
}

// Reduce the role's sums over the block's warps into one partial slot (28
// doubles: sums 0..26 and the non-finite count) and clear them; the bounds S
// restart at 0 for the next bunch piece.
template <int ROLE>
BL_DEV void seg_flush(float (&fH)[ROLE ? 13 : 14], float (&S)[6], float (&shi)[ROLE ? 13 : 14],
                      float (&slo)[ROLE ? 13 : 14], float &nf,
                      double (*red)[15], double *dst, int warp, int lane) {
  constexpr int NJ = ROLE ? 13 : 14;
  constexpr int J0 = ROLE ? 14 : 0, J1 = ROLE ? 27 : 14;
  fb_fold_subset<J0, J1>(fH, shi, slo, S);
#pragma unroll
  for (int a = 0; a < 6; ++a) S[a] = 0.0f;
#pragma unroll
  for (int i = 0; i < NJ; ++i) {
    fH[i] = 0.0f;
    ff_warp_sum(shi[i], slo[i]);
    if (lane == 0) red[warp][i] = (double)shi[i] + (double)slo[i];
    shi[i] = 0.0f;
    slo[i] = 0.0f;
  }
  if (ROLE == 0) {
    float z = 0.0f;
    ff_warp_sum(nf, z);
    if (lane == 0) red[warp][14] = (double)nf + (double)z;
    nf = 0.0f;
  }
  __syncthreads();
  const int ct = warp * 32 + lane;
  if (ct < 28) {
    // role-0 warps hold j < 14 and the count at 14; role-1 warps j >= 14 at j - 14
    const int r = (ct >= 14 && ct < 27) ? 1 : 0;
    const int k = (ct == 27) ? 14 : (r ? ct - 14 : ct);
    double t = 0.0;
    for (int w = r; w < segk::WARPS; w += 2) t += red[w][k];
    dst[ct] = t;
  }
  __syncthreads();
}

// The role's three rows of bunch b's segment matrix and (HAS_C) its centre.
template <int ROLE, bool HAS_C>
BL_DEV void seg_load_map(float (&M)[18], float (&c)[6], const float *__restrict__ mats,
                         int per_bunch, const float *__restrict__ centers, int b) {
  const float *Mb = mats + (per_bunch ? (int64_t)b * 36 : 0) + 18 * ROLE;
#pragma unroll
  for (int i = 0; i < 18; ++i) M[i] = __ldg(Mb + i);
#pragma unroll
  for (int i = 0; i < 6; ++i) c[i] = HAS_C ? __ldg(centers + (int64_t)b * 6 + i) : 0.0f;
}

// The warp is done reading ring stage s (sub-chunk j); the last warp to
// release it refills it with sub-chunk j + STAGES once every warp's arrival
// has completed the stage's empty phase.
BL_DEV void seg_release(int s, int64_t j, int64_t nsub, int64_t r_hi, int64_t r_lo,
                        const Soa<float> &zin, uint32_t sb, uint32_t full0, uint32_t empty0,
                        int *s_cnt, long long *s_issued, unsigned *err, int lane) {
  using namespace segk;
  __syncwarp();
  if (lane == 0) {
    mbar_arrive_cta(empty0 + 8 * s);
    if (atomicAdd(&s_cnt[s], 1) == WARPS - 1) {
      s_cnt[s] = 0;
      const int64_t jn = j + STAGES;
      if (jn < nsub && tc::mbar_wait(empty0 + 8 * s, (uint32_t)((j / STAGES) & 1),
                                     BL_DEVERR_TMA_TIMEOUT, err)) {
        const int64_t qn = r_lo + jn * SUB;
        seg_issue(zin, qn, min((int64_t)SUB, r_hi - qn), s, sb, full0 + 8 * s);
        *s_issued = jn + 1;
      }
    }
  }
  __syncwarp();
}

template <int ROLE, bool APPLY, bool MOMENTS, bool HAS_C>
BL_DEV void seg_consume(const Soa<float> &zin, Soa<float> &zout, int64_t n, int64_t r_lo,
                        int64_t r_hi, int64_t nsub, const int64_t *__restrict__ offsets,
                        int n_bunch, const float *__restrict__ mats, int per_bunch,
                        const float *__restrict__ centers, double *__restrict__ partials,
                        unsigned *err, const uint8_t *smem, uint32_t sb, uint32_t full0,
                        uint32_t empty0, int *s_cnt, long long *s_issued, double (*red)[15],
                        int warp, int lane) {
  using namespace segk;
  constexpr int NJ = ROLE ? 13 : 14;
  const int g = (warp >> 1) * 32 + lane;  // particle group of a pass (PPT particles)
  // biased sums fH with their coordinate bounds S, and the float-float pairs
  // (shi, slo) they are folded into; S = 0 gives the biases 0 = fH
  float fH[NJ], S[6], shi[NJ], slo[NJ], nf = 0.0f;
#pragma unroll
  for (int i = 0; i < NJ; ++i) { fH[i] = 0.0f; shi[i] = 0.0f; slo[i] = 0.0f; }
#pragma unroll
  for (int a = 0; a < 6; ++a) S[a] = 0.0f;
  float M[18], c[6];
  int b = find_bunch(offsets, n_bunch, r_lo);
  int64_t pe = bunch_end(offsets, b, n);
  if (APPLY) seg_load_map<ROLE, HAS_C>(M, c, mats, per_bunch, centers, b);
  bool ok = true, open = false;
  using V = typename VecOf<PPT>::type;
  for (int64_t j = 0; j < nsub; ++j) {
    const int s = (int)(j % STAGES);
    if (ok)
      ok = __all_sync(0xffffffffu, tc::mbar_wait(full0 + 8 * s, (uint32_t)((j / STAGES) & 1),
                                                 BL_DEVERR_TMA_TIMEOUT, err));
    const int64_t q0 = r_lo + j * SUB, q1 = min(q0 + SUB, r_hi);
    const int cnt = (int)(q1 - q0), c4 = cnt & ~3;
    const uint8_t *st = smem + s * STAGE_BYTES + 4 * PPT * g;
    if (cnt == SUB && pe >= q1) {
      // the whole stage is full and inside bunch b: four passes, no masks
#pragma unroll 1
      for (int it = 0; it < PASSES; ++it) {
        float v[PPT][6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          float w[PPT];
          vec_get(*reinterpret_cast<const V *>(st + i * COORD_BYTES + it * PASS * 4), w);
#pragma unroll
          for (int k = 0; k < PPT; ++k) v[k][i] = w[k];
        }
        if (it == PASSES - 1) seg_release(s, j, nsub, r_hi, r_lo, zin, sb, full0, empty0, s_cnt,
                                          s_issued, err, lane);
        seg_group<ROLE, APPLY, MOMENTS, false, HAS_C>(v, q0 + it * PASS + PPT * g, 0, 0, M, c,
                                                      fH, S, shi, slo, nf, zout);
      }
      open = true;
      if (pe == q1) {  // bunch b ends with this stage
        if (MOMENTS) {
          seg_flush<ROLE>(fH, S, shi, slo, nf, red,
                          partials + ((int64_t)b + blockIdx.x) * 28, warp, lane);
          open = false;
        }
        if (b + 1 < n_bunch) {
          ++b;
          pe = bunch_end(offsets, b, n);
          if (APPLY && (per_bunch || HAS_C)) seg_load_map<ROLE, HAS_C>(M, c, mats, per_bunch, centers, b);
        }
      }
    } else {
      // a stage with bunch boundaries or the array's ragged end: each pass
      // walks the bunch pieces it meets, with masks
      int64_t cur = q0;
#pragma unroll 1
      for (int it = 0; it < PASSES; ++it) {
        const int64_t a0 = q0 + it * PASS;
        if (a0 >= q1) break;
        const int64_t a1 = min(a0 + PASS, q1);
        const int64_t p0 = a0 + PPT * g;
        const int rel = it * PASS + PPT * g;  // position of this thread's first particle in the stage
        float v[PPT][6];
        if (rel + PPT <= c4) {
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            float w[PPT];
            vec_get(*reinterpret_cast<const V *>(st + i * COORD_BYTES + it * PASS * 4), w);
#pragma unroll
            for (int k = 0; k < PPT; ++k) v[k][i] = w[k];
          }
        } else {
          // past the copied multiple of four (only the array's last particles)
#pragma unroll
          for (int k = 0; k < PPT; ++k)
#pragma unroll
            for (int i = 0; i < 6; ++i)
              v[k][i] = (rel + k >= c4 && rel + k < cnt) ? zin.c[i][p0 + k] : 0.0f;
        }
        // in place, the particles past the copied part come from global
        // memory: every warp reads them before any warp stores
        if (a1 > q0 + c4) __syncthreads();
        for (;;) {
          const int64_t hi = min(a1, pe);
          if (hi > cur) {
            seg_group<ROLE, APPLY, MOMENTS, true, HAS_C>(v, p0, cur, hi, M, c, fH, S, shi, slo,
                                                         nf, zout);
            open = true;
          }
          if (hi < pe) break;  // bunch b goes on past this pass
          if (MOMENTS && open) {
            seg_flush<ROLE>(fH, S, shi, slo, nf, red,
                            partials + ((int64_t)b + blockIdx.x) * 28, warp, lane);
            open = false;
          }
          if (++b >= n_bunch) break;
          pe = bunch_end(offsets, b, n);
          if (APPLY && (per_bunch || HAS_C)) seg_load_map<ROLE, HAS_C>(M, c, mats, per_bunch, centers, b);
          cur = hi;
          if (cur >= a1) break;
        }
        cur = max(cur, a1);
      }
      seg_release(s, j, nsub, r_hi, r_lo, zin, sb, full0, empty0, s_cnt, s_issued, err, lane);
    }
    if (MOMENTS && (j % FOLD_SUBS) == FOLD_SUBS - 1)
      fb_fold_subset<ROLE ? 14 : 0, ROLE ? 27 : 14>(fH, shi, slo, S);
  }
  if (MOMENTS && open)
    seg_flush<ROLE>(fH, S, shi, slo, nf, red, partials + ((int64_t)b + blockIdx.x) * 28,
                    warp, lane);
}

template <bool APPLY, bool MOMENTS, bool HAS_C>
__global__ void __launch_bounds__(segk::THREADS, 1)
seg_f32_kernel(Soa<float> zin, Soa<float> zout, int64_t n, int64_t per_cta,
               const int64_t *__restrict__ offsets, int n_bunch, const float *__restrict__ mats,
               int per_bunch, const float *__restrict__ centers, double *__restrict__ partials,
               unsigned *err) {
  using namespace segk;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[2 * STAGES];  // full[s], then empty[s]
  __shared__ double red[WARPS][15];
  __shared__ int s_cnt[STAGES];       // warps that have released stage s in its current round
  __shared__ long long s_issued;      // sub-chunks whose copies have been issued
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nsub_all = (n + SUB - 1) / SUB;
  const int64_t j0 = (int64_t)blockIdx.x * per_cta;
  const int64_t nsub = min(nsub_all, j0 + per_cta) - j0;  // >= 1 by the grid size
  const int64_t r_lo = j0 * SUB, r_hi = min(n, (j0 + nsub) * SUB);
  const uint32_t sb = tc::smem_u32(smem);
  const uint32_t full0 = tc::smem_u32(&bars[0]), empty0 = tc::smem_u32(&bars[STAGES]);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(full0 + 8 * s, 1);
      tc::mbar_init(empty0 + 8 * s, WARPS);
      s_cnt[s] = 0;
    }
    tc::fence_mbar_init();
    const int64_t first = min((int64_t)STAGES, nsub);
    for (int64_t j = 0; j < first; ++j) {
      const int64_t q0 = r_lo + j * SUB;
      seg_issue(zin, q0, min((int64_t)SUB, r_hi - q0), (int)j, sb, full0 + 8 * (int)j);
    }
    s_issued = first;
  }
  __syncthreads();
  if ((warp & 1) == 0)
    seg_consume<0, APPLY, MOMENTS, HAS_C>(zin, zout, n, r_lo, r_hi, nsub, offsets, n_bunch, mats,
                                   per_bunch, centers, partials, err, smem, sb, full0, empty0,
                                   s_cnt, &s_issued, red, warp, lane);
  else
    seg_consume<1, APPLY, MOMENTS, HAS_C>(zin, zout, n, r_lo, r_hi, nsub, offsets, n_bunch, mats,
                                   per_bunch, centers, partials, err, smem, sb, full0, empty0,
                                   s_cnt, &s_issued, red, warp, lane);
  // no copy may still be writing this CTA's shared memory when it exits (the
  // warps have waited for every copy, unless a wait timed out)
  __syncthreads();
  if (tid == 0) {
    const long long issued = s_issued;
    for (long long j = max(0ll, issued - STAGES); j < issued; ++j)
      tc::mbar_wait(full0 + 8 * (int)(j % STAGES), (uint32_t)((j / STAGES) & 1),
                    BL_DEVERR_TMA_TIMEOUT, err);
  }
}

// Sub-chunks per CTA for n particles: the range of one CTA per SM, at least
// MIN_SUB_PER_CTA.
int64_t seg_per_cta(int64_t n, int num_sms) {
  const int64_t S = (n + segk::SUB - 1) / segk::SUB;
  const int64_t G = (int64_t)std::max(num_sms, 1);
  return std::max<int64_t>(segk::MIN_SUB_PER_CTA, (S + G - 1) / G);
}

template <bool APPLY, bool MOMENTS, bool HAS_C>
cudaError_t launch_seg(Soa<float> zin, Soa<float> zout, int64_t n, const int64_t *offsets,
                       int n_bunch, const float *mats, int per_bunch, const float *centers,
                       double *partials, int num_sms, unsigned *err, int64_t *unit,
                       cudaStream_t st) {
  static std::mutex mu;
  static bool configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!configured[dev]) {
      e = cudaFuncSetAttribute(seg_f32_kernel<APPLY, MOMENTS, HAS_C>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)segk::SMEM_BYTES);
      if (e != cudaSuccess) return e;
      configured[dev] = true;
    }
  }
  const int64_t per = seg_per_cta(n, num_sms);
  const int64_t S = (n + segk::SUB - 1) / segk::SUB;
  const int64_t grid = (S + per - 1) / per;
  if (unit) *unit = per * segk::SUB;
  seg_f32_kernel<APPLY, MOMENTS, HAS_C><<<(unsigned)grid, segk::THREADS, segk::SMEM_BYTES, st>>>(
      zin, zout, n, per, offsets, n_bunch, mats, per_bunch, centers, partials, err);
  return cudaGetLastError();
}

bool aligned16(const Soa<float> &z) {
  for (int i = 0; i < 6; ++i)
    if (reinterpret_cast<uintptr_t>(z.c[i]) & 15u) return false;
  return true;
}

template <typename T>
cudaError_t launch_stream(Soa<T> zin, Soa<T> zout, int64_t n, const int64_t *offsets,
                          int n_bunch, const T *mats, int per_bunch, const T *centers,
                          bool apply, bool moments, double *partials, cudaStream_t st,
                          int64_t *unit) {
  if (unit) *unit = STREAM_CHUNK;
  if (n <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    if (aligned16(zin) && aligned16(zout) && (apply || moments) &&
        !(apply && moments && centers)) {
      DevCtx *ctx = nullptr;
      if (current_ctx(&ctx) != BL_OK) return cudaErrorInvalidDevice;
      // the centres of the transposed maps (adjoint) never come with moments
      if (apply && moments && !centers)
        return launch_seg<true, true, false>(zin, zout, n, offsets, n_bunch, mats, per_bunch,
                                             nullptr, partials, ctx->num_sms, ctx->err_word,
                                             unit, st);
      if (apply && !moments)
        return centers ? launch_seg<true, false, true>(zin, zout, n, offsets, n_bunch, mats,
                                                       per_bunch, centers, partials, ctx->num_sms,
                                                       ctx->err_word, unit, st)
                       : launch_seg<true, false, false>(zin, zout, n, offsets, n_bunch, mats,
                                                        per_bunch, nullptr, partials,
                                                        ctx->num_sms, ctx->err_word, unit, st);
      if (!apply)
        return launch_seg<false, true, false>(zin, zout, n, offsets, n_bunch, mats, per_bunch,
                                              nullptr, partials, ctx->num_sms, ctx->err_word,
                                              unit, st);
    }
  }
  const int64_t nb = stream_blocks(n);
  dim3 grid((unsigned)nb), block(STREAM_THREADS);
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
                                          cudaStream_t, int64_t *);
template cudaError_t launch_stream<double>(Soa<double>, Soa<double>, int64_t, const int64_t *, int,
                                           const double *, int, const double *, bool, bool,
                                           double *, cudaStream_t, int64_t *);

// Sum the partial slots of bunch b (slot b + k for every unit k of `unit`
// particles that its range touches); out[b] = [N, means, central moments].
__global__ void __launch_bounds__(256)
moments_finalize_kernel(const double *__restrict__ partials, const int64_t *__restrict__ offsets,
                        int n_bunch, int64_t n, int64_t unit, double *__restrict__ out,
                        unsigned long long *nonfinite) {
  __shared__ double s_red[8 * 28];
  const int b = blockIdx.x;
  const int64_t beg = bunch_begin(offsets, b), end = bunch_end(offsets, b, n);
  double r[28];
#pragma unroll
  for (int i = 0; i < 28; ++i) r[i] = 0.0;
  if (end > beg) {
    const int64_t k0 = beg / unit, k1 = (end - 1) / unit;
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
                                    int64_t n, int64_t unit, double *out,
                                    unsigned long long *nonfinite, cudaStream_t st) {
  moments_finalize_kernel<<<n_bunch, 256, 0, st>>>(partials, offsets, n_bunch, n, unit, out,
                                                   nonfinite);
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

// FP32 form: each thread loads AP particles (strided by the block size, so
// every load is coalesced) before it uses any, keeping 48 loads in flight;
// the 36 float-float sums are reduced across the block through shared
// memory in four rounds of 9 (float-float within a round, FP64 only for the
// last 28 partials of a sum), instead of FP64 warp shuffles.
namespace adjk {
constexpr int AP = 4;                 // particles per thread and iteration
constexpr int RS = 9;                 // sums per reduction round
constexpr int PARTS = STREAM_THREADS / RS;  // 28 partials per sum in a round
}  // namespace adjk

__global__ void __launch_bounds__(STREAM_THREADS, 1)
linear_adjoint_f32_kernel(Soa<float> lam, Soa<float> zin, int64_t n,
                          const int64_t *__restrict__ offsets, int n_bunch,
                          const float *__restrict__ mats, int per_bunch,
                          double *__restrict__ partials) {
  using namespace adjk;
  __shared__ int s_b0;
  __shared__ float s_h[RS][STREAM_THREADS], s_l[RS][STREAM_THREADS];
  __shared__ float s_ph[RS][PARTS], s_pl[RS][PARTS];
  __shared__ double s_res[36];
  const int tid = threadIdx.x;
  const int64_t start = (int64_t)blockIdx.x * STREAM_CHUNK;
  const int64_t end = min(n, start + STREAM_CHUNK);
  if (tid == 0) s_b0 = find_bunch(offsets, n_bunch, start);
  __syncthreads();
  int b = s_b0;
  int64_t lo = start;
  while (lo < end) {
    const int64_t hi = min(end, bunch_end(offsets, b, n));
    if (hi > lo) {
      float M[36];
      const float *Mb = mats + (per_bunch ? (int64_t)b * 36 : 0);
#pragma unroll
      for (int i = 0; i < 36; ++i) M[i] = __ldg(Mb + i);
      float chi[36], clo[36];
#pragma unroll
      for (int i = 0; i < 36; ++i) { chi[i] = 0.f; clo[i] = 0.f; }
      for (int64_t p0 = lo + tid; p0 < hi; p0 += (int64_t)AP * STREAM_THREADS) {
        float l[AP][6], z[AP][6];
#pragma unroll
        for (int k = 0; k < AP; ++k) {
          const int64_t p = p0 + (int64_t)k * STREAM_THREADS;
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            l[k][i] = p < hi ? lam.c[i][p] : 0.f;
            z[k][i] = p < hi ? zin.c[i][p] : 0.f;
          }
        }
#pragma unroll
        for (int k = 0; k < AP; ++k) {
          const int64_t p = p0 + (int64_t)k * STREAM_THREADS;
          if (p >= hi) break;
#pragma unroll
          for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int c = 0; c < 6; ++c) ff_add_prod(chi[a * 6 + c], clo[a * 6 + c], l[k][a], z[k][c]);
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 6; ++i) s = fmaf(M[i * 6 + j], l[k][i], s);
            lam.c[j][p] = s;
          }
        }
      }
      // block reduction of the 36 sums, RS at a time
#pragma unroll
      for (int r = 0; r < 36 / RS; ++r) {
#pragma unroll
        for (int i = 0; i < RS; ++i) { s_h[i][tid] = chi[r * RS + i]; s_l[i][tid] = clo[r * RS + i]; }
        __syncthreads();
        if (tid < RS * PARTS) {
          const int j = tid / PARTS, q = tid - j * PARTS;
          float h = 0.f, l2 = 0.f;
          for (int t = q; t < STREAM_THREADS; t += PARTS) {
            ff_add(h, l2, s_h[j][t]);
            l2 = __fadd_rn(l2, s_l[j][t]);
          }
          s_ph[j][q] = h;
          s_pl[j][q] = l2;
        }
        __syncthreads();
        if (tid < RS) {
          double acc = 0.0;
          for (int q = 0; q < PARTS; ++q) acc += (double)s_ph[tid][q] + (double)s_pl[tid][q];
          s_res[r * RS + tid] = acc;
        }
        __syncthreads();
      }
      if (tid < 36) partials[((int64_t)b + blockIdx.x) * 36 + tid] = s_res[tid];
      __syncthreads();
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
  if constexpr (sizeof(T) == 4)
    linear_adjoint_f32_kernel<<<(unsigned)stream_blocks(n), STREAM_THREADS, 0, st>>>(
        lam, zin, n, offsets, n_bunch, mats, per_bunch, partials);
  else
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
