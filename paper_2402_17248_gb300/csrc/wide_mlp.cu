// The paper's own surrogate networks (Sec. 4.2: five hidden layers of 900
// units for the first stages, three of 700 for the later ones, PReLU, one
// learned slope per layer) applied to every particle in place (Sec. 4.3),
// with the same normalise / de-normalise data preparation as the small
// surrogate.
//
// A hidden layer of 900 units does not fit a 128-particle tile's activations
// on chip (128 x 960 BF16 = 240 KB), so the network runs layer by layer: each
// layer is a persistent tcgen05 GEMM C = prelu(A W^T + b) over a chunk of
// particles, with the activations of the chunk in HBM between layers (the
// GEMM is compute-bound: ~480 flop per byte at width 960).
//
// Operand layout (host-packed weights, kernel-written activations): a matrix
// [R x K] is cut into tiles of [rows x 64] K-major BF16 in the no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix; K chunks 128 bytes
// apart, row groups 1024 bytes apart), so every tile is one contiguous block
// that a single bulk async copy moves:
//  * activations: 128-row tiles (16 KB), ordered (row tile, K tile);
//  * weights [N x K]: 64-row tiles (8 KB), ordered (K tile, N tile), so the
//    up to four tiles of a 256-column output block at one K tile are
//    contiguous too.
// Per layer: one CTA per SM, warp 0 (one lane) streams A and B tiles into a
// four-stage shared-memory ring with mbarrier transaction counts, warp 1 (one
// lane) issues M=128 x N<=256 x K=16 MMAs into one of two tensor-memory
// accumulators (256 columns each), and four epilogue warps add the bias,
// apply PReLU and store the BF16 tile of the next layer's input while the
// other accumulator fills. Hidden widths are padded with zero weights to
// multiples of 64 (PReLU(0) = 0 keeps the padding at zero).
#include <algorithm>
#include <cmath>
#include <vector>

#include "mlp_common.cuh"

namespace bl {

namespace {

using namespace mlp;

constexpr int BM = 128;                    // particles per tile
constexpr int BK = 64;                     // K per tile (128-byte rows)
constexpr int BN_MAX = 256;                // output columns per work unit
constexpr int STAGES = 4;
constexpr uint32_t A_TILE = BM * BK * 2;                 // 16 KB
constexpr uint32_t B_SUB = 64 * BK * 2;                  // 8 KB (64 weight rows)
constexpr uint32_t STAGE_BYTES = A_TILE + BN_MAX * BK * 2;  // 48 KB
constexpr uint32_t OFF_BAR = STAGES * STAGE_BYTES;
constexpr uint32_t OFF_TSLOT = OFF_BAR + 8 * (2 * STAGES + 4);
constexpr uint32_t SMEM_BYTES = OFF_TSLOT + 16;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");
constexpr int THREADS = 192;  // warp 0 producer, warp 1 MMA, warps 2..5 epilogue
constexpr uint32_t TMEM_COLS = 512;

__host__ __device__ inline uint32_t tile_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Byte offset of weight (n, k) in a layer's tiled image: 64-row tiles
// ordered (K tile, N tile).
__host__ __device__ inline size_t wide_weight_offset_dev(int n, int k, int N_pad) {
  return ((size_t)(k >> 6) * (N_pad / 64) + (n >> 6)) * B_SUB + tile_off(n & 63, k & 63);
}

struct WideLayer {
  const uint8_t *A;     // activations of the chunk, tiled [RT][KT]
  const uint8_t *B;     // weights, tiled [KT][N_pad / 64]
  const float *bias;    // [N_pad]
  const float *slope;   // PReLU slope (hidden layers), device
  uint8_t *C;           // next activations, tiled [RT][N_pad / 64] (hidden layers)
  int KT, N_pad, RT;
  Soa<float> z;         // output layer: particles of the chunk (in place)
  int64_t n;            // particles in the chunk
  MlpNormF nrm;
  float *pre;           // training, hidden layers: pre-activations [RT*128][N_pad] FP32
  float *Y;             // training, output layer: raw outputs [RT*128][8] FP32
};

// Layer kernel modes: a hidden layer for inference or for training (which
// also keeps the FP32 pre-activations for the backward pass), and the output
// layer for inference (de-normalised into the particles) or for training
// (the raw normalised outputs).
enum { WL_HIDDEN = 0, WL_HIDDEN_TRAIN = 1, WL_LAST = 2, WL_LAST_TRAIN = 3 };

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) wide_layer_kernel(WideLayer p, unsigned *err) {
  constexpr bool LAST = MODE >= WL_LAST;
  extern __shared__ __align__(1024) uint8_t smem[];
  const uint32_t sbase = tc::smem_u32(smem);
  const uint32_t bar = sbase + OFF_BAR;
  // full[s] = bar + 8 s; empty[s] = bar + 8 (STAGES + s);
  // acc_full[b] = bar + 8 (2 STAGES + b); acc_empty[b] = bar + 8 (2 STAGES + 2 + b)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + OFF_TSLOT);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(bar + 8 * s, 1);
      tc::mbar_init(bar + 8 * (STAGES + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(bar + 8 * (2 * STAGES + b), 1);
      tc::mbar_init(bar + 8 * (2 * STAGES + 2 + b), 128);
    }
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tc::smem_u32(tslot), TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const int NB = (p.N_pad + BN_MAX - 1) / BN_MAX;
  const int NT = p.N_pad / 64;
  const int64_t U = (int64_t)p.RT * NB;

  if (warp == 0) {
    // ------------------------------------------------------- tile producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; ok && u < U; u += gridDim.x) {
        const int64_t rt = u / NB;
        const int nb = (int)(u % NB);
        const int bn = min(BN_MAX, p.N_pad - BN_MAX * nb);
        for (int kt = 0; kt < p.KT; ++kt) {
          ok = tc::mbar_wait(bar + 8 * (STAGES + s), ph ^ 1u, BL_DEVERR_TMA_TIMEOUT, err);
          if (!ok) break;
          const uint32_t dst = sbase + s * STAGE_BYTES;
          tc::mbar_expect_tx(bar + 8 * s, A_TILE + (uint32_t)bn * BK * 2);
          tc::bulk_g2s(dst, p.A + ((size_t)rt * p.KT + kt) * A_TILE, A_TILE, bar + 8 * s);
          tc::bulk_g2s(dst + A_TILE, p.B + ((size_t)kt * NT + 4 * nb) * B_SUB,
                       (uint32_t)bn * BK * 2, bar + 8 * s);
          if (++s == STAGES) { s = 0; ph ^= 1u; }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issue
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0, eph = 0;  // ring phase; bit b: acc_empty[b] phase
      int ab = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; ok && u < U; u += gridDim.x) {
        const int nb = (int)(u % NB);
        const int bn = min(BN_MAX, p.N_pad - BN_MAX * nb);
        ok = tc::mbar_wait(bar + 8 * (2 * STAGES + 2 + ab), ((eph >> ab) & 1u) ^ 1u,
                           BL_DEVERR_MMA_TIMEOUT, err);
        eph ^= 1u << ab;
        if (!ok) break;
        tc::fence_after();
        const uint32_t d = tmem + 256 * ab;
        const uint32_t id = tc::idesc_bf16(128, bn);
        for (int kt = 0; kt < p.KT; ++kt) {
          ok = tc::mbar_wait(bar + 8 * s, ph, BL_DEVERR_MMA_TIMEOUT, err);
          if (!ok) break;
          tc::fence_after();
          const uint64_t da = tc::sdesc(sbase + s * STAGE_BYTES, 128, 1024);
          const uint64_t db = tc::sdesc(sbase + s * STAGE_BYTES + A_TILE, 128, 1024);
#pragma unroll
          for (int j = 0; j < BK / 16; ++j)
            tc::mma_ss(d, da + 16 * j, db + 16 * j, id, (kt | j) != 0);
          tc::mma_commit(bar + 8 * (STAGES + s));  // frees the stage when these MMAs finish
          if (++s == STAGES) { s = 0; ph ^= 1u; }
        }
        tc::mma_commit(bar + 8 * (2 * STAGES + ab));  // accumulator ready
        ab ^= 1;
      }
    }
    __syncwarp();
  } else {
    // ----------------------------------------------------------- epilogue
    const int q = warp & 3;  // tensor-memory lane quarter of this warp
    const int m = q * 32 + lane;
    const uint32_t t_row = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t fph = 0;
    int ab = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; ok && u < U; u += gridDim.x) {
      const int64_t rt = u / NB;
      const int nb = (int)(u % NB);
      const int bn = min(BN_MAX, p.N_pad - BN_MAX * nb);
      ok = __all_sync(0xffffffffu, tc::mbar_wait(bar + 8 * (2 * STAGES + ab), (fph >> ab) & 1u,
                                                 BL_DEVERR_MMA_TIMEOUT, err));
      fph ^= 1u << ab;
      if (!ok) break;
      tc::fence_after();
      if constexpr (!LAST) {
        for (int c = 0; c < bn / 32; ++c) {
          uint32_t r[32];
          tc::tmem_ld32(t_row + 256 * ab + 32 * c, r);
          tc::tmem_ld_wait_regs(r);
          const int col0 = BN_MAX * nb + 32 * c;
          const float4 *bv = reinterpret_cast<const float4 *>(p.bias + col0);
          uint8_t *dst = p.C + ((size_t)rt * NT + (col0 >> 6)) * A_TILE;
          const float a = __ldg(p.slope);
#pragma unroll
          for (int g = 0; g < 4; ++g) {  // 8 columns = one 16-byte core-matrix row
            const float4 b0 = __ldg(bv + 2 * g), b1 = __ldg(bv + 2 * g + 1);
            const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
            uint32_t o[4];
            float pv[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              float v0 = __uint_as_float(r[8 * g + 2 * j]) + bb[2 * j];
              float v1 = __uint_as_float(r[8 * g + 2 * j + 1]) + bb[2 * j + 1];
              pv[2 * j] = v0;
              pv[2 * j + 1] = v1;
              v0 = v0 > 0.0f ? v0 : a * v0;
              v1 = v1 > 0.0f ? v1 : a * v1;
              o[j] = tc::pack_bf16x2(v0, v1);
            }
            if (MODE == WL_HIDDEN_TRAIN) {
              float4 *pr = reinterpret_cast<float4 *>(p.pre + ((size_t)rt * BM + m) * p.N_pad +
                                                      col0 + 8 * g);
              pr[0] = make_float4(pv[0], pv[1], pv[2], pv[3]);
              pr[1] = make_float4(pv[4], pv[5], pv[6], pv[7]);
            }
            *reinterpret_cast<uint4 *>(dst + tile_off(m, (col0 & 63) + 8 * g)) =
                make_uint4(o[0], o[1], o[2], o[3]);
          }
        }
      } else {
        uint32_t r[8];
        tc::tmem_ld8(t_row + 256 * ab, r);
        tc::tmem_ld_wait();
        const int64_t i = rt * BM + m;
        if (MODE == WL_LAST_TRAIN) {
          float y[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) y[c] = c < 6 ? __uint_as_float(r[c]) + __ldg(p.bias + c) : 0.f;
          float4 *yo = reinterpret_cast<float4 *>(p.Y + (size_t)i * 8);
          yo[0] = make_float4(y[0], y[1], y[2], y[3]);
          yo[1] = make_float4(y[4], y[5], y[6], y[7]);
        } else if (i < p.n) {
#pragma unroll
          for (int c = 0; c < 6; ++c)
            p.z.c[c][i] = df_affine(__uint_as_float(r[c]) + __ldg(p.bias + c), p.nrm.sd_out[c][0],
                                    p.nrm.sd_out[c][1], p.nrm.mu_out[c][0], p.nrm.mu_out[c][1]);
        }
      }
      tc::fence_before();
      mbar_arrive(bar + 8 * (2 * STAGES + 2 + ab));
      ab ^= 1;
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

// Normalised network input of a chunk: one 64-column K tile per 128
// particles, columns 0..5 the coordinates' BF16 high parts and 8..13 their
// low parts bf16(x - hi) (the first layer's weights repeat there), the rest
// zero.
__global__ void __launch_bounds__(256) wide_prep_kernel(Soa<float> z, int64_t n, int RT,
                                                        uint8_t *A, MlpNormF nrm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)RT * BM) return;
  float x[6];
#pragma unroll
  for (int c = 0; c < 6; ++c)
    x[c] = df_normalise(i < n ? z.c[c][i] : 0.0f, nrm.mu_in[c][0], nrm.mu_in[c][1],
                        nrm.inv_sd_in[c][0], nrm.inv_sd_in[c][1]);
  uint8_t *t = A + (size_t)(i / BM) * A_TILE;
  const int r = (int)(i % BM);
  uint32_t w[8];
  input_row(x, w);
  *reinterpret_cast<uint4 *>(t + tile_off(r, 0)) = make_uint4(w[0], w[1], w[2], 0u);
  *reinterpret_cast<uint4 *>(t + tile_off(r, 8)) = make_uint4(w[4], w[5], w[6], 0u);
#pragma unroll
  for (int k = 16; k < BK; k += 8)
    *reinterpret_cast<uint4 *>(t + tile_off(r, k)) = make_uint4(0u, 0u, 0u, 0u);
}

// ------------------------------------------------------------ training ----
// One minibatch step of a wide network (Sec. 3: MSE on normalised data,
// Adam): the forward pass runs the layer kernel above in its training modes
// (pre-activations kept in FP32, raw outputs); the backward pass is written
// out below as tiled FP32 GEMMs on the CUDA cores:
//   dW_l = dZ_l^T X_l and db_l = sum_b dZ_l   (X_l: the layer's BF16 input)
//   dX_l = dZ_l W_l                            (W_l: the BF16-valued weights)
//   dZ_{l-1} = dX_l * prelu'(pre_{l-1}),  dL/da_{l-1} = sum dX_l min(pre_{l-1}, 0)
// with prelu'(v) = 1 for v > 0 and a otherwise, then Adam on the flat FP32
// parameter vector [W_0, b_0, ..., W_{L-1}, b_{L-1}, a_0 .. a_{L-2}] and a
// re-pack of the BF16 images the layer kernel reads.

// Normalised, gathered training inputs of a minibatch: the same K tile layout
// as wide_prep_kernel; rows past the batch are zero.
__global__ void __launch_bounds__(256) wide_train_prep_kernel(Soa<float> in, const int64_t *idx,
                                                              int64_t batch, int RT, uint8_t *A,
                                                              MlpNormF nrm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)RT * BM) return;
  const bool valid = i < batch;
  const int64_t col = valid ? (idx ? idx[i] : i) : 0;
  float x[6];
#pragma unroll
  for (int c = 0; c < 6; ++c)
    x[c] = valid ? df_normalise(in.c[c][col], nrm.mu_in[c][0], nrm.mu_in[c][1],
                                nrm.inv_sd_in[c][0], nrm.inv_sd_in[c][1])
                 : 0.0f;
  uint32_t w[8];
  input_row(x, w);
  uint8_t *t = A + (size_t)(i / BM) * A_TILE;
  const int r = (int)(i % BM);
  if (!valid) w[0] = w[1] = w[2] = w[4] = w[5] = w[6] = 0u;
  *reinterpret_cast<uint4 *>(t + tile_off(r, 0)) = make_uint4(w[0], w[1], w[2], 0u);
  *reinterpret_cast<uint4 *>(t + tile_off(r, 8)) = make_uint4(w[4], w[5], w[6], 0u);
#pragma unroll
  for (int k = 16; k < BK; k += 8)
    *reinterpret_cast<uint4 *>(t + tile_off(r, k)) = make_uint4(0u, 0u, 0u, 0u);
}

// dY = d MSE / d Y = 2 (Y - T) / (6 batch) for the normalised targets T (zero
// past the batch); per-block partial sums of (Y - T)^2.
struct InvSd { float v[12]; };  // 1 / sd_out per coordinate as double-float pairs

__global__ void __launch_bounds__(256) wide_loss_kernel(const float *__restrict__ Y,
                                                        Soa<float> out, const int64_t *idx,
                                                        int64_t batch, int64_t rows,
                                                        MlpNormF nrm, InvSd inv_sd_out,
                                                        float *__restrict__ dY,
                                                        double *__restrict__ loss_part) {
  __shared__ double red[8];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l2 = 0.0;
  if (i < rows) {
    const bool valid = i < batch;
    const int64_t col = valid ? (idx ? idx[i] : i) : 0;
    const float sc = (float)(2.0 / (6.0 * (double)batch));
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float d = 0.0f;
      if (valid && c < 6) {
        const float t = df_normalise(out.c[c][col], nrm.mu_out[c][0], nrm.mu_out[c][1],
                                     inv_sd_out.v[2 * c], inv_sd_out.v[2 * c + 1]);
        const float e = Y[i * 8 + c] - t;
        l2 += (double)e * (double)e;
        d = sc * e;
      }
      dY[i * 8 + c] = d;
    }
  }
  l2 = warp_sum(l2);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    loss_part[blockIdx.x] = t;
  }
}

constexpr int GT = 64;   // output tile of the backward GEMMs
constexpr int GKC = 32;  // contraction chunk

// Element (row, k) of a tiled BF16 activation matrix with KT K tiles.
BL_DEV float act_at(const uint8_t *A, int KT, int64_t row, int k) {
  const uint8_t *t = A + ((size_t)(row / BM) * KT + (k >> 6)) * A_TILE;
  return __bfloat162float(
      *reinterpret_cast<const __nv_bfloat16 *>(t + tile_off((int)(row % BM), k & 63)));
}

// Partial weight gradients part[s][n][k] = sum over the s-th slice of the
// batch rows of dZ[b][n] X[b][k] (n < N, k < K; for the first layer X is the
// input's hi + lo pair); grid (N/64, K/64, splits), 256 threads with 4 x 4
// outputs each.
__global__ void __launch_bounds__(256) wide_dw_kernel(const float *__restrict__ dZ, int ldz,
                                                      const uint8_t *__restrict__ X, int KT, int N,
                                                      int K, int64_t rows_per_split, int first,
                                                      float *__restrict__ part) {
  __shared__ float sz[GKC][GT + 4];
  __shared__ float sx[GKC][GT + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int n0 = blockIdx.x * GT, k0 = blockIdx.y * GT;
  const int64_t b_lo = (int64_t)blockIdx.z * rows_per_split, b_hi = b_lo + rows_per_split;
  float acc[4][4] = {};
  for (int64_t b0 = b_lo; b0 < b_hi; b0 += GKC) {
    for (int e = threadIdx.x; e < GKC * GT; e += 256) {
      const int i = e / GT, j = e % GT;
      sz[i][j] = (n0 + j < N) ? dZ[(b0 + i) * ldz + n0 + j] : 0.0f;
      // the first layer's input is the pair hi (column k) + lo (column 8 + k)
      float x = 0.0f;
      if (k0 + j < K) {
        x = act_at(X, KT, b0 + i, k0 + j);
        if (first) x += act_at(X, KT, b0 + i, k0 + j + 8);
      }
      sx[i][j] = x;
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < GKC; ++i) {
      float a[4], x[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = sz[i][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = sx[i][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], x[c], acc[r][c]);
    }
    __syncthreads();
  }
  float *dst = part + (size_t)blockIdx.z * N * K;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int n = n0 + ty * 4 + r, k = k0 + tx * 4 + c;
      if (n < N && k < K) dst[(size_t)n * K + k] = acc[r][c];
    }
}

// g[i] = sum_s part[s][i] (i < count).
__global__ void __launch_bounds__(256) wide_sum_splits_kernel(const float *__restrict__ part,
                                                              int splits, int64_t count,
                                                              float *__restrict__ g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float t = 0.0f;
  for (int s = 0; s < splits; ++s) t += part[(size_t)s * count + i];
  g[i] = t;
}

// db[n] = sum_b dZ[b][n] over `rows` rows (one thread per n, 8 row phases).
__global__ void __launch_bounds__(256) wide_db_kernel(const float *__restrict__ dZ, int ldz,
                                                      int N, int64_t rows, float *__restrict__ db) {
  __shared__ float red[8][32];
  const int j = threadIdx.x & 31, ph = threadIdx.x >> 5;
  const int n = blockIdx.x * 32 + j;
  float t = 0.0f;
  if (n < N)
    for (int64_t b = ph; b < rows; b += 8) t += dZ[b * ldz + n];
  red[ph][j] = t;
  __syncthreads();
  if (ph == 0 && n < N) {
    float s = 0.0f;
    for (int q = 0; q < 8; ++q) s += red[q][j];
    db[n] = s;
  }
}

// dZ_prev[b][k] = (sum_n dZ[b][n] W[n][k]) * prelu'(pre[b][k]) for k < K, with
// the BF16 values of the FP32 masters W [N][K]; per-block partial sums of
// dX * min(pre, 0) over the batch rows b < batch (the slope's gradient).
// grid (rows/64, K/64), 256 threads with 4 x 4 outputs each.
__global__ void __launch_bounds__(256) wide_dx_kernel(const float *__restrict__ dZ, int ldz,
                                                      const float *__restrict__ W, int N, int K,
                                                      const float *__restrict__ pre, int ldp,
                                                      const float *__restrict__ slope,
                                                      int64_t batch, float *__restrict__ dZp,
                                                      int ldzp, float *__restrict__ slope_part) {
  __shared__ float sz[GT][GKC + 1];
  __shared__ float sw[GKC][GT + 4];
  __shared__ float red[8];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t b0 = (int64_t)blockIdx.x * GT;
  const int k0 = blockIdx.y * GT;
  float acc[4][4] = {};
  for (int n0 = 0; n0 < N; n0 += GKC) {
    for (int e = threadIdx.x; e < GT * GKC; e += 256) {
      const int i = e / GKC, j = e % GKC;
      sz[i][j] = (n0 + j < N) ? dZ[(b0 + i) * ldz + n0 + j] : 0.0f;
    }
    for (int e = threadIdx.x; e < GKC * GT; e += 256) {
      const int i = e / GT, j = e % GT;
      sw[i][j] = (n0 + i < N && k0 + j < K)
                     ? __bfloat162float(__float2bfloat16_rn(W[(size_t)(n0 + i) * K + k0 + j]))
                     : 0.0f;
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < GKC; ++j) {
      float a[4], w[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = sz[ty * 4 + r][j];
#pragma unroll
      for (int c = 0; c < 4; ++c) w[c] = sw[j][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], w[c], acc[r][c]);
    }
    __syncthreads();
  }
  const float a_l = __ldg(slope);
  float sp = 0.0f;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t b = b0 + ty * 4 + r;
      const int k = k0 + tx * 4 + c;
      if (k < K) {
        const float v = pre[b * ldp + k];
        if (b < batch) sp = fmaf(acc[r][c], fminf(v, 0.0f), sp);
        dZp[b * ldzp + k] = v > 0.0f ? acc[r][c] : a_l * acc[r][c];
      }
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sp += __shfl_down_sync(0xffffffffu, sp, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sp;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += red[w];
    slope_part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// out[0] = sum of the `count` partials (one block); FP32 or FP64 partials.
template <typename T, typename R>
__global__ void __launch_bounds__(256) wide_reduce_kernel(const T *__restrict__ part,
                                                          int64_t count, double scale, R *out) {
  __shared__ double red[8];
  double t = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += 256) t += (double)part[i];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    *out = (R)(s * scale);
  }
}

// Adam (Kingma and Ba, Alg. 1, bias-corrected, eps outside the root) over
// the flat parameter vector; omb1 = 1 - beta1 and omb2 = 1 - beta2 from FP64.
__global__ void __launch_bounds__(256) wide_adam_kernel(float *__restrict__ P,
                                                        const float *__restrict__ G,
                                                        float *__restrict__ M,
                                                        float *__restrict__ V, int64_t n, float lr,
                                                        float b1, float b2, float omb1, float omb2,
                                                        float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = fmaf(b1, M[i], omb1 * g);
  const float v = fmaf(b2, V[i], omb2 * g * g);
  M[i] = m;
  V[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// BF16 image and bias array of one layer from the flat masters (the padding
// stays zero); layer 0 repeats its weights for the inputs' low parts.
__global__ void __launch_bounds__(256) wide_pack_kernel(const float *__restrict__ W,
                                                        const float *__restrict__ b, int N, int K,
                                                        int N_pad, int first,
                                                        __nv_bfloat16 *__restrict__ img,
                                                        float *__restrict__ bias) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) bias[i] = b[i];
  if (i >= (int64_t)N * K) return;
  const int n = (int)(i / K), k = (int)(i % K);
  const __nv_bfloat16 v = __float2bfloat16_rn(W[i]);
  img[wide_weight_offset_dev(n, k, N_pad) / 2] = v;
  if (first) img[wide_weight_offset_dev(n, 8 + k, N_pad) / 2] = v;
}

}  // namespace

size_t wide_weight_offset(int n, int k, int N_pad) { return wide_weight_offset_dev(n, k, N_pad); }

cudaError_t wide_mlp_configure() {
  for (auto f : {wide_layer_kernel<WL_HIDDEN>, wide_layer_kernel<WL_HIDDEN_TRAIN>,
                 wide_layer_kernel<WL_LAST>, wide_layer_kernel<WL_LAST_TRAIN>}) {
    cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One chunk of particles (n <= RT * 128) through the network. act0/act1:
// ping-pong activation buffers of RT * max(K_pad) * 128 * 2 bytes.
cudaError_t launch_wide_pack(const WideNet &net, cudaStream_t st) {
  for (size_t l = 0; l < net.layers.size(); ++l) {
    const WideNet::Layer &ly = net.layers[l];
    const int64_t cnt = std::max<int64_t>((int64_t)ly.N * ly.K, ly.N);
    wide_pack_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(
        net.P + net.w_off[l], net.P + net.b_off[l], ly.N, ly.K, ly.N_pad, l == 0 ? 1 : 0,
        reinterpret_cast<__nv_bfloat16 *>(ly.W), ly.b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {
constexpr int WG_SPLITS = 4;  // batch slices of the weight-gradient GEMM

// Work buffers of a training step, carved from one workspace.
struct WideTrainBufs {
  std::vector<uint8_t *> act;  // per layer: its tiled BF16 input
  std::vector<float *> pre;    // per hidden layer: FP32 pre-activations
  float *Y = nullptr, *dY = nullptr, *dz[2] = {nullptr, nullptr}, *part = nullptr;
  float *spart = nullptr;
  double *lpart = nullptr;
  size_t bytes = 0;
};

WideTrainBufs wide_train_layout(const WideNet &net, int64_t batch, uint8_t *base) {
  WideTrainBufs b;
  const int64_t rows = (batch + BM - 1) / BM * BM;
  size_t off = 0;
  auto take = [&](size_t n) {
    uint8_t *p = base ? base + off : nullptr;
    off += (n + 255) / 256 * 256;
    return p;
  };
  const size_t L = net.layers.size();
  size_t max_nk = 0;
  for (size_t l = 0; l < L; ++l) {
    const auto &ly = net.layers[l];
    b.act.push_back(take((size_t)rows * ly.K_pad * 2));
    if (l + 1 < L) b.pre.push_back(reinterpret_cast<float *>(take((size_t)rows * ly.N_pad * 4)));
    max_nk = std::max(max_nk, (size_t)ly.N * ly.K);
  }
  b.Y = reinterpret_cast<float *>(take((size_t)rows * 8 * 4));
  b.dY = reinterpret_cast<float *>(take((size_t)rows * 8 * 4));
  for (int i = 0; i < 2; ++i)
    b.dz[i] = reinterpret_cast<float *>(take((size_t)rows * net.max_width * 4));
  b.part = reinterpret_cast<float *>(take((size_t)WG_SPLITS * max_nk * 4));
  b.spart = reinterpret_cast<float *>(take((size_t)(rows / GT + 1) * (net.max_width / GT + 1) * 4));
  b.lpart = reinterpret_cast<double *>(take((size_t)(rows / 256 + 1) * 8));
  b.bytes = off;
  return b;
}
}  // namespace

size_t wide_train_bytes(const WideNet &net, int64_t batch) {
  return wide_train_layout(net, batch, nullptr).bytes;
}

cudaError_t launch_wide_grad(const WideNet &net, const float *in, const float *out, int64_t ld,
                             const int64_t *idx, int64_t batch, float *G, float *loss_out,
                             void *ws, int num_sms, unsigned *err, cudaStream_t st) {
  const WideTrainBufs B = wide_train_layout(net, batch, static_cast<uint8_t *>(ws));
  const int RT = (int)((batch + BM - 1) / BM);
  const int64_t rows = (int64_t)RT * BM;
  const MlpNormF nrm = norm_pairs(net.nrm);
  Soa<float> si, so;
  for (int c = 0; c < 6; ++c) {
    si.c[c] = const_cast<float *>(in) + c * ld;
    so.c[c] = const_cast<float *>(out) + c * ld;
  }
  cudaError_t e;
  wide_train_prep_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(si, idx, batch, RT,
                                                                         B.act[0], nrm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int L = (int)net.layers.size();
  for (int l = 0; l < L; ++l) {
    const WideNet::Layer &ly = net.layers[l];
    WideLayer p{};
    p.A = B.act[l];
    p.B = ly.W;
    p.bias = ly.b;
    p.slope = ly.slope;
    p.C = (l + 1 < L) ? B.act[l + 1] : nullptr;
    p.KT = ly.K_pad / BK;
    p.N_pad = ly.N_pad;
    p.RT = RT;
    p.n = rows;
    p.nrm = nrm;
    p.pre = (l + 1 < L) ? B.pre[l] : nullptr;
    p.Y = B.Y;
    const int64_t units = (int64_t)RT * ((ly.N_pad + BN_MAX - 1) / BN_MAX);
    const unsigned grid = (unsigned)(units < num_sms ? units : num_sms);
    if (l + 1 < L)
      wide_layer_kernel<WL_HIDDEN_TRAIN><<<grid, THREADS, SMEM_BYTES, st>>>(p, err);
    else
      wide_layer_kernel<WL_LAST_TRAIN><<<grid, THREADS, SMEM_BYTES, st>>>(p, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // loss and dY (the targets' 1/sd as double-float pairs)
  InvSd isd;
  for (int c = 0; c < 6; ++c) {
    const double v = 1.0 / net.nrm.sd_out[c];
    isd.v[2 * c] = (float)v;
    isd.v[2 * c + 1] = (float)(v - (double)isd.v[2 * c]);
  }
  const unsigned lblocks = (unsigned)((rows + 255) / 256);
  wide_loss_kernel<<<lblocks, 256, 0, st>>>(B.Y, so, idx, batch, rows, nrm, isd, B.dY, B.lpart);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (loss_out) {
    wide_reduce_kernel<double, float><<<1, 256, 0, st>>>(B.lpart, lblocks,
                                                         1.0 / (6.0 * (double)batch), loss_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // backward
  const float *dz = B.dY;
  int ldz = 8, cur = 0;
  for (int l = L - 1; l >= 0; --l) {
    const WideNet::Layer &ly = net.layers[l];
    dim3 gw((ly.N + GT - 1) / GT, (ly.K + GT - 1) / GT, WG_SPLITS);
    wide_dw_kernel<<<gw, 256, 0, st>>>(dz, ldz, B.act[l], ly.K_pad / BK, ly.N, ly.K,
                                       rows / WG_SPLITS, l == 0 ? 1 : 0, B.part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t nk = (int64_t)ly.N * ly.K;
    wide_sum_splits_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(B.part, WG_SPLITS, nk,
                                                                         G + net.w_off[l]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    wide_db_kernel<<<(unsigned)((ly.N + 31) / 32), 256, 0, st>>>(dz, ldz, ly.N, rows,
                                                                G + net.b_off[l]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (l == 0) break;
    dim3 gx((unsigned)(rows / GT), (ly.K + GT - 1) / GT);
    float *dzp = B.dz[cur];
    wide_dx_kernel<<<gx, 256, 0, st>>>(dz, ldz, net.P + net.w_off[l], ly.N, ly.K, B.pre[l - 1],
                                       net.layers[l - 1].N_pad, net.layers[l - 1].slope, batch,
                                       dzp, net.max_width, B.spart);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    wide_reduce_kernel<float, float><<<1, 256, 0, st>>>(B.spart, (int64_t)gx.x * gx.y, 1.0,
                                                        G + net.slope_off + (l - 1));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dz = dzp;
    ldz = net.max_width;
    cur ^= 1;
  }
  return cudaSuccess;
}

cudaError_t launch_wide_adam(float *P, const float *G, float *M, float *V, int64_t n, double lr,
                             double b1, double b2, double eps, int step, cudaStream_t st) {
  const double c1 = 1.0 - std::pow(b1, (double)step), c2 = 1.0 - std::pow(b2, (double)step);
  wide_adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      P, G, M, V, n, (float)lr, (float)b1, (float)b2, (float)(1.0 - b1), (float)(1.0 - b2),
      (float)eps, (float)c1, (float)c2);
  return cudaGetLastError();
}

cudaError_t launch_wide_mlp(Soa<float> z, int64_t n, const WideNet &net, uint8_t *act0,
                            uint8_t *act1, int num_sms, unsigned *err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int RT = (int)((n + BM - 1) / BM);
  const MlpNormF nrm = norm_pairs(net.nrm);
  {
    const int64_t threads = (int64_t)RT * BM;
    wide_prep_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(z, n, RT, act0, nrm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  uint8_t *src = act0, *dst = act1;
  const int L = (int)net.layers.size();
  for (int l = 0; l < L; ++l) {
    const WideNet::Layer &ly = net.layers[l];
    WideLayer p{};
    p.A = src;
    p.B = ly.W;
    p.bias = ly.b;
    p.slope = ly.slope;
    p.C = dst;
    p.KT = ly.K_pad / BK;
    p.N_pad = ly.N_pad;
    p.RT = RT;
    p.z = z;
    p.n = n;
    p.nrm = nrm;
    const int64_t units = (int64_t)RT * ((ly.N_pad + BN_MAX - 1) / BN_MAX);
    const unsigned grid = (unsigned)(units < num_sms ? units : num_sms);
    if (l + 1 < L)
      wide_layer_kernel<WL_HIDDEN><<<grid, THREADS, SMEM_BYTES, st>>>(p, err);
    else
      wide_layer_kernel<WL_LAST><<<grid, THREADS, SMEM_BYTES, st>>>(p, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint8_t *t = src;
    src = dst;
    dst = t;
  }
  return cudaSuccess;
}

}  // namespace bl
