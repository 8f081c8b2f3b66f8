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

struct WideLayer {
  const uint8_t *A;     // activations of the chunk, tiled [RT][KT]
  const uint8_t *B;     // weights, tiled [KT][N_pad / 64]
  const float *bias;    // [N_pad]
  float slope;          // PReLU slope (hidden layers)
  uint8_t *C;           // next activations, tiled [RT][N_pad / 64] (hidden layers)
  int KT, N_pad, RT;
  Soa<float> z;         // output layer: particles of the chunk (in place)
  int64_t n;            // particles in the chunk
  MlpNormF nrm;
};

template <bool LAST>
__global__ void __launch_bounds__(THREADS, 1) wide_layer_kernel(WideLayer p, unsigned *err) {
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
#pragma unroll
          for (int g = 0; g < 4; ++g) {  // 8 columns = one 16-byte core-matrix row
            const float4 b0 = __ldg(bv + 2 * g), b1 = __ldg(bv + 2 * g + 1);
            const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
            uint32_t o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              float v0 = __uint_as_float(r[8 * g + 2 * j]) + bb[2 * j];
              float v1 = __uint_as_float(r[8 * g + 2 * j + 1]) + bb[2 * j + 1];
              v0 = v0 > 0.0f ? v0 : p.slope * v0;
              v1 = v1 > 0.0f ? v1 : p.slope * v1;
              o[j] = tc::pack_bf16x2(v0, v1);
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
        if (i < p.n) {
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

}  // namespace

size_t wide_weight_offset(int n, int k, int N_pad) {
  return ((size_t)(k >> 6) * (N_pad / 64) + (n >> 6)) * B_SUB + tile_off(n & 63, k & 63);
}

cudaError_t wide_mlp_configure() {
  cudaError_t e = cudaFuncSetAttribute(wide_layer_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(wide_layer_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES);
}

// One chunk of particles (n <= RT * 128) through the network. act0/act1:
// ping-pong activation buffers of RT * max(K_pad) * 128 * 2 bytes.
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
      wide_layer_kernel<false><<<grid, THREADS, SMEM_BYTES, st>>>(p, err);
    else
      wide_layer_kernel<true><<<grid, THREADS, SMEM_BYTES, st>>>(p, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint8_t *t = src;
    src = dst;
    dst = t;
  }
  return cudaSuccess;
}

}  // namespace bl
