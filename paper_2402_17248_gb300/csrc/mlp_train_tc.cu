// Training step of the stage surrogate on the tensor cores (Sec. 3: MSE on
// normalised pairs, minibatch gradient for Adam). One CTA per 128-sample
// tile of the batch computes the loss and the tile's gradient with respect to
// every weight and bias, in the flat parameter layout, as one partial row;
// reduce_adam_kernel (mlp_train.cu) sums the rows and applies Adam.
//
// Per tile:
//  * forward: layers 0..3 as the inference kernel computes them (same BF16
//    rounding points, FP32 accumulators, tanh.approx GELU); each hidden
//    layer's activation is also written to a global scratch tile (it is
//    needed again, in reverse order, for the weight gradients), and
//    h'(z_l) = 2 GELU'(z_l) of layers 0..2 stays in tensor memory (FP16);
//  * output layer, loss and delta_4 = dL/dy on the CUDA cores (6 outputs);
//    the last hidden layer's adjoint g_3 = (W_4^T delta_4) * h'(z_3) is
//    formed where z_3 is read again;
//  * reverse: g_{l-1} = (W_l^T g_l) * h'(z_{l-1}) by MMAs that read the
//    inference weight image as an MN-major operand, and the transposed
//    weight gradients dW_l^T = act_l^T g_l by MMAs that read the SAME
//    shared-memory buffers of act_l (reloaded from the scratch) and of g_l as
//    MN-major operands: the K dimension of these MMAs is the tile's 128
//    samples. Transposed, the accumulator's lane is an input feature, so the
//    readout stores of a warp are contiguous in the [out][in] flat layout.
//    Bias gradients sum_s g_l[s] are formed on the CUDA cores where g_l is
//    produced (a butterfly over each warp's 32 samples, then the 4 warps).
//    Adjoints enter the MMAs as BF16 hi + lo pairs (~16 significant bits).
// Hidden activations are stored as 2 GELU and the weight image holds W/2
// (the inference kernel's convention), so the weight gradients of layers
// 1..4 are half the MMA results; g_l is the true adjoint.
#include "mlp_common.cuh"

namespace bl {

namespace {

using namespace mlp;

constexpr int EPI_THREADS = 256;                 // two warpgroups, 64 features each
constexpr int THREADS = EPI_THREADS + 32;        // + the MMA warp
constexpr int MMA_WARP = EPI_THREADS / 32;
constexpr uint32_t BUF_BYTES = 128 * 128 * 2;    // one BF16 [128 x 128] operand
// The adjoint and activation buffers sit below the weight image, so that
// every operand descriptor's reach stays inside the allocation.
constexpr uint32_t OFF_GH = 0;                   // adjoint, BF16 hi term
constexpr uint32_t OFF_GL = OFF_GH + BUF_BYTES;  // adjoint, BF16 lo term
constexpr uint32_t OFF_ACT = OFF_GL + BUF_BYTES; // activation of the current layer
constexpr uint32_t OFF_IMG = OFF_ACT + BUF_BYTES;
constexpr uint32_t OFF_ONES = OFF_IMG + MLP_IMG_BYTES;
constexpr uint32_t OFF_DSUM = OFF_ONES + 128 * 16 * 2;  // [2][4 warps][128] bias sums
constexpr uint32_t OFF_RED = OFF_DSUM + 2 * 4 * 128 * 4;  // 128 x 6 floats + 4 doubles
constexpr uint32_t OFF_BAR = OFF_RED + 128 * 6 * 4 + 4 * 8;  // weights, mma, epi, reload, adj
constexpr uint32_t OFF_SLOT = OFF_BAR + 8 * 5;
constexpr uint32_t SMEM_BYTES = (OFF_SLOT + 4 + 127) / 128 * 128;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");
static_assert(OFF_IMG % 1024 == 0, "weight image alignment");
// Tensor memory: accumulator [0, 128) (rows = samples); h'(z_l), l = 0..2,
// as FP16 pairs at [128 + 64 l, 192 + 64 l); weight-gradient accumulator
// [320, 448) (rows = input features; for layer 0 rows = output features).
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_HP = 128, COL_DW = 320;
// global scratch per tile: act0 (K = 16 layout, 4 KB) then act1..act3 (32 KB each)
constexpr size_t SCRATCH_TILE = 4096 + 3 * 32768;

__host__ __device__ constexpr int woff(int l) {
  return l == 0 ? 0 : (l == 1 ? 896 : (l == 2 ? 17408 : (l == 3 ? 33920 : 50432)));
}
__host__ __device__ constexpr int boff(int l) {
  return l == 0 ? 768 : (l == 1 ? 17280 : (l == 2 ? 33792 : (l == 3 ? 50304 : 51200)));
}

// 2 GELU(x) rounded to BF16 and h'(x) = 2 GELU'(x) in FP32, for a pair of
// pre-activations. GELU'(x) = (1 + t)/2 + x (1 - t^2) u'(x) / 2 with
// t = tanh u(x), u(x) = c0 x + c1 x^3, u' = c0 + 3 c1 x^2.
BL_DEV void gelu2_and_deriv(uint32_t r0, uint32_t r1, uint32_t &act, float &h0, float &h1) {
  uint64_t x, x2, p, u, t, y, one, omt2, du, w, d;
  asm("mov.b64 %0, {%1,%2};" : "=l"(x) : "r"(r0), "r"(r1));
  asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(x2) : "l"(x));
  const uint64_t c1 = ((uint64_t)__float_as_uint(GELU_C1) << 32) | __float_as_uint(GELU_C1);
  const uint64_t c0 = ((uint64_t)__float_as_uint(GELU_C0) << 32) | __float_as_uint(GELU_C0);
  const uint64_t c13 =
      ((uint64_t)__float_as_uint(3.0f * GELU_C1) << 32) | __float_as_uint(3.0f * GELU_C1);
  one = ((uint64_t)__float_as_uint(1.0f) << 32) | __float_as_uint(1.0f);
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(p) : "l"(x2), "l"(c1), "l"(c0));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(u) : "l"(x), "l"(p));
  uint32_t ulo, uhi, tlo, thi;
  asm("mov.b64 {%0,%1}, %2;" : "=r"(ulo), "=r"(uhi) : "l"(u));
  asm("tanh.approx.f32 %0, %1;" : "=r"(tlo) : "r"(ulo));
  asm("tanh.approx.f32 %0, %1;" : "=r"(thi) : "r"(uhi));
  asm("mov.b64 %0, {%1,%2};" : "=l"(t) : "r"(tlo), "r"(thi));
  asm("fma.rn.f32x2 %0, %1, %2, %1;" : "=l"(y) : "l"(x), "l"(t));  // x (1 + t)
  uint32_t ylo, yhi;
  asm("mov.b64 {%0,%1}, %2;" : "=r"(ylo), "=r"(yhi) : "l"(y));
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(act) : "r"(yhi), "r"(ylo));
  const uint64_t nt = t ^ 0x8000000080000000ull;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(omt2) : "l"(nt), "l"(t), "l"(one));  // 1 - t^2
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(du) : "l"(x2), "l"(c13), "l"(c0));   // u'
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(w) : "l"(x), "l"(omt2));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(t), "l"(one));                  // 1 + t
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(w), "l"(du), "l"(d));
  asm("mov.b64 {%0,%1}, %2;" : "=f"(h0), "=f"(h1) : "l"(d));
}

// Two-term BF16 split of an FP32 pair: v = hi + lo to ~16 bits.
BL_DEV void split_pair(float v0, float v1, uint32_t &hi, uint32_t &lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(v1), "f"(v0));
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(v1 - h1), "f"(v0 - h0));
}

BL_DEV float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
BL_DEV float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

BL_DEV void f16x2_to_f32(uint32_t v, float &a, float &b) {
  asm("{\n .reg .f16 l, h;\n mov.b32 {l, h}, %2;\n cvt.f32.f16 %0, l;\n cvt.f32.f16 %1, h;\n}"
      : "=f"(a), "=f"(b)
      : "r"(v));
}

// 16 adjoint values (features f .. f+15 of this thread's sample row) as BF16
// hi/lo into the two adjoint buffers (K = 128 layout, row base `row`).
BL_DEV void store_g16(const float (&g)[16], uint32_t row, int f) {
  uint32_t hi[8], lo[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) split_pair(g[2 * j], g[2 * j + 1], hi[j], lo[j]);
  const uint32_t a = row + (uint32_t)(f / 8) * 128, b = a + 128;
  tc::st_shared_v4(a, hi[0], hi[1], hi[2], hi[3]);
  tc::st_shared_v4(b, hi[4], hi[5], hi[6], hi[7]);
  tc::st_shared_v4(a + BUF_BYTES, lo[0], lo[1], lo[2], lo[3]);
  tc::st_shared_v4(b + BUF_BYTES, lo[4], lo[5], lo[6], lo[7]);
}

// Sums of 16 per-sample values v[0..15] over the warp's 32 samples by a
// transposing butterfly (16 shuffles): each step halves the values a lane
// keeps and adds its partner's copy of them. Lanes 2i and 2i+1 end with the
// sum of value index 8 b4 + 4 b3 + 2 b2 + b1 (b = the lane's bits); the even
// lane stores it to dst[index].
BL_DEV void warp_colsum16(const float (&v)[16], int lane, float *dst) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool up = lane & 16;
    const float keep = up ? v[i + 8] : v[i], send = up ? v[i] : v[i + 8];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool up = lane & 8;
    const float keep = up ? a[i + 4] : a[i], send = up ? a[i] : a[i + 4];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool up = lane & 4;
    const float keep = up ? a[i + 2] : a[i], send = up ? a[i] : a[i + 2];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool up = lane & 2;
    const float keep = up ? a[1] : a[0], send = up ? a[0] : a[1];
    a[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
  if (!(lane & 1))
    dst[((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1)] =
        a[0];
}

BL_DEV void named_sync_epi() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

struct TrainArgs {
  Soa<float> zin, zout;   // sample columns (gathered through idx when idx != NULL)
  const int64_t *idx;
  int64_t batch, ntiles;
  const uint8_t *img;     // BF16 weight image (mlp_pack_kernel)
  const float *bias;      // FP32 bias block of the pack kernel (b4 at 384..389)
  MlpNormF nrm;
  float inv_sd_out[6][2];
  float two_inv_count6;   // 2 / (6 batch)
  float *part;            // [ntiles][MLP_PSTRIDE]
  double *loss_part;      // [ntiles]
  uint8_t *scratch;       // [ntiles][SCRATCH_TILE]
};

__global__ void __launch_bounds__(THREADS, 1) mlp_train_tc_kernel(TrainArgs a, unsigned *err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + OFF_SLOT);
  float *red = reinterpret_cast<float *>(smem + OFF_RED);            // [128][6]
  double *red_loss = reinterpret_cast<double *>(smem + OFF_RED + 128 * 6 * 4);
  float *dsum = reinterpret_cast<float *>(smem + OFF_DSUM);          // [2][4][128]
  const uint32_t sbase = tc::smem_u32(smem), simg = sbase + OFF_IMG;
  // bar_mma: forward and weight-gradient MMAs done; bar_adj: adjoint MMAs
  // (delta = W^T g) done; bar_epi: the epilogue has refilled the operands;
  // bar_ld: an activation reload has landed
  const uint32_t bar_w = sbase + OFF_BAR, bar_mma = bar_w + 8, bar_epi = bar_w + 16,
                 bar_ld = bar_w + 24, bar_adj = bar_w + 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_mma, 1);
    tc::mbar_init(bar_epi, EPI_THREADS);
    tc::mbar_init(bar_ld, 1);
    tc::mbar_init(bar_adj, 1);
    tc::fence_mbar_init();
  }
  if (warp == MMA_WARP) {
    tc::tmem_alloc(tc::smem_u32(tslot), TMEM_COLS);
    tc::tmem_relinquish();
  }
  init_ones(smem, OFF_ONES, tid, THREADS);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0) load_weights(simg, a.img, bar_w);

  if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      bool ok = tc::mbar_wait(bar_w, 0, BL_DEVERR_TMA_TIMEOUT, err);
      uint32_t ph = 0;
      constexpr uint32_t ID_H = tc::idesc_bf16(128, 128);
      constexpr uint32_t ID_BH = tc::idesc_bf16(128, 128) | (1u << 16);  // B MN-major
      // weight gradients: A and B both MN-major, K = the tile's samples
      constexpr uint32_t ID_DW = tc::idesc_bf16(128, 128) | (1u << 15) | (1u << 16);
      constexpr uint32_t ID_DW16 = tc::idesc_bf16(128, 16) | (1u << 15) | (1u << 16);
      const uint64_t d_ones = tc::sdesc(sbase + OFF_ONES, 128, 256);
      const uint64_t d_w0 = tc::sdesc(simg + OFF_W0, 128, 256);
      const uint64_t d_w1 = tc::sdesc(simg + OFF_W1, 128, 2048);
      const uint64_t d_b1 = tc::sdesc(simg + OFF_B1, 128, 256);
      const uint64_t d_in = tc::sdesc(sbase + OFF_GL, 128, 256);     // act0, K = 16 rows
      const uint64_t d_act = tc::sdesc(sbase + OFF_ACT, 128, 2048);  // act, K-major
      const uint64_t d_gk = tc::sdesc(sbase + OFF_GH, 128, 2048);    // g, K-major
      const uint64_t r_w1 = tc::sdesc(simg + OFF_W1, 2048, 128);     // weights, MN-major
      // the same buffers read MN-major: leading offset = sample-direction
      // stride, stride offset = feature-direction stride
      const uint64_t m_g = tc::sdesc(sbase + OFF_GH, 2048, 128);
      const uint64_t m_act = tc::sdesc(sbase + OFF_ACT, 2048, 128);
      const uint64_t m_act0 = tc::sdesc(sbase + OFF_ACT, 256, 128);  // K = 16 layout
      constexpr uint64_t G_STEP = BUF_BYTES >> 4;
      const uint32_t acc = tmem, dw = tmem + COL_DW;
      for (int64_t t = blockIdx.x; ok && t < a.ntiles; t += gridDim.x) {
#pragma unroll 1
        for (int b = 0; b < 9; ++b) {
          ok = tc::mbar_wait(bar_epi, ph, BL_DEVERR_MMA_TIMEOUT, err);
          ph ^= 1u;
          if (!ok) break;
          tc::fence_after();
          if (b == 0) {  // layer 0 forward
            tc::mma_ss(acc, d_in, d_w0, ID_H, 0);
          } else if (b <= 3) {  // layers 1..3 forward
            const uint64_t dwt = d_w1 + (uint64_t)((b - 1) * (MLP_IMG_WH >> 4));
            for (int j = 0; j < 8; ++j) tc::mma_ss(acc, d_act + 16 * j, dwt + 16 * j, ID_H, j > 0);
            tc::mma_ss(acc, d_ones, d_b1 + (uint64_t)((b - 1) * (MLP_IMG_BH >> 4)), ID_H, 1);
          } else if (b <= 7) {
            // b = 4..7, l = 4..1: dW_l^T = act_l^T g_l (N = 16 outputs for
            // l = 4), then for l = 3, 2, 1 delta_{l-1} = W_l^T g_l, each
            // group committed to its own barrier so that the epilogue reads
            // dW while the adjoint MMAs run
            const int l = 8 - b;
            const uint32_t id = (l == 4) ? ID_DW16 : ID_DW;
            for (int s_ = 0; s_ < 2; ++s_)
              for (int j = 0; j < 8; ++j)
                tc::mma_ss(dw, m_act + 256 * j, m_g + s_ * G_STEP + 256 * j, id, (s_ | j) != 0);
            if (l <= 3) {
              tc::mma_commit(bar_mma);
              const uint64_t rw = r_w1 + (uint64_t)((l - 1) * (MLP_IMG_WH >> 4));
              for (int s_ = 0; s_ < 2; ++s_)
                for (int j = 0; j < 8; ++j)
                  tc::mma_ss(acc, d_gk + s_ * G_STEP + 16 * j, rw + 256 * j, ID_BH, (s_ | j) != 0);
              tc::mma_commit(bar_adj);
              continue;
            }
          } else {  // dW0 = g_0^T act0 (rows = outputs; N = 16: inputs, bias columns)
            for (int s_ = 0; s_ < 2; ++s_)
              for (int j = 0; j < 8; ++j)
                tc::mma_ss(dw, m_g + s_ * G_STEP + 256 * j, m_act0 + 32 * j, ID_DW16, (s_ | j) != 0);
          }
          tc::mma_commit(bar_mma);
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------ epilogue warps
    const int h = warp >> 2, wq = warp & 3;
    const bool io = (h == 0);
    const int m = wq * 32 + lane;  // sample row (accumulator) / feature row (dW)
    const uint32_t t_row = tmem + ((uint32_t)(wq * 32) << 16);
    const uint32_t in_row = sbase + OFF_GL + (uint32_t)((m >> 3) * 256 + (m & 7) * 16);
    const uint32_t act_row = sbase + OFF_ACT + (uint32_t)((m >> 3) * 2048 + (m & 7) * 16);
    const uint32_t gh_row = sbase + OFF_GH + (uint32_t)((m >> 3) * 2048 + (m & 7) * 16);
    const uint8_t *w4 = smem + OFF_IMG + OFF_W4;  // [16 out][128 in] K-major (W4 / 2)
    // `ok` is kept equal across all 256 epilogue threads (every wait result
    // passes through a barrier AND), so they leave the loops together and no
    // named barrier is left waiting for a thread that has gone.
    bool ok = tc::named_bar_and(1, EPI_THREADS,
                                tc::mbar_wait(bar_w, 0, BL_DEVERR_TMA_TIMEOUT, err));
    uint32_t ph = 0, ph_ld = 0, ph_adj = 0;
    auto done = [&]() {
      tc::tmem_st_wait();
      tc::fence_proxy_async();  // operands written through the generic proxy
      tc::fence_before();
      mbar_arrive(bar_epi);
    };
    auto wait_mma = [&]() {
      const bool got = ok && tc::mbar_wait(bar_mma, ph, BL_DEVERR_MMA_TIMEOUT, err);
      ok = tc::named_bar_and(1, EPI_THREADS, got);
      ph ^= 1u;
      tc::fence_after();
    };
    auto wait_adj = [&]() {
      const bool got = ok && tc::mbar_wait(bar_adj, ph_adj, BL_DEVERR_MMA_TIMEOUT, err);
      ok = tc::named_bar_and(1, EPI_THREADS, got);
      ph_adj ^= 1u;
      tc::fence_after();
    };
    // a saved activation is reloaded into the activation buffer as soon as
    // the weight-gradient MMA that read the buffer has completed (thread 0
    // issues the copy); warp 0 waits for it before the epilogue hands the
    // buffers to the MMA warp, and a failed wait reaches the other threads
    // through the next wait_mma
    auto reload_issue = [&](const uint8_t *src, uint32_t bytes) {
      if (tid == 0) {
        tc::mbar_expect_tx(bar_ld, bytes);
        tc::bulk_g2s(sbase + OFF_ACT, src, bytes, bar_ld);
      }
    };
    auto reload_wait = [&]() {
      if (warp == 0) ok = tc::mbar_wait(bar_ld, ph_ld, BL_DEVERR_TMA_TIMEOUT, err) && ok;
      ph_ld ^= 1u;
    };
    // transposed weight-gradient readout of a layer l >= 1: accumulator row m
    // = input feature k, column j = output feature; the first warpgroup takes
    // columns [0, 64), the second [64, 128) (l = 4: the first, columns 0..5).
    // For each column the warp's 32 lanes store 32 consecutive floats.
    auto dwt_out = [&](float *P, int l) {
      const int n_out = (l == 4) ? 6 : 128;
      const int c0 = io ? 0 : 64, c1 = (l == 4) ? (io ? 16 : 0) : c0 + 64;
      float *row = P + woff(l) + m;
      for (int c = c0; c < c1; c += 16) {
        uint32_t r[16];
        tc::tmem_ld16(t_row + COL_DW + c, r);
        tc::tmem_ld_wait_regs(r);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c + j < n_out) row[(c + j) * 128] = 0.5f * __uint_as_float(r[j]);
      }
    };
    // bias gradient of the layer whose adjoint was stored one stage earlier:
    // the 4 warps' column sums from buffer `buf` (n features)
    auto db_out = [&](float *P, int l, int buf, int n) {
      if (tid < n) {
        const float *d = dsum + buf * 512;
        P[boff(l) + tid] = (d[tid] + d[128 + tid]) + (d[256 + tid] + d[384 + tid]);
      }
    };
    for (int64_t t = blockIdx.x; ok && t < a.ntiles; t += gridDim.x) {
      float *P = a.part + t * MLP_PSTRIDE;
      uint8_t *scr = a.scratch + t * SCRATCH_TILE;
      const int64_t s = t * 128 + m;
      const bool valid = s < a.batch;
      const int64_t col = valid ? (a.idx ? a.idx[s] : s) : 0;
      float tgt[6];
      // ---- inputs: normalised BF16 row into the K = 16 buffer and the scratch
      if (io) {
        float xn[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const float v = valid ? a.zin.c[c][col] : 0.0f;
          xn[c] = df_normalise(v, a.nrm.mu_in[c][0], a.nrm.mu_in[c][1], a.nrm.inv_sd_in[c][0],
                               a.nrm.inv_sd_in[c][1]);
          const float o = valid ? a.zout.c[c][col] : 0.0f;
          tgt[c] = df_normalise(o, a.nrm.mu_out[c][0], a.nrm.mu_out[c][1], a.inv_sd_out[c][0],
                                a.inv_sd_out[c][1]);
        }
        uint32_t w[8];
        input_row(xn, w);
        tc::st_shared_v4(in_row, w[0], w[1], w[2], w[3]);
        tc::st_shared_v4(in_row + 128, w[4], w[5], w[6], w[7]);
        uint8_t *g0 = scr + (m >> 3) * 256 + (m & 7) * 16;
        *reinterpret_cast<uint4 *>(g0) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(g0 + 128) = make_uint4(w[4], w[5], w[6], w[7]);
      }
      done();
      // ---- forward, hidden layers 0..2 (activations kept, h' in TMEM)
#pragma unroll 1
      for (int l = 0; l < 3 && ok; ++l) {
        wait_mma();
        if (!ok) break;
        uint8_t *gs = scr + 4096 + (size_t)l * 32768 + (m >> 3) * 2048 + (m & 7) * 16;
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          const int f = 64 * h + 16 * c;
          uint32_t r[16];
          tc::tmem_ld16(t_row + f, r);
          tc::tmem_ld_wait_regs(r);
          uint32_t av[8], hp[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float d0, d1;
            gelu2_and_deriv(r[2 * j], r[2 * j + 1], av[j], d0, d1);
            asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hp[j]) : "f"(d1), "f"(d0));
          }
          tc::st_shared_v4(act_row + (uint32_t)(f / 8) * 128, av[0], av[1], av[2], av[3]);
          tc::st_shared_v4(act_row + (uint32_t)(f / 8 + 1) * 128, av[4], av[5], av[6], av[7]);
          *reinterpret_cast<uint4 *>(gs + (f / 8) * 128) = make_uint4(av[0], av[1], av[2], av[3]);
          *reinterpret_cast<uint4 *>(gs + (f / 8 + 1) * 128) = make_uint4(av[4], av[5], av[6], av[7]);
          tc::tmem_st8(t_row + COL_HP + 64 * l + f / 2, hp);
        }
        done();
      }
      if (!ok) break;
      // ---- layer 3: act4 = 2 GELU(z3) into the buffer; output, loss and delta_4
      wait_mma();
      if (!ok) break;
      float y[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
      for (int c = 0; c < 4; ++c) {
        const int f = 64 * h + 16 * c;
        uint32_t r[16];
        tc::tmem_ld16(t_row + f, r);
        tc::tmem_ld_wait_regs(r);
        uint32_t av[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float d0, d1;
          gelu2_and_deriv(r[2 * j], r[2 * j + 1], av[j], d0, d1);
        }
        tc::st_shared_v4(act_row + (uint32_t)(f / 8) * 128, av[0], av[1], av[2], av[3]);
        tc::st_shared_v4(act_row + (uint32_t)(f / 8 + 1) * 128, av[4], av[5], av[6], av[7]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
          for (int o = 0; o < 6; ++o) {
            const uint4 wv = *reinterpret_cast<const uint4 *>(w4 + img_off(o, f + 8 * q, 128));
            const uint32_t wr[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              y[o] = fmaf(bf16_lo(wr[k]), bf16_lo(av[4 * q + k]), y[o]);
              y[o] = fmaf(bf16_hi(wr[k]), bf16_hi(av[4 * q + k]), y[o]);
            }
          }
        }
      }
      if (!io) {
#pragma unroll
        for (int o = 0; o < 6; ++o) red[m * 6 + o] = y[o];
      }
      named_sync_epi();
      float d4[6];
      if (io) {
        double lsum = 0.0;
#pragma unroll
        for (int o = 0; o < 6; ++o) {
          const float yo = y[o] + red[m * 6 + o] + __ldg(a.bias + 384 + o);
          const float diff = valid ? yo - tgt[o] : 0.0f;
          lsum += (double)diff * (double)diff;
          d4[o] = diff * a.two_inv_count6;
          red[m * 6 + o] = d4[o];  // the same thread read red[m] above
        }
        lsum = warp_sum(lsum);
        if (lane == 0) red_loss[wq] = lsum;
      }
      named_sync_epi();
      if (!io) {
#pragma unroll
        for (int o = 0; o < 6; ++o) d4[o] = red[m * 6 + o];
      }
      // the tile's saved activations (written above through the generic
      // proxy) are read back by bulk copies from the next stage on
      asm volatile("fence.proxy.async.global;" ::: "memory");
      {  // delta_4 (hi/lo) as adjoint rows: features 0..5, zeros elsewhere
        float g[16];
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          const int f = 64 * h + 16 * c;
#pragma unroll
          for (int j = 0; j < 16; ++j) g[j] = (f == 0 && j < 6) ? d4[j < 6 ? j : 0] : 0.0f;
          store_g16(g, gh_row, f);
          if (f == 0) warp_colsum16(g, lane, dsum + wq * 128);
        }
      }
      done();
      // ---- dW4 and db4 readout; g_3 = (W4^T delta_4) * h'(z_3); act3 reloaded
      wait_mma();
      if (!ok) break;
      reload_issue(scr + 4096 + 2 * 32768, 32768);  // act3
      dwt_out(P, 4);
      db_out(P, 4, 0, 6);
#pragma unroll 1
      for (int c = 0; c < 4; ++c) {
        const int f = 64 * h + 16 * c;
        uint32_t r[16];
        tc::tmem_ld16(t_row + f, r);
        tc::tmem_ld_wait_regs(r);
        float g[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          uint32_t unused;
          gelu2_and_deriv(r[2 * j], r[2 * j + 1], unused, g[2 * j], g[2 * j + 1]);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float dl[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int o = 0; o < 6; ++o) {
            const uint4 wv = *reinterpret_cast<const uint4 *>(w4 + img_off(o, f + 8 * q, 128));
            const uint32_t wr[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              dl[2 * k] = fmaf(bf16_lo(wr[k]), d4[o], dl[2 * k]);
              dl[2 * k + 1] = fmaf(bf16_hi(wr[k]), d4[o], dl[2 * k + 1]);
            }
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) g[8 * q + k] *= dl[k];
        }
        store_g16(g, gh_row, f);
        warp_colsum16(g, lane, dsum + 512 + wq * 128 + f);
      }
      reload_wait();
      done();
      // ---- layers 3, 2, 1: act_{l-1} reloaded and dW_l, db_l read out while
      // the adjoint MMA runs; then g_{l-1} = delta_{l-1} * h'
#pragma unroll 1
      for (int l = 3; l >= 1 && ok; --l) {
        wait_mma();  // dW_l done: the activation buffer is free
        if (!ok) break;
        if (l > 1) reload_issue(scr + 4096 + (size_t)(l - 2) * 32768, 32768);  // act_{l-1}
        else reload_issue(scr, 4096);                                           // act0 (K = 16)
        dwt_out(P, l);
        db_out(P, l, l & 1, 128);   // g_3, g_1: buffer 1; g_2: buffer 0
        wait_adj();  // delta_{l-1} done: the adjoint buffers are free
        if (!ok) break;
        const int nb = (l - 1) & 1;  // buffer for g_{l-1}'s sums (g_0: none)
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          const int f = 64 * h + 16 * c;
          uint32_t r[16], hp[8];
          tc::tmem_ld16(t_row + f, r);
          tc::tmem_ld8(t_row + COL_HP + 64 * (l - 1) + f / 2, hp);
          tc::tmem_ld_wait_regs(r);
          tc::tmem_ld_wait_regs(hp);
          float g[16];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float h0, h1;
            f16x2_to_f32(hp[j], h0, h1);
            g[2 * j] = __uint_as_float(r[2 * j]) * h0;
            g[2 * j + 1] = __uint_as_float(r[2 * j + 1]) * h1;
          }
          store_g16(g, gh_row, f);
          if (l > 1) warp_colsum16(g, lane, dsum + nb * 512 + wq * 128 + f);
        }
        reload_wait();
        done();
      }
      if (!ok) break;
      // ---- dW0 and db0 readout (columns 0..5 and 8..13: the inputs' high
      // and low parts, which share each weight; column 6: the bias, whose K
      // column holds 1) and the tile's loss
      wait_mma();
      if (!ok) break;
      if (io) {
        uint32_t r[16];
        tc::tmem_ld16(t_row + COL_DW, r);
        tc::tmem_ld_wait_regs(r);
#pragma unroll
        for (int k = 0; k < 6; ++k)
          P[woff(0) + m * 6 + k] = __fadd_rn(__uint_as_float(r[k]), __uint_as_float(r[8 + k]));
        P[boff(0) + m] = __uint_as_float(r[6]);
      }
      if (tid == 0) a.loss_part[t] = red_loss[0] + red_loss[1] + red_loss[2] + red_loss[3];
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == MMA_WARP) tc::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

size_t mlp_train_tc_scratch_bytes(int64_t batch) {
  return (size_t)((batch + 127) / 128) * SCRATCH_TILE;
}

cudaError_t mlp_train_tc_configure() {
  return cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES);
}

cudaError_t launch_mlp_grad_tc(const float *in, const float *out, int64_t ld, const int64_t *idx,
                               int64_t batch, const uint8_t *img, const float *bias,
                               const MlpNorm &nrm64, float *partials, double *loss_partials,
                               uint8_t *scratch, int num_sms, unsigned *err, cudaStream_t st,
                               int64_t scale_count) {
  if (batch <= 0) return cudaSuccess;
  TrainArgs a{};
  for (int c = 0; c < 6; ++c) {
    a.zin.c[c] = const_cast<float *>(in) + c * ld;
    a.zout.c[c] = const_cast<float *>(out) + c * ld;
    const double inv = 1.0 / nrm64.sd_out[c];
    a.inv_sd_out[c][0] = (float)inv;
    a.inv_sd_out[c][1] = (float)(inv - (double)a.inv_sd_out[c][0]);
  }
  a.idx = idx;
  a.batch = batch;
  a.ntiles = (batch + 127) / 128;
  a.img = img;
  a.bias = bias;
  a.nrm = norm_pairs(nrm64);
  a.two_inv_count6 = (float)(2.0 / (6.0 * (double)(scale_count > 0 ? scale_count : batch)));
  a.part = partials;
  a.loss_part = loss_partials;
  a.scratch = scratch;
  const int64_t grid = a.ntiles < num_sms ? a.ntiles : num_sms;
  mlp_train_tc_kernel<<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(a, err);
  return cudaGetLastError();
}

}  // namespace bl
