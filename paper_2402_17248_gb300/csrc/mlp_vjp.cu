// Vector-Jacobian product of the stage surrogate on the tensor cores: for
// every particle, given the adjoint lambda_out = dJ/dz_out of its stage-exit
// coordinates and its stage-entry coordinates z_in (the checkpoint), replace
// lambda_out in place by lambda_in = (dF/dz_in)^T lambda_out. This is the
// reverse sweep through a surrogate stage of the beamline gradient (Sec. 4.4
// optimises the focusing lattice by repeated tracking; the adjoint gives the
// gradient of the final moments with respect to the quadrupole strengths in
// one forward and one reverse pass).
//
// Per 128-particle tile, one CTA per SM:
//  * forward: the network's layers 0..3 exactly as the inference kernel
//    computes them (same BF16 rounding points, FP32 accumulators, tanh.approx
//    GELU), keeping h'(z_l) = 2 GELU'(z_l) of hidden layers 0..2 in tensor
//    memory in FP32 (the hidden activations are stored as 2 GELU and the
//    weight image holds W/2, so h' is the matching factor); the output layer
//    itself is not needed;
//  * the last hidden layer's adjoint g_3 = (W_4^T lambda_y) * h'(z_3) is
//    formed on the CUDA cores right where z_3 is read (W_4 has 6 rows), so
//    h'(z_3) is never stored;
//  * reverse: delta_{l-1} = W_l^T g_l by tcgen05.mma with the SAME
//    shared-memory weight image read as an MN-major B operand (instruction
//    descriptor bit 16; the descriptor's leading offset is then the
//    K-direction stride and the stride offset the N-direction stride), and
//    g_{l-1} = delta_{l-1} * h'(z_{l-1}) in FP32. Each g enters the MMA split
//    into three BF16 terms (hi + mid + lo = the FP32 value to 24 bits) and
//    the weights are BF16 values, so the products are exact and the reverse
//    sweep has the precision of an FP32 evaluation;
//  * lambda_in = (W_0^T g_0) / sd_in for the six inputs.
// The MMAs of a tile are issued by one lane of the MMA warp; two epilogue
// warpgroups own 64 features each and hand the accumulator and the operand
// buffers back and forth through mbarriers, as in the inference kernel.
#include "mlp_common.cuh"

namespace bl {

namespace {

using namespace mlp;

constexpr int EPI_THREADS = 256;                 // two warpgroups, 64 features each
constexpr int THREADS = EPI_THREADS + 32;        // + the MMA warp
constexpr int MMA_WARP = EPI_THREADS / 32;
constexpr uint32_t BUF_BYTES = 128 * 128 * 2;    // one BF16 [128 x 128] operand
constexpr uint32_t OFF_G = (MLP_IMG_BYTES + 1023) / 1024 * 1024;  // act / g hi, mid, lo
constexpr uint32_t OFF_ONES = OFF_G + 3 * BUF_BYTES;
constexpr uint32_t OFF_BAR = OFF_ONES + 128 * 16 * 2;  // weights, mma-done, epi-done
constexpr uint32_t OFF_SLOT = OFF_BAR + 8 * 3;
constexpr uint32_t SMEM_BYTES = (OFF_SLOT + 4 + 127) / 128 * 128;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");
static_assert(SMEM_BYTES > 114 * 1024, "one CTA per SM (it owns all tensor memory)");
// Tensor memory: accumulator in columns [0, 128); h'(z_l) of hidden layer
// l = 0, 1, 2 (FP32) in columns [128 (l + 1), 128 (l + 2)).
constexpr uint32_t TMEM_COLS = 512;
constexpr int NSPLIT = 3;  // BF16 terms per FP32 adjoint value

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

// Three-term BF16 split of an FP32 pair: v = hi + mid + lo to 24 bits.
BL_DEV void split3_pair(float v0, float v1, uint32_t &hi, uint32_t &mid, uint32_t &lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(v1), "f"(v0));
  v0 -= __uint_as_float(hi << 16);
  v1 -= __uint_as_float(hi & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(mid) : "f"(v1), "f"(v0));
  v0 -= __uint_as_float(mid << 16);
  v1 -= __uint_as_float(mid & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(v1), "f"(v0));
}

BL_DEV float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
BL_DEV float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// Store 16 adjoint values (features f .. f+15 of this thread's row) as three
// BF16 terms into the three operand buffers (row base `row`, K = 128 layout).
BL_DEV void store_g16(const float (&g)[16], uint32_t row, int f) {
  uint32_t hi[8], mid[8], lo[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) split3_pair(g[2 * j], g[2 * j + 1], hi[j], mid[j], lo[j]);
  const uint32_t a = row + (uint32_t)(f / 8) * 128, b = a + 128;
  tc::st_shared_v4(a, hi[0], hi[1], hi[2], hi[3]);
  tc::st_shared_v4(b, hi[4], hi[5], hi[6], hi[7]);
  tc::st_shared_v4(a + BUF_BYTES, mid[0], mid[1], mid[2], mid[3]);
  tc::st_shared_v4(b + BUF_BYTES, mid[4], mid[5], mid[6], mid[7]);
  tc::st_shared_v4(a + 2 * BUF_BYTES, lo[0], lo[1], lo[2], lo[3]);
  tc::st_shared_v4(b + 2 * BUF_BYTES, lo[4], lo[5], lo[6], lo[7]);
}

__global__ void __launch_bounds__(THREADS, 1)
mlp_vjp_kernel(Soa<float> zin, Soa<float> lam, int64_t n, int64_t ntiles,
               const uint8_t *__restrict__ img, MlpNormF nrm, unsigned *err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + OFF_SLOT);
  const uint32_t sbase = tc::smem_u32(smem);
  const uint32_t bar_w = sbase + OFF_BAR, bar_mma = bar_w + 8, bar_epi = bar_w + 16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_mma, 1);
    tc::mbar_init(bar_epi, EPI_THREADS);
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
  if (tid == 0) load_weights(sbase, img, bar_w);

  if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      bool ok = tc::mbar_wait(bar_w, 0, BL_DEVERR_TMA_TIMEOUT, err);
      uint32_t ph = 0;
      constexpr uint32_t ID_H = tc::idesc_bf16(128, 128);
      constexpr uint32_t ID_BH = tc::idesc_bf16(128, 128) | (1u << 16);  // B MN-major
      constexpr uint32_t ID_BO = tc::idesc_bf16(128, 16) | (1u << 16);
      constexpr uint64_t BUF_STEP = BUF_BYTES >> 4;
      // forward operands (K-major, as in the inference kernel)
      const uint64_t d_ones = tc::sdesc(sbase + OFF_ONES, 128, 256);
      const uint64_t d_w0 = tc::sdesc(sbase + OFF_W0, 128, 256);
      const uint64_t d_w1 = tc::sdesc(sbase + OFF_W1, 128, 2048);
      const uint64_t d_b1 = tc::sdesc(sbase + OFF_B1, 128, 256);
      const uint64_t d_in = tc::sdesc(sbase + OFF_G, 128, 256);    // K = 16 rows
      const uint64_t d_g = tc::sdesc(sbase + OFF_G, 128, 2048);    // K = 128 rows
      // reverse operands: the weight image read MN-major (B[k = out][n = in]):
      // leading offset = K-direction (out) stride, stride offset = 128 bytes
      const uint64_t r_w1 = tc::sdesc(sbase + OFF_W1, 2048, 128);  // W1..W3: K step 4096 B
      const uint64_t r_w0 = tc::sdesc(sbase + OFF_W0, 256, 128);   // N = 16, K step 512 B
      for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
#pragma unroll
        for (int ph_i = 0; ph_i < 8; ++ph_i) {
          if (!ok) break;
          ok = tc::mbar_wait(bar_epi, ph, BL_DEVERR_MMA_TIMEOUT, err);
          ph ^= 1u;
          if (!ok) break;
          tc::fence_after();
          if (ph_i == 0) {  // layer 0 forward
            tc::mma_ss(tmem, d_in, d_w0, ID_H, 0);
          } else if (ph_i <= 3) {  // layers 1..3 forward
            const int l = ph_i;
            const uint64_t dw = d_w1 + (uint64_t)((l - 1) * (MLP_IMG_WH >> 4));
#pragma unroll
            for (int j = 0; j < 8; ++j) tc::mma_ss(tmem, d_g + 16 * j, dw + 16 * j, ID_H, j > 0);
            tc::mma_ss(tmem, d_ones, d_b1 + (uint64_t)((l - 1) * (MLP_IMG_BH >> 4)), ID_H, 1);
          } else if (ph_i <= 6) {  // delta_{l-1} = W_l^T g_l, l = 3, 2, 1
            const int l = 7 - ph_i;
            const uint64_t rw = r_w1 + (uint64_t)((l - 1) * (MLP_IMG_WH >> 4));
#pragma unroll
            for (int s_ = 0; s_ < NSPLIT; ++s_)
#pragma unroll
              for (int j = 0; j < 8; ++j)
                tc::mma_ss(tmem, d_g + s_ * BUF_STEP + 16 * j, rw + 256 * j, ID_BH, s_ + j > 0);
          } else {  // lambda_x = W0^T g_0 (N = 16)
#pragma unroll
            for (int s_ = 0; s_ < NSPLIT; ++s_)
#pragma unroll
              for (int j = 0; j < 8; ++j)
                tc::mma_ss(tmem, d_g + s_ * BUF_STEP + 16 * j, r_w0 + 32 * j, ID_BO, s_ + j > 0);
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
    const int m = wq * 32 + lane;
    const uint32_t t_row = tmem + ((uint32_t)(wq * 32) << 16);
    const uint32_t row_in = sbase + OFF_G + (uint32_t)((m >> 3) * 256 + (m & 7) * 16);
    const uint32_t row_g = sbase + OFF_G + (uint32_t)((m >> 3) * 2048 + (m & 7) * 16);
    const uint8_t *w4 = smem + OFF_W4;  // [16 out][128 in], K-major core matrices
    bool ok = __all_sync(0xffffffffu, tc::mbar_wait(bar_w, 0, BL_DEVERR_TMA_TIMEOUT, err));
    uint32_t ph = 0;
    auto done = [&]() {
      tc::tmem_st_wait();
      tc::fence_proxy_async();
      tc::fence_before();
      mbar_arrive(bar_epi);
    };
    auto wait_mma = [&]() {
      ok = ok && __all_sync(0xffffffffu, tc::mbar_wait(bar_mma, ph, BL_DEVERR_MMA_TIMEOUT, err));
      ph ^= 1u;
      tc::fence_after();
    };
    for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
      const int64_t p = t * 128 + m;
      const bool valid = p < n;
      if (io) {  // normalised BF16 input row (bias hi/lo columns k = 6, 7)
        float xn[6];
#pragma unroll
        for (int c = 0; c < 6; ++c)
          xn[c] = df_normalise(valid ? zin.c[c][p] : 0.0f, nrm.mu_in[c][0], nrm.mu_in[c][1],
                               nrm.inv_sd_in[c][0], nrm.inv_sd_in[c][1]);
        uint32_t w[8];
        input_row(xn, w);
        tc::st_shared_v4(row_in, w[0], w[1], w[2], w[3]);
        tc::st_shared_v4(row_in + 128, w[4], w[5], w[6], w[7]);
      }
      done();
      // ---- forward: hidden layers 0..2 (activations and h' kept)
#pragma unroll 1
      for (int l = 0; l < 3 && ok; ++l) {
        wait_mma();
        if (!ok) break;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int f = 64 * h + 16 * c;
          uint32_t r[16];
          tc::tmem_ld16(t_row + f, r);
          tc::tmem_ld_wait_regs(r);
          uint32_t a[8], hp[16];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float d0, d1;
            gelu2_and_deriv(r[2 * j], r[2 * j + 1], a[j], d0, d1);
            hp[2 * j] = __float_as_uint(d0);
            hp[2 * j + 1] = __float_as_uint(d1);
          }
          tc::st_shared_v4(row_g + (uint32_t)(f / 8) * 128, a[0], a[1], a[2], a[3]);
          tc::st_shared_v4(row_g + (uint32_t)(f / 8 + 1) * 128, a[4], a[5], a[6], a[7]);
          tc::tmem_st16(t_row + 128 * (l + 1) + f, hp);
        }
        done();
      }
      // ---- hidden layer 3: g_3 = (W4^T lambda_y) * h'(z_3) on the CUDA cores
      if (!ok) break;
      wait_mma();
      if (!ok) break;
      {
        float ly[6];  // output adjoint in normalised units
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const float v = valid ? lam.c[c][p] : 0.0f;
          ly[c] = fmaf(v, nrm.sd_out[c][1], v * nrm.sd_out[c][0]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int f = 64 * h + 16 * c;
          uint32_t r[16];
          tc::tmem_ld16(t_row + f, r);
          tc::tmem_ld_wait_regs(r);
          float g[16];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            uint32_t a_unused;
            gelu2_and_deriv(r[2 * j], r[2 * j + 1], a_unused, g[2 * j], g[2 * j + 1]);
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {  // 8 features per 16-byte row of W4
            float dl[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) dl[k] = 0.0f;
#pragma unroll
            for (int o = 0; o < 6; ++o) {
              const uint4 wv = *reinterpret_cast<const uint4 *>(w4 + img_off(o, f + 8 * q, 128));
              const uint32_t wr[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                dl[2 * k] = fmaf(bf16_lo(wr[k]), ly[o], dl[2 * k]);
                dl[2 * k + 1] = fmaf(bf16_hi(wr[k]), ly[o], dl[2 * k + 1]);
              }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) g[8 * q + k] *= dl[k];
          }
          store_g16(g, row_g, f);
        }
        done();
      }
      // ---- reverse: g_{l} = delta_{l} * h'(z_{l}), l = 2, 1, 0
#pragma unroll 1
      for (int l = 2; l >= 0 && ok; --l) {
        wait_mma();
        if (!ok) break;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int f = 64 * h + 16 * c;
          uint32_t r[16], hp[16];
          tc::tmem_ld16(t_row + f, r);
          tc::tmem_ld16(t_row + 128 * (l + 1) + f, hp);
          tc::tmem_ld_wait_regs(r);
          tc::tmem_ld_wait_regs(hp);
          float g[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) g[j] = __uint_as_float(r[j]) * __uint_as_float(hp[j]);
          store_g16(g, row_g, f);
        }
        done();
      }
      if (!ok) break;
      wait_mma();  // lambda_x = W0^T g_0 complete
      if (!ok) break;
      if (io) {
        uint32_t r[8];
        tc::tmem_ld8(t_row, r);
        tc::tmem_ld_wait();
        if (valid) {
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const float v = __uint_as_float(r[c]);
            lam.c[c][p] = fmaf(v, nrm.inv_sd_in[c][1], v * nrm.inv_sd_in[c][0]);
          }
        }
      }
      // the next tile's first write to the operand buffers follows this
      // tile's last MMA (waited for above)
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == MMA_WARP) tc::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

cudaError_t mlp_vjp_configure() {
  return cudaFuncSetAttribute(mlp_vjp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES);
}

cudaError_t launch_mlp_vjp(Soa<float> zin, Soa<float> lam, int64_t n, const uint8_t *img,
                           const MlpNorm &nrm64, int num_sms, unsigned *err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t ntiles = (n + 127) / 128;
  const int64_t grid = ntiles < num_sms ? ntiles : num_sms;
  mlp_vjp_kernel<<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(zin, lam, n, ntiles, img,
                                                              mlp::norm_pairs(nrm64), err);
  return cudaGetLastError();
}

}  // namespace bl
