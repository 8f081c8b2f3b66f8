// Device helpers and the shared-memory weight-image layout common to the
// surrogate inference kernel (mlp_fwd.cu) and its vector-Jacobian product
// (mlp_vjp.cu).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace bl {
namespace mlp {

// Byte offsets of the BF16 weight image (built by mlp_pack_kernel): W0, W1..W3,
// W4, then the bias blocks B1..B3, B4.
constexpr uint32_t OFF_W0 = 0;
constexpr uint32_t OFF_W1 = OFF_W0 + MLP_IMG_W0;
constexpr uint32_t OFF_W4 = OFF_W1 + 3 * MLP_IMG_WH;
constexpr uint32_t OFF_B1 = OFF_W4 + MLP_IMG_W4;
constexpr uint32_t OFF_B4 = OFF_B1 + 3 * MLP_IMG_BH;
static_assert(OFF_W4 == OFF_W1 + 3 * MLP_IMG_WH && OFF_B4 == OFF_B1 + 3 * MLP_IMG_BH, "image");

constexpr float GELU_C0 = 0.7978845608028654f;               // sqrt(2/pi)
constexpr float GELU_C1 = 0.7978845608028654f * 0.044715f;

// Byte offset of element (n, k) of an [N x K] K-major BF16 block in the
// no-swizzle core-matrix layout: 8x8 core matrices of 128 contiguous bytes,
// adjacent along K at 128 bytes, adjacent along N at (K/8)*128 bytes.
__host__ __device__ inline uint32_t img_off(int n, int k, int K) {
  return (uint32_t)((n >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2);
}

// Double-float helpers: a value v is carried as hi + lo (FP32 each). The
// additions and products that must round exactly once are written with the
// _rn intrinsics, which are never contracted into an fma.
BL_DEV void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// (z - mu) * inv with mu = mh + ml and inv = ih + il, rounded to FP32.
BL_DEV float df_normalise(float z, float mh, float ml, float ih, float il) {
  float dh, dl;
  two_sum(z, -mh, dh, dl);
  dl = __fsub_rn(dl, ml);
  const float p = __fmul_rn(dh, ih);
  const float pe = fmaf(dh, ih, -p);
  return __fadd_rn(p, __fadd_rn(pe, fmaf(dh, il, __fmul_rn(dl, ih))));
}

// y * sd + mu with sd = sh + sl and mu = mh + ml, rounded to FP32.
BL_DEV float df_affine(float y, float sh, float sl, float mh, float ml) {
  const float p = __fmul_rn(y, sh);
  const float pe = fmaf(y, sh, -p);
  float s, se;
  two_sum(p, mh, s, se);
  return __fadd_rn(s, __fadd_rn(__fadd_rn(se, pe), fmaf(y, sl, ml)));
}

// The K = 16 input row of the first layer as 8 packed BF16 pairs: columns
// 0..5 the BF16 high parts of the 6 normalised inputs, 6 and 7 the constant
// 1 that multiplies the bias hi/lo weights, 8..13 the inputs' low parts
// bf16(x - hi), 14 and 15 zero. The first layer's weights repeat in columns
// 8..13, so the MMA sees each input with 16 significant bits.
BL_DEV void input_row(const float (&xn)[6], uint32_t (&w)[8]) {
  float hi[6], lo[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    hi[c] = __bfloat162float(__float2bfloat16_rn(xn[c]));
    lo[c] = __fsub_rn(xn[c], hi[c]);
  }
  w[0] = tc::pack_bf16x2(hi[0], hi[1]);
  w[1] = tc::pack_bf16x2(hi[2], hi[3]);
  w[2] = tc::pack_bf16x2(hi[4], hi[5]);
  w[3] = tc::pack_bf16x2(1.0f, 1.0f);
  w[4] = tc::pack_bf16x2(lo[0], lo[1]);
  w[5] = tc::pack_bf16x2(lo[2], lo[3]);
  w[6] = tc::pack_bf16x2(lo[4], lo[5]);
  w[7] = 0u;
}

BL_DEV void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}


// Constant A operand of a bias K-step (128 rows of (1, 1, 0, ..., 0), K = 16,
// K-major core matrices) at shared-memory byte offset `off`; all threads of
// the block take part.
BL_DEV void init_ones(uint8_t *smem, uint32_t off, int tid, int nthreads) {
  for (int i = tid; i < 128 * 16; i += nthreads) {
    const int m = i / 16, k = i % 16;
    *reinterpret_cast<__nv_bfloat16 *>(smem + off + img_off(m, k, 16)) =
        __float2bfloat16_rn(k < 2 ? 1.0f : 0.0f);
  }
}

// One thread: bulk-copy the whole weight image to shared memory at `sbase`,
// completing MLP_IMG_BYTES of transactions on mbarrier `bar`.
BL_DEV void load_weights(uint32_t sbase, const uint8_t *img, uint32_t bar) {
  tc::mbar_expect_tx(bar, MLP_IMG_BYTES);
  tc::bulk_g2s(sbase + OFF_W0, img + OFF_W0, MLP_IMG_W0, bar);
  for (int l = 0; l < 3; ++l)
    tc::bulk_g2s(sbase + OFF_W1 + l * MLP_IMG_WH, img + OFF_W1 + l * MLP_IMG_WH, MLP_IMG_WH, bar);
  tc::bulk_g2s(sbase + OFF_W4, img + OFF_W4, MLP_IMG_W4 + 3 * MLP_IMG_BH + MLP_IMG_B4, bar);
}

// FP64 normalisation constants as double-float pairs (hi, lo).
inline MlpNormF norm_pairs(const MlpNorm &n64) {
  MlpNormF n;
  auto split = [](double v, float *hl) {
    hl[0] = (float)v;
    hl[1] = (float)(v - (double)hl[0]);
  };
  for (int c = 0; c < 6; ++c) {
    split(n64.mu_in[c], n.mu_in[c]);
    split(n64.inv_sd_in[c], n.inv_sd_in[c]);
    split(n64.mu_out[c], n.mu_out[c]);
    split(n64.sd_out[c], n.sd_out[c]);
  }
  return n;
}

}  // namespace mlp
}  // namespace bl
