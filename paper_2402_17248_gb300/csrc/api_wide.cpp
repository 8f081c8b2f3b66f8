// C ABI: the paper's wide PReLU surrogate networks (create, apply, destroy).
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>

#include "runtime.h"

using namespace bl;

namespace {

void free_wide(bl_wide_mlp_s *m) {
  if (!m) return;
  for (auto &l : m->net.layers) {
    cudaFree(l.W);
    cudaFree(l.b);
  }
  delete m;
}

int pad64(int v) { return (v + 63) / 64 * 64; }

}  // namespace

extern "C" {

bl_status bl_wide_mlp_create(const bl_wide_mlp_desc *d, bl_wide_mlp **out) {
  BL_CHECK(out, "out is NULL");
  *out = nullptr;
  BL_CHECK(d && d->widths && d->W && d->b, "descriptor or its arrays are NULL");
  const int L = d->n_layers;
  BL_CHECK(L >= 2 && L <= 64, "n_layers must be in [2, 64]");
  BL_CHECK(d->widths[0] == 6 && d->widths[L] == 6, "input and output widths must be 6");
  for (int l = 1; l < L; ++l)
    BL_CHECK(d->widths[l] >= 1 && d->widths[l] <= 4096, "hidden widths must be in [1, 4096]");
  BL_CHECK(d->slopes, "slopes is NULL");
  BL_CHECK(d->mu_in && d->sd_in && d->mu_out && d->sd_out, "normalisation constants are NULL");
  for (int c = 0; c < 6; ++c) {
    BL_CHECK(std::isfinite(d->mu_in[c]) && std::isfinite(d->mu_out[c]), "means must be finite");
    BL_CHECK(d->sd_in[c] > 0.0 && d->sd_out[c] > 0.0 && std::isfinite(d->sd_in[c]) &&
                 std::isfinite(d->sd_out[c]),
             "standard deviations must be positive and finite");
  }
  for (int l = 0; l + 1 < L; ++l) BL_CHECK(std::isfinite(d->slopes[l]), "slopes must be finite");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  auto *m = new bl_wide_mlp_s();
  m->device = ctx->device;
  for (int l = 0; l < L; ++l) {
    const int K = d->widths[l], N = d->widths[l + 1];
    BL_CHECK(d->W[l] && d->b[l], "a layer's weights or biases are NULL");
    WideNet::Layer ly;
    ly.K_pad = pad64(K);
    ly.N_pad = pad64(N);
    ly.slope = (l + 1 < L) ? d->slopes[l] : 0.0f;
    std::vector<__nv_bfloat16> img((size_t)ly.K_pad * ly.N_pad, __float2bfloat16_rn(0.0f));
    for (int n = 0; n < N; ++n)
      for (int k = 0; k < K; ++k) {
        const float w = d->W[l][(size_t)n * K + k];
        if (!std::isfinite(w)) {
          free_wide(m);
          return set_error(BL_ERR_INVALID_ARG, "weights must be finite");
        }
        img[wide_weight_offset(n, k, ly.N_pad) / 2] = __float2bfloat16_rn(w);
        // the first layer sees each input as a BF16 hi (column k) + lo
        // (column 8 + k) pair sharing the weight
        if (l == 0) img[wide_weight_offset(n, 8 + k, ly.N_pad) / 2] = __float2bfloat16_rn(w);
      }
    std::vector<float> bias(ly.N_pad, 0.0f);
    for (int n = 0; n < N; ++n) {
      if (!std::isfinite(d->b[l][n])) {
        free_wide(m);
        return set_error(BL_ERR_INVALID_ARG, "biases must be finite");
      }
      bias[n] = d->b[l][n];
    }
    cudaError_t e = cudaMalloc(&ly.W, img.size() * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&ly.b, bias.size() * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpy(ly.W, img.data(), img.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(ly.b, bias.data(), bias.size() * sizeof(float), cudaMemcpyHostToDevice);
    m->net.layers.push_back(ly);
    if (e != cudaSuccess) {
      free_wide(m);
      return cuda_error(e, "wide network upload");
    }
    m->max_width = std::max(m->max_width, std::max(ly.K_pad, ly.N_pad));
  }
  for (int c = 0; c < 6; ++c) {
    m->net.nrm.mu_in[c] = d->mu_in[c];
    m->net.nrm.inv_sd_in[c] = 1.0 / d->sd_in[c];
    m->net.nrm.mu_out[c] = d->mu_out[c];
    m->net.nrm.sd_out[c] = d->sd_out[c];
  }
  *out = m;
  return BL_OK;
}

bl_status bl_wide_mlp_destroy(bl_wide_mlp *m) {
  free_wide(m);
  return BL_OK;
}

bl_status bl_wide_mlp_apply(const bl_wide_mlp *m, bl_bunch *b, int64_t chunk, bl_stream stream) {
  std::string why;
  BL_CHECK(m, "network is NULL");
  BL_CHECK(bunch_dims_ok(b, &why), why);
  BL_CHECK(b->dtype == BL_F32, "the wide network needs an FP32 bunch");
  BL_CHECK(chunk >= 0, "chunk must be >= 0");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  BL_CHECK(ctx->device == m->device, "network belongs to another device");
  if (!ctx->wide_configured) {
    BL_CUDA(wide_mlp_configure());
    ctx->wide_configured = true;
  }
  const int64_t n = b->n;
  if (n == 0) return BL_OK;
  int64_t ch = chunk > 0 ? chunk : ((int64_t)1 << 21);
  ch = (std::min(ch, n) + 127) / 128 * 128;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)ch * m->max_width * 2;
  void *a0 = nullptr, *a1 = nullptr;
  BL_TRY(ws_get(st, WS_WIDE0, bytes, &a0));
  BL_TRY(ws_get(st, WS_WIDE1, bytes, &a1));
  Soa<float> z = soa_of<float>(b);
  for (int64_t off = 0; off < n; off += ch) {
    Soa<float> zc;
    for (int c = 0; c < 6; ++c) zc.c[c] = z.c[c] + off;
    BL_CUDA(launch_wide_mlp(zc, std::min(ch, n - off), m->net, (uint8_t *)a0, (uint8_t *)a1,
                            ctx->num_sms, ctx->err_word, st));
  }
  return BL_OK;
}

}  // extern "C"
