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
  cudaFree(m->net.P);
  cudaFree(m->G);
  cudaFree(m->M);
  cudaFree(m->V);
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
  for (int l = 0; l < L; ++l) {
    BL_CHECK(d->W[l] && d->b[l], "a layer's weights or biases are NULL");
    const int K = d->widths[l], N = d->widths[l + 1];
    for (size_t i = 0; i < (size_t)N * K; ++i)
      BL_CHECK(std::isfinite(d->W[l][i]), "weights must be finite");
    for (int n = 0; n < N; ++n) BL_CHECK(std::isfinite(d->b[l][n]), "biases must be finite");
  }
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  auto *m = new bl_wide_mlp_s();
  m->device = ctx->device;
  WideNet &net = m->net;
  // flat FP32 masters: W_0, b_0, ..., W_{L-1}, b_{L-1}, then the L-1 slopes
  std::vector<float> flat;
  for (int l = 0; l < L; ++l) {
    const int K = d->widths[l], N = d->widths[l + 1];
    net.w_off.push_back((int64_t)flat.size());
    flat.insert(flat.end(), d->W[l], d->W[l] + (size_t)N * K);
    net.b_off.push_back((int64_t)flat.size());
    flat.insert(flat.end(), d->b[l], d->b[l] + N);
  }
  net.slope_off = (int64_t)flat.size();
  flat.insert(flat.end(), d->slopes, d->slopes + (L - 1));
  net.nparam = (int64_t)flat.size();
  const size_t pb = flat.size() * sizeof(float);
  cudaError_t e = cudaMalloc(&net.P, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->G, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->M, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->V, pb);
  if (e == cudaSuccess) e = cudaMemcpy(net.P, flat.data(), pb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->M, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(m->V, 0, pb);
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    WideNet::Layer ly;
    ly.K = d->widths[l];
    ly.N = d->widths[l + 1];
    ly.K_pad = pad64(ly.K);
    ly.N_pad = pad64(ly.N);
    ly.slope = (l + 1 < L) ? net.P + net.slope_off + l : nullptr;
    e = cudaMalloc(&ly.W, (size_t)ly.K_pad * ly.N_pad * 2);
    if (e == cudaSuccess) e = cudaMalloc(&ly.b, (size_t)ly.N_pad * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(ly.W, 0, (size_t)ly.K_pad * ly.N_pad * 2);
    if (e == cudaSuccess) e = cudaMemset(ly.b, 0, (size_t)ly.N_pad * sizeof(float));
    net.layers.push_back(ly);
    net.max_width = std::max(net.max_width, std::max(ly.K_pad, ly.N_pad));
  }
  // the BF16 images from the masters (the first layer repeats its weights
  // for the inputs' low parts)
  if (e == cudaSuccess) e = launch_wide_pack(net, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_wide(m);
    return cuda_error(e, "wide network upload");
  }
  for (int c = 0; c < 6; ++c) {
    net.nrm.mu_in[c] = d->mu_in[c];
    net.nrm.inv_sd_in[c] = 1.0 / d->sd_in[c];
    net.nrm.mu_out[c] = d->mu_out[c];
    net.nrm.sd_out[c] = d->sd_out[c];
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
  const size_t bytes = (size_t)ch * m->net.max_width * 2;
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

bl_status bl_wide_mlp_num_params(const bl_wide_mlp *m, int64_t *n) {
  BL_CHECK(m && n, "NULL argument");
  *n = m->net.nparam;
  return BL_OK;
}

bl_status bl_wide_mlp_get_params(const bl_wide_mlp *m, float *const *W_out, float *const *b_out,
                                 float *slopes_out) {
  BL_CHECK(m && W_out && b_out && slopes_out, "NULL argument");
  const WideNet &net = m->net;
  const int L = (int)net.layers.size();
  for (int l = 0; l < L; ++l) BL_CHECK(W_out[l] && b_out[l], "a layer's output buffer is NULL");
  std::vector<float> flat((size_t)net.nparam);
  BL_CUDA(cudaDeviceSynchronize());
  BL_CUDA(cudaMemcpy(flat.data(), net.P, flat.size() * sizeof(float), cudaMemcpyDeviceToHost));
  for (int l = 0; l < L; ++l) {
    const auto &ly = net.layers[l];
    std::memcpy(W_out[l], flat.data() + net.w_off[l], (size_t)ly.N * ly.K * sizeof(float));
    std::memcpy(b_out[l], flat.data() + net.b_off[l], (size_t)ly.N * sizeof(float));
  }
  std::memcpy(slopes_out, flat.data() + net.slope_off, (size_t)(L - 1) * sizeof(float));
  return BL_OK;
}

namespace {

bl_status wide_grad_checks(const bl_wide_mlp *m, const float *in, const float *out, int64_t ld,
                           int64_t batch, DevCtx **ctx) {
  BL_CHECK(m, "network is NULL");
  BL_CHECK(in && out, "in and out must be device arrays");
  BL_CHECK(batch >= 1 && batch <= BL_WIDE_MAX_BATCH, "batch must be in [1, BL_WIDE_MAX_BATCH]");
  BL_CHECK(ld >= 1, "ld must be positive");
  BL_TRY(current_ctx(ctx));
  BL_CHECK((*ctx)->device == m->device, "network belongs to another device");
  if (!(*ctx)->wide_configured) {
    BL_CUDA(wide_mlp_configure());
    (*ctx)->wide_configured = true;
  }
  return BL_OK;
}

}  // namespace

bl_status bl_wide_mlp_grad(const bl_wide_mlp *m, const float *in, const float *out, int64_t ld,
                           const int64_t *idx, int64_t batch, float *grad_out, float *loss_out,
                           bl_stream stream) {
  DevCtx *ctx = nullptr;
  BL_TRY(wide_grad_checks(m, in, out, ld, batch, &ctx));
  BL_CHECK(grad_out, "grad_out is NULL");
  BL_CHECK(idx || batch <= ld, "without idx the batch is the first `batch` columns");
  cudaStream_t st = (cudaStream_t)stream;
  void *ws = nullptr;
  BL_TRY(ws_get(st, WS_WIDE_TRAIN, wide_train_bytes(m->net, batch), &ws));
  BL_CUDA(launch_wide_grad(m->net, in, out, ld, idx, batch, grad_out, loss_out, ws, ctx->num_sms,
                           ctx->err_word, st));
  return BL_OK;
}

bl_status bl_wide_mlp_train_step(bl_wide_mlp *m, const float *in, const float *out, int64_t ld,
                                 const int64_t *idx, int64_t batch, const bl_adam_cfg *cfg,
                                 float *loss_out, bl_stream stream) {
  DevCtx *ctx = nullptr;
  BL_TRY(wide_grad_checks(m, in, out, ld, batch, &ctx));
  BL_CHECK(cfg && cfg->lr > 0.0 && cfg->beta1 >= 0.0 && cfg->beta1 < 1.0 && cfg->beta2 >= 0.0 &&
               cfg->beta2 < 1.0 && cfg->eps > 0.0,
           "invalid Adam configuration");
  BL_CHECK(idx || batch <= ld, "without idx the batch is the first `batch` columns");
  cudaStream_t st = (cudaStream_t)stream;
  void *ws = nullptr;
  BL_TRY(ws_get(st, WS_WIDE_TRAIN, wide_train_bytes(m->net, batch), &ws));
  BL_CUDA(launch_wide_grad(m->net, in, out, ld, idx, batch, m->G, loss_out, ws, ctx->num_sms,
                           ctx->err_word, st));
  ++m->step;
  BL_CUDA(launch_wide_adam(m->net.P, m->G, m->M, m->V, m->net.nparam, cfg->lr, cfg->beta1,
                           cfg->beta2, cfg->eps, m->step, st));
  BL_CUDA(launch_wide_pack(m->net, st));
  return BL_OK;
}

}  // extern "C"
