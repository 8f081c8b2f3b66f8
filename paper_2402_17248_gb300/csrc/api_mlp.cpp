// C ABI: stage surrogates (create, inference, training, loss, parameters).
#include <cmath>

#include "runtime.h"

using namespace bl;

namespace {

const int kWidths[6] = {6, 128, 128, 128, 128, 6};

bl_status check_desc(const bl_mlp_desc *d) {
  BL_CHECK(d, "descriptor is NULL");
  BL_CHECK(d->n_layers == 5, "this build supports 5 layers (6-128-128-128-128-6)");
  BL_CHECK(d->widths, "widths is NULL");
  for (int i = 0; i < 6; ++i)
    BL_CHECK(d->widths[i] == kWidths[i], "this build supports widths 6-128-128-128-128-6");
  BL_CHECK(d->W && d->b, "weights or biases are NULL");
  for (int l = 0; l < 5; ++l) BL_CHECK(d->W[l] && d->b[l], "a layer's weights or biases are NULL");
  BL_CHECK(d->mu_in && d->sd_in && d->mu_out && d->sd_out, "normalisation constants are NULL");
  for (int c = 0; c < 6; ++c) {
    BL_CHECK(std::isfinite(d->mu_in[c]) && std::isfinite(d->mu_out[c]), "means must be finite");
    BL_CHECK(d->sd_in[c] > 0.0 && d->sd_out[c] > 0.0 && std::isfinite(d->sd_in[c]) &&
                 std::isfinite(d->sd_out[c]),
             "standard deviations must be positive and finite");
  }
  return BL_OK;
}

bl_status check_surrogate(const bl_surrogate *s) {
  BL_CHECK(s, "surrogate is NULL");
  int dev = -1;
  BL_CUDA(cudaGetDevice(&dev));
  BL_CHECK(dev == s->device, "surrogate belongs to another device");
  return BL_OK;
}

void free_surrogate(bl_surrogate_s *s) {
  if (!s) return;
  cudaFree(s->params);
  cudaFree(s->m);
  cudaFree(s->v);
  cudaFree(s->img);
  cudaFree(s->bias);
  cudaFree(s->wt);
  cudaFree(s->wn);
  delete s;
}

bl_status train_grad(bl_surrogate *s, const float *in, const float *out, int64_t ld,
                     const int64_t *idx, int64_t batch, float **part_out, double **lp_out,
                     int *nb_out, cudaStream_t st) {
  const int nb = mlp_grad_blocks(batch);
  void *part = nullptr, *lp = nullptr;
  BL_TRY(ws_get(st, WS_TRAIN, (size_t)nb * MLP_PSTRIDE * sizeof(float), &part));
  BL_TRY(ws_get(st, WS_LOSS, (size_t)nb * sizeof(double), &lp));
  int nb2 = 0;
  BL_CUDA(launch_mlp_grad(in, out, ld, idx, batch, s->wt, s->wn, s->nrm, (float *)part,
                          (double *)lp, &nb2, st));
  *part_out = (float *)part;
  *lp_out = (double *)lp;
  *nb_out = nb2;
  return BL_OK;
}

}  // namespace

extern "C" {

bl_status bl_surrogate_create(const bl_mlp_desc *d, bl_surrogate **out) {
  BL_CHECK(out, "out is NULL");
  *out = nullptr;
  BL_TRY(check_desc(d));
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  std::vector<float> flat(MLP_NPARAM);
  for (int l = 0; l < 5; ++l) {
    const int fi = kWidths[l], fo = kWidths[l + 1];
    for (int i = 0; i < fi * fo; ++i) {
      BL_CHECK(std::isfinite(d->W[l][i]), "weights must be finite");
      flat[mlp_w_off(l) + i] = d->W[l][i];
    }
    for (int i = 0; i < fo; ++i) {
      BL_CHECK(std::isfinite(d->b[l][i]), "biases must be finite");
      flat[mlp_b_off(l) + i] = d->b[l][i];
    }
  }
  auto *s = new bl_surrogate_s();
  s->device = ctx->device;
  auto fail = [&](cudaError_t e, const char *what) {
    free_surrogate(s);
    return cuda_error(e, what);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&s->params, MLP_NPARAM * sizeof(float))) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->m, MLP_NPARAM * sizeof(float))) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->v, MLP_NPARAM * sizeof(float))) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->img, MLP_IMG_BYTES)) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->bias, MLP_BIAS_FLOATS * sizeof(float))) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->wt, MLP_NPARAM * sizeof(float))) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->wn, MLP_NPARAM * sizeof(float))) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMemcpy(s->params, flat.data(), MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e, "upload");
  if ((e = cudaMemset(s->m, 0, MLP_NPARAM * sizeof(float))) != cudaSuccess) return fail(e, "memset");
  if ((e = cudaMemset(s->v, 0, MLP_NPARAM * sizeof(float))) != cudaSuccess) return fail(e, "memset");
  if ((e = launch_mlp_pack(s->params, s->img, s->bias, s->wt, s->wn, 0)) != cudaSuccess) return fail(e, "pack");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "pack");
  for (int c = 0; c < 6; ++c) {
    s->mu_in[c] = d->mu_in[c];
    s->sd_in[c] = d->sd_in[c];
    s->mu_out[c] = d->mu_out[c];
    s->sd_out[c] = d->sd_out[c];
    s->nrm.mu_in[c] = d->mu_in[c];
    s->nrm.inv_sd_in[c] = 1.0 / d->sd_in[c];
    s->nrm.mu_out[c] = d->mu_out[c];
    s->nrm.sd_out[c] = d->sd_out[c];
  }
  *out = s;
  return BL_OK;
}

bl_status bl_surrogate_set_domain(bl_surrogate *s, const double *lo, const double *hi) {
  BL_TRY(check_surrogate(s));
  if (!lo && !hi) {
    s->has_domain = false;
    return BL_OK;
  }
  BL_CHECK(lo && hi, "give both lo and hi, or neither");
  for (int c = 0; c < 6; ++c) {
    BL_CHECK(!std::isnan(lo[c]) && !std::isnan(hi[c]) && lo[c] <= hi[c], "domain needs lo <= hi");
    // FP32 bounds that contain the FP64 box
    float l = (float)lo[c], h = (float)hi[c];
    if ((double)l > lo[c]) l = std::nextafter(l, -INFINITY);
    if ((double)h < hi[c]) h = std::nextafter(h, INFINITY);
    s->dom_lo[c] = l;
    s->dom_hi[c] = h;
  }
  s->has_domain = true;
  return BL_OK;
}

bl_status bl_surrogate_destroy(bl_surrogate *s) {
  free_surrogate(s);
  return BL_OK;
}

bl_status bl_surrogate_get_params(const bl_surrogate *s, float *const *W_out, float *const *b_out) {
  BL_TRY(check_surrogate(s));
  BL_CHECK(W_out && b_out, "output arrays are NULL");
  std::vector<float> flat(MLP_NPARAM);
  BL_CUDA(cudaDeviceSynchronize());
  BL_CUDA(cudaMemcpy(flat.data(), s->params, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
  for (int l = 0; l < 5; ++l) {
    BL_CHECK(W_out[l] && b_out[l], "an output layer buffer is NULL");
    const int fi = kWidths[l], fo = kWidths[l + 1];
    std::memcpy(W_out[l], flat.data() + mlp_w_off(l), (size_t)fi * fo * sizeof(float));
    std::memcpy(b_out[l], flat.data() + mlp_b_off(l), (size_t)fo * sizeof(float));
  }
  return BL_OK;
}

bl_status bl_surrogate_apply(const bl_surrogate *s, bl_bunch *b, bl_stream stream) {
  std::string why;
  BL_TRY(check_surrogate(s));
  BL_CHECK(bunch_dims_ok(b, &why), why);
  BL_CHECK(b->dtype == BL_F32, "surrogate inference needs an FP32 bunch");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  if (!ctx->mlp_configured) {
    BL_CUDA(mlp_forward_configure());
    ctx->mlp_configured = true;
  }
  BL_CUDA(launch_mlp_forward(soa_of<float>(b), b->n, s->img, s->nrm, ctx->num_sms,
                             ctx->err_word, (cudaStream_t)stream));
  return BL_OK;
}

bl_status bl_surrogate_train_step(bl_surrogate *s, const float *in, const float *out, int64_t ld,
                                  const int64_t *idx, int64_t batch, const bl_adam_cfg *cfg,
                                  float *loss_out, bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  BL_TRY(check_surrogate(s));
  BL_CHECK(in && out && cfg, "NULL argument");
  BL_CHECK(batch >= 1 && batch <= (int64_t)1 << 24, "batch must be in [1, 2^24]");
  BL_CHECK(ld >= (idx ? 1 : batch), "ld too small for the batch");
  BL_CHECK(cfg->lr > 0.0 && cfg->beta1 >= 0.0 && cfg->beta1 < 1.0 && cfg->beta2 >= 0.0 &&
               cfg->beta2 < 1.0 && cfg->eps > 0.0,
           "invalid Adam configuration");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  float *part = nullptr;
  double *lp = nullptr;
  int nb = 0;
  BL_TRY(train_grad(s, in, out, ld, idx, batch, &part, &lp, &nb, st));
  s->step += 1;
  BL_CUDA(launch_mlp_reduce_adam(part, nb, lp, batch, s->params, s->m, s->v, cfg->lr, cfg->beta1,
                                 cfg->beta2, cfg->eps, s->step, loss_out, nullptr, st));
  BL_CUDA(launch_mlp_pack(s->params, s->img, s->bias, s->wt, s->wn, st));
  return BL_OK;
}

bl_status bl_surrogate_grad(const bl_surrogate *s, const float *in, const float *out, int64_t ld,
                            const int64_t *idx, int64_t batch, float *grad_out, float *loss_out,
                            bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  BL_TRY(check_surrogate(s));
  BL_CHECK(in && out && grad_out, "NULL argument");
  BL_CHECK(batch >= 1 && batch <= (int64_t)1 << 24, "batch must be in [1, 2^24]");
  BL_CHECK(ld >= (idx ? 1 : batch), "ld too small for the batch");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  float *part = nullptr;
  double *lp = nullptr;
  int nb = 0;
  BL_TRY(train_grad(const_cast<bl_surrogate *>(s), in, out, ld, idx, batch, &part, &lp, &nb, st));
  BL_CUDA(launch_mlp_reduce_adam(part, nb, lp, batch, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0,
                                 0.0, 0, loss_out, grad_out, st));
  return BL_OK;
}

bl_status bl_surrogate_loss(const bl_surrogate *s, const float *in, const float *out, int64_t ld,
                            const int64_t *idx, int64_t count, double *loss_out, bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  BL_TRY(check_surrogate(s));
  BL_CHECK(in && out && loss_out, "NULL argument");
  BL_CHECK(count >= 1, "count must be >= 1");
  BL_CHECK(ld >= (idx ? 1 : count), "ld too small for the count");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  const int nb = mlp_grad_blocks(count);
  void *lp = nullptr;
  BL_TRY(ws_get(st, WS_LOSS, (size_t)nb * sizeof(double), &lp));
  int nb2 = 0;
  BL_CUDA(launch_mlp_loss(in, out, ld, idx, count, s->wt, s->wn, s->nrm, (double *)lp, &nb2, st));
  BL_CUDA(launch_loss_finalize((const double *)lp, nb2, count, loss_out, st));
  return BL_OK;
}

}  // extern "C"
