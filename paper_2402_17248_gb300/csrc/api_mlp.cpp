// C ABI: stage surrogates (create, inference, training, loss, parameters).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>

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

std::atomic<bool> g_train_simt{false};

// Samples per gradient launch: a larger minibatch is processed in chunks of
// this size, each chunk's partial rows added to one running FP64 row, so the
// partial rows (205 KB per 128-sample tile) and the tensor-core kernel's
// activation scratch (100 KB per tile) stay near 210 MB and 105 MB however
// large the batch (2^24 samples would otherwise need 27 GB and 13 GB).
constexpr int64_t TRAIN_CHUNK = (int64_t)1 << 17;

// Partial gradients and losses of `batch` samples starting at sample s0
// (scaled as a mean over scale_count samples), from the tensor-core kernel
// (default) or the SIMT FP32 kernel; *nb_out = the number of partial rows.
bl_status train_grad_part(bl_surrogate *s, const float *in, const float *out, int64_t ld,
                          const int64_t *idx, int64_t s0, int64_t batch, int64_t scale_count,
                          float **part_out, double **lp_out, int *nb_out, cudaStream_t st) {
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  const bool simt = g_train_simt.load();
  const int nb = simt ? mlp_grad_blocks(batch) : mlp_train_tc_tiles(batch);
  void *part = nullptr, *lp = nullptr;
  BL_TRY(ws_get(st, WS_TRAIN, (size_t)nb * MLP_PSTRIDE * sizeof(float), &part));
  BL_TRY(ws_get(st, WS_LOSS, (size_t)nb * sizeof(double), &lp));
  // the chunk's samples: columns s0.. of in/out, or entries s0.. of idx
  const float *ci = idx ? in : in + s0, *co = idx ? out : out + s0;
  const int64_t *cx = idx ? idx + s0 : nullptr;
  if (simt) {
    int nb2 = 0;
    BL_CUDA(launch_mlp_grad(ci, co, ld, cx, batch, s->wt, s->wn, s->nrm, (float *)part,
                            (double *)lp, &nb2, st, scale_count));
  } else {
    if (!ctx->train_tc_configured) {
      BL_CUDA(mlp_train_tc_configure());
      ctx->train_tc_configured = true;
    }
    void *scratch = nullptr;
    BL_TRY(ws_get(st, WS_TRAIN_SCRATCH, mlp_train_tc_scratch_bytes(batch), &scratch));
    BL_CUDA(launch_mlp_grad_tc(ci, co, ld, cx, batch, s->img, s->bias, s->nrm, (float *)part,
                               (double *)lp, (uint8_t *)scratch, ctx->num_sms, ctx->err_word, st,
                               scale_count));
  }
  *part_out = (float *)part;
  *lp_out = (double *)lp;
  *nb_out = nb;
  return BL_OK;
}

// Partial gradients and losses of one minibatch: *nb_out partial rows (one
// running row when the batch was processed in chunks).
bl_status train_grad(bl_surrogate *s, const float *in, const float *out, int64_t ld,
                     const int64_t *idx, int64_t batch, float **part_out, double **lp_out,
                     int *nb_out, cudaStream_t st) {
  if (batch <= TRAIN_CHUNK)
    return train_grad_part(s, in, out, ld, idx, 0, batch, batch, part_out, lp_out, nb_out, st);
  // [FP64 running row | FP64 running loss | the final FP32 row]
  const size_t acc_bytes = (MLP_PSTRIDE + 1) * sizeof(double);
  void *acc = nullptr;
  BL_TRY(ws_get(st, WS_TRAIN_ACC, acc_bytes + MLP_PSTRIDE * sizeof(float), &acc));
  double *acc_row = (double *)acc;
  double *acc_loss = acc_row + MLP_PSTRIDE;
  float *row = (float *)((uint8_t *)acc + acc_bytes);
  BL_CUDA(cudaMemsetAsync(acc, 0, acc_bytes, st));
  for (int64_t s0 = 0; s0 < batch; s0 += TRAIN_CHUNK) {
    float *part = nullptr;
    double *lp = nullptr;
    int nb = 0;
    BL_TRY(train_grad_part(s, in, out, ld, idx, s0, std::min(TRAIN_CHUNK, batch - s0), batch,
                           &part, &lp, &nb, st));
    BL_CUDA(launch_mlp_rows_accumulate(part, nb, lp, acc_row, acc_loss,
                                       s0 + TRAIN_CHUNK >= batch ? row : nullptr, st));
  }
  *part_out = row;
  *lp_out = acc_loss;
  *nb_out = 1;
  return BL_OK;
}

}  // namespace

namespace bl {
bool mlp_train_use_simt() { return g_train_simt.load(); }
}  // namespace bl

namespace {

// A surrogate from flat FP32 parameters, optional Adam moments (NULL: zero)
// and step count, and FP64 normalisation constants.
bl_status make_surrogate(const float *flat, const float *m, const float *v, int step,
                         const double *mu_in, const double *sd_in, const double *mu_out,
                         const double *sd_out, bl_surrogate **out) {
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  auto *s = new bl_surrogate_s();
  s->device = ctx->device;
  auto fail = [&](cudaError_t e, const char *what) {
    free_surrogate(s);
    return cuda_error(e, what);
  };
  const size_t pb = MLP_NPARAM * sizeof(float);
  cudaError_t e;
  if ((e = cudaMalloc(&s->params, pb)) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->m, pb)) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->v, pb)) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->img, MLP_IMG_BYTES)) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->bias, MLP_BIAS_FLOATS * sizeof(float))) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->wt, pb)) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMalloc(&s->wn, pb)) != cudaSuccess) return fail(e, "alloc");
  if ((e = cudaMemcpy(s->params, flat, pb, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "upload");
  if (m) e = cudaMemcpy(s->m, m, pb, cudaMemcpyHostToDevice);
  else e = cudaMemset(s->m, 0, pb);
  if (e != cudaSuccess) return fail(e, "upload");
  if (v) e = cudaMemcpy(s->v, v, pb, cudaMemcpyHostToDevice);
  else e = cudaMemset(s->v, 0, pb);
  if (e != cudaSuccess) return fail(e, "upload");
  if ((e = launch_mlp_pack(s->params, s->img, s->bias, s->wt, s->wn, 0)) != cudaSuccess) return fail(e, "pack");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "pack");
  s->step = step;
  for (int c = 0; c < 6; ++c) {
    s->mu_in[c] = mu_in[c];
    s->sd_in[c] = sd_in[c];
    s->mu_out[c] = mu_out[c];
    s->sd_out[c] = sd_out[c];
    s->nrm.mu_in[c] = mu_in[c];
    s->nrm.inv_sd_in[c] = 1.0 / sd_in[c];
    s->nrm.mu_out[c] = mu_out[c];
    s->nrm.sd_out[c] = sd_out[c];
  }
  *out = s;
  return BL_OK;
}

// ---- surrogate files ----
// Little-endian binary: magic "BLSURR01", int32 version (1), int32 widths[6],
// FP64 mu_in, sd_in, mu_out, sd_out (6 each), int32 has_domain, FP32
// dom_lo[6], dom_hi[6], int32 Adam step, FP32 params, m, v (MLP_NPARAM each),
// then a 64-bit FNV-1a hash of every preceding byte.
constexpr char kMagic[8] = {'B', 'L', 'S', 'U', 'R', 'R', '0', '1'};
constexpr int32_t kVersion = 1;

uint64_t fnv1a(const std::vector<uint8_t> &b, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

template <typename T> void put(std::vector<uint8_t> &b, const T *v, size_t n) {
  const uint8_t *p = reinterpret_cast<const uint8_t *>(v);
  b.insert(b.end(), p, p + n * sizeof(T));
}

struct Reader {
  const std::vector<uint8_t> &b;
  size_t pos = 0;
  template <typename T> bool get(T *v, size_t n) {
    const size_t bytes = n * sizeof(T);
    if (pos + bytes > b.size()) return false;
    std::memcpy(v, b.data() + pos, bytes);
    pos += bytes;
    return true;
  }
};

}  // namespace

extern "C" {

bl_status bl_surrogate_create(const bl_mlp_desc *d, bl_surrogate **out) {
  BL_CHECK(out, "out is NULL");
  *out = nullptr;
  BL_TRY(check_desc(d));
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
  return make_surrogate(flat.data(), nullptr, nullptr, 0, d->mu_in, d->sd_in, d->mu_out,
                        d->sd_out, out);
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

bl_status bl_surrogate_save(const bl_surrogate *s, const char *path) {
  BL_TRY(check_surrogate(s));
  BL_CHECK(path, "path is NULL");
  const size_t pb = MLP_NPARAM * sizeof(float);
  std::vector<float> P(MLP_NPARAM), M(MLP_NPARAM), V(MLP_NPARAM);
  BL_CUDA(cudaDeviceSynchronize());
  BL_CUDA(cudaMemcpy(P.data(), s->params, pb, cudaMemcpyDeviceToHost));
  BL_CUDA(cudaMemcpy(M.data(), s->m, pb, cudaMemcpyDeviceToHost));
  BL_CUDA(cudaMemcpy(V.data(), s->v, pb, cudaMemcpyDeviceToHost));
  std::vector<uint8_t> b;
  put(b, kMagic, 8);
  put(b, &kVersion, 1);
  put(b, kWidths, 6);
  put(b, s->mu_in, 6);
  put(b, s->sd_in, 6);
  put(b, s->mu_out, 6);
  put(b, s->sd_out, 6);
  const int32_t hd = s->has_domain ? 1 : 0, step = s->step;
  put(b, &hd, 1);
  put(b, s->dom_lo, 6);
  put(b, s->dom_hi, 6);
  put(b, &step, 1);
  put(b, P.data(), MLP_NPARAM);
  put(b, M.data(), MLP_NPARAM);
  put(b, V.data(), MLP_NPARAM);
  const uint64_t h = fnv1a(b, b.size());
  put(b, &h, 1);
  FILE *f = std::fopen(path, "wb");
  BL_CHECK(f, std::string("cannot open for writing: ") + path);
  const size_t w = std::fwrite(b.data(), 1, b.size(), f);
  const int c = std::fclose(f);
  BL_CHECK(w == b.size() && c == 0, std::string("write failed: ") + path);
  return BL_OK;
}

bl_status bl_surrogate_load(const char *path, bl_surrogate **out) {
  BL_CHECK(out, "out is NULL");
  *out = nullptr;
  BL_CHECK(path, "path is NULL");
  FILE *f = std::fopen(path, "rb");
  BL_CHECK(f, std::string("cannot open: ") + path);
  std::vector<uint8_t> b;
  uint8_t buf[1 << 16];
  size_t r;
  while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) b.insert(b.end(), buf, buf + r);
  std::fclose(f);
  BL_CHECK(b.size() >= 8 + sizeof(uint64_t), "surrogate file too short");
  uint64_t h = 0;
  std::memcpy(&h, b.data() + b.size() - sizeof(uint64_t), sizeof(h));
  BL_CHECK(h == fnv1a(b, b.size() - sizeof(uint64_t)), "surrogate file checksum mismatch");
  Reader rd{b};
  char magic[8];
  int32_t ver = 0, widths[6], hd = 0, step = 0;
  double mu_in[6], sd_in[6], mu_out[6], sd_out[6];
  float lo[6], hi[6];
  std::vector<float> P(MLP_NPARAM), M(MLP_NPARAM), V(MLP_NPARAM);
  BL_CHECK(rd.get(magic, 8) && std::memcmp(magic, kMagic, 8) == 0, "not a surrogate file");
  BL_CHECK(rd.get(&ver, 1) && ver == kVersion, "unsupported surrogate file version");
  BL_CHECK(rd.get(widths, 6) && std::memcmp(widths, kWidths, sizeof(widths)) == 0,
           "surrogate file widths differ from this build's 6-128-128-128-128-6");
  const bool ok = rd.get(mu_in, 6) && rd.get(sd_in, 6) && rd.get(mu_out, 6) && rd.get(sd_out, 6) &&
                  rd.get(&hd, 1) && rd.get(lo, 6) && rd.get(hi, 6) && rd.get(&step, 1) &&
                  rd.get(P.data(), MLP_NPARAM) && rd.get(M.data(), MLP_NPARAM) &&
                  rd.get(V.data(), MLP_NPARAM) && rd.pos + sizeof(uint64_t) == b.size();
  BL_CHECK(ok, "surrogate file truncated or malformed");
  for (int c = 0; c < 6; ++c)
    BL_CHECK(std::isfinite(mu_in[c]) && std::isfinite(mu_out[c]) && sd_in[c] > 0.0 &&
                 sd_out[c] > 0.0 && std::isfinite(sd_in[c]) && std::isfinite(sd_out[c]),
             "surrogate file normalisation constants invalid");
  for (int i = 0; i < MLP_NPARAM; ++i)
    BL_CHECK(std::isfinite(P[i]) && std::isfinite(M[i]) && std::isfinite(V[i]),
             "surrogate file parameters must be finite");
  BL_CHECK(step >= 0, "surrogate file step invalid");
  bl_surrogate *s = nullptr;
  BL_TRY(make_surrogate(P.data(), M.data(), V.data(), step, mu_in, sd_in, mu_out, sd_out, &s));
  if (hd) {
    for (int c = 0; c < 6; ++c) {
      s->dom_lo[c] = lo[c];
      s->dom_hi[c] = hi[c];
    }
    s->has_domain = true;
  }
  *out = s;
  return BL_OK;
}

bl_status bl_surrogate_get_domain(const bl_surrogate *s, double *lo, double *hi, int32_t *has) {
  BL_TRY(check_surrogate(s));
  BL_CHECK(lo && hi && has, "NULL argument");
  *has = s->has_domain ? 1 : 0;
  for (int c = 0; c < 6; ++c) {
    lo[c] = s->has_domain ? s->dom_lo[c] : 0.0;
    hi[c] = s->has_domain ? s->dom_hi[c] : 0.0;
  }
  return BL_OK;
}

bl_status bl_surrogate_get_norm(const bl_surrogate *s, double *mu_in, double *sd_in,
                                double *mu_out, double *sd_out) {
  BL_TRY(check_surrogate(s));
  BL_CHECK(mu_in && sd_in && mu_out && sd_out, "NULL argument");
  for (int c = 0; c < 6; ++c) {
    mu_in[c] = s->mu_in[c];
    sd_in[c] = s->sd_in[c];
    mu_out[c] = s->mu_out[c];
    sd_out[c] = s->sd_out[c];
  }
  return BL_OK;
}

}  // extern "C"

extern "C" int bl_debug_train_kernel(int simt) {
  return g_train_simt.exchange(simt != 0) ? 1 : 0;
}
