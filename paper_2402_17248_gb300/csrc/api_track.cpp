// C ABI: lattices, tracking, moments, linear maps and the plain stage push.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "runtime.h"

using namespace bl;

namespace {

bool lattice_has_per_bunch(const bl_lattice_s *L) { return L->n_bunch_k > 0; }

double element_k(const bl_lattice_s *L, int e, int b) {
  const auto &v = L->pbk[e];
  return v.empty() ? L->els[e].k : v[b];
}

}  // namespace

// Host plan (stage tables, segment and element matrices) for a reference
// energy, dtype and bunch count; uploaded to device buffers owned by the lattice.
bl_status bl::build_plan(bl_lattice_s *L, double gamma_in, int dtype, int n_bunch, cudaStream_t st) {
  int dev = -1;
  BL_CUDA(cudaGetDevice(&dev));
  auto &P = L->plan;
  if (P.valid && P.gamma_in == gamma_in && P.dtype == dtype && P.n_bunch == n_bunch &&
      P.device == dev)
    return BL_OK;
  const int nbm = lattice_has_per_bunch(L) ? n_bunch : 1;
  const size_t G = L->groups.size();
  std::vector<StageTrack> stages(G);
  std::vector<std::vector<Mat6>> seg(G);
  std::vector<std::vector<std::vector<Mat6>>> elm(G);
  std::vector<size_t> toff(G, 0), moff(G, 0);
  size_t tbytes = 0, mbytes = 0;
  const size_t esz = dtype == BL_F32 ? 4 : 8;
  double gam = gamma_in;
  for (size_t g = 0; g < G; ++g) {
    const auto &gr = L->groups[g];
    if (gr.stage) {
      BL_TRY(stage_track(L->els[gr.first], gam, dtype, &stages[g]));
      gam = stages[g].c.gamma_out;
      toff[g] = tbytes;
      tbytes += (size_t)stages[g].c.nsteps * 16 * esz;
    } else {
      const double bg = std::sqrt(gam * gam - 1.0);
      seg[g].assign(nbm, mat_identity());
      elm[g].resize(gr.last - gr.first + 1);
      for (int e = gr.first; e <= gr.last; ++e) {
        auto &em = elm[g][e - gr.first];
        em.resize(nbm);
        for (int b = 0; b < nbm; ++b) {
          em[b] = element_matrix(L->els[e], element_k(L, e, b), bg);
          seg[g][b] = mat_mul(em[b], seg[g][b]);
        }
      }
      moff[g] = mbytes;
      mbytes += (size_t)nbm * 36 * esz;
    }
  }
  // device upload
  if (P.d_tables && P.tables_bytes < tbytes) { BL_CUDA(cudaStreamSynchronize(st)); cudaFree(P.d_tables); P.d_tables = nullptr; P.tables_bytes = 0; }
  if (P.d_mats && P.mats_bytes < mbytes) { BL_CUDA(cudaStreamSynchronize(st)); cudaFree(P.d_mats); P.d_mats = nullptr; P.mats_bytes = 0; }
  if (!P.d_tables && tbytes) { BL_CUDA(cudaMalloc(&P.d_tables, tbytes)); P.tables_bytes = tbytes; }
  if (!P.d_mats && mbytes) { BL_CUDA(cudaMalloc(&P.d_mats, mbytes)); P.mats_bytes = mbytes; }
  std::vector<uint8_t> hbuf(std::max(tbytes, mbytes));
  if (tbytes) {
    for (size_t g = 0; g < G; ++g)
      if (L->groups[g].stage) {
        const void *src = dtype == BL_F32 ? (const void *)stages[g].table32.data()
                                          : (const void *)stages[g].table64.data();
        std::memcpy(hbuf.data() + toff[g], src, (size_t)stages[g].c.nsteps * 16 * esz);
      }
    BL_CUDA(cudaMemcpyAsync(P.d_tables, hbuf.data(), tbytes, cudaMemcpyHostToDevice, st));
    BL_CUDA(cudaStreamSynchronize(st));
  }
  if (mbytes) {
    for (size_t g = 0; g < G; ++g)
      if (!L->groups[g].stage)
        for (int b = 0; b < nbm; ++b)
          for (int i = 0; i < 36; ++i) {
            uint8_t *dst = hbuf.data() + moff[g] + ((size_t)b * 36 + i) * esz;
            if (dtype == BL_F32) { float v = (float)seg[g][b][i]; std::memcpy(dst, &v, 4); }
            else std::memcpy(dst, &seg[g][b][i], 8);
          }
    BL_CUDA(cudaMemcpyAsync(P.d_mats, hbuf.data(), mbytes, cudaMemcpyHostToDevice, st));
    BL_CUDA(cudaStreamSynchronize(st));
  }
  P.stages = std::move(stages);
  P.seg_mats = std::move(seg);
  P.el_mats = std::move(elm);
  P.table_off = std::move(toff);
  P.mat_off = std::move(moff);
  P.gamma_in = gamma_in;
  P.gamma_out = gam;
  P.dtype = dtype;
  P.n_bunch = n_bunch;
  P.device = dev;
  P.valid = true;
  return BL_OK;
}

namespace {

template <typename T>
bl_status run_segment(bl_bunch *b, bl_lattice_s *L, size_t g, bool moments, double *mom_dev,
                      unsigned long long *nf, cudaStream_t st) {
  auto &P = L->plan;
  Soa<T> z = soa_of<T>(b);
  const int64_t *off = b->n_bunch > 1 ? b->offsets_dev : nullptr;
  const T *mats = (const T *)((const uint8_t *)P.d_mats + P.mat_off[g]);
  const int per_bunch = lattice_has_per_bunch(L) ? 1 : 0;
  void *part = nullptr;
  if (moments)
    BL_TRY(ws_get(st, WS_PARTIALS, (size_t)stream_slots(b->n, b->n_bunch) * 28 * sizeof(double), &part));
  int64_t unit = 0;
  BL_CUDA(launch_stream<T>(z, z, b->n, off, b->n_bunch, mats, per_bunch, nullptr, true, moments,
                           (double *)part, st, &unit));
  if (moments)
    BL_CUDA(launch_moments_finalize((const double *)part, off, b->n_bunch, b->n, unit, mom_dev,
                                    nf, st));
  return BL_OK;
}

// fused: out-of-domain particles pushed by the surrogate kernel's fallback
// warp, overlapped with the network's tensor work; otherwise all by the list
// pusher after it. Every path here uses the fused form: with the chunks of
// bl_track_host on the list pusher, back-to-back calls on 2^24 particles took
// 30 ms each against 23.6 ms with the fallback warp.
bl_status run_stage(bl_bunch *b, bl_lattice_s *L, size_t g, cudaStream_t st, bool fused = true) {
  auto &P = L->plan;
  const bl_element &e = L->els[L->groups[g].first];
  const StageTrack &tr = P.stages[g];
  if (e.surrogate && e.surrogate->has_domain) {
    // surrogate inside its training domain, the plain pusher outside it
    const bl_surrogate *s = e.surrogate;
    BL_CHECK(b->dtype == BL_F32, "surrogate stages need an FP32 bunch");
    DevCtx *ctx = nullptr;
    BL_TRY(current_ctx(&ctx));
    if (!ctx->mlp_configured) {
      BL_CUDA(mlp_forward_configure());
      ctx->mlp_configured = true;
    }
    void *fb = nullptr;
    BL_TRY(ws_get(st, WS_FALLBACK, (size_t)(b->n + 1) * sizeof(int64_t), &fb));
    MlpDomain dom;
    for (int c = 0; c < 6; ++c) {
      dom.lo[c] = s->dom_lo[c];
      dom.hi[c] = s->dom_hi[c];
    }
    dom.fb_count = (unsigned long long *)fb;
    dom.fb_list = (int64_t *)fb + 1;
    dom.fb_cap = b->n;
    const float *tab = (const float *)((const uint8_t *)P.d_tables + P.table_off[g]);
    dom.stage = consts_f(tr.c);
    dom.table = tab;
    dom.fused = fused ? 1 : 0;
    BL_CUDA(cudaMemsetAsync(dom.fb_count, 0, sizeof(unsigned long long), st));
    // the surrogate kernel pushes the particles outside the domain itself
    // (a fallback warp per CTA); the list pusher takes those past a CTA's
    // queue, and exits at once when there are none
    BL_CUDA(launch_mlp_forward(soa_of<float>(b), b->n, s->img, s->nrm, ctx->num_sms,
                               ctx->err_word, st, &dom));
    BL_CUDA(launch_pusher_list(soa_of<float>(b), dom.fb_list, dom.fb_count, b->n, tr.c, tab,
                               ctx->num_sms, st));
  } else if (e.surrogate) {
    BL_TRY(bl_surrogate_apply(e.surrogate, b, st));
  } else if (e.wide_surrogate) {
    BL_TRY(bl_wide_mlp_apply(e.wide_surrogate, b, 0, st));
  } else if (b->dtype == BL_F32) {
    const float *tab = (const float *)((const uint8_t *)P.d_tables + P.table_off[g]);
    BL_CUDA(launch_pusher<float>(soa_of<float>(b), b->n, tr.c, tab, st));
  } else {
    const double *tab = (const double *)((const uint8_t *)P.d_tables + P.table_off[g]);
    BL_CUDA(launch_pusher<double>(soa_of<double>(b), b->n, tr.c, tab, st));
  }
  return BL_OK;
}

}  // namespace

namespace {

// Reduction points of a lattice: segment entries, and stage exits not
// followed by a segment. red_of[g] = index of group g's reduction or -1.
int reduction_points(const bl_lattice_s *L, std::vector<int> *red_of) {
  const size_t G = L->groups.size();
  red_of->assign(G, -1);
  int R = 0;
  for (size_t g = 0; g < G; ++g) {
    if (!L->groups[g].stage) (*red_of)[g] = R++;
    else if (g + 1 == G || L->groups[g + 1].stage) (*red_of)[g] = R++;
  }
  return R;
}

bl_status track_checks(bl_bunch *b, bl_lattice_s *L) {
  std::string why;
  BL_CHECK(bunch_dims_ok(b, &why), why);
  BL_CHECK(!lattice_has_per_bunch(L) || L->n_bunch_k == b->n_bunch,
           "lattice per-bunch strengths do not match the bunch count");
  for (const auto &gr : L->groups)
    if (gr.stage && (L->els[gr.first].surrogate || L->els[gr.first].wide_surrogate))
      BL_CHECK(b->dtype == BL_F32, "surrogate stages need an FP32 bunch");
  return BL_OK;
}

// Enqueue groups [g0, g1); the reductions of those groups (28 doubles per
// bunch per reduction point, at the point's index) go into mom_dev and their
// non-finite count into *nf (zeroed first) when mom_dev != NULL.
bl_status track_enqueue_range(bl_bunch *b, bl_lattice_s *L, size_t g0, size_t g1, double *mom_dev,
                              unsigned long long *nf, cudaStream_t st) {
  std::vector<int> red_of;
  reduction_points(L, &red_of);
  const size_t per = (size_t)b->n_bunch * 28;
  const bool want = mom_dev != nullptr;
  if (want) BL_CUDA(cudaMemsetAsync(nf, 0, sizeof(unsigned long long), st));
  for (size_t g = g0; g < g1; ++g) {
    // one NVTX range per element group, so a profiler timeline shows the
    // beamline's structure (no cost without a profiler attached)
    const bool stage = L->groups[g].stage;
    const bl_element &first = L->els[L->groups[g].first];
    nvtxRangePushA(!stage ? "bl segment"
                          : (first.surrogate ? "bl stage: surrogate"
                                             : (first.wide_surrogate ? "bl stage: wide surrogate"
                                                                     : "bl stage: pusher")));
    bl_status r = BL_OK;
    if (stage) {
      r = run_stage(b, L, g, st);
      if (r == BL_OK && want && red_of[g] >= 0) r = moments_device(b, mom_dev + red_of[g] * per, nf, st);
    } else if (b->dtype == BL_F32) {
      r = run_segment<float>(b, L, g, want, want ? mom_dev + red_of[g] * per : nullptr, nf, st);
    } else {
      r = run_segment<double>(b, L, g, want, want ? mom_dev + red_of[g] * per : nullptr, nf, st);
    }
    nvtxRangePop();
    if (r != BL_OK) return r;
  }
  return BL_OK;
}

// Every group, then the bunch's reference energy moves to the exit's.
bl_status track_enqueue(bl_bunch *b, bl_lattice_s *L, double *mom_dev, unsigned long long *nf,
                        cudaStream_t st) {
  BL_TRY(track_enqueue_range(b, L, 0, L->groups.size(), mom_dev, nf, st));
  b->gamma_ref = L->plan.gamma_out;
  return BL_OK;
}

// Moments after every element from the reductions (host, FP64): a stage's
// snapshot is the reduction at its exit (or at the next segment's entry); a
// segment's elements are reached by propagating its entry moments through
// the element matrices.
void expand_moments(const bl_lattice_s *L, int n_bunch, const double *red, double *moments_out) {
  std::vector<int> red_of;
  reduction_points(L, &red_of);
  const auto &P = L->plan;
  const size_t per = (size_t)n_bunch * 28;
  const int nbm = lattice_has_per_bunch(L) ? n_bunch : 1;
  for (size_t g = 0; g < L->groups.size(); ++g) {
    const auto &gr = L->groups[g];
    if (gr.stage) {
      const int r = red_of[g] >= 0 ? red_of[g] : red_of[g + 1];
      std::memcpy(moments_out + (size_t)gr.first * per, red + (size_t)r * per, per * sizeof(double));
    } else {
      for (int bb = 0; bb < n_bunch; ++bb) {
        double cur[28];
        std::memcpy(cur, red + (size_t)red_of[g] * per + (size_t)bb * 28, sizeof(cur));
        for (int e = gr.first; e <= gr.last; ++e) {
          double nxt[28];
          propagate_moments(P.el_mats[g][e - gr.first][nbm > 1 ? bb : 0], cur, nxt);
          std::memcpy(moments_out + (size_t)e * per + (size_t)bb * 28, nxt, sizeof(nxt));
          std::memcpy(cur, nxt, sizeof(cur));
        }
      }
    }
  }
}

// ---- host-resident bunches (bl_track_host) ----
constexpr int HOST_BUFS = 4;  // device chunk buffers in flight
// event slots: [0, 4) copied in, [4, 8) tracked, [8, 12) copied out (one per
// buffer), 12 the start, 13..16 the joins of the four pipeline streams
constexpr int EV_IN = 0, EV_TRACKED = HOST_BUFS, EV_OUT = 2 * HOST_BUFS, EV_START = 3 * HOST_BUFS,
              EV_JOIN = EV_START + 1;
static_assert(EV_JOIN + 4 == DevCtx::HOST_EVENTS, "bl_track_host event slots");
// default chunk sizes: the whole-bunch mode pays the per-chunk costs (one
// launch set, ramp and tail per kernel) only in the head and the tail, so
// smaller chunks shorten the unoverlapped first copy in and last copy out
// (measured on 2^24 particles: 27.0 ms per pass at 2^21, 27.4 at 2^22);
// the chunk-through mode pays them for every group (28.2 ms at 2^22)
constexpr int64_t HOST_CHUNK_WHOLE = (int64_t)1 << 21, HOST_CHUNK_RING = (int64_t)1 << 22;
// one bl_track_host at a time per process: the pipeline's streams and the
// work buffers of its compute streams are shared
std::mutex g_host_mu;

bl_status host_pipeline_init(DevCtx *ctx) {
  if (ctx->hp_h2d) return BL_OK;
  for (auto &s_ : ctx->hp_comp) BL_CUDA(cudaStreamCreateWithFlags(&s_, cudaStreamNonBlocking));
  BL_CUDA(cudaStreamCreateWithFlags(&ctx->hp_d2h, cudaStreamNonBlocking));
  for (auto &e : ctx->hp_ev) BL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  BL_CUDA(cudaStreamCreateWithFlags(&ctx->hp_h2d, cudaStreamNonBlocking));
  return BL_OK;
}

// Moments of a union of disjoint particle sets from the sets' own moment
// vectors [N, 6 means, 21 central second moments with 1/N]: counts add,
// means pool with weights N_c, and each central moment gains the
// parallel-axis term (mu_c - mu)(mu_c - mu)^T (FP64).
void pool_moments(const std::vector<const double *> &parts, double *out) {
  double N = 0.0;
  for (const double *p : parts) N += p[0];
  std::memset(out, 0, 28 * sizeof(double));
  out[0] = N;
  if (!(N > 0.0)) return;
  for (const double *p : parts)
    if (p[0] > 0.0)
      for (int a = 0; a < 6; ++a) out[1 + a] += p[0] * p[1 + a];
  for (int a = 0; a < 6; ++a) out[1 + a] /= N;
  for (const double *p : parts) {
    if (!(p[0] > 0.0)) continue;
    int j = 7;
    for (int a = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b, ++j) {
        const double da = p[1 + a] - out[1 + a], db = p[1 + b] - out[1 + b];
        out[j] += p[0] * (p[j] + da * db);
      }
  }
  for (int j = 7; j < 28; ++j) out[j] /= N;
}

}  // namespace

extern "C" {

bl_status bl_lattice_create(const bl_element *elements, int32_t n_elements, int32_t n_bunch_k,
                            bl_lattice **out) {
  BL_CHECK(out, "out is NULL");
  *out = nullptr;
  BL_CHECK(elements && n_elements > 0, "lattice needs at least one element");
  BL_CHECK(n_bunch_k >= 0, "n_bunch_k must be >= 0");
  auto L = std::make_unique<bl_lattice_s>();
  L->n_bunch_k = 0;
  for (int i = 0; i < n_elements; ++i) {
    const bl_element &e = elements[i];
    BL_CHECK(e.kind >= BL_DRIFT && e.kind <= BL_PLASMA_LENS, "unknown element kind");
    BL_CHECK(std::isfinite(e.L) && e.L >= 0.0, "element length must be finite and >= 0");
    if (e.kind == BL_QUAD) BL_CHECK(std::isfinite(e.k), "quad strength must be finite");
    if (e.kind == BL_PLASMA_LENS) {
      BL_CHECK(std::isfinite(e.k), "plasma lens strength must be finite");
      BL_CHECK(!e.per_bunch_k, "plasma lenses take no per-bunch strengths");
    }
    if (e.kind == BL_SBEND) {
      BL_CHECK(std::isfinite(e.angle), "bend angle must be finite");
      BL_CHECK(e.angle == 0.0 || e.L > 0.0, "a bend with an angle needs L > 0");
    }
    if (e.kind == BL_PLASMA) {
      BL_CHECK(e.L > 0.0, "plasma stage needs L > 0");
      BL_CHECK(e.nsteps >= 1 && e.nsteps <= (1 << 20), "plasma stage needs 1 <= nsteps <= 2^20");
      BL_CHECK(e.n0_cm3 > 0.0 && std::isfinite(e.E0_Vpm) && std::isfinite(e.phi0),
               "plasma stage parameters invalid");
      BL_CHECK(!(e.surrogate && e.wide_surrogate),
               "a plasma stage takes a surrogate or a wide surrogate, not both");
    } else {
      BL_CHECK(!e.surrogate && !e.wide_surrogate, "only plasma stages take surrogates");
    }
    std::vector<double> pk;
    if (e.kind == BL_QUAD && e.per_bunch_k) {
      BL_CHECK(n_bunch_k > 0, "per_bunch_k given but n_bunch_k == 0");
      pk.assign(e.per_bunch_k, e.per_bunch_k + n_bunch_k);
      for (double v : pk) BL_CHECK(std::isfinite(v), "per_bunch_k must be finite");
      L->n_bunch_k = n_bunch_k;
    }
    L->els.push_back(e);
    L->pbk.push_back(std::move(pk));
    if (e.kind == BL_QUAD) L->n_quads++;
  }
  for (int i = 0; i < n_elements; ++i) {
    const bool st = L->els[i].kind == BL_PLASMA;
    if (st || L->groups.empty() || L->groups.back().stage)
      L->groups.push_back({st, i, i});
    else
      L->groups.back().last = i;
  }
  *out = L.release();
  return BL_OK;
}

bl_status bl_lattice_destroy(bl_lattice *lat) {
  delete lat;
  return BL_OK;
}

bl_status bl_segment_matrix(const bl_element *elements, int32_t n, double gamma_ref,
                            double *M_out) {
  BL_CHECK(M_out, "M_out is NULL");
  BL_CHECK(n >= 0 && (n == 0 || elements), "elements is NULL");
  BL_CHECK(std::isfinite(gamma_ref) && gamma_ref > 1.0, "gamma_ref must be finite and > 1");
  const double bg = std::sqrt(gamma_ref * gamma_ref - 1.0);
  Mat6 M = mat_identity();
  for (int i = 0; i < n; ++i) {
    const bl_element &e = elements[i];
    BL_CHECK(e.kind == BL_DRIFT || e.kind == BL_QUAD || e.kind == BL_SBEND ||
                 e.kind == BL_PLASMA_LENS,
             "bl_segment_matrix takes linear elements only");
    BL_CHECK(std::isfinite(e.L) && e.L >= 0.0, "element length must be finite and >= 0");
    BL_CHECK(std::isfinite(e.k) && std::isfinite(e.angle), "element strengths must be finite");
    BL_CHECK(e.kind != BL_SBEND || e.angle == 0.0 || e.L > 0.0, "a bend with an angle needs L > 0");
    M = mat_mul(element_matrix(e, e.k, bg), M);
  }
  for (int i = 0; i < 36; ++i) M_out[i] = M[i];
  return BL_OK;
}

int32_t bl_lattice_num_elements(const bl_lattice *lat) { return lat ? (int32_t)lat->els.size() : -1; }
int32_t bl_lattice_num_quads(const bl_lattice *lat) { return lat ? lat->n_quads : -1; }


bl_status bl_track(bl_bunch *b, const bl_lattice *lat_c, double *moments_out,
                   int64_t *nonfinite_out, bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  BL_CHECK(lat_c, "lattice is NULL");
  bl_lattice_s *L = const_cast<bl_lattice_s *>(lat_c);
  BL_TRY(track_checks(b, L));
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  std::lock_guard<std::mutex> lk(L->mu);
  BL_TRY(build_plan(L, b->gamma_ref, b->dtype, b->n_bunch, st));
  const bool want = moments_out != nullptr || nonfinite_out != nullptr;
  std::vector<int> red_of;
  const int R = reduction_points(L, &red_of);
  const size_t per = (size_t)b->n_bunch * 28;
  double *mom_dev = nullptr;
  void *nf = nullptr;
  if (want) {
    void *p = nullptr;
    BL_TRY(ws_get(st, WS_MOMENTS, (size_t)R * per * sizeof(double), &p));
    mom_dev = (double *)p;
    BL_TRY(ws_get(st, WS_NONFINITE, sizeof(unsigned long long), &nf));
  }
  BL_TRY(track_enqueue(b, L, mom_dev, (unsigned long long *)nf, st));
  if (!want) return BL_OK;
  std::vector<double> red((size_t)R * per);
  unsigned long long nonfin = 0;
  BL_CUDA(cudaMemcpyAsync(red.data(), mom_dev, red.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  BL_CUDA(cudaMemcpyAsync(&nonfin, nf, sizeof(nonfin), cudaMemcpyDeviceToHost, st));
  BL_CUDA(cudaStreamSynchronize(st));
  if (nonfinite_out) *nonfinite_out = (int64_t)nonfin;
  if (moments_out) expand_moments(L, b->n_bunch, red.data(), moments_out);
  if (nonfin) return set_error(BL_ERR_NONFINITE, std::to_string(nonfin) + " non-finite particles seen");
  return BL_OK;
}

bl_status bl_track_host(const float *const in_host[6], float *const out_host[6], int64_t n,
                        double *gamma_ref, const bl_lattice *lat_c, int64_t chunk,
                        double *moments_out, int64_t *nonfinite_out, bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  BL_CHECK(lat_c, "lattice is NULL");
  BL_CHECK(in_host && out_host && gamma_ref, "NULL argument");
  for (int c = 0; c < 6; ++c) BL_CHECK(in_host[c] && out_host[c], "coordinate pointer is NULL");
  BL_CHECK(n >= 1, "n must be >= 1");
  BL_CHECK(chunk >= 0, "chunk must be >= 0");
  BL_CHECK(*gamma_ref > 1.0 && std::isfinite(*gamma_ref), "gamma_ref must exceed 1");
  bl_lattice_s *L = const_cast<bl_lattice_s *>(lat_c);
  BL_CHECK(L->n_bunch_k <= 1, "bl_track_host tracks one bunch: per-bunch strengths for more "
                              "than one bunch are not supported");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  std::lock_guard<std::mutex> hk(g_host_mu);
  std::lock_guard<std::mutex> lk(L->mu);
  BL_TRY(host_pipeline_init(ctx));
  const double g_in = *gamma_ref;
  BL_TRY(build_plan(L, g_in, BL_F32, 1, st));
  const bool want = moments_out != nullptr || nonfinite_out != nullptr;
  std::vector<int> red_of;
  const int R = reduction_points(L, &red_of);
  const size_t per = (size_t)R * 28 + 1;  // one region: R reductions + a non-finite count
  const size_t G = L->groups.size();
  // head: groups up to the first stage; tail: from the last stage on
  size_t first_stage = G, last_stage = G;
  for (size_t g = 0; g < G; ++g)
    if (L->groups[g].stage) {
      if (first_stage == G) first_stage = g;
      last_stage = g;
    }
  // Whole-bunch mode (the bunch fits on the device and the lattice has two
  // stages or more): only the head and the tail run chunk by chunk, so the
  // copies in overlap the first stage and the copies out the last, and the
  // groups in between run once on the whole bunch. Otherwise every chunk
  // passes through the whole lattice in a four-buffer ring.
  size_t free_b = 0, total_b = 0;
  BL_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const bool fits = first_stage < last_stage && (size_t)n * 6 * sizeof(float) <= free_b / 2;
  if (chunk == 0) chunk = fits ? HOST_CHUNK_WHOLE : HOST_CHUNK_RING;
  if (chunk > n) chunk = n;
  const int64_t nchunks = (n + chunk - 1) / chunk;
  const bool whole = fits && nchunks > 1;
  const size_t h_end = first_stage + 1, t_begin = last_stage;
  const int64_t nregions = whole ? 2 * nchunks + 1 : nchunks;
  void *buf = nullptr, *red = nullptr;
  const size_t buf_floats = whole ? (size_t)6 * n : (size_t)HOST_BUFS * 6 * chunk;
  BL_TRY(ws_get(st, WS_HOST_BUF, buf_floats * sizeof(float), &buf));
  if (want) BL_TRY(ws_get(st, WS_HOST_RED, (size_t)nregions * per * sizeof(double), &red));
  float *dbuf = (float *)buf;
  double *dred = (double *)red;
  cudaEvent_t *ev = ctx->hp_ev;
  cudaStream_t h2d = ctx->hp_h2d, d2h = ctx->hp_d2h;
  cudaStream_t pipe[4] = {h2d, d2h, ctx->hp_comp[0], ctx->hp_comp[1]};
  // the pipeline starts after the work already on the caller's stream
  BL_CUDA(cudaEventRecord(ev[EV_START], st));
  for (cudaStream_t s_ : pipe) BL_CUDA(cudaStreamWaitEvent(s_, ev[EV_START], 0));
  // a view of particles [off, off + cn) of a device SoA whose coordinate
  // arrays are `stride` floats apart
  auto view = [&](float *base, size_t stride, int64_t off, int64_t cn) {
    bl_bunch v{};
    v.x = base + off;
    v.px = base + stride + off;
    v.y = base + 2 * stride + off;
    v.py = base + 3 * stride + off;
    v.t = base + 4 * stride + off;
    v.pt = base + 5 * stride + off;
    v.n = cn;
    v.n_bunch = 1;
    v.dtype = BL_F32;
    v.gamma_ref = g_in;
    return v;
  };
  auto region = [&](int64_t k) { return want ? dred + (size_t)k * per : nullptr; };
  auto region_nf = [&](int64_t k) {
    return want ? reinterpret_cast<unsigned long long *>(dred + (size_t)k * per + per - 1) : nullptr;
  };
  auto copies = [&](float *dst_base, size_t dst_stride, const float *const *src, int64_t off,
                    int64_t cn, bool to_dev, cudaStream_t cs) {
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 6 && e == cudaSuccess; ++c) {
      float *d = dst_base + (size_t)c * dst_stride + (to_dev ? off : 0);
      e = to_dev ? cudaMemcpyAsync(d, src[c] + off, cn * sizeof(float), cudaMemcpyHostToDevice, cs)
                 : cudaMemcpyAsync(out_host[c] + off, dst_base + (size_t)c * dst_stride + off,
                                   cn * sizeof(float), cudaMemcpyDeviceToHost, cs);
    }
    return e;
  };
  // record `e_` on `from`, make `to` wait for it (the event can be reused at once)
  auto link = [&](cudaStream_t from, cudaStream_t to, cudaEvent_t e_) {
    cudaError_t e = cudaEventRecord(e_, from);
    return e == cudaSuccess ? cudaStreamWaitEvent(to, e_, 0) : e;
  };
  bl_status r = BL_OK;
  cudaError_t e = cudaSuccess;
  if (whole) {
    // head, chunk by chunk on alternating compute streams, each chunk as soon
    // as it has arrived
    for (int64_t i = 0; i < nchunks && r == BL_OK && e == cudaSuccess; ++i) {
      cudaStream_t cs = ctx->hp_comp[i % 2];
      const int64_t off = i * chunk, cn = std::min(chunk, n - off);
      e = copies(dbuf, n, in_host, off, cn, true, h2d);
      if (e == cudaSuccess) e = link(h2d, cs, ev[EV_IN]);
      if (e != cudaSuccess) break;
      bl_bunch v = view(dbuf, n, off, cn);
      r = track_checks(&v, L);
      if (r == BL_OK) r = track_enqueue_range(&v, L, 0, h_end, region(i), region_nf(i), cs);
    }
    // the groups in between, once, on the whole bunch
    if (r == BL_OK && e == cudaSuccess) e = link(ctx->hp_comp[1], ctx->hp_comp[0], ev[EV_IN + 1]);
    if (r == BL_OK && e == cudaSuccess) {
      bl_bunch v = view(dbuf, n, 0, n);
      r = track_enqueue_range(&v, L, h_end, t_begin, region(nchunks), region_nf(nchunks),
                              ctx->hp_comp[0]);
    }
    if (r == BL_OK && e == cudaSuccess) e = link(ctx->hp_comp[0], ctx->hp_comp[1], ev[EV_IN + 2]);
    // tail, chunk by chunk, each chunk copied out as soon as it is done
    for (int64_t i = 0; i < nchunks && r == BL_OK && e == cudaSuccess; ++i) {
      cudaStream_t cs = ctx->hp_comp[i % 2];
      const int64_t off = i * chunk, cn = std::min(chunk, n - off);
      bl_bunch v = view(dbuf, n, off, cn);
      r = track_enqueue_range(&v, L, t_begin, G, region(nchunks + 1 + i),
                              region_nf(nchunks + 1 + i), cs);
      if (r == BL_OK) e = link(cs, d2h, ev[EV_TRACKED]);
      if (r == BL_OK && e == cudaSuccess) e = copies(dbuf, n, nullptr, off, cn, false, d2h);
    }
  } else {
    for (int64_t i = 0; i < nchunks && r == BL_OK && e == cudaSuccess; ++i) {
      const int b = (int)(i % HOST_BUFS);
      cudaStream_t cs = ctx->hp_comp[i % 2];
      const int64_t off = i * chunk, cn = std::min(chunk, n - off);
      float *d = dbuf + (size_t)b * 6 * chunk;
      // copy in once the chunk that last used this buffer has been copied out
      if (i >= HOST_BUFS) e = cudaStreamWaitEvent(h2d, ev[EV_OUT + b], 0);
      // the chunk buffer holds coordinate arrays `chunk` floats apart; the
      // copies address it as a view at offset 0
      for (int c = 0; c < 6 && e == cudaSuccess; ++c)
        e = cudaMemcpyAsync(d + (size_t)c * chunk, in_host[c] + off, cn * sizeof(float),
                            cudaMemcpyHostToDevice, h2d);
      if (e == cudaSuccess) e = link(h2d, cs, ev[EV_IN + b]);
      if (e != cudaSuccess) break;
      bl_bunch v = view(d, chunk, 0, cn);
      r = track_checks(&v, L);
      if (r == BL_OK) r = track_enqueue_range(&v, L, 0, G, region(i), region_nf(i), cs);
      if (r != BL_OK) break;
      e = link(cs, d2h, ev[EV_TRACKED + b]);
      for (int c = 0; c < 6 && e == cudaSuccess; ++c)
        e = cudaMemcpyAsync(out_host[c] + off, d + (size_t)c * chunk, cn * sizeof(float),
                            cudaMemcpyDeviceToHost, d2h);
      if (e == cudaSuccess) e = cudaEventRecord(ev[EV_OUT + b], d2h);
    }
  }
  if (r == BL_OK && e != cudaSuccess) r = set_error(BL_ERR_CUDA, cudaGetErrorString(e));
  // join: the caller's stream waits for the whole pipeline (also after an
  // error, so that no copy into the caller's buffers is in flight on return)
  for (int k = 0; k < 4; ++k) {
    cudaEventRecord(ev[EV_JOIN + k], pipe[k]);
    cudaStreamWaitEvent(st, ev[EV_JOIN + k], 0);
  }
  std::vector<double> hred;
  if (r == BL_OK && want) {
    hred.resize((size_t)nregions * per);
    const cudaError_t e2 = cudaMemcpyAsync(hred.data(), dred, hred.size() * sizeof(double),
                                           cudaMemcpyDeviceToHost, st);
    if (e2 != cudaSuccess) r = set_error(BL_ERR_CUDA, cudaGetErrorString(e2));
  }
  const cudaError_t es = cudaStreamSynchronize(st);
  if (r != BL_OK) return r;
  if (es != cudaSuccess) return set_error(BL_ERR_CUDA, cudaGetErrorString(es));
  *gamma_ref = L->plan.gamma_out;
  if (!want) return BL_OK;
  // each reduction point from the regions that computed it: in the chunked
  // mode every chunk's; in the whole-bunch mode the head's or the tail's
  // chunks, or the middle's single region
  std::vector<int> grp_of_red((size_t)R, 0);
  for (size_t g = 0; g < G; ++g)
    if (red_of[g] >= 0) grp_of_red[red_of[g]] = (int)g;
  std::vector<double> pooled((size_t)R * 28);
  std::vector<const double *> parts;
  for (int rr = 0; rr < R; ++rr) {
    parts.clear();
    const size_t g = (size_t)grp_of_red[rr];
    if (!whole) {
      for (int64_t i = 0; i < nchunks; ++i) parts.push_back(hred.data() + (size_t)i * per + (size_t)rr * 28);
    } else if (g < h_end) {
      for (int64_t i = 0; i < nchunks; ++i) parts.push_back(hred.data() + (size_t)i * per + (size_t)rr * 28);
    } else if (g >= t_begin) {
      for (int64_t i = 0; i < nchunks; ++i)
        parts.push_back(hred.data() + (size_t)(nchunks + 1 + i) * per + (size_t)rr * 28);
    } else {
      parts.push_back(hred.data() + (size_t)nchunks * per + (size_t)rr * 28);
    }
    pool_moments(parts, pooled.data() + (size_t)rr * 28);
  }
  unsigned long long nonfin = 0;
  for (int64_t k = 0; k < nregions; ++k) {
    unsigned long long c = 0;
    std::memcpy(&c, hred.data() + (size_t)k * per + per - 1, sizeof(c));
    nonfin += c;
  }
  if (nonfinite_out) *nonfinite_out = (int64_t)nonfin;
  if (moments_out) expand_moments(L, 1, pooled.data(), moments_out);
  if (nonfin) return set_error(BL_ERR_NONFINITE, std::to_string(nonfin) + " non-finite particles seen");
  return BL_OK;
}

int32_t bl_track_num_reductions(const bl_lattice *lat) {
  if (!lat) return -1;
  std::vector<int> red_of;
  return reduction_points(lat, &red_of);
}

bl_status bl_track_async(bl_bunch *b, const bl_lattice *lat_c, double *reduced_dev,
                         bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  BL_CHECK(lat_c, "lattice is NULL");
  bl_lattice_s *L = const_cast<bl_lattice_s *>(lat_c);
  BL_TRY(track_checks(b, L));
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  std::lock_guard<std::mutex> lk(L->mu);
  auto &P = L->plan;
  int dev = -1;
  BL_CUDA(cudaGetDevice(&dev));
  const bool planned = P.valid && P.gamma_in == b->gamma_ref && P.dtype == b->dtype &&
                       P.n_bunch == b->n_bunch && P.device == dev;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  BL_CUDA(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    BL_CHECK(planned, "bl_track_async under stream capture needs the lattice's plan for this "
                      "bunch: call bl_track (or bl_track_async) once before capturing");
  BL_TRY(build_plan(L, b->gamma_ref, b->dtype, b->n_bunch, st));
  std::vector<int> red_of;
  const int R = reduction_points(L, &red_of);
  unsigned long long *nf = reduced_dev
      ? reinterpret_cast<unsigned long long *>(reduced_dev + (size_t)R * b->n_bunch * 28)
      : nullptr;
  return track_enqueue(b, L, reduced_dev, nf, st);
}

bl_status bl_track_expand_moments(const bl_lattice *lat_c, int32_t n_bunch,
                                  const double *reduced_host, double *moments_out) {
  BL_CHECK(lat_c && reduced_host && moments_out, "NULL argument");
  const bl_lattice_s *L = lat_c;
  BL_CHECK(L->plan.valid && L->plan.n_bunch == n_bunch,
           "the lattice has no plan for this bunch count: track it first");
  expand_moments(L, n_bunch, reduced_host, moments_out);
  return BL_OK;
}

bl_status bl_moments(const bl_bunch *b, double *out, bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  std::string why;
  BL_CHECK(bunch_dims_ok(b, &why), why);
  BL_CHECK(out, "out is NULL");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  void *p = nullptr;
  BL_TRY(ws_get(st, WS_MOMENTS, (size_t)b->n_bunch * 28 * sizeof(double), &p));
  BL_TRY(moments_device(b, (double *)p, nullptr, st));
  BL_CUDA(cudaMemcpyAsync(out, p, (size_t)b->n_bunch * 28 * sizeof(double), cudaMemcpyDefault, st));
  return BL_OK;
}

bl_status bl_apply_linear(bl_bunch *b, const double *M, int32_t per_bunch, bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  std::string why;
  BL_CHECK(bunch_dims_ok(b, &why), why);
  BL_CHECK(M, "matrix is NULL");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  const int nm = per_bunch ? b->n_bunch : 1;
  for (int i = 0; i < nm * 36; ++i) BL_CHECK(std::isfinite(M[i]), "matrix entries must be finite");
  const size_t esz = b->dtype == BL_F32 ? 4 : 8;
  void *d = nullptr;
  BL_TRY(ws_get(st, WS_MATS, (size_t)nm * 36 * esz, &d));
  std::vector<uint8_t> h((size_t)nm * 36 * esz);
  for (int i = 0; i < nm * 36; ++i) {
    if (esz == 4) { float v = (float)M[i]; std::memcpy(&h[i * 4], &v, 4); }
    else std::memcpy(&h[i * 8], &M[i], 8);
  }
  // a pageable-source copy has consumed the host buffer when it returns
  BL_CUDA(cudaMemcpyAsync(d, h.data(), h.size(), cudaMemcpyHostToDevice, st));
  const int64_t *off = b->n_bunch > 1 ? b->offsets_dev : nullptr;
  if (b->dtype == BL_F32) {
    Soa<float> z = soa_of<float>(b);
    BL_CUDA(launch_stream<float>(z, z, b->n, off, b->n_bunch, (const float *)d, per_bunch ? 1 : 0,
                                 nullptr, true, false, nullptr, st));
  } else {
    Soa<double> z = soa_of<double>(b);
    BL_CUDA(launch_stream<double>(z, z, b->n, off, b->n_bunch, (const double *)d, per_bunch ? 1 : 0,
                                  nullptr, true, false, nullptr, st));
  }
  return BL_OK;
}

bl_status bl_push_stage(bl_bunch *b, const bl_element *stage, bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  std::string why;
  BL_CHECK(bunch_dims_ok(b, &why), why);
  BL_CHECK(stage && stage->kind == BL_PLASMA, "stage must be a BL_PLASMA element");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  StageTrack tr;
  BL_TRY(stage_track(*stage, b->gamma_ref, b->dtype, &tr));
  const size_t bytes = (size_t)tr.c.nsteps * 16 * (b->dtype == BL_F32 ? 4 : 8);
  void *d = nullptr;
  BL_TRY(ws_get(st, WS_TABLES, bytes, &d));
  const void *src = b->dtype == BL_F32 ? (const void *)tr.table32.data() : (const void *)tr.table64.data();
  BL_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st));
  if (b->dtype == BL_F32)
    BL_CUDA(launch_pusher<float>(soa_of<float>(b), b->n, tr.c, (const float *)d, st));
  else
    BL_CUDA(launch_pusher<double>(soa_of<double>(b), b->n, tr.c, (const double *)d, st));
  b->gamma_ref = tr.c.gamma_out;
  return BL_OK;
}

}  // extern "C"

// Diagnostic entry point (declared in include/bl_debug.h): the FP64 pooling
// that bl_track_host applies to chunked moment reductions.
extern "C" int bl_debug_pool_moments(const double *parts, int32_t k, double *out) {
  if (!parts || !out || k < 1) return 1;
  std::vector<const double *> v((size_t)k);
  for (int32_t i = 0; i < k; ++i) v[i] = parts + (size_t)i * 28;
  pool_moments(v, out);
  return 0;
}
