// C ABI: gradient of a final beam quantity with respect to every quadrupole
// strength (reverse mode through segment maps and surrogate stages).
//
// Forward: the entry state of every group (segment or stage) is saved as a
// checkpoint. Seed: lambda_i = dJ/dz_i = K_b (z_i - mean_b), with K_b from
// the final moments. Reverse: a segment maps lambda <- M^T lambda and reduces
// the cross moment C = sum_i lambda_out,i z_in,i^T (z_in: the checkpoint);
// a surrogate stage maps lambda through the MLP's vector-Jacobian product,
// recomputing the forward activations from its checkpoint. For quadrupole q
// of a segment with elements M_1..M_m (q-th derivative D_q = dM_q/dk),
// dJ/dk_q = sum_ab (R_q D_q P_q)_ab C_ab with P_q = M_{q-1}..M_1 and
// R_q = M_m..M_{q+1}, evaluated on the host in FP64.
#include <cmath>

#include "runtime.h"

using namespace bl;

extern "C" {

bl_status bl_track_grad(bl_bunch *b, const bl_lattice *lat_c, int32_t objective, double *J_out,
                        double *dJ_dk, bl_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  std::string why;
  BL_CHECK(lat_c, "lattice is NULL");
  BL_CHECK(bunch_dims_ok(b, &why), why);
  BL_CHECK(b->dtype == BL_F32, "the adjoint needs an FP32 bunch");
  BL_CHECK(b->n > 0, "the adjoint needs particles");
  BL_CHECK(objective >= BL_OBJ_EPS_N_X && objective <= BL_OBJ_SIGMA_Y, "unknown objective");
  BL_CHECK(J_out && dJ_dk, "J_out and dJ_dk must be given");
  bl_lattice_s *L = const_cast<bl_lattice_s *>(lat_c);
  BL_CHECK(L->n_bunch_k == 0 || L->n_bunch_k == b->n_bunch,
           "lattice per-bunch strengths do not match the bunch count");
  for (const auto &gr : L->groups)
    if (gr.stage) BL_CHECK(L->els[gr.first].surrogate, "the adjoint covers surrogate stages only");
  DevCtx *ctx = nullptr;
  BL_TRY(current_ctx(&ctx));
  std::lock_guard<std::mutex> lk(L->mu);
  BL_TRY(build_plan(L, b->gamma_ref, BL_F32, b->n_bunch, st));
  const auto &P = L->plan;
  const size_t G = L->groups.size();
  const int64_t n = b->n;
  const int nbunch = b->n_bunch;
  const int per_bunch = L->n_bunch_k > 0 ? 1 : 0;
  const int64_t *off = nbunch > 1 ? b->offsets_dev : nullptr;

  void *ck = nullptr, *lam = nullptr;
  BL_TRY(ws_get(st, WS_CKPT, G * 6 * (size_t)n * sizeof(float), &ck));
  BL_TRY(ws_get(st, WS_LAMBDA, 6 * (size_t)n * sizeof(float), &lam));
  auto ckpt = [&](size_t g) {
    Soa<float> s;
    for (int c = 0; c < 6; ++c) s.c[c] = (float *)ck + (g * 6 + c) * (size_t)n;
    return s;
  };
  Soa<float> z = soa_of<float>(b);
  Soa<float> lm;
  for (int c = 0; c < 6; ++c) lm.c[c] = (float *)lam + c * (size_t)n;

  // ---- forward with checkpoints
  for (size_t g = 0; g < G; ++g) {
    Soa<float> cp = ckpt(g);
    for (int c = 0; c < 6; ++c)
      BL_CUDA(cudaMemcpyAsync(cp.c[c], z.c[c], n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    const auto &gr = L->groups[g];
    if (gr.stage) {
      BL_TRY(bl_surrogate_apply(L->els[gr.first].surrogate, b, st));
    } else {
      const float *mats = (const float *)((const uint8_t *)P.d_mats + P.mat_off[g]);
      BL_CUDA(launch_stream<float>(z, z, n, off, nbunch, mats, per_bunch, nullptr, true, false,
                                   nullptr, st));
    }
  }
  b->gamma_ref = P.gamma_out;

  // ---- final moments and the seed
  void *mom = nullptr;
  BL_TRY(ws_get(st, WS_MOMENTS, (size_t)nbunch * 28 * sizeof(double), &mom));
  BL_TRY(moments_device(b, (double *)mom, nullptr, st));
  std::vector<double> m((size_t)nbunch * 28);
  BL_CUDA(cudaMemcpyAsync(m.data(), mom, m.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  BL_CUDA(cudaStreamSynchronize(st));
  const double gam = P.gamma_out, bg = std::sqrt(gam * gam - 1.0);
  const int a0 = (objective == BL_OBJ_EPS_N_X || objective == BL_OBJ_SIGMA_X) ? 0 : 2;
  const bool eps = objective == BL_OBJ_EPS_N_X || objective == BL_OBJ_EPS_N_Y;
  std::vector<float> K((size_t)nbunch * 36, 0.0f), cen((size_t)nbunch * 6, 0.0f);
  auto sidx = [](int a, int c) {  // index of S_ac (a <= c) in the 28-vector
    int j = 0;
    for (int p = 0; p < 6; ++p)
      for (int q = p; q < 6; ++q) {
        if (p == a && q == c) return 7 + j;
        ++j;
      }
    return -1;
  };
  for (int bb = 0; bb < nbunch; ++bb) {
    const double *mb = m.data() + (size_t)bb * 28;
    const double N = mb[0];
    for (int c = 0; c < 6; ++c) cen[bb * 6 + c] = (float)mb[1 + c];
    const double Sxx = mb[sidx(a0, a0)], Spp = mb[sidx(a0 + 1, a0 + 1)], Sxp = mb[sidx(a0, a0 + 1)];
    float *Kb = K.data() + (size_t)bb * 36;
    if (N <= 0) { J_out[bb] = 0.0; continue; }
    if (eps) {
      const double D = Sxx * Spp - Sxp * Sxp;
      BL_CHECK(D > 0.0, "emittance objective of a bunch with zero emittance");
      J_out[bb] = bg * std::sqrt(D);
      const double c = bg / (N * std::sqrt(D));
      Kb[a0 * 6 + a0] = (float)(c * Spp);
      Kb[a0 * 6 + a0 + 1] = (float)(-c * Sxp);
      Kb[(a0 + 1) * 6 + a0 + 1] = (float)(c * Sxx);
      Kb[(a0 + 1) * 6 + a0] = (float)(-c * Sxp);
    } else {
      BL_CHECK(Sxx > 0.0, "beam-size objective of a bunch with zero size");
      J_out[bb] = std::sqrt(Sxx);
      Kb[a0 * 6 + a0] = (float)(1.0 / (N * std::sqrt(Sxx)));
    }
  }
  void *dK = nullptr, *dC = nullptr;
  BL_TRY(ws_get(st, WS_MATS, K.size() * sizeof(float) + cen.size() * sizeof(float), &dK));
  float *dcen = (float *)dK + K.size();
  BL_CUDA(cudaMemcpyAsync(dK, K.data(), K.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  BL_CUDA(cudaMemcpyAsync(dcen, cen.data(), cen.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  BL_CUDA(launch_stream<float>(z, lm, n, off, nbunch, (const float *)dK, 1, dcen, true, false,
                               nullptr, st));

  // ---- reverse sweep
  size_t nseg = 0;
  for (const auto &gr : L->groups) nseg += gr.stage ? 0 : 1;
  BL_TRY(ws_get(st, WS_CROSS, std::max<size_t>(1, nseg) * nbunch * 36 * sizeof(double), &dC));
  void *part = nullptr;
  BL_TRY(ws_get(st, WS_PARTIALS, (size_t)stream_slots(n, nbunch) * 36 * sizeof(double), &part));
  std::vector<int> seg_index(G, -1);
  {
    int si = 0;
    for (size_t g = 0; g < G; ++g)
      if (!L->groups[g].stage) seg_index[g] = si++;
  }
  for (size_t gi = G; gi-- > 0;) {
    const auto &gr = L->groups[gi];
    if (gr.stage) {
      const bl_surrogate *s = L->els[gr.first].surrogate;
      if (!ctx->mlp_vjp_configured) {
        BL_CUDA(mlp_vjp_configure());
        ctx->mlp_vjp_configured = true;
      }
      BL_CUDA(launch_mlp_vjp(ckpt(gi), lm, n, s->img, s->nrm, ctx->num_sms, ctx->err_word, st));
    } else {
      const float *mats = (const float *)((const uint8_t *)P.d_mats + P.mat_off[gi]);
      BL_CUDA(launch_linear_adjoint<float>(lm, ckpt(gi), n, off, nbunch, mats, per_bunch,
                                           (double *)part, st));
      BL_CUDA(launch_cross_finalize((const double *)part, off, nbunch, n,
                                    (double *)dC + (size_t)seg_index[gi] * nbunch * 36, st));
    }
  }
  std::vector<double> C(std::max<size_t>(1, nseg) * nbunch * 36);
  BL_CUDA(cudaMemcpyAsync(C.data(), dC, C.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  BL_CUDA(cudaStreamSynchronize(st));

  // ---- quad gradients on the host (FP64)
  const int nq = L->n_quads;
  for (int bb = 0; bb < nbunch; ++bb) {
    int q = 0;
    for (size_t g = 0; g < G; ++g) {
      const auto &gr = L->groups[g];
      if (gr.stage) continue;
      const double *Cb = C.data() + ((size_t)seg_index[g] * nbunch + bb) * 36;
      const int mi = per_bunch ? bb : 0;
      const int m_el = gr.last - gr.first + 1;
      for (int e = gr.first; e <= gr.last; ++e) {
        const bl_element &el = L->els[e];
        if (el.kind != BL_QUAD) continue;
        Mat6 Pm = mat_identity(), Rm = mat_identity();
        for (int j = 0; j < e - gr.first; ++j) Pm = mat_mul(P.el_mats[g][j][mi], Pm);
        for (int j = e - gr.first + 1; j < m_el; ++j) Rm = mat_mul(P.el_mats[g][j][mi], Rm);
        const double k = L->pbk[e].empty() ? el.k : L->pbk[e][bb];
        const Mat6 Gm = mat_mul(Rm, mat_mul(element_dmatrix_dk(el, k, bg), Pm));
        double s = 0.0;
        for (int i = 0; i < 36; ++i) s += Gm[i] * Cb[i];
        dJ_dk[(size_t)bb * nq + q] = s;
        ++q;
      }
    }
  }
  return BL_OK;
}

}  // extern "C"
