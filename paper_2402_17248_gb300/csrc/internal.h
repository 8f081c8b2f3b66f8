// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/bl.h"

namespace bl {

template <typename T> struct Soa { T *c[6]; };

// Particles per block of the streaming kernels and its thread count.
constexpr int STREAM_THREADS = 256;
constexpr int64_t STREAM_CHUNK = 4096;

inline int64_t stream_blocks(int64_t n) { return (n + STREAM_CHUNK - 1) / STREAM_CHUNK; }
// Partial-sum slots of a segmented reduction: slot (bunch + block) is unique
// because bunches and blocks both tile the particle range contiguously.
inline int64_t stream_slots(int64_t n, int n_bunch) { return stream_blocks(n) + n_bunch; }

// ---- streaming kernels (linear.cu) ----
// z_out = M_b (z_in - c_b) for particles of bunch b (c_b = 0 when c == NULL),
// optionally reducing moments of z_in into `partials` (28 doubles per slot:
// bunch b's sums over unit k, k = particle / *unit, go to slot b + k, so at
// most stream_slots(n, n_bunch) slots are written). *unit (if non-NULL)
// receives the unit length that launch_moments_finalize must be given.
template <typename T>
cudaError_t launch_stream(Soa<T> zin, Soa<T> zout, int64_t n, const int64_t *offsets,
                          int n_bunch, const T *mats, int per_bunch, const T *centers,
                          bool apply, bool moments, double *partials, cudaStream_t st,
                          int64_t *unit = nullptr);
cudaError_t launch_moments_finalize(const double *partials, const int64_t *offsets,
                                    int n_bunch, int64_t n, int64_t unit, double *out,
                                    unsigned long long *nonfinite, cudaStream_t st);
// lambda <- M_b^T lambda and cross[b] += sum_i lambda_out,i z_in,i^T (36 per slot).
template <typename T>
cudaError_t launch_linear_adjoint(Soa<T> lam, Soa<T> zin, int64_t n, const int64_t *offsets,
                                  int n_bunch, const T *mats, int per_bunch,
                                  double *partials, cudaStream_t st);
cudaError_t launch_cross_finalize(const double *partials, const int64_t *offsets,
                                  int n_bunch, int64_t n, double *out, cudaStream_t st);

// ---- plasma stage pusher (pusher.cu) ----
struct StageConsts {
  double kp, g, K0, h;
  double bg_in, gamma_in, bg_out, gamma_out;
  double uz_ref_out;
  int nsteps;
};
// The stage constants in FP32 for the FP32 pusher (push_f32.cuh).
struct ConstsF {
  float kp, g, K0, h, h2, h6;
  float bg_in, gamma_in, bg_out, gamma_out, uz_out;
  int nsteps;
};
ConstsF consts_f(const StageConsts &c);
// table: nsteps*4 entries of 4 values (T), see pusher.cu for the layout.
template <typename T>
cudaError_t launch_pusher(Soa<T> z, int64_t n, const StageConsts &c, const T *table,
                          cudaStream_t st);
// FP32 push of the particles list[0 .. min(*count, capacity)) only.
cudaError_t launch_pusher_list(Soa<float> z, const int64_t *list, const unsigned long long *count,
                               int64_t capacity, const StageConsts &c, const float *table,
                               int num_sms, cudaStream_t st);

// ---- MLP (mlp_fwd.cu, mlp_train.cu) ----
constexpr int MLP_H = 128;
constexpr int MLP_NPARAM = 128 * 6 + 128 + 3 * (128 * 128 + 128) + 6 * 128 + 6;  // 51206
// Offsets of W[l] and b[l] in the flat FP32 parameter vector.
inline int mlp_w_off(int l) {
  static const int o[5] = {0, 896, 17408, 33920, 50432};
  return o[l];
}
inline int mlp_b_off(int l) {
  static const int o[5] = {768, 17280, 33792, 50304, 51200};
  return o[l];
}
// Size in bytes of the BF16 UMMA weight image and its FP32 bias block.
constexpr int MLP_IMG_W0 = 128 * 16 * 2;
constexpr int MLP_IMG_WH = 128 * 128 * 2;
constexpr int MLP_IMG_W4 = 16 * 128 * 2;
// Bias blocks: N x 16 K-major blocks whose first two K columns hold the
// bias split into BF16 hi and lo parts (added by one extra MMA K-step).
constexpr int MLP_IMG_BH = 128 * 16 * 2;
constexpr int MLP_IMG_B4 = 16 * 16 * 2;
constexpr int MLP_IMG_BYTES =
    MLP_IMG_W0 + 3 * MLP_IMG_WH + MLP_IMG_W4 + 3 * MLP_IMG_BH + MLP_IMG_B4;  // 119296
constexpr int MLP_BIAS_FLOATS = 3 * 128 + 16;

struct MlpNorm { double mu_in[6], inv_sd_in[6], mu_out[6], sd_out[6]; };
// The same constants as double-float pairs (hi, lo) for the inference kernel.
struct MlpNormF { float mu_in[6][2], inv_sd_in[6][2], mu_out[6][2], sd_out[6][2]; };

cudaError_t launch_mlp_pack(const float *params, uint8_t *img, float *bias, float *wt,
                            float *wn, cudaStream_t st);
// err: device word that receives BL_DEVERR_* flags of bounded waits.
// Training-input box of a surrogate; particles outside it are not mapped
// but pushed by the plain FP32 pusher of the stage (constants stage, RK4
// reference table `table`): by the surrogate kernel's own fallback warp,
// or, past its per-CTA queue, listed in fb_list (fb_count counts them) for
// launch_pusher_list.
struct MlpDomain {
  float lo[6], hi[6];
  int64_t *fb_list;
  unsigned long long *fb_count;
  int64_t fb_cap;
  ConstsF stage;
  const float *table;
  int fused;  // 1: the fallback warp pushes (up to its queue); 0: every particle goes to the list
};
cudaError_t launch_mlp_forward(Soa<float> z, int64_t n, const uint8_t *img, const MlpNorm &nrm,
                               int num_sms, unsigned *err, cudaStream_t st,
                               const MlpDomain *dom = nullptr);
cudaError_t mlp_forward_configure();

// ---- wide PReLU networks (wide_mlp.cu) ----
struct WideNet {
  struct Layer {
    uint8_t *W = nullptr;  // BF16 weights, tiled (see wide_weight_offset)
    float *b = nullptr;    // FP32 bias, N_pad entries
    const float *slope = nullptr;  // PReLU slope (hidden layers), device (inside the masters)
    int K = 0, N = 0;      // real widths
    int K_pad = 0, N_pad = 0;
  };
  std::vector<Layer> layers;
  MlpNorm nrm{};
  // flat FP32 masters [W_0, b_0, ..., W_{L-1}, b_{L-1}, slopes] on the device
  float *P = nullptr;
  std::vector<int64_t> w_off, b_off;
  int64_t slope_off = 0, nparam = 0;
  int max_width = 0;
};
// Byte offset of weight (n, k) in a layer's tiled BF16 image.
size_t wide_weight_offset(int n, int k, int N_pad);
cudaError_t wide_mlp_configure();
cudaError_t launch_wide_mlp(Soa<float> z, int64_t n, const WideNet &net, uint8_t *act0,
                            uint8_t *act1, int num_sms, unsigned *err, cudaStream_t st);
// Rebuild every layer's BF16 image and bias array from the flat masters.
cudaError_t launch_wide_pack(const WideNet &net, cudaStream_t st);
// Device bytes of the training work buffers for a minibatch of `batch` pairs.
size_t wide_train_bytes(const WideNet &net, int64_t batch);
// Minibatch gradient (flat layout, into G) and loss (device float, or NULL)
// of the MSE on normalised targets; inputs/targets coordinate-major [6][ld].
cudaError_t launch_wide_grad(const WideNet &net, const float *in, const float *out, int64_t ld,
                             const int64_t *idx, int64_t batch, float *G, float *loss_out,
                             void *ws, int num_sms, unsigned *err, cudaStream_t st);
cudaError_t launch_wide_adam(float *P, const float *G, float *M, float *V, int64_t n, double lr,
                             double b1, double b2, double eps, int step, cudaStream_t st);

// Partial-gradient row stride (floats) of the training kernels, padded for
// 16-byte aligned vector stores.
constexpr int MLP_PSTRIDE = 51208;
int mlp_grad_blocks(int64_t count);

// Minibatch MSE gradient with the SIMT kernels (mlp_train.cu): in/out are
// coordinate-major [6][ld] FP32; partials: mlp_grad_blocks(batch) rows of
// MLP_PSTRIDE floats; loss_partials: one double per block.
// scale_count (0: batch) is the sample count the MSE is averaged over, so a
// large minibatch can be processed in chunks with the whole batch's scale.
cudaError_t launch_mlp_grad(const float *in, const float *out, int64_t ld, const int64_t *idx,
                            int64_t batch, const float *wt, const float *wn, const MlpNorm &nrm,
                            float *partials, double *loss_partials, int *nblocks_out,
                            cudaStream_t st, int64_t scale_count = 0);
// acc[i] += rows[b][i] (i < MLP_NPARAM) and *acc_loss += loss_rows[b] for
// b = 0 .. nrows-1, in FP64: the partial rows of one chunk of a minibatch
// added to the running sums. With `row_out`, the sums are then also written
// to it as one FP32 partial row.
cudaError_t launch_mlp_rows_accumulate(const float *rows, int nrows, const double *loss_rows,
                                       double *acc, double *acc_loss, float *row_out,
                                       cudaStream_t st);
// Sum partial gradients; if step > 0 apply Adam with bias correction for
// step t = step. grad_out (device, NPARAM) and loss_out (device) optional.
// Minibatch MSE gradient on the tensor cores (mlp_train_tc.cu): one
// partial row per 128-sample tile (mlp_train_tc_tiles(batch) rows), from the
// inference weight image and FP32 bias block; scratch holds the tiles' saved
// activations (mlp_train_tc_scratch_bytes(batch) bytes).
inline int mlp_train_tc_tiles(int64_t batch) { return (int)((batch + 127) / 128); }
size_t mlp_train_tc_scratch_bytes(int64_t batch);
cudaError_t mlp_train_tc_configure();
cudaError_t launch_mlp_grad_tc(const float *in, const float *out, int64_t ld, const int64_t *idx,
                               int64_t batch, const uint8_t *img, const float *bias,
                               const MlpNorm &nrm, float *partials, double *loss_partials,
                               uint8_t *scratch, int num_sms, unsigned *err, cudaStream_t st,
                               int64_t scale_count = 0);
// Which gradient kernel the training entry points use: false = tensor cores
// (default), true = the SIMT FP32 kernel (bl_debug_train_kernel).
bool mlp_train_use_simt();
cudaError_t launch_mlp_reduce_adam(const float *partials, int nblocks, const double *loss_partials,
                                   int64_t batch, float *params, float *m, float *v, double lr,
                                   double b1, double b2, double eps, int step, float *loss_out,
                                   float *grad_out, cudaStream_t st);
cudaError_t launch_mlp_loss(const float *in, const float *out, int64_t ld, const int64_t *idx,
                            int64_t count, const float *wt, const float *wn, const MlpNorm &nrm,
                            double *loss_partials, int *nblocks_out, cudaStream_t st);
cudaError_t launch_loss_finalize(const double *loss_partials, int nblocks, int64_t count,
                                 double *loss_out, cudaStream_t st);
// lam <- J_F(zin)^T lam for every particle (raw coordinates on both sides),
// on the tensor cores with the inference weight image (mlp_vjp.cu).
cudaError_t launch_mlp_vjp(Soa<float> zin, Soa<float> lam, int64_t n, const uint8_t *img,
                           const MlpNorm &nrm, int num_sms, unsigned *err, cudaStream_t st);
cudaError_t mlp_vjp_configure();


}  // namespace bl
