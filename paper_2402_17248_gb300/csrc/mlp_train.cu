// Training and differentiation of the stage surrogate (Sec. 3: MSE loss on
// normalised data, Adam over minibatches; Sec. 4.4 for gradients of the
// tracked beam with respect to its inputs).
//
// One block holds S samples; thread j owns hidden feature j. The forward pass
// reproduces the inference datapath's rounding points (BF16 weights, BF16
// network input and hidden activations, FP32 sums, GELU in tanh form with
// the hardware tanh); the backward pass is FP32 reverse mode treating the
// BF16 roundings as the identity. A block writes its partial weight gradient
// (flat parameter layout) and its partial loss; a second kernel sums the
// partials and applies Adam (Kingma and Ba, Algorithm 1) to the FP32 masters.
#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace bl {

namespace {

constexpr int S = 16;       // samples per block
constexpr int NT = 128;     // threads per block
// Offsets of W[l] and b[l] in the flat parameter vector.
__host__ __device__ constexpr int woff(int l) {
  return l == 0 ? 0 : (l == 1 ? 896 : (l == 2 ? 17408 : (l == 3 ? 33920 : 50432)));
}
__host__ __device__ constexpr int boff(int l) {
  return l == 0 ? 768 : (l == 1 ? 17280 : (l == 2 ? 33792 : (l == 3 ? 50304 : 51200)));
}
constexpr float C0 = 0.7978845608028654f;
constexpr float C1 = 0.7978845608028654f * 0.044715f;

enum Mode { MODE_TRAIN = 0, MODE_LOSS = 1 };

BL_DEV float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

BL_DEV void gelu_fwd(float x, float &y, float &dy) {
  const float x2 = x * x;
  const float u = x * fmaf(C1, x2, C0);
  const float t = tc::tanh_approx(u);
  y = 0.5f * x * (1.0f + t);
  const float du = fmaf(3.0f * C1, x2, C0);
  dy = 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * du;
}

struct Smem {
  float h0[S][8];          // normalised input (BF16 hi + lo)
  float h[4][S][128];      // h_1..h_4 (BF16-rounded GELU outputs)
  float dg[4][S][128];     // GELU'(a_0..a_3)
  float d[S][128];         // current delta (dL/da_l)
  float a4[S][8];          // network output (normalised)
  float d4[S][8];          // dL/da_4
  double loss[NT / 32];
};

// Inputs zin and targets zout are
// six coordinate arrays indexed by column idx[s] (or s when idx is NULL).
template <int MODE>
__global__ void __launch_bounds__(NT)
mlp_grad_kernel(Soa<float> zin, Soa<float> zout, const int64_t *__restrict__ idx, int64_t count,
                const float *__restrict__ wt, const float *__restrict__ wn, MlpNorm nrm,
                float *__restrict__ part, double *__restrict__ loss_part,
                double inv_count6) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t s0 = (int64_t)blockIdx.x * S;
  const int ns = (count - s0 < S) ? (int)(count - s0) : S;

  // ---- inputs: FP64 normalisation, carried as a BF16 hi + lo pair as on
  // the tensor-core path (zero rows past the end)
  for (int i = tid; i < S * 8; i += NT) {
    const int s = i / 8, c = i % 8;
    float v = 0.f;
    if (s < ns && c < 6) {
      const int64_t col = idx ? idx[s0 + s] : s0 + s;
      const float x = (float)(((double)zin.c[c][col] - nrm.mu_in[c]) * nrm.inv_sd_in[c]);
      const float hi = bf16r(x);
      v = __fadd_rn(hi, bf16r(__fsub_rn(x, hi)));
    }
    sm.h0[s][c] = v;
  }
  __syncthreads();

  // ---- forward: layers 0..3 (thread = output feature)
  for (int l = 0; l < 4; ++l) {
    const int fi = (l == 0) ? 6 : 128;
    const float *W = wt + woff(l);  // [in][out]
    float acc[S];
    const float bj = wt[boff(l) + tid];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = bj;
    if (l == 0) {
      for (int k = 0; k < 6; ++k) {
        const float w = W[k * 128 + tid];
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = fmaf(w, sm.h0[s][k], acc[s]);
      }
    } else {
      const float(*H)[128] = sm.h[l - 1];
      for (int k = 0; k < 128; k += 4) {
        const float w0 = W[(k + 0) * 128 + tid], w1 = W[(k + 1) * 128 + tid];
        const float w2 = W[(k + 2) * 128 + tid], w3 = W[(k + 3) * 128 + tid];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const float4 hv = *reinterpret_cast<const float4 *>(&H[s][k]);
          acc[s] = fmaf(w0, hv.x, fmaf(w1, hv.y, fmaf(w2, hv.z, fmaf(w3, hv.w, acc[s]))));
        }
      }
    }
    (void)fi;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      float y, dy;
      gelu_fwd(acc[s], y, dy);
      sm.h[l][s][tid] = bf16r(y);
      sm.dg[l][s][tid] = dy;
    }
    __syncthreads();
  }
  // ---- layer 4 (6 outputs): thread t < 6*S computes output (s, o)
  double lsum = 0.0;
  if (tid < 6 * S) {
    const int o = tid / S, s = tid % S;
    const float *W = wn + woff(4) + o * 128;  // [out][in]
    float acc = wn[boff(4) + o];
    for (int k = 0; k < 128; k += 4) {
      const float4 hv = *reinterpret_cast<const float4 *>(&sm.h[3][s][k]);
      acc = fmaf(W[k], hv.x, fmaf(W[k + 1], hv.y, fmaf(W[k + 2], hv.z, fmaf(W[k + 3], hv.w, acc))));
    }
    sm.a4[s][o] = acc;
    float d = 0.f;
    if (s < ns) {
      const int64_t col = idx ? idx[s0 + s] : s0 + s;
      const float tgt = (float)(((double)zout.c[o][col] - nrm.mu_out[o]) / nrm.sd_out[o]);
      const float diff = acc - tgt;
      lsum = (double)diff * (double)diff;
      d = (float)(2.0 * (double)diff * inv_count6);
    }
    sm.d4[s][o] = d;
  }
  lsum = warp_sum(lsum);
  if ((tid & 31) == 0) sm.loss[tid >> 5] = lsum;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += sm.loss[w];
    loss_part[blockIdx.x] = t;
  }
  if (MODE == MODE_LOSS) return;

  float *P = part + (int64_t)blockIdx.x * MLP_PSTRIDE;

  // ---- layer 4 backward: dW4, db4; dh_4 = W4^T d4
  if (MODE == MODE_TRAIN) {
    // dW4[o][k] = sum_s d4[s][o] h4[s][k]; thread = k
    for (int o = 0; o < 6; ++o) {
      float a = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s) a = fmaf(sm.d4[s][o], sm.h[3][s][tid], a);
      P[woff(4) + o * 128 + tid] = a;
    }
    if (tid < 6) {
      float a = 0.f;
      for (int s = 0; s < S; ++s) a += sm.d4[s][tid];
      P[boff(4) + tid] = a;
    }
  }
  {
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int o = 0; o < 6; ++o) {
      const float w = wn[woff(4) + o * 128 + tid];
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] = fmaf(w, sm.d4[s][o], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) sm.d[s][tid] = acc[s] * sm.dg[3][s][tid];  // d(a_3)
  }
  __syncthreads();

  // ---- layers 3..1: dW_l, db_l, then d(a_{l-1}) = (W_l^T d) * GELU'(a_{l-1})
  for (int l = 3; l >= 1; --l) {
    if (MODE == MODE_TRAIN) {
      float dj[S];
#pragma unroll
      for (int s = 0; s < S; ++s) dj[s] = sm.d[s][tid];
      const float(*H)[128] = sm.h[l - 1];
      float *Pw = P + woff(l) + tid * 128;
      for (int k = 0; k < 128; k += 4) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const float4 hv = *reinterpret_cast<const float4 *>(&H[s][k]);
          a.x = fmaf(dj[s], hv.x, a.x);
          a.y = fmaf(dj[s], hv.y, a.y);
          a.z = fmaf(dj[s], hv.z, a.z);
          a.w = fmaf(dj[s], hv.w, a.w);
        }
        *reinterpret_cast<float4 *>(Pw + k) = a;
      }
      float bsum = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s) bsum += dj[s];
      P[boff(l) + tid] = bsum;
    }
    // dh_l[s][k] = sum_j W_l[j][k] d[s][j]; thread = k
    const float *W = wn + woff(l);  // [out j][in k]
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int j = 0; j < 128; j += 4) {
      const float w0 = W[(j + 0) * 128 + tid], w1 = W[(j + 1) * 128 + tid];
      const float w2 = W[(j + 2) * 128 + tid], w3 = W[(j + 3) * 128 + tid];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const float4 dv = *reinterpret_cast<const float4 *>(&sm.d[s][j]);
        acc[s] = fmaf(w0, dv.x, fmaf(w1, dv.y, fmaf(w2, dv.z, fmaf(w3, dv.w, acc[s]))));
      }
    }
    __syncthreads();  // everyone done reading sm.d
#pragma unroll
    for (int s = 0; s < S; ++s) sm.d[s][tid] = acc[s] * sm.dg[l - 1][s][tid];
    __syncthreads();
  }

  // ---- layer 0: dW0, db0; input gradient for the VJP
  if (MODE == MODE_TRAIN) {
    float dj[S];
#pragma unroll
    for (int s = 0; s < S; ++s) dj[s] = sm.d[s][tid];
    for (int k = 0; k < 6; ++k) {
      float a = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s) a = fmaf(dj[s], sm.h0[s][k], a);
      P[woff(0) + tid * 6 + k] = a;
    }
    float bsum = 0.f;
#pragma unroll
    for (int s = 0; s < S; ++s) bsum += dj[s];
    P[boff(0) + tid] = bsum;
  }
}

__global__ void __launch_bounds__(256)
reduce_adam_kernel(const float *__restrict__ part, int nblocks, const double *__restrict__ loss_part,
                   double inv_count6, float *__restrict__ params, float *__restrict__ m,
                   float *__restrict__ v, float lr, float b1, float b2, float omb1, float omb2,
                   float eps, float c1, float c2, float *loss_out, float *grad_out, int apply) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && loss_out) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += loss_part[b];
    *loss_out = (float)(t * inv_count6);
  }
  if (i >= MLP_NPARAM) return;
  float g = 0.f;
  for (int b = 0; b < nblocks; ++b) g += part[(int64_t)b * MLP_PSTRIDE + i];
  if (grad_out) grad_out[i] = g;
  if (!apply) return;
  // omb1 = 1 - beta1 and omb2 = 1 - beta2 come from the host in FP64: formed
  // in FP32 from the rounded beta2 = 0.999f, 1 - beta2 would be off by 1.3e-5
  const float mi = fmaf(b1, m[i], omb1 * g);
  const float vi = fmaf(b2, v[i], omb2 * g * g);
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / c1, vh = vi / c2;
  params[i] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void loss_finalize_kernel(const double *__restrict__ lp, int nblocks, double inv,
                                     double *out) {
  __shared__ double red[8];
  double t = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) t += lp[b];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *out = s * inv;
  }
}

template <int MODE>
cudaError_t launch_grad_mode(Soa<float> zin, Soa<float> zout, const int64_t *idx, int64_t count,
                             const float *wt, const float *wn, const MlpNorm &nrm, float *part,
                             double *loss_part, cudaStream_t st, int64_t scale_count = 0) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel<MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(Smem));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (count <= 0) return cudaSuccess;
  const int64_t nb = (count + S - 1) / S;
  const double inv = 1.0 / (6.0 * (double)(scale_count > 0 ? scale_count : count));
  mlp_grad_kernel<MODE><<<(unsigned)nb, NT, sizeof(Smem), st>>>(zin, zout, idx, count, wt, wn,
                                                                nrm, part, loss_part, inv);
  return cudaGetLastError();
}

Soa<float> cols6(const float *base, int64_t ld) {
  Soa<float> r;
  for (int c = 0; c < 6; ++c) r.c[c] = const_cast<float *>(base) + c * ld;
  return r;
}

}  // namespace

int mlp_grad_blocks(int64_t count) { return (int)((count + S - 1) / S); }

cudaError_t launch_mlp_grad(const float *in, const float *out, int64_t ld, const int64_t *idx,
                            int64_t batch, const float *wt, const float *wn, const MlpNorm &nrm,
                            float *partials, double *loss_partials, int *nblocks_out,
                            cudaStream_t st, int64_t scale_count) {
  *nblocks_out = mlp_grad_blocks(batch);
  return launch_grad_mode<MODE_TRAIN>(cols6(in, ld), cols6(out, ld), idx, batch, wt, wn, nrm,
                                      partials, loss_partials, st, scale_count);
}

__global__ void __launch_bounds__(256)
rows_accumulate_kernel(const float *__restrict__ rows, int nrows, const double *__restrict__ lr,
                       double *__restrict__ acc, double *__restrict__ acc_loss,
                       float *__restrict__ row_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    double t = *acc_loss;
    for (int b = 0; b < nrows; ++b) t += lr[b];
    *acc_loss = t;
  }
  if (i >= MLP_NPARAM) return;
  double g = acc[i];
  for (int b = 0; b < nrows; ++b) g += (double)rows[(int64_t)b * MLP_PSTRIDE + i];
  acc[i] = g;
  if (row_out) row_out[i] = (float)g;
}

cudaError_t launch_mlp_rows_accumulate(const float *rows, int nrows, const double *loss_rows,
                                       double *acc, double *acc_loss, float *row_out,
                                       cudaStream_t st) {
  rows_accumulate_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(rows, nrows, loss_rows, acc,
                                                                   acc_loss, row_out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_reduce_adam(const float *partials, int nblocks, const double *loss_partials,
                                   int64_t batch, float *params, float *m, float *v, double lr,
                                   double b1, double b2, double eps, int step, float *loss_out,
                                   float *grad_out, cudaStream_t st) {
  const double c1 = 1.0 - pow(b1, (double)step);
  const double c2 = 1.0 - pow(b2, (double)step);
  const int apply = step > 0;
  reduce_adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(
      partials, nblocks, loss_partials, 1.0 / (6.0 * (double)batch), params, m, v, (float)lr,
      (float)b1, (float)b2, (float)(1.0 - b1), (float)(1.0 - b2), (float)eps,
      (float)(apply ? c1 : 1.0), (float)(apply ? c2 : 1.0),
      loss_out, grad_out, apply);
  return cudaGetLastError();
}

cudaError_t launch_mlp_loss(const float *in, const float *out, int64_t ld, const int64_t *idx,
                            int64_t count, const float *wt, const float *wn, const MlpNorm &nrm,
                            double *loss_partials, int *nblocks_out, cudaStream_t st) {
  *nblocks_out = mlp_grad_blocks(count);
  return launch_grad_mode<MODE_LOSS>(cols6(in, ld), cols6(out, ld), idx, count, wt, wn, nrm,
                                     nullptr, loss_partials, st);
}

cudaError_t launch_loss_finalize(const double *loss_partials, int nblocks, int64_t count,
                                 double *loss_out, cudaStream_t st) {
  loss_finalize_kernel<<<1, 256, 0, st>>>(loss_partials, nblocks, 1.0 / (6.0 * (double)count),
                                          loss_out);
  return cudaGetLastError();
}

}  // namespace bl
