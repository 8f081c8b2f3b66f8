// Plasma stage, plain method: classical RK4 in s through a prescribed linear
// wake (the per-particle stage map that the surrogate of Sec. 3/4 learns).
//
// Equations (u = p/(m_e c), gamma = sqrt(1+|u|^2), phi = k_p zeta,
// g = e E0/(m_e c^2), K0 = g k_p/2):
//   x' = u_x/u_z,  u_x' = -(gamma/u_z) K0 sin(phi) x   (same for y)
//   zeta' = 1 - gamma/u_z,  u_z' = (gamma/u_z) g cos(phi)
// Writing gamma/u_z = 1 + w with w = (1+u_perp^2)/(u_z (gamma+u_z)) removes
// the cancellation in zeta' = -w.
//
// FP32 deviation form. zeta and u_z are carried as deviations from the FP64
// reference trajectory, whose RK4 stage values Y_r,i (i = 1..4 of every step)
// the host precomputes with the same RK4. Because RK4 is linear in its stage
// derivatives, integrating dY = Y - Y_r with stage derivatives
// f(Y_r,i + dY_i) - f(Y_r,i) reproduces RK4 of the full state exactly in
// exact arithmetic, while every FP32 quantity stays small:
//   d(dzeta)/ds = -(w - w_r)
//   d(du_z)/ds  = g [(cos phi - cos phi_r)(1 + w_r) + (w - w_r) cos phi]
// cos phi - cos phi_r is formed without cancellation from sin/cos of half
// the phase deviation once per step; inside a step the phase moves by
// ~1e-5 rad, so the stage values use a first-order update whose error
// (~1e-10) is far below FP32 resolution. With a = (1+u_perp^2)/u_z^2 ~ 1e-7,
// w = a/2 (1 - a/4) to O(a^3).
//
// FP64 instantiation: same deviation form with exact trigonometry and exact
// w at every stage (used for the small FP64 configuration).
#include "common.cuh"
#include "internal.h"
#include "push_f32.cuh"

namespace bl {

namespace {

struct alignas(32) D4 { double x, y, z, w; };

// LIST: push only the particles list[0 .. min(*count, n)) (the surrogate's
// fallback particles); otherwise every particle p < n.
template <bool LIST>
__global__ void __launch_bounds__(128)
pusher_f32(Soa<float> z, int64_t n, ConstsF c, const float4 *__restrict__ table,
           const int64_t *__restrict__ list, const unsigned long long *count) {
  const int64_t m = LIST ? min(n, (int64_t)*count) : n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    push::push_particle(z, LIST ? list[i] : i, c, table);
}

// ---------------------------------------------------------------- FP64 ----
struct StateD { double x, ux, y, uy, dz, du; };

__device__ StateD eval_d(const StateD &Y, double uz_r, double w_r, double phi_r, double kp,
                         double g, double K0) {
  const double uz = uz_r + Y.du;
  const double q = 1.0 + Y.ux * Y.ux + Y.uy * Y.uy;
  const double gam = sqrt(q + uz * uz);
  const double w = q / (uz * (gam + uz));
  const double dphi = kp * Y.dz;
  double sphi, cphi;
  sincos(phi_r + dphi, &sphi, &cphi);
  const double dcos = -2.0 * sin(phi_r + 0.5 * dphi) * sin(0.5 * dphi);
  const double dw = w - w_r;
  const double F = (1.0 + w) * K0 * sphi;
  StateD k;
  k.x = Y.ux / uz;
  k.ux = -F * Y.x;
  k.y = Y.uy / uz;
  k.uy = -F * Y.y;
  k.dz = -dw;
  k.du = g * (dcos * (1.0 + w_r) + dw * cphi);
  return k;
}

__device__ StateD axpy_d(const StateD &Y, double a, const StateD &k) {
  return {fma(a, k.x, Y.x), fma(a, k.ux, Y.ux), fma(a, k.y, Y.y),
          fma(a, k.uy, Y.uy), fma(a, k.dz, Y.dz), fma(a, k.du, Y.du)};
}

__global__ void __launch_bounds__(128)
pusher_f64(Soa<double> z, int64_t n, StageConsts c, const D4 *__restrict__ table) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    StateD Y;
    {
      Y.x = z.c[0][p];
      Y.y = z.c[2][p];
      Y.ux = z.c[1][p] * c.bg_in;
      Y.uy = z.c[3][p] * c.bg_in;
      const double dg = -z.c[5][p] * c.bg_in;
      const double up2 = Y.ux * Y.ux + Y.uy * Y.uy;
      const double gam = c.gamma_in + dg;
      const double uz = sqrt(gam * gam - 1.0 - up2);
      Y.du = (dg * (gam + c.gamma_in) - up2) / (uz + c.bg_in);
      Y.dz = -z.c[4][p];
    }
    const double h = c.h, h2 = 0.5 * c.h;
    for (int s = 0; s < c.nsteps; ++s) {
      const D4 e0 = table[4 * s + 0], e1 = table[4 * s + 1];
      const D4 e2 = table[4 * s + 2], e3 = table[4 * s + 3];
      StateD k1 = eval_d(Y, e0.x, e0.y, e0.z, c.kp, c.g, c.K0);
      StateD k2 = eval_d(axpy_d(Y, h2, k1), e1.x, e1.y, e1.z, c.kp, c.g, c.K0);
      StateD k3 = eval_d(axpy_d(Y, h2, k2), e2.x, e2.y, e2.z, c.kp, c.g, c.K0);
      StateD k4 = eval_d(axpy_d(Y, h, k3), e3.x, e3.y, e3.z, c.kp, c.g, c.K0);
      StateD acc;
      acc.x = k1.x + 2.0 * (k2.x + k3.x) + k4.x;
      acc.ux = k1.ux + 2.0 * (k2.ux + k3.ux) + k4.ux;
      acc.y = k1.y + 2.0 * (k2.y + k3.y) + k4.y;
      acc.uy = k1.uy + 2.0 * (k2.uy + k3.uy) + k4.uy;
      acc.dz = k1.dz + 2.0 * (k2.dz + k3.dz) + k4.dz;
      acc.du = k1.du + 2.0 * (k2.du + k3.du) + k4.du;
      Y = axpy_d(Y, h / 6.0, acc);
    }
    const double uz = c.uz_ref_out + Y.du;
    const double up2 = Y.ux * Y.ux + Y.uy * Y.uy;
    const double gam = sqrt(1.0 + up2 + uz * uz);
    const double dg = (up2 + Y.du * (uz + c.uz_ref_out)) / (gam + c.gamma_out);
    z.c[0][p] = Y.x;
    z.c[1][p] = Y.ux / c.bg_out;
    z.c[2][p] = Y.y;
    z.c[3][p] = Y.uy / c.bg_out;
    z.c[4][p] = -Y.dz;
    z.c[5][p] = -dg / c.bg_out;
  }
}

}  // namespace

ConstsF consts_f(const StageConsts &c) {
  ConstsF f;
  f.kp = (float)c.kp;
  f.g = (float)c.g;
  f.K0 = (float)c.K0;
  f.h = (float)c.h;
  f.h2 = (float)(0.5 * c.h);
  f.h6 = (float)(c.h / 6.0);
  f.bg_in = (float)c.bg_in;
  f.gamma_in = (float)c.gamma_in;
  f.bg_out = (float)c.bg_out;
  f.gamma_out = (float)c.gamma_out;
  f.uz_out = (float)c.uz_ref_out;
  f.nsteps = c.nsteps;
  return f;
}

template <>
cudaError_t launch_pusher<float>(Soa<float> z, int64_t n, const StageConsts &c,
                                 const float *table, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 127) / 128;
  pusher_f32<false><<<(unsigned)blocks, 128, 0, st>>>(
      z, n, consts_f(c), reinterpret_cast<const float4 *>(table), nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_pusher_list(Soa<float> z, const int64_t *list, const unsigned long long *count,
                               int64_t capacity, const StageConsts &c, const float *table,
                               int num_sms, cudaStream_t st) {
  if (capacity <= 0) return cudaSuccess;
  // one-warp blocks: the list is usually short, and a block this small fits
  // beside a resident surrogate CTA (which leaves ~7.9K registers of an SM),
  // so a fallback push can overlap another bunch chunk's network pass
  int64_t blocks = (capacity + 31) / 32;
  if (blocks > 16 * (int64_t)num_sms) blocks = 16 * (int64_t)num_sms;  // grid-stride over the list
  pusher_f32<true><<<(unsigned)blocks, 32, 0, st>>>(
      z, capacity, consts_f(c), reinterpret_cast<const float4 *>(table), list, count);
  return cudaGetLastError();
}

template <>
cudaError_t launch_pusher<double>(Soa<double> z, int64_t n, const StageConsts &c,
                                  const double *table, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 127) / 128;
  pusher_f64<<<(unsigned)blocks, 128, 0, st>>>(z, n, c, reinterpret_cast<const D4 *>(table));
  return cudaGetLastError();
}

}  // namespace bl
