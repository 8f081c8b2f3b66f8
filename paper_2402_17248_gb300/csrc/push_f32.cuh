// FP32 RK4 push of one particle through a prescribed-wake plasma stage (the
// plain method of a stage, Sec. 3/4): the arithmetic of pusher_f32 in
// pusher.cu, shared with the surrogate kernel, whose fallback warp pushes the
// particles outside the network's training domain with exactly the same
// operations (so both paths give bit-identical particles). The deviation
// form and its derivation are described in pusher.cu.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace bl {
namespace push {

BL_DEV float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

struct StateF { float x, ux, y, uy, dz, du; };

// Right-hand side in deviation form. w = gamma/u_z - 1 = sqrt(1 + a) - 1 with
// a = (1 + u_perp^2)/u_z^2 is taken to second order, a/2 - a^2/8; the dropped
// a^3/16 is below FP32 rounding of w while a < 2^-10.5 (u_z > 38 sqrt(1 +
// u_perp^2)), which the host enforces as gamma_ref >= 400 at the stage entry.
BL_DEV StateF eval_f(const StateF &Y, float uz_r, float w_r, float sphi, float cphi, float dcos,
                     const ConstsF &c) {
  const float uz = uz_r + Y.du;
  const float q = fmaf(Y.uy, Y.uy, fmaf(Y.ux, Y.ux, 1.0f));
  const float r = rcp_approx(uz);
  const float a = q * r * r;
  const float w = 0.5f * a * fmaf(-0.25f, a, 1.0f);
  const float F = (1.0f + w) * c.K0 * sphi;
  const float dw = w - w_r;
  StateF k;
  k.x = Y.ux * r;
  k.ux = -F * Y.x;
  k.y = Y.uy * r;
  k.uy = -F * Y.y;
  k.dz = -dw;
  k.du = c.g * fmaf(dcos, 1.0f + w_r, dw * cphi);
  return k;
}

BL_DEV StateF axpy(const StateF &Y, float a, const StateF &k) {
  return {fmaf(a, k.x, Y.x), fmaf(a, k.ux, Y.ux), fmaf(a, k.y, Y.y),
          fmaf(a, k.uy, Y.uy), fmaf(a, k.dz, Y.dz), fmaf(a, k.du, Y.du)};
}

// Particle p of z through the stage: relative -> deviation coordinates,
// c.nsteps RK4 steps with the reference's stage values from `table`
// (4 float4 per step: uz_r, w_r, sin/cos of the reference phase or its
// stage increments), then back to relative coordinates at the exit.
BL_DEV void push_particle(Soa<float> z, int64_t p, const ConstsF &c,
                          const float4 *__restrict__ table) {
  StateF Y;
  {
    const float x = z.c[0][p], px = z.c[1][p], y = z.c[2][p], py = z.c[3][p];
    const float t = z.c[4][p], pt = z.c[5][p];
    Y.x = x;
    Y.y = y;
    Y.ux = px * c.bg_in;
    Y.uy = py * c.bg_in;
    const float dg = -pt * c.bg_in;  // gamma - gamma_ref
    const float up2 = fmaf(Y.uy, Y.uy, Y.ux * Y.ux);
    const float gam = c.gamma_in + dg;
    const float uz = sqrtf(fmaf(gam, gam, -1.0f - up2));
    Y.du = fmaf(dg, gam + c.gamma_in, -up2) / (uz + c.bg_in);
    Y.dz = -t;
  }
  for (int s = 0; s < c.nsteps; ++s) {
    const float4 e0 = __ldg(table + 4 * s + 0);
    const float4 e1 = __ldg(table + 4 * s + 1);
    const float4 e2 = __ldg(table + 4 * s + 2);
    const float4 e3 = __ldg(table + 4 * s + 3);
    const float sr = e0.z, cr = e0.w;
    float s2, c2;
    sincosf(0.5f * c.kp * Y.dz, &s2, &c2);
    const float sD = 2.0f * s2 * c2;
    const float cm1 = -2.0f * s2 * s2;
    const float sphi = fmaf(sr, cm1, fmaf(cr, sD, sr));
    const float dcos = fmaf(cr, cm1, -sr * sD);
    const float cphi = cr + dcos;
    const float dsr = sphi - sr;
    // stage 1
    StateF k1 = eval_f(Y, e0.x, e0.y, sphi, cphi, dcos, c);
    // stage 2
    StateF Y2 = axpy(Y, c.h2, k1);
    float dz = Y2.dz - Y.dz;
    float eps = fmaf(c.kp, dz, e1.z);
    StateF k2 = eval_f(Y2, e1.x, e1.y, fmaf(cphi, eps, sphi), fmaf(-sphi, eps, cphi),
                       fmaf(-dsr, e1.z, fmaf(-sphi * c.kp, dz, dcos)), c);
    // stage 3
    StateF Y3 = axpy(Y, c.h2, k2);
    dz = Y3.dz - Y.dz;
    eps = fmaf(c.kp, dz, e2.z);
    StateF k3 = eval_f(Y3, e2.x, e2.y, fmaf(cphi, eps, sphi), fmaf(-sphi, eps, cphi),
                       fmaf(-dsr, e2.z, fmaf(-sphi * c.kp, dz, dcos)), c);
    // stage 4
    StateF Y4 = axpy(Y, c.h, k3);
    dz = Y4.dz - Y.dz;
    eps = fmaf(c.kp, dz, e3.z);
    StateF k4 = eval_f(Y4, e3.x, e3.y, fmaf(cphi, eps, sphi), fmaf(-sphi, eps, cphi),
                       fmaf(-dsr, e3.z, fmaf(-sphi * c.kp, dz, dcos)), c);
    StateF acc;
    acc.x = k1.x + 2.0f * (k2.x + k3.x) + k4.x;
    acc.ux = k1.ux + 2.0f * (k2.ux + k3.ux) + k4.ux;
    acc.y = k1.y + 2.0f * (k2.y + k3.y) + k4.y;
    acc.uy = k1.uy + 2.0f * (k2.uy + k3.uy) + k4.uy;
    acc.dz = k1.dz + 2.0f * (k2.dz + k3.dz) + k4.dz;
    acc.du = k1.du + 2.0f * (k2.du + k3.du) + k4.du;
    Y = axpy(Y, c.h6, acc);
  }
  {
    const float uz = c.uz_out + Y.du;
    const float up2 = fmaf(Y.uy, Y.uy, Y.ux * Y.ux);
    const float gam = sqrtf(fmaf(uz, uz, 1.0f + up2));
    const float dg = fmaf(Y.du, uz + c.uz_out, up2) / (gam + c.gamma_out);
    const float ib = 1.0f / c.bg_out;
    z.c[0][p] = Y.x;
    z.c[1][p] = Y.ux * ib;
    z.c[2][p] = Y.y;
    z.c[3][p] = Y.uy * ib;
    z.c[4][p] = -Y.dz;
    z.c[5][p] = -dg * ib;
  }
}

}  // namespace push
}  // namespace bl
