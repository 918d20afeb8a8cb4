// mx_encounter.cuh -- the per-pair close-encounter test (arXiv 2601.16791,
// Sec. 2.1.2, mce_snif listing: flagged when min(d0, d1, d2min) <= rc^2 with
// rc = max(rcrit_i, rcrit_j)), shared by the detection kernel and the
// catch-up of deferred planetesimals so that both take the same decision.
#pragma once
#include "mx_common.cuh"

namespace mx {

// Conservative FP32 screen: false only for pairs the FP64 test cannot flag.
// The cubic Hermite interpolant p of the squared separation satisfies
// p >= min(d0, d1) - (4/27)(|D0| + |D1|) on the step (D = endpoint slopes in
// units of the step); the FP32 evaluation gets a 10% + 1e-3 relative margin,
// far above its rounding.  a, b: x0 y0 z0 u0 v0 w0 x1 y1 z1 u1 v1 w1.
__device__ __forceinline__ bool encounter_screen(const float* a, const float* b, float rc2f,
                                                 float hf) {
  const float dx0 = a[0] - b[0], dy0 = a[1] - b[1], dz0 = a[2] - b[2];
  const float du0 = a[3] - b[3], dv0 = a[4] - b[4], dw0 = a[5] - b[5];
  const float dx1 = a[6] - b[6], dy1 = a[7] - b[7], dz1 = a[8] - b[8];
  const float du1 = a[9] - b[9], dv1 = a[10] - b[10], dw1 = a[11] - b[11];
  const float d0 = fmaf(dx0, dx0, fmaf(dy0, dy0, dz0 * dz0));
  const float d1 = fmaf(dx1, dx1, fmaf(dy1, dy1, dz1 * dz1));
  const float D0 = fabsf(2.0f * hf * fmaf(dx0, du0, fmaf(dy0, dv0, dz0 * dw0)));
  const float D1 = fabsf(2.0f * hf * fmaf(dx1, du1, fmaf(dy1, dv1, dz1 * dw1)));
  const float lb = fminf(d0, d1) - (4.0f / 27.0f) * (D0 + D1);
  return lb <= 1.1f * rc2f + 1e-3f * (d0 + d1 + D0 + D1);
}

// Exact FP64 encounter test between target a and big b (6 doubles each at
// the start, 0, and end, 1, of the step).
static __device__ __noinline__ bool encounter_fp64(const double* a0, const double* b0, const double* a1,
                                           const double* b1, double h, double rc2) {
  const double dx0 = a0[0] - b0[0], dy0 = a0[1] - b0[1], dz0 = a0[2] - b0[2];
  const double du0 = a0[3] - b0[3], dv0 = a0[4] - b0[4], dw0 = a0[5] - b0[5];
  const double dx1 = a1[0] - b1[0], dy1 = a1[1] - b1[1], dz1 = a1[2] - b1[2];
  const double du1 = a1[3] - b1[3], dv1 = a1[4] - b1[4], dw1 = a1[5] - b1[5];
  const double d0 = fma(dx0, dx0, fma(dy0, dy0, dz0 * dz0));
  const double d1 = fma(dx1, dx1, fma(dy1, dy1, dz1 * dz1));
  if (d0 <= rc2 || d1 <= rc2) return true;
  // slopes of the squared separation per unit of tau = t/h
  const double D0 = 2.0 * h * fma(dx0, du0, fma(dy0, dv0, dz0 * dw0));
  const double D1 = 2.0 * h * fma(dx1, du1, fma(dy1, dv1, dz1 * dw1));
  if (!(D0 < 0.0 && D1 > 0.0)) return false;
  // p(tau) = d0 + D0 tau + c2 tau^2 + c3 tau^3 with p(1) = d1, p'(1) = D1
  const double c2 = -3.0 * d0 - 2.0 * D0 + 3.0 * d1 - D1;
  const double c3 = 2.0 * d0 + D0 - 2.0 * d1 + D1;
  // p'(tau) = 3 c3 tau^2 + 2 c2 tau + D0 has exactly one root in (0, 1)
  const double A = 3.0 * c3, B = 2.0 * c2, C = D0;
  double tau;
  if (A == 0.0) {
    tau = -C / B;
  } else {
    const double disc = fmax(B * B - 4.0 * A * C, 0.0);
    const double q = -0.5 * (B + copysign(sqrt(disc), B));
    const double r1 = q / A;
    const double r2 = (q != 0.0) ? C / q : r1;
    tau = (r1 >= 0.0 && r1 <= 1.0) ? r1 : r2;
  }
  tau = fmin(fmax(tau, 0.0), 1.0);
  const double p = fma(tau, fma(tau, fma(tau, c3, c2), D0), d0);
  return fmax(p, 0.0) <= rc2;
}

}  // namespace mx
