// mx_kepler.cuh -- universal-variable Kepler drift (arXiv 2601.16791, Sec. 2:
// the Keplerian part of the hybrid step), shared by the drift kernels and the
// adjoint.  See k_drift.cu for the method.
#pragma once
#include "mx_common.cuh"

namespace mx {

// c2(z) = sum_k (-z)^k/(2k+2)!, c3(z) = sum_k (-z)^k/(2k+3)!, eight terms,
// accurate to FP64 for |z| <= 0.3.
__device__ __forceinline__ void stumpff_series(double z, double& c2, double& c3) {
  c2 = 1.0 / 20922789888000.0;      // 1/16!
  c3 = 1.0 / 355687428096000.0;     // 1/17!
  c2 = fma(-z, c2, 1.0 / 87178291200.0);
  c3 = fma(-z, c3, 1.0 / 1307674368000.0);
  c2 = fma(-z, c2, 1.0 / 479001600.0);
  c3 = fma(-z, c3, 1.0 / 6227020800.0);
  c2 = fma(-z, c2, 1.0 / 3628800.0);
  c3 = fma(-z, c3, 1.0 / 39916800.0);
  c2 = fma(-z, c2, 1.0 / 40320.0);
  c3 = fma(-z, c3, 1.0 / 362880.0);
  c2 = fma(-z, c2, 1.0 / 720.0);
  c3 = fma(-z, c3, 1.0 / 5040.0);
  c2 = fma(-z, c2, 1.0 / 24.0);
  c3 = fma(-z, c3, 1.0 / 120.0);
  c2 = fma(-z, c2, 0.5);
  c3 = fma(-z, c3, 1.0 / 6.0);
}

// The same series with six terms, for |z| <= 0.03 (a step of up to about
// 0.17 rad of mean motion): the first term left out, z^6/14!, is below 1e-20
// of c2 there.
__device__ __forceinline__ void stumpff_series6(double z, double& c2, double& c3) {
  c2 = 1.0 / 479001600.0;           // 1/12!
  c3 = 1.0 / 6227020800.0;          // 1/13!
  c2 = fma(-z, c2, 1.0 / 3628800.0);
  c3 = fma(-z, c3, 1.0 / 39916800.0);
  c2 = fma(-z, c2, 1.0 / 40320.0);
  c3 = fma(-z, c3, 1.0 / 362880.0);
  c2 = fma(-z, c2, 1.0 / 720.0);
  c3 = fma(-z, c3, 1.0 / 5040.0);
  c2 = fma(-z, c2, 1.0 / 24.0);
  c3 = fma(-z, c3, 1.0 / 120.0);
  c2 = fma(-z, c2, 0.5);
  c3 = fma(-z, c3, 1.0 / 6.0);
}

// c0..c3 for any z: quarter the argument into the series range, then apply
// c0(4z) = 2c0^2 - 1, c1(4z) = c0 c1, c2(4z) = c1^2/2, c3(4z) = (c2 + c0 c3)/4.
static __device__ __noinline__ void stumpff_reduced(double z, double& c0, double& c1, double& c2,
                                             double& c3) {
  int m = 0;
  while (fabs(z) > 0.3 && m < 60) {
    z *= 0.25;
    ++m;
  }
  stumpff_series(z, c2, c3);
  c1 = fma(-z, c3, 1.0);
  c0 = fma(-z, c2, 1.0);
  for (; m > 0; --m) {
    c3 = 0.25 * fma(c0, c3, c2);
    c2 = 0.5 * c1 * c1;
    c1 = c0 * c1;
    c0 = fma(2.0 * c0, c0, -1.0);
  }
}

// |a| <= c for a constant c > 0, on the bit patterns (integer order is value
// order for non-negative doubles; a NaN compares false, as in FP64), so the
// test leaves the FP64 pipe free.
__device__ __forceinline__ bool abs_le(double a, double c) {
  return (__double_as_longlong(a) & 0x7fffffffffffffffLL) <= __double_as_longlong(c);
}

// G0..G3 at s for beta.
__device__ __forceinline__ void gfuns(double s, double beta, double* G) {
  const double s2 = s * s;
  const double z = beta * s2;
  double c2, c3;
  if (abs_le(z, 0.03)) {
    stumpff_series6(z, c2, c3);
  } else if (abs_le(z, 0.3)) {
    stumpff_series(z, c2, c3);
  } else {
    double c0, c1;
    stumpff_reduced(z, c0, c1, c2, c3);
  }
  G[2] = s2 * c2;
  G[3] = s2 * s * c3;
  G[1] = fma(-beta, G[3], s);
  G[0] = fma(-beta, G[2], 1.0);
}

// Returns false when the iteration cap is reached.
__device__ __forceinline__ bool kepler_drift(double mu, double h, int maxit, double& x, double& y,
                                             double& z, double& u, double& v, double& w) {
  if ((__double_as_longlong(h) << 1) == 0) return true;   // h = +-0
  const double r02 = fma(x, x, fma(y, y, z * z));
  const double ir0 = rsqrt_d(r02);
  const double r0 = r02 * ir0;
  const double v2 = fma(u, u, fma(v, v, w * w));
  const double eta = fma(x, u, fma(y, v, z * w));
  const double beta = fma(2.0 * mu, ir0, -v2);
  const double zeta = fma(-beta, r0, mu);
  // Short steps (|beta| (h/r0)^2 <= 0.1, n h below about 0.3): third-order
  // guess from inverting h = r0 s + eta s^2/2 + zeta s^3/6, s = h/r0
  // - eta h^2/(2 r0^3) + h^3 (eta^2/(2 r0^5) - zeta/(6 r0^4)), error O((n h)^4).
  // Halley's error after a correction of relative size e is about
  // (zeta/(6 r0) - eta^2/(4 r0^2)) s^2 e^3 ~ ((n h)^2/6) e^3 in relative terms,
  // below 2e-17 for e <= 1e-5 on a short step, so a correction that small
  // ends the solve there (1e-7 otherwise).  Longer steps, where the series
  // says little, start from its second-order part.
  const double hi = h * ir0;
  const bool short_step = abs_le(beta * hi * hi, 0.1);
  const double t1 = short_step ? fma(0.5 * eta * eta, ir0, -zeta * (1.0 / 6.0)) : 0.0;
  const double stop = short_step ? 1e-5 : 1e-7;
  double s = hi * fma(h * ir0 * ir0, fma(hi, t1, -0.5 * eta), 1.0);
  double G[4];
  bool done = false;
  double ds = 0.0;
  for (int it = 0; it < maxit; ++it) {
    gfuns(s, beta, G);
    const double F = fma(r0, s, fma(eta, G[2], fma(zeta, G[3], -h)));
    const double Fp = fma(eta, G[1], fma(zeta, G[2], r0));
    const double Fpp = fma(eta, G[0], zeta * G[1]);
    ds = -F * Fp * rcp_d(fma(Fp, Fp, -0.5 * F * Fpp));
    s += ds;
    if (fabs(ds) <= stop * fabs(s)) {
      done = true;
      break;
    }
  }
  if (!done) return false;
  // carry G to the stepped s: G_k(s0 + ds) = G_k + ds G_{k-1} + ds^2/2 G_{k-2},
  // with G_{-1} = -beta G1 and G_{-2} = -beta G0.
  // (f and g need only G1 and G2.)
  const double hd = 0.5 * ds;
  const double g2 = fma(ds, fma(hd, G[0], G[1]), G[2]);
  const double g1 = fma(ds, fma(-hd * beta, G[1], G[0]), G[1]);
  const double r = fma(eta, g1, fma(zeta, g2, r0));
  const double ir = rcp_d(r);
  const double f = fma(-mu * g2, ir0, 1.0);
  const double g = fma(r0, g1, eta * g2);
  const double fd = -mu * g1 * ir * ir0;
  const double gd = fma(-mu * g2, ir, 1.0);
  const double xn = fma(f, x, g * u), yn = fma(f, y, g * v), zn = fma(f, z, g * w);
  const double un = fma(fd, x, gd * u), vn = fma(fd, y, gd * v), wn = fma(fd, z, gd * w);
  x = xn; y = yn; z = zn;
  u = un; v = vn; w = wn;
  return true;
}

}  // namespace mx
