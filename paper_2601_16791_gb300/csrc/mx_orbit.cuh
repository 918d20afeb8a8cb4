// mx_orbit.cuh -- osculating two-body orbit of one body (arXiv 2601.16791,
// Sec. 3.5: the ejection criterion e >= 1 and the element conversion it runs
// on every body).  The relations are the standard two-body ones (Murray &
// Dermott 1999, Sec. 2.8): angular momentum h = x cross v; eccentricity
// vector (v cross h)/gm - x/r; semilatus rectum p = |h|^2/gm.
#pragma once
#include "mx_common.cuh"

namespace mx {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// |(v cross h)/gm - x/r|: the eccentricity.  The ejection test needs nothing
// else, so it skips the angles.
__device__ __forceinline__ double orbit_ecc(double gm, double x, double y, double z, double u,
                                            double v, double w) {
  const double r = sqrt(x * x + y * y + z * z);
  const double hx = y * w - z * v, hy = z * u - x * w, hz = x * v - y * u;
  const double ex = (v * hz - w * hy) / gm - x / r;
  const double ey = (w * hx - u * hz) / gm - y / r;
  const double ez = (u * hy - v * hx) / gm - z / r;
  return sqrt(ex * ex + ey * ey + ez * ez);
}

// The test of Sec. 3.5 on one body in DH coordinates: unbound (e >= 1)
// about gm with the heliocentric velocity v_b + P/m0.  Not inlined, so that
// the step's test and the catch-up of deferred planetesimals run the same
// instructions and take the same decision.
static __device__ __noinline__ bool dh_unbound(double gm, double inv_mu0, const double* P,
                                               double x, double y, double z, double vbx,
                                               double vby, double vbz) {
  const double u = vbx + P[0] * inv_mu0;
  const double v = vby + P[1] * inv_mu0;
  const double w = vbz + P[2] * inv_mu0;
  return orbit_ecc(gm, x, y, z, u, v, w) >= 1.0;
}

__device__ __forceinline__ double wrap_two_pi(double a) {
  a = fmod(a, kTwoPi);
  return (a < 0.0) ? a + kTwoPi : a;
}

// Elements q, e, i, varpi (longitude of pericentre), Omega (node), M (mean
// anomaly).  The true anomaly f comes from e cos f = p/r - 1 and
// e sin f = |h| (x.v)/(gm r), the argument of latitude u from the position
// along the node line and 90 degrees ahead of it in the orbit plane, and
// varpi = Omega + u - f.  M: eccentric anomaly E for e < 1 (M = E - e sin E,
// reduced to [0, 2 pi)), hyperbolic anomaly F for e > 1 (M = e sinh F - F),
// Barker's D + D^3/3 (D = tan(f/2)) for e = 1.  Degenerate cases: Omega = 0
// for an orbit in the reference plane, f = 0 for e = 0.
__device__ __forceinline__ void orbit_elements(double gm, double x, double y, double z, double u,
                                               double v, double w, double* el) {
  const double r = sqrt(x * x + y * y + z * z);
  const double hx = y * w - z * v, hy = z * u - x * w, hz = x * v - y * u;
  const double hxy = sqrt(hx * hx + hy * hy);
  const double h = sqrt(hx * hx + hy * hy + hz * hz);
  const double p = h * h / gm;
  const double ex = (v * hz - w * hy) / gm - x / r;
  const double ey = (w * hx - u * hz) / gm - y / r;
  const double ez = (u * hy - v * hx) / gm - z / r;
  const double e = sqrt(ex * ex + ey * ey + ez * ez);
  const double node = (hxy > 0.0) ? atan2(hx, -hy) : 0.0;
  double sn, cn;
  sincos(node, &sn, &cn);
  const double ci = (h > 0.0) ? hz / h : 1.0, si = (h > 0.0) ? hxy / h : 0.0;
  const double along = x * cn + y * sn;
  const double ahead = (y * cn - x * sn) * ci + z * si;
  const double ulat = atan2(ahead, along);
  const double rv = x * u + y * v + z * w;
  const double f = (e > 0.0) ? atan2(h * rv / (gm * r), p / r - 1.0) : 0.0;
  double sf, cf;
  sincos(f, &sf, &cf);
  double M;
  if (e < 1.0) {
    const double E = atan2(sqrt(1.0 - e * e) * sf, e + cf);
    M = wrap_two_pi(E - e * sin(E));
  } else if (e > 1.0) {
    const double F = asinh(sqrt(e * e - 1.0) * sf / (1.0 + e * cf));
    M = e * sinh(F) - F;
  } else {
    const double D = tan(0.5 * f);
    M = D + D * D * D / 3.0;
  }
  el[0] = p / (1.0 + e);
  el[1] = e;
  el[2] = atan2(hxy, hz);
  el[3] = wrap_two_pi(node + ulat - f);
  el[4] = wrap_two_pi(node);
  el[5] = M;
}

}  // namespace mx
