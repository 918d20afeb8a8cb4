// mx_orbit.cuh -- osculating two-body orbit of one body (arXiv 2601.16791,
// Sec. 3.5: the ejection criterion e >= 1 and the element conversion it runs
// on every body).  The relations are the standard two-body ones (Murray &
// Dermott 1999, Sec. 2.8): angular momentum h = x cross v; eccentricity
// vector (v cross h)/gm - x/r; semilatus rectum p = |h|^2/gm.
#pragma once
#include "mx_common.cuh"

namespace mx {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// The test of Sec. 3.5 on one body in DH coordinates: unbound (e >= 1)
// about gm with the heliocentric velocity v_b + P/m0.  Since
// e^2 = 1 + (v^2 - 2 gm/r) |h|^2 / gm^2, e >= 1 is v^2 >= 2 gm / r, i.e.
// (v^2)^2 r^2 >= (2 gm)^2, when h != 0; a radial orbit (h = 0) has e = 1.
// That form needs no division and no square root (the FP64 units issue
// those as long instruction sequences).  Not inlined, so that the step's
// test and the catch-up of deferred planetesimals run the same instructions
// and take the same decision.
static __device__ __noinline__ bool dh_unbound(double gm, double inv_mu0, const double* P,
                                               double x, double y, double z, double vbx,
                                               double vby, double vbz) {
  const double u = vbx + P[0] * inv_mu0;
  const double v = vby + P[1] * inv_mu0;
  const double w = vbz + P[2] * inv_mu0;
  const double v2 = u * u + v * v + w * w;
  const double r2 = x * x + y * y + z * z;
  const double hx = y * w - z * v, hy = z * u - x * w, hz = x * v - y * u;
  const double h2 = hx * hx + hy * hy + hz * hz;
  return (v2 * v2) * r2 >= 4.0 * gm * gm || h2 == 0.0;
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
// Sines and cosines come from the vectors already at hand (cos Omega =
// -h_y/|h_xy|, cos f = (e cos f)/e, sin E = sqrt(1 - e^2) sin f/(1 + e cos f),
// tan(f/2) = sin f/(1 + cos f)), so the transcendental calls are one atan2
// for each of i, Omega, u, f and E, and asinh for e > 1.
__device__ __forceinline__ void orbit_elements(double gm, double x, double y, double z, double u,
                                               double v, double w, double* el) {
  const double r = sqrt(x * x + y * y + z * z);
  const double hx = y * w - z * v, hy = z * u - x * w, hz = x * v - y * u;
  const double hxy2 = hx * hx + hy * hy;
  const double hxy = sqrt(hxy2);
  const double h2 = hxy2 + hz * hz;
  const double h = sqrt(h2);
  const double p = h2 / gm;
  const double ex = (v * hz - w * hy) / gm - x / r;
  const double ey = (w * hx - u * hz) / gm - y / r;
  const double ez = (u * hy - v * hx) / gm - z / r;
  const double e = sqrt(ex * ex + ey * ey + ez * ez);
  double node = 0.0, cn = 1.0, sn = 0.0;
  if (hxy > 0.0) {
    node = atan2(hx, -hy);
    cn = -hy / hxy;
    sn = hx / hxy;
  }
  const double ci = (h > 0.0) ? hz / h : 1.0, si = (h > 0.0) ? hxy / h : 0.0;
  const double along = x * cn + y * sn;
  const double ahead = (y * cn - x * sn) * ci + z * si;
  const double ulat = atan2(ahead, along);
  const double rv = x * u + y * v + z * w;
  const double ecf = p / r - 1.0, esf = h * rv / (gm * r);
  double f = 0.0, cf = 1.0, sf = 0.0;
  if (e > 0.0) {
    f = atan2(esf, ecf);
    cf = ecf / e;
    sf = esf / e;
  }
  double M;
  if (e < 1.0) {
    const double rt = sqrt(1.0 - e * e);
    const double E = atan2(rt * sf, e + cf);
    M = wrap_two_pi(E - e * (rt * sf / (1.0 + e * cf)));
  } else if (e > 1.0) {
    const double shF = sqrt(e * e - 1.0) * sf / (1.0 + e * cf);
    M = e * shF - asinh(shF);
  } else {
    const double D = sf / (1.0 + cf);
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
