// mx_growth.cuh -- growth tracks of the forming planets (arXiv 2601.16791,
// Sec. 3.3, Eqs. 13-16) and the gaps they open (Sec. 3.1, Eqs. 8-9).
//
// The mass follows Eq. 13 up to tau_c and Eq. 15 after it, at t = (global
// step index) x h at the start of each step, and is held for the step; the
// changeover radius follows the mass (rcrit_hill Hill radii from the
// osculating semimajor axis, as at set-up); once t > tau_c the body opens a
// gap of half-width gap_c R_H with density factor exp(-(t - tau_c)/tau_g).
// The radius (Eq. 14, k1 = 1, k2 = 1/4, c_s at the body's cylindrical
// distance; after tau_c Eq. 16 from R_c, Eq. 14 at mass M_c on the current
// orbit) does not enter the step and is computed on demand.
#pragma once
#include "mx_common.cuh"

namespace mx {

constexpr double kEulerE = 2.718281828459045235360287;

__device__ __forceinline__ double growth_mass(const Growth& g, double t) {
  if (t <= g.tc) return g.m0 + (kEulerE / (kEulerE - 1.0)) * (g.mc - g.m0) * (1.0 - exp(-t / g.tc));
  return g.mc + (g.mf - g.mc) * (1.0 - exp(-(t - g.tc) / g.tg));
}

// Eq. 14: R_p = G M / (c_s^2 / k1 + G M / (k2 R_H)).
__device__ __forceinline__ double inflated_radius(double gm, double cs, double rh) {
  return gm / (cs * cs / 1.0 + gm / (0.25 * rh));
}

// Osculating semimajor axis about gm (vis-viva), or r for an unbound orbit
// (as the set-up's changeover radius).
__device__ __forceinline__ double semimajor_or_r(double gm, double r, double v2) {
  const double a = 1.0 / (2.0 / r - v2 / gm);
  return (a > 0.0) ? a : r;
}

// Momentum sum mu_i v_i of system S's big bodies with the masses they have
// now, reduced by all threads of the block in a fixed tree.
__device__ __forceinline__ void big_momentum(const Dev& d, const SysDev& S,
                                             double (*red)[kThreads], double* P) {
  const int N = d.N;
  double p[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double m = d.bmu[S.boff + i];
    p[0] = fma(m, d.xv[3 * (size_t)N + g], p[0]);
    p[1] = fma(m, d.xv[4 * (size_t)N + g], p[1]);
    p[2] = fma(m, d.xv[5 * (size_t)N + g], p[2]);
  }
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = p[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  for (int c = 0; c < 3; ++c) P[c] = red[c][0];
  __syncthreads();
}

// Heliocentric r, v^2 of big body i of S with momentum P.
__device__ __forceinline__ void big_rv2(const Dev& d, const SysDev& S, int i, const double* P,
                                        double* r, double* v2, double* R) {
  const int N = d.N, g = S.off + i;
  const double x = d.xv[g], y = d.xv[(size_t)N + g], z = d.xv[2 * (size_t)N + g];
  const double u = d.xv[3 * (size_t)N + g] + P[0] * S.inv_mu0;
  const double v = d.xv[4 * (size_t)N + g] + P[1] * S.inv_mu0;
  const double w = d.xv[5 * (size_t)N + g] + P[2] * S.inv_mu0;
  *r = sqrt(x * x + y * y + z * z);
  *v2 = u * u + v * v + w * w;
  *R = sqrt(x * x + y * y);
}

// The growth update at the start of a step at time t: mass, changeover radius
// and gap of every growing big body of S.  All threads of the block call it.
__device__ __forceinline__ void grow_update(const Dev& d, const SysDev& S, double t,
                                            double (*red)[kThreads]) {
  double P[3];
  big_momentum(d, S, red, P);
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int b = S.boff + i;
    const Growth G = d.grow[b];
    if (!G.grows || removed(d, S.off + i)) continue;
    const double mu = S.G * growth_mass(G, t);
    double r, v2, R;
    big_rv2(d, S, i, P, &r, &v2, &R);
    const double rh = semimajor_or_r(S.mu0 + mu, r, v2) * cbrt(mu / (3.0 * S.mu0));
    d.bmu[b] = mu;
    set_rcrit(d, b, S.rcrit_hill * rh);
    const bool runaway = t > G.tc;
    d.gap_w[b] = runaway ? S.gap_c * rh : 0.0;
    d.gap_f[b] = runaway ? exp(-(t - G.tc) / G.tg) : 1.0;
  }
  __syncthreads();
}

}  // namespace mx
