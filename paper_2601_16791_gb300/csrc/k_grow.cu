// k_grow.cu -- growth tracks of the forming planets (arXiv 2601.16791,
// Sec. 3.3, Eqs. 13-16) and the gaps they open (Sec. 3.1, Eqs. 8-9).
//
// One block per system, one thread per big body, once per step before the
// step's first half kick: the mass at t = step x h (Eq. 13 up to tau_c, Eq. 15
// after), the changeover radius of that mass (rcrit_hill Hill radii from the
// osculating semimajor axis, as at set-up), the gap (half-width gap_c R_H and
// density factor exp(-(t - tau_c)/tau_g) once t > tau_c) and the radius
// (Eq. 14, k1 = 1, k2 = 1/4, with c_s at the body's cylindrical distance;
// after tau_c Eq. 16 from R_c, Eq. 14 at mass M_c on the current orbit).
#include "mx_common.cuh"
#include "mx_kernels.h"

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

__global__ void __launch_bounds__(kThreads) k_grow(Dev d, long long step) {
  const SysDev& S = d.sys[blockIdx.x];
  if (!S.grow_on) return;
  const double t = (double)step * S.h;
  const int N = d.N;
  // momentum of the state with the masses it has now (heliocentric velocities)
  __shared__ double red[3][kThreads];
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
  const double P0 = red[0][0], P1 = red[1][0], P2 = red[2][0];
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int b = S.boff + i, g = S.off + i;
    const Growth G = d.grow[b];
    if (!G.grows || removed(d, g)) continue;
    const double mu = S.G * growth_mass(G, t);
    const double x = d.xv[g], y = d.xv[(size_t)N + g], z = d.xv[2 * (size_t)N + g];
    const double u = d.xv[3 * (size_t)N + g] + P0 * S.inv_mu0;
    const double v = d.xv[4 * (size_t)N + g] + P1 * S.inv_mu0;
    const double w = d.xv[5 * (size_t)N + g] + P2 * S.inv_mu0;
    const double r = sqrt(x * x + y * y + z * z);
    const double v2 = u * u + v * v + w * w;
    const double a = semimajor_or_r(S.mu0 + mu, r, v2);
    const double rh = a * cbrt(mu / (3.0 * S.mu0));
    d.bmu[b] = mu;
    d.brc[b] = S.rcrit_hill * rh;
    const bool runaway = t > G.tc;
    d.gap_w[b] = runaway ? S.gap_c * rh : 0.0;
    d.gap_f[b] = runaway ? exp(-(t - G.tc) / G.tg) : 1.0;
    const double R = sqrt(x * x + y * y);
    const double cs = S.hr1 * pow(R, S.flare) * sqrt(S.mu0 / R);
    double rad;
    if (!runaway) {
      rad = inflated_radius(mu, cs, rh);
    } else {
      const double muc = S.G * G.mc;
      const double ac = semimajor_or_r(S.mu0 + muc, r, v2);
      rad = inflated_radius(muc, cs, ac * cbrt(muc / (3.0 * S.mu0))) -
            G.dr * (1.0 - exp(-(t - G.tc) / G.tg));
    }
    d.brad[b] = rad;
  }
}

void launch_grow(const Dev& d, long long step, cudaStream_t st) {
  k_grow<<<d.nsys, kThreads, 0, st>>>(d, step);
}

}  // namespace mx
