// k_drift.cu -- jump and Kepler drift of every body (arXiv 2601.16791, Sec. 2:
// the Keplerian part of the hybrid step, which Mercury-Arxes hands to WHFast;
// here solved in universal variables).
//
// One thread per body.  The Kepler equation in the universal anomaly s,
//   F(s) = r0 s + eta G2(s) + zeta G3(s) - h = 0,   G_k = s^k c_k(beta s^2),
// with r0 = |x|, eta = x.v, beta = 2 mu/r0 - v^2, zeta = mu - beta r0, is
// solved by Halley's method from a second-order starting guess.  Once a
// Halley correction is below 1e-7 of s, the next error is below the FP64
// resolution (cubic convergence), so the stepped s is final; the G functions
// are carried to it by a second-order Taylor step (dG_k/ds = G_{k-1}) instead
// of a fresh series evaluation.  The state then moves with the Gauss f and g
// functions.
#include "mx_common.cuh"
#include "mx_kernels.h"

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

// c0..c3 for any z: quarter the argument into the series range, then apply
// c0(4z) = 2c0^2 - 1, c1(4z) = c0 c1, c2(4z) = c1^2/2, c3(4z) = (c2 + c0 c3)/4.
__device__ __noinline__ void stumpff_reduced(double z, double& c0, double& c1, double& c2,
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

// G0..G3 at s for beta.
__device__ __forceinline__ void gfuns(double s, double beta, double* G) {
  const double s2 = s * s;
  const double z = beta * s2;
  double c2, c3;
  if (fabs(z) <= 0.3) {
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
  if (h == 0.0) return true;
  const double r02 = fma(x, x, fma(y, y, z * z));
  const double ir0 = rsqrt_d(r02);
  const double r0 = r02 * ir0;
  const double v2 = fma(u, u, fma(v, v, w * w));
  const double eta = fma(x, u, fma(y, v, z * w));
  const double beta = fma(2.0 * mu, ir0, -v2);
  const double zeta = fma(-beta, r0, mu);
  // second-order guess s = (h/r0)(1 - eta h / (2 r0^2))
  double s = h * ir0 * fma(-0.5 * eta * h, ir0 * ir0, 1.0);
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
    if (fabs(ds) <= 1e-7 * fabs(s)) {
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

// Jump by (jump_frac h) P/m0, save the pre-drift state, drift by the system's h.
__global__ void __launch_bounds__(kThreads) k_jump_drift(Dev d, double jump_frac) {
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *d.pair_count = 0;
    *d.work_count = 0;
  }
  if (threadIdx.x >= t.count) return;
  const int N = d.N;
  const int j = t.start + threadIdx.x;
  double dj[3];
  jump_vec(d.P + 3 * t.sys, S, jump_frac, dj);
  double x = d.xv[j] + dj[0];
  double y = d.xv[(size_t)N + j] + dj[1];
  double z = d.xv[2 * (size_t)N + j] + dj[2];
  double u = d.xv[3 * (size_t)N + j];
  double v = d.xv[4 * (size_t)N + j];
  double w = d.xv[5 * (size_t)N + j];
  d.xv0[j] = x;
  d.xv0[(size_t)N + j] = y;
  d.xv0[2 * (size_t)N + j] = z;
  d.xv0[3 * (size_t)N + j] = u;
  d.xv0[4 * (size_t)N + j] = v;
  d.xv0[5 * (size_t)N + j] = w;
  if (!kepler_drift(S.mu0, S.h, d.kepler_max_iter, x, y, z, u, v, w))
    atomicOr(d.status, ST_KEPLER);
  d.xv[j] = x;
  d.xv[(size_t)N + j] = y;
  d.xv[2 * (size_t)N + j] = z;
  d.xv[3 * (size_t)N + j] = u;
  d.xv[4 * (size_t)N + j] = v;
  d.xv[5 * (size_t)N + j] = w;
  d.flags[j] = 0;
}

// Drift n bodies of a caller buffer (6 x n) by h about mu.
__global__ void __launch_bounds__(kThreads) k_drift_buf(double* xv, int n, double mu, double h,
                                                        int maxit, unsigned* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double x = xv[j], y = xv[(size_t)n + j], z = xv[2 * (size_t)n + j];
  double u = xv[3 * (size_t)n + j], v = xv[4 * (size_t)n + j], w = xv[5 * (size_t)n + j];
  if (!kepler_drift(mu, h, maxit, x, y, z, u, v, w)) atomicOr(status, ST_KEPLER);
  xv[j] = x;
  xv[(size_t)n + j] = y;
  xv[2 * (size_t)n + j] = z;
  xv[3 * (size_t)n + j] = u;
  xv[4 * (size_t)n + j] = v;
  xv[5 * (size_t)n + j] = w;
}

void launch_jump_drift(const Dev& d, double jump_frac, cudaStream_t st) {
  k_jump_drift<<<d.ntiles, d.tile, 0, st>>>(d, jump_frac);
}

void launch_drift_buf(double* xv, int n, double mu, double h, int maxit, unsigned* status,
                      cudaStream_t st) {
  if (n <= 0) return;
  k_drift_buf<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(xv, n, mu, h, maxit, status);
}

}  // namespace mx
