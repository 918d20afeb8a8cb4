// k_drift.cu -- jump and Kepler drift of every body (arXiv 2601.16791, Sec. 2:
// the Keplerian part of the hybrid step, which Mercury-Arxes hands to WHFast;
// here solved in universal variables).
//
// One thread per body.  The Kepler equation in the universal anomaly s,
//   F(s) = r0 s + eta G2(s) + zeta G3(s) - h = 0,   G_k = s^k c_k(beta s^2),
// with r0 = |x|, eta = x.v, beta = 2 mu/r0 - v^2, zeta = mu - beta r0, is
// solved by Halley's method from a third-order starting guess.  Once a
// Halley correction is small enough (1e-5 of s on short steps, 1e-7 on long
// ones; mx_kepler.cuh), the next error is below the FP64 resolution (cubic
// convergence), so the stepped s is final; the G functions
// are carried to it by a second-order Taylor step (dG_k/ds = G_{k-1}) instead
// of a fresh series evaluation.  The state then moves with the Gauss f and g
// functions.
#include "mx_common.cuh"
#include "mx_kepler.cuh"
#include "mx_kernels.h"

namespace mx {

// Jump by (jump_frac h) P/m0, save the pre-drift state, drift by the system's h.
__global__ void __launch_bounds__(kThreads) k_jump_drift(Dev d, double jump_frac) {
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *d.pair_count = 0;
    *d.work_count = 0;
  }
  const int slot = d.defer ? *d.hstep : 0;
  const bool rec = d.defer && slot < d.hist_cap;
  if (rec && t.start == S.off && threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) d.h_P[(size_t)slot * 6 * d.nsys + 3 * t.sys + c] = d.P[3 * t.sys + c];
  if (threadIdx.x >= t.count) return;
  const int N = d.N;
  const int j = t.start + threadIdx.x;
  if (d.defer && d.lag[j]) return;   // waits for the window's catch-up
  const int jl = j - S.off;
  if (removed(d, j)) {   // removed: stays where it is
    d.flags[j] = 0;
    if (rec && jl < S.nbig) {   // a history that deferred planetesimals never match
      const size_t b = S.boff + jl, o0 = (size_t)slot * 6 * d.NB;
      for (int c = 0; c < 6; ++c) {
        const double q = d.xv[(size_t)c * N + j];
        d.h_b0[o0 + (size_t)c * d.NB + b] = q;
        d.h_b1[o0 + (size_t)c * d.NB + b] = q;
      }
      d.h_comp[(size_t)slot * d.NB + b] = -1;
    }
    return;
  }
  double dj[3];
  jump_vec(d.P + 3 * t.sys, S, jump_frac, dj);
  // a big body comes from the kick's output (d.bk): the kick of an interior
  // step leaves it there only
  const double* src = (jl < S.nbig) ? d.bk + S.boff + jl : d.xv + j;
  const size_t ld = (jl < S.nbig) ? (size_t)d.NB : (size_t)N;
  double x = src[0] + dj[0];
  double y = src[ld] + dj[1];
  double z = src[2 * ld] + dj[2];
  double u = src[3 * ld];
  double v = src[4 * ld];
  double w = src[5 * ld];
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
  if (rec && jl < S.nbig) {   // the big body's endpoints, for deferred planetesimals
    const size_t b = S.boff + jl, o0 = (size_t)slot * 6 * d.NB;
    const double e0[6] = {d.xv0[j], d.xv0[(size_t)N + j], d.xv0[2 * (size_t)N + j], d.xv0[3 * (size_t)N + j],
                          d.xv0[4 * (size_t)N + j], d.xv0[5 * (size_t)N + j]};
    const double e1[6] = {x, y, z, u, v, w};
    for (int c = 0; c < 6; ++c) {
      d.h_b0[o0 + (size_t)c * d.NB + b] = e0[c];
      d.h_b1[o0 + (size_t)c * d.NB + b] = e1[c];
    }
    d.h_comp[(size_t)slot * d.NB + b] = -1;
  }
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

// The kernels of a step share one shared-memory carveout (the largest), so
// the SMs are not reconfigured between consecutive kernels with different
// shared-memory needs (measured: ~12 us bubbles before k_detect and the kick).
void configure_drift() {
  cudaFuncSetAttribute(k_jump_drift, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

}  // namespace mx
