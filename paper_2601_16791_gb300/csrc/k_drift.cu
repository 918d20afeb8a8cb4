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
#include "mx_drift_body.cuh"
#include "mx_kepler.cuh"
#include "mx_kernels.h"

namespace mx {

__global__ void __launch_bounds__(kThreads) k_jump_drift(Dev d, double jump_frac) {
  jump_drift_tile(d, jump_frac, blockIdx.x);
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
