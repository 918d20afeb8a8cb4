// k_init.cu -- set-up and readout: heliocentric <-> democratic-heliocentric
// coordinates, changeover radii and per-planetesimal drag constants.
//
// DH velocities are barycentric: v_b = v_h - sum_i m_i v_h,i / (m0 + sum_i m_i)
// over the massive bodies; the way back is v_h = v_b + P/m0 with
// P = sum_i m_i v_b,i (arXiv 2601.16791, Sec. 2.1.3: mco_h2dh / mco_dh2h,
// with their momentum loops over massive bodies only).  A big body's
// changeover radius is rcrit_hill Hill radii, R_H = a (m/(3 m0))^(1/3), from
// its osculating semimajor axis with gm = G (m0 + m) (Sec. 2.1.3 mce_hill;
// Sec. 3.5 for gm).
#include "mx_common.cuh"
#include "mx_kernels.h"

namespace mx {

constexpr double kAuKm = 1.495978707e8;   // astronomical unit [km]

// One block per system: V (stored in P) and, if do_rcrit, the radii.
__global__ void __launch_bounds__(kThreads) k_init_sys(Dev d, int do_rcrit, double rcrit_hill) {
  const SysDev& S = d.sys[blockIdx.x];
  const int N = d.N;
  __shared__ double red[4][kThreads];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double mu = d.bmu[S.boff + i];
    acc[0] = fma(mu, d.xv[3 * (size_t)N + g], acc[0]);
    acc[1] = fma(mu, d.xv[4 * (size_t)N + g], acc[1]);
    acc[2] = fma(mu, d.xv[5 * (size_t)N + g], acc[2]);
    acc[3] += mu;
    if (do_rcrit) {
      const double x = d.xv[g], y = d.xv[(size_t)N + g], z = d.xv[2 * (size_t)N + g];
      const double u = d.xv[3 * (size_t)N + g], v = d.xv[4 * (size_t)N + g],
                   w = d.xv[5 * (size_t)N + g];
      const double r = sqrt(x * x + y * y + z * z);
      double a = 1.0 / (2.0 / r - (u * u + v * v + w * w) / (S.mu0 + mu));
      if (!(a > 0.0)) a = r;
      set_rcrit(d, S.boff + i, rcrit_hill * a * cbrt(mu / (3.0 * S.mu0)));
    }
  }
  for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double inv = 1.0 / (S.mu0 + red[3][0]);
    for (int c = 0; c < 3; ++c) d.P[3 * blockIdx.x + c] = red[c][0] * inv;
  }
}

// Per body: v -= V of its system; drag constants for planetesimals.
__global__ void __launch_bounds__(kThreads) k_init_bodies(Dev d, const double* rp_km,
                                                          const double* rho, int set_drag) {
  const Tile t = d.tiles[blockIdx.x];
  if (threadIdx.x >= t.count) return;
  const int N = d.N;
  const int j = t.start + threadIdx.x;
  const double* V = d.P + 3 * t.sys;
  for (int c = 0; c < 3; ++c) d.xv[(size_t)(3 + c) * N + j] -= V[c];
  if (set_drag) {
    const double r = rp_km[j], q = rho[j];
    d.rp_cm[j] = r * 1.0e5;
    d.kdrag[j] = 3.0 / (8.0 * (r / kAuKm) * q);
  }
}

// Heliocentric readout: x, v + P/m0 (P from k_prep).
__global__ void __launch_bounds__(kThreads) k_readout(Dev d, double* out) {
  const Tile t = d.tiles[blockIdx.x];
  if (threadIdx.x >= t.count) return;
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  const int j = t.start + threadIdx.x;
  const double* P = d.P + 3 * t.sys;
  for (int c = 0; c < 3; ++c) {
    out[(size_t)c * N + j] = d.xv[(size_t)c * N + j];
    out[(size_t)(3 + c) * N + j] = d.xv[(size_t)(3 + c) * N + j] + P[c] * S.inv_mu0;
  }
}

// The step counter and the half-kick counters at step `step` (kernel
// arguments, so that setting them takes no host-to-device copy).
__global__ void k_set_step(Dev d, long long step) {
  d.kick_ctr[0] = d.kick_ctr[1] = (int)(2 * step);
  d.gstep[0] = step;
}

void launch_set_step(const Dev& d, long long step, cudaStream_t st) {
  k_set_step<<<1, 1, 0, st>>>(d, step);
}

void launch_init_sys(const Dev& d, int do_rcrit, double rcrit_hill, cudaStream_t st) {
  k_init_sys<<<d.nsys, kThreads, 0, st>>>(d, do_rcrit, rcrit_hill);
}

void launch_init_bodies(const Dev& d, const double* rp_km, const double* rho, int set_drag,
                        cudaStream_t st) {
  k_init_bodies<<<d.ntiles, d.tile, 0, st>>>(d, rp_km, rho, set_drag);
}

void launch_readout(const Dev& d, double* out, cudaStream_t st) {
  k_readout<<<d.ntiles, d.tile, 0, st>>>(d, out);
}

}  // namespace mx
