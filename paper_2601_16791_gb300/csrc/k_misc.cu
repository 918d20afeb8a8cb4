// k_misc.cu -- energy / angular momentum of the massive bodies and the FP64
// throughput probe used as the roofline denominator.
//
// Energy (arXiv 2601.16791, Sec. 2.1.3: mxx_en runs over massive bodies
// only), in democratic-heliocentric form: sum_i |p_i|^2/(2 m_i) +
// |sum_i p_i|^2/(2 m0) - sum_i G m0 m_i/r_i - sum_{i<j} G m_i m_j/r_ij, and
// L = sum_i m_i x_i x v_i.  One block per system, fixed partition and tree.
#include "mx_common.cuh"
#include "mx_kernels.h"

namespace mx {

__global__ void __launch_bounds__(kThreads) k_energy(Dev d, double* out /* 7 per system */) {
  const SysDev& S = d.sys[blockIdx.x];
  const double inv_G = S.inv_G, m_star = S.m_star;
  const int N = d.N;
  __shared__ double red[8][kThreads];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // ke, pe, Px, Py, Pz, Lx, Ly, Lz
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double mu = d.bmu[S.boff + i];
    if (mu == 0.0) continue;
    const double m = mu * inv_G;
    const double x = d.xv[g], y = d.xv[(size_t)N + g], z = d.xv[2 * (size_t)N + g];
    const double u = d.xv[3 * (size_t)N + g], v = d.xv[4 * (size_t)N + g], w = d.xv[5 * (size_t)N + g];
    acc[0] += 0.5 * m * (u * u + v * v + w * w);
    acc[1] -= S.mu0 * m / sqrt(x * x + y * y + z * z);
    acc[2] += m * u;
    acc[3] += m * v;
    acc[4] += m * w;
    acc[5] += m * (y * w - z * v);
    acc[6] += m * (z * u - x * w);
    acc[7] += m * (x * v - y * u);
    for (int k = i + 1; k < S.nbig; ++k) {
      const double muk = d.bmu[S.boff + k];
      if (muk == 0.0) continue;
      const int gk = S.off + k;
      const double dx = d.xv[gk] - x, dy = d.xv[(size_t)N + gk] - y, dz = d.xv[2 * (size_t)N + gk] - z;
      acc[1] -= m * muk / sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
  for (int c = 0; c < 8; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 8; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double Px = red[2][0], Py = red[3][0], Pz = red[4][0];
    double* o = out + 7 * blockIdx.x;
    o[0] = red[0][0] + (Px * Px + Py * Py + Pz * Pz) / (2.0 * m_star);
    o[1] = red[1][0];
    o[2] = o[0] + o[1];
    o[3] = 0.0;
    o[4] = red[5][0];
    o[5] = red[6][0];
    o[6] = red[7][0];
  }
}

void launch_energy(const Dev& d, double* out, cudaStream_t st) {
  k_energy<<<d.nsys, kThreads, 0, st>>>(d, out);
}

// Independent FMA chains, eight per thread, so the FP64 pipe is the limit.
__global__ void __launch_bounds__(256) k_dfma(double* sink, int iters, double a, double b) {
  double r[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) r[k] = 1e-3 * threadIdx.x + k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = fma(r[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += r[k];
  if (s == 123.456) sink[0] = s;   // keeps the chains alive
}

void launch_dfma(double* sink, int blocks, int iters, cudaStream_t st) {
  k_dfma<<<blocks, 256, 0, st>>>(sink, iters, 0.9999999, 1e-9);
}

}  // namespace mx
