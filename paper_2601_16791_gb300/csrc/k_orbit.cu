// k_orbit.cu -- the ejection test and the element conversion of Sec. 3.5
// (arXiv 2601.16791): a body whose osculating heliocentric orbit has e >= 1
// is flagged ejected (stat -3), a massive one loses its mass; the count of
// flagged bodies is a per-system reduction over stat.
//
// One thread per body; each reads its 6 state doubles and writes at most a
// byte and a double, so the test is an O(N) pass bound by its FP64
// divisions and square roots.  Heliocentric velocities are v_b + P/m0 with
// the system's P as the last k_prep computed it.
#include "mx_common.cuh"
#include "mx_kernels.h"
#include "mx_orbit.cuh"

namespace mx {

// scheduled = 1: the test that follows a step; with deferral on, the slot
// just recorded is marked so that the catch-up runs the same test on the
// planetesimals it replays.  Lagged planetesimals are tested there instead.
__global__ void __launch_bounds__(kThreads) k_eject(Dev d, int scheduled) {
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  if (scheduled && d.defer && blockIdx.x == 0 && threadIdx.x == 0) {
    const int slot = *d.hstep - 1;   // the kick that ended the step moved hstep on
    if (slot >= 0 && slot < d.hist_cap) d.h_ej[slot] = 1;
  }
  if (threadIdx.x >= t.count) return;
  const int j = t.start + threadIdx.x;
  if (removed(d, j) || (d.defer && d.lag[j])) return;
  const int N = d.N;
  const double* P = d.P + 3 * t.sys;
  const int jl = j - S.off;
  const double gm = (jl < S.nbig) ? S.mu0 + d.bmu[S.boff + jl] : S.mu0;
  if (dh_unbound(gm, S.inv_mu0, P, d.xv[j], d.xv[(size_t)N + j], d.xv[2 * (size_t)N + j],
                 d.xv[3 * (size_t)N + j], d.xv[4 * (size_t)N + j], d.xv[5 * (size_t)N + j])) {
    d.stat[j] = kStatEjected;
    if (jl < S.nbig) d.bmu[S.boff + jl] = 0.0;   // read by no other thread of this launch
    atomicAdd(d.ej_new, 1);
  }
}

// Elements of every body (6 x N rows q, e, i, varpi, Omega, M).
__global__ void __launch_bounds__(kThreads) k_elements(Dev d, double* out) {
  const Tile t = d.tiles[blockIdx.x];
  if (threadIdx.x >= t.count) return;
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  const int j = t.start + threadIdx.x;
  const double* P = d.P + 3 * t.sys;
  const int jl = j - S.off;
  const double gm = (jl < S.nbig) ? S.mu0 + d.bmu[S.boff + jl] : S.mu0;
  double el[6];
  orbit_elements(gm, d.xv[j], d.xv[(size_t)N + j], d.xv[2 * (size_t)N + j],
                 d.xv[3 * (size_t)N + j] + P[0] * S.inv_mu0,
                 d.xv[4 * (size_t)N + j] + P[1] * S.inv_mu0,
                 d.xv[5 * (size_t)N + j] + P[2] * S.inv_mu0, el);
  for (int c = 0; c < 6; ++c) out[(size_t)c * N + j] = el[c];
}

// Removed bodies of each system (count of stat < 0); one block per system.
__global__ void __launch_bounds__(kThreads) k_stat_count(Dev d, int* out) {
  const SysDev& S = d.sys[blockIdx.x];
  __shared__ int red[kThreads];
  int c = 0;
  for (int i = threadIdx.x; i < S.n; i += blockDim.x) c += (d.stat[S.off + i] < 0) ? 1 : 0;
  red[threadIdx.x] = c;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

void launch_eject(const Dev& d, int scheduled, cudaStream_t st) {
  k_eject<<<d.ntiles, d.tile, 0, st>>>(d, scheduled);
}

void launch_elements(const Dev& d, double* out, cudaStream_t st) {
  k_elements<<<d.ntiles, d.tile, 0, st>>>(d, out);
}

void launch_stat_count(const Dev& d, int* out, cudaStream_t st) {
  k_stat_count<<<d.nsys, kThreads, 0, st>>>(d, out);
}

// The test runs between the step's kernels: the same carveout as theirs.
void configure_orbit() {
  cudaFuncSetAttribute(k_eject, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

}  // namespace mx
