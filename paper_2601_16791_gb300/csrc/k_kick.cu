// k_kick.cu -- interaction kick with the changeover function K and gas drag
// (arXiv 2601.16791, Sec. 2.1.3 mfo_drct listing; Sec. 3.1 Eqs. 1-7; the
// velocity update of the Sec. 2.1.2 listing, v += (h/2)(a + a_user)).
//
// One thread per target body, a block per tile of one system.  The system's
// big bodies are staged in shared memory in chunks with the constants each
// pair needs, so the inner loop is loads from shared memory and FP64 FMAs.
// Each target sums its sources in ascending order (the gather form of the
// parallel loop), so results do not depend on the launch shape.
#include "mx_common.cuh"
#include "mx_kernels.h"
#include "mx_kick_body.cuh"

namespace mx {

// One block per system: its momentum and the staged big positions.
__global__ void __launch_bounds__(kThreads) k_prep(Dev d, double jump_frac, int nkick) {
  prep_system(d, jump_frac, nkick, blockIdx.x);
}

// One block per tile (register use capped at 80: three resident blocks of
// 256 threads; see jump_kick_tile).
template <int NKICK, bool FUSED>
__global__ void __launch_bounds__(kThreads, 3) k_jump_kick(Dev d, double jump_frac,
                                                          double kick_frac) {
  extern __shared__ double dsm[];
  jump_kick_tile<NKICK, FUSED>(d, jump_frac, kick_frac, blockIdx.x, dsm);
}

// Kick acceleration (gravity + drag) without changing the state: 3 x N.
__global__ void __launch_bounds__(kThreads) k_accel(Dev d, double* acc, int drag_only,
                                                    int acc_stride, int acc_base) {
  extern __shared__ double dsm[];
  BigSmem sb(dsm, big_chunk(d.big_max));
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  const double* P = d.P + 3 * t.sys;
  const int N = d.N;
  const bool valid = threadIdx.x < t.count;
  const int j = t.start + threadIdx.x;
  const bool act = valid && !removed(d, j);   // a removed body gets zero
  const int jl = j - S.off;
  double x = 0, y = 0, z = 0, u = 0, v = 0, w = 0, rcj = 0.0;
  if (act) {
    x = d.xv[j];
    y = d.xv[(size_t)N + j];
    z = d.xv[2 * (size_t)N + j];
    u = d.xv[3 * (size_t)N + j];
    v = d.xv[4 * (size_t)N + j];
    w = d.xv[5 * (size_t)N + j];
    if (jl < S.nbig) rcj = d.brc[S.boff + jl];
  }
  double ax = 0, ay = 0, az = 0;
  if (!drag_only) gravity_all(d, S, sb, act, jl, rcj, x, y, z, ax, ay, az);
  if (!valid) return;
  const bool drag = act && S.gas_on && jl >= S.nbig;
  double a[3] = {0.0, 0.0, 0.0};
  if (drag) {
    int kout = 0;
    gas_drag(S, x, y, z, u + P[0] * S.inv_mu0, v + P[1] * S.inv_mu0, w + P[2] * S.inv_mu0,
             d.rp_cm[j], d.kdrag[j], a, -1, &kout, S.grow_on ? gap_factor(d, S, x, y) : 1.0);
  }
  if (drag_only) {
    if (jl < S.nbig) return;
    const int o = j - acc_base;
    acc[o] = a[0];
    acc[(size_t)acc_stride + o] = a[1];
    acc[2 * (size_t)acc_stride + o] = a[2];
  } else {
    acc[j] = ax + a[0];
    acc[(size_t)N + j] = ay + a[1];
    acc[2 * (size_t)N + j] = az + a[2];
  }
}

void launch_prep(const Dev& d, double jump_frac, int nkick, cudaStream_t st) {
  k_prep<<<d.nsys, kThreads, 0, st>>>(d, jump_frac, nkick);
}

void launch_jump_kick(const Dev& d, double jump_frac, double kick_frac, int nkick,
                      cudaStream_t st) {
  const size_t sm = kick_smem_bytes(d, false);
  if (nkick == 2) k_jump_kick<2, false><<<d.ntiles, d.tile, sm, st>>>(d, jump_frac, kick_frac);
  else k_jump_kick<1, false><<<d.ntiles, d.tile, sm, st>>>(d, jump_frac, kick_frac);
}

// The interior steps' kick with its own prep (no k_prep launch before it):
// jump 1/2, two half kicks; for forward runs without growth tracks or k
// branches recorded or replayed.
void launch_jump_kick_fused(const Dev& d, cudaStream_t st) {
  k_jump_kick<2, true><<<d.ntiles, d.tile, kick_smem_bytes(d, true), st>>>(d, 0.5, 0.5);
}

void launch_accel(const Dev& d, double* acc, int drag_only, int acc_stride, int acc_base,
                  cudaStream_t st) {
  k_accel<<<d.ntiles, d.tile, kick_smem_bytes(d, false), st>>>(d, acc, drag_only, acc_stride,
                                                              acc_base);
}

// The kernels of a step share one shared-memory carveout (the largest), so
// the SMs are not reconfigured between consecutive kernels with different
// shared-memory needs (measured: ~12 us bubbles before k_detect and the kick).
void configure_kick() {
  const int c = cudaSharedmemCarveoutMaxShared;
  cudaFuncSetAttribute(k_prep, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_jump_kick<1, false>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_jump_kick<2, false>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_jump_kick<2, true>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
}

}  // namespace mx
