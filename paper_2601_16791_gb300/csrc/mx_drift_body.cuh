// mx_drift_body.cuh -- the per-tile body of the jump and Kepler drift
// (k_drift.cu), shared by its kernel and the persistent step kernel.
#pragma once
#include "mx_common.cuh"
#include "mx_kepler.cuh"

namespace mx {

// Jump by (jump_frac h) P/m0, save the pre-drift state, drift by the system's
// h: the bodies of tile `bid`, one per thread (blockDim.x = the tile size).
__device__ __forceinline__ void jump_drift_tile(const Dev& d, double jump_frac, int bid) {
  const Tile t = d.tiles[bid];
  const SysDev& S = d.sys[t.sys];
  if (bid == 0 && threadIdx.x == 0) {
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

}  // namespace mx
