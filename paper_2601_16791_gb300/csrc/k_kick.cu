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
#include "mx_growth.cuh"
#include "mx_kernels.h"
#include "mx_physics.cuh"

namespace mx {

__device__ __forceinline__ void stage_bigs(const Dev& d, const SysDev& S, int c0, int cn,
                                           BigSmem& sb) {
  for (int k = threadIdx.x; k < cn; k += blockDim.x) {
    const int b = S.boff + c0 + k;
    const double rc = d.brc[b];
    sb.x[k] = d.bx[b];
    sb.y[k] = d.by[b];
    sb.z[k] = d.bz[b];
    sb.mu[k] = d.bmu[b];
    sb.rc[k] = rc;
    sb.rc2[k] = rc * rc;
    sb.rc2lo[k] = 0.01 * (rc * rc);
    sb.rc01[k] = 0.1 * rc;
    sb.i09rc[k] = (rc > 0.0) ? 1.0 / (0.9 * rc) : 0.0;
  }
}

// Gravity on target j (local index jl, own changeover radius rcj) from all big
// bodies of its system; every thread of the block must call it.
__device__ __forceinline__ void gravity_all(const Dev& d, const SysDev& S, BigSmem& sb, bool act,
                                            int jl, double rcj, double x, double y, double z,
                                            double& ax, double& ay, double& az) {
  const bool jbig = jl < S.nbig;
  for (int c0 = 0; c0 < S.nbig; c0 += kBigChunk) {
    const int cn = min(kBigChunk, S.nbig - c0);
    __syncthreads();
    stage_bigs(d, S, c0, cn, sb);
    __syncthreads();
    if (!act) continue;
    if (!jbig) {
      for (int k = 0; k < cn; ++k)
        pair_acc(x - sb.x[k], y - sb.y[k], z - sb.z[k], sb.mu[k], sb.rc2[k], sb.rc2lo[k],
                 sb.rc01[k], sb.i09rc[k], ax, ay, az);
    } else {
      for (int k = 0; k < cn; ++k) {
        if (c0 + k == jl) continue;
        const double rc = fmax(sb.rc[k], rcj);
        pair_acc(x - sb.x[k], y - sb.y[k], z - sb.z[k], sb.mu[k], rc * rc, 0.01 * (rc * rc),
                 0.1 * rc, 1.0 / (0.9 * rc), ax, ay, az);
      }
    }
  }
}

// Momentum of each system's massive bodies and the staged big positions.
// One block per system; a fixed partition and tree keep the sum deterministic.
// nkick > 0: the kernel that follows makes nkick half kicks; the kick counter
// (for recording or replaying the k branch of Eq. 7) advances here.
// The first launch of a step (jump_frac = 0, nkick > 0) first applies the
// growth tracks (Sec. 3.3) of a system that has them, at t = gstep x h; the
// launch that ends a step (jump_frac != 0) counts it in gstep.
__global__ void __launch_bounds__(kThreads) k_prep(Dev d, double jump_frac, int nkick) {
  const SysDev& S = d.sys[blockIdx.x];
  __shared__ double red[3][kThreads];
  if (S.grow_on && nkick > 0 && jump_frac == 0.0)
    grow_update(d, S, (double)d.gstep[0] * S.h, red);
  if (nkick > 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    d.kick_ctr[1] = d.kick_ctr[0];
    d.kick_ctr[0] += nkick;
    if (jump_frac != 0.0) d.gstep[0] += 1;   // no block reads it in this launch
  }
  const int N = d.N;
  // With at most 32 big bodies (one per lane of warp 0) the tree below adds
  // only zeros above its last five levels, so warp 0 alone takes those five
  // levels with shuffles, in the same order (the same sum, bit for bit),
  // without block barriers; the other warps have nothing to stage.
  const bool one_warp = S.nbig <= 32;
  if (one_warp && threadIdx.x >= 32) return;
  double p[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double m = d.bmu[S.boff + i];
    p[0] = fma(m, d.xv[3 * (size_t)N + g], p[0]);
    p[1] = fma(m, d.xv[4 * (size_t)N + g], p[1]);
    p[2] = fma(m, d.xv[5 * (size_t)N + g], p[2]);
  }
  double Ps[3];
  if (one_warp) {
    for (int s = 16; s > 0; s >>= 1)
      for (int c = 0; c < 3; ++c) p[c] += __shfl_down_sync(0xffffffffu, p[c], s);
    for (int c = 0; c < 3; ++c) Ps[c] = __shfl_sync(0xffffffffu, p[c], 0);
  } else {
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = p[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s)
        for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
      __syncthreads();
    }
    for (int c = 0; c < 3; ++c) Ps[c] = red[c][0];
  }
  double* P = d.P + 3 * blockIdx.x;
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) P[c] = Ps[c];
  double dj[3];
  jump_vec(Ps, S, jump_frac, dj);
  // the kicks of a history slot (the end of a step, or the leading half kick
  // of a call, recorded as -1) enter the history deferred planetesimals replay
  const int slot = d.defer ? *d.hstep : 0;
  const bool rec = d.defer && nkick > 0 && slot < d.hist_cap;
  if (rec && threadIdx.x == 0) {
    for (int c = 0; c < 3; ++c) d.h_P[(size_t)slot * 6 * d.nsys + 3 * d.nsys + 3 * blockIdx.x + c] = Ps[c];
    if (blockIdx.x == 0) {
      d.h_nkick[slot] = (jump_frac != 0.0) ? nkick : -nkick;
      d.h_ej[slot] = 0;   // k_eject marks the slots an ejection test follows
    }
  }
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double bx = d.xv[g] + dj[0];
    const double by = d.xv[(size_t)N + g] + dj[1];
    const double bz = d.xv[2 * (size_t)N + g] + dj[2];
    d.bx[S.boff + i] = bx;
    d.by[S.boff + i] = by;
    d.bz[S.boff + i] = bz;
    if (S.grow_on) d.gap_r[S.boff + i] = sqrt(bx * bx + by * by);   // gap centre (Sec. 3.1)
    if (rec) {
      const size_t o = (size_t)slot * 3 * d.NB + S.boff + i;
      d.h_bx[o] = bx;
      d.h_bx[o + d.NB] = by;
      d.h_bx[o + 2 * (size_t)d.NB] = bz;
      d.h_mu[(size_t)slot * d.NB + S.boff + i] = removed(d, g) ? -1.0 : d.bmu[S.boff + i];
      d.h_rc[(size_t)slot * d.NB + S.boff + i] = d.brc[S.boff + i];
      if (S.grow_on) {
        const size_t q = (size_t)slot * 3 * d.NB + S.boff + i;
        d.h_gap[q] = d.gap_r[S.boff + i];
        d.h_gap[q + d.NB] = d.gap_w[S.boff + i];
        d.h_gap[q + 2 * (size_t)d.NB] = d.gap_f[S.boff + i];
      }
    }
  }
}

// Jump then kick (nkick half kicks of kick_frac * h each, gravity evaluated once; the
// drag is re-evaluated before each with the updated velocity).  The momentum
// P read here is the one k_prep just computed; it stays valid across the
// kicks because the K-weighted pair forces are antisymmetric and the drag acts
// on massless bodies only.
template <int NKICK>
__global__ void __launch_bounds__(kThreads) k_jump_kick(Dev d, double jump_frac, double kick_frac) {
  __shared__ BigSmem sb;
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  const double* P = d.P + 3 * t.sys;
  const int N = d.N;
  double dj[3];
  jump_vec(P, S, jump_frac, dj);
  const double kick_h = kick_frac * S.h;
  const int j = t.start + threadIdx.x;
  // a deferred planetesimal is kicked by the window's catch-up instead; a
  // removed body is not kicked
  const bool act = threadIdx.x < t.count && !(d.defer && d.lag[j]) && !removed(d, j);
  // the last kernel of a history slot moves on to the next one
  if (d.defer && blockIdx.x == 0 && threadIdx.x == 0) *d.hstep += 1;
  const int jl = j - S.off;
  double x = 0, y = 0, z = 0, u = 0, v = 0, w = 0, rcj = 0.0;
  if (act) {
    x = d.xv[j] + dj[0];
    y = d.xv[(size_t)N + j] + dj[1];
    z = d.xv[2 * (size_t)N + j] + dj[2];
    u = d.xv[3 * (size_t)N + j];
    v = d.xv[4 * (size_t)N + j];
    w = d.xv[5 * (size_t)N + j];
    if (jl < S.nbig) rcj = d.brc[S.boff + jl];
  }
  double ax = 0, ay = 0, az = 0;
  gravity_all(d, S, sb, act, jl, rcj, x, y, z, ax, ay, az);
  if (!act) return;
  if (jump_frac != 0.0) {
    d.xv[j] = x;
    d.xv[(size_t)N + j] = y;
    d.xv[2 * (size_t)N + j] = z;
  }
  const bool drag = S.gas_on && jl >= S.nbig;
  const double hp0 = P[0] * S.inv_mu0, hp1 = P[1] * S.inv_mu0, hp2 = P[2] * S.inv_mu0;
  const double rp = drag ? d.rp_cm[j] : 0.0, kd = drag ? d.kdrag[j] : 0.0;
  const int kbase = d.kmode ? d.kick_ctr[1] : 0;
  // the gas at the (fixed) position, shared by the launch's half kicks
  GasAt gq = drag ? gas_at(S, x, y) : GasAt{false, 0.0, 0.0, 0.0};
  if (drag && S.grow_on) gq.rho *= gap_factor(d, S, x, y);
  if (drag && S.dg_on) {   // disk gravity: fixed over the launch, like the big bodies' gravity
    ax += gq.adg[0];
    ay += gq.adg[1];
  }
  const DragConst dc = drag ? drag_const(S, gq, x, y, hp0, hp1, hp2, rp, kd) : DragConst{};
#pragma unroll
  for (int kk = 0; kk < NKICK; ++kk) {
    double a[3] = {0.0, 0.0, 0.0};
    if (drag) {
      const int kidx = kbase + kk;
      const bool kuse = d.kmode != 0 && kidx < d.kcap;
      const size_t word = (size_t)kidx * d.kwords + (j >> 5);
      int kin = -1, kout = 0;
      if (kuse && d.kmode == 2) kin = (d.kbits[word] >> (j & 31)) & 1u;
      gas_drag_at(S, dc, u, v, w, a, kin, &kout);
      if (kuse && d.kmode == 1 && kout) atomicOr(&d.kbits[word], 1u << (j & 31));
    }
    u = fma(kick_h, ax + a[0], u);
    v = fma(kick_h, ay + a[1], v);
    w = fma(kick_h, az + a[2], w);
  }
  d.xv[3 * (size_t)N + j] = u;
  d.xv[4 * (size_t)N + j] = v;
  d.xv[5 * (size_t)N + j] = w;
  if (!(finite_d(x) && finite_d(y) && finite_d(z) && finite_d(u) && finite_d(v) && finite_d(w)))
    atomicOr(d.status, ST_NONFINITE);
}

// Kick acceleration (gravity + drag) without changing the state: 3 x N.
__global__ void __launch_bounds__(kThreads) k_accel(Dev d, double* acc, int drag_only,
                                                    int acc_stride, int acc_base) {
  __shared__ BigSmem sb;
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
  if (nkick == 2) k_jump_kick<2><<<d.ntiles, d.tile, 0, st>>>(d, jump_frac, kick_frac);
  else k_jump_kick<1><<<d.ntiles, d.tile, 0, st>>>(d, jump_frac, kick_frac);
}

void launch_accel(const Dev& d, double* acc, int drag_only, int acc_stride, int acc_base,
                  cudaStream_t st) {
  k_accel<<<d.ntiles, d.tile, 0, st>>>(d, acc, drag_only, acc_stride, acc_base);
}

// The kernels of a step share one shared-memory carveout (the largest), so
// the SMs are not reconfigured between consecutive kernels with different
// shared-memory needs (measured: ~12 us bubbles before k_detect and the kick).
void configure_kick() {
  const int c = cudaSharedmemCarveoutMaxShared;
  cudaFuncSetAttribute(k_prep, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_jump_kick<1>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_jump_kick<2>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
}

}  // namespace mx
