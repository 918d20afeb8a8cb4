// mx_kick_body.cuh -- the per-tile bodies of the jump and kick and of the
// momentum prep (k_kick.cu), shared by their kernels and the persistent step
// kernel.
#pragma once
#include "mx_common.cuh"
#include "mx_growth.cuh"
#include "mx_physics.cuh"

namespace mx {


// Big positions come from k_prep's copy (d.bx), or, with `dj` (a kick that
// makes its own prep), from the state plus the jump.  The block's last warp
// takes the first bodies: warp 0 makes the momentum sum of a fused kick, and
// the warps of a block share the four warp schedulers in order, so the two
// pieces of per-block work land on different schedulers.
__device__ __forceinline__ void stage_bigs(const Dev& d, const SysDev& S, int c0, int cn,
                                           BigSmem& sb, const double* dj) {
  const int first = (blockDim.x > 32) ? (int)blockDim.x - 32 : 0;
  for (int r = threadIdx.x; r < cn + first; r += blockDim.x) {
    const int k = r - first;   // threads [first, blockDim) take k = 0, 1, ...
    if (k < 0) continue;
    const int b = S.boff + c0 + k;
    const size_t NB = d.NB;
    if (dj) {
      const size_t g = (size_t)S.off + c0 + k;
      sb.x[k] = d.xv[g] + dj[0];
      sb.y[k] = d.xv[(size_t)d.N + g] + dj[1];
      sb.z[k] = d.xv[2 * (size_t)d.N + g] + dj[2];
    } else {
      sb.x[k] = d.bx[b];
      sb.y[k] = d.by[b];
      sb.z[k] = d.bz[b];
    }
    sb.mu[k] = d.bmu[b];
    sb.rc[k] = d.brc[b];
    sb.rc2[k] = d.brc4[b];
    sb.rc2lo[k] = d.brc4[NB + b];
    sb.rc01[k] = d.brc4[2 * NB + b];
    sb.i09rc[k] = d.brc4[3 * NB + b];
  }
}

// Gravity on target j (local index jl, own changeover radius rcj) from all big
// bodies of its system; every thread of the block must call it.
__device__ __forceinline__ void gravity_all(const Dev& d, const SysDev& S, BigSmem& sb, bool act,
                                            int jl, double rcj, double x, double y, double z,
                                            double& ax, double& ay, double& az,
                                            const double* dj = nullptr) {
  const bool jbig = jl < S.nbig;
  for (int c0 = 0; c0 < S.nbig; c0 += sb.chunk) {
    const int cn = min(sb.chunk, S.nbig - c0);
    __syncthreads();
    stage_bigs(d, S, c0, cn, sb, dj);
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

// P = sum of mu_i v_i over the big bodies of system S, in out[0..2] (shared)
// for every thread of the block.  The sum has one fixed partition and tree,
// whatever the block size: kThreads partial sums, partial t over the bodies
// i = t (mod kThreads) in ascending order, then a pairwise tree over the
// partials.  With at most 32 big bodies every partial past the first 32 is
// zero, so the tree adds only zeros above its last five levels, and warp 0
// takes those five levels with shuffles (the same sum, bit for bit).
// red: kThreads x 3 shared scratch.  Every thread of the block must call it.
__device__ __forceinline__ void system_momentum(const Dev& d, const SysDev& S,
                                                double (*red)[kThreads], double* out) {
  const int N = d.N;
  auto partial = [&](int t, double* p) {
    p[0] = p[1] = p[2] = 0.0;
    for (int i = t; i < S.nbig; i += kThreads) {
      const int g = S.off + i;
      const double m = d.bmu[S.boff + i];
      p[0] = fma(m, d.xv[3 * (size_t)N + g], p[0]);
      p[1] = fma(m, d.xv[4 * (size_t)N + g], p[1]);
      p[2] = fma(m, d.xv[5 * (size_t)N + g], p[2]);
    }
  };
  if (S.nbig <= 32) {
    if (threadIdx.x < 32) {
      double p[3];
      partial(threadIdx.x, p);
      // a level whose offset s >= nbig adds lanes holding +0 to every lane
      // below s (a partial is never -0: it starts at +0), which changes no
      // bit, so it is skipped
      for (int s = 16; s > 0; s >>= 1)
        if (s < S.nbig)
          for (int c = 0; c < 3; ++c) p[c] += __shfl_down_sync(0xffffffffu, p[c], s);
      if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) out[c] = p[c];
    }
  } else {
    for (int t = threadIdx.x; t < kThreads; t += blockDim.x) {
      double p[3];
      partial(t, p);
      for (int c = 0; c < 3; ++c) red[c][t] = p[c];
    }
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
      for (int t = threadIdx.x; t < s; t += blockDim.x)
        for (int c = 0; c < 3; ++c) red[c][t] += red[c][t + s];
      __syncthreads();
    }
    if (threadIdx.x == 0)
      for (int c = 0; c < 3; ++c) out[c] = red[c][0];
  }
  __syncthreads();
}

// Momentum of each system's massive bodies and the staged big positions.
// One block per system (system_momentum fixes the sum's order).
// nkick > 0: the kernel that follows makes nkick half kicks; the kick counter
// (for recording or replaying the k branch of Eq. 7) advances here.
// The first launch of a step (jump_frac = 0, nkick > 0) first applies the
// growth tracks (Sec. 3.3) of a system that has them, at t = gstep x h; the
// launch that ends a step (jump_frac != 0) counts it in gstep.
__device__ __forceinline__ void prep_system(const Dev& d, double jump_frac, int nkick, int sysi) {
  const SysDev& S = d.sys[sysi];
  __shared__ double red[3][kThreads];
  __shared__ double s_P[3];
  if (S.grow_on && nkick > 0 && jump_frac == 0.0)
    grow_update(d, S, (double)d.gstep[0] * S.h, red);
  if (nkick > 0 && sysi == 0 && threadIdx.x == 0) {
    d.kick_ctr[1] = d.kick_ctr[0];
    d.kick_ctr[0] += nkick;
    if (jump_frac != 0.0) d.gstep[0] += 1;   // no block reads it in this launch
  }
  const int N = d.N;
  system_momentum(d, S, red, s_P);
  const double Ps[3] = {s_P[0], s_P[1], s_P[2]};
  double* P = d.P + 3 * sysi;
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) P[c] = Ps[c];
  double dj[3];
  jump_vec(Ps, S, jump_frac, dj);
  // the kicks of a history slot (the end of a step, or the leading half kick
  // of a call, recorded as -1) enter the history deferred planetesimals replay
  const int slot = d.defer ? *d.hstep : 0;
  const bool rec = d.defer && nkick > 0 && slot < d.hist_cap;
  if (rec && threadIdx.x == 0) {
    for (int c = 0; c < 3; ++c) d.h_P[(size_t)slot * 6 * d.nsys + 3 * d.nsys + 3 * sysi + c] = Ps[c];
    if (sysi == 0) {
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

// The prep of a kick made inside it (the FUSED kick of an interior step):
// each block computes its system's P (system_momentum: the sum k_prep makes,
// bit for bit) and stages the big bodies from the state plus the jump.  The
// big bodies' own results go to d.bk only, so that no block of the launch
// overwrites a big body's state that another block still reads; the drift
// that follows reads them there.  The block of each system's first tile
// stores P and the history record k_prep would, and system 0's advances the
// counters.  Those blocks read the history slot before they arrive, and the
// last of them to arrive moves the slot on (no block waits for another).
struct FusedPrep {
  double P[3], dj[3], hp[3];   // P, the jump (jump_vec at jump_frac), P/m0
};

// P of a fused kick, its jump (jump_vec) and P/m0, into shared memory.  With
// at most 32 big bodies, component c is summed by warp c mod (warps) with
// system_momentum's partials and tree (the same bits), and the same warp
// forms its jump and P/m0 component: the block's few per-block instructions
// are spread over its warps, which sit on different warp schedulers.  With
// more, system_momentum.  Every thread of the block must call it; ends with a
// block barrier.
__device__ __forceinline__ void fused_momentum(const Dev& d, const SysDev& S, double jump_frac,
                                               double (*red)[kThreads], double* sP, double* sdj,
                                               double* shp) {
  const int N = d.N;
  const double cj = (jump_frac * S.h) * S.inv_mu0;
  if (S.nbig <= 32) {
    const int nw = (int)(blockDim.x >> 5), warp = (int)(threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int c = warp; c < 3; c += nw) {
      double p = 0.0;
      if (lane < S.nbig) p = fma(d.bmu[S.boff + lane], d.xv[(size_t)(3 + c) * N + S.off + lane], p);
      for (int s = 16; s > 0; s >>= 1)
        if (s < S.nbig) p += __shfl_down_sync(0xffffffffu, p, s);
      if (lane == 0) {
        sP[c] = p;
        sdj[c] = cj * p;
        shp[c] = p * S.inv_mu0;
      }
    }
  } else {
    system_momentum(d, S, red, sP);
    if (threadIdx.x < 3) {
      sdj[threadIdx.x] = cj * sP[threadIdx.x];
      shp[threadIdx.x] = sP[threadIdx.x] * S.inv_mu0;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ FusedPrep fused_prep(const Dev& d, const SysDev& S, const Tile& t,
                                                int nkick, double jump_frac,
                                                double (*red)[kThreads]) {
  __shared__ double s_P[3], s_dj[3], s_hp[3];
  __shared__ int s_slot;
  const bool head = t.start == S.off;
  if (head && threadIdx.x == 0) s_slot = d.defer ? *(volatile int*)d.hstep : 0;
  fused_momentum(d, S, jump_frac, red, s_P, s_dj, s_hp);   // ends with a block barrier
  FusedPrep f;
  for (int c = 0; c < 3; ++c) {
    f.P[c] = s_P[c];
    f.dj[c] = s_dj[c];
    f.hp[c] = s_hp[c];
  }
  if (!head) return f;
  const int slot = s_slot;
  const int sysi = t.sys;
  if (threadIdx.x == 0) {
    if (sysi == 0) {
      d.kick_ctr[1] = d.kick_ctr[0];
      d.kick_ctr[0] += nkick;
      d.gstep[0] += 1;
    }
    if (d.defer) {
      __threadfence();
      if (atomicAdd(d.arrive, 1) == d.nsys - 1) {
        *d.arrive = 0;
        *d.hstep = slot + 1;
      }
    }
  }
  const bool rec = d.defer && slot < d.hist_cap;
  if (threadIdx.x == 0) {
    for (int c = 0; c < 3; ++c) d.P[3 * sysi + c] = f.P[c];
    if (rec) {
      for (int c = 0; c < 3; ++c)
        d.h_P[(size_t)slot * 6 * d.nsys + 3 * d.nsys + 3 * sysi + c] = f.P[c];
      if (sysi == 0) {
        d.h_nkick[slot] = nkick;
        d.h_ej[slot] = 0;
      }
    }
  }
  if (rec) {
    double dj[3];
    jump_vec(f.P, S, 0.5, dj);
    const int N = d.N;
    for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
      const int g = S.off + i;
      const size_t o = (size_t)slot * 3 * d.NB + S.boff + i;
      d.h_bx[o] = d.xv[g] + dj[0];
      d.h_bx[o + d.NB] = d.xv[(size_t)N + g] + dj[1];
      d.h_bx[o + 2 * (size_t)d.NB] = d.xv[2 * (size_t)N + g] + dj[2];
      d.h_mu[(size_t)slot * d.NB + S.boff + i] = removed(d, g) ? -1.0 : d.bmu[S.boff + i];
      d.h_rc[(size_t)slot * d.NB + S.boff + i] = d.brc[S.boff + i];
    }
  }
  return f;
}

// Jump then kick (nkick half kicks of kick_frac * h each, gravity evaluated once; the
// drag is re-evaluated before each with the updated velocity).  The momentum
// P read here is the one k_prep just computed (FUSED: the one the kernel
// computes itself, for a step's end, jump_frac = 1/2, with nkick = 2); it
// stays valid across the kicks because the K-weighted pair forces are
// antisymmetric and the drag acts on massless bodies only.  Every kick also
// leaves the big bodies' results in d.bk, where the drift reads them.
// Dynamic shared memory: kick_smem_bytes(d, FUSED) (the staging; FUSED with
// more than 32 big bodies also the momentum tree, in the same space, before
// the staging).
// The kernel (k_jump_kick) caps register use at 80 (three resident blocks of
// 256 threads): with the big bodies staged in chunks of at most 256,
// registers set residency, and the extra warps outweigh the few spills
// (measured on the gas disk and the semi-active disk).  `bid` is the tile,
// `dsm` the block's dynamic shared memory (kick_smem_bytes).
template <int NKICK, bool FUSED>
__device__ __forceinline__ void jump_kick_tile(const Dev& d, double jump_frac, double kick_frac,
                                               int bid, double* dsm) {
  BigSmem sb(dsm, big_chunk(d.big_max));
  const Tile t = d.tiles[bid];
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  double dj[3], hp[3];
  if constexpr (FUSED) {
    const FusedPrep f =
        fused_prep(d, S, t, NKICK, jump_frac, reinterpret_cast<double(*)[kThreads]>(dsm));
    for (int c = 0; c < 3; ++c) {
      dj[c] = f.dj[c];
      hp[c] = f.hp[c];
    }
  } else {
    const double* Pv = d.P + 3 * t.sys;
    // the last kernel of a history slot moves on to the next one
    if (d.defer && bid == 0 && threadIdx.x == 0) *d.hstep += 1;
    jump_vec(Pv, S, jump_frac, dj);
    for (int c = 0; c < 3; ++c) hp[c] = Pv[c] * S.inv_mu0;
  }
  const double kick_h = kick_frac * S.h;
  const int j = t.start + threadIdx.x;
  // a deferred planetesimal is kicked by the window's catch-up instead; a
  // removed body is not kicked
  const bool act = threadIdx.x < t.count && !(d.defer && d.lag[j]) && !removed(d, j);
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
  gravity_all(d, S, sb, act, jl, rcj, x, y, z, ax, ay, az, FUSED ? dj : nullptr);
  if (!act) return;
  const bool big = jl < S.nbig;
  if (__double_as_longlong(jump_frac) != 0 && !(FUSED && big)) {   // jump_frac is +0 or 1/2
    d.xv[j] = x;
    d.xv[(size_t)N + j] = y;
    d.xv[2 * (size_t)N + j] = z;
  }
  const bool drag = S.gas_on && !big;
  const double hp0 = hp[0], hp1 = hp[1], hp2 = hp[2];
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
    if (drag) {
      const int kidx = kbase + kk;
      const bool kuse = d.kmode != 0 && kidx < d.kcap;
      const size_t word = (size_t)kidx * d.kwords + (j >> 5);
      int kin = -1, kout = 0;
      if (kuse && d.kmode == 2) kin = (d.kbits[word] >> (j & 31)) & 1u;
      double dvec[3];
      const double coef = gas_drag_coef(S, dc, u, v, w, dvec, kin, &kout);
      if (kuse && d.kmode == 1 && kout) atomicOr(&d.kbits[word], 1u << (j & 31));
      kick_with_drag(kick_h, ax, ay, az, coef, dvec, u, v, w);
    } else {
      u = fma(kick_h, ax, u);
      v = fma(kick_h, ay, v);
      w = fma(kick_h, az, w);
    }
  }
  if (big) {
    double* q = d.bk + S.boff + jl;
    const size_t NB = d.NB;
    q[0] = x;
    q[NB] = y;
    q[2 * NB] = z;
    q[3 * NB] = u;
    q[4 * NB] = v;
    q[5 * NB] = w;
  }
  if (!(FUSED && big)) {
    d.xv[3 * (size_t)N + j] = u;
    d.xv[4 * (size_t)N + j] = v;
    d.xv[5 * (size_t)N + j] = w;
  }
  if (!(finite_d(x) && finite_d(y) && finite_d(z) && finite_d(u) && finite_d(v) && finite_d(w)))
    atomicOr(d.status, ST_NONFINITE);
}

// Dynamic shared memory of a kick: the big bodies' staging, and for a fused
// kick with more than 32 big bodies the momentum tree (in the same space,
// before the staging).
__host__ __device__ __forceinline__ size_t kick_smem_bytes(const Dev& d, bool fused) {
  size_t n = 9 * (size_t)big_chunk(d.big_max);
  if (fused && d.big_max > 32 && n < 3 * (size_t)kThreads) n = 3 * (size_t)kThreads;
  return n * sizeof(double);
}

}  // namespace mx
