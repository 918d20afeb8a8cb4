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

namespace mx {

// Drag acceleration (Eq. 3) of one planetesimal at heliocentric position
// (x, y, z) moving with heliocentric velocity (u, v, w).  Quantities follow
// Sec. 3.1: Sigma (Eq. 1, normalised at 1 AU), rho_g (Eq. 4) at the midplane,
// v_g = v_k sqrt(1 - 2 eta) (Eqs. 5, 6), C_D (Eq. 7) from Re and Ma.
// kd = 3 / (8 r_p[AU] rho_p); rp_cm = r_p in cm.
__device__ __forceinline__ void gas_drag(const SysDev& S, double x, double y, double z, double u,
                                         double v, double w, double rp_cm, double kd, double* a) {
  a[0] = a[1] = a[2] = 0.0;
  const double R2 = fma(x, x, y * y);
  const double iR = rsqrt_d(R2);             // 1/R
  const double R = R2 * iR;
  if (R < S.r_in) return;                    // no gas inside the inner edge (Sec. 3.1.1)
  double sigma, rmh, rcs, reta, inv_cs;      // Sigma, R^-(1+f), R^(f-1/2), R^(2f), 1/c_s
  const double ih = rsqrt_d(R);              // R^-1/2
  if (S.flare_quarter) {
    const double q = rsqrt_d(ih);            // R^1/4
    rcs = q * ih;                            // R^-1/4
    rmh = iR * rcs;                          // R^-5/4
    reta = R * ih;                           // R^1/2
    inv_cs = q * S.inv_c_cs;
  } else {
    const double lr = log(R);
    rcs = exp((S.flare - 0.5) * lr);
    rmh = exp(-(1.0 + S.flare) * lr);
    reta = exp(2.0 * S.flare * lr);
    inv_cs = rcp_d(S.c_cs * rcs);
  }
  if (S.gamma_one) sigma = S.sigma1 * iR;
  else sigma = S.sigma1 * exp(-S.gamma * log(R));
  if (!S.rc_inf) sigma *= exp(-pow(R * S.inv_rc, 2.0 - S.gamma));
  const double rho = S.c_rho * sigma * rmh;
  const double vk = S.sqrt_mu0 * ih;
  const double t = fma(-2.0 * S.c_eta, reta, 1.0);   // 1 - 2 eta
  const double vg = vk * (t * rsqrt_d(t));
  const double g = vg * iR;                  // gas velocity = g * (-y, x, 0)
  const double du = fma(g, y, u);
  const double dv = fma(-g, x, v);
  const double dw = w;
  const double dv2 = fma(du, du, fma(dv, dv, dw * dw));
  if (dv2 == 0.0) return;
  const double dvm = dv2 * rsqrt_d(dv2);
  const double Ma = dvm * inv_cs;
  const double Re = S.c_re * rp_cm * Ma * rho;
  const double k = (Re < 1e5) ? 0.4 : 0.2;
  // Eq. 7 with one reciprocal: [(24/Re + 40/(10+Re))^-1 + 0.23 Ma]^-1 = D/den1
  // where D = 240 + 64 Re and den1 = Re (10 + Re) + 0.23 Ma D.
  const double D = fma(64.0, Re, 240.0);
  const double den1 = fma(0.23 * Ma, D, Re * (10.0 + Re));
  const double A = 1.6 + Ma;
  const double r = rcp_d(den1 * A);
  const double first = D * A * r;           // = D / den1
  const double second = fma(2.0, Ma, 1.6 * k) * den1 * r;
  const double cd = (S.cd_mode == 1) ? fma(first, first, second) : first + second;
  const double coef = S.cd_scale * cd * kd * rho * dvm;
  a[0] = -coef * du;
  a[1] = -coef * dv;
  a[2] = -coef * dw;
}

// K(s)/s^3 times mu for one pair, accumulated into (ax, ay, az) as -f * d
// (Sec. 2.1.3: K = 1 for s^2 >= rc^2, 0 for s^2 <= 0.01 rc^2, quintic between).
__device__ __forceinline__ void pair_acc(double dx, double dy, double dz, double mu, double rc2,
                                         double rc2lo, double rc01, double i09rc, double& ax,
                                         double& ay, double& az) {
  const double s2 = fma(dx, dx, fma(dy, dy, dz * dz));
  const double yy = rsqrt_d(s2);
  double f = yy * yy * yy;
  if (s2 < rc2) {
    if (s2 <= rc2lo) {
      f = 0.0;
    } else {
      const double q = (s2 * yy - rc01) * i09rc;
      f *= q * q * q * fma(q, fma(6.0, q, -15.0), 10.0);
    }
  }
  f *= mu;
  ax = fma(-f, dx, ax);
  ay = fma(-f, dy, ay);
  az = fma(-f, dz, az);
}

// Shared-memory staging of one chunk of big bodies.
struct BigSmem {
  double x[kBigChunk], y[kBigChunk], z[kBigChunk], mu[kBigChunk];
  double rc[kBigChunk], rc2[kBigChunk], rc2lo[kBigChunk], rc01[kBigChunk], i09rc[kBigChunk];
};

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
__global__ void __launch_bounds__(kThreads) k_prep(Dev d, double jump_frac) {
  const SysDev& S = d.sys[blockIdx.x];
  __shared__ double red[3][kThreads];
  const int N = d.N;
  double p[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double m = d.bmu[S.boff + i];
    p[0] = fma(m, d.xv[3 * (size_t)N + g], p[0]);
    p[1] = fma(m, d.xv[4 * (size_t)N + g], p[1]);
    p[2] = fma(m, d.xv[5 * (size_t)N + g], p[2]);
  }
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = p[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  double* P = d.P + 3 * blockIdx.x;
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) P[c] = red[c][0];
  double Ps[3] = {red[0][0], red[1][0], red[2][0]};
  double dj[3];
  jump_vec(Ps, S, jump_frac, dj);
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    d.bx[S.boff + i] = d.xv[g] + dj[0];
    d.by[S.boff + i] = d.xv[(size_t)N + g] + dj[1];
    d.bz[S.boff + i] = d.xv[2 * (size_t)N + g] + dj[2];
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
  const bool act = threadIdx.x < t.count;
  const int j = t.start + threadIdx.x;
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
#pragma unroll
  for (int kk = 0; kk < NKICK; ++kk) {
    double a[3] = {0.0, 0.0, 0.0};
    if (drag) gas_drag(S, x, y, z, u + hp0, v + hp1, w + hp2, rp, kd, a);
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
  const bool act = threadIdx.x < t.count;
  const int j = t.start + threadIdx.x;
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
  if (!act) return;
  const bool drag = S.gas_on && jl >= S.nbig;
  double a[3] = {0.0, 0.0, 0.0};
  if (drag) {
    gas_drag(S, x, y, z, u + P[0] * S.inv_mu0, v + P[1] * S.inv_mu0, w + P[2] * S.inv_mu0,
             d.rp_cm[j], d.kdrag[j], a);
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

void launch_prep(const Dev& d, double jump_frac, cudaStream_t st) {
  k_prep<<<d.nsys, kThreads, 0, st>>>(d, jump_frac);
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

}  // namespace mx
