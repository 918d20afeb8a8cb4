// k_adjoint.cu -- hand-written reverse-mode derivative (vector-Jacobian
// product) of one hybrid step: half kick with K-weighted gravity and gas drag,
// jump, Kepler drift, jump, half kick (arXiv 2601.16791, Sec. 2 and 3.1).
//
// mx_adjoint_step receives the state z0 at the start of a step and the
// cotangent of the state at its end, recomputes the step's intermediate
// states from z0 (a planetesimal that meets a big body is integrated by
// Bulirsch-Stoer from its pre-drift state, k_adj_bs.cu; a big-big encounter
// makes the adjoint refuse), then sweeps back:
//   kick 2 -> jump 2 -> drift or Bulirsch-Stoer -> jump 1 -> kick 1.
// Couplings of all bodies to the few big bodies -- the big sources of the
// gravity Jacobian, the momentum P inside both jumps and inside the drag's
// heliocentric velocity -- are summed per tile in a fixed order and then per
// system in a fixed order, so the result is the same on every run.
//
// Parameter cotangents (per system): d/d sigma1, d/d gamma, d/d cd_scale.
#include "mx_common.cuh"
#include "mx_kepler.cuh"
#include "mx_kernels.h"
#include "mx_physics.cuh"

namespace mx {

// ------------------------------------------------ drag derivative (Eq. 3)
// Reverse mode through the drag of one planetesimal: heliocentric position
// (x, y, z), heliocentric velocity (u, v, w), radius rp_cm, kd = 3/(8 r_p rho_p),
// k branch kb of Eq. 7; la is the cotangent of the acceleration.  Adds the
// cotangents of position (gx), velocity (gv) and of (sigma1, gamma, cd_scale)
// (gp).  The forward quantities are recomputed here in plain form.
__device__ void drag_vjp(const SysDev& S, double x, double y, double u, double v, double w,
                         double rp_cm, double kd, int kb, const double* la, double* gx,
                         double* gv, double* gp) {
  const double R2 = x * x + y * y;
  const double R = sqrt(R2);
  if (!(R >= S.r_in) || R2 == 0.0) return;
  const double lnR = log(R);
  double E = 1.0, dlnE_dR = 0.0, dlnE_dg = 0.0;
  if (!S.rc_inf) {
    const double lr = log(R * S.inv_rc);
    const double p = exp((2.0 - S.gamma) * lr);
    E = exp(-p);
    dlnE_dR = -(2.0 - S.gamma) * p / R;
    dlnE_dg = p * lr;
  }
  const double sigma = S.sigma1 * exp(-S.gamma * lnR) * E;
  const double vk = S.sqrt_mu0 / sqrt(R);
  const double cs = S.c_cs * exp((S.flare - 0.5) * lnR);
  const double rho = S.c_rho * sigma * exp(-(1.0 + S.flare) * lnR);
  const double Rf2 = exp(2.0 * S.flare * lnR);
  const double eta = S.c_eta * Rf2;
  const double t = 1.0 - 2.0 * eta;
  const double st = sqrt(t);
  const double vg = vk * st;
  const double gf = vg / R;
  const double du = u + gf * y, dv = v - gf * x, dw = w;
  const double D2 = du * du + dv * dv + dw * dw;
  if (D2 == 0.0) return;
  const double Dm = sqrt(D2);
  const double Ma = Dm / cs;
  const double Re = S.c_re * rp_cm * Ma * rho;
  const double k = kb ? 0.2 : 0.4;
  const double Dn = 240.0 + 64.0 * Re;
  const double den1 = Re * (10.0 + Re) + 0.23 * Ma * Dn;
  const double first0 = Dn / den1;
  const double first = (S.cd_mode == 1) ? first0 * first0 : first0;
  const double A = 1.6 + Ma;
  const double second = (1.6 * k + 2.0 * Ma) / A;
  const double CD = first + second;
  const double cd = S.cd_scale * CD;
  const double coef = cd * kd * rho * Dm;
  // a = -coef (du, dv, dw)
  double ldu = -coef * la[0], ldv = -coef * la[1], ldw = -coef * la[2];
  const double lcoef = -(la[0] * du + la[1] * dv + la[2] * dw);
  const double lcd = lcoef * kd * rho * Dm;
  double lrho = lcoef * cd * kd * Dm;
  double lDm = lcoef * cd * kd * rho;
  gp[2] += lcd * CD;
  const double lCD = lcd * S.cd_scale;
  // C_D of Eq. 7 through first = D/den1 (squared in the printed form) and second
  const double dfirst0_dRe = (64.0 * den1 - Dn * (10.0 + 2.0 * Re + 0.23 * 64.0 * Ma)) / (den1 * den1);
  const double dfirst0_dMa = -0.23 * Dn * Dn / (den1 * den1);
  const double fscale = (S.cd_mode == 1) ? 2.0 * first0 : 1.0;
  const double dsecond_dMa = (2.0 * A - (1.6 * k + 2.0 * Ma)) / (A * A);
  const double lRe = lCD * fscale * dfirst0_dRe;
  double lMa = lCD * (fscale * dfirst0_dMa + dsecond_dMa);
  // Re = c_re r_p Ma rho
  lMa += lRe * S.c_re * rp_cm * rho;
  lrho += lRe * S.c_re * rp_cm * Ma;
  // Ma = |dv| / c_s
  lDm += lMa / cs;
  const double lcs = -lMa * Dm / (cs * cs);
  const double lD2 = lDm / (2.0 * Dm);
  ldu += 2.0 * du * lD2;
  ldv += 2.0 * dv * lD2;
  ldw += 2.0 * dw * lD2;
  // du = u + gf y, dv = v - gf x, dw = w
  gv[0] += ldu;
  gv[1] += ldv;
  gv[2] += ldw;
  const double lgf = ldu * y - ldv * x;
  double lx = -ldv * gf, ly = ldu * gf;
  // gf = v_g / R, v_g = v_k sqrt(1 - 2 eta)
  const double lvg = lgf / R;
  double lR = -lgf * vg / R2;
  const double lvk = lvg * st;
  const double lt = lvg * vk / (2.0 * st);
  const double leta = -2.0 * lt;
  // eta = c_eta(gamma) R^(2 flare)
  lR += leta * eta * 2.0 * S.flare / R;
  gp[1] += leta * S.deta_dgamma * Rf2;
  // rho = c_rho Sigma R^-(1+flare)
  const double lsigma = lrho * rho / sigma;
  lR -= lrho * rho * (1.0 + S.flare) / R;
  // c_s = c_cs R^(flare - 1/2), v_k = sqrt(mu0) R^(-1/2)
  lR += lcs * cs * (S.flare - 0.5) / R;
  lR -= lvk * vk * 0.5 / R;
  // Sigma = sigma1 R^-gamma E(R, gamma)
  gp[0] += lsigma * sigma / S.sigma1;
  lR += lsigma * sigma * (-S.gamma / R + dlnE_dR);
  gp[1] += lsigma * sigma * (-lnR + dlnE_dg);
  // R = sqrt(x^2 + y^2)
  lx += lR * x / R;
  ly += lR * y / R;
  gx[0] += lx;
  gx[1] += ly;
}

// Reverse of the disk's gravity on a planetesimal (Eqs. 10-12), in the form
// the kick applies it: a = g(R) (x, y, 0), g = c_dg Sigma(R) R^-m, m = 2 for
// the gamma = 1 edge form (F = 2 pi G Sigma r_in / R) and m = 1 otherwise
// (F = 2 pi G Sigma S(gamma)), Sigma = sigma1 R^-gamma E(R, gamma), and no
// force inside r_in.  la is the cotangent of the acceleration.  Adds
// la . da/d(x, y) to gx and la . da/d(sigma1, gamma) to gp[0], gp[1]:
//   da/dx = g e_x + (x, y) g'(R) x / R,  g'/g = dln Sigma/dR - m/R,
//   dln g/dgamma = -ln R + dln E/dgamma + dln S/dgamma (0 for the edge form).
__device__ void disk_gravity_vjp(const SysDev& S, double x, double y, const double* la, double* gx,
                                 double* gp) {
  const double R2 = x * x + y * y;
  const double R = sqrt(R2);
  if (!(R >= S.r_in) || R2 == 0.0) return;
  const double lnR = log(R);
  double E = 1.0, dlnE_dR = 0.0, dlnE_dg = 0.0;
  if (!S.rc_inf) {
    const double lr = log(R * S.inv_rc);
    const double p = exp((2.0 - S.gamma) * lr);
    E = exp(-p);
    dlnE_dR = -(2.0 - S.gamma) * p / R;
    dlnE_dg = p * lr;
  }
  const double m = S.dg_edge ? 2.0 : 1.0;
  const double g = S.c_dg * S.sigma1 * exp(-(S.gamma + m) * lnR) * E;
  const double lr = la[0] * x + la[1] * y;
  const double c = lr * g * (-S.gamma / R + dlnE_dR - m / R) / R;
  gx[0] += g * la[0] + c * x;
  gx[1] += g * la[1] + c * y;
  gp[0] += lr * g / S.sigma1;
  gp[1] += lr * g * (-lnR + dlnE_dg + S.dlnS_dgamma);
}

// ------------------------------------------------ Kepler-drift derivative
// G4, G5 at (s, beta): series for |beta s^2| <= 0.3, else from
// G_{k+2} = (s^k/k! - G_k)/beta.
__device__ __forceinline__ void g45(double s, double beta, const double* G, double& G4,
                                    double& G5) {
  const double s2 = s * s;
  const double z = beta * s2;
  if (fabs(z) <= 0.3) {
    double c4 = 1.0 / 6402373705728000.0;     // 1/18!
    double c5 = 1.0 / 121645100408832000.0;   // 1/19!
    const double f4[8] = {1.0 / 24.0, 1.0 / 720.0, 1.0 / 40320.0, 1.0 / 3628800.0,
                          1.0 / 479001600.0, 1.0 / 87178291200.0, 1.0 / 20922789888000.0,
                          1.0 / 6402373705728000.0};
    const double f5[8] = {1.0 / 120.0, 1.0 / 5040.0, 1.0 / 362880.0, 1.0 / 39916800.0,
                          1.0 / 6227020800.0, 1.0 / 1307674368000.0, 1.0 / 355687428096000.0,
                          1.0 / 121645100408832000.0};
    c4 = f4[7];
    c5 = f5[7];
    for (int m = 6; m >= 0; --m) {
      c4 = fma(-z, c4, f4[m]);
      c5 = fma(-z, c5, f5[m]);
    }
    G4 = s2 * s2 * c4;
    G5 = s2 * s2 * s * c5;
  } else {
    G4 = (0.5 * s2 - G[2]) / beta;
    G5 = (s2 * s / 6.0 - G[3]) / beta;
  }
}

// Cotangent of the pre-drift state (x, v) from that of the post-drift state.
// The universal anomaly s solves F(s) = r0 s + eta G2 + zeta G3 - h = 0
// (implicit function: ds = -(F_r0 dr0 + F_eta deta + F_zeta dzeta +
// F_beta dbeta)/F_s with F_s = r), and dG_k/ds = G_{k-1},
// dG_k/dbeta = -(s G_{k+1} - k G_{k+2})/2.
__device__ bool kepler_vjp(double mu, double h, int maxit, const double* x, const double* v,
                           const double* lx1, const double* lv1, double* lx0, double* lv0) {
  for (int c = 0; c < 3; ++c) {
    lx0[c] = lx1[c];
    lv0[c] = lv1[c];
  }
  if (h == 0.0) return true;
  const double r02 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  const double r0 = sqrt(r02);
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const double eta = x[0] * v[0] + x[1] * v[1] + x[2] * v[2];
  const double beta = 2.0 * mu / r0 - v2;
  const double zeta = mu - beta * r0;
  double s = (h / r0) * (1.0 - 0.5 * eta * h / r02);
  double G[4];
  bool done = false;
  for (int it = 0; it < maxit; ++it) {
    gfuns(s, beta, G);
    const double F = r0 * s + eta * G[2] + zeta * G[3] - h;
    const double Fp = r0 + eta * G[1] + zeta * G[2];
    const double Fpp = eta * G[0] + zeta * G[1];
    const double ds = -F * Fp / (Fp * Fp - 0.5 * F * Fpp);
    s += ds;
    if (fabs(ds) <= 1e-7 * fabs(s)) {
      done = true;
      break;
    }
  }
  if (!done) return false;
  gfuns(s, beta, G);
  double G4, G5;
  g45(s, beta, G, G4, G5);
  const double r = r0 + eta * G[1] + zeta * G[2];
  const double f = 1.0 - mu * G[2] / r0;
  const double g = r0 * G[1] + eta * G[2];
  const double fd = -mu * G[1] / (r * r0);
  const double gd = 1.0 - mu * G[2] / r;
  double lf = 0, lg = 0, lfd = 0, lgd = 0;
  for (int c = 0; c < 3; ++c) {
    lf += lx1[c] * x[c];
    lg += lx1[c] * v[c];
    lfd += lv1[c] * x[c];
    lgd += lv1[c] * v[c];
    lx0[c] = f * lx1[c] + fd * lv1[c];
    lv0[c] = g * lx1[c] + gd * lv1[c];
  }
  double lG1 = 0, lG2 = 0, lr0 = 0, leta = 0, lr = 0, lzeta = 0, lbeta = 0;
  lG2 -= mu * lf / r0;
  lr0 += mu * G[2] * lf / r02;
  lr0 += G[1] * lg;
  lG1 += r0 * lg;
  leta += G[2] * lg;
  lG2 += eta * lg;
  lG1 -= mu * lfd / (r * r0);
  lr += mu * G[1] * lfd / (r * r * r0);
  lr0 += mu * G[1] * lfd / (r * r02);
  lG2 -= mu * lgd / r;
  lr += mu * G[2] * lgd / (r * r);
  lr0 += lr;
  leta += G[1] * lr;
  lG1 += eta * lr;
  lzeta += G[2] * lr;
  lG2 += zeta * lr;
  const double dG1b = -0.5 * (s * G[2] - G[3]);
  const double dG2b = -0.5 * (s * G[3] - 2.0 * G4);
  const double dG3b = -0.5 * (s * G4 - 3.0 * G5);
  const double ls = lG1 * G[0] + lG2 * G[1];
  lbeta += lG1 * dG1b + lG2 * dG2b;
  const double Fb = eta * dG2b + zeta * dG3b;
  lr0 -= ls * s / r;
  leta -= ls * G[2] / r;
  lzeta -= ls * G[3] / r;
  lbeta -= ls * Fb / r;
  lbeta -= r0 * lzeta;
  lr0 -= beta * lzeta;
  lr0 -= 2.0 * mu * lbeta / r02;
  const double lv2 = -lbeta;
  for (int c = 0; c < 3; ++c) {
    lx0[c] += leta * v[c] + lr0 * x[c] / r0;
    lv0[c] += leta * x[c] + 2.0 * lv2 * v[c];
  }
  return true;
}

// ------------------------------------------------------------- kernels

// Momentum sum mu_i v_i of each system's bigs from velocity rows vx, vy, vz
// (stride N); one block per system, fixed tree.
__global__ void __launch_bounds__(kThreads) k_adj_momentum(Dev d, const double* vx,
                                                           const double* vy, const double* vz,
                                                           double* P, int slot) {
  const SysDev& S = d.sys[blockIdx.x];
  __shared__ double red[3][kThreads];
  double p[3] = {0, 0, 0};
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double m = d.bmu[S.boff + i];
    p[0] = fma(m, vx[g], p[0]);
    p[1] = fma(m, vy[g], p[1]);
    p[2] = fma(m, vz[g], p[2]);
  }
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = p[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) P[9 * blockIdx.x + 3 * slot + c] = red[c][0];
}

__device__ __forceinline__ int kick_branch(const Dev& d, int kick, int j) {
  if (d.kmode != 2 || kick < 0 || kick >= d.kcap) return -1;
  return (d.kbits[(size_t)kick * d.kwords + (j >> 5)] >> (j & 31)) & 1u;
}

// Big bodies staged in shared memory per pass of the adjoint's kicks.
constexpr int kAdjChunk = 128;

// The changeover constants of a pair (rc^2, 0.01 rc^2, 0.1 rc, 1/(0.9 rc)
// with rc = max(rc_i, rc_j), Sec. 2.1.3): the big body's, or the target's
// own when the target is a big body with the larger radius.  They grow with
// rc, so comparing rc^2 picks the larger radius.
struct PairRc {
  double rc2, lo, r01, i09;
};
__device__ __forceinline__ PairRc pair_rc(const double (*sc)[kAdjChunk], int k, const PairRc& own) {
  PairRc c{sc[0][k], sc[1][k], sc[2][k], sc[3][k]};
  // compared on the bit patterns (non-negative doubles), off the FP64 pipe
  if (__double_as_longlong(own.rc2) > __double_as_longlong(c.rc2)) c = own;
  return c;
}

// A target's own changeover constants (zero for a planetesimal).
__device__ __forceinline__ PairRc target_rc(const Dev& d, const SysDev& S, int jl) {
  PairRc c{0.0, 0.0, 0.0, 0.0};
  if (jl < S.nbig) {
    const size_t b = S.boff + jl;
    c = PairRc{d.brc4[b], d.brc4[(size_t)d.NB + b], d.brc4[2 * (size_t)d.NB + b],
               d.brc4[3 * (size_t)d.NB + b]};
  }
  return c;
}

// Positions, masses and changeover constants of a chunk of big bodies.
__device__ __forceinline__ void stage_chunk(const Dev& d, const SysDev& S, const double* X, int c0,
                                            int cn, double* sx, double* sy, double* sz, double* sm,
                                            double (*sc)[kAdjChunk]) {
  const int N = d.N;
  for (int k = threadIdx.x; k < cn; k += blockDim.x) {
    const int g = S.off + c0 + k;
    const size_t b = S.boff + c0 + k;
    sx[k] = X[g]; sy[k] = X[(size_t)N + g]; sz[k] = X[2 * (size_t)N + g];
    sm[k] = d.bmu[b];
    for (int q = 0; q < 4; ++q) sc[q][k] = d.brc4[(size_t)q * d.NB + b];
  }
}

// Kick 1 forward: v1 = v0 + (h/2)(a_grav(x0) + a_drag(x0, v0 + P0/m0)).
__global__ void __launch_bounds__(kThreads) k_adj_kick1_fwd(Dev d, Adj a) {
  __shared__ double sx[kAdjChunk], sy[kAdjChunk], sz[kAdjChunk], sm[kAdjChunk];
  __shared__ double sc[4][kAdjChunk];
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  const bool act = threadIdx.x < t.count;
  const int j = t.start + threadIdx.x;
  const int jl = j - S.off;
  const double* P0 = a.P + 9 * t.sys;
  double x = 0, y = 0, z = 0, u = 0, v = 0, w = 0;
  if (act) {
    x = a.z0[j]; y = a.z0[(size_t)N + j]; z = a.z0[2 * (size_t)N + j];
    u = a.z0[3 * (size_t)N + j]; v = a.z0[4 * (size_t)N + j]; w = a.z0[5 * (size_t)N + j];
  }
  const PairRc trc = target_rc(d, S, act ? jl : S.nbig);
  double ax = 0, ay = 0, az = 0;
  for (int c0 = 0; c0 < S.nbig; c0 += kAdjChunk) {
    const int cn = min(kAdjChunk, S.nbig - c0);
    __syncthreads();
    stage_chunk(d, S, a.z0, c0, cn, sx, sy, sz, sm, sc);
    __syncthreads();
    if (!act) continue;
    for (int k = 0; k < cn; ++k) {
      if (c0 + k == jl) continue;
      const PairRc c = pair_rc(sc, k, trc);
      pair_acc(x - sx[k], y - sy[k], z - sz[k], sm[k], c.rc2, c.lo, c.r01, c.i09, ax, ay, az);
    }
  }
  if (!act) return;
  double ad[3] = {0, 0, 0};
  if (S.gas_on && jl >= S.nbig) {
    int kout = 0;
    gas_drag(S, x, y, z, u + P0[0] * S.inv_mu0, v + P0[1] * S.inv_mu0, w + P0[2] * S.inv_mu0,
             d.rp_cm[j], d.kdrag[j], ad, kick_branch(d, 2 * a.step, j), &kout);
  }
  const double th = 0.5 * S.h;
  a.v1[j] = fma(th, ax + ad[0], u);
  a.v1[(size_t)N + j] = fma(th, ay + ad[1], v);
  a.v1[2 * (size_t)N + j] = fma(th, az + ad[2], w);
}

// Jump 1 and drift forward: x2 = x0 + (h/2) P1/m0, (x3, v3) = drift(x2, v1);
// with stage 3 the drift alone, from the (x2, v1) the forward step left
// (a.pd, read only); with stage 2, jump 2: x4 = x3 + (h/2) P3/m0.
__global__ void __launch_bounds__(kThreads) k_adj_move_fwd(Dev d, Adj a, int stage) {
  const Tile t = d.tiles[blockIdx.x];
  if (threadIdx.x >= t.count) return;
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  const int j = t.start + threadIdx.x;
  const double c = 0.5 * S.h * S.inv_mu0;
  if (stage != 2) {
    double x, y, z;
    if (stage == 1) {
      const double* P1 = a.P + 9 * t.sys + 3;
      x = a.z0[j] + c * P1[0];
      y = a.z0[(size_t)N + j] + c * P1[1];
      z = a.z0[2 * (size_t)N + j] + c * P1[2];
      a.x2[j] = x; a.x2[(size_t)N + j] = y; a.x2[2 * (size_t)N + j] = z;
    } else {   // stage 3: the forward's own pre-drift state (a.pd)
      x = a.x2[j]; y = a.x2[(size_t)N + j]; z = a.x2[2 * (size_t)N + j];
    }
    double u = a.v1[j], v = a.v1[(size_t)N + j], w = a.v1[2 * (size_t)N + j];
    if (!kepler_drift(S.mu0, S.h, d.kepler_max_iter, x, y, z, u, v, w)) atomicOr(d.status, ST_KEPLER);
    a.xv3[j] = x; a.xv3[(size_t)N + j] = y; a.xv3[2 * (size_t)N + j] = z;
    a.xv3[3 * (size_t)N + j] = u; a.xv3[4 * (size_t)N + j] = v; a.xv3[5 * (size_t)N + j] = w;
  } else {
    const double* P3 = a.P + 9 * t.sys + 6;
    for (int q = 0; q < 3; ++q) a.x4[(size_t)q * N + j] = a.xv3[(size_t)q * N + j] + c * P3[q];
  }
}

// One pair's part of a half kick's reverse.  With J the Jacobian of the
// pair's acceleration -mu K(s) d/s^3 and l the cotangent of the acceleration,
// mu J l = -(A l + B d), A = mu K/s^3, B = mu (K' s - 3K)/s^5 (d.l); the big
// body's position gets A l + B d, added to (bx, by, bz), and the target's
// gets -(A l + B d), kept as the sums sa += A and sb += B d (the target adds
// -(sa l + sb) once).  nl = -3 l, so that outside the changeover shell (K = 1,
// K' = 0) B = mu/s^5 (d.nl).  1/s from the single-precision estimate with one
// correction, as in the forward's pair weight; nothing inside 0.1 rc (K = 0).
__device__ __forceinline__ void pair_vjp(double dx, double dy, double dz, double mu,
                                         const PairRc& c, double lax, double lay, double laz,
                                         double nlx, double nly, double nlz, double& bx,
                                         double& by, double& bz, double& sa, double& sbx,
                                         double& sby, double& sbz) {
  const double s2 = fma(dx, dx, fma(dy, dy, dz * dz));
  if (__double_as_longlong(s2) <= __double_as_longlong(c.lo)) return;
  const double y = float_to_double_bits(rsqrtf(abs_to_float_bits(s2)));
  const double e = fma(-s2 * y, y, 1.0);
  const double is = fma(y * e, fma(0.375, e, 0.5), y);   // 1/s
  const double is2 = is * is;
  const double mis3 = mu * (is2 * is);
  const double dl3 = fma(dx, nlx, fma(dy, nly, dz * nlz));   // -3 d.l
  double A = mis3, T = dl3;   // T = (K' s - 3K) d.l
  if (__double_as_longlong(s2) < __double_as_longlong(c.rc2)) {
    const double sv = s2 * is;
    const double q = (sv - c.r01) * c.i09;
    const double omq = 1.0 - q;
    const double K = q * q * q * fma(q, fma(6.0, q, -15.0), 10.0);
    const double Kp = 30.0 * q * q * omq * omq * c.i09;   // dK/ds
    A = mis3 * K;
    T = dl3 * fma(Kp * sv, -1.0 / 3.0, K);
  }
  const double B = (mis3 * is2) * T;
  bx = fma(A, lax, fma(B, dx, bx));
  by = fma(A, lay, fma(B, dy, by));
  bz = fma(A, laz, fma(B, dz, bz));
  sa += A;
  sbx = fma(B, dx, sbx);
  sby = fma(B, dy, sby);
  sbz = fma(B, dz, sbz);
}

// Which parts of a half kick's reverse a launch takes.  The gravity's part is
// linear in the cotangent l of the acceleration and depends on the positions
// only, so the reverse of a step's first half kick and of the previous step's
// last one (the same positions) can share one pass over the pairs: the first
// launch takes the drag and leaves its l in lout, the second adds it (lin) to
// its own before the pair pass.
//   grav: the pass over the (target, big body) pairs;
//   drag: the drag's reverse (and the disk's gravity);
//   own: l = (h/2) lam_v of this kick (0: none, a pass with lin alone);
//   lin: 3 x N, added to l for the pair pass (or null);
//   lout: 3 x N, receives this kick's own l (or null).
struct KickRev {
  int grav, drag, own;
  const double* lin;
  double* lout;
};

// Reverse of a half kick at positions X (3 x N), velocities V (3 x N) and
// momentum Pk, with the cotangent in a.lam: lam_x += (h/2) J^T lam_v,
// lam_v += (h/2) (d a_drag/d v)^T lam_v.  Per-tile partials: the cotangent
// each big body's position receives from all targets, the drag's share of
// the momentum cotangent, the sum of the targets' own position cotangents
// (for the jump before this kick), and the parameter cotangents.
//
// A warp's sums for the big bodies go round its lanes: the chunk's bodies
// are taken W at a time (W the largest power of two <= those left, at most
// 32); in round r, lane l of each W-lane group takes body (l + r) mod W of
// the batch and then passes its running sum for that body to the lane before
// it, so each body's sum visits the group's targets in a fixed order with
// one shuffle a pair, and the groups' sums are added at the end.
__global__ void __launch_bounds__(kThreads) k_adj_kick_vjp(Dev d, Adj a, const double* X,
                                                           const double* V, int pslot, int kick,
                                                           KickRev r) {
  __shared__ double sx[kAdjChunk], sy[kAdjChunk], sz[kAdjChunk], sm[kAdjChunk];
  __shared__ double sc[4][kAdjChunk];
  __shared__ double wpart[kThreads / 32][kAdjChunk][3];
  __shared__ double wsum[kThreads / 32][9];
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  const bool act = threadIdx.x < t.count;
  const int j = t.start + threadIdx.x;
  const int jl = j - S.off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  const double* Pk = a.P + 9 * t.sys + 3 * pslot;
  const double th = 0.5 * S.h;
  double* rec = a.part + a.poff[blockIdx.x];
  double x = 0, y = 0, z = 0, lvx = 0, lvy = 0, lvz = 0;
  if (act) {
    x = X[j]; y = X[(size_t)N + j]; z = X[2 * (size_t)N + j];
    lvx = a.lam[3 * (size_t)N + j]; lvy = a.lam[4 * (size_t)N + j]; lvz = a.lam[5 * (size_t)N + j];
  }
  const PairRc trc = target_rc(d, S, act ? jl : S.nbig);
  // the cotangent of this kick's acceleration (the drag's too), and the
  // gravity's: that plus the one a merged reverse carries in (r.lin)
  const double lax = r.own ? th * lvx : 0.0, lay = r.own ? th * lvy : 0.0,
               laz = r.own ? th * lvz : 0.0;
  double gax = lax, gay = lay, gaz = laz;
  if (act && r.lin) {
    gax += r.lin[j];
    gay += r.lin[(size_t)N + j];
    gaz += r.lin[2 * (size_t)N + j];
  }
  if (act && r.lout) {
    r.lout[j] = lax;
    r.lout[(size_t)N + j] = lay;
    r.lout[2 * (size_t)N + j] = laz;
  }
  const double nlx = -3.0 * gax, nly = -3.0 * gay, nlz = -3.0 * gaz;
  double sa = 0, sbx = 0, sby = 0, sbz = 0;   // the target's sums (pair_vjp)
  for (int c0 = 0; r.grav && c0 < S.nbig; c0 += kAdjChunk) {
    const int cn = min(kAdjChunk, S.nbig - c0);
    __syncthreads();
    stage_chunk(d, S, X, c0, cn, sx, sy, sz, sm, sc);
    __syncthreads();
    for (int base = 0; base < cn;) {
      const int left = cn - base;
      const int W = left >= 32 ? 32 : 1 << (31 - __clz(left));
      const int gl = lane & (W - 1);
      double bx = 0, by = 0, bz = 0;   // the running sum of the body this lane holds
      for (int r = 0; r < W; ++r) {
        const int k = base + ((gl + r) & (W - 1));
        if (act && c0 + k != jl)
          pair_vjp(x - sx[k], y - sy[k], z - sz[k], sm[k], pair_rc(sc, k, trc), gax, gay, gaz,
                   nlx, nly, nlz, bx, by, bz, sa, sbx, sby, sbz);
        if (r + 1 < W) {
          const int src = (gl + 1) & (W - 1);
          bx = __shfl_sync(0xffffffffu, bx, src, W);
          by = __shfl_sync(0xffffffffu, by, src, W);
          bz = __shfl_sync(0xffffffffu, bz, src, W);
        }
      }
      for (int off = W; off < 32; off <<= 1) {
        bx += __shfl_down_sync(0xffffffffu, bx, off);
        by += __shfl_down_sync(0xffffffffu, by, off);
        bz += __shfl_down_sync(0xffffffffu, bz, off);
      }
      if (lane < W) {
        const int k = base + ((gl + W - 1) & (W - 1));
        wpart[warp][k][0] = bx;
        wpart[warp][k][1] = by;
        wpart[warp][k][2] = bz;
      }
      base += W;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < cn; k += blockDim.x) {
      double s0 = 0, s1 = 0, s2 = 0;
      for (int q = 0; q < nwarps; ++q) {
        s0 += wpart[q][k][0];
        s1 += wpart[q][k][1];
        s2 += wpart[q][k][2];
      }
      rec[3 * (c0 + k) + 0] = s0;
      rec[3 * (c0 + k) + 1] = s1;
      rec[3 * (c0 + k) + 2] = s2;
    }
  }
  // into lam_x of this target
  double gx = -fma(sa, gax, sbx), gy = -fma(sa, gay, sby), gz = -fma(sa, gaz, sbz);
  // drag
  double own[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // dP (3), sum lam_x (3), dparams (3)
  if (act) {
    double lvxn = lvx, lvyn = lvy, lvzn = lvz;
    if (r.drag && S.gas_on && jl >= S.nbig) {
      const double u = V[j] + Pk[0] * S.inv_mu0, v = V[(size_t)N + j] + Pk[1] * S.inv_mu0,
                   w = V[2 * (size_t)N + j] + Pk[2] * S.inv_mu0;
      const double la[3] = {lax, lay, laz};
      double dx3[3] = {0, 0, 0}, dv3[3] = {0, 0, 0};
      int kb = kick_branch(d, kick, j);
      if (kb < 0) {
        double ad[3];
        gas_drag(S, x, y, z, u, v, w, d.rp_cm[j], d.kdrag[j], ad, -1, &kb);
      }
      drag_vjp(S, x, y, u, v, w, d.rp_cm[j], d.kdrag[j], kb, la, dx3, dv3, own + 6);
      if (S.dg_on) disk_gravity_vjp(S, x, y, la, dx3, own + 6);
      gx += dx3[0];
      gy += dx3[1];
      gz += dx3[2];
      lvxn += dv3[0];
      lvyn += dv3[1];
      lvzn += dv3[2];
      for (int c = 0; c < 3; ++c) own[c] = dv3[c] * S.inv_mu0;
    }
    const double lx = a.lam[j] + gx, ly = a.lam[(size_t)N + j] + gy, lz = a.lam[2 * (size_t)N + j] + gz;
    a.lam[j] = lx;
    a.lam[(size_t)N + j] = ly;
    a.lam[2 * (size_t)N + j] = lz;
    a.lam[3 * (size_t)N + j] = lvxn;
    a.lam[4 * (size_t)N + j] = lvyn;
    a.lam[5 * (size_t)N + j] = lvzn;
    own[3] = lx;
    own[4] = ly;
    own[5] = lz;
  }
  for (int q = 0; q < 9; ++q) {
    double vq = own[q];
    for (int off = 16; off > 0; off >>= 1) vq += __shfl_down_sync(0xffffffffu, vq, off);
    if (lane == 0) wsum[warp][q] = vq;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double sum = 0;
    for (int q = 0; q < nwarps; ++q) sum += wsum[q][threadIdx.x];
    rec[3 * S.nbig + threadIdx.x] = sum;
  }
}

// Sums over a system's tiles of values v < V of their partial records (the
// system's tiles are consecutive, so record k sits at p0 + k R), into out[v]
// (shared memory), on a block of kThreads threads.  Each value's tiles are
// split into P interleaved strands (strand s adds tiles s, s + P, ... in
// order; P the largest power of two <= 32 with P V <= kThreads), and the
// strands are added by a fixed butterfly, so the chain of dependent adds is
// T / P long and the order depends on nothing but V.  Every thread calls it.
__device__ void fold_tiles(const double* p0, int R, int T, int V, double* out) {
  int P = 1;
  while (2 * P <= 32 && 2 * P * V <= kThreads) P *= 2;
  const int v = threadIdx.x / P, s = threadIdx.x & (P - 1);
  double acc = 0.0;
  if (v < V) {
#pragma unroll 4
    for (int k = s; k < T; k += P) acc += p0[(size_t)k * R + v];
  }
  for (int o = P >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (v < V && s == 0) out[v] = acc;
  __syncthreads();
}

// Systems with more than (kThreads - 9) / 3 big bodies: block (sys, y) folds
// the tile partials of the big bodies' position cotangents 3 per body, values
// y kThreads .. (y + 1) kThreads - 1 of the system, one thread a value over
// four interleaved strands of tiles added in a fixed order; adds them to
// lam_x and keeps them for k_adj_fold_kick.
__global__ void __launch_bounds__(kThreads) k_adj_fold_big(Dev d, Adj a) {
  const int sys = blockIdx.x;
  const SysDev& S = d.sys[sys];
  const int nb = S.nbig, R = 3 * nb + 9;
  if (R <= kThreads) return;
  const int v = blockIdx.y * kThreads + threadIdx.x;
  if (v >= 3 * nb) return;
  const int t0 = a.sys_tiles[sys], T = a.sys_tiles[sys + 1] - t0;
  const double* p0 = a.part + (T > 0 ? a.poff[t0] : 0) + v;
  double acc[4] = {0, 0, 0, 0};
  int k = 0;
  for (; k + 4 <= T; k += 4)
    for (int q = 0; q < 4; ++q) acc[q] += p0[(size_t)(k + q) * R];
  for (int q = 0; k < T; ++k, ++q) acc[q] += p0[(size_t)k * R];
  const double f = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  const int i = v / 3, c = v - 3 * i;
  a.lam[(size_t)c * d.N + S.off + i] += f;
  a.bfold[3 * (size_t)S.boff + v] = f;
}

// Per system: fold the tile partials of a kick's reverse (fixed order).
//  kick 2: lam_x(big) += G; lam_P3 = dP_drag + (h/2)/m0 (sum_j lam_x4_j);
//          lam_v(big) += mu lam_P3.
//  kick 1: lam_x(big) += G; lam_v(big) += mu dP_drag.
__global__ void __launch_bounds__(kThreads) k_adj_fold_kick(Dev d, Adj a, int which, int grav) {
  const int sys = blockIdx.x;
  const SysDev& S = d.sys[sys];
  const int N = d.N;
  const int t0 = a.sys_tiles[sys], T = a.sys_tiles[sys + 1] - t0;
  const int nb = S.nbig, R = 3 * nb + 9;
  const double* p0 = a.part + (T > 0 ? a.poff[t0] : 0);
  __shared__ double tot[9];
  __shared__ double gsum_sh[3];
  __shared__ double fold[kThreads];
  if (R <= kThreads) {
    fold_tiles(p0, R, T, R, fold);
    // (without the pair pass, the records' big-body values are not this
    // launch's and are left out)
    for (int i = threadIdx.x; grav && i < nb; i += blockDim.x) {
      const int g = S.off + i;
      for (int c = 0; c < 3; ++c) a.lam[(size_t)c * N + g] += fold[3 * i + c];
    }
    if (threadIdx.x < 3) {   // the bigs' extra position cotangent, summed in big order
      double sum = 0.0;
      for (int i = 0; grav && i < nb; ++i) sum += fold[3 * i + threadIdx.x];
      gsum_sh[threadIdx.x] = sum;
    }
    if (threadIdx.x < 9) tot[threadIdx.x] = fold[3 * nb + threadIdx.x];
  } else {
    // many big bodies: k_adj_fold_big has added their cotangents and left
    // them in a.bfold; their sum in big order for sum_j lam_x4_j
    double gs[3] = {0, 0, 0};
    for (int i = threadIdx.x; grav && i < nb; i += blockDim.x)
      for (int c = 0; c < 3; ++c) gs[c] += a.bfold[3 * ((size_t)S.boff + i) + c];
    fold_tiles(p0 + 3 * nb, R, T, 9, tot);
    __shared__ double red[3][kThreads];
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = gs[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w)
        for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x < 3) gsum_sh[threadIdx.x] = red[threadIdx.x][0];
  }
  __syncthreads();
  double lP[3];
  for (int c = 0; c < 3; ++c) {
    lP[c] = tot[c];
    if (which == 2) lP[c] += 0.5 * S.h * S.inv_mu0 * (tot[3 + c] + gsum_sh[c]);
  }
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const int g = S.off + i;
    const double m = d.bmu[S.boff + i];
    for (int c = 0; c < 3; ++c) a.lam[(size_t)(3 + c) * N + g] += m * lP[c];
  }
  if (a.dpar && threadIdx.x < 3) a.dpar[3 * sys + threadIdx.x] += tot[6 + threadIdx.x];
}

// Reverse of the drift: (lam_x2, lam_v1) = J^T (lam_x3, lam_v3) per body,
// with the tile's sum of lam_x2 for jump 1.
__global__ void __launch_bounds__(kThreads) k_adj_drift_vjp(Dev d, Adj a) {
  __shared__ double wsum[kThreads / 32][3];
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  const bool act = threadIdx.x < t.count;
  const int j = t.start + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  double own[3] = {0, 0, 0};
  // a body an encounter group writes back (marked 2 by k_adj_tape) already
  // holds its cotangent at the pre-drift state (k_adj_bs_vjp); it only enters
  // the jump's sum
  const bool in_group = a.groups && act && d.flags[j] == 2;
  if (in_group)
    for (int c = 0; c < 3; ++c) own[c] = a.lam[(size_t)c * N + j];
  if (act && !in_group) {
    const double x[3] = {a.x2[j], a.x2[(size_t)N + j], a.x2[2 * (size_t)N + j]};
    const double v[3] = {a.v1[j], a.v1[(size_t)N + j], a.v1[2 * (size_t)N + j]};
    double l1[3], m1[3], l0[3], m0[3];
    for (int c = 0; c < 3; ++c) {
      l1[c] = a.lam[(size_t)c * N + j];
      m1[c] = a.lam[(size_t)(3 + c) * N + j];
    }
    if (!kepler_vjp(S.mu0, S.h, d.kepler_max_iter, x, v, l1, m1, l0, m0))
      atomicOr(d.status, ST_KEPLER);
    for (int c = 0; c < 3; ++c) {
      a.lam[(size_t)c * N + j] = l0[c];
      a.lam[(size_t)(3 + c) * N + j] = m0[c];
      own[c] = l0[c];
    }
  }
  for (int q = 0; q < 3; ++q) {
    double vq = own[q];
    for (int off = 16; off > 0; off >>= 1) vq += __shfl_down_sync(0xffffffffu, vq, off);
    if (lane == 0) wsum[warp][q] = vq;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double sum = 0;
    for (int q = 0; q < nwarps; ++q) sum += wsum[q][threadIdx.x];
    a.part[a.poff[blockIdx.x] + threadIdx.x] = sum;
  }
}

// Per system: jump 1 -> lam_P1 = (h/2)/m0 sum_j lam_x2_j; lam_v1(big) += mu lam_P1.
__global__ void __launch_bounds__(kThreads) k_adj_fold_jump1(Dev d, Adj a) {
  const int sys = blockIdx.x;
  const SysDev& S = d.sys[sys];
  const int N = d.N;
  __shared__ double lP[3];
  const int t0 = a.sys_tiles[sys], T = a.sys_tiles[sys + 1] - t0;
  fold_tiles(a.part + (T > 0 ? a.poff[t0] : 0), 3 * S.nbig + 9, T, 3, lP);
  if (threadIdx.x < 3) {
    double sum = lP[threadIdx.x];
    if (a.groups) sum += a.bs_xsum[3 * sys + threadIdx.x];   // the big bodies' BS shares
    lP[threadIdx.x] = 0.5 * S.h * S.inv_mu0 * sum;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double m = d.bmu[S.boff + i];
    for (int c = 0; c < 3; ++c) a.lam[(size_t)(3 + c) * N + g] += m * lP[c];
  }
}

int adjoint_vjp_blocks_per_sm(int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_adj_kick_vjp, threads, 0) != cudaSuccess)
    return 0;
  return n;
}

void launch_fold_kick(const Dev& d, const Adj& a, int which, int grav, cudaStream_t st) {
  if (grav && 3 * d.big_max + 9 > kThreads)
    k_adj_fold_big<<<dim3(d.nsys, (3 * d.big_max + kThreads - 1) / kThreads), kThreads, 0, st>>>(d, a);
  k_adj_fold_kick<<<d.nsys, kThreads, 0, st>>>(d, a, which, grav);
}

void launch_adjoint_step_a(const Dev& d, const Adj& a, cudaStream_t st) {
  const int N = d.N;
  // forward recomputation
  k_adj_momentum<<<d.nsys, kThreads, 0, st>>>(d, a.z0 + 3 * (size_t)N, a.z0 + 4 * (size_t)N,
                                               a.z0 + 5 * (size_t)N, a.P, 0);
  // (with a.pd, x2 and v1 are the forward's, and only the drift is redone)
  if (!a.pd) k_adj_kick1_fwd<<<d.ntiles, d.tile, 0, st>>>(d, a);
  k_adj_momentum<<<d.nsys, kThreads, 0, st>>>(d, a.v1, a.v1 + N, a.v1 + 2 * (size_t)N, a.P, 1);
  k_adj_move_fwd<<<d.ntiles, d.tile, 0, st>>>(d, a, a.pd ? 3 : 1);
  if (a.groups) launch_adjoint_bs_plan(d, a, st);
}

void launch_adjoint_step_b(const Dev& d, const Adj& a, cudaStream_t st) {
  const int N = d.N;
  if (a.groups) launch_adjoint_bs_fwd(d, a, a.bs_blocks, st);
  k_adj_momentum<<<d.nsys, kThreads, 0, st>>>(d, a.xv3 + 3 * (size_t)N, a.xv3 + 4 * (size_t)N,
                                               a.xv3 + 5 * (size_t)N, a.P, 2);
  k_adj_move_fwd<<<d.ntiles, d.tile, 0, st>>>(d, a, 2);
  // reverse sweep: kick 2 (at x4, v3, P3), jump 2, drift, jump 1, kick 1 (at x0, v0, P0)
  // (with a.lin, the pair pass also takes the next step's first half kick,
  // left pending at the same positions)
  k_adj_kick_vjp<<<d.ntiles, d.tile, 0, st>>>(d, a, a.x4, a.xv3 + 3 * (size_t)N, 2, 2 * a.step + 1,
                                              KickRev{1, 1, 1, a.lin, nullptr});
  launch_fold_kick(d, a, 2, 1, st);
  if (a.groups) launch_adjoint_bs_vjp(d, a, a.bs_blocks, st);
  k_adj_drift_vjp<<<d.ntiles, d.tile, 0, st>>>(d, a);
  if (a.groups) launch_adjoint_bs_fold(d, a, st);
  k_adj_fold_jump1<<<d.nsys, kThreads, 0, st>>>(d, a);
  // merged: the drag now, the pair pass with the previous step's last half kick
  const KickRev r1{a.defer_k1 ? 0 : 1, 1, 1, nullptr, a.defer_k1 ? a.lpend : nullptr};
  k_adj_kick_vjp<<<d.ntiles, d.tile, 0, st>>>(d, a, a.z0, a.z0 + 3 * (size_t)N, 0, 2 * a.step, r1);
  launch_fold_kick(d, a, 1, r1.grav, st);
}

void launch_adjoint_flush(const Dev& d, const Adj& a, const double* xpos, cudaStream_t st) {
  k_adj_kick_vjp<<<d.ntiles, d.tile, 0, st>>>(d, a, xpos, xpos, 0, 0,
                                              KickRev{1, 0, 0, a.lpend, nullptr});
  launch_fold_kick(d, a, 1, 1, st);
}

// ------------------------------------------------------ loss and set-up
// L = sum_j w_j (a_f,j - a_i,j)^2 with a = 1/(2/r - v^2/gm) from heliocentric
// states (gm = G m0 for planetesimals, G (m0 + m) for big bodies).  Per tile:
// partial L; the DH cotangent of the final state (position: dL/dx_f; velocity:
// dL/dv_h, plus on big bodies (mu_i/m0) sum_j dL/dv_h,j, added by the fold)
// and the cotangent of the initial heliocentric state.
__device__ __forceinline__ double semimajor_grad(double gm, const double* x, const double* v,
                                                 double* dadx, double* dadv) {
  const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  const double r = sqrt(r2);
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const double E = 2.0 / r - v2 / gm;
  const double aa = 1.0 / E;
  for (int c = 0; c < 3; ++c) {
    dadx[c] = 2.0 * aa * aa * x[c] / (r2 * r);
    dadv[c] = 2.0 * aa * aa * v[c] / gm;
  }
  return aa;
}

__global__ void __launch_bounds__(kThreads) k_loss(Dev d, const double* xvh0, const double* wgt,
                                                   double* seed_f, double* seed_i, double* part,
                                                   const int* poff) {
  __shared__ double wsum[kThreads / 32][4];
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  const bool act = threadIdx.x < t.count;
  const int j = t.start + threadIdx.x;
  const int jl = j - S.off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  const double* P = d.P + 3 * t.sys;
  double own[4] = {0, 0, 0, 0};
  if (act) {
    const double wj = wgt[j];
    const double gm = S.mu0 + ((jl < S.nbig) ? d.bmu[S.boff + jl] : 0.0);
    double xf[3], vf[3], xi[3], vi[3], dxf[3], dvf[3], dxi[3], dvi[3];
    for (int c = 0; c < 3; ++c) {
      xf[c] = d.xv[(size_t)c * N + j];
      vf[c] = d.xv[(size_t)(3 + c) * N + j] + P[c] * S.inv_mu0;
      xi[c] = xvh0[(size_t)c * N + j];
      vi[c] = xvh0[(size_t)(3 + c) * N + j];
    }
    double fac = 0.0;
    if (wj != 0.0) {
      const double af = semimajor_grad(gm, xf, vf, dxf, dvf);
      const double ai = semimajor_grad(gm, xi, vi, dxi, dvi);
      const double da = af - ai;
      own[0] = wj * da * da;
      fac = 2.0 * wj * da;
    }
    for (int c = 0; c < 3; ++c) {
      const double gxf = (wj != 0.0) ? fac * dxf[c] : 0.0, gvf = (wj != 0.0) ? fac * dvf[c] : 0.0;
      seed_f[(size_t)c * N + j] = gxf;
      seed_f[(size_t)(3 + c) * N + j] = gvf;
      seed_i[(size_t)c * N + j] = (wj != 0.0) ? -fac * dxi[c] : 0.0;
      seed_i[(size_t)(3 + c) * N + j] = (wj != 0.0) ? -fac * dvi[c] : 0.0;
      own[1 + c] = gvf;
    }
  }
  for (int q = 0; q < 4; ++q) {
    double vq = own[q];
    for (int off = 16; off > 0; off >>= 1) vq += __shfl_down_sync(0xffffffffu, vq, off);
    if (lane == 0) wsum[warp][q] = vq;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double sum = 0;
    for (int q = 0; q < nwarps; ++q) sum += wsum[q][threadIdx.x];
    part[poff[blockIdx.x] + threadIdx.x] = sum;
  }
}

// Per system: L, and the bigs' share of the velocity cotangent through P.
__global__ void __launch_bounds__(kThreads) k_loss_fold(Dev d, double* seed_f, const double* part,
                                                        const int* poff, double* Lsys) {
  const int sys = blockIdx.x;
  const SysDev& S = d.sys[sys];
  const int N = d.N;
  __shared__ double tot[4];
  if (threadIdx.x < 4) {
    double sum = 0;
    for (int tt = 0; tt < d.ntiles; ++tt)
      if (d.tiles[tt].sys == sys) sum += part[poff[tt] + threadIdx.x];
    tot[threadIdx.x] = sum;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double m = d.bmu[S.boff + i] * S.inv_mu0;
    for (int c = 0; c < 3; ++c) seed_f[(size_t)(3 + c) * N + g] += m * tot[1 + c];
  }
  if (threadIdx.x == 0) Lsys[sys] = tot[0];
}

// Reverse of heliocentric -> DH at set-up: v_b = v_h - sum_i m_i v_h,i / M.
// Per system: S = sum_j lam_v_j (all bodies); big i gets -(m_i/M) S.
__global__ void __launch_bounds__(kThreads) k_init_vjp(Dev d, const double* lam, double* grad) {
  const int sys = blockIdx.x;
  const SysDev& S = d.sys[sys];
  const int N = d.N;
  __shared__ double red[4][kThreads];
  double acc[4] = {0, 0, 0, 0};
  for (int j = threadIdx.x; j < S.n; j += blockDim.x) {
    const int g = S.off + j;
    for (int c = 0; c < 6; ++c) grad[(size_t)c * N + g] = lam[(size_t)c * N + g];
    for (int c = 0; c < 3; ++c) acc[c] += lam[(size_t)(3 + c) * N + g];
  }
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) acc[3] += d.bmu[S.boff + i];
  for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  const double inv_tot = 1.0 / (S.mu0 + red[3][0]);   // 1 / (G M_total)
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int g = S.off + i;
    const double f = d.bmu[S.boff + i] * inv_tot;
    for (int c = 0; c < 3; ++c) grad[(size_t)(3 + c) * N + g] -= f * red[c][0];
  }
}

void launch_loss(const Dev& d, const double* xvh0, const double* w, double* seed_f, double* seed_i,
                 double* part, const int* poff, double* Lsys, cudaStream_t st) {
  k_loss<<<d.ntiles, d.tile, 0, st>>>(d, xvh0, w, seed_f, seed_i, part, poff);
  k_loss_fold<<<d.nsys, kThreads, 0, st>>>(d, seed_f, part, poff, Lsys);
}

void launch_init_vjp(const Dev& d, const double* lam, double* grad, cudaStream_t st) {
  k_init_vjp<<<d.nsys, kThreads, 0, st>>>(d, lam, grad);
}

}  // namespace mx
