// mx_physics.cuh -- per-pair gravity with the changeover weight and the gas
// drag of one planetesimal (arXiv 2601.16791, Sec. 2.1.3 and Sec. 3.1),
// shared by the forward kick and the adjoint's recomputation.
#pragma once
#include "mx_common.cuh"

namespace mx {

// The gas at a planetesimal's heliocentric position (Sec. 3.1): rho_g
// (Eq. 4, midplane), 1/c_s and the gas velocity factor g (v_gas = g (-y, x, 0),
// v_g = v_k sqrt(1 - 2 eta), Eqs. 5, 6), and, when enabled, the disk's
// gravity (Eqs. 10-12) along the cylindrical radius.  in_gas = false inside
// the inner edge (Sec. 3.1.1).  It depends on the position only, so the two
// half kicks of one launch share it.
struct GasAt {
  bool in_gas;
  double rho, inv_cs, g;
  double adg[2];   // disk gravity (x, y), zero unless enabled
};

__device__ __forceinline__ GasAt gas_at(const SysDev& S, double x, double y) {
  GasAt q;
  q.in_gas = false;
  q.rho = q.inv_cs = q.g = 0.0;
  q.adg[0] = q.adg[1] = 0.0;
  const double R2 = fma(x, x, y * y);
  const double iR = rsqrt_d(R2);             // 1/R
  const double R = R2 * iR;
  // no gas inside the inner edge (Sec. 3.1.1); R >= 0, so the test on the bit
  // patterns is the value test, off the FP64 pipe
  if (__double_as_longlong(R) < __double_as_longlong(S.r_in)) return q;
  double sigma, rmh, rcs, reta, inv_cs;      // Sigma, R^-(1+f), R^(f-1/2), R^(2f), 1/c_s
  const double ih = rsqrt_d(R);              // R^-1/2
  if (S.flare_quarter) {
    const double qq = rsqrt_d(ih);           // R^1/4
    rcs = qq * ih;                           // R^-1/4
    rmh = iR * rcs;                          // R^-5/4
    reta = R * ih;                           // R^1/2
    inv_cs = qq * S.inv_c_cs;
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
  q.rho = S.c_rho * sigma * rmh;
  const double vk = S.sqrt_mu0 * ih;
  const double t = fma(-2.0 * S.c_eta, reta, 1.0);   // 1 - 2 eta
  const double vg = vk * (t * rsqrt_d(t));
  q.g = vg * iR;                             // gas velocity = g * (-y, x, 0)
  q.inv_cs = inv_cs;
  q.in_gas = true;
  if (S.dg_on) {   // Eqs. 10-12: 2 pi G Sigma S(gamma), or 2 pi G Sigma r_in / R
    const double F = S.c_dg * sigma * (S.dg_edge ? iR : 1.0);
    q.adg[0] = F * iR * x;
    q.adg[1] = F * iR * y;
  }
  return q;
}

// The drag's terms of one planetesimal that do not depend on its velocity,
// for the half kicks of one launch (the position, the gas there and the
// momentum P are fixed over them): the gas's velocity minus P/m0 along x and
// y (so that dv = v_b + off), and the factors of Re and of the drag magnitude.
struct DragConst {
  bool in_gas;
  double offu, offv, offw;   // dv = (u + offu, v + offv, w + offw), u barycentric
  double inv_cs;
  double re_k;               // Re = re_k |dv|
  double coef_k;             // |a| = C_D coef_k |dv|^2
};

// kd = 3 / (8 r_p[AU] rho_p); rp_cm = r_p in cm; (hp0, hp1, hp2) = P/m0.
__device__ __forceinline__ DragConst drag_const(const SysDev& S, const GasAt& q, double x,
                                                double y, double hp0, double hp1, double hp2,
                                                double rp_cm, double kd) {
  DragConst c;
  c.in_gas = q.in_gas;
  c.offu = fma(q.g, y, hp0);
  c.offv = fma(-q.g, x, hp1);
  c.offw = hp2;
  c.inv_cs = q.inv_cs;
  c.re_k = (S.c_re * rp_cm) * (q.rho * q.inv_cs);
  c.coef_k = (S.cd_scale * kd) * q.rho;
  return c;
}

// Drag (Eq. 3) of one planetesimal with barycentric velocity (u, v, w), from
// its velocity-free terms (drag_const): returns coef >= 0 with the
// acceleration -coef (du, dv, dw), the velocity relative to the gas, written
// to dvec.  C_D (Eq. 7) from Re and Ma.  kb_in: -1 takes the k of Eq. 7 from
// Re; 0 or 1 forces k = 0.4 or 0.2 (a recorded branch being replayed).
// *kb_out receives the branch used.
__device__ __forceinline__ double gas_drag_coef(const SysDev& S, const DragConst& c, double u,
                                                double v, double w, double* dvec, int kb_in,
                                                int* kb_out) {
  dvec[0] = dvec[1] = dvec[2] = 0.0;
  *kb_out = 0;
  if (!c.in_gas) return 0.0;
  const double du = u + c.offu;
  const double dv = v + c.offv;
  const double dw = w + c.offw;
  dvec[0] = du;
  dvec[1] = dv;
  dvec[2] = dw;
  const double dv2 = fma(du, du, fma(dv, dv, dw * dw));
  if (__double_as_longlong(dv2) == 0) return 0.0;   // dv2 is +0 or positive
  const double dvm = dv2 * rsqrt_d(dv2);
  const double Ma = dvm * c.inv_cs;
  const double Re = c.re_k * dvm;
  // Re < 1e5 on the bit patterns (both positive): off the FP64 pipe
  const int kb = (kb_in >= 0) ? kb_in
                              : (__double_as_longlong(Re) < __double_as_longlong(1e5) ? 0 : 1);
  *kb_out = kb;
  const double k16 = kb ? 1.6 * 0.2 : 1.6 * 0.4;   // 1.6 k, both products made by the compiler
  // Eq. 7 with one reciprocal: [(24/Re + 40/(10+Re))^-1 + 0.23 Ma]^-1 = D/den1
  // where D = 240 + 64 Re and den1 = Re (10 + Re) + 0.23 Ma D, and the second
  // term (2 Ma + 1.6 k)/(1.6 + Ma); over the common denominator den1 A:
  // C_D = [D A + (2 Ma + 1.6 k) den1] / (den1 A).
  const double D = fma(64.0, Re, 240.0);
  const double den1 = fma(0.23 * Ma, D, Re * (10.0 + Re));
  const double A = 1.6 + Ma;
  const double r = rcp_d(den1 * A);
  const double t2 = fma(2.0, Ma, k16);
  double cd;
  if (S.cd_mode == 1) {   // the first term squared
    const double first = D * A * r;
    cd = fma(first, first, t2 * den1 * r);
  } else {
    cd = fma(t2, den1, D * A) * r;
  }
  return cd * c.coef_k * dvm;
}

// The drag acceleration itself (gas_drag_coef), into a[3].
__device__ __forceinline__ void gas_drag_at(const SysDev& S, const DragConst& c, double u,
                                            double v, double w, double* a, int kb_in,
                                            int* kb_out) {
  double d[3];
  const double coef = gas_drag_coef(S, c, u, v, w, d, kb_in, kb_out);
  a[0] = -coef * d[0];
  a[1] = -coef * d[1];
  a[2] = -coef * d[2];
}

// One half kick of a planetesimal's velocity with the gravity (ax, ay, az)
// and the drag coefficient and relative velocity of gas_drag_coef:
// v + h (a_grav - coef dv), as (v + h a_grav) - (h coef) dv.
__device__ __forceinline__ void kick_with_drag(double h, double ax, double ay, double az,
                                               double coef, const double* dvec, double& u,
                                               double& v, double& w) {
  const double hc = h * coef;
  u = fma(-hc, dvec[0], fma(h, ax, u));
  v = fma(-hc, dvec[1], fma(h, ay, v));
  w = fma(-hc, dvec[2], fma(h, az, w));
}

// The gas density factor of a planetesimal at (x, y, .) (the dens_factor
// listing of Sec. 3.1): 1, or the factor gf[i] of the last big body (ascending
// index) whose open gap (Eqs. 8-9) holds the planetesimal's cylindrical
// distance R strictly inside |R - gr[i]| < gw[i].  gr (the big bodies'
// cylindrical distances at kick time) comes from k_prep, gw and gf from
// k_grow; the arrays start at the system's first big body.  Not inlined, so
// that the kick and the catch-up of deferred planetesimals decide alike.
static __device__ __noinline__ double gap_factor(const double* gr, const double* gw,
                                                 const double* gf, int nbig, double x, double y) {
  const double R = sqrt(x * x + y * y);
  double f = 1.0;
  for (int i = 0; i < nbig; ++i) {
    const double w = gw[i];
    if (w > 0.0) {
      const double r = gr[i];
      if (R < r + w && R > r - w) f = gf[i];
    }
  }
  return f;
}

__device__ __forceinline__ double gap_factor(const Dev& d, const SysDev& S, double x, double y) {
  return gap_factor(d.gap_r + S.boff, d.gap_w + S.boff, d.gap_f + S.boff, S.nbig, x, y);
}

// The gas's acceleration on one planetesimal at heliocentric position
// (x, y, z) moving with heliocentric velocity (u, v, w): the drag (gas_at,
// then gas_drag_at) plus, when enabled, the disk's gravity.  Quantities follow
// Sec. 3.1: Sigma (Eq. 1, normalised at 1 AU), rho_g (Eq. 4) at the midplane,
// v_g (Eqs. 5, 6), C_D (Eq. 7).  dfac multiplies the gas density (a gap).
// (u, v, w) is the heliocentric velocity here.
__device__ __forceinline__ void gas_drag(const SysDev& S, double x, double y, double z, double u,
                                         double v, double w, double rp_cm, double kd, double* a,
                                         int kb_in, int* kb_out, double dfac = 1.0) {
  (void)z;
  GasAt q = gas_at(S, x, y);
  q.rho *= dfac;
  gas_drag_at(S, drag_const(S, q, x, y, 0.0, 0.0, 0.0, rp_cm, kd), u, v, w, a, kb_in, kb_out);
  a[0] += q.adg[0];
  a[1] += q.adg[1];
}

// f = mu K(s)/s^3 for one pair at separation d (Sec. 2.1.3: K = 1 for
// s^2 >= rc^2, 0 for s^2 <= 0.01 rc^2, quintic between).
// mu/s^3 comes straight from the single-precision estimate y of 1/s (relative
// error ~1e-6, as in rsqrt_d): with e = 1 - s^2 y^2 (y^2 is exact, y having
// 24 significant bits), 1/s^3 = y^3 (1 - e)^(-3/2) = y^3 (1 + 3e/2 + 15e^2/8),
// the dropped terms ~2 e^3 below the FP64 rounding; 1/s itself (for the
// changeover shell only) is y (1 + e/2 + 3e^2/8), as rsqrt_d makes it.
__device__ __forceinline__ double pair_weight(double dx, double dy, double dz, double mu,
                                              double rc2, double rc2lo, double rc01,
                                              double i09rc) {
  const double s2 = fma(dx, dx, fma(dy, dy, dz * dz));
  const double y = float_to_double_bits(rsqrtf(abs_to_float_bits(s2)));
  const double y2 = y * y;
  const double e = fma(-s2, y2, 1.0);
  double f = ((mu * y) * y2) * fma(e, fma(1.875, e, 1.5), 1.0);
  // s2 < rc2 decided on the bit patterns: for non-negative doubles the integer
  // order is the value order, and the compare leaves the FP64 pipe free
  if (__double_as_longlong(s2) < __double_as_longlong(rc2)) {
    if (s2 <= rc2lo) {
      f = 0.0;
    } else {
      const double yy = fma(y * e, fma(0.375, e, 0.5), y);
      const double q = (s2 * yy - rc01) * i09rc;
      f *= q * q * q * fma(q, fma(6.0, q, -15.0), 10.0);
    }
  }
  return f;
}

// The pair's acceleration -f d accumulated into (ax, ay, az).
__device__ __forceinline__ void pair_acc(double dx, double dy, double dz, double mu, double rc2,
                                         double rc2lo, double rc01, double i09rc, double& ax,
                                         double& ay, double& az) {
  const double f = pair_weight(dx, dy, dz, mu, rc2, rc2lo, rc01, i09rc);
  ax = fma(-f, dx, ax);
  ay = fma(-f, dy, ay);
  az = fma(-f, dz, az);
}

// Shared-memory staging of one chunk of big bodies: nine arrays of `chunk`
// doubles in the block's dynamic shared memory, chunk = min(most big bodies
// of a system, kBigChunk), so that a disk with a few big bodies leaves the SM
// its shared memory (the number of resident blocks is then set by registers).
__host__ __device__ __forceinline__ int big_chunk(int big_max) {
  return big_max < 1 ? 1 : (big_max < kBigChunk ? big_max : kBigChunk);
}

struct BigSmem {
  double *x, *y, *z, *mu, *rc, *rc2, *rc2lo, *rc01, *i09rc;
  int chunk;
  __device__ BigSmem(double* base, int n)
      : x(base), y(base + n), z(base + 2 * n), mu(base + 3 * n), rc(base + 4 * n),
        rc2(base + 5 * n), rc2lo(base + 6 * n), rc01(base + 7 * n), i09rc(base + 8 * n),
        chunk(n) {}
};

}  // namespace mx
