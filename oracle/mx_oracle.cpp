// mx_oracle.cpp -- plain, slow, FP64 CPU oracle of the hybrid symplectic hot
// path of arXiv 2601.16791 (Mercury-Arxes / Mercury+).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
// bench.py's CPU-baseline leg may load this library.  It shares nothing with
// the CUDA path (paper_2601_16791_gb300/csrc): no header, helper, table or
// constant.  Every routine is written from the paper; where the paper is
// silent the reading used is stated beside the code.
//
// The routines are templates over the scalar type so that the same code,
// instantiated with a forward-mode dual number, gives the reference
// directional derivative of a loss (orc_jvp_loss).  Control flow always
// follows the real part, so the dual instantiation takes exactly the
// branches, encounter flags and Bulirsch-Stoer step decisions of the plain
// FP64 run.
//
// Compile without floating-point contraction (-ffp-contract=off) so the
// results are the same on x86-64 and AArch64 hosts.

#include "mx_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- constants
constexpr double kPi = 3.14159265358979323846;
constexpr double kAuCm = 1.495978707e13;     // astronomical unit [cm] (IAU 2012)
constexpr double kAuKm = 1.495978707e8;      // astronomical unit [km]
constexpr double kHydrogenG = 1.6735575e-24; // mass of a hydrogen atom [g]
constexpr double kMsunG = 1.98847e33;        // solar mass [g]
constexpr double kEps = std::numeric_limits<double>::epsilon();

// ------------------------------------------------------------ dual numbers
// One-direction forward-mode AD.  Real parts are computed with the same
// double operations as the plain instantiation.
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
inline Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual& a, const Dual& b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual sqrt(const Dual& a) {
  const double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline Dual exp(const Dual& a) {
  const double e = std::exp(a.v);
  return Dual(e, a.d * e);
}
inline Dual log(const Dual& a) { return Dual(std::log(a.v), a.d / a.v); }

inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
inline double dpart(double) { return 0.0; }
inline double dpart(const Dual& a) { return a.d; }

using std::exp;
using std::log;
using std::sqrt;

// a^p with both arguments possibly dual; real part is std::pow in both cases.
inline double tpow(double a, double p) { return std::pow(a, p); }
inline Dual tpow(const Dual& a, double p) {
  const double r = std::pow(a.v, p);
  return Dual(r, p * std::pow(a.v, p - 1.0) * a.d);
}
inline Dual tpow(const Dual& a, const Dual& p) {
  const double r = std::pow(a.v, p.v);
  return Dual(r, p.v * std::pow(a.v, p.v - 1.0) * a.d + r * std::log(a.v) * p.d);
}

// ------------------------------------------------------------------ state
template <class T>
struct State {
  int n = 0;
  std::vector<T> q[6];  // x, y, z, vx, vy, vz
  void resize(int nn) {
    n = nn;
    for (auto& a : q) a.assign(nn, T(0.0));
  }
};

struct Bodies {
  int nbig = 0, nsmall = 0, n = 0;
  double mu0 = 0.0;                 // G * m_star
  std::vector<double> mu, rcrit;    // per body; zero for small bodies
  std::vector<double> rp_km, rhop;  // per small body
  // per body: 0 in the integration, -3 removed as ejected (Sec. 3.5); empty:
  // every body is in.  A removed body keeps its state and takes no part in
  // the kick, jump, drift or encounter search; a removed massive body has mu 0.
  std::vector<signed char> stat;
  bool gone(int j) const { return !stat.empty() && stat[j] != 0; }
  // per massive body: gap half-width (0: no gap) and gas density factor in it
  // (Sec. 3.1, Eqs. 8-9); empty: no gaps
  std::vector<double> gap_w, gap_f;
};

template <class T>
struct GasT {
  orc_gas raw;
  double G = 0.0;             // gravitational constant (disk gravity)
  T sigma1, gamma, cd_scale;  // the three differentiable disk/drag parameters
};

template <class T>
void load_state(State<T>& s, int n, const double* xv) {
  s.resize(n);
  for (int k = 0; k < 6; ++k)
    for (int j = 0; j < n; ++j) s.q[k][j] = T(xv[(size_t)k * n + j]);
}
template <class T>
void store_state(const State<T>& s, double* xv) {
  for (int k = 0; k < 6; ++k)
    for (int j = 0; j < s.n; ++j) xv[(size_t)k * s.n + j] = val(s.q[k][j]);
}

// -------------------------------------------------- changeover (Sec. 2.1.3)
// The mfo_drct listing: with rc = max(rcrit_i, rcrit_j), a pair at distance s
// gets K = 1 for s^2 >= rc^2, K = 0 for s^2 <= 0.01 rc^2, and otherwise
// K = 10q^3 - 15q^4 + 6q^5 with q = (s - 0.1 rc)/(0.9 rc).  The kick applies
// K/s^3 times mu_i * dx.
inline double changeover_K(double s, double rc) {
  if (s * s >= rc * rc) return 1.0;
  if (s * s <= 0.01 * rc * rc) return 0.0;
  const double q = (s - 0.1 * rc) / (0.9 * rc);
  return 10.0 * q * q * q - 15.0 * q * q * q * q + 6.0 * q * q * q * q * q;
}

template <class T>
T k_over_s3(const T& s2, double rc) {
  const double rc2 = rc * rc;
  if (val(s2) >= rc2) {
    T s = sqrt(s2);
    return T(1.0) / (s2 * s);
  }
  if (val(s2) <= 0.01 * rc2) return T(0.0);
  T s = sqrt(s2);
  T q = (s - 0.1 * rc) / (0.9 * rc);
  T K = T(10.0) * q * q * q - T(15.0) * q * q * q * q + T(6.0) * q * q * q * q * q;
  return K / (s2 * s);
}

// The complement used inside an encounter: (1 - K)/s^3.
template <class T>
T one_minus_k_over_s3(const T& s2, double rc) {
  const double rc2 = rc * rc;
  if (val(s2) >= rc2) return T(0.0);
  T s = sqrt(s2);
  if (val(s2) <= 0.01 * rc2) return T(1.0) / (s2 * s);
  T q = (s - 0.1 * rc) / (0.9 * rc);
  T K = T(10.0) * q * q * q - T(15.0) * q * q * q * q + T(6.0) * q * q * q * q * q;
  return (T(1.0) - K) / (s2 * s);
}

// ------------------------------------------- interaction kick (Sec. 2.1.3)
// Rectangular (parallel) form of mfo_drct: each target j sums over the big
// sources i != j in ascending i.
template <class T>
void accel_grav(const Bodies& b, const State<T>& s, std::vector<T>* a) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < b.n; ++j) {
    T ax(0.0), ay(0.0), az(0.0);
    for (int i = 0; i < b.nbig && !b.gone(j); ++i) {
      if (i == j) continue;
      T dx = s.q[0][j] - s.q[0][i];
      T dy = s.q[1][j] - s.q[1][i];
      T dz = s.q[2][j] - s.q[2][i];
      T s2 = dx * dx + dy * dy + dz * dz;
      const double rc = std::max(b.rcrit[i], b.rcrit[j]);
      T f = k_over_s3(s2, rc) * b.mu[i];
      ax = ax - f * dx;
      ay = ay - f * dy;
      az = az - f * dz;
    }
    a[0][j] = ax;
    a[1][j] = ay;
    a[2][j] = az;
  }
}

// Serial triangular form of the same listing (Newton's third law).
void accel_grav_triangular(const Bodies& b, const State<double>& s, std::vector<double>* a) {
  for (int k = 0; k < 3; ++k) a[k].assign(b.n, 0.0);
  for (int i = 0; i < b.nbig; ++i) {
    for (int j = i + 1; j < b.n; ++j) {
      double dx = s.q[0][j] - s.q[0][i];
      double dy = s.q[1][j] - s.q[1][i];
      double dz = s.q[2][j] - s.q[2][i];
      double s2 = dx * dx + dy * dy + dz * dz;
      const double rc = std::max(b.rcrit[i], b.rcrit[j]);
      double t = k_over_s3(s2, rc);
      double fi = t * b.mu[i], fj = t * b.mu[j];
      a[0][j] -= fi * dx; a[1][j] -= fi * dy; a[2][j] -= fi * dz;
      a[0][i] += fj * dx; a[1][i] += fj * dy; a[2][i] += fj * dz;
    }
  }
}

// Momentum of the massive bodies only (Sec. 2.1.3: the loops of mco_dh2h and
// mdt_hy run over the massive bodies), G-scaled: P = sum mu_i v_i.
template <class T>
void momentum(const Bodies& b, const State<T>& s, T P[3]) {
  for (int k = 0; k < 3; ++k) {
    T acc(0.0);
    for (int i = 0; i < b.nbig; ++i) acc = acc + b.mu[i] * s.q[3 + k][i];
    P[k] = acc;
  }
}

// ------------------------------------------------------ gas drag (Sec. 3.1)
// Drag coefficient, Eq. 7 (Tanigawa et al. form).  k is 0.4 for Re < 1e5 and
// 0.2 otherwise (the paper leaves Re = 1e5 itself unassigned; it goes with
// the upper branch).  mode 0 raises the bracket to the power -1, so that
// C_D -> 24/Re in the Stokes limit; mode 1 uses the printed power -2.
template <class T>
T drag_cd(const T& Re, const T& Ma, int mode) {
  const double k = (val(Re) < 1e5) ? 0.4 : 0.2;
  T inner = T(24.0) / Re + T(40.0) / (T(10.0) + Re);
  T bracket = T(1.0) / inner + T(0.23) * Ma;
  T first = (mode == 1) ? T(1.0) / (bracket * bracket) : T(1.0) / bracket;
  return first + T(2.0) * (T(0.8 * k) + Ma) / (T(1.6) + Ma);
}

// Disk model at cylindrical radius R (AU).  Eq. 1 with the normalisation
// moved to 1 AU (Sigma1 = Sigma(1 AU) when R_C is infinite), the flared
// aspect ratio H/r = hr_1au (R/1AU)^flare, c_s = (H/r) v_k, h = c_s/Omega
// (Eq. 4), eta from Eq. 6 with temperature slope beta = 1 - 2 flare (since
// c_s^2 ~ T), and v_g from Eq. 5.
template <class T>
struct DiskAt {
  T sigma, rho_g, H_au, cs, vk, eta, vg, hr;
};

template <class T>
DiskAt<T> disk_at(const GasT<T>& g, double mu0, const T& R) {
  DiskAt<T> d;
  d.sigma = g.sigma1 * tpow(R, -g.gamma);
  if (std::isfinite(g.raw.r_c_au)) d.sigma = d.sigma * exp(-tpow(R / g.raw.r_c_au, T(2.0) - g.gamma));
  d.hr = g.raw.hr_1au * tpow(R, g.raw.flare);
  d.vk = sqrt(mu0 / R);
  d.cs = d.hr * d.vk;
  d.H_au = d.hr * R;
  d.rho_g = d.sigma / (std::sqrt(2.0 * kPi) * d.H_au * kAuCm);
  const double beta_T = 1.0 - 2.0 * g.raw.flare;
  d.eta = (T(1.0) / (2.0 * g.raw.gamma_c)) * (g.gamma + (beta_T / 2.0 + 1.5)) * d.hr * d.hr;
  d.vg = d.vk * sqrt(T(1.0) - T(2.0) * d.eta);
  return d;
}

// Drag acceleration of one small body (Eq. 3): magnitude
// (3/8)(C_D/r_p)(rho_g/rho_p)|dv|^2 against the relative velocity dv between
// the body (heliocentric velocity) and the sub-Keplerian, azimuthal gas.
// Re and Ma follow the definitions the paper defers to Brasser et al. (2007):
// Ma = |dv|/c_s; Re = 2 r_p |dv| / nu with nu = (1/2) v_th lambda,
// v_th = sqrt(8/pi) c_s and lambda = mu_mol m_H / (sigma_mol rho_g).
// rho_g is the midplane value (Eq. 4) for every height.  Inside R_in the
// density factor is zero (Sec. 3.1.1), so the drag vanishes.
// dfac multiplies the gas density (the listing's dens_factor: a gap).
template <class T>
void drag_one(const GasT<T>& g, double mu0, const T* x, const T* vh, double rp_km,
              double rhop, T* acc, double* re_ma, double dfac = 1.0) {
  acc[0] = acc[1] = acc[2] = T(0.0);
  if (re_ma) re_ma[0] = re_ma[1] = 0.0;
  if (!g.raw.enabled) return;
  T R = sqrt(x[0] * x[0] + x[1] * x[1]);
  if (val(R) < g.raw.r_in_au) return;
  DiskAt<T> d = disk_at(g, mu0, R);
  d.rho_g = d.rho_g * dfac;
  T ux = -x[1] / R, uy = x[0] / R;  // azimuthal unit vector
  T dvx = vh[0] - d.vg * ux;
  T dvy = vh[1] - d.vg * uy;
  T dvz = vh[2];
  T dv = sqrt(dvx * dvx + dvy * dvy + dvz * dvz);
  if (val(dv) == 0.0) return;
  T Ma = dv / d.cs;
  T lambda_cm = T(g.raw.mu_mol * kHydrogenG / g.raw.sigma_mol_cm2) / d.rho_g;
  T vth = std::sqrt(8.0 / kPi) * d.cs;
  T nu = T(0.5) * vth * lambda_cm;  // [AU/d * cm]
  const double rp_cm = rp_km * 1.0e5;
  T Re = T(2.0 * rp_cm) * dv / nu;
  T cd = drag_cd(Re, Ma, g.raw.cd_mode) * g.cd_scale;
  const double rp_au = rp_km / kAuKm;
  T coef = T(3.0 / 8.0) * cd / rp_au * (d.rho_g / rhop) * dv;
  acc[0] = -coef * dvx;
  acc[1] = -coef * dvy;
  acc[2] = -coef * dvz;
  if (re_ma) { re_ma[0] = val(Re); re_ma[1] = val(Ma); }
}

// ------------------------------------------- disk gravity (Sec. 3.1.2)
// The leading term of the axisymmetric thin-disk force (Eq. 10):
//   F_DG = 2 pi G Sigma(r) S(gamma),
//   S(gamma) = sum_n A_n (1 - gamma)(4n + 1) / ((2n + 2 - gamma)(2n - 1 + gamma)),
//   A_n = [(2n)! / (2^(2n) (n!)^2)]^2,
// and for gamma = 1 the leading edge term, F_DG = 2 pi G Sigma(r) R_in / r
// (Eq. 12).  The terms of S fall off as (1 - gamma)/(pi n^2), so the partial
// sums S_N approach S as S + c1/N + c2/N^2 + ...; S is taken from the
// compensated partial sums at N = 256 * 2^k by Richardson extrapolation in 1/N
// (eight levels).  Reading: F_DG is the signed radial force per unit mass in the
// midplane (positive outward), applied along the cylindrical radius; it acts
// on planetesimals only, where there is gas (r >= R_in).
// With deriv = 1 the same sums give dS/dgamma, term by term: with
// a = 2n + 2 - gamma and b = 2n - 1 + gamma, d/dgamma [(1 - gamma)/(a b)] =
// [-a b + (1 - gamma)(b - a)]/(a b)^2; those terms fall off as -1/(pi n^2),
// so the same extrapolation applies.
double dg_series_sum(double gamma, int deriv) {
  const int levels = 8;
  double S[levels];
  double sum = 0.0, comp = 0.0;      // compensated (Kahan) sum of the terms
  double An_root = 1.0;              // A_n = An_root^2, An_root = (2n)!/(4^n (n!)^2)
  int n = 0;
  for (int k = 0; k < levels; ++k) {
    const int N = 256 << k;
    for (; n < N; ++n) {
      if (n > 0) An_root *= (2.0 * n - 1.0) / (2.0 * n);
      const double An = An_root * An_root;
      double t;
      if (!deriv) {
        t = An * (1.0 - gamma) * (4.0 * n + 1.0) /
            ((2.0 * n + 2.0 - gamma) * (2.0 * n - 1.0 + gamma));
      } else {
        const double a = 2.0 * n + 2.0 - gamma, b = 2.0 * n - 1.0 + gamma;
        t = An * (4.0 * n + 1.0) * (-(a * b) + (1.0 - gamma) * (b - a)) / ((a * b) * (a * b));
      }
      const double y = t - comp;
      const double nxt = sum + y;
      comp = (nxt - sum) - y;
      sum = nxt;
    }
    S[k] = sum;
  }
  // Richardson: each level removes the next 1/N^m term (N doubles between entries)
  for (int m = 1; m < levels; ++m)
    for (int k = levels - 1; k >= m; --k) {
      const double f = std::ldexp(1.0, m);
      S[k] = (f * S[k] - S[k - 1]) / (f - 1.0);
    }
  return S[levels - 1];
}

double dg_series(double gamma) { return dg_series_sum(gamma, 0); }
double dg_series_dgamma(double gamma) { return dg_series_sum(gamma, 1); }

// S(gamma) as a function of the (possibly dual) parameter gamma: the forward
// derivative carries dS/dgamma.
inline double dg_factor(double gamma) { return dg_series(gamma); }
inline Dual dg_factor(const Dual& gamma) {
  return Dual(dg_series(gamma.v), dg_series_dgamma(gamma.v) * gamma.d);
}

template <class T>
void disk_gravity_one(const GasT<T>& g, double mu0, const T* x, T* acc) {
  if (!g.raw.enabled || !g.raw.disk_gravity) return;
  T R = sqrt(x[0] * x[0] + x[1] * x[1]);
  if (val(R) < g.raw.r_in_au || val(R) == 0.0) return;
  DiskAt<T> d = disk_at(g, mu0, R);
  const double to_code = kAuCm * kAuCm / kMsunG;   // g/cm^2 -> Msun/AU^2
  T F = T(2.0 * kPi * g.G * to_code) * d.sigma;
  if (g.raw.gamma == 1.0) F = F * (g.raw.r_in_au / R);
  else F = F * dg_factor(g.gamma);
  acc[0] = acc[0] + F * x[0] / R;
  acc[1] = acc[1] + F * x[1] / R;
}

// The gas density factor of the Sec. 3.1 listing at cylindrical distance R:
// 1, or the factor of the last massive body (ascending index) with a gap whose
// band |R - r_i| < W_i holds R, r_i the body's cylindrical distance now.
template <class T>
double gap_factor(const Bodies& b, const State<T>& s, double R) {
  double f = 1.0;
  for (int i = 0; i < (int)b.gap_w.size(); ++i) {
    if (!(b.gap_w[i] > 0.0)) continue;
    const double xi = val(s.q[0][i]), yi = val(s.q[1][i]);
    const double ri = std::sqrt(xi * xi + yi * yi);
    if (R < ri + b.gap_w[i] && R > ri - b.gap_w[i]) f = b.gap_f[i];
  }
  return f;
}

// Drag on every small body, plus the disk's gravity when enabled.  The body's
// heliocentric velocity is its DH (barycentric) velocity plus P/m0, P the
// massive-body momentum at kick time.
template <class T>
void accel_drag(const GasT<T>& g, const Bodies& b, const State<T>& s, const T P[3],
                std::vector<T>* a) {
  const int nb = b.nbig;
#pragma omp parallel for schedule(static)
  for (int j = nb; j < b.n; ++j) {
    if (b.gone(j)) {
      for (int k = 0; k < 3; ++k) a[k][j] = T(0.0);
      continue;
    }
    T x[3] = {s.q[0][j], s.q[1][j], s.q[2][j]};
    T vh[3];
    for (int k = 0; k < 3; ++k) vh[k] = s.q[3 + k][j] + P[k] / b.mu0;
    T acc[3];
    double dfac = 1.0;
    if (!b.gap_w.empty()) {
      const double xj = val(x[0]), yj = val(x[1]);
      dfac = gap_factor(b, s, std::sqrt(xj * xj + yj * yj));
    }
    drag_one(g, b.mu0, x, vh, b.rp_km[j - nb], b.rhop[j - nb], acc, nullptr, dfac);
    disk_gravity_one(g, b.mu0, x, acc);
    for (int k = 0; k < 3; ++k) a[k][j] = acc[k];
  }
}

// ----------------------------------------------------- Kepler drift (Sec. 2)
// The paper drives the Keplerian part with the WHFast solver (Sec. 2); this
// oracle solves the same two-body problem in universal variables.
// Stumpff functions c_k(z) = sum_m (-z)^m/(2m+k)!, evaluated by series after
// reducing |z| below 0.1 by quarters and restored with the quadrupling
// identities c0(4z) = 2c0^2 - 1, c1(4z) = c0 c1, c2(4z) = c1^2/2,
// c3(4z) = (c2 + c0 c3)/4 (Danby 1988, Sec. 6.9).
template <class T>
void stumpff(T z, T* c) {
  int nred = 0;
  while (std::fabs(val(z)) > 0.1) {
    z = z * 0.25;
    ++nred;
  }
  const int M = 12;
  double inv_fact[2 * M + 4];
  inv_fact[0] = 1.0;
  for (int k = 1; k < 2 * M + 4; ++k) inv_fact[k] = inv_fact[k - 1] / k;
  T c2(inv_fact[2 * M + 2]), c3(inv_fact[2 * M + 3]);
  for (int m = M - 1; m >= 0; --m) {
    c2 = T(inv_fact[2 * m + 2]) - z * c2;
    c3 = T(inv_fact[2 * m + 3]) - z * c3;
  }
  T c1 = T(1.0) - z * c3;
  T c0 = T(1.0) - z * c2;
  for (int r = 0; r < nred; ++r) {
    T n0 = T(2.0) * c0 * c0 - T(1.0);
    T n1 = c0 * c1;
    T n2 = T(0.5) * c1 * c1;
    T n3 = T(0.25) * (c2 + c0 * c3);
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  c[0] = c0; c[1] = c1; c[2] = c2; c[3] = c3;
}

// Universal Kepler equation in s: F(s) = r0 G1 + eta0 G2 + mu G3 - h = 0,
// G_k = s^k c_k(beta s^2), F'(s) = r(s) > 0.  Newton iteration kept inside a
// bisection bracket, stopped when |ds| <= 4 ulp(s).  A final Newton
// correction carries the implicit-function derivative for dual numbers.
// The state then moves by the Gauss f and g functions.
template <class T>
int drift_one(double mu, double h, T* x, T* v, int maxit, int* iters) {
  if (h == 0.0) return ORC_OK;
  T r0 = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  T v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  T eta = x[0] * v[0] + x[1] * v[1] + x[2] * v[2];
  T beta = T(2.0 * mu) / r0 - v2;
  auto eval = [&](const T& s, T& F, T& dF, T* G) {
    T c[4];
    stumpff(beta * s * s, c);
    G[0] = c[0];
    G[1] = s * c[1];
    G[2] = s * s * c[2];
    G[3] = s * s * s * c[3];
    F = r0 * G[1] + eta * G[2] + mu * G[3] - h;
    dF = r0 * G[0] + eta * G[1] + mu * G[2];
  };
  T F, dF, G[4];
  const double s0 = h / val(r0);
  double lo, hi;
  // Bracket the root; F is strictly increasing.
  {
    double a = s0;
    int grow = 0;
    eval(T(a), F, dF, G);
    if (h > 0.0) {
      lo = 0.0;
      while (val(F) < 0.0) {
        lo = a; a *= 2.0;
        eval(T(a), F, dF, G);
        if (++grow > 200) return ORC_ERR_KEPLER_NOCONV;
      }
      hi = a;
    } else {
      hi = 0.0;
      while (val(F) > 0.0) {
        hi = a; a *= 2.0;
        eval(T(a), F, dF, G);
        if (++grow > 200) return ORC_ERR_KEPLER_NOCONV;
      }
      lo = a;
    }
  }
  T s(std::min(std::max(s0, lo), hi));
  bool conv = false;
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    eval(s, F, dF, G);
    if (val(F) < 0.0) lo = std::max(lo, val(s));
    else hi = std::min(hi, val(s));
    T snew = s - F / dF;
    if (!(val(snew) > lo && val(snew) < hi)) snew = T(0.5 * (lo + hi));
    const double ds = val(snew) - val(s);
    s = snew;
    if (std::fabs(ds) <= 4.0 * kEps * std::fabs(val(s)) || lo == hi) {
      conv = true;
      break;
    }
  }
  if (iters) *iters = it;
  if (!conv) return ORC_ERR_KEPLER_NOCONV;
  eval(s, F, dF, G);
  s = s - F / dF;
  eval(s, F, dF, G);
  T r = dF;
  T f = T(1.0) - mu * G[2] / r0;
  T g = r0 * G[1] + eta * G[2];
  T fd = -(mu * G[1]) / (r * r0);
  T gd = T(1.0) - mu * G[2] / r;
  T xn[3], vn[3];
  for (int k = 0; k < 3; ++k) {
    xn[k] = f * x[k] + g * v[k];
    vn[k] = fd * x[k] + gd * v[k];
  }
  for (int k = 0; k < 3; ++k) { x[k] = xn[k]; v[k] = vn[k]; }
  return ORC_OK;
}

template <class T>
int drift_all(double mu0, double h, int maxit, State<T>& s, int* itmax,
              const Bodies* b = nullptr) {
  int err = ORC_OK, imax = 0;
#pragma omp parallel for schedule(static) reduction(max : err, imax)
  for (int j = 0; j < s.n; ++j) {
    if (b && b->gone(j)) continue;
    T x[3] = {s.q[0][j], s.q[1][j], s.q[2][j]};
    T v[3] = {s.q[3][j], s.q[4][j], s.q[5][j]};
    int it = 0;
    int e = drift_one(mu0, h, x, v, maxit, &it);
    if (e) err = std::max(err, e);
    imax = std::max(imax, it);
    for (int k = 0; k < 3; ++k) { s.q[k][j] = x[k]; s.q[3 + k][j] = v[k]; }
  }
  if (itmax) *itmax = std::max(*itmax, imax);
  return err;
}

// ------------------------------------------- encounter detection (Sec. 2.1.2)
// The mce_snif listing flags a pair when min(d0, d1, d2min) <= rc^2.  Reading
// of d2min: the minimum over the step of the cubic Hermite interpolant of the
// squared separation built from its end values d0, d1 and end time slopes
// d0t = 2 dx0.dv0, d1t = 2 dx1.dv1; it exists only when the separation is
// shrinking at the start and growing at the end.  The interior stationary
// point is found here by plain bisection on the derivative.
double hermite_d2min(double d0, double d1, double d0t, double d1t, double h) {
  const double D0 = h * d0t, D1 = h * d1t;  // slopes in tau = t/h
  if (!(D0 < 0.0 && D1 > 0.0)) return std::numeric_limits<double>::infinity();
  auto dp = [&](double t) {
    return d0 * (6.0 * t * t - 6.0 * t) + D0 * (3.0 * t * t - 4.0 * t + 1.0) +
           d1 * (6.0 * t - 6.0 * t * t) + D1 * (3.0 * t * t - 2.0 * t);
  };
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (dp(mid) < 0.0) lo = mid;
    else hi = mid;
  }
  const double t = 0.5 * (lo + hi);
  const double t2 = t * t, t3 = t2 * t;
  const double p = d0 * (2.0 * t3 - 3.0 * t2 + 1.0) + D0 * (t3 - 2.0 * t2 + t) +
                   d1 * (-2.0 * t3 + 3.0 * t2) + D1 * (t3 - t2);
  return std::max(p, 0.0);
}

// Returns the flagged pairs (i < nbig, j != i; a big-big pair once, i < j)
// sorted by (i, j).
void detect(const Bodies& b, const double* xv0, const double* xv1, double h,
            std::vector<std::pair<int, int>>& pairs) {
  const int n = b.n;
  std::vector<std::vector<std::pair<int, int>>> per_i(b.nbig);
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < b.nbig; ++i) {
    for (int j = 0; j < n; ++j) {
      if (j == i || (j < b.nbig && j < i) || b.gone(i) || b.gone(j)) continue;
      double dx0[3], dv0[3], dx1[3], dv1[3];
      for (int k = 0; k < 3; ++k) {
        dx0[k] = xv0[(size_t)k * n + j] - xv0[(size_t)k * n + i];
        dv0[k] = xv0[(size_t)(3 + k) * n + j] - xv0[(size_t)(3 + k) * n + i];
        dx1[k] = xv1[(size_t)k * n + j] - xv1[(size_t)k * n + i];
        dv1[k] = xv1[(size_t)(3 + k) * n + j] - xv1[(size_t)(3 + k) * n + i];
      }
      const double d0 = dx0[0] * dx0[0] + dx0[1] * dx0[1] + dx0[2] * dx0[2];
      const double d1 = dx1[0] * dx1[0] + dx1[1] * dx1[1] + dx1[2] * dx1[2];
      const double d0t = 2.0 * (dx0[0] * dv0[0] + dx0[1] * dv0[1] + dx0[2] * dv0[2]);
      const double d1t = 2.0 * (dx1[0] * dv1[0] + dx1[1] * dv1[1] + dx1[2] * dv1[2]);
      const double rc = std::max(b.rcrit[i], b.rcrit[j]);
      const double m = std::min(std::min(d0, d1), hermite_d2min(d0, d1, d0t, d1t, h));
      if (m <= rc * rc) per_i[i].push_back({i, j});
    }
  }
  pairs.clear();
  for (auto& v : per_i) pairs.insert(pairs.end(), v.begin(), v.end());
}

// ------------------------------------------------ Bulirsch-Stoer (Sec. 2)
// mdt_bs2 integrates encounter bodies under conservative forces.  The paper
// gives no constants; reading: Gragg-Bulirsch-Stoer with Stoermer's rule for
// y'' = f(y), sub-step counts n_k = 2k (k = 1..8), polynomial extrapolation
// in (H/n)^2, error = max over bodies of max(|dx|^2 xscal, |dv|^2 vscal)
// with xscal = 1/|x|^2 and vscal = 1/|v|^2 at the start of the sub-step (the
// Sec. 2.1.1 listing), accepted when <= tol^2.  On acceptance the next
// sub-step grows by 1.3 (capped by what remains); on failure it halves.
// Forces: the star plus (1-K)-weighted pair forces from the massive members.
template <class T>
void bs_accel(double mu0, int nb, const double* mu, const double* rcrit, const std::vector<T>& X,
              std::vector<T>& A) {
  for (int bb = 0; bb < nb; ++bb) {
    T x = X[bb], y = X[nb + bb], z = X[2 * nb + bb];
    T r2 = x * x + y * y + z * z;
    T r = sqrt(r2);
    T f = T(mu0) / (r2 * r);
    T ax = -f * x, ay = -f * y, az = -f * z;
    for (int i = 0; i < nb; ++i) {
      if (i == bb || mu[i] == 0.0) continue;
      T dx = x - X[i], dy = y - X[nb + i], dz = z - X[2 * nb + i];
      T s2 = dx * dx + dy * dy + dz * dz;
      const double rc = std::max(rcrit[bb], rcrit[i]);
      T w = one_minus_k_over_s3(s2, rc) * mu[i];
      ax = ax - w * dx;
      ay = ay - w * dy;
      az = az - w * dz;
    }
    A[bb] = ax; A[nb + bb] = ay; A[2 * nb + bb] = az;
  }
}

// Stoermer's rule over H with n sub-steps; Y = 6 x nb state.
template <class T>
void stoermer(double mu0, int nb, const double* mu, const double* rcrit, const std::vector<T>& Y,
              double H, int n, std::vector<T>& out) {
  const int m3 = 3 * nb;
  const double d = H / n;
  std::vector<T> X(Y.begin(), Y.begin() + m3), A(m3), D(m3);
  bs_accel(mu0, nb, mu, rcrit, X, A);
  for (int k = 0; k < m3; ++k) {
    D[k] = T(d) * (Y[m3 + k] + T(0.5 * d) * A[k]);
    X[k] = X[k] + D[k];
  }
  for (int s = 1; s < n; ++s) {
    bs_accel(mu0, nb, mu, rcrit, X, A);
    for (int k = 0; k < m3; ++k) {
      D[k] = D[k] + T(d * d) * A[k];
      X[k] = X[k] + D[k];
    }
  }
  bs_accel(mu0, nb, mu, rcrit, X, A);
  out.resize(2 * m3);
  for (int k = 0; k < m3; ++k) {
    out[k] = X[k];
    out[m3 + k] = D[k] / d + T(0.5 * d) * A[k];
  }
}

template <class T>
int bs_group(double mu0, int nb, const double* mu, const double* rcrit, std::vector<T>& Y,
             double h, double tol, int max_sub, int* nsub_out) {
  const int KMAX = 8;
  const int m = 6 * nb;
  double rem = h, H = h;
  int nsub = 0;
  std::vector<std::vector<T>> tab(KMAX * KMAX);
  while (rem != 0.0) {
    if (nsub >= max_sub) {
      if (nsub_out) *nsub_out = nsub;
      return ORC_ERR_BS_NOCONV;
    }
    ++nsub;
    if (std::fabs(H) > std::fabs(rem)) H = rem;
    std::vector<double> xscal(nb), vscal(nb);
    for (int b = 0; b < nb; ++b) {
      const double x = val(Y[b]), y = val(Y[nb + b]), z = val(Y[2 * nb + b]);
      const double u = val(Y[3 * nb + b]), v = val(Y[4 * nb + b]), w = val(Y[5 * nb + b]);
      xscal[b] = 1.0 / (x * x + y * y + z * z);
      vscal[b] = 1.0 / (u * u + v * v + w * w);
    }
    bool ok = false;
    int kacc = 0;
    for (int k = 0; k < KMAX && !ok; ++k) {
      const int nk = 2 * (k + 1);
      stoermer(mu0, nb, mu, rcrit, Y, H, nk, tab[k * KMAX + 0]);
      for (int j = 1; j <= k; ++j) {
        const int nkj = 2 * (k - j + 1);
        const double ratio = (double)nk / nkj;
        const double den = ratio * ratio - 1.0;
        const std::vector<T>& a = tab[k * KMAX + j - 1];
        const std::vector<T>& c = tab[(k - 1) * KMAX + j - 1];
        std::vector<T>& o = tab[k * KMAX + j];
        o.resize(m);
        for (int e = 0; e < m; ++e) o[e] = a[e] + (a[e] - c[e]) / den;
      }
      if (k >= 1) {
        const std::vector<T>& best = tab[k * KMAX + k];
        const std::vector<T>& prev = tab[k * KMAX + k - 1];
        double err = 0.0;
        for (int b = 0; b < nb; ++b) {
          double ex = 0.0, ev = 0.0;
          for (int c = 0; c < 3; ++c) {
            const double dx = val(best[c * nb + b]) - val(prev[c * nb + b]);
            const double dv = val(best[(3 + c) * nb + b]) - val(prev[(3 + c) * nb + b]);
            ex += dx * dx;
            ev += dv * dv;
          }
          err = std::max(err, std::max(ex * xscal[b], ev * vscal[b]));
        }
        if (err <= tol * tol) {
          ok = true;
          kacc = k;
        }
      }
    }
    if (ok) {
      Y = tab[kacc * KMAX + kacc];
      rem = rem - H;
      H = 1.3 * H;
    } else {
      H = 0.5 * H;
    }
  }
  if (nsub_out) *nsub_out = nsub;
  return ORC_OK;
}

// Encounter groups (reading; the paper runs one BS call over all encounter
// bodies).  Big bodies joined by flagged big-big pairs form big groups;
// each big group of two or more is integrated on its own and gives its
// members' states.  Every flagged small body forms a test-particle group with
// the big groups of the bigs it is flagged with; only the small body's state
// is taken from it (it is massless, so the bigs' copies follow their own
// motion).  Members are listed bigs ascending, then the small body.
struct Group {
  std::vector<int> members;
  int write_from;  // members[write_from..] receive the BS result
};

std::vector<Group> build_groups(const Bodies& b, const std::vector<std::pair<int, int>>& pairs) {
  std::vector<int> parent(b.nbig);
  for (int i = 0; i < b.nbig; ++i) parent[i] = i;
  auto find = [&](int i) {
    while (parent[i] != i) i = parent[i];
    return i;
  };
  for (auto& pr : pairs) {
    if (pr.second < b.nbig) {
      int ra = find(pr.first), rb = find(pr.second);
      if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
    }
  }
  std::vector<int> root(b.nbig);
  for (int i = 0; i < b.nbig; ++i) root[i] = find(i);
  std::vector<Group> groups;
  std::vector<int> size(b.nbig, 0);
  for (int i = 0; i < b.nbig; ++i) size[root[i]]++;
  for (int r = 0; r < b.nbig; ++r) {
    if (root[r] != r || size[r] < 2) continue;
    Group g;
    for (int i = 0; i < b.nbig; ++i)
      if (root[i] == r) g.members.push_back(i);
    g.write_from = 0;
    groups.push_back(g);
  }
  // small bodies, ascending; the pair list is sorted by (i, j) so collect per j
  std::vector<std::vector<int>> bigs_of(b.nsmall);
  for (auto& pr : pairs)
    if (pr.second >= b.nbig) bigs_of[pr.second - b.nbig].push_back(pr.first);
  for (int s = 0; s < b.nsmall; ++s) {
    if (bigs_of[s].empty()) continue;
    std::vector<char> use_root(b.nbig, 0);
    for (int i : bigs_of[s]) use_root[root[i]] = 1;
    Group g;
    for (int i = 0; i < b.nbig; ++i)
      if (use_root[root[i]]) g.members.push_back(i);
    g.write_from = (int)g.members.size();
    g.members.push_back(b.nbig + s);
    groups.push_back(g);
  }
  return groups;
}

// ----------------------------------------------------------- the full step
// Order (reading; the paper inherits it from Chambers 1999): half kick with
// K-weighted forces plus drag, jump h/2, Kepler drift of every body, detection,
// BS of every encounter group from the pre-drift state (replacing the drift
// for those bodies), jump h/2, half kick.
struct StepStats {
  long long pairs = 0, groups = 0, max_bs_sub = 0, max_kep_iter = 0;
};

template <class T>
int hybrid_step(const orc_params& p, const GasT<T>& g, const Bodies& b, State<T>& s,
                unsigned char* ever, int step_index, int* log, int log_cap, int* log_count,
                StepStats& st) {
  const double h = p.dt;
  const int n = b.n;
  std::vector<T> a[3], ad[3];
  for (int k = 0; k < 3; ++k) { a[k].assign(n, T(0.0)); ad[k].assign(n, T(0.0)); }
  T P[3];
  auto kick = [&]() {
    momentum(b, s, P);
    accel_grav(b, s, a);
    for (int k = 0; k < 3; ++k) std::fill(ad[k].begin(), ad[k].end(), T(0.0));
    accel_drag(g, b, s, P, ad);
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < n; ++j)
        if (!b.gone(j)) s.q[3 + k][j] = s.q[3 + k][j] + T(0.5 * h) * (a[k][j] + ad[k][j]);
  };
  auto jump = [&]() {
    momentum(b, s, P);
    for (int k = 0; k < 3; ++k) {
      T dx = T(0.5 * h) * P[k] / b.mu0;
      for (int j = 0; j < n; ++j)
        if (!b.gone(j)) s.q[k][j] = s.q[k][j] + dx;
    }
  };
  kick();
  jump();
  State<T> s0 = s;
  int itmax = 0;
  int err = drift_all(b.mu0, h, p.kepler_max_iter, s, &itmax, &b);
  st.max_kep_iter = std::max<long long>(st.max_kep_iter, itmax);
  if (err) return err;
  std::vector<double> xv0((size_t)6 * n), xv1((size_t)6 * n);
  store_state(s0, xv0.data());
  store_state(s, xv1.data());
  std::vector<std::pair<int, int>> pairs;
  detect(b, xv0.data(), xv1.data(), h, pairs);
  st.pairs += (long long)pairs.size();
  if ((int)pairs.size() > p.pair_cap) return ORC_ERR_PAIR_OVERFLOW;
  for (auto& pr : pairs) {
    if (ever) { ever[pr.first] = 1; ever[pr.second] = 1; }
    if (log) {
      if (*log_count < log_cap) {
        log[3 * *log_count + 0] = step_index;
        log[3 * *log_count + 1] = pr.first;
        log[3 * *log_count + 2] = pr.second;
      }
      ++*log_count;
    }
  }
  std::vector<Group> groups = build_groups(b, pairs);
  st.groups += (long long)groups.size();
  int gerr = ORC_OK;
  long long gmax = 0;
#pragma omp parallel for schedule(dynamic) reduction(max : gerr, gmax)
  for (int gi = 0; gi < (int)groups.size(); ++gi) {
    const Group& gr = groups[gi];
    const int nb = (int)gr.members.size();
    std::vector<double> mu(nb), rc(nb);
    std::vector<T> Y((size_t)6 * nb);
    for (int m = 0; m < nb; ++m) {
      const int j = gr.members[m];
      mu[m] = b.mu[j];
      rc[m] = b.rcrit[j];
      for (int k = 0; k < 6; ++k) Y[(size_t)k * nb + m] = s0.q[k][j];
    }
    int nsub = 0;
    int e = bs_group(b.mu0, nb, mu.data(), rc.data(), Y, h, p.bs_tol, p.bs_max_sub, &nsub);
    gmax = std::max<long long>(gmax, nsub);
    if (e) gerr = std::max(gerr, e);
    for (int m = gr.write_from; m < nb; ++m) {
      const int j = gr.members[m];
      for (int k = 0; k < 6; ++k) s.q[k][j] = Y[(size_t)k * nb + m];
    }
  }
  st.max_bs_sub = std::max(st.max_bs_sub, gmax);
  if (gerr) return gerr;
  jump();
  kick();
  for (int k = 0; k < 6; ++k)
    for (int j = 0; j < n; ++j)
      if (!std::isfinite(val(s.q[k][j]))) return ORC_ERR_NONFINITE;
  return ORC_OK;
}

// ------------------------------------- orbital elements and ejection (Sec. 3.5)
// Osculating elements of one body about gm (G(m0 + m) for a massive body,
// G m0 for a planetesimal, Sec. 3.5), from the two-body relations (Murray &
// Dermott 1999, Sec. 2.8):
//   angular momentum h = x cross v, semilatus rectum p = |h|^2/gm;
//   eccentricity vector (v cross h)/gm - x/r, e its length;
//   q = p/(1 + e); cos i = h_z/|h|; node Omega = atan2(h_x, -h_y);
//   argument of latitude u = angle of x from the node line in the orbit plane;
//   true anomaly f from e cos f = p/r - 1, e sin f = |h| (x.v)/(gm r);
//   longitude of pericentre varpi = Omega + u - f;
//   mean anomaly from the eccentric anomaly E (e < 1, M = E - e sin E), the
//   hyperbolic anomaly F (e > 1, M = e sinh F - F) or, for e = 1, Barker's
//   D + D^3/3 with D = tan(f/2).
// Conventions for the degenerate cases: Omega = 0 when the orbit lies in the
// reference plane, f = 0 when e = 0.  Angles Omega, varpi and the elliptic M
// are reduced to [0, 2 pi).
struct Elements {
  double q, e, i, varpi, node, M;
};

double wrap_2pi(double a) {
  a = std::fmod(a, 2.0 * kPi);
  return a < 0.0 ? a + 2.0 * kPi : a;
}

Elements x2el(double gm, const double* x, const double* v) {
  Elements el;
  const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  const double hx = x[1] * v[2] - x[2] * v[1];
  const double hy = x[2] * v[0] - x[0] * v[2];
  const double hz = x[0] * v[1] - x[1] * v[0];
  const double hxy = std::sqrt(hx * hx + hy * hy);
  const double h = std::sqrt(hx * hx + hy * hy + hz * hz);
  const double p = h * h / gm;
  const double ex = (v[1] * hz - v[2] * hy) / gm - x[0] / r;
  const double ey = (v[2] * hx - v[0] * hz) / gm - x[1] / r;
  const double ez = (v[0] * hy - v[1] * hx) / gm - x[2] / r;
  const double e = std::sqrt(ex * ex + ey * ey + ez * ez);
  el.e = e;
  el.q = p / (1.0 + e);
  el.i = std::atan2(hxy, hz);
  const double node = (hxy > 0.0) ? std::atan2(hx, -hy) : 0.0;
  el.node = wrap_2pi(node);
  const double cn = std::cos(node), sn = std::sin(node);
  const double ci = (h > 0.0) ? hz / h : 1.0, si = (h > 0.0) ? hxy / h : 0.0;
  // in-plane axes: the node line and the direction 90 degrees ahead of it
  const double along = x[0] * cn + x[1] * sn;
  const double ahead = (-x[0] * sn + x[1] * cn) * ci + x[2] * si;
  const double u = std::atan2(ahead, along);
  const double rv = x[0] * v[0] + x[1] * v[1] + x[2] * v[2];
  const double ecf = p / r - 1.0, esf = h * rv / (gm * r);
  const double f = (e > 0.0) ? std::atan2(esf, ecf) : 0.0;
  el.varpi = wrap_2pi(node + u - f);
  if (e < 1.0) {
    const double E = std::atan2(std::sqrt(1.0 - e * e) * std::sin(f), e + std::cos(f));
    el.M = wrap_2pi(E - e * std::sin(E));
  } else if (e > 1.0) {
    const double F = std::asinh(std::sqrt(e * e - 1.0) * std::sin(f) / (1.0 + e * std::cos(f)));
    el.M = e * std::sinh(F) - F;
  } else {
    const double D = std::tan(0.5 * f);
    el.M = D + D * D * D / 3.0;
  }
  return el;
}

// The ejection test of Sec. 3.5: a body still in the integration whose
// osculating heliocentric eccentricity is 1 or more is flagged (stat -3) and
// a massive one loses its mass (mu 0).  Heliocentric velocities are
// v_b + P/m0 with the massive-body momentum P of the state as given, taken
// once for all bodies.
int eject_check(Bodies& b, const State<double>& s) {
  double P[3];
  momentum(b, s, P);
  int removed = 0;
  for (int j = 0; j < b.n; ++j) {
    if (b.gone(j)) continue;
    const double x[3] = {s.q[0][j], s.q[1][j], s.q[2][j]};
    double vh[3];
    for (int k = 0; k < 3; ++k) vh[k] = s.q[3 + k][j] + P[k] / b.mu0;
    const double gm = (j < b.nbig) ? b.mu0 + b.mu[j] : b.mu0;
    if (x2el(gm, x, vh).e >= 1.0) {
      b.stat[j] = -3;
      if (j < b.nbig) b.mu[j] = 0.0;
      ++removed;
    }
  }
  return removed;
}

// ------------------------------------------ planet growth (Secs. 3.1, 3.3)
// Eq. 13 (core phase, t <= tau_c) and Eq. 15 (runaway gas accretion after
// it); the two meet at M_c, since (e/(e - 1))(1 - 1/e) = 1.
constexpr double kEuler = 2.718281828459045235360287;

double growth_mass(const orc_growth& g, double t) {
  if (t <= g.tau_c)
    return g.m0 + (kEuler / (kEuler - 1.0)) * (g.mc - g.m0) * (1.0 - std::exp(-t / g.tau_c));
  return g.mc + (g.mf - g.mc) * (1.0 - std::exp(-(t - g.tau_c) / g.tau_g));
}

// Eq. 14 with k1 = 1 and k2 = 1/4: R_p = G M / (c_s^2/k1 + G M/(k2 R_H)).
double inflated_radius(double gm, double cs, double rh) {
  return gm / (cs * cs / 1.0 + gm / (0.25 * rh));
}

struct GrowOut {
  double mu, rcrit, gap_w, gap_f, radius;
};

// Growth quantities of massive body i at time t (see orc_grow_state).  P is
// the momentum of the state with the masses it has now.
GrowOut grow_one(const orc_params& p, double mu0, const orc_growth& g, const double* x,
                 const double* vb, const double P[3], double t, double gap_c) {
  GrowOut o;
  const double M = growth_mass(g, t);
  o.mu = p.G * M;
  double vh[3];
  for (int k = 0; k < 3; ++k) vh[k] = vb[k] + P[k] / mu0;
  const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  const double v2 = vh[0] * vh[0] + vh[1] * vh[1] + vh[2] * vh[2];
  double a = 1.0 / (2.0 / r - v2 / (mu0 + o.mu));
  if (!(a > 0.0)) a = r;
  const double rh = a * std::cbrt(o.mu / (3.0 * mu0));
  o.rcrit = p.rcrit_hill * rh;
  const bool runaway = t > g.tau_c;
  o.gap_w = runaway ? gap_c * rh : 0.0;
  o.gap_f = runaway ? std::exp(-(t - g.tau_c) / g.tau_g) : 1.0;
  // sound speed at the body's cylindrical distance (the disk of Sec. 3.1)
  const double R = std::sqrt(x[0] * x[0] + x[1] * x[1]);
  const double cs = p.gas.hr_1au * std::pow(R, p.gas.flare) * std::sqrt(mu0 / R);
  if (!runaway) {
    o.radius = inflated_radius(o.mu, cs, rh);
  } else {   // R_c: Eq. 14 as it stood at tau_c, the mass M_c, on the current orbit
    const double muc = p.G * g.mc;
    double ac = 1.0 / (2.0 / r - v2 / (mu0 + muc));
    if (!(ac > 0.0)) ac = r;
    const double rc = inflated_radius(muc, cs, ac * std::cbrt(muc / (3.0 * mu0)));
    o.radius = rc - g.delta_r * (1.0 - std::exp(-(t - g.tau_c) / g.tau_g));
  }
  return o;
}

// Applies the growth tracks at time t to the bodies (mu, rcrit, gaps).
void grow_bodies(const orc_params& p, Bodies& b, const State<double>& s, const orc_growth* g,
                 double gap_c, double t) {
  double P[3];
  momentum(b, s, P);
  b.gap_w.assign(b.nbig, 0.0);
  b.gap_f.assign(b.nbig, 1.0);
  for (int i = 0; i < b.nbig; ++i) {
    if (!g[i].grows || b.gone(i)) continue;
    const double x[3] = {s.q[0][i], s.q[1][i], s.q[2][i]};
    const double v[3] = {s.q[3][i], s.q[4][i], s.q[5][i]};
    const GrowOut o = grow_one(p, b.mu0, g[i], x, v, P, t, gap_c);
    b.mu[i] = o.mu;
    b.rcrit[i] = o.rcrit;
    b.gap_w[i] = o.gap_w;
    b.gap_f[i] = o.gap_f;
  }
}

// ------------------------------------------------------ set-up and readout
double semimajor_of(double gm, const double* x, const double* v) {
  const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  return 1.0 / (2.0 / r - v2 / gm);
}

template <class T>
T semimajor_t(double gm, const T* x, const T* v) {
  T r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  T v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  return T(1.0) / (T(2.0) / r - v2 / gm);
}

bool make_bodies(const orc_params* p, int nbig, int nsmall, const double* mu, const double* rcrit,
                 const double* rp_km, const double* rhop, Bodies& b) {
  if (!p || nbig < 0 || nsmall < 0) return false;
  b.nbig = nbig;
  b.nsmall = nsmall;
  b.n = nbig + nsmall;
  b.mu0 = p->G * p->m_star;
  b.mu.assign(mu, mu + b.n);
  b.rcrit.assign(rcrit, rcrit + b.n);
  b.rp_km.assign(nsmall, 1.0);
  b.rhop.assign(nsmall, 1.0);
  if (rp_km) b.rp_km.assign(rp_km, rp_km + nsmall);
  if (rhop) b.rhop.assign(rhop, rhop + nsmall);
  return true;
}

template <class T>
GasT<T> make_gas(const orc_gas& raw, double G) {
  GasT<T> g;
  g.raw = raw;
  g.G = G;
  g.sigma1 = T(raw.sigma1_gcm2);
  g.gamma = T(raw.gamma);
  g.cd_scale = T(raw.cd_scale);
  return g;
}

}  // namespace

// =================================================================== C API
extern "C" {

void orc_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

double orc_changeover(double s, double rc) { return changeover_K(s, rc); }
double orc_k_over_s3(double s2, double rc) { return k_over_s3(s2, rc); }

int orc_init(const orc_params* p, int nbig, int nsmall, const double* m_big,
             const double* xv_helio, double* xv_dh, double* mu, double* rcrit) {
  if (!p || nbig < 0 || nsmall < 0 || !xv_helio || !xv_dh || !mu || !rcrit) return ORC_ERR_ARG;
  const int n = nbig + nsmall;
  const double mu0 = p->G * p->m_star;
  double msum = 0.0, mv[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < nbig; ++i) {
    msum += m_big[i];
    for (int k = 0; k < 3; ++k) mv[k] += m_big[i] * xv_helio[(size_t)(3 + k) * n + i];
  }
  // Barycentric velocity of the star is -sum m_i v_h,i / M_total; every
  // body's barycentric velocity is its heliocentric one plus that.
  const double mtot = p->m_star + msum;
  for (int k = 0; k < 3; ++k) {
    const double V = mv[k] / mtot;
    for (int j = 0; j < n; ++j) {
      xv_dh[(size_t)k * n + j] = xv_helio[(size_t)k * n + j];
      xv_dh[(size_t)(3 + k) * n + j] = xv_helio[(size_t)(3 + k) * n + j] - V;
    }
  }
  for (int j = 0; j < n; ++j) {
    mu[j] = (j < nbig) ? p->G * m_big[j] : 0.0;
    rcrit[j] = 0.0;
  }
  // Changeover radius: rcrit_hill Hill radii, R_H = a (mu/(3 mu0))^(1/3) with
  // the osculating a at t = 0 (gm = mu0 + mu, as for big bodies in Sec. 3.5).
  for (int i = 0; i < nbig; ++i) {
    double x[3], v[3];
    for (int k = 0; k < 3; ++k) {
      x[k] = xv_helio[(size_t)k * n + i];
      v[k] = xv_helio[(size_t)(3 + k) * n + i];
    }
    double a = semimajor_of(mu0 + mu[i], x, v);
    if (!(a > 0.0)) a = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    rcrit[i] = p->rcrit_hill * a * std::cbrt(mu[i] / (3.0 * mu0));
  }
  return ORC_OK;
}

int orc_readout(const orc_params* p, int nbig, int nsmall, const double* mu, const double* xv_dh,
                double* xv_helio) {
  if (!p || !mu || !xv_dh || !xv_helio) return ORC_ERR_ARG;
  const int n = nbig + nsmall;
  const double mu0 = p->G * p->m_star;
  for (int k = 0; k < 3; ++k) {
    double P = 0.0;
    for (int i = 0; i < nbig; ++i) P += mu[i] * xv_dh[(size_t)(3 + k) * n + i];
    for (int j = 0; j < n; ++j) {
      xv_helio[(size_t)k * n + j] = xv_dh[(size_t)k * n + j];
      xv_helio[(size_t)(3 + k) * n + j] = xv_dh[(size_t)(3 + k) * n + j] + P / mu0;
    }
  }
  return ORC_OK;
}

int orc_accel_grav(int nbig, int n, const double* xv, const double* mu, const double* rcrit,
                   double* acc, int triangular) {
  if (nbig < 0 || n < nbig || !xv || !mu || !rcrit || !acc) return ORC_ERR_ARG;
  Bodies b;
  b.nbig = nbig; b.n = n; b.nsmall = n - nbig;
  b.mu.assign(mu, mu + n);
  b.rcrit.assign(rcrit, rcrit + n);
  State<double> s;
  load_state(s, n, xv);
  std::vector<double> a[3];
  for (auto& v : a) v.assign(n, 0.0);
  if (triangular) accel_grav_triangular(b, s, a);
  else accel_grav(b, s, a);
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < n; ++j) acc[(size_t)k * n + j] = a[k][j];
  return ORC_OK;
}

int orc_momentum(int nbig, int n, const double* xv, const double* mu, double* P3) {
  if (!xv || !mu || !P3) return ORC_ERR_ARG;
  for (int k = 0; k < 3; ++k) {
    double acc = 0.0;
    for (int i = 0; i < nbig; ++i) acc += mu[i] * xv[(size_t)(3 + k) * n + i];
    P3[k] = acc;
  }
  return ORC_OK;
}

int orc_gas_state(const orc_params* p, double R, double* out8) {
  if (!p || !out8 || !(R > 0.0)) return ORC_ERR_ARG;
  GasT<double> g = make_gas<double>(p->gas, p->G);
  DiskAt<double> d = disk_at(g, p->G * p->m_star, R);
  out8[0] = d.sigma; out8[1] = d.rho_g; out8[2] = d.H_au; out8[3] = d.cs;
  out8[4] = d.vk; out8[5] = d.eta; out8[6] = d.vg; out8[7] = d.hr;
  return ORC_OK;
}

double orc_drag_cd(double Re, double Ma, int cd_mode) { return drag_cd(Re, Ma, cd_mode); }

double orc_dg_series(double gamma) { return dg_series(gamma); }
double orc_dg_series_dgamma(double gamma) { return dg_series_dgamma(gamma); }

int orc_disk_gravity(const orc_params* p, const double* x3, double* acc3) {
  if (!p || !x3 || !acc3) return ORC_ERR_ARG;
  GasT<double> g = make_gas<double>(p->gas, p->G);
  acc3[0] = acc3[1] = acc3[2] = 0.0;
  disk_gravity_one(g, p->G * p->m_star, x3, acc3);
  return ORC_OK;
}

int orc_drag_one(const orc_params* p, const double* x3, const double* vh3, double rp_km,
                 double rhop, double* acc3, double* re_ma2) {
  if (!p || !x3 || !vh3 || !acc3) return ORC_ERR_ARG;
  GasT<double> g = make_gas<double>(p->gas, p->G);
  drag_one(g, p->G * p->m_star, x3, vh3, rp_km, rhop, acc3, re_ma2);
  return ORC_OK;
}

int orc_gas_drag(const orc_params* p, int nbig, int nsmall, const double* xv, const double* mu,
                 const double* rp_km, const double* rhop, double* acc_small) {
  return orc_gas_drag_gap(p, nbig, nsmall, xv, mu, rp_km, rhop, nullptr, nullptr, acc_small);
}

int orc_gas_drag_gap(const orc_params* p, int nbig, int nsmall, const double* xv,
                     const double* mu, const double* rp_km, const double* rhop,
                     const double* gap_w, const double* gap_f, double* acc_small) {
  if (!p || !xv || !mu || !rp_km || !rhop || !acc_small || (!gap_w != !gap_f)) return ORC_ERR_ARG;
  const int n = nbig + nsmall;
  std::vector<double> zero(n, 0.0);
  Bodies b;
  make_bodies(p, nbig, nsmall, mu, zero.data(), rp_km, rhop, b);
  if (gap_w) {
    b.gap_w.assign(gap_w, gap_w + nbig);
    b.gap_f.assign(gap_f, gap_f + nbig);
  }
  State<double> s;
  load_state(s, n, xv);
  GasT<double> g = make_gas<double>(p->gas, p->G);
  double P[3];
  momentum(b, s, P);
  std::vector<double> a[3];
  for (auto& v : a) v.assign(n, 0.0);
  accel_drag(g, b, s, P, a);
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < nsmall; ++j) acc_small[(size_t)k * nsmall + j] = a[k][nbig + j];
  return ORC_OK;
}

void orc_stumpff(double z, double* c4) { stumpff(z, c4); }

int orc_drift(const orc_params* p, int n, double* xv, double h, int* iters_max) {
  if (!p || !xv || n < 0) return ORC_ERR_ARG;
  State<double> s;
  load_state(s, n, xv);
  int it = 0;
  int e = drift_all(p->G * p->m_star, h, p->kepler_max_iter, s, &it);
  store_state(s, xv);
  if (iters_max) *iters_max = it;
  return e;
}

double orc_hermite_d2min(double d0, double d1, double d0t, double d1t, double h) {
  return hermite_d2min(d0, d1, d0t, d1t, h);
}

int orc_detect(const orc_params* p, int nbig, int n, const double* xv0, const double* xv1,
               const double* rcrit, unsigned char* flags, int* pairs, int cap, int* npairs) {
  if (!p || !xv0 || !xv1 || !rcrit || !npairs || cap < 0) return ORC_ERR_ARG;
  Bodies b;
  b.nbig = nbig; b.n = n; b.nsmall = n - nbig;
  b.rcrit.assign(rcrit, rcrit + n);
  std::vector<std::pair<int, int>> pr;
  detect(b, xv0, xv1, p->dt, pr);
  *npairs = (int)pr.size();
  if (flags) {
    std::memset(flags, 0, (size_t)n);
    for (auto& q : pr) flags[q.first] = flags[q.second] = 1;
  }
  if (pairs)
    for (int k = 0; k < (int)pr.size() && k < cap; ++k) {
      pairs[2 * k] = pr[k].first;
      pairs[2 * k + 1] = pr[k].second;
    }
  return (int)pr.size() > cap ? ORC_ERR_PAIR_OVERFLOW : ORC_OK;
}

// Encounter groups of one step from its flagged pairs (big index first, each
// pair once, as orc_detect lists them).  Writes each group's members, bigs
// ascending then the planetesimal, back to back in members[], the start of
// group g at offsets[g] (offsets[ngroups] = total) and the first member that
// receives the group's result at write_from[g].  Big groups come first (root
// order), then the planetesimals' groups in planetesimal order.
int orc_build_groups(int nbig, int nsmall, int npairs, const int* pairs, int cap_groups,
                     int cap_members, int* members, int* offsets, int* write_from,
                     int* ngroups) {
  if (nbig < 0 || nsmall < 0 || npairs < 0 || (npairs > 0 && !pairs) || !ngroups)
    return ORC_ERR_ARG;
  Bodies b;
  b.nbig = nbig; b.nsmall = nsmall; b.n = nbig + nsmall;
  std::vector<std::pair<int, int>> pr((size_t)npairs);
  for (int k = 0; k < npairs; ++k) {
    const int i = pairs[2 * k], j = pairs[2 * k + 1];
    if (i < 0 || i >= nbig || j <= i || j >= b.n) return ORC_ERR_ARG;
    pr[k] = {i, j};
  }
  std::vector<Group> g = build_groups(b, pr);
  *ngroups = (int)g.size();
  size_t tot = 0;
  for (auto& q : g) tot += q.members.size();
  if ((int)g.size() > cap_groups || (long long)tot > cap_members) return ORC_ERR_PAIR_OVERFLOW;
  if (!members || !offsets || !write_from) return ORC_ERR_ARG;
  int o = 0;
  for (size_t k = 0; k < g.size(); ++k) {
    offsets[k] = o;
    write_from[k] = g[k].write_from;
    for (int m : g[k].members) members[o++] = m;
  }
  offsets[g.size()] = o;
  return ORC_OK;
}

int orc_bs_group(const orc_params* p, int nb, const double* mu, const double* rcrit, double* xv,
                 double h, int* nsub) {
  if (!p || nb <= 0 || !mu || !rcrit || !xv) return ORC_ERR_ARG;
  std::vector<double> Y(xv, xv + (size_t)6 * nb);
  int e = bs_group(p->G * p->m_star, nb, mu, rcrit, Y, h, p->bs_tol, p->bs_max_sub, nsub);
  std::copy(Y.begin(), Y.end(), xv);
  return e;
}

int orc_step(const orc_params* p, int nbig, int nsmall, double* xv, const double* mu,
             const double* rcrit, const double* rp_km, const double* rhop, int nsteps,
             unsigned char* ever_flag, int* pair_log, int log_cap, int* log_count,
             long long* stats) {
  Bodies b;
  if (!xv || !mu || !rcrit || nsteps < 0 || !make_bodies(p, nbig, nsmall, mu, rcrit, rp_km, rhop, b))
    return ORC_ERR_ARG;
  if (p->gas.enabled && nsmall > 0 && (!rp_km || !rhop)) return ORC_ERR_ARG;
  State<double> s;
  load_state(s, b.n, xv);
  GasT<double> g = make_gas<double>(p->gas, p->G);
  StepStats st;
  int lc = 0;
  int err = ORC_OK;
  if (p->eject_every > 0) b.stat.assign(b.n, 0);   // removals stay local (see orc_step_ex)
  for (int k = 0; k < nsteps && !err; ++k) {
    err = hybrid_step(*p, g, b, s, ever_flag, k, pair_log, log_cap, &lc, st);
    if (!err && p->eject_every > 0 && (k + 1) % p->eject_every == 0) eject_check(b, s);
  }
  store_state(s, xv);
  if (log_count) *log_count = lc;
  if (stats) {
    stats[0] = st.pairs; stats[1] = st.groups; stats[2] = st.max_bs_sub; stats[3] = st.max_kep_iter;
  }
  return err;
}

int orc_step_ex(const orc_params* p, int nbig, int nsmall, double* xv, double* mu,
                double* rcrit, const double* rp_km, const double* rhop, int nsteps,
                long long step0, signed char* stat, const orc_growth* growth, double gap_c,
                unsigned char* ever_flag, long long* stats) {
  Bodies b;
  if (!xv || !mu || !rcrit || !stat || nsteps < 0 || step0 < 0 || p->eject_every < 0 ||
      !make_bodies(p, nbig, nsmall, mu, rcrit, rp_km, rhop, b))
    return ORC_ERR_ARG;
  if (p->gas.enabled && nsmall > 0 && (!rp_km || !rhop)) return ORC_ERR_ARG;
  b.stat.assign(stat, stat + b.n);
  State<double> s;
  load_state(s, b.n, xv);
  GasT<double> g = make_gas<double>(p->gas, p->G);
  StepStats st;
  int lc = 0;
  int err = ORC_OK;
  for (int k = 0; k < nsteps && !err; ++k) {
    if (growth) grow_bodies(*p, b, s, growth, gap_c, (double)(step0 + k) * p->dt);
    err = hybrid_step(*p, g, b, s, ever_flag, k, nullptr, 0, &lc, st);
    if (!err && p->eject_every > 0 && (step0 + k + 1) % p->eject_every == 0) eject_check(b, s);
  }
  store_state(s, xv);
  std::copy(b.mu.begin(), b.mu.end(), mu);
  std::copy(b.rcrit.begin(), b.rcrit.end(), rcrit);
  std::copy(b.stat.begin(), b.stat.end(), stat);
  if (stats) {
    stats[0] = st.pairs; stats[1] = st.groups; stats[2] = st.max_bs_sub; stats[3] = st.max_kep_iter;
  }
  return err;
}

int orc_grow_state(const orc_params* p, int nbig, int n, const double* xv, const double* mu,
                   const double* rcrit, const orc_growth* g, double gap_c, double t,
                   double* mu_out, double* rcrit_out, double* gap_w, double* gap_f,
                   double* radius) {
  if (!p || !xv || !mu || !rcrit || !g || nbig < 0 || n < nbig) return ORC_ERR_ARG;
  Bodies b;
  b.nbig = nbig;
  b.nsmall = n - nbig;
  b.n = n;
  b.mu0 = p->G * p->m_star;
  b.mu.assign(mu, mu + n);
  State<double> s;
  load_state(s, n, xv);
  double P[3];
  momentum(b, s, P);
  for (int i = 0; i < nbig; ++i) {
    GrowOut o{mu[i], rcrit[i], 0.0, 1.0, 0.0};
    if (g[i].grows) {
      const double x[3] = {s.q[0][i], s.q[1][i], s.q[2][i]};
      const double v[3] = {s.q[3][i], s.q[4][i], s.q[5][i]};
      o = grow_one(*p, b.mu0, g[i], x, v, P, t, gap_c);
    }
    if (mu_out) mu_out[i] = o.mu;
    if (rcrit_out) rcrit_out[i] = o.rcrit;
    if (gap_w) gap_w[i] = o.gap_w;
    if (gap_f) gap_f[i] = o.gap_f;
    if (radius) radius[i] = o.radius;
  }
  return ORC_OK;
}

int orc_eject(const orc_params* p, int nbig, int n, const double* xv, double* mu,
              signed char* stat, int* n_new) {
  Bodies b;
  if (!p || !xv || !mu || !stat || nbig < 0 || n < nbig) return ORC_ERR_ARG;
  b.nbig = nbig;
  b.nsmall = n - nbig;
  b.n = n;
  b.mu0 = p->G * p->m_star;
  b.mu.assign(mu, mu + n);
  b.stat.assign(stat, stat + n);
  State<double> s;
  load_state(s, n, xv);
  const int k = eject_check(b, s);
  std::copy(b.mu.begin(), b.mu.end(), mu);
  std::copy(b.stat.begin(), b.stat.end(), stat);
  if (n_new) *n_new = k;
  return ORC_OK;
}

int orc_elements(int n, const double* gm, const double* xv, double* out) {
  if (n < 0 || !gm || !xv || !out) return ORC_ERR_ARG;
  for (int j = 0; j < n; ++j) {
    double x[3], v[3];
    for (int k = 0; k < 3; ++k) {
      x[k] = xv[(size_t)k * n + j];
      v[k] = xv[(size_t)(3 + k) * n + j];
    }
    const Elements el = x2el(gm[j], x, v);
    const double o[6] = {el.q, el.e, el.i, el.varpi, el.node, el.M};
    for (int k = 0; k < 6; ++k) out[(size_t)k * n + j] = o[k];
  }
  return ORC_OK;
}

int orc_energy(const orc_params* p, int nbig, int n, const double* xv, const double* mu, double* E,
               double* L3) {
  if (!p || !xv || !mu || !E || !L3) return ORC_ERR_ARG;
  const double G = p->G, mu0 = G * p->m_star;
  double ke = 0.0, P[3] = {0, 0, 0}, pe = 0.0, L[3] = {0, 0, 0};
  for (int i = 0; i < nbig; ++i) {
    if (mu[i] == 0.0) continue;
    const double x = xv[i], y = xv[n + i], z = xv[2 * (size_t)n + i];
    const double u = xv[3 * (size_t)n + i], v = xv[4 * (size_t)n + i], w = xv[5 * (size_t)n + i];
    const double m = mu[i] / G;
    ke += 0.5 * m * (u * u + v * v + w * w);
    P[0] += m * u; P[1] += m * v; P[2] += m * w;
    pe -= mu0 * m / std::sqrt(x * x + y * y + z * z);
    L[0] += m * (y * w - z * v);
    L[1] += m * (z * u - x * w);
    L[2] += m * (x * v - y * u);
    for (int j = i + 1; j < nbig; ++j) {
      if (mu[j] == 0.0) continue;
      const double dx = xv[j] - x, dy = xv[n + j] - y, dz = xv[2 * (size_t)n + j] - z;
      pe -= m * mu[j] / std::sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
  ke += (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / (2.0 * p->m_star);
  *E = ke + pe;
  for (int k = 0; k < 3; ++k) L3[k] = L[k];
  return ORC_OK;
}

int orc_semimajor(const orc_params* p, int nbig, int n, const double* mu, const double* xv_helio,
                  double* a) {
  if (!p || !mu || !xv_helio || !a) return ORC_ERR_ARG;
  const double mu0 = p->G * p->m_star;
  for (int j = 0; j < n; ++j) {
    double x[3], v[3];
    for (int k = 0; k < 3; ++k) {
      x[k] = xv_helio[(size_t)k * n + j];
      v[k] = xv_helio[(size_t)(3 + k) * n + j];
    }
    a[j] = semimajor_of(j < nbig ? mu0 + mu[j] : mu0, x, v);
  }
  return ORC_OK;
}

int orc_jvp_loss(const orc_params* p, int nbig, int nsmall, const double* m_big,
                 const double* xv_helio, const double* rp_km, const double* rhop, const double* w,
                 int nsteps, const double* dxv, const double* dpar, double* L, double* dL) {
  if (!p || !m_big || !xv_helio || !w || !dxv || !dpar || !L || !dL) return ORC_ERR_ARG;
  const int n = nbig + nsmall;
  std::vector<double> xv_dh((size_t)6 * n), mu(n), rcrit(n);
  int e = orc_init(p, nbig, nsmall, m_big, xv_helio, xv_dh.data(), mu.data(), rcrit.data());
  if (e) return e;
  Bodies b;
  make_bodies(p, nbig, nsmall, mu.data(), rcrit.data(), rp_km, rhop, b);
  // Seeded input in dual form; the heliocentric -> DH map is linear in v.
  State<Dual> hel;
  hel.resize(n);
  for (int k = 0; k < 6; ++k)
    for (int j = 0; j < n; ++j)
      hel.q[k][j] = Dual(xv_helio[(size_t)k * n + j], dxv[(size_t)k * n + j]);
  const double mu0 = b.mu0;
  double msum = 0.0;
  for (int i = 0; i < nbig; ++i) msum += m_big[i];
  const double mtot = p->m_star + msum;
  State<Dual> s;
  s.resize(n);
  for (int k = 0; k < 3; ++k) {
    Dual mv(0.0);
    for (int i = 0; i < nbig; ++i) mv = mv + m_big[i] * hel.q[3 + k][i];
    Dual V = mv / mtot;
    for (int j = 0; j < n; ++j) {
      s.q[k][j] = hel.q[k][j];
      s.q[3 + k][j] = hel.q[3 + k][j] - V;
    }
  }
  GasT<Dual> g;
  g.raw = p->gas;
  g.G = p->G;
  g.sigma1 = Dual(p->gas.sigma1_gcm2, dpar[0]);
  g.gamma = Dual(p->gas.gamma, dpar[1]);
  g.cd_scale = Dual(p->gas.cd_scale, dpar[2]);
  StepStats st;
  int lc = 0;
  for (int k = 0; k < nsteps; ++k) {
    e = hybrid_step(*p, g, b, s, nullptr, k, nullptr, 0, &lc, st);
    if (e) return e;
  }
  Dual P[3];
  momentum(b, s, P);
  Dual loss(0.0);
  for (int j = nbig; j < n; ++j) {
    if (w[j - nbig] == 0.0) continue;
    Dual xi[3] = {hel.q[0][j], hel.q[1][j], hel.q[2][j]};
    Dual vi[3] = {hel.q[3][j], hel.q[4][j], hel.q[5][j]};
    Dual xf[3] = {s.q[0][j], s.q[1][j], s.q[2][j]};
    Dual vf[3];
    for (int k = 0; k < 3; ++k) vf[k] = s.q[3 + k][j] + P[k] / mu0;
    Dual da = semimajor_t(mu0, xf, vf) - semimajor_t(mu0, xi, vi);
    loss = loss + w[j - nbig] * da * da;
  }
  *L = loss.v;
  *dL = loss.d;
  return ORC_OK;
}

}  // extern "C"
