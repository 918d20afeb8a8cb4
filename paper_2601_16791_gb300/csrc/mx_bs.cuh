// mx_bs.cuh -- the thread Bulirsch-Stoer integrator of an encounter group
// (arXiv 2601.16791, Sec. 2: mdt_bs2 for the bodies of a close encounter):
// Stoermer's rule for y'' = f(y) with n_k = 2(k+1) sub-steps, Aitken-Neville
// extrapolation in (H/n)^2, the error of the Sec. 2.1.1 listing (xscal =
// 1/|x|^2, vscal = 1/|v|^2) against tol^2, growth by 1.3 after an accepted
// macro sub-step and halving after a failure.  Forces: the star plus the
// (1 - K)-weighted pair forces of the massive members (the complement of the
// kick's changeover weight).  Shared by the step's large groups (k_bs.cu) and
// by the adjoint, which records the accepted sequence (k_adj_bs.cu).
#pragma once
#include "mx_common.cuh"

namespace mx {

struct GroupState {
  int nb;
  double mu[kMaxGroup], rc[kMaxGroup];
};

// a = -mu0 x/|x|^3 + sum over massive members i of -(1-K)/s^3 mu_i (x - x_i).
__device__ __forceinline__ void bs_accel(const GroupState& G, double mu0,
                                         const double (*X)[kMaxGroup], double (*A)[kMaxGroup]) {
  for (int b = 0; b < G.nb; ++b) {
    const double x = X[0][b], y = X[1][b], z = X[2][b];
    const double ir = rsqrt_d(fma(x, x, fma(y, y, z * z)));
    const double f = mu0 * ir * ir * ir;
    double ax = -f * x, ay = -f * y, az = -f * z;
    for (int i = 0; i < G.nb; ++i) {
      if (i == b || G.mu[i] == 0.0) continue;
      const double dx = x - X[0][i], dy = y - X[1][i], dz = z - X[2][i];
      const double s2 = fma(dx, dx, fma(dy, dy, dz * dz));
      const double rc = fmax(G.rc[b], G.rc[i]);
      const double rc2 = rc * rc;
      if (s2 >= rc2) continue;
      const double yy = rsqrt_d(s2);
      double w = yy * yy * yy;
      if (s2 > 0.01 * rc2) {
        const double q = (s2 * yy - 0.1 * rc) / (0.9 * rc);
        w *= 1.0 - q * q * q * fma(q, fma(6.0, q, -15.0), 10.0);
      }
      w *= G.mu[i];
      ax = fma(-w, dx, ax);
      ay = fma(-w, dy, ay);
      az = fma(-w, dz, az);
    }
    A[0][b] = ax;
    A[1][b] = ay;
    A[2][b] = az;
  }
}

// Stoermer's rule over H with n sub-steps from Y (6 x nb) into O.
static __device__ void stoermer(const GroupState& G, double mu0, const double (*Y)[kMaxGroup], double H,
                         int n, double (*O)[kMaxGroup]) {
  double X[3][kMaxGroup], A[3][kMaxGroup], D[3][kMaxGroup];
  const double dd = H / n;
  const double d2 = dd * dd;
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < G.nb; ++b) X[c][b] = Y[c][b];
  bs_accel(G, mu0, X, A);
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < G.nb; ++b) {
      D[c][b] = dd * fma(0.5 * dd, A[c][b], Y[3 + c][b]);
      X[c][b] += D[c][b];
    }
  for (int s = 1; s < n; ++s) {
    bs_accel(G, mu0, X, A);
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < G.nb; ++b) {
        D[c][b] = fma(d2, A[c][b], D[c][b]);
        X[c][b] += D[c][b];
      }
  }
  bs_accel(G, mu0, X, A);
  const double idd = 1.0 / dd;
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < G.nb; ++b) {
      O[c][b] = X[c][b];
      O[3 + c][b] = fma(D[c][b], idd, 0.5 * dd * A[c][b]);
    }
}

// 1 / ((n_k / n_{k-j})^2 - 1) with n_k = 2(k+1)
__device__ __forceinline__ double inv_den(int k, int j) {
  const double r = (double)(k + 1) / (double)(k - j + 1);
  return 1.0 / (r * r - 1.0);
}

// rec(H, kacc, Ystart) is called for every accepted macro sub-step with its
// length, the extrapolation row it took (rows 0..kacc, n_i = 2(i+1)) and the
// state it started from (the adjoint records that sequence; the step does not).
template <class Rec>
__device__ bool bs_integrate_rec(const GroupState& G, double mu0, double h, double tol,
                                 int max_sub, double (*Y)[kMaxGroup], int* nsub_out, Rec&& rec) {
  double row[kBsRows][6][kMaxGroup];
  double raw[6][kMaxGroup];
  double xscal[kMaxGroup], vscal[kMaxGroup];
  const double tol2 = tol * tol;
  double rem = h, H = h;
  int nsub = 0;
  while (rem != 0.0) {
    if (nsub >= max_sub) {
      *nsub_out = nsub;
      return false;
    }
    ++nsub;
    if (fabs(H) > fabs(rem)) H = rem;
    for (int b = 0; b < G.nb; ++b) {
      xscal[b] = 1.0 / fma(Y[0][b], Y[0][b], fma(Y[1][b], Y[1][b], Y[2][b] * Y[2][b]));
      vscal[b] = 1.0 / fma(Y[3][b], Y[3][b], fma(Y[4][b], Y[4][b], Y[5][b] * Y[5][b]));
    }
    int kacc = -1;
    for (int k = 0; k < kBsRows; ++k) {
      stoermer(G, mu0, Y, H, 2 * (k + 1), raw);
      for (int c = 0; c < 6; ++c)
        for (int b = 0; b < G.nb; ++b) {
          double prev = row[0][c][b];
          row[0][c][b] = raw[c][b];
          for (int jj = 1; jj <= k; ++jj) {
            const double t = row[jj][c][b];
            row[jj][c][b] = fma(row[jj - 1][c][b] - prev, inv_den(k, jj), row[jj - 1][c][b]);
            prev = t;
          }
        }
      if (k >= 1) {
        double err = 0.0;
        for (int b = 0; b < G.nb; ++b) {
          double ex = 0.0, ev = 0.0;
          for (int c = 0; c < 3; ++c) {
            const double dx = row[k][c][b] - row[k - 1][c][b];
            const double dv = row[k][3 + c][b] - row[k - 1][3 + c][b];
            ex = fma(dx, dx, ex);
            ev = fma(dv, dv, ev);
          }
          err = fmax(err, fmax(ex * xscal[b], ev * vscal[b]));
        }
        if (err <= tol2) {
          kacc = k;
          break;
        }
      }
    }
    if (kacc >= 0) {
      rec(H, kacc, (const double(*)[kMaxGroup])Y);
      for (int c = 0; c < 6; ++c)
        for (int b = 0; b < G.nb; ++b) Y[c][b] = row[kacc][c][b];
      rem -= H;
      H *= 1.3;
    } else {
      H *= 0.5;
    }
  }
  *nsub_out = nsub;
  return true;
}

struct NoTape {
  __device__ void operator()(double, int, const double (*)[kMaxGroup]) const {}
};

__device__ __forceinline__ bool bs_integrate(const GroupState& G, double mu0, double h, double tol,
                                             int max_sub, double (*Y)[kMaxGroup], int* nsub_out) {
  return bs_integrate_rec(G, mu0, h, tol, max_sub, Y, nsub_out, NoTape{});
}

}  // namespace mx
