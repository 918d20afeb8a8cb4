// mx_bs2.cuh -- Bulirsch-Stoer of two-body groups on lanes (term lanes, and
// the coordinate split over three warps), shared by the step's groups and
// catch-up (k_bs.cu) and the adjoint's recorded forward (k_adj_bs.cu).
#pragma once
#include "mx_common.cuh"

namespace mx {

// Changeover constants of one member: rc^2, 0.01 rc^2, 0.1 rc, 1/(0.9 rc).
struct MemberK {
  double rc, rc2, rc2lo, rc01, i09;
};

// Integration state of one group between macro sub-steps.
template <int NB>
struct GroupRun {
  double Y[6][NB];
  double rem, H;
  int nsub;
};

// ----------------------------------------- two-body groups, one term per lane
// A group of two bodies (a big body and a planetesimal, or two big bodies)
// runs one step candidate per warp.  Lane 4r + q holds extrapolation row r
// and one force term q: 0 the star on body 0, 1 the star on body 1, 2 body 1
// on body 0, 3 body 0 on body 1.  Every lane evaluates its term with the same
// instructions (the star is a source without changeover), the two terms of a
// body are added with one shuffle, and each lane advances only its own body
// (q & 1).  One warp scheduler issues an FP64 instruction about every 70
// cycles on this part, so a macro sub-step costs the FP64 instructions of one
// lane: about 30 per Stoermer sub-step here, against about 70 when one lane
// carries both bodies and all their terms.  The four candidates of the spread
// phase and of the catch-up are four warps, one per scheduler.  The Neville
// values of a row are split over its lanes: positions of body q & 1 on q < 2,
// velocities on q >= 2.  Rows are checked as they complete, after rows 2, 3, 5
// and 7: the round ends at the first check where candidate 0 (the largest
// step) has a converged row.  The search still accepts what trying H, then
// H/2 after a failure, with the rows in order, would accept.
constexpr unsigned kBs2Checks = (1u << 2) | (1u << 3) | (1u << 5) | (1u << 7);

constexpr double bs_inv_den_c(int r, int j) {
  return (j < 1 || j > r) ? 0.0
                          : 1.0 / (((double)(r + 1) / (double)(r - j + 1)) *
                                       ((double)(r + 1) / (double)(r - j + 1)) - 1.0);
}
#define MX_DEN_ROW(r)                                                                       \
  { bs_inv_den_c(r, 0), bs_inv_den_c(r, 1), bs_inv_den_c(r, 2), bs_inv_den_c(r, 3),          \
    bs_inv_den_c(r, 4), bs_inv_den_c(r, 5), bs_inv_den_c(r, 6), bs_inv_den_c(r, 7) }
// 1 / ((n_r / n_{r-j})^2 - 1) and 1 / n_r for n_r = 2(r+1)
static __constant__ double c_bs_inv_den[kBsRows][kBsRows] = {
    MX_DEN_ROW(0), MX_DEN_ROW(1), MX_DEN_ROW(2), MX_DEN_ROW(3),
    MX_DEN_ROW(4), MX_DEN_ROW(5), MX_DEN_ROW(6), MX_DEN_ROW(7)};
#undef MX_DEN_ROW
static __constant__ double c_bs_inv_n[kBsRows] = {1.0 / 2, 1.0 / 4, 1.0 / 6, 1.0 / 8,
                                           1.0 / 10, 1.0 / 12, 1.0 / 14, 1.0 / 16};

// The force term of one lane: source mu and the changeover of the pair
// (rc = max of the two rcrit; the star's term has rc = infinity).
struct Bs2Term {
  double musrc, rc2, rc2lo, rc01, i09;
  bool pair;
};

__device__ __forceinline__ Bs2Term bs2_term(int q, double mu0, const double* mu, const MemberK* K) {
  Bs2Term t;
  t.pair = q >= 2;
  const int ob = q & 1;
  if (!t.pair) {
    t.musrc = mu0;
    t.rc2 = t.rc2lo = INFINITY;
    t.rc01 = t.i09 = 0.0;
  } else {
    const MemberK& k = (K[0].rc > K[1].rc) ? K[0] : K[1];
    t.musrc = mu[1 - ob];
    t.rc2 = k.rc2;
    t.rc2lo = k.rc2lo;
    t.rc01 = k.rc01;
    t.i09 = k.i09;
  }
  return t;
}

// Acceleration of this lane's body (its two terms summed) at positions X.
__device__ __forceinline__ void bs2_accel(const Bs2Term& t, const double (&X)[3], double (&A)[3]) {
  double dv[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double xo = __shfl_xor_sync(0xffffffffu, X[c], 1);
    dv[c] = X[c] - (t.pair ? xo : 0.0);
  }
  const double s2 = fma(dv[0], dv[0], fma(dv[1], dv[1], dv[2] * dv[2]));
  const double yy = rsqrt_d(s2);
  double wgt = (yy * yy) * (yy * t.musrc);
  // the changeover tests on the bit patterns (s2 and the radii are
  // non-negative, the star's +infinity): off the FP64 pipe
  const long long b2 = __double_as_longlong(s2);
  if (b2 >= __double_as_longlong(t.rc2)) {
    wgt = 0.0;
  } else if (b2 > __double_as_longlong(t.rc2lo)) {
    const double q = fma(s2, yy, -t.rc01) * t.i09;
    wgt *= fma(-q * q * q, fma(q, fma(6.0, q, -15.0), 10.0), 1.0);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double a = -wgt * dv[c];
    A[c] = a + __shfl_xor_sync(0xffffffffu, a, 2);
  }
}

// Neville table of rows 0..K from the raw row values; returns the lowest row
// r in 1..K whose error max(|dx|^2 xscal, |dv|^2 vscal) over both bodies is
// within tol2, or -1.  T keeps the extrapolated values of each lane's row.
__device__ __forceinline__ int bs2_check(int K, int row, double sc, double tol2,
                                         const double (&Traw)[3], double (&T)[3]) {
  double Tp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) T[c] = Tp[c] = Traw[c];
#pragma unroll
  for (int j = 1; j < kBsRows; ++j) {
    if (j > K) break;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double up = __shfl_up_sync(0xffffffffu, T[c], 4);
      if (row >= j && row <= K) {
        if (row == j) Tp[c] = T[c];
        T[c] = fma(T[c] - up, c_bs_inv_den[row][j], T[c]);
      }
    }
  }
  double e = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double dx = T[c] - Tp[c];
    e = fma(dx, dx, e);
  }
  e *= sc;
  // max and test of non-negative errors on their bit patterns (integer order
  // is value order there), off the FP64 pipe
  long long eb = __double_as_longlong(e);
  eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 1));
  eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 2));
  const bool conv = row >= 1 && row <= K && eb <= __double_as_longlong(tol2);
  const unsigned v = __ballot_sync(0xffffffffu, conv);
  return v ? ((__ffs(v) - 1) >> 2) : -1;
}

// ------------------------------------------------ two bodies on three warps
// The catch-up's integrator for two-body groups.  A group's macro sub-steps
// form one serial chain, and a warp scheduler issues one FP64 instruction
// about every 69 cycles, so the chain's length in FP64 instructions per warp
// sets its time.  Here warp c (c = 0, 1, 2) keeps coordinate c of every lane
// of bs2_rounds' layout (lane 4r + q: Stoermer row r, force term q), so the
// per-coordinate work (differences, accelerations, the Stoermer update, the
// Aitken-Neville table) is a third of bs2_rounds'; the squared separation
// and the error, which need all three coordinates, exchange them through
// shared memory and sum them in bs2_rounds' order.  Every floating-point
// operation is bs2_rounds' own, so each try gives its bits and the step
// search, one try per round (H, then H/2 after a failure, ...), accepts what
// it accepts.  Warps 0-2 only (named barrier 1, 96 threads); g is the same
// on every lane of the three warps before and after.
struct Bs2cSmem {
  double* d;   // [2][3][32] the pair separations, by sub-step parity
  double* e;   // [3][32] the coordinates' error differences
  double* y;   // [12] the accepted state: x0, x1, v0, v1
};

__device__ __forceinline__ void bs2c_bar() { asm volatile("bar.sync 1, 96;" ::: "memory"); }

// With `rec`, the lane's term at this sub-step is also kept: its separation
// (coordinate c) in row c and, in row 3 + c, its weight (c = 0), 1/s (c = 1)
// or s^2 (c = 2), rows of 32 lanes.
__device__ __forceinline__ double bs2c_accel(const Bs2Term& t, int c, int lane, double X,
                                             const Bs2cSmem& sm, int& buf,
                                             double* rec = nullptr) {
  const double xo = __shfl_xor_sync(0xffffffffu, X, 1);
  const double dv = X - (t.pair ? xo : 0.0);
  double* sd = sm.d + buf * 96;
  sd[c * 32 + lane] = dv;
  bs2c_bar();
  const double d0 = sd[lane], d1 = sd[32 + lane], d2 = sd[64 + lane];
  buf ^= 1;
  const double s2 = fma(d0, d0, fma(d1, d1, d2 * d2));
  const double yy = rsqrt_d(s2);
  double wgt = (yy * yy) * (yy * t.musrc);
  const long long b2 = __double_as_longlong(s2);
  if (b2 >= __double_as_longlong(t.rc2)) {
    wgt = 0.0;
  } else if (b2 > __double_as_longlong(t.rc2lo)) {
    const double qv = fma(s2, yy, -t.rc01) * t.i09;
    wgt *= fma(-qv * qv * qv, fma(qv, fma(6.0, qv, -15.0), 10.0), 1.0);
  }
  if (rec) {
    rec[c * 32 + lane] = dv;
    rec[(3 + c) * 32 + lane] = (c == 0) ? wgt : ((c == 1) ? yy : s2);
  }
  const double a = -wgt * dv;
  return a + __shfl_xor_sync(0xffffffffu, a, 2);
}

// bs2_check on one coordinate: the Neville table of rows 0..K, then the error
// summed over the three coordinates in bs2_rounds' order.
__device__ __forceinline__ int bs2c_check(int K, int row, int c, int lane, double sc, double tol2,
                                          double Traw, double& T, const Bs2cSmem& sm) {
  double Tp = Traw;
  T = Traw;
#pragma unroll
  for (int j = 1; j < kBsRows; ++j) {
    if (j > K) break;
    const double up = __shfl_up_sync(0xffffffffu, T, 4);
    if (row >= j && row <= K) {
      if (row == j) Tp = T;
      T = fma(T - up, c_bs_inv_den[row][j], T);
    }
  }
  sm.e[c * 32 + lane] = T - Tp;
  bs2c_bar();
  const double x0 = sm.e[lane], x1 = sm.e[32 + lane], x2 = sm.e[64 + lane];
  double e = 0.0;
  e = fma(x0, x0, e);
  e = fma(x1, x1, e);
  e = fma(x2, x2, e);
  e *= sc;
  long long eb = __double_as_longlong(e);
  eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 1));
  eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 2));
  const bool conv = row >= 1 && row <= K && eb <= __double_as_longlong(tol2);
  const unsigned v = __ballot_sync(0xffffffffu, conv);
  return v ? ((__ffs(v) - 1) >> 2) : -1;
}

}  // namespace mx
