// k_adj_bs.cu -- reverse mode through the Bulirsch-Stoer groups of one step
// (arXiv 2601.16791, Sec. 2: bodies in a close encounter leave the Kepler
// drift and are integrated by mdt_bs2 together).
//
// The adjoint recomputes the step from its start.  After the drift it runs
// the encounter detection on the recomputed endpoints and builds the step's
// own groups from them (k_groups on the sorted pairs, so the items come in a
// fixed order): groups of big bodies joined by big-big encounters, every
// member written back, and test-particle groups, a planetesimal with the
// whole big groups of the big bodies it meets, only the planetesimal written
// back.  Every group is integrated again and each accepted macro sub-step's
// length, extrapolation row and starting state go to the group's region of a
// tape: test-particle pairs on three warps with the catch-up's two-body
// arithmetic (mx_bs2.cuh), other groups on one warp with the arithmetic of
// the step's thread integrator (mx_bs.cuh; lane r runs the Stoermer row with
// 2(r+1) sub-steps, lane 0 builds the Aitken-Neville table and takes the
// first converged row, as the sequential search does).  The members'
// results replace their drifted states.
//
// The reverse sweep treats that sequence as fixed (a discrete adjoint of the
// Gragg-Bulirsch-Stoer map with its accepted steps and rows frozen, as a
// forward-mode derivative that follows the primal's control flow gives):
// every accepted sub-step is a fixed linear combination of Stoermer runs
// (the Aitken-Neville weights of its row), and each Stoermer run is reversed
// from its recomputed positions with the Jacobian of the group's forces (the
// star and the (1 - K)-weighted pair forces), the rows' shares summed in a
// fixed butterfly.  A member written back gets its cotangent at its
// pre-drift state in place of the drift's; the big bodies of a test-particle
// group get shares, added to theirs by a per-system fold in item order.
#include "mx_bs.cuh"
#include "mx_bs2.cuh"
#include "mx_common.cuh"
#include "mx_kernels.h"

namespace mx {

namespace {

// Tape record of one accepted macro sub-step: H, row, the 6 x nb state, then
// (two-body groups) the slot of its kept Stoermer sub-steps or -1; each group
// has room for kAdjMaxSteps of them.
__device__ __forceinline__ int tape_stride(int nb) { return 3 + 6 * nb; }
constexpr int kAdjMaxSteps = 128;

// Slots of kept sub-steps are handed to a group kSubChunk at a time (one
// atomic per kSubChunk records); -1 when the pool is used up or absent.
constexpr int kSubChunk = 8;
constexpr int kSubStride = kAdjSubVals * 32;   // doubles of one sub-step in a slot
static_assert(kAdjSubRec == (2 * kBsRows + 1) * kSubStride, "a slot holds sub-steps 0..2 kBsRows");
static_assert((kAdjSubRec * sizeof(double)) % 16 == 0 && (kSubStride * sizeof(double)) % 16 == 0,
              "slots and sub-steps are whole 16-byte chunks");

__device__ __forceinline__ int take_slots(const Adj& a) {
  if (a.sub == nullptr) return -1;
  const unsigned s0 = atomicAdd(a.sub_count, (unsigned)kSubChunk);
  return (s0 <= a.sub_cap && a.sub_cap - s0 >= (unsigned)kSubChunk) ? (int)s0 : -1;
}

}  // namespace

// The items of the step's work list the adjoint takes: every one (groups 1),
// or the groups of big bodies only (groups 2: every member written back).
__device__ __forceinline__ bool adj_takes(const Dev& d, const Adj& a, int w) {
  return a.groups == 1 || (a.groups == 2 && d.work_wfrom[w] == 0);
}

// One block, after k_groups: the tape region of every item the adjoint takes
// (an exclusive scan of kAdjMaxSteps records of its size, in item order), and
// the mark flags = 2 on the members it writes back, whose drift the reverse
// then leaves to the group.  Every item starts with g_M = -1 (not processed);
// the forward kernels set it.
__global__ void __launch_bounds__(1024) k_adj_tape(Dev d, Adj a) {
  __shared__ unsigned long long s_wsum[32];
  __shared__ unsigned long long s_run, s_ent;
  const int W = min(*d.work_count, a.g_cap);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_run = 0;
    s_ent = 0;
    if (a.sub_count) *a.sub_count = 0;
  }
  __syncthreads();
  for (int base = 0; base < W; base += blockDim.x) {
    const int w = base + threadIdx.x;
    unsigned long long v = 0;
    if (w < W) {
      a.g_M[w] = -1;
      if (adj_takes(d, a, w)) {
        const int o = d.work_off[w], nb = d.work_off[w + 1] - o;
        v = (unsigned long long)kAdjMaxSteps * tape_stride(min(nb, kMaxGroup));
        for (int m = d.work_wfrom[w]; m < nb; ++m) d.flags[d.work_mem[o + m]] = 2;
        if (d.work_wfrom[w] > 0) atomicAdd(&s_ent, (unsigned long long)d.work_wfrom[w]);
      }
    }
    unsigned long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long run = s_run;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        const unsigned long long c = s_wsum[q];
        s_wsum[q] = run;
        run += c;
      }
      s_run = run;
    }
    __syncthreads();
    if (w < W) a.g_off[w] = s_wsum[warp] + inc - v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.tape_need[0] = s_run;
    a.tape_need[1] = s_ent;
  }
}

// Item w's members in the step's order (big bodies ascending, then the
// planetesimal of a test-particle group), their constants and their
// pre-drift states (x2, v1); *jj the last member, *wf the first written back.
__device__ bool load_adj_group(const Dev& d, const Adj& a, int w, GroupState& G,
                               double (*Y)[kMaxGroup], int* big, int* jj, int* sys, int* wf) {
  const int o = d.work_off[w], nb = d.work_off[w + 1] - o;
  if (nb < 2 || nb > kMaxGroup) return false;
  const int sy = d.work_sys[w];
  const SysDev& S = d.sys[sy];
  const int N = d.N;
  G.nb = nb;
  for (int m = 0; m < nb; ++m) {
    const int gi = d.work_mem[o + m];
    const int l = gi - S.off;
    const bool bm = l < S.nbig;
    big[m] = bm ? l : -1;
    G.mu[m] = bm ? d.bmu[S.boff + l] : 0.0;
    G.rc[m] = bm ? d.brc[S.boff + l] : 0.0;
    for (int c = 0; c < 3; ++c) {
      Y[c][m] = a.x2[(size_t)c * N + gi];
      Y[3 + c][m] = a.v1[(size_t)c * N + gi];
    }
  }
  *jj = d.work_mem[o + nb - 1];
  *sys = sy;
  *wf = d.work_wfrom[w];
  return true;
}

// A test-particle pair (a big body and the planetesimal): k_adj_bs_fwd2 and
// k_adj_bs_vjp2 take it; every other item goes to the general kernels.
__device__ __forceinline__ bool adj_pair(const Dev& d, int w) {
  return d.work_off[w + 1] - d.work_off[w] == 2 && d.work_wfrom[w] == 1;
}

// Forward, one warp per group: lane r < kBsRows runs Stoermer row r from the
// macro sub-step's start; lane 0 extrapolates, checks and (on acceptance)
// records the sub-step and passes the new state to the other lanes through
// shared memory.  The arithmetic and the decisions are bs_integrate's.  The
// results of the members written back (the planetesimal of a test-particle
// group, every member of a group of big bodies) replace their drifted states
// in xv3.
__global__ void __launch_bounds__(32) k_adj_bs_fwd(Dev d, Adj a) {
  __shared__ double sraw[kBsRows][6][kMaxGroup];
  __shared__ double sY[6][kMaxGroup];
  const int lane = threadIdx.x;
  const int ng = min(*d.work_count, a.g_cap);
  for (int g = blockIdx.x; g < ng; g += gridDim.x) {
    if (!adj_takes(d, a, g) || adj_pair(d, g)) continue;   // pairs: k_adj_bs_fwd2
    GroupState G;
    double Y[6][kMaxGroup];
    int big[kMaxGroup], j, sy, wf;
    if (!load_adj_group(d, a, g, G, Y, big, &j, &sy, &wf)) continue;
    const SysDev& S = d.sys[sy];
    const int nb = G.nb, stride = tape_stride(nb);
    const unsigned long long off = a.g_off[g];
    if (off + (unsigned long long)kAdjMaxSteps * stride > a.tape_cap) {
      if (lane == 0) {
        a.g_M[g] = -1;
        atomicOr(d.status, ST_WORK_OVF);
      }
      continue;
    }
    double* T = a.tape + off;
    const double tol2 = d.bs_tol * d.bs_tol;
    double rem = S.h, H = S.h;
    int nsub = 0, M = 0;
    bool ok = true;
    while (rem != 0.0) {
      if (nsub >= d.bs_max_sub || M >= kAdjMaxSteps) {
        ok = false;
        break;
      }
      ++nsub;
      if (fabs(H) > fabs(rem)) H = rem;
      if (lane < kBsRows) {
        double raw[6][kMaxGroup];
        stoermer(G, S.mu0, Y, H, 2 * (lane + 1), raw);
        for (int c = 0; c < 6; ++c)
          for (int b = 0; b < nb; ++b) sraw[lane][c][b] = raw[c][b];
      }
      __syncwarp();
      int kacc = -1;
      if (lane == 0) {
        double row[kBsRows][6][kMaxGroup];
        double xscal[kMaxGroup], vscal[kMaxGroup];
        for (int b = 0; b < nb; ++b) {
          xscal[b] = 1.0 / fma(Y[0][b], Y[0][b], fma(Y[1][b], Y[1][b], Y[2][b] * Y[2][b]));
          vscal[b] = 1.0 / fma(Y[3][b], Y[3][b], fma(Y[4][b], Y[4][b], Y[5][b] * Y[5][b]));
        }
        for (int k = 0; k < kBsRows && kacc < 0; ++k) {
          for (int c = 0; c < 6; ++c)
            for (int b = 0; b < nb; ++b) {
              double prev = row[0][c][b];
              row[0][c][b] = sraw[k][c][b];
              for (int jj = 1; jj <= k; ++jj) {
                const double t = row[jj][c][b];
                row[jj][c][b] = fma(row[jj - 1][c][b] - prev, inv_den(k, jj), row[jj - 1][c][b]);
                prev = t;
              }
            }
          if (k >= 1) {
            double err = 0.0;
            for (int b = 0; b < nb; ++b) {
              double ex = 0.0, ev = 0.0;
              for (int c = 0; c < 3; ++c) {
                const double dx = row[k][c][b] - row[k - 1][c][b];
                const double dv = row[k][3 + c][b] - row[k - 1][3 + c][b];
                ex = fma(dx, dx, ex);
                ev = fma(dv, dv, ev);
              }
              err = fmax(err, fmax(ex * xscal[b], ev * vscal[b]));
            }
            if (err <= tol2) kacc = k;
          }
        }
        if (kacc >= 0) {
          double* r = T + (size_t)M * stride;
          r[0] = H;
          r[1] = (double)kacc;
          for (int c = 0; c < 6; ++c)
            for (int b = 0; b < nb; ++b) {
              r[2 + c * nb + b] = Y[c][b];
              sY[c][b] = row[kacc][c][b];
            }
        }
      }
      kacc = __shfl_sync(0xffffffffu, kacc, 0);
      __syncwarp();
      if (kacc >= 0) {
        for (int c = 0; c < 6; ++c)
          for (int b = 0; b < nb; ++b) Y[c][b] = sY[c][b];
        rem -= H;
        H *= 1.3;
        ++M;
      } else {
        H *= 0.5;
      }
      __syncwarp();
    }
    if (lane == 0) {
      if (!ok) {
        atomicOr(d.status, M >= kAdjMaxSteps ? ST_TAPE : ST_BS);
        a.g_M[g] = -1;
      } else {
        a.g_M[g] = M;
        const int N = d.N, o = d.work_off[g];
        for (int m = wf; m < nb; ++m)
          for (int c = 0; c < 6; ++c) a.xv3[(size_t)c * N + d.work_mem[o + m]] = Y[c][m];
      }
    }
  }
}

// Forward of a two-body group (a big body and the planetesimal), one block
// of four warps per group: warps 0-2 run the catch-up's integrator with one
// coordinate each (bs2c arithmetic, the same tries and accepted sub-steps as
// the step's own two-body integrator), one try per round, and record every
// accepted macro sub-step (H, row, starting state) in the group's tape.  Each
// try also keeps its Stoermer sub-steps (every lane's term at every position
// up to its row's last) in the slot of the record it tries for; a rejected
// try's slot is rewritten by the next try, so the accepted one stays.
__global__ void __launch_bounds__(128) k_adj_bs_fwd2(Dev d, Adj a) {
  __shared__ double s_d[2 * 3 * 32], s_e[3 * 32], s_y[12];
  __shared__ int s_slot;
  const Bs2cSmem sm{s_d, s_e, s_y};
  const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
  const int row = lane >> 2, q = lane & 3, ob = q & 1;
  const bool vel = q >= 2;
  const int n = 2 * (row + 1);
  const int ng = min(*d.work_count, a.g_cap);
  for (int g = blockIdx.x; g < ng; g += gridDim.x) {
    if (!adj_takes(d, a, g) || !adj_pair(d, g)) continue;   // a big body and the planetesimal
    if (c == 3) continue;           // warps 0-2 only (named barrier 1)
    GroupState G;
    double Y0[6][kMaxGroup];
    int big[kMaxGroup], j, sy, wf;
    if (!load_adj_group(d, a, g, G, Y0, big, &j, &sy, &wf)) continue;
    const SysDev& S = d.sys[sy];
    const int stride = tape_stride(2);
    const unsigned long long off = a.g_off[g];
    if (off + (unsigned long long)kAdjMaxSteps * stride > a.tape_cap) {
      if (threadIdx.x == 0) {
        a.g_M[g] = -1;
        atomicOr(d.status, ST_WORK_OVF);
      }
      continue;
    }
    double* T = a.tape + off;
    double mu[2];
    MemberK K[2];
    for (int m = 0; m < 2; ++m) {
      const double rc = G.rc[m];
      mu[m] = G.mu[m];
      K[m].rc = rc;
      K[m].rc2 = rc * rc;
      K[m].rc2lo = 0.01 * (rc * rc);
      K[m].rc01 = 0.1 * rc;
      K[m].i09 = (rc > 0.0) ? 1.0 / (0.9 * rc) : 0.0;
    }
    const Bs2Term tm = bs2_term(q, S.mu0, mu, K);
    GroupRun<2> gr;
    for (int k = 0; k < 6; ++k) {
      gr.Y[k][0] = Y0[k][0];
      gr.Y[k][1] = Y0[k][1];
    }
    gr.rem = S.h;
    gr.H = S.h;
    gr.nsub = 0;
    const double tol2 = d.bs_tol * d.bs_tol;
    int buf = 0, M = 0;
    bool ok = true;
    if (threadIdx.x == 0) s_slot = take_slots(a);
    bs2c_bar();
    int slot0 = s_slot, m0 = 0;   // the group's current chunk of slots, from record m0
    while (gr.rem != 0.0) {
      if (gr.nsub >= d.bs_max_sub || M >= kAdjMaxSteps) {
        ok = false;
        break;
      }
      if (fabs(gr.H) > fabs(gr.rem)) gr.H = gr.rem;
      const double Hc = gr.H;
      const int slot = (slot0 >= 0) ? slot0 + (M - m0) : -1;
      double* keep = (slot >= 0) ? a.sub + (size_t)slot * kAdjSubRec : nullptr;
      double X = ob ? gr.Y[c][1] : gr.Y[c][0];
      const double V = ob ? gr.Y[3 + c][1] : gr.Y[3 + c][0];
      const int so = vel ? 3 : 0;
      const double s0 = ob ? gr.Y[so][1] : gr.Y[so][0];
      const double s1 = ob ? gr.Y[so + 1][1] : gr.Y[so + 1][0];
      const double s2v = ob ? gr.Y[so + 2][1] : gr.Y[so + 2][0];
      const double sc = rcp_d(fma(s0, s0, fma(s1, s1, s2v * s2v)));
      const double dd = Hc * c_bs_inv_n[row];
      const double d2 = dd * dd;
      double A = bs2c_accel(tm, c, lane, X, sm, buf, keep);
      double D = dd * fma(0.5 * dd, A, V);
      X += D;
      double Traw = 0.0, Tv = 0.0;
      int acc_r = -1;
      bool decided = false;
      for (int st = 1; st <= 2 * kBsRows && !decided; ++st) {
        A = bs2c_accel(tm, c, lane, X, sm, buf,
                       (keep && st <= n) ? keep + (size_t)st * kSubStride : nullptr);
        if (st < n) {
          D = fma(d2, A, D);
          X += D;
        } else if (st == n) {
          const double idd = n * rcp_d(Hc);
          Traw = vel ? fma(D, idd, 0.5 * dd * A) : X;
        }
        const int Kr = (st >> 1) - 1;
        if ((st & 1) || !((kBs2Checks >> Kr) & 1u)) continue;
        const int r = bs2c_check(Kr, row, c, lane, sc, tol2, Traw, Tv, sm);
        if (r >= 0) {
          acc_r = r;
          decided = true;
        } else if (Kr == kBsRows - 1) {
          decided = true;
        }
      }
      gr.nsub += 1;
      if (acc_r >= 0) {
        if (c == 0 && lane == 0) {   // the sub-step's record: H, row, starting state
          double* rr = T + (size_t)M * stride;
          rr[0] = Hc;
          rr[1] = (double)acc_r;
          for (int k = 0; k < 6; ++k) {
            rr[2 + 2 * k] = gr.Y[k][0];
            rr[3 + 2 * k] = gr.Y[k][1];
          }
          rr[14] = (double)slot;
        }
        const bool chunk_done = slot0 >= 0 && M + 1 - m0 == kSubChunk;
        if (chunk_done && threadIdx.x == 0) s_slot = take_slots(a);
        if (row == acc_r) sm.y[3 * q + c] = Tv;
        bs2c_bar();
        if (chunk_done) {
          slot0 = s_slot;
          m0 = M + 1;
        }
        for (int k = 0; k < 3; ++k) {
          gr.Y[k][0] = sm.y[k];
          gr.Y[k][1] = sm.y[3 + k];
          gr.Y[3 + k][0] = sm.y[6 + k];
          gr.Y[3 + k][1] = sm.y[9 + k];
        }
        bs2c_bar();
        gr.rem -= Hc;
        gr.H = 1.3 * Hc;
        ++M;
      } else {
        gr.H *= 0.5;
      }
    }
    if (c == 0 && lane == 0) {
      if (!ok) {
        atomicOr(d.status, M >= kAdjMaxSteps ? ST_TAPE : ST_BS);
        a.g_M[g] = -1;
      } else {
        a.g_M[g] = M;
        for (int k = 0; k < 6; ++k) a.xv3[(size_t)k * d.N + j] = gr.Y[k][1];
      }
    }
  }
}

// gX += J_a(X)^T lA for the group's accelerations a(X) (star plus the
// (1 - K)-weighted pair forces of the massive members, as bs_accel).  For a
// pair at separation s with weight w(s^2) = mu_i (1 - K(s))/s^3, the force on
// b is -w dx (dx = x_b - x_i), whose Jacobian in dx is -w I - 2 w' dx dx^T,
// w' = dw/d(s^2) = mu_i g'(s)/(2s), g = (1 - K)/s^3 (g = 1/s^3 inside 0.1 rc),
// K' = 30 q^2 (1 - q)^2 / (0.9 rc).
__device__ void accel_vjp(const GroupState& G, double mu0, const double (*X)[kMaxGroup],
                          const double (*lA)[kMaxGroup], double (*gX)[kMaxGroup]) {
  for (int b = 0; b < G.nb; ++b) {
    const double x = X[0][b], y = X[1][b], z = X[2][b];
    const double lx = lA[0][b], ly = lA[1][b], lz = lA[2][b];
    const double r2 = x * x + y * y + z * z;
    const double r = sqrt(r2);
    const double ir3 = 1.0 / (r2 * r);
    const double ir5 = ir3 / r2;
    const double xl = x * lx + y * ly + z * lz;
    gX[0][b] += -mu0 * (lx * ir3 - 3.0 * xl * x * ir5);
    gX[1][b] += -mu0 * (ly * ir3 - 3.0 * xl * y * ir5);
    gX[2][b] += -mu0 * (lz * ir3 - 3.0 * xl * z * ir5);
    for (int i = 0; i < G.nb; ++i) {
      if (i == b || G.mu[i] == 0.0) continue;
      const double dx = x - X[0][i], dy = y - X[1][i], dz = z - X[2][i];
      const double s2 = dx * dx + dy * dy + dz * dz;
      const double rc = fmax(G.rc[b], G.rc[i]);
      if (s2 >= rc * rc) continue;
      const double s = sqrt(s2);
      double gval, dg;
      if (s2 <= 0.01 * rc * rc) {
        gval = 1.0 / (s2 * s);
        dg = -3.0 / (s2 * s2);
      } else {
        const double q = (s - 0.1 * rc) / (0.9 * rc);
        const double K = q * q * q * (10.0 + q * (-15.0 + 6.0 * q));
        const double Kp = 30.0 * q * q * (1.0 - q) * (1.0 - q) / (0.9 * rc);
        gval = (1.0 - K) / (s2 * s);
        dg = -Kp / (s2 * s) - 3.0 * (1.0 - K) / (s2 * s2);
      }
      const double w = G.mu[i] * gval;
      const double wp = G.mu[i] * dg / (2.0 * s);
      const double dl = dx * lx + dy * ly + dz * lz;
      const double cx = -w * lx - 2.0 * wp * dl * dx;
      const double cy = -w * ly - 2.0 * wp * dl * dy;
      const double cz = -w * lz - 2.0 * wp * dl * dz;
      gX[0][b] += cx;
      gX[1][b] += cy;
      gX[2][b] += cz;
      gX[0][i] -= cx;
      gX[1][i] -= cy;
      gX[2][i] -= cz;
    }
  }
}

// Reverse of one Stoermer run (n sub-steps of length H/n from Y): adds
// J^T (lO) to lY, with the positions X_0..X_n recomputed here.
constexpr int kMaxSub = 2 * kBsRows;

__device__ void stoermer_vjp(const GroupState& G, double mu0, const double (*Y)[kMaxGroup],
                             double H, int n, const double (*lO)[kMaxGroup],
                             double (*lY)[kMaxGroup], double scale) {
  double X[kMaxSub + 1][3][kMaxGroup];
  double A[3][kMaxGroup], D[3][kMaxGroup];
  const double dd = H / n, d2 = dd * dd;
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < G.nb; ++b) X[0][c][b] = Y[c][b];
  bs_accel(G, mu0, X[0], A);
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < G.nb; ++b) {
      D[c][b] = dd * fma(0.5 * dd, A[c][b], Y[3 + c][b]);
      X[1][c][b] = X[0][c][b] + D[c][b];
    }
  for (int s = 1; s < n; ++s) {
    bs_accel(G, mu0, X[s], A);
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < G.nb; ++b) {
        D[c][b] = fma(d2, A[c][b], D[c][b]);
        X[s + 1][c][b] = X[s][c][b] + D[c][b];
      }
  }
  // reverse: O_x = X_n, O_v = D_n/dd + (dd/2) A(X_n)
  double lX[3][kMaxGroup], lD[3][kMaxGroup], lA[3][kMaxGroup];
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < G.nb; ++b) {
      lX[c][b] = scale * lO[c][b];
      lD[c][b] = scale * lO[3 + c][b] / dd;
      lA[c][b] = scale * 0.5 * dd * lO[3 + c][b];
    }
  accel_vjp(G, mu0, X[n], lA, lX);
  for (int s = n - 1; s >= 1; --s) {
    // X_{s+1} = X_s + D_{s+1};  D_{s+1} = D_s + d2 A(X_s)
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < G.nb; ++b) {
        lD[c][b] += lX[c][b];
        lA[c][b] = d2 * lD[c][b];
      }
    accel_vjp(G, mu0, X[s], lA, lX);
  }
  // X_1 = X_0 + D_1;  D_1 = dd V_0 + (dd^2/2) A(X_0)
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < G.nb; ++b) {
      lD[c][b] += lX[c][b];
      lY[3 + c][b] += dd * lD[c][b];
      lA[c][b] = 0.5 * d2 * lD[c][b];
    }
  accel_vjp(G, mu0, X[0], lA, lX);
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < G.nb; ++b) lY[c][b] += lX[c][b];
}

// The Aitken-Neville result of row K is sum_i c_i S_i over the Stoermer runs
// S_0..S_K (the recurrence of bs_integrate is linear in them); c_i is the
// recurrence applied to the unit vector e_i.
__device__ void neville_weights(int K, double* c) {
  for (int l = 0; l <= K; ++l) {
    double row[kBsRows] = {0.0};
    for (int k = 0; k <= K; ++k) {
      double prev = row[0];
      row[0] = (k == l) ? 1.0 : 0.0;
      for (int jj = 1; jj <= k; ++jj) {
        const double t = row[jj];
        row[jj] = fma(row[jj - 1] - prev, inv_den(k, jj), row[jj - 1]);
        prev = t;
      }
    }
    c[l] = row[K];
  }
}

// Reverse, one warp per group: the planetesimal's cotangent at its BS result
// (in lam) goes back through the recorded sub-steps, lane r <= K reversing
// Stoermer row r with its Aitken-Neville weight and the lanes' shares summed
// by a butterfly (every lane ends with the same sum).  The planetesimal's
// pre-drift cotangent replaces lam's; the big members' shares go to g_contrib.
__global__ void __launch_bounds__(32) k_adj_bs_vjp(Dev d, Adj a) {
  const int lane = threadIdx.x;
  const int ng = min(*d.work_count, a.g_cap);
  for (int g = blockIdx.x; g < ng; g += gridDim.x) {
    const int M = a.g_M[g];
    if (M < 0 || adj_pair(d, g)) continue;   // pairs: k_adj_bs_vjp2
    GroupState G;
    double Y0[6][kMaxGroup];
    int big[kMaxGroup], j, sy, wf;
    if (!load_adj_group(d, a, g, G, Y0, big, &j, &sy, &wf)) continue;
    const SysDev& S = d.sys[sy];
    const int N = d.N, nb = G.nb, o = d.work_off[g];
    // the cotangents of the outputs: the members written back carry theirs
    double lY[6][kMaxGroup], lO[6][kMaxGroup];
    for (int c = 0; c < 6; ++c)
      for (int m = 0; m < nb; ++m)
        lO[c][m] = (m >= wf) ? a.lam[(size_t)c * N + d.work_mem[o + m]] : 0.0;
    const int stride = tape_stride(nb);
    for (int k = M - 1; k >= 0; --k) {
      const double* r = a.tape + a.g_off[g] + (size_t)k * stride;
      const double H = r[0];
      const int K = (int)r[1];
      for (int c = 0; c < 6; ++c)
        for (int m = 0; m < nb; ++m) lY[c][m] = 0.0;
      if (lane <= K) {
        double Ys[6][kMaxGroup];
        for (int c = 0; c < 6; ++c)
          for (int m = 0; m < nb; ++m) Ys[c][m] = r[2 + c * nb + m];
        double cw[kBsRows];
        neville_weights(K, cw);
        stoermer_vjp(G, S.mu0, Ys, H, 2 * (lane + 1), lO, lY, cw[lane]);
      }
      for (int c = 0; c < 6; ++c)
        for (int m = 0; m < nb; ++m) {
          double v = lY[c][m];
          for (int o = 1; o < kBsRows; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          lO[c][m] = v;
        }
    }
    // a member written back gets its cotangent at its pre-drift state; any
    // other (a big body of a test-particle group) a share, folded per system
    if (lane == 0) {
      double* out = a.g_contrib + (size_t)g * 6 * kMaxGroup;
      for (int m = 0; m < nb; ++m)
        for (int c = 0; c < 6; ++c) {
          if (m >= wf) a.lam[(size_t)c * N + d.work_mem[o + m]] = lO[c][m];
          else out[6 * m + c] = lO[c][m];
        }
    }
  }
}

// Reverse of a two-body group, one block of three warps per group, in the
// forward's layout (lane 4r + q: Stoermer row r, force term q, as in
// bs2_rounds: 0 and 1 the star on body 0 and 1, 2 body 1 on body 0, 3 body 0
// on body 1; warp c: coordinate c).  Every term is written as a pair term
// (the star is a source at the origin): with d = x_b - x_src, s = |d|,
// w = mu (1 - K)/s^3 and w' = dw/d(s^2), the force -w d has the product
//   c = -w lA - 2 w' (d . lA) d,
// added to body b's cotangent; a pair term also gives -c to its source.  The
// dot product takes lA's three coordinates from shared memory; a body's total
// is its two terms' c plus the other body's pair reaction, gathered with
// shuffles in a fixed order (both lanes of a body get the same bits).  The
// rows' results are weighted by the Aitken-Neville coefficients of the
// recorded row and summed over rows by a fixed butterfly.
//
// The Stoermer positions of a record come from the slot the forward kept
// (copied to shared memory with cp.async one record ahead of the sweep), or,
// for a record without a slot, are recomputed with the forward's own
// arithmetic into the same layout: both give the same bits.

// -2 dw/d(s^2) of a term from its kept weight w, 1/s and s^2:
//   w' = -1.5 w / s^2 - mu K'(s) / (2 s^4),  K' = 30 q^2 (1 - q)^2 / (0.9 rc),
// the second part inside the changeover shell (0.1 rc < s < rc) only.
__device__ __forceinline__ double adj_wpm2(const Bs2Term& t, double s2, double yy, double w) {
  const long long b2 = __double_as_longlong(s2);
  if (b2 >= __double_as_longlong(t.rc2)) return 0.0;
  const double y2 = yy * yy;
  double r = 3.0 * w * y2;
  if (b2 > __double_as_longlong(t.rc2lo)) {
    const double w0 = y2 * (yy * t.musrc);   // the weight before the changeover factor
    const double q = fma(s2, yy, -t.rc01) * t.i09;
    const double om = 1.0 - q;
    const double kp = 30.0 * (q * q) * (om * om) * t.i09;
    r = fma(w0 * kp, yy, r);
  }
  return r;
}

__device__ __forceinline__ void cp_async16(double* dst, const double* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// Dynamic shared memory of k_adj_bs_vjp2: two records' sub-steps, the
// cotangent exchange (two buffers) and bs2c_accel's exchange.
constexpr int kVjp2Smem = (2 * kAdjSubRec + 2 * 96 + 2 * 96 + 96 + 12) * (int)sizeof(double);

__global__ void __launch_bounds__(96) k_adj_bs_vjp2(Dev d, Adj a) {
  extern __shared__ __align__(16) double s_v2[];
  double* s_rec = s_v2;                      // [2][kAdjSubRec]
  double* s_la = s_v2 + 2 * kAdjSubRec;      // [2][3][32]
  const Bs2cSmem sm{s_la + 2 * 96, s_la + 4 * 96, s_la + 5 * 96};
  __shared__ double s_nw[kBsRows][kBsRows];
  const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
  const int row = lane >> 2, q = lane & 3, ob = q & 1;
  const int src_r = (lane & ~3) + 3 - ob;    // the row's lane of the other body's pair term
  const int n = 2 * (row + 1);
  const int ng = min(*d.work_count, a.g_cap);
  // Aitken-Neville weights of every row K (neville_weights, with the
  // constants the two-body integrator extrapolates with)
  for (int e = threadIdx.x; e < kBsRows * kBsRows; e += blockDim.x) {
    const int K = e / kBsRows, l = e % kBsRows;
    double rw[kBsRows] = {0.0};
    for (int k = 0; k <= K; ++k) {
      double prev = rw[0];
      rw[0] = (k == l) ? 1.0 : 0.0;
      for (int jj = 1; jj <= k; ++jj) {
        const double t = rw[jj];
        rw[jj] = fma(rw[jj - 1] - prev, c_bs_inv_den[k][jj], rw[jj - 1]);
        prev = t;
      }
    }
    s_nw[K][l] = (l <= K) ? rw[K] : 0.0;
  }
  bs2c_bar();
  const int stride = tape_stride(2);
  for (int g = blockIdx.x; g < ng; g += gridDim.x) {
    if (!adj_pair(d, g)) continue;
    const int M = a.g_M[g];
    if (M < 0) continue;
    GroupState G;
    double Y0[6][kMaxGroup];
    int big[kMaxGroup], j, sy, wf;
    if (!load_adj_group(d, a, g, G, Y0, big, &j, &sy, &wf)) continue;
    const SysDev& S = d.sys[sy];
    const int N = d.N;
    Bs2Term tm;
    {
      double mu[2];
      MemberK K[2];
      for (int m = 0; m < 2; ++m) {
        const double rc = G.rc[m];
        mu[m] = G.mu[m];
        K[m].rc = rc;
        K[m].rc2 = rc * rc;
        K[m].rc2lo = 0.01 * (rc * rc);
        K[m].rc01 = 0.1 * rc;
        K[m].i09 = (rc > 0.0) ? 1.0 / (0.9 * rc) : 0.0;
      }
      tm = bs2_term(q, S.mu0, mu, K);
    }
    const double* tape = a.tape + a.g_off[g];
    // the copy of record k's kept sub-steps 0..2(K + 1), if it has a slot
    auto fetch = [&](int k) {
      const double* r = tape + (size_t)k * stride;
      const int slot = (int)r[14];
      if (slot >= 0) {
        const double* src = a.sub + (size_t)slot * kAdjSubRec;
        double* dst = s_rec + (k & 1) * kAdjSubRec;
        const int chunks = (2 * (int)r[1] + 3) * (kSubStride / 2);
        for (int i = threadIdx.x; i < chunks; i += 96) cp_async16(dst + 2 * i, src + 2 * i);
      }
      cp_async_commit();
    };
    // the cotangent of the group's output: the planetesimal's (body 1)
    double lOp = ob ? a.lam[(size_t)c * N + j] : 0.0;
    double lOv = ob ? a.lam[(size_t)(3 + c) * N + j] : 0.0;
    if (M > 0) fetch(M - 1);
    for (int k = M - 1; k >= 0; --k) {
      if (k > 0) fetch(k - 1);
      else cp_async_commit();
      cp_async_wait1();   // record k's copy (all but the newest group) has landed
      bs2c_bar();
      double* B = s_rec + (k & 1) * kAdjSubRec;
      const double* r = tape + (size_t)k * stride;
      const double H = r[0];
      const int K = (int)r[1];
      const int nmax = 2 * (K + 1);
      const double dd = H * c_bs_inv_n[row], d2 = dd * dd;
      if ((int)r[14] < 0) {   // no slot: the forward's sub-steps again, into B
        double X = r[2 + 2 * c + ob];
        const double V = r[2 + 2 * (3 + c) + ob];
        int buf = 0;
        double A = bs2c_accel(tm, c, lane, X, sm, buf, B);
        double D = dd * fma(0.5 * dd, A, V);
        X += D;
        for (int st = 1; st <= nmax; ++st) {
          A = bs2c_accel(tm, c, lane, X, sm, buf, (st <= n) ? B + (size_t)st * kSubStride : nullptr);
          if (st < n) {
            D = fma(d2, A, D);
            X += D;
          }
        }
        bs2c_bar();
      }
      // reverse, the rows in lockstep from the longest accepted row down; a
      // lane's own sweep starts at its n (a lane with nothing to do carries
      // zero cotangents at kept positions, which add nothing)
      const bool act = row <= K;
      const double scale = act ? s_nw[K][row] : 0.0;
      const int top = min(n, nmax);
      double lX = scale * lOp, lD = scale * lOv / dd, lYv = 0.0;
      const double lA = scale * 0.5 * dd * lOv;   // O_v = D_n/dd + (dd/2) A(X_n)
      int par = 0;
      for (int st = nmax; st >= 0; --st) {
        double la;
        if (st > top) {
          la = 0.0;
        } else if (st == n) {
          la = lA;
        } else if (st >= 1) {   // X_{s+1} = X_s + D_{s+1}, D_{s+1} = D_s + d2 A(X_s)
          lD += lX;
          la = d2 * lD;
        } else {                // X_1 = X_0 + D_1, D_1 = dd V_0 + (dd^2/2) A(X_0)
          lD += lX;
          lYv = dd * lD;
          la = 0.5 * d2 * lD;
        }
        double* xl = s_la + par * 96;
        xl[c * 32 + lane] = la;
        bs2c_bar();
        const double l0 = xl[lane], l1 = xl[32 + lane], l2 = xl[64 + lane];
        par ^= 1;
        const double* e = B + (size_t)min(st, top) * kSubStride;
        const double x0 = e[lane], x1 = e[32 + lane], x2 = e[64 + lane];
        const double w = e[96 + lane];
        const double f = adj_wpm2(tm, e[160 + lane], e[128 + lane], w) *
                         fma(x0, l0, fma(x1, l1, x2 * l2));
        const double xc = (c == 0) ? x0 : ((c == 1) ? x1 : x2);
        const double cs = fma(f, xc, -w * la);
        const double cr = tm.pair ? -cs : 0.0;
        const double other = __shfl_xor_sync(0xffffffffu, cs, 2);
        const double react = __shfl_sync(0xffffffffu, cr, src_r);
        lX += (cs + other) + react;
      }
      // this row's share of the input cotangent, weighted; summed over rows
      double vp = act ? lX : 0.0, vv = act ? lYv : 0.0;
      vp += __shfl_xor_sync(0xffffffffu, vp, 4);
      vv += __shfl_xor_sync(0xffffffffu, vv, 4);
      vp += __shfl_xor_sync(0xffffffffu, vp, 8);
      vv += __shfl_xor_sync(0xffffffffu, vv, 8);
      vp += __shfl_xor_sync(0xffffffffu, vp, 16);
      vv += __shfl_xor_sync(0xffffffffu, vv, 16);
      lOp = vp;
      lOv = vv;
      bs2c_bar();   // B is read by every warp before the copy of record k - 2 lands in it
    }
    if (lane == 1) {   // body 1: the planetesimal's cotangent at its pre-drift state
      a.lam[(size_t)c * N + j] = lOp;
      a.lam[(size_t)(3 + c) * N + j] = lOv;
    }
    if (lane == 0) {   // body 0: the big body's share
      double* out = a.g_contrib + (size_t)g * 6 * kMaxGroup;
      out[c] = lOp;
      out[3 + c] = lOv;
    }
  }
}

// Many big bodies: one key per share of a member that a group does not write
// back, (body << 32 | item kMaxGroup + member), for k_sort_keys; the order of
// the sorted keys does not depend on the order they are written in.
__global__ void __launch_bounds__(kThreads) k_adj_share_keys(Dev d, Adj a) {
  const int W = min(*d.work_count, a.g_cap);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < W; g += gridDim.x * blockDim.x) {
    const int wf = d.work_wfrom[g];
    if (wf == 0 || !adj_takes(d, a, g)) continue;
    const int o = d.work_off[g];
    const int e0 = atomicAdd(a.scount, wf);
    for (int m = 0; m < wf; ++m) {
      if (e0 + m >= a.skeys_cap) {
        atomicOr(d.status, ST_WORK_OVF);
        break;
      }
      a.skeys[e0 + m] = ((unsigned long long)d.work_mem[o + m] << 32) |
                        (unsigned long long)(g * kMaxGroup + m);
    }
  }
}

// Each run of sorted keys of one body: its shares added in item order.
__global__ void __launch_bounds__(kThreads) k_adj_share_sum(Dev d, Adj a) {
  const int n = min(*a.scount, a.skeys_cap);
  const int N = d.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const unsigned body = (unsigned)(a.skeys[p] >> 32);
    if (p > 0 && (unsigned)(a.skeys[p - 1] >> 32) == body) continue;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int q = p; q < n && (unsigned)(a.skeys[q] >> 32) == body; ++q) {
      const unsigned e = (unsigned)(a.skeys[q] & 0xffffffffull);
      if (a.g_M[e / kMaxGroup] < 0) continue;
      const double* c6 = a.g_contrib + (size_t)e * 6;
      for (int c = 0; c < 6; ++c) acc[c] += c6[c];
    }
    for (int c = 0; c < 6; ++c) a.lam[(size_t)c * N + body] += acc[c];
  }
}

// Per system: the shares of the members a group does not write back (big
// bodies of test-particle groups) and the sum of their position parts for
// jump 1's momentum term.  With up to 64 big bodies a system's sums run over
// the items on all threads of the block (thread t takes items t, t + 256, ...
// in order) and end in a fixed pairwise tree; with more (sorted_shares, for
// every system), k_adj_share_sum has added each body's shares in item order.
// Either way the order is fixed.
__global__ void __launch_bounds__(kThreads) k_adj_bs_fold(Dev d, Adj a) {
  __shared__ double red[6][kThreads];
  const int sys = blockIdx.x;
  const SysDev& S = d.sys[sys];
  const int N = d.N;
  const int ng = min(*d.work_count, a.g_cap);
  const int t = threadIdx.x;
  auto in_sys = [&](int g) { return d.work_sys[g] == sys && a.g_M[g] >= 0; };
  // block-wide sum of v[0..nv) into red[.][0] (every thread must call it)
  auto tree = [&](const double* v, int nv) {
    for (int c = 0; c < nv; ++c) red[c][t] = v[c];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (t < w)
        for (int c = 0; c < nv; ++c) red[c][t] += red[c][t + w];
      __syncthreads();
    }
  };
  // item g's share for big body i (local index), added to acc
  auto add_share = [&](int g, int i, double* acc) {
    const int o = d.work_off[g], wf = d.work_wfrom[g];
    for (int m = 0; m < wf; ++m) {
      if (d.work_mem[o + m] - S.off != i) continue;
      const double* c6 = a.g_contrib + (size_t)g * 6 * kMaxGroup + 6 * m;
      for (int c = 0; c < 6; ++c) acc[c] += c6[c];
    }
  };
  if (a.sorted_shares) {
    // the shares were added by k_adj_share_sum
  } else if (S.nbig <= 64) {
    for (int i = 0; i < S.nbig; ++i) {
      double acc[6] = {0, 0, 0, 0, 0, 0};
      for (int g = t; g < ng; g += kThreads)
        if (in_sys(g)) add_share(g, i, acc);
      tree(acc, 6);
      if (t == 0)
        for (int c = 0; c < 6; ++c) a.lam[(size_t)c * N + S.off + i] += red[c][0];
      __syncthreads();
    }
  }
  double sx[3] = {0, 0, 0};
  for (int g = t; g < ng; g += kThreads) {
    if (!in_sys(g)) continue;
    const int wf = d.work_wfrom[g];
    for (int m = 0; m < wf; ++m)
      for (int c = 0; c < 3; ++c) sx[c] += a.g_contrib[(size_t)g * 6 * kMaxGroup + 6 * m + c];
  }
  tree(sx, 3);
  if (t < 3) a.bs_xsum[3 * sys + t] = red[t][0];
}

void launch_adjoint_bs_plan(const Dev& d, const Adj& a, cudaStream_t st) {
  // detection on the recomputed endpoints, without touching the step's log
  // (encounter flags, big-big count, deferral history)
  Dev dd = d;
  dd.ever = nullptr;
  dd.bb_count = nullptr;
  dd.defer = 0;
  cudaMemsetAsync(d.flags, 0, d.N, st);
  cudaMemsetAsync(d.pair_count, 0, sizeof(int), st);
  launch_detect(dd, a.x2, a.xv3, d.flags, d.keys, d.pair_count, d.pair_cap, 1, st);
  // sorted keys give the work items a fixed order (the shares' fold follows it)
  launch_sort_keys(d.keys, d.pair_count, d.pair_cap, 0, st);
  launch_groups(dd, st);   // the step's own groups: big groups, then test-particle groups
  k_adj_tape<<<1, 1024, 0, st>>>(dd, a);
}

void launch_adjoint_bs_fwd(const Dev& d, const Adj& a, int nblocks, cudaStream_t st) {
  if (a.sorted_shares) {
    cudaMemsetAsync(a.scount, 0, sizeof(int), st);
    k_adj_share_keys<<<a.bs_blocks, kThreads, 0, st>>>(d, a);
    launch_sort_keys(a.skeys, a.scount, a.skeys_cap, 0, st);
  }
  k_adj_bs_fwd<<<nblocks, 32, 0, st>>>(d, a);    // every item but the test-particle pairs
  k_adj_bs_fwd2<<<nblocks, 128, 0, st>>>(d, a);  // test-particle pairs
}

void launch_adjoint_bs_vjp(const Dev& d, const Adj& a, int nblocks, cudaStream_t st) {
  k_adj_bs_vjp<<<nblocks, 32, 0, st>>>(d, a);    // every item but the test-particle pairs
  cudaFuncSetAttribute(k_adj_bs_vjp2, cudaFuncAttributeMaxDynamicSharedMemorySize, kVjp2Smem);
  k_adj_bs_vjp2<<<nblocks, 96, kVjp2Smem, st>>>(d, a);   // test-particle pairs
}

void launch_adjoint_bs_fold(const Dev& d, const Adj& a, cudaStream_t st) {
  if (a.sorted_shares) k_adj_share_sum<<<a.bs_blocks, kThreads, 0, st>>>(d, a);
  k_adj_bs_fold<<<d.nsys, kThreads, 0, st>>>(d, a);
}

}  // namespace mx
