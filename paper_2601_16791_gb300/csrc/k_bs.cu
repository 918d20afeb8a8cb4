// k_bs.cu -- encounter groups and their Bulirsch-Stoer integration
// (arXiv 2601.16791, Sec. 2: close encounters leave the symplectic map for
// mdt_bs2, Bulirsch-Stoer for conservative forces; Sec. 2.1.1 listing for the
// error scales xscal = 1/|x|^2, vscal = 1/|v|^2; Sec. 2.1.2 for the pair
// forces of mfo_hkce, here the (1 - K) complement of the kick's weight).
//
// Groups: big bodies joined by flagged big-big pairs form big groups, each
// integrated on its own and giving its members' states; every flagged
// planetesimal forms a test-particle group with the big groups of the bigs it
// meets and only its own state is taken from it (it has no mass, so the big
// copies follow the same motion as in their own group).  The list is built by
// one block from the sorted pair keys, so it is the same on every run.
//
// Integrator: Stoermer's rule for x'' = a(x) with n_k = 2k sub-steps
// (k = 1..8), Aitken-Neville extrapolation in (H/n)^2, error = max over
// bodies of max(|dx|^2 xscal, |dv|^2 vscal) <= tol^2; accepted sub-steps grow
// by 1.3 (capped by what remains), failed ones halve.  Groups of up to four
// bodies run on lanes (k_bs_pack, then k_bs_spread for the long ones); larger
// groups run one per thread (k_bs).  On this part an FP64 instruction has
// ~67-cycle latency and costs the same for 1 or 32 active lanes, so a group's
// serial chain, not its arithmetic, sets the time: the rows and step
// candidates of a macro sub-step go on separate lanes to shorten it.
#include "mx_common.cuh"
#include "mx_kernels.h"

namespace mx {

__device__ __forceinline__ int sys_of(const Dev& d, int g) {
  int lo = 0, hi = d.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d.sys[mid].off <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int key_j(unsigned long long k) { return (int)((k >> 32) & 0x7fffffffull); }
__device__ __forceinline__ int key_i(unsigned long long k) { return (int)(k & 0xffffffffull); }
__device__ __forceinline__ bool key_small(unsigned long long k) { return (k >> 63) != 0; }

// Inclusive block scan of two ints (blockDim.x = 1024).
__device__ __forceinline__ void block_scan2(int& a, int& b, int* sa, int* sb) {
  const int t = threadIdx.x;
  sa[t] = a;
  sb[t] = b;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    const int xa = (t >= off) ? sa[t - off] : 0;
    const int xb = (t >= off) ? sb[t - off] : 0;
    __syncthreads();
    sa[t] += xa;
    sb[t] += xb;
    __syncthreads();
  }
  a = sa[t];
  b = sb[t];
}

// Members of the test-particle group of the run of pairs starting at p
// (same small body j): the big groups of its bigs, ascending, then j.
// Returns the member count, or -1 when it exceeds kMaxGroup.
__device__ int run_members(const unsigned long long* keys, int p, int n, const int* nodes,
                           int nnodes, const int* comp_of, const int* comp_start,
                           const int* comp_nodes, int* mem) {
  const int j = key_j(keys[p]);
  int cnt = 0;
  for (int q = p; q < n && key_j(keys[q]) == j; ++q) {
    const int i = key_i(keys[q]);
    // is i in a big group?
    int lo = 0, hi = nnodes - 1, at = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      if (nodes[mid] == i) { at = mid; break; }
      if (nodes[mid] < i) lo = mid + 1;
      else hi = mid - 1;
    }
    const int c = (at >= 0) ? comp_of[at] : -1;
    const int b0 = (c >= 0) ? comp_start[c] : 0;
    const int b1 = (c >= 0) ? comp_start[c + 1] : 1;
    for (int b = b0; b < b1; ++b) {
      const int g = (c >= 0) ? nodes[comp_nodes[b]] : i;
      bool seen = false;
      for (int e = 0; e < cnt; ++e) seen |= (mem[e] == g);
      if (seen) continue;
      if (cnt >= kMaxGroup - 1) return -1;
      // insert keeping ascending order
      int e = cnt;
      while (e > 0 && mem[e - 1] > g) {
        mem[e] = mem[e - 1];
        --e;
      }
      mem[e] = g;
      ++cnt;
    }
  }
  mem[cnt++] = j;
  return cnt;
}

__global__ void __launch_bounds__(1024) k_groups(Dev d) {
  __shared__ int nodes[2 * kMaxBigPairs];
  __shared__ int parent[2 * kMaxBigPairs];
  __shared__ int comp_of[2 * kMaxBigPairs];
  __shared__ int comp_start[2 * kMaxBigPairs + 1];
  __shared__ int comp_nodes[2 * kMaxBigPairs];
  __shared__ int sa[1024], sb[1024];
  __shared__ int s_nbb, s_nnodes, s_ncomp, s_bw, s_bm, s_bad;
  const int count = *d.pair_count;
  if (count > d.pair_cap) {
    if (threadIdx.x == 0) atomicOr(d.status, ST_PAIR_OVF);
    return;
  }
  const int n = count;
  if (n == 0) return;
  const unsigned long long* keys = d.keys;
  if (threadIdx.x == 0) {
    s_nbb = n;
    s_bad = 0;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x)
    if (key_small(keys[p]) && (p == 0 || !key_small(keys[p - 1]))) s_nbb = p;
  __syncthreads();
  const int nbb = s_nbb;
  if (nbb > kMaxBigPairs) {
    if (threadIdx.x == 0) atomicOr(d.status, ST_GROUP);
    return;
  }
  // ---- big groups: union-find over the (few) big-big pairs, one thread
  if (threadIdx.x == 0) {
    int nn = 0;
    for (int p = 0; p < nbb; ++p) {
      const int ab[2] = {key_i(keys[p]), key_j(keys[p])};
      for (int q = 0; q < 2; ++q) {
        const int g = ab[q];
        int e = nn;
        bool dup = false;
        for (int f = 0; f < nn; ++f) dup |= (nodes[f] == g);
        if (dup) continue;
        while (e > 0 && nodes[e - 1] > g) {
          nodes[e] = nodes[e - 1];
          --e;
        }
        nodes[e] = g;
        ++nn;
      }
    }
    for (int e = 0; e < nn; ++e) parent[e] = e;
    auto find_idx = [&](int g) {
      int lo = 0, hi = nn - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (nodes[mid] < g) lo = mid + 1;
        else hi = mid;
      }
      return lo;
    };
    auto root = [&](int e) {
      while (parent[e] != e) e = parent[e];
      return e;
    };
    for (int p = 0; p < nbb; ++p) {
      const int a = root(find_idx(key_i(keys[p])));
      const int b = root(find_idx(key_j(keys[p])));
      if (a != b) parent[max(a, b)] = min(a, b);
    }
    // components numbered in order of their smallest member
    int nc = 0;
    for (int e = 0; e < nn; ++e) {
      const int r = root(e);
      if (r == e) comp_of[e] = nc++;
      else comp_of[e] = comp_of[r];
    }
    for (int c = 0; c <= nc; ++c) comp_start[c] = 0;
    for (int e = 0; e < nn; ++e) comp_start[comp_of[e] + 1]++;
    for (int c = 0; c < nc; ++c) comp_start[c + 1] += comp_start[c];
    for (int c = 0; c < nc; ++c) {
      int fill = comp_start[c];
      for (int e = 0; e < nn; ++e)
        if (comp_of[e] == c) comp_nodes[fill++] = e;
    }
    // one work item per big group
    int m = 0;
    for (int c = 0; c < nc; ++c) {
      const int sz = comp_start[c + 1] - comp_start[c];
      if (sz > kMaxGroup) s_bad = ST_GROUP;
      if (c >= d.work_cap || m + sz > d.mem_cap) {
        s_bad = ST_WORK_OVF;
        break;
      }
      d.work_off[c] = m;
      d.work_sys[c] = sys_of(d, nodes[comp_nodes[comp_start[c]]]);
      d.work_wfrom[c] = 0;
      for (int b = comp_start[c]; b < comp_start[c + 1]; ++b) d.work_mem[m++] = nodes[comp_nodes[b]];
    }
    s_nnodes = nn;
    s_ncomp = nc;
    if (d.bb_count && nbb > 0) atomicAdd(d.bb_count, (unsigned long long)nbb);
    s_bw = nc;
    s_bm = m;
  }
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) atomicOr(d.status, (unsigned)s_bad);
    return;
  }
  // ---- test-particle groups: one per run of pairs with the same small body
  for (int cs = nbb; cs < n; cs += blockDim.x) {
    const int p = cs + threadIdx.x;
    const bool start = p < n && (p == nbb || key_j(keys[p]) != key_j(keys[p - 1]));
    int mem[kMaxGroup];
    int mc = 0;
    if (start) {
      mc = run_members(keys, p, n, nodes, s_nnodes, comp_of, comp_start, comp_nodes, mem);
      if (mc < 0) {
        s_bad = ST_GROUP;
        mc = 0;
      }
    }
    int ws = start ? 1 : 0, ms = mc;
    block_scan2(ws, ms, sa, sb);
    const int bw = s_bw, bm = s_bm;
    if (start && mc > 0) {
      const int w = bw + ws - 1;
      const int o = bm + ms - mc;
      if (w >= d.work_cap || o + mc > d.mem_cap) {
        s_bad = ST_WORK_OVF;
      } else {
        d.work_off[w] = o;
        d.work_sys[w] = sys_of(d, mem[mc - 1]);
        d.work_wfrom[w] = mc - 1;
        for (int e = 0; e < mc; ++e) d.work_mem[o + e] = mem[e];
      }
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) {
      s_bw = bw + ws;
      s_bm = bm + ms;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (s_bad) {
      atomicOr(d.status, (unsigned)s_bad);
      *d.work_count = 0;
    } else {
      const int W = min(s_bw, d.work_cap);
      *d.work_count = W;
      d.work_off[W] = s_bm;
    }
  }
}

// ---------------------------------------------------------------- integrator
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
__device__ void stoermer(const GroupState& G, double mu0, const double (*Y)[kMaxGroup], double H,
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

__device__ bool bs_integrate(const GroupState& G, double mu0, double h, double tol, int max_sub,
                             double (*Y)[kMaxGroup], int* nsub_out) {
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

// ------------------------------------------------- warp-cooperative groups
// Groups of up to kLaneMaxNB bodies run on lanes: lane 8c + r of a group
// integrates extrapolation row r (n = 2(r+1) Stoermer sub-steps) with the
// candidate step H/2^c.  The rows of a macro sub-step advance side by side;
// the Aitken-Neville table of each candidate is a wavefront across its 8
// lanes (row r takes row r-1's column j-1 by a shuffle); every lane checks its
// own row's error, and the lowest converged lane of the group's vote (smallest
// c, then smallest r) is accepted -- exactly what trying H, then H/2 after a
// failure, and so on, with the rows in order, would accept.
//
// Two phases.  k_bs_pack runs four groups per warp with one candidate (8
// lanes each) for at most kPackRounds macro sub-steps: cheap in FP64 issue
// slots, which cost the same for 1 or 32 active lanes.  Groups still running
// are saved to a continuation list, and k_bs_spread finishes them one per
// warp with four candidates on a grid of one warp per SM, so the few long
// chains (deep fly-bys) neither wait behind failed attempts nor share an
// SM's FP64 pipe.
constexpr int kLaneMaxNB = 4;
constexpr int kPackRounds = 3;

// Changeover constants of one member: rc^2, 0.01 rc^2, 0.1 rc, 1/(0.9 rc).
struct MemberK {
  double rc, rc2, rc2lo, rc01, i09;
};

template <int NB>
__device__ __forceinline__ void acc_nb(double mu0, const double* mu, const MemberK* K,
                                       const double (&X)[3][NB], double (&A)[3][NB]) {
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const double x = X[0][b], y = X[1][b], z = X[2][b];
    const double ir = rsqrt_d(fma(x, x, fma(y, y, z * z)));
    const double f = mu0 * (ir * ir) * ir;
    double ax = -f * x, ay = -f * y, az = -f * z;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      if (i == b || mu[i] == 0.0) continue;
      const double dx = x - X[0][i], dy = y - X[1][i], dz = z - X[2][i];
      const double s2 = fma(dx, dx, fma(dy, dy, dz * dz));
      // rc = max(rcrit_b, rcrit_i): the constants of the member with the larger radius
      const MemberK& k = (K[b].rc > K[i].rc) ? K[b] : K[i];
      if (s2 >= k.rc2) continue;
      const double yy = rsqrt_d(s2);
      double wgt = (yy * yy) * (yy * mu[i]);
      if (s2 > k.rc2lo) {
        const double q = fma(s2, yy, -k.rc01) * k.i09;
        wgt *= fma(-q * q * q, fma(q, fma(6.0, q, -15.0), 10.0), 1.0);
      }
      ax = fma(-wgt, dx, ax);
      ay = fma(-wgt, dy, ay);
      az = fma(-wgt, dz, az);
    }
    A[0][b] = ax;
    A[1][b] = ay;
    A[2][b] = az;
  }
}

// Integration state of one group between macro sub-steps.
template <int NB>
struct GroupRun {
  double Y[6][NB];
  double rem, H;
  int nsub;
};

// Up to max_rounds macro sub-steps of one group on the lanes of `gmask`
// (8 * NCAND lanes starting at warp lane `base`; this lane is base + 8c + r).
// Returns 1 when the step is done, 0 when rounds ran out, -1 at the cap.
template <int NB, int NCAND>
__device__ int bs_rounds(unsigned gmask, int base, int lane, double mu0, const double* mu,
                         const MemberK* K, double tol, int max_sub, int max_rounds,
                         GroupRun<NB>& g) {
  const int rel = lane - base;
  const int row = rel & 7, cand = rel >> 3;
  const double tol2 = tol * tol;
  double inv_den[kBsRows];
#pragma unroll
  for (int j = 1; j < kBsRows; ++j) {
    const double r = (double)(row + 1) / (double)(row - j + 1);
    inv_den[j] = (j <= row) ? 1.0 / (r * r - 1.0) : 0.0;
  }
  const int n = 2 * (row + 1);
  const double inv_n = 1.0 / n;
  const double cscale = 1.0 / (double)(1 << cand);
  for (int round = 0; round < max_rounds; ++round) {
    if (g.rem == 0.0) return 1;
    if (g.nsub >= max_sub) return -1;
    if (fabs(g.H) > fabs(g.rem)) g.H = g.rem;
    const double Hc = g.H * cscale;
    double xscal[NB], vscal[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      xscal[b] = rcp_d(fma(g.Y[0][b], g.Y[0][b], fma(g.Y[1][b], g.Y[1][b], g.Y[2][b] * g.Y[2][b])));
      vscal[b] = rcp_d(fma(g.Y[3][b], g.Y[3][b], fma(g.Y[4][b], g.Y[4][b], g.Y[5][b] * g.Y[5][b])));
    }
    double X[3][NB], A[3][NB], D[3][NB];
    const double dd = Hc * inv_n;
    const double d2 = dd * dd;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < NB; ++b) X[c][b] = g.Y[c][b];
    acc_nb<NB>(mu0, mu, K, X, A);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        D[c][b] = dd * fma(0.5 * dd, A[c][b], g.Y[3 + c][b]);
        X[c][b] += D[c][b];
      }
    for (int s = 1; s < n; ++s) {
      acc_nb<NB>(mu0, mu, K, X, A);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          D[c][b] = fma(d2, A[c][b], D[c][b]);
          X[c][b] += D[c][b];
        }
    }
    acc_nb<NB>(mu0, mu, K, X, A);
    double T[6][NB], Tp[6][NB];
    const double idd = n * rcp_d(Hc);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        T[c][b] = X[c][b];
        T[3 + c][b] = fma(D[c][b], idd, 0.5 * dd * A[c][b]);
        Tp[c][b] = T[c][b];
        Tp[3 + c][b] = T[3 + c][b];
      }
    __syncwarp(gmask);
#pragma unroll
    for (int j = 1; j < kBsRows; ++j) {
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const double up = __shfl_up_sync(gmask, T[c][b], 1, 8);
          if (row >= j) {
            if (row == j) Tp[c][b] = T[c][b];
            T[c][b] = fma(T[c][b] - up, inv_den[j], T[c][b]);
          }
        }
    }
    bool ok = false;
    if (row >= 1) {
      double err = 0.0;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        double ex = 0.0, ev = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double dx = T[c][b] - Tp[c][b];
          const double dv = T[3 + c][b] - Tp[3 + c][b];
          ex = fma(dx, dx, ex);
          ev = fma(dv, dv, ev);
        }
        err = fmax(err, fmax(ex * xscal[b], ev * vscal[b]));
      }
      ok = err <= tol2;
    }
    const unsigned vote = __ballot_sync(gmask, ok) & gmask;
    if (vote) {
      const int src = __ffs(vote) - 1;
      const int c_acc = (src - base) >> 3;
      g.nsub += c_acc + 1;                   // attempts a one-at-a-time search makes
      if (g.nsub > max_sub) return -1;
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int b = 0; b < NB; ++b) g.Y[c][b] = __shfl_sync(gmask, T[c][b], src);
      const double Hacc = g.H / (double)(1 << c_acc);
      g.rem -= Hacc;
      g.H = 1.3 * Hacc;
    } else {
      g.nsub += NCAND;
      g.H *= 1.0 / (double)(1 << NCAND);
    }
  }
  return (g.rem == 0.0) ? 1 : 0;
}

template <int NB>
__device__ __forceinline__ void load_members(const Dev& d, const SysDev& S, int o0, double* mu,
                                             MemberK* K) {
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int g = d.work_mem[o0 + m];
    const int l = g - S.off;
    const double rc = (l < S.nbig) ? d.brc[S.boff + l] : 0.0;
    mu[m] = (l < S.nbig) ? d.bmu[S.boff + l] : 0.0;
    K[m].rc = rc;
    K[m].rc2 = rc * rc;
    K[m].rc2lo = 0.01 * (rc * rc);
    K[m].rc01 = 0.1 * rc;
    K[m].i09 = (rc > 0.0) ? 1.0 / (0.9 * rc) : 0.0;
  }
}

template <int NB>
__device__ __forceinline__ void write_members(const Dev& d, int w, int o0, int lane_rel,
                                              const GroupRun<NB>& g) {
  const int wf = d.work_wfrom[w];
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    if (lane_rel == m && m >= wf) {
      const int gi = d.work_mem[o0 + m];
#pragma unroll
      for (int c = 0; c < 6; ++c) d.xv[(size_t)c * d.N + gi] = g.Y[c][m];
    }
  }
}

// Continuation record: rem, H, nsub, then Y.
constexpr int kContDoubles = 3 + 6 * kLaneMaxNB;

template <int NB>
__device__ void pack_group(const Dev& d, int w, unsigned gmask, int base, int lane) {
  const int o0 = d.work_off[w];
  const SysDev& S = d.sys[d.work_sys[w]];
  double mu[NB];
  MemberK K[NB];
  load_members<NB>(d, S, o0, mu, K);
  GroupRun<NB> g;
#pragma unroll
  for (int m = 0; m < NB; ++m)
#pragma unroll
    for (int c = 0; c < 6; ++c) g.Y[c][m] = d.xv0[(size_t)c * d.N + d.work_mem[o0 + m]];
  g.rem = S.h;
  g.H = S.h;
  g.nsub = 0;
  const int r = bs_rounds<NB, 1>(gmask, base, lane, S.mu0, mu, K, d.bs_tol, d.bs_max_sub,
                                 kPackRounds, g);
  if (r != 0) {
    if (lane == base) {
      if (r < 0) atomicOr(d.status, ST_BS);
      d.work_nsub[w] = g.nsub;
    }
    write_members<NB>(d, w, o0, lane - base, g);
    return;
  }
  // still running: hand over to k_bs_spread
  int slot = 0;
  if (lane == base) slot = atomicAdd(d.cont_count, 1);
  slot = __shfl_sync(gmask, slot, base);
  if (slot >= d.cont_cap) {   // list full: finish here
    const int r2 = bs_rounds<NB, 1>(gmask, base, lane, S.mu0, mu, K, d.bs_tol, d.bs_max_sub,
                                    1 << 30, g);
    if (lane == base) {
      if (r2 < 0) atomicOr(d.status, ST_BS);
      d.work_nsub[w] = g.nsub;
    }
    write_members<NB>(d, w, o0, lane - base, g);
    return;
  }
  if (lane == base) {
    double* c = d.cont_state + (size_t)slot * kContDoubles;
    d.cont_item[slot] = w;
    c[0] = g.rem;
    c[1] = g.H;
    c[2] = (double)g.nsub;
#pragma unroll
    for (int m = 0; m < NB; ++m)
#pragma unroll
      for (int q = 0; q < 6; ++q) c[3 + 6 * m + q] = g.Y[q][m];
  }
}

// Four groups of LO..HI bodies per warp, 8 lanes each (separate kernels keep
// the common two-body case free of the larger cases' register pressure).
template <int LO, int HI>
__global__ void __launch_bounds__(128) k_bs_pack(Dev d) {
  const int W = *d.work_count;
  const int lane = threadIdx.x & 31;
  const int slot = lane >> 3;
  const int base = slot * 8;
  const unsigned gmask = 0xffu << base;
  const int gslot = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4 + slot;
  const int nslots = (gridDim.x * blockDim.x >> 5) * 4;
  for (int w = gslot; w < W; w += nslots) {
    const int nb = d.work_off[w + 1] - d.work_off[w];
    if (nb < LO || nb > HI) continue;
    if (LO <= 1 && nb == 1) pack_group<(LO <= 1 ? 1 : LO)>(d, w, gmask, base, lane);
    else if (LO <= 2 && HI >= 2 && nb == 2) pack_group<2>(d, w, gmask, base, lane);
    else if (LO <= 3 && HI >= 3 && nb == 3) pack_group<(HI >= 3 ? 3 : 2)>(d, w, gmask, base, lane);
    else if (HI >= 4 && nb == 4) pack_group<(HI >= 4 ? 4 : 2)>(d, w, gmask, base, lane);
  }
}

template <int NB>
__device__ void spread_group(const Dev& d, int slot, int lane) {
  const int w = d.cont_item[slot];
  const int o0 = d.work_off[w];
  const SysDev& S = d.sys[d.work_sys[w]];
  double mu[NB];
  MemberK K[NB];
  load_members<NB>(d, S, o0, mu, K);
  GroupRun<NB> g;
  const double* c = d.cont_state + (size_t)slot * kContDoubles;
  g.rem = c[0];
  g.H = c[1];
  g.nsub = (int)c[2];
#pragma unroll
  for (int m = 0; m < NB; ++m)
#pragma unroll
    for (int q = 0; q < 6; ++q) g.Y[q][m] = c[3 + 6 * m + q];
  const int r = bs_rounds<NB, 4>(0xffffffffu, 0, lane, S.mu0, mu, K, d.bs_tol, d.bs_max_sub,
                                 1 << 30, g);
  if (lane == 0) {
    if (r < 0) atomicOr(d.status, ST_BS);
    d.work_nsub[w] = g.nsub;
  }
  write_members<NB>(d, w, o0, lane, g);
}

// The continued groups of LO..HI bodies, one per warp, four step candidates
// x eight rows.
template <int LO, int HI>
__global__ void __launch_bounds__(32) k_bs_spread(Dev d) {
  const int C = min(*d.cont_count, d.cont_cap);
  const int lane = threadIdx.x & 31;
  for (int slot = blockIdx.x; slot < C; slot += gridDim.x) {
    const int w = d.cont_item[slot];
    const int nb = d.work_off[w + 1] - d.work_off[w];
    if (nb < LO || nb > HI) continue;
    if (LO <= 1 && nb == 1) spread_group<(LO <= 1 ? 1 : LO)>(d, slot, lane);
    else if (LO <= 2 && HI >= 2 && nb == 2) spread_group<2>(d, slot, lane);
    else if (LO <= 3 && HI >= 3 && nb == 3) spread_group<(HI >= 3 ? 3 : 2)>(d, slot, lane);
    else if (HI >= 4 && nb == 4) spread_group<(HI >= 4 ? 4 : 2)>(d, slot, lane);
  }
}

// One thread per work item with more than kLaneMaxNB bodies, grid-stride.
__global__ void __launch_bounds__(32) k_bs(Dev d) {
  const int W = *d.work_count;
  const int N = d.N;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x) {
    const int o0 = d.work_off[w];
    const int nb = min(d.work_off[w + 1] - o0, kMaxGroup);   // the builder caps groups
    if (nb <= kLaneMaxNB) continue;
    GroupState G;
    G.nb = nb;
    const SysDev& S = d.sys[d.work_sys[w]];
    double Y[6][kMaxGroup];
    for (int m = 0; m < nb; ++m) {
      const int g = d.work_mem[o0 + m];
      const int l = g - S.off;
      G.mu[m] = (l < S.nbig) ? d.bmu[S.boff + l] : 0.0;
      G.rc[m] = (l < S.nbig) ? d.brc[S.boff + l] : 0.0;
      for (int c = 0; c < 6; ++c) Y[c][m] = d.xv0[(size_t)c * N + g];
    }
    int nsub = 0;
    if (!bs_integrate(G, S.mu0, S.h, d.bs_tol, d.bs_max_sub, Y, &nsub))
      atomicOr(d.status, ST_BS);
    d.work_nsub[w] = nsub;
    for (int m = d.work_wfrom[w]; m < nb; ++m) {
      const int g = d.work_mem[o0 + m];
      for (int c = 0; c < 6; ++c) d.xv[(size_t)c * N + g] = Y[c][m];
    }
  }
}

void launch_groups(const Dev& d, cudaStream_t st) { k_groups<<<1, 1024, 0, st>>>(d); }

void launch_bs(const Dev& d, int nblocks, cudaStream_t st) {
  // (a group has at least two members: one big body and the body it meets)
  cudaMemsetAsync(d.cont_count, 0, sizeof(int), st);
  k_bs_pack<2, 2><<<nblocks, 128, 0, st>>>(d);
  k_bs_pack<3, 4><<<nblocks, 128, 0, st>>>(d);
  k_bs<<<nblocks, 32, 0, st>>>(d);
  k_bs_spread<2, 2><<<nblocks / 4, 32, 0, st>>>(d);
  k_bs_spread<3, 4><<<nblocks / 4, 32, 0, st>>>(d);
}

}  // namespace mx
