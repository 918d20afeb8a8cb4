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
// (k = 1..8), Aitken-Neville extrapolation in (H/n)^2 kept as one in-place
// row, error = max over bodies of max(|dx|^2 xscal, |dv|^2 vscal) <= tol^2;
// accepted sub-steps grow by 1.3 (capped by what remains), failed ones halve.
// One thread per group; groups are independent.
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
// Groups of up to kLaneMaxNB bodies run on 8 lanes each (4 groups per warp):
// lane r of a group integrates extrapolation row r (n = 2(r+1) Stoermer
// sub-steps), so the 8 rows of one macro sub-step advance side by side instead
// of one after another.  The Aitken-Neville table is then built as a wavefront
// across the 8 lanes (row r takes row r-1's column j-1 by a shuffle), each lane
// checks its own row's error, and the lowest converged row is taken -- the
// same choice as evaluating the rows in order and stopping at the first one
// that converges.
constexpr int kLaneMaxNB = 4;

template <int NB>
__device__ __forceinline__ void acc_nb(double mu0, const double* mu, const double* rc,
                                       const double (&X)[3][NB], double (&A)[3][NB]) {
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const double x = X[0][b], y = X[1][b], z = X[2][b];
    const double ir = rsqrt_d(fma(x, x, fma(y, y, z * z)));
    const double f = mu0 * ir * ir * ir;
    double ax = -f * x, ay = -f * y, az = -f * z;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      if (i == b || mu[i] == 0.0) continue;
      const double dx = x - X[0][i], dy = y - X[1][i], dz = z - X[2][i];
      const double s2 = fma(dx, dx, fma(dy, dy, dz * dz));
      const double r = fmax(rc[b], rc[i]);
      const double r2 = r * r;
      if (s2 >= r2) continue;
      const double yy = rsqrt_d(s2);
      double wgt = yy * yy * yy;
      if (s2 > 0.01 * r2) {
        const double q = (s2 * yy - 0.1 * r) * (1.0 / (0.9 * r));
        wgt *= 1.0 - q * q * q * fma(q, fma(6.0, q, -15.0), 10.0);
      }
      wgt *= mu[i];
      ax = fma(-wgt, dx, ax);
      ay = fma(-wgt, dy, ay);
      az = fma(-wgt, dz, az);
    }
    A[0][b] = ax;
    A[1][b] = ay;
    A[2][b] = az;
  }
}

// One group on the 8 lanes of `mask` (lane r = row r).  Y is the group state
// (identical in all 8 lanes); returns false when the sub-step cap is hit.
template <int NB>
__device__ bool bs_lanes(unsigned mask, int row, double mu0, const double* mu, const double* rc,
                         double h, double tol, int max_sub, double (&Y)[6][NB], int* nsub_out) {
  const double tol2 = tol * tol;
  // 1 / ((n_row / n_{row-j})^2 - 1) for j = 1..row
  double inv_den[kBsRows];
#pragma unroll
  for (int j = 1; j < kBsRows; ++j) {
    const double r = (double)(row + 1) / (double)(row - j + 1);
    inv_den[j] = (j <= row) ? 1.0 / (r * r - 1.0) : 0.0;
  }
  const int n = 2 * (row + 1);
  double rem = h, H = h;
  int nsub = 0;
  while (rem != 0.0) {
    if (nsub >= max_sub) {
      *nsub_out = nsub;
      return false;
    }
    ++nsub;
    if (fabs(H) > fabs(rem)) H = rem;
    double xscal[NB], vscal[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      xscal[b] = 1.0 / fma(Y[0][b], Y[0][b], fma(Y[1][b], Y[1][b], Y[2][b] * Y[2][b]));
      vscal[b] = 1.0 / fma(Y[3][b], Y[3][b], fma(Y[4][b], Y[4][b], Y[5][b] * Y[5][b]));
    }
    // this lane's Stoermer row
    double X[3][NB], A[3][NB], D[3][NB];
    const double dd = H / n;
    const double d2 = dd * dd;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < NB; ++b) X[c][b] = Y[c][b];
    acc_nb<NB>(mu0, mu, rc, X, A);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        D[c][b] = dd * fma(0.5 * dd, A[c][b], Y[3 + c][b]);
        X[c][b] += D[c][b];
      }
    for (int s = 1; s < n; ++s) {
      acc_nb<NB>(mu0, mu, rc, X, A);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          D[c][b] = fma(d2, A[c][b], D[c][b]);
          X[c][b] += D[c][b];
        }
    }
    acc_nb<NB>(mu0, mu, rc, X, A);
    double T[6][NB], Tp[6][NB];
    const double idd = (double)n / H;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        T[c][b] = X[c][b];
        T[3 + c][b] = fma(D[c][b], idd, 0.5 * dd * A[c][b]);
        Tp[c][b] = T[c][b];
        Tp[3 + c][b] = T[3 + c][b];
      }
    __syncwarp(mask);
    // Aitken-Neville wavefront: after step j, lane r >= j holds T[r][j]
#pragma unroll
    for (int j = 1; j < kBsRows; ++j) {
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const double up = __shfl_up_sync(mask, T[c][b], 1, 8);
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
    const unsigned vote = __ballot_sync(mask, ok) & mask;
    if (vote) {
      const int lead = __ffs(vote) - 1;          // lowest converged row (warp lane)
      const int src = lead & 7;
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int b = 0; b < NB; ++b) Y[c][b] = __shfl_sync(mask, T[c][b], src, 8);
      rem -= H;
      H *= 1.3;
    } else {
      H *= 0.5;
    }
  }
  *nsub_out = nsub;
  return true;
}

template <int NB>
__device__ void bs_slot_group(const Dev& d, int w, unsigned mask, int row) {
  const int N = d.N;
  const int o0 = d.work_off[w];
  const SysDev& S = d.sys[d.work_sys[w]];
  double mu[NB], rc[NB], Y[6][NB];
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int g = d.work_mem[o0 + m];
    const int l = g - S.off;
    mu[m] = (l < S.nbig) ? d.bmu[S.boff + l] : 0.0;
    rc[m] = (l < S.nbig) ? d.brc[S.boff + l] : 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) Y[c][m] = d.xv0[(size_t)c * N + g];
  }
  int nsub = 0;
  const bool ok = bs_lanes<NB>(mask, row, S.mu0, mu, rc, S.h, d.bs_tol, d.bs_max_sub, Y, &nsub);
  if (row == 0) {
    if (!ok) atomicOr(d.status, ST_BS);
    d.work_nsub[w] = nsub;
    for (int m = d.work_wfrom[w]; m < NB; ++m) {
      const int g = d.work_mem[o0 + m];
#pragma unroll
      for (int c = 0; c < 6; ++c) d.xv[(size_t)c * N + g] = Y[c][m];
    }
  }
}

// 4 groups per warp, 8 lanes each; groups of more than kLaneMaxNB bodies are
// left to k_bs.
__global__ void __launch_bounds__(128) k_bs_lanes(Dev d) {
  const int W = *d.work_count;
  const int lane = threadIdx.x & 31;
  const int slot = lane >> 3, row = lane & 7;
  const unsigned mask = 0xffu << (8 * slot);
  const int gslot = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4 + slot;
  const int nslots = (gridDim.x * blockDim.x >> 5) * 4;
  for (int w = gslot; w < W; w += nslots) {
    const int nb = d.work_off[w + 1] - d.work_off[w];
    switch (nb) {
      case 1: bs_slot_group<1>(d, w, mask, row); break;
      case 2: bs_slot_group<2>(d, w, mask, row); break;
      case 3: bs_slot_group<3>(d, w, mask, row); break;
      case 4: bs_slot_group<4>(d, w, mask, row); break;
      default: break;
    }
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
  k_bs_lanes<<<nblocks, 128, 0, st>>>(d);
  k_bs<<<nblocks, 32, 0, st>>>(d);
}

}  // namespace mx
