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
// one block from the pair keys, which come as one contiguous run per target
// with the big bodies ascending; the runs' order varies, but no group's
// members or arithmetic depend on it.
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
#include <cooperative_groups.h>

#include "mx_common.cuh"
#include "mx_encounter.cuh"
#include "mx_kepler.cuh"
#include "mx_kernels.h"
#include "mx_bs.cuh"
#include "mx_bs2.cuh"
#include "mx_detect_body.cuh"
#include "mx_drift_body.cuh"
#include "mx_kick_body.cuh"
#include "mx_orbit.cuh"
#include "mx_physics.cuh"

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

// 2^-c for 0 <= c <= 1022, exactly, from its bit pattern (no FP64 division).
__device__ __forceinline__ double pow2_neg(int c) { return __hiloint2double((1023 - c) << 20, 0); }

__device__ __forceinline__ int key_j(unsigned long long k) { return (int)((k >> 32) & 0x7fffffffull); }
__device__ __forceinline__ int key_i(unsigned long long k) { return (int)(k & 0xffffffffull); }
__device__ __forceinline__ bool key_small(unsigned long long k) { return (k >> 63) != 0; }

// Inclusive block scan of two ints (blockDim.x a multiple of 32, at most
// 1024): shuffles within each warp, then one warp scans the warps' totals
// (sa, sb: 32 ints each of shared scratch).  Two block barriers.
__device__ __forceinline__ void block_scan2(int& a, int& b, int* sa, int* sb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int xa = __shfl_up_sync(0xffffffffu, a, o);
    const int xb = __shfl_up_sync(0xffffffffu, b, o);
    if (lane >= o) {
      a += xa;
      b += xb;
    }
  }
  if (lane == 31) {
    sa[warp] = a;
    sb[warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int ta = (lane < nw) ? sa[lane] : 0;
    int tb = (lane < nw) ? sb[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int xa = __shfl_up_sync(0xffffffffu, ta, o);
      const int xb = __shfl_up_sync(0xffffffffu, tb, o);
      if (lane >= o) {
        ta += xa;
        tb += xb;
      }
    }
    sa[lane] = ta;
    sb[lane] = tb;
  }
  __syncthreads();
  if (warp > 0) {
    a += sa[warp - 1];
    b += sb[warp - 1];
  }
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

constexpr int kGroupKeysSmem = 2048;   // 16 KB of static shared memory

// The encounter groups of the step from its pair keys, in one block of any
// size (a multiple of 32, at most 1024): big groups by union-find over the
// big-big pairs, then one test-particle group per run of keys with the same
// planetesimal, in key order.
__device__ __forceinline__ void groups_block(const Dev& d) {
  __shared__ int nodes[2 * kMaxBigPairs];
  __shared__ int parent[2 * kMaxBigPairs];
  __shared__ int comp_of[2 * kMaxBigPairs];
  __shared__ int comp_start[2 * kMaxBigPairs + 1];
  __shared__ int comp_nodes[2 * kMaxBigPairs];
  __shared__ int sa[32], sb[32];
  __shared__ int s_nbb, s_nnodes, s_ncomp, s_bw, s_bm, s_bad, s_slot;
  __shared__ unsigned long long bbk[kMaxBigPairs];   // the big-big pairs
  // the step's keys, read once from global memory when they fit
  __shared__ unsigned long long skeys[kGroupKeysSmem];
  const int count = *d.pair_count;
  if (count > d.pair_cap) {
    if (threadIdx.x == 0) atomicOr(d.status, ST_PAIR_OVF);
    return;
  }
  const int n = count;
  if (n == 0) return;
  const bool staged = n <= kGroupKeysSmem;
  const unsigned long long* keys = staged ? skeys : d.keys;
  if (threadIdx.x == 0) {
    s_nbb = 0;
    s_bad = 0;
    s_slot = d.defer ? *d.hstep : 0;   // read early, used by thread 0 below
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const unsigned long long k = d.keys[p];
    if (staged) skeys[p] = k;
    if (!key_small(k)) {
      const int q = atomicAdd(&s_nbb, 1);
      if (q < kMaxBigPairs) bbk[q] = k;
    }
  }
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
      const int ab[2] = {key_i(bbk[p]), key_j(bbk[p])};
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
      const int a = root(find_idx(key_i(bbk[p])));
      const int b = root(find_idx(key_j(bbk[p])));
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
    // big groups of this step, for the catch-up of deferred planetesimals
    const int slot = s_slot;
    if (d.defer && slot < d.hist_cap)
      for (int e = 0; e < nn; ++e) {
        const SysDev& Sg = d.sys[sys_of(d, nodes[e])];
        d.h_comp[(size_t)slot * d.NB + Sg.boff + (nodes[e] - Sg.off)] = comp_of[e];
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
  for (int cs = 0; cs < n; cs += blockDim.x) {
    const int p = cs + threadIdx.x;
    const bool start = p < n && key_small(keys[p]) && (p == 0 || key_j(keys[p]) != key_j(keys[p - 1]));
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

__global__ void __launch_bounds__(1024) k_groups(Dev d) { groups_block(d); }

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
// With deferral on, the one round of a two-body group in the packed phase
// stops at the check after this row when nothing has converged yet.
constexpr int kDeferRow = 3;

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
  const double cscale = pow2_neg(cand);   // 2^-cand, exact
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
      const double Hacc = g.H * pow2_neg(c_acc);   // exact: a power of two
      g.rem -= Hacc;
      g.H = 1.3 * Hacc;
    } else {
      g.nsub += NCAND;
      g.H *= 1.0 / (double)(1 << NCAND);
    }
  }
  return (g.rem == 0.0) ? 1 : 0;
}

// The members' masses and changeover constants (a big body's from set_rcrit's
// table, the same bits as computed here from r_c; a planetesimal has none).
template <int NB>
__device__ __forceinline__ void load_members(const Dev& d, const SysDev& S, int o0, double* mu,
                                             MemberK* K) {
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int g = d.work_mem[o0 + m];
    const int l = g - S.off;
    const bool big = l < S.nbig;
    const size_t b = (size_t)S.boff + (big ? l : 0);
    mu[m] = big ? d.bmu[b] : 0.0;
    K[m].rc = big ? d.brc[b] : 0.0;
    K[m].rc2 = big ? d.brc4[b] : 0.0;
    K[m].rc2lo = big ? d.brc4[d.NB + b] : 0.0;
    K[m].rc01 = big ? d.brc4[2 * (size_t)d.NB + b] : 0.0;
    K[m].i09 = big ? d.brc4[3 * (size_t)d.NB + b] : 0.0;
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


// Up to max_rounds macro sub-steps of a two-body group; this warp runs step
// candidate `cand` of NCAND (NCAND warps of the block, s_row[NCAND] and
// s_y[12] in shared memory when NCAND > 1).  Returns 1 when the step is done,
// 0 when rounds ran out, -1 at the sub-step cap.  g is the same on every lane
// and warp before and after.
template <int NCAND>
__device__ int bs2_rounds(int cand, int lane, const Bs2Term& t, double tol, int max_sub,
                          int max_rounds, GroupRun<2>& g, int* s_row, double* s_y,
                          unsigned long long* fevals = nullptr, int stop_row = kBsRows - 1) {
  const int row = lane >> 2, q = lane & 3, ob = q & 1;
  const bool vel = q >= 2;
  const int n = 2 * (row + 1);
  const double tol2 = tol * tol;
  const double cscale = pow2_neg(cand);   // 2^-cand, exact
  for (int round = 0; round < max_rounds; ++round) {
    if (g.rem == 0.0) return 1;
    if (g.nsub >= max_sub) return -1;
    if (fabs(g.H) > fabs(g.rem)) g.H = g.rem;
    const double Hc = g.H * cscale;
    double X[3], V[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X[c] = ob ? g.Y[c][1] : g.Y[c][0];
      V[c] = ob ? g.Y[3 + c][1] : g.Y[3 + c][0];
    }
    const double s0 = vel ? V[0] : X[0], s1 = vel ? V[1] : X[1], s2v = vel ? V[2] : X[2];
    const double sc = rcp_d(fma(s0, s0, fma(s1, s1, s2v * s2v)));
    const double dd = Hc * c_bs_inv_n[row];
    const double d2 = dd * dd;
    double A[3], D[3], Traw[3] = {0.0, 0.0, 0.0}, T[3];
    bs2_accel(t, X, A);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      D[c] = dd * fma(0.5 * dd, A[c], V[c]);
      X[c] += D[c];
    }
    int acc_c = -1, acc_r = -1;
    bool decided = false;
    for (int s = 1; s <= 2 * kBsRows && !decided; ++s) {
      bs2_accel(t, X, A);
      if (s < n) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          D[c] = fma(d2, A[c], D[c]);
          X[c] += D[c];
        }
      } else if (s == n) {
        const double idd = n * rcp_d(Hc);
#pragma unroll
        for (int c = 0; c < 3; ++c) Traw[c] = vel ? fma(D[c], idd, 0.5 * dd * A[c]) : X[c];
      }
      const int K = (s >> 1) - 1;   // the row that completed at this sub-step
      if ((s & 1) || !((kBs2Checks >> K) & 1u)) continue;
      const int r = bs2_check(K, row, sc, tol2, Traw, T);
      if (NCAND == 1) {
        if (r >= 0) {
          acc_c = 0;
          acc_r = r;
          decided = true;
        } else if (K >= stop_row && K < kBsRows - 1) {
          return 0;   // handed over before the round is decided: g is as it was
        } else if (K == kBsRows - 1) {
          decided = true;
        }
      } else {
        if (lane == 0) s_row[cand] = r;
        __syncthreads();
        if (s_row[0] >= 0) {
          acc_c = 0;
          acc_r = s_row[0];
          decided = true;
        } else if (K == kBsRows - 1) {
          for (int c = 1; c < NCAND && acc_c < 0; ++c)
            if (s_row[c] >= 0) {
              acc_c = c;
              acc_r = s_row[c];
            }
          decided = true;
        }
        __syncthreads();
      }
    }
    if (acc_c >= 0) {
      // the accepted row's lanes hold x0, x1 (q = 0, 1) and v0, v1 (q = 2, 3)
      if (NCAND == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          g.Y[c][0] = __shfl_sync(0xffffffffu, T[c], 4 * acc_r + 0);
          g.Y[c][1] = __shfl_sync(0xffffffffu, T[c], 4 * acc_r + 1);
          g.Y[3 + c][0] = __shfl_sync(0xffffffffu, T[c], 4 * acc_r + 2);
          g.Y[3 + c][1] = __shfl_sync(0xffffffffu, T[c], 4 * acc_r + 3);
        }
      } else {
        if (cand == acc_c && row == acc_r)
#pragma unroll
          for (int c = 0; c < 3; ++c) s_y[3 * q + c] = T[c];
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          g.Y[c][0] = s_y[c];
          g.Y[c][1] = s_y[3 + c];
          g.Y[3 + c][0] = s_y[6 + c];
          g.Y[3 + c][1] = s_y[9 + c];
        }
        __syncthreads();
      }
      g.nsub += acc_c + 1;                   // attempts a one-at-a-time search makes
      // force evaluations of that search: every row of each failed try, rows
      // 0..acc_r of the accepted one (row r: 2(r + 1) sub-steps + 1)
      if (fevals && cand == 0 && lane == 0)
        atomicAdd(fevals, (unsigned long long)(80 * acc_c + (acc_r + 1) * (acc_r + 3)));
      if (g.nsub > max_sub) return -1;
      const double Hacc = g.H * pow2_neg(acc_c);   // exact: a power of two
      g.rem -= Hacc;
      g.H = 1.3 * Hacc;
    } else {
      if (fevals && cand == 0 && lane == 0) atomicAdd(fevals, (unsigned long long)(80 * NCAND));
      g.nsub += NCAND;
      g.H *= 1.0 / (double)(1 << NCAND);
    }
  }
  return (g.rem == 0.0) ? 1 : 0;
}

// The two CTAs of a catch-up cluster try H (rank 0) and H/2 (rank 1) in the
// same round, as the first two candidates of bs2_rounds.  Each CTA's mailbox
// receives the other's message: rank 0's the H/2 try (its lowest converged
// row, or -1, and that row's state), rank 1's the round's outcome (the
// accepted candidate and row, or -1, and the new state).  A message is
// written, then fenced at cluster scope, then its round number is stored in
// `seq`; the reader polls `seq` (at most kMailSpin polls).
struct ClusterMail {
  double* y;          // [12] state in the message
  volatile int* hdr;  // [2] candidate, row
  volatile int* seq;  // [1] round number of the message
  volatile int* ack;  // [1] rank 0's: the last outcome rank 1 has read
  int* round;         // [1] rounds run by this CTA's catch-up so far (both CTAs alike)
  int* flag;          // [1] scratch: a word one thread read, for the three warps
  int cta;            // 0 or 1
  unsigned* status;
};
constexpr long long kMailSpin = 1ll << 26;   // about a second of polls

// Writes this CTA's message into the other CTA's mailbox: lanes of row
// `row_sel` hold coordinate c of the state's four vectors (x0, x1, v0, v1).
__device__ __forceinline__ void mail_send(const ClusterMail& mb, int c, int lane, int row,
                                          int row_sel, int cand, int r, double T, int seq) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned other = (unsigned)(1 - mb.cta);
  double* ry = cl.map_shared_rank(mb.y, other);
  int* rh = cl.map_shared_rank(const_cast<int*>(mb.hdr), other);
  int* rs = cl.map_shared_rank(const_cast<int*>(mb.seq), other);
  if (r >= 0 && row == row_sel) ry[3 * (lane & 3) + c] = T;
  if (c == 0 && lane == 0) {
    rh[0] = cand;
    rh[1] = r;
  }
  bs2c_bar();
  if (c == 0 && lane == 0) {
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
    *reinterpret_cast<volatile int*>(rs) = seq;
  }
}

// Waits until *w >= v (one thread polls, the three warps get its answer);
// false if that did not happen within kMailSpin polls (ST_BARRIER).
__device__ __forceinline__ bool mail_wait_word(const ClusterMail& mb, volatile int* w, int v,
                                               int c, int lane) {
  if (c == 0 && lane == 0) {
    long long k = 0;
    int ok = 1;
    while (*w < v) {   // a shared-memory word: a poll costs tens of cycles
      if (++k > kMailSpin) {
        atomicOr(mb.status, ST_BARRIER);
        ok = 0;
        break;
      }
    }
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
    *mb.flag = ok;
  }
  bs2c_bar();
  const bool ok = *mb.flag != 0;
  bs2c_bar();
  return ok;
}

// The message of round `seq` in this CTA's mailbox.  Round numbers only grow,
// and the other CTA sends the message of a round only after this CTA's
// message of the round before has been read, so the word reaches `seq` and
// stays there while this CTA waits.
__device__ __forceinline__ bool mail_wait(const ClusterMail& mb, int seq, int c, int lane) {
  return mail_wait_word(mb, mb.seq, seq, c, lane);
}

// Up to max_rounds tries per CTA (one per round); returns 1 when the step is
// done, 0 when rounds ran out, -1 at the sub-step cap, as bs2_rounds does.
// With `mb` the CTA is one of a cluster pair (above); without, it tries one
// candidate per round alone.
__device__ int bs2c_rounds(int c, int lane, const Bs2Term& t, double tol, int max_sub,
                           int max_rounds, GroupRun<2>& g, const Bs2cSmem& sm,
                           unsigned long long* fevals, const ClusterMail* mb = nullptr) {
  const int row = lane >> 2, q = lane & 3, ob = q & 1;
  const bool vel = q >= 2;
  const int n = 2 * (row + 1);
  const double tol2 = tol * tol;
  const int cand = mb ? mb->cta : 0;
  const int ncand = mb ? 2 : 1;
  int buf = 0;
  for (int round = 0; round < max_rounds; ++round) {
    if (g.rem == 0.0) return 1;
    if (g.nsub >= max_sub) return -1;
    if (fabs(g.H) > fabs(g.rem)) g.H = g.rem;
    int seq = 0;
    if (mb) {
      seq = *mb->round + 1;
      bs2c_bar();   // every warp has read the round number
      if (c == 0 && lane == 0) *mb->round = seq;
    }
    const double Hc = g.H * pow2_neg(cand);
    double X = ob ? g.Y[c][1] : g.Y[c][0];
    const double V = ob ? g.Y[3 + c][1] : g.Y[3 + c][0];
    const int so = vel ? 3 : 0;
    const double s0 = ob ? g.Y[so][1] : g.Y[so][0];
    const double s1 = ob ? g.Y[so + 1][1] : g.Y[so + 1][0];
    const double s2v = ob ? g.Y[so + 2][1] : g.Y[so + 2][0];
    const double sc = rcp_d(fma(s0, s0, fma(s1, s1, s2v * s2v)));
    const double dd = Hc * c_bs_inv_n[row];
    const double d2 = dd * dd;
    double A = bs2c_accel(t, c, lane, X, sm, buf);
    double D = dd * fma(0.5 * dd, A, V);
    X += D;
    double Traw = 0.0, T = 0.0;
    int acc_r = -1;
    bool decided = false, moot = false;
    for (int st = 1; st <= 2 * kBsRows && !decided; ++st) {
      A = bs2c_accel(t, c, lane, X, sm, buf);
      if (st < n) {
        D = fma(d2, A, D);
        X += D;
      } else if (st == n) {
        const double idd = n * rcp_d(Hc);
        Traw = vel ? fma(D, idd, 0.5 * dd * A) : X;
      }
      const int K = (st >> 1) - 1;   // the row that completed at this sub-step
      if ((st & 1) || !((kBs2Checks >> K) & 1u)) continue;
      const int r = bs2c_check(K, row, c, lane, sc, tol2, Traw, T, sm);
      if (r >= 0) {
        acc_r = r;
        decided = true;
      } else if (K == kBsRows - 1) {
        decided = true;
      } else if (mb && cand == 1) {
        // rank 0 has already decided the round: this try no longer matters
        if (c == 0 && lane == 0) *mb->flag = (*mb->seq >= seq) ? 1 : 0;
        bs2c_bar();
        moot = *mb->flag != 0;
        bs2c_bar();
        decided = moot;
      }
    }
    int acc_c = (acc_r >= 0) ? cand : -1;
    if (mb) {
      bool ok = true;
      if (cand == 1) {
        if (!moot) mail_send(*mb, c, lane, row, acc_r, 1, acc_r, T, seq);
        ok = mail_wait(*mb, seq, c, lane);
        acc_c = ok ? mb->hdr[0] : -1;
        acc_r = ok ? mb->hdr[1] : -1;
        if (ok && acc_c >= 0 && row == acc_r) T = mb->y[3 * q + c];
        bs2c_bar();   // every warp has read the outcome: rank 0 may send the next one
        if (c == 0 && lane == 0) {
          namespace cg = cooperative_groups;
          int* rack = cg::this_cluster().map_shared_rank(const_cast<int*>(mb->ack), 0u);
          asm volatile("fence.acq_rel.cluster;" ::: "memory");
          *reinterpret_cast<volatile int*>(rack) = seq;
        }
      } else {
        if (acc_c < 0) {   // H failed: the round is H/2's try
          ok = mail_wait(*mb, seq, c, lane);
          acc_r = ok ? mb->hdr[1] : -1;
          acc_c = (acc_r >= 0) ? 1 : -1;
          if (acc_c == 1 && row == acc_r) T = mb->y[3 * q + c];
        }
        // rank 1 has read the last round's outcome before this one replaces it
        ok = ok && mail_wait_word(*mb, mb->ack, seq - 1, c, lane);
        mail_send(*mb, c, lane, row, acc_r, acc_c, acc_r, T, seq);
      }
      bs2c_bar();
      if (!ok) return -1;
      if (acc_c >= 0) {
        // the accepted state: both ranks hold it on the lanes of row acc_r
        // (the own try's, or the other's copied in from the mailbox)
        if (row == acc_r) sm.y[3 * q + c] = T;
        bs2c_bar();
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          g.Y[k][0] = sm.y[k];
          g.Y[k][1] = sm.y[3 + k];
          g.Y[3 + k][0] = sm.y[6 + k];
          g.Y[3 + k][1] = sm.y[9 + k];
        }
        bs2c_bar();
        g.nsub += acc_c + 1;
        if (fevals && cand == 0 && c == 0 && lane == 0)
          atomicAdd(fevals, (unsigned long long)(80 * acc_c + (acc_r + 1) * (acc_r + 3)));
        if (g.nsub > max_sub) return -1;
        const double Hacc = g.H * pow2_neg(acc_c);
        g.rem -= Hacc;
        g.H = 1.3 * Hacc;
      } else {
        if (fevals && cand == 0 && c == 0 && lane == 0)
          atomicAdd(fevals, (unsigned long long)(80 * ncand));
        g.nsub += ncand;
        g.H *= 1.0 / (double)(1 << 2);
      }
      continue;
    }
    if (acc_r >= 0) {
      // the accepted row's lanes hold coordinate c of x0, x1 (q = 0, 1) and
      // v0, v1 (q = 2, 3)
      if (row == acc_r) sm.y[3 * q + c] = T;
      bs2c_bar();
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        g.Y[k][0] = sm.y[k];
        g.Y[k][1] = sm.y[3 + k];
        g.Y[3 + k][0] = sm.y[6 + k];
        g.Y[3 + k][1] = sm.y[9 + k];
      }
      bs2c_bar();
      g.nsub += 1;
      if (fevals && c == 0 && lane == 0)
        atomicAdd(fevals, (unsigned long long)((acc_r + 1) * (acc_r + 3)));
      if (g.nsub > max_sub) return -1;
      const double Hacc = g.H * pow2_neg(0);
      g.rem -= Hacc;
      g.H = 1.3 * Hacc;
    } else {
      if (fevals && c == 0 && lane == 0) atomicAdd(fevals, 80ull);
      g.nsub += 1;
      g.H *= 1.0 / (double)(1 << 1);
    }
  }
  return (g.rem == 0.0) ? 1 : 0;
}

// Continuation record: rem, H, nsub, then Y.
constexpr int kContDoubles = 3 + 6 * kLaneMaxNB;

// After the packed rounds (result r of the round function): finished groups
// are written; a test-particle group still running is deferred to the
// window's catch-up when deferral is on; anything else goes to the spread
// phase, or, with its list full, is finished here by `finish_here`.
template <int NB, class Finish>
__device__ void pack_tail(const Dev& d, int w, unsigned gmask, int base, int lane, int o0, int r,
                          GroupRun<NB>& g, Finish&& finish_here) {
  if (r != 0) {
    if (lane == base) {
      if (r < 0) atomicOr(d.status, ST_BS);
      d.work_nsub[w] = g.nsub;
    }
    write_members<NB>(d, w, o0, lane - base, g);
    return;
  }
  // still running.  A test-particle group (only the planetesimal's state is
  // kept) leaves the step: the body is deferred to the window's catch-up.
  if (d.defer && d.work_wfrom[w] == NB - 1 && d.sys[d.work_sys[w]].nbig <= kDeferMaxBig) {
    const int hs = *d.hstep;
    int rr = d.dcap;
    if (lane == base && hs < d.hist_cap) rr = atomicAdd(&d.rcount[0], 1);
    rr = __shfl_sync(gmask, rr, base);
    if (rr < d.dcap) {
      if (lane == base) {
        const int j = d.work_mem[o0 + NB - 1];
        int* R = d.d_rec + (size_t)rr * kRecInts;   // bank 0: deferred in this window
        R[0] = j;
        R[1] = hs;
        R[2] = NB;
#pragma unroll
        for (int m = 0; m < kLaneMaxNB; ++m) R[3 + m] = (m < NB) ? d.work_mem[o0 + m] : j;
        R[7] = -1;
        R[8] = 0;
        double* c = d.d_state + (size_t)rr * kRecDoubles;
        c[0] = g.rem;
        c[1] = g.H;
        c[2] = (double)g.nsub;
#pragma unroll
        for (int m = 0; m < NB; ++m)
#pragma unroll
          for (int q = 0; q < 6; ++q) c[3 + 6 * m + q] = g.Y[q][m];
        d.work_nsub[w] = g.nsub;
        d.lag[j] = 1;
        atomicAdd(d.defer_total, 1ull);
      }
      return;
    }
  }
  // hand over to the spread phase; with deferral on (no spread launches) a
  // big-body group, or a group the record banks had no room for, finishes here
  int slot = d.cont_cap;
  if (!d.defer) {
    if (lane == base) slot = atomicAdd(d.cont_count, 1);
    slot = __shfl_sync(gmask, slot, base);
  }
  if (slot >= d.cont_cap) {   // list full or no spread phase: finish here
    const int r2 = finish_here(g);
    if (r2 == 2) return;   // the caller finishes the group itself
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

template <int NB>
__device__ __noinline__ void pack_group(const Dev& d, int w, unsigned gmask, int base, int lane) {
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
  // with deferral on, a group that needs a second round leaves the step at once
  const int r = bs_rounds<NB, 1>(gmask, base, lane, S.mu0, mu, K, d.bs_tol, d.bs_max_sub,
                                 d.defer ? 1 : kPackRounds, g);
  pack_tail<NB>(d, w, gmask, base, lane, o0, r, g, [&](GroupRun<NB>& gg) {
    return bs_rounds<NB, 1>(gmask, base, lane, S.mu0, mu, K, d.bs_tol, d.bs_max_sub, 1 << 30, gg);
  });
}

__device__ void pack_two(const Dev& d, int w, int lane);
__device__ void pack_two_pair(const Dev& d, int a, int b, int lane);
__device__ __noinline__ void thread_group(const Dev& d, int w);

// Two-body groups, one per warp (term lanes, one candidate).
__global__ void __launch_bounds__(32) k_bs_pack2(Dev d) {
  const int W = *d.work_count;
  for (int w = blockIdx.x; w < W; w += gridDim.x)
    if (d.work_off[w + 1] - d.work_off[w] == 2) pack_two(d, w, threadIdx.x);
}

// Every group, one per warp, in one launch: two bodies on term lanes, three
// or four on the lane integrator (eight lanes), more on one thread.  Used
// with deferral on, where nothing is handed to a spread phase.
__device__ __forceinline__ void bs_one_warp(const Dev& d, int w, int lane) {
  const int nb = d.work_off[w + 1] - d.work_off[w];
  if (nb == 2) pack_two(d, w, lane);
  else if (nb == 3) { if (lane < 8) pack_group<3>(d, w, 0xffu, 0, lane); }
  else if (nb == 4) { if (lane < 8) pack_group<4>(d, w, 0xffu, 0, lane); }
  else if (nb > kLaneMaxNB && lane == 0) thread_group(d, w);
  __syncwarp();
}

// A two-body group whose planetesimal may be deferred: with deferral on,
// pack_two makes one try and gives it up at row kDeferRow, so only rows
// 0..kDeferRow of its lanes ever count.
__device__ __forceinline__ bool two_deferrable(const Dev& d, int w) {
  return d.defer && d.work_off[w + 1] - d.work_off[w] == 2 && d.work_wfrom[w] == 1 &&
         d.sys[d.work_sys[w]].nbig <= kDeferMaxBig;
}

// The work items go to the warps in pairs (2s, 2s + 1).  A pair of deferrable
// two-body groups shares the warp (pack_two_pair, 16 lanes each); any other
// pair is taken one item after the other.
__device__ __forceinline__ void bs_all_warps(const Dev& d, int w0, int nw) {
  const int W = *d.work_count;
  const int lane = threadIdx.x & 31;
  for (int sp = w0; 2 * sp < W; sp += nw) {
    const int a = 2 * sp, b = 2 * sp + 1;
    if (b < W && two_deferrable(d, a) && two_deferrable(d, b)) {
      pack_two_pair(d, a, b, lane);
    } else {
      bs_one_warp(d, a, lane);
      if (b < W) bs_one_warp(d, b, lane);
    }
  }
}

__global__ void __launch_bounds__(32) k_bs_all(Dev d) { bs_all_warps(d, blockIdx.x, gridDim.x); }

__device__ void pack_two(const Dev& d, int w, int lane) {
  const int o0 = d.work_off[w];
  const SysDev& S = d.sys[d.work_sys[w]];
  double mu[2];
  MemberK K[2];
  load_members<2>(d, S, o0, mu, K);
  const Bs2Term t = bs2_term(lane & 3, S.mu0, mu, K);
  GroupRun<2> g;
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int c = 0; c < 6; ++c) g.Y[c][m] = d.xv0[(size_t)c * d.N + d.work_mem[o0 + m]];
  g.rem = S.h;
  g.H = S.h;
  g.nsub = 0;
  // with deferral on, a group whose first try has not converged by row
  // kDeferRow goes to the catch-up, which runs that macro sub-step again
  // from the start with four candidates (the same steps are accepted)
  const int r = bs2_rounds<1>(0, lane, t, d.bs_tol, d.bs_max_sub, d.defer ? 1 : kPackRounds, g,
                              nullptr, nullptr, nullptr, d.defer ? kDeferRow : kBsRows - 1);
  pack_tail<2>(d, w, 0xffffffffu, 0, lane, o0, r, g, [&](GroupRun<2>& gg) {
    return bs2_rounds<1>(0, lane, t, d.bs_tol, d.bs_max_sub, 1 << 30, gg, nullptr, nullptr);
  });
}

// bs2_check on the 16 lanes of half `hs` (0 or 16) of the warp: the lowest
// converged row of that half.  Every lane of the warp calls it.
__device__ __forceinline__ int bs2_check_half(int K, int row, int hs, double sc, double tol2,
                                              const double (&Traw)[3], double (&T)[3]) {
  double Tp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) T[c] = Tp[c] = Traw[c];
#pragma unroll
  for (int j = 1; j <= kDeferRow; ++j) {
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
  long long eb = __double_as_longlong(e);
  eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 1));
  eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 2));
  const bool conv = row >= 1 && row <= K && eb <= __double_as_longlong(tol2);
  const unsigned v = (__ballot_sync(0xffffffffu, conv) >> hs) & 0xffffu;
  return v ? ((__ffs(v) - 1) >> 2) : -1;
}

// One round of bs2_rounds<1> (max_rounds 1, stop_row kDeferRow) on the 16
// lanes of this lane's half of the warp: lane 16h + 4r + q holds row r <=
// kDeferRow and force term q of the half's group.  The arithmetic of every
// row and check is bs2_rounds' own, so the round returns what bs2_rounds
// returns and leaves g as it leaves it.  The halves run in lockstep (every
// shuffle and vote takes the whole warp) until both have decided.
__device__ int bs2_half_round(int lane, const Bs2Term& t, double tol, int max_sub,
                              GroupRun<2>& g) {
  const int hs = lane & 16, row = (lane >> 2) & 3, q = lane & 3, ob = q & 1;
  const bool vel = q >= 2;
  const int n = 2 * (row + 1);
  const double tol2 = tol * tol;
  int res = 2;   // 2: the try decides
  if (g.rem == 0.0) res = 1;
  else if (g.nsub >= max_sub) res = -1;
  if (res == 2 && fabs(g.H) > fabs(g.rem)) g.H = g.rem;
  const double Hc = g.H * pow2_neg(0);
  double X[3], V[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    X[c] = ob ? g.Y[c][1] : g.Y[c][0];
    V[c] = ob ? g.Y[3 + c][1] : g.Y[3 + c][0];
  }
  const double s0 = vel ? V[0] : X[0], s1 = vel ? V[1] : X[1], s2v = vel ? V[2] : X[2];
  const double sc = rcp_d(fma(s0, s0, fma(s1, s1, s2v * s2v)));
  const double dd = Hc * c_bs_inv_n[row];
  const double d2 = dd * dd;
  double A[3], D[3], Traw[3] = {0.0, 0.0, 0.0}, T[3], Tacc[3] = {0.0, 0.0, 0.0};
  bs2_accel(t, X, A);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    D[c] = dd * fma(0.5 * dd, A[c], V[c]);
    X[c] += D[c];
  }
  int acc_r = -1;
  bool done = res != 2;
  for (int s = 1; s <= 2 * (kDeferRow + 1); ++s) {
    if (__all_sync(0xffffffffu, done)) break;
    bs2_accel(t, X, A);
    if (s < n) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        D[c] = fma(d2, A[c], D[c]);
        X[c] += D[c];
      }
    } else if (s == n) {
      const double idd = n * rcp_d(Hc);
#pragma unroll
      for (int c = 0; c < 3; ++c) Traw[c] = vel ? fma(D[c], idd, 0.5 * dd * A[c]) : X[c];
    }
    const int K = (s >> 1) - 1;   // the row that completed at this sub-step
    if ((s & 1) || !((kBs2Checks >> K) & 1u)) continue;
    const int r = bs2_check_half(K, row, hs, sc, tol2, Traw, T);
    if (!done) {
      if (r >= 0) {
        acc_r = r;
        done = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) Tacc[c] = T[c];
      } else if (K >= kDeferRow) {
        done = true;   // handed over before the round is decided: g is as it was
      }
    }
  }
  // the accepted row's lanes hold x0, x1 (q = 0, 1) and v0, v1 (q = 2, 3)
  const int src = hs + 4 * (acc_r >= 0 ? acc_r : 0);
  double Yn[6][2];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Yn[c][0] = __shfl_sync(0xffffffffu, Tacc[c], src + 0);
    Yn[c][1] = __shfl_sync(0xffffffffu, Tacc[c], src + 1);
    Yn[3 + c][0] = __shfl_sync(0xffffffffu, Tacc[c], src + 2);
    Yn[3 + c][1] = __shfl_sync(0xffffffffu, Tacc[c], src + 3);
  }
  if (res != 2) return res;
  if (acc_r < 0) return 0;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    g.Y[c][0] = Yn[c][0];
    g.Y[c][1] = Yn[c][1];
  }
  g.nsub += 1;
  if (g.nsub > max_sub) return -1;
  const double Hacc = g.H * pow2_neg(0);
  g.rem -= Hacc;
  g.H = 1.3 * Hacc;
  return (g.rem == 0.0) ? 1 : 0;
}

// Two deferrable two-body groups a and b on one warp, 16 lanes each (lanes
// 0-15: a, 16-31: b): pack_two's round on the half (bs2_half_round), then
// pack_tail.  A group pack_tail would finish in the step (the record banks
// full) is finished afterwards by the whole warp from where its half left it,
// as pack_two finishes it.
__device__ void pack_two_pair(const Dev& d, int a, int b, int lane) {
  const int hs = lane & 16;
  const int w = hs ? b : a;
  const int o0 = d.work_off[w];
  const SysDev& S = d.sys[d.work_sys[w]];
  double mu[2];
  MemberK K[2];
  load_members<2>(d, S, o0, mu, K);
  const Bs2Term t = bs2_term(lane & 3, S.mu0, mu, K);
  GroupRun<2> g;
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int c = 0; c < 6; ++c) g.Y[c][m] = d.xv0[(size_t)c * d.N + d.work_mem[o0 + m]];
  g.rem = S.h;
  g.H = S.h;
  g.nsub = 0;
  const int r = bs2_half_round(lane, t, d.bs_tol, d.bs_max_sub, g);
  bool fin = false;
  pack_tail<2>(d, w, 0xffffu << hs, hs, lane, o0, r, g, [&](GroupRun<2>&) {
    fin = true;
    return 2;
  });
  const unsigned fins = __ballot_sync(0xffffffffu, fin && (lane & 15) == 0);
  for (int h = 0; h < 32; h += 16) {
    if (!(fins & (1u << h))) continue;
    const int wf = h ? b : a;
    const int of = d.work_off[wf];
    const SysDev& Sf = d.sys[d.work_sys[wf]];
    double muf[2];
    MemberK Kf[2];
    load_members<2>(d, Sf, of, muf, Kf);
    const Bs2Term tf = bs2_term(lane & 3, Sf.mu0, muf, Kf);
    GroupRun<2> gf;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int c = 0; c < 6; ++c) gf.Y[c][m] = __shfl_sync(0xffffffffu, g.Y[c][m], h);
    gf.rem = __shfl_sync(0xffffffffu, g.rem, h);
    gf.H = __shfl_sync(0xffffffffu, g.H, h);
    gf.nsub = __shfl_sync(0xffffffffu, g.nsub, h);
    const int r2 = bs2_rounds<1>(0, lane, tf, d.bs_tol, d.bs_max_sub, 1 << 30, gf, nullptr, nullptr);
    if (lane == 0) {
      if (r2 < 0) atomicOr(d.status, ST_BS);
      d.work_nsub[wf] = gf.nsub;
    }
    write_members<2>(d, wf, of, lane, gf);
  }
  __syncwarp();
}

// Two-body groups handed over by k_bs_pack2: one per block of four warps,
// one step candidate per warp.
__global__ void __launch_bounds__(128) k_bs_spread2(Dev d) {
  __shared__ int s_row[4];
  __shared__ double s_y[12];
  const int C = min(*d.cont_count, d.cont_cap);
  const int lane = threadIdx.x & 31, cand = threadIdx.x >> 5;
  for (int slot = blockIdx.x; slot < C; slot += gridDim.x) {
    const int w = d.cont_item[slot];
    const int o0 = d.work_off[w];
    if (d.work_off[w + 1] - o0 != 2) continue;
    const SysDev& S = d.sys[d.work_sys[w]];
    double mu[2];
    MemberK K[2];
    load_members<2>(d, S, o0, mu, K);
    const Bs2Term t = bs2_term(lane & 3, S.mu0, mu, K);
    GroupRun<2> g;
    const double* c = d.cont_state + (size_t)slot * kContDoubles;
    g.rem = c[0];
    g.H = c[1];
    g.nsub = (int)c[2];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int q = 0; q < 6; ++q) g.Y[q][m] = c[3 + 6 * m + q];
    const int r = bs2_rounds<4>(cand, lane, t, d.bs_tol, d.bs_max_sub, 1 << 30, g, s_row, s_y);
    if (cand == 0) {
      if (lane == 0) {
        if (r < 0) atomicOr(d.status, ST_BS);
        d.work_nsub[w] = g.nsub;
      }
      write_members<2>(d, w, o0, lane, g);
    }
  }
}

// Four groups of LO..HI bodies per warp, 8 lanes each (separate kernels keep
// the common two-body case free of the larger cases' register pressure).  One
// warp per block: consecutive blocks land on different SMs, so the groups
// spread over all SMs' FP64 pipes instead of filling a few SMs' worth of
// four-warp blocks.
template <int LO, int HI>
__global__ void __launch_bounds__(32) k_bs_pack(Dev d) {
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

// A group of more than kLaneMaxNB bodies on one thread.
__device__ __noinline__ void thread_group(const Dev& d, int w) {
  const int N = d.N;
  const int o0 = d.work_off[w];
  const int nb = min(d.work_off[w + 1] - o0, kMaxGroup);   // the builder caps groups
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
  if (!bs_integrate(G, S.mu0, S.h, d.bs_tol, d.bs_max_sub, Y, &nsub)) atomicOr(d.status, ST_BS);
  d.work_nsub[w] = nsub;
  for (int m = d.work_wfrom[w]; m < nb; ++m) {
    const int g = d.work_mem[o0 + m];
    for (int c = 0; c < 6; ++c) d.xv[(size_t)c * N + g] = Y[c][m];
  }
}

// One thread per work item with more than kLaneMaxNB bodies, grid-stride.
__global__ void __launch_bounds__(32) k_bs(Dev d) {
  const int W = *d.work_count;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x)
    if (d.work_off[w + 1] - d.work_off[w] > kLaneMaxNB) thread_group(d, w);
}

// ----------------------------------------------- deferred planetesimals
// k_catchup replays the steps of deferred planetesimals (one body per block
// of four warps).  A window's history slots are whole steps and the leading
// half kicks of calls.  Each step is the direct path's own arithmetic on the
// big bodies' recorded history: jump (P of jump 1), Kepler drift, the
// encounter test against every big body (same screen and FP64 test as
// k_detect), Bulirsch-Stoer of its test-particle group from the pre-drift
// states (the integrators of the packed and spread phases, which accept the
// same sub-steps), jump (P of jump 2), gravity of the staged big positions in
// ascending order and the half kick(s) with drag.  So a deferred body ends
// where the direct path would have put it, bit for bit.  Each body has a
// cluster of two CTAs of four warps, on two SMs.  Both CTAs and all their
// warps take the same path (each warp on its own scheduler, so the repeated
// work costs no time); in a two-body group's Bulirsch-Stoer rounds warps 0-2
// of each CTA split the coordinates and the CTAs try H and H/2
// (bs2c_rounds); only warp 0 of rank 0 writes.
//
// Modes (CatchArgs::mode):
//  0  window end, main stream: every body deferred in the window and every
//     body carried from the last one is replayed towards the window's end;
//     a two-body group met on the way (or still running) may take at most
//     kCatchBudget macro sub-steps here.  Bodies that get to the end rejoin
//     the step; the others are carried (copied to bank_out).
//  1  side stream, while the main stream runs the next window: the carried
//     bodies are replayed to the window's end without a budget (in place).
//     This mode writes no state, lag flag or pair list, only the records.
//  2  settle: everything is replayed to the end and rejoins the step.
// Zero: any encounter goes to the side stream.  Measured on the gas disk,
// budgets of 1, 2 and 4 sub-steps made the main-stream pass (which the step
// waits for) 2.2-2.5x longer and the step about 6% slower.
constexpr int kCatchBudget = 0;
// Group-size field of a record whose body the ejection test removed during a
// side-stream pass (the state in the record is the one it keeps).
constexpr int kRecEjected = -3;

struct CatchArgs {
  int mode;
  int bank_a, bank_b;   // input banks (-1: none)
  int bank_out;         // mode 0: bank of the carried bodies
  int t_end;            // replay slots up to (not including) t_end
  int tl;               // the range's last whole-step slot (pair list), -1 none
  int next_slot;        // the history slot of the next step (modes 0 and 2, else -1)
  int t_next;           // where the next range starts: a body that reached t_end is kept there
};

// Big-body mu and changeover radius during slot t (the history's: masses
// and radii can change after the slot, by growth or removal).
template <int NB>
__device__ __forceinline__ void load_members_g(const Dev& d, const SysDev& S, const int* gid,
                                               int t, double* mu, MemberK* K) {
  const double* hmu = d.h_mu + (size_t)t * d.NB + S.boff;
  const double* hrc = d.h_rc + (size_t)t * d.NB + S.boff;
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int l = gid[m] - S.off;
    const double rc = (l < S.nbig) ? hrc[l] : 0.0;
    mu[m] = (l < S.nbig) ? hmu[l] : 0.0;
    K[m].rc = rc;
    K[m].rc2 = rc * rc;
    K[m].rc2lo = 0.01 * (rc * rc);
    K[m].rc01 = 0.1 * rc;
    K[m].i09 = (rc > 0.0) ? 1.0 / (0.9 * rc) : 0.0;
  }
}

struct CatchBlk {
  int lane, wq;
  int cta;                   // rank in the cluster pair (only rank 0 writes)
  unsigned long long* ops;   // work counters of this pass (main or side stream)
  Bs2cSmem b2;               // two-body groups on three warps (bs2c_rounds)
  const ClusterMail* mail;   // the pair's mailboxes
  double* s_g;               // [15] a group's run state, broadcast to the block
  int* s_row;     // [4]
  double* s_y;    // [12]
  double* s_bc;   // [6] broadcast of a body state
  int* s_r;       // [1] broadcast of a result code
};

// A test-particle group in progress: members, integration state.
struct CatchGroup {
  int nb;
  int gid[kLaneMaxNB];
  double rem, H;
  int nsub;
  double Y[6][kLaneMaxNB];
};

// Three or four bodies: the lane integrator of k_bs_spread on one warp, run
// to the end of the step.
template <int NB>
__device__ __noinline__ int catch_bs(const Dev& d, const SysDev& S, const CatchGroup& G, int t,
                                     int lane, double* s6) {
  double mu[NB];
  MemberK K[NB];
  load_members_g<NB>(d, S, G.gid, t, mu, K);
  GroupRun<NB> g;
#pragma unroll
  for (int m = 0; m < NB; ++m)
#pragma unroll
    for (int q = 0; q < 6; ++q) g.Y[q][m] = G.Y[q][m];
  g.rem = G.rem;
  g.H = G.H;
  g.nsub = G.nsub;
  const int r = bs_rounds<NB, 4>(0xffffffffu, 0, lane, S.mu0, mu, K, d.bs_tol, d.bs_max_sub,
                                 1 << 30, g);
#pragma unroll
  for (int q = 0; q < 6; ++q) s6[q] = g.Y[q][NB - 1];
  return r;
}

// Runs the group for at most max_rounds macro sub-steps (two bodies: term
// lanes, one candidate per warp; three or four: to the end of the step on
// warp 0, then broadcast).  Returns 1 (done, body state in s6), 0 (rounds ran
// out, G updated) or -1 (sub-step cap).
__device__ int catch_bs_any(const Dev& d, const SysDev& S, CatchGroup& G, int t,
                            int max_rounds, const CatchBlk& B, double* s6) {
  if (G.nb == 2) {
    double mu[2];
    MemberK K[2];
    load_members_g<2>(d, S, G.gid, t, mu, K);
    const Bs2Term t = bs2_term(B.lane & 3, S.mu0, mu, K);
    GroupRun<2> g;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int q = 0; q < 6; ++q) g.Y[q][m] = G.Y[q][m];
    g.rem = G.rem;
    g.H = G.H;
    g.nsub = G.nsub;
    // warps 0-2 integrate; the result reaches warp 3 through shared memory
    int r = 0;
    if (B.wq < 3) r = bs2c_rounds(B.wq, B.lane, t, d.bs_tol, d.bs_max_sub, max_rounds, g, B.b2,
                                  B.cta == 0 ? B.ops + 2 : nullptr, B.mail);
    __syncthreads();
    if (threadIdx.x == 0) {
      *B.s_r = r;
      B.s_g[0] = g.rem;
      B.s_g[1] = g.H;
      B.s_g[2] = (double)g.nsub;
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int q = 0; q < 6; ++q) B.s_g[3 + 6 * m + q] = g.Y[q][m];
    }
    __syncthreads();
    r = *B.s_r;
    G.rem = B.s_g[0];
    G.H = B.s_g[1];
    G.nsub = (int)B.s_g[2];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int q = 0; q < 6; ++q) G.Y[q][m] = B.s_g[3 + 6 * m + q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 6; ++q) s6[q] = G.Y[q][1];
    return r;
  }
  if (B.wq == 0) {
    const int r = (G.nb == 3) ? catch_bs<3>(d, S, G, t, B.lane, s6)
                              : catch_bs<4>(d, S, G, t, B.lane, s6);
    if (B.lane == 0) {
      for (int q = 0; q < 6; ++q) B.s_bc[q] = s6[q];
      *B.s_r = r;
    }
  }
  __syncthreads();
  for (int q = 0; q < 6; ++q) s6[q] = B.s_bc[q];
  const int r = *B.s_r;
  __syncthreads();
  return r;
}

// The thread integrator of k_bs for a group of more than four bodies
// (cnt big bodies mem[], then the planetesimal with pre-drift state a0).
__device__ __noinline__ void catch_bs_thread(const Dev& d, const SysDev& S, const int* mem, int cnt,
                                             const double* a0, int t, double* out) {
  const size_t NBs = (size_t)d.NB;
  const double* B0 = d.h_b0 + (size_t)t * 6 * NBs + S.boff;
  const int nb = cnt + 1;
  const double* hmu = d.h_mu + (size_t)t * NBs + S.boff;
  const double* hrc = d.h_rc + (size_t)t * NBs + S.boff;
  GroupState G;
  G.nb = nb;
  double Y[6][kMaxGroup];
  for (int m = 0; m < nb; ++m) {
    const bool big = m < cnt;
    G.mu[m] = big ? hmu[mem[m]] : 0.0;
    G.rc[m] = big ? hrc[mem[m]] : 0.0;
    for (int q = 0; q < 6; ++q) Y[q][m] = big ? B0[(size_t)q * NBs + mem[m]] : a0[q];
  }
  int nsub = 0;
  if (!bs_integrate(G, S.mu0, S.h, d.bs_tol, d.bs_max_sub, Y, &nsub)) atomicOr(d.status, ST_BS);
  for (int q = 0; q < 6; ++q) out[q] = Y[q][nb - 1];
}

// Jump 1, drift and the encounter test of step t.  No encounter: returns 0
// with the drifted state in s6.  A group of up to four bodies: returns its
// size with the group set up in G (pre-drift states, a fresh step).  Larger
// groups are integrated here (returns 0).  keys: 0 ignore, 1 append the
// pairs to the pair list (the last step of a range on the main stream), 2
// keep them in *kn / kl for the record (the side stream).
__device__ int catch_front(const Dev& d, const SysDev& S, int sys, int j, int t, int keys,
                           const CatchBlk& B, double* s6, CatchGroup& G, int* kn, int* kl) {
  const int lane = B.lane;
  const bool w0 = B.wq == 0;
  const bool wr = w0 && B.cta == 0;   // the warp that writes (rank 1 replays alike, silently)
  const size_t NBs = (size_t)d.NB;
  if (wr && lane == 0) atomicAdd(B.ops + 0, 1ull);
  double dj[3];
  jump_vec(d.h_P + (size_t)t * 6 * d.nsys + 3 * sys, S, 0.5, dj);
  double x = s6[0] + dj[0], y = s6[1] + dj[1], z = s6[2] + dj[2];
  double u = s6[3], v = s6[4], w = s6[5];
  const double a0[6] = {x, y, z, u, v, w};
  if (!kepler_drift(S.mu0, S.h, d.kepler_max_iter, x, y, z, u, v, w) && wr && lane == 0)
    atomicOr(d.status, ST_KEPLER);
  const double a1[6] = {x, y, z, u, v, w};
  float af[12];
  for (int k = 0; k < 6; ++k) {
    af[k] = to_float_bits(a0[k]);
    af[6 + k] = to_float_bits(a1[k]);
  }
  const double* B0 = d.h_b0 + (size_t)t * 6 * NBs + S.boff;
  const double* B1 = d.h_b1 + (size_t)t * 6 * NBs + S.boff;
  const double* hmu = d.h_mu + (size_t)t * NBs + S.boff;
  const double* hrc = d.h_rc + (size_t)t * NBs + S.boff;
  const float hf = to_float_bits(S.h);
  // flagged big bodies, ascending
  int fl[kMaxGroup];
  int nf = 0;
  bool over = false;
  for (int c0 = 0; c0 < S.nbig; c0 += 32) {
    const int l = c0 + lane;
    bool hit = false;
    if (l < S.nbig && hmu[l] >= 0.0) {   // a body removed by then meets nothing
      const double rcb = hrc[l];
      const float rcf = fmaxf(to_float_bits(rcb), 0.0f);
      float bf[12];
      double b0[6], b1[6];
      for (int q = 0; q < 6; ++q) {
        b0[q] = B0[(size_t)q * NBs + l];
        b1[q] = B1[(size_t)q * NBs + l];
        bf[q] = to_float_bits(b0[q]);
        bf[6 + q] = to_float_bits(b1[q]);
      }
      if (encounter_screen(af, bf, rcf * rcf, hf)) {
        const double rc = fmax(rcb, 0.0);
        hit = encounter_fp64(a0, b0, a1, b1, S.h, rc * rc);
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit && wr) {
      const int gi = S.off + l;
      if (d.ever) {
        d.ever[gi] = 1;
        d.ever[j] = 1;
      }
      if (keys == 1) {
        d.flags[gi] = 1;
        const int pos = atomicAdd(d.pair_count, 1);
        if (pos < d.pair_cap)
          d.keys[pos] = (1ull << 63) | ((unsigned long long)(unsigned)j << 32) | (unsigned)gi;
      }
    }
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      if (nf < kMaxGroup) fl[nf++] = c0 + b;
      else over = true;
    }
  }
  if (keys == 1 && wr && lane == 0) d.flags[j] = nf > 0 ? 1 : 0;
  if (keys == 2) {
    *kn = nf;
    for (int e = 0; e < nf; ++e) kl[e] = fl[e];
  }
  for (int q = 0; q < 6; ++q) s6[q] = a1[q];
  if (nf == 0) return 0;
  // members: the big groups of the flagged bodies (ascending), then j
  const int* comp = d.h_comp + (size_t)t * NBs + S.boff;
  int mem[kMaxGroup];
  int cnt = 0;
  bool bad = over;
  for (int e = 0; e < nf && !bad; ++e) {
    const int ce = comp[fl[e]];
    const int b0 = (ce >= 0) ? 0 : fl[e];
    const int b1 = (ce >= 0) ? S.nbig : fl[e] + 1;
    for (int b = b0; b < b1 && !bad; ++b) {
      if (ce >= 0 && comp[b] != ce) continue;
      bool seen = false;
      for (int q = 0; q < cnt; ++q) seen |= (mem[q] == b);
      if (seen) continue;
      if (cnt >= kMaxGroup - 1) {
        bad = true;
        break;
      }
      int q = cnt;
      while (q > 0 && mem[q - 1] > b) {
        mem[q] = mem[q - 1];
        --q;
      }
      mem[q] = b;
      ++cnt;
    }
  }
  if (bad) {   // the direct path skips the step's Bulirsch-Stoer and reports it
    if (wr && lane == 0) atomicOr(d.status, ST_GROUP);
    return 0;
  }
  const int nb = cnt + 1;
  if (nb <= kLaneMaxNB) {
    G.nb = nb;
    for (int m = 0; m < kLaneMaxNB; ++m) {
      const bool big = m < cnt;
      G.gid[m] = big ? S.off + mem[m] : j;
      for (int q = 0; q < 6; ++q) G.Y[q][m] = big ? B0[(size_t)q * NBs + mem[m]] : a0[q];
    }
    G.rem = S.h;
    G.H = S.h;
    G.nsub = 0;
    return nb;
  }
  // more than four bodies: the thread integrator of k_bs, on one thread
  if (w0 && lane == 0) catch_bs_thread(d, S, mem, cnt, a0, t, B.s_bc);
  __syncthreads();
  for (int q = 0; q < 6; ++q) s6[q] = B.s_bc[q];
  __syncthreads();
  return 0;
}

// Jump 2 and the half kick(s) that end step t, or (head) the leading half
// kick of a call, which has no jump and keeps the positions as they are.
__device__ void catch_back(const Dev& d, const SysDev& S, int sys, int j, int t, bool lead,
                           double* s6, unsigned long long* ops) {
  const double* P2 = d.h_P + (size_t)t * 6 * d.nsys + 3 * d.nsys + 3 * sys;
  const int hk = d.h_nkick[t];
  const bool head = hk < 0;
  double dj[3];
  jump_vec(P2, S, head ? 0.0 : 0.5, dj);
  const double x = s6[0] + dj[0], y = s6[1] + dj[1], z = s6[2] + dj[2];
  double u = s6[3], v = s6[4], w = s6[5];
  const double* BX = d.h_bx + (size_t)t * 3 * d.NB + S.boff;
  const double* hmu = d.h_mu + (size_t)t * d.NB + S.boff;
  const double* hrc = d.h_rc + (size_t)t * d.NB + S.boff;
  // the pairs' weights on the lanes (lane l: big body c0 + l), then the sum
  // in ascending order, as the kick's loop makes it (the same bits)
  double ax = 0, ay = 0, az = 0;
  const int lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < S.nbig; c0 += 32) {
    const int l = c0 + lane;
    double f = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    if (l < S.nbig) {
      const double rc = hrc[l];
      ex = x - BX[l];
      ey = y - BX[d.NB + l];
      ez = z - BX[2 * (size_t)d.NB + l];
      f = pair_weight(ex, ey, ez, fmax(hmu[l], 0.0), rc * rc, 0.01 * (rc * rc), 0.1 * rc,
                      (rc > 0.0) ? 1.0 / (0.9 * rc) : 0.0);
    }
    const int cn = min(32, S.nbig - c0);
    for (int k = 0; k < cn; ++k) {
      const double fk = __shfl_sync(0xffffffffu, f, k);
      ax = fma(-fk, __shfl_sync(0xffffffffu, ex, k), ax);
      ay = fma(-fk, __shfl_sync(0xffffffffu, ey, k), ay);
      az = fma(-fk, __shfl_sync(0xffffffffu, ez, k), az);
    }
  }
  const int nk = head ? -hk : hk;
  if (lead) atomicAdd(ops + 1, (unsigned long long)nk);
  const double kick_h = 0.5 * S.h;
  const double hp0 = P2[0] * S.inv_mu0, hp1 = P2[1] * S.inv_mu0, hp2 = P2[2] * S.inv_mu0;
  const double rp = S.gas_on ? d.rp_cm[j] : 0.0, kd = S.gas_on ? d.kdrag[j] : 0.0;
  GasAt gq = S.gas_on ? gas_at(S, x, y) : GasAt{false, 0.0, 0.0, 0.0};
  if (S.gas_on && S.grow_on) {   // the slot's gaps, as in k_jump_kick
    const double* hg = d.h_gap + (size_t)t * 3 * d.NB + S.boff;
    gq.rho *= gap_factor(hg, hg + d.NB, hg + 2 * (size_t)d.NB, S.nbig, x, y);
  }
  if (S.gas_on && S.dg_on) {   // as in k_jump_kick
    ax += gq.adg[0];
    ay += gq.adg[1];
  }
  const DragConst dc = S.gas_on ? drag_const(S, gq, x, y, hp0, hp1, hp2, rp, kd) : DragConst{};
  for (int kk = 0; kk < nk; ++kk) {   // as in k_jump_kick
    if (S.gas_on) {
      int kout = 0;
      double dvec[3];
      const double coef = gas_drag_coef(S, dc, u, v, w, dvec, -1, &kout);
      kick_with_drag(kick_h, ax, ay, az, coef, dvec, u, v, w);
    } else {
      u = fma(kick_h, ax, u);
      v = fma(kick_h, ay, v);
      w = fma(kick_h, az, w);
    }
  }
  if (!(finite_d(x) && finite_d(y) && finite_d(z) && finite_d(u) && finite_d(v) && finite_d(w)) &&
      lead)
    atomicOr(d.status, ST_NONFINITE);
  if (!head) {
    s6[0] = x;
    s6[1] = y;
    s6[2] = z;
  }
  s6[3] = u;
  s6[4] = v;
  s6[5] = w;
}

__device__ __forceinline__ int* rec_ints(const Dev& d, int bank, int idx) {
  return d.d_rec + ((size_t)bank * d.dcap + idx) * kRecInts;
}
__device__ __forceinline__ double* rec_state(const Dev& d, int bank, int idx) {
  return d.d_state + ((size_t)bank * d.dcap + idx) * kRecDoubles;
}

// One record from the start of its progress to a.t_end (or, mode 0, until a
// group outruns the budget).
__device__ void catch_record(const Dev& d, const CatchArgs& a, int bank, int idx,
                             const CatchBlk& B) {
  const bool lead = threadIdx.x == 0 && B.cta == 0;
  const int* R = rec_ints(d, bank, idx);
  const double* Cs = rec_state(d, bank, idx);
  const int j = R[0];
  int t = R[1];
  int kslot = R[7], kn = R[8];
  int kl[kMaxGroup];
  for (int e = 0; e < kMaxGroup; ++e) kl[e] = (e < kn) ? R[9 + e] : 0;
  const int sys = sys_of(d, j);
  const SysDev& S = d.sys[sys];
  // settle: pairs the side stream found at the range's last step
  if (a.mode == 2 && kslot >= 0 && kslot == a.tl && lead) {
    for (int e = 0; e < kn; ++e) {
      const int gi = S.off + kl[e];
      d.flags[gi] = 1;
      const int pos = atomicAdd(d.pair_count, 1);
      if (pos < d.pair_cap)
        d.keys[pos] = (1ull << 63) | ((unsigned long long)(unsigned)j << 32) | (unsigned)gi;
    }
    d.flags[j] = kn > 0 ? 1 : 0;
  }
  if (R[2] == kRecEjected) {   // removed during a side-stream pass: the main stream finishes it
    if (a.mode != 1 && lead) {
      for (int q = 0; q < 6; ++q) d.xv[q * (size_t)d.N + j] = Cs[3 + q];
      d.stat[j] = kStatEjected;
      atomicAdd(d.ej_new, 1);
      d.lag[j] = 0;
    }
    return;
  }
  // stored pairs are valid only until the next pass over the record (slots are reused)
  kslot = -1;
  kn = 0;
  CatchGroup G;
  G.nb = R[2];
  double s6[6];
  for (int q = 0; q < 6; ++q) s6[q] = 0.0;
  if (G.nb >= 2) {
    for (int m = 0; m < kLaneMaxNB; ++m) {
      G.gid[m] = (m < G.nb) ? R[3 + m] : j;
      for (int q = 0; q < 6; ++q) G.Y[q][m] = (m < G.nb) ? Cs[3 + 6 * m + q] : 0.0;
    }
    G.rem = Cs[0];
    G.H = Cs[1];
    G.nsub = (int)Cs[2];
  } else {
    for (int q = 0; q < 6; ++q) s6[q] = Cs[3 + q];
  }
  const int budget = (a.mode == 0) ? kCatchBudget : (1 << 30);
  bool carried = false, ejected = false;
  // the ejection test that follows slot tt, as k_eject runs it (planetesimal:
  // gm = mu0; P of the slot's kicks)
  auto eject_after = [&](int tt) {
    if (!d.h_ej[tt]) return false;
    const double* P2 = d.h_P + (size_t)tt * 6 * d.nsys + 3 * d.nsys + 3 * sys;
    return dh_unbound(S.mu0, S.inv_mu0, P2, s6[0], s6[1], s6[2], s6[3], s6[4], s6[5]);
  };
  for (;;) {
    if (G.nb >= 2) {
      const int r = catch_bs_any(d, S, G, t, budget, B, s6);
      if (r == 0) {
        carried = true;
        break;
      }
      if (r < 0 && lead) atomicOr(d.status, ST_BS);
      G.nb = 0;
      catch_back(d, S, sys, j, t, lead, s6, B.ops);
      ejected = eject_after(t);
      ++t;
      if (ejected) break;
    }
    if (t >= a.t_end) break;
    if (d.h_nkick[t] > 0) {
      const int km = (t == a.tl) ? (a.mode == 1 ? 2 : 1) : 0;
      int kn2 = 0;
      const int nb = catch_front(d, S, sys, j, t, km, B, s6, G, &kn2, kl);
      if (km == 2) {
        kslot = t;
        kn = kn2;
      }
      if (nb >= 2) continue;   // the group runs at the top of the loop
    }
    catch_back(d, S, sys, j, t, lead, s6, B.ops);
    ejected = eject_after(t);
    ++t;
    if (ejected) break;
  }
  if (ejected && a.mode != 1) {   // removed (Sec. 3.5), with the state it has now
    if (lead) {
      for (int q = 0; q < 6; ++q) d.xv[q * (size_t)d.N + j] = s6[q];
      d.stat[j] = kStatEjected;
      atomicAdd(d.ej_new, 1);
      d.lag[j] = 0;
    }
    return;
  }
  if (a.mode != 1 && !carried) {   // up to date: the body rejoins the step
    if (lead) {
      for (int q = 0; q < 6; ++q) d.xv[q * (size_t)d.N + j] = s6[q];
      d.lag[j] = 0;
    }
    return;
  }
  // carried: mode 0 copies the record to bank_out, mode 1 updates it in place
  __shared__ int s_slot;
  if (lead) s_slot = (a.mode == 0) ? atomicAdd(&d.rcount[a.bank_out], 1) : idx;
  __syncthreads();
  const int ob = (a.mode == 0) ? a.bank_out : bank;
  const int oi = s_slot;
  __syncthreads();
  if (!lead || oi >= d.dcap) {
    if (lead && oi >= d.dcap) atomicOr(d.status, ST_WORK_OVF);
    return;
  }
  int* O = rec_ints(d, ob, oi);
  double* Os = rec_state(d, ob, oi);
  O[0] = j;
  O[1] = (t >= a.t_end) ? a.t_next : t;
  O[2] = ejected ? kRecEjected : (carried ? G.nb : 0);
  for (int m = 0; m < kLaneMaxNB; ++m) O[3 + m] = carried ? G.gid[m] : 0;
  O[7] = kslot;
  O[8] = kn;
  for (int e = 0; e < kMaxGroup; ++e) O[9 + e] = kl[e];
  if (carried) {
    Os[0] = G.rem;
    Os[1] = G.H;
    Os[2] = (double)G.nsub;
    for (int m = 0; m < kLaneMaxNB; ++m)
      for (int q = 0; q < 6; ++q) Os[3 + 6 * m + q] = G.Y[q][m];
  } else {
    for (int q = 0; q < 6; ++q) Os[3 + q] = s6[q];
  }
}

// A cluster of two CTAs per deferred body, on two SMs: both replay the body
// alike (only rank 0 writes), and in a two-body group's Bulirsch-Stoer rounds
// rank 0 tries H and rank 1 tries H/2 (bs2c_rounds with a ClusterMail).
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(128) k_catchup(Dev d, CatchArgs a) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ int s_row[4], s_r;
  __shared__ double s_y[12], s_bc[6], s_g[15];
  __shared__ double s_b2d[2 * 3 * 32], s_b2e[3 * 32], s_b2y[12];
  __shared__ double s_my[12];
  __shared__ int s_mw[6];   // header (2), seq, ack, round, scratch flag
  const int cta = (int)cl.block_rank();
  if (threadIdx.x < 6) s_mw[threadIdx.x] = 0;
  const ClusterMail mail{s_my, s_mw, s_mw + 2, s_mw + 3, s_mw + 4, s_mw + 5, cta, d.status};
  const CatchBlk B{(int)(threadIdx.x & 31), (int)(threadIdx.x >> 5), cta,
                   d.work_ops + (a.mode == 1 ? 4 : 0), Bs2cSmem{s_b2d, s_b2e, s_b2y}, &mail, s_g,
                   s_row, s_y, s_bc, &s_r};
  // both mailboxes are zeroed before either CTA can write into the other's
  cl.sync();
  const int na = (a.bank_a >= 0) ? min(d.rcount[a.bank_a], d.dcap) : 0;
  const int nb = (a.bank_b >= 0) ? min(d.rcount[a.bank_b], d.dcap) : 0;
  if (a.next_slot >= 0 && blockIdx.x == 0 && threadIdx.x == 0) d.hstep[0] = a.next_slot;
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  for (int r = pair; r < na + nb; r += npairs) {
    if (r < na) catch_record(d, a, a.bank_a, r, B);
    else catch_record(d, a, a.bank_b, r - na, B);
    __syncthreads();
  }
  // no CTA leaves while the other may still write into its shared memory
  cl.sync();
}

// ------------------------------------------------------ the persistent step
// One interior step of every system of a batch as one cooperative launch
// (all blocks resident): the phases of the per-kernel step -- jump and drift,
// detection, groups, Bulirsch-Stoer of every group, the kick with its own
// prep -- run the same device functions on the same tiles, separated by grid
// barriers, so the result is the per-kernel step's, bit for bit.  Blocks
// claim tiles from a counter per phase, warps take groups in turn, and block
// 0 builds the groups.
//
// A barrier waits at most `spin` polls of its generation word; a block that
// gives up sets ST_BARRIER and the abort flag, and every block leaves at the
// next barrier it reaches (a wait never outlasts its limit, so the launch
// ends whatever happens).  Returns false to every thread once that happened.
__device__ bool grid_sync(unsigned* bar, long long spin, unsigned* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vb = bar;
    int ok = vb[2] == 0;
    if (ok) {
      const unsigned gen = vb[1];
      __threadfence();
      if (atomicAdd(bar, 1u) == gridDim.x - 1) {
        vb[0] = 0;   // every block has arrived: ready for the next barrier
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        long long k = 0;
        while (vb[1] == gen) {
          if (vb[2] != 0) {
            ok = 0;
            break;
          }
          if (++k > spin) {
            atomicOr(status, ST_BARRIER);
            atomicExch(bar + 2, 1u);
            ok = 0;
            break;
          }
          __nanosleep(128);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The next tile of a phase for this block, claimed from the phase's counter
// (tiles come in the tiling's order, costliest first when the autotuner
// picked that, and each block takes the next one when it is free).  The
// barrier also ends every read of the last tile's shared staging (a fused
// kick's momentum tree shares that space).
__device__ __forceinline__ int next_tile(unsigned* ctr) {
  __shared__ int s_t;
  __syncthreads();
  if (threadIdx.x == 0) s_t = (int)atomicAdd(ctr, 1u);
  __syncthreads();
  return s_t;
}

// Dynamic shared memory: the larger of detection's and the fused kick's.
__global__ void __launch_bounds__(kThreads, 3) k_step_persist(Dev d, long long spin) {
  extern __shared__ __align__(16) unsigned char dsm_p[];
  unsigned* ctr = d.gbar + 4;   // tile counters of the three per-body phases
  for (int t = next_tile(ctr); t < d.ntiles; t = next_tile(ctr)) jump_drift_tile(d, 0.5, t);
  if (!grid_sync(d.gbar, spin, d.status)) return;
  for (int t = next_tile(ctr + 1); t < d.ntiles; t = next_tile(ctr + 1))
    detect_tile(d, d.xv0, d.xv, d.flags, d.keys, d.pair_count, d.pair_cap, 1, t, dsm_p);
  if (!grid_sync(d.gbar, spin, d.status)) return;
  if (blockIdx.x == 0) groups_block(d);
  if (!grid_sync(d.gbar, spin, d.status)) return;
  const int wpb = blockDim.x >> 5;
  bs_all_warps(d, blockIdx.x * wpb + (threadIdx.x >> 5), gridDim.x * wpb);
  __syncwarp();
  if (!grid_sync(d.gbar, spin, d.status)) return;
  for (int t = next_tile(ctr + 2); t < d.ntiles; t = next_tile(ctr + 2))
    jump_kick_tile<2, true>(d, 0.5, 0.5, t, reinterpret_cast<double*>(dsm_p));
}

static size_t persist_smem_bytes(const Dev& d) {
  const size_t a = det_smem_bytes(det_chunk(d.tile, d.big_max));
  const size_t b = kick_smem_bytes(d, true);
  return a > b ? a : b;
}

int persist_grid(const Dev& d) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaFuncSetAttribute(k_step_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)persist_smem_bytes(d)) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_persist, d.tile,
                                                    persist_smem_bytes(d)) != cudaSuccess)
    return 0;
  const int g = per_sm * sms;
  return g < d.ntiles ? g : d.ntiles;
}

cudaError_t launch_step_persist(const Dev& d, int grid, long long spin, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d.gbar, 0, 8 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(d.tile);
  cfg.dynamicSmemBytes = persist_smem_bytes(d);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_step_persist, d, spin);
}

void launch_groups(const Dev& d, cudaStream_t st) { k_groups<<<1, 1024, 0, st>>>(d); }

void launch_bs(const Dev& d, int nblocks, cudaStream_t st) {
  // (a group has at least two members: one big body and the body it meets)
  if (d.defer) {   // no spread phase: one launch
    k_bs_all<<<nblocks, 32, 0, st>>>(d);   // one wave; pairs of groups per warp
    return;
  }
  cudaMemsetAsync(d.cont_count, 0, sizeof(int), st);
  k_bs_pack2<<<4 * nblocks, 32, 0, st>>>(d);
  k_bs_pack<3, 4><<<4 * nblocks, 32, 0, st>>>(d);
  k_bs<<<nblocks, 32, 0, st>>>(d);
  k_bs_spread2<<<nblocks / 4, 128, 0, st>>>(d);
  k_bs_spread<3, 4><<<nblocks / 4, 32, 0, st>>>(d);
}

void launch_catchup(const Dev& d, int nblocks, int mode, int bank_a, int bank_b, int bank_out,
                    int t_end, int tl, int next_slot, int t_next, cudaStream_t st) {
  const CatchArgs a{mode, bank_a, bank_b, bank_out, t_end, tl, next_slot, t_next};
  k_catchup<<<(nblocks + 1) & ~1, 128, 0, st>>>(d, a);   // whole cluster pairs
}

// The kernels of a step share one shared-memory carveout (the largest), so
// the SMs are not reconfigured between consecutive kernels with different
// shared-memory needs (measured: ~12 us bubbles before k_detect and the kick).
void configure_bs() {
  const int c = cudaSharedmemCarveoutMaxShared;
  cudaFuncSetAttribute(k_groups, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_bs_all, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_bs_pack2, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_bs_pack<3, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_bs, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_bs_spread2, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_bs_spread<3, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_catchup, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_step_persist, cudaFuncAttributePreferredSharedMemoryCarveout, c);
}

}  // namespace mx
