// k_detect.cu -- close-encounter detection and pair compaction
// (arXiv 2601.16791, Sec. 2.1.2, mce_snif listing: a pair is flagged when
// min(d0, d1, d2min) <= rc^2, rc = max(rcrit_i, rcrit_j)).
//
// One thread per target body against the big bodies of its system, staged in
// shared memory with FP64 endpoint states and FP32 copies.  A provably
// conservative FP32 test discards far pairs: the cubic Hermite interpolant p
// of the squared separation satisfies p >= min(d0, d1) - (4/27)(|D0| + |D1|)
// on the step (D = endpoint slopes in units of the step), and the FP32
// evaluation gets a 10% + 1e-3 relative margin, far above its rounding.
// Surviving pairs are decided in FP64 with the closed-form minimum of p.
// Flagged pairs are appended with one atomic per warp (ballot compaction);
// the pair order is then fixed by sorting the 64-bit keys.
#include "mx_common.cuh"
#include "mx_kernels.h"

namespace mx {

// Exact FP64 encounter test between target a and big b (6 doubles each at
// the start, 0, and end, 1, of the step).
__device__ __noinline__ bool encounter_fp64(const double* a0, const double* b0, const double* a1,
                                           const double* b1, double h, double rc2) {
  const double dx0 = a0[0] - b0[0], dy0 = a0[1] - b0[1], dz0 = a0[2] - b0[2];
  const double du0 = a0[3] - b0[3], dv0 = a0[4] - b0[4], dw0 = a0[5] - b0[5];
  const double dx1 = a1[0] - b1[0], dy1 = a1[1] - b1[1], dz1 = a1[2] - b1[2];
  const double du1 = a1[3] - b1[3], dv1 = a1[4] - b1[4], dw1 = a1[5] - b1[5];
  const double d0 = fma(dx0, dx0, fma(dy0, dy0, dz0 * dz0));
  const double d1 = fma(dx1, dx1, fma(dy1, dy1, dz1 * dz1));
  if (d0 <= rc2 || d1 <= rc2) return true;
  // slopes of the squared separation per unit of tau = t/h
  const double D0 = 2.0 * h * fma(dx0, du0, fma(dy0, dv0, dz0 * dw0));
  const double D1 = 2.0 * h * fma(dx1, du1, fma(dy1, dv1, dz1 * dw1));
  if (!(D0 < 0.0 && D1 > 0.0)) return false;
  // p(tau) = d0 + D0 tau + c2 tau^2 + c3 tau^3 with p(1) = d1, p'(1) = D1
  const double c2 = -3.0 * d0 - 2.0 * D0 + 3.0 * d1 - D1;
  const double c3 = 2.0 * d0 + D0 - 2.0 * d1 + D1;
  // p'(tau) = 3 c3 tau^2 + 2 c2 tau + D0 has exactly one root in (0, 1)
  const double A = 3.0 * c3, B = 2.0 * c2, C = D0;
  double tau;
  if (A == 0.0) {
    tau = -C / B;
  } else {
    const double disc = fmax(B * B - 4.0 * A * C, 0.0);
    const double q = -0.5 * (B + copysign(sqrt(disc), B));
    const double r1 = q / A;
    const double r2 = (q != 0.0) ? C / q : r1;
    tau = (r1 >= 0.0 && r1 <= 1.0) ? r1 : r2;
  }
  tau = fmin(fmax(tau, 0.0), 1.0);
  const double p = fma(tau, fma(tau, fma(tau, c3, c2), D0), d0);
  return fmax(p, 0.0) <= rc2;
}

struct DetSmem {
  double s[12][kThreads];   // x0 y0 z0 u0 v0 w0 x1 y1 z1 u1 v1 w1
  float f[12][kThreads];
  double rc[kThreads];
  float rcf[kThreads];
};

// xv0, xv1: 6 x N endpoint states; keys/count/cap: pair output.
__global__ void __launch_bounds__(kThreads) k_detect(Dev d, const double* xv0, const double* xv1,
                                                     unsigned char* flags,
                                                     unsigned long long* keys, int* count,
                                                     int cap) {
  __shared__ DetSmem sm;
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  const bool act = threadIdx.x < t.count;
  const int j = t.start + threadIdx.x;
  const int jl = j - S.off;
  const bool jbig = jl < S.nbig;
  const int lane = threadIdx.x & 31;
  const double h = S.h;
  const float hf = (float)h;
  double a0[6], a1[6];
  float af[12];
  double rcj = 0.0;
  for (int k = 0; k < 6; ++k) {
    a0[k] = act ? xv0[(size_t)k * N + j] : 0.0;
    a1[k] = act ? xv1[(size_t)k * N + j] : 0.0;
    af[k] = (float)a0[k];
    af[6 + k] = (float)a1[k];
  }
  if (act && jbig) rcj = d.brc[S.boff + jl];
  const float rcjf = (float)rcj;
  for (int c0 = 0; c0 < S.nbig; c0 += blockDim.x) {
    const int cn = min((int)blockDim.x, S.nbig - c0);
    __syncthreads();
    if (threadIdx.x < cn) {
      const int g = S.off + c0 + threadIdx.x;
      for (int k = 0; k < 6; ++k) {
        const double p0 = xv0[(size_t)k * N + g], p1 = xv1[(size_t)k * N + g];
        sm.s[k][threadIdx.x] = p0;
        sm.s[6 + k][threadIdx.x] = p1;
        sm.f[k][threadIdx.x] = (float)p0;
        sm.f[6 + k][threadIdx.x] = (float)p1;
      }
      const double rcb = d.brc[S.boff + c0 + threadIdx.x];
      sm.rc[threadIdx.x] = rcb;
      sm.rcf[threadIdx.x] = (float)rcb;
    }
    __syncthreads();
    for (int k = 0; k < cn; ++k) {
      const int il = c0 + k;
      // big-big pairs are tested once, with the lower index as the big one
      bool ok = act && (!jbig || il < jl);
      bool hit = false;
      if (ok) {
        const float rcf = fmaxf(sm.rcf[k], rcjf);
        const float rc2f = rcf * rcf;
        const float dx0 = af[0] - sm.f[0][k], dy0 = af[1] - sm.f[1][k], dz0 = af[2] - sm.f[2][k];
        const float du0 = af[3] - sm.f[3][k], dv0 = af[4] - sm.f[4][k], dw0 = af[5] - sm.f[5][k];
        const float dx1 = af[6] - sm.f[6][k], dy1 = af[7] - sm.f[7][k], dz1 = af[8] - sm.f[8][k];
        const float du1 = af[9] - sm.f[9][k], dv1 = af[10] - sm.f[10][k], dw1 = af[11] - sm.f[11][k];
        const float d0 = fmaf(dx0, dx0, fmaf(dy0, dy0, dz0 * dz0));
        const float d1 = fmaf(dx1, dx1, fmaf(dy1, dy1, dz1 * dz1));
        const float D0 = fabsf(2.0f * hf * fmaf(dx0, du0, fmaf(dy0, dv0, dz0 * dw0)));
        const float D1 = fabsf(2.0f * hf * fmaf(dx1, du1, fmaf(dy1, dv1, dz1 * dw1)));
        const float lb = fminf(d0, d1) - (4.0f / 27.0f) * (D0 + D1);
        if (lb <= 1.1f * rc2f + 1e-3f * (d0 + d1 + D0 + D1)) {
          const double rc = fmax(sm.rc[k], rcj);
          const double rc2 = rc * rc;
          double b0[6], b1[6];
          for (int q = 0; q < 6; ++q) {
            b0[q] = sm.s[q][k];
            b1[q] = sm.s[6 + q][k];
          }
          hit = encounter_fp64(a0, b0, a1, b1, h, rc2);
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (m) {
        const int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (hit) {
          const int pos = base + __popc(m & ((1u << lane) - 1u));
          const int gi = S.off + il;
          if (pos < cap)
            keys[pos] = ((unsigned long long)(jbig ? 0u : 1u) << 63) |
                        ((unsigned long long)(unsigned)j << 32) | (unsigned)gi;
          flags[gi] = 1;
          flags[j] = 1;
          if (d.ever) {
            d.ever[gi] = 1;
            d.ever[j] = 1;
          }
        }
      }
    }
  }
}

// Sorts min(*count, cap) keys ascending in one block (bitonic; shared memory
// up to kSortSmem keys, global memory beyond).  swap_ij turns the step's
// (small-flag, j, i) keys into (i, j) keys first.
constexpr int kSortSmem = 4096;   // 32 KB of static shared memory
__global__ void __launch_bounds__(1024) k_sort_keys(unsigned long long* keys, const int* count,
                                                    int cap, int swap_ij) {
  __shared__ unsigned long long sk[kSortSmem];
  const int n = min(*count, cap);
  if (n <= 0) return;
  if (swap_ij) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned long long k = keys[i];
      const unsigned long long jj = (k >> 32) & 0x7fffffffull, ii = k & 0xffffffffull;
      keys[i] = (ii << 32) | jj;
    }
    __syncthreads();
  }
  int P2 = 1;
  while (P2 < n) P2 <<= 1;
  const bool in_smem = P2 <= kSortSmem;
  unsigned long long* a = in_smem ? sk : keys;
  if (in_smem) {
    for (int i = threadIdx.x; i < P2; i += blockDim.x) sk[i] = (i < n) ? keys[i] : ~0ull;
  } else {
    for (int i = n + threadIdx.x; i < P2; i += blockDim.x) keys[i] = ~0ull;
  }
  __syncthreads();
  for (int k = 2; k <= P2; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        const int ixj = i ^ jj;
        if (ixj > i) {
          const unsigned long long x = a[i], y = a[ixj];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  if (in_smem)
    for (int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = sk[i];
}

// (i, j) int pairs from sorted (i << 32 | j) keys.
__global__ void k_keys_to_pairs(const unsigned long long* keys, const int* count, int cap,
                                int* pairs) {
  const int n = min(*count, cap);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const unsigned long long k = keys[p];
    pairs[2 * p] = (int)(k >> 32);
    pairs[2 * p + 1] = (int)(k & 0xffffffffull);
  }
}

void launch_keys_to_pairs(const unsigned long long* keys, const int* count, int cap, int* pairs,
                          cudaStream_t st) {
  k_keys_to_pairs<<<64, 256, 0, st>>>(keys, count, cap, pairs);
}

void launch_detect(const Dev& d, const double* xv0, const double* xv1, unsigned char* flags,
                   unsigned long long* keys, int* count, int cap, cudaStream_t st) {
  k_detect<<<d.ntiles, d.tile, 0, st>>>(d, xv0, xv1, flags, keys, count, cap);
}

void launch_sort_keys(unsigned long long* keys, const int* count, int cap, int swap_ij,
                      cudaStream_t st) {
  k_sort_keys<<<1, 1024, 0, st>>>(keys, count, cap, swap_ij);
}

}  // namespace mx
