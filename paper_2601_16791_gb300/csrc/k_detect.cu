// k_detect.cu -- close-encounter detection and pair compaction
// (arXiv 2601.16791, Sec. 2.1.2, mce_snif listing: a pair is flagged when
// min(d0, d1, d2min) <= rc^2, rc = max(rcrit_i, rcrit_j)).
//
// One thread per target body against the big bodies of its system, staged in
// shared memory with FP64 endpoint states and FP32 copies.  A provably
// conservative FP32 screen discards far pairs (mx_encounter.cuh); surviving
// pairs are decided in FP64 with the closed-form minimum of the cubic Hermite
// interpolant of the squared separation.
// Each target keeps its flagged big bodies (ascending) and writes them as one
// contiguous run, with one atomic per warp; runs of different targets come in
// any order.  The step groups runs as they are; callers that want the pairs
// in order sort the keys (k_sort_keys).
#include "mx_common.cuh"
#include "mx_encounter.cuh"
#include "mx_kernels.h"

namespace mx {

// Big bodies staged per pass, in the block's dynamic shared memory: `chunk`
// = min(threads per block, most big bodies of a system) entries of each
// array (a disk with a few big bodies leaves the SM its shared memory).
__host__ __device__ __forceinline__ int det_chunk(int tile, int big_max) {
  const int c = big_max < tile ? big_max : tile;
  return c < 1 ? 1 : c;
}

__host__ __device__ __forceinline__ size_t det_smem_bytes(int chunk) {
  return (size_t)chunk * (13 * sizeof(double) + 13 * sizeof(float) + 1);
}

struct DetSmem {
  double* s[12];   // x0 y0 z0 u0 v0 w0 x1 y1 z1 u1 v1 w1
  float* f[12];
  double* rc;
  float* rcf;
  unsigned char* out;   // big body removed from the integration (Sec. 3.5)
  __device__ DetSmem(unsigned char* base, int n) {
    double* db = reinterpret_cast<double*>(base);
    for (int q = 0; q < 12; ++q) s[q] = db + q * n;
    rc = db + 12 * n;
    float* fb = reinterpret_cast<float*>(db + 13 * n);
    for (int q = 0; q < 12; ++q) f[q] = fb + q * n;
    rcf = fb + 12 * n;
    out = reinterpret_cast<unsigned char*>(fb + 13 * n);
  }
};

// xv0, xv1: 6 x N endpoint states; keys/count/cap: pair output.
// runs = 1 (the step): a target with more than kMaxGroup flagged big bodies
// would make a group larger than kMaxGroup, reported as ST_GROUP.
__global__ void __launch_bounds__(kThreads) k_detect(Dev d, const double* xv0, const double* xv1,
                                                     unsigned char* flags,
                                                     unsigned long long* keys, int* count,
                                                     int cap, int runs) {
  extern __shared__ __align__(16) unsigned char dsm_det[];
  const int chunk = det_chunk(blockDim.x, d.big_max);
  DetSmem sm(dsm_det, chunk);
  const Tile t = d.tiles[blockIdx.x];
  const SysDev& S = d.sys[t.sys];
  const int N = d.N;
  const int j = t.start + threadIdx.x;
  // a deferred planetesimal is tested by the window's catch-up instead; a
  // removed body meets nothing
  const bool act = threadIdx.x < t.count && !(d.defer && d.lag[j]) && !removed(d, j);
  const int jl = j - S.off;
  const bool jbig = jl < S.nbig;
  const int lane = threadIdx.x & 31;
  const double h = S.h;
  const float hf = to_float_bits(h);
  double a0[6], a1[6];
  float af[12];
  double rcj = 0.0;
  for (int k = 0; k < 6; ++k) {
    a0[k] = act ? xv0[(size_t)k * N + j] : 0.0;
    a1[k] = act ? xv1[(size_t)k * N + j] : 0.0;
    af[k] = to_float_bits(a0[k]);
    af[6 + k] = to_float_bits(a1[k]);
  }
  if (act && jbig) rcj = d.brc[S.boff + jl];
  const float rcjf = to_float_bits(rcj);
  int hits[kMaxGroup];
  int nh = 0;
  const unsigned long long tag = ((unsigned long long)(jbig ? 0u : 1u) << 63) |
                                 ((unsigned long long)(unsigned)j << 32);
  // writes the buffered hits of the lanes with `mine` set, each lane's as one
  // run (the warp takes its space with one atomic); every lane calls it
  auto flush = [&](bool mine) {
    const int own = mine ? nh : 0;
    int inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    if (total == 0) return;
    int base = 0;
    if (lane == 31) base = atomicAdd(count, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    const int start = base + inc - own;
    for (int e = 0; e < own; ++e)
      if (start + e < cap) keys[start + e] = tag | (unsigned)(S.off + hits[e]);
    if (mine) nh = 0;
  };
  for (int c0 = 0; c0 < S.nbig; c0 += chunk) {
    const int cn = min(chunk, S.nbig - c0);
    __syncthreads();
    if (threadIdx.x < cn) {
      const int g = S.off + c0 + threadIdx.x;
      for (int k = 0; k < 6; ++k) {
        const double p0 = xv0[(size_t)k * N + g], p1 = xv1[(size_t)k * N + g];
        sm.s[k][threadIdx.x] = p0;
        sm.s[6 + k][threadIdx.x] = p1;
        sm.f[k][threadIdx.x] = to_float_bits(p0);
        sm.f[6 + k][threadIdx.x] = to_float_bits(p1);
      }
      const double rcb = d.brc[S.boff + c0 + threadIdx.x];
      sm.rc[threadIdx.x] = rcb;
      sm.rcf[threadIdx.x] = to_float_bits(rcb);
      sm.out[threadIdx.x] = removed(d, g);
    }
    __syncthreads();
    for (int k = 0; k < cn; ++k) {
      const int il = c0 + k;
      // big-big pairs are tested once, with the lower index as the big one
      bool ok = act && (!jbig || il < jl) && !sm.out[k];
      bool hit = false;
      if (ok) {
        const float rcf = fmaxf(sm.rcf[k], rcjf);
        const float rc2f = rcf * rcf;
        float bf[12];
        for (int q = 0; q < 12; ++q) bf[q] = sm.f[q][k];
        if (encounter_screen(af, bf, rc2f, hf)) {
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
      if (hit) {
        const int gi = S.off + il;
        flags[gi] = 1;
        flags[j] = 1;
        if (d.ever) {
          d.ever[gi] = 1;
          d.ever[j] = 1;
        }
        if (nh == kMaxGroup) {   // a run split in two: only past the group limit
          if (runs) atomicOr(d.status, ST_GROUP);
          nh = -1;               // marks the flush below as due
        } else {
          hits[nh++] = il;
        }
      }
      // a full buffer is written out (every lane of the warp takes part)
      if (__any_sync(0xffffffffu, nh < 0)) {
        const bool redo = nh < 0;
        if (redo) nh = kMaxGroup;
        flush(redo);
        if (redo) hits[nh++] = il;
      }
    }
  }
  flush(true);
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
                   unsigned long long* keys, int* count, int cap, int runs, cudaStream_t st) {
  const size_t sm = det_smem_bytes(det_chunk(d.tile, d.big_max));
  k_detect<<<d.ntiles, d.tile, sm, st>>>(d, xv0, xv1, flags, keys, count, cap, runs);
}

void launch_sort_keys(unsigned long long* keys, const int* count, int cap, int swap_ij,
                      cudaStream_t st) {
  k_sort_keys<<<1, 1024, 0, st>>>(keys, count, cap, swap_ij);
}

// The kernels of a step share one shared-memory carveout (the largest), so
// the SMs are not reconfigured between consecutive kernels with different
// shared-memory needs (measured: ~12 us bubbles before k_detect and the kick).
void configure_detect() {
  cudaFuncSetAttribute(k_detect, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

}  // namespace mx
