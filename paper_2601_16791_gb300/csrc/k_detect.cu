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
#include "mx_detect_body.cuh"
#include "mx_kernels.h"

namespace mx {

__global__ void __launch_bounds__(kThreads) k_detect(Dev d, const double* xv0, const double* xv1,
                                                     unsigned char* flags,
                                                     unsigned long long* keys, int* count,
                                                     int cap, int runs) {
  extern __shared__ __align__(16) unsigned char dsm_det[];
  detect_tile(d, xv0, xv1, flags, keys, count, cap, runs, blockIdx.x, dsm_det);
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
