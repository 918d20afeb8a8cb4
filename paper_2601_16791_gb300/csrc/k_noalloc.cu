// k_noalloc.cu -- encounter detection for callers that cannot allocate device
// memory.
//
// Some callers of this library cannot call cudaMalloc: for instance a host
// application that owns all of the GPU's memory through its own pool and
// forbids other allocations, or a latency-critical loop that cannot afford the
// device-wide synchronisation a fresh allocation may cause.  For them,
// mx_detect_encounters_noalloc runs the same detection, sort and pair output
// as mx_detect_encounters without an mx_system, keeping its working memory
// (pair keys, pair counter, the system record and the tile list) in one
// fixed-size array that lives in the library's static device memory.
//
// That array is a host-side stand-in in host code: its device address is
// fetched with cudaGetSymbolAddress once per device (on the first call made
// while that device is current) and only that address is handed to kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mx.h"
#include "mx_common.cuh"
#include "mx_kernels.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kNaMaxTiles = MX_NOALLOC_MAX_BODIES / mx::kThreads;
// The key sort pads the keys up to the next power of two of the pair count;
// with a power-of-two capacity the padding stays inside the key region.
static_assert((MX_NOALLOC_MAX_PAIRS & (MX_NOALLOC_MAX_PAIRS - 1)) == 0,
              "the pair capacity must be a power of two");
static_assert(MX_NOALLOC_MAX_BODIES % mx::kThreads == 0,
              "the body limit must be a whole number of tiles");

// Byte offsets of the pieces inside the scratch array.
constexpr size_t kOffKeys = 0;
constexpr size_t kOffCount = kOffKeys + sizeof(unsigned long long) * MX_NOALLOC_MAX_PAIRS;
constexpr size_t kOffSys = kOffCount + 256;
constexpr size_t kOffTiles = kOffSys + ((sizeof(mx::SysDev) + 255) / 256) * 256;
constexpr size_t kScratchBytes = kOffTiles + sizeof(mx::Tile) * kNaMaxTiles;

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Writes the system record and the tiles for n bodies, zeroes the counter.
__global__ void k_noalloc_setup(unsigned char* scratch, mx::SysDev sys, int n) {
  mx::Tile* tiles = reinterpret_cast<mx::Tile*>(scratch + kOffTiles);
  const int ntiles = (n + mx::kThreads - 1) / mx::kThreads;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
    const int start = t * mx::kThreads;
    tiles[t] = mx::Tile{0, start, min(mx::kThreads, n - start), 0};
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *reinterpret_cast<mx::SysDev*>(scratch + kOffSys) = sys;
    int* cnt = reinterpret_cast<int*>(scratch + kOffCount);
    cnt[0] = 0;
    cnt[1] = 0;
  }
}

}  // namespace

extern "C" mx_status mx_detect_encounters_noalloc(const mx_params* p, int n_big, int n,
                                                  const double* dev_rcrit, const double* dev_xv0,
                                                  const double* dev_xv1,
                                                  unsigned char* dev_flags, int* dev_pairs,
                                                  int cap, int* n_pairs, void* cuda_stream) {
  if (!p || !dev_rcrit || !dev_xv0 || !dev_xv1 || !dev_flags || !n_pairs || cap < 0 ||
      (cap > 0 && !dev_pairs) || n_big < 0 || n < n_big || n <= 0 || !std::isfinite(p->dt))
    return MX_ERR_ARG;
  if (n > MX_NOALLOC_MAX_BODIES) return MX_ERR_ARG;   // beyond the static scratch
  // An error left pending by earlier work is the caller's: report it before
  // launching anything, rather than as this call's launch failure.
  if (cudaPeekAtLastError() != cudaSuccess) return MX_ERR_CUDA;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MX_ERR_CUDA;
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr)
        return MX_ERR_CUDA;
      g_scratch_addr[dev] = static_cast<unsigned char*>(addr);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  mx::SysDev sys;
  std::memset(&sys, 0, sizeof(sys));
  sys.off = 0;
  sys.nbig = n_big;
  sys.n = n;
  sys.boff = 0;
  sys.h = p->dt;
  sys.mu0 = p->G * p->m_star;
  mx::Dev d;
  std::memset(&d, 0, sizeof(d));
  d.brc = const_cast<double*>(dev_rcrit);
  d.sys = reinterpret_cast<const mx::SysDev*>(scratch + kOffSys);
  d.tiles = reinterpret_cast<const mx::Tile*>(scratch + kOffTiles);
  d.N = n;
  d.NB = n_big;
  d.nsys = 1;
  d.ntiles = (n + mx::kThreads - 1) / mx::kThreads;
  d.tile = mx::kThreads;
  d.big_max = n_big;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(scratch + kOffKeys);
  int* count = reinterpret_cast<int*>(scratch + kOffCount);
  if (cudaMemsetAsync(dev_flags, 0, (size_t)n, st) != cudaSuccess) return MX_ERR_CUDA;
  k_noalloc_setup<<<32, 256, 0, st>>>(scratch, sys, n);
  if (cudaGetLastError() != cudaSuccess) return MX_ERR_CUDA;
  mx::launch_detect(d, dev_xv0, dev_xv1, dev_flags, keys, count, MX_NOALLOC_MAX_PAIRS, 0, st);
  if (cudaGetLastError() != cudaSuccess) return MX_ERR_CUDA;
  mx::launch_sort_keys(keys, count, MX_NOALLOC_MAX_PAIRS, 1, st);
  if (cudaGetLastError() != cudaSuccess) return MX_ERR_CUDA;
  if (cap > 0) {
    mx::launch_keys_to_pairs(keys, count, cap < MX_NOALLOC_MAX_PAIRS ? cap : MX_NOALLOC_MAX_PAIRS,
                             dev_pairs, st);
    if (cudaGetLastError() != cudaSuccess) return MX_ERR_CUDA;
  }
  int found = 0;
  if (cudaMemcpyAsync(&found, count, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MX_ERR_CUDA;
  *n_pairs = found;
  if (found > MX_NOALLOC_MAX_PAIRS || found > cap) return MX_ERR_PAIR_OVERFLOW;
  return MX_OK;
}
