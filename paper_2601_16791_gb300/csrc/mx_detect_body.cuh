// mx_detect_body.cuh -- the per-tile body of close-encounter detection
// (k_detect.cu), shared by its kernel and the persistent step kernel.
#pragma once
#include "mx_common.cuh"
#include "mx_encounter.cuh"

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
// Tile `bid`, one target per thread; dsm_det: the block's dynamic shared
// memory (det_smem_bytes).
__device__ __forceinline__ void detect_tile(const Dev& d, const double* xv0, const double* xv1,
                                            unsigned char* flags, unsigned long long* keys,
                                            int* count, int cap, int runs, int bid,
                                            unsigned char* dsm_det) {
  const int chunk = det_chunk(blockDim.x, d.big_max);
  DetSmem sm(dsm_det, chunk);
  const Tile t = d.tiles[bid];
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

}  // namespace mx
