// mx_api.cu -- the C ABI (include/mx.h): owns the device buffers of one or
// more systems, records the step as CUDA graphs, and maps device status bits to
// mx_status.  All arithmetic on bodies runs in the kernels; the host only
// folds parameters into per-system constants and lays out the buffers.
#include <cuda_runtime.h>

#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mx.h"
#include "mx_common.cuh"
#include "mx_kernels.h"

namespace {

thread_local std::string g_last_error;

mx_status fail(mx_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

constexpr double kPi = 3.14159265358979323846;
constexpr double kAuCm = 1.495978707e13;
constexpr double kHydrogenG = 1.6735575e-24;
constexpr double kMsunG = 1.98847e33;   // solar mass [g]

// S(gamma) = sum_n A_n (1-gamma)(4n+1)/((2n+2-gamma)(2n-1+gamma)),
// A_n = [(2n)!/(2^(2n) (n!)^2)]^2 (Eq. 10, gamma != 1).  The first 2^20 terms
// are summed with compensation; the rest is the tail of the terms' expansion
// t_n = (1-gamma)/(pi n^2) (1 - 1/(2n)) + O(n^-4), i.e.
// (1-gamma)/pi (1/N + 1/(4N^2)) + O(N^-3).  Cached per gamma.
double disk_gravity_series(double gamma) {
  static std::vector<std::pair<double, double>> cache;
  for (auto& kv : cache)
    if (kv.first == gamma) return kv.second;
  const int N = 1 << 20;
  double sum = 0.0, comp = 0.0, b = 1.0;   // b = (2n)!/(4^n (n!)^2), A_n = b^2
  for (int n = 0; n < N; ++n) {
    if (n > 0) b *= (2.0 * n - 1.0) / (2.0 * n);
    const double t = b * b * (1.0 - gamma) * (4.0 * n + 1.0) /
                     ((2.0 * n + 2.0 - gamma) * (2.0 * n - 1.0 + gamma));
    const double y = t - comp;
    const double nx = sum + y;
    comp = (nx - sum) - y;
    sum = nx;
  }
  const double Nd = (double)N;
  const double tail = (1.0 - gamma) / kPi * (1.0 / Nd + 0.25 / (Nd * Nd));
  const double S = sum + tail;
  cache.push_back({gamma, S});
  return S;
}

// dS/dgamma (gamma != 1), for the adjoint: each term's logarithmic
// derivative is -1/(1-gamma) + 1/(2n+2-gamma) - 1/(2n-1+gamma), summed as
// S is; the tail's derivative is -(1/pi)(1/N + 1/(4N^2)).  Cached per gamma.
double disk_gravity_series_dgamma(double gamma) {
  static std::vector<std::pair<double, double>> cache;
  for (auto& kv : cache)
    if (kv.first == gamma) return kv.second;
  const int N = 1 << 20;
  double sum = 0.0, comp = 0.0, b = 1.0;
  for (int n = 0; n < N; ++n) {
    if (n > 0) b *= (2.0 * n - 1.0) / (2.0 * n);
    const double p = 2.0 * n + 2.0 - gamma, q = 2.0 * n - 1.0 + gamma;
    const double t = b * b * (1.0 - gamma) * (4.0 * n + 1.0) / (p * q);
    const double dt = t * (-1.0 / (1.0 - gamma) + 1.0 / p - 1.0 / q);
    const double y = dt - comp;
    const double nx = sum + y;
    comp = (nx - sum) - y;
    sum = nx;
  }
  const double Nd = (double)N;
  const double dS = sum - (1.0 / kPi) * (1.0 / Nd + 0.25 / (Nd * Nd));
  cache.push_back({gamma, dS});
  return dS;
}

#define MX_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? MX_ERR_OOM : MX_ERR_CUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

mx_status status_to_code(unsigned st) {
  if (st & mx::ST_NONFINITE) return fail(MX_ERR_NONFINITE, "non-finite position or velocity");
  if (st & mx::ST_KEPLER) return fail(MX_ERR_KEPLER_NOCONV, "Kepler solve hit its iteration cap");
  if (st & mx::ST_PAIR_OVF) return fail(MX_ERR_PAIR_OVERFLOW, "more encounter pairs than pair_cap");
  if (st & mx::ST_GROUP)
    return fail(MX_ERR_GROUP_TOO_LARGE, "encounter group larger than MX_MAX_GROUP bodies");
  if (st & mx::ST_WORK_OVF) return fail(MX_ERR_PAIR_OVERFLOW, "encounter work list overflow");
  if (st & mx::ST_BS) return fail(MX_ERR_BS_NOCONV, "Bulirsch-Stoer hit its sub-step cap");
  if (st & mx::ST_TAPE)
    return fail(MX_ERR_BS_NOCONV, "an adjoint encounter group took more than 128 accepted sub-steps");
  if (st & mx::ST_BARRIER) return fail(MX_ERR_BARRIER_TIMEOUT, "device wait gave up");
  if (st & mx::ST_WINDOW) return fail(MX_ERR_CUDA, "deferral window longer than its history");
  return MX_OK;
}

bool valid_params(const mx_params* p) {
  return p && std::isfinite(p->G) && p->G > 0 && p->m_star > 0 && std::isfinite(p->dt) &&
         p->rcrit_hill >= 0 && p->bs_tol > 0 && p->kepler_max_iter > 0 && p->bs_max_sub > 0 &&
         p->pair_cap > 0 && p->pair_cap <= (1 << 26) && p->eject_every >= 0;
}

// Per-system constants folded from the parameters.
mx::SysDev make_sysdev(const mx_params& p, int off, int nbig, int n, int boff) {
  mx::SysDev s;
  std::memset(&s, 0, sizeof(s));
  s.off = off;
  s.nbig = nbig;
  s.n = n;
  s.boff = boff;
  s.mu0 = p.G * p.m_star;
  s.inv_mu0 = 1.0 / s.mu0;
  s.sqrt_mu0 = std::sqrt(s.mu0);
  s.h = p.dt;
  s.inv_G = 1.0 / p.G;
  s.m_star = p.m_star;
  const mx_gas& g = p.gas;
  s.gas_on = g.enabled ? 1 : 0;
  s.cd_mode = g.cd_mode;
  s.gamma_one = (g.gamma == 1.0) ? 1 : 0;
  s.flare_quarter = (g.flare == 0.25) ? 1 : 0;
  s.rc_inf = std::isinf(g.r_c_au) ? 1 : 0;
  s.sigma1 = g.sigma1_gcm2;
  s.gamma = g.gamma;
  s.inv_rc = s.rc_inf ? 0.0 : 1.0 / g.r_c_au;
  s.r_in = g.r_in_au;
  s.hr1 = g.hr_1au;
  s.flare = g.flare;
  s.cd_scale = g.cd_scale;
  s.c_rho = 1.0 / (std::sqrt(2.0 * kPi) * kAuCm * g.hr_1au);
  s.c_cs = g.hr_1au * s.sqrt_mu0;
  s.inv_c_cs = 1.0 / s.c_cs;
  const double beta_T = 1.0 - 2.0 * g.flare;
  s.c_eta = g.hr_1au * g.hr_1au * (g.gamma + beta_T / 2.0 + 1.5) / (2.0 * g.gamma_c);
  s.deta_dgamma = g.hr_1au * g.hr_1au / (2.0 * g.gamma_c);
  const double c_lam = g.mu_mol * kHydrogenG / g.sigma_mol_cm2;
  s.c_re = 4.0 / (std::sqrt(8.0 / kPi) * c_lam);
  // disk gravity: 2 pi G Sigma [Msun/AU^2] times S(gamma), or r_in / R at gamma = 1
  s.dg_on = (g.enabled && g.disk_gravity) ? 1 : 0;
  s.dg_edge = (g.gamma == 1.0) ? 1 : 0;
  const double two_pi_g = 2.0 * kPi * p.G * (kAuCm * kAuCm / kMsunG);
  s.c_dg = s.dg_on ? two_pi_g * (s.dg_edge ? g.r_in_au : disk_gravity_series(g.gamma)) : 0.0;
  s.dlnS_dgamma = (s.dg_on && !s.dg_edge)
                      ? disk_gravity_series_dgamma(g.gamma) / disk_gravity_series(g.gamma)
                      : 0.0;
  s.grow_on = 0;                 // mx_set_growth
  s.G = p.G;
  s.rcrit_hill = p.rcrit_hill;
  s.gap_c = 4.0;
  return s;
}

}  // namespace

struct mx_system {
  int device = 0;
  cudaStream_t st = nullptr;
  cudaStream_t cap_st = nullptr;
  std::vector<mx_params> params;   // per system
  std::vector<int> nbig, nsmall;
  int N = 0, NB = 0;
  mx::Dev d{};
  mx::SysDev* d_sys = nullptr;
  mx::Tile* d_tiles = nullptr;
  double* d_tmp = nullptr;        // 6 x N scratch for readout / set_state
  double* d_energy = nullptr;
  double* d_sink = nullptr;
  unsigned* h_status = nullptr;   // pinned
  int* h_count = nullptr;         // pinned
  std::vector<void*> allocs;
  cudaGraphExec_t g_head = nullptr, g_mid = nullptr, g_last = nullptr;
  cudaGraphExec_t gt_head = nullptr, gt_mid = nullptr, gt_last = nullptr;   // timed variants
  cudaEvent_t mk_head[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t mk_step[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  long long step = 0;
  int eject_every = 0;            // ejection test schedule (Sec. 3.5), 0: none
  bool removed_any = false;       // a test outside the schedule removed bodies
  bool grow_any = false;          // some system follows growth tracks (mx_set_growth)
  mx::Growth* d_grow = nullptr;   // [NB]
  int* d_counts = nullptr;        // [nsys] removed bodies per system
  int bs_blocks = 0;
  int catch_blocks = 0;
  int window = 0;                 // history slots per catch-up of deferred planetesimals (0: off)
  int pending = 0;                // slots recorded in the current window
  int wbase = 0;                  // first history slot of the current window (0 or window)
  int last_full = -1;             // history slot of the last whole step, -1 none
  int carried = 1;                // bank of the bodies carried from the last window (1 or 2)
  bool side_busy = false;         // a side-stream pass is in flight
  cudaStream_t side_st = nullptr; // highest priority: its blocks take SMs as soon as they free up
  int prio_low = 0, prio_high = 0;
  cudaEvent_t ev_main = nullptr, ev_side = nullptr;
  long long catchups = 0;
  // side-stream launches timed by mx_step_profiled, read once they complete
  struct Span {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Span> side_spans;
  int persist = 0;                // interior steps as one cooperative launch (k_step_persist)
  long long persist_spin = 1ll << 24;   // polls a grid barrier waits before it gives up
  int persist_grid = 0;           // blocks of that launch (all resident)
  int tile = mx::kThreads;        // targets per tile (autotuned)
  int order = 0;                  // 0: tiles in system order; 1: costliest first
  int tiles_cap = 0;
  std::vector<mx::SysDev> h_sys;
  // adjoint scratch (allocated on first use)
  double *a_v1 = nullptr, *a_x2 = nullptr, *a_xv3 = nullptr, *a_x4 = nullptr;
  double *a_part = nullptr, *a_P = nullptr, *a_L = nullptr;
  // adjoint through the encounter groups (k_adj_bs.cu)
  int a_gcap = 0;
  int* a_gM = nullptr;
  unsigned long long* a_goff = nullptr;
  double *a_gcontrib = nullptr, *a_tape = nullptr, *a_bsx = nullptr;
  unsigned long long a_tape_cap = 0;
  unsigned long long* a_need = nullptr;   // device [2]: tape doubles, big bodies' shares
  unsigned long long* h_need = nullptr;   // pinned copy
  unsigned long long* a_skeys = nullptr;  // sorted share keys (many big bodies)
  int* a_scount = nullptr;
  int a_skeys_cap = 0;
  double* a_bfold = nullptr;              // 3 x NB
  // merged reverse of consecutive half kicks (mx_adjoint_merge): the pair
  // pass of the last adjoint step's first half kick, pending with its
  // cotangent (a_lpend) and positions (a_xpend), both 3 x N
  int a_merge = 0, a_pend = 0;
  int pd_ok = 0;   // d.xv0 holds the pre-drift state of every body for the last mx_step
  long long a_pend_step = -1;
  double* a_pend_lam = nullptr;
  double *a_lpend = nullptr, *a_xpend = nullptr;
  // kept Stoermer sub-steps of two-body records (mx_adjoint_store)
  double* a_sub = nullptr;
  unsigned* a_subn = nullptr;
  unsigned a_sub_cap = 0, a_sub_want = 1u << 14;
  int a_groups = 1;               // mx_adjoint_encounters
  int* a_poff = nullptr;
  int* a_systiles = nullptr;
  size_t a_part_cap = 0;
  // the adjoint's own tiling (kThreads targets, system order), whatever the
  // forward step's autotuner picked: its kernels are faster on full blocks,
  // and its per-tile partial sums then do not depend on the forward tiling
  mx::Tile* a_tiles = nullptr;
  int a_ntiles = 0;
  int a_tile = mx::kThreads;   // targets per block of the adjoint's per-target kernels
  long long kbits_cap = 0;
};

namespace {

template <class T>
mx_status dalloc(mx_system* s, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return fail(MX_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  s->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return MX_OK;
}

#define MX_TRY(x)                 \
  do {                            \
    mx_status r_ = (x);           \
    if (r_ != MX_OK) return r_;   \
  } while (0)

mx_status set_device(mx_system* s) {
  int cur = -1;
  MX_CUDA(cudaGetDevice(&cur));
  if (cur != s->device) MX_CUDA(cudaSetDevice(s->device));
  return MX_OK;
}

mx_status sync_status(mx_system* s) {
  MX_CUDA(cudaMemcpyAsync(s->h_status, s->d.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
  MX_CUDA(cudaStreamSynchronize(s->st));
  MX_CUDA(cudaGetLastError());
  const unsigned st = *s->h_status;
  if (st) {
    MX_CUDA(cudaMemsetAsync(s->d.status, 0, sizeof(unsigned), s->st));
    MX_CUDA(cudaStreamSynchronize(s->st));
    return status_to_code(st);
  }
  return MX_OK;
}

// The device work of one interior step, or the last step of a call
// (one half kick at its end), or the leading half kick.
// With `marks` (the timed graphs of mx_step_timed), an event is recorded
// before the first launch and after each one (as graph nodes: external
// records, so that launching the graph records them).
void mark_event(cudaEvent_t e, cudaStream_t st) { cudaEventRecordWithFlags(e, st, cudaEventRecordExternal); }

void enqueue_head(mx_system* s, cudaStream_t st, cudaEvent_t* marks) {
  if (marks) mark_event(marks[0], st);
  mx::launch_prep(s->d, 0.0, 1, st);
  if (marks) mark_event(marks[1], st);
  mx::launch_jump_kick(s->d, 0.0, 0.5, 1, st);
  if (marks) mark_event(marks[2], st);
}

// An interior step's kick makes its own prep (k_jump_kick<2, true>) in forward
// runs without growth tracks (their update sits in k_prep) and without k
// branches recorded or replayed (the kick counter k_prep advances).
bool fuse_prep(const mx_system* s) { return s->d.kmode == 0 && !s->grow_any; }

// The persistent form of an interior step (mx_set_persistent): with deferral
// on, in forward runs whose interior kick makes its own prep.
bool persist_step(const mx_system* s, int last) {
  return s->persist && !last && fuse_prep(s) && s->d.defer && s->persist_grid > 0;
}

void enqueue_step(mx_system* s, int last, cudaStream_t st, cudaEvent_t* marks) {
  if (!marks && persist_step(s, last)) {
    mx::launch_step_persist(s->d, s->persist_grid, s->persist_spin, st);
    return;
  }
  int m = 0;
  auto mark = [&] {
    if (marks) mark_event(marks[m++], st);
  };
  mark();
  mx::launch_jump_drift(s->d, 0.5, st);
  mark();
  mx::launch_detect(s->d, s->d.xv0, s->d.xv, s->d.flags, s->d.keys, s->d.pair_count,
                    s->d.pair_cap, 1, st);
  mark();
  mx::launch_groups(s->d, st);
  mark();
  mx::launch_bs(s->d, s->bs_blocks, st);
  mark();
  if (!last && fuse_prep(s)) {
    mark();   // no k_prep: an empty span keeps the timed graphs' layout
    mx::launch_jump_kick_fused(s->d, st);
  } else {
    mx::launch_prep(s->d, 0.5, last ? 1 : 2, st);
    mark();
    mx::launch_jump_kick(s->d, 0.5, 0.5, last ? 1 : 2, st);
  }
  mark();
}

void enqueue_head(mx_system* s, cudaStream_t st) { enqueue_head(s, st, nullptr); }
void enqueue_step(mx_system* s, int last, cudaStream_t st) { enqueue_step(s, last, st, nullptr); }

// The ejection test (Sec. 3.5) follows step number gstep (1-based, global)
// when it is a multiple of eject_every.  Such a step ends with its own half
// kick (the last-step form), so that the test sees the state at the step's
// end and a removed massive body no longer acts in the next step's kick.
bool eject_after(const mx_system* s, long long gstep) {
  return s->eject_every > 0 && gstep % s->eject_every == 0;
}

// With growth tracks every step ends with its own half kick, and the next one
// starts with the masses of its own start time (k_prep applies them).
bool split_after(const mx_system* s, long long gstep) {
  return s->grow_any || eject_after(s, gstep);
}

// Deferral is on for forward runs with a window; recording or replaying the
// drag branches (kmode != 0) keeps every body on the direct path.
void update_defer(mx_system* s) { s->d.defer = (s->window > 0 && s->d.kmode == 0) ? 1 : 0; }

// The end of a window of history slots [wbase, wbase + window).  On the main
// stream, after the side stream's pass over the last window: bodies deferred
// in this window and bodies carried from the last one are replayed with a
// round budget; those that reach the end rejoin the step, the rest are
// carried.  Then, on the side stream, the carried bodies are replayed to the
// window's end while the main stream goes on with the next window (it writes
// the other half of the history ring).  `timed(kind, stream, launch)` wraps
// each launch (event timing in mx_step_profiled).
template <class Timed>
cudaError_t window_end(mx_system* s, Timed&& timed) {
  const int out = 3 - s->carried;
  const int t_end = s->wbase + s->window;
  const int next = (s->wbase == 0) ? s->window : 0;
  const int tl = (s->last_full >= s->wbase && s->last_full < t_end) ? s->last_full : -1;
  cudaError_t e = cudaSuccess;
  if (s->side_busy) {
    // Bodies deferred in this window (bank 0) do not depend on the side
    // stream's pass (it works on the other carried bank and on the other half
    // of the history ring), so they are replayed before the main stream waits
    // for it; the carried bank follows once the side pass is done.
    e = timed(MX_K_CATCHUP, s->st, [&] {
      mx::launch_catchup(s->d, s->catch_blocks, 0, 0, -1, out, t_end, tl, next, next, s->st);
    });
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->st, s->ev_side, 0);
    if (e == cudaSuccess)
      e = timed(MX_K_CATCHUP, s->st, [&] {
        mx::launch_catchup(s->d, s->catch_blocks, 0, s->carried, -1, out, t_end, tl, next, next,
                           s->st);
        cudaMemsetAsync(s->d.rcount + s->carried, 0, sizeof(int), s->st);
        cudaMemsetAsync(s->d.rcount, 0, sizeof(int), s->st);
      });
  } else {
    e = timed(MX_K_CATCHUP, s->st, [&] {
      mx::launch_catchup(s->d, s->catch_blocks, 0, s->carried, 0, out, t_end, tl, next, next, s->st);
      cudaMemsetAsync(s->d.rcount + s->carried, 0, sizeof(int), s->st);
      cudaMemsetAsync(s->d.rcount, 0, sizeof(int), s->st);
    });
  }
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_main, s->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side_st, s->ev_main, 0);
  if (e == cudaSuccess)
    e = timed(MX_K_CATCHUP_SIDE, s->side_st, [&] {
      mx::launch_catchup(s->d, s->catch_blocks, 1, out, -1, out, t_end, tl, -1, next, s->side_st);
    });
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_side, s->side_st);
  s->side_busy = true;
  s->carried = out;
  s->wbase = next;
  s->pending = 0;
  ++s->catchups;
  return e;
}

// A history slot (a whole step, or the leading half kick of a call) has been
// enqueued on the main stream.
template <class Timed>
cudaError_t slot_done(mx_system* s, bool full, Timed&& timed) {
  if (!s->d.defer) return cudaSuccess;
  if (full) s->last_full = s->wbase + s->pending;
  if (++s->pending < s->window) return cudaSuccess;
  return window_end(s, timed);
}

auto untimed = [](int, cudaStream_t, auto&& launch) -> cudaError_t {
  launch();
  return cudaGetLastError();
};

// Brings every deferred planetesimal up to date (the main stream waits for
// the side stream, then replays what is left of the current window with no
// budget) before the state is read or replaced, or the parameters the history
// was recorded under change.  The history ring starts again at slot 0.
template <class Timed>
cudaError_t settle_with(mx_system* s, Timed&& timed) {
  if (!s->d.defer || (s->pending == 0 && !s->side_busy)) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  const int t_end = s->wbase + s->pending;
  if (s->side_busy) {
    // as at a window's end: the bodies deferred in this window first, while
    // the side stream may still run; then, after it, the carried bank
    e = timed(MX_K_CATCHUP, s->st, [&] {
      mx::launch_catchup(s->d, s->catch_blocks, 2, 0, -1, -1, t_end, s->last_full, 0, 0, s->st);
    });
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->st, s->ev_side, 0);
    if (e == cudaSuccess)
      e = timed(MX_K_CATCHUP, s->st, [&] {
        mx::launch_catchup(s->d, s->catch_blocks, 2, s->carried, -1, -1, t_end, s->last_full, 0, 0,
                           s->st);
        cudaMemsetAsync(s->d.rcount, 0, 3 * sizeof(int), s->st);
      });
  } else {
    e = timed(MX_K_CATCHUP, s->st, [&] {
      mx::launch_catchup(s->d, s->catch_blocks, 2, s->carried, 0, -1, t_end, s->last_full, 0, 0,
                         s->st);
      cudaMemsetAsync(s->d.rcount, 0, 3 * sizeof(int), s->st);
    });
  }
  s->side_busy = false;
  s->pending = 0;
  s->wbase = 0;
  s->last_full = -1;
  ++s->catchups;
  return e;
}

mx_status settle(mx_system* s) {
  MX_CUDA(settle_with(s, untimed));
  return MX_OK;
}

mx_status capture(mx_system* s, int which, cudaGraphExec_t* out, cudaEvent_t* marks = nullptr) {
  cudaGraph_t g = nullptr;
  MX_CUDA(cudaStreamBeginCapture(s->cap_st, cudaStreamCaptureModeThreadLocal));
  if (which == 0) enqueue_head(s, s->cap_st, marks);
  else enqueue_step(s, which == 2, s->cap_st, marks);
  cudaError_t e = cudaStreamEndCapture(s->cap_st, &g);
  if (e != cudaSuccess) return fail(MX_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(MX_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  return MX_OK;
}

mx_status ensure_graphs(mx_system* s) {
  if (s->g_head) return MX_OK;
  MX_TRY(capture(s, 0, &s->g_head));
  MX_TRY(capture(s, 1, &s->g_mid));
  MX_TRY(capture(s, 2, &s->g_last));
  return MX_OK;
}

// The step graphs with event nodes between the kernels (mx_step_timed).
mx_status ensure_timed_graphs(mx_system* s) {
  if (s->gt_head) return MX_OK;
  for (auto& e : s->mk_head)
    if (!e) MX_CUDA(cudaEventCreate(&e));
  for (auto& e : s->mk_step)
    if (!e) MX_CUDA(cudaEventCreate(&e));
  MX_TRY(capture(s, 0, &s->gt_head, s->mk_head));
  MX_TRY(capture(s, 1, &s->gt_mid, s->mk_step));
  MX_TRY(capture(s, 2, &s->gt_last, s->mk_step));
  return MX_OK;
}

constexpr int kMinTile = 64;
constexpr int kMaxWindow = 64;       // steps of big-body history kept for deferred planetesimals
constexpr int kDefaultWindow = 10;
constexpr size_t kHistBudget = 256ull << 20;   // bytes the history may take

// Tiles of `tile` targets per system; order 1 puts the costliest first (work
// per target grows with the system's big bodies and with gas drag), so the
// block scheduler starts the long blocks early and the tail is short.
std::vector<mx::Tile> make_tiles(const std::vector<mx::SysDev>& sys, int tile, int order) {
  std::vector<mx::Tile> tiles;
  std::vector<double> cost;
  for (int k = 0; k < (int)sys.size(); ++k) {
    for (int t = 0; t < sys[k].n; t += tile) {
      const int cnt = std::min(tile, sys[k].n - t);
      tiles.push_back({k, sys[k].off + t, cnt, 0});
      cost.push_back((double)cnt * (sys[k].nbig + 1 + (sys[k].gas_on ? 4 : 0)));
    }
  }
  if (order == 1) {
    std::vector<int> idx(tiles.size());
    for (size_t q = 0; q < idx.size(); ++q) idx[q] = (int)q;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<mx::Tile> sorted;
    for (int q : idx) sorted.push_back(tiles[q]);
    tiles.swap(sorted);
  }
  return tiles;
}

void drop_graphs(mx_system* s) {
  if (s->g_head) cudaGraphExecDestroy(s->g_head);
  if (s->g_mid) cudaGraphExecDestroy(s->g_mid);
  if (s->g_last) cudaGraphExecDestroy(s->g_last);
  if (s->gt_head) cudaGraphExecDestroy(s->gt_head);
  if (s->gt_mid) cudaGraphExecDestroy(s->gt_mid);
  if (s->gt_last) cudaGraphExecDestroy(s->gt_last);
  s->g_head = s->g_mid = s->g_last = nullptr;
  s->gt_head = s->gt_mid = s->gt_last = nullptr;
}

mx_status set_tiling(mx_system* s, int tile, int order) {
  std::vector<mx::Tile> tiles = make_tiles(s->h_sys, tile, order);
  if ((int)tiles.size() > s->tiles_cap) return fail(MX_ERR_ARG, "tile size below the minimum");
  MX_CUDA(cudaMemcpyAsync(s->d_tiles, tiles.data(), tiles.size() * sizeof(mx::Tile),
                          cudaMemcpyHostToDevice, s->st));
  MX_CUDA(cudaStreamSynchronize(s->st));
  s->tile = tile;
  s->order = order;
  s->d.tile = tile;
  s->d.ntiles = (int)tiles.size();
  if (s->persist) s->persist_grid = mx::persist_grid(s->d);
  drop_graphs(s);
  return MX_OK;
}

// ---------------------------------------------------------------- autotuner
// Picks the tile size (targets per block) and the tile order for a size
// bucket by timing one plain step per candidate, state saved and restored
// (results do not depend on the choice: every target sums its sources in
// the same order and the pair keys are sorted).  Choices are kept in a
// small JSON file ($MX_AUTOTUNE_CACHE, else ~/.cache/mx/autotune.json);
// MX_AUTOTUNE=0 keeps the defaults.
std::string tune_key(const mx_system* s) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, s->device);
  auto bucket = [](double x) { return x <= 0 ? 0 : (int)std::lround(4.0 * std::log2(x)); };
  bool gas = false;
  for (auto& p : s->params) gas |= (p.gas.enabled != 0);
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s/%d|nsys%d|N%d|NB%d|gas%d", prop.name, prop.multiProcessorCount,
                bucket(s->params.size()), bucket(s->N), bucket(s->NB), gas ? 1 : 0);
  return buf;
}

std::string tune_path() {
  const char* p = std::getenv("MX_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/mx/autotune.json";
}

// Flat {"key": [tile, order], ...} file.
std::vector<std::pair<std::string, std::pair<int, int>>> tune_load() {
  std::vector<std::pair<std::string, std::pair<int, int>>> out;
  FILE* f = std::fopen(tune_path().c_str(), "r");
  if (!f) return out;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
  std::fclose(f);
  size_t pos = 0;
  while ((pos = txt.find('"', pos)) != std::string::npos) {
    const size_t end = txt.find('"', pos + 1);
    if (end == std::string::npos) break;
    std::string key = txt.substr(pos + 1, end - pos - 1);
    int a = 0, b = 0;
    if (std::sscanf(txt.c_str() + end + 1, " : [ %d , %d ]", &a, &b) == 2) out.push_back({key, {a, b}});
    pos = end + 1;
  }
  return out;
}

void tune_store(const std::string& key, int tile, int order) {
  auto all = tune_load();
  bool found = false;
  for (auto& kv : all)
    if (kv.first == key) { kv.second = {tile, order}; found = true; }
  if (!found) all.push_back({key, {tile, order}});
  const std::string path = tune_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    std::string dir = path.substr(0, slash), cur;
    for (size_t q = 1; q <= dir.size(); ++q)
      if (q == dir.size() || dir[q] == '/') { cur = dir.substr(0, q); mkdir(cur.c_str(), 0755); }
  }
  const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  for (size_t q = 0; q < all.size(); ++q)
    std::fprintf(f, "  \"%s\": [%d, %d]%s\n", all[q].first.c_str(), all[q].second.first,
                 all[q].second.second, q + 1 < all.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
}

void enqueue_head(mx_system* s, cudaStream_t st);
void enqueue_step(mx_system* s, int last, cudaStream_t st);

mx_status trial_ms(mx_system* s, double* ms) {
  const size_t bytes = (size_t)6 * s->N * sizeof(double);
  MX_CUDA(cudaMemcpyAsync(s->d_tmp, s->d.xv, bytes, cudaMemcpyDeviceToDevice, s->st));
  cudaEvent_t e0, e1;
  MX_CUDA(cudaEventCreate(&e0));
  MX_CUDA(cudaEventCreate(&e1));
  // a warm-up call of two steps, then the timed one: an interior step (its
  // kick makes its own prep) and a call's last step, as the production graphs
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) MX_CUDA(cudaEventRecord(e0, s->st));
    enqueue_head(s, s->st);
    MX_CUDA(slot_done(s, false, untimed));
    enqueue_step(s, 0, s->st);
    MX_CUDA(slot_done(s, true, untimed));
    enqueue_step(s, 1, s->st);
    MX_CUDA(slot_done(s, true, untimed));
    MX_CUDA(settle_with(s, untimed));
  }
  MX_CUDA(cudaEventRecord(e1, s->st));
  MX_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  MX_CUDA(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MX_CUDA(cudaMemcpyAsync(s->d.xv, s->d_tmp, bytes, cudaMemcpyDeviceToDevice, s->st));
  MX_CUDA(cudaMemsetAsync(s->d.status, 0, sizeof(unsigned), s->st));
  MX_CUDA(cudaMemsetAsync(s->d.pair_count, 0, 2 * sizeof(int), s->st));
  // trials run at creation: the encounter log and the counters start empty
  MX_CUDA(cudaMemsetAsync(s->d.ever, 0, s->N, s->st));
  MX_CUDA(cudaMemsetAsync(s->d.bb_count, 0, sizeof(unsigned long long), s->st));
  MX_CUDA(cudaMemsetAsync(s->d.defer_total, 0, sizeof(unsigned long long), s->st));
  MX_CUDA(cudaMemsetAsync(s->d.work_ops, 0, 8 * sizeof(unsigned long long), s->st));
  MX_CUDA(cudaMemsetAsync(s->d.kick_ctr, 0, 2 * sizeof(int), s->st));
  MX_CUDA(cudaMemsetAsync(s->d.gstep, 0, sizeof(long long), s->st));
  MX_CUDA(cudaStreamSynchronize(s->st));
  *ms = t;
  return MX_OK;
}

// A tile is whole warps, from 64 to 256 targets.
bool valid_tile(int tile) { return tile >= 64 && tile <= mx::kThreads && tile % 32 == 0; }

mx_status autotune(mx_system* s) {
  const char* env = std::getenv("MX_AUTOTUNE");
  if (env && std::strcmp(env, "0") == 0) return MX_OK;
  const std::string key = tune_key(s);
  for (auto& kv : tune_load())
    if (kv.first == key) {
      const int tile = kv.second.first, order = kv.second.second;
      if (valid_tile(tile) && (order == 0 || order == 1)) return set_tiling(s, tile, order);
    }
  double best = 1e300;
  int bt = s->tile, bo = s->order;
  // whole warps from 64 to 256 targets: besides the powers of two, sizes whose
  // block count fills the resident slots' waves more evenly (a long kernel
  // ends with its last, partly filled wave)
  for (int tile : {64, 96, 128, 160, 192, 224, 256})
    for (int order : {0, 1}) {
      if (order == 1 && s->params.size() == 1) continue;   // one system: order is moot
      MX_TRY(set_tiling(s, tile, order));
      double ms = 1e300;
      for (int rep = 0; rep < 2; ++rep) {   // the better of two trials
        double t = 0.0;
        MX_TRY(trial_ms(s, &t));
        ms = std::min(ms, t);
      }
      if (ms < best) { best = ms; bt = tile; bo = order; }
    }
  MX_TRY(set_tiling(s, bt, bo));
  tune_store(key, bt, bo);
  return MX_OK;
}

// Builds the device side of a batch of systems (one system = batch of one).
mx_status build(mx_system* s, const std::vector<const double*>& m_big,
                const std::vector<const double*>& xv_helio, const std::vector<const double*>& rp,
                const std::vector<const double*>& rho) {
  const int nsys = (int)s->params.size();
  std::vector<mx::SysDev> sys(nsys);
  std::vector<mx::Tile> tiles;
  int off = 0, boff = 0, tiles_cap = 0;
  for (int k = 0; k < nsys; ++k) {
    const int n = s->nbig[k] + s->nsmall[k];
    sys[k] = make_sysdev(s->params[k], off, s->nbig[k], n, boff);
    tiles_cap += (n + kMinTile - 1) / kMinTile;
    off += n;
    boff += s->nbig[k];
  }
  s->h_sys = sys;
  s->tiles_cap = tiles_cap;
  tiles = make_tiles(sys, s->tile, s->order);
  s->N = off;
  s->NB = boff;
  const int N = s->N, NB = s->NB;
  if (N <= 0) return fail(MX_ERR_ARG, "empty system");
  mx::Dev& d = s->d;
  int cap = 0;
  for (auto& p : s->params) cap = std::max(cap, p.pair_cap);
  int cap2 = 1;
  while (cap2 < cap) cap2 <<= 1;
  MX_TRY(dalloc(s, &d.xv, (size_t)6 * N));
  MX_TRY(dalloc(s, &d.xv0, (size_t)6 * N));
  MX_TRY(dalloc(s, &s->d_tmp, (size_t)6 * N));
  MX_TRY(dalloc(s, &d.rp_cm, N));
  MX_TRY(dalloc(s, &d.kdrag, N));
  MX_TRY(dalloc(s, &d.bx, NB));
  MX_TRY(dalloc(s, &d.by, NB));
  MX_TRY(dalloc(s, &d.bz, NB));
  MX_TRY(dalloc(s, &d.bmu, NB));
  MX_TRY(dalloc(s, &d.brc, NB));
  MX_TRY(dalloc(s, &d.brc4, 4 * (size_t)NB));
  MX_TRY(dalloc(s, &d.P, 3 * (size_t)nsys));
  MX_TRY(dalloc(s, &d.bk, 6 * (size_t)NB));
  MX_TRY(dalloc(s, &d.arrive, 1));
  MX_TRY(dalloc(s, &d.flags, N));
  MX_TRY(dalloc(s, &d.keys, cap2));
  MX_TRY(dalloc(s, &d.pair_count, 2));
  d.work_count = d.pair_count + 1;
  const int work_cap = cap + NB;
  const int mem_cap = 4 * cap + NB;
  MX_TRY(dalloc(s, &d.work_off, work_cap + 1));
  MX_TRY(dalloc(s, &d.work_mem, mem_cap));
  MX_TRY(dalloc(s, &d.work_sys, work_cap));
  MX_TRY(dalloc(s, &d.work_wfrom, work_cap));
  MX_TRY(dalloc(s, &d.work_nsub, work_cap));
  d.cont_cap = std::min(work_cap, 1 << 14);
  MX_TRY(dalloc(s, &d.cont_count, 1));
  MX_TRY(dalloc(s, &d.ever, N));
  MX_TRY(dalloc(s, &d.bb_count, 1));
  MX_TRY(dalloc(s, &d.kick_ctr, 2));
  d.kbits = nullptr;
  d.kmode = 0;
  d.kwords = (N + 31) / 32;
  d.kcap = 0;
  MX_TRY(dalloc(s, &d.cont_item, d.cont_cap));
  MX_TRY(dalloc(s, &d.cont_state, (size_t)d.cont_cap * 27));
  // deferred planetesimals: per-step history of the big bodies, records
  {
    const size_t per_step = (size_t)20 * NB * sizeof(double) + (size_t)NB * sizeof(int) +
                            (size_t)6 * nsys * sizeof(double) + 2 * sizeof(int);
    int hc = kMaxWindow;
    while (hc > 1 && (size_t)hc * per_step > kHistBudget) hc >>= 1;
    d.hist_cap = hc;
    d.dcap = 1 << 14;
    MX_TRY(dalloc(s, &d.lag, N));
    MX_TRY(dalloc(s, &d.hstep, 1));
    MX_TRY(dalloc(s, &d.rcount, 3));
    MX_TRY(dalloc(s, &d.defer_total, 1));
    MX_TRY(dalloc(s, &d.work_ops, 8));
    MX_TRY(dalloc(s, &d.h_P, (size_t)hc * 6 * nsys));
    MX_TRY(dalloc(s, &d.h_b0, (size_t)hc * 6 * NB));
    MX_TRY(dalloc(s, &d.h_b1, (size_t)hc * 6 * NB));
    MX_TRY(dalloc(s, &d.h_bx, (size_t)hc * 3 * NB));
    MX_TRY(dalloc(s, &d.h_mu, (size_t)hc * NB));
    MX_TRY(dalloc(s, &d.h_rc, (size_t)hc * NB));
    MX_TRY(dalloc(s, &d.h_gap, (size_t)hc * 3 * NB));
    MX_TRY(dalloc(s, &d.h_ej, hc));
    MX_TRY(dalloc(s, &d.h_comp, (size_t)hc * NB));
    MX_TRY(dalloc(s, &d.h_nkick, hc));
    MX_TRY(dalloc(s, &d.d_rec, (size_t)3 * d.dcap * mx::kRecInts));
    MX_TRY(dalloc(s, &d.d_state, (size_t)3 * d.dcap * mx::kRecDoubles));
    s->window = std::min(kDefaultWindow, hc / 2);
  }
  MX_TRY(dalloc(s, &d.status, 1));
  MX_TRY(dalloc(s, &d.gbar, 8));
  MX_TRY(dalloc(s, &d.stat, N));
  MX_TRY(dalloc(s, &s->d_grow, NB));
  MX_TRY(dalloc(s, &d.gap_r, NB));
  MX_TRY(dalloc(s, &d.gap_w, NB));
  MX_TRY(dalloc(s, &d.gap_f, NB));
  MX_TRY(dalloc(s, &d.brad, NB));
  MX_TRY(dalloc(s, &d.gstep, 1));
  d.grow = s->d_grow;
  MX_TRY(dalloc(s, &d.ej_new, 1));
  MX_TRY(dalloc(s, &s->d_counts, nsys));
  MX_TRY(dalloc(s, &s->d_sys, nsys));
  MX_TRY(dalloc(s, &s->d_tiles, tiles_cap));
  MX_TRY(dalloc(s, &s->d_energy, 7 * (size_t)nsys));
  MX_TRY(dalloc(s, &s->d_sink, 1));
  d.sys = s->d_sys;
  d.tiles = s->d_tiles;
  d.N = N;
  d.NB = NB;
  d.nsys = nsys;
  d.ntiles = (int)tiles.size();
  d.tile = s->tile;
  d.big_max = 0;
  for (auto& q : sys) d.big_max = std::max(d.big_max, q.nbig);
  d.pair_cap = cap;
  d.work_cap = work_cap;
  d.mem_cap = mem_cap;
  d.kepler_max_iter = s->params[0].kepler_max_iter;
  d.bs_max_sub = s->params[0].bs_max_sub;
  d.bs_tol = s->params[0].bs_tol;
  cudaStream_t st = s->st;
  MX_CUDA(cudaMemcpyAsync(s->d_sys, sys.data(), nsys * sizeof(mx::SysDev), cudaMemcpyHostToDevice, st));
  MX_CUDA(cudaMemcpyAsync(s->d_tiles, tiles.data(), tiles.size() * sizeof(mx::Tile),
                          cudaMemcpyHostToDevice, st));
  MX_CUDA(cudaMemsetAsync(d.status, 0, sizeof(unsigned), st));
  MX_CUDA(cudaMemsetAsync(d.gbar, 0, 8 * sizeof(unsigned), st));
  MX_CUDA(cudaMemsetAsync(d.pair_count, 0, 2 * sizeof(int), st));
  MX_CUDA(cudaMemsetAsync(d.flags, 0, N, st));
  MX_CUDA(cudaMemsetAsync(d.stat, 0, N, st));
  MX_CUDA(cudaMemsetAsync(s->d_grow, 0, std::max(NB, 1) * sizeof(mx::Growth), st));
  MX_CUDA(cudaMemsetAsync(d.gap_r, 0, std::max(NB, 1) * sizeof(double), st));
  MX_CUDA(cudaMemsetAsync(d.gap_w, 0, std::max(NB, 1) * sizeof(double), st));
  MX_CUDA(cudaMemsetAsync(d.gap_f, 0, std::max(NB, 1) * sizeof(double), st));
  MX_CUDA(cudaMemsetAsync(d.brad, 0, std::max(NB, 1) * sizeof(double), st));
  MX_CUDA(cudaMemsetAsync(d.gstep, 0, sizeof(long long), st));
  MX_CUDA(cudaMemsetAsync(d.ej_new, 0, sizeof(int), st));
  MX_CUDA(cudaMemsetAsync(d.ever, 0, N, st));
  MX_CUDA(cudaMemsetAsync(d.bb_count, 0, sizeof(unsigned long long), st));
  MX_CUDA(cudaMemsetAsync(d.kick_ctr, 0, 2 * sizeof(int), st));
  MX_CUDA(cudaMemsetAsync(d.arrive, 0, sizeof(int), st));
  MX_CUDA(cudaMemsetAsync(d.lag, 0, N, st));
  MX_CUDA(cudaMemsetAsync(d.hstep, 0, sizeof(int), st));
  MX_CUDA(cudaMemsetAsync(d.rcount, 0, 3 * sizeof(int), st));
  MX_CUDA(cudaMemsetAsync(d.defer_total, 0, sizeof(unsigned long long), st));
  MX_CUDA(cudaMemsetAsync(d.work_ops, 0, 8 * sizeof(unsigned long long), st));
  update_defer(s);
  // host staging: state rows, masses as mu = G m, per-body drag inputs
  std::vector<double> xv((size_t)6 * N), bmu(NB, 0.0), rpb(N, 1.0), rhob(N, 1.0);
  for (int k = 0; k < nsys; ++k) {
    const int n = s->nbig[k] + s->nsmall[k], o = sys[k].off;
    for (int c = 0; c < 6; ++c)
      std::memcpy(&xv[(size_t)c * N + o], xv_helio[k] + (size_t)c * n, n * sizeof(double));
    for (int i = 0; i < s->nbig[k]; ++i) bmu[sys[k].boff + i] = s->params[k].G * m_big[k][i];
    for (int q = 0; q < s->nsmall[k]; ++q) {
      if (rp[k]) rpb[o + s->nbig[k] + q] = rp[k][q];
      if (rho[k]) rhob[o + s->nbig[k] + q] = rho[k][q];
    }
  }
  double *d_rp = nullptr, *d_rho = nullptr;
  MX_CUDA(cudaMalloc(&d_rp, N * sizeof(double)));
  MX_CUDA(cudaMalloc(&d_rho, N * sizeof(double)));
  MX_CUDA(cudaMemcpyAsync(d.xv, xv.data(), xv.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  MX_CUDA(cudaMemcpyAsync(d.bmu, bmu.data(), NB * sizeof(double), cudaMemcpyHostToDevice, st));
  MX_CUDA(cudaMemcpyAsync(d_rp, rpb.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
  MX_CUDA(cudaMemcpyAsync(d_rho, rhob.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
  MX_CUDA(cudaMemsetAsync(d.brc, 0, NB * sizeof(double), st));
  mx::launch_init_sys(d, 1, s->params[0].rcrit_hill, st);
  mx::launch_init_bodies(d, d_rp, d_rho, 1, st);
  MX_CUDA(cudaGetLastError());
  MX_CUDA(cudaStreamSynchronize(st));
  cudaFree(d_rp);
  cudaFree(d_rho);
  int nsm = 0;
  MX_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device));
  s->bs_blocks = 4 * nsm;
  s->catch_blocks = 4 * nsm;
  mx::configure_drift();
  mx::configure_detect();
  mx::configure_kick();
  mx::configure_bs();
  mx::configure_orbit();
  s->eject_every = s->params[0].eject_every;
  return sync_status(s);
}

void destroy_impl(mx_system* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  if (s->st) cudaStreamSynchronize(s->st);
  drop_graphs(s);
  for (void* p : s->allocs) cudaFree(p);
  if (s->h_status) cudaFreeHost(s->h_status);
  if (s->h_count) cudaFreeHost(s->h_count);
  if (s->h_need) cudaFreeHost(s->h_need);
  if (s->side_st) {
    cudaStreamSynchronize(s->side_st);
    cudaStreamDestroy(s->side_st);
  }
  for (auto& sp : s->side_spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  for (auto e : s->mk_head)
    if (e) cudaEventDestroy(e);
  for (auto e : s->mk_step)
    if (e) cudaEventDestroy(e);
  if (s->ev_main) cudaEventDestroy(s->ev_main);
  if (s->ev_side) cudaEventDestroy(s->ev_side);
  if (s->cap_st) cudaStreamDestroy(s->cap_st);
  delete s;
}

mx_status create(mx_system** out, void* stream) {
  mx_system* s = new mx_system();
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    delete s;
    return fail(MX_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  s->st = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaDeviceGetStreamPriorityRange(&s->prio_low, &s->prio_high) != cudaSuccess ||
      cudaStreamCreateWithPriority(&s->side_st, cudaStreamNonBlocking, s->prio_high) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_main, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_side, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&s->h_status, sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&s->h_count, 2 * sizeof(int)) != cudaSuccess) {
    destroy_impl(s);
    return fail(MX_ERR_CUDA, "stream or pinned allocation failed");
  }
  *out = s;
  return MX_OK;
}

}  // namespace

extern "C" {

const char* mx_last_error(void) { return g_last_error.c_str(); }

mx_status mx_init_system(const mx_params* p, int n_big, int n_small, const double* m_big,
                         const double* xv_helio, const double* rp_km, const double* rho_gcm3,
                         void* cuda_stream, mx_system** out) {
  g_last_error.clear();
  if (!out) return fail(MX_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!valid_params(p)) return fail(MX_ERR_ARG, "invalid parameters");
  if (n_big < 0 || n_small < 0 || n_big + n_small <= 0 || (long long)n_big + n_small > (1 << 30))
    return fail(MX_ERR_ARG, "invalid body counts");
  if ((n_big > 0 && !m_big) || !xv_helio) return fail(MX_ERR_ARG, "NULL input array");
  if (p->gas.enabled && n_small > 0 && (!rp_km || !rho_gcm3))
    return fail(MX_ERR_ARG, "gas drag needs rp_km and rho_gcm3");
  if (p->gas.enabled && !(p->gas.hr_1au > 0 && p->gas.gamma_c > 0 && p->gas.sigma_mol_cm2 > 0))
    return fail(MX_ERR_ARG, "invalid gas parameters");
  for (int i = 0; i < n_big; ++i)
    if (!(m_big[i] >= 0.0)) return fail(MX_ERR_ARG, "negative or NaN mass");
  mx_system* s = nullptr;
  MX_TRY(create(&s, cuda_stream));
  s->params.assign(1, *p);
  s->nbig.assign(1, n_big);
  s->nsmall.assign(1, n_small);
  mx_status r = build(s, {m_big}, {xv_helio}, {rp_km}, {rho_gcm3});
  if (r == MX_OK) r = autotune(s);
  if (r != MX_OK) {
    std::string msg = g_last_error;
    destroy_impl(s);
    return fail(r, msg);
  }
  *out = s;
  return MX_OK;
}

mx_status mx_init_batch(int n_sys, const mx_params* params, const int* n_big, const int* n_small,
                        const double* const* m_big, const double* const* xv_helio,
                        const double* const* rp_km, const double* const* rho_gcm3,
                        void* cuda_stream, mx_system** out) {
  g_last_error.clear();
  if (!out) return fail(MX_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_sys <= 0 || !params || !n_big || !n_small || !m_big || !xv_helio)
    return fail(MX_ERR_ARG, "invalid batch arguments");
  long long total = 0;
  for (int k = 0; k < n_sys; ++k) {
    const mx_params* p = &params[k];
    if (!valid_params(p)) return fail(MX_ERR_ARG, "invalid parameters of system " + std::to_string(k));
    if (n_big[k] < 0 || n_small[k] < 0 || n_big[k] + n_small[k] <= 0)
      return fail(MX_ERR_ARG, "invalid body counts of system " + std::to_string(k));
    if ((n_big[k] > 0 && !m_big[k]) || !xv_helio[k]) return fail(MX_ERR_ARG, "NULL input array");
    if (p->gas.enabled && n_small[k] > 0 && (!rp_km || !rho_gcm3 || !rp_km[k] || !rho_gcm3[k]))
      return fail(MX_ERR_ARG, "gas drag needs rp_km and rho_gcm3");
    for (int i = 0; i < n_big[k]; ++i)
      if (!(m_big[k][i] >= 0.0)) return fail(MX_ERR_ARG, "negative or NaN mass");
    if (p->eject_every != params[0].eject_every)
      return fail(MX_ERR_ARG, "eject_every differs between systems");
    total += n_big[k] + n_small[k];
  }
  if (total > (1LL << 30)) return fail(MX_ERR_ARG, "too many bodies");
  mx_system* s = nullptr;
  MX_TRY(create(&s, cuda_stream));
  s->params.assign(params, params + n_sys);
  s->nbig.assign(n_big, n_big + n_sys);
  s->nsmall.assign(n_small, n_small + n_sys);
  std::vector<const double*> mb(m_big, m_big + n_sys), xv(xv_helio, xv_helio + n_sys);
  std::vector<const double*> rp(n_sys, nullptr), rh(n_sys, nullptr);
  for (int k = 0; k < n_sys; ++k) {
    if (rp_km) rp[k] = rp_km[k];
    if (rho_gcm3) rh[k] = rho_gcm3[k];
  }
  mx_status r = build(s, mb, xv, rp, rh);
  if (r == MX_OK) r = autotune(s);
  if (r != MX_OK) {
    std::string msg = g_last_error;
    destroy_impl(s);
    return fail(r, msg);
  }
  *out = s;
  return MX_OK;
}

mx_status mx_batch_offsets(mx_system* s, int* offsets) {
  if (!s || !offsets) return fail(MX_ERR_ARG, "invalid arguments");
  for (size_t k = 0; k < s->h_sys.size(); ++k) offsets[k] = s->h_sys[k].off;
  offsets[s->h_sys.size()] = s->N;
  return MX_OK;
}

mx_status mx_batch_size(mx_system* s, int* n_sys, int* n_total) {
  if (!s) return fail(MX_ERR_ARG, "NULL system");
  if (n_sys) *n_sys = (int)s->h_sys.size();
  if (n_total) *n_total = s->N;
  return MX_OK;
}

mx_status mx_tiling(mx_system* s, int* tile, int* order) {
  if (!s) return fail(MX_ERR_ARG, "NULL system");
  if (tile) *tile = s->tile;
  if (order) *order = s->order;
  return MX_OK;
}

mx_status mx_set_tiling(mx_system* s, int tile, int order) {
  if (!s || !valid_tile(tile) || !(order == 0 || order == 1))
    return fail(MX_ERR_ARG, "tile must be a multiple of 32 from 64 to 256 and order 0 or 1");
  MX_TRY(set_device(s));
  return set_tiling(s, tile, order);
}

mx_status mx_set_defer_window(mx_system* s, int window) {
  if (!s || window < 0) return fail(MX_ERR_ARG, "invalid arguments");
  if (2 * window > s->d.hist_cap)
    return fail(MX_ERR_ARG, "window longer than half the history (" + std::to_string(s->d.hist_cap / 2) + " slots)");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  s->window = window;
  update_defer(s);
  drop_graphs(s);
  return MX_OK;
}

mx_status mx_defer_stats(mx_system* s, int* window, int* max_window, long long* deferred,
                         long long* catchups) {
  if (!s) return fail(MX_ERR_ARG, "NULL system");
  MX_TRY(set_device(s));
  unsigned long long n = 0;
  MX_CUDA(cudaMemcpyAsync(&n, s->d.defer_total, sizeof(n), cudaMemcpyDeviceToHost, s->st));
  MX_CUDA(cudaStreamSynchronize(s->st));
  if (window) *window = s->d.defer ? s->window : 0;
  if (max_window) *max_window = s->d.hist_cap / 2;
  if (deferred) *deferred = (long long)n;
  if (catchups) *catchups = s->catchups;
  return MX_OK;
}

mx_status mx_set_persistent(mx_system* s, int on, long long spin_limit) {
  if (!s || on < 0 || on > 1) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  if (on && s->tile < mx::kThreads) MX_TRY(set_tiling(s, mx::kThreads, s->order));
  s->persist = on;
  s->persist_spin = spin_limit < 0 ? (1ll << 24) : spin_limit;
  s->persist_grid = on ? mx::persist_grid(s->d) : 0;
  if (on && s->persist_grid <= 0) {
    s->persist = 0;
    return fail(MX_ERR_CUDA, "no resident grid for the persistent step");
  }
  drop_graphs(s);
  return MX_OK;
}

mx_status mx_catchup_work(mx_system* s, long long* ops6, int reset) {
  if (!s || !ops6) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  unsigned long long w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // after the side stream's last pass, so its counts are complete
  if (s->side_busy) MX_CUDA(cudaStreamWaitEvent(s->st, s->ev_side, 0));
  MX_CUDA(cudaMemcpyAsync(w, s->d.work_ops, sizeof(w), cudaMemcpyDeviceToHost, s->st));
  if (reset) MX_CUDA(cudaMemsetAsync(s->d.work_ops, 0, sizeof(w), s->st));
  MX_CUDA(cudaStreamSynchronize(s->st));
  for (int k = 0; k < 3; ++k) {
    ops6[k] = (long long)w[k];
    ops6[3 + k] = (long long)w[4 + k];
  }
  return MX_OK;
}

mx_status mx_energy_batch(mx_system* s, double* E, double* L3) {
  if (!s || !E || !L3) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  const int nsys = (int)s->h_sys.size();
  mx::launch_energy(s->d, s->d_energy, s->st);
  std::vector<double> o(7 * (size_t)nsys);
  MX_CUDA(cudaMemcpyAsync(o.data(), s->d_energy, o.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  MX_TRY(sync_status(s));
  for (int k = 0; k < nsys; ++k) {
    E[k] = o[7 * k + 2];
    for (int c = 0; c < 3; ++c) L3[3 * k + c] = o[7 * k + 4 + c];
  }
  return MX_OK;
}

void mx_destroy(mx_system* s) { destroy_impl(s); }

mx_status mx_sizes(mx_system* s, int* n_big, int* n_small) {
  if (!s) return fail(MX_ERR_ARG, "NULL system");
  if (n_big) *n_big = s->nbig[0];
  if (n_small) *n_small = s->nsmall[0];
  return MX_OK;
}

mx_status mx_step(mx_system* s, int n_steps) {
  if (!s || n_steps < 0) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  if (n_steps == 0) {
    MX_TRY(settle(s));
    return sync_status(s);
  }
  MX_TRY(ensure_graphs(s));
  MX_CUDA(cudaGraphLaunch(s->g_head, s->st));
  MX_CUDA(slot_done(s, false, untimed));
  for (int k = 0; k < n_steps; ++k) {
    const bool test = eject_after(s, s->step + k + 1);
    const bool split = split_after(s, s->step + k + 1);
    MX_CUDA(cudaGraphLaunch((k + 1 == n_steps || split) ? s->g_last : s->g_mid, s->st));
    if (test) mx::launch_eject(s->d, 1, s->st);
    MX_CUDA(cudaGetLastError());
    MX_CUDA(slot_done(s, true, untimed));
    if (split && k + 1 < n_steps) {   // the next step starts with its own half kick
      MX_CUDA(cudaGraphLaunch(s->g_head, s->st));
      MX_CUDA(slot_done(s, false, untimed));
    }
  }
  s->step += n_steps;
  // a deferred body's drift is the catch-up's; only planetesimals of systems
  // with at most kDeferMaxBig big bodies are ever deferred
  bool deferrable = false;
  if (s->d.defer)
    for (const auto& sy : s->h_sys) deferrable |= sy.nbig <= mx::kDeferMaxBig;
  s->pd_ok = !deferrable;
  return sync_status(s);
}

}  // extern "C"

namespace {

// mx_step_profiled / mx_step_timed: launch by launch with events.  total_ms
// sums each step's span (its first launch to its last, a window-end
// catch-up included); with a flush buffer, the buffer is overwritten before
// every step, outside the spans.
mx_status profiled_run(mx_system* s, int n_steps, void* flush, size_t flush_bytes,
                       double* kernel_ms, int* launches, double* total_ms) {
  if (!s || n_steps < 0 || (flush_bytes > 0 && !flush)) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  cudaStream_t st = s->st;
  // (kind, event-before, event-after) per launch
  std::vector<mx_system::Span> spans;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> steps;   // per-step spans, main stream
  auto mk = [&](cudaStream_t sm, cudaEvent_t* ev) -> cudaError_t {
    cudaError_t r = cudaEventCreate(ev);
    return (r != cudaSuccess) ? r : cudaEventRecord(*ev, sm);
  };
  auto timed3 = [&](int k, cudaStream_t sm, auto&& launch) -> cudaError_t {
    mx_system::Span sp{k, nullptr, nullptr};
    cudaError_t r = mk(sm, &sp.a);
    if (r != cudaSuccess) return r;
    launch();
    r = mk(sm, &sp.b);
    if (r != cudaSuccess) return r;
    if (sm == st) {
      spans.push_back(sp);
    } else {
      s->side_spans.push_back(sp);
    }
    return cudaGetLastError();
  };
  auto timed = [&](int k, auto&& launch) { return timed3(k, st, launch); };
  auto step_open = [&](int k) -> cudaError_t {
    cudaError_t r = cudaSuccess;
    if (flush_bytes > 0) r = cudaMemsetAsync(flush, k & 0xff, flush_bytes, st);
    steps.push_back({nullptr, nullptr});
    return (r != cudaSuccess) ? r : mk(st, &steps.back().first);
  };
  auto step_close = [&]() -> cudaError_t { return mk(st, &steps.back().second); };
  cudaError_t e = cudaSuccess;
  if (n_steps == 0) {   // only the pending catch-up, timed
    e = step_open(0);
    if (e == cudaSuccess) e = settle_with(s, timed3);
    if (e == cudaSuccess) e = step_close();
  } else {
    e = step_open(0);
    if (e == cudaSuccess) e = timed(MX_K_PREP, [&] { mx::launch_prep(s->d, 0.0, 1, st); });
    if (e == cudaSuccess) e = timed(MX_K_JUMP_KICK, [&] { mx::launch_jump_kick(s->d, 0.0, 0.5, 1, st); });
    if (e == cudaSuccess) e = slot_done(s, false, timed3);
  }
  for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
    const bool test = eject_after(s, s->step + k + 1);
    const bool last_step = (k + 1 == n_steps) || split_after(s, s->step + k + 1);
    if (k > 0) e = step_open(k);
    if (e == cudaSuccess && k > 0 && split_after(s, s->step + k)) {   // a fresh half kick
      e = timed(MX_K_PREP, [&] { mx::launch_prep(s->d, 0.0, 1, st); });
      if (e == cudaSuccess) e = timed(MX_K_JUMP_KICK, [&] { mx::launch_jump_kick(s->d, 0.0, 0.5, 1, st); });
      if (e == cudaSuccess) e = slot_done(s, false, timed3);
    }
    if (e == cudaSuccess) e = timed(MX_K_JUMP_DRIFT, [&] { mx::launch_jump_drift(s->d, 0.5, st); });
    if (e == cudaSuccess)
      e = timed(MX_K_DETECT, [&] {
        mx::launch_detect(s->d, s->d.xv0, s->d.xv, s->d.flags, s->d.keys, s->d.pair_count, s->d.pair_cap, 1, st);
      });
    if (e == cudaSuccess) e = timed(MX_K_GROUPS, [&] { mx::launch_groups(s->d, st); });
    if (e == cudaSuccess) e = timed(MX_K_BS, [&] { mx::launch_bs(s->d, s->bs_blocks, st); });
    if (!last_step && fuse_prep(s)) {
      if (e == cudaSuccess) e = timed(MX_K_JUMP_KICK, [&] { mx::launch_jump_kick_fused(s->d, st); });
    } else {
      if (e == cudaSuccess) e = timed(MX_K_PREP, [&] { mx::launch_prep(s->d, 0.5, last_step ? 1 : 2, st); });
      if (e == cudaSuccess)
        e = timed(MX_K_JUMP_KICK, [&] { mx::launch_jump_kick(s->d, 0.5, 0.5, last_step ? 1 : 2, st); });
    }
    if (e == cudaSuccess && test) e = timed(MX_K_EJECT, [&] { mx::launch_eject(s->d, 1, st); });
    if (e == cudaSuccess) e = slot_done(s, true, timed3);
    if (e == cudaSuccess) e = step_close();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  double sum[MX_NKERN] = {0};
  int cnt[MX_NKERN] = {0};
  float ms = 0.f;
  for (auto& sp : spans) {
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, sp.a, sp.b);
    sum[sp.kind] += ms;
    cnt[sp.kind]++;
  }
  // side-stream launches: those that have completed (all of them after a settle)
  std::vector<mx_system::Span> keep;
  for (auto& sp : s->side_spans) {
    if (e == cudaSuccess && cudaEventQuery(sp.b) == cudaSuccess) {
      e = cudaEventElapsedTime(&ms, sp.a, sp.b);
      sum[sp.kind] += ms;
      cnt[sp.kind]++;
      cudaEventDestroy(sp.a);
      cudaEventDestroy(sp.b);
    } else {
      keep.push_back(sp);
    }
  }
  s->side_spans.swap(keep);
  double tot = 0.0;
  for (auto& sp : steps) {
    if (e == cudaSuccess && sp.first && sp.second) {
      e = cudaEventElapsedTime(&ms, sp.first, sp.second);
      tot += ms;
    }
  }
  if (total_ms) *total_ms = tot;
  for (auto& sp : spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  for (auto& sp : steps) {
    if (sp.first) cudaEventDestroy(sp.first);
    if (sp.second) cudaEventDestroy(sp.second);
  }
  if (e != cudaSuccess) return fail(MX_ERR_CUDA, std::string("profiled step: ") + cudaGetErrorString(e));
  for (int k = 0; k < MX_NKERN; ++k) {
    if (kernel_ms) kernel_ms[k] = sum[k];
    if (launches) launches[k] = cnt[k];
  }
  s->step += n_steps;
  return sync_status(s);
}

// mx_step_timed: the step graphs of mx_step, in their timed variants (an
// event node between kernels), one step at a time.  Before every step the
// flush buffer is overwritten; after it the host waits for the step's end and
// reads its events.  A step's span runs from its first event to its end (a
// window-end catch-up included).  Deferral's side-stream launches are timed
// as in profiled_run.
mx_status timed_graph_run(mx_system* s, int n_steps, void* flush, size_t flush_bytes,
                          double* kernel_ms, int* launches, double* total_ms) {
  if (!s || n_steps < 0 || (flush_bytes > 0 && !flush)) return fail(MX_ERR_ARG, "invalid arguments");
  if (n_steps == 0) return profiled_run(s, 0, flush, flush_bytes, kernel_ms, launches, total_ms);
  MX_TRY(set_device(s));
  MX_TRY(ensure_graphs(s));
  // with no per-kernel output asked for, the production graphs run as they
  // are, with events only around each step
  const bool per_kernel = kernel_ms || launches;
  if (per_kernel) MX_TRY(ensure_timed_graphs(s));
  cudaGraphExec_t gh = per_kernel ? s->gt_head : s->g_head;
  cudaGraphExec_t gm = per_kernel ? s->gt_mid : s->g_mid;
  cudaGraphExec_t gl = per_kernel ? s->gt_last : s->g_last;
  cudaStream_t st = s->st;
  double sum[MX_NKERN] = {0};
  int cnt[MX_NKERN] = {0};
  std::vector<mx_system::Span> spans;   // window-end launches on the main stream
  auto timed3 = [&](int k, cudaStream_t sm, auto&& launch) -> cudaError_t {
    mx_system::Span sp{k, nullptr, nullptr};
    cudaError_t r = cudaEventCreate(&sp.a);
    if (r == cudaSuccess) r = cudaEventRecord(sp.a, sm);
    if (r != cudaSuccess) return r;
    launch();
    r = cudaEventCreate(&sp.b);
    if (r == cudaSuccess) r = cudaEventRecord(sp.b, sm);
    if (r != cudaSuccess) return r;
    if (sm == st) spans.push_back(sp);
    else s->side_spans.push_back(sp);
    return cudaGetLastError();
  };
  static const int kHeadKind[2] = {MX_K_PREP, MX_K_JUMP_KICK};
  static const int kStepKind[6] = {MX_K_JUMP_DRIFT, MX_K_DETECT, MX_K_GROUPS, MX_K_BS, MX_K_PREP,
                                   MX_K_JUMP_KICK};
  cudaEvent_t e_end = nullptr, e_start = nullptr;
  MX_CUDA(cudaEventCreate(&e_end));
  MX_CUDA(cudaEventCreate(&e_start));
  double tot = 0.0;
  float ms = 0.f;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
    // a call's first step, and a step after an ejection test, start with a half kick
    const bool head = (k == 0) || split_after(s, s->step + k);
    const bool test = eject_after(s, s->step + k + 1);
    const bool split = split_after(s, s->step + k + 1);
    if (flush_bytes > 0) e = cudaMemsetAsync(flush, k & 0xff, flush_bytes, st);
    if (e == cudaSuccess && !per_kernel) e = cudaEventRecord(e_start, st);
    if (e == cudaSuccess && head) {
      e = cudaGraphLaunch(gh, st);
      if (e == cudaSuccess) e = slot_done(s, false, timed3);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch((k + 1 == n_steps || split) ? gl : gm, st);
    if (e == cudaSuccess && test) e = timed3(MX_K_EJECT, st, [&] { mx::launch_eject(s->d, 1, st); });
    if (e == cudaSuccess) e = slot_done(s, true, timed3);
    if (e == cudaSuccess) e = cudaEventRecord(e_end, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e_end);
    if (e != cudaSuccess) break;
    if (head && per_kernel)
      for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
        e = cudaEventElapsedTime(&ms, s->mk_head[q], s->mk_head[q + 1]);
        sum[kHeadKind[q]] += ms;
        cnt[kHeadKind[q]]++;
      }
    // a fused interior kick has no k_prep: its span (empty) is not counted
    const bool fused = !(k + 1 == n_steps || split) && fuse_prep(s);
    for (int q = 0; q < 6 && per_kernel && e == cudaSuccess; ++q) {
      e = cudaEventElapsedTime(&ms, s->mk_step[q], s->mk_step[q + 1]);
      if (fused && kStepKind[q] == MX_K_PREP) continue;
      sum[kStepKind[q]] += ms;
      cnt[kStepKind[q]]++;
    }
    for (auto& sp : spans) {
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, sp.a, sp.b);
      sum[sp.kind] += ms;
      cnt[sp.kind]++;
      cudaEventDestroy(sp.a);
      cudaEventDestroy(sp.b);
    }
    spans.clear();
    if (e == cudaSuccess)
      e = cudaEventElapsedTime(&ms, !per_kernel ? e_start : head ? s->mk_head[0] : s->mk_step[0],
                               e_end);
    tot += ms;
  }
  for (auto& sp : spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  cudaEventDestroy(e_end);
  cudaEventDestroy(e_start);
  // side-stream launches that have completed
  std::vector<mx_system::Span> keep;
  for (auto& sp : s->side_spans) {
    if (e == cudaSuccess && cudaEventQuery(sp.b) == cudaSuccess) {
      e = cudaEventElapsedTime(&ms, sp.a, sp.b);
      sum[sp.kind] += ms;
      cnt[sp.kind]++;
      cudaEventDestroy(sp.a);
      cudaEventDestroy(sp.b);
    } else {
      keep.push_back(sp);
    }
  }
  s->side_spans.swap(keep);
  if (e != cudaSuccess) return fail(MX_ERR_CUDA, std::string("timed step: ") + cudaGetErrorString(e));
  for (int q = 0; q < MX_NKERN; ++q) {
    if (kernel_ms) kernel_ms[q] = sum[q];
    if (launches) launches[q] = cnt[q];
  }
  if (total_ms) *total_ms = tot;
  s->step += n_steps;
  return sync_status(s);
}

}  // namespace

extern "C" {

mx_status mx_step_profiled(mx_system* s, int n_steps, double* kernel_ms, int* launches,
                           double* total_ms) {
  if (s) s->pd_ok = 0;
  return profiled_run(s, n_steps, nullptr, 0, kernel_ms, launches, total_ms);
}

mx_status mx_step_timed(mx_system* s, int n_steps, void* dev_flush, size_t flush_bytes,
                        double* kernel_ms, int* launches, double* total_ms) {
  if (s) s->pd_ok = 0;
  return timed_graph_run(s, n_steps, dev_flush, flush_bytes, kernel_ms, launches, total_ms);
}

mx_status mx_step_wall(mx_system* s, int n_steps, void* dev_flush, size_t flush_bytes,
                       double* wall_ms, double* flush_ms) {
  if (!s || n_steps < 1 || (flush_bytes > 0 && !dev_flush) || !wall_ms)
    return fail(MX_ERR_ARG, "invalid arguments");
  s->pd_ok = 0;
  MX_TRY(set_device(s));
  MX_TRY(ensure_graphs(s));
  MX_TRY(settle(s));   // nothing pending from earlier calls enters the span
  cudaStream_t st = s->st;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (auto& e : ev) MX_CUDA(cudaEventCreate(&e));
  cudaError_t e = cudaEventRecord(ev[0], st);
  for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
    const bool head = (k == 0) || split_after(s, s->step + k);
    const bool test = eject_after(s, s->step + k + 1);
    const bool split = split_after(s, s->step + k + 1);
    if (flush_bytes > 0) e = cudaMemsetAsync(dev_flush, k & 0xff, flush_bytes, st);
    if (e == cudaSuccess && head) {
      e = cudaGraphLaunch(s->g_head, st);
      if (e == cudaSuccess) e = slot_done(s, false, untimed);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch((k + 1 == n_steps || split) ? s->g_last : s->g_mid, st);
    if (e == cudaSuccess && test) {
      mx::launch_eject(s->d, 1, st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = slot_done(s, true, untimed);
  }
  // the settle waits for the side stream on the main stream, so the end event
  // follows every catch-up of the steps
  if (e == cudaSuccess) e = settle_with(s, untimed);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
  if (e == cudaSuccess && flush_ms) {   // the flushes alone, nothing else in flight
    e = cudaEventRecord(ev[2], st);
    for (int k = 0; k < n_steps && e == cudaSuccess && flush_bytes > 0; ++k)
      e = cudaMemsetAsync(dev_flush, (k + 1) & 0xff, flush_bytes, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], st);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(flush_ms ? ev[3] : ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  *wall_ms = ms;
  if (e == cudaSuccess && flush_ms) {
    e = cudaEventElapsedTime(&ms, ev[2], ev[3]);
    *flush_ms = ms;
  }
  for (auto& q : ev) cudaEventDestroy(q);
  if (e != cudaSuccess) return fail(MX_ERR_CUDA, std::string("wall step: ") + cudaGetErrorString(e));
  s->step += n_steps;
  return sync_status(s);
}

mx_status mx_last_encounters(mx_system* s, int* host_pairs, int cap, int* n_pairs) {
  if (!s || !n_pairs || cap < 0 || (cap > 0 && !host_pairs)) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  MX_CUDA(cudaMemcpyAsync(s->h_count, s->d.pair_count, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  MX_CUDA(cudaStreamSynchronize(s->st));
  const int n = std::min(*s->h_count, s->d.pair_cap);
  *n_pairs = *s->h_count;
  std::vector<unsigned long long> keys(n);
  if (n > 0)
    MX_CUDA(cudaMemcpy(keys.data(), s->d.keys, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  std::vector<std::pair<int, int>> pr(n);
  for (int k = 0; k < n; ++k)
    pr[k] = {(int)(keys[k] & 0xffffffffull), (int)((keys[k] >> 32) & 0x7fffffffull)};
  std::sort(pr.begin(), pr.end());
  for (int k = 0; k < n && k < cap; ++k) {
    host_pairs[2 * k] = pr[k].first;
    host_pairs[2 * k + 1] = pr[k].second;
  }
  return (*s->h_count > s->d.pair_cap) ? fail(MX_ERR_PAIR_OVERFLOW, "pair list overflow") : MX_OK;
}

mx_status mx_accel(mx_system* s, double* dev_acc) {
  if (!s || !dev_acc) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  mx::launch_prep(s->d, 0.0, 0, s->st);
  mx::launch_accel(s->d, dev_acc, 0, s->N, 0, s->st);
  return sync_status(s);
}

mx_status mx_gas_drag(mx_system* s, double* dev_acc) {
  if (!s || !dev_acc) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  const int ns = s->nsmall[0];
  if (ns == 0) return MX_OK;
  MX_CUDA(cudaMemsetAsync(dev_acc, 0, (size_t)3 * ns * sizeof(double), s->st));
  mx::launch_prep(s->d, 0.0, 0, s->st);
  mx::launch_accel(s->d, dev_acc, 1, ns, s->nbig[0], s->st);
  return sync_status(s);
}

mx_status mx_detect_encounters(mx_system* s, const double* dev_xv0, const double* dev_xv1,
                               unsigned char* dev_flags, int* dev_pairs, int cap, int* n_pairs) {
  if (!s || !dev_xv0 || !dev_xv1 || !n_pairs || cap < 0 || (cap > 0 && !dev_pairs) ||
      s->params.size() != 1)
    return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  unsigned char* flags = dev_flags ? dev_flags : s->d.flags;
  MX_CUDA(cudaMemsetAsync(flags, 0, s->N, s->st));
  MX_CUDA(cudaMemsetAsync(s->d.pair_count, 0, sizeof(int), s->st));
  mx::Dev dd = s->d;
  dd.ever = nullptr;        // caller-supplied states do not enter the encounter log
  dd.bb_count = nullptr;
  dd.defer = 0;
  mx::launch_detect(dd, dev_xv0, dev_xv1, flags, s->d.keys, s->d.pair_count, s->d.pair_cap, 0, s->st);
  mx::launch_sort_keys(s->d.keys, s->d.pair_count, s->d.pair_cap, 1, s->st);
  if (dev_pairs && cap > 0)
    mx::launch_keys_to_pairs(s->d.keys, s->d.pair_count, std::min(cap, s->d.pair_cap), dev_pairs, s->st);
  MX_CUDA(cudaMemcpyAsync(s->h_count, s->d.pair_count, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  MX_TRY(sync_status(s));
  *n_pairs = *s->h_count;
  // the step's own pair list is overwritten; it is rebuilt by the next step
  MX_CUDA(cudaMemsetAsync(s->d.pair_count, 0, 2 * sizeof(int), s->st));
  MX_CUDA(cudaStreamSynchronize(s->st));
  if (*n_pairs > cap || *n_pairs > s->d.pair_cap)
    return fail(MX_ERR_PAIR_OVERFLOW, "more flagged pairs than cap");
  return MX_OK;
}

mx_status mx_kepler_drift(mx_system* s, double* dev_xv, double h) {
  if (!s || !dev_xv || !std::isfinite(h)) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  const mx_params& p = s->params[0];
  mx::launch_drift_buf(dev_xv, s->N, p.G * p.m_star, h, p.kepler_max_iter, s->d.status, s->st);
  return sync_status(s);
}

mx_status mx_energy(mx_system* s, double* E, double* L3) {
  if (!s || !E || !L3) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  mx::launch_energy(s->d, s->d_energy, s->st);
  double o[7];
  MX_CUDA(cudaMemcpyAsync(o, s->d_energy, sizeof(o), cudaMemcpyDeviceToHost, s->st));
  MX_TRY(sync_status(s));
  *E = o[2];
  L3[0] = o[4];
  L3[1] = o[5];
  L3[2] = o[6];
  return MX_OK;
}

mx_status mx_get_state(mx_system* s, double* xv_host, int coords, long long* step) {
  if (!s || !xv_host || (coords != MX_COORD_HELIO && coords != MX_COORD_DH))
    return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  const double* src = s->d.xv;
  if (coords == MX_COORD_HELIO) {
    mx::launch_prep(s->d, 0.0, 0, s->st);
    mx::launch_readout(s->d, s->d_tmp, s->st);
    src = s->d_tmp;
  }
  MX_CUDA(cudaMemcpyAsync(xv_host, src, (size_t)6 * s->N * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  MX_TRY(sync_status(s));
  if (step) *step = s->step;
  return MX_OK;
}

mx_status mx_set_state(mx_system* s, const double* xv_host, int coords, long long step) {
  if (!s || !xv_host || (coords != MX_COORD_HELIO && coords != MX_COORD_DH))
    return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  MX_CUDA(cudaMemcpyAsync(s->d.xv, xv_host, (size_t)6 * s->N * sizeof(double), cudaMemcpyHostToDevice, s->st));
  if (coords == MX_COORD_HELIO) {
    mx::launch_init_sys(s->d, 0, 0.0, s->st);
    mx::launch_init_bodies(s->d, nullptr, nullptr, 0, s->st);
  }
  mx::launch_set_step(s->d, step, s->st);
  MX_TRY(sync_status(s));
  s->step = step;
  return MX_OK;
}

mx_status mx_get_state_device(mx_system* s, double* dev_xv) {
  if (!s || !dev_xv) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  MX_CUDA(cudaMemcpyAsync(dev_xv, s->d.xv, (size_t)6 * s->N * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
  return MX_OK;
}

mx_status mx_set_state_device(mx_system* s, const double* dev_xv) {
  if (!s || !dev_xv) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  MX_CUDA(cudaMemcpyAsync(s->d.xv, dev_xv, (size_t)6 * s->N * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
  return MX_OK;
}

mx_status mx_check_ejections(mx_system* s, int* n_removed) {
  if (!s) return fail(MX_ERR_ARG, "NULL system");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  MX_CUDA(cudaMemsetAsync(s->d.ej_new, 0, sizeof(int), s->st));
  mx::launch_prep(s->d, 0.0, 0, s->st);   // P of the current state
  mx::launch_eject(s->d, 0, s->st);
  MX_CUDA(cudaMemcpyAsync(s->h_count, s->d.ej_new, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  MX_TRY(sync_status(s));
  if (*s->h_count > 0) s->removed_any = true;
  if (n_removed) *n_removed = *s->h_count;
  return MX_OK;
}

mx_status mx_body_status(mx_system* s, signed char* host_stat, int* n_removed) {
  if (!s) return fail(MX_ERR_ARG, "NULL system");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  if (host_stat)
    MX_CUDA(cudaMemcpyAsync(host_stat, s->d.stat, s->N, cudaMemcpyDeviceToHost, s->st));
  const int nsys = (int)s->h_sys.size();
  std::vector<int> counts(nsys, 0);
  if (n_removed) {
    mx::launch_stat_count(s->d, s->d_counts, s->st);
    MX_CUDA(cudaMemcpyAsync(counts.data(), s->d_counts, nsys * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  }
  MX_TRY(sync_status(s));
  if (n_removed) std::copy(counts.begin(), counts.end(), n_removed);
  return MX_OK;
}

mx_status mx_set_growth(mx_system* s, int sys, const mx_growth* g, double gap_c) {
  if (!s || !g || sys < 0 || sys >= (int)s->h_sys.size() || !(gap_c >= 0.0))
    return fail(MX_ERR_ARG, "invalid arguments");
  const int nb = s->nbig[sys];
  std::vector<mx::Growth> gr(nb);
  bool any = false;
  for (int i = 0; i < nb; ++i) {
    const mx_growth& q = g[i];
    gr[i] = mx::Growth{q.m0, q.mc, q.mf, q.tau_c, q.tau_g, q.delta_r, q.grows ? 1 : 0, 0};
    if (!q.grows) continue;
    any = true;
    if (!(q.m0 >= 0.0 && q.mc >= 0.0 && q.mf >= 0.0 && q.tau_c > 0.0 && q.tau_g > 0.0 &&
          std::isfinite(q.delta_r) && std::isfinite(q.mf) && std::isfinite(q.tau_c) &&
          std::isfinite(q.tau_g)))
      return fail(MX_ERR_ARG, "invalid growth track of body " + std::to_string(i));
  }
  if (any && !(s->params[sys].dt > 0.0)) return fail(MX_ERR_ARG, "growth needs dt > 0");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  mx::SysDev& S = s->h_sys[sys];
  if (nb > 0)
    MX_CUDA(cudaMemcpyAsync(s->d_grow + S.boff, gr.data(), nb * sizeof(mx::Growth),
                            cudaMemcpyHostToDevice, s->st));
  S.grow_on = any ? 1 : 0;
  S.gap_c = gap_c;
  MX_CUDA(cudaMemcpyAsync(s->d_sys + sys, &S, sizeof(mx::SysDev), cudaMemcpyHostToDevice, s->st));
  // no gap until the first step with the track
  if (nb > 0) MX_CUDA(cudaMemsetAsync(s->d.gap_w + S.boff, 0, nb * sizeof(double), s->st));
  s->grow_any = false;
  for (auto& y : s->h_sys) s->grow_any = s->grow_any || y.grow_on;
  update_defer(s);
  drop_graphs(s);
  return sync_status(s);
}

mx_status mx_planets(mx_system* s, double* m_host, double* r_host) {
  if (!s) return fail(MX_ERR_ARG, "NULL system");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  const int NB = s->NB;
  std::vector<double> mu(NB), rad(NB);
  if (r_host) mx::launch_radius(s->d, s->st);
  if (NB > 0) {
    MX_CUDA(cudaMemcpyAsync(mu.data(), s->d.bmu, NB * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    MX_CUDA(cudaMemcpyAsync(rad.data(), s->d.brad, NB * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  }
  MX_TRY(sync_status(s));
  for (size_t k = 0; k < s->h_sys.size(); ++k) {
    const mx::SysDev& S = s->h_sys[k];
    for (int i = 0; i < S.nbig; ++i) {
      if (m_host) m_host[S.boff + i] = mu[S.boff + i] / s->params[k].G;
      if (r_host) r_host[S.boff + i] = rad[S.boff + i];
    }
  }
  return MX_OK;
}

mx_status mx_elements(mx_system* s, double* dev_el) {
  if (!s || !dev_el) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  mx::launch_prep(s->d, 0.0, 0, s->st);
  mx::launch_elements(s->d, dev_el, s->st);
  return sync_status(s);
}

mx_status mx_fp64_peak(void* cuda_stream, double ms_target, double* tflops) {
  if (!tflops || !(ms_target > 0)) return fail(MX_ERR_ARG, "invalid arguments");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  MX_CUDA(cudaGetDevice(&dev));
  MX_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  double* sink = nullptr;
  MX_CUDA(cudaMalloc(&sink, sizeof(double)));
  cudaEvent_t e0, e1;
  MX_CUDA(cudaEventCreate(&e0));
  MX_CUDA(cudaEventCreate(&e1));
  const int blocks = nsm * 8;
  int iters = 256;
  float ms = 0.f;
  for (int rep = 0; rep < 8; ++rep) {
    MX_CUDA(cudaEventRecord(e0, st));
    mx::launch_dfma(sink, blocks, iters, st);
    MX_CUDA(cudaEventRecord(e1, st));
    MX_CUDA(cudaEventSynchronize(e1));
    MX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms >= 0.8 * ms_target) break;
    const double scale = std::min(16.0, ms_target / std::max(ms, 0.01f));
    iters = (int)std::min(1 << 24, (int)(iters * scale) + 1);
  }
  const double flops = 2.0 * 8.0 * (double)iters * blocks * 256.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return MX_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ adjoint
namespace {

// Per-tile partial records for the adjoint and the loss: 3 doubles per big
// body of the tile's system plus 9.
// The doubles of the adjoint's recorded Bulirsch-Stoer sub-steps to start
// with (each group reserves room for 128 sub-steps; a two-body group's
// sub-step takes 15 doubles).  The tape grows to what a step's groups reserve.
constexpr size_t kAdjTape = (size_t)1 << 23;

// Makes the share keys hold `n` (a power of two for the bitonic sort's
// padding; the stream is idle).
mx_status grow_share_keys(mx_system* s, unsigned long long n) {
  if (n <= (unsigned long long)s->a_skeys_cap) return MX_OK;
  unsigned long long cap = 1024;
  while (cap < n) cap <<= 1;
  if (cap > (1ull << 30)) return fail(MX_ERR_PAIR_OVERFLOW, "too many encounter shares");
  if (s->a_skeys) {
    MX_CUDA(cudaFree(s->a_skeys));
    s->allocs.erase(std::remove(s->allocs.begin(), s->allocs.end(), (void*)s->a_skeys), s->allocs.end());
    s->a_skeys = nullptr;
    s->a_skeys_cap = 0;
  }
  MX_TRY(dalloc(s, &s->a_skeys, (size_t)cap));
  s->a_skeys_cap = (int)cap;
  return MX_OK;
}

// Makes the tape hold `need` doubles, with a quarter to spare (the stream is
// idle: the caller has synchronised it).
mx_status grow_tape(mx_system* s, unsigned long long need) {
  if (need <= s->a_tape_cap) return MX_OK;
  const unsigned long long cap = std::max(need + need / 4, 2 * s->a_tape_cap);
  MX_CUDA(cudaFree(s->a_tape));
  s->allocs.erase(std::remove(s->allocs.begin(), s->allocs.end(), (void*)s->a_tape), s->allocs.end());
  s->a_tape = nullptr;
  s->a_tape_cap = 0;
  MX_TRY(dalloc(s, &s->a_tape, (size_t)cap));
  s->a_tape_cap = cap;
  return MX_OK;
}

// The step's device view with the adjoint's tiling.
mx::Dev adjoint_dev(const mx_system* s) {
  mx::Dev d = s->d;
  d.tiles = s->a_tiles;
  d.ntiles = s->a_ntiles;
  d.tile = s->a_tile;
  return d;
}

// The adjoint's targets per block.  With few big bodies, 256 (the per-tile
// partial records and their folds favour full blocks: 0.62 against 1.01 ms a
// step with 64 on the 4-core disk).  With many, the kick's reverse is a long
// pass over the pairs in which every block does the same work, so the block
// count is chosen to fill whole waves of the resident blocks: of 160 to 256
// targets (whole warps), the size whose waves come closest to a whole number
// (902 blocks of 224 targets make 2.97 waves on 152 SMs, where 790 of 256
// make 2.6 and a third of the SMs idle through the last).
int adjoint_tile(const mx_system* s) {
  if (s->d.big_max <= 64) return mx::kThreads;
  const int nsm = s->bs_blocks / 4;
  int best_tile = mx::kThreads;
  double best = -1.0;
  for (int w = mx::kThreads / 32; w >= 5; --w) {
    const int t = 32 * w;
    const int occ = mx::adjoint_vjp_blocks_per_sm(t);
    if (occ <= 0 || nsm <= 0) continue;
    const double waves = (double)make_tiles(s->h_sys, t, 0).size() / ((double)occ * nsm);
    const double eff = waves / std::ceil(waves);
    if (eff > best + 1e-9) {
      best = eff;
      best_tile = t;
    }
  }
  return best_tile;
}

mx_status ensure_adjoint_store(mx_system* s) {
  if (s->a_sub_want == 0 || s->a_sub) return MX_OK;
  MX_TRY(dalloc(s, &s->a_sub, (size_t)s->a_sub_want * mx::kAdjSubRec));
  s->a_sub_cap = s->a_sub_want;
  return MX_OK;
}

mx_status ensure_adjoint(mx_system* s) {
  MX_TRY(ensure_adjoint_store(s));
  const int N = s->N;
  if (!s->a_tiles) {
    MX_TRY(dalloc(s, &s->a_x2, (size_t)6 * N));   // x2 and v1: one 6 x N pre-drift state
    s->a_v1 = s->a_x2 + 3 * (size_t)N;
    const int gcap = s->d.work_cap;   // one entry per item of the step's work list
    s->a_gcap = gcap;
    MX_TRY(dalloc(s, &s->a_gM, gcap));
    MX_TRY(dalloc(s, &s->a_goff, gcap));
    MX_TRY(dalloc(s, &s->a_gcontrib, (size_t)gcap * mx::kMaxGroup * 6));
    MX_TRY(dalloc(s, &s->a_tape, kAdjTape));
    MX_TRY(dalloc(s, &s->a_need, 2));
    if (cudaMallocHost(&s->h_need, 2 * sizeof(unsigned long long)) != cudaSuccess)
      return fail(MX_ERR_OOM, "cudaMallocHost");
    MX_TRY(dalloc(s, &s->a_scount, 1));
    MX_TRY(dalloc(s, &s->a_bfold, 3 * (size_t)s->NB));
    MX_TRY(dalloc(s, &s->a_lpend, (size_t)6 * N));
    s->a_xpend = s->a_lpend + 3 * (size_t)N;
    MX_TRY(dalloc(s, &s->a_subn, 1));
    MX_TRY(dalloc(s, &s->a_bsx, 3 * s->h_sys.size()));
    s->a_tape_cap = kAdjTape;
    MX_TRY(dalloc(s, &s->a_xv3, (size_t)6 * N));
    MX_TRY(dalloc(s, &s->a_x4, (size_t)3 * N));
    MX_TRY(dalloc(s, &s->a_P, 9 * s->h_sys.size()));
    MX_TRY(dalloc(s, &s->a_L, s->h_sys.size()));
    s->a_tile = adjoint_tile(s);
    std::vector<mx::Tile> tiles = make_tiles(s->h_sys, s->a_tile, 0);
    std::vector<int> poff(tiles.size());
    size_t off = 0;
    for (size_t t = 0; t < tiles.size(); ++t) {
      poff[t] = (int)off;
      off += 3 * (size_t)s->h_sys[tiles[t].sys].nbig + 9;
    }
    if (off > (size_t)INT32_MAX) return fail(MX_ERR_ARG, "adjoint partials too large");
    MX_TRY(dalloc(s, &s->a_part, off));
    s->a_part_cap = off;
    MX_TRY(dalloc(s, &s->a_poff, tiles.size()));
    std::vector<int> systiles(s->h_sys.size() + 1, 0);   // tiles come in system order
    for (const mx::Tile& t : tiles) systiles[t.sys + 1] += 1;
    for (size_t k = 1; k < systiles.size(); ++k) systiles[k] += systiles[k - 1];
    MX_TRY(dalloc(s, &s->a_systiles, systiles.size()));
    MX_CUDA(cudaMemcpyAsync(s->a_systiles, systiles.data(), systiles.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s->st));
    MX_TRY(dalloc(s, &s->a_tiles, tiles.size()));
    s->a_ntiles = (int)tiles.size();
    MX_CUDA(cudaMemcpyAsync(s->a_poff, poff.data(), poff.size() * sizeof(int), cudaMemcpyHostToDevice, s->st));
    MX_CUDA(cudaMemcpyAsync(s->a_tiles, tiles.data(), tiles.size() * sizeof(mx::Tile),
                            cudaMemcpyHostToDevice, s->st));
    MX_CUDA(cudaStreamSynchronize(s->st));
  }
  return MX_OK;
}

// The adjoint's view of the system's buffers for one call on dev_lambda and
// dev_dparams (the per-step fields are the caller's).
mx::Adj make_adj(const mx_system* s, double* dev_lambda, double* dev_dparams) {
  mx::Adj a{};
  a.v1 = s->a_v1;
  a.x2 = s->a_x2;
  a.xv3 = s->a_xv3;
  a.x4 = s->a_x4;
  a.lam = dev_lambda;
  a.part = s->a_part;
  a.poff = s->a_poff;
  a.sys_tiles = s->a_systiles;
  a.P = s->a_P;
  a.dpar = dev_dparams;
  a.groups = s->a_groups;
  a.g_cap = s->a_gcap;
  a.bs_blocks = s->bs_blocks;
  a.g_M = s->a_gM;
  a.g_off = s->a_goff;
  a.g_contrib = s->a_gcontrib;
  a.tape = s->a_tape;
  a.tape_cap = s->a_tape_cap;
  a.tape_need = s->a_need;
  a.sorted_shares = s->d.big_max > 64;
  a.skeys = s->a_skeys;
  a.scount = s->a_scount;
  a.skeys_cap = s->a_skeys_cap;
  a.bfold = s->a_bfold;
  a.bs_xsum = s->a_bsx;
  a.sub = s->a_sub;
  a.sub_count = s->a_subn;
  a.sub_cap = s->a_sub_cap;
  a.lin = nullptr;
  a.lpend = s->a_lpend;
  a.defer_k1 = 0;
  return a;
}

// The pending pair pass of a merged reverse, on its own, into the cotangent
// it belongs to (enqueued; the caller reads the status).
mx_status flush_adjoint(mx_system* s) {
  if (!s->a_pend) return MX_OK;
  mx::Adj a = make_adj(s, s->a_pend_lam, nullptr);
  mx::launch_adjoint_flush(adjoint_dev(s), a, s->a_xpend, s->st);
  s->a_pend = 0;
  return MX_OK;
}

}  // namespace

extern "C" {

mx_status mx_set_gas_params(mx_system* s, int k, double sigma1, double gamma, double cd_scale) {
  if (!s || k < 0 || k >= (int)s->h_sys.size() || !std::isfinite(sigma1) || !std::isfinite(gamma) ||
      !std::isfinite(cd_scale))
    return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  mx_params& p = s->params[k];
  p.gas.sigma1_gcm2 = sigma1;
  p.gas.gamma = gamma;
  p.gas.cd_scale = cd_scale;
  const mx::SysDev old = s->h_sys[k];
  mx::SysDev nw = make_sysdev(p, old.off, old.nbig, old.n, old.boff);
  s->h_sys[k] = nw;
  MX_CUDA(cudaMemcpyAsync(s->d_sys + k, &s->h_sys[k], sizeof(mx::SysDev), cudaMemcpyHostToDevice, s->st));
  MX_CUDA(cudaStreamSynchronize(s->st));
  return MX_OK;
}

mx_status mx_kick_branches(mx_system* s, int mode, long long max_kicks) {
  if (!s || mode < 0 || mode > 2 || max_kicks < 0 || max_kicks > (1LL << 30))
    return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  if (mode == 0) {
    s->d.kmode = 0;
    update_defer(s);
    drop_graphs(s);
    return MX_OK;
  }
  if (mode == 1) {
    const size_t words = (size_t)max_kicks * s->d.kwords;
    if (max_kicks > s->kbits_cap) {
      if (s->d.kbits) {
        cudaFree(s->d.kbits);
        s->allocs.erase(std::remove(s->allocs.begin(), s->allocs.end(), (void*)s->d.kbits), s->allocs.end());
        s->d.kbits = nullptr;
      }
      MX_TRY(dalloc(s, &s->d.kbits, words));
      s->kbits_cap = max_kicks;
    }
    MX_CUDA(cudaMemsetAsync(s->d.kbits, 0, words * sizeof(unsigned), s->st));
    s->d.kcap = (int)max_kicks;
  } else if (!s->d.kbits) {
    return fail(MX_ERR_ARG, "no recorded branches to replay");
  }
  s->d.kmode = mode;
  update_defer(s);
  drop_graphs(s);
  MX_CUDA(cudaStreamSynchronize(s->st));
  return MX_OK;
}

mx_status mx_encounter_log(mx_system* s, unsigned char* dev_ever, long long* n_big_big, int reset) {
  if (!s) return fail(MX_ERR_ARG, "NULL system");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  if (dev_ever) MX_CUDA(cudaMemcpyAsync(dev_ever, s->d.ever, s->N, cudaMemcpyDeviceToDevice, s->st));
  unsigned long long bb = 0;
  MX_CUDA(cudaMemcpyAsync(&bb, s->d.bb_count, sizeof(bb), cudaMemcpyDeviceToHost, s->st));
  if (reset) {
    MX_CUDA(cudaMemsetAsync(s->d.ever, 0, s->N, s->st));
    MX_CUDA(cudaMemsetAsync(s->d.bb_count, 0, sizeof(unsigned long long), s->st));
  }
  MX_CUDA(cudaStreamSynchronize(s->st));
  if (n_big_big) *n_big_big = (long long)bb;
  return MX_OK;
}

mx_status mx_set_step_index(mx_system* s, long long step) {
  if (!s || step < 0 || step > (1LL << 29)) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  mx::launch_set_step(s->d, step, s->st);
  MX_CUDA(cudaStreamSynchronize(s->st));
  s->step = step;
  return MX_OK;
}

mx_status mx_loss_semimajor(mx_system* s, const double* dev_xv_helio0, const double* dev_w,
                            double* L, double* dev_seed_final, double* dev_seed_init) {
  if (!s || !dev_xv_helio0 || !dev_w || !L || !dev_seed_final || !dev_seed_init)
    return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  MX_TRY(ensure_adjoint(s));
  mx::launch_prep(s->d, 0.0, 0, s->st);
  mx::launch_loss(adjoint_dev(s), dev_xv_helio0, dev_w, dev_seed_final, dev_seed_init, s->a_part,
                  s->a_poff, s->a_L, s->st);
  MX_CUDA(cudaMemcpyAsync(L, s->a_L, s->h_sys.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  return sync_status(s);
}

mx_status mx_adjoint_encounters(mx_system* s, int on) {
  if (!s || on < 0 || on > 2) return fail(MX_ERR_ARG, "invalid arguments");
  s->a_groups = on;
  return MX_OK;
}

mx_status mx_adjoint_store(mx_system* s, long long slots) {
  if (!s || slots < 0 || slots > (1ll << 20)) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  if (s->a_sub) {   // the pool is replaced at the next adjoint step
    MX_CUDA(cudaStreamSynchronize(s->st));
    MX_CUDA(cudaFree(s->a_sub));
    s->allocs.erase(std::remove(s->allocs.begin(), s->allocs.end(), (void*)s->a_sub), s->allocs.end());
    s->a_sub = nullptr;
    s->a_sub_cap = 0;
  }
  s->a_sub_want = (unsigned)slots;
  return MX_OK;
}

mx_status mx_adjoint_init(mx_system* s, const double* dev_lambda, double* dev_grad_helio) {
  if (!s || !dev_lambda || !dev_grad_helio) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  MX_TRY(flush_adjoint(s));   // a merged reverse's pending pair pass first
  mx::launch_init_vjp(s->d, dev_lambda, dev_grad_helio, s->st);
  return sync_status(s);
}

static mx_status adjoint_step(mx_system* s, const double* dev_state_k, const double* dev_pd,
                       long long step_k, double* dev_lambda, double* dev_dparams) {
  if (!s || !dev_state_k || !dev_lambda || !dev_dparams || step_k < 0 || step_k > (1LL << 29))
    return fail(MX_ERR_ARG, "invalid arguments");
  if (s->eject_every > 0 || s->removed_any)
    return fail(MX_ERR_ARG, "the adjoint does not follow bodies removed by ejection");
  if (s->grow_any) return fail(MX_ERR_ARG, "the adjoint does not follow growing masses");
  MX_TRY(set_device(s));
  MX_TRY(settle(s));
  MX_TRY(ensure_adjoint(s));
  // a pending pair pass joins this step's last half kick only when this is
  // the step before it, on the same cotangent; otherwise it runs on its own
  const bool merge_in = s->a_pend && s->a_merge && s->a_pend_step == step_k + 1 &&
                        s->a_pend_lam == dev_lambda;
  if (s->a_pend && !merge_in) MX_TRY(flush_adjoint(s));
  mx::Adj a = make_adj(s, dev_lambda, dev_dparams);
  a.z0 = dev_state_k;
  a.step = (int)step_k;
  if (dev_pd) {   // read only: the kernels that write x2 and v1 do not run
    a.pd = dev_pd;
    a.x2 = const_cast<double*>(dev_pd);
    a.v1 = a.x2 + 3 * (size_t)s->N;
  }
  a.lin = merge_in ? s->a_lpend : nullptr;
  a.defer_k1 = s->a_merge;
  const mx::Dev d = adjoint_dev(s);
  mx::launch_adjoint_step_a(d, a, s->st);
  if (a.groups) {   // the groups' tape, sized from their plan
    MX_CUDA(cudaMemcpyAsync(s->h_need, s->a_need, 2 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s->st));
    MX_TRY(sync_status(s));
    MX_TRY(grow_tape(s, s->h_need[0]));
    if (a.sorted_shares) MX_TRY(grow_share_keys(s, s->h_need[1]));
    a.tape = s->a_tape;
    a.tape_cap = s->a_tape_cap;
    a.skeys = s->a_skeys;
    a.skeys_cap = s->a_skeys_cap;
  }
  mx::launch_adjoint_step_b(d, a, s->st);
  s->a_pend = 0;
  if (s->a_merge) {   // this step's first half kick waits for its pair pass
    MX_CUDA(cudaMemcpyAsync(s->a_xpend, dev_state_k, 3 * (size_t)s->N * sizeof(double),
                            cudaMemcpyDeviceToDevice, s->st));
    s->a_pend = 1;
    s->a_pend_step = step_k;
    s->a_pend_lam = dev_lambda;
  }
  const mx_status r = sync_status(s);
  if (r != MX_OK) s->a_pend = 0;
  return r;
}

mx_status mx_adjoint_step(mx_system* s, const double* dev_state_k, long long step_k,
                          double* dev_lambda, double* dev_dparams) {
  return adjoint_step(s, dev_state_k, nullptr, step_k, dev_lambda, dev_dparams);
}

mx_status mx_adjoint_step_predrift(mx_system* s, const double* dev_state_k,
                                   const double* dev_predrift_k, long long step_k,
                                   double* dev_lambda, double* dev_dparams) {
  if (!dev_predrift_k) return fail(MX_ERR_ARG, "invalid arguments");
  return adjoint_step(s, dev_state_k, dev_predrift_k, step_k, dev_lambda, dev_dparams);
}

mx_status mx_predrift_state(mx_system* s, double* dev_xv) {
  if (!s || !dev_xv) return fail(MX_ERR_ARG, "invalid arguments");
  if (!s->pd_ok)
    return fail(MX_ERR_ARG, "no pre-drift state: the last mx_step had deferral on, or none ran");
  MX_TRY(set_device(s));
  MX_CUDA(cudaMemcpyAsync(dev_xv, s->d.xv0, 6 * (size_t)s->N * sizeof(double),
                          cudaMemcpyDeviceToDevice, s->st));
  return sync_status(s);
}

mx_status mx_adjoint_merge(mx_system* s, int on) {
  if (!s || on < 0 || on > 1) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  if (!on && s->a_pend) {
    MX_TRY(flush_adjoint(s));
    MX_TRY(sync_status(s));
  }
  s->a_merge = on;
  return MX_OK;
}

mx_status mx_adjoint_flush(mx_system* s) {
  if (!s) return fail(MX_ERR_ARG, "invalid arguments");
  MX_TRY(set_device(s));
  if (!s->a_pend) return MX_OK;
  MX_TRY(flush_adjoint(s));
  return sync_status(s);
}

}  // extern "C"
