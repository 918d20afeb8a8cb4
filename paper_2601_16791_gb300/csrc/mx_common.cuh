// mx_common.cuh -- device data layout and FP64 helpers shared by the sm_103a
// kernels of the hybrid symplectic step (arXiv 2601.16791, Sec. 2 and 3.1).
//
// Layout in HBM (all float64 unless noted), for all systems of a batch back to
// back (a single system is a batch of one):
//   state  6 x N   x, y, z, vx, vy, vz rows; each system's big bodies first.
//                  DH coordinates: heliocentric x, barycentric v.
//   xv0    6 x N   the post-jump, pre-drift state of the current step
//                  (detection endpoints and Bulirsch-Stoer starting point).
//   rp_cm, kdrag [N]  planetesimal radius [cm] and 3/(8 r_p[AU] rho_p).
//   bx,by,bz,bmu,brc [NB]  big bodies of every system, compact: positions
//                  staged for the kick (already jumped), mu = G m, rcrit.
//   P      [3 x nsys]  massive-body momentum sum mu_i v_i of each system.
//   flags  [N] uint8, pair keys [cap] uint64, Bulirsch-Stoer work list.
// Every kernel reads its system's constants from a SysDev record.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mx {

constexpr int kThreads = 256;     // threads per block of the per-body kernels (= tile)
constexpr int kBigChunk = 256;    // big bodies staged in shared memory per pass
constexpr int kMaxGroup = 16;     // bodies per Bulirsch-Stoer group (MX_MAX_GROUP)
constexpr int kBsRows = 8;        // extrapolation rows: n_k = 2, 4, ..., 16
constexpr int kMaxBigPairs = 512; // big-big encounter pairs handled per step
// Planetesimals are deferred only in systems with at most this many big
// bodies: a replayed step sums the gravity of every big body on one lane (in
// the direct path's order), so with many big bodies a replay costs more than
// the encounter it moves off the step.
constexpr int kDeferMaxBig = 64;
// Status of a body removed from the integration as ejected (Sec. 3.5).
constexpr signed char kStatEjected = -3;

// Device status bits, OR-ed by kernels and turned into mx_status on the host.
enum : unsigned {
  ST_KEPLER = 1u << 0,
  ST_BS = 1u << 1,
  ST_PAIR_OVF = 1u << 2,
  ST_NONFINITE = 1u << 3,
  ST_BARRIER = 1u << 4,
  ST_GROUP = 1u << 5,
  ST_WORK_OVF = 1u << 6,
  ST_TAPE = 1u << 7,     // an adjoint group needed more sub-steps than its tape holds
  ST_WINDOW = 1u << 8
};

// Constants of one system.
struct SysDev {
  int off;        // global index of the system's first body
  int nbig;       // massive bodies
  int n;          // all bodies
  int boff;       // index of its first big body in the compact big arrays
  double mu0, inv_mu0, sqrt_mu0;
  double h;       // step
  double inv_G, m_star;
  // gas (Sec. 3.1)
  int gas_on, cd_mode, gamma_one, flare_quarter;
  int rc_inf, pad0;
  double sigma1, gamma, inv_rc, r_in, hr1, flare, cd_scale;
  double c_rho;   // rho_g = c_rho * Sigma * R^-(1+flare)     [g/cm^3]
  double c_cs;    // c_s  = c_cs * R^(flare-1/2)              [AU/d]
  double inv_c_cs;
  double c_eta;   // eta  = c_eta * R^(2 flare)
  double deta_dgamma;  // d c_eta / d gamma
  double c_re;    // Re   = c_re * r_p[cm] * Ma * rho_g
  // disk gravity (Eqs. 10-12): radial force per unit mass c_dg * Sigma[g/cm^2],
  // times 1/R for gamma = 1 (dg_edge), outward positive
  int dg_on, dg_edge;
  double c_dg;
  double dlnS_dgamma;   // d ln S / d gamma of the series (0 for the edge form), for the adjoint
  // planet growth (Sec. 3.3) and gaps (Sec. 3.1, Eqs. 8-9)
  int grow_on, pad1;
  double G, rcrit_hill, gap_c;
};

// Growth track of one big body (Eqs. 13, 15; radius Eqs. 14, 16).
struct Growth {
  double m0, mc, mf;   // Msun
  double tc, tg;       // d
  double dr;           // AU
  int grows, pad;
};

// A block's worth of targets, never spanning two systems.
struct Tile {
  int sys, start, count, pad;
};

// Pointers to the device buffers.
struct Dev {
  double* xv;      // 6 x N
  double* xv0;     // 6 x N
  double* rp_cm;   // N
  double* kdrag;   // N
  double *bx, *by, *bz, *bmu, *brc;   // NB
  double* brc4;    // 4 x NB: rc^2, 0.01 rc^2, 0.1 rc, 1/(0.9 rc) of each big body (set_rcrit)
  double* P;       // 3 x nsys
  double* bk;      // 6 x NB: big bodies after the latest kick, the drift's source for them
  int* arrive;     // [1] blocks of a kick with its own prep that have read the history slot
  unsigned char* flags;               // N
  unsigned long long* keys;           // pair keys [pair_cap]
  int* pair_count;
  int* work_count;
  int* work_off;   // [work_cap + 1]
  int* work_mem;   // [mem_cap]
  int* work_sys;   // [work_cap]
  int* work_wfrom; // [work_cap]
  int* work_nsub;  // [work_cap] macro sub-steps used (diagnostic)
  int* cont_count; // groups handed from the packed to the spread BS phase
  int* cont_item;  // [cont_cap] their work items
  double* cont_state; // [cont_cap x (3 + 6 x 4)] their integration state
  int cont_cap;
  unsigned char* ever;          // [N] bodies flagged since the log was reset
  unsigned long long* bb_count; // big-big pairs flagged since the log was reset
  int* kick_ctr;   // [0]: half kicks made so far, [1]: index of the next launch's first
  unsigned* kbits; // recorded k branch of Eq. 7, one bit per (half kick, body)
  int kmode;       // 0: compute k from Re, 1: record, 2: replay
  int kwords;      // 32-bit words per half kick
  int kcap;        // half kicks the bit array holds
  unsigned* status;
  // Ejection (Sec. 3.5): a body with stat != 0 is out of the integration; it
  // keeps its state and every kernel of the step passes it by.  A removed
  // big body has mu = 0.
  signed char* stat;   // [N] 0, or kStatEjected
  int* ej_new;         // bodies removed by ejection tests since the host last cleared it
  // Growth (Sec. 3.3): tracks, and per big body the gap's centre (cylindrical
  // distance at kick time, k_prep), half-width (0: none) and density factor,
  // and the radius (k_grow).
  const Growth* grow;  // [NB]
  long long* gstep;    // [0] global index of the step under way (its first k_prep reads it)
  double *gap_r, *gap_w, *gap_f, *brad;   // [NB]
  const SysDev* sys;
  const Tile* tiles;
  int N, NB, nsys, ntiles;
  int tile;        // targets per tile = threads per block of the per-body kernels
  int big_max;     // most big bodies of any system (sizes the kernels' shared staging)
  int pair_cap, work_cap, mem_cap;
  int kepler_max_iter, bs_max_sub;
  double bs_tol;
  // Deferred planetesimals.  A planetesimal is massless, so its own close
  // encounter changes no other body: when its Bulirsch-Stoer group outlasts
  // the packed phase, the rest of its steps wait for the end of the window,
  // where k_catchup replays them from the big bodies' recorded history with
  // the same device functions (so the result is the one the direct path
  // gives, bit for bit).  defer = 0 leaves every step on the direct path.
  int defer;
  int hist_cap;        // history slots (two windows)
  int dcap;            // records per bank
  unsigned char* lag;  // [N] 1 while the body waits for a catch-up
  int* hstep;          // [0] history slot of the current step
  int* rcount;         // [3] records in each bank
  unsigned long long* defer_total;  // bodies deferred since creation
  // Work done by catch-ups, in units with a fixed algorithmic cost: [0]
  // body-slots drifted (jump + drift + encounter test), [1] half kicks of
  // one body, [2] force evaluations of two-body Bulirsch-Stoer groups that
  // the one-at-a-time step search makes (rows of the accepted try and of
  // every failed try before it); [0..2] main-stream passes, [4..6] the side
  // stream's.
  unsigned long long* work_ops;   // [8]
  // Grid barrier of the persistent step (k_step_persist): arrivals, the
  // barrier's generation, a flag set once any block gave up waiting, and
  // (from [4]) the tile counters of its per-body phases.
  unsigned* gbar;                   // [8]
  double* h_P;         // [hist_cap][2][3 nsys] P of jump 1, P of jump 2 and the kicks
  double* h_b0;        // [hist_cap][6][NB] big bodies after jump 1 (pre-drift)
  double* h_b1;        // [hist_cap][6][NB] big bodies after the drift (detection endpoint)
  double* h_bx;        // [hist_cap][3][NB] big positions after jump 2 (kick sources)
  double* h_mu;        // [hist_cap][NB] big mu during the slot, -1 for a removed body
  double* h_rc;        // [hist_cap][NB] big changeover radius during the slot
  double* h_gap;       // [hist_cap][3][NB] gaps during the slot: centre, half-width, factor
  int* h_ej;           // [hist_cap] 1: the ejection test follows the slot
  int* h_comp;         // [hist_cap][NB] big group of each big body, -1 for none
  int* h_nkick;        // [hist_cap] half kicks ending the slot; -1: a call's leading half kick
  int* d_rec;          // [3][dcap][kRecInts] records: bank 0 deferred in this window,
                       // banks 1 and 2 carried between windows
  double* d_state;     // [3][dcap][kRecDoubles]
};

// Record of a deferred body.  Ints: body, history slot t, group size (0: at
// the start of slot t with the body's state in doubles 3..8; >= 2: in the
// middle of slot t's Bulirsch-Stoer group), four member indices, the slot and
// count of pairs found at the last step of a side-stream pass, their big
// bodies (local indices).  Doubles: rem, H, nsub, 6 x 4 group state.
constexpr int kRecInts = 32;
constexpr int kRecDoubles = 3 + 6 * 4;

// Buffers of one adjoint step (k_adjoint.cu).
struct Adj {
  const double* z0;   // 6 x N state at the start of the step
  double* v1;         // 3 x N after kick 1
  double* x2;         // 3 x N after jump 1
  double* xv3;        // 6 x N after the drift
  double* x4;         // 3 x N after jump 2
  double* lam;        // 6 x N cotangent, in/out
  double* part;       // per-tile partial sums
  const int* poff;    // [ntiles] offset of each tile's partial record
  const int* sys_tiles;   // [nsys + 1] first tile of each system (tiles in system order)
  double* P;          // 9 per system: P0, P1, P3
  double* dpar;       // 3 per system, accumulated
  int step;           // index of the step (recorded k branches)
  // Bulirsch-Stoer groups (k_adj_bs.cu): x2 and v1 are the two halves of one
  // 6 x N pre-drift state.  The groups are the step's own work list (d.work_*,
  // built by k_groups from the recomputed endpoints), item by item.
  // groups: 0 none (the caller asserts no big-big encounter: bodies in groups
  // carry no cotangent); 1 every group; 2 groups of big bodies only (a loss
  // that leaves out the planetesimals that met a big body)
  int groups;
  int g_cap, bs_blocks;          // g_cap: work items (d.work_cap)
  int* g_M;                      // accepted sub-steps recorded per item, -1: not processed
  unsigned long long* g_off;     // tape offset of each item
  double* g_contrib;             // [g_cap][kMaxGroup][6] shares of members not written back
  double* tape;                  // accepted sub-steps: H, row, 6 x nb start state, slot
  unsigned long long tape_cap;   // doubles
  unsigned long long* tape_need; // [2]: doubles the step's groups reserve, and the
                                 // shares of big bodies not written back (k_adj_tape)
  // many big bodies (sorted_shares): each big body's shares are added in the
  // order of (body, item, member) keys sorted once, skeys_cap >= their count
  int sorted_shares;
  unsigned long long* skeys;
  int* scount;
  int skeys_cap;
  double* bfold;                 // 3 per big body: its folded kick cotangent (many big bodies)
  // merged reverse of consecutive half kicks (k_adjoint.cu, KickRev): lin
  // (or null) is the pending cotangent of the next step's first half kick,
  // taken in this step's last-kick pair pass; with defer_k1 this step's first
  // half kick leaves its own in lpend (3 x N) instead of a pair pass
  const double* lin;
  double* lpend;
  int defer_k1;
  // the forward step's pre-drift state (x2, v1), 6 x N (mx_predrift_state),
  // or null: recomputed.  When set, x2 and v1 point into it and are only read
  const double* pd;
  double* bs_xsum;               // 3 per system: sum of the big shares' position parts
  // two-body groups: the Stoermer sub-steps of each accepted macro sub-step,
  // kAdjSubRec doubles a slot (null: none are kept, the reverse recomputes)
  double* sub;
  unsigned* sub_count;           // slots handed out in this step
  unsigned sub_cap;              // slots
};

// One slot of kept Stoermer sub-steps: sub-steps 0..16, each six rows of 32
// lanes (separation x, y, z, force weight, 1/s, s^2 of the lane's term).
constexpr int kAdjSubVals = 6;
constexpr int kAdjSubRec = 17 * kAdjSubVals * 32;

// ------------------------------------------------------------------ helpers
// On this part FP64 instructions (conversions included) issue at ~1/60 of the
// FP32 rate with ~67-cycle dependent latency, so seeds are built with integer
// and FP32 instructions only.
//
// |x| as a float, read off the binary64 bit pattern: the exponent is rebased
// from bias 1023 to 127 and the top 20 mantissa bits are kept (truncation,
// relative error < 2^-20).  Valid for 2^-126 <= |x| < 2^128.
__device__ __forceinline__ float abs_to_float_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu;
  return __uint_as_float((hi - ((1023u - 127u) << 20)) << 3);
}

// x as a float for the FP32 encounter screen, read off the binary64 bit
// pattern like abs_to_float_bits (20 mantissa bits kept, relative error
// < 2^-20, far inside the screen's margin), sign kept; zero for
// |x| < 2^-126.  Valid for |x| < 2^128.  Integer instructions only, where a
// conversion would take an FP64 issue slot.
__device__ __forceinline__ float to_float_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned a = hi & 0x7fffffffu;
  const unsigned f = (a < (897u << 20)) ? 0u : ((a - ((1023u - 127u) << 20)) << 3);
  return __uint_as_float(f | (hi & 0x80000000u));
}

// A positive normal float as a double, exactly, by moving its bits.
__device__ __forceinline__ double float_to_double_bits(float f) {
  const unsigned u = __float_as_uint(f);
  return __hiloint2double((int)((u >> 3) + ((1023u - 127u) << 20)), (int)(u << 29));
}

// 1/sqrt(x) for x > 0 (in the range above): single-precision hardware
// estimate of the truncated argument (~1e-6), then one third-order Householder
// correction y <- y (1 + e/2 + 3e^2/8), e = 1 - x y^2 (error ~ e^3, below the
// FP64 rounding).
__device__ __forceinline__ double rsqrt_d(double x) {
  const double y = float_to_double_bits(rsqrtf(abs_to_float_bits(x)));
  const double e = fma(-x * y, y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}

// 1/x for |x| in the range above: estimate from the truncated |x|, sign put
// back by bits, then y <- y (1 + e + e^2), e = 1 - x y.
__device__ __forceinline__ double rcp_d(double x) {
  const double a = float_to_double_bits(__frcp_rn(abs_to_float_bits(x)));
  const double y = __hiloint2double(__double2hiint(a) | (__double2hiint(x) & (int)0x80000000),
                                    __double2loint(a));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// A double is finite when its exponent field is not all ones: tested on the
// high word with integer instructions, off the FP64 pipe.
__device__ __forceinline__ bool finite_d(double a) {
  return (__double2hiint(a) & 0x7ff00000) != 0x7ff00000;
}

// A big body's changeover radius and the constants the pair weight takes
// from it (rc^2, 0.01 rc^2, 0.1 rc, 1/(0.9 rc), as the kick's staging had
// computed them per block), so that the kick only loads them.
__device__ __forceinline__ void set_rcrit(const Dev& d, int b, double rc) {
  d.brc[b] = rc;
  d.brc4[b] = rc * rc;
  d.brc4[(size_t)d.NB + b] = 0.01 * (rc * rc);
  d.brc4[2 * (size_t)d.NB + b] = 0.1 * rc;
  d.brc4[3 * (size_t)d.NB + b] = (rc > 0.0) ? 1.0 / (0.9 * rc) : 0.0;
}

// A body removed from the integration (Sec. 3.5).  Detection also runs on
// a Dev without bodies' status (the no-alloc entry), where nobody is removed.
__device__ __forceinline__ bool removed(const Dev& d, int j) {
  return d.stat != nullptr && d.stat[j] != 0;
}

// Jump displacement (h/2) P / m0 of the step's democratic-heliocentric split
// (Sec. 2.1.3: momentum of massive bodies only).  Every kernel that applies
// the same jump evaluates this same expression, so a big body's staged
// position and its own update agree bit for bit.
// jump_frac is the jump's length in units of the system's step h.
__device__ __forceinline__ void jump_vec(const double* P, const SysDev& S, double jump_frac,
                                         double* dj) {
  const double c = (jump_frac * S.h) * S.inv_mu0;
  dj[0] = c * P[0];
  dj[1] = c * P[1];
  dj[2] = c * P[2];
}

}  // namespace mx
