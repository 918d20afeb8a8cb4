/*
 * mx.h -- C ABI of the GB300 (sm_103a) hybrid symplectic hot path.
 *
 * The library advances planetary systems with the hybrid symplectic step that
 * Mercury+ parallelises (arXiv 2601.16791, Sec. 2): a kick with forces from the
 * massive ("big") bodies weighted by the changeover function K (Sec. 2.1.3,
 * mfo_drct listing) plus gas drag on the planetesimals (Sec. 3.1, Eqs. 1-7),
 * a jump of all heliocentric positions by the massive bodies' momentum
 * (Sec. 2.1.3, the massive-body momentum loops), a Kepler drift of every body
 * (Sec. 2: the WHFast Kepler part, here universal variables), detection of
 * close encounters (Sec. 2.1.2, mce_snif listing), and Bulirsch-Stoer
 * integration of the encounter groups (Sec. 2: mdt_bs2).
 *
 * Conventions shared by every entry point:
 *  - Units: AU, day, solar mass.  Gravity enters as mu = G*m.
 *  - "6xN" buffers are structure-of-arrays float64: x[N], y[N], z[N], vx[N],
 *    vy[N], vz[N] back to back; big (massive) bodies come first.
 *  - dev_* arguments are device pointers owned by the caller (for instance
 *    torch tensors on the system's device); host_* or unprefixed pointers are
 *    host memory owned by the caller.  The library never frees caller memory.
 *  - Every call is ordered on the CUDA stream given to mx_init_system.  Calls
 *    that return host values synchronise that stream before returning.
 *  - No call aborts, traps or waits without a bound.  Device-side failures set
 *    bits of a status word that the next synchronising call turns into the
 *    returned mx_status.  On MX_ERR_ARG nothing was changed.
 *  - mx_last_error() gives a one-line description of the last failure on the
 *    calling thread.
 */
#ifndef MX_H
#define MX_H
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MX_OK = 0,
  MX_ERR_ARG = 1,                 /* bad argument; state unchanged */
  MX_ERR_CUDA = 2,                /* a CUDA runtime call failed */
  MX_ERR_OOM = 3,                 /* device allocation failed */
  MX_ERR_KEPLER_NOCONV = 4,       /* Kepler solve hit its iteration cap */
  MX_ERR_BS_NOCONV = 5,           /* Bulirsch-Stoer hit its sub-step cap */
  MX_ERR_PAIR_OVERFLOW = 6,       /* more encounter pairs than pair_cap */
  MX_ERR_NONFINITE = 7,           /* a non-finite position or velocity */
  MX_ERR_BARRIER_TIMEOUT = 8,     /* a bounded device-side wait gave up */
  MX_ERR_ENCOUNTER_IN_ADJOINT = 9,/* reserved (the adjoint now follows big-big
                                     encounters through their groups) */
  MX_ERR_GROUP_TOO_LARGE = 10     /* an encounter group exceeds MX_MAX_GROUP */
} mx_status;

#define MX_MAX_GROUP 16           /* bodies per Bulirsch-Stoer group */

typedef struct mx_system mx_system;   /* opaque; owns its device memory */

/* Gas disk (Sec. 3.1).  Sigma(R) = sigma1 (R/1AU)^-gamma exp[-(R/r_c)^(2-gamma)]
 * (Eq. 1 normalised at 1 AU), zero inside r_in; H/r = hr_1au (R/1AU)^flare;
 * temperature slope beta = 1 - 2 flare (Eq. 2 through c_s^2 ~ T). */
typedef struct {
  double sigma1_gcm2;   /* g/cm^2 at 1 AU */
  double gamma;         /* surface-density slope */
  double r_c_au;        /* characteristic radius; +inf for a pure power law */
  double r_in_au;       /* inner edge */
  double hr_1au;        /* aspect ratio at 1 AU */
  double flare;         /* aspect-ratio exponent */
  double gamma_c;       /* ratio of specific heats (Eq. 6), 7/5 */
  double mu_mol;        /* mean molecular weight (mean free path) */
  double sigma_mol_cm2; /* molecular cross-section */
  double cd_scale;      /* factor on C_D */
  int enabled;          /* 0: no drag */
  int cd_mode;          /* 0: Eq. 7 bracket to the power -1; 1: power -2 as printed */
  int disk_gravity;     /* 1: the disk's gravity on planetesimals (Eqs. 10-12): a radial
                           force per unit mass 2 pi G Sigma(R) S(gamma) (gamma != 1) or
                           2 pi G Sigma(R) r_in / R (gamma = 1), outward positive, along the
                           cylindrical radius, where R >= r_in; the adjoint differentiates
                           it (position, sigma1, gamma) */
  int reserved;         /* 0 */
} mx_gas;

typedef struct {
  double G;             /* AU^3 Msun^-1 d^-2 */
  double m_star;        /* Msun */
  double dt;            /* step h, days (may be negative) */
  double rcrit_hill;    /* changeover radius in Hill radii (3) */
  double bs_tol;        /* Bulirsch-Stoer tolerance (1e-12) */
  int kepler_max_iter;  /* Kepler iteration cap */
  int bs_max_sub;       /* Bulirsch-Stoer macro sub-step cap per group and step */
  int pair_cap;         /* encounter pair capacity */
  int eject_every;      /* ejection test (Sec. 3.5, see mx_check_ejections) after every step
                           whose global index (steps taken, counting it) is a multiple of
                           this; 0: never.  The same for every system of a batch. */
  mx_gas gas;
} mx_params;

/* Coordinates of mx_get_state / mx_set_state. */
#define MX_COORD_HELIO 0  /* heliocentric x and v */
#define MX_COORD_DH 1     /* heliocentric x, barycentric v (what the step works in) */

/*
 * mx_init_system -- copy one system to the device and prepare it.
 *  p          parameters (copied).
 *  n_big      massive bodies (>= 0); n_small massless planetesimals (>= 0).
 *  m_big      [n_big] masses in Msun (host).
 *  xv_helio   6xN heliocentric state (host), N = n_big + n_small.
 *  rp_km, rho_gcm3  [n_small] radius and density of each planetesimal (host);
 *             may be NULL when p->gas.enabled == 0.
 *  cuda_stream a cudaStream_t (NULL: the legacy default stream).
 *  out        receives the system.
 * Converts to democratic-heliocentric coordinates (barycentric velocities)
 * and sets each big body's changeover radius to rcrit_hill Hill radii from its
 * osculating semimajor axis (Sec. 2.1.3 mce_hill; Sec. 3.5 for gm).
 * Errors: MX_ERR_ARG, MX_ERR_OOM, MX_ERR_CUDA.
 */
mx_status mx_init_system(const mx_params* p, int n_big, int n_small, const double* m_big,
                         const double* xv_helio, const double* rp_km, const double* rho_gcm3,
                         void* cuda_stream, mx_system** out);

/*
 * mx_init_batch -- n_sys independent systems of uneven size in one mx_system
 * (the batched ensemble).  Arrays of n_sys entries: params[k], n_big[k],
 * n_small[k], and per-system host pointers m_big[k], xv_helio[k], rp_km[k],
 * rho_gcm3[k] with the layout of mx_init_system (rp_km / rho_gcm3 may be NULL
 * when no system has gas).  Every kernel of mx_step then runs once over all
 * systems: targets are cut into tiles that never span two systems, and the
 * step is replayed as CUDA graphs.  The integrator caps (kepler_max_iter,
 * bs_max_sub, bs_tol) and the pair capacity are taken from params[0]; dt,
 * masses and gas may differ per system.  The state of system k occupies
 * columns [off[k], off[k+1]) of the 6xN state (mx_batch_offsets).  Tile size
 * and order are autotuned per size bucket at set-up and cached
 * ($MX_AUTOTUNE_CACHE, default ~/.cache/mx/autotune.json; MX_AUTOTUNE=0 keeps
 * tiles of 256 in system order); the choice does not change any result.
 */
mx_status mx_init_batch(int n_sys, const mx_params* params, const int* n_big, const int* n_small,
                        const double* const* m_big, const double* const* xv_helio,
                        const double* const* rp_km, const double* const* rho_gcm3,
                        void* cuda_stream, mx_system** out);
/* offsets [n_sys + 1]: first body of each system in the 6xN state. */
mx_status mx_batch_offsets(mx_system* s, int* offsets);
mx_status mx_batch_size(mx_system* s, int* n_sys, int* n_total);
/* Energy and angular momentum of every system: E [n_sys], L3 [3 n_sys]. */
mx_status mx_energy_batch(mx_system* s, double* E, double* L3);
/* Tile size (targets per block: a multiple of 32 from 64 to 256) and order
 * (0: system order, 1: costliest tiles first) in use; mx_set_tiling overrides
 * the autotuner.  MX_ERR_ARG for another size or order. */
mx_status mx_tiling(mx_system* s, int* tile, int* order);
mx_status mx_set_tiling(mx_system* s, int tile, int order);

/*
 * Deferred planetesimals (an execution choice of this library; the paper has
 * no counterpart).  A planetesimal is massless (Sec. 3.4), so its own close
 * encounter changes no other body.  When its Bulirsch-Stoer group needs more
 * than a few macro sub-steps, the body leaves the step and the other bodies go
 * on.  One catch-up launch later replays its remaining steps from the big
 * bodies' recorded states with the same device arithmetic.  That happens when
 * `window` history slots have been recorded (a slot is a step, or the leading
 * half kick of an mx_step / mx_step_profiled call, so a window may span calls),
 * or earlier, before any call that reads or replaces the state, changes the
 * gas parameters or the branch mode, or reads the encounter log or pair list.
 * The state every such call sees is the one the direct path gives, bit for
 * bit.  Big-body groups are never deferred, nor are planetesimals of systems
 * with more than 64 big bodies (a replay sums every big body's gravity on one
 * lane, in the direct path's order).  Recording or replaying drag
 * branches (mx_kick_branches) turns deferral off.  A catch-up's device errors
 * are reported by the call that launched it.
 *
 * mx_set_defer_window: window = 0 keeps every body on the direct path;
 * 1 <= window <= the history length (*max_window of mx_defer_stats, at most
 * 64) sets the slots per catch-up.  Default: min(10, history length).
 * MX_ERR_ARG for a window outside that range.
 * mx_defer_stats: window in effect (0 when off), history length, bodies
 * deferred since creation, catch-up launches made (host pointers, each may
 * be NULL).
 */
mx_status mx_set_defer_window(mx_system* s, int window);
/*
 * mx_set_persistent -- run each interior step of mx_step (every step of a
 * call but its last; the leading half kick stays a launch of its own) as ONE
 * cooperative launch over all systems of the handle, captured in the step's
 * CUDA graph: the phases of the step (jump and drift, detection, groups,
 * Bulirsch-Stoer of every group, the kick with its own momentum) run in
 * turn, separated by grid barriers, on the same device functions and tiles
 * as the per-kernel step, so the state is the same bit for bit (spec:
 * the batched ensemble advances in one persistent launch per step; the
 * paper has no counterpart).  Applies to forward runs with deferral on and
 * no growth tracks, ejection schedule or recorded k branches; other steps
 * keep the per-kernel graphs.  on = 1 switches the tiling to 256 targets per
 * block if it was smaller (results do not depend on the tiling).
 *  spin_limit  polls a grid barrier waits for the other blocks before it
 *              gives up (< 0: the default, 2^24, about two seconds); a step
 *              whose barrier gave up returns MX_ERR_BARRIER_TIMEOUT (the
 *              launch still ends; the state is then that of a partial step).
 * Errors: MX_ERR_ARG, MX_ERR_CUDA (no resident grid).  Settles first.
 */
mx_status mx_set_persistent(mx_system* s, int on, long long spin_limit);

/* mx_catchup_work -- work the catch-ups have done since creation or the last
 * reset, in units of fixed algorithmic cost (host ops6[6]): [0] body-slots
 * replayed through jump, drift and the encounter test, [1] half kicks of one
 * body, [2] force evaluations of two-body Bulirsch-Stoer groups as the
 * one-try-at-a-time step search makes them (every row of each failed try,
 * rows up to the accepted one of the accepted try); [0..2] by the main
 * stream's catch-ups (MX_K_CATCHUP), [3..5] by the side stream's
 * (MX_K_CATCHUP_SIDE).  Waits for the side stream's last pass.  Groups of
 * three or more bodies are not counted.  reset != 0 zeroes the counters
 * after reading. */
mx_status mx_catchup_work(mx_system* s, long long* ops6, int reset);
mx_status mx_defer_stats(mx_system* s, int* window, int* max_window, long long* deferred,
                         long long* catchups);

/* Frees the system's device memory and graphs.  NULL is ignored. */
void mx_destroy(mx_system* s);

/*
 * mx_step -- advance n_steps hybrid steps (Sec. 2; step order: half kick,
 * half jump, drift, detection, Bulirsch-Stoer of encounter groups, half jump,
 * half kick).  Runs as CUDA graphs on the system's stream and synchronises
 * once at the end to read the status word.  n_steps >= 0; n_steps = 0 only
 * brings deferred planetesimals up to date (see mx_set_defer_window).  With
 * eject_every > 0 the ejection test of mx_check_ejections follows every step
 * on that schedule (the step then ends with its own half kick, and the next
 * one starts with a fresh half kick).
 */
mx_status mx_step(mx_system* s, int n_steps);

/* Kernels of one step, in launch order, for mx_step_profiled. */
#define MX_NKERN 10
#define MX_K_PREP 0       /* momentum + staged big positions: before a call's first and
                             last half kick, and before every kick of runs with growth
                             tracks or recorded/replayed k branches; the other kicks
                             compute them themselves */
#define MX_K_JUMP_KICK 1  /* jump + half kick(s): gravity and drag */
#define MX_K_JUMP_DRIFT 2 /* jump + Kepler drift */
#define MX_K_DETECT 3     /* encounter detection + compaction */
#define MX_K_SORT 4       /* pair-key sort */
#define MX_K_GROUPS 5     /* encounter groups */
#define MX_K_BS 6         /* Bulirsch-Stoer of the groups */
#define MX_K_CATCHUP 7    /* deferred planetesimals: window-end and settling catch-ups */
#define MX_K_CATCHUP_SIDE 8 /* carried planetesimals on the side stream (overlaps the steps) */
#define MX_K_EJECT 9      /* ejection test (steps on the eject_every schedule) */

/*
 * mx_step_profiled -- the same n_steps as mx_step, launched kernel by kernel
 * (no graph) with CUDA events around every launch on the system's stream.
 *  kernel_ms [MX_NKERN]  summed device time per kernel (host, may be NULL)
 *  launches  [MX_NKERN]  launches per kernel (host, may be NULL)
 *  total_ms              sum over the steps of each step's device time, from
 *                        before its first launch to after its last (a
 *                        window-end catch-up belongs to the step that ends
 *                        the window) (host, may be NULL)
 * Synchronises once at the end.  n_steps = 0 only runs (and times) the
 * pending catch-up of deferred planetesimals, if any.  Side-stream launches
 * (MX_K_CATCHUP_SIDE) are counted in the call during which they complete.
 */
mx_status mx_step_profiled(mx_system* s, int n_steps, double* kernel_ms, int* launches,
                           double* total_ms);

/*
 * mx_step_timed -- the CUDA graphs of mx_step, in variants with an event
 * between kernels, one step at a time, with a cache flush: before every step
 * the device buffer dev_flush (flush_bytes bytes, e.g. more than the L2 cache;
 * caller-owned) is overwritten on the system's stream, outside the steps'
 * timed spans; after every step the host waits for it and reads its events.
 * Outputs as mx_step_profiled.  flush_bytes = 0 means no flush; n_steps = 0
 * runs the pending catch-up, timed.  With kernel_ms and launches both NULL
 * the production graphs run unchanged, with events only around each step
 * (the event nodes between kernels add about 7% to a step), and only
 * total_ms is written.
 */
mx_status mx_step_timed(mx_system* s, int n_steps, void* dev_flush, size_t flush_bytes,
                        double* kernel_ms, int* launches, double* total_ms);

/*
 * mx_step_wall -- n_steps steps through the production CUDA graphs of
 * mx_step, then the catch-up that brings every deferred planetesimal to the
 * last step, all enqueued with no host wait in between; before every step the
 * device buffer dev_flush (flush_bytes bytes, caller-owned; 0 = no flush) is
 * overwritten on the system's stream.
 *  wall_ms   device time from before the first flush to after the catch-up
 *            (the side stream's work is joined into it), host, required
 *  flush_ms  if not NULL: the same n_steps flushes enqueued alone after the
 *            span, with nothing else in flight, timed the same way
 * Anything pending from earlier calls is settled before the span starts.
 * Synchronises before returning.  n_steps >= 1.
 */
mx_status mx_step_wall(mx_system* s, int n_steps, void* dev_flush, size_t flush_bytes,
                       double* wall_ms, double* flush_ms);

/* Encounter pairs found by the last step (sorted by (i, j), i big, body
 * indices), copied to host_pairs [2*cap]; *n_pairs gets the full count. */
mx_status mx_last_encounters(mx_system* s, int* host_pairs, int cap, int* n_pairs);

/*
 * mx_accel -- kick acceleration at the current state into dev_acc (3xN):
 * the K-weighted gravity of the big bodies (Sec. 2.1.3, rectangular loop)
 * plus, on planetesimals, the gas drag of mx_gas_drag.
 */
mx_status mx_accel(mx_system* s, double* dev_acc);

/*
 * mx_gas_drag -- gas-drag acceleration of every planetesimal at the current
 * state into dev_acc (3 x n_small): Eq. 3 with C_D from Eq. 7, rho_g from
 * Eq. 4, sub-Keplerian gas speed from Eqs. 5-6, relative to the body's
 * heliocentric velocity.  Zeros when the gas is disabled.
 */
mx_status mx_gas_drag(mx_system* s, double* dev_acc);

/*
 * mx_detect_encounters -- close-encounter test (Sec. 2.1.2, mce_snif) between
 * the states dev_xv0 (start of the step) and dev_xv1 (end), both 6xN DH
 * device buffers.  A pair (big i, body j) is flagged when the smallest of the
 * squared separations at the two ends and the minimum of their cubic Hermite
 * interpolant over the step is at most max(rcrit_i, rcrit_j)^2.
 *  dev_flags  [N] bytes, 1 for bodies in a flagged pair (may be NULL).
 *  dev_pairs  [2*cap] ints, (i, j) pairs sorted by (i, j) (may be NULL).
 *  n_pairs    host; receives the number of flagged pairs (also when > cap,
 *             which returns MX_ERR_PAIR_OVERFLOW).
 */
mx_status mx_detect_encounters(mx_system* s, const double* dev_xv0, const double* dev_xv1,
                               unsigned char* dev_flags, int* dev_pairs, int cap, int* n_pairs);

/*
 * mx_detect_encounters_noalloc -- the encounter test of mx_detect_encounters
 * for callers that cannot allocate device memory (the paper has no
 * counterpart; it is a library-usage variant).  Some callers cannot call
 * cudaMalloc -- a host application that owns all of the GPU's memory through
 * its own pool, or a latency-critical loop that cannot take the device-wide
 * synchronisation an allocation may cause -- so this call needs no mx_system
 * and allocates nothing: its working memory is a fixed array in the
 * library's static device memory (about 0.7 MB, held on every GPU that loads
 * the library until the process exits).
 *  p          parameters; only G, m_star and dt are used.
 *  n_big, n   big bodies and all bodies (n <= MX_NOALLOC_MAX_BODIES).
 *  dev_rcrit  [n] changeover radius per body (0 for planetesimals), device.
 *  dev_xv0, dev_xv1  6xn DH states at the start and end of the step, device.
 *  dev_flags  [n] bytes, set to 1 for bodies in a flagged pair (required).
 *  dev_pairs  [2*cap] ints, (i, j) sorted by (i, j) (may be NULL if cap = 0).
 *  n_pairs    host; receives the number of flagged pairs.
 *  cuda_stream  stream to run on (NULL: legacy default stream).
 * The first call on a device, made with that device current, looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  The address is kept for the life of the process: a
 * cudaDeviceReset (or any reset of the device's primary context) unloads the
 * array, and the kept address is then stale, so after such a reset this
 * entry point must not be called again on that device in the same process.
 * Every call shares the one array, which keeps the last call's contents; the
 * call clears what must start at zero.  Calls that overlap on the GPU (other
 * threads or streams) race on the array.
 * Errors: MX_ERR_ARG (including n above the limit), MX_ERR_CUDA (also when a
 * CUDA error was already pending at entry: it is left pending and nothing
 * runs), MX_ERR_PAIR_OVERFLOW when more than cap or MX_NOALLOC_MAX_PAIRS
 * pairs (n_pairs still receives the full count, and with at most
 * MX_NOALLOC_MAX_PAIRS pairs the first cap of the sorted list are written).
 * Synchronises the stream before returning.
 */
#define MX_NOALLOC_MAX_BODIES (1 << 21)
#define MX_NOALLOC_MAX_PAIRS (1 << 16)
mx_status mx_detect_encounters_noalloc(const mx_params* p, int n_big, int n,
                                       const double* dev_rcrit, const double* dev_xv0,
                                       const double* dev_xv1, unsigned char* dev_flags,
                                       int* dev_pairs, int cap, int* n_pairs, void* cuda_stream);

/* mx_kepler_drift -- Kepler drift by h of the N bodies of dev_xv (6xN, in
 * place) about mu0 = G m_star, universal variables (Sec. 2). */
mx_status mx_kepler_drift(mx_system* s, double* dev_xv, double h);

/* mx_energy -- energy and angular momentum of the massive bodies, DH form
 * (kinetic sum_i |p_i|^2/2m_i + |sum p|^2/2m0, full Newtonian potential;
 * Sec. 2.1.3: the energy loop runs over massive bodies only).  Host outputs. */
mx_status mx_energy(mx_system* s, double* E, double* L3);

/* State transfer.  coords: MX_COORD_HELIO or MX_COORD_DH.  step: the number
 * of steps taken so far (may be NULL on get). */
mx_status mx_get_state(mx_system* s, double* xv_host, int coords, long long* step);
mx_status mx_set_state(mx_system* s, const double* xv_host, int coords, long long step);
/* Device-to-device copies of the DH state (6xN), ordered on the stream. */
mx_status mx_get_state_device(mx_system* s, double* dev_xv);
mx_status mx_set_state_device(mx_system* s, const double* dev_xv);

/* ------------------------------------------------------------------------
 * Differentiation: a hand-written adjoint (reverse mode) of the hybrid step.
 * The loss provided (mx_loss_semimajor) is the weighted squared change of the
 * planetesimals' semimajor axes; its gradient is taken with respect to the
 * initial heliocentric state and to the gas parameters (Sigma normalisation,
 * Sigma slope, C_D factor).  Planetesimals that met a big body either carry
 * weight 0 (they are massless, so nothing else depends on them and the
 * encounter groups are skipped), or are differentiated through their
 * Bulirsch-Stoer groups (mx_adjoint_encounters).  Big bodies that meet form
 * groups of their own, which the adjoint always differentiates when asked to
 * (modes 1 and 2 of mx_adjoint_encounters).  The disk's gravity (Eqs. 10-12), when on, is
 * differentiated too: with respect to position, sigma1 and gamma (through
 * Sigma and, for gamma != 1, through the series S(gamma)); at gamma = 1 the
 * force is the edge form of Eq. 12, and its gamma derivative is the one of
 * that form.  Systems with growth or the ejection test have no adjoint.
 * The Python layer (paper_2601_16791_gb300.autograd) drives checkpointing:
 * the state is stored every k steps and each segment is recomputed before
 * its reverse sweep.
 * ------------------------------------------------------------------------ */

/* Gas parameters of system k (Sec. 3.1): Sigma at 1 AU, slope gamma (Eq. 1),
 * and the factor on C_D (Eq. 7).  Takes effect at the next launch. */
mx_status mx_set_gas_params(mx_system* s, int k, double sigma1_gcm2, double gamma,
                            double cd_scale);

/* The k switch of Eq. 7 (k = 0.4 below Re = 1e5, 0.2 above) is a jump; for
 * finite differences and for the adjoint's recomputation the branch taken at
 * each (half kick, planetesimal) can be recorded and replayed.
 * mode 0: off; 1: record (clears, room for max_kicks half kicks, counted from
 * step 0 as 2 per step); 2: replay the recording. */
mx_status mx_kick_branches(mx_system* s, int mode, long long max_kicks);

/* Encounter log since the last reset: dev_ever [N] bytes (device, may be
 * NULL) = 1 for every body flagged in any step; *n_big_big = flagged big-big
 * pairs summed over steps.  reset != 0 clears the log afterwards. */
mx_status mx_encounter_log(mx_system* s, unsigned char* dev_ever, long long* n_big_big,
                           int reset);

/* Sets the step counter (used to index recorded branches). */
mx_status mx_set_step_index(mx_system* s, long long step);

/* Loss at the current state against the initial heliocentric state
 * dev_xv_helio0 (6xN, device): L[k] = sum over bodies j of system k of
 * w[j] (a_final,j - a_initial,j)^2, a = 1/(2/r - v^2/gm) (gm = G m0 for
 * planetesimals, G (m0 + m) for big bodies; Sec. 3.5).  dev_w [N] device.
 * Writes L [n_sys] (host), dev_seed_final (6xN device: dL/d of the current DH
 * state) and dev_seed_init (6xN device: dL/d of the initial heliocentric
 * state through a_initial). */
mx_status mx_loss_semimajor(mx_system* s, const double* dev_xv_helio0, const double* dev_w,
                            double* L, double* dev_seed_final, double* dev_seed_init);

/* Reverse of one hybrid step.  dev_state_k: 6xN DH state at the start of
 * step step_k (device); dev_lambda: 6xN cotangent of the state at the end of
 * the step, replaced by the cotangent at its start; dev_dparams [3 n_sys]
 * (device) accumulates d/d(sigma1, gamma, cd_scale) of each system.
 * With encounter groups on (mx_adjoint_encounters), a planetesimal that meets
 * a big body in the step is differentiated through its Bulirsch-Stoer
 * integration (Sec. 2: the recomputed group's accepted sub-steps and
 * extrapolation rows held fixed); with them off it is differentiated as if
 * drifted, which is exact when its cotangent is zero (a loss that leaves it
 * out; it is massless, so nothing else depends on it).  Big bodies that meet
 * are differentiated through their own groups in modes 1 and 2.
 * The groups' record (128 accepted sub-steps reserved per group) grows to
 * what the step needs; the step waits once on the device to size it.
 * Errors: MX_ERR_ARG; MX_ERR_OOM when the record cannot grow;
 * MX_ERR_BS_NOCONV when a group needs more than 128 accepted sub-steps or
 * hits the sub-step cap; the step's own errors (MX_ERR_PAIR_OVERFLOW,
 * MX_ERR_GROUP_TOO_LARGE, ...).  On an error in the recomputation up to the
 * groups' plan, dev_lambda and dev_dparams are unchanged. */
mx_status mx_adjoint_step(mx_system* s, const double* dev_state_k, long long step_k,
                          double* dev_lambda, double* dev_dparams);

/* The pre-drift state of the last step mx_step took (Sec. 2.1: the state the
 * Kepler drift starts from): heliocentric positions after the first jump and
 * barycentric velocities after the first half kick, 6xN into dev_xv (device).
 * MX_ERR_ARG when the last step-taking call was not mx_step, or deferral was
 * on in it for a system that can defer (a deferred planetesimal is drifted by
 * the catch-up instead; recording or replaying drag branches turns deferral
 * off, and systems with more than 64 big bodies never defer, see
 * mx_set_defer_window). */
mx_status mx_predrift_state(mx_system* s, double* dev_xv);

/* mx_adjoint_step with the step's pre-drift state from the forward run
 * (mx_predrift_state after the mx_step(1) that started from dev_state_k),
 * read only, instead of recomputing the first half kick and jump: one pass
 * over the (target, big body) pairs less.  The same derivative; it follows
 * the forward's values where the recomputation would differ from them by
 * rounding. */
mx_status mx_adjoint_step_predrift(mx_system* s, const double* dev_state_k,
                                   const double* dev_predrift_k, long long step_k,
                                   double* dev_lambda, double* dev_dparams);

/* Which of the step's encounter groups mx_adjoint_step integrates and
 * differentiates.  The groups are the step's own (rebuilt from the
 * recomputed endpoints): groups of big bodies joined by big-big encounters,
 * and test-particle groups, a planetesimal with the whole big groups of the
 * big bodies it meets.
 *   on = 1 (the default): every group;
 *   on = 2: the groups of big bodies only, for a loss that gives the
 *           planetesimals that met a big body weight 0 (they are massless,
 *           so nothing else depends on them);
 *   on = 0: none; the caller asserts that no big bodies met in the step
 *           (mx_encounter_log), or the big bodies' derivative is wrong. */
mx_status mx_adjoint_encounters(mx_system* s, int on);

/* Memory for the reverse of two-body encounter groups.  The adjoint's
 * recomputation keeps the Stoermer sub-steps of each accepted macro sub-step
 * of a two-body group (26,112 bytes a slot; default 16,384 slots, 428 MB,
 * allocated at the first mx_adjoint_step), so that the reverse reads them
 * back instead of integrating the sub-step again.  Records beyond the pool
 * are recomputed; the result is the same to the bit either way.  slots = 0
 * keeps none; at most 2^20.  The pool in place is freed (after the stream's
 * work) and the new one allocated at the next adjoint step. */
mx_status mx_adjoint_store(mx_system* s, long long slots);

/* Merged reverse of consecutive steps.  Both half kicks of the hybrid step
 * (Sec. 2.1) sit between a step's last drift and the next step's first at the
 * same positions, and the gravity part of a half kick's reverse is linear in
 * its cotangent.  With on = 1, mx_adjoint_step of step k takes the drag part
 * of its first half kick's reverse and leaves the pair pass pending: its
 * cotangent and positions (2 x 3 x N doubles) are kept in the system, and the
 * next call, for step k - 1 on the same dev_lambda, takes it in the pass of
 * that step's last half kick.  That saves one pass over the (target, big body)
 * pairs a step, most of an adjoint step with many big bodies.  Until then,
 * the position rows of that dev_lambda lack the pending term, and the buffer
 * must stay allocated: the term is added into it later (mx_destroy drops a
 * pending term without touching it).
 * mx_adjoint_init, mx_adjoint_flush, mx_adjoint_merge(s, 0), or an
 * mx_adjoint_step of any other step or cotangent adds it first.  The shared
 * pass runs at the recomputed positions of step k - 1's last half kick, which
 * are step k's starting positions for every body the mode integrates
 * faithfully: every body in mode 1; in mode 2 all but the planetesimals that
 * met a big body, and in mode 0 all but the members of encounter groups,
 * whose cotangents the mode's loss must leave at zero anyway
 * (mx_adjoint_encounters).  The results then agree with the unmerged reverse
 * to rounding; the order of every sum stays fixed.  Default 0. */
mx_status mx_adjoint_merge(mx_system* s, int on);

/* Adds a merged reverse's pending pair pass (mx_adjoint_merge) to the
 * cotangent it belongs to, so that buffer holds the cotangent at the start
 * of the step it was last given to.  No-op without one.  Synchronises. */
mx_status mx_adjoint_flush(mx_system* s);

/* Reverse of the set-up transform: cotangent of the initial DH state ->
 * cotangent of the initial heliocentric state (6xN device buffers).  Adds a
 * pending pair pass (mx_adjoint_merge) to its cotangent first. */
mx_status mx_adjoint_init(mx_system* s, const double* dev_lambda, double* dev_grad_helio);

/* ------------------------------------------------------------------------
 * Ejection and orbital elements (Sec. 3.5).  A body is ejected when its
 * osculating heliocentric orbit is unbound, e >= 1, with gm = G (m0 + m) for
 * a massive body and G m0 for a planetesimal.  An ejected body is removed
 * from the integration (its status becomes MX_STAT_EJECTED): it keeps the
 * state it had at the test and takes no further part in the kick, the jump,
 * the drift or the encounter search; a massive one also loses its mass
 * (mu = 0), so it no longer pulls on the others and drops out of the momentum
 * P and of mx_energy.  mx_accel gives it zero acceleration.  Systems with
 * removed bodies, or with eject_every > 0, have no adjoint (MX_ERR_ARG).
 * ------------------------------------------------------------------------ */
#define MX_STAT_EJECTED (-3)

/* Runs the ejection test now on the current state (heliocentric velocities
 * v_b + P/m0 with P the momentum of that state); *n_removed (host, may be
 * NULL) gets the number of bodies it removed, over all systems. */
mx_status mx_check_ejections(mx_system* s, int* n_removed);

/* host_stat [N] (host, may be NULL): 0 for a body in the integration,
 * MX_STAT_EJECTED for a removed one.  n_removed [n_sys] (host, may be NULL):
 * removed bodies of each system (the count of status < 0 over its bodies). */
mx_status mx_body_status(mx_system* s, signed char* host_stat, int* n_removed);

/* Osculating heliocentric elements of every body (removed ones: of the state
 * they keep) into dev_el (6xN device buffer, caller-owned), rows: q [AU], e,
 * i [rad], longitude of pericentre, longitude of the node, mean anomaly
 * (e < 1: in [0, 2 pi); e > 1: e sinh F - F; e = 1: D + D^3/3 with D the
 * tangent of half the true anomaly).  Node 0 for an orbit in the reference
 * plane; angles in [0, 2 pi). */
mx_status mx_elements(mx_system* s, double* dev_el);

/* ------------------------------------------------------------------------
 * Planet growth and gas gaps (Sec. 3.3, Eqs. 13-16; Sec. 3.1, Eqs. 8-9 and
 * the dens_factor listing).  A growing massive body follows
 *   M(t) = m0 + (e/(e-1)) (mc - m0) (1 - exp(-t/tau_c))      t <= tau_c (Eq. 13)
 *   M(t) = mc + (mf - mc) (1 - exp(-(t - tau_c)/tau_g))      t >  tau_c (Eq. 15)
 * with t = (global step index) x dt at the start of each step (applied by
 * the step's first kick launch, MX_K_PREP); the mass is held for the step.  Its changeover radius follows the mass (rcrit_hill Hill
 * radii, R_H = a (M/3 m0)^(1/3) from the osculating a), and once t > tau_c it
 * opens a gap: planetesimals whose cylindrical distance lies strictly within
 * gap_c R_H of the body's cylindrical distance (at kick time) see the gas
 * density times exp(-(t - tau_c)/tau_g); with overlapping gaps the body with
 * the highest index wins.  The radius (Eq. 14 before tau_c with c_s at the
 * body's cylindrical distance, k1 = 1, k2 = 1/4; Eq. 16 after it, R_c from
 * Eq. 14 at mass mc on the current orbit) is not used by the step; mx_planets
 * computes it for the current state at t = (steps taken) x dt.
 * With growth on, every step ends with its own half kick (the next one starts
 * with the new masses), and there is no adjoint.  Deferred planetesimals
 * replay each step with the masses, changeover radii and gaps it had.
 * ------------------------------------------------------------------------ */
typedef struct {
  double m0, mc, mf;    /* Msun: at t = 0, at t = tau_c, for t -> inf */
  double tau_c, tau_g;  /* days, > 0 */
  double delta_r;       /* AU: radius lost after tau_c (Eq. 16) */
  int grows;            /* 0: the body keeps its mass (and has no gap) */
  int reserved;         /* 0 */
} mx_growth;

/* Growth tracks of system sys (0 for a single system): g [n_big of that
 * system] (host, copied), gap_c the gap half-width in Hill radii (Eq. 8: 4).
 * Takes effect at the next step.  MX_ERR_ARG for a bad index, non-positive
 * times, negative masses, dt <= 0 with a growing body, or gap_c < 0. */
mx_status mx_set_growth(mx_system* s, int sys, const mx_growth* g, double gap_c);

/* Masses [Msun] and radii [AU] of the massive bodies of every system, in
 * system order (host arrays of the total number of massive bodies, may be
 * NULL).  Radius 0 for a body that does not grow. */
mx_status mx_planets(mx_system* s, double* m_host, double* r_host);

/* Sizes of the system. */
mx_status mx_sizes(mx_system* s, int* n_big, int* n_small);

/* One-line description of the last error on this thread ("" if none). */
const char* mx_last_error(void);

/*
 * mx_fp64_peak -- measures this GPU's FP64 fused-multiply-add rate: every SM
 * runs independent FMA chains for about ms_target milliseconds; *tflops gets
 * 2 * FMAs / second / 1e12.  Used for the roofline denominator.
 */
mx_status mx_fp64_peak(void* cuda_stream, double ms_target, double* tflops);

#ifdef __cplusplus
}
#endif
#endif
