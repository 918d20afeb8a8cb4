/*
 * mx_oracle.h -- plain FP64 CPU oracle for the hybrid symplectic hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline leg (and its --impl reference arm) may load this
 * library.  It shares no code, header, table or constant with the CUDA path
 * in paper_2601_16791_gb300/csrc; both are written from the paper
 * (arXiv 2601.16791, "Mercury-Arxes") independently.
 *
 * Units: AU, day, solar mass.  Masses enter as G-scaled mu = G*m
 * (the paper's Sec. 2.1.3 force loop multiplies by m(i) with no G).
 * Arrays are structure-of-arrays: a "6xN" buffer holds x[N], y[N], z[N],
 * vx[N], vy[N], vz[N] back to back.  Big (massive) bodies come first.
 * In the democratic-heliocentric (DH) coordinates that the step works in,
 * x is heliocentric position and v is barycentric velocity.
 *
 * Every function returns 0 on success or a positive ORC_ERR_* code.
 */
#ifndef MX_ORACLE_H
#define MX_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_KEPLER_NOCONV = 2,
  ORC_ERR_BS_NOCONV = 3,
  ORC_ERR_PAIR_OVERFLOW = 4,
  ORC_ERR_NONFINITE = 5
};

typedef struct {
  double sigma1_gcm2;   /* surface density at 1 AU [g/cm^2] (Eq. 1 normalised at 1 AU) */
  double gamma;         /* surface-density slope (Eq. 1) */
  double r_c_au;        /* characteristic radius R_C [AU]; +inf = pure power law */
  double r_in_au;       /* inner edge R_in [AU]: no gas inward (Sec. 3.1) */
  double hr_1au;        /* aspect ratio H/r at 1 AU */
  double flare;         /* H/r grows as r^flare; temperature slope beta = 1 - 2*flare */
  double gamma_c;       /* ratio of specific heats, 7/5 (Eq. 6) */
  double mu_mol;        /* mean molecular weight, for the mean free path */
  double sigma_mol_cm2; /* molecular cross-section [cm^2] */
  double cd_scale;      /* multiplies C_D (differentiable drag-coefficient factor) */
  int enabled;          /* 0 = no gas drag */
  int cd_mode;          /* 0: bracket of Eq. 7 to the power -1; 1: power -2 as printed */
  int disk_gravity;     /* 1: add the disk's gravity on planetesimals (Eqs. 10-12) */
  int reserved;
} orc_gas;

typedef struct {
  double G;             /* gravitational constant [AU^3 Msun^-1 d^-2] */
  double m_star;        /* central mass [Msun] */
  double dt;            /* step h [d] */
  double rcrit_hill;    /* changeover radius in Hill radii */
  double bs_tol;        /* Bulirsch-Stoer relative tolerance */
  int kepler_max_iter;  /* iteration cap of the universal Kepler solve */
  int bs_max_sub;       /* cap on BS macro sub-steps per group and step */
  int pair_cap;         /* capacity of the encounter pair list */
  int eject_every;      /* ejection test (Sec. 3.5) after every step whose global index
                           k + 1 is a multiple of this; 0: never */
  orc_gas gas;
} orc_params;

/* Growth track of one massive body (Sec. 3.3): core growth to mc at t =
 * tau_c (Eq. 13), runaway gas accretion towards mf with e-folding time tau_g
 * (Eq. 15); the radius of Eq. 14 before tau_c and Eq. 16 after it. */
typedef struct {
  double m0, mc, mf;    /* masses [Msun] at t = 0, t = tau_c, t -> inf */
  double tau_c, tau_g;  /* [d] */
  double delta_r;       /* radius lost in the collapse after tau_c (Eq. 16) [AU] */
  int grows;            /* 0: the body keeps its mass */
  int reserved;
} orc_growth;

void orc_set_threads(int n);

/* Changeover function K(s) for changeover radius rc (Sec. 2.1.3 listing). */
double orc_changeover(double s, double rc);
/* K(s)/s^3 written in terms of s^2, the factor the kick multiplies by mu*dx. */
double orc_k_over_s3(double s2, double rc);

/* Heliocentric (x, v_h) -> DH (x, v_b); mu = G*m; rcrit = rcrit_hill * R_Hill. */
int orc_init(const orc_params* p, int nbig, int nsmall, const double* m_big,
             const double* xv_helio, double* xv_dh, double* mu, double* rcrit);
/* DH -> heliocentric. */
int orc_readout(const orc_params* p, int nbig, int nsmall, const double* mu,
                const double* xv_dh, double* xv_helio);

/* K-weighted gravity on every body from the big bodies, acc is 3xN.
 * triangular=0: the paper's rectangular gather loop; 1: its serial
 * triangular loop with Newton's third law. */
int orc_accel_grav(int nbig, int n, const double* xv, const double* mu,
                   const double* rcrit, double* acc, int triangular);
/* P = sum over massive bodies of mu_i v_i (G-scaled momentum). */
int orc_momentum(int nbig, int n, const double* xv, const double* mu, double* P3);

/* Gas-drag acceleration on every small body (3 x nsmall), Eqs. 1, 3-7. */
int orc_gas_drag(const orc_params* p, int nbig, int nsmall, const double* xv,
                 const double* mu, const double* rp_km, const double* rhop,
                 double* acc_small);
/* As orc_gas_drag with gaps (Sec. 3.1 listing, Eqs. 8-9): gap_w [nbig]
 * half-widths (0: none) and gap_f [nbig] density factors, centred on each
 * massive body's cylindrical distance in xv (both NULL: no gaps). */
int orc_gas_drag_gap(const orc_params* p, int nbig, int nsmall, const double* xv,
                     const double* mu, const double* rp_km, const double* rhop,
                     const double* gap_w, const double* gap_f, double* acc_small);
/* Disk quantities at cylindrical radius R [AU]:
 * out = {Sigma [g/cm^2], rho_g [g/cm^3], H [AU], c_s [AU/d], v_k [AU/d],
 *        eta, v_g [AU/d], H/r}. */
int orc_gas_state(const orc_params* p, double R, double* out8);
/* The series S(gamma) of Eq. 10 (gamma != 1): F_DG = 2 pi G Sigma(r) S(gamma). */
double orc_dg_series(double gamma);
/* dS/dgamma of the same series (the forward derivative of the disk's gravity
 * with respect to gamma). */
double orc_dg_series_dgamma(double gamma);
/* Disk-gravity acceleration (Eqs. 10-12) on a planetesimal at x3 (AU/d^2). */
int orc_disk_gravity(const orc_params* p, const double* x3, double* acc3);
/* Drag coefficient of Eq. 7 (k = 0.4 below Re = 1e5, 0.2 from 1e5 up). */
double orc_drag_cd(double Re, double Ma, int cd_mode);
/* Drag acceleration of one small body with given heliocentric x and v_h. */
int orc_drag_one(const orc_params* p, const double* x3, const double* vh3,
                 double rp_km, double rhop, double* acc3, double* re_ma2);

/* Stumpff functions c0..c3 at z. */
void orc_stumpff(double z, double* c4);
/* Kepler drift of n bodies by h about mu0 = G*m_star (universal variables).
 * iters_max receives the largest iteration count used. */
int orc_drift(const orc_params* p, int n, double* xv, double h, int* iters_max);

/* Minimum over [0,1] of the cubic Hermite interpolant of the squared
 * distance (endpoint values d0, d1, time slopes d0t, d1t over step h);
 * +inf unless the separation shrinks at the start and grows at the end. */
double orc_hermite_d2min(double d0, double d1, double d0t, double d1t, double h);
/* Encounter detection over big x body pairs between the pre-drift (xv0) and
 * post-drift (xv1) states.  flags[n] = 1 for bodies in a flagged pair;
 * pairs = (i, j) int pairs sorted by (i, j), at most cap. */
int orc_detect(const orc_params* p, int nbig, int n, const double* xv0,
               const double* xv1, const double* rcrit, unsigned char* flags,
               int* pairs, int cap, int* npairs);

/* Encounter groups of one step (reading of Sec. 2's single BS call over the
 * encounter bodies): bigs joined by flagged big-big pairs form big groups;
 * each flagged planetesimal forms a group of the whole big groups of the
 * bigs it meets, then itself, and only it is written back.  pairs: npairs
 * (i, j) with i < nbig, i < j < nbig + nsmall.  Output: members[] back to
 * back (bigs ascending, then the planetesimal), offsets[ngroups + 1],
 * write_from[ngroups] (index within the group of the first member written).
 * Big groups (two or more bigs) come first, then the planetesimals' groups
 * in planetesimal order.  ORC_ERR_PAIR_OVERFLOW if the groups exceed
 * cap_groups or cap_members (ngroups still set). */
int orc_build_groups(int nbig, int nsmall, int npairs, const int* pairs,
                     int cap_groups, int cap_members, int* members,
                     int* offsets, int* write_from, int* ngroups);

/* Bulirsch-Stoer integration over h of a group of nb bodies (6 x nb SoA
 * state, modified in place) under the star plus (1-K)-weighted pair forces
 * from the group's massive members. nsub receives the macro sub-steps. */
int orc_bs_group(const orc_params* p, int nb, const double* mu,
                 const double* rcrit, double* xv, double h, int* nsub);

/* nsteps hybrid steps of the full system, in place (DH state), the first
 * one with global index 0 (with p->eject_every > 0 the ejection test of
 * orc_step_ex runs on its schedule; removals are not returned).  Masses are
 * fixed (orc_step_ex follows growth tracks).
 * ever_flag[n] (may be NULL) is OR-ed with 1 for every body flagged in any
 * step.  pair_log (may be NULL) receives (step, i, j) triples, up to
 * log_cap of them; log_count receives how many were found in total.
 * stats (may be NULL) receives {pairs, groups, max BS sub-steps,
 * max Kepler iterations}. */
int orc_step(const orc_params* p, int nbig, int nsmall, double* xv,
             const double* mu, const double* rcrit, const double* rp_km,
             const double* rhop, int nsteps, unsigned char* ever_flag,
             int* pair_log, int log_cap, int* log_count, long long* stats);

/* As orc_step, with bodies that can be removed (Sec. 3.5) and masses that can
 * grow (Sec. 3.3; growth may be NULL).  With growth, every step k (global index
 * step0 + k) starts by taking mu, rcrit and the gaps from orc_grow_state at
 * t = (step0 + k) h; the planetesimals' drag then sees Sigma times the gap
 * factor of the last growing body (ascending index) whose gap, centred on its
 * cylindrical distance at kick time, holds the planetesimal's cylindrical
 * distance strictly inside (the Sec. 3.1 listing).  rcrit[n] is in/out.  stat[n] (in/out):
 * 0 for a body in the integration, -3 for one removed as ejected; a removed
 * body keeps its state and takes no further part in the step.  mu[n] (in/out):
 * an ejected massive body's mu becomes 0.  step0 is the global index of the
 * first step (the ejection test follows steps with (step0 + k + 1) a multiple
 * of p->eject_every). */
int orc_step_ex(const orc_params* p, int nbig, int nsmall, double* xv, double* mu,
                double* rcrit, const double* rp_km, const double* rhop, int nsteps,
                long long step0, signed char* stat, const orc_growth* growth, double gap_c,
                unsigned char* ever_flag, long long* stats);

/* What the growth tracks give at time t (Sec. 3.3 and the gap of Sec. 3.1),
 * from the DH state xv (6 x n) whose momentum is taken with the masses mu:
 * for every growing massive body i < nbig, mu_out = G M_p(t), rcrit_out =
 * rcrit_hill R_H with R_H = a (M_p / 3 m0)^(1/3) from the osculating a
 * (gm = G (m0 + M_p)), the gap half-width gap_c R_H and density factor
 * exp(-(t - tau_c)/tau_g) once t > tau_c (else half-width 0 and factor 1),
 * and the radius (Eq. 14 with c_s at the body's cylindrical distance, or
 * Eq. 16 with R_c = Eq. 14 at M_p = mc).  Bodies that do not grow keep mu and
 * rcrit and get no gap and radius 0.  Any output may be NULL. */
int orc_grow_state(const orc_params* p, int nbig, int n, const double* xv, const double* mu,
                   const double* rcrit, const orc_growth* g, double gap_c, double t,
                   double* mu_out, double* rcrit_out, double* gap_w, double* gap_f,
                   double* radius);

/* The ejection test of Sec. 3.5 on a DH state: every body still in the
 * integration whose heliocentric osculating eccentricity (gm = G(m0 + m) for
 * massive bodies, G m0 for planetesimals) is >= 1 gets stat -3 and mu 0.
 * Returns the number of bodies removed in *n_new. */
int orc_eject(const orc_params* p, int nbig, int n, const double* xv, double* mu,
              signed char* stat, int* n_new);

/* Osculating heliocentric elements of n bodies about gm[j] from the
 * heliocentric state xv (6 x n): out (6 x n) rows q [AU], e, i [rad],
 * varpi = longitude of pericentre, Omega = longitude of the node, M = mean
 * anomaly (e < 1: in [0, 2 pi); e > 1: e sinh F - F; e = 1: Barker's
 * D + D^3/3 with D = tan(f/2)). */
int orc_elements(int n, const double* gm, const double* xv, double* out);

/* Energy (M_sun AU^2 d^-2) and angular momentum of the massive bodies. */
int orc_energy(const orc_params* p, int nbig, int n, const double* xv,
               const double* mu, double* E, double* L3);

/* Semimajor axes from heliocentric states (vis-viva, gm = G*m_star for
 * small bodies, G*(m_star + m) for big ones). */
int orc_semimajor(const orc_params* p, int nbig, int n, const double* mu,
                  const double* xv_helio, double* a);

/* Forward-mode reference derivative of the loss
 *   L = sum_j w[j] * (a_final_j - a_initial_j)^2   (small bodies j)
 * after nsteps steps from the heliocentric input state, along the direction
 * (dxv [6xN], dpar = {d sigma1, d gamma, d cd_scale}).  Returns L and dL. */
int orc_jvp_loss(const orc_params* p, int nbig, int nsmall, const double* m_big,
                 const double* xv_helio, const double* rp_km, const double* rhop,
                 const double* w, int nsteps, const double* dxv,
                 const double* dpar, double* L, double* dL);

#ifdef __cplusplus
}
#endif
#endif
