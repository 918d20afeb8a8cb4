// mx_kernels.h -- host-side launchers of the sm_103a kernels (internal to the
// library; the public C ABI is include/mx.h).
#pragma once
#include <cuda_runtime.h>

namespace mx {

struct Dev;

// One shared-memory carveout for all kernels of a step (set once per system).
void configure_drift();
void configure_detect();
void configure_kick();
void configure_bs();
void configure_orbit();

// k_init.cu / k_misc.cu
void launch_init_sys(const Dev& d, int do_rcrit, double rcrit_hill, cudaStream_t st);
void launch_set_step(const Dev& d, long long step, cudaStream_t st);
void launch_init_bodies(const Dev& d, const double* rp_km, const double* rho, int set_drag,
                        cudaStream_t st);
void launch_readout(const Dev& d, double* out, cudaStream_t st);
void launch_energy(const Dev& d, double* out, cudaStream_t st);
void launch_dfma(double* sink, int blocks, int iters, cudaStream_t st);

// k_kick.cu
void launch_prep(const Dev& d, double jump_frac, int nkick, cudaStream_t st);
void launch_jump_kick(const Dev& d, double jump_frac, double kick_frac, int nkick, cudaStream_t st);
void launch_jump_kick_fused(const Dev& d, cudaStream_t st);
void launch_accel(const Dev& d, double* acc, int drag_only, int acc_stride, int acc_base,
                  cudaStream_t st);

// k_drift.cu
void launch_jump_drift(const Dev& d, double jump_frac, cudaStream_t st);
void launch_drift_buf(double* xv, int n, double mu, double h, int maxit, unsigned* status,
                      cudaStream_t st);

// k_detect.cu
void launch_detect(const Dev& d, const double* xv0, const double* xv1, unsigned char* flags,
                   unsigned long long* keys, int* count, int cap, int runs, cudaStream_t st);
void launch_sort_keys(unsigned long long* keys, const int* count, int cap, int swap_ij,
                      cudaStream_t st);
void launch_keys_to_pairs(const unsigned long long* keys, const int* count, int cap, int* pairs,
                          cudaStream_t st);

// k_bs.cu
void launch_groups(const Dev& d, cudaStream_t st);
void launch_bs(const Dev& d, int nblocks, cudaStream_t st);
// The persistent interior step (one cooperative launch, grid barriers with
// at most `spin` polls each): its largest resident grid for the current
// tiling (0 if the occupancy query failed), and the launch (barrier words
// zeroed first).
int persist_grid(const Dev& d);
cudaError_t launch_step_persist(const Dev& d, int grid, long long spin, cudaStream_t st);
// mode 0: window end (budgeted, carried bodies to bank_out); 1: side stream
// (bank_a in place); 2: settle (everything rejoins).  Slots up to t_end; a
// body kept at t_end is stored at slot t_next (the next range's start).
void launch_catchup(const Dev& d, int nblocks, int mode, int bank_a, int bank_b, int bank_out,
                    int t_end, int tl, int next_slot, int t_next, cudaStream_t st);

// k_orbit.cu (Sec. 3.5): ejection test (scheduled = 1 after a step), elements
// (6 x N), removed bodies per system
void launch_eject(const Dev& d, int scheduled, cudaStream_t st);
void launch_elements(const Dev& d, double* out, cudaStream_t st);
void launch_stat_count(const Dev& d, int* out, cudaStream_t st);

// k_grow.cu (Sec. 3.3): radii of the growing planets now (mx_planets)
void launch_radius(const Dev& d, cudaStream_t st);

// k_adjoint.cu
// The adjoint step in two parts: the forward recomputation up to the drift,
// with the encounter groups' tape plan (its size in doubles in *a.tape_need)
// when a.groups; then the groups' integration and the reverse sweep.
void launch_adjoint_step_a(const Dev& d, const Adj& a, cudaStream_t st);
void launch_adjoint_step_b(const Dev& d, const Adj& a, cudaStream_t st);
// The pending pair pass of a merged reverse on its own (a.lpend at the
// positions xpos, 3 x N), into a.lam.
void launch_adjoint_flush(const Dev& d, const Adj& a, const double* xpos, cudaStream_t st);
// Resident blocks per SM of the kick's reverse at `threads` threads a block.
int adjoint_vjp_blocks_per_sm(int threads);
// k_adj_bs.cu: the step's encounter groups inside the adjoint (forward with a
// tape, reverse, per-system fold of the big bodies' shares)
void launch_adjoint_bs_plan(const Dev& d, const Adj& a, cudaStream_t st);
void launch_adjoint_bs_fwd(const Dev& d, const Adj& a, int nblocks, cudaStream_t st);
void launch_adjoint_bs_vjp(const Dev& d, const Adj& a, int nblocks, cudaStream_t st);
void launch_adjoint_bs_fold(const Dev& d, const Adj& a, cudaStream_t st);
void launch_loss(const Dev& d, const double* xvh0, const double* w, double* seed_f, double* seed_i,
                 double* part, const int* poff, double* Lsys, cudaStream_t st);
void launch_init_vjp(const Dev& d, const double* lam, double* grad, cudaStream_t st);

}  // namespace mx
