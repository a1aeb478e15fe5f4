/*
 * lbpf.h -- C ABI of the GB300 (sm_103a) lattice-Boltzmann phase-field solver.
 *
 * The solver advances the coupled phase field phi, supersaturation U and
 * temperature theta of Cartalade, Younsi & Plapp (arXiv 1602.07483, Sec. 2,
 * Eqs. PhaseField_KarmaRappel, Concentration_Echebarria, Temp_Ramirez) with
 * the lattice-Boltzmann schemes of Sec. 3:
 *   - phi: non-local BGK collision, Eqs. (LBE_Eq_Phase)-(LBE_RelaxationTime)
 *     and the collision stage of Sec. 3.4, anisotropy Eq. (Anisotropic-
 *     Function_As) or Eq. (As_K41-K61), N vector Eq. (TermesAnisotropes);
 *   - U: BGK with the modified equilibrium, Eqs. (Supersaturation_Bis)-
 *     (RelaxationTime_Concentration), anti-trapping Eq. (AntiTrapping_Current);
 *   - theta: standard BGK with a source, Eqs. (LBE_Eq_Temp)-(ThermalDiffusivity);
 *   - streaming with bounce-back zero-flux walls (Sec. 3.4, Sec. 4).
 * Lattices D3Q7, D3Q15, D3Q19 (Tables 1-2), or D2Q5, D2Q9 (Tables 3-4) on an
 * nz = 1 grid, where the z walls carry no links and bound no wall nodes.
 * One step is: phi collision and
 * streaming with phi^n, U^n, theta^n; then U and theta with phi^{n+1} and
 * dphi/dt = (phi^{n+1} - phi^n)/dt (Sec. 3.4, "Algorithm implementation").
 *
 * Conventions for every call:
 *   - Return value: LBPF_OK (0) or a negative LBPF_E* code; lbpf_strerror()
 *     names it.  A CUDA failure is sticky: every later call on the handle
 *     returns LBPF_ECUDA.
 *   - Host arrays are owned by the caller, FP64, site-major with x fastest:
 *     index ((z*ny + y)*nx + x).  Population arrays are population-major,
 *     [Q][nz][ny][nx], in the paper's direction order (Table 1 or 3), and hold the
 *     POST-STREAMING populations g_i(x,t), h_i(x,t), f_i(x,t).
 *   - Device memory is owned by the handle (allocated in lbpf_create, freed
 *     in lbpf_destroy).  Work is enqueued on the caller's CUDA stream (or on
 *     a non-blocking stream owned by the handle when NULL); calls that return
 *     host data synchronise that stream.
 *   - There is no CPU fallback: without a usable CUDA device lbpf_create
 *     returns LBPF_ECUDA.
 *   - Handles are not thread-safe; use one handle per host thread.
 */
#ifndef LBPF_H
#define LBPF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBPF_OK 0
#define LBPF_EINVAL (-1)    /* bad argument (sizes, lattice, null pointer) */
#define LBPF_EUNSTABLE (-2) /* parameters give a relaxation time <= 1/2 somewhere */
#define LBPF_ENOMEM (-3)    /* device allocation failed */
#define LBPF_ENAN (-4)      /* a non-finite value was found in the fields */
#define LBPF_ETIMEOUT (-5)  /* a bounded wait of the one-launch step gave up (sticky; see
                               lbpf_set_schedule) */
#define LBPF_ECUDA (-6)     /* CUDA runtime error (sticky) */

/* storage of the distributions; arithmetic is FP64 for LBPF_F64, FP32 otherwise */
#define LBPF_F64 0
#define LBPF_F32 1
#define LBPF_F16 2  /* (f - shift) * scale in binary16, decoded to FP32 */
#define LBPF_BF16 3 /* same codec in bfloat16 */

/* field mask for lbpf_read_fields */
#define LBPF_PHI 1u
#define LBPF_U 2u
#define LBPF_THETA 4u

typedef struct {
  int32_t nx, ny, nz; /* nodes per edge, each >= 1; nx*ny*nz < 2^32 / 19 (226,050,910) */
} lbpf_grid;

/* 3D: every lattice in {7, 15, 19}.  2D: every lattice in {5, 9} and nz = 1.
 * Mixing 2D and 3D lattices is LBPF_EINVAL. */
typedef struct {
  int32_t q_phi;   /* 7 | 15 | 19  or  5 | 9 */
  int32_t q_u;     /* 7 | 15 | 19  or  5 | 9 */
  int32_t q_theta; /* 0 (theta frozen at theta0) | 7 | 15 | 19  or  0 | 5 | 9 */
} lbpf_lattice;

typedef struct {
  double W0, tau0;      /* interface width, relaxation time (Eq. PhaseField_KarmaRappel) */
  double D, kappa;      /* solute and thermal diffusivity */
  double lambda;        /* coupling constant */
  double Mc_inf;        /* scaled liquidus slope M c_inf */
  double k;             /* partition coefficient, 0 < k <= 1 */
  int32_t aniso;        /* 0: Eq. (Anisotropic-Function_As); 1: Eq. (As_K41-K61) */
  double eps1, eps2;    /* aniso 0: eps_s, unused; aniso 1: eps_s, delta */
  double dx, dt;        /* lattice spacing and time step */
  int32_t antitrapping; /* 1: anti-trapping current on; 0: off */
  int32_t storage;      /* LBPF_F64 | LBPF_F32 | LBPF_F16 | LBPF_BF16 */
  double grad2_min;     /* |grad phi|^2 below which n, N, j_at are taken as 0 and a_s = 1;
                           0 selects the default 1e-12 */
} lbpf_params;

typedef struct lbpf_sim lbpf_sim;

/* Create a simulation on the current CUDA device.  Validates every argument,
 * derives the relaxation times eta_U (Eq. RelaxationTime_Concentration) and
 * eta_theta (Eq. ThermalDiffusivity), and rejects parameter sets for which
 * a_s^2 eta_phi(a_s) <= 1/2 for some orientation (the non-local collision then
 * over-relaxes), or eta_U, eta_theta <= 1/2, with LBPF_EUNSTABLE.  Allocates all
 * device state (two copies of each distribution, three levels of phi, two of
 * U and theta).  `cuda_stream` is a cudaStream_t or NULL; it is borrowed.
 * The state is zero until lbpf_init_seed or lbpf_set_state. */
int lbpf_create(const lbpf_grid* grid, const lbpf_lattice* lattice, const lbpf_params* params,
                void* cuda_stream, lbpf_sim** out);

/* Initial condition of Sec. 4: n_seeds diffuse spheres
 * phi = tanh((R - r) dx / (sqrt2 W0)) (the largest value where seeds overlap),
 * U = U0 and theta = theta0 everywhere.  centres: 3*n_seeds lattice coordinates
 * (x,y,z; fractional allowed), radii: n_seeds lattice units.  Populations start
 * at g = w phi, h = (A + B q/zeta) U, f = w theta.  Resets the step counter. */
int lbpf_init_seed(lbpf_sim* sim, int32_t n_seeds, const double* centres, const double* radii,
                   double U0, double theta0);

/* Replace the state by post-streaming populations from the host (FP64, layout
 * above; f may be NULL when q_theta == 0).  Moments are recomputed as sums of
 * the populations; theta0 is the frozen temperature when q_theta == 0.
 * Resets the step counter.  Synchronous. */
int lbpf_set_state(lbpf_sim* sim, const double* g, const double* h, const double* f, double theta0);

/* Copy the post-streaming populations to the host (FP64; any pointer may be
 * NULL to skip that field).  Synchronous. */
int lbpf_get_state(lbpf_sim* sim, double* g, double* h, double* f);

/* Enqueue n_steps time steps (asynchronous).  Steps are replayed from a CUDA
 * graph captured on first use.  Returns LBPF_OK, or a sticky error. */
int lbpf_step(lbpf_sim* sim, int64_t n_steps);

/* Same as lbpf_step but without graphs: each kernel launch is bracketed by CUDA
 * events recorded on the handle's stream, and the call returns (synchronously)
 * the summed device time of the phase-field kernels in ms_kernels[0], of the
 * U/theta kernels in ms_kernels[1], and the wall span of the n steps in
 * ms_kernels[2].  Under the one-launch schedule the whole step is one kernel:
 * its time is in ms_kernels[0] and ms_kernels[1] is 0.  Used to measure
 * per-kernel bandwidth. */
int lbpf_step_timed(lbpf_sim* sim, int64_t n_steps, double ms_kernels[3]);

/* Copy phi, U and/or theta (as selected by mask) of the current step to the
 * host in FP64; unselected pointers may be NULL.  Synchronous. */
int lbpf_read_fields(lbpf_sim* sim, uint32_t mask, double* phi, double* U, double* theta);

/* FP64 sums over all sites, computed on the device in a fixed order:
 * out[0] = sum phi, out[1] = sum U, out[2] = sum theta,
 * out[3] = sum zeta(phi) (1 + (1-k) U)  (total solute, c / c_inf).
 * Returns LBPF_ENAN (after filling out) when any sum is not finite.  Synchronous. */
int lbpf_sums(lbpf_sim* sim, double out[4]);

/* Dendrite tip and tip radius (the tip velocity of Sec. 4.1 is the tip's displacement per
 * unit time).  axis: 0, 1, 2 = scan along +x, +y, +z (0 or 1 on a 2D grid).  centre_lu:
 * 3 lattice coordinates (x, y, z; z ignored on a 2D grid, give 0); the scan starts at the
 * node nearest to them, which must lie in the grid.  x_tip_lu: the first crossing
 * phi_i >= 0 > phi_{i+1} along the axis from that node, linearly interpolated, as a
 * coordinate along the axis in lattice units (-1 when none).  rho_lu (may be NULL): tip
 * radius in lattice units, a least-squares parabola t(j) = t_tip - j^2 / (2 rho) through
 * the crossings of the lines offset by j = +-1..+-4 along each other axis, one fit per
 * plane spanned by the scan axis and an axis with more than one node, averaged (the two
 * planes in 3D, the grid plane on a 2D or nz = 1 grid; -1 when undefined).
 * LBPF_EINVAL for a bad axis or a centre outside the grid.  Synchronous. */
int lbpf_tip(lbpf_sim* sim, int32_t axis, const double centre_lu[3], double* x_tip_lu, double* rho_lu);

/* Number of steps taken since the last init / set_state / load. */
int64_t lbpf_steps_done(const lbpf_sim* sim);

/* Checkpoint: write / read a self-describing binary file (header with grid,
 * lattices, parameters, step count; then the post-streaming populations and the
 * moment fields phi^n, phi^{n-1}, U^n, theta^n, theta^{n-1}, all in FP64), so that a
 * run restarts bit for bit in every storage type (the FP16/BF16 codec is shifted by
 * phi^{n-1} and theta^{n-1}, and decodes to FP64 exactly).  lbpf_load requires a handle
 * created with the same grid and lattices, and a file of this format (version 3). */
int lbpf_save(lbpf_sim* sim, const char* path);
int lbpf_load(lbpf_sim* sim, const char* path);

/* Tiling of the step kernels: node rows per block `by` (4..8; a block is
 * 32 x by threads, one node per thread and plane) and z-chunk length
 * (>= 1; the z range is split into chunks processed by separate thread
 * blocks).  0 keeps the current value.  Takes effect at the next lbpf_step
 * (the step graph is re-captured). */
int lbpf_set_tiling(lbpf_sim* sim, int32_t by, int32_t zchunk);
int lbpf_get_tiling(const lbpf_sim* sim, int32_t* by, int32_t* zchunk);

/* Autotuner: times `steps` steps for each candidate tiling on a snapshot of
 * the current state, keeps the fastest, and restores the state.  best_ms
 * (may be NULL) receives the best time per step.  Synchronous. */
int lbpf_autotune(lbpf_sim* sim, int32_t steps, double* best_ms);

/* How a step is launched (the order of the work within a step follows Sec. 3.4:
 * phi first, then U and theta with phi^{n+1}; both schedules give bit-identical results).
 *   LBPF_SCHED_TWO_KERNELS (default): the phase-field kernel over all tiles, then the
 *     U/theta kernel over all tiles.
 *   LBPF_SCHED_ONE_LAUNCH: one persistent kernel per step in which the U/theta tile of a
 *     region starts as soon as the phase-field tiles that write phi^{n+1} around it are done,
 *     so that both phases run side by side on the SMs.  Its blocks wait on flags set by
 *     other blocks of the same launch, in an order that always lets them finish; every wait
 *     is bounded (about a second), and a wait that gives up makes the handle fail with
 *     LBPF_ETIMEOUT at the next call that returns data.  Available for FP32, FP16 and BF16
 *     storage with the lattice triples D3Q19 x D3Q19 x {frozen theta, D3Q7, D3Q19} and
 *     D2Q9 x D2Q5 x D2Q5 (LBPF_EINVAL otherwise).
 * Synchronises the handle's stream; the step graph is re-captured at the next step. */
#define LBPF_SCHED_TWO_KERNELS 0
#define LBPF_SCHED_ONE_LAUNCH 1
int lbpf_set_schedule(lbpf_sim* sim, int32_t schedule);
int lbpf_get_schedule(const lbpf_sim* sim, int32_t* schedule);
/* Bound of each wait of the one-launch step, in polling rounds of about 0.25 us (default
 * 2^22, about a second; the ordered schedule never needs more than the time one tile takes).
 * 0 makes every wait give up at once: the step then runs with the flag of a failed wait set,
 * and the next call that returns data reports LBPF_ETIMEOUT (sticky), which is how the
 * failure path is tested without a device hang.  LBPF_EINVAL for a negative value.
 * Synchronises the handle's stream; takes effect at the next step. */
int lbpf_set_wait_polls(lbpf_sim* sim, int32_t polls);

/* Diagnostic of the bounded wait the one-launch step uses: one warp waits on a device flag
 * initialised to `flag_value` for at most `polls` rounds (each about 0.25 us); *seen is 1
 * when the wait saw the flag set (flag_value != 0), 0 when it gave up.  The device stays
 * usable either way.  Synchronous (synchronises the device). */
int lbpf_wait_probe(int32_t flag_value, int32_t polls, int32_t* seen);

int lbpf_destroy(lbpf_sim* sim);

/* Batched stepping: several independent simulations with identical lattices and storage
 * (grids and physical parameters may differ, e.g. the parameter sweeps over Delta, eps
 * and k of the paper's Sec. 4 studies) advance together, one launch per kernel phase
 * covering the tiles of all members, with the time loop captured in one CUDA graph.
 *
 * lbpf_batch_create: creates n member simulations, member i from grids[i], lattices[i]
 * and params[i] as lbpf_create would (all lattices[i] equal, all params[i].storage equal,
 * else LBPF_EINVAL; a failing member's lbpf_create code is returned).  The batch owns the
 * members and destroys them in lbpf_batch_destroy.  All members run on `cuda_stream`
 * (borrowed), or on a non-blocking stream the batch owns when it is NULL.  Get a member's
 * handle with lbpf_batch_member to seed it, read it or step it alone. */
typedef struct lbpf_batch lbpf_batch;
int lbpf_batch_create(int32_t n, const lbpf_grid* grids, const lbpf_lattice* lattices, const lbpf_params* params,
                      void* cuda_stream, lbpf_batch** out);
/* The i-th member of a batch (0 <= i < n); the handle stays owned by whoever created it. */
int lbpf_batch_member(const lbpf_batch* batch, int32_t i, lbpf_sim** out);
/* A batch over handles the caller already created (they stay the caller's; destroy the
 * batch before them).  The batch runs on `cuda_stream`, or on the first member's stream
 * when NULL; lbpf_batch_step orders itself after the work each member has enqueued on its
 * own stream and makes each member's stream wait for the batch's work, so calls on a
 * member between batch steps need no extra synchronisation. */
int lbpf_batch_from_sims(int32_t n, lbpf_sim* const* sims, void* cuda_stream, lbpf_batch** out);
/* Enqueue n_steps steps of every member (asynchronous).  All members must have taken the
 * same number of steps (LBPF_EINVAL otherwise). */
int lbpf_batch_step(lbpf_batch* batch, int64_t n_steps);
/* Tiling of the batched launches, as lbpf_set_tiling for one handle: `by` block
 * rows (4..8, 0 keeps the current; ignored for 2D lattices, which use one-row
 * blocks) and z-chunks of `zchunk` planes for every member (0: each member's
 * default).  Results do not depend on the tiling.  LBPF_EINVAL for values out of
 * range.  Synchronises the batch stream. */
int lbpf_batch_set_tiling(lbpf_batch* batch, int32_t by, int32_t zchunk);
/* The batch's current tiling: block rows and the z-chunk request (0: each member's
 * default).  Either pointer may be NULL. */
int lbpf_batch_get_tiling(const lbpf_batch* batch, int32_t* by, int32_t* zchunk);
/* Times the candidate batch tilings and keeps the fastest, as lbpf_autotune does for
 * one handle: block rows 4, 6 and 8 with z-chunks of each member's default, 12, 16 and
 * 24 planes (2D lattices: one-row blocks with chunks of the default, 8, 16 and 32 rows).
 * Each candidate runs single steps up to the next multiple of 6 steps, 6 warm-up steps,
 * then `steps` rounded up to a multiple of 6, timed with CUDA events on the batch
 * stream; every member's state and step count are restored afterwards, so the batch
 * continues exactly as if the call had not been made (the state is copied on the device:
 * LBPF_ENOMEM, tiling unchanged, when the copy of all members does not fit).
 * best_ms (may be NULL): milliseconds per batch step of the tiling kept.  All members
 * must have taken the same number of steps (LBPF_EINVAL otherwise).  Synchronous. */
int lbpf_batch_autotune(lbpf_batch* batch, int32_t steps, double* best_ms);
/* The step schedule of the batched launches, as lbpf_set_schedule for one handle (the
 * one-launch schedule spans the tiles of all members).  Synchronises the batch stream. */
int lbpf_batch_set_schedule(lbpf_batch* batch, int32_t schedule);
int lbpf_batch_get_schedule(const lbpf_batch* batch, int32_t* schedule);
int lbpf_batch_destroy(lbpf_batch* batch);

/* Largest n_sites that lbpf_field_sums_noalloc accepts (65536 partial sums of
 * 4096 sites each). */
#define LBPF_NOALLOC_MAX_SITES (268435456LL)

/* The same four FP64 sums as lbpf_sums, over caller-owned DEVICE arrays, with
 * no memory allocation at all.  The paper has no counterpart: this serves
 * callers that hold device fields but cannot call cudaMalloc -- loops that must
 * avoid the implicit device synchronisation of cudaMalloc/cudaFree, and hosts
 * whose device memory is fully reserved by another allocator.
 *   phi, U, theta: device arrays of n_sites elements of the compute type of
 *     `storage` (double for LBPF_F64, float otherwise); theta may be NULL, then
 *     theta0 is used at every site.
 *   k: partition coefficient of the solute sum.  out: HOST array of 4 doubles.
 *   cuda_stream: stream to run on (NULL = legacy default stream); the call
 *     copies the sums to `out` and synchronises the stream before returning, so
 *     a stream that is being captured is refused (LBPF_EINVAL, nothing enqueued).
 * The reduction scratch (2 MiB) is a file-scope device array that every GPU
 * loading the library keeps until the process exits; all calls on a device
 * share it and each call overwrites the part it uses, so nothing in it needs
 * clearing.  Calls that overlap on the GPU (several streams or host threads at
 * once) race on that scratch and must be serialised by the caller.  The first
 * call on a device looks up the scratch's device address with
 * cudaGetSymbolAddress and keeps it for the process; make that first call before
 * any stream capture, and do not call again on a device after cudaDeviceReset.
 * Returns LBPF_EINVAL for NULL inputs, n_sites < 1 or
 * n_sites > LBPF_NOALLOC_MAX_SITES, LBPF_ENAN when a sum is not finite,
 * LBPF_ECUDA on a CUDA error. */
int lbpf_field_sums_noalloc(const void* phi, const void* U, const void* theta, int32_t storage, int64_t n_sites,
                            double k, double theta0, double out[4], void* cuda_stream);

/* Static description of an error code. */
const char* lbpf_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBPF_H */
