/*
 * ccmsav.h -- C ABI of the GB300 (sm_103a) CC-MSAV vesicle time stepper.
 *
 * The library advances the coupled Allen-Cahn (membrane phase phi) /
 * variable-mobility Cahn-Hilliard (concentration psi) system with the
 * constant-coefficient MSAV scheme of Zhang, Li, Lowengrub and Wise,
 * "An Efficient Constant-Coefficient MSAV Scheme for Computing Vesicle Growth
 * and Shrinkage" (arXiv 2601.10057):
 *   - model and energy: Sec. 2.1 (eqs. AC, CH, energy_functional,
 *     energy_densities) with the MSAV reformulation of Sec. 2.2 (eqs.
 *     modified_energy, aux_vars, msav_mu, msav_nu);
 *   - time step: CC-MSAV-BDF2 of Sec. 3.2 (eqs. AC_BDF2 ... Z_BDF2); the first
 *     step after ccmsav_set_state is the CC-MSAV-BDF1 variant (Appendix B,
 *     remark on the BDF1 scheme);
 *   - space: cell-centred staggered grid with homogeneous Neumann ghost cells
 *     (Sec. 3.4, Appendix D), face mobility and nonlocal bending terms of
 *     Sec. 3.4.1;
 *   - solution procedure: Appendix B (Steps 1-4, Algorithm "BDF2 MSAV Solution
 *     Procedure") with the constant-coefficient operators chi and zeta solved
 *     by DCT-II / eigenvalue divide / DCT-III (Appendix C).
 *
 * Conventions for every call:
 *   - Return value: 0 on success, a negative CCMSAV_E* code otherwise;
 *     ccmsav_strerror() gives a message.  No call aborts the process.
 *   - Fields are N*N arrays, row-major: a[j*N + i] is cell (i, j) with centre
 *     ((i + 1/2) h, (j + 1/2) h), h = L / N.
 *   - The library owns all of its device memory and frees it in
 *     ccmsav_destroy().  It never frees or keeps caller memory: host pointers
 *     are read or written only during the call.
 *   - Work is queued on the CUDA stream given to ccmsav_create(); calls that
 *     return data to the host synchronise that stream.
 *   - After a device-side error (CCMSAV_ENONFINITE) the handle refuses to
 *     step until the next ccmsav_set_state().
 *   - A handle must not be used from two host threads at once.
 */
#ifndef CCMSAV_H
#define CCMSAV_H

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CCMSAV_OK           0
#define CCMSAV_EINVAL      -1   /* bad argument (size, parameter, index, NULL) */
#define CCMSAV_ENOMEM      -2   /* device or host allocation failed */
#define CCMSAV_ECUDA       -3   /* a CUDA runtime call failed */
#define CCMSAV_ESTATE      -4   /* call out of order (e.g. step before set_state) */
#define CCMSAV_ENONFINITE  -5   /* NaN/Inf input or state, a SAV radicand <= 0,
                                   or a face mobility M_psi(A phi*) <= 0 */
#define CCMSAV_ETIMEOUT    -6   /* reserved for a bounded device-side wait that
                                   gives up; no kernel of this library waits on
                                   another (stream order and last-block arrival
                                   counters order the phases), so no call
                                   returns it */

/* Precision of the field arithmetic. */
#define CCMSAV_FP64       0     /* fields, stencils, DCTs and reductions in FP64 */
#define CCMSAV_FP32_BULK  1     /* fields, stencils and DCTs in FP32; SAV inner
                                   products, scalar updates, the 5x5 solve and
                                   mass/energy reductions accumulated in FP64 */

/* Flags for ccmsav_create(). */
#define CCMSAV_TRACK_ENERGY 1   /* accumulate the lambda-sum of the modified
                                   energy each BDF2 step (one extra reduction
                                   kernel per step); needed for E_mod in
                                   ccmsav_energy() */
#define CCMSAV_CLASSICAL    4   /* the classical MSAV scheme instead of CC-MSAV
                                   (the paper's baseline, Sec. 3.5.2; Appendix B
                                   remarks on the Classical-MSAV schemes): the
                                   Cahn-Hilliard stabilisation inside the
                                   chemical potential, so both Cahn-Hilliard
                                   solves use 3/(2 dt) - lam div(M_psi(phi*) grad),
                                   solved by DCT-preconditioned conjugate
                                   gradients (the constant-coefficient
                                   operator with the mean face mobility as
                                   preconditioner); the Allen-Cahn part is the
                                   CC-MSAV one.  Steps are launched directly
                                   (no CUDA graphs): the host reads the
                                   convergence flags every four iterations */
#define CCMSAV_BDF1_ALWAYS  2   /* every step is the first-order CC-MSAV-BDF1
                                   scheme (Appendix B, remark on the BDF1
                                   scheme: level n in place of the
                                   extrapolations, 1/dt in place of 3/(2 dt),
                                   phi^n/dt in place of (4 phi^n - phi^{n-1})/(2 dt),
                                   SAV updates X^{n+1} = X^n + (F, phi^{n+1} - phi^n)) */

/* Model and scheme parameters.  Symbols and default values are those of the
 * paper's parameter table (Appendix G): gamma_surf, gamma_bend, gamma_area
 * (surface, bending and arc-length penalty), gamma_in/out, psi_in/out,
 * beta_in/out (osmotic densities f_in/out, Sec. 2.1), eps (interface width),
 * M_phi (Allen-Cahn mobility), M0 (Cahn-Hilliard mobility parameter in
 * M_psi = 1 - M0 (phi^2 - 1)^2), theta and lam (Allen-Cahn and Cahn-Hilliard
 * stabilisation, Sec. 3.2), beta (SAV splitting parameter), dt (time step)
 * and L (side of the square domain [0, L]^2). */
typedef struct {
    double gamma_surf, gamma_bend, gamma_area;
    double gamma_in, gamma_out;
    double psi_in, psi_out;
    double beta_in, beta_out;
    double eps, M_phi, M0;
    double theta, beta, lam;
    double dt, L;
} ccmsav_params;

typedef struct ccmsav ccmsav_t;   /* opaque handle */

/* Create a stepper for n_sims independent simulations (n_sims >= 1).
 *   N[s]      grid size of simulation s: a power of two in [8, 8192].
 *   params    parameters shared by all simulations; per_sim (may be NULL)
 *             gives one parameter set per simulation instead.
 *   precision CCMSAV_FP64 or CCMSAV_FP32_BULK.
 *   flags     0 or a combination of CCMSAV_TRACK_ENERGY, CCMSAV_BDF1_ALWAYS
 *             and CCMSAV_CLASSICAL.
 *   stream    a cudaStream_t (NULL: the legacy default stream).
 * Validates every parameter (eps, dt, L, lam, M_phi > 0; theta, beta,
 * gamma_* >= 0; 0 < M0 < 1) and returns CCMSAV_EINVAL otherwise.
 * Allocates all device memory; no device compute is queued.
 * On success *out receives the handle. */
int ccmsav_create(ccmsav_t** out, const ccmsav_params* params, int n_sims,
                  const int* N, const ccmsav_params* per_sim, int precision,
                  int flags, void* stream);

/* Load the initial state of simulation `sim` from host FP64 arrays phi, psi
 * (N*N each; copied before return).  Computes V^0, W^0, Z^0 from their
 * definitions (Sec. 2.2, eq. msav_ic) and sets the target arc length A of
 * U to the initial arc length int f_surf(phi^0) (so U^0 = 0; the paper does
 * not state A).  Resets the step counter, the lambda-sum and the error
 * state; the next step of this simulation is the BDF1 start step.
 * Returns CCMSAV_ENONFINITE if an input value is not finite (checked on the
 * device while the fields are uploaded); the simulation then holds no state
 * until the next successful set_state. */
int ccmsav_set_state(ccmsav_t* h, int sim, const double* phi, const double* psi);

/* As ccmsav_set_state, from device memory of the handle's precision (FP64
 * for CCMSAV_FP64, FP32 for CCMSAV_FP32_BULK).  The pointers are only read
 * during the call (stream-ordered). */
int ccmsav_set_state_device(ccmsav_t* h, int sim, const void* phi, const void* psi);

/* Advance every simulation by nsteps >= 0 time steps.  Asynchronous: work is
 * queued on the handle's stream; device-side errors are reported by the next
 * synchronising call (ccmsav_sync, get_state, energy, mass, get_aux).
 * Several simulations: their BDF2 steps run three at a time from one CUDA
 * graph per rotation phase of the three time levels.  Inside it, FP32
 * simulations of the same N on the warp-FFT kernels (N = 128 .. 2048, no
 * CCMSAV_CLASSICAL, CCMSAV_TRACK_ENERGY or CCMSAV_BDF1_ALWAYS) share each
 * kernel launch (one
 * launch per kernel, step and N for the whole group); the others run their
 * own launches concurrently.  Every simulation's results are the same bits
 * as a run of that simulation alone.
 * Returns CCMSAV_ESTATE if some simulation has no state yet or is in error. */
int ccmsav_step(ccmsav_t* h, int nsteps);

/* Wait for queued work and return the first device-side error, if any. */
int ccmsav_sync(ccmsav_t* h);

/* Copy the current phi^n, psi^n of simulation `sim` into caller-owned host
 * FP64 arrays (N*N each; FP32 fields are widened).  Synchronises. */
int ccmsav_get_state(ccmsav_t* h, int sim, double* phi, double* psi);

/* Diagnostics of simulation `sim` at the current level (synchronises):
 *   out[0] E_mod   modified discrete energy E^{n+1,n}_mod (eq.
 *                  modified_discrete_energy, discrete norms of Appendix D);
 *                  includes the lambda-sum only with CCMSAV_TRACK_ENERGY.
 *                  With CCMSAV_BDF1_ALWAYS: the one-level energy of the BDF1
 *                  scheme, c_b/2 ||Lap phi||^2 + (c_s - theta~)/2 ||grad phi||^2
 *                  + c_beta/2 ||phi||^2 + the SAV terms at level n
 *   out[1] F_surf  gamma_surf * int f_surf
 *   out[2] F_bend  gamma_bend * int f_bend
 *   out[3] F_area  gamma_area/2 (int f_surf - A)^2
 *   out[4] F_osm   int f_osm
 *   out[5] arc     int f_surf (the diffuse arc length)
 *   out[6] lamsum  sum_{j>=2} dt/2 ||d^j||^2 (0 without CCMSAV_TRACK_ENERGY)
 *   out[7] F       F_surf + F_bend + F_area + F_osm
 * All sums are accumulated in FP64. */
int ccmsav_energy(ccmsav_t* h, int sim, double out[8]);

/* Discrete mass h^2 sum_ij psi_ij of the stored concentration, summed in FP64
 * (Sec. 3.4.2, remark on mass conservation).  Synchronises. */
int ccmsav_mass(ccmsav_t* h, int sim, double* mass);

/* Scalar state of simulation `sim`:
 *   aux[0..3]  V^n, U^n, W^n, Z^n      aux[4..7]  V^{n-1}, U^{n-1}, W^{n-1}, Z^{n-1}
 *   aux[8]     A (target arc length)   aux[9]     lambda-sum
 *   aux[10]    steps taken since set_state
 *   aux[11]    the conserved mean of psi (FP64) that the FP32-bulk path keeps
 *              exactly (restored by set_aux when nonzero)
 * get synchronises; set replaces the scalars (the fields are untouched), for
 * example to restore a checkpoint together with set_state_levels. */
int ccmsav_get_aux(ccmsav_t* h, int sim, double aux[12]);
int ccmsav_set_aux(ccmsav_t* h, int sim, const double aux[12]);

/* The same twelve scalars copied to the caller's host buffer asynchronously:
 * the copy is queued on the simulation's stream behind the steps queued so
 * far, and the call returns at once.  `aux` must stay valid until that copy
 * has run (ccmsav_sync, or any synchronising call); with page-locked memory
 * the copy overlaps the following steps.  aux[10] is the device's own count
 * of steps (it equals get_aux's after set_state, or after set_aux).  The
 * device status is not checked here: ccmsav_sync reports a device error.
 * Lets a caller read every step's scalars without stalling the GPU between
 * steps.  Returns CCMSAV_ESTATE before set_state. */
int ccmsav_get_aux_async(ccmsav_t* h, int sim, double aux[12]);

/* Two-level field access for exact checkpoint/resume: the previous level
 * phi^{n-1}, psi^{n-1} (host FP64, N*N each). */
int ccmsav_get_prev_state(ccmsav_t* h, int sim, double* phi_prev, double* psi_prev);
int ccmsav_set_state_levels(ccmsav_t* h, int sim, const double* phi, const double* psi,
                            const double* phi_prev, const double* psi_prev);

/* Grid size of simulation `sim`, or a negative code. */
int ccmsav_grid_size(ccmsav_t* h, int sim);

/* Number of CUDA kernel launches queued by this handle since creation. */
long long ccmsav_launch_count(ccmsav_t* h);

/* Per-kernel tracing with CUDA events recorded on the handle's stream around
 * every kernel of every step while enabled (enable = 1; 0 stops recording).
 * ccmsav_profile_read() synchronises and returns, for simulation `sim`, the
 * accumulated device time in milliseconds of each step kernel in the order
 *   [0] stencil/pointwise + reductions   [1] forward row DCT (transposed)
 *   [2] forward column DCT + Gram sums   [3] 5x5 solve + SAV update
 *   [4] recovery + inverse column DCT    [5] inverse row DCT
 *   [6] lambda-sum reduction (CCMSAV_TRACK_ENERGY only)
 *   [7] the conjugate-gradient Cahn-Hilliard solves (CCMSAV_CLASSICAL only)
 * and in *nsteps the number of steps traced; it then resets the counters. */
int ccmsav_profile(ccmsav_t* h, int enable);
int ccmsav_profile_read(ccmsav_t* h, int sim, double ms[8], long long* nsteps);

/* Autotuner of the line-transform schedule.  It times `steps` BDF2 steps
 * (rounded up to a multiple of three, after three warm-up steps) of each
 * candidate schedule from the current state -- for a handle of one
 * simulation that simulation alone, for several simulations the handle's
 * batched step with the candidate applied to all of them (what the handle
 * runs) -- keeps the fastest (the default schedule unless another is at
 * least 2 % faster) and restores the state (the
 * fields and scalars are unchanged afterwards).  Candidates (FP32): the
 * warp-level four-step FFT kernels with a shared-memory carveout of 72, 58
 * or 100 percent for the three 8-line transform kernels, and the CTA-level
 * Stockham FFT kernels; FP64 has only the latter.  The choice is recorded
 * for each (N, precision) of the handle in a process-wide table, from which
 * handles created later start.  For several simulations a second stage then
 * times the launch-group size (ccmsav_set_group_points: the current value,
 * no grouping, 2^17 .. 2^22 and 2^26 grid points per group) with the chosen
 * schedule and keeps the fastest for this handle (the current value unless
 * another is at least 2 % faster).
 * report (may be NULL) receives 4 doubles per simulation: warp path (1/0),
 * carveout, best ms/step, ms/step of the default schedule (0 when not timed).
 * Needs set_state for every simulation (CCMSAV_ESTATE otherwise); steps in
 * [1, 3000]; not for CCMSAV_CLASSICAL handles (CCMSAV_EINVAL).  Synchronises. */
int ccmsav_autotune(ccmsav_t* h, int steps, double* report);

/* Launch groups of a handle of several simulations (see ccmsav_step): FP32
 * simulations of the same N on the warp-FFT kernels are grouped, in handle
 * order, until a group holds about `points` grid points (at least two
 * simulations); each group's six kernels per step are one launch each, and
 * the groups run concurrently on different streams.  points = 0: no
 * grouping.  Default 2^21.  Setting it synchronises and drops the handle's
 * batch graphs (they are captured again at the next step); results do not
 * depend on it (every simulation's bits equal its own run).
 * ccmsav_group_points returns the current value (-1 for a NULL handle). */
int ccmsav_set_group_points(ccmsav_t* h, long long points);
long long ccmsav_group_points(ccmsav_t* h);

/* Index checks of a library built with -DCCMSAV_BOUNDS (a separate
 * libccmsav_bounds.so, for testing): the step kernels check every element
 * index of their field, spectrum and level accesses against the array's
 * size; an index outside sets bit 1 (a load, redirected to element 0) or
 * bit 2 (a store, dropped) of a device flag.  Returns the flags raised by
 * the kernels of the handle's precisions since the last call (0: none) and
 * clears them; synchronises.  CCMSAV_EINVAL in a library built without the
 * checks. */
int ccmsav_bounds_flag(ccmsav_t* h);

/* Conjugate-gradient settings of a CCMSAV_CLASSICAL handle (all its
 * simulations): stop when ||r||_2 <= rtol ||b||_2 (rtol > 0; default 1e-10
 * for FP64, 1e-6 for FP32) or after max_iter iterations (>= 1; default 200).
 * CCMSAV_EINVAL on a bad value or a handle without CCMSAV_CLASSICAL. */
int ccmsav_set_pcg(ccmsav_t* h, double rtol, int max_iter);

/* Conjugate-gradient statistics of simulation `sim` (synchronises):
 *   out[0] iterations of the last step (the larger of its two solves)
 *   out[1] iterations of all steps since creation
 *   out[2], out[3] final relative residuals ||r|| / ||b|| of the last step's
 *          two solves (zeta_c^{-1} g0c and zeta_c^{-1} div(M grad P))
 * CCMSAV_EINVAL for a handle without CCMSAV_CLASSICAL. */
int ccmsav_pcg_stats(ccmsav_t* h, int sim, double out[4]);

/* Largest grid side accepted by ccmsav_mass_noalloc(): the largest grid a
 * handle accepts.  The scratch does not grow with N (see below). */
#define CCMSAV_NOALLOC_MAX_N 8192

/* ccmsav_mass_noalloc -- h^2 * sum_ij psi_ij (h = L / N) of a caller-owned
 * device field, with no device or host allocation by the library.
 * The paper has no counterpart: this is a service for callers that cannot
 * let a library allocate, e.g. services whose device memory is reserved up
 * front by a pooling allocator or capped by a framework, or real-time loops
 * that must not pay allocation latency.  It computes what ccmsav_mass()
 * computes for a handle's state, but for any N x N field the caller holds.
 *   psi        device pointer, N*N values, FP64 (precision CCMSAV_FP64) or
 *              FP32 (CCMSAV_FP32_BULK); summed in FP64 in a fixed order
 *   N          1 <= N <= CCMSAV_NOALLOC_MAX_N, else CCMSAV_EINVAL
 *   L          domain side (> 0)
 *   mass       host pointer to one double (output)
 *   stream     cudaStream_t the work is queued on; the call copies the result
 *              to *mass and synchronises that stream before it returns
 * Returns CCMSAV_ECUDA if a launch, the copy or the synchronisation fails.
 * Scratch is a fixed array of 1185 doubles (under 10 KB, whatever N is)
 * compiled into the library; every GPU that loads the library holds it until
 * the process exits.  Each call looks up that array's device address for
 * the current device and context (nothing is cached across calls).  All
 * calls share the array: calls whose work
 * overlaps on the GPU (different streams or host threads) race and must be
 * serialised by the caller. */
int ccmsav_mass_noalloc(const void* psi, int N, int precision, double L,
                        double* mass, void* stream);

/* ---------------------------------------------------------------------------
 * Standalone constant-coefficient spectral solver and initial-condition
 * smoother.
 *
 * ccmsav_solver_solve computes u = (c0 - c1 Lap_h + c2 Lap_h^2)^{-1} f on an
 * N x N cell-centred grid (h = L / N) with the 5-point Laplacian Lap_h and
 * one of three boundary rules, by forward transform, division by the
 * closed-form eigenvalues and inverse transform (Appendix C; the paper's
 * closing remarks name the DST and the FFT as the fast solvers for Dirichlet
 * and periodic boundaries):
 *   CCMSAV_BC_NEUMANN    mirror ghosts (u_{-1} = u_0, Appendix D), DCT-II/III;
 *   CCMSAV_BC_DIRICHLET  odd ghosts (u_{-1} = -u_0: u = 0 on the boundary
 *                        faces), DST-II/III;
 *   CCMSAV_BC_PERIODIC   wrapped ghosts (u_{-1} = u_{N-1}), complex FFT.
 * ccmsav_solver_smooth runs the smoother of Appendix F in place on a device
 * field phi: nsteps steps of the constant-mobility Cahn-Hilliard equation
 * phi_t = Mob Lap((phi^3 - phi)/eps - eps Lap phi), semi-implicit first order
 * (the nonlinear term explicit, the biharmonic term implicit):
 *   (1/dt + Mob eps Lap_h^2) phi^{n+1} = phi^n/dt + Mob Lap_h((phi^n^3 - phi^n)/eps),
 * each step one solve above, then phi <- max(-1, min(1, phi)).  The paper
 * uses Mob = 0.01, dt = 1e-6 and ten steps (T = 1e-5) with Neumann ghosts.
 *
 * Device pointers f, u, phi hold N*N values of the solver's precision
 * (FP64 or FP32), row-major, 16-byte aligned; f and u may be the same array.
 * The calls are asynchronous on the solver's stream (ccmsav_solver_sync waits
 * for it).  The solver owns its tables and one N x N scratch field (complex
 * for periodic) and frees them in ccmsav_solver_destroy. */
#define CCMSAV_BC_NEUMANN   0
#define CCMSAV_BC_DIRICHLET 1
#define CCMSAV_BC_PERIODIC  2

typedef struct ccmsav_solver ccmsav_solver_t;   /* opaque solver handle */

/* N a power of two in [8, 8192], L > 0, bc one of CCMSAV_BC_*, precision
 * CCMSAV_FP64 or CCMSAV_FP32_BULK (FP32 fields and transforms), stream a
 * cudaStream_t (NULL: a stream owned by the solver).  CCMSAV_EINVAL on a bad
 * argument, CCMSAV_ENOMEM if device memory runs out. */
int ccmsav_solver_create(ccmsav_solver_t** out, int N, double L, int bc, int precision, void* stream);

/* coef = {c0, c1, c2}: finite, c1 >= 0, c2 >= 0 and c0 + c1 s + c2 s^2 > 0 at
 * the smallest eigenvalue s of -Lap_h (0 for Neumann and periodic), else
 * CCMSAV_EINVAL.  CCMSAV_ECUDA if a launch fails. */
int ccmsav_solver_solve(ccmsav_solver_t* s, const double coef[3], const void* f, void* u);

/* eps > 0, mobility >= 0, dt > 0, nsteps >= 0 (0: only the clamp). */
int ccmsav_solver_smooth(ccmsav_solver_t* s, double eps, double mobility, double dt, int nsteps, void* phi);

/* Wait for the solver's queued work. */
int ccmsav_solver_sync(ccmsav_solver_t* s);

/* Kernel launches queued by the solver since creation. */
long long ccmsav_solver_launch_count(ccmsav_solver_t* s);

/* Free the solver (synchronises its stream first).  NULL is accepted. */
void ccmsav_solver_destroy(ccmsav_solver_t* s);

/* Message for a status code (static storage). */
const char* ccmsav_strerror(int status);

/* Free all device memory of the handle (synchronises its stream first).
 * NULL is accepted. */
void ccmsav_destroy(ccmsav_t* h);

#ifdef __cplusplus
}
#endif
#endif /* CCMSAV_H */
