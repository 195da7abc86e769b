/*
 * rve.h -- C ABI of the GB300 library for non-local ductile damage in
 * voxelised periodic RVEs (Magri, Lucarini, Lemoine, Adam, Segurado, "An FFT
 * framework for simulating non-local ductile failure in heterogeneous
 * materials").
 *
 * The library solves, for every load increment, the coupled problem of the
 * paper's Section 3.1 (Eq. governing_non-local): equilibrium div sigma = 0
 * under mixed macroscopic control (E_hk prescribed, Sigma_HK prescribed) and
 * one generalised Helmholtz equation abar_j - div(l_j^2(x) grad abar_j) =
 * alpha_j per non-local variable, with periodic boundary conditions, by the
 * iterated staggered scheme of Algorithm 1: a Newton / conjugate-gradient
 * FFT-Galerkin solve of the mechanics (Section 3.2.2) and a preconditioned
 * CG solve of each Helmholtz equation in Fourier space (Algorithm 2).  The
 * constitutive law is the non-local Lemaitre model (Section 2.2.3, Appendix
 * A.2): J2 plasticity with linear hardening on the effective stress and a
 * linear damage law driven by the non-local equivalent plastic strain.
 *
 * Conventions (all entry points):
 *  - Every call returns an int status (rve_status); none aborts or throws.
 *  - Grid sizes n = {N1, N2, N3} (N3 ignored in 2D); fields are stored
 *    component-major, x1 fastest: f[c][N3][N2][N1].
 *  - Strain/stress vectors exchanged through the handle-level calls
 *    (targets, homogenised values) use the component order 11, 22, 33, 23,
 *    13, 12 with TENSOR shears.  Fields passed to the operator-level calls
 *    (rve_op_*) carry Mandel components (shears times sqrt 2): 6 in 3D,
 *    the in-plane 11, 22, 12 in 2D (plane strain).
 *  - Pointers documented as "device" are CUDA device pointers valid on the
 *    handle's device; calls are enqueued on the handle's stream and are
 *    ordered with each other.  Calls that return host values synchronise
 *    that stream.  Inputs are copied; the caller keeps ownership of every
 *    buffer it passes.
 *  - One handle must not be used from two threads at once.
 *  - Stresses are in the units of the elastic moduli given (MPa in the
 *    shipped workloads); lengths in the units of L.
 */
#ifndef RVE_H
#define RVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rve rve_t;

typedef enum {
  RVE_OK = 0,
  RVE_ERR_ARG = -1,            /* invalid argument (null, size, range) */
  RVE_ERR_STATE = -2,          /* call out of order (e.g. no phases set) */
  RVE_ERR_CUDA = -3,           /* a CUDA runtime call failed */
  RVE_ERR_OOM = -4,            /* device allocation failed */
  RVE_ERR_NOT_CONVERGED = -5,  /* an iteration budget ran out; the state is
                                  left at the last converged increment */
  RVE_ERR_NUMERIC = -6,        /* NaN/Inf or Krylov breakdown */
  RVE_ERR_TIMEOUT = -7,        /* a device-side wait for a tile copy ran out
                                  of its budget (a hardware or driver fault);
                                  the handle should be freed */
  RVE_ERR_LOAD_PATH_END = -8   /* every increment of the load path is done */
} rve_status;

/* Per-phase constitutive parameters (Section 2.1.2; Section 4 for the damage
 * cap).  damage_law: 0 = linear elastic (E, nu only); 1 = J2 plasticity with
 * isotropic hardening sigma_0(eps_p) on the effective stress and Lemaitre
 * damage D = clamp((abar - eps_C)/(eps_R - eps_C), 0, D_max)
 * (Eq. non-local_damage_lemaitre); 2 = cracking elastic particle, an
 * extension of the multi-variable framework of Section 3.1 that the paper
 * does not print: local variable kappa = max(kappa_n, ||<eps>_+||) (norm of
 * the positive principal strains), D = clamp((abar - eps_C)/(eps_R - eps_C),
 * 0, D_max) with eps_C, eps_R read as kappa_C, kappa_R, sigma = (1 - D) C eps.
 * nonlocal_var: index j of the non-local variable this phase feeds with
 * alpha_j = eps_p (law 1) or kappa (law 2) and reads abar_j from, or -1
 * (Section 3.1: alpha_j = 0 outside the damaging phase).
 * 3 = non-local Gurson-Tvergaard-Needleman (Sections 2.1.1 and 2.2.2,
 * Appendix A.1): yield surface (s/sigma_0)^2 + 2 f* q1 cosh(3 q2 p /
 * (2 sigma_0)) - 1 - q3 f*^2 with normal flow, matrix equivalent plastic
 * strain eps_0^p by the work balance sigma : d eps^p = (1 - f) sigma_0
 * d eps_0^p, porosity f driven by the non-local eps_0^p and tr eps^p
 * (Eq. non-local_porosity_gurson, Chu-Needleman nucleation f_N, eps_N, s_N
 * from the initial porosity f_0), effective porosity f*(f) with coalescence
 * between f_C and f_F, capped at fstar_max < f_V* (Section 4: 0.9 f_V*).
 * The phase feeds variables nonlocal_var (alpha = eps_0^p) and
 * nonlocal_var + 1 (alpha = tr eps^p); damage fields report f*.
 * hardening (laws 1 and 3): 0 = linear, sigma_0 = sigma_y + H e; 1 = the
 * Aravas power law of Section 4.1 (Eq. aravas), sigma_0 / sigma_y =
 * (sigma_0 / sigma_y + 3 mu e / sigma_y)^N with mu this phase's shear
 * modulus and 0 < N < 1.  The remaining fields are read only when they
 * apply; reserved must be 0. */
typedef struct {
  double E, nu, sigma_y, H;
  int damage_law;
  int nonlocal_var;
  double eps_C, eps_R, D_max;
  int hardening;
  int reserved;
  double N;
  double q1, q2, q3;          /* GTN surface coefficients */
  double f_C, f_F;            /* coalescence onset, porosity at fracture */
  double f_N, eps_N, s_N;     /* Chu-Needleman nucleation (Eq. nucleation) */
  double f_0;                 /* initial porosity */
  double fstar_max;           /* cap on the effective porosity */
} rve_phase_params;

/* Solver tolerances and budgets.  The paper prints no values (Algorithm 1,
 * Algorithm 2 use a symbolic TOL); rve_default_options fills the production
 * set (tol_stag = tol_newton = 1e-6, cg_rtol 1e-3 mixed / 1e-8 FP64,
 * pcg_rtol 1e-7 mixed, the FP32 round-off level / 1e-8 FP64).  In the mixed
 * form each Newton correction is solved inexactly in FP32 while the Newton
 * residual is evaluated in FP64. */
typedef struct {
  double tol_stag;     /* staggered ERR tolerance (Algorithm 1 (iii)) */
  double tol_newton;   /* Newton residual and correction tolerance */
  double cg_rtol;      /* mechanical CG: ||r|| <= cg_rtol ||b|| */
  double pcg_rtol;     /* Helmholtz PCG: ||r|| <= pcg_rtol ||b|| (Algorithm 2) */
  int max_stag, max_newton, max_cg, max_pcg;
  int min_stag;        /* minimum staggered iterations (>= 2 so ERR compares
                          two solutions) */
  int check_every;     /* Krylov iterations launched between host checks */
} rve_solver_options;

/* Result of one load increment. */
typedef struct {
  int status;                /* rve_status of the increment */
  int increment;             /* 1-based index of the increment just solved */
  int staggered_iters;
  int newton_iters;          /* summed over staggered iterations */
  long long cg_iters;        /* mechanical CG iterations, summed */
  long long pcg_iters;       /* Helmholtz PCG iterations, summed over j */
  double err;                /* last staggered ERR */
  double voxel_iterations;   /* V * (cg_iters + pcg_iters) */
  double sigma[6];           /* <sigma>, tensor shears */
  double eps[6];             /* <eps>, tensor shears */
  double D_mean, D_max;
  int fail_stage;            /* on failure: 1 Newton budget, 2 CG, 3 PCG,
                                4 staggered budget, 5 numeric; 0 on success */
  int reserved;
} rve_step_info;

/* Precision modes: RVE_FP64 runs every operator in double precision;
 * RVE_MIXED runs FFTs, the projection, Krylov vectors and matvecs in FP32
 * while reductions (dot products, norms), the return map, the strain and
 * internal-variable state and the zero-frequency macroscopic block stay in
 * FP64. */
enum { RVE_FP64 = 0, RVE_MIXED = 1 };

/* ----------------------------------------------------------------- handle */

/* Fills *opt with the production defaults for the given precision. */
int rve_default_options(int precision, rve_solver_options* opt);

/* Creates a handle for a dim-dimensional grid n[0..dim-1] of a periodic cell
 * of size L[0..dim-1] (Section 3.2.1: voxel centres at (1/2 + n_i) L_i/N_i).
 * N1 must be even (real-to-complex transform along x1); every N_i must be a
 * product of 2, 3 and 5.  n_nonlocal = J non-local variables (0..4).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  Allocates all
 * device memory of the handle (cudaMalloc) on the current device.
 * Errors: RVE_ERR_ARG, RVE_ERR_OOM, RVE_ERR_CUDA. */
int rve_create(rve_t** out, int dim, const int n[3], const double L[3], int precision,
               int n_nonlocal, void* cuda_stream);

/* Releases every resource of the handle.  Accepts NULL. */
void rve_free(rve_t* h);

int rve_set_options(rve_t* h, const rve_solver_options* opt);

/* Phase map and per-phase laws (Sections 2.2.1 and 3.1).  phase: N3*N2*N1
 * uint8 (x1 fastest), host or device pointer, values < n_phases (<= 8).
 * ell: [J][n_phases] characteristic lengths l_j of each phase (the piecewise
 * l(x) of Eq. piecewiseell, with l_j small but nonzero outside the phase that
 * carries variable j, Section 2.2.1 remark).  Resets the state to the
 * undeformed one.  Errors: RVE_ERR_ARG (phase id out of range, bad
 * parameters), RVE_ERR_CUDA. */
int rve_set_phases(rve_t* h, const uint8_t* phase, int n_phases, const rve_phase_params* params,
                   const double* ell);

/* Macroscopic load history (Section 3.1): strain_ctrl[6] = 1 where E_hk is
 * prescribed, 0 where Sigma_HK is; target[n_incr][6] holds the prescribed
 * value of each component at the end of each increment (host pointer).  In
 * 2D, components 33, 23, 13 must be strain-controlled with target 0 (plane
 * strain).  Resets the increment counter (not the state). */
int rve_set_load_path(rve_t* h, int n_incr, const uint8_t strain_ctrl[6], const double* target);

/* Solves the next load increment by Algorithm 1 and commits it.  info may be
 * NULL.  Synchronises the stream.  On RVE_ERR_NOT_CONVERGED or
 * RVE_ERR_NUMERIC the state stays at the last converged increment. */
int rve_step_increment(rve_t* h, rve_step_info* info);

/* The next load increment with automatic cut-back of the strain increment
 * (Section 4: a variable increment, reduced where the solution needs it,
 * down to a minimum admissible size).  The path from the last converged
 * (sub-)step to the increment's target is tried whole; on
 * RVE_ERR_NOT_CONVERGED the state stays at the last converged sub-step and
 * the sub-step is halved; after each converged sub-step it doubles again
 * (capped by what is left).  Targets of both control kinds are interpolated
 * linearly along the remaining path.  The sub-step never falls below
 * 2^-max_cuts (0..60) of the path left at the call: then the call returns
 * RVE_ERR_NOT_CONVERGED with the state at the last converged sub-step, and
 * a later call (or rve_step_increment) continues from there.  info (may be
 * NULL): the last sub-step's result with the iteration counts summed over
 * every attempt; info->reserved receives the number of converged
 * sub-steps.  Other errors are returned as they occur. */
int rve_step_increment_adaptive(rve_t* h, int max_cuts, rve_step_info* info);

/* Homogenised stress / strain (volume averages, Section 3.1) of the last
 * converged increment, tensor shears, host output. */
int rve_homogenized_stress(const rve_t* h, double sigma[6]);
int rve_homogenized_strain(const rve_t* h, double eps[6]);

/* Copies a field of the last converged increment to dst (device or host
 * memory; the call returns once the copy is done), FP64, component-major.  which: 0 strain (Mandel, nc comps), 1 stress
 * (Mandel, 6 comps), 2 damage D (1), 3 non-local abar (J comps), 4 eps_p (1),
 * 5 plastic strain (Mandel, 6 comps), 6 porosity f (1; 0 outside GTN
 * phases).  For GTN phases field 2 holds f* and field 4 eps_0^p. */
int rve_get_field(const rve_t* h, int which, double* dst, size_t n_doubles);

/* Number of voxels and carried Mandel components of a handle. */
int rve_get_sizes(const rve_t* h, long long* n_voxels, int* n_comp, int* n_nonlocal);

/* Kernel-launch accounting of a handle (a profiling aid, not part of the
 * method).  Launches are counted per kernel class at all times, together
 * with their algorithmic bytes (every operand read once, every result
 * written once); with rve_profile(h, 1) each launch is also bracketed by a
 * pair of CUDA events recorded on the handle's stream and its device time
 * accumulated.  rve_profile_read fills total_ms[k], launches[k] and
 * bytes[k] for k < n_classes (any may be NULL), synchronising the stream
 * first, and returns the number of classes; rve_profile_reset zeroes them.
 * Class names come from rve_profile_class_name(k) (NULL past the last). */
int rve_profile(rve_t* h, int enable);
int rve_profile_read(rve_t* h, int n_classes, double* total_ms, long long* launches, double* bytes);
int rve_profile_reset(rve_t* h);
const char* rve_profile_class_name(int k);

/* Human-readable name of a status code (static string). */
const char* rve_status_string(int status);

/* ------------------------------------------------ operator-level calls
 * One step of the hot path each, on caller-owned DEVICE buffers in FP64
 * (converted to the handle's working precision inside).  They use the
 * handle's phase map, parameters and load-path stress mask (or pure strain
 * control if no load path is set) and do not change its increment state.
 */

/* Backward-Euler Lemaitre return map at every voxel (Appendix A.2, Eq.
 * non-local_damage_lemaitre, with the non-local variables frozen as in
 * Algorithm 1 (i)).  eps: [nc][V] Mandel total strain; epsp_n: [6][V] Mandel
 * plastic strain of the last converged increment; ep_n: [V] equivalent
 * plastic strain; abar: [J][V] non-local variables.  Outputs sigma [6][V],
 * epsp [6][V], ep [V], D [V], alpha [J][V].  Stores the tangent for
 * rve_op_tangent_apply / rve_op_matvec. */
int rve_op_return_map(rve_t* h, const double* eps, const double* epsp_n, const double* ep_n,
                      const double* abar, double* sigma, double* epsp, double* ep, double* D,
                      double* alpha);

/* The same with the history of the GTN law (law 3) given explicitly:
 * abar_n [J][V] the non-local variables of the last converged increment and
 * f_n [V] its porosity (device; NULL = the handle's converged state); the
 * new porosity goes to f [V] (device; NULL = handle scratch).  The porosity
 * of GTN voxels is (f_n + A_N(abar_0) (abar_0 - abar_0,n) + d) / (1 + d),
 * d = abar_1 - abar_1,n (Appendix A.1 with the non-local variables frozen);
 * D receives f*, ep eps_0^p, alpha eps_0^p and tr eps^p. */
int rve_op_return_map_ex(rve_t* h, const double* eps, const double* epsp_n, const double* ep_n,
                         const double* abar, const double* abar_n, const double* f_n, double* sigma,
                         double* epsp, double* ep, double* D, double* alpha, double* f);

/* tau = C_T : p with the tangent of the last rve_op_return_map (Eq.
 * lin_stress); p, tau: [nc][V]. */
int rve_op_tangent_apply(rve_t* h, const double* p, double* tau);

/* out = G*(tau) = F^-1 { G*(xi) : F(tau) } (Eq. eqdiscrete2): the Galerkin
 * projection with the rotated-scheme derivative and the zero frequency
 * projected on the stress-controlled components.  tau, out: [nc][V].
 * Errors: RVE_ERR_ARG, RVE_ERR_CUDA, RVE_ERR_TIMEOUT (a tile copy of the 3D
 * projection pass did not arrive within its wait budget). */
int rve_op_apply_gamma(rve_t* h, const double* tau, double* out);

/* Test hook of the timeout path of the 3D projection pass (not part of the
 * method): wait_s (0 < wait_s <= 60, default 2) is how long a CTA waits for
 * its tile copy before it gives up and the call returns RVE_ERR_TIMEOUT;
 * extra_tx_bytes (0..4096, default 0) are added to the byte count the
 * tile's barrier expects, which no copy delivers, so that the wait runs out
 * although the copy lands (the CTA then counts those bytes itself, so that
 * no copy is in flight when it returns).  A handle that has reported
 * RVE_ERR_TIMEOUT keeps reporting it and should be freed.
 * Errors: RVE_ERR_ARG. */
int rve_test_tile_wait(rve_t* h, double wait_s, int extra_tx_bytes);

/* Ap = G*(C_T : p), the operator of the mechanical CG (Section 3.2.2). */
int rve_op_matvec(rve_t* h, const double* p, double* Ap);

/* Solves G*(C_T : x) = b by conjugate gradients from x = 0, stopping when
 * ||r|| <= rtol ||b|| or after maxit iterations; *iters receives the count.
 * b must lie in the range of G* (for instance b = G*(t) for some t): the
 * curvature (p, G*(C_T : p)) is evaluated as (p, C_T : p), equal for
 * directions in that range. */
int rve_op_cg(rve_t* h, const double* b, double* x, double rtol, int maxit, int* iters);

/* out = L(a) = a - div(l_j^2 grad a) evaluated spectrally (Eq.
 * LhelmFourier); a, out: [V]. */
int rve_op_helmholtz_apply(rve_t* h, int j, const double* a, double* out);

/* Algorithm 2: abar = F^-1 ConjGrad(GC, M, F(alpha), rtol) for variable j;
 * alpha, abar: [V]. */
int rve_op_helmholtz_solve(rve_t* h, int j, const double* alpha, double* abar, double rtol,
                           int maxit, int* iters);

/* ------------------------------------------------ checkpoint / resume
 * The converged state after the last increment (strain, plastic strain,
 * local history variable, non-local variables, porosity and the
 * homogenised values)
 * as a self-describing byte image, so a long load path can be saved and
 * resumed (also on another handle of the same grid and variable count; the
 * phases, options and load path are not part of the image and must be set
 * on the target handle).  The image is FP64 in both forms, so an image
 * written by a mixed-precision handle loads into an FP64 handle and the
 * other way round. */

/* Bytes of the image of this handle (header + (nc + 8 + J) V doubles). */
long long rve_state_bytes(const rve_t* h);

/* Write the image into the caller's host buffer `buf` of `bytes` bytes.
 * Errors: RVE_ERR_ARG (NULL, buffer too small), RVE_ERR_STATE (phases not
 * set), RVE_ERR_CUDA. */
int rve_save_state(const rve_t* h, void* buf, long long bytes);

/* Restore an image written by rve_save_state: the next rve_step_increment
 * solves increment (saved count + 1) of the handle's load path.  The image's
 * grid and variable count must match the handle.
 * Errors: RVE_ERR_ARG (NULL, size or header mismatch), RVE_ERR_STATE
 * (phases not set), RVE_ERR_CUDA. */
int rve_load_state(rve_t* h, const void* buf, long long bytes);

/* ------------------------------------------------ graphs, autotuning, batches
 * The paper solves one RVE at a time; these calls serve many RVEs of
 * different grids advanced together on one GPU. */

/* Replay each Krylov chunk (check_every CG or PCG iterations, Algorithms 1
 * and 2) from a CUDA graph captured on its first use instead of launching
 * its kernels one by one.  Results are identical.  Captured chunks are
 * dropped by rve_set_options, rve_set_phases, rve_set_load_path and
 * rve_autotune; profiling (rve_profile) launches directly.  A capture the
 * runtime refuses falls back to direct launches.  Off by default.
 * Errors: RVE_ERR_ARG, RVE_ERR_CUDA. */
int rve_set_graphs(rve_t* h, int enable);

/* Width of the tile of the 3D projection pass (G* of Eq. eqdiscrete2 with the
 * last-axis transform, six-component handles whose last axis has 64, 128
 * or 256 points): narrow = 0 (default) moves 8 columns (FP32; 4 in FP64)
 * per CTA of 256 threads, narrow = 1 half as many per CTA of 128 threads,
 * so that twice as many CTAs share an SM.  Results are identical; only the
 * time differs (rve_autotune picks it).  Drops captured Krylov chunks.
 * Errors: RVE_ERR_ARG (h null, narrow not 0 or 1), RVE_ERR_CUDA. */
int rve_set_gamma_tile(rve_t* h, int narrow);
/* The current choice of rve_set_gamma_tile.  Errors: RVE_ERR_ARG. */
int rve_get_gamma_tile(const rve_t* h, int* narrow);

/* Pick the FFT schedule of the handle's mechanical matvec by timing:
 * for every axis transformed by the runtime mixed-radix code, each radix
 * order with the fewest stages; then the column-tile width of the strided
 * passes; then the width of the 3D projection pass's tile
 * (rve_set_gamma_tile).  Each candidate is timed over `reps` matvecs G*(C_T : p) that
 * overwrite only the Krylov scratch vectors (CUDA events on the handle's
 * stream); a candidate replaces
 * the current choice when it is at least 2 % faster.  Axes with compile-time
 * schedules (64-, 128- and 256-point y / last axes; N1 = 64, 96, 128 and
 * 256 rows) are left alone.  Allowed
 * after rve_set_phases and before the first rve_step_increment (else
 * RVE_ERR_STATE); the state is not changed.  best_ms (nullable): time of
 * one matvec with the chosen schedule; tx (nullable): chosen tile width;
 * radix (nullable): radices per axis, 0-terminated.
 * Errors: RVE_ERR_ARG, RVE_ERR_STATE, RVE_ERR_CUDA. */
int rve_autotune(rve_t* h, int reps, double* best_ms, int* tx, int radix[3][8]);

/* A batch of independent handles advanced together: each member gets its
 * own non-blocking stream (its previous stream is restored by
 * rve_batch_free) and CUDA-graph replay of its Krylov chunks, and each
 * rve_batch_step runs one increment of every member, one host worker thread
 * per member, so the members' kernels overlap on the GPU.  members: handles
 * with phases and load path set, distinct, owned by the caller, which must
 * not use them directly while the batch exists.  autotune_reps > 0 runs
 * rve_autotune(member, autotune_reps) on members that have not stepped yet.
 * Errors: RVE_ERR_ARG, RVE_ERR_STATE, RVE_ERR_CUDA, RVE_ERR_OOM. */
typedef struct rve_batch rve_batch_t;
int rve_batch_create(rve_batch_t** out, int count, rve_t* const* members, int autotune_reps);

/* One increment of every member (members whose load path is finished report
 * RVE_ERR_LOAD_PATH_END in their info and are skipped).  infos: [count],
 * filled per member as by rve_step_increment.  Returns RVE_OK when every
 * member returned RVE_OK (or had finished), else the first member's error. */
int rve_batch_step(rve_batch_t* b, rve_step_info* infos);

/* Number of members (0 for NULL). */
int rve_batch_size(const rve_batch_t* b);

/* Synchronise and release the batch; the members keep their state and get
 * their original streams back. */
void rve_batch_free(rve_batch_t* b);

/* ------------------------------------------------ adjoint over the load path
 * The paper has no adjoint; these calls give the exact derivative of the
 * discrete converged load path, for inverse problems and gradient-based
 * design.  Objective: J = <sigma_N>_11, the homogenised axial stress after
 * the last increment N of the load path.  FP64 handles only. */

/* Per-voxel factor s(x) > 0 on the Young's modulus of the voxel's phase (K
 * and mu scale with it) for the forward solve and the adjoint; s: host array
 * [V] (x1 fastest), copied; NULL removes the field (s = 1).
 * Errors: RVE_ERR_ARG (non-positive or non-finite entry), RVE_ERR_OOM,
 * RVE_ERR_CUDA. */
int rve_set_stiffness_field(rve_t* h, const double* s);

/* Forward pass of the adjoint: re-initialise the state, run every increment
 * of the load path (Algorithm 1) and keep a checkpoint of the converged
 * state after 0, k, 2k, ... increments (k = checkpoint_every) in device
 * memory owned by the handle (about (nc + 8 + J) V doubles each, plus k
 * increments' states for the recomputation).  J (nullable): the objective.
 * Errors: RVE_ERR_ARG (FP32/mixed handle, k < 1, a phase with the Aravas
 * flow stress), RVE_ERR_STATE (phases or load path not set), the step
 * errors of rve_step_increment. */
int rve_adjoint_forward(rve_t* h, int checkpoint_every, double* J);

typedef struct {
  int status;
  int increments;       /* N */
  int recomputed;       /* increments re-solved from checkpoints */
  int checkpoints;
  int transposed_staggered_iters;      /* sum over increments */
  int max_transposed_staggered_iters;
  long long cg_iters, pcg_iters;       /* adjoint linear solves */
} rve_adjoint_info;

/* Reverse pass after rve_adjoint_forward: for n = N .. 1, re-solve the
 * increments of each checkpoint segment from its checkpoint, then solve the
 * adjoint of increment n: the transposed staggered scheme alternates
 *   P C_T lambda_n = P [d(sigma, alpha, h)/d eps]^T (s_n, mu_n, eta_n)   (CG
 *     on G* C_T, Eqs. eqdiscrete2 / lin_stress; P = G*, lambda_n in the
 *     compatible, mixed-control space)
 *   L_j mu_{n,j} = [d sigma / d abar_j]^T (s_n - lambda_n)   (Algorithm 2)
 * until both change by at most tol_stag (relative, max_stag sweeps), with
 * s_N = dJ e_11 / V, s_n = 0 before, and carries the history adjoint
 * eta_{n-1} = [d(sigma, alpha, h_n)/d h_{n-1}]^T (s_n - lambda_n, mu_n,
 * eta_n).  The linear solves use cg_rtol / pcg_rtol and max_cg / max_pcg of
 * the handle's options.  Outputs, each scaled by dJ (the upstream
 * derivative), any may be NULL:
 *   grad_params [n_phases][4]: dJ/d(sigma_y, H, eps_C, eps_R) per phase
 *     (kappa_C, kappa_R in the eps_C, eps_R slots of cracking phases);
 *   grad_ell [J]: dJ/dl_j, l_j the largest entry of row j of the length
 *     table, the whole row scaling with it;
 *   grad_stiff [V] (host): dJ/ds(x) at the current stiffness field.
 * The handle is left at the converged state after increment N (its
 * per-voxel sigma and D buffers hold the last adjoint linearisation).
 * Errors: RVE_ERR_STATE (no forward pass), RVE_ERR_NOT_CONVERGED,
 * RVE_ERR_NUMERIC, RVE_ERR_CUDA. */
int rve_adjoint_backward(rve_t* h, double dJ, double* grad_params, double* grad_ell, double* grad_stiff,
                         rve_adjoint_info* info);

/* ------------------------------------------------ allocation-free variant
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory, such as an application that hands
 * all device memory out of its own pool at start-up and forbids later
 * cudaMalloc calls, or a plug-in running inside a host framework that owns
 * the device's memory.  Such a caller cannot create a handle (rve_create
 * allocates), so this call computes the same out = G*(tau) as
 * rve_op_apply_gamma (FP64) without one, and allocates
 * nothing: its half-spectrum scratch (32 MiB) and its FFT tables sit in
 * static device arrays that every GPU which loads the library holds until
 * the process exits.
 *  - dim, n, L: grid as in rve_create (N1 even, axes products of 2, 3, 5,
 *    every axis <= 1024); strain_ctrl[6]: 1 where the mean strain is
 *    prescribed (the zero frequency keeps the other, stress-controlled,
 *    components), as in rve_set_load_path.
 *  - tau, out: caller-owned DEVICE buffers [nc][V] (Mandel, FP64).
 *  - cuda_stream: the stream the work is enqueued on; the call returns after
 *    synchronising it.
 *  - Grids whose FP64 half spectrum (nc * N3 * N2 * ps * 16 bytes, ps = N1/2+1
 *    rounded up to 16) exceeds 32 MiB, e.g. beyond 64^3 in 3D, are rejected
 *    with RVE_ERR_ARG before any device work.
 *  - The first call on a device (with that device current) looks up the
 *    static arrays' device addresses.  Every call copies the grid's tables
 *    from host memory and synchronises the stream, so the call must not be
 *    made while its stream (or, in global capture mode, any stream) is being
 *    captured into a CUDA graph.
 *  - Every call shares the same static scratch, tables and wait flag, which
 *    keep the last call's contents (the call clears the flag itself): calls
 *    that overlap on the GPU (other streams, other host threads) race and
 *    must be serialised by the caller.
 * Errors: RVE_ERR_ARG, RVE_ERR_CUDA, RVE_ERR_TIMEOUT (a tile copy of the 3D
 * projection pass did not arrive within its wait budget; out is then
 * incomplete). */
int rve_op_apply_gamma_noalloc(int dim, const int n[3], const double L[3], const uint8_t strain_ctrl[6],
                               const double* tau, double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* RVE_H */
