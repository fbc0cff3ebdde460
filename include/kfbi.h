/*
 * kfbi.h -- C ABI of the GB300 (sm_103a) KFBI operator-application library.
 *
 * The library implements the hot path of the GPU-accelerated kernel-free
 * boundary integral (KFBI) method of Tan, Huang and Ying (arXiv 2404.14864):
 * one application of the boundary-integral operator of the Dirichlet BIE
 * (Eq. 3.17), i.e. Procedure 2 of Sec. 3.3 --
 *   (a) jumps at the interface (Eq. 3.35 and the 3x3 system of Sec. 3.2.5)
 *       and the corrected five-point right-hand side (Sec. 3.2.4),
 *   (b) the box solve of Delta_h u - kappa u = R with u = 0 on the box
 *       (Eq. 3.31) by DST-I transforms and an eigenvalue division
 *       (Sec. 3.4.2),
 *   (c) extraction of u+ at the boundary nodes (Eq. 3.36, Sec. 3.2.6) --
 * and the time steppers of Sec. 3.1 / Procedure 3 that call it inside a
 * GMRES solve of the BIE (the Krylov alternative named in Sec. 5).
 *
 * Conventions (all entry points):
 *  - Plain C types only.  Device pointers are CUDA global-memory pointers
 *    owned by the caller; the library never frees them.  Everything reached
 *    through an opaque handle is owned by the library.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on it; kfbi_create_domain, the
 *    kfbi_step_* calls and kfbi_destroy_* synchronise the stream before
 *    returning (the step calls read GMRES convergence scalars on the host).
 *  - Grid arrays exchanged with the caller are the (M-1) x (M-1) interior
 *    nodes x_i = lo + i h, y_j = lo + j h, i, j = 1..M-1, h = (hi - lo)/M,
 *    row-major with y slow: element (j-1)*(M-1) + (i-1).
 *  - Boundary arrays have n_boundary entries, node k at curve parameter
 *    2 pi k / n_boundary.
 *  - Complex data are interleaved (re, im) pairs of doubles (complex128).
 *    An operator call is complex iff kappa_im != 0.
 *  - Every call returns a kfbi_status; the library never aborts or exits.
 *    On failure the message is available from kfbi_last_error(dom) (or
 *    kfbi_last_global_error() when no domain exists yet).
 */
#ifndef KFBI_H
#define KFBI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KFBI_OK = 0,
  KFBI_ERR_ARG = 1,           /* invalid argument or size */
  KFBI_ERR_GEOMETRY = 2,      /* interface too close to the box, bad stencil */
  KFBI_ERR_OOM = 3,           /* device allocation failed or admission refused */
  KFBI_ERR_NOT_CONVERGED = 4, /* GMRES reached gmres_maxit */
  KFBI_ERR_NONFINITE = 5,     /* NaN/Inf in a residual */
  KFBI_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  KFBI_ERR_CUDA = 7,          /* a CUDA runtime/driver call failed */
  KFBI_ERR_UNSUPPORTED = 8    /* feature not available in this build */
} kfbi_status;

typedef enum {
  KFBI_FP64 = 0,        /* plain path: every kernel in float64 */
  KFBI_MIXED_TF32 = 1,  /* DST on tcgen05 tensor cores, TF32 split in 3
                           passes with FP32 accumulation; correction and
                           extraction in FP32; GMRES in FP64 */
  KFBI_MIXED_FFT32 = 2  /* DST-I by FP32 FFT on the CUDA cores (M = 32 N1,
                           N1 in {2, 4, 6, 8, 12, 16, 24, 32, 48, 64}, i.e.
                           64 <= M <= 2048 with M / 32 a power of two or
                           three times one; otherwise KFBI_ERR_UNSUPPORTED at
                           creation); correction, extraction, GMRES and
                           refinement as KFBI_MIXED_TF32 */
} kfbi_precision;

typedef enum {
  KFBI_CURVE_POLAR = 0,  /* z(t) = c + r(t)(cos t, sin t),
                            r(t) = params[0] + params[1] sin(params[2] t + params[3]) */
  KFBI_CURVE_ELLIPSE = 1 /* z(t) = c + Rot(params[2]) (params[0] cos t, params[1] sin t) */
} kfbi_curve_kind;

typedef struct {
  int M;               /* grid intervals per side (unknowns (M-1)^2), 8 <= M <= 4096 */
  double box_lo;       /* box [box_lo, box_hi]^2 */
  double box_hi;
  int n_boundary;      /* boundary nodes, 16 <= n_boundary <= 16384 */
  int curve_kind;      /* kfbi_curve_kind */
  double cx, cy;       /* curve centre */
  double params[6];    /* curve parameters (see kfbi_curve_kind) */
  int precision;       /* kfbi_precision */
  int gmres_restart;   /* GMRES restart length m, 1..64 */
  double gmres_tol;    /* stop when ||r||_2 <= gmres_tol * ||b||_2 */
  int gmres_maxit;     /* total GMRES iterations per solve */
  int solver;          /* kfbi_solver: how the density equation is solved;
                          0 (a zero-initialised description) = GMRES */
  double richardson_gamma; /* KFBI_RICHARDSON step gamma, 0 < gamma < 2 */
} kfbi_domain_desc;

/* Iterative solver of the density equation (Eq. 3.17) behind
 * kfbi_solve_density and the time steppers of one domain.  gmres_tol and
 * gmres_maxit bound both (for Richardson, maxit counts its updates).
 *   KFBI_GMRES      restarted GMRES(gmres_restart), CGS2 Arnoldi in FP64.
 *   KFBI_RICHARDSON the Richardson iteration of Eq. 3.21,
 *                   phi <- phi + gamma (b - A phi), one operator application
 *                   and one fused residual/update kernel per iteration.  The
 *                   paper takes gamma in (0, 1); it converges whenever
 *                   |1 - gamma lambda| < 1 on the spectrum of A = 1/2 I + W,
 *                   so 0 < gamma < 2 is accepted.  Single domains only:
 *                   batches and the server refuse such domains. */
typedef enum { KFBI_GMRES = 0, KFBI_RICHARDSON = 1 } kfbi_solver;

typedef struct {
  int iters;           /* solver iterations (GMRES: operator applications inside
                          GMRES; Richardson: updates of phi) */
  double rel_residual; /* final rotated-residual estimate / ||b|| */
  int converged;       /* 1 if rel_residual <= gmres_tol */
  int applications;    /* operator applications in the step (GMRES + 2) */
} kfbi_solve_info;

typedef struct kfbi_domain kfbi_domain; /* opaque, library-owned */
typedef struct kfbi_state kfbi_state;   /* opaque, library-owned time-level fields */
typedef struct kfbi_plan kfbi_plan;     /* opaque, host-only setup tables */

/* ---- setup (Procedure 1 of Sec. 3.3) ------------------------------------ */

/* Build the geometry (boundary nodes, inside mask, irregular nodes, cut-edge
 * intersections), the per-target coefficient tables and the DST tables on
 * the host, upload them once to the current CUDA device and allocate the
 * domain's work buffers.  Synchronous.  Errors: KFBI_ERR_ARG (sizes),
 * KFBI_ERR_GEOMETRY (interface closer than 2h to the box, empty stencil),
 * KFBI_ERR_OOM, KFBI_ERR_CUDA.  On error *out is NULL. */
kfbi_status kfbi_create_domain(const kfbi_domain_desc* desc, void* stream, kfbi_domain** out);
void kfbi_destroy_domain(kfbi_domain* dom);

/* ---- the hot path (Procedure 2 of Sec. 3.3) ----------------------------- */

/* out_dev[k] = u+(z_k): interior limit at boundary node k of the solution u
 * of the interface problem (Eq. 3.30) Delta u - kappa u = f-tilde off Gamma,
 * [u] = phi, [u_n] = 0 on Gamma, u = 0 on the box.
 *   phi_dev : n_boundary doubles (complex128 if kappa_im != 0), device.
 *   f_dev   : (M-1)^2 grid of f (same type as phi) or NULL for f = 0; values
 *             at nodes outside Omega are ignored (f-tilde of Eq. 3.25).
 *   out_dev : n_boundary doubles (complex128 if kappa_im != 0), device.
 * kappa = kappa_re + i kappa_im; (lambda_a + lambda_b - kappa) must not
 * vanish for any DST mode (true for kappa_re > 0 or kappa_im != 0).
 * Asynchronous on `stream`; uses the domain's work buffers, so calls on one
 * domain must not overlap. */
kfbi_status kfbi_apply_operator(kfbi_domain* dom, double kappa_re, double kappa_im,
                                const void* phi_dev, const void* f_dev, void* out_dev,
                                void* stream);

/* As kfbi_apply_operator, and also writes the grid solution u of Eq. 3.30 at
 * all (M-1)^2 interior nodes (inside and outside Omega) to u_grid_dev (same
 * element type).  u_plus_dev may be NULL. */
kfbi_status kfbi_interface_solve(kfbi_domain* dom, double kappa_re, double kappa_im,
                                 const void* phi_dev, const void* f_dev, void* u_grid_dev,
                                 void* u_plus_dev, void* stream);

/* Solve the Dirichlet BIE (Eq. 3.17) (1/2 I + W) phi = b with the domain's
 * solver (kfbi_solver: GMRES(m) with FP64 Arnoldi (CGS2) and Givens
 * rotations, or the Richardson iteration of Eq. 3.21) and operator;
 * phi_dev holds the initial guess on entry and the solution on exit.
 * Synchronous.  KFBI_ERR_NOT_CONVERGED if gmres_maxit is reached. */
kfbi_status kfbi_solve_density(kfbi_domain* dom, double kappa_re, double kappa_im,
                               const void* b_dev, void* phi_dev, kfbi_solve_info* info,
                               void* stream);

/* ---- Neumann BVP (Eqs. 3.19, 3.20, 3.22) ---------------------------------
 * Delta u - kappa u = f in Omega, d_n u = g_N on Gamma (n the outward
 * normal), on domains of every precision (mixed domains iterate with the
 * fast operator and refine with the float64 one, as for Dirichlet data).
 * The box condition is u = 0 on the box (the Green's function of the
 * Dirichlet box; the solution in Omega does not depend on that choice). */

/* out_dev[k] = d_n u+(z_k): interior normal derivative at boundary node k of
 * the solution of the interface problem (Eq. 3.30) with [u] = 0,
 * [u_n] = psi, F = f-tilde (f_dev may be NULL).  With f = 0 this is the
 * Neumann BIE operator psi/2 - d_n (V psi) of Eq. 3.19 (u = -V psi).
 * Layouts and types as kfbi_apply_operator.  Asynchronous on `stream`. */
kfbi_status kfbi_apply_neumann(kfbi_domain* dom, double kappa_re, double kappa_im,
                               const void* psi_dev, const void* f_dev, void* out_dev,
                               void* stream);

/* Solve the Neumann BVP: b = g_N - d_n (Y f)+, the BIE of Eq. 3.19 for psi
 * with the domain's solver (GMRES or the Richardson iteration of Eq. 3.22),
 * then u = Y f - V psi (Eq. 3.20) on the grid.
 *   gn_dev     : n_boundary values of g_N (complex128 if kappa_im != 0).
 *   f_dev      : (M-1)^2 grid of f or NULL (values outside Omega ignored).
 *   psi_dev    : n_boundary, initial guess on entry, density on exit.
 *   u_grid_dev : (M-1)^2 grid solution on exit (NULL: not formed).
 * Synchronous.  KFBI_ERR_NOT_CONVERGED if gmres_maxit is reached. */
kfbi_status kfbi_solve_neumann(kfbi_domain* dom, double kappa_re, double kappa_im,
                               const void* gn_dev, const void* f_dev, void* psi_dev,
                               void* u_grid_dev, kfbi_solve_info* info, void* stream);

/* Allocation-free box solve, for callers that cannot allocate device memory
 * (code that runs where cudaMalloc is not allowed, e.g. inside a graph
 * capture it does not own, or a plugin whose host program owns every device
 * allocation).  The paper has no counterpart to this entry point.
 * Solves (D_xx + D_yy - kappa) u = rhs on the (M-1)^2 interior nodes of the
 * box [box_lo, box_hi]^2 with u = 0 on the box boundary (the five-point
 * operator of the box solve) by float64 DST-I passes, without a domain.
 *   rhs_dev, u_dev : (M-1)^2 doubles, complex128 if kappa_im != 0, caller
 *                    layout, device memory owned by the caller.
 * Work space is a static device array of 2.5 MiB that every GPU loading the
 * library holds until exit, so M - 1 <= 256; larger M returns KFBI_ERR_ARG.
 * The first call in a device's context looks up the array's address (call
 * it once before any stream capture); after cudaDeviceReset, or from
 * another context, the next call looks it up again.  All calls share the
 * array, so calls that overlap on the GPU race.  Allocates nothing;
 * asynchronous on `stream`. */
kfbi_status kfbi_box_solve_noalloc(int M, double box_lo, double box_hi, double kappa_re,
                                   double kappa_im, const void* rhs_dev, void* u_dev,
                                   void* stream);

/* ---- time stepping (Sec. 3.1, Procedure 3) ------------------------------ */

typedef enum { KFBI_HEAT = 0, KFBI_WAVE = 1, KFBI_SCHRODINGER = 2 } kfbi_equation;

kfbi_status kfbi_state_create(kfbi_domain* dom, int equation, kfbi_state** out);
void kfbi_state_destroy(kfbi_state* st);

/* Heat u_t = Delta u + s, Crank-Nicolson (Eqs. 3.1-3.4), kappa = 2/dt:
 * F^1 = (2/dt) u0 + lap_u0 + src_sum (src_sum = s^0 + s^1 or NULL). */
kfbi_status kfbi_state_init_heat(kfbi_state* st, double dt, const double* u0_dev,
                                 const double* lap_u0_dev, const double* src_sum_dev,
                                 void* stream);
/* Wave u_tt = Delta u, theta-scheme (Eq. 3.5), kappa = 1/(theta dt^2);
 * the state starts at time level 1: u1 is the current field. */
kfbi_status kfbi_state_init_wave(kfbi_state* st, double dt, double theta, const double* u0_dev,
                                 const double* lap_u0_dev, const double* u1_dev,
                                 const double* lap_u1_dev, void* stream);
/* Schroedinger -i u_t + Delta u + v u + w|u|^2 u = 0 (Eq. 2.2), Strang
 * splitting (Eqs. 3.8-3.12), kappa = 2i/dt; u0, lap_u0 complex128. */
kfbi_status kfbi_state_init_schrodinger(kfbi_state* st, double dt, const void* u0_dev,
                                        const void* lap_u0_dev, void* stream);

/* One heat step: solve for u^{n+1} with Dirichlet data g_next_dev
 * (n_boundary doubles at t^{n+1}), then F^{n+2} = (4/dt) u^{n+1} - F^{n+1}
 * + src_sum_next (s^{n+1} + s^{n+2} on the grid, or NULL).  info may be NULL. */
kfbi_status kfbi_step_heat(kfbi_domain* dom, kfbi_state* st, const double* g_next_dev,
                           const double* src_sum_next_dev, kfbi_solve_info* info,
                           void* stream);
/* One wave step: u^{n+1} with data g_next_dev, then
 * F^{n+2} = (kappa/theta) u^{n+1} - ((1-2theta)/theta) F^{n+1} - F^n. */
kfbi_status kfbi_step_wave(kfbi_domain* dom, kfbi_state* st, const double* g_next_dev,
                           kfbi_solve_info* info, void* stream);
/* One Strang step of -i u_t + Delta u + v u + w |u|^2 u = 0 (Eq. 2.2):
 * the pointwise Crank-Nicolson step of Eq. 3.10,
 * u** = ((1 - i a)/(1 + i a)) u* with a = (dt/2)(v + w |u*|^2) (the
 * modulus-preserving root of Eq. 3.10, which the paper's Newton iteration
 * reaches from u*; unique while dt |w| |u|^2 / 2 < 1), then Eq. 3.12 for
 * u^{n+1} with data g_next_dev (complex128), then u* = 2 u^{n+1} - u**.
 * v_dev: (M-1)^2 doubles (the potential v); w: real, finite (else
 * KFBI_ERR_ARG).  Batched steps take each state's kfbi_state_set_w; the
 * server steps Schroedinger requests with w = 0. */
kfbi_status kfbi_step_schrodinger(kfbi_domain* dom, kfbi_state* st, const double* v_dev,
                                  double w, const void* g_next_dev, kfbi_solve_info* info,
                                  void* stream);

/* Boundary condition of the state's steps: neumann = 0 (default) takes
 * g_next as Dirichlet data u = g (Eq. 3.17), neumann = 1 as Neumann data
 * d_n u = g with the outward normal (Eq. 3.19; the density is then psi and
 * u = Y f - V psi, Eq. 3.20).  Resets the density to zero.  Batches and
 * the server take Dirichlet states only (KFBI_ERR_ARG). */
kfbi_status kfbi_state_set_neumann(kfbi_state* st, int neumann);

/* Nonlinear coefficient w of a Schroedinger state's batched steps
 * (kfbi_batch_step takes no w; single steps pass theirs to
 * kfbi_step_schrodinger).  Default 0; KFBI_ERR_ARG for another equation or
 * a non-finite w. */
kfbi_status kfbi_state_set_w(kfbi_state* st, double w);

/* Checkpoint and resume: the state's time-level data (fields, densities,
 * extrapolation history, superposition caches, step parameters) as one
 * host blob of kfbi_state_blob_bytes bytes (caller-owned host memory).
 * Importing into a state of the same equation on a domain with the same
 * description continues the run bit for bit.  Both synchronous; import
 * returns KFBI_ERR_ARG for a blob of another equation, grid, node count or
 * domain precision. */
long long kfbi_state_blob_bytes(const kfbi_state* st);
kfbi_status kfbi_state_export(kfbi_state* st, void* host_buf, long long bytes);
kfbi_status kfbi_state_import(kfbi_state* st, const void* host_buf, long long bytes);

/* Copy the current field u^n (all (M-1)^2 nodes; values outside Omega are
 * the exterior part of the interface solution) or the current density. */
kfbi_status kfbi_state_get_u(kfbi_state* st, void* u_out_dev, void* stream);
kfbi_status kfbi_state_get_phi(kfbi_state* st, void* phi_out_dev, void* stream);

/* ---- batched time steps ------------------------------------------------- */

/* A batch groups n mixed-precision domains of one device (KFBI_MIXED_TF32
 * and KFBI_MIXED_FFT32 in any mix; any sizes and curves, same
 * gmres_restart) so that one time step of all of them runs as grouped
 * launches (Sec. 3.4.2's box solve and Procedure 2's operator application
 * for many instances at once): the tcgen05 DST passes of every TF32
 * instance are one persistent launch over all their tiles, the FFT passes
 * of the FFT32 instances one launch per grid size, every other kernel takes
 * the instance from its grid, and one lockstep GMRES iteration of the whole
 * batch is a CUDA graph replayed until every instance has converged.  The
 * first step binds the states, runs the autotuner (below) and captures the
 * graph.
 * An instance's result does not depend on what it is batched with (same
 * bits alone or in any mix); against kfbi_step_* on its own domain it agrees
 * to the GMRES tolerance (reduction orders differ).
 * The domains must outlive the batch. */
typedef struct kfbi_batch kfbi_batch;
kfbi_status kfbi_batch_create(kfbi_domain* const* domains, int n, void* stream, kfbi_batch** out);
void kfbi_batch_destroy(kfbi_batch* batch);
/* One time step of every instance: states[i] (initialised, on domains[i])
 * advances with Dirichlet data g_next_dev[i] (n_boundary doubles, or
 * complex128 for Schroedinger).  src_or_v_dev[i]: the heat source sum
 * s^{n+1} + s^{n+2} (or NULL), the Schroedinger potential v (required), or
 * unused for the wave equation; src_or_v_dev itself may be NULL.
 * infos: n entries or NULL.  Synchronous. */
kfbi_status kfbi_batch_step(kfbi_batch* batch, kfbi_state* const* states,
                            const void* const* g_next_dev, const double* const* src_or_v_dev,
                            kfbi_solve_info* infos, void* stream);
/* Autotuner result for the TF32 instances: chosen tile order (0 as given,
 * 1 largest instances first) and the measured microseconds of the grouped
 * fast passes for the first candidate of each order. */
kfbi_status kfbi_batch_tuning(const kfbi_batch* batch, int* tile_order, double* us_natural,
                              double* us_largest_first);
/* One autotuned group.  The autotuner times each candidate launch shape of
 * a group on the group's fast application (the passes one GMRES iteration
 * runs; CUDA events, one warm-up and three timed repetitions) and keeps the
 * fastest:
 *   engine 1: the FFT32 instances of grid size M; candidates: rows (warps)
 *             per block of the FFT passes, param[c][0] in {8, 4};
 *   engine 0: all TF32 instances; candidates: param[c][0] tile order (0 as
 *             given, 1 largest first), param[c][1] persistent CTAs of the
 *             tensor passes (one per SM, or half as many).
 * No candidate changes the arithmetic of a tile or a row, so an instance's
 * bits do not depend on the choice (split K, which would, follows the tile
 * count: CTA pairs when a pass's tiles fill at most half of the SMs).
 * FFT choices are cached per M and kept across rebinds; a grid size new to
 * the batch is tuned at its first step. */
typedef struct {
  int engine;        /* 0 TF32 tensor passes, 1 FFT passes */
  int M;             /* grid size of an FFT group (0 for TF32) */
  int instances;     /* instances in the group */
  int n_candidates;  /* candidates considered (at most 4) */
  int chosen;        /* index of the kept candidate */
  int param[4][2];   /* the candidates' launch parameters (see above) */
  double us[4];      /* measured microseconds per candidate (0 when forced) */
} kfbi_batch_tuning_t;
int kfbi_batch_tuning_count(const kfbi_batch* batch);
kfbi_status kfbi_batch_tuning_get(const kfbi_batch* batch, int i, kfbi_batch_tuning_t* out);
/* candidate >= 0: skip the timing and use candidate (modulo each group's
 * candidate count) in every group from the next step on, so that every
 * configuration can be checked; -1 restores the autotuner.  KFBI_ERR_ARG
 * for candidate < -1. */
kfbi_status kfbi_batch_force_candidate(kfbi_batch* batch, int candidate);
const char* kfbi_batch_last_error(const kfbi_batch* batch);

/* ---- inspection and diagnostics ----------------------------------------- */

const char* kfbi_last_error(const kfbi_domain* dom);
const char* kfbi_last_global_error(void);
/* Number of CUDA kernels this library has launched since it was loaded. */
long long kfbi_launch_count(void);
/* Device bytes held by the domain (work buffers + its own tables; the DST-I
 * tables shared by all domains on one grid are counted by
 * kfbi_table_cache_bytes). */
long long kfbi_domain_device_bytes(const kfbi_domain* dom);
/* Device bytes held by a state's time-level fields and vectors. */
long long kfbi_state_device_bytes(const kfbi_state* st);
/* Device bytes of the shared DST-I tables (S and eigenvalues, and their
 * TF32/FP32 forms) alive for all grids (M, h) in use. */
long long kfbi_table_cache_bytes(void);

/* Kernel timing with CUDA events recorded on the launching stream around
 * every launch of the enabled kernel classes (off by default).
 * kfbi_profile_enable takes a bit mask of kfbi_prof_class bits (1 << cls;
 * 0 disables); each timed launch adds two event records.
 * kfbi_profile_read synchronises the recorded events and returns the launch
 * count and summed duration of one class. */
typedef enum {
  KFBI_PROF_DST = 0,     /* one DST-I pass (GEMM) of the box solve */
  KFBI_PROF_CORRECT = 1, /* corrected right-hand side */
  KFBI_PROF_EXTRACT = 2, /* boundary extraction */
  KFBI_PROF_KRYLOV = 3,  /* GMRES kernels */
  KFBI_PROF_GRID = 4,    /* elementwise grid kernels (steppers, layout) */
  KFBI_PROF_SPARSE = 5,  /* first DST pass of a sparse right-hand side (CUDA cores) */
  KFBI_PROF_NCLASS = 6
} kfbi_prof_class;
void kfbi_profile_enable(int class_mask);
void kfbi_profile_reset(void);
kfbi_status kfbi_profile_read(int cls, long long* launches, double* total_ms);
/* Floating-point operations the recorded launches of a class issued, for
 * the classes whose launches count them (KFBI_PROF_DST: the executed dense
 * products of each pass, three TF32 products per pass on a mixed domain). */
kfbi_status kfbi_profile_work(int cls, double* flops);
/* Algorithmic bytes the recorded launches of a class move (counted by the
 * launches that declare them: the FFT DST passes count the rows they read
 * and write, 4 (M - 1) bytes per row each way; a first pass built from the
 * irregular nodes counts only its writes). */
kfbi_status kfbi_profile_bytes(int cls, double* bytes);

/* Self-check of the FP32 <-> FP64 conversions the refinement kernels do on
 * the integer and FP32 pipes (the GPU's FP64 pipe is narrow): on the current
 * device, n seeded bit patterns (doubles of every exponent, rounding ties
 * and carries; floats of every exponent) are converted both ways and by the
 * hardware conversions, and *mismatches receives the number of results whose
 * bits differ (0 expected).  Synchronous on `stream` (NULL: the legacy
 * default stream).  KFBI_ERR_ARG for n < 1 or a NULL mismatches pointer. */
kfbi_status kfbi_check_conversions(unsigned long long seed, long long n, long long* mismatches,
                                   void* stream);

/* Self-check of the bounded device-side waits (the tensor-core passes'
 * pipeline waits give up after a cycle limit, record the failure in the
 * domain's error word, and the call returns KFBI_ERR_TIMEOUT): one block
 * waits, with the same wait routine and a limit of `seconds`, on an mbarrier
 * that nothing completes.  Returns KFBI_ERR_TIMEOUT when the wait gave up as
 * designed (the expected result; the device stays usable), KFBI_OK if the
 * wait completed, KFBI_ERR_ARG unless 0 < seconds <= 1.  Synchronous on
 * `stream`. */
kfbi_status kfbi_check_wait_timeout(double seconds, void* stream);

/* Host-only plan: the geometry and coefficient tables kfbi_create_domain
 * uploads, built without touching the GPU, for inspection and tests. */
typedef enum {
  KFBI_PLAN_N_EDGES = 0,     /* count: cut edges */
  KFBI_PLAN_EDGE_I = 1,      /* int32[n_edges]: i of the lower/left endpoint */
  KFBI_PLAN_EDGE_J = 2,      /* int32[n_edges]: j of the lower/left endpoint */
  KFBI_PLAN_EDGE_DIR = 3,    /* int32[n_edges]: 0 along x, 1 along y */
  KFBI_PLAN_EDGE_COORD = 4,  /* double[n_edges]: intersection coordinate on the edge's line */
  KFBI_PLAN_EDGE_THETA = 5,  /* double[n_edges]: curve parameter of the intersection */
  KFBI_PLAN_INSIDE = 6,      /* uint8[(M+1)^2]: inside mask, [j*(M+1)+i] */
  KFBI_PLAN_N_IRREGULAR = 7, /* count: irregular nodes */
  KFBI_PLAN_IRREGULAR = 8,   /* int32[n_irr]: interior index (j-1)*(M-1)+(i-1), ascending */
  KFBI_PLAN_N_ARMS = 9,      /* count: correction arms (two per cut edge) */
  KFBI_PLAN_ARM_NODE = 10,   /* int32[n_arms]: index into the irregular list */
  KFBI_PLAN_ARM_K0 = 11,     /* int32[n_arms]: first density node of the 6-point stencil */
  KFBI_PLAN_ARM_ALPHA = 12,  /* double[n_arms*6]: kappa-free density weights (scaled by s/h^2) */
  KFBI_PLAN_ARM_BETA = 13,   /* double[n_arms*6]: density weights multiplying kappa */
  KFBI_PLAN_ARM_FIDX = 14,   /* int32[n_arms*2]: interior indices of the f extrapolation */
  KFBI_PLAN_ARM_FCOEF = 15,  /* double[n_arms*2]: their coefficients */
  KFBI_PLAN_NODE_GIDX = 16,  /* int32[nb*6]: interior indices of the extraction stencil */
  KFBI_PLAN_NODE_W = 17,     /* double[nb*6]: extraction weights on U */
  KFBI_PLAN_NODE_A = 18,     /* double[nb*6]: kappa-free density weights, nodes k-2..k+3 */
  KFBI_PLAN_NODE_B = 19,     /* double[nb*6]: density weights multiplying kappa */
  KFBI_PLAN_NODE_FIDX = 20,  /* int32[nb]: interior index of f at the node */
  KFBI_PLAN_NODE_FCOEF = 21, /* double[nb]: its coefficient */
  KFBI_PLAN_ARM_DELTA = 22,  /* double[n_arms*6]: weights of the Neumann density psi */
  KFBI_PLAN_NODE_WN = 23,    /* double[nb*6]: normal-derivative extraction weights on U */
  KFBI_PLAN_NODE_E = 24,     /* double[nb*6]: psi weights of d_n u+, nodes k-2..k+3 */
  KFBI_PLAN_NODE_FCOEF_N = 25 /* double[nb]: coefficient of f (at NODE_FIDX) in d_n u+ */
} kfbi_plan_field;

kfbi_status kfbi_plan_create(const kfbi_domain_desc* desc, kfbi_plan** out);
void kfbi_plan_destroy(kfbi_plan* plan);
/* Element count of a field (or the value of a count field). */
long long kfbi_plan_size(const kfbi_plan* plan, int field);
/* Copy a field into host memory dst (kfbi_plan_size elements of its type). */
kfbi_status kfbi_plan_export(const kfbi_plan* plan, int field, void* dst);
/* Exact device bytes that a domain created from this plan's description
 * plus one state of the given equation hold (kfbi_domain_device_bytes +
 * kfbi_state_device_bytes), computed on the host; -1 on bad arguments. */
long long kfbi_plan_device_bytes(const kfbi_plan* plan, int equation);

/* ---- served stream (continuous batching) --------------------------------- */

/* A server runs many independent time-stepping requests (heat, wave and
 * Schroedinger solves of any grid size and domain) on one device.  A request
 * is admitted when its arrival time has passed, a slot is free
 * (max_resident) and its exact device bytes fit both the server's budget and
 * the device's free memory less hbm_reserve_bytes; admission is first come
 * first served (a request that does not fit holds back later ones).  On
 * admission its domain, state, boundary data and source/potential are made
 * resident on the device.  Each tick then advances every resident request
 * by one time step in one batch step (kfbi_batch_step semantics: grouped
 * launches, lockstep GMRES), so requests that arrive while others run join
 * at the next tick and share their launches.  A request that has taken all
 * its steps is retired: its final field is copied to its host u_out and its
 * device memory is freed for the next admissions.  A request's result does
 * not depend on the other requests it ran with.
 * Lanes: with lanes > 1 requests are split by padded grid size (up to 512,
 * up to 1024, larger; lane = min(class, lanes - 1)), each lane with its own
 * batch, stream and admission queue under the shared slot and byte limits.
 * kfbi_server_run drives every lane from its own host thread, so small
 * requests are not held to the pace of the largest grid; kfbi_server_tick
 * steps the lanes one after another.  Tick indices in kfbi_request_info
 * count the request's lane's ticks.
 * Host threads (plan_threads) build the host plans of arrived requests
 * while the device works; with plan_threads = 0 plans are built at
 * admission.  Submit, tick and run are called from one thread. */
typedef struct kfbi_server kfbi_server;

typedef struct {
  int max_resident;            /* requests on the device at once, 1..4096 */
  long long hbm_budget_bytes;  /* device bytes the resident requests may hold;
                                  0 = the free memory at creation less hbm_reserve_bytes */
  long long hbm_reserve_bytes; /* free device memory every admission leaves untouched */
  int gmres_restart;           /* GMRES restart shared by all requests (lockstep batch) */
  int plan_threads;            /* host threads building request plans, 0..64 */
  int lanes;                   /* size lanes, 0..3 (0 and 1: one lane on the given stream;
                                  more: one stream and host thread per lane) */
} kfbi_server_desc;

typedef struct {
  kfbi_domain_desc domain; /* precision KFBI_MIXED_TF32 or KFBI_MIXED_FFT32 (M with an FFT
                              pass, else KFBI_ERR_UNSUPPORTED at submission);
                              gmres_restart = the server's */
  int equation;            /* kfbi_equation */
  int steps;               /* time steps, >= 1 */
  double dt;               /* time step */
  double theta;            /* theta of the wave scheme (wave only) */
  double arrival;          /* arrival time, seconds on the server clock */
  /* Host buffers read at admission; they must stay valid until the request
   * is resident.  Grids are (M-1)^2 row-major interior values, float64, or
   * complex128 interleaved for the Schroedinger equation. */
  const void* u0;          /* u at t_0 */
  const void* lap_u0;      /* Laplacian of u at t_0 */
  const double* u1;        /* wave: u at t_1 */
  const double* lap_u1;    /* wave: Laplacian of u at t_1 */
  const void* g;           /* steps x n_boundary Dirichlet values at t_1..t_steps
                              (wave: t_2..t_{steps+1}; complex128 for Schroedinger) */
  const double* src_init;  /* heat: first source sum s^0 + s^1 (grid) or NULL */
  const double* src_profile; /* heat: spatial source profile p (grid) or NULL */
  const double* src_coef;  /* heat: steps coefficients; step n (0-based) uses the
                              source sum src_coef[n] * p; NULL = 1 */
  const double* potential; /* Schroedinger: potential v (grid, float64) */
  void* u_out;             /* host, written at completion: the final field (grid);
                              must stay valid until the request is done */
} kfbi_request;

typedef enum {
  KFBI_REQ_QUEUED = 0,
  KFBI_REQ_RESIDENT = 1,
  KFBI_REQ_DONE = 2,
  KFBI_REQ_FAILED = 3
} kfbi_request_state;

typedef struct {
  int state;               /* kfbi_request_state */
  int status;              /* kfbi_status of a failed request */
  double arrival, admitted, finished; /* server clock seconds (-1: not yet) */
  int admit_tick, finish_tick;        /* tick indices (-1: not yet) */
  int steps_done;
  int max_iters;           /* most GMRES iterations of one of its steps */
  double max_rel_residual; /* largest final relative residual of its steps */
  long long device_bytes;  /* device bytes it held while resident */
} kfbi_request_info;

typedef struct {
  int ticks, admitted, completed, failed; /* ticks summed over lanes */
  double busy_seconds;         /* inside batch steps, summed over lanes */
  double admit_seconds;        /* admitting (plan wait, uploads, init) on the calling thread */
  double resident_ticks;       /* sum over ticks of the resident count */
  long long peak_device_bytes; /* most bytes held by resident requests at once */
  long long h2d_bytes, d2h_bytes;
  double grid_point_steps;     /* sum over completed steps of M^2 */
} kfbi_server_stats;

kfbi_status kfbi_server_create(const kfbi_server_desc* desc, void* stream, kfbi_server** out);
void kfbi_server_destroy(kfbi_server* server);
/* Queue a request; *id receives its index (0, 1, ... in submission order). */
kfbi_status kfbi_server_submit(kfbi_server* server, const kfbi_request* req, int* id);
/* One tick at server time now (seconds; now < 0 reads the server's wall
 * clock): admissions, one batch step of the resident requests, retirement.
 * *n_resident (may be NULL) receives the requests that stepped. */
kfbi_status kfbi_server_tick(kfbi_server* server, double now, int* n_resident);
/* Restart the wall clock at 0 and tick until every submitted request is
 * done or failed, sleeping while nothing is resident and the next arrival
 * lies ahead; KFBI_ERR_TIMEOUT if time_limit (> 0) seconds pass first. */
kfbi_status kfbi_server_run(kfbi_server* server, double time_limit);
kfbi_status kfbi_server_request_info(const kfbi_server* server, int id, kfbi_request_info* info);
kfbi_status kfbi_server_get_stats(const kfbi_server* server, kfbi_server_stats* stats);
const char* kfbi_server_last_error(const kfbi_server* server);

#ifdef __cplusplus
}
#endif

#endif /* KFBI_H */
