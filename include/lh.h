/*
 * lh.h -- C ABI of liblh.so, a single-GPU (NVIDIA B300, sm_103a) implementation of
 * the matrix-free, partially assembled, sum-factorized Lagrange-phase hot path of
 * high-order finite-element Lagrangian hydrodynamics (arXiv 2112.07075).
 *
 * Method (paper Section 3.3, Eqs. 14-18, single material):
 *     M_v dv/dt = -F.1,   rho|J| = rho0|J0|,   M_E de/dt = F^T v,   dx/dt = v,
 * with every operator applied through the decomposition A = G^T B^T D B G of
 * Section 3.1 (the parallel P/P^T factor is the identity on one GPU) and the
 * tensor-product sum factorization of Section 3.2.
 *
 * Spaces: continuous H1 velocity/position space Q_p on GLL nodes, discontinuous
 * L2 energy space Q_{p-1} on Gauss-Legendre nodes, Gauss-Legendre quadrature with
 * q1 points per direction, structured nx x ny (x nz) quad/hex mesh of a box whose
 * vertices the caller supplies (they may be jittered inside the box).
 *
 * Data layout (all FP64, little endian):
 *   H1 vector fields x, v, accelerations, F.1 : [dim][N_H1], component-major;
 *       node g = gx + N1x*(gy + N1y*gz), N1x = nx*p + 1 (likewise y, z).
 *   L2 fields e, F^T v                        : [NE][p^dim]; element
 *       e = ex + nx*(ey + ny*ez), local node jx + p*(jy + p*jz).
 *   Force quadrature data (lh_copy_qdata)     : [NE][dim*dim][q1^dim], entry
 *       (c, l) = omega detJ (sigma J^{-T})_{c l}, qpoint kx + q1*(ky + q1*kz).
 *
 * Ownership: state buffers (x, v, e, right-hand sides, outputs) are caller-owned
 * DEVICE memory. The context owns every other device buffer; all of them are
 * allocated once in lh_setup (one arena) and freed in lh_destroy. No entry point
 * allocates device memory after setup.
 *
 * Streams: every compute call is asynchronous on the given stream (0 = legacy
 * default stream) and returns after enqueueing. Scalar results (time-step
 * estimate, solver info) are written to caller-provided DEVICE memory.
 *
 * Errors: every call returns an lh_status. Argument errors are detected on the
 * host before anything is enqueued. Conditions found on the device (inverted
 * element, CG not converged, bounded wait expired) are written to the status
 * field of the info struct of the call that found them and are also latched in
 * the context; lh_sync_status() waits for the context's work and returns (and
 * clears) the latched device status. lh_last_error() describes the last error.
 *
 * Threading: a context must not be used from two host threads at once, and
 * calls on one context that overlap on the GPU (different streams without
 * ordering) race on the context's internal buffers.
 */
#ifndef LH_H
#define LH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *lh_stream_t; /* a cudaStream_t */

typedef enum {
  LH_OK = 0,
  LH_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, bad option) */
  LH_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  LH_ERR_OOM = 3,           /* the setup arena could not be allocated */
  LH_ERR_INVERTED = 4,      /* det J <= 0 at some quadrature point */
  LH_ERR_NOT_CONVERGED = 5, /* CG reached max_it before the tolerance */
  LH_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired */
  LH_ERR_UNSUPPORTED = 7    /* (dim, order, q1) combination not compiled */
} lh_status;

typedef enum {
  LH_PROBLEM_TAYLOR_GREEN = 0,
  LH_PROBLEM_GRESHO = 1,    /* 2D only */
  LH_PROBLEM_SEDOV = 2      /* blast: rho0 = 1, v0 = 0, internal energy 0.25 deposited uniformly in
                               element 0 (the corner at the origin), e = 0 elsewhere; the box
                               faces are symmetry planes. Exercises the viscosity's linear term
                               and the step control (lh_set_dt_control). */
} lh_problem;
typedef enum { LH_SOURCE_NONE = 0, LH_SOURCE_TAYLOR_GREEN_2D = 1 } lh_source;
typedef enum { LH_PRECISION_FP64 = 0, LH_PRECISION_FP32_IR = 1, LH_PRECISION_BF16TC_IR = 2 } lh_precision;

typedef struct {
  int dim;                  /* 2 or 3 */
  int nx, ny, nz;           /* elements per direction (nz ignored for dim 2) */
  const double *vertices;   /* HOST, [(nx+1)(ny+1)(nz+1)][dim], vertex vx + (nx+1)(vy + (ny+1) vz);
                               copied during lh_setup, may be freed afterwards */
  int order;                /* H1 order p in 1..4; L2 order is p-1 */
  int q1;                   /* Gauss-Legendre points per direction */
  double gamma;             /* ideal-gas exponent (> 1) */
  double cfl;               /* CFL number of the time-step estimate (> 0) */
  int use_viscosity;        /* 1: tensor artificial viscosity on, 0: off */
  int source;               /* lh_source */
  int precision;            /* lh_precision of the velocity mass solves (lh_mass_cg and
                               lh_rk2avg_step): LH_PRECISION_FP64 = FP64 Jacobi PCG;
                               LH_PRECISION_FP32_IR = FP32 Jacobi PCG inner solves (FP32
                               mass data, vectors, contractions) under FP64 iterative
                               refinement (FP64 residual b - M x, norms, x update);
                               LH_PRECISION_BF16TC_IR = the same refinement with the inner
                               element contractions on the tensor cores (BF16 hi/lo split
                               operands, FP32 accumulation; dim 3, order >= 3,
                               q1^3 <= 256, else lh_setup returns LH_ERR_UNSUPPORTED) */
} lh_params;

/* Sizes of a context's spaces. */
typedef struct {
  int64_t ne;      /* elements */
  int64_t n_h1;    /* scalar H1 nodes */
  int64_t nv;      /* vector H1 DOFs = dim * n_h1 */
  int64_t n_l2;    /* L2 DOFs = ne * p^dim */
  int64_t nq;      /* quadrature points = ne * q1^dim */
  int64_t arena_bytes; /* device bytes owned by the context */
} lh_sizes;

/* Result of one mass solve; lives in DEVICE memory. */
typedef struct {
  int iters;        /* CG iterations taken (FP32 inner iterations for LH_PRECISION_FP32_IR) */
  int status;       /* LH_OK or LH_ERR_NOT_CONVERGED / LH_ERR_TIMEOUT */
  double rel_res;   /* final ||r||_2 / ||b||_2 (0 when b = 0) */
  double b_norm;    /* ||b||_2 over free DOFs */
  int refinements;  /* FP64 refinement steps (LH_PRECISION_FP32_IR), 0 otherwise */
  int reserved;
} lh_cg_info;

/* Running time-integration record; lives in DEVICE memory. The caller sets t and
   t_end before the first step (e.g. by cudaMemcpy); lh_rk2avg_step updates it. */
typedef struct {
  double t;           /* current time, advanced by dt each step */
  double t_end;       /* final time used to cap a CFL-controlled step */
  double dt;          /* step size used by the last step */
  double dt_est;      /* CFL time-step estimate from the last step's stage 1 */
  double energy_src;  /* dt * sum_j b_j of the last step (energy added by the source) */
  double cg_rel_res[2];
  int cg_iters[2];    /* CG iterations of the last step's two mass solves */
  int status;         /* LH_OK or the first device-side error of the last step */
  int steps;          /* steps taken with this record */
  long long cg_iters_total; /* sum of cg_iters over all steps taken with this record
                               (lh_rk2avg_step only; the batch step leaves it alone) */
  /* step control with rejection (lh_set_dt_control); untouched otherwise */
  double dt_ctl;      /* controller cap c on dt (<= 0: none); the caller may start it at 0 */
  double dt_est_half; /* CFL estimate at the half-step state of the last attempt */
  int rejected;       /* 1 if the last attempt was rejected (state left unchanged) */
  int rejections;     /* rejected attempts with this record */
} lh_step_info;

typedef struct lh_ctx lh_ctx;

/* Set up a context: copies the vertices, builds the H1 node positions x0
 * (multilinear vertex map at the GLL nodes), the basis tables, the mass
 * quadrature data omega*rho0*detJ0 (Section 3.2), the initial inverse
 * Jacobians, the element energy-mass inverses M_E^{-1} (Eq. 17), the Jacobi
 * diagonal of M_v, and allocates the arena. rho0_q: optional DEVICE array
 * [NE][q1^dim] of initial densities at quadrature points (NULL: rho0 = 1).
 * Returns LH_ERR_INVERTED if det J0 <= 0 anywhere, LH_ERR_UNSUPPORTED if the
 * (dim, order, q1) kernels are not compiled in. Synchronous. */
lh_status lh_setup(const lh_params *params, const double *rho0_q, lh_ctx **out);

/* Release every resource of the context (NULL is accepted). Synchronous. */
void lh_destroy(lh_ctx *ctx);

/* Sizes of the context's spaces. */
lh_status lh_get_sizes(const lh_ctx *ctx, lh_sizes *out);

/* Message of the last error on this context (or of the last failed lh_setup when
 * ctx is NULL). Never NULL. */
const char *lh_last_error(const lh_ctx *ctx);

/* Wait for all work enqueued by the context and return the first device-side
 * error latched since the last call (then clear it), or LH_ERR_CUDA. */
lh_status lh_sync_status(lh_ctx *ctx);

/* Initial state of an analytic problem: x = x0 (H1 node positions), v = nodal
 * interpolation of the problem's velocity (zero on constrained DOFs), e = the
 * element-local L2 projection of p0 / ((gamma - 1) rho0) (Section 3.3 spaces).
 * x, v: DEVICE [dim][N_H1]; e: DEVICE [NE][p^dim]. */
lh_status lh_init_state(lh_ctx *ctx, int problem, double *x, double *v, double *e,
                        lh_stream_t stream);

/* Quadrature-point data update (Section 6, "quadrature point data" and
 * "artificial viscosity"; Eqs. 1-5 stress, Eq. 16 density): from the state
 * (x, v: DEVICE [dim][N_H1]; e: DEVICE [NE][p^dim]) computes, per quadrature
 * point, the Jacobian, its determinant and inverse, rho = rho0 detJ0 / detJ,
 * ideal-gas pressure and sound speed, tensor artificial viscosity, the stress
 * sigma and the force data omega detJ sigma J^{-T}, stored in the context for
 * the following force products. If dt_est is not NULL, also writes the CFL
 * time-step estimate (one DEVICE double; 0 if an element is inverted). */
lh_status lh_update_qdata(lh_ctx *ctx, const double *x, const double *v, const double *e,
                          double *dt_est, lh_stream_t stream);

/* Copy the force quadrature data of the last lh_update_qdata into out (DEVICE,
 * [NE][dim*dim][q1^dim]). */
lh_status lh_copy_qdata(lh_ctx *ctx, double *out, lh_stream_t stream);

/* Force product (Eq. 14 right-hand side): rhs = F u, where
 * F_{(i,c),j} = sum_q phi_j(q) sum_l dw_i/dxi_l(q) D_q[c,l] with the force data
 * of the last lh_update_qdata. u: DEVICE [NE][p^dim] or NULL for u = 1 (F.1).
 * rhs: DEVICE [dim][N_H1], overwritten; no boundary conditions applied. */
lh_status lh_force_mult(lh_ctx *ctx, const double *u, double *rhs, lh_stream_t stream);

/* Transposed force product (Eq. 17 right-hand side): out = F^T v.
 * v: DEVICE [dim][N_H1]; out: DEVICE [NE][p^dim], overwritten. */
lh_status lh_force_mult_t(lh_ctx *ctx, const double *v, double *out, lh_stream_t stream);

/* Mass product (Section 3.2, y = B^T D B x per element, then G^T):
 * y = M_v x with M_v = I_dim (x) M, M_ij = sum_q omega rho0 detJ0 w_i w_j.
 * x, y: DEVICE [dim][N_H1] (must not alias); no boundary conditions applied. */
lh_status lh_mass_mult(lh_ctx *ctx, const double *x, double *y, lh_stream_t stream);

/* Velocity mass action with the tensor-core element operator of
 * LH_PRECISION_BF16TC_IR (the operator its inner solves use): y = M x in FP32,
 * x masked to the free DOFs (constrained DOFs count as 0), no boundary conditions
 * on y. x, y: DEVICE FP32 [dim][N_H1], must not alias. Returns LH_ERR_UNSUPPORTED
 * for contexts of another precision. */
lh_status lh_mass_mult_tc(lh_ctx *ctx, const float *x, float *y, lh_stream_t stream);

/* Velocity mass solve (Eq. 14, "inversion of a global CG mass matrix", Section 6):
 * Jacobi-preconditioned CG for M_v x = b on the free DOFs (v.n = 0 on the box
 * faces; x is set to 0 on constrained DOFs and b is ignored there), stopping when
 * the FP64 residual satisfies ||b - M x||_2 <= rel_tol ||b||_2. x: in = initial
 * guess, out = solution. b, x: DEVICE [dim][N_H1]. info: DEVICE lh_cg_info or NULL.
 * With the context's precision LH_PRECISION_FP64, max_it bounds the CG iterations;
 * with LH_PRECISION_FP32_IR (LH_PRECISION_BF16TC_IR) each refinement step runs an
 * FP32 PCG to a relative residual of 1e-6 (3e-5) (at most 200 iterations), at most
 * 40 steps are taken, max_it bounds the total inner iterations, and info->iters
 * reports that total.
 * One persistent cooperative launch; convergence is decided on the device. */
lh_status lh_mass_cg(lh_ctx *ctx, const double *b, double *x, double rel_tol, int max_it,
                     lh_cg_info *info, lh_stream_t stream);

/* Energy solve (Eq. 17): out = M_E^{-1} rhs element by element with the dense
 * inverses built at setup. rhs, out: DEVICE [NE][p^dim] (must not alias). */
lh_status lh_energy_solve(lh_ctx *ctx, const double *rhs, double *out, lh_stream_t stream);

/* One RK2-average step of Eqs. 14-18 (two stages; the force data of a stage is
 * computed once and used for both F.1 and F^T v, which conserves total energy
 * up to the solver tolerance). x, v, e: DEVICE state, updated in place.
 * dt > 0: fixed step. dt <= 0: dt = min(dt_est(stage 1), info->t_end - info->t).
 * info: DEVICE lh_step_info (required; t and t_end must be initialised).
 * Mass solves: Jacobi-PCG to rel_tol (<= 0: 1e-12), max_it (<= 0: 1000),
 * warm-started from the previous solve's acceleration. */
lh_status lh_rk2avg_step(lh_ctx *ctx, double *x, double *v, double *e, double dt,
                         double rel_tol, int max_it, lh_step_info *info, lh_stream_t stream);

/* Step control with rejection for the CFL-controlled steps (dt <= 0) of
 * lh_rk2avg_step (no counterpart in the paper, which names no integrator; used by
 * shock workloads). With it enabled, an attempt takes dt = min(info->dt_ctl (if > 0),
 * dt_est(S_n), t_end - t); the stage-2 quadrature update also estimates the CFL step
 * at the half-step state S_h. If dt_est(S_h) < dt the attempt is rejected on the
 * device: x, v, e stay unchanged, t does not advance, info->rejected = 1,
 * info->rejections += 1 and dt_ctl = 0.85 dt_est(S_h) (0.5 dt if S_h is inverted);
 * otherwise the step is taken as usual and a positive dt_ctl grows by 2 %. The
 * caller repeats calls until info->t reaches t_end. enable = 0 restores plain CFL
 * steps. Returns LH_ERR_ARG for a NULL context. */
lh_status lh_set_dt_control(lh_ctx *ctx, int enable);

/* Solver timing probe (measurement support; no counterpart in the paper).
 * lh_timing_enable(ctx, 1) makes every later mass solve of this context
 * (lh_mass_cg and the two solves inside lh_rk2avg_step) record a pair of CUDA
 * events on its stream around the solver launch; up to 64 solves are kept.
 * lh_timing_read waits for the recorded events, returns the summed solver time
 * in milliseconds and the number of solves since the previous read, and starts
 * a new record. Leave timing disabled while capturing a CUDA graph (the events
 * would become capture dependencies, not timestamps). Returns LH_ERR_ARG on NULL
 * arguments, LH_ERR_CUDA if an event call fails. */
lh_status lh_timing_enable(lh_ctx *ctx, int enable);
lh_status lh_timing_read(lh_ctx *ctx, double *solver_ms, int *solves);

/* ---------------------------------------------------------------------------
 * Remap phase, velocity (Section 3.5; the continuous advection of Section 2.3).
 *
 * The remap moves the velocity from the mesh at the H1 node positions x0 to the
 * mesh at x1 (same topology) by integrating, over the pseudo-time tau in [0, 1]
 * with the mesh moving as x(tau) = x0 + tau u, u = x1 - x0,
 *     M(tau) dv/dtau = K(tau) v,
 *     M(tau)_ij = int w_i w_j dx,   K(tau)_ij = int w_i (u . grad w_j) dx
 * (unit density; the scalar matrices act on each component). Both operators are
 * partially assembled: per stage one element pass computes omega detJ(tau) and
 * omega adj(J(tau)) u at the quadrature points and applies K element by element
 * with sum factorization; M(tau) is inverted by the Lagrange phase's persistent
 * solver in the context's precision (FP64 Jacobi-PCG, or the FP32 / tensor-core
 * inner solver under FP64 refinement), always to the FP64 residual criterion.
 * ------------------------------------------------------------------------- */

/* Result of one lh_remap_velocity call; lives in DEVICE memory, reset by the call. */
typedef struct {
  int status;             /* LH_OK or the context's latched device status (first error
                             since the last lh_sync_status): LH_ERR_INVERTED when
                             det J(tau) <= 0 at a qpoint, or a solver status */
  int solves;             /* mass solves taken (2 per pseudo-time step) */
  int cg_iters_max;       /* largest iteration count of one solve */
  int reserved;
  long long cg_iters_total;
  double cg_rel_res_max;  /* largest final relative residual of one solve */
} lh_remap_info;

/* Remap the velocity v (DEVICE [dim][N_H1], updated in place) from the node
 * positions x0 to x1 (DEVICE [dim][N_H1]) with `steps` >= 1 equal pseudo-time
 * steps h = 1/steps of the explicit midpoint rule:
 *     k1 = M(tau)^-1 K(tau) v,   k2 = M(tau + h/2)^-1 K(tau + h/2) (v + h/2 k1),
 *     v <- v + h k2.
 * constrained != 0: the Lagrange phase's v.n = 0 DOFs keep their value (the solves
 * act on the free DOFs); 0: every DOF is remapped. Mass solves: the context's
 * solver (see lh_mass_cg) to rel_tol (<= 0: 1e-12) and max_it (<= 0: 1000),
 * warm-started from the previous stage's rate. info: DEVICE lh_remap_info or NULL.
 * Works in the context's solver and stage scratch and in its force quadrature data
 * buffer: call lh_update_qdata again before a later lh_force_mult/lh_force_mult_t.
 * v must not alias x0 or x1 (LH_ERR_ARG). */
lh_status lh_remap_velocity(lh_ctx *ctx, const double *x0, const double *x1, double *v, int steps,
                            int constrained, double rel_tol, int max_it, lh_remap_info *info,
                            lh_stream_t stream);

/* The remap operators at one pseudo-time, without boundary conditions:
 * kv = K(tau) v and mv = M(tau) v on the mesh x0 + tau (x1 - x0). kv or mv may be
 * NULL. All DEVICE [dim][N_H1]; kv and mv must not alias v (LH_ERR_ARG). Uses the
 * same context scratch as lh_remap_velocity. */
lh_status lh_remap_apply(lh_ctx *ctx, const double *x0, const double *x1, double tau, const double *v,
                         double *kv, double *mv, lh_stream_t stream);

/* ---------------------------------------------------------------------------
 * Stiffness (diffusion) operator of the hyper-viscosity and artificial-viscosity
 * terms (Sections 2.1 and 3.3 name it beside the mass and force operators;
 * Section 6 names the diffusion-integrator kernels of the viscosity calculation).
 *
 * On the mesh with H1 node positions x, S_ij = int grad w_i . grad w_j dx (scalar,
 * applied to each component), partially assembled as in Section 3.1 with the
 * reference gradients as B and, per quadrature point, the symmetric matrix
 * G = omega det J J^-1 J^-T (omega adj(J) adj(J)^T / det J) as D; the action is
 * sum factorized (reference gradient, G, transposed reference gradient) plus the
 * deterministic node gather.
 * ------------------------------------------------------------------------- */

/* PA setup on the mesh at node positions x (DEVICE [dim][N_H1]): stores G
 * ([NE][dim(dim+1)/2][q1^dim] in the context), the unit-density mass data
 * omega det J and the Jacobi inverse of that mass matrix M_x (every DOF). An
 * element with det J <= 0 latches LH_ERR_INVERTED in the context status. The data
 * stays valid until the next lh_stiffness_setup. */
lh_status lh_stiffness_setup(lh_ctx *ctx, const double *x, lh_stream_t stream);

/* y = S_x u for u, y DEVICE [dim][N_H1] (must not alias), no boundary conditions.
 * LH_ERR_ARG before the first lh_stiffness_setup. */
lh_status lh_stiffness_mult(lh_ctx *ctx, const double *u, double *y, lh_stream_t stream);

/* Discrete Laplacian of an H1 field (natural boundary conditions): lap solves
 * M_x lap = -S_x v per component on every DOF with the context's solver (see
 * lh_mass_cg), stopping at ||b - M x||_2 <= rel_tol ||b||_2 (rel_tol <= 0: 1e-12;
 * max_it <= 0: 1000).
 * v, lap: DEVICE [dim][N_H1], must not alias; lap in = initial guess.
 * info: DEVICE lh_cg_info or NULL. LH_ERR_ARG before the first lh_stiffness_setup. */
lh_status lh_laplacian(lh_ctx *ctx, const double *v, double *lap, double rel_tol, int max_it,
                       lh_cg_info *info, lh_stream_t stream);

/* ---------------------------------------------------------------------------
 * Mesh optimisation kernels (TMOP; Section 2.2 objective, Section 3.4 Eqs. 6-7).
 *
 * F(x) = int mu(T(x)) + gamma int |x - x0|^2 / d^2 over the target elements
 * (quadrature weights w_q det W), T = A W^-1 with A = dx/dxbar on the reference
 * element [0,1]^dim and the target W = h I (the ideal element of size h). Metric:
 * mu_2(T) = |T|^2 / (2 det T) - 1 in 2D, mu_303(T) = |T|^2 / (3 det(T)^(2/3)) - 1 in
 * 3D (shape metrics, zero on scaled rotations). Fully matrix-free: the metric and
 * its first and second derivatives are evaluated at each quadrature point inside
 * one sum-factorized element pass per call; vectors are gathered deterministically.
 * An element with det T <= 0 latches LH_ERR_INVERTED in the context status.
 * ------------------------------------------------------------------------- */
typedef struct {
  double target_size;  /* h of W = h I (> 0) */
  double lim_weight;   /* gamma (>= 0; 0 switches the limiting term off) */
  double lim_dist;     /* d, the constant displacement limit (> 0 when gamma > 0) */
} lh_tmop_params;

/* F(x) -> *F (DEVICE double). x, x0: DEVICE [dim][N_H1]; x0 may be NULL when
 * gamma = 0. Deterministic (fixed-order block sums). */
lh_status lh_tmop_objective(lh_ctx *ctx, const lh_tmop_params *prm, const double *x, const double *x0,
                            double *F, lh_stream_t stream);

/* g = dF/dx (Eq. 6 plus the limiting term), DEVICE [dim][N_H1], no boundary
 * conditions; g must not alias x or x0. */
lh_status lh_tmop_gradient(lh_ctx *ctx, const lh_tmop_params *prm, const double *x, const double *x0,
                           double *g, lh_stream_t stream);

/* y = (d^2F/dx^2) u (Eq. 7 plus the limiting term) at x; x, u, y DEVICE
 * [dim][N_H1]; y must not alias x or u. */
lh_status lh_tmop_hessian_mult(lh_ctx *ctx, const lh_tmop_params *prm, const double *x, const double *u,
                               double *y, lh_stream_t stream);

/* diag = the diagonal of d^2F/dx^2 at x (the Jacobi preconditioner of the Newton
 * solve), DEVICE [dim][N_H1]; must not alias x. */
lh_status lh_tmop_hessian_diag(lh_ctx *ctx, const lh_tmop_params *prm, const double *x, double *diag,
                               lh_stream_t stream);

/* Partially assembled Hessian, for the repeated Hessian products of a Newton-Krylov
 * solve at fixed x (a departure from Section 3.4's fully matrix-free choice: on this
 * GPU the FP64 rate, not memory, bounds the recomputation of the metric).
 * lh_tmop_workspace_size: the workspace length in doubles, NE * n(n+1)/2 * q1^dim
 * with n = dim^2 (the symmetric second-derivative tensor of mu per quadrature point,
 * scaled by w_q det W / h^2). lh_tmop_hessian_setup fills the caller's DEVICE
 * workspace at x (LH_ERR_INVERTED latched for det T <= 0); lh_tmop_hessian_mult_pa
 * then gives y = (d^2F/dx^2) u from it (limiting term included, same prm), equal to
 * lh_tmop_hessian_mult at that x up to rounding. work must not alias x, u or y. */
lh_status lh_tmop_workspace_size(const lh_ctx *ctx, int64_t *doubles);
lh_status lh_tmop_hessian_setup(lh_ctx *ctx, const lh_tmop_params *prm, const double *x, double *work,
                                lh_stream_t stream);
lh_status lh_tmop_hessian_mult_pa(lh_ctx *ctx, const lh_tmop_params *prm, const double *work,
                                  const double *u, double *y, lh_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batching form: many independent problems advanced together.
 *
 * A batch references existing contexts (2D, q1 = 2*order, LH_PRECISION_FP64;
 * orders 1..4 may be mixed) and their caller-owned state buffers. Every hot-path
 * operation of lh_rk2avg_step (quadrature data, F.1, mass CG, F^T v with the
 * energy solve, state updates) becomes ONE persistent launch over all problems:
 * element work items are sorted by order and each runs the kernel family of its
 * order; the mass solves of all problems run in one cooperative launch with
 * per-problem scalars and convergence (each to rel_tol). The step is captured
 * into a CUDA graph on first use and replayed. The arithmetic per problem is the
 * same as lh_rk2avg_step with a fixed dt, except for the summation order of the
 * CG dot products.
 * ------------------------------------------------------------------------- */
typedef struct lh_batch lh_batch;

/* Create a batch of n problems. ctxs[i]: context of problem i; x, v, e: HOST
 * arrays of n DEVICE pointers to each problem's state (as for lh_rk2avg_step);
 * dt: HOST array of n fixed step sizes (> 0); infos: DEVICE array of n
 * lh_step_info records updated by every step (t, dt, steps, cg_iters, cg_rel_res,
 * status), or NULL. The contexts and buffers must outlive the batch; the batch
 * owns one small device arena (work lists, argument records, solver scalars). */
lh_status lh_batch_create(int n, lh_ctx *const *ctxs, double *const *x, double *const *v, double *const *e,
                          const double *dt, lh_step_info *infos, lh_batch **out);

/* Tile shapes of the batched step (the RAJA-teams style tiles of Section 4.2, as
 * an autotuned choice): cfg[0..3] = element batches per work item of the element
 * passes for orders 1..4 (1, 2 or 4), cfg[4..7] = element batches per work item
 * of the solver for orders 1..4 (1, 2 or 4), cfg[8] = threads per block of the
 * element passes, i.e. how many threads share one tile's quadrature slab (128,
 * 256 or 512; every per-value result is the same for any choice).
 *
 * lh_batch_autotune times whole batched steps (element passes and solver) for
 * candidate shapes -- per order element tiles 1, 2, 4 and solver tiles 1, 2, 4, then
 * 128, 256, 512 threads per block -- and keeps each change that makes the step at
 * least 1 % faster. Every trial starts from the same state and the problems'
 * states, warm starts and step records are restored at the end, so tuning leaves
 * no trace in the results. cfg_out: optional HOST int[9], the chosen shape.
 * Synchronous; allocates and frees one snapshot buffer of the problems' states.
 * lh_batch_set_config sets a shape directly (HOST int[9]; LH_ERR_ARG for values
 * outside the lists above). The default is all tiles 1 and 256 threads. */
lh_status lh_batch_autotune(lh_batch *b, int *cfg_out);
lh_status lh_batch_set_config(lh_batch *b, const int *cfg);

/* One RK2-average step of every problem (fixed dt per problem), enqueued on
 * `stream` as one CUDA graph launch (captured on the first call and whenever
 * rel_tol, max_it or the tile shape change; rel_tol <= 0: 1e-12, max_it <= 0:
 * 1000). The graph holds six launches, three per stage: the fused quadrature-data
 * and F.1 element pass; one cooperative launch with the right-hand-side gather,
 * every problem's mass solve and the stage's node update; the F^T v element pass
 * with the energy update. */
lh_status lh_batch_step(lh_batch *b, double rel_tol, int max_it, lh_stream_t stream);

/* Message of the last error of a batch call. */
const char *lh_batch_last_error(const lh_batch *b);

/* Release the batch (not its contexts). NULL is accepted. */
void lh_batch_destroy(lh_batch *b);

/* ---------------------------------------------------------------------------
 * Learned form: a small per-element MLP predicts the initial guess of the
 * velocity mass solves of lh_rk2avg_step. Network: 586 -> 128 -> 128 -> 192,
 * GELU (erf) after both hidden layers, BF16 weights and activations on the
 * tensor cores with FP32 accumulation, FP32 master weights, Adam (0.9, 0.999,
 * 1e-8), mean-squared-error loss. Inputs per element (3D Q3), from the three most
 * recent mass-solve solutions a_1, a_2, a_3 at its 64 nodes (3 x 192 values):
 * a_1 / s, (a_1 - a_2) / s_d and (a_2 - a_3) / s_d with s, s_d the RMS of a_1 and
 * of a_1 - a_2 over the free DOFs; then its Jacobian at the centroid divided by
 * h0*p (9) and det J / (h0*p)^3 (1). Output: (a_new - a_1) / s_d at its nodes.
 * Parameters are one flat FP32 vector: W1 [128][592] (input padded to 592;
 * columns 586..591 stay zero), b1[128], W2 [128][128], b2[128], W3 [192][128], b3[192].
 * ------------------------------------------------------------------------- */
typedef struct lh_mlp lh_mlp;

/* Create an MLP for batches of up to max_rows elements; weights uniform in
 * +-sqrt(6 / fan_in) from `seed`, biases zero. Allocates its device buffers. */
lh_status lh_mlp_create(unsigned long long seed, int max_rows, lh_mlp **out);
void lh_mlp_destroy(lh_mlp *m);
/* Number of FP32 parameters. */
int lh_mlp_num_params(void);
/* Copy the FP32 parameters to / from HOST memory (set also resets Adam). Synchronous. */
lh_status lh_mlp_get_params(const lh_mlp *m, float *host_out);
lh_status lh_mlp_set_params(lh_mlp *m, const float *host_in);
/* Y[n][192] = MLP(X[n][586]); X, Y DEVICE FP32. */
lh_status lh_mlp_forward(lh_mlp *m, const float *X, int n, float *Y, lh_stream_t stream);
/* Loss (mean over n*192 outputs of (Y - T)^2, one DEVICE float) and, if grads is
 * not NULL, its gradient (DEVICE FP32, lh_mlp_num_params() values); no update. */
lh_status lh_mlp_gradients(lh_mlp *m, const float *X, const float *T, int n, float *grads, float *loss,
                           lh_stream_t stream);
/* One Adam step with learning rate lr on the batch (X, T); loss as above. */
lh_status lh_mlp_train_step(lh_mlp *m, const float *X, const float *T, int n, float lr, float *loss,
                            lh_stream_t stream);
const char *lh_mlp_last_error(const lh_mlp *m);
/* Waits for the device, then returns LH_ERR_TIMEOUT (and clears it) if a GEMM of
 * this MLP gave up a bounded wait since the last call, else LH_OK. */
lh_status lh_mlp_sync_status(lh_mlp *m);

/* Attach the learned form to a context (3D, order 3, q1 = 6). mode 1: record a
 * training example per element at every mass solve of lh_rk2avg_step that has
 * three earlier solutions (features into X_buf[row][586], targets into
 * T_buf[row][192], DEVICE, until capacity_rows rows are filled). mode 2: predict
 * the initial guess with `mlp`: the guess g and the previous solution a_1 are
 * compared by the Jacobi-preconditioned residual norm (r, D^-1 r): r = b - M g
 * (FP32 mass action, FP64 sums) for the guess, r = b - b_prev for a_1 (the mass
 * matrix is constant in time and a_1 solved the previous right-hand side b_prev
 * to the CG tolerance); the smaller starts CG; CG still runs to its tolerance
 * (either precision). mode 0: detach.
 * Allocates the form's device buffers (a set-up call); synchronous. */
lh_status lh_learn_attach(lh_ctx *ctx, lh_mlp *mlp, int mode, float *X_buf, float *T_buf, int capacity_rows);
/* Recording mode keeps every stride-th element of each solve (a rotating subset:
 * solve k records elements e = (k mod stride) + j * stride), so long runs on large
 * meshes fit the example buffer; default 1 (every element). LH_ERR_ARG without an
 * attached learned form or for stride < 1. */
lh_status lh_learn_set_record_stride(lh_ctx *ctx, int stride);
/* HOST counters of the attached learned form: rows recorded, mass solves seen,
 * predictions made, predictions that won the residual comparison, and the mean
 * over predictions of the ratio of the two compared norms, learned over previous
 * (square root of (r, D^-1 r) ratios; the last two read
 * device memory; synchronous). Any pointer may be NULL. */
lh_status lh_learn_stats(const lh_ctx *ctx, int *rows_recorded, int *solves, int *predictions, int *learned_used,
                         double *mean_ratio);

/* Mass product without any device allocation (the paper has no counterpart; this
 * is a convenience of this library). Computes the same y = M_v x as lh_mass_mult,
 * but takes everything from the caller and needs no context, so nothing is
 * allocated: not by this call and not by an lh_setup before it. It is meant for
 * callers that may not call cudaMalloc -- for example code that runs inside a
 * latency-critical loop where cudaMalloc's implicit device synchronisation is not
 * acceptable, or an embedding application that owns all device memory through its
 * own pool and forbids other allocations.
 *
 * dim, nx, ny, nz (ignored for dim 2), order, q1: as in lh_params (same compiled
 *   (dim, order, q1) families as lh_setup; LH_ERR_UNSUPPORTED otherwise).
 * mq: DEVICE [NE][q1^dim], the mass quadrature data omega_q * rho0 * detJ0 at each
 *   quadrature point (element and point numbering as in the layout notes above).
 * x, y: DEVICE [dim][N_H1], must not alias; y is overwritten, no boundary
 *   conditions are applied.
 * Scratch: the element vector (dim * NE * (order+1)^dim doubles) lives in a
 *   file-scope static device array of 32 MiB (plus a 24 KiB array with the basis
 *   tables of every compiled family); every GPU that loads liblh holds these until
 *   the process exits. Larger meshes are rejected with LH_ERR_ARG and a message
 *   giving the bytes needed, before anything is enqueued. The scratch holds the
 *   previous call's contents; every entry this call reads is written first by
 *   this call, so nothing has to start at zero.
 * Set-up: the first call on each device (with that device current) does a
 *   one-time set-up: it looks up the arrays' device addresses with
 *   cudaGetSymbolAddress, uploads the basis tables of every compiled family with
 *   a synchronous cudaMemcpy followed by cudaDeviceSynchronize, and sets the mass
 *   kernels' shared-memory attribute. Make that first call before any stream
 *   capture. With CUDA's default lazy module loading, the first use of the
 *   library's kernels on a device also loads its module, and the two static
 *   arrays are created on the device at that moment: an application that hands
 *   all device memory to its own pool should make the first call at start-up,
 *   before the pool takes the memory (or run with CUDA_MODULE_LOADING=EAGER).
 *   Every later call only enqueues two kernels on `stream`.
 * Concurrency: all calls share the one scratch array per device, so calls whose
 *   execution overlaps on the GPU (different streams without ordering, or
 *   several host threads) race and give wrong results; order them on one stream.
 * Errors: lh_last_error(NULL) describes the last failure of this call. */
lh_status lh_mass_mult_noalloc(int dim, int nx, int ny, int nz, int order, int q1, const double *mq,
                               const double *x, double *y, lh_stream_t stream);

/* Diagnostic (no counterpart in the paper): runs the library's bounded
 * grid-wide wait with one block that never arrives, so the waiting block gives
 * up after about one second instead of hanging; writes the device status it
 * latched (LH_ERR_TIMEOUT when the bound works) to *status_out. Allocates and
 * frees 256 bytes; synchronous. */
lh_status lh_selftest_barrier_timeout(int *status_out);

#ifdef __cplusplus
}
#endif
#endif /* LH_H */
