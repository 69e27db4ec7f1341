/*
 * libmhfp -- GB300 (sm_103a) solver for the stabilized, hybridized
 * Q1-RT0-P0 three-field poromechanics system of Frigo, Castelletto,
 * Ferronato & White, "Efficient solvers for hybridized three-field mixed
 * finite element coupled poromechanics" (arXiv:2002.09603).
 *
 * One backward-Euler step solves A_H x = b (Eq. stab_A, hybrid form),
 *
 *     [ A_uu   A_up            0         ] [u]   [f_u]
 *     [ A_pu   Abar_pp+A_stab  dt A_ppi  ] [p] = [f_p]
 *     [ 0      A_pip           A_pipi    ] [pi]  [f_pi]
 *
 * by right-preconditioned flexible GMRES with the block upper-triangular
 * preconditioner M of Eq. (hybridPrec), whose A_uu and C~_pi solves are
 * multigrid V-cycles.
 *
 * Conventions for every call below:
 *  - Vectors are FP64 DEVICE pointers in the layout
 *      [ u (3 per node, node-major: u_x,u_y,u_z of node 0, then node 1, ...)
 *      | p (one per cell) | pi (one per face) ],
 *    nodes n = i + (nx+1)(j + (ny+1)k), cells c = i + nx(j + ny k), faces
 *    x-normal family first (i <= nx, j < ny, k < nz), then y, then z, each
 *    lexicographic.  The caller owns every vector it passes; the handle owns
 *    all matrices, multigrid levels and Krylov workspace.
 *  - All device work is issued on the CUDA stream given to mhfp_create.
 *    Calls return after their work is queued, except those that report
 *    statistics or sizes (mhfp_solve, mhfp_setup_precond), which
 *    synchronise the stream.
 *  - Errors are returned as mhfp_status; mhfp_last_error gives the text.
 *    Host-side validation happens before any launch.  No call traps,
 *    asserts on the device or waits without bound.
 */
#ifndef MHFP_H
#define MHFP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhfp_ctx* mhfp_handle;

typedef enum {
  MHFP_OK = 0,
  MHFP_ERR_ARG = 1,            /* bad argument (null pointer, size, value)      */
  MHFP_ERR_MESH = 2,           /* inverted/degenerate element (det J <= 0)      */
  MHFP_ERR_OOM = 3,            /* device allocation failed                      */
  MHFP_ERR_CUDA = 4,           /* a CUDA runtime call failed                    */
  MHFP_ERR_NOT_CONVERGED = 5,  /* maxit reached; x holds the last iterate       */
  MHFP_ERR_NONFINITE = 6,      /* NaN/Inf in the right-hand side or residual    */
  MHFP_ERR_BREAKDOWN = 7,      /* Krylov breakdown that is not convergence      */
  MHFP_ERR_STATE = 8           /* call out of order (e.g. solve before setup)   */
} mhfp_status;

/* Structured hexahedral mesh of a box (nx*ny*nz cells), host arrays, copied
 * at create time.  coords: (nx+1)(ny+1)(nz+1)*3 node coordinates (any
 * positively oriented hexahedra).  node_fix: per node, bit0/1/2 = u_x/u_y/u_z
 * prescribed to zero.  face_bc: per face, bit0 = the uniform traction acts on
 * it, bit1 = drained (interface pressure prescribed to zero), bit2 = no-flow
 * (the default for boundary faces that are not drained). */
typedef struct {
  int nx, ny, nz;
  const double* coords;
  const unsigned char* node_fix;
  const unsigned char* face_bc;
} mhfp_mesh;

/* Per-cell material fields, host arrays of n_T values (kappa: 3 per cell,
 * the diagonal of the permeability tensor).  E [Pa], nu [-], biot [-],
 * Seps [1/Pa], mu [Pa s], kappa [m^2]. */
typedef struct {
  const double *E, *nu, *biot, *Seps, *mu, *kappa;
} mhfp_materials;

typedef struct {
  int restart;          /* FGMRES restart length m, 1..63 (default 50)         */
  int maxit;            /* maximum total FGMRES iterations (default 1000)      */
  int cheb_degree;      /* Chebyshev smoother degree (default 2); 0: chosen by */
                        /* the set-up autotuner (autotune = 1 required): the   */
                        /* step's load right-hand side is solved to 1e-8 with  */
                        /* degrees 1, 2 and 3 and the fastest is kept          */
  double cheb_ratio;    /* lmax / lmin of the smoother interval (default 10)   */
  int coarse_max;       /* coarsen while a level has more lattice points       */
                        /* (default 125, at most 4096); the last level is      */
                        /* solved with a dense FP64 inverse built on the GPU   */
                        /* by Gauss-Jordan elimination (2 n^3 FMA for its n    */
                        /* unknowns; MHFP_ERR_ARG if a pivot is not positive)  */
  int power_iters;      /* power iterations for rho(D^-1 A) (default 15)       */
  int precision;        /* 0: FP64 preconditioner (default); 1: FP32 V-cycles  */
                        /* and Schur steps inside the FP64 FGMRES (residuals,  */
                        /* Gram-Schmidt, Hessenberg and the coarsest dense     */
                        /* solve stay FP64)                                    */
  int graphs;           /* 2 (default): the whole solve is one CUDA graph      */
                        /* (restart cycles in a WHILE node, Arnoldi steps in   */
                        /* IF nodes, decisions taken on the device); 1: each   */
                        /* Arnoldi step is one graph replay driven by the      */
                        /* host (used whenever kernel timing is enabled);      */
                        /* 0: kernels are launched one by one                  */
  int autotune;         /* 1 (default): time the launch schedules of each      */
                        /* coarse level's smoother at set-up (one point per    */
                        /* thread, or the stencil offsets split over 4, 8 or   */
                        /* 16 warps) and the two occupancy variants of the     */
                        /* finest FP32 displacement sweep, and keep the        */
                        /* fastest (schedule only: the same products, summed   */
                        /* in a schedule-dependent fixed order)                */
  int reorth;           /* Gram-Schmidt of each Arnoldi step (the paper names  */
                        /* GMRES in PETSc, Section 5, and no orthogonalisation)*/
                        /* 1 (default): classical Gram-Schmidt, repeated once  */
                        /* when the norm falls below 1/sqrt(2) of its value    */
                        /* (DGKS test); 0: one classical pass, never repeated  */
                        /* (PETSc's GMRES default)                             */
  int schedule;         /* 0 (default): each coarse lattice level's sweeps and */
                        /* residuals take the autotuner's schedule (the size   */
                        /* rule when autotune = 0); 1, 4, 8 or 16: every       */
                        /* coarse lattice level uses that schedule (1 = one    */
                        /* point per thread, W = offsets over W warps)         */
  int fine_blocks;      /* finest FP32 displacement sweep and residual         */
                        /* (precision = 1): 0 (default) autotuned (size rule   */
                        /* without it); 5, 6, 7 or 8: one node per thread with */
                        /* that many resident blocks of 256 per SM (5: two     */
                        /* neighbour slots per loop iteration); 4: persistent  */
                        /* CTAs (4 per SM) fed by bulk copies of the stored    */
                        /* rows into shared memory (same sums, same order)     */
  int near_kernel;      /* near-kernel of the displacement multigrid (Section  */
                        /* 5): 0 (default) the three translations per          */
                        /* aggregate, separate displacement components         */
                        /* (M_II^(h)); 1 the six rigid-body modes (M_III^(h)): */
                        /* per aggregate a Gram-Schmidt factorisation of the   */
                        /* modes restricted to its dofs, six dofs per coarse   */
                        /* point (a mode the aggregate cannot represent leaves */
                        /* a decoupled dof with a unit diagonal)               */
  int formulation;      /* 0 (default): the hybridized system [u | p | pi]     */
                        /* (Eq. hmfeSys) with M_II^(h) / M_III^(h); 1: the     */
                        /* mixed system [u | p | q] (Eq. mfeSys, one RT0 flux  */
                        /* per face, q = 0 imposed on no-flow faces) with the  */
                        /* block-triangular preconditioner M_II^(m) of         */
                        /* Eq. (prec): a displacement V-cycle, Chebyshev on    */
                        /* A_qq preconditioned by its diagonal, and a V-cycle  */
                        /* on C~_p = A_pp + A_stab + the fixed-stress diagonal */
                        /* - dt A_pq L_qq^-1 A_qp (L_qq the lumped A_qq).      */
                        /* Same vector length as 0; the face entries are the   */
                        /* fluxes.  Needs precision = 0; the transposed,       */
                        /* adjoint, gradient, permeability-update and no-      */
                        /* allocation residual calls return MHFP_ERR_STATE     */
} mhfp_options;

typedef struct {
  int iterations;       /* FGMRES iterations (all cycles)                      */
  int restarts;         /* completed restart cycles                            */
  int converged;        /* 1 if the true residual met tol                      */
  double rel_residual;  /* Arnoldi estimate |g_{j+1}| / ||D_s b||              */
  double true_rel_residual; /* ||D_s (b - A x)|| / ||D_s b|| at exit           */
  double solve_ms;      /* wall time of the call (host clock)                  */
} mhfp_stats;

typedef struct {
  int levels;           /* number of levels (>= 1)                             */
  long long points[8];  /* lattice points (or faces) per level                 */
  int block[8];         /* unknowns per point (3 for u, 6 on the coarse u      */
                        /* levels with the rigid-body modes, 1 for pi)         */
  double lmax[8];       /* 1.1 * rho(D^-1 A) per level (0 on the last level)   */
  int schedule[8];      /* launch schedule of the level's sweeps: 1 = one point */
                        /* per thread, 4/8/16 = offsets split over that many    */
                        /* warps; finest FP32 displacement level: fine_blocks  */
                        /* (4, 6 or 8); 0 = not a lattice sweep                */
  double sweep_us[8];   /* set-up autotuner's time of one sweep under that     */
                        /* schedule, microseconds (0 when not timed)           */
  int cheb_degree;      /* Chebyshev degree of the smoothers in use            */
} mhfp_hierarchy_info;

/* Fill *opt with the defaults listed above. */
void mhfp_default_options(mhfp_options* opt);

/* Validate and copy mesh + materials, record dt (Section 2.1, backward
 * Euler) and the uniform traction vector (Appendix A, f_u) acting on faces
 * with face_bc bit0.  stream: a cudaStream_t (may be NULL = legacy default).
 * The device current at the call is the one the handle uses. */
mhfp_status mhfp_create(const mhfp_mesh* mesh, const mhfp_materials* mat, double dt,
                        const double traction[3], void* stream, mhfp_handle* out);

/* Element kernels and assembly (Appendix A; Eq. hmfeSys / A_33H static
 * condensation of the RT0 fluxes; Eq. J_def / stab_A macro-element
 * stabilization with beta_M = (3b)^2 / [32 (lambda + 4G)]).  Returns
 * MHFP_ERR_MESH if any element has det J <= 0 at a quadrature point. */
mhfp_status mhfp_assemble_condense(mhfp_handle h);

/* Preconditioner set-up (Section 4, Eq. hybridPrec, Eq. app_Bp):
 * B~_p = S_eps|T| + diag(A_stab) + diag(A_up^T diag(A_uu)^-1 A_up)
 *        + dt diag(A_wp^T A_ww^-1 A_wp),
 * C~_pi = A_pipi - dt A_pip B~_p^-1 A_ppi, and the two multigrid
 * hierarchies.  opt may be NULL (defaults).  Synchronises the stream. */
mhfp_status mhfp_setup_precond(mhfp_handle h, const mhfp_options* opt);

/* Right-hand side of one backward-Euler step (Section 2.1, Appendix A):
 * b = [ load_scale * f_u ; A_pu u_prev + S_eps |T| p_prev ; 0 ].
 * d_x_prev: previous solution in the vector layout (only u and p are read),
 * or NULL for u_0 = 0, p_0 = 0.  d_rhs: output, n = n_u + n_p + n_pi. */
mhfp_status mhfp_build_rhs(mhfp_handle h, const double* d_x_prev, double load_scale, double* d_rhs);

/* Solve A_H x = b by FGMRES(restart) with right preconditioning M^-1, zero
 * initial guess (Section 5), on the equilibrated system D_s A_H D_s with
 * D_s = diag(A_uu, B~_p, C~_pi)^(-1/2); stops when ||D_s (b - A x)|| <=
 * tol ||D_s b||.  d_rhs, d_x: device vectors (d_x is overwritten).
 * stats may be NULL.  Synchronises the stream. */
mhfp_status mhfp_solve(mhfp_handle h, const double* d_rhs, double* d_x, double tol, mhfp_stats* stats);

/* Solve `count` independent systems (different handles: meshes, materials,
 * dt, right-hand sides) together.  Each handle's FGMRES (the same algorithm
 * as mhfp_solve) is advanced step by step in round-robin order; the work of
 * every Arnoldi step is one CUDA-graph replay on the handle's own stream, so
 * handles created on distinct streams run concurrently on the device.
 * stats and statuses (count entries each) may be NULL; returns the first
 * non-OK status (in handle order), MHFP_OK if every solve converged.  Not in
 * the paper: batching of its solve over parameter samples and loads. */
mhfp_status mhfp_solve_batch(int count, const mhfp_handle* hs, const double* const* d_rhs, double* const* d_x,
                             double tol, mhfp_stats* stats, mhfp_status* statuses);

/* Many solves in one CUDA graph launch (not in the paper: batching of its
 * solve over parameter samples, meshes and loads).  Entry i solves handle
 * hs[i] for d_rhs[i] into d_x[i] (device vectors of that handle's size) with
 * the algorithm of mhfp_solve.  Entries of one handle run one after another
 * in list order (they share its Krylov workspace); entries of different
 * handles are independent branches of the graph and run concurrently.  The
 * graph is built and instantiated once by mhfp_batch_create (the device-
 * driven solve of mhfp_solve, with the copies of b and x and the control
 * block's reset as graph nodes), and every mhfp_batch_run is one
 * cudaGraphLaunch on `stream` (NULL: the legacy default stream) followed by
 * a synchronisation; the handles' own streams are synchronised first.  The
 * vector pointers are fixed at creation.  After mhfp_update_logk on any of
 * its handles a batch reports MHFP_ERR_STATE and must be created again.
 * stats / statuses: count entries each (may be NULL); solve_ms is the whole
 * launch's wall time.  Returns the first non-OK status. */
typedef struct mhfp_batch_s* mhfp_batch;
mhfp_status mhfp_batch_create(int count, const mhfp_handle* hs, const double* const* d_rhs, double* const* d_x,
                              double tol, mhfp_batch* out);
/* The same batch with several right-hand sides of one handle solved in
 * lockstep (multi-right-hand-side kernels; not in the paper: its solve
 * batched over the loads of one discretisation, as with the four load
 * scales of one mesh).  Entries of one handle are taken, in list order, in
 * sets of at most max_lanes (1 <= max_lanes <= MHFP_MAX_LANES; 1 gives
 * mhfp_batch_create).  A set of K > 1 entries is one FGMRES run for all K:
 * each kernel of the solve is launched once with the K right-hand sides as
 * its third grid dimension, the handle's matrices shared by all of them; each right-hand side keeps its own Krylov basis, Hessenberg
 * matrix, restarts and stopping decision, and its result is bit-identical to
 * the same entry in mhfp_batch_create.  The set runs until its last member
 * has stopped; a member that stops earlier keeps its solution and
 * statistics.  Sets of one handle run one after another in its branch;
 * different handles concurrently.  The batch allocates, for each (handle,
 * set size K) it uses, a workspace of K copies of the handle's solve vectors
 * (about (1.5 restart + 14) n doubles per right-hand side), freed by
 * mhfp_batch_destroy.  Only for handles of the hybrid system (formulation
 * = 0, either precision); otherwise MHFP_ERR_STATE. */
#define MHFP_MAX_LANES 16
mhfp_status mhfp_batch_create_lanes(int count, const mhfp_handle* hs, const double* const* d_rhs,
                                    double* const* d_x, double tol, int max_lanes, mhfp_batch* out);
mhfp_status mhfp_batch_run(mhfp_batch b, void* stream, mhfp_stats* stats, mhfp_status* statuses);
void mhfp_batch_destroy(mhfp_batch b);

/* y = A_H x (Eq. stab_A, hybrid form), unscaled. */
mhfp_status mhfp_apply_operator(mhfp_handle h, const double* d_x, double* d_y);

/* y = A_H x as the mixed-precision solve's Arnoldi step forms it
 * (precision = 1 set-ups only, else MHFP_ERR_STATE): float-float arithmetic
 * (every FP64 coefficient as a pair of FP32 words, exact products, sums
 * carried as unevaluated pairs) from x rounded to FP32 (the Arnoldi step's
 * vectors are FP32 values).  Relative error about 2^-44 of the sum of the
 * |terms| of a row.  The handle's FP32 work vector is overwritten. */
mhfp_status mhfp_apply_operator_ff(mhfp_handle h, const double* d_x, double* d_y);

/* y = A_H^T x.  The condensed operator satisfies A_H^T = D A_H D^-1 with
 * D = diag(I, -I, -dt I) (A_pu = -A_up^T, A_pip = A_ppi^T; A_uu, A_pipi,
 * Abar_pp + A_stab symmetric; Section 2 and the remark on symmetrisation
 * after Eq. stab_A), so this applies the same blocks with the signs and dt
 * factors of the off-diagonal blocks moved. */
mhfp_status mhfp_apply_operator_t(mhfp_handle h, const double* d_x, double* d_y);

/* Adjoint solve A_H^T lambda = g by FGMRES with the transposed
 * preconditioner M^T (lower block-triangular, forward substitution u, p, pi,
 * with the same symmetric V-cycles), on the equilibrated system
 * D_s A_H^T D_s; same stopping rule, stats and synchronisation as
 * mhfp_solve.  Not in the paper: the adjoint of its forward solve. */
mhfp_status mhfp_adjoint_solve(mhfp_handle h, const double* d_g, double* d_lambda, double tol, mhfp_stats* stats);

/* d_grad[T] -= lambda^T (d A_H / d ln kappa_T) x for every cell T (n_T
 * values, accumulated).  kappa_T scales the cell's whole diagonal
 * permeability, so W_T = A_ww,T^-1 is proportional to kappa_T and the
 * derivative is cell T's condensed flow contribution (Eq. hmfeSys):
 * p row dt (1^T W_T 1 p_T - (W_T 1)^T pi_T), pi rows W_T pi_T - W_T 1 p_T.
 * With lambda_n the adjoint states of a time-stepped misfit J, summing this
 * over the steps gives dJ / d ln kappa (the right-hand side does not depend
 * on kappa). */
mhfp_status mhfp_grad_logk(mhfp_handle h, const double* d_lambda, const double* d_x, double* d_grad);

/* New per-cell log-permeability for an existing, set-up handle (the
 * adjoint loop's parameter update; not in the paper, which solves for fixed
 * materials).  d_logk: device array of n_T values theta_T; every cell gets
 * kappa_T = exp(theta_T) times its create-time anisotropy ratios
 * (kappa_T,q / kappa_T,x), so theta_T = ln kappa_T,x.  Recomputes in place
 * what depends on kappa: the RT0 condensation W_T = A_ww,T^-1, W_T 1,
 * 1^T W_T 1 and Abar_pp (Eq. hmfeSys), B~_p and C~_pi (Eq. app_Bp, Section
 * 4), the equilibration D_s, the interface-pressure multigrid hierarchy
 * (same levels and launch schedules, no autotuning) and the FP32 copies.
 * A_uu, A_up, the stabilization and the displacement hierarchy do not
 * depend on kappa and are kept.  No device buffer of the handle is
 * reallocated (the first update allocates its scratch once: the anisotropy
 * ratios, the Galerkin product workspace and the dense-inverse workspace).
 * The captured solve graphs are dropped and captured again by the next
 * solve.  MHFP_ERR_ARG if some exp(theta_T) is not a positive finite
 * permeability (nothing is changed then).  Synchronises the stream. */
mhfp_status mhfp_update_logk(mhfp_handle h, const double* d_logk);

/* Misfit of one time step (not in the paper; the objective of the gradient
 * growth): *d_J += 1/2 inv_su2 sum_top (u_z - u_z*)^2 + 1/2 inv_sp2
 * sum_cells (p - p*)^2, and d_g (n values, overwritten) = dJ/dx.  The top
 * u_z* are the (nx+1)(ny+1) nodes of the plane k = nz in lexicographic
 * order; p* has n_T values.  d_J is a device scalar. */
mhfp_status mhfp_misfit(mhfp_handle h, const double* d_x, const double* d_uz_target, const double* d_p_target,
                        double inv_su2, double inv_sp2, double* d_J, double* d_g);

/* Adjoint right-hand side of step n: d_rhs = d_g + C^T lambda_{n+1}, where
 * C x = [0 ; A_pu u + S_eps|T| p ; 0] is how step n+1's right-hand side
 * depends on step n (Section 2.1).  d_lambda_next may be NULL (last step). */
mhfp_status mhfp_adjoint_rhs(mhfp_handle h, const double* d_g, const double* d_lambda_next, double* d_rhs);

/* z = M^-T v (the adjoint's preconditioner), unscaled. */
mhfp_status mhfp_apply_precond_t(mhfp_handle h, const double* d_v, double* d_z);

/* z = M^-1 v with the multigrid inner solves (Eq. hybridPrec back
 * substitution: pi, then p, then u), unscaled.  With formulation = 1 the
 * block-triangular M_II^(m) of Eq. (prec) by forward substitution: u and q,
 * then p. */
mhfp_status mhfp_apply_precond(mhfp_handle h, const double* d_v, double* d_z);

/* One V-cycle x = V(b) of the displacement (which = 0, length n_u) or the
 * interface-pressure (which = 1, length n_pi) hierarchy, in the precision
 * the solve uses: with precision = 1 the FP64 b is rounded to FP32, the
 * FP32 cycle runs, and x is its FP32 result widened to FP64.  With
 * formulation = 1, which = 1 is the hierarchy of C~_p (length n_p). */
mhfp_status mhfp_vcycle(mhfp_handle h, int which, const double* d_b, double* d_x);

/* y = A_l x for level `level` of hierarchy `which` (lengths from
 * mhfp_hierarchy).  Level 0 of which = 1 is C~_pi (C~_p with formulation =
 * 1); with formulation = 1, which = 2 is the one-level A_qq (length n_pi)
 * that the flux block's Chebyshev smoother runs on. */
mhfp_status mhfp_level_apply(mhfp_handle h, int which, int level, const double* d_x, double* d_y);

/* Hierarchy description (after mhfp_setup_precond); which as for
 * mhfp_level_apply. */
mhfp_status mhfp_hierarchy(mhfp_handle h, int which, mhfp_hierarchy_info* info);

/* Copy the diagonal approximation B~_p (n_p values; with formulation = 1
 * the diagonal of C~_p) and the equilibration scaling D_s (n values) into
 * device buffers (either may be NULL). */
mhfp_status mhfp_get_scalings(mhfp_handle h, double* d_btilde, double* d_ds);

/* Sizes: n_u = 3 (nx+1)(ny+1)(nz+1), n_p = nx ny nz, n_pi = number of faces
 * (every dof is kept, Table tab:grids counting). */
mhfp_status mhfp_sizes(mhfp_handle h, long long* n_u, long long* n_p, long long* n_pi);

/* Per-kernel-class device time accumulated with CUDA events on the
 * handle's stream while timing is enabled (kernel classes: 0 = Chebyshev
 * sweeps of the finest displacement level; 1 = FP64 operator apply; 2 =
 * Gram-Schmidt; 3 = preconditioner apply M^-1 with its precision
 * conversions; 4 = displacement V-cycle; 5 = interface-pressure V-cycle;
 * classes 4, 5 and 0 lie inside 3; 6 = the float-float operator of the
 * mixed-precision Arnoldi step).  bytes_per_launch is the algorithmic
 * traffic of classes 0-2 and 6 (matrix values, inverse diagonal blocks and
 * vectors touched once) and 0 for classes 3-5.
 * mhfp_timing(h, 1) resets and enables, mhfp_timing(h, 0) disables. */
mhfp_status mhfp_timing(mhfp_handle h, int enable);
mhfp_status mhfp_timing_read(mhfp_handle h, int kernel_class, long long* launches,
                             double* total_ms, double* bytes_per_launch);

/* ||D_s (b - A_H x)|| and ||D_s b|| without allocating anything (the paper
 * has no counterpart; this is a service of this library).
 *
 * Who needs it: callers that cannot call cudaMalloc at this point, such as
 * hosts that hand all device memory to their own pool allocator up front, or
 * loops that must not allocate once running.  mhfp_solve computes the same
 * norm through the handle's Krylov workspace, which it allocates (about
 * (2m+4) n doubles) on its first call; this entry point needs only an
 * assembled and set-up handle.
 *
 * d_b, d_x: device vectors of length n (layout above).  d_out: device buffer
 * of 2 doubles, receives { ||D_s (b - A_H x)||_2, ||D_s b||_2 }, with D_s the
 * equilibration of mhfp_solve; their ratio is mhfp_solve's true relative
 * residual.
 *
 * Scratch: a file-scope static __device__ array of 65536 x 2 doubles (1 MiB)
 * that every GPU which loads the library holds until the process exits.
 * The call needs ceil(n_nodes/256) + ceil(n_T/256) + ceil(n_faces/256) row
 * blocks (one partial-sum pair each); meshes needing more than 65536 are
 * rejected with MHFP_ERR_ARG and a message saying so (a cube of 149^3 cells
 * needs 65,132 and is accepted, 150^3 needs 66,449 and is not; 128^3 needs
 * 41,346).  The first call on each device looks up the array's device
 * address with cudaGetSymbolAddress (with that device current) and caches
 * it for the life of the process, so the device's primary context must not
 * be reset (cudaDeviceReset) between calls; make that first call before any
 * stream capture.  All calls share the array and it keeps the last
 * call's partial sums; every call overwrites each partial sum it reads, so
 * nothing has to start at zero, but calls that overlap on the GPU (for
 * example on two streams) race and must be serialised by the caller. */
mhfp_status mhfp_residual_norm_noalloc(mhfp_handle h, const double* d_b, const double* d_x, double* d_out);

/* Number of kernels this library has launched in the process so far (all
 * handles); a caller brackets a region with two reads to count its launches. */
long long mhfp_launch_count(void);

const char* mhfp_last_error(mhfp_handle h);
const char* mhfp_status_string(mhfp_status s);
void mhfp_destroy(mhfp_handle h);

#ifdef __cplusplus
}
#endif
#endif /* MHFP_H */
