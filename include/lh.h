/*
 * lh.h - C ABI of the B300-native implicit high-order Lagrangian hydrodynamics library.
 *
 * The library evaluates, matrix-free and sum-factorised on tensor-product quad/hex
 * elements, the stage residual of the implicit time step of the paper
 * "Implicit Lagrangian Hydrodynamics with High-Order Finite Elements" (arxiv 2609.16424)
 * and its Jacobian actions, and drives the Newton-Krylov solve of that stage.
 *
 * Discretisation (paper Sec. 2.1): kinematic space Q_k (continuous, order 1 <= k <= 4)
 * for position x and velocity v, thermodynamic space Q_{k-1} (discontinuous) for the
 * specific internal energy e.  Readings of points the paper leaves open: H1 basis =
 * Lagrange at Gauss-Lobatto points, L2 basis = Lagrange at Gauss-Legendre points,
 * quadrature = Gauss-Legendre with 2k points per direction (or lh_mesh_desc.quad_1d).
 *
 * State vectors (all double unless stated):  U = [ x | v | e ]
 *   x, v : dim components, each all N_V H1 nodes of the (k n_0 + 1) x (k n_1 + 1)
 *          [x (k n_2 + 1)] lattice, x-fastest;                       length dim*N_V each
 *   e    : element-major, element e = e0 + n_0 (e1 + n_1 e2), then its k^dim dofs
 *          x-fastest;                                                 length N_E = NE k^dim
 *   n = 2 dim N_V + N_E unknowns.
 *
 * Stage residual (paper Sec. 3.5, Eq. (21), at w = u + tau k), mass-weighted form that
 * matches the blocks of Eq. (23):
 *   R_x = k_x - w_v
 *   R_v = M_V k_v + F(w) . 1         rows of fixed normal velocity (bc_mask): R_v = k_v
 *   R_e = M_E k_e - F(w)^T w_v - b(w)
 * with M_V, M_E, F from Eq. (7), the stress of Eqs. (11), (13)-(20), rho = rho0 detJ0 /
 * detJ at quadrature points, and b the optional Taylor-Green energy source.
 *
 * Conventions:
 *  - Vector arguments are DEVICE pointers owned by the caller unless stated otherwise.
 *  - Work is queued on the mesh's stream (lh_mesh_desc.stream / lh_set_stream); calls
 *    that return host scalars synchronise that stream.
 *  - No exception crosses the ABI.  Failures return a status; lh_last_error(mesh)
 *    returns a message for the last failing call on that mesh.
 */
#ifndef LH_H
#define LH_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lh_mesh lh_mesh;

typedef enum {
  LH_OK = 0,
  LH_EINVAL = 1,      /* invalid argument (NULL pointer, unsupported order/dim, ...) */
  LH_ECUDA = 2,       /* a CUDA runtime call failed */
  LH_ENOMEM = 3,      /* device allocation failed */
  LH_ETANGLED = 4,    /* a quadrature point has det J <= 0 */
  LH_ENOCONV = 5,     /* Newton did not reach its tolerance; state left unchanged */
  LH_ENONFINITE = 6   /* a residual norm is NaN or Inf */
} lh_status;

typedef enum {
  LH_FP64 = 0,        /* double in, double out, double arithmetic */
  LH_FP32 = 1,        /* float in, float out, float arithmetic (state gathered in double) */
  LH_FP32_LIN = 2,    /* float in, float out, float arithmetic from the linearisation record
                         of the last lh_linearize (same u, k, tau pointers/value required) */
  LH_TF32 = 3,        /* as LH_FP32_LIN, with the element contractions (B and B^T of Eq. (8))
                         on the tensor cores: TF32 operands, FP32 accumulation; quadrature-
                         point arithmetic in float.  2D orders 1-4 and 3D orders 1-2. */
  LH_BF16 = 4         /* as LH_TF32 with BF16 operands */
} lh_prec;

/* Mesh and model description.  Call lh_mesh_desc_init first to get the defaults. */
typedef struct {
  int dim;                 /* 2 or 3 */
  int n[3];                /* elements per direction (n[2] ignored for dim 2) */
  double lo[3], hi[3];     /* box corners */
  int order;               /* H1 order k, 1..4 (L2 order k-1) */
  int quad_1d;             /* Gauss points per direction; 0 -> 2k (only 2k is supported) */
  const double* rho0;      /* HOST array [NE] of initial densities, or NULL -> rho0_value */
  const double* gamma;     /* HOST array [NE] of adiabatic indices, or NULL -> gamma_value */
  double rho0_value;       /* default 1.0 */
  double gamma_value;      /* default 1.4 */
  unsigned bc_mask;        /* bit 2c+s: v_c = 0 on the face of axis c at low (s=0) / high
                              (s=1) end; default all faces */
  int visc;                /* smooth artificial viscosity mu_imp (Eq. (13)) on/off; default 1 */
  double q1, q2, psi0;     /* Eq. (13), (17); defaults 0.5, 1.0, 0.5 */
  double eps_e;            /* Eq. (19); default 1e-6 */
  double h0;               /* Eq. (14) initial length scale; <= 0 -> (|Omega0| / NE)^(1/dim) */
  double h_coarse;         /* Eq. (18) coarse length scale; <= 0 -> h0 */
  int tg_source;           /* Taylor-Green manufactured energy source (dim 2); default 0 */
  void* stream;            /* cudaStream_t for all work; NULL = legacy default stream */
} lh_mesh_desc;

/* Fill *desc with the defaults listed above (unit box, dim 3, 4^3 elements, order 2). */
void lh_mesh_desc_init(lh_mesh_desc* desc);

/* Create a mesh: builds the 1D bases and quadrature, copies materials to the device and
 * allocates the mesh's work buffers (element scratch, reduction partials).  Memory owned
 * by the mesh is released by lh_mesh_destroy.  Writes *out = NULL on failure. */
lh_status lh_mesh_create(const lh_mesh_desc* desc, lh_mesh** out);
lh_status lh_mesh_destroy(lh_mesh* mesh);

/* Host array out[6] = { NE, N_V, N_E, n, NQ (quadrature points), dim }. */
lh_status lh_sizes(const lh_mesh* mesh, long long* out);

/* Change the stream used by all later calls on this mesh. */
lh_status lh_set_stream(lh_mesh* mesh, void* stream);

/* x0: device [dim*N_V]; writes the undeformed node positions of the box. */
lh_status lh_initial_nodes(lh_mesh* mesh, double* x0);

/* Stage residual R(k; tau, u) of Eq. (21).  u, k, r: device [n] double.  r may not alias
 * u or k.  If min_detj (HOST pointer) is non-NULL the call synchronises and stores the
 * minimum over quadrature points of det J at w (the line-search test of Sec. 3.5). */
lh_status lh_residual(lh_mesh* mesh, const double* u, const double* k, double tau,
                      double* r, double* min_detj);

/* Jacobian action out = (dR/dk)(u, k; tau) dk of Eq. (22), matrix-free (paper Sec. 3.1,
 * Eq. (10): transfers B, G unchanged, only the quadrature-point kernel differentiated).
 * dk and out are device [n] arrays of double (LH_FP64) or float (LH_FP32); u and k are
 * double.  With LH_FP32 the state is gathered and re-centred per element in double,
 * then all arithmetic runs in float.  LH_FP32_LIN, LH_TF32 and LH_BF16 take float dk/out
 * and need the record of a preceding lh_linearize(u, k, tau); LH_TF32/LH_BF16 return
 * LH_EINVAL for 3D orders >= 3 (the dense element operator does not fit in shared memory).
 * A tensor-core wait that times out writes NaN into the affected element rows and is
 * reported by the next lh_newton_step (LH_ECUDA) and by lh_tc_status.  The same holds for
 * LH_FP32_LIN on elements of 64 points (3D Q2, 2D Q4), whose kernel copies each element's
 * record into shared memory asynchronously and waits on the copy with a bounded wait
 * (about 1 s): if that wait runs out, the rows of the warp's later elements are NaN, a
 * failing lh_newton_step reports LH_ECUDA and lh_tc_status reports it. */
lh_status lh_jvp(lh_mesh* mesh, const double* u, const double* k, double tau,
                 const void* dk, void* out, lh_prec prec);

/* Box decomposition (paper Sec. 2.2, Eq. (8) with P != I).  A partition is a mesh of a
 * sub-box of the global box: same element size, the global h0 and h_coarse, walls only on
 * the global boundary (the shared face unmasked).  On a shared face the velocity rows of
 * the residual and of J.w hold each side's partial sums (mass and force terms of its own
 * elements); summing the two sides' values gives the global operator there.  x rows,
 * fixed velocity rows and L2 rows are complete on each side.
 * face = 2 axis + side (side 0 low, 1 high, numbered as bc_mask).  buf holds
 * dim * (nodes of the face) entries, component-major, the face nodes lexicographic over the
 * remaining axes.  prec LH_FP64: r, buf double; any other precision: float.
 * lh_halo_pack copies the velocity rows of the face nodes of r into buf; lh_halo_add adds
 * buf (the other side's packed rows) into the free velocity rows of r.  Asynchronous. */
lh_status lh_halo_len(const lh_mesh* mesh, int face, long long* len);
lh_status lh_halo_pack(lh_mesh* mesh, int face, const void* r, void* buf, lh_prec prec);
lh_status lh_halo_add(lh_mesh* mesh, int face, const void* buf, void* r, lh_prec prec);

/* Status of the bounded waits of the tensor-core J.w (on the tensor cores) and of the
 * LH_FP32_LIN J.w of 64-point elements (on its record copies): LH_OK, or LH_ECUDA if one of
 * them timed out since the last call or the mesh's creation (synchronises; clears the
 * flag). */
lh_status lh_tc_status(lh_mesh* mesh);

/* Poll limit of every bounded wait of the tensor-core J.w on its MMA completions (process
 * wide, all devices; default 2^22 polls, about 1 s at most).  After the first wait that runs
 * out, the kernel skips all later MMA issues and waits of that launch, writes NaN into the
 * element rows it has not finished, sets the flag lh_tc_status reports, lets the MMAs it
 * already issued drain (one more wait with the default limit) and releases its tensor
 * memory.  A diagnostic switch: a limit of 0 makes every launch take that path at once.
 * Returns the previous limit. */
unsigned lh_tc_set_wait_polls(unsigned polls);

/* Linearisation record (partial assembly of the tangent, paper Sec. 2.2: store the
 * quadrature-point data once, reuse it for every action): evaluates the residual at
 * w = u + tau k in FP64 and keeps, rounded to float, the linearisation of the
 * quadrature-point map at every point ([NE][25 (3D) or 18 (2D)][quadrature points]:
 * J^-1, grad v, and the pressure and linearised viscosity scalars of Eqs. (11)-(20): W, p,
 * dp/de, mu and the three coefficients of dmu in theta = d detJ / detJ, d(div v) and de).
 * Later lh_jvp calls with LH_FP32_LIN, LH_TF32 or LH_BF16 and the same u, k (pointers)
 * and tau apply the linearised map instead of re-evaluating the point kernel.
 * lh_newton_step with a reduced-precision J.w writes the record at every Newton iterate
 * and invalidates it on return.  Asynchronous; allocates the record on first use. */
lh_status lh_linearize(lh_mesh* mesh, const double* u, const double* k, double tau);

/* Diagonal of the velocity block dR_v/dk_v = M_V + tau dF.1/dv of the stage Jacobian at
 * (u, k, tau) (the block the paper's Eq. (23) preconditions): 1 on fixed rows, diag(M_V) plus
 * tau times the viscous part (from the FP32 linearisation record, which this call writes as
 * lh_linearize does) on free rows.  u, k: device [n]; out: device double [dim * NV], the
 * velocity rows in the layout of the state.  Asynchronous. */
lh_status lh_jvv_diagonal(lh_mesh* mesh, const double* u, const double* k, double tau, double* out);

/* Transpose action out = (dR/dk)^T y (paper Sec. 3.1: transpose actions share the
 * gather-apply-scatter structure).  LH_FP64: y, out device [n] double, the point kernel's
 * hand-written reverse mode.  LH_FP32_LIN: y, out float, the transpose of the linearised
 * point map of the record of a preceding lh_linearize(u, k, tau). */
lh_status lh_jtvp(lh_mesh* mesh, const double* u, const double* k, double tau,
                  const void* y, void* out, lh_prec prec);

/* Mass matrices of Eq. (7) (constant in time since rho detJ = rho0 detJ0).
 * which = 0: H1 mass M_V applied to each of the dim components, f/out device [dim*N_V];
 * which = 1: L2 mass M_E (block diagonal), f/out device [N_E]. */
lh_status lh_mass_apply(lh_mesh* mesh, int which, const double* f, double* out);

/* Solve M z = rhs.  which = 0: M_V, Jacobi-preconditioned CG per component to relative
 * tolerance rtol (maxit iterations); which = 1: M_E by the exact per-element inverse
 * (rtol, maxit ignored).  *iters (HOST, may be NULL) receives the CG iterations used.
 * Synchronises.  Returns LH_ENOCONV if CG stopped at maxit above tolerance. */
lh_status lh_mass_solve(lh_mesh* mesh, int which, const double* rhs, double* sol,
                        double rtol, int maxit, int* iters);

/* Apply the Newton-GMRES preconditioner of lh_newton_step (a stand-in for Eq. (23)):
 *   z = P^-1 r,  P^-1 = [I, tau M_V^-1, 0; 0, M_V^-1, 0; 0, 0, M_E^-1],
 * with M_V^-1 the diagonal of M_V (kind 0) or its exact Kronecker-product inverse (kind 1,
 * float arithmetic; exact for uniform rho0) on free velocity rows and identity on fixed rows.
 * Kind 2 of lh_newton_opts.precond (the diagonal of M_V + tau dF/dv at the current Newton
 * iterate) exists only inside lh_newton_step and is rejected here with LH_EINVAL; its
 * diagonal is available from lh_jvv_diagonal.
 * r, z: device [n] double, not aliased.  Asynchronous. */
lh_status lh_precond(lh_mesh* mesh, int kind, double tau, const double* r, double* z);

/* Explicit time step estimate used to set "CFL multiple" time steps (reading: the
 * paper's first-step CFL refers to an estimate it does not print):
 *   dt = min_q h_min,q / (c_s,q + mu_q / (rho_q h_min,q)),  h_min,q = sigma_min(J_q) / k.
 * u device [n]; *dt (HOST).  Synchronises. */
lh_status lh_dt_estimate(lh_mesh* mesh, const double* u, double* dt);

/* L1 velocity error of the 2D Taylor-Green vortex (Sec. 4.1): sum over elements and the
 * 2k-point Gauss rule of alpha_q detJ_q |v_h(x_q) - v*(x_q)|_2 with the steady exact
 * velocity v* = (sin pi x cos pi y, -cos pi x sin pi y) at the moved points x_q.  u: device
 * state [n]; l1: HOST output.  LH_EINVAL on a 3D mesh.  Synchronises. */
lh_status lh_tg_velocity_error(lh_mesh* mesh, const double* u, double* l1);

/* Kinetic 1/2 v^T M_V v and internal 1^T M_E e energies of state u (HOST outputs). */
lh_status lh_energies(lh_mesh* mesh, const double* u, double* kinetic, double* internal);

typedef struct {
  double newton_rtol;      /* ||R|| <= rtol ||R^0|| stops; default 1e-10 */
  double newton_atol;      /* ... or ||R|| <= atol; default 0 */
  double gmres_rtol;       /* relative tolerance of each linear solve; default 1e-12 */
  int newton_maxit;        /* default 20 */
  int gmres_maxit;         /* total GMRES iterations per linear solve; default 60 */
  int restart;             /* GMRES restart length (<= 64); default 30 */
  int max_halvings;        /* line-search halvings of the Newton step; default 10 */
  lh_prec jvp_prec;        /* precision of the J.w inside GMRES; default LH_FP64.  LH_FP32,
                              LH_TF32 and LH_BF16 use an FP32 Krylov basis and the linearisation
                              record written at every Newton iterate */
  int precond;             /* velocity block of the preconditioner: 0 = diagonal of M_V,
                              1 = exact M_V inverse as a Kronecker product of 1D inverses
                              (exact for uniform rho0; rho0-scaled otherwise); 2 = inverse of
                              the diagonal of the paper's velocity block M_V + tau dF/dv
                              (Eq. (23)), recomputed from the linearisation record at every
                              Newton iterate, each free entry kept at >= 0.5 diag(M_V) (the
                              viscous tangent is not sign-definite) (needs jvp_prec other than
                              LH_FP64); 3 = a Chebyshev iteration (the matrix-free smoother the
                              paper's Sec. 5 points to) on the velocity Schur block
                              S = M_V + tau dF.1/dv + tau^2 dF.1/dx (the block Eq. (23)'s velocity
                              part approximates, with the exact elimination of the x rows),
                              Jacobi-scaled by the diagonal of kind 2, S applied by the record
                              J.w (reduced-precision J.w only); default 1 */
  int forcing;             /* 0: every linear solve to gmres_rtol (default); 1: adaptive
                              forcing terms (Eisenstat and Walker 1996, choice 2 with gamma 0.9,
                              alpha 2, and the safeguard against oversolving the last step):
                              eta_0 = eta_max, eta_k = 0.9 (|R_k| / |R_{k-1}|)^2, kept >= 0.9
                              eta_{k-1}^2 when that exceeds 0.1 and >= 0.5 target / |R_k|,
                              clamped to [gmres_rtol, eta_max] */
  double eta_max;          /* largest forcing term; default 0.1 */
  int scaled_norm;         /* 0: the Newton test and GMRES use ||R||_2 (default); 1: both use
                              ||W R||_2 with W = 1 on x rows and fixed v rows, 1/(M_V)_ii on
                              free v rows and (M_E^-1)_ii on e rows (GMRES then solves the
                              row-scaled system W J dk = -W R), so the v and e rows are not
                              weighted by mass factors that shrink with the mesh size; stats
                              r0 / rfinal are then in that norm */
  int cheb_degree;         /* precond 3: degree of the Chebyshev polynomial (>= 1; degree m
                              costs m - 1 Jacobian actions per application); default 3 */
  double cheb_ratio;       /* precond 3: the Chebyshev interval is [b / ratio, b], b = 1.1 x the
                              largest eigenvalue of D^-1 S estimated by 5 power steps at every
                              Newton iterate; default 20 */
  int arnoldi;             /* driver of the Arnoldi iterations of an FP32-basis GMRES: 1 = on
                              the device (default): each restart cycle is one launch of a CUDA
                              graph whose WHILE conditional node repeats one iteration (operator,
                              both Gram-Schmidt passes, the exact-norm fallback, the Givens
                              rotation and the stopping test, all in kernels) until the device
                              ends the cycle; the host reads the cycle's Hessenberg matrix once.
                              The first solve with a new operator kind runs on the host (the
                              kernels' one-time set-up cannot be recorded).  0 = host loop, one
                              read-back per iteration.  Same arithmetic either way (the Givens
                              rotations in double on the device instead of the host). */
} lh_newton_opts;

typedef struct {
  int newton_its;          /* Newton iterations taken */
  int gmres_its_total;     /* GMRES iterations over all linear solves */
  int backtracks;          /* line-search halvings */
  int residual_evals;      /* residual evaluations (incl. line-search trials) */
  int jvp_evals;           /* Jacobian actions */
  int reorth;              /* second Gram-Schmidt passes taken */
  double r0, rfinal;       /* ||R|| at the initial guess and at exit */
  double min_detj;         /* min det J at the accepted stage state */
  int newton_its_max;      /* most Newton iterations of one stage solve (the count the
                              Newton-count time-step control of Sec. 4 reads) */
} lh_step_stats;

void lh_newton_opts_init(lh_newton_opts* opts);

/* One implicit midpoint step (paper Sec. 4.1, SD2): tau = dt/2, solve R(k; tau, u) = 0
 * by inexact Newton-GMRES with the right preconditioner
 *   P^-1 = [I, tau M_V^-1, 0; 0, M_V^-1, 0; 0, 0, M_E^-1]
 * (M_V^-1 as opts.precond selects; the upper block eliminates dR_x/dk_v = -tau I exactly;
 * a stand-in for the block-diagonal AMG of Eq. (23)) with the det J line search of Sec.
 * 3.5, then u <- u + dt k.  u: device [n] in/out.  k_prev: device [n] initial guess on
 * entry and the converged k on exit, or NULL (zero initial guess).  Synchronises.
 * On LH_ENOCONV / LH_ETANGLED / LH_ENONFINITE u and k_prev are left unchanged. */
lh_status lh_newton_step(lh_mesh* mesh, double* u, double* k_prev, double dt,
                         const lh_newton_opts* opts, lh_step_stats* stats);

/* Solve one SDIRK stage system R(k; tau, u_base) = 0 (Eq. (21)) by the Newton-GMRES of
 * lh_newton_step, without changing any state.  u_base: device [n] stage base state (read
 * only).  k: device [n], the initial guess on entry and the converged stage increment on
 * exit (unchanged on failure); must not alias u_base.  tau > 0: the stage scaling (the
 * diagonal entry of the tableau times dt).  stats as for lh_newton_step (also written on
 * LH_ENOCONV).  Synchronises. */
lh_status lh_stage_solve(lh_mesh* mesh, const double* u_base, double* k, double tau,
                         const lh_newton_opts* opts, lh_step_stats* stats);

/* One step of the SDIRK scheme SD<scheme> of Sec. 4: 2 = implicit midpoint (one stage,
 * tau = dt/2; the same arithmetic as lh_newton_step), 3 = the 3-stage L-stable method of
 * order 3 (Alexander; diagonal gamma = 0.43586652150845899...), 4 = the 3-stage A-stable
 * method of order 4 (Crouzeix; gamma = 1/2 + cos(pi/18)/sqrt(3)).  Stage i solves
 * R(k_i; a_ii dt, u + dt sum_{j<i} a_ij k_j) = 0 from the initial guess k_{i-1} (k_prev, or
 * zero, for the first stage); then u <- u + dt sum_i b_i k_i.
 *  u: device [n] in/out.  k_prev: device [n] first-stage initial guess on entry and the last
 *  stage's k on exit, or NULL.  stats: sums over the stages of the counts, newton_its_max
 *  the largest stage count, r0 / rfinal the largest and min_detj the smallest over the
 *  stages.  Allocates 4 n doubles of stage storage on the first call.  Synchronises.
 *  On any error u and k_prev are left unchanged; LH_EINVAL for a scheme other than 2-4. */
lh_status lh_sdirk_step(lh_mesh* mesh, int scheme, double* u, double* k_prev, double dt,
                        const lh_newton_opts* opts, lh_step_stats* stats);

/* ---- Time loop with the paper's implicit time step control (Sec. 4, "implicit time step
 * control"; the first step at FS-CFL times the explicit estimate of lh_dt_estimate).
 * After a step whose largest stage solve took <= grow_its Newton iterations dt grows by
 * `grow`; with more, up to reject_its - 1, dt is kept; a step with >= reject_its iterations,
 * or whose solve fails (LH_ENOCONV, LH_ETANGLED, LH_ENONFINITE), is rejected: the state goes
 * back to the start of the step and the step is retried with shrink * dt.  The last step is
 * clipped to reach t_end exactly.
 * Initial guess: each step starts from the previous step's last-stage increment (zero at
 * the first step, or k_prev's content on entry).  The paper leaves the initial guess open;
 * a predicted guess (for example the learned proposal of lh_mlp_*) is formed by the caller
 * into k_prev between calls of lh_newton_step, since it needs the caller's network and the
 * increments of earlier steps; this loop does not call a predictor. */
typedef struct {
  int scheme;              /* 2 = implicit midpoint, 3 = SD3, 4 = SD4 (lh_sdirk_step); default 2 */
  double fs_cfl;           /* first dt = fs_cfl * lh_dt_estimate(u); default 2 */
  double dt0;              /* if > 0, the first dt instead (fs_cfl ignored); default 0 */
  double grow, shrink;     /* dt factors; defaults 1.05 and 0.85 */
  int grow_its;            /* <= this many Newton iterations: grow; default 1 */
  int reject_its;          /* >= this many: reject; default 4 */
  int enlarge;             /* 0: never grow dt (rejections still shrink it); default 1 */
  int max_steps;           /* accepted steps at most; default 1000000 */
  int max_attempts;        /* attempts (accepted or not) at most, <= 0: no limit; default 0 */
  double dt_min;           /* LH_ENOCONV once the controller's dt falls below this; default 0 */
} lh_advance_opts;

typedef struct {           /* one attempt of the time loop */
  double dt;               /* the controller's dt at the attempt */
  double h;                /* the step taken (dt, or less for the last step) */
  int newton_its;          /* largest stage Newton count, or -1 if the solve failed */
  int accepted;
} lh_advance_attempt;

typedef struct {
  int steps, rejected, attempts;
  double t;                /* time reached (t_end unless a limit ended the loop) */
  double dt_next;          /* the controller's dt after the last attempt */
  long long newton_its, gmres_its;   /* totals over the accepted steps */
} lh_advance_stats;

void lh_advance_opts_init(lh_advance_opts* opts);

/* Advance u from t = 0 to t_end (in place) with the control above.  u: device [n];
 * k_prev: device [n] first initial guess on entry and the last accepted step's increment on
 * exit, or NULL (zero first guess, kept internally).  nopts: the Newton-GMRES options of
 * every stage solve (NULL: defaults).  hist: HOST array of hist_cap attempts (may be NULL);
 * the first min(attempts, hist_cap) attempts are written.  Allocates 2 n doubles of trial
 * state on the first call.  Synchronises.  Errors other than the rejectable solve failures
 * end the loop and are returned with u at the last accepted step; LH_ENOCONV also if dt
 * falls below dt_min. */
lh_status lh_advance(lh_mesh* mesh, double* u, double* k_prev, double t_end, const lh_newton_opts* nopts,
                     const lh_advance_opts* aopts, lh_advance_stats* stats, lh_advance_attempt* hist,
                     int hist_cap);

/* The same loop without a mesh (host only, no GPU): each attempt's Newton count is taken in
 * order from counts[0 .. ncounts) (a negative entry: the solve failed; past the end: 2), the
 * explicit estimate is dt_est.  Lets the controller be checked without solving anything. */
lh_status lh_advance_replay(const int* counts, int ncounts, double dt_est, double t_end,
                            const lh_advance_opts* aopts, lh_advance_stats* stats, lh_advance_attempt* hist,
                            int hist_cap);

/* ---- Explicit path: the paper's comparison method (Sec. 2.2, Sec. 4.1: ORIG-E / dFEM-E)
 * Eqs. (6a)-(6b) integrated explicitly: M_V dv/dt = -F.1 (dv/dt = 0 on fixed rows),
 * M_E de/dt = F^T v + b, dx/dt = v, with F's quadrature data formed once per stage and
 * applied twice (Sec. 2.2).  M_V is inverted by conjugate gradients preconditioned with the
 * Kronecker-product inverse of lh_precond kind 1 (exact for uniform rho0, so a few
 * iterations reach rounding); M_E^-1 is exact.  Viscosity: the smooth mu_imp of Eqs.
 * (13)-(18) (visc_model 0) or the original tensor viscosity mu_exp of Sec. 3.4 (visc_model
 * 1; the paper defers its ingredients to Dobrev et al. 2012, Sec. 6.2; readings:
 * mu = rho (q2 l^2 |lambda_1| + q1 psi_1 psi_0 l c_s), (lambda_1, s_1) the smallest
 * eigenpair of eps(v), l = l0 |J J0^-1 s_1|, psi_1 = [lambda_1 < 0], psi_0 = 1 or, with
 * the vorticity switch, |div v| / (sqrt(dim) |grad v|_F)).  Integrators (Sec. 4.1; the
 * schemes are defined in Dobrev et al. 2012, Sec. 7.1): scheme 2 = RK2-average
 *   v_h = v + dt/2 a(U), e_h = e + dt/2 g(U, v_h), x_h = x + dt/2 v_h;
 *   v' = v + dt a(U_h), vbar = (v + v') / 2, e' = e + dt g(U_h, vbar), x' = x + dt vbar
 * with a = -M_V^-1 F.1 and g(U, w) = M_E^-1 (F(U)^T w + b) (total energy changes by
 * exactly dt 1^T b per step); 3 = SSP RK3 (Shu-Osher); 4 = classical RK4, both on
 * dU/dt = (v, a(U), g(U, v)).  All in FP64. */
typedef struct {
  int scheme;              /* 2 = RK2-average, 3 = RK3 SSP, 4 = RK4; default 2 */
  int visc_model;          /* 0 = mu_imp (the mesh's q1, q2, psi0), 1 = mu_exp; default 1 */
  double q1_exp, q2_exp;   /* mu_exp coefficients; defaults 0.5 and 2 */
  double l0_exp;           /* mu_exp initial length l0; 0 = h0 / order (default) */
  int vorticity;           /* mu_exp vorticity switch psi_0; default 0 (psi_0 = 1) */
  double cfl;              /* lh_explicit_advance: dt = cfl x the explicit estimate; default 0.5 */
  double mass_rtol;        /* relative tolerance of the M_V solves; default 1e-13 */
  int mass_maxit;          /* CG iterations per M_V solve at most; default 200 */
} lh_explicit_opts;

typedef struct {
  int steps, rejected;     /* accepted / repeated steps (lh_explicit_advance) */
  double t;                /* time reached */
  double dt_last;          /* the controller's dt after the last step */
  long long force_evals;   /* evaluations of F's quadrature data */
  long long mass_iters;    /* CG iterations over all M_V solves */
} lh_explicit_stats;

void lh_explicit_opts_init(lh_explicit_opts* opts);

/* F's two applications at state u (device [n]): f1 = F(u).1 (device [dim N_V], every row
 * assembled, fixed rows included) and ftw = F(u)^T w + b (device [N_E]; w: device [dim N_V]
 * velocity field, or NULL for the velocity of u; b the Taylor-Green source if enabled).
 * Either output may be NULL.  dt_est (HOST, may be NULL; then no synchronisation): the
 * explicit estimate min_q h_min / (c_s + mu / (rho h_min)) of lh_dt_estimate with the
 * viscosity model of opts.  Allocates the explicit work arrays on first use. */
lh_status lh_force(lh_mesh* mesh, const double* u, const double* w, const lh_explicit_opts* opts, double* f1,
                   double* ftw, double* dt_est);

/* One explicit step of size dt in place on u (device [n]).  Synchronises.  LH_ENOCONV if a
 * mass solve did not reach mass_rtol (u is then unchanged); LH_ENONFINITE if the new state is
 * not finite (u unchanged). */
lh_status lh_explicit_step(lh_mesh* mesh, double* u, double dt, const lh_explicit_opts* opts,
                           lh_explicit_stats* stats);

/* Explicit run from t = 0 to t_end in place on u with the step control of the explicit
 * method (reading of Dobrev et al. 2012, Sec. 7.3, which the paper cites): the first dt is
 * cfl x the estimate at u; after each step the estimate at the new state (cfl x) is
 * compared with the step taken: below it, the step is repeated with 0.85 dt; above 1.25 dt,
 * the next dt is 1.02 dt.  The last step is clipped to reach t_end.  max_steps bounds the
 * accepted steps.  Synchronises. */
lh_status lh_explicit_advance(lh_mesh* mesh, double* u, double t_end, int max_steps, const lh_explicit_opts* opts,
                              lh_explicit_stats* stats);

/* The Butcher tableau lh_sdirk_step uses for a scheme (host only, no GPU): *stages = s, A:
 * HOST double[9] row-major 3 x 3 (entries beyond s x s are 0), b: HOST double[3].
 * LH_EINVAL for a scheme other than 2-4. */
lh_status lh_sdirk_tableau(int scheme, int* stages, double* A, double* b);

/* Stage residual R(k; tau, u), the same operator and kernel as lh_residual, for callers
 * that must not allocate device memory when they call the library (for example code
 * inside a host application that owns all device memory through its own pool, or
 * latency-critical loops that cannot accept cudaMalloc's implicit synchronisation).
 * The paper has no counterpart; it is a deployment variant.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.  The
 *    element scratch (16 MiB), per-block minima (512 KiB) and 1D tables of orders 1-4
 *    (8 KiB) live in file-scope __device__ arrays that every GPU loading the library holds
 *    until exit.
 *  - Maximum size: NE * dim * (order+1)^dim <= 2^21 (e.g. 3D Q2: NE <= 25890; 2D Q2:
 *    NE <= 116508); larger meshes are rejected with LH_EINVAL and a message naming the
 *    limit.  No min det J is returned.
 *  - desc: as for lh_mesh_create (desc->rho0 / desc->gamma host arrays are ignored; the
 *    work runs on desc->stream).  rho0, gamma: DEVICE arrays [NE] of initial densities and
 *    adiabatic indices.  u, k, r: DEVICE [n] double, r must not alias u or k.
 *  - The first call on each device looks up the device addresses of those arrays
 *    (cudaGetSymbolAddress) and writes the tables of all orders with synchronous copies;
 *    later calls copy nothing.  Make that first call before any stream capture.
 *  - Every call shares the arrays and overwrites them (the scratch keeps the last call's
 *    contents; nothing in it must start at zero).  Calls that overlap on the GPU, e.g. on
 *    two streams at once, race on them.
 *  - Asynchronous on desc->stream; errors are reported by lh_last_error(NULL). */
lh_status lh_residual_noalloc(const lh_mesh_desc* desc, const double* rho0, const double* gamma,
                              const double* u, const double* k, double tau, double* r);

/* ---- Learned Newton initial guess (an addition to the paper's method) -------------------
 * The paper starts each stage solve from the previous increment (Sec. 3.5 leaves the
 * initial guess open).  A per-element MLP predicts the correction k^n - k^{n-1} from the
 * element dofs of the last two increments and dt:
 *   Linear(n_in, h) -> GELU -> [Linear(h, h) -> GELU] x (layers - 1) -> Linear(h, n_out),
 * exact GELU z Phi(z), mean-squared-error loss, Adam (beta 0.9 / 0.999, eps 1e-8).  Matrix
 * products on the tensor cores with BF16 operands and FP32 accumulation; FP32 master weights.
 * Parameters are flat FP32: W_1 [h][n_in], b_1 [h], ..., W_last [n_out][h], b_last [n_out].
 * All arrays are DEVICE float arrays, row-major [M][features], unless stated. */
typedef struct lh_mlp lh_mlp;
/* init_params: HOST array of lh_mlp_num_params floats, or NULL (zeros).  Synchronises. */
lh_status lh_mlp_create(int n_in, int hidden, int layers, int n_out, const float* init_params, void* stream,
                        lh_mlp** out);
lh_status lh_mlp_destroy(lh_mlp* mlp);
long long lh_mlp_num_params(const lh_mlp* mlp);
/* copy the parameters to a HOST array (synchronises) */
lh_status lh_mlp_params(lh_mlp* mlp, float* host_out);
/* Y [M][n_out] = network(X [M][n_in]) */
lh_status lh_mlp_forward(lh_mlp* mlp, const float* X, int M, float* Y);
/* gradient of the mean squared error of network(X) against T [M][n_out]; grad_out (device,
 * may be NULL) receives it; *loss (HOST, may be NULL) the loss (synchronises if non-NULL) */
lh_status lh_mlp_grad(lh_mlp* mlp, const float* X, const float* T, int M, float* grad_out, double* loss);
/* one Adam step on the batch (X, T) with learning rate lr; *loss as in lh_mlp_grad */
lh_status lh_mlp_train_step(lh_mlp* mlp, const float* X, const float* T, int M, float lr, double* loss);
const char* lh_mlp_last_error(const lh_mlp* mlp);
/* Features of every element: X [NE][2 F1 + 1], F1 = 2 dim (k+1)^dim + k^dim: the element dofs
 * [x | v | e] of k1 (device [n] double) divided by scale[0] (x rows), scale[1] (v rows),
 * scale[2] (e rows), then the same for k2, then dt / scale[3].  scale: device float[4]. */
lh_status lh_mlp_features(lh_mesh* mesh, const double* k1, const double* k2, double dt, const float* scale,
                          float* X);
/* Initial guess of the stage solve at (u, tau) from element predictions Y [NE][F2],
 * F2 = dim (k+1)^dim + k^dim: corrections of the v rows then the e rows (scaled by scale[1],
 * scale[2]).  k0_v = k1_v + average over the elements sharing each node (0 on fixed rows),
 * k0_e = k1_e + the element's prediction, k0_x = u_v + tau k0_v (R_x = 0 exactly).
 * u, k1, k0: device [n] double. */
lh_status lh_mlp_apply_prediction(lh_mesh* mesh, const double* u, double tau, const double* k1, const float* Y,
                                  const float* scale, double* k0);

/* Message for the last failing call on mesh (or a global message if mesh is NULL). */
const char* lh_last_error(const lh_mesh* mesh);

/* Kernel timing (measurement support).  While enabled, each element-kernel launch of the
 * kinds below is bracketed by CUDA events on the mesh's stream; lh_profile_read returns
 * the accumulated device milliseconds and launch counts per kind (HOST arrays of
 * LH_PROF_KINDS entries) and synchronises.  Enabling resets the accumulators. */
enum { LH_PROF_RESIDUAL = 0, LH_PROF_JVP64 = 1, LH_PROF_JVP32 = 2, LH_PROF_JTVP = 3, LH_PROF_MASS = 4,
       LH_PROF_JVPTC = 5, LH_PROF_KINDS = 6 };
lh_status lh_profile_enable(lh_mesh* mesh, int enable);
lh_status lh_profile_read(lh_mesh* mesh, double* ms, long long* count);

/* Arithmetic operations (+ - * / sqrt tanh cbrt cos sin, one each) of one evaluation of
 * the quadrature-point kernel, counted by running the kernel's code on the host with a
 * counting scalar.  kind 0: stress (residual), 1: tangent (J.w), 2: adjoint (J^T.y),
 * 3: tangent from the linearisation record (reduced-precision J.w); 4: the float
 * operations the residual's stress (kind 0) costs in the double-word arithmetic it runs in
 * on the GPU (each double-word sum, product, quotient, root and tanh weighed by its count
 * of float operations).
 * Needs no GPU.  *ops is a HOST pointer. */
lh_status lh_qp_flops(int dim, int kind, int visc, long long* ops);

/* Host check of the double-word (float pair) arithmetic the residual's point kernel runs
 * in (needs no GPU): `trials` seeded cases of which = 0 sum / difference, 1 product,
 * 2 quotient, 3 square root, 4 cube root (relative errors against double), 5 tanh on
 * [-25, 25] (absolute error), 6-9 the whole quadrature-point stress (S, E, det J) in
 * double-word against double, 2D / 2D viscous / 3D / 3D viscous.  *max_err: HOST. */
lh_status lh_dd_check(int which, int trials, unsigned seed, double* max_err);

/* Floats per quadrature point in the linearisation record of lh_linearize (dim 2 or 3).
 * Needs no GPU.  *len is a HOST pointer. */
lh_status lh_record_len(int dim, int* len);

/* Host check of the linearisation record: on `trials` random points near the undeformed
 * element (seeded), compares the tangent formed from the record (lin_record + the linear
 * map of the J.w kernels) with the dual-number tangent of the point kernel.  Writes the
 * largest relative error of the record path evaluated in double (formula check) and the
 * median relative error of dS when the record and the tangent are float (as on the GPU).
 * Needs no GPU.  Output pointers are HOST pointers. */
lh_status lh_qp_tangent_check(int dim, int visc, int trials, unsigned seed, double* max_err_double,
                              double* median_err_float);

/* Host check of the transposed linearised map used by the reduced-precision J^T y: the
 * dot-product identity <L x, y> = <x, L^T y> on `trials` random records, directions and
 * adjoints (double).  Writes the largest relative defect.  Needs no GPU. */
lh_status lh_qp_adjoint_check(int dim, int visc, int trials, unsigned seed, double* max_rel);

/* Number of CUDA kernels this library has launched in the process so far. */
long long lh_launch_count(void);

/* Measurement helper: throughput (TFLOP/s, HOST *tflops) of independent FMA chains on
 * every SM of the current device; prec LH_FP64 or LH_FP32.  Used as the roofline
 * denominator of FP64/FP32-pipe-bound kernels.  Synchronises the device. */
lh_status lh_probe_fma(int prec, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* LH_H */
