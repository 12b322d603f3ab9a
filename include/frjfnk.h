/*
 * frjfnk.h - C ABI of the GB300 Jacobian-free Newton-Krylov library for
 * high-order flux reconstruction (FR/CPR) on 2D quadrilaterals.
 *
 * Method: Wang & Yu, "A comparative study of implicit Jacobian-free
 * Rosenbrock-Wanner, ESDIRK and BDF methods for unsteady flow simulation with
 * high-order flux reconstruction formulations" (arXiv 1904.04825).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an int status (FR_OK = 0 or an FR_ERR_* code); the
 *    message of the last failure is returned by fr_last_error(ctx).
 *  - State-shaped vectors (U, R, z, y, b, x, ...) are caller-owned DEVICE
 *    pointers to double[Ne][4][Np] with Np = (p+1)^2: element ix + Nx*iy,
 *    variable (rho, rho*u, rho*v, E) of Sec. 2, point i + (p+1)*j where i
 *    runs along x and j along y over the Gauss-Legendre solution points.
 *    The total length is ndof = Ne * 4 * Np doubles.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered; calls that return a convergence
 *    result (gmres_solve, step_*) synchronise the stream before returning.
 *  - A context owns all workspace (Krylov basis, element blocks, stage
 *    buffers), allocated once by fr_ctx_create on the device that is current
 *    at that time; that device must be current for every later call on the
 *    context.  Calls on one context must not overlap (one stream at a time).
 *    Nothing is allocated after fr_ctx_create.
 *  - The mesh is a periodic tensor-product mesh of axis-aligned quads; the
 *    edge arrays are HOST pointers copied at creation.
 */
#ifndef FRJFNK_H
#define FRJFNK_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FR_OK = 0,
  FR_ERR_INVALID_ARG = 1,   /* bad pointer, size, degree or option */
  FR_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
  FR_ERR_NONFINITE = 3,     /* a NaN/Inf norm was met; the stepper's U is unchanged */
  FR_ERR_NOT_CONVERGED = 4, /* GMRES hit its restart limit / PTC hit max iterations */
  FR_ERR_PTC_STALLED = 5,   /* too many rejected pseudo-time steps */
  FR_ERR_TIMEOUT = 6,       /* reserved for bounded device-side waits */
  FR_ERR_UNSUPPORTED = 7    /* degree or configuration not compiled in */
};

typedef struct fr_ctx fr_ctx;

/* Periodic mesh: nx*ny quads, element ix+nx*iy spans
 * [x_edges[ix], x_edges[ix+1]] x [y_edges[iy], y_edges[iy+1]] (Sec. 3:
 * affine elements, |J| = hx*hy/4).  nx, ny >= 2.  Host arrays of length
 * nx+1 and ny+1, strictly increasing. */
typedef struct fr_mesh_desc {
  int nx, ny;
  const double* x_edges;
  const double* y_edges;
  int wall_y;            /* 0: periodic in y; 1: isothermal no-slip walls at
                            y_edges[0] and y_edges[ny] (viscous runs only) */
} fr_mesh_desc;

/* Options (fill with fr_default_opts first). */
typedef struct fr_opts {
  double gamma;          /* ratio of specific heats, 1.4 (Sec. 2) */
  int m_max;             /* largest GMRES restart length the workspace holds (30; at
                            most 63, so the paper's GMRES(60) fits) */
  double eps_rel;        /* FD Jv step eps = eps_rel (1 + ||U||_2) / ||z||_2 (1e-7) */
  double eps_fixed;      /* > 0: fixed eps instead (the paper's 1e-8, Sec. 4.5) */
  double block_eps_rel;  /* element-block FD step eps_j = block_eps_rel (1 + |U_j|) (1e-7) */
  int precond;           /* 1: element-Jacobi right preconditioner (Sec. 4.5), 0: none */
  int gmres_m;           /* restart length used by the steppers (30) */
  int gmres_max_restarts;/* restart limit used by the steppers (20) */
  double tol_lin;        /* ROW: GMRES relative tolerance tol_rel,linear (1e-8) */
  double reorth_eta;     /* Arnoldi: classical Gram-Schmidt, repeated once when the
                            first pass leaves ||w|| < reorth_eta ||w_in|| (1/64);
                            1 = always two passes (the paper names no variant) */
  double mu;             /* dynamic viscosity; > 0 selects the Navier-Stokes
                            residual with BR2 viscous fluxes (Sec. 2-3), 0 = Euler */
  double prandtl;        /* Pr (0.72); kappa = mu Cp / Pr, gas constant R = 1 */
  double body_force_x;   /* force per unit mass along x (drives channel flow) */
  double wall_temperature; /* T at isothermal walls */
  int block_precision;   /* element-Jacobi blocks: 0 = FP64 (default); 1 = FP32
                            inversion and storage; 2 = FP32 inversion, BF16
                            storage.  The FD columns (unless block_columns = 1),
                            the FD matvec (unless jv_precision = 1), Arnoldi and
                            all updates stay FP64 (reduced precision changes
                            only the preconditioner, not the converged answer).
                            3D degree 3 (320-row blocks) takes 1 or 2 only */
  int precond_refresh;   /* pseudo-transient continuation (ESDIRK, BDF2): 0 = form
                            J_ee once per stage at its first pseudo iterate and
                            re-invert shift*I - J_ee when dtau changes (default);
                            1 = form the blocks again at every pseudo iterate;
                            2 = form them once per stage and keep them, shift
                            included (no re-inversion when dtau changes: any
                            fixed right preconditioner leaves the converged
                            answer unchanged, and the loose inner solves of
                            PTC need no exact one).
                            The paper does not say; ROW forms them once per step */
  int guess;             /* initial guess of ROW stage solves: 0 = zero (the
                            paper's); 1 = the same stage's solution at the previous
                            step (zero on a first step); 2 = learned (an attached
                            fr_mlp fed [b, previous-step stage solution, previous
                            stage solution]; falls back to 1 without a model).
                            GMRES stops at tol_lin * ||b|| whatever the guess */
  int jv_precision;      /* finite-difference operator A z (2D Euler residual and
                            3D contexts):
                            0 = FP64 throughout (default, the paper's);
                            1 = the linear parts of R(U+eps z) - R(U) -- solution and
                            flux interpolation, derivative and correction -- in
                            FP32 on eps z, the nonlinear pointwise and common
                            fluxes and their differences from the cached
                            F(U), f^num(U) in FP64.  A z then carries a relative
                            error of ~1e-7, so use it only with tol_lin >= 1e-6
                            (ROW at loose tolerances, ESDIRK/BDF2 inner solves).
                            3D (BR2 Navier-Stokes): reference derivatives,
                            traces, BR2 liftings, corrected gradient and
                            corrected divergence act on z in FP32; the
                            inviscid and viscous fluxes at U + eps z (state,
                            traces and gradient from caches at U plus eps
                            times their FP32 parts of z) in FP64, differenced
                            against the fluxes cached at U */
  int riemann;           /* common inviscid flux at the faces (Sec. 3, Eq. invis_com):
                            0 = Rusanov (default), 1 = Roe without entropy fix (the
                            paper's); Euler residual only */
  int block_columns;     /* arithmetic of the FD columns of J_ee (Sec. 4.5):
                            0 = FP64 (default); 1 = FP32, with the step
                            eps_j = max(block_eps_rel, 2^-12) (1 + |U_j|) (about
                            the square root of FP32's unit roundoff) divided by
                            the step the FP32 rounding actually took, and R(U)
                            of each element formed by the same FP32 arithmetic.
                            The columns then carry a relative error of ~1e-3,
                            which changes only the preconditioner.  3D contexts
                            with block_precision 1 or 2 only */
} fr_opts;

/* Pseudo-transient continuation options (Sec. 4.4; fill with
 * fr_default_ptc_opts first). */
typedef struct fr_ptc_opts {
  double tol_nl;         /* ||F^k|| / ||F^0|| stopping tolerance (1e-6) */
  double tol_lin;        /* GMRES relative tolerance inside PTC (1e-1) */
  double dtau_init;      /* <= 0: dtau_init = dt (the paper's default) */
  double dtau_max;       /* 1e20 (the paper's default) */
  int max_iters;         /* accepted pseudo steps per solve (200) */
  int max_rejections;    /* rejected pseudo steps before FR_ERR_PTC_STALLED (30) */
  double reject_above;   /* reject when the GMRES relative residual exceeds this (0.1) */
} fr_ptc_opts;

typedef struct fr_gmres_info {
  int iters;             /* Arnoldi iterations over all cycles */
  int restarts;          /* cycles after the first that iterated */
  int converged;         /* 1 if relres <= rtol */
  double relres;         /* Givens estimate of ||b - A x|| / ||b|| */
} fr_gmres_info;

typedef struct fr_step_stats {
  int gmres_iters;       /* sum over all linear solves of the step */
  int gmres_calls;       /* number of linear solves */
  int ptc_iters;         /* accepted pseudo steps (ESDIRK / BDF2) */
  int rejections;        /* rejected pseudo steps (ESDIRK / BDF2) */
  int residual_evals;    /* R(q) evaluations outside the Jv products */
  int converged;         /* 1 if every solve met its tolerance */
} fr_step_stats;

void fr_default_opts(fr_opts* opts);
void fr_default_ptc_opts(fr_ptc_opts* opts);

/* Create a context for degree p (2 <= p <= 4) on the current device.
 * Copies the mesh, builds the 1D tables (Gauss-Legendre points, Lagrange
 * basis, Radau g_DG correction derivatives, Sec. 3) and allocates every
 * workspace buffer.  *out receives the handle (NULL on failure). */
int fr_ctx_create(const fr_mesh_desc* mesh, int p, const fr_opts* opts, fr_ctx** out);
/* ---- 3D hexahedral Navier-Stokes path (Sec. 2-3 in three directions;
 * the Taylor-Green vortex of Sec. 5) ----
 * Periodic tensor-product mesh of axis-aligned hexahedra: element
 * ix + nx (iy + ny iz) spans [x_edges[ix], x_edges[ix+1]] x [y_edges[iy], ...]
 * x [z_edges[iz], ...].  nx, ny, nz >= 2; host arrays of nx+1, ny+1, nz+1
 * strictly increasing values. */
typedef struct fr_mesh3d_desc {
  int nx, ny, nz;
  const double* x_edges;
  const double* y_edges;
  const double* z_edges;
} fr_mesh3d_desc;
/* Create a 3D context: state layout double[Ne][5][(p+1)^3] with variables
 * (rho, rho u, rho v, rho w, E) and point index i + N j + N^2 k (N = p+1, i
 * along x).  1 <= p <= 4.  R(q) is the FR residual with the Rusanov common
 * flux and, for opts->mu > 0, the BR2 viscous terms (kappa = mu Cp / Pr,
 * R_gas = 1); mu = 0 gives the Euler residual.  Every call of this header
 * that takes a context works on a 3D one (fr_residual, fr_jv, ejacobi_*,
 * gmres_solve, the steppers, fr_autotune, profiling) except the batch and
 * learned-guess calls.  Element-Jacobi blocks (5 (p+1)^3 rows) are built
 * for p <= 3 (p = 3: 320-row blocks stored in FP32 or BF16, block_precision
 * 1 or 2, staged in chunks of 4096 elements); opts->precond with p > 3 or
 * with p = 3 and FP64 blocks, opts->riemann = 1, opts->guess = 2 or a body
 * force return FR_ERR_UNSUPPORTED.  The blocks and their staging are
 * allocated only when opts->precond is set; jv_precision = 1 allocates its
 * caches (traces and face data at U, 6 values per DOF at the points, and
 * FP32 buffers). */
int fr_ctx_create_3d(const fr_mesh3d_desc* mesh, int p, const fr_opts* opts, fr_ctx** out);
/* Kinetic-energy dissipation rate of the Taylor-Green study (Sec. 5) of the
 * 3D state U (device, ndof doubles): out[0] = eps1 = 2 mu / rho0 <S^d : S^d>,
 * out[1] = eps3 = -<p div v> / rho0 (eps2 = 0: zero bulk viscosity), out[2] =
 * <rho |v|^2 / 2> / rho0, <.> the volume average by Gauss-Legendre
 * quadrature at the solution points, the velocity differentiated as each
 * element's degree-p interpolant.  out: host, 3 doubles.  Synchronises the
 * stream.  FR_ERR_UNSUPPORTED on a 2D context. */
int fr_dissipation_rate(fr_ctx* ctx, const double* U, double rho0, double* out, void* stream);

/* ---- accuracy of the isentropic vortex study (Sec. 5.1) ----------------
 * The exact solution of Eq. VP_Solution: a free stream (rho_inf, u_inf,
 * v_inf) with gas constant R = 1 carries, centred at (x0 + u_inf t,
 * y0 + v_inf t) (nearest periodic image on the mesh's box),
 *   du = -alpha/(2 pi) (y - yc) e^{phi (1 - r^2)},
 *   dv =  alpha/(2 pi) (x - xc) e^{phi (1 - r^2)},
 *   dT = -alpha^2 (gamma - 1)/(16 phi gamma pi^2) e^{2 phi (1 - r^2)},
 * dS = 0, r the distance to the centre (the paper prints its square; the
 * exponent is read as phi (1 - r^2)).  The Mach number is taken on the
 * free-stream speed, T_inf = (u_inf^2 + v_inf^2) / (gamma mach^2). */
typedef struct fr_vortex {
  double alpha, phi;     /* strength and width (5, 1/2) */
  double mach;           /* free-stream Mach number on |V| (0.5) */
  double rho_inf, u_inf, v_inf;  /* free stream (1, 1, 1) */
  double x0, y0;         /* centre at t = 0 (0, 0) */
} fr_vortex;
void fr_default_vortex(fr_vortex* v);
/* Error(s) = sqrt( int (s_exact - s_num)^2 dV / V ) of Sec. 5.1 for
 * s = rho, u, v, p of the conserved state U (device, ndof doubles) against
 * the exact vortex at time t, the integral by the Gauss-Legendre rule of the
 * solution points on every element (weights w_i w_j |J_e|), V the area of
 * the mesh's box.  err: HOST array of 4 doubles (E(rho), E(u), E(v), E(p)).
 * 2D Euler contexts; synchronises the stream. */
int fr_vortex_error(fr_ctx* ctx, const double* U, const fr_vortex* vortex, double t, double* err,
                    void* stream);

/* Free the context and its device memory. NULL is accepted. */
int fr_ctx_destroy(fr_ctx* ctx);
/* Message of the last failing call on ctx ("" if none); static string for ctx == NULL. */
const char* fr_last_error(const fr_ctx* ctx);
/* Number of doubles in one state vector (2D: Ne * 4 * (p+1)^2; 3D: Ne * 5 * (p+1)^3). */
long long fr_ndof(const fr_ctx* ctx);

/* R = R(U), the FR/CPR semi-discrete right-hand side dq/dt = R(q)
 * (Sec. 3 Eqs. discrete_ns and simplified_ode): Lagrange extrapolation of
 * the solution to the flux points, Rusanov common flux F^num scaled as in
 * Eq. norm_num_f, divergence of the local flux plus the Radau correction.
 * U, R: device, ndof doubles, must not alias. */
int fr_residual(fr_ctx* ctx, const double* U, double* R, void* stream);

/* y = shift*z - (R(U + eps z) - R0) / eps, the finite-difference
 * Jacobian-vector product of Sec. 4.5 applied as A z with
 * A = D - dR/dq, D = shift*I (Eq. linear).  eps follows fr_opts; a zero z
 * gives y = 0.  R0 must equal R(U).  All device, ndof doubles; y must not
 * alias the inputs.  With fr_opts.jv_precision = 1 the product is formed
 * from fluxes cached at U (recomputed by this call and at the start of every
 * GMRES solve) instead of R0, with the linear parts in FP32. */
int fr_jv(fr_ctx* ctx, const double* U, const double* R0, const double* z, double shift,
          double* y, void* stream);

/* Form and invert the element-Jacobi preconditioner blocks
 * M_e = shift*I - dR_e/dq_e (the diagonal blocks of A, Sec. 4.5) at the
 * state U, stored inside ctx.  The paper does not say how the blocks are
 * formed: here by element-local forward differences with every neighbour
 * trace frozen, step block_eps_rel (1 + |U_j|).  Block rows/columns follow
 * the element's slice of the state.  R0 is accepted for interface symmetry
 * and may be NULL (the local differences need only U). */
int ejacobi_factor(fr_ctx* ctx, const double* U, const double* R0, double shift, void* stream);

/* z_e = M_e^{-1} r_e for every element with the blocks of the last
 * ejacobi_factor call (FR_ERR_INVALID_ARG if there was none).  r, z: device,
 * ndof doubles, must not alias; r 16-byte aligned (FR_ERR_INVALID_ARG
 * otherwise: element blocks and rows of r are streamed into shared memory
 * by bulk copies).  A copy that never completes (bounded wait) sets the
 * context's error flag; the next GMRES cycle then returns FR_ERR_TIMEOUT
 * and the context should be destroyed. */
int ejacobi_apply(fr_ctx* ctx, const double* r, double* z, void* stream);

/* Solve A x = b, A z = shift*z - (R(U+eps z) - R0)/eps, with restarted
 * GMRES(m) (Sec. 4.5), right-preconditioned by the current element-Jacobi
 * blocks when fr_opts.precond = 1 (call ejacobi_factor with the same U and
 * shift first).  x is the initial guess on entry and the solution on exit.
 * Stops when the Givens estimate of ||b - A x|| <= rtol*||b|| or after
 * max_restarts+1 cycles (then FR_ERR_NOT_CONVERGED, x holds the last
 * iterate).  m <= fr_opts.m_max.  info may be NULL. */
int gmres_solve(fr_ctx* ctx, const double* U, const double* R0, double shift, const double* b,
                double* x, int m, double rtol, int max_restarts, fr_gmres_info* info,
                void* stream);

/* One linearly implicit Rosenbrock-Wanner step of Eq. Rosenbrock_General,
 * q^{n+1} = q^n + sum_j m_j Y_j, with (I/(omega dt) - dR/dq)^n frozen at
 * q^n.  scheme = 2 (ROW2, 3 stages), 3 (ROS34PW2, 4 stages), 4 (RODASP,
 * 6 stages).  Linear solves use fr_opts.gmres_m / gmres_max_restarts /
 * tol_lin from a zero guess.  U (device) is advanced in place.  stats may be
 * NULL. */
int step_row(fr_ctx* ctx, int scheme, double dt, double* U, fr_step_stats* stats, void* stream);

/* One ESDIRK step (Eq. ESDIRK2); every implicit stage (Eq. SDIRK_newton) is
 * solved by pseudo-transient continuation with SER time-step control and
 * rejection (Eq. linearized_pseudo_transient_final, Sec. 4.4), the
 * element-Jacobi blocks re-formed at every pseudo step.  scheme = 2, 3, 4
 * (3, 4, 6 stages).  ptc may be NULL (defaults).  U advanced in place. */
int step_esdirk(fr_ctx* ctx, int scheme, double dt, double* U, const fr_ptc_opts* ptc,
                fr_step_stats* stats, void* stream);

/* One BDF2 step (Eq. BDF with omega = 2/3, a = (4/3, -1/3); Eq. BDF_newton
 * solved by pseudo-transient continuation).  U holds q^n on entry and
 * q^{n+1} on exit; U_prev holds q^{n-1} on entry and q^n on exit.
 * first_step != 0 takes one backward-Euler step instead (the paper does not
 * say how BDF2 starts) and ignores U_prev's input. */
int step_bdf2(fr_ctx* ctx, double dt, double* U, double* U_prev, int first_step,
              const fr_ptc_opts* ptc, fr_step_stats* stats, void* stream);

/* One explicit SSPRK3 step (the three-stage, third-order strong-stability-
 * preserving Runge-Kutta scheme the paper's introduction sets the implicit
 * schemes against): u1 = U + dt R(U), u2 = 3/4 U + 1/4 (u1 + dt R(u1)),
 * U <- 1/3 U + 2/3 (u2 + dt R(u2)).  Three residual evaluations, no
 * linear solves; stable only below the explicit CFL limit.  U (device) is
 * advanced in place; FR_ERR_NONFINITE leaves it unchanged. */
int step_ssprk3(fr_ctx* ctx, double dt, double* U, fr_step_stats* stats, void* stream);

/* ---- learned initial guess (no counterpart in the paper) ---------------
 * A per-element MLP for ROW stage i of step n, features
 * [b_e/s, (b - b^{n-1})_e/s, Y_i^{n-1}_e/s] -> (Y_i^n - Y_i^{n-1})_e/s with
 * s = ||b||_2/sqrt(ndof) (the stage's right-hand side and solution at the
 * previous step; zero when absent); the guess is Y_i^{n-1} + s MLP(features),
 * kept only when its residual ||b - A x0|| is below that of Y_i^{n-1}.
 * Network 3nb -> hidden -> hidden -> nb, ReLU,
 * FP32 master weights.  Training kernels run in FP32 on the CUDA cores
 * (gradients checkable against an FP64 reference); inference runs BF16
 * operands on the tcgen05 tensor cores with FP32 accumulation.  GMRES tests the
 * guess: a stage solved from it still stops at tol_lin * ||b||. */
typedef struct fr_mlp fr_mlp;
/* Create a model (device memory for up to max_batch samples). */
int fr_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, fr_mlp** out);
int fr_mlp_destroy(fr_mlp* m);
const char* fr_mlp_last_error(const fr_mlp* m);
/* Parameter count and the flat FP32 layout [W1 b1 W2 b2 W3 b3], W row-major (out x in). */
long long fr_mlp_num_params(const fr_mlp* m);
/* HOST parameter arrays of fr_mlp_num_params floats; set also resets Adam. */
int fr_mlp_set_params(fr_mlp* m, const float* host, void* stream);
int fr_mlp_get_params(fr_mlp* m, float* host, void* stream);
int fr_mlp_get_grads(fr_mlp* m, float* host, void* stream);
/* Y[M][n_out] = MLP(X[M][n_in]) (device FP32 arrays, M <= max_batch);
 * bf16 = 0: FP32 training path (keeps the activations for fr_mlp_backward);
 * bf16 = 1: BF16 inference on the 5th-generation tensor cores (tcgen05 MMA,
 * FP32 accumulation in tensor memory; inputs and hidden activations rounded
 * to BF16).  A GEMM whose bounded wait gave up sets a flag that the next
 * fr_mlp_forward reports as FR_ERR_TIMEOUT. */
int fr_mlp_forward(fr_mlp* m, const float* X, int M, float* Y, int bf16, void* stream);
/* Gradients of mean((Y - T)^2)/2 after an FP32 forward on the same X;
 * loss_host (may be NULL) receives the loss (synchronises). */
int fr_mlp_backward(fr_mlp* m, const float* X, const float* T, int M, double* loss_host, void* stream);
/* One Adam step (with bias correction) on the FP32 weights; refreshes the BF16 copy. */
int fr_mlp_adam(fr_mlp* m, float lr, float beta1, float beta2, float eps, void* stream);
/* Model for fr_opts.guess = 2 (NULL detaches).  Allocates the feature
 * buffers once. */
int fr_attach_guess_model(fr_ctx* ctx, fr_mlp* model);
/* Record training pairs from step_row: after each stage solve, features and
 * targets (Y_i^n - Y_i^{n-1})_e/s of every elem_stride-th element (offset rotating per stage)
 * into the device arrays X [max][3nb] and T [max][nb] until max samples.
 * X = T = NULL stops.  fr_stage_capture_count gives the samples recorded. */
int fr_set_stage_capture(fr_ctx* ctx, float* X, float* T, long long max_samples, int elem_stride);
long long fr_stage_capture_count(const fr_ctx* ctx);
/* Features of every element for (b, bl, yl) into X [ne][3nb]; bl / yl = the
 * stage's previous-step right-hand side / solution (NULL = zero). */
int fr_stage_features(fr_ctx* ctx, const double* b, const double* bl, const double* yl, float* X,
                      void* stream);
/* Forget the stage solutions of the last step (call when U is replaced by an
 * unrelated state); the next ROW step then starts from zero guesses. */
int fr_reset_history(fr_ctx* ctx);
/* Stage solves where a learned guess was formed, and where it was kept. */
int fr_guess_stats(const fr_ctx* ctx, long long* tried, long long* used);

/* ---- allocation-free variant (no counterpart in the paper) -------------
 * y = shift*z - (R(U + eps z) - R0)/eps exactly as fr_jv computes it, but
 * without a context and without allocating device memory.  It is for
 * callers that cannot call cudaMalloc at the point where they need the
 * product: applications whose own allocator has reserved the GPU's memory
 * up front, or code that must not allocate after start-up (cudaMalloc can
 * synchronise the device and fail under memory pressure).
 *  - Working memory is one fixed static device array inside the library
 *    (about 365 KB, held on every GPU that loads the library until the
 *    process exits).  It limits the mesh to 2 <= nx, ny <= 4096; larger
 *    meshes are rejected with FR_ERR_INVALID_ARG.  p must be 2, 3 or 4.
 *  - Every call looks up the array's device address on the current device
 *    (this allocates nothing).  The first lookup on a device also loads the
 *    library's device code there.  The call copies the host edges on
 *    `stream` and cannot be captured into a graph: on a stream that is being
 *    captured it returns FR_ERR_UNSUPPORTED.
 *  - Every call uses the same array and leaves its contents behind; calls
 *    that overlap on the GPU (other streams, other host threads) race.
 *    Serialise them on one stream.
 *  - mesh: HOST edge arrays (copied on `stream`); opts may be NULL
 *    (defaults; gamma, eps_rel, eps_fixed and riemann are used).  The
 *    product is the periodic FP64 Euler one: mesh->wall_y != 0,
 *    opts->mu > 0 or opts->jv_precision != 0 return FR_ERR_UNSUPPORTED.
 *    U, R0, z, y: device, ndof doubles as for fr_jv.  Errors are reported
 *    by fr_last_error(NULL). */
int fr_jv_noalloc(const fr_mesh_desc* mesh, int p, const fr_opts* opts, const double* U,
                  const double* R0, const double* z, double shift, double* y, void* stream);

/* ---- batches of independent instances (no counterpart in the paper) ----
 * Many small problems (uneven meshes and degrees, one fr_opts for all)
 * advanced with one call per time step.  Each instance keeps its own
 * context and kernels; they run concurrently on one CUDA stream per
 * instance, and every restart cycle of the stage GMRES of all instances is
 * replayed as one CUDA graph: one graph launch and one host wait per cycle
 * for the whole batch instead of one host round trip per chunk of Arnoldi
 * steps per instance.  Instances that converged skip the cycle's work on
 * the device (the GMRES kernels test a device flag). */
typedef struct fr_batch fr_batch;

/* Create `count` instances: meshes[k] (host edges, copied), degrees[k] in
 * {2,3,4}, opts shared (NULL = defaults; opts->guess must be 0, else
 * FR_ERR_UNSUPPORTED).  *out = NULL on failure. */
int fr_batch_create(int count, const fr_mesh_desc* meshes, const int* degrees, const fr_opts* opts,
                    fr_batch** out);
int fr_batch_destroy(fr_batch* batch);
const char* fr_batch_last_error(const fr_batch* batch);
/* Launch structure of the batch's GMRES cycles.  on = 1 (the default): when
 * every instance is a 2D Euler context of degree 2..4 with element-Jacobi
 * blocks and the FP64 FD operator, each Arnoldi iteration of all instances
 * runs as one batched launch per kernel (per degree for the block apply
 * and the FD operator): the grid holds the CTAs of every instance, each CTA
 * finds its instance from a device table of per-instance arguments and CTA
 * ranges, and instances whose cycle is done skip their work on the device.
 * Every instance keeps the CTA partition of its own launches, so results
 * equal those of single-instance steps.  on = 0: every instance enqueues its
 * own cycle kernels on its stream.  Changing it drops the captured graphs. */
int fr_batch_set_batched(fr_batch* batch, int on);
/* Kernel nodes of the largest captured cycle graph (0 before the first step). */
int fr_batch_cycle_kernels(const fr_batch* batch, long long* kernels);
/* Context of instance k (owned by the batch; NULL when out of range), for
 * fr_residual, fr_set_launch_config, fr_autotune and friends. */
fr_ctx* fr_batch_member(fr_batch* batch, int k);

/* One ROW step (scheme as fr_step_row: 2, 3 or 4) of size dt on every
 * instance: U[k] (device, ndof(k) doubles) is replaced by its new state;
 * stats[k] (host, may be NULL) as fr_step_row reports them.  The stage
 * solves are restarted GMRES(gmres_m) from a zero guess with the stopping
 * test of fr_gmres_solve (Givens residual <= tol_lin * ||b||), so each
 * instance takes the same iterations as fr_step_row with guess 0 on its
 * own; per-instance results agree to round-off (reduction grids may differ).
 * The cycle graphs are captured on the first call and replayed while the
 * U pointers, dt, scheme and launch configurations stay the same.  Ordered
 * after the work queued on `stream` and blocks the host until the step is
 * done.  Errors: FR_ERR_NOT_CONVERGED when an instance's stage solve
 * reached gmres_max_restarts (states still advanced), FR_ERR_NONFINITE
 * (states untouched), FR_ERR_CUDA. */
int fr_batch_step_row(fr_batch* batch, int scheme, double dt, double* const* U, fr_step_stats* stats,
                      void* stream);

/* One ESDIRK step (scheme 2, 3 or 4, as step_esdirk) / one BDF2 step (as
 * step_bdf2; U_prev[k] in/out) of every instance.  Each pseudo-transient
 * iteration decides on the host from its own residual norms, so instances
 * run their own control loops: `threads` host threads (0 = one per host
 * core, at most one per instance) take instances in turn and step each on
 * the instance's stream, so the kernels of different instances overlap on
 * the device.  Blocks until every instance finished.  stats[k] as for the
 * single-instance calls.  Returns FR_OK, or the most severe instance status
 * (FR_ERR_CUDA / FR_ERR_NONFINITE / FR_ERR_INVALID_ARG before
 * FR_ERR_NOT_CONVERGED / FR_ERR_PTC_STALLED); fr_batch_last_error names the
 * instance.  Each instance's U (and U_prev) follows that instance's status
 * as the single-instance calls document it. */
int fr_batch_step_esdirk(fr_batch* batch, int scheme, double dt, double* const* U, const fr_ptc_opts* ptc,
                         int threads, fr_step_stats* stats, void* stream);
int fr_batch_step_bdf2(fr_batch* batch, double dt, double* const* U, double* const* U_prev, int first_step,
                       const fr_ptc_opts* ptc, int threads, fr_step_stats* stats, void* stream);

/* ---- launch configuration (no counterpart in the paper) ----------------
 * vec_blocks: grid of the streaming Krylov-vector kernels (dots, updates,
 * norms, block apply), 1..4096 CTAs; tile_variant: element-tile shape of
 * the Euler residual kernel (0 or 1; results are identical, only the
 * speed differs).  Reductions are deterministic for a fixed vec_blocks;
 * another vec_blocks changes their rounding order. */
int fr_set_launch_config(fr_ctx* ctx, int vec_blocks, int tile_variant);
int fr_get_launch_config(const fr_ctx* ctx, int* vec_blocks, int* tile_variant);
/* Time full GMRES(gmres_m) cycles of A = shift I - dR/dU at U (device) for
 * vec_blocks in {152, 304, 456, 608, 912, 1216} x both tile variants and
 * keep the fastest; ms_best / ms_default (host, may be NULL) = time of one
 * cycle with the chosen / the configuration found on entry.  Overwrites the
 * element blocks (formed at `shift`) and the internal work vectors;
 * synchronises `stream`. */
int fr_autotune(fr_ctx* ctx, const double* U, double shift, int reps, double* ms_best, double* ms_default,
                void* stream);

/* ---- measurement hooks (no counterpart in the paper) -------------------
 * Kernel families for fr_profile_*: */
enum {
  FR_KF_RESIDUAL = 0,  /* R(U) */
  FR_KF_JV = 1,        /* FD operator A z and b - A z */
  FR_KF_FACTOR = 2,    /* element-block formation (+ inversion where one kernel does both) */
  FR_KF_APPLY = 3,     /* element-Jacobi apply (incl. basis normalisation) */
  FR_KF_DOTS = 4,      /* Gram-Schmidt multi-dot products */
  FR_KF_UPDATE = 5,    /* Gram-Schmidt multi-AXPY updates */
  FR_KF_SOLUPDATE = 6, /* x += M^-1 V y */
  FR_KF_OTHER = 7,     /* norms, linear combinations, copies, Givens */
  FR_KF_INVERT = 8,    /* inversion of staged element blocks (viscous and 3D contexts) */
  FR_KF_COUNT = 9
};

/* Test hook (no counterpart in the paper) for the bounded waits of the
 * element-Jacobi apply, whose CTAs wait on shared-memory barriers for the
 * bulk copies of the blocks: polls = the poll limit of every such wait
 * (0 = the default, 2^22); skip_first_copy = 1 makes CTA 0 of every later
 * apply launch leave its first element's copies unissued, so that its wait
 * runs out.  The CTA then flags the context, waits (bounded) for the copies
 * it did issue and leaves; the GMRES cycle that launched it returns
 * FR_ERR_TIMEOUT (as gmres_solve and the steppers do whenever a bounded wait
 * gave up).  Nothing faults.  A context that reported FR_ERR_TIMEOUT keeps
 * reporting it: destroy it. */
int fr_set_wait_test(fr_ctx* ctx, unsigned polls, int skip_first_copy);

/* Elements whose FD element blocks (Sec. 4.5) are staged in FP64 and
 * inverted at a time.  3D degree-3 contexts (320-row blocks, 800 KB each in
 * FP64) stage 4096 elements at a time; every other context stages all
 * elements at once.  n may lower the chunk (1 <= n <= the chunk the context
 * allocated; a smaller chunk changes no result, only the number of
 * launches); FR_ERR_INVALID_ARG otherwise.  With chunks, a new shift of the
 * pseudo-transient iteration forms the blocks again instead of re-inverting
 * the staging. */
int fr_set_block_chunk(fr_ctx* ctx, long long n);

/* Number of kernels this library has launched in this process. */
long long fr_kernel_launches(void);

/* Start timing every launch of the families whose bit (1 << FR_KF_*) is set
 * in family_mask with CUDA events on the launching stream.  Creates the
 * events (host-side setup, no device allocation). */
int fr_profile_begin(fr_ctx* ctx, unsigned family_mask);

/* Stop timing; synchronises the recorded events and writes, per family
 * (arrays of FR_KF_COUNT entries, any may be NULL): the summed kernel time in
 * ms, the number of launches that did work (GMRES-cycle kernels launched
 * after the cycle finished return at once and are not counted), and the
 * algorithmic bytes and floating-point operations of the timed launches
 * (the counting rules are stated beside each launch in the sources). */
int fr_profile_end(fr_ctx* ctx, double* ms, long long* launches, double* bytes, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* FRJFNK_H */
