/*
 * m1.h — C ABI of the grey M1 radiation step on one GB300 GPU (sm_103a).
 *
 * The library implements the time-implicit grey M1 radiative-transfer step of
 * Bloch, Tremblin, Gonzalez, Padioleau & Audit (A&A 2021), Sects. 2-3:
 *   - the M1 closure P = D(f) E (Sect. 2.2) and the M1 eigenvalues
 *     (Eq. eigenvalues, Sect. 3.1.1);
 *   - the HLL interface fluxes F*, P* (Sect. 3.1.1) with the asymptotic-
 *     preserving correction alpha (Eq. asymptoticCorrection, Sect. 3.1.3);
 *   - the well-balanced flux source (Eqs. wb_smart, boundaryCondition,
 *     Sect. 3.1.2) or the centred one (Eq. wb_naive);
 *   - absorption/emission exchange with the gas (Eqs. momentModel,
 *     internalEnergyEqua, Sect. 2.1);
 *   - the backward-Euler residual of Sect. 3.1.1, its Jacobian-vector product
 *     and point-block Jacobi preconditioner, restarted GMRES and Newton-Raphson
 *     (Sects. 3.3.1-3.3.2);
 *   - the semi-implicit step of Sect. 3.1 (sources implicit, fluxes explicit),
 *     whose WB source is the tridiagonal system of Appendix B.
 *
 * Conventions (all entry points):
 *   - Every call returns an m1_status; nothing throws or exits across the ABI.
 *     m1_last_error() gives a human-readable reason for the last failure.
 *   - Arrays are structure-of-arrays, x fastest, WITHOUT ghost cells: a field
 *     is N = nx*ny*nz doubles; F is dim consecutive fields (F_x, F_y, F_z);
 *     an unknown vector is [E, F_x, (F_y), (F_z), (T)] = n_u*N doubles with
 *     n_u = 1 + dim (+1 with gas coupling).
 *   - Caller pointers are host or device memory as the m1_mem argument says.
 *     They are read/written on the context's stream and not retained after the
 *     call returns (the call synchronises that stream before returning).
 *   - The context owns all the device memory it allocates (m1_init_grid and,
 *     lazily, the first implicit call). M1_ERR_NOMEM reports a failed allocation.
 *   - Units are the caller's: c and a_r are grid parameters (c = a_r = 1 in the
 *     workloads shipped with this library).
 */
#ifndef M1_H
#define M1_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    M1_OK = 0,
    M1_ERR_ARG = 1,           /* invalid argument (message in m1_last_error) */
    M1_ERR_CUDA = 2,          /* a CUDA call failed */
    M1_ERR_NOMEM = 3,         /* device allocation failed */
    M1_ERR_NOT_CONVERGED = 4, /* Newton/GMRES did not reach the tolerance */
    M1_ERR_NONFINITE = 5,     /* NaN/Inf met in a residual or a norm */
    M1_ERR_TIMEOUT = 6,       /* a bounded device wait ran out */
    M1_ERR_STATE = 7          /* call out of order (e.g. no state set) */
} m1_status;

typedef enum { M1_BC_OUTFLOW = 0, M1_BC_PERIODIC = 1, M1_BC_REFLECT = 2, M1_BC_DIRICHLET = 3 } m1_bc;
typedef enum { M1_MEM_HOST = 0, M1_MEM_DEVICE = 1 } m1_mem;
typedef enum { M1_PREC_FP64 = 0, M1_PREC_MIXED = 1 } m1_precision;
/* Krylov method of the Newton linear solves: restarted GMRES(restart), or the
 * paper's BiCGStab (Sect. 3.3.1), right-preconditioned, the recurrence scalars on
 * the device; gmres_max and gmres_rtol bound either. */
typedef enum { M1_KRYLOV_GMRES = 0, M1_KRYLOV_BICGSTAB = 1 } m1_krylov;
typedef enum {
    M1_PRECOND_NONE = 0,
    M1_PRECOND_BJ = 1,
    M1_PRECOND_LEARNED = 2,
    M1_PRECOND_MG = 3,
    M1_PRECOND_LINE = 4
} m1_precond;

/* Grid and discretisation flags (one context per grid). */
typedef struct {
    int dim;              /* 1, 2 or 3 */
    int n[3];             /* cells per axis; unused axes must be 1 */
    double lo[3], hi[3];  /* box; dx_a = (hi_a - lo_a) / n_a */
    int bc[3][2];         /* m1_bc per axis and side (0 = low, 1 = high); periodic on both sides or neither */
    double c, a_r;        /* speed of light and radiation constant */
    int gas_coupling;     /* 1: T is an unknown (Eq. internalEnergyEqua); 0: frozen emission B */
    int well_balanced;    /* 1: Eq. wb_smart; 0: Eq. wb_naive */
    int ap_correction;    /* 1: alpha of Eq. asymptoticCorrection; 0: alpha = 1 (plain HLL) */
    int fixed_eigs;       /* 1: lambda+- = +-c; 0: Eq. eigenvalues */
    double lambda_floor;  /* lambda+ = max(floor, ...), lambda- = min(-floor, ...) (0 in the paper's default) */
    int wb_boundary;      /* 1: Eq. boundaryCondition at non-periodic boundary faces; 0: plain face average */
    int implicit_eigs;    /* 1: lambda in F*, P* at the new time level; 0: frozen at time n */
} m1_grid_desc;

/* Solver options (m1_default_opts fills the defaults shown). */
typedef struct {
    double newton_rtol;   /* 1e-8: stop when ||R(U^k)||_2 <= rtol ||R(U^n)||_2 */
    int newton_max;       /* 30 */
    int restart;          /* 30 (at most 30): GMRES(restart) */
    int gmres_max;        /* 3000 total Arnoldi iterations per linear solve */
    double gmres_rtol;    /* 1e-4: forcing term ||J d + R|| <= rtol ||R|| */
    int precision;        /* m1_precision: FP64, or FP32 inner FGMRES under FP64 refinement */
    int precond;          /* m1_precond; M1_PRECOND_LEARNED needs M1_PREC_MIXED and m1_set_preconditioner;
                             M1_PRECOND_LINE (the block-tridiagonal part of J, solved exactly along the
                             line: J itself on a non-periodic 1D grid) needs dim 1, M1_PREC_FP64 and >= 3
                             cells; M1_PRECOND_MG needs M1_PREC_MIXED, dim 2 and frozen or fixed wave speeds
                             (see m1_mg_apply) */
    int line_search;      /* 1 (default): halve theta up to 6 times until the Armijo decrease holds; 0: full
                             Newton steps (theta = 1) */
    int advance;          /* 1: on success U^n <- U^{n+1}; 0: keep U^n (result in m1_get_solution) */
    int refine_max;       /* mixed precision: max FP64 refinement sweeps per Newton step (4) */
    int krylov;           /* an m1_krylov value, default M1_KRYLOV_GMRES; the learned preconditioner needs GMRES */
    int pc_rebuild;       /* M1_PRECOND_MG: rebuild the hierarchy on Newton steps 0, k, 2k, ... of each implicit
                             step (1, the default: every Newton step; values < 1 act as 1); in between, the
                             cycle keeps its smoothers and coarse operators and applies the current J on level 0 */
    int realizability;    /* 0 (default): the result may leave the admissible set (E > 0, |F| <= cE); its
                             violations are counted. 1: the a posteriori admissibility fallback (Sect. 3.1.3
                             names the centred source as the remedy for f > 1). Checks run when Newton has
                             converged and after every check_every Newton steps without convergence. A check
                             flags the unflagged cells with E <= 0 or |F| > cE; if there are none and Newton has
                             not converged, the unflagged cells whose largest residual component is at least a
                             tenth of the largest one. A flagged cell takes the centred flux source
                             (Eq. wb_naive); its faces take alpha = 1 and the speeds -c, +c. The iterate of a
                             flagged inadmissible cell is reset to U^n, ||R(U^n)|| of the new scheme becomes the
                             reference, and every later Newton
                             update of a flagged cell is scaled so that the cell stays admissible. Newton steps
                             of all rounds count against newton_max. Needs frozen (implicit_eigs = 0) or fixed
                             wave speeds. */
    int check_every;      /* realizability = 1: Newton steps between checks before convergence (5; 0: only at
                             convergence) */
    int forcing;          /* 0 (default): every linear solve to gmres_rtol. 1: Eisenstat-Walker forcing (their
                             choice 2, gamma 0.9, exponent 2): eta_k = 0.9 (||R_k|| / ||R_{k-1}||)^2, safeguarded by
                             0.9 eta_{k-1}^2 when that exceeds 0.1, clipped to [gmres_rtol, 0.1], and not below
                             0.5 newton_rtol ||R(U^n)|| / ||R_k|| (no solve tighter than the Newton test needs);
                             eta_0 = 0.1. Only the path to the root changes, not the root. */
} m1_solver_opts;

#define M1_HIST 64  /* length of the per-Newton-iteration histories */

typedef struct {
    int converged;        /* 1 when ||R|| <= newton_rtol * ||R^0|| */
    int newton_iters;
    int gmres_iters;      /* total Arnoldi iterations over all linear solves */
    int refinements;      /* FP64 refinement sweeps (mixed precision) */
    double res0, res;     /* ||R(U^n)||_2 (of the last scheme when the fallback flagged cells) and the final ||R||_2 */
    long long realizability_violations; /* cells with |F| > c E in the result (Sect. 3.1.3) */
    double time_ms;       /* wall time of the step measured on the stream */
    /* per Newton iteration k < min(newton_iters, M1_HIST): ||R|| after the
     * update, Arnoldi iterations of its linear solve, line-search theta */
    double res_hist[M1_HIST];
    int gmres_hist[M1_HIST];
    double theta_hist[M1_HIST];
    long long fallback_cells;  /* realizability = 1: cells flagged in this step (m1_get_fallback) */
    int fallback_rounds;       /* realizability = 1: checks that flagged cells */
    int fp64_double_word;      /* 1: the step's FP64 residuals and J v ran in double words (m1_set_fp64_arithmetic) */
    double fp64_floor;         /* M1_FP64_AUTO: ||R_dw(U^n) - R_fp64(U^n)|| / ||R(U^n)||, the double-word
                                  rounding floor measured at the start of the step (0 when not measured) */
} m1_step_info;

typedef struct {
    int converged;
    int iters;
    double res0, res;     /* ||b|| and the true ||b - J x|| at exit */
} m1_solve_info;

/* kernel classes of the per-class timers (m1_profile) */
typedef enum {
    M1_K_RESIDUAL = 0,   /* FP64 residual stencil */
    M1_K_JV64 = 1,       /* FP64 J v stencil */
    M1_K_JV32 = 2,       /* FP32 J v stencil */
    M1_K_PC_BUILD = 3,   /* point blocks, dP/dU, multigrid levels and their inverses */
    M1_K_PC_APPLY = 4,   /* block-Jacobi apply or one multigrid cycle */
    M1_K_ORTHO = 5,      /* Gram-Schmidt dots, updates, norms, Givens */
    M1_K_VECTOR = 6,     /* other vector kernels (axpy, conversions) */
    M1_K_EXPLICIT = 7,   /* semi-implicit step kernels */
    M1_K_CLASSES = 8
} m1_kernel_class;

typedef struct {
    long long newton_iters, gmres_iters, jv_calls, residual_calls, precond_builds;
    long long explicit_steps, implicit_steps, kernel_launches;
    double bytes_per_jv, bytes_per_residual;  /* algorithmic bytes of one launch (FP64) */
    double bytes_per_jv32;                     /* algorithmic bytes of one FP32 J v launch */
    /* with profiling on (m1_profile): device time (CUDA events on the
     * context's stream) and launch count per m1_kernel_class */
    double kernel_ms[M1_K_CLASSES];
    long long kernel_count[M1_K_CLASSES];
    double ortho_bytes;   /* algorithmic bytes moved by the Gram-Schmidt kernels so far */
    double bytes_per_mg_cycle;  /* algorithmic bytes of one multigrid cycle (0 before a hierarchy is built) */
} m1_stats_t;

typedef struct m1_ctx m1_ctx;

void m1_default_opts(m1_solver_opts* opts);

/* Create a context on the current CUDA device. cuda_stream: a cudaStream_t
 * (NULL = the legacy default stream). Validates the descriptor (M1_ERR_ARG).
 * Allocates the fields, the time-n state and the face arrays. */
m1_status m1_init_grid(const m1_grid_desc* desc, void* cuda_stream, m1_ctx** out);

/* Free every device allocation of the context. NULL is accepted. */
m1_status m1_destroy(m1_ctx* ctx);

/* Opacities: sigma_a (absorption/emission, Eq. momentModel energy row) and
 * sigma_f (flux source and alpha). sigma_f == NULL uses sigma_a. N doubles each. */
m1_status m1_set_opacity(m1_ctx* ctx, const double* sigma_a, const double* sigma_f, m1_mem mem);

/* Time-n state. E: N, F: dim*N. With gas coupling T (N) and rho_cv (N) are
 * required; otherwise they must be NULL. Resets the time-n face data (alpha,
 * lambda at time n). */
m1_status m1_set_state(m1_ctx* ctx, const double* E, const double* F, const double* T,
                       const double* rho_cv, m1_mem mem);

/* Copy the context's current state out (T may be NULL without gas coupling). */
m1_status m1_get_state(const m1_ctx* ctx, double* E, double* F, double* T, m1_mem mem);

/* The result U^{n+1} of the last m1_implicit_step / m1_explicit_step, as an
 * unknown vector (n_u*N doubles). */
m1_status m1_get_solution(const m1_ctx* ctx, double* U, m1_mem mem);

/* Dirichlet ghost data of one face (axis, side) whose bc is M1_BC_DIRICHLET:
 * E (M cells of the face, M = N / n[axis], face cells ordered x fastest over
 * the remaining axes), F (dim*M), mask (M bytes; 1 = use the given ghost,
 * 0 = zero-gradient copy; NULL = all 1). */
m1_status m1_set_boundary(m1_ctx* ctx, int axis, int side, const double* E, const double* F,
                          const unsigned char* mask, m1_mem mem);

/* Frozen emission B = a_r T_g^4 (N doubles; only without gas coupling; default 0). */
m1_status m1_set_emission(m1_ctx* ctx, const double* B, m1_mem mem);

/* External energy source S added to dE/dt (N doubles, NULL = none). */
m1_status m1_set_source(m1_ctx* ctx, const double* S, m1_mem mem);

/* Prescribed gas velocity on the faces: u[a] holds the normal velocity of every
 * face of axis a (N / n_a * (n_a + 1) doubles, the face index runs fastest
 * along x as for cells, with n_a + 1 faces along a). Used by m1_advect (gas
 * coupling) and m1_velocity_sources. */
m1_status m1_set_velocity(m1_ctx* ctx, const double* ux, const double* uy, const double* uz, m1_mem mem);

/* Explicit first-order upwind transport of the gas internal energy rho c_v T by
 * the prescribed velocity over dt (the frozen-hydrodynamics step of the
 * operator split of Sect. 3.2); updates T of the current state. */
m1_status m1_advect(m1_ctx* ctx, double dt);

/* The explicit velocity-dependent radiation sources over dt (Sect. 2.1 at first
 * order in u/c, applied after the implicit step: step 3 of the splitting of
 * Sect. 2.3). With u the mean of a cell's two face velocities per axis, P the
 * closure pressure of the current state, B = a_r T^4 (gas coupling) or the
 * frozen emission and sigma the flux opacity:
 *   S_E = (sigma/c) u.F + (sigma/c) E |u|^2 + (sigma/c) u.(P u)
 *   S_F = sigma P u + sigma B u + (sigma/c^2) u (u.F)
 * E += dt S_E, F += c dt S_F and, with gas coupling, rho c_v T -= dt S_E.
 * Updates the current state; needs m1_set_velocity. */
m1_status m1_velocity_sources(m1_ctx* ctx, double dt);

/* One semi-implicit step of size dt (Sect. 3.1): HLL fluxes and alpha at time n,
 * backward-Euler exchange and flux source (tridiagonal WB solves along each
 * component's own axis, Appendix B form). Advances the state. */
m1_status m1_explicit_step(m1_ctx* ctx, double dt);

/* One backward-Euler step of size dt by Newton-Raphson + right-preconditioned
 * restarted (F)GMRES (Sect. 3.3). On failure returns M1_ERR_NOT_CONVERGED
 * (or M1_ERR_NONFINITE) and leaves the state unchanged; info is filled either way. */
m1_status m1_implicit_step(m1_ctx* ctx, double dt, const m1_solver_opts* opts, m1_step_info* info);

/* The cells the admissibility fallback flagged in the last m1_implicit_step
 * (realizability = 1): N bytes, 1 = flagged (centred source, alpha = 1 and
 * speeds -c, +c on its faces), 0 otherwise; all 0 after a step without it. */
m1_status m1_get_fallback(const m1_ctx* ctx, unsigned char* mask, m1_mem mem);

/* R(U) of the backward-Euler step of size dt from the context's time-n state
 * (the scheme of Sect. 3.1.1). U, R: n_u*N doubles. */
m1_status m1_residual(m1_ctx* ctx, double dt, const double* U, double* R, m1_mem mem);

/* J(U) v, the exact directional derivative of m1_residual. precision:
 * M1_PREC_FP64, forward-mode dual numbers in the context's FP64 arithmetic
 * (m1_set_fp64_arithmetic; the operator of the mixed path's refinement), or
 * M1_PREC_MIXED, the FP32 operator of the inner solver (in 2D with frozen or
 * fixed wave speeds the linear stencil of dP/dU at U, else dual numbers; inputs
 * rounded to FP32, result widened to FP64). */
m1_status m1_jv(m1_ctx* ctx, double dt, const double* U, const double* v, double* Jv,
                int precision, m1_mem mem);

/* Point blocks J_ii = dR_i/dU_i of m1_residual at U (Sect. 3.3.2 block Jacobi):
 * n_u*n_u*N doubles laid out blocks[(row*n_u + col)*N + cell]. */
m1_status m1_diag_blocks(m1_ctx* ctx, double dt, const double* U, double* blocks, m1_mem mem);

/* The multigrid preconditioner (M1_PRECOND_MG): the structured-grid analogue of
 * the algebraic multigrid the paper found best among its preconditioners
 * (Sect. 3.3.2, Sect. 4). 2D, frozen or fixed wave speeds, FP32. Level 0 is
 * J(U) itself (applied as J v) with the point-block inverses as smoother; its
 * 5-point stencil of n_u x n_u blocks is assembled directly from the stored
 * pressure Jacobian (radiation only) or read off J v by coloured probes (gas
 * coupling); levels >= 1 aggregate 2 x 2 cells (piecewise-constant prolongation,
 * summing restriction, Galerkin stencil P^T A P) until both sides are <= 16
 * cells. One application is a V(1,1) cycle from zero with damped point-block
 * Jacobi (omega 0.7) and 10 damped sweeps on the coarsest level; it is linear in
 * r. Periodic axes need at least 3 cells.
 *
 * m1_mg_apply builds the hierarchy at U (U NULL = the time-n state) for step
 * size dt and returns z = one cycle applied to r (n_u*N doubles each, rounded to
 * FP32 and widened back). */
m1_status m1_mg_apply(m1_ctx* ctx, double dt, const double* U, const double* r, double* z, m1_mem mem);

/* After m1_mg_apply: the number of levels, and the stencil of one level as
 * 5*n_u*n_u*N_level doubles, A[((s*n_u + row)*n_u + col)*N_level + cell] with s =
 * 0..4 the (self, -x, +x, -y, +y) neighbour; N_level = nx*ny of that level
 * (sizes halve with ceil from the grid's). A NULL out only reports nlev. */
m1_status m1_mg_blocks(m1_ctx* ctx, int level, int* nlev, double* out, m1_mem mem);

/* Solve J(U) x = b with the step's GMRES (U NULL = the time-n state).
 * x is the output (initial guess 0). */
m1_status m1_gmres_solve(m1_ctx* ctx, double dt, const double* U, const double* b, double* x,
                         const m1_solver_opts* opts, m1_solve_info* info, m1_mem mem);

/* Cumulative counters of the context. */
m1_status m1_stats(const m1_ctx* ctx, m1_stats_t* out);

/* FP64 arithmetic of the residual and J v stencils (the outer Newton residual
 * and the FP64 J v of the plain path and of the mixed path's refinement).
 * This GPU issues FP64 operations at about 1/64 of the FP32 rate, and these
 * stencils are bound by them; M1_FP64_DOUBLE_WORD evaluates them in
 * double-word arithmetic instead (each value a sum hi + lo of two FP32 numbers,
 * about 48 significant bits, operations of Joldes, Muller and Popescu, ACM TOMS
 * 2017, relative error <= 15 * 2^-48 per operation) on FP32 operations, with
 * FP32's exponent range; arrays stay FP64. M1_FP64_AUTO (the default) takes it
 * when c, a_r and every dx lie within 2^-30 .. 2^30, and in m1_implicit_step only
 * when the step can reach its Newton tolerance in it: each step first evaluates
 * R(U^n) in both arithmetics, and keeps double words when newton_rtol ||R(U^n)||
 * is at least 32 times ||R_dw(U^n) - R_fp64(U^n)|| (stiff exchange terms, c sigma
 * dt >> 1, cancel in the residual and raise the double-word floor 2^5-2^6 times
 * above FP64's). In either double-word case
 * a residual that is not finite or exceeds 2^100 in some component is computed
 * again in FP64, and the context stays on FP64 from then on (counted in
 * *fallbacks). M1_FP64_NATIVE: FP64 operations throughout. */
typedef enum { M1_FP64_AUTO = 0, M1_FP64_NATIVE = 1, M1_FP64_DOUBLE_WORD = 2 } m1_fp64_arith;
m1_status m1_set_fp64_arithmetic(m1_ctx* ctx, int mode);
/* The arithmetic in use (M1_FP64_NATIVE or M1_FP64_DOUBLE_WORD) and the number
 * of range fallbacks so far; either pointer may be NULL. */
m1_status m1_get_fp64_arithmetic(const m1_ctx* ctx, int* mode, long long* fallbacks);

/* Turn the per-kernel-class event timers on (1) or off (0) and reset them.
 * Timers add two event records per timed launch on the context's stream. */
m1_status m1_profile(m1_ctx* ctx, int enable);

/* ---------------------------------------------------------------------------
 * Learned preconditioner (not in the paper; the library's own addition).
 *
 * A 3-level 2D U-Net (63,875 parameters; 3x3 convolutions 7-16-16 | 16-32-32 |
 * 32-32-32 | 64-32-16 | 32-16-3, ReLU, 2x2 average pooling, nearest 2x
 * upsampling with skip concatenation) maps a Krylov vector v of a 2D
 * radiation-only grid (channels E, F_x, F_y, scaled by s = ||v|| / sqrt(n)),
 * the normalised log opacity (log10(sigma_f dx) - 0.5) / 2.5, and the state U
 * at which the Jacobian is taken (F_x / (cE), F_y / (cE) clipped to [-1, 1], and
 * (log10 E + 3) / 3, E floored at 1e-30) to a correction. As the right
 * preconditioner of flexible GMRES it applies
 *     z = J_bj^-1 v + s * N(v / s, log sigma, U),
 * the point-block Jacobi result plus the learned correction. Weights are FP32
 * masters with a BF16 copy; the convolutions multiply BF16 weights and BF16
 * activations on the tensor cores with FP32 accumulation (activations stored in
 * BF16 in inference, FP32 in training), or, after m1_nn_set_tensor_cores(nn, 0),
 * FP32 activations on the CUDA cores (the precise path of the gradient checks).
 * Tensors are NHWC float arrays: inputs B*H*W*7, outputs/targets B*H*W*3.
 * ------------------------------------------------------------------------- */
typedef struct m1_nn m1_nn;

typedef struct {
    int epochs;           /* passes over the pairs */
    double lr;            /* Adam step size (beta1 0.9, beta2 0.999, eps 1e-8) */
    double lr_decay;      /* lr *= lr_decay each epoch (0 or 1: constant) */
    unsigned long long seed; /* shuffle seed (SplitMix64) */
} m1_train_opts;

typedef struct {
    int steps;            /* Adam steps taken */
    double first_loss, final_loss; /* batch loss of the first step, mean loss of the last epoch */
} m1_train_info;

size_t m1_nn_num_params(void);
/* Network for batches of `batch` H x W images (H, W multiples of 4) on cuda_stream. */
m1_status m1_nn_create(int H, int W, int batch, void* cuda_stream, m1_nn** out);
m1_status m1_nn_destroy(m1_nn* nn);
/* FP32 parameters in layer order (weights W[ky][kx][ci][co] then biases); resets Adam. */
m1_status m1_nn_set_params(m1_nn* nn, const float* theta, m1_mem mem);
m1_status m1_nn_get_params(const m1_nn* nn, float* theta, m1_mem mem);
/* y = N(x) for one batch; bf16 = 1 stores activations in BF16 (inference path). */
m1_status m1_nn_forward(m1_nn* nn, const float* x, float* y, int bf16, m1_mem mem);
/* Loss (1/B) sum_b ||N(x_b) - t_b||^2 / (H W 3) (mean squared error per output element)
 * and its gradient. */
m1_status m1_nn_loss_grad(m1_nn* nn, const float* x, const float* t, double* loss, float* grad, m1_mem mem);
/* Adam on npairs (x, t) pairs held as consecutive images; batches of the network's size. */
m1_status m1_nn_train(m1_nn* nn, const float* X, const float* T, int npairs, const m1_train_opts* opts,
                      m1_train_info* info, m1_mem mem);
/* 1 (default): convolutions on the tensor cores (BF16 operands, FP32 accumulation);
 * 0: FP32 activations and products on the CUDA cores. Applies to every later call. */
m1_status m1_nn_set_tensor_cores(m1_nn* nn, int on);
const char* m1_nn_last_error(const m1_nn* nn);

/* One training pair from the context's own Jacobian (2D, radiation only):
 * r = J(U) e (U NULL = the time-n state), s = ||r|| / sqrt(n), x = [r / s, log sigma,
 * the state channels of U] (NHWC, 7 channels), t = (e - J_bj(U)^-1 r) / s (NHWC,
 * 3 channels): the part of the exact inverse that point-block Jacobi misses. */
m1_status m1_nn_make_pair(m1_ctx* ctx, double dt, const double* U, const double* e, float* x, float* t,
                          m1_mem mem);

/* Attach (nn != NULL) or detach the learned preconditioner. The network must be
 * built for batch 1 and the grid's n[1] x n[0]; the context does not own it. */
m1_status m1_set_preconditioner(m1_ctx* ctx, m1_nn* nn);

/* How flexible GMRES combines the learned correction with point-block Jacobi (a
 * context setting, default M1_LEARNED_ADDITIVE; the paper has no learned
 * component, this is the library's own design):
 *   M1_LEARNED_ADDITIVE: z = J_bj^-1 v + s (N(v / s) - N(0)) on odd Arnoldi steps,
 *     z = J_bj^-1 v on even ones; s = ||v|| / sqrt(n);
 *   M1_LEARNED_TWO_STAGE: on odd Arnoldi steps a point-block Jacobi stage first,
 *     z1 = J_bj^-1 v and r1 = v - J z1 (FP32 J v), then
 *     z = z1 + J_bj^-1 r1 + s1 (N(r1 / s1) - N(0)), s1 = ||r1|| / sqrt(n) (taken on
 *     the device): the network sees the residual the first stage leaves, J times
 *     an error point-block Jacobi resolves slowly, which is what the pairs of
 *     m1_nn_make_pair teach it; even steps as above;
 *   M1_LEARNED_TWO_STAGE_ALL: the two-stage form on every Arnoldi step.
 * N(0) is the network's response to a zero vector at the same Newton iterate.
 * M1_ERR_ARG for another value. */
#define M1_LEARNED_ADDITIVE 0
#define M1_LEARNED_TWO_STAGE 1
#define M1_LEARNED_TWO_STAGE_ALL 2
m1_status m1_set_learned_form(m1_ctx* ctx, int form);

/* ---------------------------------------------------------------------------
 * Batched steps: many independent 2D radiation-only problems (periodic,
 * outflow or reflecting boundaries; frozen or fixed wave speeds) solved by one
 * persistent launch per size class, all classes replayed from one CUDA graph.
 * Each CTA takes problems from a device work queue and runs a whole
 * backward-Euler step (Newton, FP32 GMRES under FP64 refinement, point-block
 * Jacobi, line search) with CTA-wide barriers only. Classes of more than
 * 128 x 128 cells (or any class, see m1_batch_set_class and m1_batch_tune) run
 * instead through single-grid contexts, one problem after another on a side
 * stream, concurrently with the graph.
 * ------------------------------------------------------------------------- */
typedef struct m1_batch m1_batch;

typedef struct {
    int converged, newton_iters, gmres_iters;
    double res0, res;
} m1_batch_problem_info;

/* nprob grids (descs[k]); size classes are the distinct cell counts. */
m1_status m1_batch_create(int nprob, const m1_grid_desc* descs, void* cuda_stream, m1_batch** out);
m1_status m1_batch_destroy(m1_batch* b);
/* Problem k's opacities, time-n state (E: N, F: 2N) and frozen emission (NULL = 0). */
m1_status m1_batch_set_problem(m1_batch* b, int k, const double* sigma_a, const double* sigma_f, const double* E,
                               const double* F, const double* B, m1_mem mem);
/* Time each class on the single-grid path and with persistent CTAs of 128, 256
 * and 512 threads (a size more than 3x slower than the best so far ends the
 * class's search) and keep the fastest: chosen[c] receives the CTA size, or 0
 * for the single-grid path (may be NULL). */
m1_status m1_batch_tune(m1_batch* b, const double* dts, const m1_solver_opts* opts, int* chosen);
/* Run class c with persistent CTAs of `threads` (128, 256 or 512), or, with
 * threads = 0, through single-grid contexts one problem after another on a side
 * stream while the persistent classes run (the default for classes of more than
 * 128 x 128 cells: one SM per problem is slow there). The single-grid path uses
 * FP32 inner GMRES under FP64 refinement with the caller's multigrid, else
 * point-block Jacobi preconditioner. */
m1_status m1_batch_set_class(m1_batch* b, int c, int threads);
/* One implicit step of every problem (dts[k]); info[k] per problem (may be
 * NULL); *elapsed_ms = device time of the graph launch (may be NULL). The
 * solutions are read with m1_batch_get_solution; the time-n states are kept. */
m1_status m1_batch_implicit_step(m1_batch* b, const double* dts, const m1_solver_opts* opts,
                                 m1_batch_problem_info* info, double* elapsed_ms);
m1_status m1_batch_get_solution(const m1_batch* b, int k, double* U, m1_mem mem);
int m1_batch_num_classes(const m1_batch* b);
const char* m1_batch_last_error(const m1_batch* b);

/* ---------------------------------------------------------------------------
 * Allocation-free residual.
 *
 * The paper has no counterpart of this entry point. It serves callers that
 * cannot allocate device memory at the point of the call: code running inside
 * a memory pool or arena that forbids cudaMalloc/cudaFree, a host thread that
 * must not trigger the implicit synchronisation of an allocation, or a
 * framework that owns all allocations itself. It computes the same R(U) as
 * m1_residual, but without a context: every input and output is a device
 * pointer passed by the caller, and the working memory (the time-n face data
 * and the reduction partials) lives in one file-scope __device__ array of the
 * library, sized for at most M1_NOALLOC_MAX_CELLS cells. Every GPU that loads
 * the library holds that array (about 9.4 MB) until the process exits.
 *
 * Rules:
 *   - N = n[0]*n[1]*n[2] above M1_NOALLOC_MAX_CELLS is rejected with
 *     M1_ERR_ARG before anything is launched.
 *   - The call allocates nothing (no cudaMalloc, cudaFree or allocating
 *     library routine). Its first call in each CUDA context (the device's
 *     primary context, made current by the call) looks up the array's device
 *     address (cudaGetSymbolAddress) and caches it under the context's unique
 *     id; make that first call before any stream capture. After a device reset
 *     the next call runs in a new context and looks the address up again.
 *   - Every call shares the one array, which keeps the last call's contents:
 *     the call clears what must start at zero, but calls that overlap on the
 *     GPU (different streams, or different host threads on one device) race.
 *     Serialise them.
 *   - The call is asynchronous on cuda_stream: R and *norm2 are valid once the
 *     stream has reached this point. Only launch errors are reported.
 * ------------------------------------------------------------------------- */
#define M1_NOALLOC_MAX_CELLS 65536

typedef struct {
    const double* Un;        /* time-n state, n_u*N (device) */
    const double* sigma_a;   /* N (device) */
    const double* sigma_f;   /* N (device), NULL = sigma_a */
    const double* B;         /* N frozen emission without gas coupling, NULL = 0 */
    const double* S;         /* N source, NULL = none */
    const double* rho_cv;    /* N, required with gas coupling */
    const double* bE[3][2];  /* Dirichlet ghost data of each face, as m1_set_boundary (device) */
    const double* bF[3][2];
    const unsigned char* bmask[3][2];
} m1_device_fields;

/* R(U) of the backward-Euler step of size dt (same result as m1_residual for
 * the same inputs) and its squared 2-norm into *norm2 (a device double; NULL
 * = not wanted). U and R: n_u*N device doubles. */
m1_status m1_residual_noalloc(const m1_grid_desc* desc, double dt, const m1_device_fields* fields,
                              const double* U, double* R, double* norm2, void* cuda_stream);

/* Message of the last failed call on this context (never NULL). */
const char* m1_last_error(const m1_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* M1_H */
