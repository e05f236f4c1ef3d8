/*
 * rann_dd.h -- C ABI of the GB300 (sm_103a) RaNN domain-decomposition solver.
 *
 * The method (Shang, Heinlein, Mishra, Wang, "Overlapping Schwarz
 * preconditioners for randomized neural networks with domain decomposition"):
 * each overlapping box subdomain Omega_j carries a randomized single-hidden-
 * layer tanh network Phi_j with fixed uniform weights (Sec. 2, Eq. (net));
 * the networks are glued by a partition of unity omega_j and a constraining
 * operator C u = L u + G that enforces the Dirichlet data (Eq. (operator),
 * (netdd)); collocation gives the block least-squares system H W = F
 * (Eq. (system)); PCA of each local basis Psi_j reduces H_j to H_j V_{p_j}
 * (Sec. 4, Eq. (system_new)); the normal equations H^T H W = H^T F are solved
 * by additive-Schwarz preconditioned CG or restricted-additive-Schwarz
 * preconditioned GMRES (Sec. 3).  Algorithm 1 lists the steps in this order.
 *
 * Conventions for every entry point:
 *  - Every call returns a rann_status; RANN_OK on success.  On error the
 *    handle is left usable unless the status is RANN_ECUDA (a CUDA error,
 *    after which the handle should be destroyed).  rann_dd_last_error()
 *    returns a human-readable message for the last failing call of the
 *    calling thread.
 *  - "_dev" pointers are CUDA device pointers to contiguous float64 (or
 *    int64 where stated) arrays owned by the caller; "_host" pointers are host
 *    memory owned by the caller.  The handle owns all internal device memory
 *    (allocated at create/assemble/pca/setup time, released by destroy).
 *  - All work is enqueued on the CUDA stream given to rann_dd_create and is
 *    stream-ordered.  Calls that return host data (pca ranks, solver stats,
 *    inspection getters) synchronise that stream.
 *  - Calls out of Algorithm 1's order (solve before setup_precond, pca
 *    before assemble, ...) return RANN_EORDER.
 *  - No process-global state: handles are independent; a handle must not be
 *    used from two host threads at once.
 */
#ifndef RANN_DD_H
#define RANN_DD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RANN_OK = 0,
  RANN_EINVAL = 1,          /* an argument is out of range or inconsistent */
  RANN_ENOMEM = 2,          /* device or host allocation failed */
  RANN_ECUDA = 3,           /* a CUDA runtime error */
  RANN_NOT_CONVERGED = 4,   /* Krylov solve hit maxit; W holds the last iterate */
  RANN_BREAKDOWN = 5,       /* CG p^T A p <= 0, or NaN/Inf met in a reduction */
  RANN_LOCAL_SINGULAR = 6,  /* warning: a local Cholesky needed a diagonal shift */
  RANN_EORDER = 7,          /* call made out of Algorithm 1's order */
  RANN_TIMEOUT = 8          /* a bounded device wait (tensor-core product pipeline) gave up;
                               the work it fed is invalid, the handle stays usable */
} rann_status;

/* PDE operator A of Eq. (1). */
enum { RANN_OP_POISSON = 0,    /* -Lap u + c0 u                          */
       RANN_OP_DIFFUSION = 1,  /* -div(a grad u), spatial dims only        */
       RANN_OP_HEAT = 2 };     /* u_t - nu Lap_x u; last coordinate is t   */
/* Diffusion coefficient a(x). */
enum { RANN_COEF_CONST = 0,      /* a = coef_value                                  */
       RANN_COEF_MULTISCALE = 1, /* a = 2 + sin(2 pi x/eps) sin(2 pi y/eps)        */
       RANN_COEF_PIECEWISE = 2 };/* a = sum_c coef_vals[c] s_c(x,y), g x g smoothed cells */
/* G of the constraining operator C u = L u + G (Eq. (operator)). */
enum { RANN_G_ZERO = 0, RANN_G_SINPROD = 1 /* G = prod_{spatial i} sin(pi x_i) */ };
/* Subdomain layout. */
enum { RANN_LAYOUT_CELL = 0,   /* mu_k = (k+1/2)/l, half-width (1/l + overlap)/2 */
       RANN_LAYOUT_PAPER = 1 };/* mu_k = k/(l-1), half-width (delta/2)/(l-1) (Sec. 5, Ex. 1) */
/* PCA rank rule (Sec. 4). */
enum { RANN_PCA_ABS = 0,       /* p_j = #{sigma_k > thr}                            */
       RANN_PCA_VARIANCE = 1,  /* smallest p: sum_{k<=p} sigma_k^2 >= (1-thr) sum sigma^2 */
       RANN_PCA_NONE = 2 };    /* p_j = m, V = I                                    */
/* Schwarz preconditioner kind (Sec. 3). */
enum { RANN_PREC_NONE = 0, RANN_PREC_AS = 1, RANN_PREC_SAS = 2, RANN_PREC_RAS = 3 };

/*
 * Problem descriptor: the statement of Eq. (1) with Dirichlet data through
 * C u = L u + G, the subdomain grid and overlap, the local networks, the
 * collocation grid.  Host memory, read during rann_dd_create only.
 *
 * Collocation points: the cell-centred grid x_q = (q + 1/2)/(sub[i]*pts[i])
 * per dimension, q = 0 .. sub[i]*pts[i]-1; global point index
 * g = q_0 + G_0 (q_1 + G_1 q_2) (dimension 0 fastest).
 * Source: f(x) = f0 + sum_{t < f_terms} fc[t] prod_{spatial i} sin(pi fa[t*dim+i] x_i).
 * Constraint: L = prod_{spatial i} tanh(x_i/rho) tanh((1-x_i)/rho)
 *             [* tanh(t/rho) for RANN_OP_HEAT] (Eq. (cons1), (cons2)).
 * Piecewise coefficient: s_c(x,y) = S(x; c mod g) S(y; c div g) with the
 * smooth cell indicator S(x; i) = [tanh((x-i/g)/w) - tanh((x-(i+1)/g)/w)]/2,
 * w = 1/(8g), and the outer edges pushed to -inf/+inf (so sum_c s_c = 1).
 * Weights: R [J][m][dim] and b [J][m] if given, else drawn from the
 * SplitMix64 stream `seed` as U[-w_range, w_range] in the order
 * (subdomain j: R_j in (neuron, dim) order, then b_j).
 */
typedef struct {
  int dim;                 /* 2 or 3 (a space-time problem counts t)          */
  int op;                  /* RANN_OP_*                                       */
  double c0;               /* Poisson reaction coefficient                    */
  double nu;               /* heat diffusivity                                */
  int coef;                /* RANN_COEF_*                                     */
  double coef_value;       /* RANN_COEF_CONST value                           */
  double eps;              /* RANN_COEF_MULTISCALE period                     */
  int coef_grid;           /* RANN_COEF_PIECEWISE g (<= 8)                    */
  const double* coef_vals; /* [g*g], cell (cx, cy) at cy*g + cx               */
  int layout;              /* RANN_LAYOUT_*                                   */
  int sub[3];              /* subdomains per dimension (l_i)                  */
  double overlap[3];       /* RANN_LAYOUT_CELL: absolute overlap per dim      */
  double delta;            /* RANN_LAYOUT_PAPER: overlap ratio delta > 1      */
  int pts[3];              /* collocation points per subdomain cell per dim   */
  int neurons;             /* m, 1 .. 1024                                    */
  double w_range;          /* weights ~ U[-w_range, w_range]                  */
  uint64_t seed;           /* SplitMix64 stream when R/b are NULL             */
  const double* R;         /* optional [J][m][dim]                            */
  const double* b;         /* optional [J][m]                                 */
  double rho;              /* constraint sharpness                            */
  int g_kind;              /* RANN_G_*                                        */
  double f0;               /* constant part of f                              */
  int f_terms;             /* 0 .. 16                                         */
  const double* fc;        /* [f_terms]                                       */
  const double* fa;        /* [f_terms][dim]                                  */
} rann_dd_desc;

/* Per-solve statistics. */
typedef struct {
  int iters;               /* Krylov iterations (inner steps for GMRES)       */
  double rel_res_true;     /* ||H^T(F - H W)|| / ||H^T F|| recomputed at exit */
  double rel_res_rec;      /* the solver's own stopping quantity at exit      */
  double rel_res_prec;     /* ||M^{-1}(b - A W)|| / ||M^{-1} b|| at exit (GMRES) */
  double ms_solve;         /* device time of the solve                        */
  int n_shifted;           /* local factors that needed a shift (from setup)  */
  double ms_assemble;      /* device time of the handle's last assemble (+ rhs) */
  double ms_pca;           /* device time of the last pca                     */
  double ms_setup;         /* device time of the last setup_precond           */
  double kappa_est;        /* estimate of kappa(M^{-1} H^T H) from the first
                              refinement cycle's Krylov coefficients: the
                              Lanczos tridiagonal of CG (Ritz values) or the
                              Arnoldi Hessenberg of GMRES (singular values);
                              a lower bound that tightens with the iteration
                              count; -1 where not formed (CGS, BiCG, < 2 steps) */
} rann_dd_stats;

typedef struct rann_dd_handle rann_dd_handle;

/* Algorithm 1 steps 1-2: subdomains, collocation grid, networks.  Copies the
 * descriptor; `cuda_stream` is a cudaStream_t (NULL = legacy default). */
rann_status rann_dd_create(const rann_dd_desc* desc, void* cuda_stream, rann_dd_handle** out);
/* Releases all device memory of the handle (stream-ordered, then synchronises). */
void rann_dd_destroy(rann_dd_handle* h);

/* Sizes: N global collocation points, total block rows sum_j N_j, J, m, and
 * the current number of unknowns DoF = sum_j p_j (J*m before pca). */
rann_status rann_dd_sizes(rann_dd_handle* h, int64_t* n_points, int64_t* n_block_rows,
                          int* J, int* m, int64_t* dof);
/* Collocation point coordinates into xyz_dev [N][dim]. */
rann_status rann_dd_points(rann_dd_handle* h, double* xyz_dev);

/* Algorithm 1 steps 3 and 5 (Sec. 2 Eq. (system), Sec. 4 Psi_j): for every
 * subdomain j and collocation point x in box_j, Psi_j = omega_j Phi_j and
 * H_j = A[L omega_j Phi_j], float64, kept in the handle. */
rann_status rann_dd_assemble(rann_dd_handle* h);
/* F_i = f(x_i) - A[G](x_i) at the N global points into F_dev [N]. */
rann_status rann_dd_rhs(rann_dd_handle* h, double* F_dev);

/* Algorithm 1 step 4 (Sec. 4, Eq. (pca), (system_new)): eigen-decomposition of
 * each Gram matrix Psi_j^T Psi_j = V diag(sigma^2) V^T, rank p_j by `mode` and
 * `thr`, then H_j <- H_j V_{p_j}.  Writes the ranks to ranks_host [J] (may be
 * NULL).  Synchronises. */
rann_status rann_dd_pca(rann_dd_handle* h, int mode, double thr, int* ranks_host);

/* Algorithm 1 step 6, preconditioner part (Sec. 3): for every subdomain i the
 * extended set N(i) (subdomains whose box shares a collocation point with
 * box_i; overlap_level = 0: {i} only), A_i = R_i H^T H R_i^T assembled from
 * the neighbour Gram blocks, and its Cholesky factor (float64; a diagonal
 * shift is applied and counted where a pivot fails).  `kind` is
 * RANN_PREC_AS / SAS / RAS / NONE and fixes D_i (Sec. 3, Sec. 5).
 * Returns RANN_LOCAL_SINGULAR (a warning) if any factor was shifted. */
rann_status rann_dd_setup_precond(rann_dd_handle* h, int kind, int overlap_level);

/* Algorithm 1 step 6, solve part: preconditioned CG on H^T H W = H^T F
 * (Sec. 3, Sec. 5 Table 1b/3) from W = 0, stopping when the recursive
 * ||H^T F - H^T H W|| / ||H^T F|| <= rtol (true residual recomputed at exit).
 * Needs a symmetric preconditioner (AS or NONE).  F_dev [N], W_dev [DoF]. */
rann_status rann_dd_solve_cg_as(rann_dd_handle* h, const double* F_dev, double* W_dev,
                                double rtol, int maxit, rann_dd_stats* stats);
/* Left-preconditioned restarted GMRES(restart) on the normal equations from
 * W = 0, stopping when ||M^{-1}(H^T F - H^T H W)|| / ||M^{-1} H^T F|| <= rtol
 * (Sec. 5 Example 1 stopping rule).  Any preconditioner kind. */
rann_status rann_dd_solve_gmres_ras(rann_dd_handle* h, const double* F_dev, double* W_dev,
                                    double rtol, int restart, int maxit, rann_dd_stats* stats);
/* The CG variants of Sec. 5 (Table 1b) on the normal equations from W = 0,
 * with any preconditioner kind: conjugate gradient squared (Sonneveld) and
 * biconjugate gradients (Fletcher; its shadow sequence applies A^T = A and
 * M^{-T}), both preconditioned as in Barrett et al., Templates (1994), and
 * both stopping when ||H^T F - H^T H W|| / ||H^T F|| <= rtol (the float64
 * residual; the recurrences run as iterative refinement like CG).  Returns
 * RANN_BREAKDOWN when a recurrence scalar vanishes or is not finite.
 * F_dev [N], W_dev [DoF]. */
rann_status rann_dd_solve_cgs(rann_dd_handle* h, const double* F_dev, double* W_dev,
                              double rtol, int maxit, rann_dd_stats* stats);
rann_status rann_dd_solve_bicg(rann_dd_handle* h, const double* F_dev, double* W_dev,
                               double rtol, int maxit, rann_dd_stats* stats);

/* Adjoint of the solve (differentiation through Algorithm 1 step 6; the
 * paper's normal equations of Sec. 2 are symmetric, so the adjoint system is
 * the same): lam_dev [DoF] receives lam = (H^T H)^{-1} gW for a loss gradient
 * gW_dev = dl/dW [DoF], solved to rtol with the stored preconditioner (CG if
 * it is AS or none, left-preconditioned GMRES(50) otherwise).  Then
 * dl/dF = H lam (rann_dd_matvec).  Krylov iterates are recomputed, not
 * stored.  Needs setup_precond. */
rann_status rann_dd_solve_backward(rann_dd_handle* h, const double* gW_dev, double* lam_dev,
                                   double rtol, int maxit, rann_dd_stats* stats);

/* Derivative of a loss through the solve with respect to the reaction
 * coefficient c0 of the Poisson operator -Lap u + c0 u (the coefficient
 * enters Sec. 2 Eq. (sum) linearly, and Psi_j, hence the PCA basis, does not
 * depend on it): dH/dc0 = L Psi V and, for F from rann_dd_rhs, dF/dc0 = -G.
 * Given F_dev [N] (the right-hand side the solve used), the solution W_dev
 * [DoF] and lam_dev [DoF] = (H^T H)^{-1} dl/dW from rann_dd_solve_backward,
 * *grad_host receives
 *   dl/dc0 = r . (H_c lam) - (H lam) . G - (H lam) . (H_c W),   r = F - H W,
 * for a loss that depends on c0 only through W.  H_c x is formed as
 * u_hat(x) - G at the collocation points (rann_dd_eval).  All device
 * pointers are the caller's; synchronises the stream.  RANN_EINVAL for other
 * operators, RANN_EORDER before rann_dd_pca. */
rann_status rann_dd_grad_c0(rann_dd_handle* h, const double* F_dev, const double* W_dev, const double* lam_dev,
                            double* grad_host);

/* Derivative of a loss through the solve with respect to the cell values a_c
 * (c < g*g) of the piecewise diffusion coefficient a = sum_c a_c s_c of
 * -div(a grad u) (RANN_OP_DIFFUSION with RANN_COEF_PIECEWISE).  The operator
 * of Sec. 2 Eq. (sum) is linear in a and Psi_j (hence the PCA basis) does
 * not depend on a, so dH/da_c x = A_c[v_x] at the collocation points, with
 * A_c v = -s_c Lap v - grad s_c . grad v and v_x = L sum_j omega_j
 * (Phi_j . V_{p_j} x_j), and dF/da_c = -A_c[G] for F from rann_dd_rhs.
 * Given F_dev [N], W_dev [DoF] and lam_dev [DoF] = (H^T H)^{-1} dl/dW (from
 * rann_dd_solve_backward), grad_host [g*g] receives
 *   dl/da_c = r . (dH/da_c lam) + (H lam) . (dF/da_c - dH/da_c W),  r = F - H W,
 * for a loss that depends on a only through W (fixed-order sums; one kernel
 * forms v, grad v and Lap v of both vectors per point).  Synchronises.
 * RANN_EINVAL for other operators or coefficients, RANN_EORDER before pca. */
rann_status rann_dd_grad_coef(rann_dd_handle* h, const double* F_dev, const double* W_dev, const double* lam_dev,
                              double* grad_host);
/* Replaces the piecewise coefficient values a_c (host [g*g], finite) of a
 * RANN_COEF_PIECEWISE diffusion handle.  H and F depend on them, so the
 * handle returns to Algorithm 1 step 3: assemble, rhs, pca and
 * setup_precond must run again. */
rann_status rann_dd_set_coef(rann_dd_handle* h, const double* vals_host);
/* Adjoint of the evaluation at the collocation points (Eq. (netdd),
 * (pca_net)): with u_hat = E W + G on the N points, gW_dev [DoF] = E^T r for
 * r_dev [N]; block j is (E^T r)_j = V_{p_j}^T Psi_j^T (L r)|_{rows_j}.  Used for
 * losses on u_hat, e.g. dl/dW = 2 E^T (u_hat - u_obs) for ||u_hat - u_obs||^2.
 * Synchronises. */
rann_status rann_dd_eval_grid_t(rann_dd_handle* h, const double* r_dev, double* gW_dev);

/* Precision policy.  Mode 1 (default): the work that only shapes the
 * preconditioner or the Krylov iterates -- the neighbour Gram blocks of A_i,
 * the Cholesky trailing updates, L_i^{-1}, and every operator and
 * preconditioner application inside the Krylov iterations -- runs in
 * double-float (float32 hi + lo pairs, about 48 significant bits; GB300
 * executes float32 at 70x its float64 rate), while the PCA, the reduced
 * blocks B_j and every residual that decides a restart or convergence stay
 * float64-accurate, so the solve is an iterative refinement converging to the
 * float64 solution.  In mode 1 the two dense products of the PCA (the Gram
 * matrices Psi_j^T Psi_j and B_j = H_j V_{p_j}) and the neighbour Gram blocks
 * are formed on the bf16 tensor cores (tcgen05) from exact 7-bit digit slices
 * of float64 operands (Ozaki splitting), with an error of the float64
 * product's order; the Gram-Schmidt and back-transformation of the kept
 * eigenvectors and the 32 x 32 diagonal blocks of the local Cholesky factors
 * are double-float (the eigenvalues, hence the PCA ranks, stay float64).
 * Mode 0: float64 SIMT
 * arithmetic throughout (needed where the preconditioner must be exact to
 * float64 rounding, e.g. the unreduced system with PCA off).  Affects the
 * next pca, setup_precond and solve. */
rann_status rann_dd_set_precision(rann_dd_handle* h, int mode);

/* u_hat(x) = L(x) sum_j omega_j(x) (V_{p_j}^T Phi_j(x)) . W_j + G(x)
 * (Eq. (netdd), (pca_net)) at n points x_dev [n][dim] (inside [0,1]^dim)
 * into u_dev [n]. */
rann_status rann_dd_eval(rann_dd_handle* h, const double* W_dev, const double* x_dev,
                         int64_t n, double* u_dev);

/* Building blocks of the solve, exposed for tests and composition
 * (all device vectors float64): y = H x (y_dev [N], x_dev [DoF]);
 * z = H^T y; z = H^T H x (float64, B^T (B x)); z = M^{-1} r with the stored
 * local factors (double-float after a set-up in precision mode 1, float64
 * after one in mode 0). */
rann_status rann_dd_matvec(rann_dd_handle* h, const double* x_dev, double* y_dev);
rann_status rann_dd_matvec_t(rann_dd_handle* h, const double* y_dev, double* z_dev);
rann_status rann_dd_normal_matvec(rann_dd_handle* h, const double* x_dev, double* z_dev);
rann_status rann_dd_precond_apply(rann_dd_handle* h, const double* r_dev, double* z_dev);
/* z = M^{-T} r = sum_i R_i^T A_i^{-1} D_i R_i r (the transposed Schwarz
 * preconditioner of Sec. 3; equals M^{-1} for AS). */
rann_status rann_dd_precond_apply_t(rann_dd_handle* h, const double* r_dev, double* z_dev);

/* Many right-hand sides per launch (the batching the weak-scaling runs of
 * Sec. 5 / Table 2 call for; the operator and the local factors are shared).
 * Vectors of one call are stored one after another: R_dev, Z_dev [nrhs][DoF],
 * F_dev [nrhs][N], W_dev [nrhs][DoF], device, caller-owned; stats: nrhs
 * entries or NULL.
 * rann_dd_precond_apply_multi: Z_c = M^{-1} R_c for c < nrhs; every column
 * equals rann_dd_precond_apply of that column.
 * rann_dd_solve_cg_as_multi: rann_dd_solve_cg_as for every column, in
 * lockstep: each step reads the local factors and the block rows of H^T H
 * once for (up to four) columns at a time; every column keeps its own
 * scalars, convergence flag and refinement decisions, with the arithmetic
 * of the one-column solve (same iterates while a column is below its own
 * maxit).  The return value is the first non-OK column status (RANN_OK if
 * all converged).  With the float64 factors (precision mode 0) or without
 * the block-row operator the columns are solved one after another.
 * rann_dd_solve_gmres_ras_multi: rann_dd_solve_gmres_ras for every column in
 * the same way: each Arnoldi step applies the block-row operator and the
 * Schwarz preconditioner to all columns' current basis vectors at once; the
 * Gram-Schmidt passes, the Givens bookkeeping, the restarts and the float64
 * residual decisions are per column, so every column equals the one-column
 * solve (a column that converged keeps stepping with a frozen Hessenberg
 * matrix while others run). */
rann_status rann_dd_precond_apply_multi(rann_dd_handle* h, const double* R_dev, double* Z_dev, int nrhs);
rann_status rann_dd_solve_cg_as_multi(rann_dd_handle* h, const double* F_dev, double* W_dev, int nrhs,
                                      double rtol, int maxit, rann_dd_stats* stats);
rann_status rann_dd_solve_gmres_ras_multi(rann_dd_handle* h, const double* F_dev, double* W_dev, int nrhs,
                                          double rtol, int restart, int maxit, rann_dd_stats* stats);

/* Inspection (synchronising copies to host memory).
 * which = 0: Psi_j, 1: H_j (both N_j x m, after assemble, before pca);
 *         2: reduced block B_j = H_j V_{p_j} (N_j x p_j, after pca).
 * rows_host [N_j] receives the global point index of each row. */
rann_status rann_dd_block_info(rann_dd_handle* h, int j, int64_t* n_rows, int* n_cols);
rann_status rann_dd_get_block(rann_dd_handle* h, int j, int which, double* out_host,
                              int64_t* rows_host);
/* Eigenvalues sigma^2 (descending, [m]) and the kept V_{p_j} ([m][p_j] row-major). */
rann_status rann_dd_get_pca(rann_dd_handle* h, int j, double* eig_host, double* V_host);

/* The transposed block product z_j = B_j^T y(rows_j) without any allocation.
 * The paper has no counterpart: it exists for callers that cannot allocate
 * device memory -- a program whose device memory is all owned by its own
 * allocator (a framework's caching pool or a fixed arena reserved at
 * start-up), where cudaMalloc fails, or a latency-critical loop that cannot
 * take the device-wide synchronisation cudaMalloc/cudaFree may imply.  It
 * needs no handle and allocates nothing: partial sums live in a fixed device
 * array of 2^20 doubles (8 MiB) and block descriptors in a fixed table of
 * 4096 entries, both held by every GPU that loads the library until exit.
 * Host arrays [J]: block j is n_rows[j] x ld[j] row-major at B_dev + boff[j]
 * (its first n_cols[j] columns are used); its rows read y_dev at the indices
 * rows_dev[row_off[j] .. row_off[j] + n_rows[j]) (int64, device); z_j goes to
 * z_dev[zoff[j] ..].  RANN_EINVAL if J is outside 1..4096, a pointer is NULL,
 * a descriptor is negative or n_cols > ld, or (number of 256-row tiles) x
 * (largest n_cols) exceeds 2^20.  The first call on a device looks up the
 * arrays' device addresses (with that device current).  All calls share
 * the arrays, which keep the last call's
 * contents; every value a call reads is written earlier by the same call.
 * Calls that overlap on the GPU race.  Enqueued on `cuda_stream`. */
rann_status rann_dd_matvec_t_noalloc(int J, const int64_t* boff, const int* n_rows, const int* n_cols,
                                     const int* ld, const int64_t* row_off, const int64_t* zoff,
                                     const double* B_dev, const int64_t* rows_dev, const double* y_dev,
                                     double* z_dev, void* cuda_stream);

/* Kernel accounting (tracing for the roofline; the paper has no
 * counterpart).  Every kernel launch is counted per kernel family together
 * with its algorithmic bytes and flops (the minimal traffic and arithmetic
 * of the operation it performs, computed from the sizes); with
 * profile_enable(h, 1) each launch is also bracketed by CUDA events on the
 * handle's stream.  profile_enable resets all counters.  profile_get returns,
 * for family idx = 0, 1, ... (RANN_EINVAL past the last one): its name (a
 * static string), kernels launched, summed device time in ms (0 unless
 * profiling was on), summed algorithmic bytes and flops, and its roofline
 * class (0 = memory-bound, 1 = float64-ALU-bound, 2 = bf16-tensor-core-bound,
 * whose flops are those of the digit-slice products, 3 = double-float
 * arithmetic on the float32 pipe, float64-equivalent flops; the class of a
 * family can depend on the precision mode).  It synchronises the
 * pending events.  Any output pointer may be NULL. */
rann_status rann_dd_profile_enable(rann_dd_handle* h, int on);
rann_status rann_dd_profile_get(rann_dd_handle* h, int idx, const char** name, int64_t* launches,
                                double* ms, double* alg_bytes, double* alg_flops, int* bound);

/* Schwarz apply configurations (precision mode 1).  0: the fused kernel that
 * reads 32-row blocks of L_i^{-1} twice (the second time from L2); 1..3: the
 * streaming kernel that reads every row of L_i^{-1} once through shared
 * memory, with row chunks of about 1/6, 1/12, 1/24 of an SM's share of the
 * factor entries (sets of at most 6144 unknowns).  setup_precond picks 2 for
 * sets of 2048 unknowns and more, else 0.  The configurations differ only in
 * the summation order (results agree to the double-float factor accuracy);
 * each is deterministic.
 * rann_dd_set_apply_config: after setup_precond; RANN_EINVAL for a
 * configuration this set-up cannot run (or out of range).
 * rann_dd_tune_apply: times every configuration this set-up can run (one
 * warm-up and `reps` timed applies each, CUDA events on the handle's
 * stream; a configuration's time is its fastest apply, robust to other
 * work sharing the GPU) and keeps the configuration in effect unless
 * another is more than 10 % faster, in which case it keeps the fastest of
 * those (work sharing the GPU can slow all of one configuration's samples;
 * a small gain does not outweigh that noise); best_out gets the choice,
 * ms_out [RANN_APPLY_NCFG] (or NULL) the ms per apply, -1 where a
 * configuration cannot run.
 * Synchronises. */
#define RANN_APPLY_NCFG 4
rann_status rann_dd_set_apply_config(rann_dd_handle* h, int cfg);
rann_status rann_dd_get_apply_config(rann_dd_handle* h, int* cfg);
rann_status rann_dd_tune_apply(rann_dd_handle* h, int reps, int* best_out, float* ms_out);

/* Moves the handle's work to another CUDA stream (0 = legacy default):
 * waits for the current stream's work first. */
rann_status rann_dd_set_stream(rann_dd_handle* h, void* cuda_stream);

/* ---- Batches of instances (Sec. 5, Table 2: many independent problems) ----
 * rann_dd_batch_run takes n instances (handles of any problem and grid size,
 * created and left unassembled or assembled, in any precision mode) through
 * the whole path -- assemble, F, PCA, Schwarz set-up, the preconditioned
 * solve and, with backward set, the gradient of the grid misfit
 * l = ||u_hat - u_obs||^2 over the collocation points: dl/dW = 2 E^T (u_hat -
 * u_obs), the adjoint solve, dl/dF = H lam and, for the piecewise
 * coefficient, dl/da_c (rann_dd_grad_coef).  A batch owns `nworkers` host
 * threads (1..64), each with its own CUDA stream; a worker moves an
 * instance's handle onto its stream for the run and back afterwards, so the
 * kernels of different instances overlap on the device while every worker
 * drives its instance's host-side control (rank decisions, Krylov
 * convergence checks).  Instances start largest first (points x neurons).
 * With autotune set, the first instance of each size class (subdomain
 * count, largest extended set rounded up to 64 unknowns) runs
 * rann_dd_tune_apply(reps 5) and the others of the class wait for and reuse
 * its choice.
 * Per instance (arrays of n pointers, device buffers caller-owned):
 *   F_dev [n_points] written; W_dev with room for J*m entries, dof written;
 *   backward only: u_obs_dev [n_points] read, grad_F_dev [n_points] written
 *   (or NULL), grad_coef_host [g*g] written for RANN_COEF_PIECEWISE handles
 *   (or NULL).
 * out[k]: the first failing step's status (RANN_NOT_CONVERGED of a solve is
 * recorded, not failing), dof, the apply configuration used, the loss, and
 * the forward and adjoint statistics.  Returns RANN_OK when every instance
 * succeeded, else the first failing instance's status (the others still
 * run).  A handle must not be used by the caller while the call runs. */
typedef struct rann_dd_batch rann_dd_batch;
typedef struct {
  int pca_mode;           /* RANN_PCA_*                                     */
  double pca_thr;
  int prec_kind;          /* RANN_PREC_*                                    */
  int solver;             /* 0: CG (prec AS or NONE), 1: GMRES(restart)     */
  double rtol;
  int restart;
  int maxit;
  int autotune;           /* 1: tune the Schwarz apply per size class       */
  int backward;           /* 1: also the misfit gradient                    */
} rann_dd_pipeline;
typedef struct {
  rann_status status;
  int64_t dof;
  int apply_config;
  double loss;
  rann_dd_stats forward, adjoint;
} rann_dd_pipeline_out;
rann_status rann_dd_batch_create(int nworkers, rann_dd_batch** out);
void rann_dd_batch_destroy(rann_dd_batch* b);
rann_status rann_dd_batch_run(rann_dd_batch* b, int n, rann_dd_handle* const* hs, const rann_dd_pipeline* cfg,
                              double* const* F_dev, double* const* W_dev, const double* const* u_obs_dev,
                              double* const* grad_F_dev, double* const* grad_coef_host, rann_dd_pipeline_out* out);


/* Measured device rates for roofline denominators (TFLOP/s, 2 flops per
 * multiply-add): df32_tflops, the double-float multiply-add of the Schwarz
 * apply and the inner operator on the float32 pipe; fp64_tflops, float64
 * FMAs.  Each is a timed loop of independent chains on every SM (legacy
 * default stream, synchronises).  Either pointer may be NULL. */
rann_status rann_dd_device_rates(double* df32_tflops, double* fp64_tflops);

/* Host-side fault injection for failure-detection tests (the paper has no
 * counterpart; no device code is made to fault, trap or hang):
 *   RANN_FAULT_WAIT_EXPIRED: writes `value` (non-zero) into the handle's
 *     device error word of the tensor-core product pipelines, exactly what a
 *     bounded mbarrier wait writes when it gives up; the next pca,
 *     setup_precond or solve that reads the word back returns RANN_TIMEOUT
 *     (and clears it).  value = 0 clears the word.
 *   RANN_FAULT_ALLOC_CAP: from now on the handle's device allocations fail
 *     (RANN_ENOMEM, before any cudaMalloc) whenever its live bytes would
 *     exceed `value`; value < 0 removes the cap.
 * A failed pca or setup_precond leaves the handle at the previous step of
 * Algorithm 1 (solves then return RANN_EORDER until the step succeeds). */
enum { RANN_FAULT_WAIT_EXPIRED = 1, RANN_FAULT_ALLOC_CAP = 2 };
rann_status rann_dd_inject_fault(rann_dd_handle* h, int kind, int64_t value);

const char* rann_dd_status_string(rann_status s);
const char* rann_dd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RANN_DD_H */
