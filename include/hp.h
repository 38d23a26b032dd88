/*
 * hp.h -- C ABI of the GB300 Gauss-Newton Hessian-action engine for the
 * log-coefficient Poisson inverse problem (hIPPYlib paper, Villa/Petra/Ghattas).
 *
 * Problem (Section 5.1, eqs. (poi), (poisson_weak)):
 *     -div(e^m grad u) = f  in the unit square (dim 2) or cube (dim 3),
 *     u = u_top on the face x_last = 1, u = u_bottom on x_last = 0,
 *     zero Neumann elsewhere;
 * P1 elements on a structured mesh of N^dim cells (2 right triangles per
 * square, 6 Kuhn tetrahedra per cube), nodes (N+1)^dim, lexicographic with the
 * first axis fastest.  The element coefficient is the element mean of e^m.
 *
 * Prior (Section 5.1.1, eq. (PoissonPrior); Section 2.3): A = gamma*K(1) + delta*M
 * with zero Neumann, precision R = A M^{-1} A.  Noise: Gamma = sigma^2 I,
 * B = P1 interpolation at the observation points (Section 5.1.1).
 *
 * Conventions (all entry points):
 *  - Vectors and blocks are DEVICE pointers to FP64, column-major, one column
 *    per right-hand side, leading dimension ld >= n (in elements).  They are
 *    owned by the caller; the library never frees them.
 *  - The library owns the opaque handle and its device workspace.  All work is
 *    enqueued on the stream set by hp_set_stream (default: the legacy stream)
 *    and each call synchronises that stream before returning, so outputs are
 *    ready when the call returns.  Scalars returned through host pointers are
 *    host memory.
 *  - Return value: HP_OK or a negative HP_ERR_* code; hp_status_string()
 *    names it and hp_last_error() gives a one-line detail.  Nothing throws
 *    across the ABI.  HP_ERR_NOT_CONVERGED leaves the best iterate in the
 *    outputs.
 *  - There is no CPU fallback: every numerical step runs in this library's
 *    CUDA kernels (sm_103a).
 */
#ifndef HP_H
#define HP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HP_OK 0
#define HP_ERR_INVALID (-1)
#define HP_ERR_NOT_CONVERGED (-2)
#define HP_ERR_NONFINITE (-3)
#define HP_ERR_CUDA (-4)
#define HP_ERR_NOMEM (-5)
#define HP_ERR_STATE (-6) /* a call needs hp_set_point first */

/* precision of the PDE solves */
#define HP_FP64_PLAIN 0 /* FP64 multigrid-preconditioned CG throughout       */
#define HP_FP32_IR 1    /* FP32 MG-PCG inside FP64 iterative refinement     */

/* flags of hp_hessian_apply */
#define HP_MISFIT_ONLY 0 /* Y = H_misfit X                                 */
#define HP_WITH_PRIOR 1  /* Y = (H_misfit + R) X                           */
#define HP_FULL_NEWTON 2 /* add the adjoint terms (full Hessian, see below)  */

typedef struct hp_problem hp_problem;

typedef struct {
  int dim;               /* 2 or 3                                            */
  int N;                 /* cells per axis (>= 1); nodes n = (N+1)^dim        */
  double gamma, delta;   /* prior operator A = gamma K(Theta) + delta M (> 0) */
  double sigma;          /* noise standard deviation (> 0)                    */
  int nobs;              /* number of pointwise observations (>= 0)          */
  const double *obs_xyz; /* HOST, nobs*dim, point-major, inside [0,1]^dim     */
  const double *d_obs;   /* HOST, nobs observed values (NULL = zeros)         */
  const double *m_prior; /* HOST, n prior mean (NULL = 0)                     */
  const double *f;       /* HOST, n nodal source, load = M f (NULL = 0)       */
  double u_top, u_bottom;/* Dirichlet data on x_last = 1 / x_last = 0         */
  int precision;         /* HP_FP64_PLAIN or HP_FP32_IR                       */
  double rtol;           /* relative residual of every PDE solve (e.g. 1e-8)  */
  int max_iter;          /* cap on CG iterations per solve (e.g. 500)         */
  double theta[6];       /* prior anisotropy Theta (s.p.d.): T00, T11, T22, T01,
                            T02, T12 (2D uses T00, T11, T01); all zero = identity */
  double robin_beta;     /* Robin condition Theta grad m . n + beta m = 0 of the
                            prior (Section 5.1.1): A gains gamma beta M_boundary;
                            0 = zero Neumann                                   */
} hp_problem_desc;

typedef struct {
  int iterations;        /* inner CG iterations (max over columns, summed over refinement steps) */
  int outer;             /* FP64 refinement steps (0 for HP_FP64_PLAIN)                        */
  int solves;            /* number of block solves performed by the call                     */
  double rel_res;        /* max over columns of the final FP64 relative residual             */
} hp_solve_stats;

typedef struct {
  double rel_tol;        /* stop when |g_i| <= rel_tol |g_0| (|g| = sqrt(g^T R^{-1} g)) */
  double abs_tol;        /* ... or |g_i| <= abs_tol                                       */
  int max_iter;          /* Newton iterations (Algorithm 1: max_iter)                     */
  int max_backtrack;     /* Armijo backtracks (Algorithm 1: max_backtracking_iter)        */
  double c_armijo;       /* Armijo constant (Section 4.1: 1e-5 .. 1e-4)                   */
  int cg_max_iter;       /* inner CG cap                                                  */
  int full_newton;       /* 0: Gauss-Newton Hessian; 1: full Hessian (HP_FULL_NEWTON); the
                            CG stops on non-positive curvature (Steihaug) either way       */
  int lowrank_k;         /* 0: CG preconditioned by R^-1 (Section 4.1).  > 0: by
                            R^-1 - V diag(lambda / (1 + lambda)) V^T, the inverse (Woodbury)
                            of R + R V Lambda V^T R with the lowrank_k leading eigenpairs of
                            H_misfit v = lambda R v (double pass, Philox directions)        */
  int lowrank_p;         /* oversampling of that eigensolve                                */
  int lowrank_refresh;   /* recompute the eigenpairs every lowrank_refresh Newton
                            iterations (0: only at the first)                              */
  double prec_rtol;      /* relative tolerance of the two prior solves of R^-1 when it
                            preconditions the CG (0: the problem's tolerance).  The
                            gradient and its R^-1 norm, which decide convergence, always
                            use the problem's tolerance.  A looser value makes the
                            preconditioner vary between CG iterations: it saved a few
                            percent where the CG needs few iterations, and stalled Newton
                            where it needs many (64^3 with k = 100).  No counterpart in
                            the paper.                                                     */
} hp_newton_opts;

typedef struct {
  int iterations;        /* Newton iterations taken                        */
  int cg_iterations;     /* total inner CG iterations (Hessian actions)    */
  int converged;         /* 1 if the gradient test was met                 */
  double J0, J;          /* initial and final cost                         */
  double gnorm0, gnorm;  /* initial and final |g|                          */
  int pde_solves;        /* total PDE block solves (state, adjoint, incremental, prior, mass) */
  int eig_solves;        /* low-rank preconditioner eigensolves                         */
} hp_newton_stats;

/* ---- lifetime ------------------------------------------------------------ */

/* Validates desc, copies its host arrays to the device, builds the observation
 * operator, the prior hierarchy and the workspace.  HP_ERR_INVALID on bad
 * sizes or parameters (dim not 2/3, N < 1, gamma/delta/sigma <= 0, points
 * outside the domain, coarsest multigrid grid too large). */
int hp_problem_create(const hp_problem_desc *desc, hp_problem **out);
void hp_problem_destroy(hp_problem *P);
/* cudaStream_t passed as void*; NULL = legacy default stream. */
int hp_set_stream(hp_problem *P, void *stream);
int hp_set_precision(hp_problem *P, int precision);
int hp_set_tolerance(hp_problem *P, double rtol, int max_iter);
/* Replaces observed data (HOST array of nobs values) and sigma (> 0). */
int hp_set_data(hp_problem *P, const double *d_obs_host, double sigma);
int hp_num_nodes(const hp_problem *P);
int hp_num_elements(const hp_problem *P);
/* Copies the device observation vector back: d_out HOST, nobs values. */
int hp_get_data(const hp_problem *P, double *d_out_host);

/* ---- forward problem / cost / gradient (Section 5.1, Appendix A) -------- */

/* Linearisation point: builds e^m coefficients and the multigrid hierarchy of
 * K(m), solves the state u(m).  m_dev: n values.  If J_out != NULL the cost
 * J(m) (eq. (cost-elliptic)) is written to J_out[0..2] = {J, misfit, reg}. */
int hp_set_point(hp_problem *P, const double *m_dev, double *J_out);
/* State u(m) (eq. (firststate)) into u_dev (n values, Dirichlet values included). */
int hp_forward(hp_problem *P, const double *m_dev, double *u_dev, hp_solve_stats *st);
/* y_dev[0..nobs) = B u for a device state u_dev. */
int hp_observe(hp_problem *P, const double *u_dev, double *y_dev);
/* Gradient g = R (m - m_pr) + C^T p with K p = -B^T (B u - d)/sigma^2
 * (eqs. (firstadj), (firstcontrol)).  Sets the linearisation point to m.
 * J_out (HOST, may be NULL) receives {J, misfit, reg}. */
int hp_gradient(hp_problem *P, const double *m_dev, double *g_dev, double *J_out);

/* ---- Hessian action (Appendix A, eqs. (incrementals1)-(incrementals3)) -- */

/* Gauss-Newton Hessian action at the current linearisation point on a block
 * of nrhs columns:  K Uh = -C X,  K Ph = -B^T B Uh / sigma^2,  Y = C^T Ph
 * (+ R X if flags & HP_WITH_PRIOR).  With flags & HP_FULL_NEWTON the adjoint
 * terms of the same equations are kept (the full Hessian):
 *   K Ph = -B^T B Uh / sigma^2 - C(p) X,  Y = C^T Ph + C(p)^T Uh + X (.) C^T p,
 * where p is the adjoint at the point (solved on first use after hp_set_point /
 * hp_set_data and kept) and C(p) is C built from p instead of u.  X and Y may
 * not alias. */
int hp_hessian_apply(hp_problem *P, const double *X_dev, int ldx, double *Y_dev, int ldy,
                     int nrhs, int flags, hp_solve_stats *st);

/* ---- operator pieces (exposed for parity tests and composition) --------- */

/* Y = K(m) X at the current point with Dirichlet rows as identity and the
 * couplings to Dirichlet nodes removed (the zero-Dirichlet operator). */
int hp_stiffness_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs);
/* X = K(m)^{-1} B on the zero-Dirichlet space (Dirichlet rows of B ignored). */
int hp_state_solve(hp_problem *P, const double *B, int ldb, double *X, int ldx, int nrhs,
                   hp_solve_stats *st);
/* Y = C X (all rows; C X = K(kappa_hat) u, kappa_hat = elem-mean(e^m X)). */
int hp_C_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs);
/* Y = C^T W,  (C^T W)_v = e^{m_v}/(dim+1) sum_{e ni v} |e| grad u . grad W. */
int hp_Ct_apply(hp_problem *P, const double *W, int ldw, double *Y, int ldy, int nrhs);
/* Prior operator A = gamma K(1) + delta M, mass M (Section 2.3). */
int hp_prior_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs);
int hp_mass_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs);
/* X = A^{-1} B (multigrid PCG). */
int hp_prior_solve(hp_problem *P, const double *B, int ldb, double *X, int ldx, int nrhs,
                   hp_solve_stats *st);
/* X = M^{-1} B (Jacobi PCG). */
int hp_mass_solve(hp_problem *P, const double *B, int ldb, double *X, int ldx, int nrhs,
                  hp_solve_stats *st);
/* Y = R X = A M^{-1} A X  and  Y = R^{-1} X = A^{-1} M A^{-1} X. */
int hp_R_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs);
int hp_Rinv_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs);
/* W = C_M eta: rectangular factor of M (Appendix C, eq. (rect_decomp)) with a
 * degree-2 element rule.  eta: (dim+1)*nelems normals per column, element-major. */
int hp_mass_factor_apply(hp_problem *P, const double *eta, int ldeta, double *W, int ldw, int nsamples);

/* ---- batches of independent problems ---------------------------------------
 * Many independent inverse problems of uneven size on one GPU (the batched
 * workload of the build; the paper treats one problem at a time).  Each problem
 * gets its own non-blocking CUDA stream (set with hp_set_stream; restored to the
 * legacy stream by hp_batch_destroy) and a pool of nthreads host threads (0 =
 * min(hardware threads, 16)) drives the problems, so their kernel sequences
 * run concurrently.  The problems stay owned by the caller.  Per-problem
 * arrays are indexed by problem; status[i] receives each problem's return
 * code and the call returns the first failure, else HP_OK.  Results equal
 * those of the same calls made on each problem alone.  The streams share the
 * device's hardware work queues, of which CUDA gives a process 8 unless the
 * environment variable CUDA_DEVICE_MAX_CONNECTIONS is set (up to 32) before CUDA
 * starts: with 32, a block of Hessian actions on 64 problems ran 7.8 % faster and
 * MAP + eigenpairs 35 % faster.  hp_batch_map_and_eig hands out the largest
 * problems first; the other calls go in index order. */
typedef struct hp_batch hp_batch;
int hp_batch_create(hp_problem *const *problems, int nproblems, int nthreads, hp_batch **out);
void hp_batch_destroy(hp_batch *B);
/* hp_set_point on every problem (m[i]: device, n_i values). */
int hp_batch_set_point(hp_batch *B, const double *const *m, int *status);
/* hp_newton_cg_map then hp_lowrank_eig (Algorithms 1, 2, 4) on every problem:
 * m_inout[i] (device, n_i) in: start, out: MAP point; Omega[i] n_i x (k+p), ld
 * ldo[i]; lambda[i] (k) and V[i] (n_i x k, ld ldv[i]) out; nstats may be NULL. */
int hp_batch_map_and_eig(hp_batch *B, double *const *m_inout, const hp_newton_opts *opts, int k, int p,
                         const double *const *Omega, const int *ldo, double *const *lambda,
                         double *const *V, const int *ldv, hp_newton_stats *nstats, int *status);
/* hp_hessian_apply on every problem at its current point. */
int hp_batch_hessian_apply(hp_batch *B, const double *const *X, const int *ldx, double *const *Y,
                           const int *ldy, const int *nrhs, int flags, int *status);

/* ---- solve without device allocation ---------------------------------------
 * The paper has no counterpart to this entry point: it serves callers that
 * cannot allocate device memory when they solve.  hp_mass_solve grows the
 * problem's workspace with cudaMalloc on first use; an application that reserves
 * all device memory at start-up, or must keep its device footprint fixed while it
 * runs, cannot allow that.  hp_mass_solve_noalloc computes the same X = M^{-1} B
 * (FP64 diagonally preconditioned CG, per-column relative residual
 * min(rtol, 1e-10)) using one fixed file-scope device array as scratch, and
 * calls no cudaMalloc / cudaFree or allocating library routine.
 *  - Limits: nrhs <= HP_NOALLOC_MAX_COLS and n * nrhs <= HP_NOALLOC_MAX_ENTRIES,
 *    else HP_ERR_INVALID.  The scratch array (4 * HP_NOALLOC_MAX_ENTRIES doubles
 *    plus per-column partials, about 8.5 MB) lives on every GPU that loads the
 *    library until the process exits.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress).
 *  - All calls share the one array: calls that overlap on the GPU (other streams,
 *    other threads, other problems) race and must be serialised by the caller.
 *    Each call re-initialises what it reads, so no state carries over.
 *  - The call synchronises the problem's stream once per CG iteration (it reads
 *    the per-column convergence flags into a host array), so it cannot be
 *    recorded into a CUDA graph. */
#define HP_NOALLOC_MAX_COLS 64
#define HP_NOALLOC_MAX_ENTRIES 262144
int hp_mass_solve_noalloc(hp_problem *P, const double *B, int ldb, double *X, int ldx, int nrhs,
                          hp_solve_stats *st);

/* ---- algorithms (Section 4) ---------------------------------------------- */

/* Inexact Newton-CG (Algorithm 1) from m_dev_inout (n values) to the MAP point.
 * opts may be NULL (defaults: rel_tol 1e-6, abs_tol 0, max_iter 50,
 * max_backtrack 10, c_armijo 1e-4, cg_max_iter 200, Gauss-Newton, R^-1
 * preconditioner).  The linearisation point
 * is left at the returned m. */
int hp_newton_cg_map(hp_problem *P, double *m_dev_inout, const hp_newton_opts *opts,
                     hp_newton_stats *st);
/* Double-pass randomized generalized eigensolver (Algorithm 2 with PreCholQR,
 * Algorithm 4) for H_misfit v = lambda R v at m_map_dev.  Omega_dev: n x (k+p)
 * Gaussian test matrix (caller-drawn), ld ldo.  Outputs: lambda_dev (k values,
 * descending), V_dev (n x k, ld ldv, R-orthonormal, sign: largest-magnitude
 * entry positive).  single_pass != 0 selects Algorithm 3 instead: one block of
 * k+p Hessian actions, T the least-squares fit of eq. (Tsinglepass) over
 * symmetric matrices (solved exactly as the Lyapunov equation X M + M X = C,
 * M = W W^T, C = Zs W^T + W Zs^T, W = Qb^T Omega, Zs = Qb^T Y, Qb = R Q). */
int hp_lowrank_eig(hp_problem *P, const double *m_map_dev, int k, int p, const double *Omega_dev,
                   int ldo, double *lambda_dev, double *V_dev, int ldv, int single_pass,
                   hp_solve_stats *st);
/* Laplace-approximation samples (Section 4.3): for each sample j, prior sample
 * m_pr + x with x = A^{-1} C_M eta_j (eq. (sample_prior)) and posterior sample
 * m_map + x - V S V^T R x, S = diag(1 - 1/sqrt(1+lambda)) (eq. (sample_post)).
 * eta_j ((dim+1)*nelems standard normals, element-major) is column j of eta_dev
 * (ld ldeta) or, when eta_dev is NULL, drawn on the device from Philox4x32-10
 * with the given seed (see hp_philox_normals; sample index j).  prior_dev /
 * post_dev: n x nsamples, ld lds (either may be NULL). */
int hp_laplace_sample(hp_problem *P, const double *m_map_dev, const double *lambda_dev,
                      const double *V_dev, int ldv, int k, const double *eta_dev, int ldeta,
                      unsigned long long seed, int nsamples, double *prior_dev, double *post_dev,
                      int lds, hp_solve_stats *st);

/* Standard normals from Philox4x32-10 (Salmon et al., SC'11), as the sampler draws
 * them: out[ld*j + t] is normal t of sample first_sample + j.  Call g = t/4 uses
 * counter (g, g>>32, sample, sample>>32) and key (seed, seed>>32); its words
 * (x0,x1), (x2,x3) give two FP32 Box-Muller pairs with u = ((x>>8) + 1/2) 2^-24.
 * raw != 0 writes the 32-bit words themselves (as doubles).  DEVICE out,
 * enqueued on stream (cudaStream_t; NULL = legacy) and synchronised. */
int hp_philox_normals(unsigned long long seed, long long first_sample, int nsamples, int nper,
                      double *out, int ld, int raw, void *stream);

/* Pointwise variance (Section 4.4).  The prior part, diag(R^-1), by
 *   HP_VAR_RANDOMIZED: Algorithm 2 with A = R^-1, B = I on the r columns of Z
 *     (Gaussian, caller-drawn): diag(R^-1) ~ sum_i mu_i vbar_i (.) vbar_i
 *     (eq. (prior_mvar)); or
 *   HP_VAR_STOCHASTIC: diag(R^-1) ~ [sum_j z_j (.) w_j] / [sum_j z_j (.) z_j] with
 *     R w_j = z_j for the r probe columns of Z (eq. (stoc_diag_estimator)).
 * prior_var_dev (n) receives it.  With k > 0 eigenpairs (lambda_dev, V_dev) of
 * the prior-preconditioned misfit Hessian, post_var_dev (n) receives
 * prior_var - sum_i lambda_i / (1 + lambda_i) v_i (.) v_i (eq. (post_mvar));
 * post_var_dev may be NULL.  Z_dev: n x r, ld ldz; r <= min(n, 1024) for the
 * randomized method.  Needs no linearisation point (R does not depend on m). */
#define HP_VAR_RANDOMIZED 0
#define HP_VAR_STOCHASTIC 1
int hp_pointwise_variance(hp_problem *P, int method, const double *Z_dev, int ldz, int r,
                          const double *lambda_dev, const double *V_dev, int ldv, int k,
                          double *prior_var_dev, double *post_var_dev, hp_solve_stats *st);

/* ---- tuning ----------------------------------------------------------------
 * Knobs of the PDE solver (no counterpart in the paper): nu damped-Jacobi sweeps
 * before and after each coarse correction and damping omega, the number of RHS
 * columns solved together (0 = all), and the grid-size cap of the node kernels.
 * Defaults: nu 3, nu_coarse 0, omega 0.7, col_chunk 0, max_blocks 4096, smoother 1
 * (Chebyshev), cheb_alpha 10, fuse_transfer 0, fuse_from 0, tma_tiles 0, smem_tail 0.  Every setting solves to the same
 * tolerance; only speed changes. */
typedef struct {
  int nu;          /* 1..4 */
  int nu_coarse;   /* 0 = nu, else the sweeps on the levels below the finest (1..4) */
  double omega;    /* (0, 1) */
  int col_chunk;   /* >= 0 */
  int max_blocks;  /* >= 64 */
  int smoother;    /* 0 damped Jacobi with omega; 1 Chebyshev: sweep k uses the
                      reciprocal of root k of the degree-nu Chebyshev polynomial on
                      [lmax / cheb_alpha, lmax] (lmax: Gershgorin bound of D^-1 S on
                      each level), post-smoothing in reverse order */
  double cheb_alpha; /* > 1 */
  int fuse_transfer; /* 1: the residual and its restriction run as one kernel, and so
                        do the prolongation and the first post-smoothing sweep (the
                        fine residual and the prolonged iterate are never stored);
                        2: the same on the levels below the finest only */
  int fuse_from;   /* reserved: must be 0 (HP_ERR_INVALID otherwise) */
  int tma_tiles;   /* 1: on the multigrid levels of stiffness solves whose grid has np - 1 a
                      multiple of 32 (2D: and of 16; 3D: and of 16 planes), the stencil
                      kernels work on tiles that bulk tensor copies (TMA) bring into shared
                      memory with their halo -- 32 x 16 nodes in 2D, 32 x 8 nodes marching
                      through z segments of 16 or 8 planes in 3D (the launch picks the
                      length that fills the GPU's last wave of CTAs better); 2: the same on
                      the finest level only (the coarser levels keep the row kernels); 0:
                      every warp loads its own row of nodes */
  int smem_tail;   /* k >= 1: the coarse end of the V-cycle -- from the finest level l >= k
                      whose vectors, and those of every level below it, fit in one CTA's
                      shared memory -- runs as one launch of one CTA per column group, its
                      steps separated by block barriers only; the result equals the
                      per-level kernels' bit for bit.
                      0: off */
  int refine_df;   /* arithmetic of the FP64 iterative refinement around FP32 inner solves
                      (the residual b - K x with its norm, the scaling into the inner
                      precision and the update x += d): 0 FP64 instructions; 1 (default)
                      double-float arithmetic for solve tolerances >= 1e-9 on blocks of at
                      least 2^24 values (n times the columns), FP64 otherwise:
                      b and x held as pairs of floats (about 48 significand bits) in the
                      refinement's workspace, compensated products and sums on the FP32
                      pipe, the caller's FP64 blocks converted once per solve by bit
                      manipulation (C and C^T follow the same rule); 2 the same at every
                      tolerance and block size.  Any nonzero value also runs the eigensolver's
                      dense products (Gram, triangular solve, block product, the small
                      Jacobi eigensolver) in double-float with compensated sums. */
} hp_tuning;
int hp_set_tuning(hp_problem *P, const hp_tuning *t);
int hp_get_tuning(const hp_problem *P, hp_tuning *t);
/* Times one block of nrhs Gauss-Newton Hessian actions at the current point
 * (CUDA events, the mean of reps timed runs after a warm-up per candidate) over a
 * small candidate set by coordinate descent in two passes (smoother, column
 * chunk, fused transfers, coarse tails, tiled kernels, grid cap; a candidate must
 * be at least 1 % faster to be taken) and applies the fastest.  best / best_ms
 * (HOST, may be NULL) receive it.  Needs hp_set_point first; allocates its test
 * block (setup-time call). */
int hp_autotune(hp_problem *P, int nrhs, int reps, hp_tuning *best, double *best_ms);
/* The same search timed on the caller's block: X (DEVICE, column-major n x nrhs,
 * ldx >= n) is the block of directions the settings are for (the iteration count
 * of a candidate depends on the right-hand sides, so a random block can favour
 * another smoother than the block that will run).  X is only read. */
int hp_autotune_block(hp_problem *P, const double *X, int ldx, int nrhs, int reps, hp_tuning *best,
                      double *best_ms);

/* ---- learned warm start (2D stiffness solves; no counterpart in the paper) --
 * A 4-level U-Net (16-32-64-128 channels, 3x3 convolutions with zero padding,
 * 2x2 mean pooling, nearest 2x upsampling, skip concatenation [upsampled, skip],
 * ReLU, 1x1 output layer) on an H x W grid, H and W multiples of 8.  Weights are
 * kept in FP32 (master copy, Adam) and used by every kernel as BF16; activations
 * and accumulation are FP32.  All tensors are NCHW FP32, batch first.
 * Parameters are packed layer by layer, each layer its weights (co, ci, k, k)
 * then its biases (co), in the order enc1a 3->16, enc1b 16->16, enc2a 16->32,
 * enc2b 32->32, enc3a 32->64, enc3b 64->64, bota 64->128, botb 128->128,
 * dec3a 192->64, dec3b 64->64, dec2a 96->32, dec2b 32->32, dec1a 48->16,
 * dec1b 16->16, out 16->1 (1x1).  A network is used by one thread at a time.
 *
 * Training loss: the relative residual of the output y in the sample's own
 * stiffness system.  A sample is an input x (3,H,W), whose channel 2 is the 0/1
 * mask of the free nodes, and loss data aux (4,H,W) = (b, diag, cx, cy): the
 * right-hand side and the symmetric 5-point stencil of K on the grid (cx couples
 * a pixel to its right neighbour, cy to the one below).  With S = mask K mask,
 *   L = 1/(2N) sum_n |mask_n b_n - S_n y_n|^2 / |mask_n b_n|^2
 * (a sample with a zero right-hand side counts 0). */
typedef struct hp_unet hp_unet;
/* batch_cap: largest N of a forward / gradient call.  Parameters start at zero:
 * set them with hp_unet_set_params. */
int hp_unet_create(int H, int W, int batch_cap, hp_unet **out);
void hp_unet_destroy(hp_unet *U);
long hp_unet_num_params(const hp_unet *U);
/* HOST arrays of hp_unet_num_params floats.  set_params also rounds the weights
 * to BF16 for the kernels and resets the Adam state. */
int hp_unet_set_params(hp_unet *U, const float *params);
int hp_unet_get_params(const hp_unet *U, float *params);
/* y (N,1,H,W) = net(x (N,3,H,W)); DEVICE arrays, 1 <= N <= batch_cap; synchronous. */
int hp_unet_forward(hp_unet *U, const float *x, int N, float *y);
/* Loss (HOST double, may be NULL) and its gradient with respect to the packed
 * parameters (HOST floats, may be NULL) for DEVICE x (N,3,H,W) and aux (N,4,H,W). */
int hp_unet_loss_grad(hp_unet *U, const float *x, const float *aux, int N, double *loss, float *grad);
/* Adam (beta 0.9, 0.999, eps 1e-8, step size lr) over `epochs` passes of the
 * nsamples DEVICE samples X (nsamples,3,H,W), A (nsamples,4,H,W) in shuffled
 * batches of `batch` (a trailing partial batch is skipped); the order comes from
 * seed.  loss_per_epoch (HOST, epochs doubles, may be NULL) gets the mean batch
 * loss of each epoch. */
int hp_unet_train(hp_unet *U, const float *X, const float *A, int nsamples, int epochs, int batch, double lr,
                  unsigned long long seed, double *loss_per_epoch);
/* Where the 3x3 convolutions with a multiple of 16 output channels run (the forward
 * pass, and the input gradient of the backward pass): on = 1 (the default), on the
 * tensor cores as implicit GEMMs (tcgen05 MMAs on BF16 operands, FP32 accumulators in
 * tensor memory; each FP32 activation or gradient enters as three BF16 terms, its full
 * significand, and the tensor core's accumulation truncates: outputs agree with the
 * FP32-pipe kernels to about 1e-5 relative); on = 0, on the FP32 pipes.  The
 * weight gradients and the 1x1 output layer use the FP32 pipes either way.  A
 * tensor-core convolution whose MMAs have not completed after about a second gives up
 * and makes the forward, gradient or training call fail with HP_ERR_CUDA.
 * get_tensor_cores returns the setting (-1 for NULL).  Not part of the paper. */
int hp_unet_set_tensor_cores(hp_unet *U, int on);
int hp_unet_get_tensor_cores(const hp_unet *U);

/* The network's view of a 2D problem: grid H = W = the node count per axis
 * rounded up to a multiple of 8; node (ix, iy) sits at row iy, column ix.  For a
 * solve K x = b (b zero on the Dirichlet faces iy = 0, N): z = D^-1 b with D the
 * diagonal of K, c = |z| / sqrt(nfree) its RMS over the nfree free nodes.  Input
 * channels: m; z / c; the 0/1 mask of the free nodes.  The output y is the
 * solution in the same scaling, so the initial guess is x0 = c y on the free
 * nodes, 0 elsewhere.  HP_ERR_INVALID for a 3D problem. */
int hp_warmstart_grid(const hp_problem *P, int *H, int *W);
/* Attaches a network (not owned; NULL detaches) of the problem's grid.  While
 * attached and enabled, every stiffness solve (state, adjoint, incremental
 * forward and adjoint) starts from the network's guess instead of zero; a
 * column whose guess has a residual no smaller than |b| (or non-finite) starts
 * from zero instead.  Every solve still runs to the same relative tolerance. */
int hp_warmstart_attach(hp_problem *P, hp_unet *U);
int hp_warmstart_enable(hp_problem *P, int on);
/* Records the problem's stiffness solves as training samples: after each solve,
 * column j appends its network input to X (capacity,3,H,W), its loss data
 * (b / c, diag, cx, cy) of the current level-0 stiffness stencil to A
 * (capacity,4,H,W) and, if T is not NULL, its solution x / c to T
 * (capacity,1,H,W) (DEVICE arrays) until capacity is reached.  X = NULL stops
 * recording (the count of the last recording stays readable); a new recording
 * starts the count from zero. */
int hp_warmstart_record(hp_problem *P, float *X, float *A, float *T, int capacity);
/* Samples recorded, columns that started from a guess, columns that fell back
 * to zero (HOST, each may be NULL); since attach / record. */
int hp_warmstart_counts(const hp_problem *P, long long *recorded, long long *guesses, long long *fallbacks);

/* ---- measurement ---------------------------------------------------------- */

/* Kernel families timed when profiling is on (CUDA events on the problem's
 * stream around each launch):  0 level-0 PCG matvec (stencil + <p,Kp>),
 * 1 level-0 Jacobi smoothing sweep, 2 level-0 V-cycle residual, 3 FP64
 * refinement residual, 4 CG vector update (+ <r,r>), 5 whole V-cycle,
 * 6 level-0 fused two-sweep pre-smoothing. */
#define HP_PROF_NIDS 7
/* Turns event timing on (on != 0) or off and clears the records. */
int hp_profile_enable(hp_problem *P, int on);
/* Synchronises the stream and returns, per family id < nids, the number of
 * timed launches and their summed duration in ms (HOST arrays); clears.
 * While profiling, kernels are launched directly (not as graphs) and each PCG
 * iteration is headed by a short bounded clock-spin kernel, so the iteration's
 * kernels run back to back and each event pair times its kernel alone. */
int hp_profile_read(hp_problem *P, int nids, int *counts, double *total_ms);
/* Replays one level-0 kernel of the last FP32 block solve on its live workspace
 * (same columns, launch configuration and tuning), reps times back to back on the
 * problem's stream, with CUDA events around the burst: family 0 damped-Jacobi
 * sweep, 1 V-cycle residual, 2 fused two-sweep pre-smoothing.  The kernels read
 * the workspace and write a scratch level vector, so the solver state is kept.
 * us_warm (HOST, may be NULL): mean microseconds per launch back to back (data
 * largely L2-resident).  us_cold (HOST, may be NULL): each launch preceded by a
 * read of the DEVICE buffer `flush` (>= 64 MB; pass one larger than L2), minus
 * the same reads timed alone -- the launch with its data in HBM.  Needs a prior
 * FP32 solve with at least 4 columns on a multilevel hierarchy (HP_ERR_STATE). */
int hp_replay_kernel(hp_problem *P, int family, int reps, void *flush, size_t flush_bytes, double *us_warm,
                     double *us_cold);
/* The same kernel replayed inside a CUDA graph: reps launches captured into one
 * graph, which is launched once untimed and once timed (CUDA events around the
 * graph launch).  us (HOST) receives the mean microseconds per launch -- the cost
 * of the kernel as the solver's captured PCG loop runs it, without the ~2 us
 * granularity of back-to-back stream launches.  Same preconditions as above;
 * allocates and frees the graph (a measurement call, not for the hot path). */
int hp_replay_kernel_graph(hp_problem *P, int family, int reps, double *us);

/* ---- status --------------------------------------------------------------- */
const char *hp_status_string(int status);
const char *hp_last_error(void);
/* Number of this library's kernel launches since load (for launch accounting). */
unsigned long long hp_kernel_launches(void);
/* Launches of the TMA-tiled stencil kernels (2D tiles and the 3D z-marching kernel)
 * made directly, so that a caller can tell which kernel form a solve ran.  Kernels
 * recorded into or replayed from CUDA graphs are not counted: with profiling on
 * (hp_profile_enable) every kernel is launched directly. */
unsigned long long hp_tiled_kernel_launches(void);
/* Algorithmic DRAM bytes (every array a kernel must read or write, counted once per
 * launch) of the kernels on the Hessian-action path since load, summed over direct
 * launches only: launches recorded into CUDA graphs are not counted, so measure a
 * step with profiling on (hp_profile_enable, which launches directly) and divide the
 * difference by the step's duration for its bandwidth.  out (HOST) receives nfam
 * cumulative totals, indexed by the families below (entries past the last family
 * are 0).  Kernels counted: the stencil kernels on every level (row and tiled forms),
 * the dense coarse solve, restriction and prolongation, the PCG vector updates and
 * inner products, the FP64 refinement passes, C, C^T and the observation operator. */
#define HP_BYTES_STENCIL0 0 /* stencil kernels on the finest level (PCG matvec, sweeps, residual) */
#define HP_BYTES_STENCILC 1 /* stencil kernels on coarser levels and the dense coarse solve   */
#define HP_BYTES_TRANSFER 2 /* restriction and prolongation                                  */
#define HP_BYTES_VECTOR 3   /* PCG vector updates and inner products                         */
#define HP_BYTES_REFINE 4   /* FP64 refinement: start, residual with norm, scaling, update   */
#define HP_BYTES_CCT 5      /* C, C^T and the observation gather / scatter                   */
#define HP_BYTES_FAMILIES 6
int hp_algorithmic_bytes(double *out, int nfam);

#ifdef __cplusplus
}
#endif
#endif /* HP_H */
