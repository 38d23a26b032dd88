// internal.h -- library-internal types and the host launchers shared between
// the translation units of libhp.so.  Not part of the ABI (see include/hp.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hp.h"
#include "common.cuh"

namespace hp {

// Grids whose stiffness stencils run as TMA-tiled kernels (2D, np - 1 a multiple of the
// 32 x 16 tile, at least one tile wide): the last tile in each direction also takes the
// grid's final node / row.
constexpr int TILE_X = 32, TILE_Y = 16;
inline bool tile_grid(const GridDesc &g) {
  return g.dim == 2 && g.np >= TILE_X + 1 && (g.np - 1) % TILE_X == 0 && (g.np - 1) % TILE_Y == 0;
}
// 3D: 32 x 8-node xy tiles marching through z segments of 16 planes, or of 8 where that
// fills the GPU's last wave of CTAs better (the last tile or segment in each direction also
// takes the grid's final node / row / plane)
constexpr int TILE3_X = 32, TILE3_Y = 8, TILE3_Z = 16;
inline bool tile3_grid(const GridDesc &g) {
  return g.dim == 3 && g.np >= TILE3_X + 1 && (g.np - 1) % TILE3_X == 0 && (g.np - 1) % TILE3_Y == 0 &&
         (g.np - 1) % TILE3_Z == 0;
}

// Symmetric stencil stored by "forward" couplings: y_i = diag_i x_i +
// sum_f [c_f(i) x_{i+o_f} + c_f(i-o_f) x_{i-o_f}], with o_f the 0/1 corner
// masks of the Kuhn edges.  full = false: axis offsets only (stiffness,
// 5-/7-point); full = true: all 2^D - 1 edge directions (prior / mass,
// 7-/15-point).  Coefficient f of node i is at c[f * n + i].
template <typename T> struct Stencil {
  T *diag = nullptr;
  T *invdiag = nullptr;
  T *c = nullptr;
  T *pk = nullptr;  // axis stencils on tiled grids: one record {diag, invdiag, c_0, c_1} per node
                    // (16 B); in 3D followed by c_2 in rows of (np + 3) / 4 * 4 (16-byte strides)
  int nf = 0;
  bool full = false;
  double lmax = 2.0;  // upper bound of the spectrum of diag^-1 S (Gershgorin)
  // FP64 stencils: the coefficients as double-float pairs {hi, lo} (c_f at [f n + i], the
  // diagonal at [nf n + i]) for the double-float refinement, made on first use after the
  // coefficients change (cpr_ok is cleared wherever they are rebuilt)
  float2 *cpr = nullptr;
  bool cpr_ok = false;
};

struct Level {
  GridDesc g{};
  long nelems = 0;
  double *kappa = nullptr;   // element coefficients of K on this level
  Stencil<double> K64, A64;
  Stencil<float> K32, A32;
};

struct CoarseInv {
  int nc = 0;
  bool fp64_valid = false;   // inv64 holds the FP64 inverse (else only inv32 is current)
  double *dense = nullptr;   // work: nc x nc
  double *inv64 = nullptr;
  float *inv32 = nullptr;
};

enum OpKind { OP_K = 0, OP_A = 1, OP_M = 2 };

// growable device buffer
struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  int ensure(size_t b);
  void release();
  template <typename T> T *as() const { return static_cast<T *>(p); }
};

template <typename T> struct BlockWS {
  int scap = 0;       // column capacity
  long ldn = 0;       // padded column stride
  DBuf x, r, z, p, q;               // PCG vectors
  DBuf lr[HP_MAXL], la[HP_MAXL], lb[HP_MAXL];  // MG level vectors (level 0 uses r/z and lb[0])
};

// a captured PCG loop (init + device-side while node), cached per configuration
struct PcgGraph {
  int op, tbytes, vw, s, maxit;
  double tol;
  cudaGraphExec_t exec;
};

// Device-side state of a graph-driven iterative refinement (one solve at a time).
struct RefineCtl {
  int outer;       // refinement steps run
  int total_its;   // inner PCG iterations, summed over the steps
  int flags;       // 1: not converged within max_outer, 2: non-finite residual
  int pad;
  double worst;    // max_j |r_j| / |b_j| at the last check
};

// a captured refinement loop: a while node over the refinement steps, each with the
// scaling into the inner precision, the PCG (nested while node), the accumulation,
// the FP64 residual and the convergence control; cached per configuration
struct SolveGraph {
  int op, tbytes, vw, s, maxit, max_outer;
  double rtol, tol_in;
  cudaGraphExec_t exec;
};

struct ScalarWS {
  int scap = 0;
  DBuf rz, pq, rr, bb, alpha, beta, scale, iscale, tol2col, tmp;   // double per column
  DBuf bbr;                                        // |b|^2 of a graph-driven refinement (the PCG reuses bb)
  DBuf active;                                     // int per column
  DBuf partial;                                    // double [slot][col][block]
  DBuf counter;                                    // unsigned [slot][col]
  DBuf iter;                                       // int: PCG iteration counter
  int hcap = 0;                                    // pinned host mirrors
  int *h_active = nullptr, *h_iter = nullptr;
  double *h_rr = nullptr, *h_bb = nullptr;
};

}  // namespace hp

struct hp_problem {
  // description
  int dim = 2, N = 0, L = 0;
  long n = 0, nelems = 0;
  double gamma = 0, delta = 0, sigma = 1, u_top = 1, u_bottom = 0;
  double theta[6] = {1, 1, 1, 0, 0, 0};  // prior anisotropy (T00, T11, T22, T01, T02, T12)
  double robin_beta = 0;                 // prior Robin coefficient beta (0 = zero Neumann)
  int precision = HP_FP32_IR;
  double rtol = 1e-8;
  double u_rtol = 0.0;          // tolerance the current state u was solved to
  int max_iter = 500;
  double inner_rtol = 1e-5;     // FP32 inner tolerance of the refinement
  int max_outer = 12;
  int nu = 3;                   // pre/post smoothing sweeps         (tuning)
  int nu_coarse = 0;            // sweeps on the coarser levels, 0 = nu (tuning)
  double omega = 0.7;           // Jacobi damping                     (tuning)
  int col_chunk = 0;            // RHS columns per solve, 0 = all     (tuning)
  long max_blocks = 4096;       // grid cap of the node kernels       (tuning)
  int fuse_from = 0;            // first multigrid level of the fused coarse tail, 0 = none (tuning)
  int smoother = 1;             // 0 damped Jacobi (omega), 1 Chebyshev (cheb_alpha)   (tuning)
  int fuse_transfer = 0;        // residual + restriction and prolongation + first post sweep fused (tuning)
  double cheb_alpha = 10.0;     // Chebyshev interval [lmax / alpha, lmax]             (tuning)
  int tma_tiles = 0;            // 2D stiffness levels as TMA-tiled stencil kernels       (tuning)
  int smem_tail = 0;            // coarse V-cycle levels in one shared-memory CTA per group (tuning)
  int refine_df = 1;            // FP64 refinement arithmetic in double-float on the FP32 pipe:
                                // 0 never, 1 for tolerances >= DF_MIN_RTOL, 2 always (tuning)
  cudaStream_t st = nullptr;
  cudaStream_t cap = nullptr;   // private stream used to capture CUDA graphs
  bool use_graphs = true;       // inner PCG loops as graphs with a device-side while node
  std::vector<hp::PcgGraph> graphs;
  std::vector<hp::SolveGraph> sgraphs;

  hp::Level lv[HP_MAXL];
  hp::CoarseInv cK, cA;
  hp::Stencil<double> M64;
  hp::Stencil<float> M32;

  // point-dependent state
  bool have_point = false;
  double *m = nullptr, *E = nullptr, *u = nullptr, *lift = nullptr;
  double *Cbeta = nullptr;      // C as a stencil on e^m (.) X: (2^{D+1}-1) x n, built from u
  // double-float pairs of CbetaE, Cbeta and e^m for the double-float C / C^T kernels, made on
  // first use after C is rebuilt; the input block of those kernels as pairs (grouped by 4)
  float2 *CbetaE_pr = nullptr, *Cbeta_pr = nullptr, *E_pr = nullptr;
  bool cct_pr_ok = false;
  hp::DBuf xpairs;
  hp::DBuf dense_tmp;  // n x s scratch of the eigensolver's double-float triangular solves
  double *CbetaE = nullptr;     // the same coefficients with e^m folded in (C X = CbetaE-stencil X)
  // adjoint terms of the full Newton Hessian (built on demand at the current point)
  double *padj = nullptr;       // adjoint p
  double *Cbeta_p = nullptr;    // C(p): the same stencil built from p
  double *CbetaE_p = nullptr;   // ... with e^m folded in
  double *wmm = nullptr;        // C(u)^T p: weights of the diagonal second-derivative term
  bool have_p = false, have_full = false;
  // data
  double *m_prior = nullptr, *f_load = nullptr, *d_obs = nullptr;
  int nobs = 0;
  int *obs_node = nullptr;      // nobs * (dim+1)
  double *obs_w = nullptr;      // nobs * (dim+1)
  int *bt_row = nullptr;        // n: CSR row of B^T for the node, -1 if untouched
  int *bt_ptr = nullptr;        // rows + 1
  int *bt_ent = nullptr;        // entries: obs * (dim+1) + k
  int bt_rows = 0;

  // workspaces
  hp::BlockWS<float> w32;
  hp::BlockWS<double> w64;
  hp::ScalarWS sc;
  hp::DBuf r64, b64, t64a, t64b, t64c, obsbuf, small, etabuf, vtmp[6];
  hp::DBuf x64;                     // iterate of a graph-driven refinement (copied out at the end)
  hp::DBuf rctl;                    // RefineCtl of the graph-driven refinement
  hp::RefineCtl *h_rctl = nullptr;  // pinned host mirror

  // optional CUDA-event timing of selected kernels (hp_profile_*)
  bool prof_on = false;
  std::vector<int> prof_id;
  std::vector<cudaEvent_t> prof_ev;   // 2 per record
  size_t prof_used = 0;
  bool prof_failed = false;            // graph-recorded event timing unavailable
  long prof_cnt[16] = {};              // harvested totals per family
  double prof_ms[16] = {};

  // learned warm start of the stiffness solves (warm.cu)
  hp_unet *ws_net = nullptr;
  bool ws_on = false;
  float *ws_rx = nullptr, *ws_ra = nullptr, *ws_rt = nullptr;  // recorder targets (caller's)
  long ws_rcap = 0, ws_rcount = 0;
  long long ws_guesses = 0, ws_fallbacks = 0;
  hp::DBuf ws_flag, ws_bb, ws_z;
};

namespace hp {

int set_error(int code, const std::string &msg);
int cuda_check(cudaError_t e, const char *where);
#define HP_CUDA(call)                                              \
  do {                                                             \
    int _rc = ::hp::cuda_check((call), #call);                     \
    if (_rc) return _rc;                                           \
  } while (0)
#define HP_TRY(call)              \
  do {                            \
    int _rc = (call);             \
    if (_rc) return _rc;          \
  } while (0)

// ---- profiling ids (kernel families timed by hp_profile_*) ----------------
enum ProfId {
  PROF_MATVEC = 0,     // level-0 stencil apply fused with <p, Kp> (PCG matvec)
  PROF_SMOOTH = 1,     // level-0 damped-Jacobi sweep
  PROF_RESID_MG = 2,   // level-0 residual inside the V-cycle
  PROF_RESID64 = 3,    // FP64 refinement residual
  PROF_CG_UPDATE = 4,  // x += a p, r -= a q, <r, r>
  PROF_VCYCLE = 5,     // whole preconditioner application
  PROF_PRESMOOTH = 6,  // level-0 fused two-sweep pre-smoothing from zero
  PROF_COUNT = 7
};
int prof_start(hp_problem *P, int id);   // returns a record index or -1
void prof_stop(hp_problem *P, int rec);
void prof_harvest(hp_problem *P, size_t from, size_t to, bool keep);
void prof_spin(hp_problem *P);  // profiling only: keep the GPU busy while the host enqueues  // add records' times to the totals

// ---- fem.cu -------------------------------------------------------------
int build_hierarchy_geometry(hp_problem *P);  // levels, allocs, prior/mass stencils, coarse A inverse
int build_point(hp_problem *P, const double *m_dev);  // E, kappa hierarchy, K stencils, lift, coarse K inverse
void launch_build_C(hp_problem *P);  // after the state solve
// C(w) stencil of any nodal w: beta (for C^T) and betaE (beta with e^m folded in, for C)
void launch_build_C_from(hp_problem *P, const double *w, double *beta, double *betaE);
void launch_C_apply_beta(hp_problem *P, const double *betaE, const double *X, long ldx, double *Y, long ldy, int s,
                         double scale, double yb);
void launch_Ct_apply_beta(hp_problem *P, const double *beta_c, const double *W, long ldw, double *Y, long ldy, int s,
                          double scale, double beta);
void launch_C_apply(hp_problem *P, const double *X, long ldx, double *Y, long ldy, int s, double scale);
void launch_Ct_apply(hp_problem *P, const double *W, long ldw, double *Y, long ldy, int s, double scale,
                     double beta);
void launch_obs_gather(hp_problem *P, const double *X, long ldx, double *Yq, int s);
void launch_obs_scatter(hp_problem *P, const double *Yq, double *X, long ldx, int s, double scale);
void launch_mass_factor(hp_problem *P, const double *eta, long ldeta, double *W, long ldw, int s);
void launch_zero_dirichlet(hp_problem *P, double *X, long ldx, int s);

// ---- rng.cu ----------------------------------------------------------------
void launch_philox_normals(unsigned long long seed, long long first, int nsamples, int nper, double *out, long ld,
                           int raw, cudaStream_t st);
template <typename T>
void launch_stencil_apply(const hp_problem *P, const GridDesc &g, const Stencil<T> &S, const T *X, long ldx,
                          T *Y, long ldy, int s, cudaStream_t st);
int coarse_setup(hp_problem *P, hp::OpKind op);
// Gershgorin bound of the spectrum of diag^-1 S for a level stencil (host value, synchronises)
int gershgorin_bound(hp_problem *P, const GridDesc &g, const Stencil<double> &S, double *out);

// ---- vec.cu ---------------------------------------------------------------
void launch_copy(const double *X, long ldx, double *Y, long ldy, long n, int s, cudaStream_t st);
void launch_fill(double *X, long ldx, long n, int s, double v, cudaStream_t st);
void launch_axpby(double a, const double *X, long ldx, double b, double *Y, long ldy, long n, int s,
                  cudaStream_t st);   // Y = a X + b Y
void launch_ew_exp(const double *m, double *E, long n, cudaStream_t st);
// B0 = B (the `face` nodes at each end of a column zeroed), X = 0, bb[j] = |B0_j|^2 and,
// if rr_dev is non-null, rr[j] = bb[j]
int ir_start(hp_problem *P, const double *B, long ldb, double *B0, long ld0, double *X, long ldx, long n, int s,
             long face, double *bb_dev, double *rr_dev);
// per-column deterministic dots: out[j] = sum_i X_ij Y_ij (FP64)
int block_dot(hp_problem *P, const double *X, long ldx, const double *Y, long ldy, long n, int s,
              double *out_dev);

// ---- unet.cu / warm.cu -------------------------------------------------------
float *unet_input(hp_unet *U);          // (cap,3,H,W) input buffer of the network
const float *unet_output(const hp_unet *U);  // (cap,1,H,W) output of the last unet_run
int unet_cap(const hp_unet *U);
void unet_dims(const hp_unet *U, int *H, int *W);
void unet_run(hp_unet *U, int N, cudaStream_t st);  // forward of the first N inputs, enqueued on st
// Stiffness solves: X (n x s) = initial guesses for the Dirichlet-zeroed right-hand
// sides B when a network is attached and enabled; returns 1 if X was written, 0 if not.
int warm_guess(hp_problem *P, const double *B, long ldb, double *X, long ldx, int s);
// True when warm_guess would try a guess (a network attached and enabled, 2D).
bool warm_attached(const hp_problem *P);
bool warm_recording(const hp_problem *P);  // stiffness solves are being recorded as training samples
// Columns j with flag[j] != 0 restart from zero: X_j = 0, R_j = B_j.
void warm_fallback(hp_problem *P, const int *flag_host, int s, const double *B, long ldb, double *X, long ldx,
                   double *R, long ldr);
// Appends the finished solves (B_j, X_j) to the recorder, if one is set.
void warm_record(hp_problem *P, const double *B, long ldb, const double *X, long ldx, int s);

// ---- solver.cu --------------------------------------------------------------
int ensure_scalars(hp_problem *P, int s);
void drop_graphs(hp_problem *P);
void free_scalars_host(hp_problem *P);
int solve_block(hp_problem *P, OpKind op, const double *B, long ldb, double *X, long ldx, int s,
                double rtol, hp_solve_stats *st);
int apply_op64(hp_problem *P, OpKind op, const double *X, long ldx, double *Y, long ldy, int s);

// ---- dense.cu ---------------------------------------------------------------
// G (s1 x s2, column-major, ldg) = X^T Y ; X: n x s1, Y: n x s2 (FP64)
int gram(hp_problem *P, const double *X, long ldx, int s1, const double *Y, long ldy, int s2, double *G,
         int ldg, long n);
// Y (n x s2) = X (n x s1) * S (s1 x s2, ld lds) [+ beta * Y]
void launch_gemm_nn(const double *X, long ldx, int s1, const double *S, int lds, int s2, double *Y,
                    long ldy, long n, double alpha, double beta, hp_problem *P);
// in-place CGS2 orthonormalisation of the columns of Y (n x s)
int cgs2_qr(hp_problem *P, double *Y, long ldy, long n, int s);
int thin_qr(hp_problem *P, double *Y, long ldy, long n, int s);  // shifted Cholesky QR, cgs2_qr fallback
// upper Cholesky R^T R = G (s x s, ld s) in place; returns HP_ERR_NONFINITE if not SPD
int small_cholesky(hp_problem *P, double *G, int s);
// Y <- Y R^{-1}, R upper (s x s)
void launch_trsm_right_upper(double *Y, long ldy, long n, int s, const double *R, hp_problem *P);
// symmetric eigen-decomposition of T (s x s) by cyclic Jacobi: lambda (s), S (s x s) columns
int small_symeig(hp_problem *P, const double *T, int s, double *lambda, double *S);

}  // namespace hp
