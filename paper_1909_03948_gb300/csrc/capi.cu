// capi.cu -- the hp_* C ABI (include/hp.h): problem lifetime, forward /
// gradient / Gauss-Newton Hessian action, inexact Newton-CG (Algorithm 1),
// double-pass randomized eigensolver with PreCholQR (Algorithms 2, 4) and
// Laplace-approximation sampling (Section 4.3).  The host code here only
// orchestrates; every numerical step is one of this library's kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

namespace hp {

static thread_local std::string g_err;

int set_error(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int cuda_check(cudaError_t e, const char *where) {
  if (e == cudaSuccess) return 0;
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? HP_ERR_NOMEM : HP_ERR_CUDA;
}

static long padded(long n) { return (n + 63) / 64 * 64; }

__global__ void k_set_dirichlet(long face, long top_off, double *u, double u_bottom, double u_top) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < face; t += (long)gridDim.x * blockDim.x) {
    u[t] = u_bottom;
    u[top_off + t] = u_top;
  }
}

__global__ void k_sub_vec(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ c, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) c[i] = a[i] - b[i];
}

// Y[:, j] = X[:, j] + v
__global__ void k_add_vec_cols(const double *__restrict__ X, long ldx, const double *__restrict__ v,
                               double *__restrict__ Y, long ldy, long n) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    Y[ldy * j + i] = X[ldx * j + i] + v[i];
}

// z (k x s) *= S_i = 1 - 1/sqrt(1 + lambda_i)
__global__ void k_scale_rows_S(double *z, int k, int s, const double *__restrict__ lam) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * s) return;
  const int i = t % k;
  z[t] *= 1.0 - 1.0 / sqrt(1.0 + lam[i]);
}

__global__ void k_symmetrize(const double *__restrict__ T, double *__restrict__ Ts, int s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s * s) return;
  const int a = t % s, b = t / s;
  Ts[t] = 0.5 * (T[a + (long)s * b] + T[b + (long)s * a]);
}

// sign of each column: largest-magnitude entry (first on ties) made positive
__global__ void k_sign_normalise(double *V, long ldv, long n) {
  const int j = blockIdx.x;
  double *v = V + ldv * j;
  __shared__ double bv[NT];
  __shared__ long bi[NT];
  double best = -1.0;
  long besti = 0;
  for (long i = threadIdx.x; i < n; i += NT) {
    const double a = fabs(v[i]);
    if (a > best) {
      best = a;
      besti = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = bv[threadIdx.x + o];
      const long ia = bi[threadIdx.x + o];
      if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ia < bi[threadIdx.x])) {
        bv[threadIdx.x] = a;
        bi[threadIdx.x] = ia;
      }
    }
    __syncthreads();
  }
  const double sg = v[bi[0]] < 0.0 ? -1.0 : 1.0;
  __syncthreads();
  if (sg < 0.0)
    for (long i = threadIdx.x; i < n; i += NT) v[i] = -v[i];
}

static int sync(hp_problem *P) {
  HP_CUDA(cudaGetLastError());
  HP_CUDA(cudaStreamSynchronize(P->st));
  return 0;
}

static double *col64(DBuf &b, hp_problem *P, int s, int *rc) {
  *rc = b.ensure(sizeof(double) * padded(P->n) * std::max(s, 1));
  return b.as<double>();
}

// ---------------------------------------------------------------------------
// observation operator setup (host): containing simplex + barycentric weights
// ---------------------------------------------------------------------------
static int setup_observations(hp_problem *P, const double *xyz) {
  const int D = P->dim, nv = D + 1, N = P->N, np = N + 1;
  P->nobs = std::max(P->nobs, 0);
  const int q = P->nobs;
  std::vector<std::vector<int>> perms;
  {
    std::vector<int> a(D);
    std::iota(a.begin(), a.end(), 0);
    do perms.push_back(a);
    while (std::next_permutation(a.begin(), a.end()));
  }
  std::vector<int> node((size_t)q * nv);
  std::vector<double> w((size_t)q * nv);
  for (int o = 0; o < q; ++o) {
    int c[3] = {0, 0, 0};
    double loc[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
      const double x = xyz[(size_t)o * D + a];
      if (!(x >= -1e-12 && x <= 1.0 + 1e-12)) return set_error(HP_ERR_INVALID, "observation point outside the domain");
      const double t = std::min(std::max(x, 0.0), 1.0) * N;
      c[a] = std::min(std::max((int)std::floor(t), 0), N - 1);
      loc[a] = t - c[a];
    }
    std::vector<int> pi(D);
    std::iota(pi.begin(), pi.end(), 0);
    std::stable_sort(pi.begin(), pi.end(), [&](int a, int b) { return loc[a] > loc[b]; });
    int mask = 0;
    for (int k = 0; k <= D; ++k) {
      double lam;
      if (k == 0)
        lam = 1.0 - loc[pi[0]];
      else if (k == D)
        lam = loc[pi[D - 1]];
      else
        lam = loc[pi[k - 1]] - loc[pi[k]];
      if (k > 0) mask |= 1 << pi[k - 1];
      long idx = 0, stride = 1;
      for (int a = 0; a < D; ++a) {
        idx += (long)(c[a] + ((mask >> a) & 1)) * stride;
        stride *= np;
      }
      node[(size_t)o * nv + k] = (int)idx;
      w[(size_t)o * nv + k] = lam;
    }
  }
  // B^T as node-sorted CSR
  std::vector<int> row(P->n, -1), ptr, ent;
  {
    std::vector<std::pair<int, int>> pairs;
    pairs.reserve((size_t)q * nv);
    for (int e = 0; e < q * nv; ++e) pairs.push_back({node[e], e});
    std::sort(pairs.begin(), pairs.end());
    int cur = -1;
    for (auto &pr : pairs) {
      if (pr.first != cur) {
        cur = pr.first;
        row[cur] = (int)ptr.size();
        ptr.push_back((int)ent.size());
      }
      ent.push_back(pr.second);
    }
    ptr.push_back((int)ent.size());
  }
  P->bt_rows = (int)ptr.size() - 1;
  HP_CUDA(cudaMalloc(&P->obs_node, sizeof(int) * std::max<size_t>(1, node.size())));
  HP_CUDA(cudaMalloc(&P->obs_w, sizeof(double) * std::max<size_t>(1, w.size())));
  HP_CUDA(cudaMalloc(&P->bt_row, sizeof(int) * P->n));
  HP_CUDA(cudaMalloc(&P->bt_ptr, sizeof(int) * ptr.size()));
  HP_CUDA(cudaMalloc(&P->bt_ent, sizeof(int) * std::max<size_t>(1, ent.size())));
  if (q) {
    HP_CUDA(cudaMemcpy(P->obs_node, node.data(), sizeof(int) * node.size(), cudaMemcpyHostToDevice));
    HP_CUDA(cudaMemcpy(P->obs_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice));
    HP_CUDA(cudaMemcpy(P->bt_ent, ent.data(), sizeof(int) * ent.size(), cudaMemcpyHostToDevice));
  }
  HP_CUDA(cudaMemcpy(P->bt_row, row.data(), sizeof(int) * P->n, cudaMemcpyHostToDevice));
  HP_CUDA(cudaMemcpy(P->bt_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice));
  return 0;
}

// ---------------------------------------------------------------------------
// forward / cost
// ---------------------------------------------------------------------------
static int forward_state(hp_problem *P, hp_solve_stats *st) {
  int rc = 0;
  double *rhs = col64(P->t64a, P, 1, &rc);
  HP_TRY(rc);
  launch_axpby(1.0, P->lift, P->n, 0.0, rhs, P->n, P->n, 1, P->st);
  launch_axpby(1.0, P->f_load, P->n, 1.0, rhs, P->n, P->n, 1, P->st);
  HP_TRY(solve_block(P, OP_K, rhs, P->n, P->u, P->n, 1, P->rtol, st));
  const GridDesc &g = P->lv[0].g;
  const long face = P->dim == 2 ? g.np : (long)g.np * g.np;
  k_set_dirichlet<<<(int)std::min<long>(64, (face + 255) / 256), 256, 0, P->st>>>(face, g.n - face, P->u,
                                                                                  P->u_bottom, P->u_top);
  count_launch();
  launch_build_C(P);
  return 0;
}

// J = misfit + reg at the current point; also leaves R (m - m_pr) in Rdm if non-null
static int cost_at_point(hp_problem *P, double *J3, double *Rdm) {
  int rc = 0;
  const long n = P->n;
  HP_TRY(P->obsbuf.ensure(sizeof(double) * (2 * (size_t)std::max(P->nobs, 1) + 8)));
  double *yq = P->obsbuf.as<double>();
  double *scal = yq + 2 * std::max(P->nobs, 1);
  double misfit = 0.0;
  if (P->nobs > 0) {
    launch_obs_gather(P, P->u, n, yq, 1);
    k_sub_vec<<<1, 256, 0, P->st>>>(yq, P->d_obs, yq, P->nobs);
    count_launch();
    HP_TRY(block_dot(P, yq, P->nobs, yq, P->nobs, P->nobs, 1, scal));
  }
  double *dm = col64(P->t64b, P, 1, &rc);
  HP_TRY(rc);
  double *z = col64(P->t64c, P, 1, &rc);
  HP_TRY(rc);
  double *w = col64(P->vtmp[0], P, 1, &rc);
  HP_TRY(rc);
  k_sub_vec<<<blocks_for(n, 1), NT, 0, P->st>>>(P->m, P->m_prior, dm, n);
  count_launch();
  HP_TRY(apply_op64(P, OP_A, dm, n, z, n, 1));
  HP_TRY(solve_block(P, OP_M, z, n, w, n, 1, std::min(P->rtol, 1e-10), nullptr));
  HP_TRY(block_dot(P, z, n, w, n, n, 1, scal + 1));
  if (Rdm) HP_TRY(apply_op64(P, OP_A, w, n, Rdm, n, 1));
  double h[2] = {0, 0};
  HP_CUDA(cudaMemcpyAsync(h, scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, P->st));
  HP_TRY(sync(P));
  if (P->nobs > 0) misfit = 0.5 * h[0] / (P->sigma * P->sigma);
  const double reg = 0.5 * h[1];
  if (!std::isfinite(misfit) || !std::isfinite(reg)) return set_error(HP_ERR_NONFINITE, "non-finite cost");
  if (J3) {
    J3[0] = misfit + reg;
    J3[1] = misfit;
    J3[2] = reg;
  }
  return 0;
}

// flag = 1 if a and b differ anywhere (bitwise; the flag starts at 0)
__global__ void k_differs(const double *__restrict__ a, const double *__restrict__ b, long n, int *flag) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (__double_as_longlong(a[i]) != __double_as_longlong(b[i])) {
      *flag = 1;
      return;
    }
}

// true when m_dev is bitwise the current linearisation point and its state was solved to
// the current tolerance: everything set_point would build is still current
static bool is_current_point(hp_problem *P, const double *m_dev) {
  if (!P->have_point || P->u_rtol != P->rtol) return false;
  int *flag = P->sc.active.as<int>();
  if (!flag || cudaMemsetAsync(flag, 0, sizeof(int), P->st) != cudaSuccess) return false;
  k_differs<<<blocks_for(P->n, 1), NT, 0, P->st>>>(m_dev, P->m, P->n, flag);
  count_launch();
  int h = 1;
  if (cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, P->st) != cudaSuccess ||
      cudaStreamSynchronize(P->st) != cudaSuccess)
    return false;
  return h == 0;
}

static int set_point(hp_problem *P, const double *m_dev, double *J3, hp_solve_stats *st) {
  if (!is_current_point(P, m_dev)) {
    HP_TRY(build_point(P, m_dev));
    HP_TRY(forward_state(P, st));
    P->have_point = true;
    P->u_rtol = P->rtol;
  }
  if (J3) HP_TRY(cost_at_point(P, J3, nullptr));
  return sync(P);
}

// adjoint p at the current point into P->padj (one stiffness solve, kept until the point
// or the data change): K p = -B^T (B u - d) / sigma^2
static int adjoint_at_point(hp_problem *P) {
  if (P->have_p) return 0;
  int rc = 0;
  const long n = P->n;
  if (!P->padj && cudaMalloc(&P->padj, sizeof(double) * n) != cudaSuccess)
    return set_error(HP_ERR_NOMEM, "adjoint");
  double *rhs = col64(P->t64a, P, 1, &rc);
  HP_TRY(rc);
  HP_TRY(P->obsbuf.ensure(sizeof(double) * (2 * (size_t)std::max(P->nobs, 1) + 8)));
  double *yq = P->obsbuf.as<double>();
  if (P->nobs > 0) {
    launch_obs_gather(P, P->u, n, yq, 1);
    k_sub_vec<<<1, 256, 0, P->st>>>(yq, P->d_obs, yq, P->nobs);
    count_launch();
  }
  launch_obs_scatter(P, yq, rhs, n, 1, -1.0 / (P->sigma * P->sigma));
  HP_TRY(solve_block(P, OP_K, rhs, n, P->padj, n, 1, P->rtol, nullptr));
  P->have_p = true;
  return 0;
}

// the adjoint terms of the full Hessian at the current point: C(p) and C(u)^T p
static int full_terms_at_point(hp_problem *P) {
  if (P->have_full) return 0;
  HP_TRY(adjoint_at_point(P));
  const long n = P->n;
  const int nC = (1 << (P->dim + 1)) - 1;
  if (!P->Cbeta_p && cudaMalloc(&P->Cbeta_p, sizeof(double) * n * nC) != cudaSuccess)
    return set_error(HP_ERR_NOMEM, "full Hessian terms");
  if (!P->CbetaE_p && cudaMalloc(&P->CbetaE_p, sizeof(double) * n * nC) != cudaSuccess)
    return set_error(HP_ERR_NOMEM, "full Hessian terms");
  if (!P->wmm && cudaMalloc(&P->wmm, sizeof(double) * n) != cudaSuccess)
    return set_error(HP_ERR_NOMEM, "full Hessian terms");
  launch_build_C_from(P, P->padj, P->Cbeta_p, P->CbetaE_p);
  launch_Ct_apply(P, P->padj, n, P->wmm, n, 1, 1.0, 0.0);
  P->have_full = true;
  return 0;
}

__global__ void k_add_diag_cols(const double *__restrict__ w, const double *__restrict__ X, long ldx,
                                double *__restrict__ Y, long ldy, long n) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    Y[ldy * j + i] += w[i] * X[ldx * j + i];
}

// g = R (m - m_pr) + C^T p at the current point
static int gradient_at_point(hp_problem *P, double *g, double *J3) {
  int rc = 0;
  const long n = P->n;
  double *Rdm = col64(P->vtmp[2], P, 1, &rc);
  HP_TRY(rc);
  HP_TRY(adjoint_at_point(P));
  double J3l[3];
  HP_TRY(cost_at_point(P, J3 ? J3 : J3l, Rdm));
  launch_Ct_apply(P, P->padj, n, g, n, 1, 1.0, 0.0);
  launch_axpby(1.0, Rdm, n, 1.0, g, n, n, 1, P->st);
  return sync(P);
}

static int hessian_block(hp_problem *P, const double *X, long ldx, double *Y, long ldy, int s, int flags,
                         hp_solve_stats *st) {
  if (!P->have_point) return set_error(HP_ERR_STATE, "hp_set_point must be called first");
  int rc = 0;
  const long n = P->n, ld = padded(n);
  double *t1 = col64(P->t64a, P, s, &rc);
  HP_TRY(rc);
  double *t2 = col64(P->t64b, P, s, &rc);
  HP_TRY(rc);
  HP_TRY(P->obsbuf.ensure(sizeof(double) * ((size_t)std::max(P->nobs, 1) * s + 8)));
  double *yq = P->obsbuf.as<double>();
  const bool full = (flags & HP_FULL_NEWTON) != 0;
  double *uh = nullptr;
  if (full) {
    HP_TRY(full_terms_at_point(P));
    uh = col64(P->t64c, P, s, &rc);
    HP_TRY(rc);
  }
  // incremental forward (eq. incrementals1): K Uh = -C X
  launch_C_apply(P, X, ldx, t1, ld, s, -1.0);
  HP_TRY(solve_block(P, OP_K, t1, ld, t2, ld, s, P->rtol, st));
  // incremental adjoint (eq. incrementals2): K Ph = -B^T B Uh / sigma^2 [- C(p) X]
  launch_obs_gather(P, t2, ld, yq, s);
  launch_obs_scatter(P, yq, t1, ld, s, -1.0 / (P->sigma * P->sigma));
  if (full) {
    launch_copy(t2, ld, uh, ld, n, s, P->st);
    launch_C_apply_beta(P, P->CbetaE_p, X, ldx, t1, ld, s, -1.0, 1.0);
  }
  HP_TRY(solve_block(P, OP_K, t1, ld, t2, ld, s, P->rtol, st));
  // eq. incrementals3: Y = C^T Ph [+ C(p)^T Uh + X (.) C^T p]
  launch_Ct_apply(P, t2, ld, Y, ldy, s, 1.0, 0.0);
  if (full) {
    launch_Ct_apply_beta(P, P->Cbeta_p, uh, ld, Y, ldy, s, 1.0, 1.0);
    k_add_diag_cols<<<dim3(blocks_for(n, s), s), NT, 0, P->st>>>(P->wmm, X, ldx, Y, ldy, n);
    count_launch();
  }
  if (flags & HP_WITH_PRIOR) {
    double *t3 = col64(P->t64c, P, s, &rc);
    HP_TRY(rc);
    HP_TRY(apply_op64(P, OP_A, X, ldx, t1, ld, s));
    HP_TRY(solve_block(P, OP_M, t1, ld, t2, ld, s, std::min(P->rtol, 1e-10), st));
    HP_TRY(apply_op64(P, OP_A, t2, ld, t3, ld, s));
    launch_axpby(1.0, t3, ld, 1.0, Y, ldy, n, s, P->st);
  }
  return sync(P);
}

static int R_apply(hp_problem *P, const double *X, long ldx, double *Y, long ldy, int s) {
  int rc = 0;
  const long ld = padded(P->n);
  double *t1 = col64(P->t64a, P, s, &rc);
  HP_TRY(rc);
  double *t2 = col64(P->t64b, P, s, &rc);
  HP_TRY(rc);
  HP_TRY(apply_op64(P, OP_A, X, ldx, t1, ld, s));
  HP_TRY(solve_block(P, OP_M, t1, ld, t2, ld, s, std::min(P->rtol, 1e-10), nullptr));
  HP_TRY(apply_op64(P, OP_A, t2, ld, Y, ldy, s));
  return 0;
}

static int Rinv_apply(hp_problem *P, const double *X, long ldx, double *Y, long ldy, int s, double tol = 0.0) {
  int rc = 0;
  const long ld = padded(P->n);
  const double rt = tol > 0.0 ? tol : P->rtol;
  double *t1 = col64(P->t64a, P, s, &rc);
  HP_TRY(rc);
  double *t2 = col64(P->t64b, P, s, &rc);
  HP_TRY(rc);
  HP_TRY(solve_block(P, OP_A, X, ldx, t1, ld, s, rt, nullptr));
  HP_TRY(apply_op64(P, OP_M, t1, ld, t2, ld, s));
  HP_TRY(solve_block(P, OP_A, t2, ld, Y, ldy, s, rt, nullptr));
  return 0;
}

// t_i *= lambda_i / (1 + lambda_i)
__global__ void k_lowrank_scale(double *t, const double *__restrict__ lam, int k) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) t[i] *= lam[i] / (1.0 + lam[i]);
}

static int dot1(hp_problem *P, const double *a, const double *b, double *out) {
  HP_TRY(P->small.ensure(sizeof(double) * 64));
  double *d = P->small.as<double>();
  HP_TRY(block_dot(P, a, P->n, b, P->n, P->n, 1, d));
  HP_CUDA(cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, P->st));
  return sync(P);
}

}  // namespace hp

using namespace hp;

// ===========================================================================
// ABI
// ===========================================================================
extern "C" {

const char *hp_status_string(int s) {
  switch (s) {
    case HP_OK: return "ok";
    case HP_ERR_INVALID: return "invalid argument";
    case HP_ERR_NOT_CONVERGED: return "not converged";
    case HP_ERR_NONFINITE: return "non-finite value";
    case HP_ERR_CUDA: return "CUDA error";
    case HP_ERR_NOMEM: return "out of device memory";
    case HP_ERR_STATE: return "no linearisation point (call hp_set_point)";
    default: return "unknown status";
  }
}

const char *hp_last_error(void) { return g_err.c_str(); }
unsigned long long hp_kernel_launches(void) { return g_launches.load(); }
unsigned long long hp_tiled_kernel_launches(void) { return g_tiled_launches.load(); }
int hp_algorithmic_bytes(double *out, int nfam) {
  if (!out || nfam < 0) return set_error(HP_ERR_INVALID, "hp_algorithmic_bytes: bad arguments");
  for (int f = 0; f < nfam; ++f) out[f] = f < BYTES_FAMILIES ? (double)g_alg_bytes[f].load() : 0.0;
  return HP_OK;
}

int hp_problem_create(const hp_problem_desc *d, hp_problem **out) {
  if (!d || !out) return set_error(HP_ERR_INVALID, "null argument");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return set_error(HP_ERR_INVALID, "dim must be 2 or 3");
  if (d->N < 1 || d->N > 8192) return set_error(HP_ERR_INVALID, "N out of range");
  if (!(d->gamma > 0) || !(d->delta > 0)) return set_error(HP_ERR_INVALID, "gamma and delta must be > 0");
  if (!(d->sigma > 0)) return set_error(HP_ERR_INVALID, "sigma must be > 0");
  if (d->nobs < 0 || (d->nobs > 0 && !d->obs_xyz)) return set_error(HP_ERR_INVALID, "bad observations");
  if (d->precision != HP_FP64_PLAIN && d->precision != HP_FP32_IR) return set_error(HP_ERR_INVALID, "bad precision");
  hp_problem *P = new hp_problem();
  P->dim = d->dim;
  P->N = d->N;
  P->n = 1;
  for (int a = 0; a < d->dim; ++a) P->n *= (d->N + 1);
  P->nelems = (d->dim == 2 ? 2 : 6);
  for (int a = 0; a < d->dim; ++a) P->nelems *= d->N;
  P->gamma = d->gamma;
  P->delta = d->delta;
  P->sigma = d->sigma;
  P->u_top = d->u_top;
  P->u_bottom = d->u_bottom;
  P->precision = d->precision;
  P->rtol = d->rtol > 0 ? d->rtol : 1e-8;
  P->max_iter = d->max_iter > 0 ? d->max_iter : 500;
  P->nobs = d->nobs;
  {
    bool zero = true;
    for (int q = 0; q < 6; ++q) zero = zero && d->theta[q] == 0.0;
    if (!zero) {
      const double *t = d->theta;
      const double m1 = t[0], m2 = t[0] * t[1] - t[3] * t[3];
      const double m3 = d->dim == 3 ? t[0] * (t[1] * t[2] - t[5] * t[5]) - t[3] * (t[3] * t[2] - t[5] * t[4]) +
                                          t[4] * (t[3] * t[5] - t[1] * t[4])
                                    : 1.0;
      if (!(m1 > 0 && m2 > 0 && m3 > 0)) {
        delete P;
        return set_error(HP_ERR_INVALID, "theta must be symmetric positive definite");
      }
      for (int q = 0; q < 6; ++q) P->theta[q] = t[q];
      if (d->dim == 2) P->theta[2] = 1.0, P->theta[4] = P->theta[5] = 0.0;
    }
    if (!(d->robin_beta >= 0.0)) {
      delete P;
      return set_error(HP_ERR_INVALID, "robin_beta must be >= 0");
    }
    P->robin_beta = d->robin_beta;
  }
  if (const char *e = getenv("HP_GRAPHS")) P->use_graphs = !(e[0] == '0');
  int rc = 0;
  auto fail = [&](int code) {
    hp_problem_destroy(P);
    return code;
  };
  if ((rc = ensure_scalars(P, 1))) return fail(rc);
  if ((rc = build_hierarchy_geometry(P))) return fail(rc);
  const size_t nb = sizeof(double) * P->n;
  for (double **pp : {&P->m, &P->E, &P->u, &P->lift, &P->m_prior, &P->f_load}) {
    if (cudaMalloc(pp, nb) != cudaSuccess) return fail(set_error(HP_ERR_NOMEM, "allocation"));
  }
  const int nC = (1 << (P->dim + 1)) - 1;
  if (cudaMalloc(&P->Cbeta, sizeof(double) * P->n * nC) != cudaSuccess ||
      cudaMalloc(&P->CbetaE, sizeof(double) * P->n * nC) != cudaSuccess)
    return fail(set_error(HP_ERR_NOMEM, "allocation"));
  if (cudaMalloc(&P->d_obs, sizeof(double) * std::max(1, P->nobs)) != cudaSuccess)
    return fail(set_error(HP_ERR_NOMEM, "allocation"));
  cudaMemset(P->d_obs, 0, sizeof(double) * std::max(1, P->nobs));
  if (d->d_obs && P->nobs)
    cudaMemcpy(P->d_obs, d->d_obs, sizeof(double) * P->nobs, cudaMemcpyHostToDevice);
  cudaMemset(P->m_prior, 0, nb);
  if (d->m_prior) cudaMemcpy(P->m_prior, d->m_prior, nb, cudaMemcpyHostToDevice);
  cudaMemset(P->f_load, 0, nb);
  if (d->f) {
    int r2 = 0;
    double *tmp = col64(P->t64a, P, 1, &r2);
    if (r2) return fail(r2);
    cudaMemcpy(tmp, d->f, nb, cudaMemcpyHostToDevice);
    if ((rc = apply_op64(P, OP_M, tmp, P->n, P->f_load, P->n, 1))) return fail(rc);
  }
  if ((rc = setup_observations(P, d->obs_xyz))) return fail(rc);
  if ((rc = cuda_check(cudaDeviceSynchronize(), "create"))) return fail(rc);
  *out = P;
  return HP_OK;
}

void hp_problem_destroy(hp_problem *P) {
  if (!P) return;
  cudaDeviceSynchronize();
  for (int l = 0; l < HP_MAXL; ++l) {
    Level &lv = P->lv[l];
    for (void *p : {(void *)lv.kappa, (void *)lv.K64.diag, (void *)lv.K64.invdiag, (void *)lv.K64.c,
                    (void *)lv.K32.diag, (void *)lv.K32.invdiag, (void *)lv.K32.c, (void *)lv.K32.pk, (void *)lv.A64.diag,
                    (void *)lv.A64.invdiag, (void *)lv.A64.c, (void *)lv.A32.diag, (void *)lv.A32.invdiag,
                    (void *)lv.A32.c, (void *)lv.K64.cpr, (void *)lv.A64.cpr})
      if (p) cudaFree(p);
  }
  for (CoarseInv *C : {&P->cK, &P->cA})
    for (void *p : {(void *)C->dense, (void *)C->inv64, (void *)C->inv32})
      if (p) cudaFree(p);
  for (void *p : {(void *)P->CbetaE_pr, (void *)P->Cbeta_pr, (void *)P->E_pr})
    if (p) cudaFree(p);
  P->xpairs.release();
  P->dense_tmp.release();
  for (void *p : {(void *)P->M64.diag, (void *)P->M64.invdiag, (void *)P->M64.c, (void *)P->M64.cpr, (void *)P->M32.diag,
                  (void *)P->M32.invdiag, (void *)P->M32.c, (void *)P->m, (void *)P->E, (void *)P->u,
                  (void *)P->lift, (void *)P->Cbeta, (void *)P->CbetaE, (void *)P->padj, (void *)P->Cbeta_p, (void *)P->CbetaE_p, (void *)P->wmm, (void *)P->m_prior, (void *)P->f_load, (void *)P->d_obs, (void *)P->obs_node,
                  (void *)P->obs_w, (void *)P->bt_row, (void *)P->bt_ptr, (void *)P->bt_ent})
    if (p) cudaFree(p);
  for (BlockWS<float> *W = &P->w32; W; W = nullptr) {
    for (DBuf *b : {&W->x, &W->r, &W->z, &W->p, &W->q}) b->release();
    for (int l = 0; l < HP_MAXL; ++l) {
      W->lr[l].release();
      W->la[l].release();
      W->lb[l].release();
    }
  }
  {
    BlockWS<double> *W = &P->w64;
    for (DBuf *b : {&W->x, &W->r, &W->z, &W->p, &W->q}) b->release();
    for (int l = 0; l < HP_MAXL; ++l) {
      W->lr[l].release();
      W->la[l].release();
      W->lb[l].release();
    }
  }
  drop_graphs(P);
  if (P->cap) cudaStreamDestroy(P->cap);
  free_scalars_host(P);
  ScalarWS &S = P->sc;
  for (DBuf *b : {&S.iter, &S.rz, &S.pq, &S.rr, &S.bb, &S.alpha, &S.beta, &S.scale, &S.iscale, &S.tol2col, &S.bbr, &S.tmp, &S.active, &S.partial, &S.counter})
    b->release();
  for (DBuf *b : {&P->r64, &P->b64, &P->x64, &P->rctl, &P->t64a, &P->t64b, &P->t64c, &P->obsbuf, &P->small,
                  &P->etabuf, &P->ws_flag, &P->ws_bb, &P->ws_z})
    b->release();
  if (P->h_rctl) cudaFreeHost(P->h_rctl);
  for (int i = 0; i < 6; ++i) P->vtmp[i].release();
  for (cudaEvent_t e : P->prof_ev) cudaEventDestroy(e);
  delete P;
}

int hp_set_stream(hp_problem *P, void *stream) {
  if (!P) return set_error(HP_ERR_INVALID, "null problem");
  P->st = static_cast<cudaStream_t>(stream);
  return HP_OK;
}

int hp_set_precision(hp_problem *P, int precision) {
  if (!P || (precision != HP_FP64_PLAIN && precision != HP_FP32_IR)) return set_error(HP_ERR_INVALID, "precision");
  const bool changed = precision != P->precision;
  P->precision = precision;
  if (changed) {  // the coarse inverses are factored in the precision of the inner solves
    HP_TRY(coarse_setup(P, OP_A));
    if (P->have_point) HP_TRY(coarse_setup(P, OP_K));
  }
  return HP_OK;
}

int hp_set_tolerance(hp_problem *P, double rtol, int max_iter) {
  if (!P || !(rtol > 0) || rtol >= 1 || max_iter < 1) return set_error(HP_ERR_INVALID, "tolerance");
  P->rtol = rtol;
  P->max_iter = max_iter;
  return HP_OK;
}

int hp_set_data(hp_problem *P, const double *d_obs_host, double sigma) {
  if (!P || !(sigma > 0)) return set_error(HP_ERR_INVALID, "sigma");
  P->sigma = sigma;
  if (d_obs_host && P->nobs) HP_CUDA(cudaMemcpy(P->d_obs, d_obs_host, sizeof(double) * P->nobs, cudaMemcpyHostToDevice));
  P->have_p = P->have_full = false;  // the adjoint depends on the data
  return HP_OK;
}

int hp_get_data(const hp_problem *P, double *d_out_host) {
  if (!P || !d_out_host) return set_error(HP_ERR_INVALID, "null");
  if (P->nobs) HP_CUDA(cudaMemcpy(d_out_host, P->d_obs, sizeof(double) * P->nobs, cudaMemcpyDeviceToHost));
  return HP_OK;
}

int hp_profile_enable(hp_problem *P, int on) {
  if (!P) return set_error(HP_ERR_INVALID, "null problem");
  HP_CUDA(cudaStreamSynchronize(P->st));
  P->prof_on = on != 0;
  P->prof_used = 0;
  P->prof_failed = false;
  for (int i = 0; i < 16; ++i) {
    P->prof_cnt[i] = 0;
    P->prof_ms[i] = 0.0;
  }
  return HP_OK;
}

int hp_profile_read(hp_problem *P, int nids, int *counts, double *total_ms) {
  if (!P || nids < 0 || nids > 16 || (nids > 0 && (!counts || !total_ms)))
    return set_error(HP_ERR_INVALID, "arguments");
  HP_CUDA(cudaStreamSynchronize(P->st));
  prof_harvest(P, 0, P->prof_used, false);
  for (int i = 0; i < nids; ++i) {
    counts[i] = (int)P->prof_cnt[i];
    total_ms[i] = P->prof_ms[i];
    P->prof_cnt[i] = 0;
    P->prof_ms[i] = 0.0;
  }
  P->prof_used = 0;
  return HP_OK;
}

int hp_num_nodes(const hp_problem *P) { return P ? (int)P->n : 0; }
int hp_num_elements(const hp_problem *P) { return P ? (int)P->nelems : 0; }

int hp_set_point(hp_problem *P, const double *m_dev, double *J_out) {
  if (!P || !m_dev) return set_error(HP_ERR_INVALID, "null");
  return set_point(P, m_dev, J_out, nullptr);
}

int hp_forward(hp_problem *P, const double *m_dev, double *u_dev, hp_solve_stats *st) {
  if (!P || !m_dev) return set_error(HP_ERR_INVALID, "null");
  if (st) *st = hp_solve_stats{};
  HP_TRY(build_point(P, m_dev));
  HP_TRY(forward_state(P, st));
  P->have_point = true;
  P->u_rtol = P->rtol;
  if (u_dev) HP_CUDA(cudaMemcpyAsync(u_dev, P->u, sizeof(double) * P->n, cudaMemcpyDeviceToDevice, P->st));
  return sync(P);
}

int hp_observe(hp_problem *P, const double *u_dev, double *y_dev) {
  if (!P || !u_dev || !y_dev) return set_error(HP_ERR_INVALID, "null");
  launch_obs_gather(P, u_dev, P->n, y_dev, 1);
  return sync(P);
}

int hp_gradient(hp_problem *P, const double *m_dev, double *g_dev, double *J_out) {
  if (!P || !m_dev || !g_dev) return set_error(HP_ERR_INVALID, "null");
  HP_TRY(set_point(P, m_dev, nullptr, nullptr));
  return gradient_at_point(P, g_dev, J_out);
}

int hp_hessian_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs, int flags,
                     hp_solve_stats *st) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !X || !Y || nrhs < 0 || ldx < P->n || ldy < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (st) *st = hp_solve_stats{};
  if (nrhs == 0) return HP_OK;
  return hessian_block(P, X, ldx, Y, ldy, nrhs, flags, st);
}

int hp_stiffness_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !X || !Y || nrhs < 0 || ldx < P->n || ldy < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (!P->have_point) return set_error(HP_ERR_STATE, "hp_set_point must be called first");
  if (nrhs == 0) return HP_OK;
  HP_TRY(apply_op64(P, OP_K, X, ldx, Y, ldy, nrhs));
  return sync(P);
}

int hp_state_solve(hp_problem *P, const double *B, int ldb, double *X, int ldx, int nrhs, hp_solve_stats *st) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !B || !X || nrhs < 0 || ldb < P->n || ldx < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (!P->have_point) return set_error(HP_ERR_STATE, "hp_set_point must be called first");
  if (st) *st = hp_solve_stats{};
  if (nrhs == 0) return HP_OK;
  HP_TRY(solve_block(P, OP_K, B, ldb, X, ldx, nrhs, P->rtol, st));
  return sync(P);
}

int hp_C_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !X || !Y || nrhs < 0 || ldx < P->n || ldy < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (!P->have_point) return set_error(HP_ERR_STATE, "hp_set_point must be called first");
  if (nrhs == 0) return HP_OK;
  launch_C_apply(P, X, ldx, Y, ldy, nrhs, 1.0);
  return sync(P);
}

int hp_Ct_apply(hp_problem *P, const double *W, int ldw, double *Y, int ldy, int nrhs) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !W || !Y || nrhs < 0 || ldw < P->n || ldy < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (!P->have_point) return set_error(HP_ERR_STATE, "hp_set_point must be called first");
  if (nrhs == 0) return HP_OK;
  launch_Ct_apply(P, W, ldw, Y, ldy, nrhs, 1.0, 0.0);
  return sync(P);
}

int hp_prior_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !X || !Y || nrhs < 0 || ldx < P->n || ldy < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (nrhs == 0) return HP_OK;
  HP_TRY(apply_op64(P, OP_A, X, ldx, Y, ldy, nrhs));
  return sync(P);
}

int hp_mass_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !X || !Y || nrhs < 0 || ldx < P->n || ldy < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (nrhs == 0) return HP_OK;
  HP_TRY(apply_op64(P, OP_M, X, ldx, Y, ldy, nrhs));
  return sync(P);
}

int hp_prior_solve(hp_problem *P, const double *B, int ldb, double *X, int ldx, int nrhs, hp_solve_stats *st) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !B || !X || nrhs < 0 || ldb < P->n || ldx < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (st) *st = hp_solve_stats{};
  if (nrhs == 0) return HP_OK;
  HP_TRY(solve_block(P, OP_A, B, ldb, X, ldx, nrhs, P->rtol, st));
  return sync(P);
}

int hp_mass_solve(hp_problem *P, const double *B, int ldb, double *X, int ldx, int nrhs, hp_solve_stats *st) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !B || !X || nrhs < 0 || ldb < P->n || ldx < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (st) *st = hp_solve_stats{};
  if (nrhs == 0) return HP_OK;
  HP_TRY(solve_block(P, OP_M, B, ldb, X, ldx, nrhs, std::min(P->rtol, 1e-10), st));
  return sync(P);
}

int hp_R_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !X || !Y || nrhs < 0 || ldx < P->n || ldy < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (nrhs == 0) return HP_OK;
  HP_TRY(R_apply(P, X, ldx, Y, ldy, nrhs));
  return sync(P);
}

int hp_Rinv_apply(hp_problem *P, const double *X, int ldx, double *Y, int ldy, int nrhs) {
  if (P && nrhs == 0) return HP_OK;
  if (!P || !X || !Y || nrhs < 0 || ldx < P->n || ldy < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (nrhs == 0) return HP_OK;
  HP_TRY(Rinv_apply(P, X, ldx, Y, ldy, nrhs));
  return sync(P);
}

int hp_mass_factor_apply(hp_problem *P, const double *eta, int ldeta, double *W, int ldw, int nsamples) {
  if (P && nsamples == 0) return HP_OK;
  if (!P || !eta || !W || nsamples < 0 || ldeta < P->nelems * (P->dim + 1) || ldw < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  if (nsamples == 0) return HP_OK;
  launch_mass_factor(P, eta, ldeta, W, ldw, nsamples);
  return sync(P);
}

// ---------------------------------------------------------------------------
// Algorithm 1: inexact Newton-CG
// ---------------------------------------------------------------------------
int hp_newton_cg_map(hp_problem *P, double *m, const hp_newton_opts *opts_in, hp_newton_stats *out) {
  if (!P || !m) return set_error(HP_ERR_INVALID, "null");
  hp_newton_opts o{1e-6, 0.0, 50, 10, 1e-4, 200, 0, 0, 10, 0, 0.0};
  if (opts_in) o = *opts_in;
  if (!(o.prec_rtol >= 0.0 && o.prec_rtol < 1.0)) return set_error(HP_ERR_INVALID, "prec_rtol in [0, 1)");
  const int lk = std::max(0, o.lowrank_k), lp = std::max(0, o.lowrank_p), ls = lk + lp;
  if (lk > 0 && (ls > P->n || ls > 1024)) return set_error(HP_ERR_INVALID, "lowrank_k + lowrank_p too large");
  hp_newton_stats S{};
  const long n = P->n;
  std::vector<double *> v(8, nullptr);
  for (auto &p : v)
    if (cudaMalloc(&p, sizeof(double) * n) != cudaSuccess) {
      for (auto q : v)
        if (q) cudaFree(q);
      return set_error(HP_ERR_NOMEM, "newton workspace");
    }
  // low-rank preconditioner: V (n x k), lambda (k), Omega (n x (k+p)), scratch (k)
  double *Vl = nullptr, *laml = nullptr, *Oml = nullptr, *tk = nullptr;
  auto free_lr = [&]() {
    for (double *q : {Vl, laml, Oml, tk})
      if (q) cudaFree(q);
  };
  if (lk > 0 && (cudaMalloc(&Vl, sizeof(double) * n * lk) != cudaSuccess ||
                 cudaMalloc(&laml, sizeof(double) * lk) != cudaSuccess ||
                 cudaMalloc(&Oml, sizeof(double) * n * ls) != cudaSuccess ||
                 cudaMalloc(&tk, sizeof(double) * lk) != cudaSuccess)) {
    free_lr();
    for (auto q : v) cudaFree(q);
    return set_error(HP_ERR_NOMEM, "newton low-rank workspace");
  }
  double *g = v[0], *x = v[1], *r = v[2], *z = v[3], *d = v[4], *Hd = v[5], *mt = v[6];
  auto cleanup = [&](int rc) {
    for (auto q : v) cudaFree(q);
    free_lr();
    if (out) *out = S;
    return rc;
  };
  bool have_lr = false;
  // z -= V diag(lambda / (1 + lambda)) V^T r   (after z = R^-1 r)
  auto lowrank_correct = [&](const double *rv, double *zv) -> int {
    if (!have_lr) return 0;
    HP_TRY(gram(P, Vl, n, lk, rv, n, 1, tk, lk, n));
    k_lowrank_scale<<<1, 256, 0, P->st>>>(tk, laml, lk);
    count_launch();
    launch_gemm_nn(Vl, n, lk, tk, lk, 1, zv, n, n, -1.0, 1.0, P);
    return 0;
  };
  int rc = 0;
  double J3[3];
  if ((rc = set_point(P, m, J3, nullptr))) return cleanup(rc);
  double J = J3[0];
  S.J0 = J;
  double g0 = -1.0, gn = 0.0;
  int solves = 1;
  for (int it = 0; it < o.max_iter; ++it) {
    if ((rc = gradient_at_point(P, g, nullptr))) return cleanup(rc);
    solves += 2;
    if ((rc = Rinv_apply(P, g, n, z, n, 1))) return cleanup(rc);
    solves += 2;
    double gRg = 0.0;
    if ((rc = dot1(P, g, z, &gRg))) return cleanup(rc);
    gn = std::sqrt(std::max(gRg, 0.0));
    if (!std::isfinite(gn)) return cleanup(set_error(HP_ERR_NONFINITE, "non-finite gradient"));
    if (g0 < 0) {
      g0 = gn;
      S.gnorm0 = g0;
    }
    S.gnorm = gn;
    if (gn <= std::max(o.rel_tol * g0, o.abs_tol)) {
      S.converged = 1;
      break;
    }
    const double eta = std::min(0.5, std::sqrt(gn / g0));
    if (lk > 0 && (!have_lr || (o.lowrank_refresh > 0 && it % o.lowrank_refresh == 0))) {
      // leading eigenpairs of the prior-preconditioned misfit Hessian at the current point
      launch_philox_normals(0x6c72ULL + (unsigned long long)it, 0, ls, (int)n, Oml, n, 0, P->st);
      hp_solve_stats es{};
      if ((rc = hp_lowrank_eig(P, m, lk, lp, Oml, (int)n, laml, Vl, (int)n, 0, &es))) return cleanup(rc);
      solves += es.solves;
      S.eig_solves += 1;
      have_lr = true;
    }
    // CG-Steihaug on H x = -g, preconditioner R^{-1} [- V D V^T]: r0 = -g, z0 = preconditioned r0
    launch_fill(x, n, n, 1, 0.0, P->st);
    launch_axpby(-1.0, g, n, 0.0, r, n, n, 1, P->st);
    launch_axpby(-1.0, z, n, 0.0, z, n, n, 1, P->st);
    if ((rc = lowrank_correct(r, z))) return cleanup(rc);
    double rz = gRg;
    if (have_lr && (rc = dot1(P, r, z, &rz))) return cleanup(rc);
    const double r0 = std::sqrt(rz);
    launch_axpby(1.0, z, n, 0.0, d, n, n, 1, P->st);
    int k = 0;
    for (k = 1; k <= o.cg_max_iter; ++k) {
      hp_solve_stats hs{};
      if ((rc = hessian_block(P, d, n, Hd, n, 1, HP_WITH_PRIOR | (o.full_newton ? HP_FULL_NEWTON : 0), &hs)))
        return cleanup(rc);
      solves += hs.solves;
      double dHd = 0.0;
      if ((rc = dot1(P, d, Hd, &dHd))) return cleanup(rc);
      if (dHd <= 0.0) {
        if (k == 1) launch_axpby(1.0, z, n, 0.0, x, n, n, 1, P->st);
        break;
      }
      const double alpha = rz / dHd;
      launch_axpby(alpha, d, n, 1.0, x, n, n, 1, P->st);
      launch_axpby(-alpha, Hd, n, 1.0, r, n, n, 1, P->st);
      if ((rc = Rinv_apply(P, r, n, z, n, 1, o.prec_rtol))) return cleanup(rc);
      solves += 2;
      if ((rc = lowrank_correct(r, z))) return cleanup(rc);
      double rzn = 0.0;
      if ((rc = dot1(P, r, z, &rzn))) return cleanup(rc);
      if (std::sqrt(std::max(rzn, 0.0)) <= eta * r0) break;
      const double beta = rzn / rz;
      launch_axpby(1.0, z, n, beta, d, n, n, 1, P->st);
      rz = rzn;
    }
    S.cg_iterations += std::min(k, o.cg_max_iter);
    double gdm = 0.0;
    if ((rc = dot1(P, g, x, &gdm))) return cleanup(rc);
    // Armijo backtracking
    double alpha = 1.0;
    bool accepted = false;
    for (int j = 0; j < o.max_backtrack; ++j) {
      launch_copy(m, n, mt, n, n, 1, P->st);
      launch_axpby(alpha, x, n, 1.0, mt, n, n, 1, P->st);
      if ((rc = set_point(P, mt, J3, nullptr))) return cleanup(rc);
      solves += 2;
      if (J3[0] < J + alpha * o.c_armijo * gdm) {
        launch_copy(mt, n, m, n, n, 1, P->st);
        J = J3[0];
        accepted = true;
        break;
      }
      alpha *= 0.5;
    }
    S.iterations = it + 1;
    if (!accepted) {
      if ((rc = set_point(P, m, nullptr, nullptr))) return cleanup(rc);
      break;
    }
  }
  S.J = J;
  S.pde_solves = solves;
  if ((rc = sync(P))) return cleanup(rc);
  return cleanup(S.converged ? HP_OK : set_error(HP_ERR_NOT_CONVERGED, "Newton-CG did not converge"));
}

// ---------------------------------------------------------------------------
// Algorithms 2 and 4: double-pass randomized generalized eigensolver
// ---------------------------------------------------------------------------
}  // extern "C"

namespace hp {

// C (s x s) = op(A) op(B) for s x s column-major matrices (ta, tb: transpose flags)
__global__ void k_small_gemm(int s, int ta, int tb, const double *__restrict__ A, const double *__restrict__ B,
                             double *__restrict__ C) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s * s) return;
  const int i = t % s, j = t / s;
  double acc = 0.0;
  for (int k = 0; k < s; ++k) {
    const double a = ta ? A[k + (long)s * i] : A[i + (long)s * k];
    const double b = tb ? B[j + (long)s * k] : B[k + (long)s * j];
    acc += a * b;
  }
  C[t] = acc;
}

static void small_gemm(hp_problem *P, int s, int ta, int tb, const double *A, const double *B, double *C) {
  k_small_gemm<<<(s * s + 255) / 256, 256, 0, P->st>>>(s, ta, tb, A, B, C);
  count_launch();
}

// C = E + E^T
__global__ void k_sym_sum(const double *__restrict__ E, double *__restrict__ C, int s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s * s) return;
  const int i = t % s, j = t / s;
  C[t] = E[i + (long)s * j] + E[j + (long)s * i];
}

// Lyapunov solve in the eigenbasis of M: Ct_ij /= (d_i + d_j); pairs with d_i + d_j below
// 1e-14 d_max (a rank-deficient M) get the minimum-norm value 0
__global__ void k_lyap_div(double *__restrict__ Ct, const double *__restrict__ d, int s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s * s) return;
  const int i = t % s, j = t / s;
  const double den = d[i] + d[j], dmax = fmax(fabs(d[0]), fabs(d[s - 1]));
  Ct[t] = den > 1e-14 * dmax ? Ct[t] / den : 0.0;
}

// out_i = base_i + sgn sum_j w_j V_ij^2 with w_j = mu_j (xf = 0) or mu_j / (1 + mu_j) (xf = 1)
__global__ void k_diag_lowrank(const double *__restrict__ V, long ldv, long n, int k, const double *__restrict__ mu,
                               int xf, double sgn, const double *__restrict__ base, double *__restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) {
      const double v = V[ldv * j + i];
      const double w = xf ? mu[j] / (1.0 + mu[j]) : mu[j];
      acc += w * v * v;
    }
    out[i] = (base ? base[i] : 0.0) + sgn * acc;
  }
}

// stochastic diagonal estimator: out_i = sum_j Z_ij W_ij / sum_j Z_ij^2
__global__ void k_stoch_diag(const double *__restrict__ Z, long ldz, const double *__restrict__ Wm, long ldw, long n,
                             int r, double *__restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double num = 0.0, den = 0.0;
    for (int j = 0; j < r; ++j) {
      const double z = Z[ldz * j + i];
      num += z * Wm[ldw * j + i];
      den += z * z;
    }
    out[i] = den > 0.0 ? num / den : 0.0;
  }
}

}  // namespace hp

extern "C" {

int hp_lowrank_eig(hp_problem *P, const double *m_map, int k, int p, const double *Omega, int ldo, double *lambda,
                   double *V, int ldv, int single_pass, hp_solve_stats *st) {
  if (!P || !m_map || !Omega || !lambda || !V || k < 1 || p < 0 || ldo < P->n || ldv < P->n)
    return set_error(HP_ERR_INVALID, "arguments");
  const int s = k + p;
  if (s > P->n || s > 1024) return set_error(HP_ERR_INVALID, "k + p too large");
  if (st) *st = hp_solve_stats{};
  int rc = 0;
  const long n = P->n, ld = padded(n);
  HP_TRY(set_point(P, m_map, nullptr, nullptr));
  double *Y = col64(P->vtmp[0], P, s, &rc);
  HP_TRY(rc);
  double *Zb = col64(P->vtmp[1], P, s, &rc);
  HP_TRY(rc);
  double *H = col64(P->vtmp[2], P, s, &rc);
  HP_TRY(rc);
  const size_t s2 = (size_t)s * s;
  HP_TRY(P->small.ensure(sizeof(double) * (12 * s2 + 4 * s + 64)));
  double *G = P->small.as<double>(), *T = G + s2, *Sm = T + s2, *Ts = Sm + s2;
  double *lam = Ts + s2;
  double *Wm = lam + 2 * s, *Zs = Wm + s2, *M = Zs + s2, *Cm = M + s2, *E = Cm + s2, *U = E + s2, *tmp = U + s2,
         *d = tmp + s2;
  // Ybar = A Omega ; Y = B^{-1} Ybar
  HP_TRY(hessian_block(P, Omega, ldo, H, ld, s, HP_MISFIT_ONLY, st));
  HP_TRY(Rinv_apply(P, H, ld, Y, ld, s));
  double *Ysave = nullptr;
  if (single_pass) {  // Y is needed again after the QR overwrites it
    Ysave = col64(P->t64c, P, s, &rc);
    HP_TRY(rc);
    launch_copy(Y, ld, Ysave, ld, n, s, P->st);
  }
  // PreCholQR: Z = qr(Y); Zb = B Z; R_Z = chol(Z^T Zb); Q = Z R_Z^{-1} (and Qb = Zb R_Z^{-1})
  HP_TRY(thin_qr(P, Y, ld, n, s));
  HP_TRY(R_apply(P, Y, ld, Zb, ld, s));
  HP_TRY(gram(P, Y, ld, s, Zb, ld, s, G, s, n));
  k_symmetrize<<<(s * s + 255) / 256, 256, 0, P->st>>>(G, Ts, s);
  count_launch();
  HP_TRY(small_cholesky(P, Ts, s));
  launch_trsm_right_upper(Y, ld, n, s, Ts, P);
  if (!single_pass) {
    // Algorithm 2: T = Q^T A Q (the second pass)
    HP_TRY(hessian_block(P, Y, ld, H, ld, s, HP_MISFIT_ONLY, st));
    HP_TRY(gram(P, Y, ld, s, H, ld, s, T, s, n));
  } else {
    // Algorithm 3, eq. (Tsinglepass): T = argmin over symmetric X of |X W - Zs|_F with
    // W = Qb^T Omega, Zs = Qb^T Y.  Its normal equations restricted to symmetric X are the
    // Lyapunov equation X M + M X = C, M = W W^T, C = Zs W^T + W Zs^T, solved in the
    // eigenbasis of M: with M = U D U^T, (U^T X U)_ij = (U^T C U)_ij / (d_i + d_j).
    launch_trsm_right_upper(Zb, ld, n, s, Ts, P);
    HP_TRY(gram(P, Zb, ld, s, Omega, ldo, s, Wm, s, n));
    HP_TRY(gram(P, Zb, ld, s, Ysave, ld, s, Zs, s, n));
    small_gemm(P, s, 0, 1, Wm, Wm, M);   // M = W W^T
    small_gemm(P, s, 0, 1, Zs, Wm, E);   // E = Zs W^T
    k_sym_sum<<<(s * s + 255) / 256, 256, 0, P->st>>>(E, Cm, s);
    k_symmetrize<<<(s * s + 255) / 256, 256, 0, P->st>>>(M, E, s);
    count_launch(2);
    HP_TRY(small_symeig(P, E, s, d, U));
    small_gemm(P, s, 1, 0, U, Cm, tmp);  // U^T C
    small_gemm(P, s, 0, 0, tmp, U, E);   // U^T C U
    k_lyap_div<<<(s * s + 255) / 256, 256, 0, P->st>>>(E, d, s);
    count_launch();
    small_gemm(P, s, 0, 0, U, E, tmp);   // U Xt
    small_gemm(P, s, 0, 1, tmp, U, T);   // X = U Xt U^T
  }
  k_symmetrize<<<(s * s + 255) / 256, 256, 0, P->st>>>(T, Ts, s);
  count_launch();
  HP_TRY(small_symeig(P, Ts, s, lam, Sm));
  // V = Q S(:, 1:k), Lambda_r = Lambda(1:k)
  launch_gemm_nn(Y, ld, s, Sm, s, k, V, ldv, n, 1.0, 0.0, P);
  k_sign_normalise<<<k, NT, 0, P->st>>>(V, ldv, n);
  count_launch();
  HP_CUDA(cudaMemcpyAsync(lambda, lam, sizeof(double) * k, cudaMemcpyDeviceToDevice, P->st));
  return sync(P);
}

// ---------------------------------------------------------------------------
// Section 4.4: pointwise variance
// ---------------------------------------------------------------------------
int hp_pointwise_variance(hp_problem *P, int method, const double *Z, int ldz, int r, const double *lambda,
                          const double *V, int ldv, int k, double *prior_var, double *post_var,
                          hp_solve_stats *st) {
  if (!P || !Z || !prior_var || r < 1 || ldz < P->n || (method != HP_VAR_RANDOMIZED && method != HP_VAR_STOCHASTIC))
    return set_error(HP_ERR_INVALID, "hp_pointwise_variance: arguments");
  if (k < 0 || (k > 0 && (!lambda || !V || ldv < P->n)))
    return set_error(HP_ERR_INVALID, "hp_pointwise_variance: eigenpair arguments");
  if (method == HP_VAR_RANDOMIZED && (r > P->n || r > 1024))
    return set_error(HP_ERR_INVALID, "hp_pointwise_variance: r <= min(n, 1024)");
  if (st) *st = hp_solve_stats{};
  int rc = 0;
  const long n = P->n, ld = padded(n);
  double *Y = col64(P->vtmp[0], P, r, &rc);
  HP_TRY(rc);
  const unsigned nb = (unsigned)blocks_for(n, 1);
  if (method == HP_VAR_STOCHASTIC) {
    HP_TRY(Rinv_apply(P, Z, ldz, Y, ld, r));
    k_stoch_diag<<<nb, NT, 0, P->st>>>(Z, ldz, Y, ld, n, r, prior_var);
    count_launch();
  } else {
    // Algorithm 2 with A = R^-1, B = I: Q = qr(R^-1 Z) (PreCholQR with B = I is a plain QR),
    // T = Q^T R^-1 Q = S diag(mu) S^T, vbar = Q S
    double *AQ = col64(P->vtmp[1], P, r, &rc);
    HP_TRY(rc);
    double *Vb = col64(P->vtmp[2], P, r, &rc);
    HP_TRY(rc);
    const size_t r2 = (size_t)r * r;
    HP_TRY(P->small.ensure(sizeof(double) * (3 * r2 + 2 * r + 64)));
    double *T = P->small.as<double>(), *Ts = T + r2, *Sm = Ts + r2, *mu = Sm + r2;
    HP_TRY(Rinv_apply(P, Z, ldz, Y, ld, r));
    HP_TRY(thin_qr(P, Y, ld, n, r));
    HP_TRY(Rinv_apply(P, Y, ld, AQ, ld, r));
    HP_TRY(gram(P, Y, ld, r, AQ, ld, r, T, r, n));
    k_symmetrize<<<(unsigned)((r2 + 255) / 256), 256, 0, P->st>>>(T, Ts, r);
    count_launch();
    HP_TRY(small_symeig(P, Ts, r, mu, Sm));
    launch_gemm_nn(Y, ld, r, Sm, r, r, Vb, ld, n, 1.0, 0.0, P);
    k_diag_lowrank<<<nb, NT, 0, P->st>>>(Vb, ld, n, r, mu, 0, 1.0, nullptr, prior_var);
    count_launch();
  }
  if (post_var) {
    if (k > 0) {
      k_diag_lowrank<<<nb, NT, 0, P->st>>>(V, ldv, n, k, lambda, 1, -1.0, prior_var, post_var);
      count_launch();
    } else {
      HP_CUDA(cudaMemcpyAsync(post_var, prior_var, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->st));
    }
  }
  return sync(P);
}

// ---------------------------------------------------------------------------
// Section 4.3: prior and Laplace-posterior samples
// ---------------------------------------------------------------------------
int hp_laplace_sample(hp_problem *P, const double *m_map, const double *lambda, const double *V, int ldv, int k,
                      const double *eta, int ldeta, unsigned long long seed, int nsamples, double *prior, double *post,
                      int lds, hp_solve_stats *st) {
  if (P && nsamples == 0) return HP_OK;
  if (!P || nsamples < 0 || (eta && ldeta < P->nelems * (P->dim + 1)) || (!prior && !post) ||
      ((prior || post) && lds < P->n))
    return set_error(HP_ERR_INVALID, "arguments");
  if (post && (!m_map || !lambda || !V || k < 0 || ldv < P->n)) return set_error(HP_ERR_INVALID, "posterior arguments");
  if (st) *st = hp_solve_stats{};
  int rc = 0;
  const long n = P->n, ld = padded(n);
  const int chunk = std::min(nsamples, eta ? 128 : 64);
  if (chunk == 0) return HP_OK;
  const long nper = P->nelems * (P->dim + 1);
  double *etag = nullptr;
  if (!eta) {
    HP_TRY(P->etabuf.ensure(sizeof(double) * (size_t)nper * chunk));
    etag = P->etabuf.as<double>();
  }
  double *W = col64(P->vtmp[0], P, chunk, &rc);
  HP_TRY(rc);
  double *X = col64(P->vtmp[1], P, chunk, &rc);
  HP_TRY(rc);
  double *RX = col64(P->vtmp[2], P, chunk, &rc);
  HP_TRY(rc);
  double *t = col64(P->t64c, P, chunk, &rc);
  HP_TRY(rc);
  HP_TRY(P->small.ensure(sizeof(double) * ((size_t)std::max(k, 1) * chunk + 64)));
  double *z = P->small.as<double>();
  for (int c0 = 0; c0 < nsamples; c0 += chunk) {
    const int cs = std::min(chunk, nsamples - c0);
    if (eta) {
      launch_mass_factor(P, eta + (long)ldeta * c0, ldeta, W, ld, cs);
    } else {
      launch_philox_normals(seed, c0, cs, (int)nper, etag, nper, 0, P->st);
      launch_mass_factor(P, etag, nper, W, ld, cs);
    }
    HP_TRY(solve_block(P, OP_A, W, ld, X, ld, cs, P->rtol, st));
    if (prior) {
      k_add_vec_cols<<<dim3(blocks_for(n, cs), cs), NT, 0, P->st>>>(X, ld, P->m_prior, prior + (long)lds * c0, lds, n);
      count_launch();
    }
    if (post) {
      // R x = A M^{-1} (A x) = A M^{-1} W
      HP_TRY(solve_block(P, OP_M, W, ld, t, ld, cs, std::min(P->rtol, 1e-10), st));
      HP_TRY(apply_op64(P, OP_A, t, ld, RX, ld, cs));
      if (k > 0) {
        HP_TRY(gram(P, V, ldv, k, RX, ld, cs, z, k, n));
        k_scale_rows_S<<<(k * cs + 255) / 256, 256, 0, P->st>>>(z, k, cs, lambda);
        count_launch();
        launch_gemm_nn(V, ldv, k, z, k, cs, X, ld, n, -1.0, 1.0, P);
      }
      k_add_vec_cols<<<dim3(blocks_for(n, cs), cs), NT, 0, P->st>>>(X, ld, m_map, post + (long)lds * c0, lds, n);
      count_launch();
    }
  }
  return sync(P);
}

}  // extern "C"
