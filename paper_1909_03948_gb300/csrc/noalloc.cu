// noalloc.cu -- hp_mass_solve_noalloc: the mass-matrix solve X = M^{-1} B
// without any device allocation.
//
// hp_mass_solve grows the problem's workspace on first use (cudaMalloc).  Some
// callers cannot allocate at solve time: a host application that reserves all
// device memory at start-up and forbids allocation afterwards, or one that must
// not change the device's memory footprint while it runs.  This variant keeps its
// temporaries in one file-scope device array of fixed size instead (about 8.5 MB:
// four vectors of HP_NOALLOC_MAX_ENTRIES doubles plus per-column partials).
//
// Method: FP64 conjugate gradients on M preconditioned by diag(M), per-column
// stopping at |r| <= tol |b| with tol = min(problem rtol, 1e-10) and at most
// the problem's max_iter iterations -- the same operator and stopping rule as
// the FP64 path of hp_mass_solve.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.h"

namespace hp {

// Scratch: 4 work vectors (r, z, p, q) of up to HP_NOALLOC_MAX_ENTRIES
// (= n * nrhs) doubles, per-column dot partials and per-column scalars.
constexpr long kNaMaxEntries = HP_NOALLOC_MAX_ENTRIES;
constexpr int kNaMaxCols = HP_NOALLOC_MAX_COLS;
constexpr int kNaBlocks = 128;  // blocks per column of the reductions
constexpr int kNaScalars = 8;   // per column: bb, rr, rz, alpha, beta, active, spare
constexpr long kNaSize = 4 * kNaMaxEntries + (long)kNaMaxCols * (kNaBlocks + kNaScalars);

static __device__ __align__(256) double g_na_scratch[kNaSize];

static std::mutex g_na_mutex;
static double *g_na_ptr[256] = {};  // device address of g_na_scratch, per device

// Device address of the scratch array on the current device, resolved with
// cudaGetSymbolAddress by the first call on that device.
static int na_scratch(double **out) {
  int dev = 0;
  HP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return set_error(HP_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void *p = nullptr;
    HP_CUDA(cudaGetSymbolAddress(&p, g_na_scratch));
    g_na_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_na_ptr[dev];
  return 0;
}

enum { NA_INIT = 0, NA_ALPHA = 1, NA_RR = 2, NA_BETA = 3 };

struct NaScal {
  double *bb, *rr, *rz, *alpha, *beta, *active;  // column-indexed, "active" as 0.0 / 1.0
};

__global__ void k_na_start(long n, const double *__restrict__ B, long ldb, double *__restrict__ X, long ldx,
                           double *__restrict__ r, double *__restrict__ p, NaScal sc, int it_zero) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    r[n * j + i] = B[ldb * j + i];
    p[n * j + i] = 0.0;
    X[ldx * j + i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sc.beta[j] = 0.0;
  (void)it_zero;
}

// partial of <a, b> per (column, block)
__global__ void k_na_dot(long n, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ part) {
  const int j = blockIdx.y;
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    acc += a[n * j + i] * b[n * j + i];
  acc = block_sum<NT>(acc);
  if (threadIdx.x == 0) part[(long)j * gridDim.x + blockIdx.x] = acc;
}

// fixed-order sum of the partials of column j, then the CG scalar step
__global__ void k_na_fin(const double *__restrict__ part, int nblk, NaScal sc, int mode, double tol2, int first) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += NT) s += part[(long)j * nblk + b];
  s = block_sum<NT>(s);
  if (threadIdx.x != 0) return;
  const bool act = sc.active[j] != 0.0;
  switch (mode) {
    case NA_INIT:
      sc.bb[j] = s;
      sc.rr[j] = s;
      sc.active[j] = s > 0.0 ? 1.0 : 0.0;
      break;
    case NA_ALPHA: sc.alpha[j] = (act && s > 0.0) ? sc.rz[j] / s : 0.0; break;
    case NA_RR:
      sc.rr[j] = s;
      sc.active[j] = (act && s > tol2 * sc.bb[j]) ? 1.0 : 0.0;
      break;
    case NA_BETA:
      sc.beta[j] = (!first && act && sc.rz[j] != 0.0) ? s / sc.rz[j] : 0.0;
      sc.rz[j] = s;
      break;
  }
}

__global__ void k_na_precond(long n, const double *__restrict__ invdiag, const double *__restrict__ r,
                             double *__restrict__ z, double *__restrict__ p, const double *__restrict__ beta, int pass) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    if (pass == 0) {
      z[n * j + i] = invdiag[i] * r[n * j + i];
    } else {
      p[n * j + i] = z[n * j + i] + beta[j] * p[n * j + i];
    }
  }
}

__global__ void k_na_update(long n, const double *__restrict__ p, const double *__restrict__ q, double *__restrict__ X,
                            long ldx, double *__restrict__ r, const double *__restrict__ alpha) {
  const int j = blockIdx.y;
  const double a = alpha[j];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    X[ldx * j + i] += a * p[n * j + i];
    r[n * j + i] -= a * q[n * j + i];
  }
}

static int na_mass_solve(hp_problem *P, const double *B, long ldb, double *X, long ldx, int s, hp_solve_stats *stats) {
  const long n = P->n;
  if ((long)s > kNaMaxCols || n * (long)s > kNaMaxEntries)
    return set_error(HP_ERR_INVALID, "hp_mass_solve_noalloc: nrhs <= 64 and n * nrhs <= 262144 required");
  double *base = nullptr;
  HP_TRY(na_scratch(&base));
  double *r = base, *z = base + kNaMaxEntries, *p = base + 2 * kNaMaxEntries, *q = base + 3 * kNaMaxEntries;
  double *part = base + 4 * kNaMaxEntries;
  double *scal = part + (long)kNaMaxCols * kNaBlocks;
  NaScal sc{scal, scal + kNaMaxCols, scal + 2 * kNaMaxCols, scal + 3 * kNaMaxCols, scal + 4 * kNaMaxCols,
            scal + 5 * kNaMaxCols};
  cudaStream_t st = P->st;
  const double tol = std::min(P->rtol, 1e-10);
  const int nb = (int)std::min<long>(kNaBlocks, std::max<long>(1, (n + NT - 1) / NT));
  const dim3 grid(nb, s);
  const Stencil<double> &M = P->M64;
  k_na_start<<<grid, NT, 0, st>>>(n, B, ldb, X, ldx, r, p, sc, 0);
  k_na_dot<<<grid, NT, 0, st>>>(n, r, r, part);
  k_na_fin<<<s, NT, 0, st>>>(part, nb, sc, NA_INIT, tol * tol, 1);
  count_launch(3);
  double h_active[kNaMaxCols];
  int it = 0;
  for (it = 1; it <= P->max_iter; ++it) {
    k_na_precond<<<grid, NT, 0, st>>>(n, M.invdiag, r, z, p, sc.beta, 0);
    k_na_dot<<<grid, NT, 0, st>>>(n, r, z, part);
    k_na_fin<<<s, NT, 0, st>>>(part, nb, sc, NA_BETA, 0.0, it == 1);
    k_na_precond<<<grid, NT, 0, st>>>(n, M.invdiag, r, z, p, sc.beta, 1);
    launch_stencil_apply<double>(P, P->lv[0].g, M, p, n, q, n, s, st);
    k_na_dot<<<grid, NT, 0, st>>>(n, p, q, part);
    k_na_fin<<<s, NT, 0, st>>>(part, nb, sc, NA_ALPHA, 0.0, 0);
    k_na_update<<<grid, NT, 0, st>>>(n, p, q, X, ldx, r, sc.alpha);
    k_na_dot<<<grid, NT, 0, st>>>(n, r, r, part);
    k_na_fin<<<s, NT, 0, st>>>(part, nb, sc, NA_RR, tol * tol, 0);
    count_launch(9);
    HP_CUDA(cudaMemcpyAsync(h_active, sc.active, sizeof(double) * s, cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaStreamSynchronize(st));
    int nact = 0;
    for (int j = 0; j < s; ++j) nact += h_active[j] != 0.0;
    if (nact == 0) break;
  }
  if (stats) {
    stats->iterations += std::min(it, P->max_iter);
    stats->solves += 1;
  }
  if (it > P->max_iter) return set_error(HP_ERR_NOT_CONVERGED, "hp_mass_solve_noalloc did not converge");
  return cuda_check(cudaGetLastError(), "hp_mass_solve_noalloc");
}

}  // namespace hp

extern "C" int hp_mass_solve_noalloc(hp_problem *P, const double *B, int ldb, double *X, int ldx, int nrhs,
                                     hp_solve_stats *st) {
  using namespace hp;
  if (P && nrhs == 0) return HP_OK;
  if (!P || !B || !X || nrhs < 0 || ldb < P->n || ldx < P->n) return set_error(HP_ERR_INVALID, "arguments");
  if (st) *st = hp_solve_stats{};
  return na_mass_solve(P, B, ldb, X, ldx, nrhs, st);
}
