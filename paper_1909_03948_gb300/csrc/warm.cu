// warm.cu -- the learned initial guess of the 2D stiffness solves, and the
// recorder that turns the method's own solves into training samples for it.
//
// The network sees a solve K x = b on the padded nodal grid (row iy, column ix;
// H = W = the node count per axis rounded up to a multiple of 8): channel 0 the
// nodal log-coefficient m, channel 1 the Jacobi-scaled right-hand side z = D^-1 b
// (D = diag K) divided by its RMS c = |z| / sqrt(nfree) over the free nodes,
// channel 2 the 0/1 mask of the free nodes.  Its output y is the solution in the
// same scaling: x0 = c y.  A guess only changes where PCG starts: every solve
// still runs to the same relative tolerance, and a column whose guess leaves a
// residual no smaller than |b| starts from zero instead.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace hp {

static long nfree_of(const hp_problem *P) { return (long)(P->N + 1) * (P->N - 1); }

// Z = D^-1 B on the free nodes (B is zero on the Dirichlet faces, where D = 1)
__global__ void k_ws_jacobi(long n, const double *__restrict__ B, long ldb, const double *__restrict__ diag,
                            double *__restrict__ Z, long ldz) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    Z[ldz * j + i] = B[ldb * j + i] / diag[i];
}

// sample j: (m, z_j / c_j, mask) on the padded grid, zero outside the nodes; c_j^2 = zz_j / nfree
__global__ void k_ws_inputs(int np, int H, int W, const double *__restrict__ m, const double *__restrict__ Z, long ldz,
                            const double *__restrict__ zz, double nfree, float *__restrict__ X) {
  const int j = blockIdx.y;
  const long HW = (long)H * W;
  const double ic = zz[j] > 0.0 ? sqrt(nfree / zz[j]) : 0.0;
  float *o = X + (long)j * 3 * HW;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < HW; t += (long)gridDim.x * blockDim.x) {
    const int y = (int)(t / W), x = (int)(t % W);
    float a = 0.f, b = 0.f, c = 0.f;
    if (x < np && y < np) {
      const long i = x + (long)np * y;
      const bool fr = y > 0 && y < np - 1;
      a = (float)m[i];
      b = fr ? (float)(ic * Z[ldz * j + i]) : 0.f;
      c = fr ? 1.f : 0.f;
    }
    o[t] = a;
    o[HW + t] = b;
    o[2 * HW + t] = c;
  }
}

// loss data of sample j: (b_j / c_j, diag, cx, cy) of the level-0 stiffness stencil, and
// (optional) the solution x_j / c_j; zero outside the nodes
__global__ void k_ws_aux(int np, long n, int H, int W, const double *__restrict__ B, long ldb,
                         const double *__restrict__ Xs, long ldx, const double *__restrict__ zz, double nfree,
                         const double *__restrict__ diag, const double *__restrict__ cst, float *__restrict__ A,
                         float *__restrict__ T) {
  const int j = blockIdx.y;
  const long HW = (long)H * W;
  const double ic = zz[j] > 0.0 ? sqrt(nfree / zz[j]) : 0.0;
  float *a = A + (long)j * 4 * HW;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < HW; t += (long)gridDim.x * blockDim.x) {
    const int y = (int)(t / W), x = (int)(t % W);
    float b = 0.f, d = 0.f, cx = 0.f, cy = 0.f, u = 0.f;
    if (x < np && y < np) {
      const long i = x + (long)np * y;
      const bool fr = y > 0 && y < np - 1;
      b = fr ? (float)(ic * B[ldb * j + i]) : 0.f;
      d = (float)diag[i];
      cx = (float)cst[i];
      cy = (float)cst[n + i];
      u = fr ? (float)(ic * Xs[ldx * j + i]) : 0.f;
    }
    a[t] = b;
    a[HW + t] = d;
    a[2 * HW + t] = cx;
    a[3 * HW + t] = cy;
    if (T) T[(long)j * HW + t] = u;
  }
}

// guess of column j: X_j = c_j y_j on the free nodes, 0 on the Dirichlet faces
__global__ void k_ws_guess(int np, long n, int W, long HW, const float *__restrict__ Y, const double *__restrict__ zz,
                           double nfree, double *__restrict__ X, long ldx) {
  const int j = blockIdx.y;
  const double sc = sqrt(zz[j] / nfree);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int y = (int)(i / np), x = (int)(i % np);
    X[ldx * j + i] = (y > 0 && y < np - 1) ? sc * (double)Y[(long)j * HW + (long)y * W + x] : 0.0;
  }
}

__global__ void k_ws_restart(long n, const int *__restrict__ flag, const double *__restrict__ B, long ldb,
                             double *__restrict__ X, long ldx, double *__restrict__ R, long ldr) {
  const int j = blockIdx.y;
  if (!flag[j]) return;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    X[ldx * j + i] = 0.0;
    R[ldr * j + i] = B[ldb * j + i];
  }
}

static unsigned grid_of(long cnt) { return (unsigned)std::max<long>(1, std::min<long>((cnt + 255) / 256, 256)); }

static void padded_grid(const hp_problem *P, int *H, int *W) {
  const int np = P->N + 1;
  *H = *W = (np + 7) / 8 * 8;
}

// Z = D^-1 B into Z (ldz) and zz_j = |Z_j|^2 into P->ws_bb
static int jacobi_scaled(hp_problem *P, const double *B, long ldb, double *Z, long ldz, int s) {
  k_ws_jacobi<<<dim3(grid_of(P->n), s), 256, 0, P->st>>>(P->n, B, ldb, P->lv[0].K64.diag, Z, ldz);
  count_launch();
  HP_TRY(P->ws_bb.ensure(sizeof(double) * s));
  return block_dot(P, Z, ldz, Z, ldz, P->n, s, P->ws_bb.as<double>());
}

bool warm_attached(const hp_problem *P) { return P->ws_on && P->ws_net && P->dim == 2; }

int warm_guess(hp_problem *P, const double *B, long ldb, double *X, long ldx, int s) {
  if (!warm_attached(P)) return 0;
  hp_unet *U = P->ws_net;
  int H, W;
  unet_dims(U, &H, &W);
  const int np = P->N + 1;
  const long HW = (long)H * W;
  const double nfree = (double)nfree_of(P);
  const int cap = unet_cap(U);
  if (jacobi_scaled(P, B, ldb, X, ldx, s)) return 0;   // X holds z until the guesses overwrite it
  const double *zz = P->ws_bb.as<double>();
  for (int c0 = 0; c0 < s; c0 += cap) {
    const int cs = std::min(cap, s - c0);
    k_ws_inputs<<<dim3(grid_of(HW), cs), 256, 0, P->st>>>(np, H, W, P->m, X + ldx * c0, ldx, zz + c0, nfree,
                                                           unet_input(U));
    count_launch();
    unet_run(U, cs, P->st);
    k_ws_guess<<<dim3(grid_of(P->n), cs), 256, 0, P->st>>>(np, P->n, W, HW, unet_output(U), zz + c0, nfree,
                                                            X + ldx * c0, ldx);
    count_launch();
  }
  P->ws_guesses += s;
  return 1;
}

void warm_fallback(hp_problem *P, const int *flag_host, int s, const double *B, long ldb, double *X, long ldx,
                   double *R, long ldr) {
  int nf = 0;
  for (int j = 0; j < s; ++j) nf += flag_host[j] != 0;
  if (!nf) return;
  P->ws_fallbacks += nf;
  if (P->ws_flag.ensure(sizeof(int) * s)) return;
  cudaMemcpyAsync(P->ws_flag.p, flag_host, sizeof(int) * s, cudaMemcpyHostToDevice, P->st);
  k_ws_restart<<<dim3(grid_of(P->n), s), 256, 0, P->st>>>(P->n, P->ws_flag.as<int>(), B, ldb, X, ldx, R, ldr);
  count_launch();
}

bool warm_recording(const hp_problem *P) { return P->ws_rx && P->dim == 2 && P->ws_rcount < P->ws_rcap; }

void warm_record(hp_problem *P, const double *B, long ldb, const double *X, long ldx, int s) {
  if (!warm_recording(P)) return;
  int H, W;
  padded_grid(P, &H, &W);
  const long HW = (long)H * W;
  const int np = P->N + 1;
  const double nfree = (double)nfree_of(P);
  const int cs = (int)std::min<long>(s, P->ws_rcap - P->ws_rcount);
  const long k = P->ws_rcount, ldz = (P->n + 63) / 64 * 64;
  if (P->ws_z.ensure(sizeof(double) * ldz * cs) || jacobi_scaled(P, B, ldb, P->ws_z.as<double>(), ldz, cs)) return;
  const double *zz = P->ws_bb.as<double>();
  const Stencil<double> &K = P->lv[0].K64;
  k_ws_inputs<<<dim3(grid_of(HW), cs), 256, 0, P->st>>>(np, H, W, P->m, P->ws_z.as<double>(), ldz, zz, nfree,
                                                         P->ws_rx + k * 3 * HW);
  k_ws_aux<<<dim3(grid_of(HW), cs), 256, 0, P->st>>>(np, P->n, H, W, B, ldb, X, ldx, zz, nfree, K.diag, K.c,
                                                      P->ws_ra + k * 4 * HW, P->ws_rt ? P->ws_rt + k * HW : nullptr);
  count_launch(2);
  P->ws_rcount += cs;
}

}  // namespace hp

using namespace hp;

extern "C" {

int hp_warmstart_grid(const hp_problem *P, int *H, int *W) {
  if (!P || !H || !W) return set_error(HP_ERR_INVALID, "hp_warmstart_grid: null");
  if (P->dim != 2) return set_error(HP_ERR_INVALID, "hp_warmstart_grid: the warm start is 2D only");
  padded_grid(P, H, W);
  return HP_OK;
}

int hp_warmstart_attach(hp_problem *P, hp_unet *U) {
  if (!P) return set_error(HP_ERR_INVALID, "hp_warmstart_attach: null problem");
  if (U) {
    if (P->dim != 2) return set_error(HP_ERR_INVALID, "hp_warmstart_attach: the warm start is 2D only");
    int H, W, h, w;
    padded_grid(P, &H, &W);
    unet_dims(U, &h, &w);
    if (h != H || w != W) return set_error(HP_ERR_INVALID, "hp_warmstart_attach: network grid differs from the problem's");
  }
  HP_CUDA(cudaStreamSynchronize(P->st));
  P->ws_net = U;
  P->ws_on = U != nullptr;
  P->ws_guesses = P->ws_fallbacks = 0;
  return HP_OK;
}

int hp_warmstart_enable(hp_problem *P, int on) {
  if (!P) return set_error(HP_ERR_INVALID, "hp_warmstart_enable: null problem");
  if (on && !P->ws_net) return set_error(HP_ERR_STATE, "hp_warmstart_enable: no network attached");
  HP_CUDA(cudaStreamSynchronize(P->st));
  P->ws_on = on != 0;
  return HP_OK;
}

int hp_warmstart_record(hp_problem *P, float *X, float *A, float *T, int capacity) {
  if (!P) return set_error(HP_ERR_INVALID, "hp_warmstart_record: null problem");
  if (X && (P->dim != 2 || !A || capacity < 1))
    return set_error(HP_ERR_INVALID, "hp_warmstart_record: 2D problem, X, A and capacity >= 1");
  HP_CUDA(cudaStreamSynchronize(P->st));
  P->ws_rx = X;
  P->ws_ra = X ? A : nullptr;
  P->ws_rt = X ? T : nullptr;
  P->ws_rcap = X ? capacity : 0;
  if (X) P->ws_rcount = 0;
  return HP_OK;
}

int hp_warmstart_counts(const hp_problem *P, long long *recorded, long long *guesses, long long *fallbacks) {
  if (!P) return set_error(HP_ERR_INVALID, "hp_warmstart_counts: null problem");
  if (recorded) *recorded = P->ws_rcount;
  if (guesses) *guesses = P->ws_guesses;
  if (fallbacks) *fallbacks = P->ws_fallbacks;
  return HP_OK;
}

}  // extern "C"
