// vec.cu -- column-block vector kernels (FP64) and deterministic block dots.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace hp {

std::atomic<unsigned long long> g_launches{0};
std::atomic<unsigned long long> g_tiled_launches{0};
std::atomic<unsigned long long> g_alg_bytes[BYTES_FAMILIES] = {};
thread_local long tl_n0 = 0;
thread_local int tl_no_count = 0;

int DBuf::ensure(size_t b) {
  if (b <= bytes) return 0;
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
  if (cudaMalloc(&p, b) != cudaSuccess) {
    cudaGetLastError();
    return set_error(HP_ERR_NOMEM, "device allocation failed");
  }
  bytes = b;
  return 0;
}

void DBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

__global__ void k_copy(const double *__restrict__ X, long ldx, double *__restrict__ Y, long ldy, long n) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    Y[ldy * j + i] = X[ldx * j + i];
}

__global__ void k_fill(double *X, long ldx, long n, double v) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    X[ldx * j + i] = v;
}

__global__ void k_axpby(double a, const double *__restrict__ X, long ldx, double b, double *__restrict__ Y,
                        long ldy, long n) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double y = b == 0.0 ? 0.0 : b * Y[ldy * j + i];
    Y[ldy * j + i] = a * X[ldx * j + i] + y;
  }
}

__global__ void k_exp(const double *__restrict__ m, double *__restrict__ E, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    E[i] = exp(m[i]);
}

void launch_copy(const double *X, long ldx, double *Y, long ldy, long n, int s, cudaStream_t st) {
  k_copy<<<dim3(blocks_for(n, s), s), NT, 0, st>>>(X, ldx, Y, ldy, n);
  count_launch();
}
void launch_fill(double *X, long ldx, long n, int s, double v, cudaStream_t st) {
  k_fill<<<dim3(blocks_for(n, s), s), NT, 0, st>>>(X, ldx, n, v);
  count_launch();
}
void launch_axpby(double a, const double *X, long ldx, double b, double *Y, long ldy, long n, int s,
                  cudaStream_t st) {
  k_axpby<<<dim3(blocks_for(n, s), s), NT, 0, st>>>(a, X, ldx, b, Y, ldy, n);
  count_launch();
}
void launch_ew_exp(const double *m, double *E, long n, cudaStream_t st) {
  k_exp<<<blocks_for(n, 1), NT, 0, st>>>(m, E, n);
  count_launch();
}

// Two-stage deterministic dot: block partials then a fixed-order sum.
__global__ void k_dot_partial(const double *__restrict__ X, long ldx, const double *__restrict__ Y, long ldy,
                              long n, double *__restrict__ part) {
  const int j = blockIdx.y;
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    acc += X[ldx * j + i] * Y[ldy * j + i];
  acc = block_sum<NT>(acc);
  if (threadIdx.x == 0) part[(long)j * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_dot_final(const double *__restrict__ part, int nb, double *__restrict__ out,
                            double *__restrict__ out2) {
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(long)j * nb + b];
  acc = block_sum<NT>(acc);
  if (threadIdx.x == 0) {
    out[j] = acc;
    if (out2) out2[j] = acc;
  }
}

// Start of an iterative-refinement solve from x = 0, in one pass over B: B0 = B with the
// `face` nodes at each end of a column zeroed (the Dirichlet rows; face = 0 keeps all),
// X = 0, and the block partials of |B0_j|^2.  X may alias B (each thread reads its
// entry of B before writing the same entry of X).
__global__ void k_ir_start(const double *B, long ldb, double *__restrict__ B0, long ld0, double *X, long ldx,
                           long n, long face, double *__restrict__ part) {
  const int j = blockIdx.y;
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double v = (i < face || i >= n - face) ? 0.0 : B[ldb * j + i];
    B0[ld0 * j + i] = v;
    X[ldx * j + i] = 0.0;
    acc += v * v;
  }
  acc = block_sum<NT>(acc);
  if (threadIdx.x == 0) part[(long)j * gridDim.x + blockIdx.x] = acc;
}

int ir_start(hp_problem *P, const double *B, long ldb, double *B0, long ld0, double *X, long ldx, long n, int s,
             long face, double *bb_dev, double *rr_dev) {
  const int nb = blocks_for(n, s);
  HP_TRY(P->sc.tmp.ensure(sizeof(double) * (size_t)nb * s));
  double *part = P->sc.tmp.as<double>();
  k_ir_start<<<dim3(nb, s), NT, 0, P->st>>>(B, ldb, B0, ld0, X, ldx, n, face, part);
  k_dot_final<<<s, NT, 0, P->st>>>(part, nb, bb_dev, rr_dev);
  count_launch(2);
  count_bytes(BY_REFINE, 3.0 * 8.0 * (double)n * s);  // read B, write B0 and X
  return 0;
}

int block_dot(hp_problem *P, const double *X, long ldx, const double *Y, long ldy, long n, int s,
              double *out_dev) {
  const int nb = blocks_for(n, s);
  HP_TRY(P->sc.tmp.ensure(sizeof(double) * (size_t)nb * s));
  double *part = P->sc.tmp.as<double>();
  k_dot_partial<<<dim3(nb, s), NT, 0, P->st>>>(X, ldx, Y, ldy, n, part);
  k_dot_final<<<s, NT, 0, P->st>>>(part, nb, out_dev, nullptr);
  count_launch(2);
  return 0;
}

}  // namespace hp
