// dense.cu -- FP64 tall-skinny and small dense linear algebra of the
// randomized eigensolver (Algorithms 2-4) and the low-rank sampling update.
//
//   gram          G = X^T Y (n x s1, n x s2), tiled, deterministic two-stage sum
//   gemm_nn       Y = alpha X S + beta Y (X: n x s1, S: s1 x s2)
//   thin_qr       orthonormal Z with range(Z) = range(Y), the thin-QR step of
//                 PreCholQR (Algorithm 4): shifted Cholesky QR in three passes
//   cgs2_qr       the same by classical Gram-Schmidt with one full
//                 re-orthogonalisation per column ("twice is enough"), the
//                 fallback for a rank-deficient block
//   small_cholesky, trsm_right_upper   R_Z = chol(Z^T Zb), Q = Z R_Z^{-1}
//   small_symeig  cyclic Jacobi with a round-robin parallel ordering, sorted
//                 descending (Algorithm 2: T = S Lambda S^T), A in shared memory up
//                 to 160 x 160 (and V with it up to 90 x 90)
// GB300's FP64 rate is low (a few percent of FP32), so these are written as
// plain FP64 FMA kernels; they are a small share of the eigensolver's time,
// which is dominated by the 2(k+p) Hessian actions.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"

namespace hp {

constexpr int GT = 32;  // gram tile

__global__ void k_gram_partial(const double *__restrict__ X, long ldx, int s1, const double *__restrict__ Y, long ldy,
                               int s2, long n, long rows_per_chunk, double *__restrict__ part) {
  __shared__ double xs[GT][GT + 1], ys[GT][GT + 1];
  const int ta = blockIdx.x, tb = blockIdx.y, ch = blockIdx.z;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const long r0 = ch * rows_per_chunk, r1 = std::min<long>(n, r0 + rows_per_chunk);
  double acc[4] = {0, 0, 0, 0};
  for (long rb = r0; rb < r1; rb += GT) {
    for (int k = ty; k < GT; k += 8) {
      const long row = rb + tx;
      const int ca = ta * GT + k, cb = tb * GT + k;
      xs[k][tx] = (row < r1 && ca < s1) ? X[ldx * ca + row] : 0.0;
      ys[k][tx] = (row < r1 && cb < s2) ? Y[ldy * cb + row] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < GT; ++rr) {
      const double yv = ys[tx][rr];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += xs[ty + 8 * q][rr] * yv;
    }
    __syncthreads();
  }
  const int nta = gridDim.x, ntb = gridDim.y;
  for (int q = 0; q < 4; ++q) {
    const int a = ty + 8 * q, b = tx;
    part[(((long)ch * nta + ta) * ntb + tb) * GT * GT + a * GT + b] = acc[q];
  }
}

// The same partial Gram in double-float arithmetic on the FP32 pipe: the FP64 tiles are
// split into pairs as they are loaded into shared memory (bit manipulation), each thread
// keeps compensated (Dot2) sums for its 4 entries over the chunk's rows, and the chunk's
// entries are stored as doubles.  With sym (X = Y) only the tiles on and above the
// diagonal are formed; k_gram_final mirrors the others.  The compensated sum over a chunk
// is more accurate than FP64 accumulation of the same products (about 2^-48 of the result
// plus n 2^-96 of the terms' magnitudes).
__global__ void k_gram_partial_df(const double *__restrict__ X, long ldx, int s1, const double *__restrict__ Y,
                                  long ldy, int s2, long n, long rows_per_chunk, int sym, double *__restrict__ part) {
  __shared__ float2 xs[GT][GT + 1], ys[GT][GT + 1];
  const int ta = blockIdx.x, tb = blockIdx.y, ch = blockIdx.z;
  if (sym && ta > tb) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const long r0 = ch * rows_per_chunk, r1 = std::min<long>(n, r0 + rows_per_chunk);
  Dot2 acc[4];
  for (long rb = r0; rb < r1; rb += GT) {
    for (int k = ty; k < GT; k += 8) {
      const long row = rb + tx;
      const int ca = ta * GT + k, cb = tb * GT + k;
      const dfl a = d2df((row < r1 && ca < s1) ? X[ldx * ca + row] : 0.0);
      const dfl b = d2df((row < r1 && cb < s2) ? Y[ldy * cb + row] : 0.0);
      xs[k][tx] = make_float2(a.hi, a.lo);
      ys[k][tx] = make_float2(b.hi, b.lo);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < GT; ++rr) {
      const float2 yv = ys[tx][rr];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 xv = xs[ty + 8 * q][rr];
        acc[q].fma(dfl{xv.x, xv.y}, dfl{yv.x, yv.y});
      }
    }
    __syncthreads();
  }
  const int nta = gridDim.x, ntb = gridDim.y;
  for (int q = 0; q < 4; ++q) {
    const int a = ty + 8 * q, b = tx;
    part[(((long)ch * nta + ta) * ntb + tb) * GT * GT + a * GT + b] = df2d(acc[q].result());
  }
}

__global__ void k_gram_final(const double *__restrict__ part, int nchunk, int nta, int ntb, int s1, int s2,
                             double *__restrict__ G, int ldg, int sym) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= s1 * s2) return;
  int a = idx % s1, b = idx / s1;
  if (sym && a / GT > b / GT) {  // a tile below the diagonal: the mirrored entry of the one above
    const int t = a;
    a = b;
    b = t;
  }
  const int ta = a / GT, tb = b / GT;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(((long)c * nta + ta) * ntb + tb) * GT * GT + (a % GT) * GT + (b % GT)];
  G[idx % s1 + (long)ldg * (idx / s1)] = s;
}

// G = X^T y for a single column y: each block sums its chunk of rows for 8 columns of X at a
// time (coalesced along the rows), the partials [chunk][column] are added in chunk order
__global__ void k_gemv_t_partial(const double *__restrict__ X, long ldx, int s1, const double *__restrict__ y,
                                 long n, long rows_per_chunk, double *__restrict__ part) {
  __shared__ double red[8][8];  // [warp][column of the group]
  const int ch = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long r0 = ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  for (int a0 = 0; a0 < s1; a0 += 8) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double yi = y[i];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (a0 + q < s1) acc[q] = fmadd(X[ldx * (a0 + q) + i], yi, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
      if (lane == 0) red[w][q] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < 8 && a0 + (int)threadIdx.x < s1) {
      double t = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += red[ww][threadIdx.x];
      part[(long)ch * s1 + a0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void k_gemv_t_final(const double *__restrict__ part, int nchunk, int s1, double *__restrict__ G) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= s1) return;
  double t = 0.0;
  for (int c = 0; c < nchunk; ++c) t += part[(long)c * s1 + a];
  G[a] = t;
}

int gram(hp_problem *P, const double *X, long ldx, int s1, const double *Y, long ldy, int s2, double *G, int ldg,
         long n) {
  if (s2 == 1) {  // a matrix-vector product: the tiled kernel would compute a whole tile of X^T Y
    int nchunk = 2 * NSM;
    const long rpc = std::max<long>(256, (n + nchunk - 1) / nchunk);
    nchunk = (int)((n + rpc - 1) / rpc);
    HP_TRY(P->vtmp[5].ensure(sizeof(double) * (size_t)nchunk * s1));
    double *part = P->vtmp[5].as<double>();
    k_gemv_t_partial<<<nchunk, 256, 0, P->st>>>(X, ldx, s1, Y, n, rpc, part);
    k_gemv_t_final<<<(s1 + 255) / 256, 256, 0, P->st>>>(part, nchunk, s1, G);
    count_launch(2);
    return cuda_check(cudaGetLastError(), "gram");
  }
  const int nta = (s1 + GT - 1) / GT, ntb = (s2 + GT - 1) / GT;
  int nchunk = std::max(1, (2 * NSM) / (nta * ntb));
  long rpc = (n + nchunk - 1) / nchunk;
  rpc = (rpc + GT - 1) / GT * GT;
  nchunk = (int)((n + rpc - 1) / rpc);
  if (nchunk < 1) nchunk = 1;
  const size_t need = sizeof(double) * (size_t)nchunk * nta * ntb * GT * GT;
  HP_TRY(P->vtmp[5].ensure(need));
  double *part = P->vtmp[5].as<double>();
  const bool df = P->refine_df != 0;  // the Gram in double-float (see k_gram_partial_df)
  const int sym = df && X == Y && ldx == ldy && s1 == s2;
  if (df)
    k_gram_partial_df<<<dim3(nta, ntb, nchunk), 256, 0, P->st>>>(X, ldx, s1, Y, ldy, s2, n, rpc, sym, part);
  else
    k_gram_partial<<<dim3(nta, ntb, nchunk), 256, 0, P->st>>>(X, ldx, s1, Y, ldy, s2, n, rpc, part);
  k_gram_final<<<(s1 * s2 + 255) / 256, 256, 0, P->st>>>(part, nchunk, nta, ntb, s1, s2, G, ldg, sym);
  count_launch(2);
  return cuda_check(cudaGetLastError(), "gram");
}

__global__ void k_gemm_nn(const double *__restrict__ X, long ldx, int s1, const double *__restrict__ S, int lds,
                          int s2, double *__restrict__ Y, long ldy, long n, double alpha, double beta) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < s1; ++k) acc += X[ldx * k + i] * __ldg(&S[k + (long)lds * j]);
    const double y = beta == 0.0 ? 0.0 : beta * Y[ldy * j + i];
    Y[ldy * j + i] = alpha * acc + y;
  }
}

// The same product in double-float on the FP32 pipe: each thread forms 8 output columns of
// its row as compensated (Dot2) sums, so every element of X is split into a pair once per 8
// columns instead of read and multiplied in FP64 for each; S's entries are split as they
// are used (from L1).  alpha and beta are applied in FP64 once per output.
constexpr int GM_NJ = 8;
__global__ void k_gemm_nn_df(const double *__restrict__ X, long ldx, int s1, const double *__restrict__ S, int lds,
                             int s2, double *__restrict__ Y, long ldy, long n, double alpha, double beta) {
  extern __shared__ float2 sp[];  // the block's 8 columns of S as pairs, [k][q]
  const int j0 = blockIdx.y * GM_NJ;
  for (int t = threadIdx.x; t < s1 * GM_NJ; t += blockDim.x) {
    const int k = t / GM_NJ, q = t % GM_NJ;
    const dfl d = d2df(j0 + q < s2 ? S[k + (long)lds * (j0 + q)] : 0.0);
    sp[t] = make_float2(d.hi, d.lo);
  }
  __syncthreads();
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Dot2 acc[GM_NJ];
    for (int k = 0; k < s1; ++k) {
      const dfl x = d2df(X[ldx * k + i]);
#pragma unroll
      for (int q = 0; q < GM_NJ; ++q) {
        const float2 sv = sp[k * GM_NJ + q];
        acc[q].fma(dfl{sv.x, sv.y}, x);
      }
    }
#pragma unroll
    for (int q = 0; q < GM_NJ; ++q) {
      const int j = j0 + q;
      if (j >= s2) break;
      const double y = beta == 0.0 ? 0.0 : beta * Y[ldy * j + i];
      Y[ldy * j + i] = alpha * df2d(acc[q].result()) + y;
    }
  }
}

// R^{-1} of an upper-triangular R (column-major, s x s) in FP64, one thread per column:
// back substitution of R x = e_j (the upper triangle of the result; zeros below)
__global__ void k_tri_inv(const double *__restrict__ R, int s, double *__restrict__ Ri) {
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    for (int i = s - 1; i > j; --i) Ri[i + (long)s * j] = 0.0;
    Ri[j + (long)s * j] = 1.0 / R[j + (long)s * j];
    for (int i = j - 1; i >= 0; --i) {
      double t = 0.0;
      for (int k = i + 1; k <= j; ++k) t = fma(R[i + (long)s * k], Ri[k + (long)s * j], t);
      Ri[i + (long)s * j] = -t / R[i + (long)s * i];
    }
  }
}

void launch_gemm_nn(const double *X, long ldx, int s1, const double *S, int lds, int s2, double *Y, long ldy, long n,
                    double alpha, double beta, hp_problem *P) {
  if (P->refine_df != 0 && s2 > 1 && sizeof(float2) * (size_t)s1 * GM_NJ <= 48 * 1024) {
    const int nj = (s2 + GM_NJ - 1) / GM_NJ;
    k_gemm_nn_df<<<dim3(blocks_for(n, nj), nj), NT, sizeof(float2) * (size_t)s1 * GM_NJ, P->st>>>(
        X, ldx, s1, S, lds, s2, Y, ldy, n, alpha, beta);
  } else {
    k_gemm_nn<<<dim3(blocks_for(n, s2), s2), NT, 0, P->st>>>(X, ldx, s1, S, lds, s2, Y, ldy, n, alpha, beta);
  }
  count_launch();
}

// y <- y - Q c  with c (device, length j) ; then optionally report |y|^2
__global__ void k_scale_col(double *__restrict__ y, long n, const double *__restrict__ nrm2) {
  const double nv = sqrt(*nrm2);
  const double inv = nv > 0.0 ? 1.0 / nv : 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) y[i] *= inv;
}

int cgs2_qr(hp_problem *P, double *Y, long ldy, long n, int s) {
  HP_TRY(P->vtmp[4].ensure(sizeof(double) * (size_t)(s + 2)));
  double *c = P->vtmp[4].as<double>();
  for (int j = 0; j < s; ++j) {
    double *y = Y + ldy * j;
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      HP_TRY(gram(P, Y, ldy, j, y, ldy, 1, c, j, n));
      launch_gemm_nn(Y, ldy, j, c, j, 1, y, ldy, n, -1.0, 1.0, P);
    }
    HP_TRY(block_dot(P, y, ldy, y, ldy, n, 1, c + s));
    k_scale_col<<<blocks_for(n, 1), NT, 0, P->st>>>(y, n, c + s);
    count_launch();
  }
  return cuda_check(cudaGetLastError(), "cgs2_qr");
}

// ---------------------------------------------------------------------------
// Thin QR of a tall block by shifted Cholesky QR, three passes (Fukaya, Kannan,
// Nakatsukasa, Yamamoto, Yanagisawa, "Shifted Cholesky QR for computing the QR
// factorization of ill-conditioned matrices", SIAM J. Sci. Comput. 2020): each pass forms
// G = Y^T Y, factors G = R^T R and sets Y <- Y R^{-1}; the first pass factors G + sigma I
// with sigma = 11 (n s + s (s + 1)) u tr(G) (tr(G) >= |Y|_2^2, u the unit roundoff), which
// keeps the Cholesky factorisable for any numerically full-rank Y and makes Y well enough
// conditioned for the two plain passes to reach orthogonality at the rounding level.
// Three full-width Gram products replace the 2(s - 1) one-column products of
// column-by-column Gram-Schmidt, which waste most of each FP64 Gram tile.  A Gram matrix
// that still is not positive definite (a rank-deficient block) falls back to cgs2_qr.
// ---------------------------------------------------------------------------
__global__ void k_sym_copy(const double *__restrict__ G, double *__restrict__ R, int s) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= s * s) return;
  const int a = idx % s, b = idx / s;
  R[idx] = 0.5 * (G[a + (long)s * b] + G[b + (long)s * a]);
}

__global__ void k_shift_diag(double *R, int s, long n) {
  __shared__ double tr;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < s; ++i) t += R[i + (long)s * i];
    tr = t;
  }
  __syncthreads();
  const double sigma = 11.0 * ((double)n * s + (double)s * (s + 1)) * 0x1p-53 * tr;
  for (int i = threadIdx.x; i < s; i += blockDim.x) R[i + (long)s * i] += sigma;
}

int thin_qr(hp_problem *P, double *Y, long ldy, long n, int s) {
  HP_TRY(P->vtmp[4].ensure(sizeof(double) * (2 * (size_t)s * s + (size_t)s + 2)));
  double *G = P->vtmp[4].as<double>(), *R = G + (size_t)s * s;
  for (int pass = 0; pass < 3; ++pass) {
    HP_TRY(gram(P, Y, ldy, s, Y, ldy, s, G, s, n));
    k_sym_copy<<<(s * s + 255) / 256, 256, 0, P->st>>>(G, R, s);
    count_launch();
    if (pass == 0) {
      k_shift_diag<<<1, 256, 0, P->st>>>(R, s, n);
      count_launch();
    }
    if (small_cholesky(P, R, s) != 0) return cgs2_qr(P, Y, ldy, n, s);
    launch_trsm_right_upper(Y, ldy, n, s, R, P);
  }
  return cuda_check(cudaGetLastError(), "thin_qr");
}

// lower Cholesky in place (row-major) == upper R in column-major
__global__ void k_small_chol(double *A, int s, int *status) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < s; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[(long)k * s + k];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      A[(long)k * s + k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double dk = A[(long)k * s + k];
    for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) A[(long)i * s + k] /= dk;
    __syncthreads();
    const int m = s - k - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = k + 1 + t / m, jj = k + 1 + t % m;
      if (jj <= i) A[(long)i * s + jj] -= A[(long)i * s + k] * A[(long)jj * s + k];
    }
    __syncthreads();
  }
  // clear the strictly lower part of the column-major R (upper part of row-major)
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    const int i = t / s, jj = t % s;
    if (jj > i) A[(long)i * s + jj] = 0.0;
  }
  if (threadIdx.x == 0) *status = bad;
}

int small_cholesky(hp_problem *P, double *G, int s) {
  int *d = P->sc.active.as<int>();
  k_small_chol<<<1, 1024, 0, P->st>>>(G, s, d);
  count_launch();
  int h = 0;
  HP_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, P->st));
  HP_CUDA(cudaStreamSynchronize(P->st));
  if (h) return set_error(HP_ERR_NONFINITE, "Gram matrix of PreCholQR is not positive definite");
  return 0;
}

// Y <- Y R^{-1} (R upper, column-major s x s): row-wise forward substitution
__global__ void k_trsm_ru(double *__restrict__ Y, long ldy, long n, int s, const double *__restrict__ R) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    for (int j = 0; j < s; ++j) {
      double v = Y[ldy * j + i];
      for (int k = 0; k < j; ++k) v -= Y[ldy * k + i] * __ldg(&R[k + (long)s * j]);
      Y[ldy * j + i] = v / __ldg(&R[j + (long)s * j]);
    }
  }
}

void launch_trsm_right_upper(double *Y, long ldy, long n, int s, const double *R, hp_problem *P) {
  // double-float: Y R^{-1} as a product with the explicit inverse (FP64, one small kernel),
  // formed into a scratch block by the double-float product and copied back.  The inverse's
  // rounding is about cond(R) 2^-48 relative; the QR passes that use it are self-correcting
  // and the eigensolver's R-orthonormality is checked to 1e-7.
  const long ldt = (n + 63) / 64 * 64;
  if (P->refine_df != 0 && s > 1 && sizeof(float2) * (size_t)s * GM_NJ <= 48 * 1024 &&
      P->vtmp[3].ensure(sizeof(double) * (size_t)s * s) == 0 && P->dense_tmp.ensure(sizeof(double) * ldt * s) == 0) {
    double *Ri = P->vtmp[3].as<double>(), *T = P->dense_tmp.as<double>();
    k_tri_inv<<<1, 128, 0, P->st>>>(R, s, Ri);
    count_launch();
    launch_gemm_nn(Y, ldy, s, Ri, s, s, T, ldt, n, 1.0, 0.0, P);
    cudaMemcpy2DAsync(Y, sizeof(double) * ldy, T, sizeof(double) * ldt, sizeof(double) * n, s,
                      cudaMemcpyDeviceToDevice, P->st);
    return;
  }
  (void)cudaGetLastError();
  k_trsm_ru<<<blocks_for(n, 1), NT, 0, P->st>>>(Y, ldy, n, s, R);
  count_launch();
}

// ---------------------------------------------------------------------------
// cyclic Jacobi eigen-solver, one block.  A (s x s) and V in global scratch.
// ---------------------------------------------------------------------------
__global__ void k_jacobi_eig(double *A, double *V, int s, int m, double *lam_out, double *S_out, int max_sweeps) {
  extern __shared__ double sh[];
  double *cs = sh;          // m/2 cosines
  double *sn = sh + m / 2;  // m/2 sines
  int *pp = reinterpret_cast<int *>(sn + m / 2);
  int *qq = pp + m / 2;
  __shared__ double off_s, tot_s;
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) V[t] = (t % s == t / s) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence test
    if (threadIdx.x == 0) {
      double off = 0.0, tot = 0.0;
      for (int t = 0; t < s * s; ++t) {
        const double v = A[t] * A[t];
        tot += v;
        if (t % s != t / s) off += v;
      }
      off_s = off;
      tot_s = tot;
    }
    __syncthreads();
    if (off_s <= 1e-30 * tot_s || off_s == 0.0) break;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = threadIdx.x; k < m / 2; k += blockDim.x) {
        int p, q;
        if (k == 0) {
          p = r;
          q = m - 1;
        } else {
          p = (r + k) % (m - 1);
          q = (r - k + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, sv = 0.0;
        if (q < s) {
          const double apq = A[p + (long)s * q];
          if (apq != 0.0) {
            const double theta = (A[q + (long)s * q] - A[p + (long)s * p]) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sv = t * c;
          }
        }
        cs[k] = c;
        sn[k] = sv;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int t = threadIdx.x; t < (m / 2) * s; t += blockDim.x) {
        const int k = t / s, col = t % s;
        const int p = pp[k], q = qq[k];
        if (q >= s) continue;
        const double c = cs[k], sv = sn[k];
        const double ap = A[p + (long)s * col], aq = A[q + (long)s * col];
        A[p + (long)s * col] = c * ap - sv * aq;
        A[q + (long)s * col] = sv * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int t = threadIdx.x; t < (m / 2) * s; t += blockDim.x) {
        const int k = t / s, row = t % s;
        const int p = pp[k], q = qq[k];
        if (q >= s) continue;
        const double c = cs[k], sv = sn[k];
        const double ap = A[row + (long)s * p], aq = A[row + (long)s * q];
        A[row + (long)s * p] = c * ap - sv * aq;
        A[row + (long)s * q] = sv * ap + c * aq;
        const double vp = V[row + (long)s * p], vq = V[row + (long)s * q];
        V[row + (long)s * p] = c * vp - sv * vq;
        V[row + (long)s * q] = sv * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // sort descending (selection order computed by thread 0), write outputs
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int a = 0; a < s; ++a) pp[a] = a;
    for (int a = 0; a < s; ++a) {
      int best = a;
      for (int b = a + 1; b < s; ++b)
        if (A[pp[b] + (long)s * pp[b]] > A[pp[best] + (long)s * pp[best]]) best = b;
      const int t = pp[a];
      pp[a] = pp[best];
      pp[best] = t;
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < s; a += blockDim.x) lam_out[a] = A[pp[a] + (long)s * pp[a]];
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    const int row = t % s, col = t / s;
    S_out[row + (long)s * col] = V[row + (long)s * pp[col]];
  }
}

// The same cyclic Jacobi method (same rotations in the same order) with A in shared memory
// and the off-diagonal norm of the convergence test as a block reduction: V shares the
// shared memory for s <= JS_MAX, and lives in the global scratch Vg up to JS_MAX_A.
constexpr int JS_MAX = 90, JS_MAX_A = 160;

__global__ void __launch_bounds__(1024) k_jacobi_eig_sm(const double *__restrict__ Ain, int s, int m,
                                                        double *lam_out, double *S_out, int max_sweeps,
                                                        double *Vg) {
  extern __shared__ double sh[];
  double *A = sh, *V = Vg ? Vg : A + s * s;
  double *cs = A + s * s + (Vg ? 0 : s * s), *sn = cs + m / 2, *red = sn + m / 2;  // red: [2][32]
  int *pp = reinterpret_cast<int *>(red + 64);
  int *qq = pp + (m > s ? m : s);
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    A[t] = Ain[t];
    V[t] = (t % s == t / s) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
      const double v = A[t] * A[t];
      tot += v;
      if (t % s != t / s) off += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (lane == 0) {
      red[wid] = off;
      red[32 + wid] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < nw; ++w) {
        a += red[w];
        b += red[32 + w];
      }
      red[0] = a;
      red[32] = b;
    }
    __syncthreads();
    const double off_s = red[0], tot_s = red[32];
    __syncthreads();
    if (off_s <= 1e-30 * tot_s || off_s == 0.0) break;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = threadIdx.x; k < m / 2; k += blockDim.x) {
        int p, q;
        if (k == 0) {
          p = r;
          q = m - 1;
        } else {
          p = (r + k) % (m - 1);
          q = (r - k + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, sv = 0.0;
        if (q < s) {
          const double apq = A[p + s * q];
          if (apq != 0.0) {
            const double theta = (A[q + s * q] - A[p + s * p]) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sv = t * c;
          }
        }
        cs[k] = c;
        sn[k] = sv;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < (m / 2) * s; t += blockDim.x) {  // rows: A <- J^T A
        const int k = t / s, col = t % s;
        const int p = pp[k], q = qq[k];
        if (q >= s) continue;
        const double c = cs[k], sv = sn[k];
        const double ap = A[p + s * col], aq = A[q + s * col];
        A[p + s * col] = c * ap - sv * aq;
        A[q + s * col] = sv * ap + c * aq;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < (m / 2) * s; t += blockDim.x) {  // columns: A <- A J, V <- V J
        const int k = t / s, row = t % s;
        const int p = pp[k], q = qq[k];
        if (q >= s) continue;
        const double c = cs[k], sv = sn[k];
        const double ap = A[row + s * p], aq = A[row + s * q];
        A[row + s * p] = c * ap - sv * aq;
        A[row + s * q] = sv * ap + c * aq;
        const double vp = V[row + s * p], vq = V[row + s * q];
        V[row + s * p] = c * vp - sv * vq;
        V[row + s * q] = sv * vp + c * vq;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int a = 0; a < s; ++a) pp[a] = a;
    for (int a = 0; a < s; ++a) {
      int best = a;
      for (int b = a + 1; b < s; ++b)
        if (A[pp[b] + s * pp[b]] > A[pp[best] + s * pp[best]]) best = b;
      const int t = pp[a];
      pp[a] = pp[best];
      pp[best] = t;
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < s; a += blockDim.x) lam_out[a] = A[pp[a] + s * pp[a]];
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    const int row = t % s, col = t / s;
    S_out[row + (long)s * col] = V[row + s * pp[col]];
  }
}

// The same cyclic Jacobi with its rotations applied in double-float on the FP32 pipe: A
// (and V while it fits) held as float pairs in shared memory, V in the global scratch Vg
// beyond that.  Each rotation's angle is computed in FP64 from the three entries it needs
// (joined from their pairs), its cosine and sine split into pairs, and every update
// x' = c x - s y, y' = s x + c y is a compensated (Dot2) two-term sum.  The off-diagonal
// test uses the leading floats' squares, in FP64.
__device__ __forceinline__ dfl rot_mix(dfl a, dfl x, dfl b, dfl y) {  // a x + b y
  Dot2 d;
  d.fma(a, x);
  d.fma(b, y);
  return d.result();
}

__global__ void __launch_bounds__(1024) k_jacobi_eig_sm_df(const double *__restrict__ Ain, int s, int m,
                                                           double *lam_out, double *S_out, int max_sweeps,
                                                           float2 *Vg) {
  extern __shared__ float2 shp[];
  // A (and V while it fits) with leading dimension la = s + 1: a rotation's row pass reads
  // A[p + la col] for consecutive col, which a stride of s would put in two banks only
  const int la = s + 1;
  float2 *A = shp, *V = Vg ? Vg : A + la * s;
  const int lv = Vg ? s : la;
  float2 *csp = A + la * s + (Vg ? 0 : la * s), *snp = csp + m / 2;
  double *red = reinterpret_cast<double *>(snp + m / 2);  // [2][32]
  int *pp = reinterpret_cast<int *>(red + 64);
  int *qq = pp + (m > s ? m : s);
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    const int row = t % s, col = t / s;
    const dfl a = d2df(Ain[t]);
    A[row + la * col] = make_float2(a.hi, a.lo);
    V[row + lv * col] = make_float2(row == col ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto J = [](float2 v) { return df2d(dfl{v.x, v.y}); };
  double off_prev = 0.0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
      const int row = t % s, col = t / s;
      const double v = J(A[row + la * col]);
      tot += v * v;
      if (row != col) off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (lane == 0) {
      red[wid] = off;
      red[32 + wid] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < nw; ++w) {
        a += red[w];
        b += red[32 + w];
      }
      red[0] = a;
      red[32] = b;
    }
    __syncthreads();
    const double off_s = red[0], tot_s = red[32];
    __syncthreads();
    // the pairs carry about 48 bits, so the off-diagonal mass stops falling near
    // s (2^-48)^2 of the total: stop at 1e-26 of it (1e-13 in norm), or once a sweep no longer
    // halves it (the rounding floor; the sweeps before it converge quadratically)
    if (off_s <= 1e-26 * tot_s || off_s == 0.0 || (sweep >= 3 && off_s > 0.5 * off_prev)) break;
    off_prev = off_s;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = threadIdx.x; k < m / 2; k += blockDim.x) {
        int p, q;
        if (k == 0) {
          p = r;
          q = m - 1;
        } else {
          p = (r + k) % (m - 1);
          q = (r - k + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, sv = 0.0;
        if (q < s) {
          const double apq = J(A[p + la * q]);
          if (apq != 0.0) {
            const double theta = (J(A[q + la * q]) - J(A[p + la * p])) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sv = t * c;
          }
        }
        const dfl cd = d2df(c), sd = d2df(sv);
        csp[k] = make_float2(cd.hi, cd.lo);
        snp[k] = make_float2(sd.hi, sd.lo);
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < (m / 2) * s; t += blockDim.x) {  // rows: A <- J^T A
        const int k = t / s, col = t % s;
        const int p = pp[k], q = qq[k];
        if (q >= s) continue;
        const dfl c{csp[k].x, csp[k].y}, sn{snp[k].x, snp[k].y}, msn{-snp[k].x, -snp[k].y};
        const float2 ap2 = A[p + la * col], aq2 = A[q + la * col];
        const dfl ap{ap2.x, ap2.y}, aq{aq2.x, aq2.y};
        const dfl np_ = rot_mix(c, ap, msn, aq), nq = rot_mix(sn, ap, c, aq);
        A[p + la * col] = make_float2(np_.hi, np_.lo);
        A[q + la * col] = make_float2(nq.hi, nq.lo);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < (m / 2) * s; t += blockDim.x) {  // columns: A <- A J, V <- V J
        const int k = t / s, row = t % s;
        const int p = pp[k], q = qq[k];
        if (q >= s) continue;
        const dfl c{csp[k].x, csp[k].y}, sn{snp[k].x, snp[k].y}, msn{-snp[k].x, -snp[k].y};
        const float2 ap2 = A[row + la * p], aq2 = A[row + la * q];
        const dfl ap{ap2.x, ap2.y}, aq{aq2.x, aq2.y};
        const dfl np_ = rot_mix(c, ap, msn, aq), nq = rot_mix(sn, ap, c, aq);
        A[row + la * p] = make_float2(np_.hi, np_.lo);
        A[row + la * q] = make_float2(nq.hi, nq.lo);
        const float2 vp2 = V[row + lv * p], vq2 = V[row + lv * q];
        const dfl vp{vp2.x, vp2.y}, vq{vq2.x, vq2.y};
        const dfl nvp = rot_mix(c, vp, msn, vq), nvq = rot_mix(sn, vp, c, vq);
        V[row + lv * p] = make_float2(nvp.hi, nvp.lo);
        V[row + lv * q] = make_float2(nvq.hi, nvq.lo);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int a = 0; a < s; ++a) pp[a] = a;
    for (int a = 0; a < s; ++a) {
      int best = a;
      for (int b = a + 1; b < s; ++b)
        if (J(A[pp[b] * (la + 1)]) > J(A[pp[best] * (la + 1)])) best = b;
      const int t = pp[a];
      pp[a] = pp[best];
      pp[best] = t;
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < s; a += blockDim.x) lam_out[a] = J(A[pp[a] * (la + 1)]);
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    const int row = t % s, col = t / s;
    S_out[row + (long)s * col] = J(V[row + lv * pp[col]]);
  }
}

int small_symeig(hp_problem *P, const double *T, int s, double *lambda, double *S) {
  const int m = s + (s & 1);
  if (s <= JS_MAX_A && P->refine_df != 0) {  // double-float rotations (same layouts, pairs for doubles)
    const bool v_shared = s <= JS_MAX;
    float2 *Vg = nullptr;
    if (!v_shared) {
      HP_TRY(P->vtmp[3].ensure(sizeof(float2) * (size_t)s * s));
      Vg = P->vtmp[3].as<float2>();
    }
    const size_t shm = sizeof(float2) * ((v_shared ? 2 : 1) * (size_t)(s + 1) * s + m) + sizeof(double) * 64 +
                       sizeof(int) * 2 * (size_t)std::max(m, s);
    static std::atomic<unsigned long long> attr_df{0};
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !(attr_df.load(std::memory_order_acquire) & (1ull << dev))) {
      const size_t cap = std::max(sizeof(float2) * (2 * (JS_MAX + 1) * JS_MAX + JS_MAX + 1) + sizeof(double) * 64 +
                                      sizeof(int) * 2 * (JS_MAX + 1),
                                  sizeof(float2) * ((JS_MAX_A + 1) * JS_MAX_A + JS_MAX_A) + sizeof(double) * 64 +
                                      sizeof(int) * 2 * JS_MAX_A);
      HP_CUDA(cudaFuncSetAttribute(k_jacobi_eig_sm_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
      attr_df.fetch_or(1ull << dev, std::memory_order_release);
    }
    k_jacobi_eig_sm_df<<<1, 1024, shm, P->st>>>(T, s, m, lambda, S, 60, Vg);
    count_launch();
    return cuda_check(cudaGetLastError(), "small_symeig");
  }
  if (s <= JS_MAX_A) {
    const bool v_shared = s <= JS_MAX;
    double *Vg = nullptr;
    if (!v_shared) {
      HP_TRY(P->vtmp[3].ensure(sizeof(double) * (size_t)s * s));
      Vg = P->vtmp[3].as<double>();
    }
    const size_t shm = sizeof(double) * ((v_shared ? 2 : 1) * (size_t)s * s + m + 64) +
                       sizeof(int) * 2 * (size_t)std::max(m, s);
    static std::atomic<unsigned long long> attr_set{0};  // once per device: the largest size either layout needs
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !(attr_set.load(std::memory_order_acquire) & (1ull << dev))) {
      const size_t cap = std::max(sizeof(double) * (2 * JS_MAX * JS_MAX + JS_MAX + 1 + 64) +
                                      sizeof(int) * 2 * (JS_MAX + 1),
                                  sizeof(double) * (JS_MAX_A * JS_MAX_A + JS_MAX_A + 64) +
                                      sizeof(int) * 2 * JS_MAX_A);
      HP_CUDA(cudaFuncSetAttribute(k_jacobi_eig_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
      attr_set.fetch_or(1ull << dev, std::memory_order_release);
    }
    k_jacobi_eig_sm<<<1, 1024, shm, P->st>>>(T, s, m, lambda, S, 60, Vg);
    count_launch();
    return cuda_check(cudaGetLastError(), "small_symeig");
  }
  HP_TRY(P->vtmp[3].ensure(sizeof(double) * 2 * (size_t)s * s));
  double *A = P->vtmp[3].as<double>(), *V = A + (size_t)s * s;
  HP_CUDA(cudaMemcpyAsync(A, T, sizeof(double) * s * s, cudaMemcpyDeviceToDevice, P->st));
  const size_t shm = sizeof(double) * m + sizeof(int) * std::max(m, s) * 2 + 64;
  k_jacobi_eig<<<1, 1024, shm, P->st>>>(A, V, s, m, lambda, S, 60);
  count_launch();
  return cuda_check(cudaGetLastError(), "small_symeig");
}

}  // namespace hp
