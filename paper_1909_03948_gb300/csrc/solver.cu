// solver.cu -- multi-right-hand-side geometric-multigrid PCG with FP64
// iterative refinement.
//
// Every PDE solve of the method (state, adjoint, incremental forward /
// adjoint, prior A, mass M) goes through solve_block(): s columns at once.
//   * Inner solver: PCG in T (float for HP_FP32_IR, double for HP_FP64_PLAIN)
//     with a symmetric V-cycle preconditioner (damped Jacobi smoothing, P1
//     interpolation / its transpose, Galerkin coarse operators, dense coarse
//     inverse) -- or diagonal scaling for the mass matrix.  alpha, beta and
//     the per-column convergence flags live on the device; converged columns
//     are frozen by alpha = 0.
//   * Outer loop: r = b - K x in FP64, inner solve on r / |r| in T, x += d.
//     Stops when every column has |r|/|b| <= rtol (FP64 residual).
//   * Inner products: per-column block partials in fixed order, the last
//     block to finish sums them (deterministic) and applies the scalar step
//     of CG (alpha, beta, convergence test) in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace hp {

void drop_graphs(hp_problem *P);

enum { FIN_STORE = 0, FIN_ALPHA = 1, FIN_RR = 2, FIN_BETA = 3, FIN_INIT = 4 };

struct Fin {
  double *part = nullptr;
  unsigned *cnt = nullptr;
  int kind = FIN_STORE;
  double *rz = nullptr, *alpha = nullptr, *beta = nullptr, *rr = nullptr, *bb = nullptr, *out = nullptr;
  int *active = nullptr;
  int *iter = nullptr;   // PCG iteration counter (FIN_BETA: beta = 0 on the first iteration)
  double tol2 = 0.0;
};

__device__ __forceinline__ void fin_apply(const Fin &f, int j, double s) {
  switch (f.kind) {
    case FIN_STORE: f.out[j] = s; break;
    case FIN_ALPHA: f.alpha[j] = (f.active[j] && s > 0.0) ? f.rz[j] / s : 0.0; break;
    case FIN_RR:
      f.rr[j] = s;
      f.active[j] = f.active[j] && (s > f.tol2 * f.bb[j]);
      break;
    case FIN_BETA: {
      const double b = (*f.iter > 0 && f.active[j] && f.rz[j] != 0.0) ? s / f.rz[j] : 0.0;
      f.beta[j] = b;
      f.rz[j] = s;
    } break;
    case FIN_INIT:
      f.bb[j] = s;
      f.rr[j] = s;
      f.active[j] = s > 0.0;
      break;
  }
}

// block partial -> last block sums the partials of column j in order
__device__ __forceinline__ void dot_finish(double acc, const Fin &f, int j) {
  __shared__ bool last;
  const double bs = block_sum<NT>(acc);
  if (threadIdx.x == 0) {
    f.part[(long)j * gridDim.x + blockIdx.x] = bs;
    __threadfence();
    const unsigned t = atomicAdd(&f.cnt[j], 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += NT) s += __ldcg(&f.part[(long)j * gridDim.x + b]);
    s = block_sum<NT>(s);
    if (threadIdx.x == 0) {
      f.cnt[j] = 0u;
      fin_apply(f, j, s);
    }
  }
}

// ---------------------------------------------------------------------------
// stencil kernels
// ---------------------------------------------------------------------------
template <typename T, int D, bool FULL>
__device__ __forceinline__ T stencil_row(const GridDesc &g, const T *__restrict__ diag, const T *__restrict__ c,
                                         const T *__restrict__ x, long i, const int v[3]) {
  T acc = diag[i] * x[i];
  constexpr int NF = FULL ? (1 << D) - 1 : D;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int b = FULL ? f + 1 : (1 << f);
    bool fw = true, bw = true;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if ((b >> a) & 1) {
        fw = fw && (v[a] < g.N);
        bw = bw && (v[a] > 0);
      }
    const long off = mask_offset(g, b);
    if (fw) acc += c[(long)f * g.n + i] * x[i + off];
    if (bw) acc += c[(long)f * g.n + i - off] * x[i - off];
  }
  return acc;
}

enum { M_APPLY = 0, M_APPLY_DOT = 1, M_RESID = 2, M_JACOBI = 3, M_JACOBI_DOT = 4 };

template <typename T, int D, bool FULL, int MODE>
__global__ void __launch_bounds__(NT) k_stencil(GridDesc g, const T *__restrict__ diag, const T *__restrict__ invdiag,
                                                const T *__restrict__ c, const T *__restrict__ X, long ldx,
                                                const T *__restrict__ B, long ldb, T *__restrict__ Y, long ldy,
                                                T omega, Fin fin) {
  const int j = blockIdx.y;
  const T *x = X + ldx * j;
  const T *b = B ? B + ldb * j : nullptr;
  T *y = Y + ldy * j;
  T acc = T(0);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    const T sx = stencil_row<T, D, FULL>(g, diag, c, x, i, v);
    T out;
    if (MODE == M_APPLY || MODE == M_APPLY_DOT) {
      out = sx;
      if (MODE == M_APPLY_DOT) acc += x[i] * out;
    } else if (MODE == M_RESID) {
      out = b[i] - sx;
    } else {
      const T bi = b[i];
      out = x[i] + omega * invdiag[i] * (bi - sx);
      if (MODE == M_JACOBI_DOT) acc += bi * out;
    }
    y[i] = out;
  }
  if (MODE == M_APPLY_DOT || MODE == M_JACOBI_DOT) dot_finish((double)acc, fin, j);
}

template <typename T>
__global__ void k_jacobi0(long n, const T *__restrict__ invdiag, const T *__restrict__ B, long ldb, T *__restrict__ Y,
                          long ldy, T omega, Fin fin, int with_dot) {
  const int j = blockIdx.y;
  T acc = T(0);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T bi = B[ldb * j + i];
    const T z = omega * invdiag[i] * bi;
    Y[ldy * j + i] = z;
    acc += bi * z;
  }
  if (with_dot) dot_finish((double)acc, fin, j);
}

template <typename T, int D>
__global__ void k_restrict(GridDesc gf, GridDesc gc, const T *__restrict__ rf, long ldf, T *__restrict__ rc, long ldc,
                           int zero_dirichlet) {
  const int j = blockIdx.y;
  const T *r = rf + ldf * j;
  for (long I = blockIdx.x * (long)blockDim.x + threadIdx.x; I < gc.n; I += (long)gridDim.x * blockDim.x) {
    int J[3];
    node_coords<D>(gc, I, J);
    T out;
    if (zero_dirichlet && (J[D - 1] == 0 || J[D - 1] == gc.N)) {
      out = T(0);
    } else {
      const long f0 = 2 * (long)J[0] + (long)gf.np * (2 * (long)J[1] + (D == 3 ? (long)gf.np * 2 * J[2] : 0));
      T acc = r[f0];
#pragma unroll
      for (int b = 1; b < (1 << D); ++b) {
        bool fw = true, bw = true;
#pragma unroll
        for (int a = 0; a < D; ++a)
          if ((b >> a) & 1) {
            fw = fw && (J[a] < gc.N);
            bw = bw && (J[a] > 0);
          }
        const long off = mask_offset(gf, b);
        if (fw) acc += T(0.5) * r[f0 + off];
        if (bw) acc += T(0.5) * r[f0 - off];
      }
      out = acc;
    }
    rc[ldc * j + I] = out;
  }
}

template <typename T, int D>
__global__ void k_prolong_add(GridDesc gf, GridDesc gc, const T *__restrict__ ec, long ldc, T *__restrict__ ef,
                              long ldf) {
  const int j = blockIdx.y;
  const T *e = ec + ldc * j;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < gf.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(gf, i, v);
    int I[3] = {v[0] >> 1, v[1] >> 1, v[2] >> 1};
    const int b = (v[0] & 1) | ((v[1] & 1) << 1) | ((v[2] & 1) << 2);
    const long ic = I[0] + (long)gc.np * (I[1] + (long)gc.np * I[2]);
    T val = e[ic];
    if (b) val = T(0.5) * (val + e[ic + mask_offset(gc, b)]);
    ef[ldf * j + i] += val;
  }
}

template <typename T>
__global__ void k_coarse_apply(const T *__restrict__ inv, int nc, const T *__restrict__ R, long ldr, T *__restrict__ E,
                               long lde) {
  extern __shared__ unsigned char smem_raw[];
  T *r = reinterpret_cast<T *>(smem_raw);
  const int j = blockIdx.x;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) r[k] = R[ldr * j + k];
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    T acc = T(0);
    for (int k = 0; k < nc; ++k) acc += inv[(long)k * nc + i] * r[k];
    E[lde * j + i] = acc;
  }
}

template <typename T>
__global__ void k_cg_update(long n, const T *__restrict__ p, const T *__restrict__ q, T *__restrict__ x,
                            T *__restrict__ r, long ld, const double *__restrict__ alpha, Fin fin) {
  const int j = blockIdx.y;
  const T a = (T)alpha[j];
  T acc = T(0);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long o = ld * j + i;
    x[o] += a * p[o];
    const T rn = r[o] - a * q[o];
    r[o] = rn;
    acc += rn * rn;
  }
  dot_finish((double)acc, fin, j);
}

template <typename T>
__global__ void k_p_update(long n, const T *__restrict__ z, T *__restrict__ p, long ld, const double *__restrict__ beta) {
  const int j = blockIdx.y;
  const T b = (T)beta[j];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long o = ld * j + i;
    p[o] = z[o] + b * p[o];
  }
}

// End of a PCG iteration: count it and decide whether another one runs.  In
// graph mode the decision drives the device-side while loop.
__global__ void k_pcg_cond(const int *__restrict__ active, int s, int *iter, int maxit, int bump,
                           cudaGraphConditionalHandle h, int use_handle) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < s; j += blockDim.x)
    if (active[j]) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int it = *iter + bump;
    *iter = it;
    if (use_handle) cudaGraphSetConditional(h, (any && it < maxit) ? 1u : 0u);
  }
}

template <typename T>
__global__ void k_selfdot(long n, const T *__restrict__ r, long ld, Fin fin) {
  const int j = blockIdx.y;
  T acc = T(0);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T v = r[ld * j + i];
    acc += v * v;
  }
  dot_finish((double)acc, fin, j);
}

// r_T = scale * r64 ; (scale 0 for converged columns)
template <typename T>
__global__ void k_to_inner(long n, const double *__restrict__ R, long ldr, const double *__restrict__ scale,
                           T *__restrict__ rt, long ldt) {
  const int j = blockIdx.y;
  const double sc = scale[j];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    rt[ldt * j + i] = (T)(sc * R[ldr * j + i]);
}

// X += d / scale  (skip columns with scale 0)
template <typename T>
__global__ void k_accum(long n, const T *__restrict__ d, long ldd, const double *__restrict__ scale,
                        double *__restrict__ X, long ldx) {
  const int j = blockIdx.y;
  const double sc = scale[j];
  if (sc == 0.0) return;
  const double inv = 1.0 / sc;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    X[ldx * j + i] += inv * (double)d[ldd * j + i];
}

// ---------------------------------------------------------------------------
// profiling: a pair of events around selected launches (off by default)
// ---------------------------------------------------------------------------
int prof_start(hp_problem *P, int id) {
  if (!P->prof_on || id < 0) return -1;
  const size_t r = P->prof_used;
  while (P->prof_ev.size() < 2 * (r + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    P->prof_ev.push_back(e);
  }
  if (P->prof_id.size() < r + 1) P->prof_id.resize(r + 1);
  P->prof_id[r] = -1;  // open
  cudaEventRecord(P->prof_ev[2 * r], P->st);
  P->prof_used = r + 1;
  P->prof_id[r] = -(id + 2);
  return (int)r;
}

void prof_stop(hp_problem *P, int rec) {
  if (rec < 0) return;
  cudaEventRecord(P->prof_ev[2 * rec + 1], P->st);
  P->prof_id[rec] = -P->prof_id[rec] - 2;  // closed: store the id
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename T> static const Stencil<T> &stencil_of(const hp_problem *P, OpKind op, int l);
template <> const Stencil<float> &stencil_of<float>(const hp_problem *P, OpKind op, int l) {
  return op == OP_K ? P->lv[l].K32 : (op == OP_A ? P->lv[l].A32 : P->M32);
}
template <> const Stencil<double> &stencil_of<double>(const hp_problem *P, OpKind op, int l) {
  return op == OP_K ? P->lv[l].K64 : (op == OP_A ? P->lv[l].A64 : P->M64);
}
template <typename T> static const T *coarse_inv(const hp_problem *P, OpKind op);
template <> const float *coarse_inv<float>(const hp_problem *P, OpKind op) {
  return op == OP_K ? P->cK.inv32 : P->cA.inv32;
}
template <> const double *coarse_inv<double>(const hp_problem *P, OpKind op) {
  return op == OP_K ? P->cK.inv64 : P->cA.inv64;
}

template <typename T, int MODE>
static void stencil_launch(const GridDesc &g, const Stencil<T> &S, const T *X, long ldx, const T *B, long ldb, T *Y,
                           long ldy, int s, T omega, const Fin &fin, cudaStream_t st) {
  dim3 grid(blocks_for(g.n, s), s);
  if (g.dim == 2) {
    if (S.full)
      k_stencil<T, 2, true, MODE><<<grid, NT, 0, st>>>(g, S.diag, S.invdiag, S.c, X, ldx, B, ldb, Y, ldy, omega, fin);
    else
      k_stencil<T, 2, false, MODE><<<grid, NT, 0, st>>>(g, S.diag, S.invdiag, S.c, X, ldx, B, ldb, Y, ldy, omega, fin);
  } else {
    if (S.full)
      k_stencil<T, 3, true, MODE><<<grid, NT, 0, st>>>(g, S.diag, S.invdiag, S.c, X, ldx, B, ldb, Y, ldy, omega, fin);
    else
      k_stencil<T, 3, false, MODE><<<grid, NT, 0, st>>>(g, S.diag, S.invdiag, S.c, X, ldx, B, ldb, Y, ldy, omega, fin);
  }
  count_launch();
}

template <typename T>
void launch_stencil_apply(const hp_problem *P, const GridDesc &g, const Stencil<T> &S, const T *X, long ldx, T *Y,
                          long ldy, int s, cudaStream_t st) {
  stencil_launch<T, M_APPLY>(g, S, X, ldx, nullptr, 0, Y, ldy, s, T(0), Fin{}, st);
}
template void launch_stencil_apply<double>(const hp_problem *, const GridDesc &, const Stencil<double> &,
                                           const double *, long, double *, long, int, cudaStream_t);
template void launch_stencil_apply<float>(const hp_problem *, const GridDesc &, const Stencil<float> &, const float *,
                                          long, float *, long, int, cudaStream_t);

static long padded(long n) { return (n + 63) / 64 * 64; }

template <typename T> static BlockWS<T> &ws_of(hp_problem *P);
template <> BlockWS<float> &ws_of<float>(hp_problem *P) { return P->w32; }
template <> BlockWS<double> &ws_of<double>(hp_problem *P) { return P->w64; }

template <typename T> static int ensure_ws(hp_problem *P, int s) {
  BlockWS<T> &W = ws_of<T>(P);
  if (W.scap >= s) return 0;
  W.ldn = padded(P->n);
  const size_t blk = sizeof(T) * (size_t)W.ldn * s;
  HP_TRY(W.x.ensure(blk));
  HP_TRY(W.r.ensure(blk));
  HP_TRY(W.z.ensure(blk));
  HP_TRY(W.p.ensure(blk));
  HP_TRY(W.q.ensure(blk));
  HP_TRY(W.lb[0].ensure(blk));
  for (int l = 1; l < P->L; ++l) {
    const size_t b = sizeof(T) * (size_t)padded(P->lv[l].g.n) * s;
    HP_TRY(W.lr[l].ensure(b));
    HP_TRY(W.la[l].ensure(b));
    HP_TRY(W.lb[l].ensure(b));
  }
  W.scap = s;
  drop_graphs(P);  // captured graphs hold the old workspace pointers
  return 0;
}

void free_scalars_host(hp_problem *P) {
  ScalarWS &S = P->sc;
  for (void *p : {(void *)S.h_active, (void *)S.h_iter, (void *)S.h_rr, (void *)S.h_bb})
    if (p) cudaFreeHost(p);
  S.h_active = S.h_iter = nullptr;
  S.h_rr = S.h_bb = nullptr;
  S.hcap = 0;
}

int ensure_scalars(hp_problem *P, int s) {
  ScalarWS &S = P->sc;
  const int nbmax = blocks_for(P->n, 1);
  if (S.scap >= s && S.partial.bytes >= sizeof(double) * (size_t)nbmax * s) return 0;
  const size_t b = sizeof(double) * s;
  HP_TRY(S.rz.ensure(b));
  HP_TRY(S.pq.ensure(b));
  HP_TRY(S.rr.ensure(b));
  HP_TRY(S.bb.ensure(b));
  HP_TRY(S.alpha.ensure(b));
  HP_TRY(S.beta.ensure(b));
  HP_TRY(S.scale.ensure(b));
  HP_TRY(S.active.ensure(sizeof(int) * std::max(s, 4)));
  HP_TRY(S.partial.ensure(sizeof(double) * (size_t)nbmax * s));
  HP_TRY(S.counter.ensure(sizeof(unsigned) * s));
  HP_TRY(S.iter.ensure(sizeof(int) * 4));
  HP_CUDA(cudaMemsetAsync(S.counter.p, 0, sizeof(unsigned) * s, P->st));
  if (S.hcap < s) {
    free_scalars_host(P);
    HP_CUDA(cudaMallocHost(&S.h_active, sizeof(int) * s));
    HP_CUDA(cudaMallocHost(&S.h_iter, sizeof(int) * 4));
    HP_CUDA(cudaMallocHost(&S.h_rr, sizeof(double) * s));
    HP_CUDA(cudaMallocHost(&S.h_bb, sizeof(double) * s));
    S.hcap = s;
  }
  drop_graphs(P);  // captured graphs hold the old scalar pointers
  S.scap = s;
  return 0;
}

static Fin make_fin(hp_problem *P, int kind, double tol2 = 0.0, double *out = nullptr) {
  Fin f;
  f.part = P->sc.partial.as<double>();
  f.cnt = P->sc.counter.as<unsigned>();
  f.kind = kind;
  f.rz = P->sc.rz.as<double>();
  f.alpha = P->sc.alpha.as<double>();
  f.beta = P->sc.beta.as<double>();
  f.rr = P->sc.rr.as<double>();
  f.bb = P->sc.bb.as<double>();
  f.active = P->sc.active.as<int>();
  f.iter = P->sc.iter.as<int>();
  f.tol2 = tol2;
  f.out = out;
  return f;
}

// Preconditioner z = M^{-1} r with the fused <r, z> -> fin.
template <typename T>
static void precondition(hp_problem *P, OpKind op, int s, const T *r0, T *z0, const Fin &fin) {
  BlockWS<T> &W = ws_of<T>(P);
  cudaStream_t st = P->st;
  const T om = (T)P->omega;
  if (op == OP_M) {  // Jacobi
    const Stencil<T> &S = stencil_of<T>(P, op, 0);
    k_jacobi0<T><<<dim3(blocks_for(P->n, s), s), NT, 0, st>>>(P->n, S.invdiag, r0, W.ldn, z0, W.ldn, T(1), fin, 1);
    count_launch();
    return;
  }
  const int L = P->L;
  if (L == 1) {  // the coarse solve is the whole preconditioner; the caller forms <r, z>
    const int nc = (int)P->lv[0].g.n;
    k_coarse_apply<T><<<s, 256, sizeof(T) * nc, st>>>(coarse_inv<T>(P, op), nc, r0, W.ldn, z0, W.ldn);
    count_launch();
    return;
  }
  const T *rl[HP_MAXL];
  T *ea[HP_MAXL], *eb[HP_MAXL];
  long ld[HP_MAXL];
  rl[0] = r0;
  ea[0] = z0;
  eb[0] = W.lb[0].template as<T>();
  ld[0] = W.ldn;
  for (int l = 1; l < L; ++l) {
    rl[l] = W.lr[l].template as<T>();
    ea[l] = W.la[l].template as<T>();
    eb[l] = W.lb[l].template as<T>();
    ld[l] = padded(P->lv[l].g.n);
  }
  T *cur[HP_MAXL], *oth[HP_MAXL];
  const Fin nofin{};
  for (int l = 0; l + 1 < L; ++l) {
    const GridDesc &g = P->lv[l].g;
    const Stencil<T> &S = stencil_of<T>(P, op, l);
    T *c = eb[l], *o = ea[l];
    k_jacobi0<T><<<dim3(blocks_for(g.n, s), s), NT, 0, st>>>(g.n, S.invdiag, rl[l], ld[l], c, ld[l], om, nofin, 0);
    count_launch();
    for (int k = 1; k < P->nu; ++k) {
      const int pr = prof_start(P, l == 0 ? PROF_SMOOTH : -1);
      stencil_launch<T, M_JACOBI>(g, S, c, ld[l], rl[l], ld[l], o, ld[l], s, om, nofin, st);
      prof_stop(P, pr);
      std::swap(c, o);
    }
    {
      const int pr = prof_start(P, l == 0 ? PROF_RESID_MG : -1);
      stencil_launch<T, M_RESID>(g, S, c, ld[l], rl[l], ld[l], o, ld[l], s, om, nofin, st);
      prof_stop(P, pr);
    }
    const GridDesc &gc = P->lv[l + 1].g;
    dim3 grid(blocks_for(gc.n, s), s);
    T *rc = const_cast<T *>(rl[l + 1]);
    if (g.dim == 2)
      k_restrict<T, 2><<<grid, NT, 0, st>>>(g, gc, o, ld[l], rc, ld[l + 1], op == OP_K);
    else
      k_restrict<T, 3><<<grid, NT, 0, st>>>(g, gc, o, ld[l], rc, ld[l + 1], op == OP_K);
    count_launch();
    cur[l] = c;
    oth[l] = o;
  }
  {
    const int lc = L - 1;
    const int nc = (int)P->lv[lc].g.n;
    k_coarse_apply<T><<<s, 256, sizeof(T) * nc, st>>>(coarse_inv<T>(P, op), nc, rl[lc], ld[lc], ea[lc], ld[lc]);
    count_launch();
    cur[lc] = ea[lc];
  }
  for (int l = L - 2; l >= 0; --l) {
    const GridDesc &g = P->lv[l].g, &gc = P->lv[l + 1].g;
    const Stencil<T> &S = stencil_of<T>(P, op, l);
    dim3 grid(blocks_for(g.n, s), s);
    if (g.dim == 2)
      k_prolong_add<T, 2><<<grid, NT, 0, st>>>(g, gc, cur[l + 1], ld[l + 1], cur[l], ld[l]);
    else
      k_prolong_add<T, 3><<<grid, NT, 0, st>>>(g, gc, cur[l + 1], ld[l + 1], cur[l], ld[l]);
    count_launch();
    T *c = cur[l], *o = oth[l];
    for (int k = 0; k < P->nu; ++k) {
      const int pr = prof_start(P, l == 0 ? PROF_SMOOTH : -1);
      if (l == 0 && k == P->nu - 1)
        stencil_launch<T, M_JACOBI_DOT>(g, S, c, ld[l], rl[l], ld[l], o, ld[l], s, om, fin, st);
      else
        stencil_launch<T, M_JACOBI>(g, S, c, ld[l], rl[l], ld[l], o, ld[l], s, om, nofin, st);
      prof_stop(P, pr);
      std::swap(c, o);
    }
    cur[l] = c;
  }
}

template <typename T>
__global__ void k_dot2(long n, const T *__restrict__ a, const T *__restrict__ b, long ld, Fin fin) {
  const int j = blockIdx.y;
  T acc = T(0);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    acc += a[ld * j + i] * b[ld * j + i];
  dot_finish((double)acc, fin, j);
}

// PCG on W.r (overwritten) -> W.x.
//   init:  x = 0, p = 0, bb = rr = <r, r>, active = bb > 0, iter = 0
//   body:  z = M r, beta = <r,z>/rz (0 at iter 0), p = z + beta p,
//          q = K p, alpha = rz/<p,q>, x += alpha p, r -= alpha q, rr = <r,r>,
//          active &= rr > tol^2 bb, iter += 1; repeat while any active and iter < maxit.
template <typename T>
static void pcg_init(hp_problem *P, OpKind op, int s, cudaGraphConditionalHandle h, int use_handle, int maxit) {
  BlockWS<T> &W = ws_of<T>(P);
  cudaStream_t st = P->st;
  const long n = P->n, ld = W.ldn;
  dim3 grid(blocks_for(n, s), s);
  cudaMemsetAsync(W.x.p, 0, sizeof(T) * ld * s, st);
  cudaMemsetAsync(W.p.p, 0, sizeof(T) * ld * s, st);
  cudaMemsetAsync(P->sc.iter.p, 0, sizeof(int), st);
  k_selfdot<T><<<grid, NT, 0, st>>>(n, W.r.template as<T>(), ld, make_fin(P, FIN_INIT));
  k_pcg_cond<<<1, 256, 0, st>>>(P->sc.active.as<int>(), s, P->sc.iter.as<int>(), maxit, 0, h, use_handle);
  count_launch(2);
}

template <typename T>
static void pcg_body(hp_problem *P, OpKind op, int s, double tol2, cudaGraphConditionalHandle h, int use_handle,
                     int maxit) {
  BlockWS<T> &W = ws_of<T>(P);
  cudaStream_t st = P->st;
  const long n = P->n, ld = W.ldn;
  T *x = W.x.template as<T>(), *r = W.r.template as<T>(), *z = W.z.template as<T>();
  T *p = W.p.template as<T>(), *q = W.q.template as<T>();
  const GridDesc &g0 = P->lv[0].g;
  const Stencil<T> &S0 = stencil_of<T>(P, op, 0);
  dim3 grid(blocks_for(n, s), s);
  int pr = prof_start(P, PROF_VCYCLE);
  precondition<T>(P, op, s, r, z, make_fin(P, FIN_BETA));
  prof_stop(P, pr);
  if (op != OP_M && P->L == 1) {
    k_dot2<T><<<grid, NT, 0, st>>>(n, r, z, ld, make_fin(P, FIN_BETA));
    count_launch();
  }
  k_p_update<T><<<grid, NT, 0, st>>>(n, z, p, ld, P->sc.beta.as<double>());
  count_launch();
  pr = prof_start(P, PROF_MATVEC);
  stencil_launch<T, M_APPLY_DOT>(g0, S0, p, ld, nullptr, 0, q, ld, s, T(0), make_fin(P, FIN_ALPHA), st);
  prof_stop(P, pr);
  pr = prof_start(P, PROF_CG_UPDATE);
  k_cg_update<T><<<grid, NT, 0, st>>>(n, p, q, x, r, ld, P->sc.alpha.as<double>(), make_fin(P, FIN_RR, tol2));
  prof_stop(P, pr);
  k_pcg_cond<<<1, 256, 0, st>>>(P->sc.active.as<int>(), s, P->sc.iter.as<int>(), maxit, 1, h, use_handle);
  count_launch(2);
}

struct PcgGraph {
  int op, fp32, s, maxit;
  double tol;
  cudaGraphExec_t exec;
  int nkernels;
};
static std::vector<std::pair<hp_problem *, PcgGraph>> g_graphs;

void drop_graphs(hp_problem *P) {
  for (auto it = g_graphs.begin(); it != g_graphs.end();) {
    if (it->first == P) {
      cudaGraphExecDestroy(it->second.exec);
      it = g_graphs.erase(it);
    } else {
      ++it;
    }
  }
}

// Captures init + a conditional WHILE node whose body is one PCG iteration.
template <typename T>
static int build_graph(hp_problem *P, OpKind op, int s, double tol, int maxit, PcgGraph *out) {
  if (!P->cap) HP_CUDA(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
  cudaStream_t saved = P->st;
  const bool saved_prof = P->prof_on;
  P->prof_on = false;
  P->st = P->cap;
  const unsigned long long l0 = g_launches;
  cudaGraph_t g = nullptr;
  int rc = 0;
  auto fail = [&](cudaError_t e, const char *w) {
    rc = cuda_check(e, w);
    P->st = saved;
    P->prof_on = saved_prof;
    if (g) cudaGraphDestroy(g);
    return rc;
  };
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return fail(e, "cudaGraphCreate");
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(e, "cudaGraphConditionalHandleCreate");
  e = cudaStreamBeginCaptureToGraph(P->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail(e, "capture init");
  pcg_init<T>(P, op, s, h, 1, maxit);
  e = cudaStreamEndCapture(P->cap, &g);
  if (e != cudaSuccess) return fail(e, "end capture init");
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  cudaGraphNode_t leaf = nullptr;
  for (auto nd : nodes) {
    size_t nd_out = 0;
    cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nd_out);
    if (nd_out == 0) leaf = nd;
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  e = cudaGraphAddNode(&cn, g, leaf ? &leaf : nullptr, nullptr, leaf ? 1 : 0, &cp);
  if (e != cudaSuccess) return fail(e, "add conditional node");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(P->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail(e, "capture body");
  pcg_body<T>(P, op, s, tol * tol, h, 1, maxit);
  e = cudaStreamEndCapture(P->cap, &body);
  if (e != cudaSuccess) return fail(e, "end capture body");
  cudaGraphExec_t ex;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) return fail(e, "instantiate");
  cudaGraphDestroy(g);
  P->st = saved;
  P->prof_on = saved_prof;
  g_launches = l0;  // captured launches are counted when the graph runs
  *out = PcgGraph{(int)op, sizeof(T) == 4, s, maxit, tol, ex, 0};
  return 0;
}

template <typename T>
static int pcg(hp_problem *P, OpKind op, int s, double rtol, int maxit, int *its) {
  cudaStream_t st = P->st;
  int *h_it = P->sc.h_iter;
  if (P->use_graphs && !P->prof_on) {
    PcgGraph *G = nullptr;
    for (auto &pg : g_graphs)
      if (pg.first == P && pg.second.op == (int)op && pg.second.fp32 == (sizeof(T) == 4) && pg.second.s == s &&
          pg.second.maxit == maxit && pg.second.tol == rtol)
        G = &pg.second;
    if (!G) {
      PcgGraph ng;
      HP_TRY(build_graph<T>(P, op, s, rtol, maxit, &ng));
      g_graphs.push_back({P, ng});
      G = &g_graphs.back().second;
    }
    HP_CUDA(cudaGraphLaunch(G->exec, st));
    HP_CUDA(cudaMemcpyAsync(h_it, P->sc.iter.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaStreamSynchronize(st));
    const int per_it = 12 + 7 * P->L;  // approximate kernels per iteration, for launch accounting
    count_launch((unsigned long long)(*h_it) * per_it + 3);
    *its = *h_it;
    return *h_it >= maxit ? HP_ERR_NOT_CONVERGED : 0;
  }
  const double tol2 = rtol * rtol;
  pcg_init<T>(P, op, s, 0, 0, maxit);
  int *hact = P->sc.h_active;
  for (;;) {
    pcg_body<T>(P, op, s, tol2, 0, 0, maxit);
    HP_CUDA(cudaMemcpyAsync(hact, P->sc.active.p, sizeof(int) * s, cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaMemcpyAsync(h_it, P->sc.iter.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaStreamSynchronize(st));
    int nact = 0;
    for (int j = 0; j < s; ++j) nact += hact[j] != 0;
    if (nact == 0 || *h_it >= maxit) break;
  }
  *its = *h_it;
  HP_CUDA(cudaGetLastError());
  return *h_it >= maxit ? HP_ERR_NOT_CONVERGED : 0;
}

int apply_op64(hp_problem *P, OpKind op, const double *X, long ldx, double *Y, long ldy, int s) {
  launch_stencil_apply<double>(P, P->lv[0].g, stencil_of<double>(P, op, 0), X, ldx, Y, ldy, s, P->st);
  return cuda_check(cudaGetLastError(), "apply");
}

// FP64 residual R = B - S X with per-column |R|^2 -> rr (host)
static int residual64(hp_problem *P, OpKind op, const double *B, long ldb, const double *X, long ldx, double *R,
                      long ldr, int s) {
  const int pr = prof_start(P, PROF_RESID64);
  stencil_launch<double, M_RESID>(P->lv[0].g, stencil_of<double>(P, op, 0), X, ldx, B, ldb, R, ldr, s, 0.0, Fin{},
                                  P->st);
  prof_stop(P, pr);
  HP_TRY(block_dot(P, R, ldr, R, ldr, P->n, s, P->sc.rr.as<double>()));
  return 0;
}

template <typename T>
static int ir_solve(hp_problem *P, OpKind op, const double *B, long ldb, double *X, long ldx, int s, double rtol,
                    double tol_in, hp_solve_stats *stats) {
  BlockWS<T> &W = ws_of<T>(P);
  cudaStream_t st = P->st;
  const long n = P->n;
  const long ld64 = padded(n);
  HP_TRY(P->r64.ensure(sizeof(double) * ld64 * s));
  HP_TRY(P->b64.ensure(sizeof(double) * ld64 * s));
  double *r64 = P->r64.as<double>(), *b64 = P->b64.as<double>();
  launch_copy(B, ldb, b64, ld64, n, s, st);
  if (op == OP_K) launch_zero_dirichlet(P, b64, ld64, s);
  launch_fill(X, ldx, n, s, 0.0, st);
  HP_TRY(block_dot(P, b64, ld64, b64, ld64, n, s, P->sc.bb.as<double>()));
  launch_copy(b64, ld64, r64, ld64, n, s, st);
  HP_TRY(block_dot(P, r64, ld64, r64, ld64, n, s, P->sc.rr.as<double>()));
  double *hrr = P->sc.h_rr, *hbb = P->sc.h_bb;
  HP_CUDA(cudaMemcpyAsync(hbb, P->sc.bb.p, sizeof(double) * s, cudaMemcpyDeviceToHost, st));
  std::vector<double> hscale(s);
  int total_its = 0, outer = 0, rc = 0;
  double worst = 0.0;
  for (outer = 0; outer <= P->max_outer; ++outer) {
    HP_CUDA(cudaMemcpyAsync(hrr, P->sc.rr.p, sizeof(double) * s, cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaStreamSynchronize(st));
    int nact = 0;
    worst = 0.0;
    for (int j = 0; j < s; ++j) {
      if (!std::isfinite(hrr[j])) return set_error(HP_ERR_NONFINITE, "non-finite residual in a PDE solve");
      const double rel = hbb[j] > 0 ? std::sqrt(hrr[j] / hbb[j]) : 0.0;
      worst = std::max(worst, rel);
      const bool done = hbb[j] == 0.0 || hrr[j] <= rtol * rtol * hbb[j];
      hscale[j] = done ? 0.0 : 1.0 / std::sqrt(hrr[j]);
      nact += !done;
    }
    if (nact == 0) break;
    if (outer == P->max_outer) {
      rc = HP_ERR_NOT_CONVERGED;
      break;
    }
    HP_CUDA(cudaMemcpyAsync(P->sc.scale.p, hscale.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
    dim3 grid(blocks_for(n, s), s);
    k_to_inner<T><<<grid, NT, 0, st>>>(n, r64, ld64, P->sc.scale.as<double>(), W.r.template as<T>(), W.ldn);
    count_launch();
    int its = 0;
    const int prc = pcg<T>(P, op, s, tol_in, P->max_iter, &its);
    total_its += its;
    k_accum<T><<<grid, NT, 0, st>>>(n, W.x.template as<T>(), W.ldn, P->sc.scale.as<double>(), X, ldx);
    count_launch();
    HP_TRY(residual64(P, op, b64, ld64, X, ldx, r64, ld64, s));
    if (prc == HP_ERR_NOT_CONVERGED && its >= P->max_iter) {
      // keep refining: a stalled inner solve still reduces the residual
    }
  }
  if (stats) {
    stats->iterations += total_its;
    stats->outer += outer;
    stats->solves += 1;
    stats->rel_res = std::max(stats->rel_res, worst);
  }
  if (rc) return set_error(rc, "PDE solve did not reach the requested tolerance");
  return cuda_check(cudaGetLastError(), "ir_solve");
}

int solve_block(hp_problem *P, OpKind op, const double *B, long ldb, double *X, long ldx, int s, double rtol,
                hp_solve_stats *st) {
  if (s <= 0) return 0;
  HP_TRY(ensure_scalars(P, s));
  if (P->precision == HP_FP64_PLAIN) {
    HP_TRY(ensure_ws<double>(P, s));
    return ir_solve<double>(P, op, B, ldb, X, ldx, s, rtol, 0.5 * rtol, st);
  }
  HP_TRY(ensure_ws<float>(P, s));
  return ir_solve<float>(P, op, B, ldb, X, ldx, s, rtol, P->inner_rtol, st);
}

}  // namespace hp
