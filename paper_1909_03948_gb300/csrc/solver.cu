// solver.cu -- multi-right-hand-side geometric-multigrid PCG with FP64
// iterative refinement.
//
// Every PDE solve of the method (state, adjoint, incremental forward /
// adjoint, prior A, mass M) goes through solve_block(): s columns at once.
//   * Inner solver: PCG in T (float for HP_FP32_IR, double for HP_FP64_PLAIN)
//     with a symmetric V-cycle preconditioner (polynomial smoothing: Chebyshev
//     weights on [lmax / alpha, lmax] by default, or damped Jacobi; P1
//     interpolation / its transpose, Galerkin coarse operators, dense coarse
//     inverse) -- or diagonal scaling for the mass matrix.  alpha, beta and
//     the per-column convergence flags live on the device; converged columns
//     are frozen by alpha = 0.  The iteration loop is a CUDA graph with a
//     device-side while node, so a solve costs one graph launch.
//   * Inner layout: columns are packed in groups of VW (VW = 4 for FP32 blocks:
//     [group][node][4], one 16-byte access per node covers 4 right-hand sides
//     and one coefficient load serves all 4; VW = 1 is plain column-major).
//   * Outer loop: r = b - K x in FP64 (column-major, the ABI layout), inner solve
//     on r / |r| in T, x += d.  Stops when every column has |r|/|b| <= rtol.
//   * Inner products: per-block partials (warp sums in T, block sums in FP64),
//     then one small kernel per product sums the partials of each column in a
//     fixed order (deterministic) and applies the scalar step of CG in FP64.
//   * Level stencils of 2D stiffness solves: one CTA per 32 x 16-node tile, its
//     data brought into shared memory by TMA bulk tensor copies (k_st_tile).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

#include <cuda.h>

#include "dfloat.cuh"
#include "internal.h"

namespace hp {

void drop_graphs(hp_problem *P);

constexpr int NB = 128;  // threads per block of the node kernels (4 warps)

enum { FIN_STORE = 0, FIN_ALPHA = 1, FIN_RR = 2, FIN_BETA = 3, FIN_INIT = 4 };

struct Fin {
  double *part = nullptr;
  unsigned *cnt = nullptr;
  int kind = FIN_STORE;
  double *rz = nullptr, *alpha = nullptr, *beta = nullptr, *rr = nullptr, *bb = nullptr, *out = nullptr;
  int *active = nullptr;
  int *iter = nullptr;  // PCG iteration counter (FIN_BETA: beta = 0 on the first iteration)
  const double *tol2col = nullptr;  // per-column squared relative tolerance (FIN_RR), else tol2
  const double *open = nullptr;     // FIN_INIT: columns with open[j] == 0 start inactive
  double tol2 = 0.0;
};

__device__ __forceinline__ void fin_apply(const Fin &f, int j, double s) {
  switch (f.kind) {
    case FIN_STORE: f.out[j] = s; break;
    case FIN_ALPHA: f.alpha[j] = (f.active[j] && s > 0.0) ? f.rz[j] / s : 0.0; break;
    case FIN_RR:
      f.rr[j] = s;
      f.active[j] = f.active[j] && (s > (f.tol2col ? f.tol2col[j] : f.tol2) * f.bb[j]);
      break;
    case FIN_BETA: {
      const double b = (*f.iter > 0 && f.active[j] && f.rz[j] != 0.0) ? s / f.rz[j] : 0.0;
      f.beta[j] = b;
      f.rz[j] = s;
    } break;
    case FIN_INIT:
      f.bb[j] = s;
      f.rr[j] = s;
      f.active[j] = s > 0.0 && (f.open == nullptr || f.open[j] != 0.0);
      break;
  }
}

// ---------------------------------------------------------------------------
// packs of VW values of one node (VW consecutive columns of a group)
// ---------------------------------------------------------------------------
template <typename T, int VW> struct Pack {
  T v[VW];
  __device__ __forceinline__ static Pack ld(const T *p) {
    Pack r;
    if constexpr (VW == 4 && sizeof(T) == 4) {
      const float4 t = *reinterpret_cast<const float4 *>(p);
      r.v[0] = t.x;
      r.v[1] = t.y;
      r.v[2] = t.z;
      r.v[3] = t.w;
    } else {
#pragma unroll
      for (int q = 0; q < VW; ++q) r.v[q] = p[q];
    }
    return r;
  }
  __device__ __forceinline__ void st(T *p) const {
    if constexpr (VW == 4 && sizeof(T) == 4) {
      *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int q = 0; q < VW; ++q) p[q] = v[q];
    }
  }
  __device__ __forceinline__ static Pack zero() {
    Pack r;
#pragma unroll
    for (int q = 0; q < VW; ++q) r.v[q] = T(0);
    return r;
  }
  __device__ __forceinline__ void axpy(T a, const Pack &x) {  // this += a x
#pragma unroll
    for (int q = 0; q < VW; ++q) v[q] = fmadd(a, x.v[q], v[q]);
  }
};

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Per-column dot partial of one block (NB threads) for the VW columns of group grp:
// warp sums in T, the 4 warp sums added in FP64, stored at part[col * nblk + blin].
// k_dot_finalize then sums the nblk partials of each column in a fixed order
// (deterministic, no atomics) and applies the CG scalar step.
template <typename T, int VW>
__device__ __forceinline__ void dot_partial(const Pack<T, VW> &acc, double *part, int grp, int s, unsigned blin,
                                            unsigned nblk) {
  __shared__ double sh[NB / 32][VW];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < VW; ++q) {
    const T w = warp_sum_t(acc.v[q]);
    if (lane == 0) sh[wy][q] = (double)w;
  }
  __syncthreads();
  if (threadIdx.x < VW) {
    const int q = threadIdx.x, col = grp * VW + q;
    if (col < s) {
      double bs = 0.0;
#pragma unroll
      for (int w = 0; w < NB / 32; ++w) bs += sh[w][q];
      part[(long)col * nblk + blin] = bs;
    }
  }
}

__global__ void k_dot_finalize(const double *__restrict__ part, unsigned nblk, Fin fin) {
  const int col = blockIdx.x;
  double sum = 0.0;
  for (unsigned b = threadIdx.x; b < nblk; b += NB) sum += part[(long)col * nblk + b];
  sum = block_sum<NB>(sum);
  if (threadIdx.x == 0) fin_apply(fin, col, sum);
}

static void dot_finalize(const Fin &fin, unsigned nblk, int s, cudaStream_t st) {
  k_dot_finalize<<<s, NB, 0, st>>>(fin.part, nblk, fin);
  count_launch();
}

// ---------------------------------------------------------------------------
// stencil kernels: one node per thread, 32 x-nodes per warp, rows over warps
// and blocks, column groups over blockIdx.z.  Element (node i, group g) of a
// block with group stride gs is at base + g*gs + i*VW.
// ---------------------------------------------------------------------------
enum { M_APPLY = 0, M_APPLY_DOT = 1, M_RESID = 2, M_JACOBI = 3, M_JACOBI_DOT = 4, M_JAC2 = 5, M_RESID_DOT = 6 };

template <typename T, int VW, int D, bool FULL, int MODE>
__global__ void __launch_bounds__(NB) k_st(GridDesc g, const T *__restrict__ diag, const T *__restrict__ invdiag,
                                           const T *__restrict__ c, const T *__restrict__ X, long gx,
                                           const T *__restrict__ B, long gb, T *__restrict__ Y, long gy, int s,
                                           T omega, T omega2, Fin fin) {
  using PK = Pack<T, VW>;
  const int lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * 32 + lane;
  const int nrows = D == 2 ? g.np : g.np * g.np;
  const int grp = blockIdx.z;
  constexpr bool DOT = (MODE == M_APPLY_DOT || MODE == M_JACOBI_DOT || MODE == M_RESID_DOT);
  PK acc = PK::zero();
  for (int row = blockIdx.y * (NB / 32) + (threadIdx.x >> 5); row < nrows; row += gridDim.y * (NB / 32)) {
    if (i0 >= g.np) break;
    const int v[3] = {i0, D == 2 ? row : row % g.np, D == 2 ? 0 : row / g.np};
    const long id = i0 + (long)g.np * row;
    const T *x = X + grp * gx;
    constexpr int NF = FULL ? (1 << D) - 1 : D;
    PK out;
    if (MODE == M_JAC2) {
      // two damped-Jacobi sweeps from zero: e1 = w1 D^-1 r, e2 = e1 + w2 D^-1 (r - S e1)
      const T wi = omega * invdiag[id], wi2 = omega2 * invdiag[id];
      const PK r = PK::ld(x + id * VW);
      PK e1c;
#pragma unroll
      for (int q = 0; q < VW; ++q) e1c.v[q] = wi * r.v[q];
      PK sx;
      const T dg = diag[id];
#pragma unroll
      for (int q = 0; q < VW; ++q) sx.v[q] = dg * e1c.v[q];
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
        if (fw) sx.axpy(c[(long)f * g.n + id] * omega * invdiag[id + off], PK::ld(x + (id + off) * VW));
        if (bw) sx.axpy(c[(long)f * g.n + id - off] * omega * invdiag[id - off], PK::ld(x + (id - off) * VW));
      }
#pragma unroll
      for (int q = 0; q < VW; ++q) out.v[q] = fmadd(wi2, r.v[q] - sx.v[q], e1c.v[q]);
    } else {
      const PK xc = PK::ld(x + id * VW);
      PK sx;
      const T dg = diag[id];
#pragma unroll
      for (int q = 0; q < VW; ++q) sx.v[q] = dg * xc.v[q];
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
        if (fw) sx.axpy(c[(long)f * g.n + id], PK::ld(x + (id + off) * VW));
        if (bw) sx.axpy(c[(long)f * g.n + id - off], PK::ld(x + (id - off) * VW));
      }
      if (MODE == M_APPLY || MODE == M_APPLY_DOT) {
        out = sx;
        if (DOT)
#pragma unroll
          for (int q = 0; q < VW; ++q) acc.v[q] = fmadd(xc.v[q], out.v[q], acc.v[q]);
      } else {
        const PK bb = PK::ld(B + grp * gb + id * VW);
        if (MODE == M_RESID || MODE == M_RESID_DOT) {
#pragma unroll
          for (int q = 0; q < VW; ++q) out.v[q] = bb.v[q] - sx.v[q];
          if (DOT)
#pragma unroll
            for (int q = 0; q < VW; ++q) acc.v[q] = fmadd(out.v[q], out.v[q], acc.v[q]);
        } else {
          const T wi = omega * invdiag[id];
#pragma unroll
          for (int q = 0; q < VW; ++q) out.v[q] = fmadd(wi, bb.v[q] - sx.v[q], xc.v[q]);
          if (DOT)
#pragma unroll
            for (int q = 0; q < VW; ++q) acc.v[q] = fmadd(bb.v[q], out.v[q], acc.v[q]);
        }
      }
    }
    out.st(Y + grp * gy + id * VW);
  }
  if (DOT) dot_partial<T, VW>(acc, fin.part, grp, s, blockIdx.x + gridDim.x * blockIdx.y, gridDim.x * gridDim.y);
}

// ---------------------------------------------------------------------------
// TMA-tiled stencil kernels (2D stiffness levels, FP32, 4 columns per node).
// One CTA per tile of TILE_X x TILE_Y nodes of one column group.  Thread 0 issues
// bulk tensor copies (cp.async.bulk.tensor) of the tile's x with a one-node halo,
// of its right-hand side and of the packed coefficients {diag, 1/diag, c_x, c_y}
// (also with the halo) into shared memory; all three complete on one mbarrier.  The
// CTA therefore has its whole working set in flight at once, where the row kernel
// above issues one row of loads per warp at a time and waits for each.  The last
// tile in x (in y) also takes the grid's final node (row), so every box is sized
// for TILE + 1 nodes plus the halo; copies that reach past the grid read zeros.
// The arithmetic is k_st's, operation for operation, on the same values.
// ---------------------------------------------------------------------------
constexpr int TL_NT = NB;                                   // 4 warps
constexpr int TLB_X = TILE_X + 3, TLB_Y = TILE_Y + 3;       // x / coefficient boxes
constexpr int TLR_X = TILE_X + 1, TLR_Y = TILE_Y + 1;       // right-hand-side box
constexpr unsigned TL_XBYTES = TLB_X * TLB_Y * 16u, TL_RBYTES = TLR_X * TLR_Y * 16u;
constexpr unsigned TL_OFF_R = (TL_XBYTES + 127u) / 128u * 128u;
constexpr unsigned TL_OFF_C = TL_OFF_R + (TL_RBYTES + 127u) / 128u * 128u;
constexpr unsigned TL_OFF_M = TL_OFF_C + (TL_XBYTES + 127u) / 128u * 128u;
constexpr unsigned TL_SMEM = TL_OFF_M + 16u + 128u;  // + alignment slack

// set by a tile kernel whose copies did not arrive within its wait limit
__device__ int g_tile_timeout;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// waits for phase 0 of the barrier for at most ~2^31 clocks (about a second)
__device__ __forceinline__ bool mbar_wait0(uint32_t bar) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

template <int MODE>
__global__ void __launch_bounds__(TL_NT) k_st_tile(const __grid_constant__ CUtensorMap mx,
                                                   const __grid_constant__ CUtensorMap mr,
                                                   const __grid_constant__ CUtensorMap mc, GridDesc g, int ntx,
                                                   int nty, float *__restrict__ Y, long gy, int s, float omega,
                                                   float omega2, Fin fin) {
  using PK = Pack<float, 4>;
  extern __shared__ __align__(128) unsigned char tl_smem_raw[];
  // the boxes start on 128-byte boundaries (the launch adds 128 bytes of slack)
  unsigned char *tl_smem = tl_smem_raw + ((128u - (smem_u32(tl_smem_raw) & 127u)) & 127u);
  const float *xs = reinterpret_cast<const float *>(tl_smem);
  const float *rs = reinterpret_cast<const float *>(tl_smem + TL_OFF_R);
  const float4 *cs = reinterpret_cast<const float4 *>(tl_smem + TL_OFF_C);
  const uint32_t bar = smem_u32(tl_smem + TL_OFF_M);
  constexpr bool HAS_B = (MODE == M_RESID || MODE == M_JACOBI || MODE == M_JACOBI_DOT);
  constexpr bool DOT = (MODE == M_APPLY_DOT || MODE == M_JACOBI_DOT);
  const int tile = blockIdx.x, grp = blockIdx.y;
  const int tx = tile % ntx, ty = tile / ntx;
  const int x0 = tx * TILE_X, y0 = ty * TILE_Y;
  const int wx = TILE_X + (tx == ntx - 1), hy = TILE_Y + (ty == nty - 1);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(2u * TL_XBYTES + (HAS_B ? TL_RBYTES : 0u))
                 : "memory");
    tma_load_3d(smem_u32(xs), &mx, 4 * (x0 - 1), y0 - 1, grp, bar);
    if (HAS_B) tma_load_3d(smem_u32(rs), &mr, 4 * x0, y0, grp, bar);
    tma_load_2d(smem_u32(cs), &mc, 4 * (x0 - 1), y0 - 1, bar);
  }
  if (!__syncthreads_and(mbar_wait0(bar))) {  // every thread leaves together if any wait ran out
    // thread 0 raises the flag and waits once more (again bounded) for the copies it issued,
    // so that the CTA's shared memory is not released with bulk copies still landing in it
    if (threadIdx.x == 0) {
      atomicExch(&g_tile_timeout, 1);
      (void)mbar_wait0(bar);
    }
    return;
  }
  PK acc = PK::zero();
  for (int t = threadIdx.x; t < wx * hy; t += TL_NT) {
    const int lx = t % wx, ly = t / wx;
    const int v0 = x0 + lx, v1 = y0 + ly;
    const int ci = (ly + 1) * TLB_X + lx + 1;  // this node in the halo boxes
    const bool fx = v0 < g.N, bx = v0 > 0, fy = v1 < g.N, by = v1 > 0;
    const float4 cc = cs[ci];
    PK out;
    if (MODE == M_JAC2) {
      // two damped-Jacobi sweeps from zero: e1 = w1 D^-1 r, e2 = e1 + w2 D^-1 (r - S e1)
      const float wi = omega * cc.y, wi2 = omega2 * cc.y;
      const PK r = PK::ld(xs + ci * 4);
      PK e1c;
#pragma unroll
      for (int q = 0; q < 4; ++q) e1c.v[q] = wi * r.v[q];
      PK sx;
#pragma unroll
      for (int q = 0; q < 4; ++q) sx.v[q] = cc.x * e1c.v[q];
      if (fx) sx.axpy(cc.z * omega * cs[ci + 1].y, PK::ld(xs + (ci + 1) * 4));
      if (bx) sx.axpy(cs[ci - 1].z * omega * cs[ci - 1].y, PK::ld(xs + (ci - 1) * 4));
      if (fy) sx.axpy(cc.w * omega * cs[ci + TLB_X].y, PK::ld(xs + (ci + TLB_X) * 4));
      if (by) sx.axpy(cs[ci - TLB_X].w * omega * cs[ci - TLB_X].y, PK::ld(xs + (ci - TLB_X) * 4));
#pragma unroll
      for (int q = 0; q < 4; ++q) out.v[q] = fmadd(wi2, r.v[q] - sx.v[q], e1c.v[q]);
    } else {
      const PK xc = PK::ld(xs + ci * 4);
      PK sx;
#pragma unroll
      for (int q = 0; q < 4; ++q) sx.v[q] = cc.x * xc.v[q];
      if (fx) sx.axpy(cc.z, PK::ld(xs + (ci + 1) * 4));
      if (bx) sx.axpy(cs[ci - 1].z, PK::ld(xs + (ci - 1) * 4));
      if (fy) sx.axpy(cc.w, PK::ld(xs + (ci + TLB_X) * 4));
      if (by) sx.axpy(cs[ci - TLB_X].w, PK::ld(xs + (ci - TLB_X) * 4));
      if (MODE == M_APPLY || MODE == M_APPLY_DOT) {
        out = sx;
        if (DOT)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc.v[q] = fmadd(xc.v[q], out.v[q], acc.v[q]);
      } else {
        const PK bb = PK::ld(rs + (ly * TLR_X + lx) * 4);
        if (MODE == M_RESID) {
#pragma unroll
          for (int q = 0; q < 4; ++q) out.v[q] = bb.v[q] - sx.v[q];
        } else {
          const float wi = omega * cc.y;
#pragma unroll
          for (int q = 0; q < 4; ++q) out.v[q] = fmadd(wi, bb.v[q] - sx.v[q], xc.v[q]);
          if (DOT)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc.v[q] = fmadd(bb.v[q], out.v[q], acc.v[q]);
        }
      }
    }
    out.st(Y + grp * gy + ((long)v0 + (long)g.np * v1) * 4);
  }
  if (DOT) dot_partial<float, 4>(acc, fin.part, grp, s, tile, ntx * nty);
}

// ---------------------------------------------------------------------------
// TMA z-marching stencil kernels (3D stiffness levels, FP32, 4 columns per node).
// One CTA per xy tile of TILE3_X x TILE3_Y nodes, one z segment (16 or 8 planes, chosen per
// launch) and one column group.  A ring of TL3_NS = 3 shared-memory slots holds consecutive planes: the
// plane of x with a one-node xy halo, the plane of 16-byte coefficient records with the
// same halo, the z couplings and the plane of b; each slot completes on its own mbarrier
// (the use count's parity is the phase).  Plane p is computed from the slots of p and
// p + 1 while the copy of plane p + 2 is in flight, in the slot plane p - 1 has left.  What
// the march needs of plane p - 1 (x, c_z, 1/diag) stays in registers from the step before;
// at a segment's first plane it comes from global memory with plain loads that overlap the
// first copies.  Copies past the grid read zeros; the boundary tests keep them out of the
// arithmetic, which is k_st's, operation for operation.
// ---------------------------------------------------------------------------
constexpr int TL3_NT = NB;
constexpr int TL3_NS = 3;                                          // ring slots
constexpr int TL3B_X = TILE3_X + 3, TL3B_Y = TILE3_Y + 3;          // x / record boxes (one plane)
constexpr int TL3R_X = TILE3_X + 1, TL3R_Y = TILE3_Y + 1;          // b box (one plane)
constexpr int TL3Z_X = TILE3_X + 4;                                // c_z box width (16-byte multiple)
constexpr unsigned TL3_XB = TL3B_X * TL3B_Y * 16u, TL3_CB = TL3B_X * TL3B_Y * 16u, TL3_RB = TL3R_X * TL3R_Y * 16u;
constexpr unsigned TL3_ZB = TL3Z_X * TL3R_Y * 4u;
constexpr unsigned TL3_OFF_C = (TL3_XB + 127u) / 128u * 128u;
constexpr unsigned TL3_OFF_Z = TL3_OFF_C + (TL3_CB + 127u) / 128u * 128u;
constexpr unsigned TL3_OFF_R = TL3_OFF_Z + (TL3_ZB + 127u) / 128u * 128u;
constexpr unsigned TL3_SLOT = TL3_OFF_R + (TL3_RB + 127u) / 128u * 128u;
// A mode that reads no b (the matvecs, the two fused sweeps from zero, which take r as x)
// has slots that end before the b plane: 42 KB instead of 56.6 KB per CTA, so five CTAs fit
// on an SM instead of four.
template <int MODE> constexpr bool tl3_has_b() { return MODE == M_RESID || MODE == M_JACOBI || MODE == M_JACOBI_DOT; }
template <int MODE> constexpr unsigned tl3_slot() { return tl3_has_b<MODE>() ? TL3_SLOT : TL3_OFF_R; }
template <int MODE> constexpr unsigned tl3_smem() {
  return TL3_NS * tl3_slot<MODE>() + 8u * TL3_NS + 128u;  // slots, barriers, alignment slack
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// waits for the given phase parity of a barrier for at most ~2^31 clocks
__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

template <int MODE>
__global__ void __launch_bounds__(TL3_NT) k_st_tile3(const __grid_constant__ CUtensorMap mx,
                                                     const __grid_constant__ CUtensorMap mr,
                                                     const __grid_constant__ CUtensorMap mc,
                                                     const __grid_constant__ CUtensorMap mz, GridDesc g, int ntx,
                                                     int nty, int nzs, const float *__restrict__ Xg, long gx,
                                                     const float *__restrict__ pkg, const float *__restrict__ czg,
                                                     float *__restrict__ Y, long gy, int s, float omega, float omega2,
                                                     Fin fin) {
  using PK = Pack<float, 4>;
  extern __shared__ __align__(128) unsigned char tl3_raw[];
  unsigned char *sm = tl3_raw + ((128u - (smem_u32(tl3_raw) & 127u)) & 127u);
  constexpr bool HAS_B = (MODE == M_RESID || MODE == M_JACOBI || MODE == M_JACOBI_DOT);
  constexpr bool DOT = (MODE == M_APPLY_DOT || MODE == M_JACOBI_DOT);
  const int tile = blockIdx.x, grp = blockIdx.y;
  const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
  const int zs = (g.np - 1) / nzs;  // planes per z segment
  const int x0 = tx * TILE3_X, y0 = ty * TILE3_Y, zb = tz * zs;
  const int wx = TILE3_X + (tx == ntx - 1), hy = TILE3_Y + (ty == nty - 1);
  const int ze = zb + zs + (tz == nzs - 1);  // planes zb .. ze - 1
  constexpr unsigned SLOT = tl3_slot<MODE>();
  const uint32_t bar0 = smem_u32(sm + TL3_NS * SLOT);
  const unsigned bytes = TL3_XB + TL3_CB + TL3_ZB + (HAS_B ? TL3_RB : 0u);
  // plane q sits in slot (q - zb) % NS; its barrier's phase is the slot's use count
  auto issue = [&](int q) {
    const int r = q - zb, k = r % TL3_NS;
    unsigned char *sl = sm + k * SLOT;
    const uint32_t bar = bar0 + 8u * k;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    tma_load_4d(smem_u32(sl), &mx, 4 * (x0 - 1), y0 - 1, q, grp, bar);
    tma_load_3d(smem_u32(sl + TL3_OFF_C), &mc, 4 * (x0 - 1), y0 - 1, q, bar);
    tma_load_3d(smem_u32(sl + TL3_OFF_Z), &mz, x0, y0, q, bar);
    if (HAS_B) tma_load_4d(smem_u32(sl + TL3_OFF_R), &mr, 4 * x0, y0, q, grp, bar);
  };
  auto ready = [&](int q) {
    const int r = q - zb;
    return mbar_wait_parity(bar0 + 8u * (r % TL3_NS), (unsigned)((r / TL3_NS) & 1));
  };
  if (threadIdx.x == 0) {
    for (int k = 0; k < TL3_NS; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * k) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)  // the first plane and the one above it
    for (int q = zb; q <= zb + 1 && q <= ze; ++q) issue(q);
  PK acc = PK::zero();
  bool ok = true;
  int p_fail = ze;  // the plane whose wait ran out (planes up to p_fail + 2 may have copies in flight)
  // Each thread keeps its nodes (t = threadIdx.x + j * TL3_NT) for the whole march, so x at
  // planes p - 1 and p, and c_z and 1/diag at p - 1, rotate through registers: per node and
  // plane only x at p + 1 and the xy neighbours come from shared memory.
  constexpr int NPT = (TL3R_X * TL3R_Y + TL3_NT - 1) / TL3_NT;
  PK rxm[NPT], rx0[NPT];
  float rzm[NPT], rvm[NPT];
  {
    const long np = g.np, ldr = (np + 3) / 4 * 4;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {  // plane zb - 1 (absent below the grid: never read there)
      const int t = threadIdx.x + j * TL3_NT;
      rxm[j] = PK::zero();
      rzm[j] = 0.f;
      rvm[j] = 0.f;
      if (t >= wx * hy || zb == 0) continue;
      const long v0 = x0 + t % wx, v1 = y0 + t / wx, row = (long)(zb - 1) * np + v1;
      rxm[j] = PK::ld(Xg + grp * gx + (row * np + v0) * 4);
      rzm[j] = czg[row * ldr + v0];
      rvm[j] = pkg[(row * np + v0) * 4 + 1];
    }
  }
  for (int p = zb; p < ze; ++p) {
    __syncthreads();  // every thread is done with plane p - 1's slot
    if (threadIdx.x == 0 && p + 2 <= ze) issue(p + 2);
    ok = ready(p) && ready(p + 1);
    if (!__syncthreads_and(ok)) {  // every thread leaves together if any wait ran out
      ok = false;
      p_fail = p;
      break;
    }
    const unsigned char *sm_0 = sm + ((p - zb) % TL3_NS) * SLOT;       // plane p
    const unsigned char *sm_p = sm + ((p - zb + 1) % TL3_NS) * SLOT;   // plane p + 1
    const float *x0s = reinterpret_cast<const float *>(sm_0), *xp = reinterpret_cast<const float *>(sm_p);
    const float4 *c0s = reinterpret_cast<const float4 *>(sm_0 + TL3_OFF_C),
                 *cp = reinterpret_cast<const float4 *>(sm_p + TL3_OFF_C);
    const float *z0 = reinterpret_cast<const float *>(sm_0 + TL3_OFF_Z);
    const float *rs = reinterpret_cast<const float *>(sm_0 + TL3_OFF_R);
    const bool fz = p < g.N, bz = p > 0;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const int t = threadIdx.x + j * TL3_NT;
      if (t >= wx * hy) continue;
      const int lx = t % wx, ly = t / wx;
      const int v0 = x0 + lx, v1 = y0 + ly;
      const int ci = (ly + 1) * TL3B_X + lx + 1;  // this node in the halo boxes
      const int zi = ly * TL3Z_X + lx;            // ... in the c_z box
      const bool fx = v0 < g.N, bx = v0 > 0, fy = v1 < g.N, by = v1 > 0;
      const float4 cc = c0s[ci];  // diag, invdiag, c_x, c_y
      const float cz = z0[zi];    // c_z
      if (p == zb) rx0[j] = PK::ld(x0s + ci * 4);  // first plane: x at p from its slot
      const PK xpv = PK::ld(xp + ci * 4);  // x at p + 1
      PK out;
      if (MODE == M_JAC2) {
        const float wi = omega * cc.y, wi2 = omega2 * cc.y;
        const PK r = rx0[j];
        PK e1c;
#pragma unroll
        for (int q = 0; q < 4; ++q) e1c.v[q] = wi * r.v[q];
        PK sx;
#pragma unroll
        for (int q = 0; q < 4; ++q) sx.v[q] = cc.x * e1c.v[q];
        if (fx) sx.axpy(cc.z * omega * c0s[ci + 1].y, PK::ld(x0s + (ci + 1) * 4));
        if (bx) sx.axpy(c0s[ci - 1].z * omega * c0s[ci - 1].y, PK::ld(x0s + (ci - 1) * 4));
        if (fy) sx.axpy(cc.w * omega * c0s[ci + TL3B_X].y, PK::ld(x0s + (ci + TL3B_X) * 4));
        if (by) sx.axpy(c0s[ci - TL3B_X].w * omega * c0s[ci - TL3B_X].y, PK::ld(x0s + (ci - TL3B_X) * 4));
        if (fz) sx.axpy(cz * omega * cp[ci].y, xpv);
        if (bz) sx.axpy(rzm[j] * omega * rvm[j], rxm[j]);
#pragma unroll
        for (int q = 0; q < 4; ++q) out.v[q] = fmadd(wi2, r.v[q] - sx.v[q], e1c.v[q]);
      } else {
        const PK xc = rx0[j];
        PK sx;
#pragma unroll
        for (int q = 0; q < 4; ++q) sx.v[q] = cc.x * xc.v[q];
        if (fx) sx.axpy(cc.z, PK::ld(x0s + (ci + 1) * 4));
        if (bx) sx.axpy(c0s[ci - 1].z, PK::ld(x0s + (ci - 1) * 4));
        if (fy) sx.axpy(cc.w, PK::ld(x0s + (ci + TL3B_X) * 4));
        if (by) sx.axpy(c0s[ci - TL3B_X].w, PK::ld(x0s + (ci - TL3B_X) * 4));
        if (fz) sx.axpy(cz, xpv);
        if (bz) sx.axpy(rzm[j], rxm[j]);
        if (MODE == M_APPLY || MODE == M_APPLY_DOT) {
          out = sx;
          if (DOT)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc.v[q] = fmadd(xc.v[q], out.v[q], acc.v[q]);
        } else {
          const PK bb = PK::ld(rs + (ly * TL3R_X + lx) * 4);
          if (MODE == M_RESID) {
#pragma unroll
            for (int q = 0; q < 4; ++q) out.v[q] = bb.v[q] - sx.v[q];
          } else {
            const float wi = omega * cc.y;
#pragma unroll
            for (int q = 0; q < 4; ++q) out.v[q] = fmadd(wi, bb.v[q] - sx.v[q], xc.v[q]);
            if (DOT)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc.v[q] = fmadd(bb.v[q], out.v[q], acc.v[q]);
          }
        }
      }
      out.st(Y + grp * gy + ((long)v0 + (long)g.np * ((long)v1 + (long)g.np * p)) * 4);
      rxm[j] = rx0[j];
      rx0[j] = xpv;
      rzm[j] = cz;
      rvm[j] = cc.y;
    }
  }
  if (!ok) {
    // thread 0 raises the flag and waits once more (each wait bounded) for the planes it may
    // still have copies in flight for, so that the CTA does not leave with bulk copies
    // landing in shared memory that the next CTA on the SM receives
    if (threadIdx.x == 0) {
      atomicExch(&g_tile_timeout, 1);
      for (int q = p_fail; q <= p_fail + 2 && q <= ze; ++q) (void)ready(q);
    }
    return;
  }
  if (DOT) dot_partial<float, 4>(acc, fin.part, grp, s, tile, ntx * nty * nzs);
}

// ---------------------------------------------------------------------------
// grid transfer, coarse solve, vector kernels (grouped layout)
// ---------------------------------------------------------------------------
// Restriction = transpose of the P1 prolongation: r_c(J) = r_f(2J) +
// 1/2 sum_{b != 0} [r_f(2J + b) + r_f(2J - b)] over the 2^D - 1 Kuhn edge
// directions b; Dirichlet rows of the zero-BC space are zeroed.
template <typename T, int VW, int D>
__global__ void __launch_bounds__(NB) k_restrict(GridDesc gf, GridDesc gc, const T *__restrict__ rf, long gsf,
                                                 T *__restrict__ rc, long gsc, int zero_dirichlet) {
  using PK = Pack<T, VW>;
  // one coarse node per thread over the flattened grid (every lane busy whatever np is)
  const unsigned I = blockIdx.x * NB + threadIdx.x;
  if (I >= (unsigned)gc.n) return;
  const unsigned t = div_np(gc, I), t2 = D == 2 ? 0u : div_np(gc, t);
  const int J[3] = {(int)(I - t * (unsigned)gc.np), D == 2 ? (int)t : (int)(t - t2 * (unsigned)gc.np), (int)t2};
  const T *r = rf + blockIdx.z * gsf;
  PK out = PK::zero();
  if (!(zero_dirichlet && (J[D - 1] == 0 || J[D - 1] == gc.N))) {
    const long f0 = 2 * (long)J[0] + (long)gf.np * (2 * (long)J[1] + (D == 3 ? (long)gf.np * 2 * J[2] : 0));
    out = PK::ld(r + f0 * VW);
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
      if (fw) out.axpy(T(0.5), PK::ld(r + (f0 + off) * VW));
      if (bw) out.axpy(T(0.5), PK::ld(r + (f0 - off) * VW));
    }
  }
  out.st(rc + blockIdx.z * gsc + I * VW);
}

// e_f += P e_c: fine node 2I + b takes e_c(I) (b = 0) or the mean of e_c(I) and
// e_c(I + b) (midpoint of the coarse Kuhn edge in direction b).
template <typename T, int VW, int D>
__global__ void __launch_bounds__(NB) k_prolong_add(GridDesc gf, GridDesc gc, const T *__restrict__ ec, long gsc,
                                                    T *__restrict__ ef, long gsf) {
  using PK = Pack<T, VW>;
  // one fine node per thread over the flattened grid (every lane busy whatever np is)
  const unsigned i = blockIdx.x * NB + threadIdx.x;
  if (i >= (unsigned)gf.n) return;
  const unsigned t = div_np(gf, i), t2 = D == 2 ? 0u : div_np(gf, t);
  const int v[3] = {(int)(i - t * (unsigned)gf.np), D == 2 ? (int)t : (int)(t - t2 * (unsigned)gf.np), (int)t2};
  const T *e = ec + blockIdx.z * gsc;
  const int b = (v[0] & 1) | ((v[1] & 1) << 1) | ((v[2] & 1) << 2);
  const long ic = (v[0] >> 1) + (long)gc.np * ((v[1] >> 1) + (long)gc.np * (v[2] >> 1));
  PK val = PK::ld(e + ic * VW);
  if (b) {
    const PK v2 = PK::ld(e + (ic + mask_offset(gc, b)) * VW);
#pragma unroll
    for (int q = 0; q < VW; ++q) val.v[q] = mulr(T(0.5), val.v[q] + v2.v[q]);
  }
  T *o = ef + blockIdx.z * gsf + i * VW;
  PK cur = PK::ld(o);
#pragma unroll
  for (int q = 0; q < VW; ++q) cur.v[q] = addr(cur.v[q], val.v[q]);
  cur.st(o);
}

// (S x)(id) for node id with coordinates v (level stencil, boundary-aware)
template <typename T, int VW, int D, bool FULL>
__device__ __forceinline__ Pack<T, VW> stencil_at(const GridDesc &g, const T *__restrict__ diag,
                                                  const T *__restrict__ c, const T *__restrict__ x, long id,
                                                  const int v[3]) {
  using PK = Pack<T, VW>;
  constexpr int NF = FULL ? (1 << D) - 1 : D;
  const PK xc = PK::ld(x + id * VW);
  PK sx;
  const T dg = diag[id];
#pragma unroll
  for (int q = 0; q < VW; ++q) sx.v[q] = dg * xc.v[q];
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
    if (fw) sx.axpy(c[(long)f * g.n + id], PK::ld(x + (id + off) * VW));
    if (bw) sx.axpy(c[(long)f * g.n + id - off], PK::ld(x + (id - off) * VW));
  }
  return sx;
}

// Residual and restriction in one pass: r_c(J) = sum over the fine nodes j of the
// restriction stencil of 2J (weight 1 at 2J, 1/2 at 2J +- b) of (b_f - S e)(j).  The fine
// residual is never stored.  One coarse node per thread.
template <typename T, int VW, int D, bool FULL>
__global__ void __launch_bounds__(NB) k_resid_restrict(GridDesc gf, GridDesc gc, const T *__restrict__ diag,
                                                       const T *__restrict__ c, const T *__restrict__ e,
                                                       const T *__restrict__ bf, long gsf, T *__restrict__ rc,
                                                       long gsc, int zero_dirichlet) {
  using PK = Pack<T, VW>;
  const int I0 = blockIdx.x * 32 + (threadIdx.x & 31);
  const int row = blockIdx.y * (NB / 32) + (threadIdx.x >> 5);
  const int nrows = D == 2 ? gc.np : gc.np * gc.np;
  if (I0 >= gc.np || row >= nrows) return;
  const int J[3] = {I0, D == 2 ? row : row % gc.np, D == 2 ? 0 : row / gc.np};
  const long I = I0 + (long)gc.np * row;
  const T *eg = e + blockIdx.z * gsf, *bg = bf + blockIdx.z * gsf;
  PK out = PK::zero();
  auto resid = [&](long j, const int vj[3]) {
    const PK sx = stencil_at<T, VW, D, FULL>(gf, diag, c, eg, j, vj);
    PK r = PK::ld(bg + j * VW);
#pragma unroll
    for (int q = 0; q < VW; ++q) r.v[q] -= sx.v[q];
    return r;
  };
  if (!(zero_dirichlet && (J[D - 1] == 0 || J[D - 1] == gc.N))) {
    const int v0[3] = {2 * J[0], 2 * J[1], 2 * J[2]};
    const long f0 = v0[0] + (long)gf.np * (v0[1] + (long)gf.np * v0[2]);
    out = resid(f0, v0);
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
      if (fw) {
        const int vf[3] = {v0[0] + (b & 1), v0[1] + ((b >> 1) & 1), v0[2] + ((b >> 2) & 1)};
        out.axpy(T(0.5), resid(f0 + off, vf));
      }
      if (bw) {
        const int vb[3] = {v0[0] - (b & 1), v0[1] - ((b >> 1) & 1), v0[2] - ((b >> 2) & 1)};
        out.axpy(T(0.5), resid(f0 - off, vb));
      }
    }
  }
  out.st(rc + blockIdx.z * gsc + I * VW);
}

// Prolongation and the first post-smoothing sweep in one pass:
//   x' = x + P e_c (at the node and its stencil neighbours, recomputed on the fly),
//   y  = x' + w D^-1 (b - S x')
// The prolonged x' is never stored.
template <typename T, int VW, int D, bool FULL>
__global__ void __launch_bounds__(NB) k_prolong_sweep(GridDesc gf, GridDesc gc, const T *__restrict__ diag,
                                                      const T *__restrict__ invdiag, const T *__restrict__ c,
                                                      const T *__restrict__ x, const T *__restrict__ ec,
                                                      long gsc, const T *__restrict__ bf, T *__restrict__ y,
                                                      long gsf, T omega) {
  using PK = Pack<T, VW>;
  constexpr int NF = FULL ? (1 << D) - 1 : D;
  const int lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * 32 + lane;
  const int nrows = D == 2 ? gf.np : gf.np * gf.np;
  const T *xg = x + blockIdx.z * gsf, *bg = bf + blockIdx.z * gsf, *eg = ec + blockIdx.z * gsc;
  // x' at fine node j with coordinates vj
  auto xp = [&](long j, const int vj[3]) {
    PK val = PK::ld(xg + j * VW);
    const int bm = (vj[0] & 1) | ((vj[1] & 1) << 1) | ((vj[2] & 1) << 2);
    const long ic = (vj[0] >> 1) + (long)gc.np * ((vj[1] >> 1) + (long)gc.np * (vj[2] >> 1));
    const PK e0 = PK::ld(eg + ic * VW);
    if (bm) {
      const PK e1 = PK::ld(eg + (ic + mask_offset(gc, bm)) * VW);
#pragma unroll
      for (int q = 0; q < VW; ++q) val.v[q] = addr(val.v[q], mulr(T(0.5), e0.v[q] + e1.v[q]));
    } else {
#pragma unroll
      for (int q = 0; q < VW; ++q) val.v[q] = addr(val.v[q], e0.v[q]);
    }
    return val;
  };
  for (int row = blockIdx.y * (NB / 32) + (threadIdx.x >> 5); row < nrows; row += gridDim.y * (NB / 32)) {
    if (i0 >= gf.np) break;
    const int v[3] = {i0, D == 2 ? row : row % gf.np, D == 2 ? 0 : row / gf.np};
    const long id = i0 + (long)gf.np * row;
    const PK xc = xp(id, v);
    PK sx;
    const T dg = diag[id];
#pragma unroll
    for (int q = 0; q < VW; ++q) sx.v[q] = dg * xc.v[q];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int b = FULL ? f + 1 : (1 << f);
      bool fw = true, bw = true;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if ((b >> a) & 1) {
          fw = fw && (v[a] < gf.N);
          bw = bw && (v[a] > 0);
        }
      const long off = mask_offset(gf, b);
      if (fw) {
        const int vf[3] = {v[0] + (b & 1), v[1] + ((b >> 1) & 1), v[2] + ((b >> 2) & 1)};
        sx.axpy(c[(long)f * gf.n + id], xp(id + off, vf));
      }
      if (bw) {
        const int vb[3] = {v[0] - (b & 1), v[1] - ((b >> 1) & 1), v[2] - ((b >> 2) & 1)};
        sx.axpy(c[(long)f * gf.n + id - off], xp(id - off, vb));
      }
    }
    const PK bb = PK::ld(bg + id * VW);
    const T wi = omega * invdiag[id];
    PK out;
#pragma unroll
    for (int q = 0; q < VW; ++q) out.v[q] = fmadd(wi, bb.v[q] - sx.v[q], xc.v[q]);
    out.st(y + blockIdx.z * gsf + id * VW);
  }
}

// dense coarse-grid inverse: e = A_c^{-1} r.  blockIdx.x = chunk of 32 rows (lanes),
// blockIdx.y = column group; the 8 warps of a block split the k sum, then add.
template <typename T, int VW>
__global__ void __launch_bounds__(256) k_coarse_apply(const T *__restrict__ inv, int nc, const T *__restrict__ R,
                                                      long gsr, T *__restrict__ E, long gse) {
  using PK = Pack<T, VW>;
  extern __shared__ unsigned char smem_raw[];
  T *r = reinterpret_cast<T *>(smem_raw);
  __shared__ T red[8][32][VW];
  const T *rg = R + blockIdx.y * gsr;
  for (int k = threadIdx.x; k < nc * VW; k += blockDim.x) r[k] = rg[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  PK acc = PK::zero();
  if (i < nc) {
    for (int k = w; k < nc; k += 8) {
      const T a = inv[(long)k * nc + i];
#pragma unroll
      for (int q = 0; q < VW; ++q) acc.v[q] = fmadd(a, r[k * VW + q], acc.v[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < VW; ++q) red[w][lane][q] = acc.v[q];
  __syncthreads();
  if (w == 0 && i < nc) {
    PK out = PK::zero();
#pragma unroll
    for (int ww = 0; ww < 8; ++ww)
#pragma unroll
      for (int q = 0; q < VW; ++q) out.v[q] += red[ww][lane][q];
    out.st(E + blockIdx.y * gse + (long)i * VW);
  }
}

// 1-D node kernels: blockIdx.x over nodes (NB each), blockIdx.y = group
template <typename T, int VW>
__global__ void __launch_bounds__(NB) k_jacobi0(long n, const T *__restrict__ invdiag, const T *__restrict__ B, long gs,
                                                T *__restrict__ Y, T omega, int s, Fin fin, int with_dot) {
  using PK = Pack<T, VW>;
  const int grp = blockIdx.y;
  PK acc = PK::zero();
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    const PK b = PK::ld(B + grp * gs + i * VW);
    const T w = omega * invdiag[i];
    PK z;
#pragma unroll
    for (int q = 0; q < VW; ++q) {
      z.v[q] = w * b.v[q];
      acc.v[q] = fmadd(b.v[q], z.v[q], acc.v[q]);
    }
    z.st(Y + grp * gs + i * VW);
  }
  if (with_dot) dot_partial<T, VW>(acc, fin.part, grp, s, blockIdx.x, gridDim.x);
}

template <typename T, int VW>
__global__ void __launch_bounds__(NB) k_cg_update(long n, long gs, const T *__restrict__ p, const T *__restrict__ q,
                                                  T *__restrict__ x, T *__restrict__ r,
                                                  const double *__restrict__ alpha, int s, Fin fin) {
  using PK = Pack<T, VW>;
  const int grp = blockIdx.y;
  PK acc = PK::zero();
  T a[VW];
#pragma unroll
  for (int c = 0; c < VW; ++c) a[c] = (T)alpha[grp * VW + c];
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    const long o = grp * gs + i * VW;
    const PK pp = PK::ld(p + o), qq = PK::ld(q + o);
    PK xx = PK::ld(x + o), rr = PK::ld(r + o);
#pragma unroll
    for (int c = 0; c < VW; ++c) {
      xx.v[c] += a[c] * pp.v[c];
      rr.v[c] -= a[c] * qq.v[c];
      acc.v[c] += rr.v[c] * rr.v[c];
    }
    xx.st(x + o);
    rr.st(r + o);
  }
  dot_partial<T, VW>(acc, fin.part, grp, s, blockIdx.x, gridDim.x);
}

template <typename T, int VW>
__global__ void __launch_bounds__(NB) k_p_update(long n, long gs, const T *__restrict__ z, T *__restrict__ p,
                                                 const double *__restrict__ beta) {
  using PK = Pack<T, VW>;
  const int grp = blockIdx.y;
  T b[VW];
#pragma unroll
  for (int c = 0; c < VW; ++c) b[c] = (T)beta[grp * VW + c];
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    const long o = grp * gs + i * VW;
    const PK zz = PK::ld(z + o);
    PK pp = PK::ld(p + o);
#pragma unroll
    for (int c = 0; c < VW; ++c) pp.v[c] = zz.v[c] + b[c] * pp.v[c];
    pp.st(p + o);
  }
}

// <a, b> per column (a == b: squared norm)
template <typename T, int VW>
__global__ void __launch_bounds__(NB) k_dot(long n, long gs, const T *__restrict__ a, const T *__restrict__ b, int s,
                                            Fin fin) {
  using PK = Pack<T, VW>;
  const int grp = blockIdx.y;
  PK acc = PK::zero();
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    const PK aa = PK::ld(a + grp * gs + i * VW), bb = PK::ld(b + grp * gs + i * VW);
#pragma unroll
    for (int c = 0; c < VW; ++c) acc.v[c] += aa.v[c] * bb.v[c];
  }
  dot_partial<T, VW>(acc, fin.part, grp, s, blockIdx.x, gridDim.x);
}

// r_T (grouped) = scale * r64 (column-major); columns >= s and converged ones are 0
template <typename T, int VW>
__global__ void __launch_bounds__(NB) k_to_inner(long n, const double *__restrict__ R, long ldr,
                                                 const double *__restrict__ scale, int s, T *__restrict__ rt, long gs) {
  using PK = Pack<T, VW>;
  const int grp = blockIdx.y;
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    PK o;
#pragma unroll
    for (int q = 0; q < VW; ++q) {
      const int col = grp * VW + q;
      o.v[q] = col < s ? (T)(scale[col] * R[ldr * col + i]) : T(0);
    }
    o.st(rt + grp * gs + i * VW);
  }
}

// The same scaling inside a graph-driven refinement: the first step (ctl->outer == 1,
// counted before the step runs) starts from x = 0, so its residual is b0 itself.
template <typename T, int VW>
__global__ void __launch_bounds__(NB) k_to_inner_ctl(long n, const double *__restrict__ B0,
                                                     const double *__restrict__ R, long ldr,
                                                     const RefineCtl *__restrict__ ctl,
                                                     const double *__restrict__ scale, int s, T *__restrict__ rt,
                                                     long gs) {
  using PK = Pack<T, VW>;
  const double *src = ctl->outer == 1 ? B0 : R;
  const int grp = blockIdx.y;
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    PK o;
#pragma unroll
    for (int q = 0; q < VW; ++q) {
      const int col = grp * VW + q;
      o.v[q] = col < s ? (T)(scale[col] * src[ldr * col + i]) : T(0);
    }
    o.st(rt + grp * gs + i * VW);
  }
}

// Convergence control of a graph-driven refinement (one block): for every column the
// test |r|^2 <= rtol^2 |b|^2, the scale 1/|r| into the inner solve and back, and the
// inner tolerance (the finer of tol_in and what is left to reach rtol, with a factor 1/4
// of margin); then the loop condition: another step while a column is open, a
// non-finite residual or max_outer steps end the loop with a flag.  after_body adds the
// inner iterations of the step that just ran.
__global__ void k_refine_ctl(int s, const double *__restrict__ rr, const double *__restrict__ bb, double rtol,
                             double tol_in, double *__restrict__ scale, double *__restrict__ iscale,
                             double *__restrict__ tol2col, const int *__restrict__ pcg_iter, int after_body,
                             int max_outer, RefineCtl *ctl, cudaGraphConditionalHandle h) {
  __shared__ int nact_s, bad_s;
  __shared__ double worst_s[256];
  if (threadIdx.x == 0) nact_s = bad_s = 0;
  __syncthreads();
  int nact = 0, bad = 0;
  double worst = 0.0;
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    const double r2 = rr[j], b2 = bb[j];
    if (!isfinite(r2)) bad = 1;
    const double rel = b2 > 0 ? sqrt(r2 / b2) : 0.0;
    worst = fmax(worst, rel);
    const bool done = b2 == 0.0 || r2 <= rtol * rtol * b2;
    scale[j] = done ? 0.0 : 1.0 / sqrt(r2);
    iscale[j] = done ? 0.0 : sqrt(r2);
    const double need = r2 > 0 ? 0.25 * rtol * sqrt(b2 / r2) : 1.0;
    const double t = fmin(0.5, fmax(tol_in, need));
    tol2col[j] = t * t;
    nact += !done;
  }
  if (nact) atomicAdd(&nact_s, nact);
  if (bad) atomicOr(&bad_s, 1);
  worst_s[threadIdx.x] = worst;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) worst_s[threadIdx.x] = fmax(worst_s[threadIdx.x], worst_s[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (after_body) ctl->total_its += *pcg_iter;
    ctl->worst = worst_s[0];
    unsigned cond = 0;
    if (bad_s) {
      ctl->flags |= 2;
    } else if (nact_s > 0) {
      if (ctl->outer >= max_outer) {
        ctl->flags |= 1;
      } else {
        cond = 1;
        ctl->outer += 1;
      }
    }
    cudaGraphSetConditional(h, cond);
  }
}

// X (column-major FP64) += d / scale for the columns with scale != 0
template <typename T, int VW>
__global__ void __launch_bounds__(NB) k_accum(long n, const T *__restrict__ d, long gs, const double *__restrict__ iscale,
                                              int s, double *__restrict__ X, long ldx) {
  using PK = Pack<T, VW>;
  const int grp = blockIdx.y;
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    const PK v = PK::ld(d + grp * gs + i * VW);
#pragma unroll
    for (int q = 0; q < VW; ++q) {
      const int col = grp * VW + q;
      if (col < s) {
        const double is = iscale[col];  // |r| of the column, 0 when it has converged
        if (is != 0.0) X[ldx * col + i] += (double)v.v[q] * is;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 iterative refinement in double-float arithmetic (tuning refine_df).  GB300 runs
// FP64 at a small fraction of its FP32 rate, so around FP32 inner solves the refinement
// can keep its right-hand side b and iterate x as double-float pairs (about 48
// significand bits) and do its arithmetic on the FP32 pipe:
//  * the pairs live in the refinement's workspace in the inner solver's grouped layout,
//    one record {hi of 4 columns, lo of 4 columns} (two float4) per node and group, so
//    every access is a 16-byte load or store and no value is converted on the way;
//  * the caller's FP64 B is split into pairs once when the solve starts and x joined back
//    into its FP64 X once when it ends (bit manipulation, no FP64 instruction);
//  * the residual b - S x is a compensated (Dot2) sum of pair products with the level-0
//    stencil's coefficients, also held as pairs; its leading float, scaled per column by
//    a power of two sb with sb |b| in [0.5, 1), is written straight into the inner solve's
//    right-hand side (the scaling is exact, and keeps the FP32 inner solve's values far
//    from the float range's ends), with the column's |r|^2;
//  * the update x += d / sb adds the inner solution to the pairs (two_sum).
// Columns that have converged keep their residual in the inner right-hand side, but the
// PCG starts them inactive (the open mask of FIN_INIT), so their x stays as it is.
// ---------------------------------------------------------------------------

// sb for a column with |b|^2 = b2 (1 when b = 0)
__device__ __forceinline__ float col_scale(double b2) {
  if (!(b2 > 0.0)) return 1.f;
  int e;
  (void)frexp(sqrt(b2), &e);  // |b| = f 2^e, f in [0.5, 1)
  e = max(-125, min(125, e));
  return __uint_as_float((unsigned)(127 - e) << 23);  // 2^-e
}

// coefficient pairs of a stencil: c_f at [f n + i] (f < nf), the diagonal at [nf n + i]
__global__ void k_coef_pairs(long n, int nf, const double *__restrict__ diag, const double *__restrict__ c,
                             float2 *__restrict__ cpr) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    for (int f = 0; f < nf; ++f) {
      const dfl d = d2df(c[(long)f * n + i]);
      cpr[(long)f * n + i] = make_float2(d.hi, d.lo);
    }
    const dfl d = d2df(diag[i]);
    cpr[(long)nf * n + i] = make_float2(d.hi, d.lo);
  }
}

// b pairs = B (the `face` nodes at each end zeroed), x pairs = 0, |B|^2 block partials;
// columns past s are zero
__global__ void __launch_bounds__(NB) k_ir_start_dfp(const double *__restrict__ B, long ldb, int s, float4 *Bp,
                                                     float4 *Xp, long ldp, long n, long face, double *part) {
  const int grp = blockIdx.y;
  Pack<double, 4> acc = Pack<double, 4>::zero();
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    const bool inner = i >= face && i < n - face;
    float hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = grp * 4 + q;
      const double v = (inner && col < s) ? B[ldb * col + i] : 0.0;
      const dfl d = d2df(v);
      hi[q] = d.hi;
      lo[q] = d.lo;
      acc.v[q] = fma(v, v, acc.v[q]);
    }
    const long k = 2 * ((long)grp * ldp + i);
    Bp[k] = make_float4(hi[0], hi[1], hi[2], hi[3]);
    Bp[k + 1] = make_float4(lo[0], lo[1], lo[2], lo[3]);
    Xp[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    Xp[k + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  dot_partial<double, 4>(acc, part, grp, s, blockIdx.x, gridDim.x);
}

// the first inner right-hand side, from x = 0: rt = hi(b) sb
__global__ void __launch_bounds__(NB) k_first_inner_dfp(const float4 *__restrict__ Bp, long ldp, long n,
                                                        const double *__restrict__ bb, int s, float *__restrict__ rt,
                                                        long gs) {
  const int grp = blockIdx.y;
  float sb[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) sb[q] = col_scale(grp * 4 + q < s ? bb[grp * 4 + q] : 0.0);
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    const float4 h = Bp[2 * ((long)grp * ldp + i)];
    *reinterpret_cast<float4 *>(rt + grp * gs + i * 4) = make_float4(h.x * sb[0], h.y * sb[1], h.z * sb[2], h.w * sb[3]);
  }
}

__device__ __forceinline__ void ld_pair4(const float4 *p, long k, dfl out[4]) {
  const float4 h = p[k], l = p[k + 1];
  out[0] = {h.x, l.x};
  out[1] = {h.y, l.y};
  out[2] = {h.z, l.z};
  out[3] = {h.w, l.w};
}

// rt = (b - S x) sb from the pairs (four columns per thread, one node per thread over the
// flattened grid), |r|^2 block partials.  Every load of a node's stencil is issued before
// the arithmetic starts (2 NF + 2 pair records and 2 NF + 1 coefficient pairs in flight
// per thread), and the four columns' compensated sums advance term by term.
template <int D, bool FULL>
__global__ void __launch_bounds__(NB) k_resid_dfp(GridDesc g, const float2 *__restrict__ cpr,
                                                  const float4 *__restrict__ Xp, const float4 *__restrict__ Bp,
                                                  long ldp, float *__restrict__ rt, long gs, int s,
                                                  const double *__restrict__ bb, Fin fin) {
  constexpr int NF = FULL ? (1 << D) - 1 : D;
  const int grp = blockIdx.y;
  float sb[4], accf[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < 4; ++q) sb[q] = col_scale(grp * 4 + q < s ? bb[grp * 4 + q] : 0.0);
  const float4 *xg = Xp + 2 * (long)grp * ldp, *bg = Bp + 2 * (long)grp * ldp;
  const unsigned np = (unsigned)g.np, n = (unsigned)g.n;
  for (unsigned i = blockIdx.x * NB + threadIdx.x; i < n; i += gridDim.x * NB) {
    int v[3];
    const unsigned t = div_np(g, i), t2 = D == 2 ? 0u : div_np(g, t);
    v[0] = (int)(i - t * np);
    v[1] = D == 2 ? (int)t : (int)(t - t2 * np);
    v[2] = (int)t2;
    // the stencil's points: 0 the node, 1 + 2f / 2 + 2f the forward / backward neighbour f
    unsigned pt[2 * NF + 1];
    bool ok[2 * NF + 1];
    pt[0] = i;
    ok[0] = true;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int b = FULL ? f + 1 : (1 << f);
      bool fw = true, bw = true;
#pragma unroll
      for (int k = 0; k < D; ++k)
        if ((b >> k) & 1) {
          fw = fw && (v[k] < g.N);
          bw = bw && (v[k] > 0);
        }
      const unsigned off = (unsigned)mask_offset(g, b);
      ok[1 + 2 * f] = fw;
      ok[2 + 2 * f] = bw;
      pt[1 + 2 * f] = fw ? i + off : i;
      pt[2 + 2 * f] = bw ? i - off : i;
    }
    // loads: b, x at every point, the coefficient pair of every coupling
    const float4 bh = bg[2 * i], bl = bg[2 * i + 1];
    float4 xh[2 * NF + 1], xl[2 * NF + 1];
    float2 cp[2 * NF + 1];
#pragma unroll
    for (int k = 0; k < 2 * NF + 1; ++k) {
      xh[k] = xg[2 * pt[k]];
      xl[k] = xg[2 * pt[k] + 1];
    }
    cp[0] = cpr[(unsigned)NF * n + i];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      cp[1 + 2 * f] = cpr[(unsigned)f * n + i];
      cp[2 + 2 * f] = cpr[(unsigned)f * n + pt[2 + 2 * f]];
    }
    Dot2 a[4];
    a[0].add(dfl{bh.x, bl.x});
    a[1].add(dfl{bh.y, bl.y});
    a[2].add(dfl{bh.z, bl.z});
    a[3].add(dfl{bh.w, bl.w});
#pragma unroll
    for (int k = 0; k < 2 * NF + 1; ++k) {
      if (!ok[k]) continue;
      const dfl c{cp[k].x, cp[k].y};
      a[0].fms(c, dfl{xh[k].x, xl[k].x});
      a[1].fms(c, dfl{xh[k].y, xl[k].y});
      a[2].fms(c, dfl{xh[k].z, xl[k].z});
      a[3].fms(c, dfl{xh[k].w, xl[k].w});
    }
    float r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      r[q] = a[q].result().hi * sb[q];
      accf[q] = fmaf(r[q], r[q], accf[q]);
    }
    *reinterpret_cast<float4 *>(rt + grp * gs + (long)i * 4) = make_float4(r[0], r[1], r[2], r[3]);
  }
  Pack<double, 4> acc;
#pragma unroll
  for (int q = 0; q < 4; ++q) acc.v[q] = (double)accf[q] / ((double)sb[q] * (double)sb[q]);
  dot_partial<double, 4>(acc, fin.part, grp, s, blockIdx.x, gridDim.x);
}

// x pairs += d / sb for the open columns (iscale != 0)
__global__ void __launch_bounds__(NB) k_accum_dfp(long n, const float *__restrict__ d, long gs,
                                                  const double *__restrict__ iscale, const double *__restrict__ bb,
                                                  int s, float4 *__restrict__ Xp, long ldp) {
  const int grp = blockIdx.y;
  float isb[4];
  bool open[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int col = grp * 4 + q;
    open[q] = col < s && iscale[col] != 0.0;
    isb[q] = 1.f / col_scale(col < s ? bb[col] : 0.0);  // a power of two: exact
  }
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    const float4 dv = *reinterpret_cast<const float4 *>(d + grp * gs + i * 4);
    const float dd[4] = {dv.x, dv.y, dv.z, dv.w};
    const long k = 2 * ((long)grp * ldp + i);
    dfl x[4];
    ld_pair4(Xp, k, x);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!open[q]) continue;
      Dot2 a;
      a.add(x[q]);
      a.add(dfl{dd[q] * isb[q], 0.f});
      x[q] = a.result();
    }
    Xp[k] = make_float4(x[0].hi, x[1].hi, x[2].hi, x[3].hi);
    Xp[k + 1] = make_float4(x[0].lo, x[1].lo, x[2].lo, x[3].lo);
  }
}

// X (FP64, column-major) = the x pairs joined, for the s columns
__global__ void __launch_bounds__(NB) k_df_out_dfp(const float4 *__restrict__ Xp, long ldp, long n, int s,
                                                   double *__restrict__ X, long ldx) {
  const int grp = blockIdx.y;
  for (long i = blockIdx.x * (long)NB + threadIdx.x; i < n; i += (long)gridDim.x * NB) {
    dfl x[4];
    ld_pair4(Xp, 2 * ((long)grp * ldp + i), x);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (grp * 4 + q < s) X[ldx * (grp * 4 + q) + i] = df2d(x[q]);
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
  cudaEventRecord(P->prof_ev[2 * r], P->st);
  P->prof_used = r + 1;
  P->prof_id[r] = -(id + 2);  // open
  return (int)r;
}

void prof_stop(hp_problem *P, int rec) {
  if (rec < 0) return;
  cudaEventRecord(P->prof_ev[2 * rec + 1], P->st);
  P->prof_id[rec] = -P->prof_id[rec] - 2;  // closed: store the id
}

// bounded busy wait (clock cycles), used only while profiling
__global__ void k_spin(long long cycles) {
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) {
  }
}

void prof_spin(hp_problem *P) {
  if (!P->prof_on) return;
  k_spin<<<1, 32, 0, P->st>>>(300000LL);  // ~150 us at 2 GHz
}

// Adds the durations of records [from, to) to the per-family totals; unless keep,
// the records are retired (id -1) so that a later harvest skips them.
void prof_harvest(hp_problem *P, size_t from, size_t to, bool keep) {
  for (size_t r = from; r < to && r < P->prof_used; ++r) {
    const int id = P->prof_id[r];
    if (id < 0 || id >= 16) continue;
    float ms = 0.f;
    const bool clean = cudaPeekAtLastError() == cudaSuccess;  // an earlier error stays for the caller
    if (cudaEventElapsedTime(&ms, P->prof_ev[2 * r], P->prof_ev[2 * r + 1]) == cudaSuccess) {
      P->prof_cnt[id] += 1;
      P->prof_ms[id] += ms;
    } else {
      if (clean) (void)cudaGetLastError();  // a failed timing query must not surface as a solver error
      P->prof_failed = true;
    }
    if (!keep) P->prof_id[r] = -1;
  }
}

// ---------------------------------------------------------------------------
// host side
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

// grid-size cap of the node kernels (a tuning knob; the default 4096 is about 27 128-thread
// blocks per SM on 152 SMs, two rounds of the ~13-16 that are resident at once, which keeps
// a launch's tail short), set per solve from the problem's tuning
static thread_local long tl_max_blocks = 4096;

// uncapped row grid: one node per thread, warps along x rows
static dim3 rowgrid(const GridDesc &g, int ngroups) {
  const long nrows = g.dim == 2 ? g.np : (long)g.np * g.np;
  return dim3((g.np + 31) / 32, (unsigned)((nrows + NB / 32 - 1) / (NB / 32)), ngroups);
}
// one node per thread over the flattened grid, column groups over blockIdx.z (grid transfers)
static dim3 flatgrid(const GridDesc &g, int ngroups) {
  return dim3((unsigned)((g.n + NB - 1) / NB), 1, (unsigned)ngroups);
}
// row grid of the stencil kernels: warps loop over rows so that the grid stays near
// the grid-size cap (fewer per-block dot partials)
static dim3 rowgrid_capped(const GridDesc &g, int ngroups) {
  dim3 d = rowgrid(g, ngroups);
  const long cap = std::max<long>(1, tl_max_blocks / ((long)d.x * ngroups));
  if ((long)d.y > cap) d.y = (unsigned)cap;
  return d;
}
static long rowgrid_blocks(const GridDesc &g) {
  const dim3 d = rowgrid(g, 1);
  return (long)d.x * d.y;
}

// level stencils of 2D stiffness solves as TMA tiles (a tuning knob), set per solve
static thread_local int tl_tma = 0;

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime
static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map over a grouped FP32 block ([group][node][4], group stride gs floats) as a
// rank-3 tensor {4 np floats (one grid row), np rows, ng groups}; boxes of box_nodes x
// box_rows nodes of one group.  Zeros are read outside the grid.
static bool tile_map_block(CUtensorMap *m, const float *base, long gs, const GridDesc &g, int ng, int box_nodes,
                           int box_rows) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dim[3] = {4ull * (cuuint64_t)g.np, (cuuint64_t)g.np, (cuuint64_t)ng};
  const cuuint64_t str[2] = {16ull * (cuuint64_t)g.np, 4ull * (cuuint64_t)gs};
  const cuuint32_t box[3] = {4u * (cuuint32_t)box_nodes, (cuuint32_t)box_rows, 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dim, str, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the packed coefficient records (one float4 per node) as a rank-2 tensor {4 np, np}
static bool tile_map_coef(CUtensorMap *m, const float *pk, const GridDesc &g) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dim[2] = {4ull * (cuuint64_t)g.np, (cuuint64_t)g.np};
  const cuuint64_t str[1] = {16ull * (cuuint64_t)g.np};
  const cuuint32_t box[2] = {4u * TLB_X, (cuuint32_t)TLB_Y};
  const cuuint32_t es[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(pk), dim, str, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launches the tiled kernel for a tile grid; false (nothing launched) when a tensor
// map cannot be encoded, and the caller uses the row kernel.
template <int MODE>
static bool tile_launch(const GridDesc &g, const Stencil<float> &S, const float *X, long gx, const float *B, long gb,
                        float *Y, long gy, int s, float omega, float omega2, const Fin &fin, cudaStream_t st) {
  constexpr bool HAS_B = (MODE == M_RESID || MODE == M_JACOBI || MODE == M_JACOBI_DOT);
  const int ng = (s + 3) / 4;
  CUtensorMap mx, mr, mc;
  if (!tile_map_block(&mx, X, gx, g, ng, TLB_X, TLB_Y) || !tile_map_coef(&mc, S.pk, g)) return false;
  if (HAS_B) {
    if (!tile_map_block(&mr, B, gb, g, ng, TLR_X, TLR_Y)) return false;
  } else {
    mr = mx;
  }
  const int ntx = (g.np - 1) / TILE_X, nty = (g.np - 1) / TILE_Y;
  k_st_tile<MODE><<<dim3(ntx * nty, ng), TL_NT, TL_SMEM, st>>>(mx, mr, mc, g, ntx, nty, Y, gy, s, omega, omega2, fin);
  count_launch();
  if (!tl_no_count) g_tiled_launches.fetch_add(1, std::memory_order_relaxed);
  if (MODE == M_APPLY_DOT || MODE == M_JACOBI_DOT) dot_finalize(fin, ntx * nty, s, st);
  return true;
}

// 3D: a grouped block as a rank-4 tensor {4 np floats (one grid row), np rows, np planes,
// ng groups}; boxes of box_x x box_y nodes of one plane of one group
static bool tile3_map_block(CUtensorMap *m, const float *base, long gs, const GridDesc &g, int ng, int box_x,
                            int box_y) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t np = (cuuint64_t)g.np;
  const cuuint64_t dim[4] = {4ull * np, np, np, (cuuint64_t)ng};
  const cuuint64_t str[3] = {16ull * np, 16ull * np * np, 4ull * (cuuint64_t)gs};
  const cuuint32_t box[4] = {4u * (cuuint32_t)box_x, (cuuint32_t)box_y, 1u, 1u};
  const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dim, str, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3D coefficient records as a rank-3 tensor {4 np floats, np, np} (halo boxes), and the
// z couplings in padded rows as a rank-3 tensor {ldr, np, np} (boxes without halo)
static bool tile3_map_coef(CUtensorMap *m, CUtensorMap *mz, const float *pk, const GridDesc &g) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t np = (cuuint64_t)g.np, ldr = (np + 3) / 4 * 4;
  const cuuint64_t dim[3] = {4ull * np, np, np};
  const cuuint64_t str[2] = {16ull * np, 16ull * np * np};
  const cuuint32_t box[3] = {4u * TL3B_X, (cuuint32_t)TL3B_Y, 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  if (fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(pk), dim, str, box, es,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const cuuint64_t dimz[3] = {ldr, np, np};
  const cuuint64_t strz[2] = {4ull * ldr, 4ull * ldr * np};
  const cuuint32_t boxz[3] = {(cuuint32_t)TL3Z_X, (cuuint32_t)TL3R_Y, 1u};
  return fn(mz, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(pk + 4 * g.n), dimz, strz, boxz, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE>
static bool tile3_launch(const GridDesc &g, const Stencil<float> &S, const float *X, long gx, const float *B,
                         long gb, float *Y, long gy, int s, float omega, float omega2, const Fin &fin,
                         cudaStream_t st) {
  constexpr bool HAS_B = (MODE == M_RESID || MODE == M_JACOBI || MODE == M_JACOBI_DOT);
  const int ng = (s + 3) / 4;
  CUtensorMap mx, mr, mc, mz;
  if (!tile3_map_block(&mx, X, gx, g, ng, TL3B_X, TL3B_Y) || !tile3_map_coef(&mc, &mz, S.pk, g)) return false;
  if (HAS_B) {
    if (!tile3_map_block(&mr, B, gb, g, ng, TL3R_X, TL3R_Y)) return false;
  } else {
    mr = mx;
  }
  // the opt-in shared-memory size and the device's resident CTAs, once per mode and device
  // (solves of a batch launch from several host threads; setting the attribute twice is harmless)
  static std::atomic<int> slots[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return false;
  if (slots[dev].load(std::memory_order_acquire) == 0) {
    // an error left pending by earlier work stays for the caller to see: give up the tiled
    // form for this launch without touching it
    if (cudaPeekAtLastError() != cudaSuccess) return false;
    int per_sm = 0, sms = 0;
    if (cudaFuncSetAttribute(k_st_tile3<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tl3_smem<MODE>()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_st_tile3<MODE>, TL3_NT, tl3_smem<MODE>()) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1) {
      (void)cudaGetLastError();  // clears only the refused set-up call's error: the row kernels run instead
      return false;
    }
    slots[dev].store(per_sm * sms, std::memory_order_release);
  }
  const int nslots = slots[dev].load(std::memory_order_acquire);
  // z segments of 16 or 8 planes, whichever the model ceil(w) / w * (zs + 1) / zs puts
  // lower, w being the launch's CTAs over the resident slots: the last, partly filled wave
  // against the per-segment start (the first plane's copies and the plane below).
  // Measured on 64^3 with 120 columns (1920 or 3840 CTAs over 608 slots): 80.3 us with 16
  // planes, 76.2 us with 8 (and 82.3 / 82.1 us with 32 / 4).
  const int ntx = (g.np - 1) / TILE3_X, nty = (g.np - 1) / TILE3_Y;
  int nzs = (g.np - 1) / TILE3_Z;
  {
    double best = 0.0;
    for (int zs = TILE3_Z; zs >= TILE3_Z / 2; zs /= 2) {
      if ((g.np - 1) % zs) continue;
      const double w = (double)ntx * nty * ((g.np - 1) / zs) * ng / nslots;
      const double cost = std::ceil(w) / w * (zs + 1.0) / zs;
      if (best == 0.0 || cost < best * (1.0 - 1e-9)) {
        best = cost;
        nzs = (g.np - 1) / zs;
      }
    }
  }
  k_st_tile3<MODE><<<dim3(ntx * nty * nzs, ng), TL3_NT, tl3_smem<MODE>(), st>>>(
      mx, mr, mc, mz, g, ntx, nty, nzs, X, gx, S.pk, S.pk + 4 * g.n, Y, gy, s, omega, omega2, fin);
  count_launch();
  if (!tl_no_count) g_tiled_launches.fetch_add(1, std::memory_order_relaxed);
  if (MODE == M_APPLY_DOT || MODE == M_JACOBI_DOT) dot_finalize(fin, ntx * nty * nzs, s, st);
  return true;
}

// Algorithmic bytes of one stencil launch: the vectors it reads and writes once (x and y;
// b as well for the residual and sweep modes) and the per-node coefficients (the diagonal
// and the forward couplings; the inverse diagonal as well for the sweeps).
template <typename T, int MODE> static double st_bytes(const GridDesc &g, const Stencil<T> &S, int s) {
  const bool sweep = MODE == M_JACOBI || MODE == M_JACOBI_DOT || MODE == M_JAC2;
  const bool two = MODE == M_APPLY || MODE == M_APPLY_DOT || MODE == M_JAC2;
  return (double)sizeof(T) * (double)g.n * ((two ? 2.0 : 3.0) * s + (sweep ? 2.0 : 1.0) + S.nf);
}

template <typename T, int VW, int MODE>
static void st_launch(const GridDesc &g, const Stencil<T> &S, const T *X, long gx, const T *B, long gb, T *Y, long gy,
                      int s, T omega, const Fin &fin, cudaStream_t st, T omega2 = T(0)) {
  count_bytes(sizeof(T) == 8 && MODE == M_RESID_DOT ? BY_REFINE : level_family(g.n), st_bytes<T, MODE>(g, S, s));
  if constexpr (sizeof(T) == 4 && VW == 4 && MODE != M_RESID_DOT) {
    // tma_tiles 1: every eligible level; 2: the finest level only
    const bool tma = tl_tma == 1 || (tl_tma == 2 && g.n == tl_n0);
    if (tma && S.pk && !S.full && tile_grid(g) &&
        tile_launch<MODE>(g, S, X, gx, B, gb, Y, gy, s, omega, omega2, fin, st))
      return;
    if (tma && S.pk && !S.full && tile3_grid(g) &&
        tile3_launch<MODE>(g, S, X, gx, B, gb, Y, gy, s, omega, omega2, fin, st))
      return;
  }
  const int ng = (s + VW - 1) / VW;
  const dim3 grid = rowgrid_capped(g, ng);
  if (g.dim == 2) {
    if (S.full)
      k_st<T, VW, 2, true, MODE><<<grid, NB, 0, st>>>(g, S.diag, S.invdiag, S.c, X, gx, B, gb, Y, gy, s, omega,
                                                     omega2, fin);
    else
      k_st<T, VW, 2, false, MODE><<<grid, NB, 0, st>>>(g, S.diag, S.invdiag, S.c, X, gx, B, gb, Y, gy, s, omega,
                                                     omega2, fin);
  } else {
    if (S.full)
      k_st<T, VW, 3, true, MODE><<<grid, NB, 0, st>>>(g, S.diag, S.invdiag, S.c, X, gx, B, gb, Y, gy, s, omega,
                                                     omega2, fin);
    else
      k_st<T, VW, 3, false, MODE><<<grid, NB, 0, st>>>(g, S.diag, S.invdiag, S.c, X, gx, B, gb, Y, gy, s, omega,
                                                     omega2, fin);
  }
  count_launch();
  if (MODE == M_APPLY_DOT || MODE == M_JACOBI_DOT || MODE == M_RESID_DOT) dot_finalize(fin, grid.x * grid.y, s, st);
}

template <typename T>
void launch_stencil_apply(const hp_problem *P, const GridDesc &g, const Stencil<T> &S, const T *X, long ldx, T *Y,
                          long ldy, int s, cudaStream_t st) {
  st_launch<T, 1, M_APPLY>(g, S, X, ldx, nullptr, 0, Y, ldy, s, T(0), Fin{}, st);
}
template void launch_stencil_apply<double>(const hp_problem *, const GridDesc &, const Stencil<double> &,
                                           const double *, long, double *, long, int, cudaStream_t);
template void launch_stencil_apply<float>(const hp_problem *, const GridDesc &, const Stencil<float> &, const float *,
                                          long, float *, long, int, cudaStream_t);

static long padded(long n) { return (n + 63) / 64 * 64; }
static int round4(int s) { return (s + 3) / 4 * 4; }

template <typename T> static BlockWS<T> &ws_of(hp_problem *P);
template <> BlockWS<float> &ws_of<float>(hp_problem *P) { return P->w32; }
template <> BlockWS<double> &ws_of<double>(hp_problem *P) { return P->w64; }

// workspace for s columns (capacity rounded up to whole groups of 4)
template <typename T> static int ensure_ws(hp_problem *P, int s) {
  BlockWS<T> &W = ws_of<T>(P);
  const int sc = round4(s);
  if (W.scap >= sc) return 0;
  W.ldn = padded(P->n);
  const size_t blk = sizeof(T) * (size_t)W.ldn * sc;
  HP_TRY(W.x.ensure(blk));
  HP_TRY(W.r.ensure(blk));
  HP_TRY(W.z.ensure(blk));
  HP_TRY(W.p.ensure(blk));
  HP_TRY(W.q.ensure(blk));
  HP_TRY(W.lb[0].ensure(blk));
  for (int l = 1; l < P->L; ++l) {
    const size_t b = sizeof(T) * (size_t)padded(P->lv[l].g.n) * sc;
    HP_TRY(W.lr[l].ensure(b));
    HP_TRY(W.la[l].ensure(b));
    HP_TRY(W.lb[l].ensure(b));
  }
  W.scap = sc;
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
  const int sc = round4(s);
  long nbmax = blocks_for(P->n, 1);
  for (int l = 0; l < std::max(P->L, 1); ++l) nbmax = std::max(nbmax, rowgrid_blocks(P->lv[l].g));
  nbmax = std::max(nbmax, (P->n + NB - 1) / NB);
  if (S.scap >= sc && S.partial.bytes >= sizeof(double) * (size_t)nbmax * sc) return 0;
  const size_t b = sizeof(double) * sc;
  HP_TRY(S.rz.ensure(b));
  HP_TRY(S.pq.ensure(b));
  HP_TRY(S.rr.ensure(b));
  HP_TRY(S.bb.ensure(b));
  HP_TRY(S.alpha.ensure(b));
  HP_TRY(S.beta.ensure(b));
  HP_TRY(S.scale.ensure(b));
  HP_TRY(S.iscale.ensure(b));
  HP_TRY(S.tol2col.ensure(b));
  HP_TRY(S.bbr.ensure(b));
  HP_TRY(S.active.ensure(sizeof(int) * sc));
  HP_TRY(S.partial.ensure(sizeof(double) * (size_t)nbmax * sc));
  HP_TRY(S.counter.ensure(sizeof(unsigned) * sc));
  HP_TRY(S.iter.ensure(sizeof(int) * 4));
  for (DBuf *d : {&S.rz, &S.pq, &S.rr, &S.bb, &S.alpha, &S.beta, &S.scale, &S.iscale, &S.tol2col, &S.bbr})
    HP_CUDA(cudaMemsetAsync(d->p, 0, b, P->st));
  HP_CUDA(cudaMemsetAsync(S.active.p, 0, sizeof(int) * sc, P->st));
  HP_CUDA(cudaMemsetAsync(S.counter.p, 0, sizeof(unsigned) * sc, P->st));
  if (S.hcap < sc) {
    free_scalars_host(P);
    HP_CUDA(cudaMallocHost(&S.h_active, sizeof(int) * sc));
    HP_CUDA(cudaMallocHost(&S.h_iter, sizeof(int) * 4));
    HP_CUDA(cudaMallocHost(&S.h_rr, sizeof(double) * sc));
    HP_CUDA(cudaMallocHost(&S.h_bb, sizeof(double) * sc));
    S.hcap = sc;
  }
  drop_graphs(P);  // captured graphs hold the old scalar pointers
  S.scap = sc;
  return 0;
}

// set while a double-float refinement runs: its converged columns start each inner PCG
// inactive (their scale is 0)
static thread_local const double *tl_open = nullptr;

static Fin make_fin(hp_problem *P, int kind, double tol2 = 0.0, double *out = nullptr) {
  Fin f;
  if (kind == FIN_INIT) f.open = tl_open;
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
  f.tol2col = P->sc.tol2col.as<double>();
  f.tol2 = tol2;
  f.out = out;
  return f;
}

static dim3 nodegrid(long n, int ng) {
  const long b = std::min<long>((n + NB - 1) / NB, std::max<long>(1, tl_max_blocks / ng));
  return dim3((unsigned)b, ng);
}

// ---------------------------------------------------------------------------
// Node steps shared by the coarse-tail kernel below (the same arithmetic as the per-level
// kernels, node by node).
// ---------------------------------------------------------------------------
// S x at node id with the centre value xc given; JS: the
// neighbour values enter as omega D^-1 x (the first sweep of a pair from zero),
// in the same operation order as k_st
template <typename T, int VW, int D, bool FULL, bool JS>
__device__ __forceinline__ Pack<T, VW> vt_apply(const GridDesc &g, const T *diag, const T *invdiag, const T *c,
                                                const T *x, long id, const int v[3], T omega,
                                                const Pack<T, VW> &xc) {
  using PK = Pack<T, VW>;
  constexpr int NF = FULL ? (1 << D) - 1 : D;
  PK sx;
  const T dg = diag[id];
#pragma unroll
  for (int q = 0; q < VW; ++q) sx.v[q] = dg * xc.v[q];
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
    if (fw) {
      const T cf = JS ? c[(long)f * g.n + id] * omega * invdiag[id + off] : c[(long)f * g.n + id];
      sx.axpy(cf, PK::ld(x + (id + off) * VW));
    }
    if (bw) {
      const T cb = JS ? c[(long)f * g.n + id - off] * omega * invdiag[id - off] : c[(long)f * g.n + id - off];
      sx.axpy(cb, PK::ld(x + (id - off) * VW));
    }
  }
  return sx;
}

template <int D>
__device__ __forceinline__ void vt_coords(const GridDesc &g, long id, int v[3]) {
  v[0] = (int)(id % g.np);
  const long t = id / g.np;
  v[1] = D == 2 ? (int)t : (int)(t % g.np);
  v[2] = D == 2 ? 0 : (int)(t / g.np);
}

// ---------------------------------------------------------------------------
// Shared-memory coarse tail: the levels l0 .. L-2 of one column group run in one CTA of
// VS_NT threads with their vectors in shared memory -- the two iterates of level l0 (its
// right-hand side stays in global memory, where the restriction of level l0 - 1 wrote
// it), and the right-hand side and both iterates of each level below -- so the smoothing
// and transfer steps are separated by __syncthreads only, not by launches.  Two launches
// bracket the dense coarse solve (k_coarse_apply, spread over many CTAs): PART 0 runs the
// down leg and leaves each level's iterate (and the right-hand sides below l0) in its
// global level buffers; PART 1 reloads them with the coarse solution and runs the up leg.
// The arithmetic mirrors k_st / k_jacobi0 / k_restrict / k_prolong_add step for step
// (same operations in the same order, explicitly rounded), so the result equals the
// per-level path bit for bit.  The level-l0 correction is written to `dst`.
// ---------------------------------------------------------------------------
constexpr int VS_NT = 1024;

template <typename T> struct VTailS {
  int l0, L, zero_dirichlet, nc;
  int nu[HP_MAXL];
  T w[HP_MAXL][4];
  GridDesc g[HP_MAXL];
  const T *diag[HP_MAXL], *invdiag[HP_MAXL], *c[HP_MAXL];
  const T *r0;  // level-l0 right-hand side (global, group stride gs0)
  T *dst;       // level-l0 correction (global, group stride gs0)
  long gs0;
  T *rg[HP_MAXL], *ag[HP_MAXL];  // global right-hand side / iterate buffers of each level
  long gs[HP_MAXL];               // their group strides
  unsigned off_r[HP_MAXL], off_a[HP_MAXL], off_b[HP_MAXL];  // shared-memory byte offsets
};

template <typename T, int VW, int D, bool FULL, int PART>
__global__ void __launch_bounds__(VS_NT) k_vtail_smem(VTailS<T> vt) {
  using PK = Pack<T, VW>;
  extern __shared__ __align__(16) unsigned char vs_smem[];
  const int grp = blockIdx.y;
  auto S = [&](unsigned off) { return reinterpret_cast<T *>(vs_smem + off); };
  // one node step over level l: mode 0 two sweeps from zero (x = rhs, weights w1, w2),
  // 1 one sweep from zero (w1), 2 sweep (x, rhs b, w1), 3 residual b - S x
  auto sweep = [&](int l, int mode, const T *x, const T *b, T *y, T w1, T w2) {
    const GridDesc &g = vt.g[l];
    const T *dg = vt.diag[l], *iv = vt.invdiag[l], *cc = vt.c[l];
    for (long id = threadIdx.x; id < g.n; id += VS_NT) {
      int v[3];
      vt_coords<D>(g, id, v);
      PK out;
      if (mode == 0) {
        const T wi = w1 * iv[id], wi2 = w2 * iv[id];
        const PK r = PK::ld(x + id * VW);
        PK e1c;
#pragma unroll
        for (int q = 0; q < VW; ++q) e1c.v[q] = wi * r.v[q];
        const PK sx = vt_apply<T, VW, D, FULL, true>(g, dg, iv, cc, x, id, v, w1, e1c);
#pragma unroll
        for (int q = 0; q < VW; ++q) out.v[q] = fmadd(wi2, r.v[q] - sx.v[q], e1c.v[q]);
      } else if (mode == 1) {
        const T wi = w1 * iv[id];
        const PK r = PK::ld(x + id * VW);
#pragma unroll
        for (int q = 0; q < VW; ++q) out.v[q] = wi * r.v[q];
      } else {
        const PK xc = PK::ld(x + id * VW);
        const PK sx = vt_apply<T, VW, D, FULL, false>(g, dg, iv, cc, x, id, v, T(0), xc);
        const PK bb = PK::ld(b + id * VW);
        if (mode == 3) {
#pragma unroll
          for (int q = 0; q < VW; ++q) out.v[q] = bb.v[q] - sx.v[q];
        } else {
          const T wi = w1 * iv[id];
#pragma unroll
          for (int q = 0; q < VW; ++q) out.v[q] = fmadd(wi, bb.v[q] - sx.v[q], xc.v[q]);
        }
      }
      out.st(y + id * VW);
    }
    __syncthreads();
  };
  auto copy = [&](long n, const T *src, T *dst_) {
    for (long id = threadIdx.x; id < n; id += VS_NT) PK::ld(src + id * VW).st(dst_ + id * VW);
  };
  const T *r0 = vt.r0 + grp * vt.gs0;
  T *cur[HP_MAXL], *oth[HP_MAXL];
  if (PART == 1) {
    // reload: each level's iterate and the right-hand sides below l0, the coarse solution
    for (int l = vt.l0; l < vt.L; ++l) {
      copy(vt.g[l].n, vt.ag[l] + grp * vt.gs[l], S(vt.off_a[l]));
      if (l > vt.l0 && l + 1 < vt.L) copy(vt.g[l].n, vt.rg[l] + grp * vt.gs[l], S(vt.off_r[l]));
      cur[l] = S(vt.off_a[l]);
      oth[l] = S(vt.off_b[l]);
    }
    __syncthreads();
  }
  for (int l = vt.l0; PART == 0 && l + 1 < vt.L; ++l) {
    const T *rl = l == vt.l0 ? r0 : S(vt.off_r[l]);
    const int nul = vt.nu[l];
    T *c = nul >= 2 ? S(vt.off_a[l]) : S(vt.off_b[l]);
    T *o = nul >= 2 ? S(vt.off_b[l]) : S(vt.off_a[l]);
    sweep(l, nul >= 2 ? 0 : 1, rl, nullptr, c, vt.w[l][0], vt.w[l][1]);
    for (int k = 2; k < nul; ++k) {
      sweep(l, 2, c, rl, o, vt.w[l][k], T(0));
      T *t = c;
      c = o;
      o = t;
    }
    sweep(l, 3, c, rl, o, T(0), T(0));
    // restriction to level l + 1 (transpose of the P1 prolongation)
    {
      const GridDesc &gf = vt.g[l], &gc = vt.g[l + 1];
      T *rc = S(vt.off_r[l + 1]);
      for (long I = threadIdx.x; I < gc.n; I += VS_NT) {
        int J[3];
        vt_coords<D>(gc, I, J);
        PK out = PK::zero();
        if (!(vt.zero_dirichlet && (J[D - 1] == 0 || J[D - 1] == gc.N))) {
          const long f0 = 2 * (long)J[0] + (long)gf.np * (2 * (long)J[1] + (D == 3 ? (long)gf.np * 2 * J[2] : 0));
          out = PK::ld(o + f0 * VW);
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
            if (fw) out.axpy(T(0.5), PK::ld(o + (f0 + off) * VW));
            if (bw) out.axpy(T(0.5), PK::ld(o + (f0 - off) * VW));
          }
        }
        out.st(rc + I * VW);
      }
    }
    __syncthreads();
    cur[l] = c;
    oth[l] = o;
  }
  if (PART == 0) {
    // hand over through the global level buffers: iterates, and the right-hand sides
    // below l0 (the coarsest one is the coarse solve's input)
    for (int l = vt.l0; l < vt.L; ++l) {
      if (l + 1 < vt.L) copy(vt.g[l].n, cur[l], vt.ag[l] + grp * vt.gs[l]);
      if (l > vt.l0) copy(vt.g[l].n, S(vt.off_r[l]), vt.rg[l] + grp * vt.gs[l]);
    }
    return;
  }
  for (int l = vt.L - 2; l >= vt.l0; --l) {
    // e_l += P e_{l+1}
    {
      const GridDesc &gf = vt.g[l], &gc = vt.g[l + 1];
      const T *e = cur[l + 1];
      T *ef = cur[l];
      for (long i = threadIdx.x; i < gf.n; i += VS_NT) {
        int v[3];
        vt_coords<D>(gf, i, v);
        const int b = (v[0] & 1) | ((v[1] & 1) << 1) | ((v[2] & 1) << 2);
        const long ic = (v[0] >> 1) + (long)gc.np * ((v[1] >> 1) + (long)gc.np * (v[2] >> 1));
        PK val = PK::ld(e + ic * VW);
        if (b) {
          const PK v2 = PK::ld(e + (ic + mask_offset(gc, b)) * VW);
#pragma unroll
          for (int q = 0; q < VW; ++q) val.v[q] = mulr(T(0.5), val.v[q] + v2.v[q]);
        }
        PK cv = PK::ld(ef + i * VW);
#pragma unroll
        for (int q = 0; q < VW; ++q) cv.v[q] = addr(cv.v[q], val.v[q]);
        cv.st(ef + i * VW);
      }
    }
    __syncthreads();
    const T *rl = l == vt.l0 ? r0 : S(vt.off_r[l]);
    T *c = cur[l], *o = oth[l];
    const int nul = vt.nu[l];
    for (int k = 0; k < nul; ++k) {
      T *y = (l == vt.l0 && k == nul - 1) ? vt.dst + grp * vt.gs0 : o;
      sweep(l, 2, c, rl, y, vt.w[l][nul - 1 - k], T(0));
      T *t = c;
      c = o;
      o = t;
    }
    cur[l] = c;
  }
}

// Smoothing weights of level l, sweep k = 0 .. nu-1 (pre-smoothing applies them in this
// order, post-smoothing in reverse, so the V-cycle stays symmetric).  Damped Jacobi: omega
// every sweep.  Chebyshev: the reciprocals of the roots of the degree-nu Chebyshev
// polynomial on [lmax / alpha, lmax], lmax the Gershgorin bound of diag^-1 S, so that the
// smoother damps that interval optimally and every |1 - w lambda| product stays below 1 on
// (0, lmax].
// smoothing sweeps at level l (nu_coarse, when set, on the coarser levels)
static int nu_at(const hp_problem *P, int l) { return (l > 0 && P->nu_coarse > 0) ? P->nu_coarse : P->nu; }
// residual + restriction and prolongation + first post sweep fused at level l: on every
// level (fuse_transfer 1) or below the finest only (2), where launches, not bytes, dominate
static bool fuse_at(const hp_problem *P, int l) { return P->fuse_transfer == 1 || (P->fuse_transfer == 2 && l >= 1); }

template <typename T>
static void smooth_weights(const hp_problem *P, OpKind op, int l, T w[4]) {
  const int nu = nu_at(P, l);
  if (P->smoother != 1) {
    for (int k = 0; k < 4; ++k) w[k] = (T)P->omega;
    return;
  }
  const double b = stencil_of<double>(P, op, l).lmax, a = b / P->cheb_alpha;
  const double c = 0.5 * (a + b), d = 0.5 * (b - a);
  for (int k = 0; k < 4; ++k)
    w[k] = k < nu ? (T)(1.0 / (c - d * std::cos(M_PI * (2.0 * k + 1.0) / (2.0 * nu)))) : T(0);
}

// opt-in maximum of shared memory per CTA on the current device
static int smem_optin() {
  static thread_local int dev = -1, val = 0;
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return 0;
  if (d != dev) {
    if (cudaDeviceGetAttribute(&val, cudaDevAttrMaxSharedMemoryPerBlockOptin, d) != cudaSuccess) val = 0;
    dev = d;
  }
  return val;
}

// Shared-memory layout of the coarse tail from level l0 for node_bytes per node (bytes of
// one group's values at one node); fills the offsets when vt is given, returns the total.
template <typename T>
static size_t smem_tail_layout(const hp_problem *P, int l0, int node_bytes, VTailS<T> *vt) {
  const int L = P->L;
  size_t off = 0;
  auto take = [&](long n) {
    const size_t o = off;
    off += ((size_t)n * node_bytes + 15) / 16 * 16;
    return (unsigned)o;
  };
  for (int l = l0; l < L; ++l) {
    const long n = P->lv[l].g.n;
    const unsigned r = (l > l0) ? take(n) : 0u;  // level l0 reads its right-hand side from global memory
    const unsigned a = take(n);
    const unsigned b = (l < L - 1) ? take(n) : 0u;
    if (vt) {
      vt->off_r[l] = r;
      vt->off_a[l] = a;
      vt->off_b[l] = b;
    }
  }
  return off;
}

// first level of the shared-memory coarse tail for this solve, or L (no fusion): the lowest
// level, from smem_tail on, whose tail fits in a CTA's shared memory (at least one level
// above the coarsest)
static int tail_level(const hp_problem *P, int node_bytes) {
  if (P->smem_tail) {
    const size_t cap = (size_t)smem_optin();
    for (int l0 = std::max(1, P->smem_tail); l0 + 2 <= P->L; ++l0)
      if (smem_tail_layout<float>(P, l0, node_bytes, nullptr) <= cap) return l0;
  }
  return P->L;
}

// Algorithmic bytes of the V-cycle's levels l0 .. L-1 as the per-level kernels would move
// them (smoothing sweeps, residual, restriction, prolongation, the dense coarse solve): the
// fused tails do the same work in fewer launches, and are counted with these bytes.
template <typename T>
static double tail_bytes(const hp_problem *P, OpKind op, int s, int l0) {
  const double w = sizeof(T);
  double b = 0.0;
  for (int l = l0; l + 1 < P->L; ++l) {
    const double n = (double)P->lv[l].g.n, nc = (double)P->lv[l + 1].g.n;
    const double nf = stencil_of<T>(P, op, l).nf;
    const int nu = nu_at(P, l);
    const double sweep = (3.0 * s + 2.0 + nf) * n * w;
    b += nu >= 2 ? (2.0 * s + 2.0 + nf) * n * w + (nu - 2) * sweep : (2.0 * s + 1.0) * n * w;  // pre-smoothing
    b += (3.0 * s + 1.0 + nf) * n * w + s * (n + nc) * w;                                     // residual, restriction
    b += s * (2.0 * n + nc) * w + nu * sweep;                                                  // prolongation, post-smoothing
  }
  const double nc = (double)P->lv[P->L - 1].g.n;
  return b + (nc * nc + 2.0 * nc * s) * w;
}

// The shared-memory tail as its two launches around the dense coarse solve.
template <typename T, int VW>
static void launch_vtail_smem(hp_problem *P, OpKind op, int s, int l0, const T *const *rl, T *const *ea,
                              const long *gsl, T *dst) {
  const int L = P->L, ng = (s + VW - 1) / VW;
  VTailS<T> vt{};
  vt.l0 = l0;
  vt.L = L;
  vt.zero_dirichlet = op == OP_K;
  vt.nc = (int)P->lv[L - 1].g.n;
  for (int l = 0; l < L; ++l) {
    vt.nu[l] = nu_at(P, l);
    smooth_weights<T>(P, op, l, vt.w[l]);
    const Stencil<T> &S = stencil_of<T>(P, op, l);
    vt.g[l] = P->lv[l].g;
    vt.diag[l] = S.diag;
    vt.invdiag[l] = S.invdiag;
    vt.c[l] = S.c;
    vt.rg[l] = const_cast<T *>(rl[l]);
    vt.ag[l] = ea[l];
    vt.gs[l] = gsl[l];
  }
  vt.r0 = rl[l0];
  vt.dst = dst;
  vt.gs0 = gsl[l0];
  const size_t bytes = smem_tail_layout<T>(P, l0, (int)(sizeof(T) * VW), &vt);
  const bool full = stencil_of<T>(P, op, l0).full;
  void (*down)(VTailS<T>) = nullptr, (*up)(VTailS<T>) = nullptr;
  if (P->lv[0].g.dim == 2) {
    down = full ? k_vtail_smem<T, VW, 2, true, 0> : k_vtail_smem<T, VW, 2, false, 0>;
    up = full ? k_vtail_smem<T, VW, 2, true, 1> : k_vtail_smem<T, VW, 2, false, 1>;
  } else {
    down = full ? k_vtail_smem<T, VW, 3, true, 0> : k_vtail_smem<T, VW, 3, false, 0>;
    up = full ? k_vtail_smem<T, VW, 3, true, 1> : k_vtail_smem<T, VW, 3, false, 1>;
  }
  // every caller sets the same limit (the device's opt-in maximum less the kernel's static
  // shared memory), so solves launching from several host threads never lower it under
  // one another's launch; the launch's own size is the fallback
  auto allow = [&](void (*k)(VTailS<T>)) {
    cudaFuncAttributes fa{};
    int cap = smem_optin();
    const bool clean = cudaPeekAtLastError() == cudaSuccess;  // an earlier error stays for the caller
    if (cudaFuncGetAttributes(&fa, k) == cudaSuccess) cap -= (int)fa.sharedSizeBytes;
    if (cap < (int)bytes || cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess) {
      if (clean) (void)cudaGetLastError();  // a refused limit is not an error of the solve
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    }
  };
  allow(down);
  allow(up);
  down<<<dim3(1, ng), VS_NT, bytes, P->st>>>(vt);
  const int lc = L - 1, nc = (int)P->lv[lc].g.n;
  k_coarse_apply<T, VW><<<dim3((nc + 31) / 32, ng), 256, sizeof(T) * nc * VW, P->st>>>(
      coarse_inv<T>(P, op), nc, rl[lc], gsl[lc], ea[lc], gsl[lc]);
  up<<<dim3(1, ng), VS_NT, bytes, P->st>>>(vt);
  count_launch(3);
  count_bytes(BY_STENCILC, tail_bytes<T>(P, op, s, l0));
}

// Preconditioner z = M^{-1} r with the fused <r, z> -> fin.
template <typename T, int VW>
static void precondition(hp_problem *P, OpKind op, int s, const T *r0, T *z0, const Fin &fin) {
  BlockWS<T> &W = ws_of<T>(P);
  cudaStream_t st = P->st;
  const T om = (T)P->omega;
  const int ng = (s + VW - 1) / VW;
  const long gs0 = W.ldn * VW;
  if (op == OP_M) {  // Jacobi
    const Stencil<T> &S = stencil_of<T>(P, op, 0);
    const dim3 gr = nodegrid(P->n, ng);
    k_jacobi0<T, VW><<<gr, NB, 0, st>>>(P->n, S.invdiag, r0, gs0, z0, T(1), s, fin, 1);
    count_launch();
    count_bytes(BY_STENCIL0, (double)sizeof(T) * (double)P->n * (2.0 * s + 1.0));
    dot_finalize(fin, gr.x, s, st);
    return;
  }
  const int L = P->L;
  if (L == 1) {  // the coarse solve is the whole preconditioner; the caller forms <r, z>
    const int nc = (int)P->lv[0].g.n;
    k_coarse_apply<T, VW><<<dim3((nc + 31) / 32, ng), 256, sizeof(T) * nc * VW, st>>>(coarse_inv<T>(P, op), nc, r0,
                                                                                       gs0, z0, gs0);
    count_launch();
    count_bytes(BY_STENCILC, (double)sizeof(T) * ((double)nc * nc + 2.0 * nc * s));
    return;
  }
  const T *rl[HP_MAXL];
  T *ea[HP_MAXL], *eb[HP_MAXL];
  long gsl[HP_MAXL];
  rl[0] = r0;
  ea[0] = z0;
  eb[0] = W.lb[0].template as<T>();
  gsl[0] = gs0;
  for (int l = 1; l < L; ++l) {
    rl[l] = W.lr[l].template as<T>();
    ea[l] = W.la[l].template as<T>();
    eb[l] = W.lb[l].template as<T>();
    gsl[l] = padded(P->lv[l].g.n) * VW;
  }
  T *cur[HP_MAXL], *oth[HP_MAXL];
  const Fin nofin{};
  const int l0 = tail_level(P, (int)(sizeof(T) * VW));  // levels >= l0 run inside one launch
  for (int l = 0; l + 1 < L; ++l) {
    const int nu = nu_at(P, l);
    if (l >= l0) {  // buffer bookkeeping only: the fused kernel makes the same choices
      T *c = nu >= 2 ? ea[l] : eb[l], *o = nu >= 2 ? eb[l] : ea[l];
      for (int k = 2; k < nu; ++k) std::swap(c, o);
      cur[l] = c;
      oth[l] = o;
      continue;
    }
    const GridDesc &g = P->lv[l].g;
    const Stencil<T> &S = stencil_of<T>(P, op, l);
    T w[4];
    smooth_weights<T>(P, op, l, w);
    // Pre-smoothing from zero.  Each later sweep flips buffers (nu - 2 more pre, nu post), so the
    // fused two-sweep kernel writes ea[l] and the single sweep (nu = 1) writes eb[l]: either way the
    // level's final correction lands in ea[l] (z0 at level 0).
    T *c = nu >= 2 ? ea[l] : eb[l], *o = nu >= 2 ? eb[l] : ea[l];
    int pr = prof_start(P, l == 0 ? (nu >= 2 ? PROF_PRESMOOTH : PROF_SMOOTH) : -1);
    if (nu >= 2) {
      st_launch<T, VW, M_JAC2>(g, S, rl[l], gsl[l], nullptr, 0, c, gsl[l], s, w[0], nofin, st, w[1]);
    } else {
      k_jacobi0<T, VW><<<nodegrid(g.n, ng), NB, 0, st>>>(g.n, S.invdiag, rl[l], gsl[l], c, w[0], s, nofin, 0);
      count_launch();
      count_bytes(level_family(g.n), (double)sizeof(T) * (double)g.n * (2.0 * s + 1.0));
    }
    prof_stop(P, pr);
    for (int k = 2; k < nu; ++k) {
      pr = prof_start(P, l == 0 ? PROF_SMOOTH : -1);
      st_launch<T, VW, M_JACOBI>(g, S, c, gsl[l], rl[l], gsl[l], o, gsl[l], s, w[k], nofin, st);
      prof_stop(P, pr);
      std::swap(c, o);
    }
    const GridDesc &gc = P->lv[l + 1].g;
    T *rc = const_cast<T *>(rl[l + 1]);
    if (fuse_at(P, l)) {
      // residual and restriction in one pass (the fine residual is not stored)
      const dim3 gr = rowgrid(gc, ng);
      const int zd = op == OP_K;
      if (g.dim == 2) {
        if (S.full)
          k_resid_restrict<T, VW, 2, true><<<gr, NB, 0, st>>>(g, gc, S.diag, S.c, c, rl[l], gsl[l], rc, gsl[l + 1], zd);
        else
          k_resid_restrict<T, VW, 2, false><<<gr, NB, 0, st>>>(g, gc, S.diag, S.c, c, rl[l], gsl[l], rc, gsl[l + 1], zd);
      } else {
        if (S.full)
          k_resid_restrict<T, VW, 3, true><<<gr, NB, 0, st>>>(g, gc, S.diag, S.c, c, rl[l], gsl[l], rc, gsl[l + 1], zd);
        else
          k_resid_restrict<T, VW, 3, false><<<gr, NB, 0, st>>>(g, gc, S.diag, S.c, c, rl[l], gsl[l], rc, gsl[l + 1], zd);
      }
      count_launch();
      count_bytes(BY_TRANSFER, (double)sizeof(T) * ((2.0 * s + 1.0 + S.nf) * (double)g.n + (double)s * gc.n));
    } else {
      pr = prof_start(P, l == 0 ? PROF_RESID_MG : -1);
      st_launch<T, VW, M_RESID>(g, S, c, gsl[l], rl[l], gsl[l], o, gsl[l], s, om, nofin, st);
      prof_stop(P, pr);
      if (g.dim == 2)
        k_restrict<T, VW, 2><<<flatgrid(gc, ng), NB, 0, st>>>(g, gc, o, gsl[l], rc, gsl[l + 1], op == OP_K);
      else
        k_restrict<T, VW, 3><<<flatgrid(gc, ng), NB, 0, st>>>(g, gc, o, gsl[l], rc, gsl[l + 1], op == OP_K);
      count_launch();
      count_bytes(BY_TRANSFER, (double)sizeof(T) * s * ((double)g.n + (double)gc.n));
    }
    cur[l] = c;
    oth[l] = o;
  }
  if (l0 < L) {
    cur[L - 1] = ea[L - 1];
    for (int l = L - 2; l >= l0; --l) {
      T *c = cur[l], *o = oth[l];
      for (int k = 0; k < nu_at(P, l); ++k) std::swap(c, o);
      cur[l] = c;
    }
    launch_vtail_smem<T, VW>(P, op, s, l0, rl, ea, gsl, cur[l0]);
  } else {
    const int lc = L - 1;
    const int nc = (int)P->lv[lc].g.n;
    k_coarse_apply<T, VW><<<dim3((nc + 31) / 32, ng), 256, sizeof(T) * nc * VW, st>>>(coarse_inv<T>(P, op), nc,
                                                                                       rl[lc], gsl[lc], ea[lc], gsl[lc]);
    count_launch();
    count_bytes(BY_STENCILC, (double)sizeof(T) * ((double)nc * nc + 2.0 * nc * s));
    cur[lc] = ea[lc];
  }
  for (int l = std::min(L, l0) - 2 + (l0 < L ? 1 : 0); l >= 0; --l) {
    const GridDesc &g = P->lv[l].g, &gc = P->lv[l + 1].g;
    const Stencil<T> &S = stencil_of<T>(P, op, l);
    const int nu = nu_at(P, l);
    T *c = cur[l], *o = oth[l];
    T w[4];
    smooth_weights<T>(P, op, l, w);
    int k0 = 0;
    if (fuse_at(P, l) && nu >= 2) {
      // prolongation and the first post-smoothing sweep in one pass (x + P e_c is not stored)
      const dim3 gr = rowgrid_capped(g, ng);
      const T *ec = cur[l + 1];
      if (g.dim == 2) {
        if (S.full)
          k_prolong_sweep<T, VW, 2, true><<<gr, NB, 0, st>>>(g, gc, S.diag, S.invdiag, S.c, c, ec, gsl[l + 1], rl[l],
                                                             o, gsl[l], w[nu - 1]);
        else
          k_prolong_sweep<T, VW, 2, false><<<gr, NB, 0, st>>>(g, gc, S.diag, S.invdiag, S.c, c, ec, gsl[l + 1], rl[l],
                                                              o, gsl[l], w[nu - 1]);
      } else {
        if (S.full)
          k_prolong_sweep<T, VW, 3, true><<<gr, NB, 0, st>>>(g, gc, S.diag, S.invdiag, S.c, c, ec, gsl[l + 1], rl[l],
                                                             o, gsl[l], w[nu - 1]);
        else
          k_prolong_sweep<T, VW, 3, false><<<gr, NB, 0, st>>>(g, gc, S.diag, S.invdiag, S.c, c, ec, gsl[l + 1], rl[l],
                                                              o, gsl[l], w[nu - 1]);
      }
      count_launch();
      count_bytes(BY_TRANSFER, (double)sizeof(T) * ((3.0 * s + 2.0 + S.nf) * (double)g.n + (double)s * gc.n));
      std::swap(c, o);
      k0 = 1;
    } else {
      if (g.dim == 2)
        k_prolong_add<T, VW, 2><<<flatgrid(g, ng), NB, 0, st>>>(g, gc, cur[l + 1], gsl[l + 1], cur[l], gsl[l]);
      else
        k_prolong_add<T, VW, 3><<<flatgrid(g, ng), NB, 0, st>>>(g, gc, cur[l + 1], gsl[l + 1], cur[l], gsl[l]);
      count_launch();
      count_bytes(BY_TRANSFER, (double)sizeof(T) * s * (2.0 * (double)g.n + (double)gc.n));
    }
    for (int k = k0; k < nu; ++k) {
      const int pr = prof_start(P, l == 0 ? PROF_SMOOTH : -1);
      if (l == 0 && k == nu - 1)
        st_launch<T, VW, M_JACOBI_DOT>(g, S, c, gsl[l], rl[l], gsl[l], o, gsl[l], s, w[nu - 1 - k], fin, st);
      else
        st_launch<T, VW, M_JACOBI>(g, S, c, gsl[l], rl[l], gsl[l], o, gsl[l], s, w[nu - 1 - k], nofin, st);
      prof_stop(P, pr);
      std::swap(c, o);
    }
    cur[l] = c;
  }
}

// PCG on W.r (overwritten) -> W.x.
//   init:  x = 0, p = 0, bb = rr = <r, r>, active = bb > 0, iter = 0
//   body:  z = M r, beta = <r,z>/rz (0 at iter 0), p = z + beta p,
//          q = K p, alpha = rz/<p,q>, x += alpha p, r -= alpha q, rr = <r,r>,
//          active &= rr > tol^2 bb, iter += 1; repeat while any active and iter < maxit.
template <typename T, int VW>
static void pcg_init(hp_problem *P, OpKind op, int s, cudaGraphConditionalHandle h, int use_handle, int maxit) {
  BlockWS<T> &W = ws_of<T>(P);
  cudaStream_t st = P->st;
  const int ng = (s + VW - 1) / VW;
  const long gs = W.ldn * VW;
  cudaMemsetAsync(W.x.p, 0, sizeof(T) * gs * ng, st);
  cudaMemsetAsync(W.p.p, 0, sizeof(T) * gs * ng, st);
  cudaMemsetAsync(P->sc.iter.p, 0, sizeof(int), st);
  T *r = W.r.template as<T>();
  const dim3 gr = nodegrid(P->n, ng);
  k_dot<T, VW><<<gr, NB, 0, st>>>(P->n, gs, r, r, s, make_fin(P, FIN_INIT));
  dot_finalize(make_fin(P, FIN_INIT), gr.x, s, st);
  count_bytes(BY_VECTOR, (double)sizeof(T) * (double)P->n * s);
  k_pcg_cond<<<1, 256, 0, st>>>(P->sc.active.as<int>(), s, P->sc.iter.as<int>(), maxit, 0, h, use_handle);
  count_launch(2);
}

template <typename T, int VW>
static void pcg_body(hp_problem *P, OpKind op, int s, double tol2, cudaGraphConditionalHandle h, int use_handle,
                     int maxit) {
  BlockWS<T> &W = ws_of<T>(P);
  cudaStream_t st = P->st;
  const long n = P->n;
  const int ng = (s + VW - 1) / VW;
  const long gs = W.ldn * VW;
  T *x = W.x.template as<T>(), *r = W.r.template as<T>(), *z = W.z.template as<T>();
  T *p = W.p.template as<T>(), *q = W.q.template as<T>();
  const GridDesc &g0 = P->lv[0].g;
  const Stencil<T> &S0 = stencil_of<T>(P, op, 0);
  int pr = prof_start(P, PROF_VCYCLE);
  precondition<T, VW>(P, op, s, r, z, make_fin(P, FIN_BETA));
  prof_stop(P, pr);
  if (op != OP_M && P->L == 1) {
    const dim3 gr = nodegrid(n, ng);
    k_dot<T, VW><<<gr, NB, 0, st>>>(n, gs, r, z, s, make_fin(P, FIN_BETA));
    count_launch();
    count_bytes(BY_VECTOR, (double)sizeof(T) * (double)n * 2.0 * s);
    dot_finalize(make_fin(P, FIN_BETA), gr.x, s, st);
  }
  k_p_update<T, VW><<<nodegrid(n, ng), NB, 0, st>>>(n, gs, z, p, P->sc.beta.as<double>());
  count_launch();
  count_bytes(BY_VECTOR, (double)sizeof(T) * (double)n * 3.0 * s);
  pr = prof_start(P, PROF_MATVEC);
  st_launch<T, VW, M_APPLY_DOT>(g0, S0, p, gs, nullptr, 0, q, gs, s, T(0), make_fin(P, FIN_ALPHA), st);
  prof_stop(P, pr);
  pr = prof_start(P, PROF_CG_UPDATE);
  const dim3 gu = nodegrid(n, ng);
  k_cg_update<T, VW><<<gu, NB, 0, st>>>(n, gs, p, q, x, r, P->sc.alpha.as<double>(), s, make_fin(P, FIN_RR, tol2));
  dot_finalize(make_fin(P, FIN_RR, tol2), gu.x, s, st);
  count_bytes(BY_VECTOR, (double)sizeof(T) * (double)n * 6.0 * s);
  prof_stop(P, pr);
  k_pcg_cond<<<1, 256, 0, st>>>(P->sc.active.as<int>(), s, P->sc.iter.as<int>(), maxit, 1, h, use_handle);
  count_launch(2);
}

void drop_graphs(hp_problem *P) {
  for (auto &g : P->graphs) cudaGraphExecDestroy(g.exec);
  P->graphs.clear();
  for (auto &g : P->sgraphs) cudaGraphExecDestroy(g.exec);
  P->sgraphs.clear();
}

// the node a capture on `st` would depend on next (the last one captured)
static cudaError_t capture_leaf(cudaStream_t st, cudaGraphNode_t *leaf) {
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive || nd != 1) return cudaErrorStreamCaptureInvalidated;
  *leaf = deps[0];
  return cudaSuccess;
}

// Appends the PCG to graph g after node dep (none if null): the captured init, then a
// conditional WHILE node whose body is one PCG iteration; *last receives the while node.
// Capture runs on P->cap with P->st pointed at it by the caller.
template <typename T, int VW>
static cudaError_t append_pcg(hp_problem *P, OpKind op, int s, double tol, int maxit, cudaGraph_t g,
                              cudaGraphNode_t dep, cudaGraphNode_t *last) {
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(P->cap, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0,
                                    cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  pcg_init<T, VW>(P, op, s, h, 1, maxit);
  cudaGraphNode_t leaf = nullptr;
  const cudaError_t el = capture_leaf(P->cap, &leaf);
  cudaGraph_t gg = g;
  e = cudaStreamEndCapture(P->cap, &gg);
  if (el != cudaSuccess) return el;
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  e = cudaGraphAddNode(last, g, &leaf, nullptr, 1, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(P->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  pcg_body<T, VW>(P, op, s, tol * tol, h, 1, maxit);
  return cudaStreamEndCapture(P->cap, &body);
}

// Runs fn with launches redirected to the capture stream, profiling off and the launch
// counter paused (captured launches are counted when the graph runs).
template <typename F>
static int with_capture_stream(hp_problem *P, F fn) {
  if (!P->cap) HP_CUDA(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
  cudaStream_t saved = P->st;
  const bool saved_prof = P->prof_on;
  P->prof_on = false;
  P->st = P->cap;
  tl_no_count = 1;
  const int rc = fn();
  P->st = saved;
  P->prof_on = saved_prof;
  tl_no_count = 0;
  return rc;
}

// Captures init + a conditional WHILE node whose body is one PCG iteration.
template <typename T, int VW>
static int build_graph(hp_problem *P, OpKind op, int s, double tol, int maxit, PcgGraph *out) {
  return with_capture_stream(P, [&]() -> int {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    cudaGraphNode_t last = nullptr;
    if (e == cudaSuccess) e = append_pcg<T, VW>(P, op, s, tol, maxit, g, nullptr, &last);
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_check(e, "PCG graph");
    *out = PcgGraph{(int)op, (int)sizeof(T), VW, s, maxit, tol, ex};
    return 0;
  });
}

static int kernels_per_iteration(const hp_problem *P, OpKind op, int node_bytes) {
  if (op == OP_M) return 8;
  // V-cycle: per non-coarsest level pre (1 + nu - 2), resid, restrict, prolong, nu post; coarse 1
  // (with the shared-memory tail from tail_level on: down leg, coarse solve, up leg = 3
  // launches); plus p update, matvec, cg update, condition and three dot finalisations
  const int tl = tail_level(P, node_bytes);
  const int separate = std::min(P->L, tl) - 1 + (tl < P->L ? 1 : 0);
  int vc = 0;
  for (int l = 0; l < separate; ++l) {
    const int nu = nu_at(P, l);
    vc += (nu >= 2 ? nu - 1 : 1) + nu + (fuse_at(P, l) ? (nu >= 2 ? 1 : 2) : 3);
  }
  return 7 + vc + 1 + 2 * (P->L == 1) + ((P->smem_tail && tl < P->L) ? 2 : 0);
}

// after a PCG: fails the solve if a tile kernel gave up waiting for its copies
// (h_it[1] holds the flag read back with the iteration count), and clears the flag
static int tile_timeout_check(hp_problem *P, const int *h_it) {
  if (!h_it[1]) return 0;
  static const int zero = 0;
  cudaMemcpyToSymbolAsync(g_tile_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, P->st);
  cudaStreamSynchronize(P->st);
  return set_error(HP_ERR_CUDA, "a tiled stencil kernel timed out waiting for its tensor copies");
}

template <typename T, int VW>
static int pcg(hp_problem *P, OpKind op, int s, double rtol, int maxit, int *its) {
  cudaStream_t st = P->st;
  int *h_it = P->sc.h_iter;
  if (P->use_graphs && !P->prof_on) {
    PcgGraph *G = nullptr;
    for (auto &pg : P->graphs)
      if (pg.op == (int)op && pg.tbytes == (int)sizeof(T) && pg.vw == VW && pg.s == s && pg.maxit == maxit &&
          pg.tol == rtol)
        G = &pg;
    if (!G) {
      PcgGraph ng;
      HP_TRY((build_graph<T, VW>(P, op, s, rtol, maxit, &ng)));
      P->graphs.push_back(ng);
      G = &P->graphs.back();
    }
    HP_CUDA(cudaGraphLaunch(G->exec, st));
    HP_CUDA(cudaMemcpyAsync(h_it, P->sc.iter.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaMemcpyFromSymbolAsync(h_it + 1, g_tile_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaStreamSynchronize(st));
    count_launch((unsigned long long)(*h_it) * kernels_per_iteration(P, op, (int)(sizeof(T) * VW)) + 2);
    *its = *h_it;
    HP_TRY(tile_timeout_check(P, h_it));
    return *h_it >= maxit ? HP_ERR_NOT_CONVERGED : 0;
  }
  const double tol2 = rtol * rtol;
  pcg_init<T, VW>(P, op, s, 0, 0, maxit);
  int *hact = P->sc.h_active;
  // Profiling: a bounded clock spin heads each iteration so that the host has
  // enqueued the whole iteration before the GPU reaches it; the kernels then run
  // back to back and each event pair times its kernel, not the host's launch rate.
  for (;;) {
    prof_spin(P);
    pcg_body<T, VW>(P, op, s, tol2, 0, 0, maxit);
    HP_CUDA(cudaMemcpyAsync(hact, P->sc.active.p, sizeof(int) * s, cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaMemcpyAsync(h_it, P->sc.iter.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaStreamSynchronize(st));
    int nact = 0;
    for (int j = 0; j < s; ++j) nact += hact[j] != 0;
    if (nact == 0 || *h_it >= maxit) break;
  }
  *its = *h_it;
  HP_CUDA(cudaMemcpyFromSymbolAsync(h_it + 1, g_tile_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaStreamSynchronize(st));
  HP_TRY(tile_timeout_check(P, h_it));
  HP_CUDA(cudaGetLastError());
  return *h_it >= maxit ? HP_ERR_NOT_CONVERGED : 0;
}

int apply_op64(hp_problem *P, OpKind op, const double *X, long ldx, double *Y, long ldy, int s) {
  st_launch<double, 1, M_APPLY>(P->lv[0].g, stencil_of<double>(P, op, 0), X, ldx, nullptr, 0, Y, ldy, s, 0.0, Fin{},
                                P->st);
  return cuda_check(cudaGetLastError(), "apply");
}

// FP64 residual R = B - S X (column-major) with the per-column |R|^2 -> sc.rr in the same pass
// Whether the FP64 refinement of the solve being launched evaluates its residuals, scaling
// and updates in double-float arithmetic (FP32 inner solves only).  Double-float carries
// about 48 significand bits against FP64's 53, and its residual's error grows with
// |S| |x| / |b|: at tolerances from DF_MIN_RTOL up it leaves a wide margin (the attained
// FP64 residual is checked against the oracle at 1e-8), below it the solve keeps the FP64
// arithmetic.
constexpr double DF_MIN_RTOL = 1e-9;
// Blocks below DF_MIN_ENTRIES values (n times s) keep the FP64 refinement with refine_df 1:
// there the FP64 kernels are latency-bound rather than FP64-bound, and the double-float path's
// extra passes (the pair conversions at a solve's start and end) cost more than they save
// (measured: 64 uneven 2D problems with 40 columns each, 24,738 vs 27,940 actions/s; a
// 257^2 x 60 block, 18,357 vs 18,108; 65^3 x 120, 3,735 vs 3,275).
constexpr double DF_MIN_ENTRIES = 16.0 * 1024 * 1024;
static bool use_df(const hp_problem *P, int tbytes, double rtol, int s) {
  return tbytes == 4 && (P->refine_df == 2 || (P->refine_df == 1 && rtol >= DF_MIN_RTOL &&
                                               (double)P->n * s >= DF_MIN_ENTRIES));
}

static int residual64(hp_problem *P, OpKind op, const double *B, long ldb, const double *X, long ldx, double *R,
                      long ldr, int s) {
  const int pr = prof_start(P, PROF_RESID64);
  st_launch<double, 1, M_RESID_DOT>(P->lv[0].g, stencil_of<double>(P, op, 0), X, ldx, B, ldb, R, ldr, s, 0.0,
                                    make_fin(P, FIN_STORE, 0.0, P->sc.rr.as<double>()), P->st);
  prof_stop(P, pr);
  return cuda_check(cudaGetLastError(), "residual");
}

// DBuf::ensure that drops the captured graphs when the buffer moves (they hold its address)
static int ensure_kept(hp_problem *P, DBuf &b, size_t bytes) {
  void *old = b.p;
  HP_TRY(b.ensure(bytes));
  if (b.p != old) drop_graphs(P);
  return 0;
}

// Captures the whole refinement loop of one configuration: reset of the control block and
// the first convergence check, then a WHILE node whose body is one refinement step --
// scaling into the inner precision, the PCG (a nested WHILE node), x += d, the FP64
// residual with its norm, and the control kernel that sets the loop condition.
template <typename T, int VW>
static int build_solve_graph(hp_problem *P, OpKind op, int s, double rtol, double tol_in, SolveGraph *out) {
  BlockWS<T> &W = ws_of<T>(P);
  const long n = P->n, ld64 = padded(n);
  const int ng = (s + VW - 1) / VW;
  const long gs = W.ldn * VW;
  double *r64 = P->r64.as<double>(), *b64 = P->b64.as<double>(), *x64 = P->x64.as<double>();
  RefineCtl *ctl = P->rctl.as<RefineCtl>();
  const int maxit = P->max_iter, max_outer = P->max_outer;
  double *scale = P->sc.scale.as<double>(), *iscale = P->sc.iscale.as<double>();
  double *tol2col = P->sc.tol2col.as<double>(), *rr = P->sc.rr.as<double>(), *bb = P->sc.bbr.as<double>();
  const int *iter = P->sc.iter.as<int>();
  return with_capture_stream(P, [&]() -> int {
    cudaStream_t cs = P->cap;
    cudaGraph_t g = nullptr, body = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaGraphConditionalHandle ho;
    cudaGraphNode_t leaf = nullptr, wn = nullptr, pw = nullptr;
    auto end_capture = [&](cudaGraph_t gr, bool want_leaf) {
      cudaError_t el = want_leaf ? capture_leaf(cs, &leaf) : cudaSuccess;
      cudaGraph_t gg = gr;
      const cudaError_t ee = cudaStreamEndCapture(cs, &gg);
      return el != cudaSuccess ? el : ee;
    };
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&ho, g, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaMemsetAsync(ctl, 0, sizeof(RefineCtl), cs);
      k_refine_ctl<<<1, 256, 0, cs>>>(s, rr, bb, rtol, tol_in, scale, iscale, tol2col, iter, 0, max_outer, ctl, ho);
      e = end_capture(g, true);
    }
    if (e == cudaSuccess) {
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = ho;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&wn, g, &leaf, nullptr, 1, &cp);
      if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      k_to_inner_ctl<T, VW><<<nodegrid(n, ng), NB, 0, cs>>>(n, b64, r64, ld64, ctl, scale, s, W.r.template as<T>(),
                                                            gs);
      e = end_capture(body, true);
    }
    if (e == cudaSuccess) e = append_pcg<T, VW>(P, op, s, tol_in, maxit, body, leaf, &pw);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, &pw, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      k_accum<T, VW><<<nodegrid(n, ng), NB, 0, cs>>>(n, W.x.template as<T>(), gs, iscale, s, x64, ld64);
      const int rc = residual64(P, op, b64, ld64, x64, ld64, r64, ld64, s);
      k_refine_ctl<<<1, 256, 0, cs>>>(s, rr, bb, rtol, tol_in, scale, iscale, tol2col, iter, 1, max_outer, ctl, ho);
      e = end_capture(body, false);
      if (e == cudaSuccess && rc) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_check(e, "refinement graph");
    *out = SolveGraph{(int)op, (int)sizeof(T), VW, s, maxit, max_outer, rtol, tol_in, ex};
    return 0;
  });
}

// The refinement of ir_solve from x = 0 as one graph launch: the one-pass start, the
// captured loop, the copy of the iterate to X and one read-back of the control block.
template <typename T, int VW>
static int ir_solve_graph(hp_problem *P, OpKind op, const double *B, long ldb, double *X, long ldx, int s,
                          double rtol, double tol_in, hp_solve_stats *stats) {
  cudaStream_t st = P->st;
  const long n = P->n, ld64 = padded(n);
  HP_TRY(ensure_kept(P, P->x64, sizeof(double) * ld64 * s));
  HP_TRY(ensure_kept(P, P->rctl, sizeof(RefineCtl)));
  if (!P->h_rctl) HP_CUDA(cudaMallocHost(&P->h_rctl, sizeof(RefineCtl)));
  double *b64 = P->b64.as<double>(), *x64 = P->x64.as<double>();
  const GridDesc &g0 = P->lv[0].g;
  const long face = op == OP_K ? (P->dim == 2 ? g0.np : (long)g0.np * g0.np) : 0;
  HP_TRY(ir_start(P, B, ldb, b64, ld64, x64, ld64, n, s, face, P->sc.bbr.as<double>(), P->sc.rr.as<double>()));
  SolveGraph *G = nullptr;
  for (auto &sg : P->sgraphs)
    if (sg.op == (int)op && sg.tbytes == (int)sizeof(T) && sg.vw == VW && sg.s == s && sg.maxit == P->max_iter &&
        sg.max_outer == P->max_outer && sg.rtol == rtol && sg.tol_in == tol_in)
      G = &sg;
  if (!G) {
    SolveGraph ng;
    HP_TRY((build_solve_graph<T, VW>(P, op, s, rtol, tol_in, &ng)));
    P->sgraphs.push_back(ng);
    G = &P->sgraphs.back();
  }
  HP_CUDA(cudaGraphLaunch(G->exec, st));
  HP_CUDA(cudaMemcpy2DAsync(X, sizeof(double) * ldx, x64, sizeof(double) * ld64, sizeof(double) * n, s,
                            cudaMemcpyDeviceToDevice, st));
  int *h_it = P->sc.h_iter;
  HP_CUDA(cudaMemcpyAsync(P->h_rctl, P->rctl.p, sizeof(RefineCtl), cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaMemcpyFromSymbolAsync(h_it + 1, g_tile_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaStreamSynchronize(st));
  const RefineCtl c = *P->h_rctl;
  HP_TRY(tile_timeout_check(P, h_it));
  // kernels run: the first check, and per step the scaling, the PCG init (3) and
  // iterations, the accumulation, the residual with its finalisation and the check
  count_launch(1ull + 8ull * (unsigned long long)c.outer +
               (unsigned long long)c.total_its * (unsigned long long)kernels_per_iteration(P, op, (int)(sizeof(T) * VW)));
  if (c.flags & 2) return set_error(HP_ERR_NONFINITE, "non-finite residual in a PDE solve");
  if (stats) {
    stats->iterations += c.total_its;
    stats->outer += c.outer;
    stats->solves += 1;
    stats->rel_res = std::max(stats->rel_res, c.worst);
  }
  if (c.flags & 1) return set_error(HP_ERR_NOT_CONVERGED, "PDE solve did not reach the requested tolerance");
  if (op == OP_K) warm_record(P, b64, ld64, X, ldx, s);
  return cuda_check(cudaGetLastError(), "ir_solve");
}

// ---- the double-float refinement (tuning refine_df; FP32 inner solves, 4 columns per group)

// the double-float coefficient pairs of a level-0 FP64 stencil, made when missing or stale
static int ensure_cpr(hp_problem *P, OpKind op) {
  Stencil<double> &S = const_cast<Stencil<double> &>(stencil_of<double>(P, op, 0));
  const long n = P->lv[0].g.n;
  if (!S.cpr) HP_CUDA(cudaMalloc(&S.cpr, sizeof(float2) * (size_t)(S.nf + 1) * n));
  if (!S.cpr_ok) {
    k_coef_pairs<<<blocks_for(n, 1), NT, 0, P->st>>>(n, S.nf, S.diag, S.c, S.cpr);
    count_launch();
    S.cpr_ok = true;
  }
  return cuda_check(cudaGetLastError(), "coefficient pairs");
}

// rt = (b - S x) sb and the columns' |r|^2 -> sc.rr
static void launch_resid_dfp(hp_problem *P, OpKind op, const float4 *Xp, const float4 *Bp, long ldp, float *rt,
                             long gs, int s, const double *bb) {
  const Stencil<double> &S = stencil_of<double>(P, op, 0);
  const GridDesc &g = P->lv[0].g;
  const int ng = (s + 3) / 4;
  const dim3 gr = nodegrid(g.n, ng);
  const Fin fin = make_fin(P, FIN_STORE, 0.0, P->sc.rr.as<double>());
  const int pr = prof_start(P, PROF_RESID64);
  if (g.dim == 2) {
    if (S.full)
      k_resid_dfp<2, true><<<gr, NB, 0, P->st>>>(g, S.cpr, Xp, Bp, ldp, rt, gs, s, bb, fin);
    else
      k_resid_dfp<2, false><<<gr, NB, 0, P->st>>>(g, S.cpr, Xp, Bp, ldp, rt, gs, s, bb, fin);
  } else {
    if (S.full)
      k_resid_dfp<3, true><<<gr, NB, 0, P->st>>>(g, S.cpr, Xp, Bp, ldp, rt, gs, s, bb, fin);
    else
      k_resid_dfp<3, false><<<gr, NB, 0, P->st>>>(g, S.cpr, Xp, Bp, ldp, rt, gs, s, bb, fin);
  }
  count_launch();
  // x and b pairs, the inner right-hand side written, the coefficient pairs
  count_bytes(BY_REFINE, (double)g.n * (20.0 * s + 8.0 * (S.nf + 1)));
  dot_finalize(fin, gr.x, s, P->st);
  prof_stop(P, pr);
}

static void launch_accum_dfp(hp_problem *P, const float *d, long gs, int s, float4 *Xp, long ldp) {
  const int ng = (s + 3) / 4;
  k_accum_dfp<<<nodegrid(P->n, ng), NB, 0, P->st>>>(P->n, d, gs, P->sc.iscale.as<double>(), P->sc.bbr.as<double>(),
                                                     s, Xp, ldp);
  count_launch();
  count_bytes(BY_REFINE, 20.0 * (double)P->n * s);  // read the correction, read and write the x pairs
}

static void launch_first_inner_dfp(hp_problem *P, const float4 *Bp, long ldp, int s, float *rt, long gs) {
  const int ng = (s + 3) / 4;
  k_first_inner_dfp<<<nodegrid(P->n, ng), NB, 0, P->st>>>(Bp, ldp, P->n, P->sc.bbr.as<double>(), s, rt, gs);
  count_launch();
  count_bytes(BY_REFINE, 8.0 * (double)P->n * s);  // hi(b) read, the inner right-hand side written
}

// Captures the double-float refinement loop of one configuration: the first convergence
// check and the first inner right-hand side, then a WHILE node over the steps -- the PCG
// (a nested WHILE node), the update of the x pairs, the residual into the next inner
// right-hand side with its norm, and the control kernel.
template <typename T, int VW>
static int build_solve_graph_dfp(hp_problem *P, OpKind op, int s, double rtol, double tol_in, SolveGraph *out) {
  BlockWS<T> &W = ws_of<T>(P);
  const long ldp = padded(P->n);
  const long gs = W.ldn * VW;
  float4 *Bp = reinterpret_cast<float4 *>(P->b64.p), *Xp = reinterpret_cast<float4 *>(P->x64.p);
  RefineCtl *ctl = P->rctl.as<RefineCtl>();
  const int maxit = P->max_iter, max_outer = P->max_outer;
  double *scale = P->sc.scale.as<double>(), *iscale = P->sc.iscale.as<double>();
  double *tol2col = P->sc.tol2col.as<double>(), *rr = P->sc.rr.as<double>(), *bb = P->sc.bbr.as<double>();
  const int *iter = P->sc.iter.as<int>();
  float *rt = reinterpret_cast<float *>(W.r.p), *d = reinterpret_cast<float *>(W.x.p);
  return with_capture_stream(P, [&]() -> int {
    cudaStream_t cs = P->cap;
    cudaGraph_t g = nullptr, body = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaGraphConditionalHandle ho;
    cudaGraphNode_t leaf = nullptr, wn = nullptr, pw = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&ho, g, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaMemsetAsync(ctl, 0, sizeof(RefineCtl), cs);
      k_refine_ctl<<<1, 256, 0, cs>>>(s, rr, bb, rtol, tol_in, scale, iscale, tol2col, iter, 0, max_outer, ctl, ho);
      launch_first_inner_dfp(P, Bp, ldp, s, rt, gs);
      const cudaError_t el = capture_leaf(cs, &leaf);
      cudaGraph_t gg = g;
      e = cudaStreamEndCapture(cs, &gg);
      if (e == cudaSuccess) e = el;
    }
    if (e == cudaSuccess) {
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = ho;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&wn, g, &leaf, nullptr, 1, &cp);
      if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess) e = append_pcg<T, VW>(P, op, s, tol_in, maxit, body, nullptr, &pw);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, &pw, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      launch_accum_dfp(P, d, gs, s, Xp, ldp);
      launch_resid_dfp(P, op, Xp, Bp, ldp, rt, gs, s, bb);
      k_refine_ctl<<<1, 256, 0, cs>>>(s, rr, bb, rtol, tol_in, scale, iscale, tol2col, iter, 1, max_outer, ctl, ho);
      cudaGraph_t bg = body;
      e = cudaStreamEndCapture(cs, &bg);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_check(e, "double-float refinement graph");
    *out = SolveGraph{(int)op, 100 + (int)sizeof(T), VW, s, maxit, max_outer, rtol, tol_in, ex};
    return 0;
  });
}

// The refinement of ir_solve in double-float (from x = 0): b and x as pairs in the
// workspace, the loop as one graph launch (or, with profiling or graphs off, a host loop
// over the same kernels), the pairs joined into X at the end.
template <typename T, int VW>
static int ir_solve_dfp(hp_problem *P, OpKind op, const double *B, long ldb, double *X, long ldx, int s, double rtol,
                        double tol_in, hp_solve_stats *stats) {
  if constexpr (sizeof(T) != 4 || VW != 4) {
    return set_error(HP_ERR_INVALID, "double-float refinement needs FP32 inner solves");
  } else {
    BlockWS<T> &W = ws_of<T>(P);
    cudaStream_t st = P->st;
    const long n = P->n, ldp = padded(n);
    const int ng = (s + 3) / 4;
    const long gs = W.ldn * VW;
    const size_t pbytes = sizeof(float4) * 2 * (size_t)ldp * ng;
    HP_TRY(ensure_kept(P, P->b64, pbytes));
    HP_TRY(ensure_kept(P, P->x64, pbytes));
    HP_TRY(ensure_kept(P, P->rctl, sizeof(RefineCtl)));
    if (!P->h_rctl) HP_CUDA(cudaMallocHost(&P->h_rctl, sizeof(RefineCtl)));
    HP_TRY(ensure_cpr(P, op));
    struct OpenGuard {
      OpenGuard(const double *p) { tl_open = p; }
      ~OpenGuard() { tl_open = nullptr; }
    } open_guard(P->sc.scale.as<double>());
    float4 *Bp = reinterpret_cast<float4 *>(P->b64.p), *Xp = reinterpret_cast<float4 *>(P->x64.p);
    float *rt = reinterpret_cast<float *>(W.r.p), *d = reinterpret_cast<float *>(W.x.p);
    double *bb = P->sc.bbr.as<double>(), *rr = P->sc.rr.as<double>();
    const GridDesc &g0 = P->lv[0].g;
    const long face = op == OP_K ? (P->dim == 2 ? g0.np : (long)g0.np * g0.np) : 0;
    {  // b, x = 0 and |b|^2 (= the first |r|^2) in one pass over B
      const dim3 gr = nodegrid(n, ng);
      const Fin fin = make_fin(P, FIN_STORE, 0.0, bb);
      k_ir_start_dfp<<<gr, NB, 0, st>>>(B, ldb, s, Bp, Xp, ldp, n, face, fin.part);
      count_launch();
      count_bytes(BY_REFINE, 24.0 * (double)n * s);  // B read, b and x pairs written
      dot_finalize(fin, gr.x, s, st);
      launch_copy(bb, 0, rr, 0, s, 1, st);
    }
    int total_its = 0, outer = 0, rc = 0;
    double worst = 0.0;
    if (P->use_graphs && !P->prof_on) {
      SolveGraph *G = nullptr;
      for (auto &sg : P->sgraphs)
        if (sg.op == (int)op && sg.tbytes == 100 + (int)sizeof(T) && sg.vw == VW && sg.s == s &&
            sg.maxit == P->max_iter && sg.max_outer == P->max_outer && sg.rtol == rtol && sg.tol_in == tol_in)
          G = &sg;
      if (!G) {
        SolveGraph ngr;
        HP_TRY((build_solve_graph_dfp<T, VW>(P, op, s, rtol, tol_in, &ngr)));
        P->sgraphs.push_back(ngr);
        G = &P->sgraphs.back();
      }
      HP_CUDA(cudaGraphLaunch(G->exec, st));
      k_df_out_dfp<<<nodegrid(n, ng), NB, 0, st>>>(Xp, ldp, n, s, X, ldx);
      count_launch();
      count_bytes(BY_REFINE, 16.0 * (double)n * s);
      int *h_it = P->sc.h_iter;
      HP_CUDA(cudaMemcpyAsync(P->h_rctl, P->rctl.p, sizeof(RefineCtl), cudaMemcpyDeviceToHost, st));
      HP_CUDA(cudaMemcpyFromSymbolAsync(h_it + 1, g_tile_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
      HP_CUDA(cudaStreamSynchronize(st));
      const RefineCtl c = *P->h_rctl;
      HP_TRY(tile_timeout_check(P, h_it));
      // kernels run: the first check and right-hand side, per step the PCG init (3) and
      // iterations, the update, the residual with its finalisation and the check
      count_launch(2ull + 7ull * (unsigned long long)c.outer +
                   (unsigned long long)c.total_its * (unsigned long long)kernels_per_iteration(P, op, (int)(sizeof(T) * VW)));
      if (c.flags & 2) return set_error(HP_ERR_NONFINITE, "non-finite residual in a PDE solve");
      total_its = c.total_its;
      outer = c.outer;
      worst = c.worst;
      if (c.flags & 1) rc = HP_ERR_NOT_CONVERGED;
    } else {
      double *hrr = P->sc.h_rr, *hbb = P->sc.h_bb;
      HP_CUDA(cudaMemcpyAsync(hbb, bb, sizeof(double) * s, cudaMemcpyDeviceToHost, st));
      std::vector<double> hscale(s), hiscale(s), htol2(s);
      for (outer = 0; outer <= P->max_outer; ++outer) {
        HP_CUDA(cudaMemcpyAsync(hrr, rr, sizeof(double) * s, cudaMemcpyDeviceToHost, st));
        HP_CUDA(cudaStreamSynchronize(st));
        int nact = 0;
        worst = 0.0;
        for (int j = 0; j < s; ++j) {  // the test and inner tolerance of k_refine_ctl
          if (!std::isfinite(hrr[j])) return set_error(HP_ERR_NONFINITE, "non-finite residual in a PDE solve");
          const double rel = hbb[j] > 0 ? std::sqrt(hrr[j] / hbb[j]) : 0.0;
          worst = std::max(worst, rel);
          const bool done = hbb[j] == 0.0 || hrr[j] <= rtol * rtol * hbb[j];
          hscale[j] = done ? 0.0 : 1.0 / std::sqrt(hrr[j]);
          hiscale[j] = done ? 0.0 : std::sqrt(hrr[j]);
          const double need = hrr[j] > 0 ? 0.25 * rtol * std::sqrt(hbb[j] / hrr[j]) : 1.0;
          const double t = std::min(0.5, std::max(tol_in, need));
          htol2[j] = t * t;
          nact += !done;
        }
        if (nact == 0) break;
        if (outer == P->max_outer) {
          rc = HP_ERR_NOT_CONVERGED;
          break;
        }
        HP_CUDA(cudaMemcpyAsync(P->sc.scale.p, hscale.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
        HP_CUDA(cudaMemcpyAsync(P->sc.iscale.p, hiscale.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
        HP_CUDA(cudaMemcpyAsync(P->sc.tol2col.p, htol2.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
        if (outer == 0) launch_first_inner_dfp(P, Bp, ldp, s, rt, gs);
        int its = 0;
        const int prc = pcg<T, VW>(P, op, s, tol_in, P->max_iter, &its);
        if (prc && prc != HP_ERR_NOT_CONVERGED) return prc;
        total_its += its;
        prof_spin(P);
        launch_accum_dfp(P, d, gs, s, Xp, ldp);
        launch_resid_dfp(P, op, Xp, Bp, ldp, rt, gs, s, bb);
      }
      k_df_out_dfp<<<nodegrid(n, ng), NB, 0, st>>>(Xp, ldp, n, s, X, ldx);
      count_launch();
      count_bytes(BY_REFINE, 16.0 * (double)n * s);
    }
    if (stats) {
      stats->iterations += total_its;
      stats->outer += outer;
      stats->solves += 1;
      stats->rel_res = std::max(stats->rel_res, worst);
    }
    if (rc) return set_error(rc, "PDE solve did not reach the requested tolerance");
    return cuda_check(cudaGetLastError(), "ir_solve (double-float)");
  }
}

template <typename T, int VW>
static int ir_solve(hp_problem *P, OpKind op, const double *B, long ldb, double *X, long ldx, int s, double rtol,
                    double tol_in, hp_solve_stats *stats) {
  BlockWS<T> &W = ws_of<T>(P);
  cudaStream_t st = P->st;
  const long n = P->n;
  const long ld64 = padded(n);
  const int ng = (s + VW - 1) / VW;
  const long gs = W.ldn * VW;
  HP_TRY(ensure_kept(P, P->r64, sizeof(double) * ld64 * s));
  HP_TRY(ensure_kept(P, P->b64, sizeof(double) * ld64 * s));
  // double-float refinement (not with a learned initial guess, nor while stiffness solves are
  // recorded for its training: those paths keep the FP64 layout)
  if (use_df(P, (int)sizeof(T), rtol, s) && VW == 4 && !(op == OP_K && (warm_attached(P) || warm_recording(P))))
    return ir_solve_dfp<T, VW>(P, op, B, ldb, X, ldx, s, rtol, tol_in, stats);
  // from x = 0 with graphs on, the whole refinement runs as one captured loop
  if (P->use_graphs && !P->prof_on && !(op == OP_K && warm_attached(P)))
    return ir_solve_graph<T, VW>(P, op, B, ldb, X, ldx, s, rtol, tol_in, stats);
  double *r64 = P->r64.as<double>(), *b64 = P->b64.as<double>();
  // one pass over B: b64 = B (Dirichlet rows of a stiffness solve zeroed), X = 0, |b|^2;
  // from x = 0 the first residual is b64 itself, so rr = bb
  const GridDesc &g0 = P->lv[0].g;
  const long face = op == OP_K ? (P->dim == 2 ? g0.np : (long)g0.np * g0.np) : 0;
  const bool want_warm = op == OP_K && warm_attached(P);
  HP_TRY(ir_start(P, B, ldb, b64, ld64, X, ldx, n, s, face, P->sc.bb.as<double>(),
                  want_warm ? nullptr : P->sc.rr.as<double>()));
  // start from the learned guess (stiffness solves with a network attached) or from zero
  const bool warm = want_warm && warm_guess(P, b64, ld64, X, ldx, s);
  if (warm) HP_TRY(residual64(P, op, b64, ld64, X, ldx, r64, ld64, s));
  else if (want_warm) {  // the guess was not made: X (possibly partly written) back to zero, rr = bb
    launch_fill(X, ldx, n, s, 0.0, st);
    launch_copy(P->sc.bb.as<double>(), 0, P->sc.rr.as<double>(), 0, s, 1, st);
  }
  double *hrr = P->sc.h_rr, *hbb = P->sc.h_bb;
  HP_CUDA(cudaMemcpyAsync(hbb, P->sc.bb.p, sizeof(double) * s, cudaMemcpyDeviceToHost, st));
  std::vector<double> hscale(s), hiscale(s), htol2(s);
  int total_its = 0, outer = 0, rc = 0;
  double worst = 0.0;
  for (outer = 0; outer <= P->max_outer; ++outer) {
    HP_CUDA(cudaMemcpyAsync(hrr, P->sc.rr.p, sizeof(double) * s, cudaMemcpyDeviceToHost, st));
    HP_CUDA(cudaStreamSynchronize(st));
    if (warm && outer == 0) {
      // a guess whose residual is no smaller than |b| (or non-finite) is dropped for zero;
      // |r|^2 and |b|^2 come from differently ordered reductions, so "no smaller" allows
      // a relative rounding margin
      std::vector<int> flag(s);
      for (int j = 0; j < s; ++j) {
        flag[j] = hbb[j] > 0.0 && !(hrr[j] < (1.0 - 1e-10) * hbb[j]);
        if (flag[j]) hrr[j] = hbb[j];
      }
      warm_fallback(P, flag.data(), s, b64, ld64, X, ldx, r64, ld64);
    }
    int nact = 0;
    worst = 0.0;
    for (int j = 0; j < s; ++j) {
      if (!std::isfinite(hrr[j])) return set_error(HP_ERR_NONFINITE, "non-finite residual in a PDE solve");
      const double rel = hbb[j] > 0 ? std::sqrt(hrr[j] / hbb[j]) : 0.0;
      worst = std::max(worst, rel);
      const bool done = hbb[j] == 0.0 || hrr[j] <= rtol * rtol * hbb[j];
      hscale[j] = done ? 0.0 : 1.0 / std::sqrt(hrr[j]);
      hiscale[j] = done ? 0.0 : std::sqrt(hrr[j]);
      // inner relative tolerance: the finer of tol_in and what is left to reach rtol
      // (with a factor 1/4 of margin), so the last refinement step does no extra work
      const double need = hrr[j] > 0 ? 0.25 * rtol * std::sqrt(hbb[j] / hrr[j]) : 1.0;
      const double t = std::min(0.5, std::max(tol_in, need));
      htol2[j] = t * t;
      nact += !done;
    }
    if (nact == 0) break;
    if (outer == P->max_outer) {
      rc = HP_ERR_NOT_CONVERGED;
      break;
    }
    HP_CUDA(cudaMemcpyAsync(P->sc.scale.p, hscale.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
    HP_CUDA(cudaMemcpyAsync(P->sc.iscale.p, hiscale.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
    HP_CUDA(cudaMemcpyAsync(P->sc.tol2col.p, htol2.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
    // the first residual of a solve from zero is b64 (r64 not yet written)
    const double *rsrc = (outer == 0 && !warm) ? b64 : r64;
    k_to_inner<T, VW><<<nodegrid(n, ng), NB, 0, st>>>(n, rsrc, ld64, P->sc.scale.as<double>(), s,
                                                      W.r.template as<T>(), gs);
    count_launch();
    count_bytes(BY_REFINE, (8.0 + sizeof(T)) * (double)n * s);  // read the FP64 residual, write the inner one
    int its = 0;
    // a stalled inner solve still reduces the residual; other failures end the solve
    const int prc = pcg<T, VW>(P, op, s, tol_in, P->max_iter, &its);
    if (prc && prc != HP_ERR_NOT_CONVERGED) return prc;
    total_its += its;
    prof_spin(P);
    k_accum<T, VW><<<nodegrid(n, ng), NB, 0, st>>>(n, W.x.template as<T>(), gs, P->sc.iscale.as<double>(), s, X,
                                                   ldx);
    count_launch();
    count_bytes(BY_REFINE, (16.0 + sizeof(T)) * (double)n * s);  // read the correction, read and write x
    HP_TRY(residual64(P, op, b64, ld64, X, ldx, r64, ld64, s));
  }
  if (stats) {
    stats->iterations += total_its;
    stats->outer += outer;
    stats->solves += 1;
    stats->rel_res = std::max(stats->rel_res, worst);
  }
  if (rc) return set_error(rc, "PDE solve did not reach the requested tolerance");
  if (op == OP_K) warm_record(P, b64, ld64, X, ldx, s);
  return cuda_check(cudaGetLastError(), "ir_solve");
}

static int solve_chunk(hp_problem *P, OpKind op, const double *B, long ldb, double *X, long ldx, int s, double rtol,
                       hp_solve_stats *st) {
  HP_TRY(ensure_scalars(P, s));
  if (P->precision == HP_FP64_PLAIN) {
    HP_TRY(ensure_ws<double>(P, s));
    return ir_solve<double, 1>(P, op, B, ldb, X, ldx, s, rtol, 0.5 * rtol, st);
  }
  HP_TRY(ensure_ws<float>(P, s));
  if (s >= 2) return ir_solve<float, 4>(P, op, B, ldb, X, ldx, s, rtol, P->inner_rtol, st);
  return ir_solve<float, 1>(P, op, B, ldb, X, ldx, s, rtol, P->inner_rtol, st);
}

// Solves the s columns in chunks of the tuned width (0: all at once).
int solve_block(hp_problem *P, OpKind op, const double *B, long ldb, double *X, long ldx, int s, double rtol,
                hp_solve_stats *st) {
  if (s <= 0) return 0;
  tl_max_blocks = P->max_blocks;
  tl_tma = P->tma_tiles;
  tl_n0 = P->n;
  const int w = (P->col_chunk > 0 && P->col_chunk < s) ? P->col_chunk : s;
  for (int c0 = 0; c0 < s; c0 += w) {
    const int cs = std::min(w, s - c0);
    HP_TRY(solve_chunk(P, op, B + ldb * c0, ldb, X + ldx * c0, ldx, cs, rtol, st));
  }
  return 0;
}

}  // namespace hp

// ---------------------------------------------------------------------------
// kernel replay for the roofline (hp_replay_kernel)
// ---------------------------------------------------------------------------
namespace hp {

// reads a buffer larger than L2 so that the next kernel finds its data in HBM
__global__ void k_flush_read(const float4 *__restrict__ a, long n4, float *__restrict__ sink) {
  float acc = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
    const float4 v = a[i];
    acc += v.x + v.y + v.z + v.w;
  }
  if (acc == -1.2345e30f) *sink = acc;  // keeps the loads; never taken for finite data
}

}  // namespace hp

extern "C" int hp_replay_kernel(hp_problem *P, int family, int reps, void *flush, size_t flush_bytes,
                                double *us_warm, double *us_cold) {
  using namespace hp;
  if (!P || reps < 1 || family < 0 || family > 2 || (us_cold && (!flush || flush_bytes < (64u << 20))))
    return set_error(HP_ERR_INVALID, "hp_replay_kernel: family 0..2, reps >= 1, flush buffer >= 64 MB");
  BlockWS<float> &W = P->w32;
  if (W.scap < 4 || P->L < 2 || !P->have_point)
    return set_error(HP_ERR_STATE, "hp_replay_kernel: needs an FP32 multi-column solve at a point first");
  const int s = W.scap, VW = 4;
  const long gs = W.ldn * VW;
  tl_max_blocks = P->max_blocks;
  tl_tma = P->tma_tiles;
  tl_n0 = P->n;
  const GridDesc &g = P->lv[0].g;
  const Stencil<float> &S = P->lv[0].K32;
  const float om = (float)P->omega;
  float *z = W.z.as<float>(), *r = W.r.as<float>(), *y = W.lb[0].as<float>();
  auto launch = [&]() {
    if (family == 0)
      st_launch<float, 4, M_JACOBI>(g, S, z, gs, r, gs, y, gs, s, om, Fin{}, P->st);
    else if (family == 1)
      st_launch<float, 4, M_RESID>(g, S, z, gs, r, gs, y, gs, s, om, Fin{}, P->st);
    else
      st_launch<float, 4, M_JAC2>(g, S, r, gs, nullptr, 0, y, gs, s, om, Fin{}, P->st, om);
  };
  const long n4 = (long)(flush_bytes / sizeof(float4));
  HP_TRY(P->sc.tmp.ensure(64));
  float *sink = P->sc.tmp.as<float>();
  auto flush_read = [&]() {
    k_flush_read<<<4 * 152, 512, 0, P->st>>>(reinterpret_cast<const float4 *>(flush), n4, sink);
    count_launch();
  };
  cudaEvent_t e[6];
  for (auto &x : e) HP_CUDA(cudaEventCreate(&x));
  launch();  // warm-up
  cudaEventRecord(e[0], P->st);
  for (int k = 0; k < reps; ++k) launch();
  cudaEventRecord(e[1], P->st);
  if (us_cold) {
    cudaEventRecord(e[2], P->st);
    for (int k = 0; k < reps; ++k) {
      flush_read();
      launch();
    }
    cudaEventRecord(e[3], P->st);
    cudaEventRecord(e[4], P->st);
    for (int k = 0; k < reps; ++k) flush_read();
    cudaEventRecord(e[5], P->st);
  }
  const int rc = cuda_check(cudaEventSynchronize(us_cold ? e[5] : e[1]), "hp_replay_kernel");
  float t01 = 0.f, t23 = 0.f, t45 = 0.f;
  if (!rc) {
    cudaEventElapsedTime(&t01, e[0], e[1]);
    if (us_cold) {
      cudaEventElapsedTime(&t23, e[2], e[3]);
      cudaEventElapsedTime(&t45, e[4], e[5]);
    }
  }
  for (auto &x : e) cudaEventDestroy(x);
  if (rc) return rc;
  if (us_warm) *us_warm = 1e3 * t01 / reps;
  if (us_cold) *us_cold = 1e3 * (t23 - t45) / reps;
  return HP_OK;
}

extern "C" int hp_replay_kernel_graph(hp_problem *P, int family, int reps, double *us) {
  using namespace hp;
  if (!P || reps < 1 || reps > 100000 || family < 0 || family > 2 || !us)
    return set_error(HP_ERR_INVALID, "hp_replay_kernel_graph: family 0..2, reps in [1, 1e5], us non-null");
  BlockWS<float> &W = P->w32;
  if (W.scap < 4 || P->L < 2 || !P->have_point)
    return set_error(HP_ERR_STATE, "hp_replay_kernel_graph: needs an FP32 multi-column solve at a point first");
  const int s = W.scap;
  const long gs = W.ldn * 4;
  tl_max_blocks = P->max_blocks;
  tl_tma = P->tma_tiles;
  tl_n0 = P->n;
  const GridDesc &g = P->lv[0].g;
  const Stencil<float> &S = P->lv[0].K32;
  const float om = (float)P->omega;
  float *z = W.z.as<float>(), *r = W.r.as<float>(), *y = W.lb[0].as<float>();
  HP_CUDA(cudaStreamSynchronize(P->st));
  if (!P->cap) HP_CUDA(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  HP_CUDA(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < reps; ++k) {
    if (family == 0)
      st_launch<float, 4, M_JACOBI>(g, S, z, gs, r, gs, y, gs, s, om, Fin{}, P->cap);
    else if (family == 1)
      st_launch<float, 4, M_RESID>(g, S, z, gs, r, gs, y, gs, s, om, Fin{}, P->cap);
    else
      st_launch<float, 4, M_JAC2>(g, S, r, gs, nullptr, 0, y, gs, s, om, Fin{}, P->cap, om);
  }
  cudaError_t ce = cudaStreamEndCapture(P->cap, &graph);
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    if (exec) cudaGraphExecDestroy(exec);
    return cuda_check(ce, "hp_replay_kernel_graph capture");
  }
  cudaEvent_t e0, e1;
  HP_CUDA(cudaEventCreate(&e0));
  HP_CUDA(cudaEventCreate(&e1));
  cudaGraphLaunch(exec, P->st);  // warm-up
  cudaEventRecord(e0, P->st);
  cudaGraphLaunch(exec, P->st);
  cudaEventRecord(e1, P->st);
  const int rc = cuda_check(cudaEventSynchronize(e1), "hp_replay_kernel_graph");
  float ms = 0.f;
  if (!rc) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(exec);
  count_launch((unsigned long long)reps);  // the capture counted reps; the graph ran twice
  if (rc) return rc;
  *us = 1e3 * ms / reps;
  return HP_OK;
}
