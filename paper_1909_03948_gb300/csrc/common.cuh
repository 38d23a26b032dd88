// common.cuh -- shared device helpers: structured-mesh combinatorics, block
// reductions, launch accounting.  Internal to libhp.so.
//
// Mesh (Section 2.3 / Section 5.1): (N+1)^D nodes, lexicographic with the
// first axis fastest.  Cell c = (c_0..c_{D-1}) holds D! simplices, one per
// axis permutation pi: the chain of corner subsets
//     S_0 = {} < S_1 = {pi_0} < ... < S_D = {0..D-1},
// i.e. the vertices c + S_k (as 0/1 offsets).  In 2D this is the split of the
// square along its (0,0)-(1,1) diagonal (pi = (0,1): lower triangle,
// pi = (1,0): upper); in 3D the six Kuhn tetrahedra.  Element index =
// cell_linear * D! + perm, perms in lexicographic order.
//
// On such a simplex the P1 barycentric gradients are differences of unit axis
// vectors, so grad(lambda_{S_k}) . grad(lambda_{S_j}) is non-zero only for
// |k - j| <= 1: the stiffness couples only "path" (axis) edges and the
// element integral of grad u . grad w is (|e|/h^2) sum_k du_k dw_k with
// du_k = u(S_{k+1}) - u(S_k).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define HP_MAXL 16

struct GridDesc {
  int dim;    // 2 or 3
  int N;      // cells per axis
  int np;     // N + 1
  long n;     // nodes
  double h;   // 1/N
  unsigned mnp = 0;  // floor(2^32 / np): division by np as a multiplication (div_np)
};

// i / np for i < 2^32 without an integer division: floor(i mnp / 2^32) is the quotient or
// one less, and the remainder test corrects it
__device__ __forceinline__ unsigned div_np(const GridDesc &g, unsigned i) {
  unsigned q = __umulhi(i, g.mnp);
  unsigned r = i - q * (unsigned)g.np;
  if (r >= (unsigned)g.np) {
    ++q;
    r -= (unsigned)g.np;
  }
  if (r >= (unsigned)g.np) ++q;
  return q;
}

// chain masks of the permutations, [perm][k], k = 0..D
__constant__ static int c_chain2[2][3] = {{0, 1, 3}, {0, 2, 3}};
__constant__ static int c_chain3[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                                          {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

template <int D> struct MeshT;
template <> struct MeshT<2> {
  static constexpr int NPERM = 2;
  static constexpr int NCORN = 4;
  __device__ static __forceinline__ int chain(int p, int k) { return c_chain2[p][k]; }
};
template <> struct MeshT<3> {
  static constexpr int NPERM = 6;
  static constexpr int NCORN = 8;
  __device__ static __forceinline__ int chain(int p, int k) { return c_chain3[p][k]; }
};

__host__ __device__ __forceinline__ int popc3(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }

template <int D>
__device__ __forceinline__ void node_coords(const GridDesc &g, long i, int c[3]) {
  c[0] = (int)(i % g.np);
  long t = i / g.np;
  if (D == 2) {
    c[1] = (int)t;
    c[2] = 0;
  } else {
    c[1] = (int)(t % g.np);
    c[2] = (int)(t / g.np);
  }
}

// linear offset of a 0/1 corner mask
__device__ __forceinline__ long mask_offset(const GridDesc &g, int b) {
  return (long)(b & 1) + ((b >> 1) & 1) * (long)g.np + ((b >> 2) & 1) * (long)g.np * g.np;
}

template <int D>
__device__ __forceinline__ long cell_linear(const GridDesc &g, const int c[3]) {
  return D == 2 ? (long)c[0] + (long)g.N * c[1] : (long)c[0] + (long)g.N * (c[1] + (long)g.N * c[2]);
}

// |e| / h^2 for the simplices of this grid
template <int D> __host__ __device__ __forceinline__ double vol_over_h2(double h) {
  return D == 2 ? 0.5 : h / 6.0;
}
template <int D> __host__ __device__ __forceinline__ double elem_vol(double h) {
  return D == 2 ? 0.5 * h * h : h * h * h / 6.0;
}

// Enumerate the simplices that contain both node v and node v + b (b a 0/1
// mask; b = 0 enumerates the simplices containing v).  For each one calls
// f(cell coords, perm, k) where v = cell + S_k.  A simplex contains both iff
// its chain passes through p = v - cell and p | b.
template <int D, class F>
__device__ __forceinline__ void for_elems_with(const GridDesc &g, const int v[3], int b, F &&f) {
  const int kb = popc3(b);
#pragma unroll
  for (int sh = 0; sh < (1 << D); ++sh) {
    if (sh & b) continue;
    int c[3] = {0, 0, 0};
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      c[a] = v[a] - ((sh >> a) & 1);
      ok = ok && (c[a] >= 0) && (c[a] < g.N);
    }
    if (!ok) continue;
    const int k = popc3(sh);
#pragma unroll
    for (int p = 0; p < MeshT<D>::NPERM; ++p) {
      if (MeshT<D>::chain(p, k) == sh && MeshT<D>::chain(p, k + kb) == (sh | b)) f(c, p, k);
    }
  }
}

// ---- reductions -------------------------------------------------------------
// Multiply-add with one rounding, and a product / sum each rounded on its own: the
// compiler never fuses or splits these, so kernels that mirror one another's arithmetic
// (the per-level, fused-tail and tiled stencil kernels) produce the same bits.
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mulr(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulr(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float addr(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double addr(double a, double b) { return __dadd_rn(a, b); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum (fixed order -> deterministic).  Result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[NT / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < NT / 32 ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// ---- host side --------------------------------------------------------------
#include <atomic>
namespace hp {
extern std::atomic<unsigned long long> g_launches;
extern std::atomic<unsigned long long> g_tiled_launches;  // TMA-tiled stencil kernels alone
extern thread_local int tl_no_count;  // set while capturing graphs: launches count when the graph runs
inline void count_launch(unsigned long long k = 1) {
  if (!tl_no_count) g_launches.fetch_add(k, std::memory_order_relaxed);
}
// Algorithmic DRAM bytes of the launches on the Hessian-action path (each array read or
// written once per launch), by family (HP_BYTES_* in hp.h).  Only direct launches count:
// launches recorded into a CUDA graph do not, so a caller measures per-step bytes on a
// pass with graphs off (profiling on) and carries them over to the graph-driven steps,
// which launch the same kernels.
constexpr int BYTES_FAMILIES = 6;
enum : int { BY_STENCIL0 = 0, BY_STENCILC = 1, BY_TRANSFER = 2, BY_VECTOR = 3, BY_REFINE = 4, BY_CCT = 5 };
extern std::atomic<unsigned long long> g_alg_bytes[BYTES_FAMILIES];
extern thread_local long tl_n0;  // finest-level node count of the solve being launched (0: none)
inline void count_bytes(int fam, double bytes) {
  if (!tl_no_count && bytes > 0.0) g_alg_bytes[fam].fetch_add((unsigned long long)(bytes + 0.5), std::memory_order_relaxed);
}
inline int level_family(long n) { return n == tl_n0 ? BY_STENCIL0 : BY_STENCILC; }
constexpr int NT = 256;   // threads per block of the streaming kernels
constexpr int NSM = 152;  // SMs of a GB300
inline int blocks_for(long n, int s) {
  long b = (n + NT - 1) / NT;
  long cap = (long)(NSM * 16) / (s > 0 ? s : 1);
  if (cap < 1) cap = 1;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}
}  // namespace hp
