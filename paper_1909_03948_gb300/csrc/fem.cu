// fem.cu -- operators of the discretised log-coefficient Poisson problem.
//
// Coefficient:  kappa_e = mean_{v in e} e^{m_v}  (exact element integral of the
//               P1 interpolant of e^m, divided by |e|).
// Stiffness K(kappa): only axis (path) edges couple (see common.cuh), with
//               edge weight w = (|e|/h^2) sum_{e contains the edge} kappa_e; stored
//               as a 5-point (2D) / 7-point (3D) symmetric stencil.  Dirichlet
//               rows (last coordinate 0 or N) become identity rows and their
//               couplings are removed; the removed couplings times the Dirichlet
//               data form the lifting right-hand side (Section 5.1.3 boundary
//               conditions).
// Multigrid coarse operators: the meshes are nested (the fine simplices refine
//               the coarse ones, 2^D children each) and P1 interpolation is the
//               prolongation, so the Galerkin operator P^T K(kappa) P is the coarse
//               FE stiffness with kappa_coarse = mean of the children's kappa.
// Prior A = gamma K(1) + delta M (Section 5.1.1, eq. (PoissonPrior), Theta = I,
//               zero Neumann) and mass M couple along all 2^D - 1 Kuhn edge
//               directions (7-point / 15-point).
// C X   = K(kappa_hat) u, kappa_hat_e = mean_{v in e}(e^m X)_v   (Appendix A,
//               eq. (incrementals1): the term (mhat e^m grad u, grad p~)).
// C^T W = e^{m_v}/(D+1) sum_{e ni v} |e| grad u . grad W          (Appendix A,
//               eqs. (firstcontrol), (incrementals3)).
// B     = P1 interpolation at the observation points (Section 5.1.1).
// C_M   = rectangular factor of M from a degree-2 element rule (Appendix C,
//               eq. (rect_decomp)).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"

namespace hp {

// children of each coarse simplex: (fine cell offset mask) | (fine perm << 3)
__constant__ int c_child2[2][4];
__constant__ int c_child3[6][8];

// quadrature: barycentric coordinate of vertex k at point q (degree-2 rules)
__constant__ double c_quad2[3][3] = {{0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}};

static std::mutex g_children_mutex;
static int g_children_ready = 0;

// The coarse simplex (cell C, perm pi) = {x in C : x_{pi_0} >= x_{pi_1} >= ...}
// (local coordinates); a fine simplex belongs to it iff its centroid does.
static void compute_children(int D, std::vector<std::vector<int>> &out) {
  std::vector<std::vector<int>> perms;
  std::vector<int> a(D);
  for (int i = 0; i < D; ++i) a[i] = i;
  do perms.push_back(a);
  while (std::next_permutation(a.begin(), a.end()));
  out.assign(perms.size(), {});
  for (size_t cp = 0; cp < perms.size(); ++cp) {
    for (int o = 0; o < (1 << D); ++o) {
      for (size_t fp = 0; fp < perms.size(); ++fp) {
        double s[3] = {0, 0, 0};
        for (int ax = 0; ax < D; ++ax) s[ax] = (o >> ax) & 1;
        for (int j = 0; j < D; ++j) s[perms[fp][j]] += double(D - j) / double(D + 1);
        bool in = true;
        for (int j = 0; j + 1 < D; ++j) in = in && (s[perms[cp][j]] > s[perms[cp][j + 1]]);
        if (in) out[cp].push_back(o | (int(fp) << 3));
      }
    }
  }
}

static int ensure_children() {
  std::lock_guard<std::mutex> lock(g_children_mutex);
  if (g_children_ready) return 0;
  std::vector<std::vector<int>> c2, c3;
  compute_children(2, c2);
  compute_children(3, c3);
  int t2[2][4], t3[6][8];
  for (int p = 0; p < 2; ++p) {
    if (c2[p].size() != 4) return set_error(HP_ERR_INVALID, "internal: 2D refinement table");
    for (int q = 0; q < 4; ++q) t2[p][q] = c2[p][q];
  }
  for (int p = 0; p < 6; ++p) {
    if (c3[p].size() != 8) return set_error(HP_ERR_INVALID, "internal: 3D refinement table");
    for (int q = 0; q < 8; ++q) t3[p][q] = c3[p][q];
  }
  HP_CUDA(cudaMemcpyToSymbol(c_child2, t2, sizeof(t2)));
  HP_CUDA(cudaMemcpyToSymbol(c_child3, t3, sizeof(t3)));
  g_children_ready = 1;
  return 0;
}

// ---------------------------------------------------------------------------
// element coefficients
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_elem_kappa_fine(GridDesc g, const double *__restrict__ E, double *__restrict__ kappa,
                                  long nelems) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nelems; e += (long)gridDim.x * blockDim.x) {
    const long cell = e / MeshT<D>::NPERM;
    const int p = (int)(e % MeshT<D>::NPERM);
    int c[3];
    c[0] = (int)(cell % g.N);
    const long t = cell / g.N;
    c[1] = D == 2 ? (int)t : (int)(t % g.N);
    c[2] = D == 2 ? 0 : (int)(t / g.N);
    const long base = c[0] + (long)g.np * (c[1] + (long)g.np * c[2]);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k <= D; ++k) s += E[base + mask_offset(g, MeshT<D>::chain(p, k))];
    kappa[e] = s / (D + 1);
  }
}

template <int D>
__global__ void k_elem_kappa_coarsen(GridDesc gc, GridDesc gf, const double *__restrict__ kf,
                                     double *__restrict__ kc, long nelems_c) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nelems_c; e += (long)gridDim.x * blockDim.x) {
    const long cell = e / MeshT<D>::NPERM;
    const int p = (int)(e % MeshT<D>::NPERM);
    int c[3];
    c[0] = (int)(cell % gc.N);
    const long t = cell / gc.N;
    c[1] = D == 2 ? (int)t : (int)(t % gc.N);
    c[2] = D == 2 ? 0 : (int)(t / gc.N);
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < (1 << D); ++q) {
      const int code = D == 2 ? c_child2[p][q] : c_child3[p][q];
      const int o = code & 7, fp = code >> 3;
      int fc[3] = {2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + ((o >> 2) & 1)};
      s += kf[cell_linear<D>(gf, fc) * MeshT<D>::NPERM + fp];
    }
    kc[e] = s / (1 << D);
  }
}

// ---------------------------------------------------------------------------
// stencils
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ bool is_dirichlet(const GridDesc &g, const int v[3]) {
  return v[D - 1] == 0 || v[D - 1] == g.N;
}

template <int D>
__device__ __forceinline__ double edge_weight(const GridDesc &g, const double *__restrict__ kappa, const int v[3],
                                              int b) {
  double s = 0.0;
  for_elems_with<D>(g, v, b, [&](const int c[3], int p, int k) {
    s += kappa[cell_linear<D>(g, c) * MeshT<D>::NPERM + p];
  });
  return s * vol_over_h2<D>(g.h);
}

template <int D>
__global__ void k_build_K(GridDesc g, const double *__restrict__ kappa, double *diag, double *invdiag, double *c,
                          float *diag32, float *invdiag32, float *c32, double *lift, double u_top,
                          double u_bottom) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    const bool dv = is_dirichlet<D>(g, v);
    double dsum = 0.0, lf = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double wf = 0.0, wb = 0.0;
      int vn[3] = {v[0], v[1], v[2]};
      if (v[a] < g.N) {
        wf = edge_weight<D>(g, kappa, v, 1 << a);
        vn[a] = v[a] + 1;
        const bool dn = is_dirichlet<D>(g, vn);
        const double cf = (dv || dn) ? 0.0 : -wf;
        c[(long)a * g.n + i] = cf;
        c32[(long)a * g.n + i] = (float)cf;
        if (!dv && dn) lf += wf * (vn[D - 1] == g.N ? u_top : u_bottom);
      } else {
        c[(long)a * g.n + i] = 0.0;
        c32[(long)a * g.n + i] = 0.0f;
      }
      if (v[a] > 0) {
        int vb[3] = {v[0], v[1], v[2]};
        vb[a] = v[a] - 1;
        wb = edge_weight<D>(g, kappa, vb, 1 << a);
        if (!dv && is_dirichlet<D>(g, vb)) lf += wb * (vb[D - 1] == g.N ? u_top : u_bottom);
      }
      dsum += wf + wb;
    }
    const double dg = dv ? 1.0 : dsum;
    diag[i] = dg;
    invdiag[i] = 1.0 / dg;
    diag32[i] = (float)dg;
    invdiag32[i] = (float)(1.0 / dg);
    if (lift) lift[i] = dv ? 0.0 : lf;
  }
}

// 2D stiffness in FP32, one 16-byte record per node for the tiled stencil kernels:
// {diag, 1 / diag, coupling to x + 1, coupling to y + 1}
__global__ void k_pack_K2(long n, const float *__restrict__ diag, const float *__restrict__ invdiag,
                          const float *__restrict__ c, float4 *__restrict__ pk) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    pk[i] = make_float4(diag[i], invdiag[i], c[i], c[n + i]);
}

// 3D stiffness in FP32 for the tiled kernels: one 16-byte record per node {diag, 1 / diag,
// coupling to x + 1, coupling to y + 1}, and the coupling to z + 1 in rows padded to a
// multiple of 4 nodes (a tensor map's row stride must be a multiple of 16 bytes)
__global__ void k_pack_K3(GridDesc g, const float *__restrict__ diag, const float *__restrict__ invdiag,
                          const float *__restrict__ c, float4 *__restrict__ pk, float *__restrict__ cz) {
  const long n = g.n, ldr = (g.np + 3) / 4 * 4;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    pk[i] = make_float4(diag[i], invdiag[i], c[i], c[n + i]);
    const long x = i % g.np, row = i / g.np;
    cz[row * ldr + x] = c[2 * n + i];
  }
}

template <int D>
__device__ __forceinline__ int count_elems(const GridDesc &g, const int v[3], int b) {
  int n = 0;
  for_elems_with<D>(g, v, b, [&](const int *, int, int) { ++n; });
  return n;
}

// Symmetric anisotropy tensor: t[0..2] = (T00, T11, T22), t[3..5] = (T01, T02, T12).
struct Theta6 {
  double t[6];
};
__device__ __forceinline__ double theta_ab(const Theta6 &T, int a, int b) {
  if (a == b) return T.t[a];
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? (hi == 1 ? T.t[3] : T.t[4]) : T.t[5];
}

// Gradient (in units of 1/h) of the barycentric function of chain vertex t of Kuhn simplex p:
// with pi_t the axis added at step t, lambda_0 = 1 - x_{pi_1}, lambda_t = x_{pi_t} - x_{pi_{t+1}},
// lambda_D = x_{pi_D} in the cell's local coordinates.
template <int D>
__device__ __forceinline__ void kuhn_grad(int p, int t, double gv[3]) {
  gv[0] = gv[1] = gv[2] = 0.0;
  if (t >= 1) gv[__ffs(MeshT<D>::chain(p, t) ^ MeshT<D>::chain(p, t - 1)) - 1] += 1.0;
  if (t < D) gv[__ffs(MeshT<D>::chain(p, t + 1) ^ MeshT<D>::chain(p, t)) - 1] -= 1.0;
}

// A = gamma K(Theta) + delta M + cR M_boundary (all nodes, no Dirichlet rows), assembled per
// node from the simplices that contain it (each node keeps its diagonal and its forward
// couplings along the 2^D - 1 Kuhn edge directions) and from the boundary facets that
// contain it (the facets of a face of the cube are the Kuhn triangulation of that face).
// With Theta = I and cR = 0 this is gamma K(1) + delta M with zero Neumann.
template <int D>
__global__ void k_build_A(GridDesc g, double gamma, double delta, double cR, Theta6 Th, double *diag,
                          double *invdiag, double *c, float *diag32, float *invdiag32, float *c32) {
  constexpr int NF = (1 << D) - 1;
  const double vh2 = vol_over_h2<D>(g.h);
  const double mc = elem_vol<D>(g.h) / ((D + 1) * (D + 2));
  const double fvol = D == 2 ? g.h : 0.5 * g.h * g.h;   // boundary facet measure
  const double fm = fvol / (D * (D + 1));                // off-diagonal boundary facet mass
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    double cf[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) cf[f] = 0.0;
    double dg = 0.0;
    for_elems_with<D>(g, v, 0, [&](const int *, int p, int k) {
      double gk[3];
      kuhn_grad<D>(p, k, gk);
      for (int t = k; t <= D; ++t) {
        double gt[3];
        kuhn_grad<D>(p, t, gt);
        double e = 0.0;
        for (int a = 0; a < D; ++a)
          for (int b = 0; b < D; ++b) e += gk[a] * theta_ab(Th, a, b) * gt[b];
        const double val = gamma * vh2 * e + delta * mc * (t == k ? 2.0 : 1.0);
        if (t == k)
          dg += val;
        else
          cf[(MeshT<D>::chain(p, t) ^ MeshT<D>::chain(p, k)) - 1] += val;
      }
    });
    if (cR != 0.0) {
      for (int a = 0; a < D; ++a) {
        if (v[a] != 0 && v[a] != g.N) continue;
        int ax[2] = {0, 0}, na = 0;
        for (int o = 0; o < D; ++o)
          if (o != a) ax[na++] = o;
        for (int s0 = 0; s0 < 2; ++s0)
          for (int s1 = 0; s1 < (D == 3 ? 2 : 1); ++s1) {
            int cc[3] = {v[0], v[1], v[2]};
            cc[ax[0]] -= s0;
            if (D == 3) cc[ax[1]] -= s1;
            if (cc[ax[0]] < 0 || cc[ax[0]] >= g.N) continue;
            if (D == 3 && (cc[ax[1]] < 0 || cc[ax[1]] >= g.N)) continue;
            const int vm = (s0 << ax[0]) | (D == 3 ? (s1 << ax[1]) : 0);  // v - cc as a corner mask
            for (int perm = 0; perm < (D == 3 ? 2 : 1); ++perm) {
              const int p1 = D == 3 ? ax[perm] : ax[0];
              const int m[3] = {0, 1 << p1, D == 3 ? ((1 << p1) | (1 << ax[1 - perm])) : 0};
              int k = -1;
              for (int t = 0; t < D; ++t)
                if (m[t] == vm) k = t;
              if (k < 0) continue;
              dg += cR * 2.0 * fm;
              for (int t = k + 1; t < D; ++t) cf[(m[t] ^ m[k]) - 1] += cR * fm;
            }
          }
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      c[(long)f * g.n + i] = cf[f];
      c32[(long)f * g.n + i] = (float)cf[f];
    }
    diag[i] = dg;
    invdiag[i] = 1.0 / dg;
    diag32[i] = (float)dg;
    invdiag32[i] = (float)(1.0 / dg);
  }
}

// max over nodes of (diag_i + sum_j |s_ij|) / diag_i: a bound of the spectrum of diag^-1 S
template <int D>
__global__ void k_gersh(GridDesc g, const double *__restrict__ diag, const double *__restrict__ c, int nf, bool full,
                        unsigned long long *out) {
  double mx = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    double sum = fabs(diag[i]);
    for (int f = 0; f < nf; ++f) {
      const int b = full ? f + 1 : (1 << f);
      bool fw = true, bw = true;
      for (int a = 0; a < D; ++a)
        if ((b >> a) & 1) {
          fw = fw && (v[a] < g.N);
          bw = bw && (v[a] > 0);
        }
      const long off = mask_offset(g, b);
      if (fw) sum += fabs(c[(long)f * g.n + i]);
      if (bw) sum += fabs(c[(long)f * g.n + i - off]);
    }
    mx = fmax(mx, sum / diag[i]);
  }
  // positive doubles order like their bit patterns
  atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

int gershgorin_bound(hp_problem *P, const GridDesc &g, const Stencil<double> &S, double *out) {
  unsigned long long *d = reinterpret_cast<unsigned long long *>(P->sc.tmp.p);
  HP_TRY(P->sc.tmp.ensure(64));
  d = reinterpret_cast<unsigned long long *>(P->sc.tmp.p);
  HP_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), P->st));
  const int nb = (int)std::min<long>((g.n + 255) / 256, 1024);
  if (g.dim == 2)
    k_gersh<2><<<nb, 256, 0, P->st>>>(g, S.diag, S.c, S.nf, S.full, d);
  else
    k_gersh<3><<<nb, 256, 0, P->st>>>(g, S.diag, S.c, S.nf, S.full, d);
  count_launch();
  unsigned long long h = 0;
  HP_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, P->st));
  HP_CUDA(cudaStreamSynchronize(P->st));
  double v;
  std::memcpy(&v, &h, sizeof(v));
  *out = v;
  return 0;
}

// ---------------------------------------------------------------------------
// dense coarse-grid inverse
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_dense_from_stencil(GridDesc g, const double *diag, const double *c, int nf, bool full,
                                     double *A) {
  const long nc = g.n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nc; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    A[i * nc + i] = diag[i];
    for (int f = 0; f < nf; ++f) {
      const int b = full ? f + 1 : (1 << f);
      bool fwd = true;
      for (int a = 0; a < D; ++a)
        if ((b >> a) & 1) fwd = fwd && (v[a] < g.N);
      if (!fwd) continue;
      const long j = i + mask_offset(g, b);
      const double w = c[(long)f * g.n + i];
      A[i * nc + j] = w;
      A[j * nc + i] = w;
    }
  }
}

// In-place lower Cholesky of a dense SPD matrix (row-major), one block.
__global__ void k_dense_cholesky(double *A, int nc, int *status) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < nc; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[(long)k * nc + k];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      A[(long)k * nc + k] = (d > 0.0) ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double dk = A[(long)k * nc + k];
    for (int i = k + 1 + threadIdx.x; i < nc; i += blockDim.x) A[(long)i * nc + k] /= dk;
    __syncthreads();
    const int m = nc - k - 1;
    for (long t = threadIdx.x; t < (long)m * m; t += blockDim.x) {
      const int i = k + 1 + (int)(t / m), j = k + 1 + (int)(t % m);
      if (j <= i) A[(long)i * nc + j] -= A[(long)i * nc + k] * A[(long)j * nc + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *status = bad;
}

// Column j of the inverse from the Cholesky factor, one thread per column.  The inverse is
// symmetric, so thread j keeps its column as row j of the output, x[i] at inv[i * nc + j]:
// the threads of a warp then touch consecutive addresses at every step (and all read the same
// L entry), and the substitutions start at row j (rows above it are zero in L^-1 e_j).
__global__ void k_dense_inverse(const double *L, int nc, double *inv, float *inv32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nc) return;
  for (int i = 0; i < j; ++i) inv[(long)i * nc + j] = 0.0;
  for (int i = j; i < nc; ++i) {  // L y = e_j
    double s = (i == j) ? 1.0 : 0.0;
    for (int k = j; k < i; ++k) s -= L[(long)i * nc + k] * inv[(long)k * nc + j];
    inv[(long)i * nc + j] = s / L[(long)i * nc + i];
  }
  for (int i = nc - 1; i >= 0; --i) {  // L^T x = y
    double s = inv[(long)i * nc + j];
    for (int k = i + 1; k < nc; ++k) s -= L[(long)k * nc + i] * inv[(long)k * nc + j];
    inv[(long)i * nc + j] = s / L[(long)i * nc + i];
  }
  for (int i = 0; i < nc; ++i) inv32[(long)i * nc + j] = (float)inv[(long)i * nc + j];
}

// FP32 coarse factorisation for the FP32 inner solves (the only consumer of inv32 when the
// refinement runs in FP32): one CTA, the lower triangle packed in shared memory (row i at
// offset i (i + 1) / 2), right-looking Cholesky; FP32 runs at 64x the FP64 rate of an SM.
// L (row-major, lower) goes to Lg for the triangular solves.
__device__ __forceinline__ int tri_at(int i, int j) { return i * (i + 1) / 2 + j; }

__global__ void __launch_bounds__(1024) k_dense_cholesky32(const double *__restrict__ A, int nc, float *Lg,
                                                           int *status) {
  extern __shared__ float tri[];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int t = threadIdx.x; t < nc * (nc + 1) / 2; t += blockDim.x) {
    int i = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
    while (tri_at(i, 0) > t) --i;
    while (tri_at(i + 1, 0) <= t) ++i;
    tri[t] = (float)A[(long)i * nc + (t - tri_at(i, 0))];
  }
  __syncthreads();
  for (int k = 0; k < nc; ++k) {
    if (threadIdx.x == 0) {
      const float d = tri[tri_at(k, k)];
      if (!(d > 0.f) || !isfinite(d)) bad = 1;
      tri[tri_at(k, k)] = d > 0.f ? sqrtf(d) : 1.f;
    }
    __syncthreads();
    const float dk = tri[tri_at(k, k)];
    for (int i = k + 1 + threadIdx.x; i < nc; i += blockDim.x) tri[tri_at(i, k)] /= dk;
    __syncthreads();
    const int m = nc - k - 1;
    for (int t = threadIdx.x; t < m * (m + 1) / 2; t += blockDim.x) {  // i >= j > k
      int a = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
      while (a * (a + 1) / 2 > t) --a;
      while ((a + 1) * (a + 2) / 2 <= t) ++a;
      const int i = k + 1 + a, j = k + 1 + (t - a * (a + 1) / 2);
      tri[tri_at(i, j)] -= tri[tri_at(i, k)] * tri[tri_at(j, k)];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nc * nc; t += blockDim.x) {
    const int i = t / nc, j = t % nc;
    Lg[t] = j <= i ? tri[tri_at(i, j)] : 0.f;
  }
  if (threadIdx.x == 0) *status = bad;
}

// Column j of the inverse from L, one warp per column: the forward substitution L y = e_j
// from row j on (rows above are zero), then L^T x = y, each row's sum split over the 32
// lanes and reduced; the column is kept in shared memory and written as row j of inv32
// (the inverse is symmetric).
__global__ void __launch_bounds__(128) k_dense_inverse32(const float *__restrict__ L, int nc, float *inv32) {
  extern __shared__ float colbuf[];  // [4 warps][nc]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 4 + w;
  if (j >= nc) return;
  float *x = colbuf + (long)w * nc;
  for (int i = lane; i < nc; i += 32) x[i] = 0.f;
  __syncwarp();
  for (int i = j; i < nc; ++i) {
    float sum = 0.f;
    for (int k = j + lane; k < i; k += 32) sum += L[(long)i * nc + k] * x[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) x[i] = ((i == j ? 1.f : 0.f) - sum) / L[(long)i * nc + i];
    __syncwarp();
  }
  for (int i = nc - 1; i >= 0; --i) {
    float sum = 0.f;
    for (int k = i + 1 + lane; k < nc; k += 32) sum += L[(long)k * nc + i] * x[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) x[i] = (x[i] - sum) / L[(long)i * nc + i];
    __syncwarp();
  }
  for (int i = lane; i < nc; i += 32) inv32[(long)j * nc + i] = x[i];
}

int coarse_setup(hp_problem *P, OpKind op) {
  const Level &lc = P->lv[P->L - 1];
  CoarseInv &C = op == OP_K ? P->cK : P->cA;
  const Stencil<double> &S = op == OP_K ? lc.K64 : lc.A64;
  const long nc = lc.g.n;
  HP_CUDA(cudaMemsetAsync(C.dense, 0, sizeof(double) * nc * nc, P->st));
  const int nb = (int)std::min<long>((nc + 255) / 256, 1024);
  if (P->dim == 2)
    k_dense_from_stencil<2><<<nb, 256, 0, P->st>>>(lc.g, S.diag, S.c, S.nf, S.full, C.dense);
  else
    k_dense_from_stencil<3><<<nb, 256, 0, P->st>>>(lc.g, S.diag, S.c, S.nf, S.full, C.dense);
  int *dstat = P->sc.active.as<int>();
  const size_t tri_bytes = sizeof(float) * (size_t)nc * (nc + 1) / 2;
  if (P->precision == HP_FP32_IR && tri_bytes <= 200u * 1024u) {
    // only inv32 is used by FP32 inner solves: factor and invert in FP32 (inv64 is
    // rebuilt by hp_set_precision if the plain FP64 path is selected later)
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !(attr_set.load(std::memory_order_acquire) & (1ull << dev))) {
      HP_CUDA(cudaFuncSetAttribute(k_dense_cholesky32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   200 * 1024));
      attr_set.fetch_or(1ull << dev, std::memory_order_release);
    }
    float *L32 = reinterpret_cast<float *>(C.inv64);  // scratch: the FP64 inverse is not kept in this mode
    k_dense_cholesky32<<<1, 1024, tri_bytes, P->st>>>(C.dense, (int)nc, L32, dstat);
    k_dense_inverse32<<<(int)((nc + 3) / 4), 128, sizeof(float) * 4 * nc, P->st>>>(L32, (int)nc, C.inv32);
    C.fp64_valid = false;
  } else {
    k_dense_cholesky<<<1, 1024, 0, P->st>>>(C.dense, (int)nc, dstat);
    k_dense_inverse<<<(int)((nc + 31) / 32), 32, 0, P->st>>>(C.dense, (int)nc, C.inv64, C.inv32);
    C.fp64_valid = true;
  }
  count_launch(3);
  int h = 0;
  HP_CUDA(cudaMemcpyAsync(&h, dstat, sizeof(int), cudaMemcpyDeviceToHost, P->st));
  HP_CUDA(cudaStreamSynchronize(P->st));
  HP_CUDA(cudaGetLastError());
  if (h) return set_error(HP_ERR_NONFINITE, "coarse-grid operator is not SPD (non-finite coefficient?)");
  return 0;
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
static int alloc_stencil(Stencil<double> &S64, Stencil<float> &S32, long n, int nf, bool full) {
  S64.nf = S32.nf = nf;
  S64.full = S32.full = full;
  HP_CUDA(cudaMalloc(&S64.diag, sizeof(double) * n));
  HP_CUDA(cudaMalloc(&S64.invdiag, sizeof(double) * n));
  HP_CUDA(cudaMalloc(&S64.c, sizeof(double) * n * nf));
  HP_CUDA(cudaMalloc(&S32.diag, sizeof(float) * n));
  HP_CUDA(cudaMalloc(&S32.invdiag, sizeof(float) * n));
  HP_CUDA(cudaMalloc(&S32.c, sizeof(float) * n * nf));
  return 0;
}

static int grid_blocks(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, 8192)); }

int build_hierarchy_geometry(hp_problem *P) {
  HP_TRY(ensure_children());
  const int D = P->dim;
  const int ncmax = D == 2 ? 16 : 4;  // coarsest grid: <= 17^2 or 5^3 nodes, dense inverse
  int N = P->N, L = 1;
  while (N % 2 == 0 && N > ncmax && L < HP_MAXL) {
    N /= 2;
    ++L;
  }
  long nc = 1;
  for (int a = 0; a < D; ++a) nc *= (N + 1);
  if (nc > 1600)
    return set_error(HP_ERR_INVALID, "coarsest multigrid grid too large: N must be 2^k times a small factor");
  P->L = L;
  const int nfK = D, nfA = (1 << D) - 1;
  const int nperm = D == 2 ? 2 : 6;
  for (int l = 0; l < L; ++l) {
    Level &lv = P->lv[l];
    lv.g.dim = D;
    lv.g.N = P->N >> l;
    lv.g.np = lv.g.N + 1;
    lv.g.mnp = (unsigned)((1ull << 32) / (unsigned long long)lv.g.np);
    lv.g.n = 1;
    for (int a = 0; a < D; ++a) lv.g.n *= lv.g.np;
    lv.g.h = 1.0 / lv.g.N;
    lv.nelems = nperm;
    for (int a = 0; a < D; ++a) lv.nelems *= lv.g.N;
    HP_CUDA(cudaMalloc(&lv.kappa, sizeof(double) * lv.nelems));
    HP_TRY(alloc_stencil(lv.K64, lv.K32, lv.g.n, nfK, false));
    if (tile_grid(lv.g)) HP_CUDA(cudaMalloc(&lv.K32.pk, sizeof(float4) * lv.g.n));
    if (tile3_grid(lv.g)) {
      const long ldr = (lv.g.np + 3) / 4 * 4;
      const size_t bytes = sizeof(float4) * lv.g.n + sizeof(float) * ldr * lv.g.np * lv.g.np;
      HP_CUDA(cudaMalloc(&lv.K32.pk, bytes));
      HP_CUDA(cudaMemset(lv.K32.pk, 0, bytes));  // the row padding of the z couplings stays zero
    }
    HP_TRY(alloc_stencil(lv.A64, lv.A32, lv.g.n, nfA, true));
    const int nb = grid_blocks(lv.g.n);
    Theta6 th;
    for (int q = 0; q < 6; ++q) th.t[q] = P->theta[q];
    const double cR = P->gamma * P->robin_beta;
    if (D == 2)
      k_build_A<2><<<nb, 256, 0, P->st>>>(lv.g, P->gamma, P->delta, cR, th, lv.A64.diag, lv.A64.invdiag, lv.A64.c,
                                          lv.A32.diag, lv.A32.invdiag, lv.A32.c);
    else
      k_build_A<3><<<nb, 256, 0, P->st>>>(lv.g, P->gamma, P->delta, cR, th, lv.A64.diag, lv.A64.invdiag, lv.A64.c,
                                          lv.A32.diag, lv.A32.invdiag, lv.A32.c);
    count_launch();
  }
  // mass matrix on the fine grid
  const Level &l0 = P->lv[0];
  HP_TRY(alloc_stencil(P->M64, P->M32, l0.g.n, nfA, true));
  const Theta6 eye{{1.0, 1.0, 1.0, 0.0, 0.0, 0.0}};
  if (D == 2)
    k_build_A<2><<<grid_blocks(l0.g.n), 256, 0, P->st>>>(l0.g, 0.0, 1.0, 0.0, eye, P->M64.diag, P->M64.invdiag,
                                                         P->M64.c, P->M32.diag, P->M32.invdiag, P->M32.c);
  else
    k_build_A<3><<<grid_blocks(l0.g.n), 256, 0, P->st>>>(l0.g, 0.0, 1.0, 0.0, eye, P->M64.diag, P->M64.invdiag,
                                                         P->M64.c, P->M32.diag, P->M32.invdiag, P->M32.c);
  count_launch();
  // coarse inverses
  const long ncn = P->lv[L - 1].g.n;
  for (CoarseInv *C : {&P->cK, &P->cA}) {
    C->nc = (int)ncn;
    HP_CUDA(cudaMalloc(&C->dense, sizeof(double) * ncn * ncn));
    HP_CUDA(cudaMalloc(&C->inv64, sizeof(double) * ncn * ncn));
    HP_CUDA(cudaMalloc(&C->inv32, sizeof(float) * ncn * ncn));
  }
  HP_TRY(coarse_setup(P, OP_A));
  for (int l = 0; l < L; ++l) {
    double b = 2.0;
    HP_TRY(gershgorin_bound(P, P->lv[l].g, P->lv[l].A64, &b));
    P->lv[l].A64.lmax = P->lv[l].A32.lmax = b;
  }
  return 0;
}

int build_point(hp_problem *P, const double *m_dev) {
  const long n = P->n;
  P->have_p = P->have_full = false;
  P->have_point = false;  // until the state solve at the new point succeeds
  HP_CUDA(cudaMemcpyAsync(P->m, m_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->st));
  launch_ew_exp(P->m, P->E, n, P->st);
  const int D = P->dim;
  Level &l0 = P->lv[0];
  if (D == 2)
    k_elem_kappa_fine<2><<<grid_blocks(l0.nelems), 256, 0, P->st>>>(l0.g, P->E, l0.kappa, l0.nelems);
  else
    k_elem_kappa_fine<3><<<grid_blocks(l0.nelems), 256, 0, P->st>>>(l0.g, P->E, l0.kappa, l0.nelems);
  count_launch();
  for (int l = 1; l < P->L; ++l) {
    Level &lc = P->lv[l], &lf = P->lv[l - 1];
    if (D == 2)
      k_elem_kappa_coarsen<2><<<grid_blocks(lc.nelems), 256, 0, P->st>>>(lc.g, lf.g, lf.kappa, lc.kappa, lc.nelems);
    else
      k_elem_kappa_coarsen<3><<<grid_blocks(lc.nelems), 256, 0, P->st>>>(lc.g, lf.g, lf.kappa, lc.kappa, lc.nelems);
    count_launch();
  }
  for (int l = 0; l < P->L; ++l) {
    Level &lv = P->lv[l];
    double *lift = l == 0 ? P->lift : nullptr;
    if (D == 2)
      k_build_K<2><<<grid_blocks(lv.g.n), 256, 0, P->st>>>(lv.g, lv.kappa, lv.K64.diag, lv.K64.invdiag, lv.K64.c,
                                                           lv.K32.diag, lv.K32.invdiag, lv.K32.c, lift, P->u_top,
                                                           P->u_bottom);
    else
      k_build_K<3><<<grid_blocks(lv.g.n), 256, 0, P->st>>>(lv.g, lv.kappa, lv.K64.diag, lv.K64.invdiag, lv.K64.c,
                                                           lv.K32.diag, lv.K32.invdiag, lv.K32.c, lift, P->u_top,
                                                           P->u_bottom);
    count_launch();
    lv.K64.cpr_ok = false;  // the double-float coefficient pairs follow on first use
    if (lv.K32.pk) {
      if (D == 2)
        k_pack_K2<<<grid_blocks(lv.g.n), 256, 0, P->st>>>(lv.g.n, lv.K32.diag, lv.K32.invdiag, lv.K32.c,
                                                          reinterpret_cast<float4 *>(lv.K32.pk));
      else
        k_pack_K3<<<grid_blocks(lv.g.n), 256, 0, P->st>>>(lv.g, lv.K32.diag, lv.K32.invdiag, lv.K32.c,
                                                          reinterpret_cast<float4 *>(lv.K32.pk),
                                                          lv.K32.pk + 4 * lv.g.n);
      count_launch();
    }
  }
  HP_CUDA(cudaGetLastError());
  HP_TRY(coarse_setup(P, OP_K));
  return 0;
}

// ---------------------------------------------------------------------------
// C, C^T
//
// (C X)_v = sum_{e ni v} kappa_hat_e (K_e^1 u_e)_v with kappa_hat_e the element mean of
// E X, so C X = S_C (E (.) X) where S_C couples v to the nodes w that share a simplex
// with v: beta_{v,w} = sum_{e ni v,w} (K_e^1 u_e)_v / (D+1), K_e^1 the unit-coefficient
// element stiffness.  beta depends only on u, so it is built once per linearisation
// point; C X and C^T W = E (.) S_C^T W are then FP64 stencil applications.
// Offsets w - v: index 0 = v itself, idx = b for +b, idx = 2^D - 1 + b for -b
// (b a Kuhn edge mask), 2^{D+1} - 1 coefficients per node.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ int coff_index(int from_mask, int to_mask) {
  // simplex vertices S_k (from) and S_t (to) of one chain: to - from is +/- a Kuhn edge
  if (to_mask == from_mask) return 0;
  if ((to_mask & from_mask) == from_mask) return to_mask ^ from_mask;        // +b
  return (1 << D) - 1 + (from_mask ^ to_mask);                               // -b
}

template <int D>
__global__ void k_build_C(GridDesc g, const double *__restrict__ u, double *__restrict__ beta) {
  constexpr int NC = (1 << (D + 1)) - 1;
  const double vh2 = vol_over_h2<D>(g.h) / (D + 1);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    double b[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) b[q] = 0.0;
    const double uv = u[i];
    for_elems_with<D>(g, v, 0, [&](const int c[3], int p, int k) {
      const long base = c[0] + (long)g.np * (c[1] + (long)g.np * c[2]);
      double a = 0.0;
      if (k > 0) a += uv - u[base + mask_offset(g, MeshT<D>::chain(p, k - 1))];
      if (k < D) a += uv - u[base + mask_offset(g, MeshT<D>::chain(p, k + 1))];
      a *= vh2;
      const int mk = MeshT<D>::chain(p, k);
#pragma unroll
      for (int t = 0; t <= D; ++t) b[coff_index<D>(mk, MeshT<D>::chain(p, t))] += a;
    });
#pragma unroll
    for (int q = 0; q < NC; ++q) beta[(long)q * g.n + i] = b[q];
  }
}

// signed offset of coefficient index q: returns the mask and the sign (+1 / -1; 0 for q = 0)
template <int D>
__device__ __forceinline__ int coff_mask(int q, int *sign) {
  if (q == 0) {
    *sign = 0;
    return 0;
  }
  if (q < (1 << D)) {
    *sign = 1;
    return q;
  }
  *sign = -1;
  return q - ((1 << D) - 1);
}

template <int D>
__device__ __forceinline__ bool shift_ok(const GridDesc &g, const int v[3], int mask, int sign) {
  bool ok = true;
#pragma unroll
  for (int a = 0; a < D; ++a)
    if ((mask >> a) & 1) ok = ok && (sign > 0 ? v[a] < g.N : v[a] > 0);
  return ok;
}

// betaE_q(i) = beta_q(i) E(i + o_q): the coefficients of C with e^m folded in (once per point),
// so that C X costs one FMA per coupling
template <int D>
__global__ void k_scale_C(GridDesc g, const double *__restrict__ E, const double *__restrict__ beta,
                          double *__restrict__ betaE) {
  constexpr int NC = (1 << (D + 1)) - 1;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    betaE[i] = beta[i] * E[i];
#pragma unroll
    for (int q = 1; q < NC; ++q) {
      int sg;
      const int m = coff_mask<D>(q, &sg);
      betaE[(long)q * g.n + i] =
          shift_ok<D>(g, v, m, sg) ? beta[(long)q * g.n + i] * E[i + sg * mask_offset(g, m)] : 0.0;
    }
  }
}

// Y = scale * S_C (E (.) X) + yb * Y with the E-scaled coefficients betaE
template <int D>
__global__ void k_C_apply(GridDesc g, const double *__restrict__ betaE, const double *__restrict__ X, long ldx,
                          double *__restrict__ Y, long ldy, double scale, double yb) {
  constexpr int NC = (1 << (D + 1)) - 1;
  const int j = blockIdx.y;
  const double *x = X + ldx * j;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    double acc = betaE[i] * x[i];
#pragma unroll
    for (int q = 1; q < NC; ++q) {
      int sg;
      const int m = coff_mask<D>(q, &sg);
      if (!shift_ok<D>(g, v, m, sg)) continue;
      acc += betaE[(long)q * g.n + i] * x[i + sg * mask_offset(g, m)];
    }
    Y[ldy * j + i] = yb == 0.0 ? scale * acc : scale * acc + yb * Y[ldy * j + i];
  }
}

// Y = scale * E (.) S_C^T W + beta_acc * Y
template <int D>
__global__ void k_Ct_apply(GridDesc g, const double *__restrict__ E, const double *__restrict__ beta,
                           const double *__restrict__ W, long ldw, double *__restrict__ Y, long ldy, double scale,
                           double yb) {
  constexpr int NC = (1 << (D + 1)) - 1;
  const int j = blockIdx.y;
  const double *w = W + ldw * j;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    double acc = beta[i] * w[i];
#pragma unroll
    for (int q = 1; q < NC; ++q) {
      int sg;
      const int m = coff_mask<D>(q, &sg);
      // the row r whose offset q points at node i is r = i - (sg * m)
      if (!shift_ok<D>(g, v, m, -sg)) continue;
      const long r = i - sg * mask_offset(g, m);
      acc += beta[(long)q * g.n + r] * w[r];
    }
    const double val = scale * E[i] * acc;
    Y[ldy * j + i] = yb == 0.0 ? val : val + yb * Y[ldy * j + i];
  }
}

// The same two stencils in double-float arithmetic on the FP32 pipe (at the solve
// tolerances where the refinement runs in double-float): the input block is split into
// pairs once (k_to_pairs, grouped by 4 columns: one {hi x4, lo x4} record per node, 32
// bytes), the coefficients are kept as pairs (made once per linearisation point), and each
// thread forms the compensated (Dot2) sums of one node for 4 columns, its stencil's points
// taken in chunks whose loads are all issued before their arithmetic.  The final scaling
// (and the accumulation into Y when yb != 0) is one FP64 operation or two per element.
__global__ void k_to_pairs(const double *__restrict__ X, long ldx, int s, long n, float4 *__restrict__ Xp, long ldp) {
  const int grp = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = grp * 4 + q;
      const dfl d = d2df(col < s ? X[ldx * col + i] : 0.0);
      hi[q] = d.hi;
      lo[q] = d.lo;
    }
    const long k = 2 * ((long)grp * ldp + i);
    Xp[k] = make_float4(hi[0], hi[1], hi[2], hi[3]);
    Xp[k + 1] = make_float4(lo[0], lo[1], lo[2], lo[3]);
  }
}

__global__ void k_pairs_of(const double *__restrict__ a, long m, float2 *__restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < m; i += (long)gridDim.x * blockDim.x) {
    const dfl d = d2df(a[i]);
    out[i] = make_float2(d.hi, d.lo);
  }
}

// TRANS false: Y = scale * sum_q cpr[q][i] x[i + o_q] (+ yb Y)            (C, coefficients betaE)
// TRANS true:  Y = scale * E_i sum_q cpr[q][i + o'_q] x[i + o'_q] (+ yb Y)  (C^T, coefficients beta)
template <int D, bool TRANS>
__global__ void __launch_bounds__(NT, 2) k_cct_dfp(GridDesc g, const float2 *__restrict__ cpr,
                                                   const float2 *__restrict__ Epr, const float4 *__restrict__ Xp,
                                                   long ldp, double *__restrict__ Y, long ldy, int s, double scale,
                                                   double yb) {
  constexpr int NC = (1 << (D + 1)) - 1;
  constexpr int CH = 5;  // points per chunk of loads
  const int grp = blockIdx.y;
  const float4 *xg = Xp + 2 * (long)grp * ldp;
  const unsigned np = (unsigned)g.np, n = (unsigned)g.n;
  for (unsigned i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    int v[3];
    const unsigned t = div_np(g, i), t2 = D == 2 ? 0u : div_np(g, t);
    v[0] = (int)(i - t * np);
    v[1] = D == 2 ? (int)t : (int)(t - t2 * np);
    v[2] = (int)t2;
    Dot2 a[4];
#pragma unroll
    for (int q0 = 0; q0 < NC; q0 += CH) {
      float4 xh[CH], xl[CH];
      float2 cp[CH];
      bool ok[CH];
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        const int q = q0 + k;
        ok[k] = false;
        if (q >= NC) continue;
        int sg;
        const int m = coff_mask<D>(q, &sg);
        const int sgn = TRANS ? -sg : sg;
        ok[k] = q == 0 || shift_ok<D>(g, v, m, sgn);
        const unsigned pt = ok[k] && q > 0 ? (unsigned)((long)i + sgn * mask_offset(g, m)) : i;
        xh[k] = xg[2 * pt];
        xl[k] = xg[2 * pt + 1];
        cp[k] = cpr[(unsigned)q * n + (TRANS ? pt : i)];
      }
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        if (!ok[k]) continue;
        const dfl c{cp[k].x, cp[k].y};
        a[0].fma(c, dfl{xh[k].x, xl[k].x});
        a[1].fma(c, dfl{xh[k].y, xl[k].y});
        a[2].fma(c, dfl{xh[k].z, xl[k].z});
        a[3].fma(c, dfl{xh[k].w, xl[k].w});
      }
    }
    dfl e{1.f, 0.f};
    if (TRANS) {
      const float2 ep = Epr[i];
      e = dfl{ep.x, ep.y};
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = grp * 4 + j;
      if (col >= s) break;
      dfl r = a[j].result();
      if (TRANS) {
        Dot2 b;  // e^{m_i} times the sum
        b.fma(e, r);
        r = b.result();
      }
      const double val = scale * df2d(r);
      Y[ldy * col + i] = yb == 0.0 ? val : val + yb * Y[ldy * col + i];
    }
  }
}

// double-float C and C^T where the refinement runs in double-float (the same tolerance and
// block-size rule as the solves')
static bool cct_df(const hp_problem *P, int s) {
  return P->precision == HP_FP32_IR &&
         (P->refine_df == 2 || (P->refine_df == 1 && P->rtol >= 1e-9 && (double)P->n * s >= 16.0 * 1024 * 1024));
}

// the coefficient and e^m pairs of the u-based C, made when missing or stale
static int ensure_cct_pairs(hp_problem *P) {
  const long n = P->n, nc = P->dim == 2 ? 7 : 15;
  if (!P->CbetaE_pr) {
    HP_CUDA(cudaMalloc(&P->CbetaE_pr, sizeof(float2) * nc * n));
    HP_CUDA(cudaMalloc(&P->Cbeta_pr, sizeof(float2) * nc * n));
    HP_CUDA(cudaMalloc(&P->E_pr, sizeof(float2) * n));
  }
  if (!P->cct_pr_ok) {
    k_pairs_of<<<blocks_for(nc * n, 1), NT, 0, P->st>>>(P->CbetaE, nc * n, P->CbetaE_pr);
    k_pairs_of<<<blocks_for(nc * n, 1), NT, 0, P->st>>>(P->Cbeta, nc * n, P->Cbeta_pr);
    k_pairs_of<<<blocks_for(n, 1), NT, 0, P->st>>>(P->E, n, P->E_pr);
    count_launch(3);
    P->cct_pr_ok = true;
  }
  return cuda_check(cudaGetLastError(), "C pairs");
}

// Y = scale (C or C^T) X (+ yb Y) in double-float; false when not applicable (the caller
// then runs the FP64 kernel)
static bool cct_dfp(hp_problem *P, bool trans, const double *X, long ldx, double *Y, long ldy, int s, double scale,
                    double yb) {
  const long n = P->n, ldp = (n + 63) / 64 * 64;
  const int ng = (s + 3) / 4;
  if (ensure_cct_pairs(P) || P->xpairs.ensure(sizeof(float4) * 2 * (size_t)ldp * ng)) {
    (void)cudaGetLastError();
    return false;
  }
  float4 *Xp = P->xpairs.as<float4>();
  const dim3 gd(blocks_for(n, ng), ng);
  k_to_pairs<<<gd, NT, 0, P->st>>>(X, ldx, s, n, Xp, ldp);
  const GridDesc &g = P->lv[0].g;
  const dim3 gc(blocks_for(n, ng), ng);
  if (P->dim == 2) {
    if (trans)
      k_cct_dfp<2, true><<<gc, NT, 0, P->st>>>(g, P->Cbeta_pr, P->E_pr, Xp, ldp, Y, ldy, s, scale, yb);
    else
      k_cct_dfp<2, false><<<gc, NT, 0, P->st>>>(g, P->CbetaE_pr, nullptr, Xp, ldp, Y, ldy, s, scale, yb);
  } else {
    if (trans)
      k_cct_dfp<3, true><<<gc, NT, 0, P->st>>>(g, P->Cbeta_pr, P->E_pr, Xp, ldp, Y, ldy, s, scale, yb);
    else
      k_cct_dfp<3, false><<<gc, NT, 0, P->st>>>(g, P->CbetaE_pr, nullptr, Xp, ldp, Y, ldy, s, scale, yb);
  }
  count_launch(2);
  const double nc = P->dim == 2 ? 7.0 : 15.0;
  // the split: read X, write the pairs; the stencil: the pairs, Y (read as well when yb != 0)
  // and the coefficient pairs (and e^m for C^T)
  count_bytes(BY_CCT, 16.0 * (double)n * s);
  count_bytes(BY_CCT, (double)n * ((yb == 0.0 ? 16.0 : 24.0) * s + 8.0 * (nc + (trans ? 1.0 : 0.0))));
  return true;
}

void launch_build_C_from(hp_problem *P, const double *w, double *beta, double *betaE) {
  if (P->dim == 2) {
    k_build_C<2><<<grid_blocks(P->n), 256, 0, P->st>>>(P->lv[0].g, w, beta);
    k_scale_C<2><<<grid_blocks(P->n), 256, 0, P->st>>>(P->lv[0].g, P->E, beta, betaE);
  } else {
    k_build_C<3><<<grid_blocks(P->n), 256, 0, P->st>>>(P->lv[0].g, w, beta);
    k_scale_C<3><<<grid_blocks(P->n), 256, 0, P->st>>>(P->lv[0].g, P->E, beta, betaE);
  }
  count_launch(2);
}

void launch_build_C(hp_problem *P) {
  launch_build_C_from(P, P->u, P->Cbeta, P->CbetaE);
  P->cct_pr_ok = false;  // the double-float pairs follow on first use
}

void launch_C_apply_beta(hp_problem *P, const double *betaE, const double *X, long ldx, double *Y, long ldy, int s,
                         double scale, double yb) {
  if (betaE == P->CbetaE && cct_df(P, s) && cct_dfp(P, false, X, ldx, Y, ldy, s, scale, yb)) return;
  dim3 grid(blocks_for(P->n, s), s);
  if (P->dim == 2)
    k_C_apply<2><<<grid, NT, 0, P->st>>>(P->lv[0].g, betaE, X, ldx, Y, ldy, scale, yb);
  else
    k_C_apply<3><<<grid, NT, 0, P->st>>>(P->lv[0].g, betaE, X, ldx, Y, ldy, scale, yb);
  count_launch();
  {  // read X (and Y when yb != 0), write Y, the (2^{D+1} - 1) coefficients per node
    const double nc = P->dim == 2 ? 7.0 : 15.0;
    count_bytes(BY_CCT, 8.0 * (double)P->n * ((yb == 0.0 ? 2.0 : 3.0) * s + nc));
  }
}

void launch_C_apply(hp_problem *P, const double *X, long ldx, double *Y, long ldy, int s, double scale) {
  launch_C_apply_beta(P, P->CbetaE, X, ldx, Y, ldy, s, scale, 0.0);
}

void launch_Ct_apply_beta(hp_problem *P, const double *beta_c, const double *W, long ldw, double *Y, long ldy, int s,
                          double scale, double beta) {
  if (beta_c == P->Cbeta && cct_df(P, s) && cct_dfp(P, true, W, ldw, Y, ldy, s, scale, beta)) return;
  dim3 grid(blocks_for(P->n, s), s);
  if (P->dim == 2)
    k_Ct_apply<2><<<grid, NT, 0, P->st>>>(P->lv[0].g, P->E, beta_c, W, ldw, Y, ldy, scale, beta);
  else
    k_Ct_apply<3><<<grid, NT, 0, P->st>>>(P->lv[0].g, P->E, beta_c, W, ldw, Y, ldy, scale, beta);
  count_launch();
  {  // read W (and Y when beta != 0), write Y, e^m and the coefficients per node
    const double nc = P->dim == 2 ? 7.0 : 15.0;
    count_bytes(BY_CCT, 8.0 * (double)P->n * ((beta == 0.0 ? 2.0 : 3.0) * s + nc + 1.0));
  }
}

void launch_Ct_apply(hp_problem *P, const double *W, long ldw, double *Y, long ldy, int s, double scale,
                     double beta) {
  launch_Ct_apply_beta(P, P->Cbeta, W, ldw, Y, ldy, s, scale, beta);
}

// ---------------------------------------------------------------------------
// observation operator
// ---------------------------------------------------------------------------
__global__ void k_obs_gather(const int *__restrict__ node, const double *__restrict__ w, int nobs, int nv,
                             const double *__restrict__ X, long ldx, double *__restrict__ Yq) {
  const int j = blockIdx.y;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nobs; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nv; ++k) s += w[o * nv + k] * X[ldx * j + node[o * nv + k]];
    Yq[(long)nobs * j + o] = s;
  }
}

__global__ void k_obs_scatter(long n, const int *__restrict__ row, const int *__restrict__ ptr,
                              const int *__restrict__ ent, const double *__restrict__ w, int nobs, int nv,
                              const double *__restrict__ Yq, double *__restrict__ X, long ldx, double scale) {
  const int j = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int r = row[i];
    double s = 0.0;
    if (r >= 0) {
      for (int t = ptr[r]; t < ptr[r + 1]; ++t) {
        const int e = ent[t];
        s += w[e] * Yq[(long)nobs * j + e / nv];
      }
    }
    X[ldx * j + i] = scale * s;
  }
}

void launch_obs_gather(hp_problem *P, const double *X, long ldx, double *Yq, int s) {
  if (P->nobs == 0) return;
  dim3 grid((P->nobs + 127) / 128, s);
  k_obs_gather<<<grid, 128, 0, P->st>>>(P->obs_node, P->obs_w, P->nobs, P->dim + 1, X, ldx, Yq);
  count_launch();
  count_bytes(BY_CCT, 8.0 * (double)P->nobs * s * (P->dim + 2));
}

void launch_obs_scatter(hp_problem *P, const double *Yq, double *X, long ldx, int s, double scale) {
  dim3 grid(blocks_for(P->n, s), s);
  k_obs_scatter<<<grid, NT, 0, P->st>>>(P->n, P->bt_row, P->bt_ptr, P->bt_ent, P->obs_w, P->nobs, P->dim + 1,
                                        Yq, X, ldx, scale);
  count_launch();
  count_bytes(BY_CCT, 8.0 * ((double)P->n + (double)P->nobs) * s);
}

// ---------------------------------------------------------------------------
// rectangular factor of the mass matrix
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_mass_factor(GridDesc g, const double *__restrict__ eta, long ldeta, double *__restrict__ W,
                              long ldw) {
  const int j = blockIdx.y;
  const double *et = eta + ldeta * j;
  const double sw = sqrt(elem_vol<D>(g.h) / (D + 1));
  const double qa = (5.0 + 3.0 * sqrt(5.0)) / 20.0, qb = (5.0 - sqrt(5.0)) / 20.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.n; i += (long)gridDim.x * blockDim.x) {
    int v[3];
    node_coords<D>(g, i, v);
    double acc = 0.0;
    for_elems_with<D>(g, v, 0, [&](const int c[3], int p, int k) {
      const long e = cell_linear<D>(g, c) * MeshT<D>::NPERM + p;
#pragma unroll
      for (int q = 0; q <= D; ++q) {
        const double lam = D == 2 ? c_quad2[q][k] : (q == k ? qa : qb);
        acc += lam * et[e * (D + 1) + q];
      }
    });
    W[ldw * j + i] = sw * acc;
  }
}

void launch_mass_factor(hp_problem *P, const double *eta, long ldeta, double *W, long ldw, int s) {
  dim3 grid(blocks_for(P->n, s), s);
  if (P->dim == 2)
    k_mass_factor<2><<<grid, NT, 0, P->st>>>(P->lv[0].g, eta, ldeta, W, ldw);
  else
    k_mass_factor<3><<<grid, NT, 0, P->st>>>(P->lv[0].g, eta, ldeta, W, ldw);
  count_launch();
}

// ---------------------------------------------------------------------------
// Dirichlet rows
// ---------------------------------------------------------------------------
__global__ void k_zero_dirichlet(long face, long top_off, double *X, long ldx) {
  const int j = blockIdx.y;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < face; t += (long)gridDim.x * blockDim.x) {
    X[ldx * j + t] = 0.0;
    X[ldx * j + top_off + t] = 0.0;
  }
}

void launch_zero_dirichlet(hp_problem *P, double *X, long ldx, int s) {
  const GridDesc &g = P->lv[0].g;
  const long face = P->dim == 2 ? g.np : (long)g.np * g.np;
  dim3 grid((unsigned)std::max<long>(1, std::min<long>((face + 255) / 256, 64)), s);
  k_zero_dirichlet<<<grid, 256, 0, P->st>>>(face, g.n - face, X, ldx);
  count_launch();
}

}  // namespace hp
