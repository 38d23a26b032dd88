// tune.cu -- solver tuning knobs and the autotuner.
//
// Knobs: the V-cycle's smoother (nu sweeps, damped Jacobi with omega or Chebyshev
// weights on [lmax / alpha, lmax]), the RHS column chunk processed per solve (0 = all
// columns at once), fused grid transfers, the shared-memory coarse tail, the TMA-tiled
// stencil kernels, the double-float refinement and the grid-size cap of the node
// kernels.  hp_autotune times one block of Gauss-Newton Hessian actions at the current
// linearisation point (CUDA events on the problem's stream) for each candidate, by
// coordinate descent over the groups of knobs, and keeps the fastest.  Every candidate
// solves to the same tolerance, so tuning changes speed, not the stopping rule.
#include <algorithm>
#include <vector>

#include "internal.h"

using namespace hp;

extern "C" {

int hp_set_tuning(hp_problem *P, const hp_tuning *t) {
  if (!P || !t) return set_error(HP_ERR_INVALID, "hp_set_tuning: null");
  if (t->nu < 1 || t->nu > 4 || t->nu_coarse < 0 || t->nu_coarse > 4 || !(t->omega > 0.0 && t->omega < 1.0) || t->col_chunk < 0 || t->max_blocks < 64 ||
      t->max_blocks > (1 << 20) || t->fuse_from != 0 || t->smoother < 0 ||
      t->smoother > 1 || (t->smoother == 1 && !(t->cheb_alpha > 1.0 && t->cheb_alpha < 1e6)) ||
      t->fuse_transfer < 0 || t->fuse_transfer > 2 || t->tma_tiles < 0 || t->tma_tiles > 2 ||
      t->smem_tail < 0 || t->smem_tail >= HP_MAXL || t->refine_df < 0 || t->refine_df > 2)
    return set_error(HP_ERR_INVALID, "hp_set_tuning: nu in [1,4], omega in (0,1), col_chunk >= 0, max_blocks >= 64, "
                                     "fuse_from 0 (reserved), smoother 0/1, cheb_alpha > 1, fuse_transfer 0..2, tma_tiles 0..2, smem_tail in [0, 15], "
                                     "refine_df 0..2");
  HP_CUDA(cudaStreamSynchronize(P->st));
  if (t->nu != P->nu || t->nu_coarse != P->nu_coarse || t->omega != P->omega || t->max_blocks != P->max_blocks || t->fuse_from != P->fuse_from ||
      t->smoother != P->smoother || (t->smoother == 1 && t->cheb_alpha != P->cheb_alpha) ||
      t->fuse_transfer != P->fuse_transfer || t->tma_tiles != P->tma_tiles || t->smem_tail != P->smem_tail ||
      t->refine_df != P->refine_df)
    drop_graphs(P);
  P->refine_df = t->refine_df;
  P->tma_tiles = t->tma_tiles;
  P->smem_tail = t->smem_tail;
  P->fuse_transfer = t->fuse_transfer;
  P->fuse_from = t->fuse_from;
  P->smoother = t->smoother;
  if (t->smoother == 1) P->cheb_alpha = t->cheb_alpha;
  P->nu = t->nu;
  P->nu_coarse = t->nu_coarse;
  P->omega = t->omega;
  P->col_chunk = t->col_chunk;
  P->max_blocks = t->max_blocks;
  return HP_OK;
}

int hp_get_tuning(const hp_problem *P, hp_tuning *t) {
  if (!P || !t) return set_error(HP_ERR_INVALID, "hp_get_tuning: null");
  t->nu = P->nu;
  t->nu_coarse = P->nu_coarse;
  t->omega = P->omega;
  t->col_chunk = P->col_chunk;
  t->max_blocks = (int)P->max_blocks;
  t->fuse_from = P->fuse_from;
  t->smoother = P->smoother;
  t->cheb_alpha = P->cheb_alpha;
  t->fuse_transfer = P->fuse_transfer;
  t->tma_tiles = P->tma_tiles;
  t->smem_tail = P->smem_tail;
  t->refine_df = P->refine_df;
  return HP_OK;
}

}  // extern "C"

// The search of hp_autotune / hp_autotune_block on the device block X (n x nrhs, ldx).
static int autotune_on(hp_problem *P, const double *X, int ldx, int nrhs, int reps, hp_tuning *best,
                       double *best_ms) {
  const long n = P->n;
  double *Y = nullptr;
  if (cudaMalloc(&Y, sizeof(double) * n * nrhs) != cudaSuccess) return set_error(HP_ERR_NOMEM, "autotune: workspace");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto cleanup = [&](int rc) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(Y);
    return rc;
  };
  auto time_it = [&](const hp_tuning &t, double *ms) -> int {
    int rc = hp_set_tuning(P, &t);
    if (rc) return rc;
    rc = hp_hessian_apply(P, X, ldx, Y, (int)n, nrhs, HP_MISFIT_ONLY, nullptr);  // warm: builds graphs
    if (rc) return rc;
    double acc = 0.0;
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(e0, P->st);
      rc = hp_hessian_apply(P, X, ldx, Y, (int)n, nrhs, HP_MISFIT_ONLY, nullptr);
      if (rc) return rc;
      cudaEventRecord(e1, P->st);
      cudaEventSynchronize(e1);
      float f = 0.f;
      cudaEventElapsedTime(&f, e0, e1);
      acc += f;
    }
    *ms = acc / reps;
    return 0;
  };
  hp_tuning cur;
  hp_get_tuning(P, &cur);
  double cur_ms = 0.0;
  int rc = time_it(cur, &cur_ms);
  if (rc) return cleanup(rc);
  // a candidate replaces the current settings only when it is at least 1 % faster, so that
  // timing noise does not walk the search away from a good point
  auto consider = [&](const hp_tuning &t) -> int {
    double ms;
    const int r = time_it(t, &ms);
    if (r) return r;
    if (ms < 0.99 * cur_ms) {
      cur = t;
      cur_ms = ms;
    }
    return 0;
  };
  struct SmoothC {
    int nu, kind;
    double omega, alpha;
  };
  const SmoothC smooth[] = {{2, 0, 0.8, 10.0}, {2, 1, 0.7, 5.0}, {2, 1, 0.7, 12.0}, {3, 1, 0.7, 8.0},
                            {3, 1, 0.7, 10.0}, {3, 1, 0.7, 12.0}, {4, 1, 0.7, 12.0}};
  // coordinate descent over the settings, twice: the second pass re-times the point the first
  // one reached and revisits every coordinate from there
  for (int pass = 0; pass < 2; ++pass) {
    if (pass > 0 && (rc = time_it(cur, &cur_ms))) return cleanup(rc);
    for (const SmoothC &sm : smooth) {
      if (sm.nu == cur.nu && sm.kind == cur.smoother && (sm.kind == 0 ? sm.omega == cur.omega
                                                                       : sm.alpha == cur.cheb_alpha))
        continue;
      hp_tuning t = cur;
      t.nu = sm.nu;
      t.omega = sm.omega;
      t.smoother = sm.kind;
      t.cheb_alpha = sm.alpha;
      if ((rc = consider(t))) return cleanup(rc);
    }
    for (int w : {0, 32, 16}) {
      if (w >= nrhs || w == cur.col_chunk) continue;
      hp_tuning t = cur;
      t.col_chunk = w;
      if ((rc = consider(t))) return cleanup(rc);
    }
    for (int ft : {0, 2, 1}) {
      if (ft == cur.fuse_transfer) continue;
      hp_tuning t = cur;
      t.fuse_transfer = ft;
      if ((rc = consider(t))) return cleanup(rc);
    }
    for (int st : {0, 1}) {
      if (st == cur.smem_tail) continue;
      hp_tuning t = cur;
      t.smem_tail = st;
      if ((rc = consider(t))) return cleanup(rc);
    }
    for (int tt : {0, 1, 2}) {
      if (tt == cur.tma_tiles) continue;
      hp_tuning t = cur;
      t.tma_tiles = tt;
      if ((rc = consider(t))) return cleanup(rc);
    }
    for (int mb : {1024, 2048, 4096}) {
      if (mb == cur.max_blocks) continue;
      hp_tuning t = cur;
      t.max_blocks = mb;
      if ((rc = consider(t))) return cleanup(rc);
    }
  }
  if ((rc = hp_set_tuning(P, &cur))) return cleanup(rc);
  if (best) *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return cleanup(HP_OK);
}

extern "C" {

int hp_autotune(hp_problem *P, int nrhs, int reps, hp_tuning *best, double *best_ms) {
  if (!P || nrhs < 1 || reps < 1) return set_error(HP_ERR_INVALID, "hp_autotune: arguments");
  if (!P->have_point) return set_error(HP_ERR_STATE, "hp_set_point must be called first");
  const long n = P->n;
  double *X = nullptr;
  HP_CUDA(cudaMalloc(&X, sizeof(double) * n * nrhs));
  launch_philox_normals(0x7475ULL, 0, nrhs, (int)n, X, n, 0, P->st);
  const int rc = autotune_on(P, X, (int)n, nrhs, reps, best, best_ms);
  cudaFree(X);
  return rc;
}

int hp_autotune_block(hp_problem *P, const double *X, int ldx, int nrhs, int reps, hp_tuning *best,
                      double *best_ms) {
  if (!P || !X || nrhs < 1 || reps < 1 || ldx < P->n) return set_error(HP_ERR_INVALID, "hp_autotune_block: arguments");
  if (!P->have_point) return set_error(HP_ERR_STATE, "hp_set_point must be called first");
  return autotune_on(P, X, ldx, nrhs, reps, best, best_ms);
}

}  // extern "C"
