// batch.cu -- many independent inverse problems of uneven size on one GPU.
//
// Each problem gets its own CUDA stream; a pool of host threads drives the
// problems (one at a time per thread), so the per-problem kernel sequences --
// each inner solve a CUDA graph with a device-side while loop -- run
// concurrently and fill the SMs that a single small problem leaves idle.  A
// problem's own sequence is unchanged, so batched results equal the results of
// the same calls made one problem at a time.  The streams share the device's
// hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 unless the process sets
// it before CUDA starts; 32 measured 7.8 % more actions/s on 64 problems and a
// third off MAP + eigenpairs).
#include <algorithm>
#include <atomic>
#include <functional>
#include <thread>
#include <vector>

#include "internal.h"

struct hp_batch {
  std::vector<hp_problem *> P;
  std::vector<cudaStream_t> streams;
  int nthreads = 1;
  int device = 0;
};

namespace hp {

// Runs work(i) for every problem on the thread pool, handing problems out in index order,
// or largest first when weight is given (by weight(i), ties in index order: the
// longest-processing-time rule, which keeps a long problem from starting last and running
// alone at the end).  Largest first took MAP + eigenpairs of 64 problems from 9.94 to
// 9.77 s but made one block of Hessian actions 1 % slower, so only the former uses it.
template <class F>
static void run_pool(hp_batch *B, F &&work, const std::function<double(int)> *weight) {
  std::atomic<int> next{0};
  const int n = (int)B->P.size();
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  if (weight) std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return (*weight)(a) > (*weight)(b); });
  auto body = [&]() {
    cudaSetDevice(B->device);
    for (int k = next.fetch_add(1); k < n; k = next.fetch_add(1)) work(order[k]);
  };
  std::vector<std::thread> pool;
  const int nt = std::max(1, std::min(B->nthreads, n));
  for (int t = 1; t < nt; ++t) pool.emplace_back(body);
  body();
  for (auto &t : pool) t.join();
}

}  // namespace hp

using namespace hp;

extern "C" {

int hp_batch_create(hp_problem *const *problems, int nproblems, int nthreads, hp_batch **out) {
  if (!problems || nproblems < 1 || !out) return set_error(HP_ERR_INVALID, "hp_batch_create: arguments");
  hp_batch *B = new hp_batch();
  HP_CUDA(cudaGetDevice(&B->device));
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  B->nthreads = nthreads > 0 ? nthreads : (int)std::min<unsigned>(hw, 16u);
  for (int i = 0; i < nproblems; ++i) {
    if (!problems[i]) {
      delete B;
      return set_error(HP_ERR_INVALID, "hp_batch_create: null problem");
    }
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto q : B->streams) cudaStreamDestroy(q);
      delete B;
      return set_error(HP_ERR_CUDA, "hp_batch_create: stream");
    }
    B->streams.push_back(s);
    B->P.push_back(problems[i]);
    hp_set_stream(problems[i], s);
  }
  *out = B;
  return HP_OK;
}

void hp_batch_destroy(hp_batch *B) {
  if (!B) return;
  for (size_t i = 0; i < B->P.size(); ++i) {
    cudaStreamSynchronize(B->streams[i]);
    hp_set_stream(B->P[i], nullptr);
    cudaStreamDestroy(B->streams[i]);
  }
  delete B;
}

int hp_batch_map_and_eig(hp_batch *B, double *const *m_inout, const hp_newton_opts *opts, int k, int p,
                         const double *const *Omega, const int *ldo, double *const *lambda, double *const *V,
                         const int *ldv, hp_newton_stats *nstats, int *status) {
  if (!B || !m_inout || !Omega || !ldo || !lambda || !V || !ldv || !status)
    return set_error(HP_ERR_INVALID, "hp_batch_map_and_eig: arguments");
  const std::function<double(int)> largest = [&](int i) { return (double)B->P[i]->n; };
  run_pool(
      B,
      [&](int i) {
    hp_newton_stats st{};
    int rc = hp_newton_cg_map(B->P[i], m_inout[i], opts, &st);
    if (nstats) nstats[i] = st;
    if (rc == HP_OK || rc == HP_ERR_NOT_CONVERGED)
      rc = hp_lowrank_eig(B->P[i], m_inout[i], k, p, Omega[i], ldo[i], lambda[i], V[i], ldv[i], 0, nullptr);
    status[i] = rc;
      },
      &largest);
  for (size_t i = 0; i < B->P.size(); ++i)
    if (status[i] != HP_OK) return set_error(status[i], "hp_batch_map_and_eig: a problem failed (see status)");
  return HP_OK;
}

int hp_batch_hessian_apply(hp_batch *B, const double *const *X, const int *ldx, double *const *Y, const int *ldy,
                           const int *nrhs, int flags, int *status) {
  if (!B || !X || !ldx || !Y || !ldy || !nrhs || !status)
    return set_error(HP_ERR_INVALID, "hp_batch_hessian_apply: arguments");
  run_pool(
      B, [&](int i) { status[i] = hp_hessian_apply(B->P[i], X[i], ldx[i], Y[i], ldy[i], nrhs[i], flags, nullptr); },
      nullptr);
  for (size_t i = 0; i < B->P.size(); ++i)
    if (status[i] != HP_OK) return set_error(status[i], "hp_batch_hessian_apply: a problem failed (see status)");
  return HP_OK;
}

int hp_batch_set_point(hp_batch *B, const double *const *m, int *status) {
  if (!B || !m || !status) return set_error(HP_ERR_INVALID, "hp_batch_set_point: arguments");
  run_pool(B, [&](int i) { status[i] = hp_set_point(B->P[i], m[i], nullptr); }, nullptr);
  for (size_t i = 0; i < B->P.size(); ++i)
    if (status[i] != HP_OK) return set_error(status[i], "hp_batch_set_point: a problem failed (see status)");
  return HP_OK;
}

}  // extern "C"
