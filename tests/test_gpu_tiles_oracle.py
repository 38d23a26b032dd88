"""GPU parity of the TMA-tiled stencil kernels against the FP64 oracle.

The level stencils of the FP32 inner solves have two kernel forms: the row kernel and the
TMA-tiled kernels (2D 32 x 16-node tiles; the 3D z-marching kernel on 32 x 8-node xy tiles).
The tiled forms run on every level whose node count per axis minus one is a multiple of
32, with the tma_tiles setting on.  These cases turn it on, check through the library's
own launch counter that tiled launches ran (the calls that check it run with profiling
on, which launches every kernel directly: launches replayed from a CUDA graph are not
counted), and compare state solves and Gauss-Newton Hessian actions (Appendix A, eqs.
incrementals1-3 without the adjoint terms) with the oracle element by element:

  3D 64^3 (274,625 nodes, the oracle's CG solves), 118 columns (a ragged last group of 4)
  2D 256^2 (66,049 nodes), 60 columns; 2D 512^2 (263,169 nodes), 57 columns (ragged)

Tolerances as in the other parity tests: state solves 1e-8, Hessian actions 1e-7, both
with the GPU solves at relative residual 1e-11.  A second pass at the production
tolerance 1e-8 states the error of the FP32-in-FP64-refinement path per output: the
oracle's FP64 relative residual of the state solve (at most 1e-8 by construction) and the
Hessian action's error against the exact one.
"""
import numpy as np
import pytest

import workloads as W
from oracle.inverse import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"

CASES = [(3, 64, 118, 3), (2, 256, 60, 8), (2, 512, 57, 6)]


def _colrel(A, B):
    return max(np.linalg.norm(A[:, j] - B[:, j]) / np.linalg.norm(B[:, j]) for j in range(B.shape[1]))


def _cols(s, nsample):
    """Sampled columns: spread over the block, always the first and the last (ragged) one."""
    return sorted(set(np.linspace(0, s - 1, nsample).round().astype(int).tolist()))


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"d{c[0]}N{c[1]}s{c[2]}")
def case(request):
    from paper_1909_03948_gb300 import Problem
    dim, N, s, nsample = request.param
    w = W.make_workload(dim, N, 60 if dim == 2 else 120, gamma=0.1 if dim == 2 else 0.05,
                        seed=W.SEED_BASE + 700 + N + dim)
    dr = W.draws(w)
    orc, m_true, _ = make_problem(w, dr)
    P = Problem(dim, N, w.gamma, w.delta, orc.sigma, dr.obs_xyz, d_obs=orc.d_obs, rtol=1e-11)
    P.set_tuning(tma_tiles=1)
    m = 0.8 * m_true
    P.set_point(torch.tensor(m, device=DEV))
    X = W.random_block(orc.n, s, 1000 + N)
    yield dict(P=P, orc=orc, m=m, u=orc.forward(m), X=X, cols=_cols(s, nsample), s=s)
    P.close()


def _T(X):
    return torch.tensor(np.ascontiguousarray(X.T), device=DEV)


def test_tiled_state_solve_matches_oracle(case):
    from paper_1909_03948_gb300 import tiled_kernel_launches
    P, orc, m, X, cols = case["P"], case["orc"], case["m"], case["X"], case["cols"]
    t0 = tiled_kernel_launches()
    P.profile_enable(True)
    try:
        U, st = P.state_solve(_T(X))
    finally:
        P.profile_enable(False)
    assert tiled_kernel_launches() > t0, "the TMA-tiled kernels did not run"
    U = U.cpu().numpy().T
    ref = orc.solve_state(m, X[:, cols])
    assert _colrel(U[:, cols], ref) < 1e-8
    assert st["rel_res"] <= 1e-11


def test_tiled_hessian_action_matches_oracle(case):
    from paper_1909_03948_gb300 import tiled_kernel_launches
    P, orc, m, X, cols = case["P"], case["orc"], case["m"], case["X"], case["cols"]
    t0 = tiled_kernel_launches()
    P.profile_enable(True)
    try:
        Y, _ = P.hessian_apply(_T(X))
    finally:
        P.profile_enable(False)
    assert tiled_kernel_launches() > t0, "the TMA-tiled kernels did not run"
    Y = Y.cpu().numpy().T
    ref = orc.hessian_misfit(m, case["u"], X[:, cols])
    assert _colrel(Y[:, cols], ref) < 1e-7


def test_tiled_path_at_the_production_tolerance(case):
    """rtol 1e-8 (the benchmark's tolerance): the oracle's own FP64 relative residual of
    the GPU state solve is at most 1e-8, and the Hessian action is within 1e-5 of the
    exact one (errors measured on the GPU are recorded in the design notes)."""
    P, orc, m, X, cols = case["P"], case["orc"], case["m"], case["X"], case["cols"]
    P.set_tolerance(1e-8)
    try:
        P.set_point(torch.tensor(m, device=DEV))
        U, _ = P.state_solve(_T(X))
        U = U.cpu().numpy().T
        free = orc.free
        Kff = orc.stiffness(m)[free][:, free]
        for j in cols:
            b = X[free, j]
            r = b - Kff @ U[free, j]
            assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(b)
        Y, _ = P.hessian_apply(_T(X))
        Y = Y.cpu().numpy().T
        err = _colrel(Y[:, cols], orc.hessian_misfit(m, case["u"], X[:, cols]))
        print(f"production-tolerance Hessian action error (max over sampled columns): {err:.2e}")
        assert err < 1e-5
    finally:
        P.set_tolerance(1e-11)
        P.set_point(torch.tensor(m, device=DEV))
