"""The FP64 iterative refinement in double-float arithmetic (tuning refine_df) against the
FP64 oracle.

Around the FP32 inner solves, the refinement's residual b - K x (with its norm), the
scaling of the residual into the inner precision and the update x += d run either with
FP64 instructions (refine_df 0) or in double-float arithmetic on the FP32 pipe (pairs of
floats, compensated products and sums; refine_df 1, the default, at tolerances >= 1e-9 on
blocks of at least 2^24 values, and 2 always, with the C and C^T stencils in double-float
too).  These cases are small, so they force it with 2.  The data stay FP64 either way.
Checked here:

* at the production tolerance 1e-8, the oracle's own FP64 relative residual of every
  column is at most 1e-8, and the solution's error against the oracle's exact solve is
  within 10x that of the FP64-instruction refinement (plus 1e-10);
* forced at 1e-10, the double-float refinement still converges, to an oracle-measured
  residual of at most 1e-10;
* Gauss-Newton Hessian actions at 1e-8: the same error bound against the oracle;
* the C and C^T stencils, which run in double-float at the same tolerances, equal the
  FP64-instruction kernels to 1e-13 and the oracle to 1e-9.
"""
import numpy as np
import pytest

import workloads as W
from oracle.inverse import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"

CASES = [(2, 128, 12), (3, 32, 9), (3, 64, 3)]


def _rel_cols(A, B):
    return np.array([np.linalg.norm(A[:, j] - B[:, j]) / np.linalg.norm(B[:, j]) for j in range(B.shape[1])])


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"d{c[0]}N{c[1]}s{c[2]}")
def case(request):
    from paper_1909_03948_gb300 import Problem
    dim, N, s = request.param
    w = W.make_workload(dim, N, 40, gamma=0.1 if dim == 2 else 0.05, seed=W.SEED_BASE + 500 + N + dim)
    dr = W.draws(w)
    orc, m_true, _ = make_problem(w, dr)
    P = Problem(dim, N, w.gamma, w.delta, orc.sigma, dr.obs_xyz, d_obs=orc.d_obs, rtol=1e-8)
    m = 0.8 * m_true
    X = W.random_block(orc.n, s, 2000 + N)
    free = orc.free
    Kff = orc.stiffness(m)[free][:, free]
    yield dict(P=P, orc=orc, m=m, X=X, free=free, Kff=Kff)
    P.close()


def _T(X):
    return torch.tensor(np.ascontiguousarray(X.T), device=DEV)


def _solve(P, m, X, refine_df, rtol):
    P.set_tuning(refine_df=refine_df)
    P.set_tolerance(rtol)
    P.set_point(torch.tensor(m, device=DEV))
    U, st = P.state_solve(_T(X))
    return U.cpu().numpy().T, st


def _oracle_residuals(c, U):
    free, Kff, X = c["free"], c["Kff"], c["X"]
    R = X[free] - Kff @ U[free]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(X[free], axis=0)


def test_df_state_solve_at_the_production_tolerance(case):
    P, orc, m, X = case["P"], case["orc"], case["m"], case["X"]
    try:
        U64, _ = _solve(P, m, X, 0, 1e-8)
        Udf, st = _solve(P, m, X, 2, 1e-8)
    finally:
        P.set_tuning()
        P.set_tolerance(1e-8)
    assert _oracle_residuals(case, Udf).max() <= 1.01e-8
    assert _oracle_residuals(case, U64).max() <= 1.01e-8
    ref = orc.solve_state(m, X)
    e_df, e_64 = _rel_cols(Udf, ref), _rel_cols(U64, ref)
    print(f"state solve error at 1e-8: double-float {e_df.max():.2e}, FP64 {e_64.max():.2e}")
    assert np.all(e_df <= 10.0 * e_64 + 1e-10)


def test_df_refinement_converges_at_1e_10(case):
    P, m, X = case["P"], case["m"], case["X"]
    try:
        U, st = _solve(P, m, X, 2, 1e-10)
    finally:
        P.set_tuning()
        P.set_tolerance(1e-8)
    res = _oracle_residuals(case, U)
    print(f"double-float refinement at 1e-10: oracle residual {res.max():.2e}, {st['outer']} steps")
    assert res.max() <= 1.01e-10


def test_df_hessian_action_at_the_production_tolerance(case):
    P, orc, m, X = case["P"], case["orc"], case["m"], case["X"]
    out = {}
    try:
        for rd in (0, 2):
            P.set_tuning(refine_df=rd)
            P.set_tolerance(1e-8)
            P.set_point(torch.tensor(m, device=DEV))
            out[rd] = P.hessian_apply(_T(X))[0].cpu().numpy().T
    finally:
        P.set_tuning()
    ref = orc.hessian_misfit(m, orc.forward(m), X)
    e_df, e_64 = _rel_cols(out[2], ref), _rel_cols(out[0], ref)
    print(f"Hessian action error at 1e-8: double-float {e_df.max():.2e}, FP64 {e_64.max():.2e}")
    assert np.all(e_df <= 10.0 * e_64 + 1e-9)


def test_df_C_and_Ct_equal_the_fp64_kernels(case):
    """The C and C^T stencils (Appendix A: the incremental forward right-hand side and the
    Hessian action's last step) in double-float against the FP64-instruction kernels on the
    same linearisation point, and both against the oracle."""
    P, orc, m, X = case["P"], case["orc"], case["m"], case["X"]
    Wm = W.random_block(orc.n, X.shape[1], 3000)
    Wm[orc.dmask] = 0.0
    out = {}
    try:
        P.set_tolerance(1e-11)
        P.set_point(torch.tensor(m, device=DEV))
        for rd in (0, 2):
            P.set_tuning(refine_df=rd)
            out[rd] = (P.C_apply(_T(X)).cpu().numpy().T, P.Ct_apply(_T(Wm)).cpu().numpy().T)
    finally:
        P.set_tuning()
        P.set_tolerance(1e-8)
    assert _rel_cols(out[2][0], out[0][0]).max() < 1e-13
    assert _rel_cols(out[2][1], out[0][1]).max() < 1e-13
    u = orc.forward(m)
    assert _rel_cols(out[2][0], orc.C_apply(m, u, X)).max() < 1e-9
    assert _rel_cols(out[2][1], orc.Ct_apply(m, u, Wm)).max() < 1e-9


def test_df_host_loop_equals_graph(case):
    """The double-float refinement as one graph launch and as a host loop over the same
    kernels (profiling on) gives the same solution bit for bit."""
    P, m, X = case["P"], case["m"], case["X"]
    try:
        Ug, _ = _solve(P, m, X, 2, 1e-8)
        P.profile_enable(True)
        try:
            U = P.state_solve(_T(X))[0].cpu().numpy().T
        finally:
            P.profile_enable(False)
    finally:
        P.set_tuning()
    assert np.array_equal(U, Ug)
