"""Parity at the workloads' full sizes, in the launch configuration bench.py times: the
same block width, and the solver settings the autotuner (``tuning.tuned``) picks for it.

medium2d: 256^2 right triangles, 66,049 nodes, 400 observations, a block of k + p = 60
Gauss-Newton actions on the benchmark's directions.  The oracle computes single columns
of the action (two sparse direct solves each), so sampled columns are compared with it.
The solves run at relative residual 1e-11 rather than the benchmark's 1e-8: at 1e-8
the action's error against the exact one is not fixed by the tolerance.  An FP32-inner /
FP64-refined solve emulated on the CPU at this size left action errors about 20 times the
final relative residual; the bound of 1e-7 used here is the small-case parity bound.

cube3d: 64^3 Kuhn tetrahedra, 274,625 nodes, 1000 observations, 120 actions.  The
oracle solves this size by Jacobi-preconditioned CG to relative residual 1e-13 (a sparse
direct factorisation does not finish in minutes in 3D), about ten seconds per column, so
two sampled columns (the first and the last) are compared with it; the whole block is also checked through properties that hold at any
size: Omega^T H Omega is symmetric and positive semi-definite (H is, Section 2.2), and a
column applied on its own equals the block's column.
"""
import numpy as np
import pytest

import workloads as W
from oracle.inverse import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = 1e-7


def _colrel(A, B):
    return max(np.linalg.norm(A[:, j] - B[:, j]) / np.linalg.norm(B[:, j]) for j in range(B.shape[1]))


def _bench_settings(P, s, tmp_path):
    """The autotuned settings bench.py runs this block with (a private tuning table, so
    the test leaves the user's table alone)."""
    from paper_1909_03948_gb300 import tuning
    settings, _, _ = tuning.tuned(P, s, "fp32_ir", path=str(tmp_path / "tuning.json"))
    return settings


def _projected_checks(Om, Y):
    """Omega^T H Omega symmetric and positive semi-definite to TOL of its largest entry."""
    G = Om.T @ Y
    scale = np.abs(G).max()
    assert np.abs(G - G.T).max() <= TOL * scale
    ev = np.linalg.eigvalsh(0.5 * (G + G.T))
    assert ev.min() >= -TOL * scale


def test_medium2d_block_against_the_oracle(tmp_path):
    from paper_1909_03948_gb300 import Problem
    w = W.WORKLOADS["medium2d"]
    dr = W.draws(w)
    orc, m_true, _ = make_problem(w, dr)
    P = Problem(w.dim, w.N, w.gamma, w.delta, orc.sigma, dr.obs_xyz, d_obs=orc.d_obs, rtol=1e-8)
    try:
        m = torch.tensor(m_true, device=DEV)
        P.set_point(m)
        _bench_settings(P, w.k + w.p, tmp_path)
        P.set_tolerance(1e-11)
        P.set_point(m)  # the state again, at the tighter tolerance
        Om = W.omega(w)
        Y, st = P.hessian_apply(torch.tensor(np.ascontiguousarray(Om.T), device=DEV))
        Y = Y.cpu().numpy().T
        assert np.isfinite(Y).all()
        cols = [0, 29, 59]
        ref = orc.hessian_misfit(m_true, orc.forward(m_true), Om[:, cols])
        assert _colrel(Y[:, cols], ref) < TOL
        _projected_checks(Om, Y)
    finally:
        P.close()


def test_cube3d_block_against_the_oracle(tmp_path):
    from paper_1909_03948_gb300 import Problem, tiled_kernel_launches
    w = W.WORKLOADS["cube3d"]
    dr = W.draws(w)
    s = w.k + w.p
    orc, m_true, _ = make_problem(w, dr)
    assert orc.solver == "cg"
    P = Problem(w.dim, w.N, w.gamma, w.delta, orc.sigma, dr.obs_xyz, d_obs=orc.d_obs, rtol=1e-8)
    try:
        m = torch.tensor(m_true, device=DEV)
        P.set_point(m)
        _bench_settings(P, s, tmp_path)
        P.set_tolerance(1e-11)
        P.set_point(m)
        Om = W.omega(w)
        t0 = tiled_kernel_launches()
        P.profile_enable(True)       # direct launches, so that the tiled-launch counter sees them
        try:
            Y, _ = P.hessian_apply(torch.tensor(np.ascontiguousarray(Om.T), device=DEV))
        finally:
            P.profile_enable(False)
        tiled = tiled_kernel_launches() > t0
        Y = Y.cpu().numpy().T
        assert np.isfinite(Y).all()
        cols = [0, s - 1]
        ref = orc.hessian_misfit(m_true, orc.forward(m_true), Om[:, cols])
        err = _colrel(Y[:, cols], ref)
        print(f"cube3d Hessian action error against the oracle: {err:.2e} (tiled kernels: {tiled})")
        assert err < TOL
        _projected_checks(Om, Y)
        y0, _ = P.hessian_apply(torch.tensor(np.ascontiguousarray(Om[:, :1].T), device=DEV))
        y0 = y0.cpu().numpy().T
        assert _colrel(y0, Y[:, :1]) < TOL
    finally:
        P.close()
