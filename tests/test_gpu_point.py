"""Linearisation-point bookkeeping on the GPU: a call at the current point rebuilds nothing
(only a bitwise comparison and, if asked, the cost), a changed point or a tighter solve
tolerance rebuilds everything, and switching the inner-solve precision after creation
refactors the coarse-grid inverses in that precision (FP32 factorisation for FP32 inner
solves, FP64 for the plain FP64 path) with unchanged results."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _problem(precision="fp32_ir", rtol=1e-8, N=64):
    from paper_1909_03948_gb300 import Problem
    w = W.make_workload(2, N, 40, seed=17)
    dr = W.draws(w)
    return Problem(2, N, w.gamma, w.delta, 0.01, dr.obs_xyz, rtol=rtol, precision=precision)


def test_current_point_is_kept_and_changes_rebuild():
    from paper_1909_03948_gb300 import kernel_launches
    P = _problem()
    m = 0.3 * torch.tensor(np.random.default_rng(1).standard_normal(P.n), device=DEV)
    l0 = kernel_launches()
    J1 = P.set_point(m)
    full = kernel_launches() - l0
    # the cost (with its mass solve) is evaluated either way; the operators' rebuild and the
    # state solve are the difference
    l0 = kernel_launches()
    J2 = P.set_point(m.clone())                      # same values, another buffer
    kept = kernel_launches() - l0
    assert J2 == J1 and kept < 0.75 * full, (kept, full)
    m2 = m.clone()
    m2[P.n // 2] += 1e-12                            # one entry changed
    l0 = kernel_launches()
    P.set_point(m2)
    assert kernel_launches() - l0 >= 0.9 * full, (kernel_launches() - l0, full)
    P.set_point(m)
    P.set_tolerance(1e-10)                           # the state must be solved again, tighter
    l0 = kernel_launches()
    J3 = P.set_point(m)
    assert kernel_launches() - l0 >= 0.9 * full
    assert abs(J3[0] - J1[0]) <= 1e-6 * abs(J1[0])
    P.close()


def test_precision_switch_refactors_coarse_inverse():
    m = 0.3 * torch.tensor(np.random.default_rng(2).standard_normal(65 * 65), device=DEV)
    X = torch.tensor(np.random.default_rng(3).standard_normal((3, 65 * 65)), device=DEV)
    ref = _problem("fp64", rtol=1e-10)
    ref.set_point(m)
    Y_ref, _ = ref.hessian_apply(X)
    Z_ref, _ = ref.prior_solve(X)
    ref.close()
    P = _problem("fp32_ir", rtol=1e-10)
    P.set_point(m)
    Y32, _ = P.hessian_apply(X)
    P.set_precision("fp64")                          # inv64 is rebuilt for the plain path
    Y64, _ = P.hessian_apply(X)
    Z64, _ = P.prior_solve(X)
    P.set_precision("fp32_ir")
    Y32b, _ = P.hessian_apply(X)
    P.close()
    for Y in (Y32, Y64, Y32b):
        assert float(torch.linalg.norm(Y - Y_ref) / torch.linalg.norm(Y_ref)) <= 1e-8
    assert float(torch.linalg.norm(Z64 - Z_ref) / torch.linalg.norm(Z_ref)) <= 1e-8
