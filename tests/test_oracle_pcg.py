"""Pins for the oracle's iterative solves (oracle/pcg.py), used on the 3D meshes where a
sparse direct factorisation does not finish in minutes:

* the Jacobi-PCG solution equals a sparse direct solve (SuperLU) and its true residual is
  at the requested tolerance;
* a Problem solved by CG equals the same Problem solved directly in every quantity that
  involves a solve (state, adjoint, prior and mass solves, gradient, Hessian action);
* through the CG path alone: m = 0 gives the exact linear state u = x_last (a case P1
  reproduces exactly), and a 3D manufactured solution converges at O(h^2);
* the columns of a block are independent (a block equals its columns solved one by one).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle.fem import Mesh
from oracle.inverse import CG_RTOL, Problem, make_problem
from oracle.pcg import jacobi_pcg


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _stiffness_ff(N, seed=0):
    mesh = Mesh(3, N)
    m = 0.8 * np.random.default_rng(seed).standard_normal(mesh.n)
    K = mesh.stiffness(mesh.elem_mean(np.exp(m)))
    free = np.flatnonzero(~mesh.dirichlet_mask)
    return K[free][:, free].tocsr()


def test_pcg_equals_direct_solve_and_meets_its_residual():
    K = _stiffness_ff(10)
    B = np.random.default_rng(1).standard_normal((K.shape[0], 3))
    X = jacobi_pcg(K, B, rtol=1e-13)
    ref = spla.splu(K.tocsc()).solve(B)
    for j in range(3):
        assert _rel(X[:, j], ref[:, j]) < 1e-10
        assert np.linalg.norm(B[:, j] - K @ X[:, j]) <= 1e-13 * np.linalg.norm(B[:, j])


def test_pcg_block_columns_are_independent():
    K = _stiffness_ff(8, seed=2)
    rng = np.random.default_rng(3)
    B = rng.standard_normal((K.shape[0], 4))
    B[:, 2] *= 1e-6                              # columns of very different size converge apart
    X = jacobi_pcg(K, B, rtol=1e-12)
    for j in range(4):
        assert _rel(X[:, j], jacobi_pcg(K, B[:, j], rtol=1e-12)) < 1e-11
    assert np.all(jacobi_pcg(K, np.zeros(K.shape[0])) == 0.0)


def test_pcg_raises_when_it_cannot_converge():
    K = _stiffness_ff(6)
    with pytest.raises(RuntimeError):
        jacobi_pcg(K, np.ones(K.shape[0]), rtol=1e-13, maxiter=3, restarts=0, accept=1.0)


def test_cg_problem_equals_direct_problem():
    w = W.make_workload(3, 10, 20, gamma=0.05, seed=W.SEED_BASE + 900)
    dr = W.draws(w)
    pd, m_true, _ = make_problem(w, dr, solver="direct")
    pc, m_true_c, _ = make_problem(w, dr, solver="cg")
    assert pc.solver == "cg" and pd.solver == "direct"
    assert _rel(m_true_c, m_true) < 1e-10                       # prior draw: an A solve
    assert abs(pc.sigma - pd.sigma) <= 1e-10 * pd.sigma
    m = 0.8 * m_true
    u_d, u_c = pd.forward(m), pc.forward(m)
    assert _rel(u_c, u_d) < 1e-10
    X = W.random_block(pd.n, 3, 11)
    assert _rel(pc.M_solve(X), pd.M_solve(X)) < 1e-10
    assert _rel(pc.A_solve(X), pd.A_solve(X)) < 1e-10
    assert _rel(pc.solve_state(m, X), pd.solve_state(m, X)) < 1e-10
    g_d, J_d, _, _ = pd.gradient(m)
    g_c, J_c, _, _ = pc.gradient(m)
    assert _rel(g_c, g_d) < 1e-9 and abs(J_c - J_d) <= 1e-10 * abs(J_d)
    assert _rel(pc.hessian_misfit(m, u_c, X), pd.hessian_misfit(m, u_d, X)) < 1e-9


def test_cg_problem_linear_state_is_exact():
    """m = 0: u = x_last exactly (P1 reproduces the linear solution), through the CG path."""
    mesh = Mesh(3, 12)
    prob = Problem(mesh, 0.05, 0.5, np.zeros((0, 3)), np.zeros(0), 1.0, solver="cg")
    u = prob.forward(np.zeros(mesh.n))
    assert np.abs(u - mesh.coords[:, -1]).max() < 1e-11


def test_cg_problem_manufactured_solution_second_order():
    """-div(e^m grad u) = f in the cube with u* = sin(pi x) sin(pi y) sin(pi z), m = a x y z,
    all-Dirichlet, solved by the CG path: L2 nodal error ratio about 4 per halving."""
    a = 0.7
    errs = []
    for N in (6, 12, 24):
        mesh = Mesh(3, N)
        x, y, z = mesh.coords.T
        m = a * x * y * z
        s = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        gx = np.pi * np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        gy = np.pi * np.sin(np.pi * x) * np.cos(np.pi * y) * np.sin(np.pi * z)
        gz = np.pi * np.sin(np.pi * x) * np.sin(np.pi * y) * np.cos(np.pi * z)
        f = -np.exp(m) * (a * y * z * gx + a * x * z * gy + a * x * y * gz - 3 * np.pi ** 2 * s)
        bnd = np.zeros(mesh.n, dtype=bool)
        for c in (x, y, z):
            bnd |= (c < 1e-12) | (c > 1 - 1e-12)
        prob = Problem(mesh, 0.1, 0.5, np.zeros((0, 3)), np.zeros(0), 1.0, f=f,
                       dirichlet_mask=bnd, dirichlet_values=np.zeros(mesh.n), solver="cg")
        e = prob.forward(m) - s
        errs.append(np.sqrt(e @ (mesh.mass @ e)))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.4 < r < 4.6 for r in ratios), ratios


def test_auto_solver_choice():
    assert Problem(Mesh(2, 8), 0.1, 0.5, np.zeros((0, 2)), np.zeros(0), 1.0).solver == "direct"
    assert Problem(Mesh(3, 6), 0.1, 0.5, np.zeros((0, 3)), np.zeros(0), 1.0).solver == "direct"
    assert CG_RTOL <= 1e-13
