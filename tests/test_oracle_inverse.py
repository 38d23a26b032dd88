"""Pins for oracle/inverse.py: exact solutions, O(h^2) convergence, finite-difference
derivative checks, symmetry of the Gauss-Newton Hessian, and the full Hessian (with
the adjoint terms) against finite differences of the gradient at a nonzero residual."""
import numpy as np
import pytest

import workloads as W
from oracle.fem import Mesh
from oracle.inverse import Problem, make_problem


def _problem(dim, N, nobs, seed=0, sigma=0.01, gamma=0.1, delta=0.5):
    mesh = Mesh(dim, N)
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.05, 0.95, (nobs, dim))
    d = rng.uniform(0, 1, nobs)
    return Problem(mesh, gamma, delta, pts, d, sigma)


def _smooth_m(mesh, scale=1.0):
    X = mesh.coords
    return scale * (0.6 * np.sin(2 * X[:, 0] + 0.3) * np.cos(1.5 * X[:, -1]) - 0.2 * X[:, 0])


@pytest.mark.parametrize("dim,N", [(2, 8), (3, 4)])
def test_m_zero_gives_linear_state(dim, N):
    """m = 0, f = 0, u = 0 / 1 on bottom / top, zero Neumann: exact solution u = x_last,
    reproduced exactly by P1 (textbook special case)."""
    prob = _problem(dim, N, 3)
    u = prob.forward(np.zeros(prob.n))
    assert np.allclose(u, prob.mesh.coords[:, -1], atol=1e-13)


def test_maximum_principle():
    prob = _problem(2, 16, 3)
    u = prob.forward(2.0 * _smooth_m(prob.mesh))
    assert u.min() >= -1e-12 and u.max() <= 1 + 1e-12


def test_manufactured_solution_second_order():
    """-div(e^m grad u) = f with u* = sin(pi x) sin(pi y), m = a x y, all-Dirichlet:
    discrete L2 nodal error ratio ~ 4 per halving (O(h^2))."""
    a = 0.8
    errs = []
    for N in (8, 16, 32, 64):
        mesh = Mesh(2, N)
        x, y = mesh.coords[:, 0], mesh.coords[:, 1]
        m = a * x * y
        us = np.sin(np.pi * x) * np.sin(np.pi * y)
        dm_dx, dm_dy = a * y, a * x
        ux = np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)
        uy = np.pi * np.sin(np.pi * x) * np.cos(np.pi * y)
        lap = -2 * np.pi ** 2 * us
        f = -np.exp(m) * (dm_dx * ux + dm_dy * uy + lap)
        bnd = (x < 1e-12) | (x > 1 - 1e-12) | (y < 1e-12) | (y > 1 - 1e-12)
        prob = Problem(mesh, 0.1, 0.5, np.zeros((0, 2)), np.zeros(0), 1.0, f=f,
                       dirichlet_mask=bnd, dirichlet_values=np.zeros(mesh.n))
        u = prob.forward(m)
        e = u - us
        errs.append(np.sqrt(e @ (mesh.mass @ e)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 4.0) < 0.4), ratios


def test_C_is_derivative_of_K_u():
    """C v = d/de [K(m + e v) u] at e = 0 (central difference)."""
    prob = _problem(2, 6, 4)
    m = _smooth_m(prob.mesh)
    u = prob.forward(m)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(prob.n)
    eps = 1e-5
    fd = (prob.stiffness(m + eps * v) @ u - prob.stiffness(m - eps * v) @ u) / (2 * eps)
    assert np.allclose(prob.C_apply(m, u, v), fd, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("dim,N", [(2, 5), (3, 2)])
def test_Ct_is_transpose_of_C(dim, N):
    prob = _problem(dim, N, 4)
    m = _smooth_m(prob.mesh)
    u = prob.forward(m)
    rng = np.random.default_rng(6)
    V = rng.standard_normal((prob.n, 3))
    Wm = rng.standard_normal((prob.n, 3))
    lhs = Wm.T @ prob.C_apply(m, u, V)
    rhs = (V.T @ prob.Ct_apply(m, u, Wm)).T
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim,N", [(2, 8), (3, 3)])
def test_gradient_matches_finite_differences(dim, N):
    prob = _problem(dim, N, 10, seed=2)
    m = _smooth_m(prob.mesh, 0.7)
    g, J, _, _ = prob.gradient(m)
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = rng.standard_normal(prob.n)
        eps = 1e-5
        fd = (prob.cost(m + eps * v)[0] - prob.cost(m - eps * v)[0]) / (2 * eps)
        assert abs(fd - g @ v) <= 1e-6 * max(abs(fd), 1e-8), (fd, g @ v)


@pytest.mark.parametrize("dim,N", [(2, 6), (3, 2)])
def test_gn_hessian_equals_JtJ_by_finite_differences(dim, N):
    """w^T H_misfit v = (J w)^T Gamma^{-1} (J v) with J = dF/dm by central differences."""
    prob = _problem(dim, N, 8, seed=3)
    m = _smooth_m(prob.mesh)
    u = prob.forward(m)
    rng = np.random.default_rng(8)
    v, w = rng.standard_normal(prob.n), rng.standard_normal(prob.n)
    eps = 1e-5
    F = prob.parameter_to_observable
    Jv = (F(m + eps * v) - F(m - eps * v)) / (2 * eps)
    Jw = (F(m + eps * w) - F(m - eps * w)) / (2 * eps)
    ref = Jw @ Jv / prob.sigma ** 2
    got = w @ prob.hessian_misfit(m, u, v)
    assert abs(got - ref) <= 1e-6 * abs(ref)


def test_gn_hessian_is_full_hessian_at_zero_residual():
    """With d = F(m) exactly the adjoint vanishes, so the Gauss-Newton Hessian equals the
    true Hessian: finite differences of the gradient reproduce H v."""
    prob = _problem(2, 6, 8, seed=4)
    m = _smooth_m(prob.mesh)
    prob.d_obs = prob.parameter_to_observable(m)
    u = prob.forward(m)
    rng = np.random.default_rng(9)
    v = rng.standard_normal(prob.n)
    eps = 1e-5
    fd = (prob.gradient(m + eps * v)[0] - prob.gradient(m - eps * v)[0]) / (2 * eps)
    Hv = prob.hessian(m, u, v)
    assert np.linalg.norm(fd - Hv) <= 1e-6 * np.linalg.norm(Hv)


@pytest.mark.parametrize("dim,N", [(2, 6), (3, 2)])
def test_full_hessian_is_the_derivative_of_the_gradient(dim, N):
    """At a nonzero data residual (the adjoint p is not 0) the full Hessian action of
    eqs. incrementals1-3 equals central differences of the gradient, while the
    Gauss-Newton Hessian does not."""
    prob = _problem(dim, N, 8, seed=11)
    m = _smooth_m(prob.mesh)
    g, _, u, p = prob.gradient(m)
    assert np.linalg.norm(p) > 1e-3 * np.linalg.norm(u)
    rng = np.random.default_rng(12)
    for _ in range(2):
        v = rng.standard_normal(prob.n)
        eps = 1e-5
        fd = (prob.gradient(m + eps * v)[0] - prob.gradient(m - eps * v)[0]) / (2 * eps)
        Hv = prob.hessian_full(m, u, p, v)
        assert np.linalg.norm(fd - Hv) <= 1e-6 * np.linalg.norm(Hv)
        gn = prob.hessian(m, u, v)
        assert np.linalg.norm(fd - gn) > 1e-3 * np.linalg.norm(Hv)
    # blocks act column by column
    V = rng.standard_normal((prob.n, 3))
    HV = prob.hessian_full(m, u, p, V)
    assert np.allclose(HV[:, 1], prob.hessian_full(m, u, p, V[:, 1]), rtol=1e-12, atol=1e-12)


def test_full_hessian_is_symmetric():
    prob = _problem(2, 5, 6, seed=13)
    m = _smooth_m(prob.mesh)
    _, _, u, p = prob.gradient(m)
    H = prob.hessian_full_misfit(m, u, p, np.eye(prob.n))
    assert np.abs(H - H.T).max() <= 1e-10 * np.abs(H).max()


def test_hessian_symmetry_and_rank():
    prob = _problem(2, 6, 5, seed=5)
    m = _smooth_m(prob.mesh)
    u = prob.forward(m)
    H = prob.hessian_misfit(m, u, np.eye(prob.n))
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert ev.min() > -1e-10 * ev.max()
    assert np.sum(ev > 1e-9 * ev.max()) <= 5          # rank <= q


def test_R_is_spd_and_matches_definition():
    prob = _problem(2, 4, 2)
    A = prob.A.toarray()
    M = prob.M.toarray()
    R = A @ np.linalg.solve(M, A)
    X = np.eye(prob.n)
    assert np.allclose(prob.R_apply(X), R, rtol=1e-11, atol=1e-11)
    assert np.allclose(prob.Rinv_apply(X), np.linalg.inv(R), rtol=1e-9, atol=1e-11)
    assert np.linalg.eigvalsh(R).min() > 0


def test_workload_problem_builds():
    w = W.WORKLOADS["small2d"]
    prob, m_true, u_true = make_problem(w, W.draws(w))
    assert prob.B.shape == (50, 33 * 33)
    assert np.isclose(prob.sigma, 0.01 * np.abs(u_true).max())


@pytest.mark.parametrize("dim,N", [(2, 9), (3, 4)])
def test_prior_precision_on_constants(dim, N):
    """R = A M^{-1} A with A = gamma K(Theta) + delta M and zero Neumann: K(Theta) 1 = 0, so
    A 1 = delta M 1, M^{-1} A 1 = delta 1 and R 1 = delta^2 M 1; with 1^T M 1 = |D| = 1,
    1^T R 1 = delta^2.  Holds for any s.p.d. Theta, so a random one is used."""
    mesh = Mesh(dim, N)
    rng = np.random.default_rng(11)
    G = rng.standard_normal((dim, dim))
    theta = G @ G.T + dim * np.eye(dim)
    prob = Problem(mesh, 0.13, 0.7, np.zeros((0, dim)), np.zeros(0), 1.0, theta=theta)
    one = np.ones(mesh.n)
    R1 = prob.R_apply(one)
    assert np.abs(R1 - 0.7 ** 2 * (mesh.mass @ one)).max() <= 1e-9 * np.abs(mesh.mass @ one).max()
    assert abs(one @ R1 - 0.7 ** 2) <= 1e-11
