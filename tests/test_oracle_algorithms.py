"""Pins for oracle/algorithms.py: Newton-CG against an independent optimiser,
randomized eigensolvers against the dense generalized eigendecomposition, and the
exact covariance of the linear sampling maps (Section 4.3)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as so

import workloads as W
from oracle import algorithms as A
from oracle.fem import Mesh
from oracle.inverse import Problem, make_problem


def _problem(dim, N, nobs, seed=0, noise=0.01):
    w = W.make_workload(dim, N, nobs, seed=seed)
    prob, m_true, _ = make_problem(w, W.draws(w))
    return prob, w


def _dense(apply, n):
    return apply(np.eye(n))


def test_newton_matches_independent_optimizer():
    prob, _ = _problem(2, 6, 12, seed=11)
    res = A.newton_cg(prob, rel_tol=1e-10)
    assert res.converged
    assert all(b <= a + 1e-12 for a, b in zip(res.costs, res.costs[1:]))   # monotone
    f = lambda m: prob.cost(m)[0]
    gfun = lambda m: prob.gradient(m)[0]
    ref = so.minimize(f, np.zeros(prob.n), jac=gfun, method="L-BFGS-B",
                      options=dict(gtol=1e-12, ftol=1e-15, maxiter=5000))
    assert np.linalg.norm(res.m - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    assert f(res.m) <= f(ref.x) + 1e-9


def test_full_newton_reaches_the_same_map_in_fewer_iterations():
    """Newton-CG with the full Hessian minimises the same cost: same MAP as the
    Gauss-Newton run, and no more Newton iterations."""
    prob, _ = _problem(2, 6, 12, seed=11)
    gn = A.newton_cg(prob, rel_tol=1e-10)
    fn = A.newton_cg(prob, rel_tol=1e-10, full=True)
    assert gn.converged and fn.converged
    assert np.linalg.norm(fn.m - gn.m) <= 1e-7 * np.linalg.norm(gn.m)
    assert fn.iterations <= gn.iterations


def test_cg_steihaug_solves_spd_system():
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((20, 20))
    H = Q @ Q.T + 20 * np.eye(20)
    P = np.diag(1 / np.diag(H))
    b = rng.standard_normal(20)
    x, it, why = A.cg_steihaug(lambda v: H @ v, lambda v: P @ v, b, 1e-12, max_iter=100)
    assert why == "converged"
    assert np.allclose(H @ x, b, atol=1e-9)
    # negative curvature at the first iteration returns the preconditioned steepest descent
    x, it, why = A.cg_steihaug(lambda v: -v, lambda v: v, b, 1e-8)
    assert why == "negative_curvature" and it == 1 and np.allclose(x, b)


@pytest.mark.parametrize("dim,N,q", [(2, 5, 6), (3, 2, 5)])
def test_double_pass_equals_dense_generalized_eig(dim, N, q):
    """With k + p = n the randomized basis spans R^n, so Algorithm 2 reproduces the
    dense generalized eigenvalues H v = lambda R v exactly; V^T R V = I."""
    prob, _ = _problem(dim, N, q, seed=12)
    m = 0.3 * np.sin(np.arange(prob.n))
    u = prob.forward(m)
    n = prob.n
    H = _dense(lambda X: prob.hessian_misfit(m, u, X), n)
    R = _dense(prob.R_apply, n)
    lam_ref = sla.eigh(0.5 * (H + H.T), 0.5 * (R + R.T), eigvals_only=True)[::-1]
    Om = W.random_block(n, n, 5)
    lam, V = A.lowrank_eig(prob, m, Om, k=n)
    scale = lam_ref[0]
    assert np.allclose(lam, lam_ref, atol=1e-9 * scale)
    assert np.allclose(V.T @ R @ V, np.eye(n), atol=1e-8)
    # residual of the generalized eigenproblem for the non-trivial pairs
    nz = lam > 1e-6 * scale
    res = H @ V[:, nz] - (R @ V[:, nz]) * lam[nz]
    assert np.abs(res).max() <= 1e-8 * scale


def test_double_and_single_pass_exact_when_rank_below_sample_size():
    """rank(H_misfit) <= q < k + p: the range is captured exactly, so both Algorithm 2
    and Algorithm 3 return the non-zero eigenvalues of the dense problem."""
    prob, _ = _problem(2, 8, 6, seed=13)
    m = np.zeros(prob.n)
    u = prob.forward(m)
    n = prob.n
    H = _dense(lambda X: prob.hessian_misfit(m, u, X), n)
    R = _dense(prob.R_apply, n)
    lam_ref = sla.eigh(0.5 * (H + H.T), R, eigvals_only=True)[::-1][:6]
    Om = W.random_block(n, 12, 7)
    lam2, V2 = A.lowrank_eig(prob, m, Om, k=6)
    lam1, V1 = A.lowrank_eig(prob, m, Om, k=6, single=True)
    assert np.allclose(lam2, lam_ref, rtol=1e-8)
    assert np.allclose(lam1, lam_ref, rtol=1e-6)
    # the eigenvectors agree up to sign (distinct eigenvalues)
    for a in range(6):
        c = abs(V1[:, a] @ R @ V2[:, a])
        assert abs(c - 1) < 1e-5


def test_pre_chol_qr_b_orthonormal():
    rng = np.random.default_rng(3)
    n, s = 30, 8
    G = rng.standard_normal((n, n))
    B = G @ G.T + n * np.eye(n)
    Y = rng.standard_normal((n, s))
    Q, Qb, Rf = A.pre_chol_qr(Y, lambda X: B @ X)
    assert np.allclose(Q.T @ B @ Q, np.eye(s), atol=1e-12)
    assert np.allclose(Q @ Rf, Y, atol=1e-12)
    assert np.allclose(Qb, B @ Q, atol=1e-10)
    assert np.allclose(np.triu(Rf), Rf)


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 1)])
def test_sampling_maps_have_exact_covariances(dim, N):
    """Prior map eta -> A^{-1} C_M eta has covariance R^{-1} (eq. (sample_prior)); the
    posterior map has covariance R^{-1} - V D V^T (eq. (sample_post)), which with all
    eigenpairs retained equals (H_misfit + R)^{-1} (Woodbury, eq. (sm))."""
    prob, _ = _problem(dim, N, 3, seed=14)
    n = prob.n
    m = 0.2 * np.cos(np.arange(n))
    u = prob.forward(m)
    H = _dense(lambda X: prob.hessian_misfit(m, u, X), n)
    H = 0.5 * (H + H.T)
    R = _dense(prob.R_apply, n)
    R = 0.5 * (R + R.T)
    lam, V = sla.eigh(H, R)
    lam, V = lam[::-1], V[:, ::-1]
    ne = prob.mesh.nelems * (dim + 1)
    prior, post = A.laplace_samples(prob, np.zeros(n), lam, V, np.eye(ne))
    Rinv = np.linalg.inv(R)
    assert np.allclose(prior @ prior.T, Rinv, atol=1e-10 * np.abs(Rinv).max())
    Hinv = np.linalg.inv(H + R)
    assert np.allclose(post @ post.T, Hinv, atol=1e-9 * np.abs(Hinv).max())
    D = lam / (1 + lam)
    assert np.allclose(post @ post.T, Rinv - (V * D) @ V.T, atol=1e-9 * np.abs(Hinv).max())


def test_pointwise_variances():
    prob, _ = _problem(2, 6, 4, seed=15)
    n = prob.n
    Rinv = np.linalg.inv(_dense(prob.R_apply, n))
    nodes = np.array([0, 7, 20, n - 1])
    assert np.allclose(A.prior_variance_exact(prob, nodes), np.diag(Rinv)[nodes], rtol=1e-10)
    # randomized prior variance with rbar = n is exact
    Om = W.random_block(n, n, 4)
    pv = A.prior_variance_randomized(prob, Om, n)
    assert np.allclose(pv, np.diag(Rinv), rtol=1e-8)
    # stochastic estimator is unbiased: with many probes it approaches the diagonal
    Z = np.sign(W.random_block(n, 4000, 9))
    est = A.stochastic_diag_estimator(prob, Z)
    assert np.median(np.abs(est / np.diag(Rinv) - 1)) < 0.15


def test_small2d_workload_pipeline_qualitative():
    """Paper-level qualitative facts (Section 5.1.3): the spectrum decays rapidly and the
    numerical rank stays below the number of observations."""
    w = W.WORKLOADS["small2d"]
    prob, m_true, _ = make_problem(w, W.draws(w))
    res = A.newton_cg(prob)
    assert res.converged and res.iterations < 20
    lam, V = A.lowrank_eig(prob, res.m, W.omega(w), w.k)
    assert lam[0] / lam[-1] > 100
    assert np.all(np.diff(lam) <= 0)
