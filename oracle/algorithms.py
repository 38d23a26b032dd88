"""Newton-CG, randomized generalized eigensolvers, Laplace sampling (oracle; test infrastructure).

All quantities FP64.  Readings of the paper where it is silent:

* Newton-CG (Algorithm 1): the Newton system is solved by CG preconditioned
  with R^{-1} (Section 4.1: preconditioning with the inverse regularization
  operator); the norm of g is the preconditioned norm sqrt(g^T R^{-1} g);
  eta_i = min(0.5, sqrt(|g_i| / |g_0|)); at least one CG iteration;
  Armijo constant 1e-4 (Section 4.1 gives [1e-5, 1e-4]); step halving with at
  most 10 backtracks; at most 50 Newton iterations; Steihaug exit on
  non-positive curvature (with the preconditioned steepest-descent direction
  if it happens at the first CG iteration).
* Newton-CG uses the Gauss-Newton Hessian by default; full=True uses the
  Hessian with the adjoint terms (Appendix A), which may be indefinite away
  from the MAP point -- the Steihaug exit handles that.
* Double pass (Algorithm 2) with PreCholQR (Algorithm 4), A = H_misfit,
  B = R; the eigenvector sign is normalised so that the entry of largest
  magnitude is positive.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------------------
# Algorithm 1: inexact Newton-CG
# ---------------------------------------------------------------------------
@dataclass
class NewtonResult:
    m: np.ndarray
    converged: bool
    iterations: int
    cg_iterations: list = field(default_factory=list)
    costs: list = field(default_factory=list)
    gnorms: list = field(default_factory=list)
    alphas: list = field(default_factory=list)


def cg_steihaug(apply_H, apply_P, b, rtol, max_iter=200, min_iter=1):
    """Preconditioned CG for H x = b from x = 0.  Stops when
    sqrt(r^T P r) <= rtol * sqrt(b^T P b) (after at least min_iter iterations)
    or on non-positive curvature (Steihaug).  Returns (x, iterations, reason)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_P(r)
    rz = float(r @ z)
    r0 = np.sqrt(rz)
    if r0 == 0.0:
        return x, 0, "zero_rhs"
    d = z.copy()
    for it in range(1, max_iter + 1):
        Hd = apply_H(d)
        dHd = float(d @ Hd)
        if dHd <= 0.0:
            if it == 1:
                x = z.copy()        # preconditioned steepest descent direction
            return x, it, "negative_curvature"
        alpha = rz / dHd
        x += alpha * d
        r -= alpha * Hd
        z = apply_P(r)
        rz_new = float(r @ z)
        if it >= min_iter and np.sqrt(max(rz_new, 0.0)) <= rtol * r0:
            return x, it, "converged"
        beta = rz_new / rz
        d = z + beta * d
        rz = rz_new
    return x, max_iter, "max_iter"


def newton_cg(prob, m0=None, rel_tol=1e-6, abs_tol=0.0, max_iter=50, max_backtrack=10,
              c_armijo=1e-4, cg_max_iter=200, full=False):
    m = prob.m_prior.copy() if m0 is None else np.array(m0, dtype=float)
    u = prob.forward(m)
    J = prob.cost(m, u)[0]
    res = NewtonResult(m=m, converged=False, iterations=0, costs=[J])
    g0norm = None
    for it in range(max_iter):
        p = prob.adjoint(m, u)
        g = prob.R_apply(m - prob.m_prior) + prob.Ct_apply(m, u, p)
        gnorm = np.sqrt(max(float(g @ prob.Rinv_apply(g)), 0.0))
        if g0norm is None:
            g0norm = gnorm
        res.gnorms.append(gnorm)
        if gnorm <= max(rel_tol * g0norm, abs_tol):
            res.converged = True
            break
        eta = min(0.5, np.sqrt(gnorm / g0norm))
        if full:
            H = lambda v, m=m, u=u, p=p: prob.hessian_full(m, u, p, v)
        else:
            H = lambda v, m=m, u=u: prob.hessian(m, u, v)
        mhat, ncg, _ = cg_steihaug(H, prob.Rinv_apply, -g, eta, max_iter=cg_max_iter)
        res.cg_iterations.append(ncg)
        gdm = float(g @ mhat)
        alpha = 1.0
        accepted = False
        for _ in range(max_backtrack):
            m_try = m + alpha * mhat
            u_try = prob.forward(m_try)
            J_try = prob.cost(m_try, u_try)[0]
            if J_try < J + alpha * c_armijo * gdm:
                m, u, J = m_try, u_try, J_try
                accepted = True
                break
            alpha *= 0.5
        res.alphas.append(alpha if accepted else 0.0)
        res.costs.append(J)
        res.iterations = it + 1
        if not accepted:
            break
    res.m = m
    return res


# ---------------------------------------------------------------------------
# Algorithm 4: PreCholQR;  Algorithms 2 and 3: randomized generalized eig
# ---------------------------------------------------------------------------
def pre_chol_qr(Y, apply_B):
    """[Z, R_Y] = qr(Y); Zb = B Z; R_Z = chol(Z^T Zb) (upper, R_Z^T R_Z = Z^T Zb);
    Q = Z R_Z^{-1}, Qb = Zb R_Z^{-1}, R = R_Z R_Y."""
    Z, RY = np.linalg.qr(Y)
    Zb = apply_B(Z)
    G = Z.T @ Zb
    G = 0.5 * (G + G.T)
    RZ = np.linalg.cholesky(G).T
    Q = np.linalg.solve(RZ.T, Z.T).T          # Z R_Z^{-1}
    Qb = np.linalg.solve(RZ.T, Zb.T).T
    return Q, Qb, RZ @ RY


def _normalise_signs(V):
    idx = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[idx, np.arange(V.shape[1])])
    sgn[sgn == 0] = 1.0
    return V * sgn


def double_pass(apply_A, apply_B, apply_Binv, Omega, k):
    """Algorithm 2.  Returns (lambda[:k] descending, V[:, :k], Q)."""
    Ybar = apply_A(Omega)
    Y = apply_Binv(Ybar)
    Q, _, _ = pre_chol_qr(Y, apply_B)
    AQ = apply_A(Q)
    T = Q.T @ AQ
    T = 0.5 * (T + T.T)
    lam, S = np.linalg.eigh(T)
    order = np.argsort(lam)[::-1]
    lam, S = lam[order], S[:, order]
    V = Q @ S[:, :k]
    return lam[:k], _normalise_signs(V), Q


def single_pass(apply_A, apply_B, apply_Binv, Omega, k):
    """Algorithm 3, eq. (Tsinglepass): T = argmin_X |X (Qb^T Omega) - Qb^T Y|_F over symmetric X
    (least squares over the upper-triangular unknowns), Y = B^{-1} A Omega."""
    Ybar = apply_A(Omega)
    Y = apply_Binv(Ybar)
    Q, Qb, _ = pre_chol_qr(Y, apply_B)
    W = Qb.T @ Omega                  # (s, s)
    Z = Qb.T @ Y                      # (s, s)
    s = W.shape[0]
    iu = np.triu_indices(s)
    # vec(X W) is linear in the symmetric unknowns: build the (s*s, s(s+1)/2) design matrix
    cols = []
    for a, b in zip(*iu):
        E = np.zeros((s, s))
        E[a, b] = 1.0
        E[b, a] = 1.0
        cols.append((E @ W).ravel())
    D = np.stack(cols, axis=1)
    t, *_ = np.linalg.lstsq(D, Z.ravel(), rcond=None)
    T = np.zeros((s, s))
    T[iu] = t
    T = T + T.T - np.diag(np.diag(T))
    lam, S = np.linalg.eigh(T)
    order = np.argsort(lam)[::-1]
    lam, S = lam[order], S[:, order]
    V = Q @ S[:, :k]
    return lam[:k], _normalise_signs(V), Q


def lowrank_eig(prob, m_map, Omega, k, single=False):
    u = prob.forward(m_map)
    A = lambda X: prob.hessian_misfit(m_map, u, X)
    f = single_pass if single else double_pass
    lam, V, _ = f(A, prob.R_apply, prob.Rinv_apply, Omega, k)
    return lam, V


# ---------------------------------------------------------------------------
# Sampling (Section 4.3, eqs. (sample_prior), (sample_post)) and pointwise
# variance (Section 4.4, eqs. (stoc_diag_estimator), (prior_mvar), (post_mvar))
# ---------------------------------------------------------------------------
def laplace_samples(prob, m_map, lam, V, eta):
    """eta: (nelems*(d+1), N) normals.  Prior sample x = A^{-1} C_M eta (covariance R^{-1});
    posterior sample y = m_map + x - V S V^T R x with S = I - (Lambda + I)^{-1/2}.
    Returns (prior_samples = m_pr + x, posterior_samples)."""
    w = prob.mesh.mass_factor_apply(eta)
    x = prob.A_solve(w)
    Rx = prob.A @ prob.M_solve(w)
    S = 1.0 - 1.0 / np.sqrt(lam + 1.0)
    y = x - V @ (S[:, None] * (V.T @ Rx))
    return prob.m_prior[:, None] + x, m_map[:, None] + y


def prior_variance_exact(prob, nodes):
    """diag(R^{-1}) at the given nodes: e_i^T A^{-1} M A^{-1} e_i."""
    E = np.zeros((prob.n, len(nodes)))
    E[nodes, np.arange(len(nodes))] = 1.0
    Z = prob.A_solve(E)
    return np.einsum("ij,ij->j", Z, prob.M @ Z)


def posterior_variance_lowrank(prob, lam, V, nodes):
    """diag(R^{-1}) - sum_i lam_i/(1+lam_i) v_i (.) v_i at the given nodes (eq. (post_mvar))."""
    D = lam / (1.0 + lam)
    return prior_variance_exact(prob, nodes) - (V[nodes] ** 2) @ D


def prior_variance_randomized(prob, Omega, rbar):
    """Eq. (prior_mvar): diag(R^{-1}) ~ sum mu_i vbar_i^2 with (mu, vbar) from Algorithm 2
    with l = 0, A = R^{-1}, B = I."""
    I = lambda X: X
    mu, Vb, _ = double_pass(prob.Rinv_apply, I, I, Omega[:, :rbar], rbar)
    return (Vb ** 2) @ mu


def stochastic_diag_estimator(prob, Z):
    """Eq. (stoc_diag_estimator): diag(R^{-1}) ~ [sum z_j (.) w_j] / [sum z_j (.) z_j], R w_j = z_j."""
    W = prob.Rinv_apply(Z)
    return (Z * W).sum(axis=1) / (Z * Z).sum(axis=1)
