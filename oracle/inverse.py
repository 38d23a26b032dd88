"""Log-coefficient Poisson inverse problem, FP64 (oracle; test infrastructure).

Forward problem (Section 5.1, eqs. (poi) and (poisson_weak)):  -div(e^m grad u) = f, u = 1 on the
top face, u = 0 on the bottom face, zero Neumann elsewhere (Section 5.1.3).  Discrete reading: the element coefficient is the element
mean of the nodal field E = e^m, kappa_e = (1/(d+1)) sum_{v in e} E_v, i.e. the
exact integral of the P1 interpolant of e^m; this makes the discrete map
exactly differentiable, with d kappa_e / d m_v = E_v / (d+1).

Prior (Section 5.1.1, eq. (PoissonPrior); Section 2.3): C = A^{-2}, A = gamma*K(Theta) + delta*M
+ gamma*beta*M_boundary: the weak form of -gamma div(Theta grad m) + delta m with the Robin
condition Theta grad m . n + beta m = 0.  Defaults Theta = I, beta = 0 (zero Neumann);
discrete precision R = A M^{-1} A.

Misfit (Section 5.1.1): B = P1 interpolation at q points, Gamma_noise = sigma^2 I.

Cost  J(m) = 1/2 |B u - d|^2 / sigma^2 + 1/2 (m - m_pr)^T R (m - m_pr)     (Section 5.1.2, eq. (cost-elliptic))
Adjoint (Appendix A, eq. (firstadj)):   K p = -B^T (B u - d) / sigma^2 on the zero-Dirichlet space
Gradient (Appendix A, eq. (firstcontrol)):        g = R (m - m_pr) + C^T p
Gauss-Newton Hessian action (Appendix A, eqs. (incrementals1)-(incrementals3)
with the p-dependent terms dropped; Gauss-Newton per the footnote of Section 2.2):
    K uhat = -C mhat,  K phat = -B^T B uhat / sigma^2,  H_misfit mhat = C^T phat
where (C mhat)_i = (K(kappa_hat) u)_i with kappa_hat_e = mean_{v in e}(E_v mhat_v), and
(C^T w)_v = E_v/(d+1) * sum_{e ni v} |e| grad(u)_e . grad(w)_e.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import Mesh
from .pcg import jacobi_pcg

# Meshes with more nodes than this in 3D are solved by Jacobi-preconditioned CG to
# relative residual CG_RTOL instead of a sparse direct factorisation, which does not
# finish in minutes on 3D meshes of that size.
CG_NODES_3D = 20_000
CG_RTOL = 1e-13


class Problem:
    def __init__(self, mesh: Mesh, gamma: float, delta: float, obs_xyz: np.ndarray,
                 d_obs: np.ndarray | None, sigma: float, m_prior: np.ndarray | None = None,
                 f: np.ndarray | None = None, u_top: float = 1.0, u_bottom: float = 0.0,
                 dirichlet_mask: np.ndarray | None = None, dirichlet_values: np.ndarray | None = None,
                 theta=None, robin_beta: float = 0.0, solver: str = "auto"):
        """solver: "direct" (scipy SuperLU, exact to rounding), "cg" (Jacobi-preconditioned
        CG to relative residual CG_RTOL in the true residual), or "auto" (cg for 3D meshes
        above CG_NODES_3D nodes, else direct)."""
        if solver == "auto":
            solver = "cg" if (mesh.dim == 3 and mesh.n > CG_NODES_3D) else "direct"
        assert solver in ("direct", "cg")
        self.solver = solver
        self.mesh = mesh
        self.n = mesh.n
        self.gamma, self.delta, self.sigma = float(gamma), float(delta), float(sigma)
        self.obs_xyz = np.asarray(obs_xyz, dtype=float)
        self.B = mesh.observation_operator(self.obs_xyz) if len(self.obs_xyz) else sp.csr_matrix((0, mesh.n))
        self.d_obs = None if d_obs is None else np.asarray(d_obs, dtype=float)
        self.m_prior = np.zeros(self.n) if m_prior is None else np.asarray(m_prior, dtype=float)
        self.f = np.zeros(self.n) if f is None else np.asarray(f, dtype=float)
        if dirichlet_mask is None:
            dirichlet_mask = mesh.dirichlet_mask
            dirichlet_values = np.where(mesh.top_mask, u_top, u_bottom)
        self.dmask = np.asarray(dirichlet_mask, dtype=bool)
        self.gD = np.where(self.dmask, dirichlet_values, 0.0)
        self.free = np.flatnonzero(~self.dmask)
        # prior operator A = gamma K(Theta) + delta M + gamma beta M_boundary (all nodes)
        self.theta = np.eye(mesh.dim) if theta is None else np.asarray(theta, dtype=float)
        self.robin_beta = float(robin_beta)
        self.K1 = mesh.stiffness_tensor(self.theta)
        self.M = mesh.mass
        A = self.gamma * self.K1 + self.delta * self.M
        if self.robin_beta != 0.0:
            A = A + self.gamma * self.robin_beta * mesh.boundary_mass
        if solver == "direct":
            self.A = A.tocsc()
            self._A_lu = spla.splu(self.A)
            self._M_lu = spla.splu(self.M.tocsc())
        else:
            self.A = A.tocsr()
        self._cache_key = None

    # ---- state operator ----------------------------------------------------
    def coefficient(self, m: np.ndarray) -> np.ndarray:
        return self.mesh.elem_mean(np.exp(m))

    def stiffness(self, m: np.ndarray) -> sp.csr_matrix:
        return self.mesh.stiffness(self.coefficient(m))

    def _factor(self, m: np.ndarray):
        key = m.tobytes()
        if key != self._cache_key:
            K = self.stiffness(m)
            self._K = K
            if self.solver == "direct":
                Kff = K[self.free][:, self.free].tocsc()
                self._Kff_lu = spla.splu(Kff)
            else:
                Kff = K[self.free][:, self.free].tocsr()
                Kff.eliminate_zeros()       # the exactly-zero off-axis couplings (same operator)
                self._Kff_lu = _CGSolve(Kff)
            self._cache_key = key
        return self._K, self._Kff_lu

    def solve_state(self, m: np.ndarray, rhs: np.ndarray) -> np.ndarray:
        """Solve K(m) x = rhs on the zero-Dirichlet space; Dirichlet rows of rhs are ignored
        and Dirichlet entries of x are zero.  rhs: (n,) or (n, s)."""
        _, lu = self._factor(m)
        x = np.zeros_like(rhs, dtype=float)
        x[self.free] = lu.solve(np.ascontiguousarray(rhs[self.free]))
        return x

    def forward(self, m: np.ndarray) -> np.ndarray:
        K, lu = self._factor(m)
        load = self.M @ self.f - K @ self.gD
        u = self.gD.copy()
        u[self.free] = lu.solve(load[self.free])
        return u

    def observe(self, u: np.ndarray) -> np.ndarray:
        return self.B @ u

    # ---- prior -------------------------------------------------------------
    def A_solve(self, b: np.ndarray) -> np.ndarray:
        if self.solver == "cg":
            return jacobi_pcg(self.A, b, CG_RTOL)
        return self._A_lu.solve(np.ascontiguousarray(b))

    def M_solve(self, b: np.ndarray) -> np.ndarray:
        if self.solver == "cg":
            return jacobi_pcg(self.M, b, CG_RTOL)
        return self._M_lu.solve(np.ascontiguousarray(b))

    def R_apply(self, x: np.ndarray) -> np.ndarray:
        """R x = A M^{-1} A x."""
        return self.A @ self.M_solve(self.A @ x)

    def Rinv_apply(self, x: np.ndarray) -> np.ndarray:
        """R^{-1} x = A^{-1} M A^{-1} x."""
        return self.A_solve(self.M @ self.A_solve(x))

    def prior_sample(self, eta: np.ndarray) -> np.ndarray:
        """x = A^{-1} C_M eta, so that R x = C eta with C = A M^{-1} C_M, C C^T = R
        (Section 4.3.1, eq. (sample_prior), with the rectangular factor of Appendix C); returns m_pr + x."""
        x = self.A_solve(self.mesh.mass_factor_apply(eta))
        return (self.m_prior if x.ndim == 1 else self.m_prior[:, None]) + x

    # ---- cost, gradient ------------------------------------------------------
    def cost(self, m: np.ndarray, u: np.ndarray | None = None):
        if u is None:
            u = self.forward(m)
        r = self.observe(u) - self.d_obs
        misfit = 0.5 * float(r @ r) / self.sigma ** 2
        dm = m - self.m_prior
        reg = 0.5 * float(dm @ self.R_apply(dm))
        return misfit + reg, misfit, reg

    def adjoint(self, m: np.ndarray, u: np.ndarray) -> np.ndarray:
        rhs = -(self.B.T @ (self.observe(u) - self.d_obs)) / self.sigma ** 2
        return self.solve_state(m, rhs)

    def C_apply(self, m: np.ndarray, u: np.ndarray, mhat: np.ndarray) -> np.ndarray:
        """(C mhat) = K(kappa_hat) u with kappa_hat_e = mean_{v in e} E_v mhat_v (all rows)."""
        E = np.exp(m)
        kh = self.mesh.elem_mean(E[:, None] * (mhat if mhat.ndim == 2 else mhat[:, None]))
        Kl = self.mesh.local_stiffness()
        el = self.mesh.elements
        ue = u[el]                                            # (ne, d+1)
        le = np.einsum("eab,eb->ea", Kl, ue)                  # unit-coefficient local K_e u_e
        out = np.zeros((self.n, kh.shape[1]))
        np.add.at(out, el, le[:, :, None] * kh[:, None, :])
        return out if mhat.ndim == 2 else out[:, 0]

    def Ct_apply(self, m: np.ndarray, u: np.ndarray, w: np.ndarray) -> np.ndarray:
        """(C^T w)_v = E_v/(d+1) * sum_{e ni v} |e| grad u_e . grad w_e."""
        E = np.exp(m)
        vol, G = self.mesh.geometry
        el = self.mesh.elements
        w2 = w if w.ndim == 2 else w[:, None]
        gu = np.einsum("eak,ea->ek", G, u[el])                # (ne, d)
        gw = np.einsum("eak,eas->eks", G, w2[el])             # (ne, d, s)
        ce = vol[:, None] * np.einsum("ek,eks->es", gu, gw)   # (ne, s)
        acc = np.zeros((self.n, w2.shape[1]))
        for a in range(el.shape[1]):
            np.add.at(acc, el[:, a], ce)
        out = E[:, None] * acc / (self.mesh.dim + 1)
        return out if w.ndim == 2 else out[:, 0]

    def gradient(self, m: np.ndarray):
        """Returns (g, J, u, p)."""
        u = self.forward(m)
        p = self.adjoint(m, u)
        g = self.R_apply(m - self.m_prior) + self.Ct_apply(m, u, p)
        J = self.cost(m, u)[0]
        return g, J, u, p

    # ---- Gauss-Newton Hessian action ---------------------------------------
    def hessian_misfit(self, m: np.ndarray, u: np.ndarray, X: np.ndarray) -> np.ndarray:
        """H_misfit X for a block X (n, s) or a vector (n,)."""
        uhat = self.solve_state(m, -self.C_apply(m, u, X))
        rhs = -(self.B.T @ (self.B @ uhat)) / self.sigma ** 2
        phat = self.solve_state(m, rhs)
        return self.Ct_apply(m, u, phat)

    def hessian(self, m: np.ndarray, u: np.ndarray, X: np.ndarray) -> np.ndarray:
        return self.hessian_misfit(m, u, X) + self.R_apply(X)

    # ---- full Newton Hessian action (Appendix A with the adjoint terms) -------
    def hessian_full_misfit(self, m: np.ndarray, u: np.ndarray, p: np.ndarray, X: np.ndarray) -> np.ndarray:
        """Misfit part of the Hessian action with every term of eqs. incrementals1-3:

            K uhat = -C(u) X                               (incrementals1)
            K phat = -B^T B uhat / sigma^2 - C(p) X         (incrementals2)
            H X    = C(u)^T phat + C(p)^T uhat + X (.) C(u)^T p   (incrementals3)

        C(w) X = K(kappa_hat) w is the derivative of K(m) w in direction X; the last term
        is the second derivative of p^T K(m) u, diagonal because each element coefficient
        is linear in e^m."""
        uhat = self.solve_state(m, -self.C_apply(m, u, X))
        rhs = -(self.B.T @ (self.B @ uhat)) / self.sigma ** 2 - self.C_apply(m, p, X)
        phat = self.solve_state(m, rhs)
        wmm = self.Ct_apply(m, u, p)
        diag = wmm[:, None] * X if X.ndim == 2 else wmm * X
        return self.Ct_apply(m, u, phat) + self.Ct_apply(m, p, uhat) + diag

    def hessian_full(self, m: np.ndarray, u: np.ndarray, p: np.ndarray, X: np.ndarray) -> np.ndarray:
        return self.hessian_full_misfit(m, u, p, X) + self.R_apply(X)

    def parameter_to_observable(self, m: np.ndarray) -> np.ndarray:
        return self.observe(self.forward(m))


class _CGSolve:
    """The .solve interface of a factorisation, by Jacobi-preconditioned CG on K_ff."""

    def __init__(self, K):
        self.K = K

    def solve(self, b):
        return jacobi_pcg(self.K, np.asarray(b), CG_RTOL)


def make_problem(w, draws, dtype=float, solver: str = "auto"):
    """Build the oracle problem for a workload: m_true = prior draw from the
    workload's normals, d = B u(m_true) + sigma * xi with sigma = level * max|u|."""
    mesh = Mesh(w.dim, w.N)
    prob = Problem(mesh, w.gamma, w.delta, draws.obs_xyz, None, 1.0, solver=solver)
    m_true = prob.prior_sample(draws.eta_true.reshape(-1))
    u_true = prob.forward(m_true)
    sigma = w.noise_level * float(np.max(np.abs(u_true)))
    d = prob.observe(u_true) + sigma * draws.xi_noise
    prob.sigma = sigma
    prob.d_obs = d
    return prob, m_true, u_true
