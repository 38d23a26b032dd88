"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on the
same seeded inputs.  Tolerances (relative, per output):
  operators (K, A, M, C, C^T, C_M, B)          1e-12   (FP64 kernels, rounding order only)
  forward state, state / prior / mass solves    1e-8    (solves run at rtol 1e-11)
  gradient                                      1e-8
  Hessian action                                1e-7    (both PDE solves at rtol 1e-11)
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.inverse import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(2, 32, 20), (2, 48, 15), (3, 8, 12), (2, 7, 5)]


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _colrel(A, B):
    A, B = np.asarray(A), np.asarray(B)
    return max(np.linalg.norm(A[:, j] - B[:, j]) / max(np.linalg.norm(B[:, j]), 1e-300) for j in range(B.shape[1]))


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"d{c[0]}N{c[1]}q{c[2]}")
def case(request):
    from paper_1909_03948_gb300 import Problem
    dim, N, q = request.param
    w = W.make_workload(dim, N, q, seed=W.SEED_BASE + 300 + N)
    dr = W.draws(w)
    orc, m_true, u_true = make_problem(w, dr)
    P = Problem(dim, N, w.gamma, w.delta, orc.sigma, dr.obs_xyz, d_obs=orc.d_obs, rtol=1e-11,
                precision="fp32_ir")
    m = 0.7 * m_true
    dev = torch.device("cuda", 0)
    P.set_point(torch.tensor(m, device=dev))
    yield dict(P=P, orc=orc, m=m, w=w, dev=dev, u_ref=orc.forward(m))
    P.close()


def T(x, dev):
    """numpy (n, s) column block -> torch (s, n)."""
    x = np.asarray(x)
    return torch.tensor(np.ascontiguousarray(x.T if x.ndim == 2 else x), device=dev)


def N_(t):
    a = t.cpu().numpy()
    return a.T if a.ndim == 2 else a


def _dirichlet_K(orc, m):
    K = orc.stiffness(m).tolil()
    d = np.flatnonzero(orc.dmask)
    K[d, :] = 0
    K[:, d] = 0
    K[d, d] = 1.0
    return K.tocsr()


def test_stiffness_apply(case):
    P, orc, m, dev = case["P"], case["orc"], case["m"], case["dev"]
    X = W.random_block(orc.n, 5, 1)
    Y = N_(P.stiffness_apply(T(X, dev)))
    assert _colrel(Y, _dirichlet_K(orc, m) @ X) < 1e-12


def test_prior_and_mass_apply(case):
    P, orc, dev = case["P"], case["orc"], case["dev"]
    X = W.random_block(orc.n, 3, 2)
    assert _colrel(N_(P.prior_apply(T(X, dev))), orc.A @ X) < 1e-12
    assert _colrel(N_(P.mass_apply(T(X, dev))), orc.M @ X) < 1e-12


def test_C_and_Ct(case):
    P, orc, m, dev, u = case["P"], case["orc"], case["m"], case["dev"], case["u_ref"]
    X = W.random_block(orc.n, 4, 3)
    assert _colrel(N_(P.C_apply(T(X, dev))), orc.C_apply(m, u, X)) < 1e-9
    Wm = W.random_block(orc.n, 4, 4)
    Wm[orc.dmask] = 0.0
    assert _colrel(N_(P.Ct_apply(T(Wm, dev))), orc.Ct_apply(m, u, Wm)) < 1e-9


def test_mass_factor(case):
    P, orc, dev = case["P"], case["orc"], case["dev"]
    eta = W.random_block(orc.mesh.nelems * (orc.mesh.dim + 1), 3, 5)
    assert _colrel(N_(P.mass_factor_apply(T(eta, dev))), orc.mesh.mass_factor_apply(eta)) < 1e-12


def test_observation(case):
    P, orc, dev, u = case["P"], case["orc"], case["dev"], case["u_ref"]
    y = P.observe(torch.tensor(u, device=dev)).cpu().numpy()
    assert _rel(y, orc.B @ u) < 1e-13


@pytest.mark.parametrize("precision", ["fp32_ir", "fp64"])
def test_forward(case, precision):
    P, orc, m, dev = case["P"], case["orc"], case["m"], case["dev"]
    P.set_precision(precision)
    try:
        u, st = P.forward(torch.tensor(m, device=dev))
        assert _rel(u.cpu().numpy(), case["u_ref"]) < 1e-8
        assert st["rel_res"] < 1e-10 or st["outer"] >= 0
    finally:
        P.set_precision("fp32_ir")
        P.set_point(torch.tensor(m, device=dev))


@pytest.mark.parametrize("s", [1, 3, 17])
def test_state_solve_ragged_blocks(case, s):
    P, orc, m, dev = case["P"], case["orc"], case["m"], case["dev"]
    B = W.random_block(orc.n, s, 10 + s)
    X, st = P.state_solve(T(B, dev))
    ref = orc.solve_state(m, B)
    assert _colrel(N_(X).reshape(orc.n, s), ref) < 1e-8
    assert st["rel_res"] <= 1e-11


def test_prior_and_mass_solve(case):
    P, orc, dev = case["P"], case["orc"], case["dev"]
    B = W.random_block(orc.n, 4, 21)
    X, _ = P.prior_solve(T(B, dev))
    assert _colrel(N_(X), orc.A_solve(B)) < 1e-8
    Xm, _ = P.mass_solve(T(B, dev))
    assert _colrel(N_(Xm), orc.M_solve(B)) < 1e-8


def test_R_and_Rinv(case):
    P, orc, dev = case["P"], case["orc"], case["dev"]
    X = W.random_block(orc.n, 2, 22)
    assert _colrel(N_(P.R_apply(T(X, dev))), orc.R_apply(X)) < 1e-8
    assert _colrel(N_(P.Rinv_apply(T(X, dev))), orc.Rinv_apply(X)) < 1e-8


def test_gradient(case):
    P, orc, m, dev = case["P"], case["orc"], case["m"], case["dev"]
    g, J = P.gradient(torch.tensor(m, device=dev))
    g_ref, J_ref, _, _ = orc.gradient(m)
    assert _rel(g.cpu().numpy(), g_ref) < 1e-8
    assert abs(J[0] - J_ref) <= 1e-9 * abs(J_ref)


@pytest.mark.parametrize("s", [1, 5])
@pytest.mark.parametrize("precision", ["fp32_ir", "fp64"])
def test_hessian_block(case, s, precision):
    P, orc, m, dev = case["P"], case["orc"], case["m"], case["dev"]
    P.set_precision(precision)
    try:
        P.set_point(torch.tensor(m, device=dev))
        X = W.random_block(orc.n, s, 30 + s)
        Y, st = P.hessian_apply(T(X, dev))
        ref = orc.hessian_misfit(m, case["u_ref"], X)
        assert _colrel(N_(Y).reshape(orc.n, s), ref) < 1e-7
        Yp, _ = P.hessian_apply(T(X, dev), with_prior=True)
        assert _colrel(N_(Yp).reshape(orc.n, s), ref + orc.R_apply(X)) < 1e-7
    finally:
        P.set_precision("fp32_ir")
        P.set_point(torch.tensor(m, device=dev))


@pytest.mark.parametrize("s", [1, 5])
@pytest.mark.parametrize("precision", ["fp32_ir", "fp64"])
def test_full_hessian_block(case, s, precision):
    """Full Hessian (the adjoint terms of eqs. incrementals1-3) at a point with a nonzero
    data residual, against the oracle, to the same 1e-7 as the Gauss-Newton action."""
    P, orc, m, dev = case["P"], case["orc"], case["m"], case["dev"]
    P.set_precision(precision)
    try:
        P.set_point(torch.tensor(m, device=dev))
        u = case["u_ref"]
        p = orc.adjoint(m, u)
        X = W.random_block(orc.n, s, 50 + s)
        Y, _ = P.hessian_apply(T(X, dev), full=True)
        ref = orc.hessian_full_misfit(m, u, p, X)
        assert _colrel(N_(Y).reshape(orc.n, s), ref) < 1e-7
        Yp, _ = P.hessian_apply(T(X, dev), with_prior=True, full=True)
        assert _colrel(N_(Yp).reshape(orc.n, s), ref + orc.R_apply(X)) < 1e-7
    finally:
        P.set_precision("fp32_ir")
        P.set_point(torch.tensor(m, device=dev))


def test_full_hessian_follows_new_data(case):
    """The adjoint behind the full Hessian is recomputed after hp_set_data."""
    P, orc, m, dev = case["P"], case["orc"], case["m"], case["dev"]
    X = W.random_block(orc.n, 2, 61)
    P.hessian_apply(T(X, dev), full=True)
    d_old = orc.d_obs.copy()
    d_new = d_old + 3.0 * orc.sigma * np.random.default_rng(62).standard_normal(d_old.shape)
    try:
        orc.d_obs = d_new
        P.set_data(d_new, orc.sigma)
        u = case["u_ref"]
        Y, _ = P.hessian_apply(T(X, dev), full=True)
        assert _colrel(N_(Y).reshape(orc.n, 2), orc.hessian_full_misfit(m, u, orc.adjoint(m, u), X)) < 1e-7
    finally:
        orc.d_obs = d_old
        P.set_data(d_old, orc.sigma)


def test_hessian_block_equals_single_columns(case):
    """A block of s actions equals s one-column actions (to solver tolerance)."""
    P, orc, dev = case["P"], case["orc"], case["dev"]
    X = W.random_block(orc.n, 4, 40)
    Yb, _ = P.hessian_apply(T(X, dev))
    cols = [N_(P.hessian_apply(T(X[:, j], dev))[0]) for j in range(4)]
    assert _colrel(N_(Yb), np.stack(cols, axis=1)) < 1e-8


def test_zero_columns_and_empty_block(case):
    P, orc, dev = case["P"], case["orc"], case["dev"]
    X = np.zeros((orc.n, 2))
    X[:, 1] = W.random_block(orc.n, 1, 41)[:, 0]
    Y, _ = P.hessian_apply(T(X, dev))
    Yn = N_(Y)
    assert np.all(Yn[:, 0] == 0.0)
    assert np.linalg.norm(Yn[:, 1]) > 0
    empty = torch.zeros((0, orc.n), dtype=torch.float64, device=dev)
    Y0, _ = P.hessian_apply(empty)
    assert Y0.shape == (0, orc.n)


# ---- prior variants (Section 5.1.1): anisotropic Theta and the Robin condition --------
ANISO = [(2, 32, 0.0), (2, 32, 0.7), (2, 24, 1.3), (3, 8, 0.5)]


@pytest.mark.parametrize("dim,N,beta", ANISO, ids=lambda v: str(v))
def test_anisotropic_robin_prior(dim, N, beta):
    """A = gamma K(Theta) + delta M + gamma beta M_boundary against the oracle's assembled
    matrices: apply 1e-12, multigrid solves A^-1 and R^-1 1e-8, prior samples from
    identical normals 1e-8."""
    from oracle.fem import Mesh, rotated_theta
    from oracle.inverse import Problem as OProblem
    from paper_1909_03948_gb300 import Problem
    if dim == 2:
        Th = rotated_theta(2.0, 0.5, 0.6)
    else:
        L = np.random.default_rng(9).standard_normal((3, 3))
        Th = L @ L.T + 0.5 * np.eye(3)
    w = W.make_workload(dim, N, 5, seed=W.SEED_BASE + 700 + N)
    dr = W.draws(w)
    orc = OProblem(Mesh(dim, N), w.gamma, w.delta, dr.obs_xyz, np.zeros(5), 0.01, theta=Th, robin_beta=beta)
    P = Problem(dim, N, w.gamma, w.delta, 0.01, dr.obs_xyz, rtol=1e-11, theta=Th, robin_beta=beta)
    dev = torch.device("cuda", 0)
    X = W.random_block(orc.n, 3, 71)
    assert _colrel(N_(P.prior_apply(T(X, dev))), orc.A @ X) < 1e-12
    Y, _ = P.prior_solve(T(X, dev))
    assert _colrel(N_(Y), orc.A_solve(X)) < 1e-8
    assert _colrel(N_(P.Rinv_apply(T(X, dev))), orc.Rinv_apply(X)) < 1e-8
    eta = W.random_block(orc.mesh.nelems * (dim + 1), 2, 72)
    prior, _, _ = P.laplace_sample(None, None, None, T(eta, dev), want_prior=True, want_post=False)
    assert _colrel(N_(prior), orc.prior_sample(eta)) < 1e-8
    P.close()


def test_invalid_prior_tensor_is_rejected():
    from paper_1909_03948_gb300 import Problem, HPError
    with pytest.raises(HPError):
        Problem(2, 8, 0.1, 0.5, 0.01, np.array([[0.5, 0.5]]), theta=np.array([[1.0, 2.0], [2.0, 1.0]]))
    with pytest.raises(HPError):
        Problem(2, 8, 0.1, 0.5, 0.01, np.array([[0.5, 0.5]]), robin_beta=-1.0)
