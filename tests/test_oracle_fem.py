"""Pins for oracle/fem.py: closed-form element matrices, an independent stencil
derivation, exact integration identities and the rectangular mass factor."""
import numpy as np
import pytest

from oracle.fem import Mesh


def test_2d_element_matrices_closed_form():
    # Right triangle with legs h: unit-coefficient stiffness is (1/2) * path Laplacian of
    # the two legs (hypotenuse coupling zero), independent of h; mass is |e|/12 (1 + delta).
    for N in (1, 3, 7):
        mesh = Mesh(2, N)
        h = 1.0 / N
        K = mesh.local_stiffness()
        M = mesh.local_mass()
        Kref = 0.5 * np.array([[1, -1, 0], [-1, 2, -1], [0, -1, 1]], dtype=float)
        Mref = (h * h / 2) / 12 * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]], dtype=float)
        assert np.allclose(K, Kref[None], atol=1e-14)
        assert np.allclose(M, Mref[None], atol=1e-16)
        vol, _ = mesh.geometry
        assert np.isclose(vol.sum(), 1.0, atol=1e-14)


def test_3d_kuhn_element_matrices_closed_form():
    # Kuhn tetrahedron with path vertices 0, e_a, e_a+e_b, 1: barycentric gradients are
    # -e_a, e_a-e_b, e_b-e_c, e_c (over h); |e| = h^3/6 -> K_e = (h/6) * path Laplacian.
    N = 2
    mesh = Mesh(3, N)
    h = 1.0 / N
    Kref = (h / 6) * np.array([[1, -1, 0, 0], [-1, 2, -1, 0], [0, -1, 2, -1], [0, 0, -1, 1]], dtype=float)
    assert np.allclose(mesh.local_stiffness(), Kref[None], atol=1e-14)
    vol, _ = mesh.geometry
    assert np.allclose(vol, h ** 3 / 6)
    assert np.isclose(vol.sum(), 1.0)
    Mref = (h ** 3 / 6) / 20 * (np.ones((4, 4)) + np.eye(4))
    assert np.allclose(mesh.local_mass(), Mref[None])


def _tri_index(N, i, j, lower):
    return 2 * (i + N * j) + (0 if lower else 1)


def test_2d_stiffness_equals_independent_edge_formula():
    """K(kappa) off-diagonals: horizontal edge (i,j)-(i+1,j) couples through the lower
    triangle of cell (i,j) and the upper triangle of cell (i,j-1), vertical edge
    (i,j)-(i,j+1) through the upper triangle of cell (i,j) and the lower triangle of
    cell (i-1,j); each contributes -kappa/2.  Diagonal couplings vanish; rows sum to 0."""
    N = 5
    mesh = Mesh(2, N)
    rng = np.random.default_rng(0)
    kap = rng.uniform(0.2, 3.0, mesh.nelems)
    K = mesh.stiffness(kap).toarray()
    nd = lambda i, j: i + (N + 1) * j
    Kref = np.zeros_like(K)
    for j in range(N + 1):
        for i in range(N + 1):
            if i < N:
                w = 0.0
                if j < N:
                    w += kap[_tri_index(N, i, j, True)]
                if j > 0:
                    w += kap[_tri_index(N, i, j - 1, False)]
                Kref[nd(i, j), nd(i + 1, j)] = Kref[nd(i + 1, j), nd(i, j)] = -0.5 * w
            if j < N:
                w = 0.0
                if i < N:
                    w += kap[_tri_index(N, i, j, False)]
                if i > 0:
                    w += kap[_tri_index(N, i - 1, j, True)]
                Kref[nd(i, j), nd(i, j + 1)] = Kref[nd(i, j + 1), nd(i, j)] = -0.5 * w
    np.fill_diagonal(Kref, -Kref.sum(axis=1))
    assert np.allclose(K, Kref, atol=1e-13)


def test_3d_laplacian_is_seven_point():
    """P1 on the Kuhn triangulation reproduces the 7-point Laplacian scaled by h
    (interior rows: 6h on the diagonal, -h on the six axis neighbours, 0 elsewhere);
    for any element coefficient only axis couplings are non-zero."""
    N = 4
    mesh = Mesh(3, N)
    h = 1.0 / N
    K = mesh.stiffness(np.ones(mesh.nelems)).toarray()
    nd = lambda i, j, k: i + (N + 1) * (j + (N + 1) * k)
    c = nd(2, 2, 2)
    row = np.zeros(mesh.n)
    row[c] = 6 * h
    for o in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        row[nd(2 + o[0], 2 + o[1], 2 + o[2])] = -h
        row[nd(2 - o[0], 2 - o[1], 2 - o[2])] = -h
    assert np.allclose(K[c], row, atol=1e-14)
    rng = np.random.default_rng(1)
    Kk = mesh.stiffness(rng.uniform(0.1, 5, mesh.nelems)).toarray()
    X = mesh.coords
    d = np.abs(X[:, None, :] - X[None, :, :]) > 1e-12
    offaxis = d.sum(axis=2) >= 2
    assert np.abs(Kk[offaxis]).max() < 1e-14
    assert np.allclose(Kk.sum(axis=1), 0, atol=1e-13)


@pytest.mark.parametrize("dim,N", [(2, 1), (2, 3), (3, 1), (3, 2)])
def test_mass_factor_reproduces_mass(dim, N):
    """C_M C_M^T = M exactly (Appendix C, eq. (rect_decomp))."""
    mesh = Mesh(dim, N)
    C = mesh.mass_factor_dense()
    assert np.allclose(C @ C.T, mesh.mass.toarray(), atol=1e-15, rtol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_integrates_polynomials(dim):
    """1^T M 1 = |D| = 1 and 1^T M x = integral of x_a = 1/2, x^T M x = 1/3 (exact for P1 data)."""
    mesh = Mesh(dim, 3)
    M = mesh.mass
    one = np.ones(mesh.n)
    assert np.isclose(one @ M @ one, 1.0, atol=1e-14)
    for a in range(dim):
        x = mesh.coords[:, a]
        assert np.isclose(one @ M @ x, 0.5, atol=1e-14)
    # integral of x^2 with x the P1 interpolant of x (exact since x is linear): 1/3
    x = mesh.coords[:, 0]
    assert np.isclose(x @ M @ x, 1.0 / 3.0, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_observation_reproduces_linear_functions(dim):
    mesh = Mesh(dim, 4)
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, (40, dim))
    pts[:4] = 0.5      # on element boundaries
    pts[4] = 1.0
    pts[5] = 0.0
    B = mesh.observation_operator(pts)
    coef = rng.standard_normal(dim + 1)
    f = coef[0] + mesh.coords @ coef[1:]
    assert np.allclose(B @ f, coef[0] + pts @ coef[1:], atol=1e-13)
    assert np.allclose(np.asarray(B.sum(axis=1)).ravel(), 1.0)
    assert (B.data >= -1e-12).all()


# ---- anisotropic stiffness and boundary mass (prior variants, Section 5.1.1) ----------
@pytest.mark.parametrize("dim,N", [(2, 5), (3, 3)])
def test_tensor_stiffness_reduces_to_unit_and_integrates_linear_energy(dim, N):
    mesh = Mesh(dim, N)
    assert abs(mesh.stiffness_tensor(np.eye(dim)) - mesh.stiffness(np.ones(mesh.nelems))).max() < 1e-15
    rng = np.random.default_rng(dim)
    L = rng.standard_normal((dim, dim))
    Th = L @ L.T + 0.1 * np.eye(dim)                       # any s.p.d. tensor
    K = mesh.stiffness_tensor(Th)
    assert abs(K - K.T).max() < 1e-14
    assert np.abs(K @ np.ones(mesh.n)).max() < 1e-13      # constants in the kernel
    a = rng.standard_normal(dim)
    x = mesh.coords @ a                                   # linear field: energy a^T Theta a |D|
    assert np.isclose(x @ (K @ x), a @ Th @ a, rtol=1e-12)


@pytest.mark.parametrize("dim,N,area,x2", [(2, 4, 4.0, 5.0 / 3.0), (3, 3, 6.0, 7.0 / 3.0)])
def test_boundary_mass_closed_forms(dim, N, area, x2):
    """1^T Mb 1 = |boundary|; x^T Mb x = integral of x^2 over the boundary (P1 exact for
    products of linear functions): 2D 0 + 1 + 1/3 + 1/3, 3D 0 + 1 + 4/3."""
    mesh = Mesh(dim, N)
    Mb = mesh.boundary_mass
    one = np.ones(mesh.n)
    assert np.isclose(one @ (Mb @ one), area, rtol=1e-13)
    x = mesh.coords[:, 0]
    assert np.isclose(x @ (Mb @ x), x2, rtol=1e-13)
    interior = np.all((mesh.coords > 1e-12) & (mesh.coords < 1 - 1e-12), axis=1)
    assert abs(Mb[interior]).max() == 0.0


def test_rotated_theta_is_spd_with_given_eigenpairs():
    from oracle.fem import rotated_theta
    Th = rotated_theta(2.0, 0.5, 0.3)
    ev, V = np.linalg.eigh(Th)
    assert np.allclose(ev, [0.5, 2.0])
    assert np.isclose(abs(V[:, 1] @ np.array([np.cos(0.3), np.sin(0.3)])), 1.0)
