"""Structured P1 finite elements on the unit square / cube (oracle; test infrastructure).

Discretisation (Section 2.3: continuous Lagrange P1 basis; Section 5.1: unit
domain, Dirichlet on the bottom/top faces, zero Neumann elsewhere):

* nodes (N+1)^d, lexicographic with the first axis fastest, spacing h = 1/N;
* 2D: each cell split along its (0,0)-(1,1) diagonal into two right triangles;
* 3D: each cell split into the six Kuhn tetrahedra, one per axis permutation,
  all sharing the cell's (0,0,0)-(1,1,1) diagonal.

Element matrices are computed generically from vertex coordinates (barycentric
gradients), never from a stencil formula, and summed into CSR matrices
(the assembly sum over elements of G_e^T A_e G_e, Appendix C).
"""
from __future__ import annotations

import itertools
from functools import cached_property

import numpy as np
import scipy.sparse as sp


class Mesh:
    def __init__(self, dim: int, N: int):
        assert dim in (2, 3) and N >= 1
        self.dim, self.N = dim, N
        self.h = 1.0 / N
        self.nper = N + 1
        self.n = self.nper ** dim

    # ---- nodes -----------------------------------------------------------
    def node(self, *ijk):
        idx = 0
        stride = 1
        for a in ijk:
            idx = idx + a * stride
            stride *= self.nper
        return idx

    @cached_property
    def coords(self) -> np.ndarray:
        g = np.arange(self.nper) * self.h
        if self.dim == 2:
            y, x = np.meshgrid(g, g, indexing="ij")
            return np.stack([x.ravel(), y.ravel()], axis=1)
        z, y, x = np.meshgrid(g, g, g, indexing="ij")
        return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)

    # ---- elements --------------------------------------------------------
    @cached_property
    def local_offsets(self) -> list:
        """Vertex offsets (in cells) of the elements of one cell, in local order."""
        if self.dim == 2:
            return [[(0, 0), (1, 0), (1, 1)],      # lower triangle (below the diagonal)
                    [(0, 0), (0, 1), (1, 1)]]      # upper triangle
        out = []
        for perm in itertools.permutations(range(3)):
            v = [0, 0, 0]
            verts = [tuple(v)]
            for a in perm:
                v[a] += 1
                verts.append(tuple(v))
            out.append(verts)
        return out

    @cached_property
    def elements(self) -> np.ndarray:
        """(nelems, d+1) vertex indices; cell-major, cells lexicographic."""
        N, d = self.N, self.dim
        cell = np.arange(N ** d, dtype=np.int64)
        c = [(cell // N ** a) % N for a in range(d)]          # first axis fastest
        offs = self.local_offsets
        out = np.empty((N ** d, len(offs), d + 1), dtype=np.int64)
        for loc, verts in enumerate(offs):
            for v, o in enumerate(verts):
                out[:, loc, v] = sum((c[a] + o[a]) * self.nper ** a for a in range(d))
        return out.reshape(-1, d + 1)

    @property
    def nelems(self) -> int:
        return self.elements.shape[0]

    @cached_property
    def geometry(self):
        """Per element: volume |e| and barycentric gradients (nelems, d+1, d)."""
        X = self.coords[self.elements]                 # (ne, d+1, d)
        T = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))   # columns X_a - X_0
        det = np.linalg.det(T)
        vol = np.abs(det) / (1.0 if self.dim == 1 else (2.0 if self.dim == 2 else 6.0))
        Tinv = np.linalg.inv(T)                        # rows: grad lambda_a, a = 1..d
        G = np.empty((X.shape[0], self.dim + 1, self.dim))
        G[:, 1:, :] = Tinv
        G[:, 0, :] = -Tinv.sum(axis=1)
        return vol, G

    # ---- element matrices and assembly -----------------------------------
    def local_stiffness(self) -> np.ndarray:
        """Unit-coefficient element stiffness |e| G G^T, shape (ne, d+1, d+1)."""
        vol, G = self.geometry
        return vol[:, None, None] * np.einsum("eak,ebk->eab", G, G)

    def local_stiffness_tensor(self, Theta) -> np.ndarray:
        """Element stiffness of -div(Theta grad): |e| G Theta G^T, shape (ne, d+1, d+1)."""
        vol, G = self.geometry
        Th = np.asarray(Theta, dtype=float).reshape(self.dim, self.dim)
        return vol[:, None, None] * np.einsum("eak,kl,ebl->eab", G, Th, G)

    def stiffness_tensor(self, Theta) -> sp.csr_matrix:
        return self.assemble(self.local_stiffness_tensor(Theta))

    @cached_property
    def boundary_mass(self) -> sp.csr_matrix:
        """P1 mass matrix of the boundary: sum over the element facets that lie on a face of
        the unit square / cube of |f| (1 + delta_ab) / (d (d + 1)) (the facets are segments
        in 2D and triangles in 3D)."""
        el, X = self.elements, self.coords
        d = self.dim
        rows, cols, vals = [], [], []
        base = (np.ones((d, d)) + np.eye(d)) / (d * (d + 1))
        for drop in range(d + 1):
            fv = np.delete(el, drop, axis=1)                     # (ne, d) facet vertices
            P = X[fv]                                            # (ne, d, d)
            on = np.zeros(len(fv), dtype=bool)
            for a in range(d):
                for side in (0.0, 1.0):
                    on |= np.all(np.abs(P[:, :, a] - side) < 1e-12, axis=1)
            if not on.any():
                continue
            Pf = P[on]
            if d == 2:
                meas = np.linalg.norm(Pf[:, 1] - Pf[:, 0], axis=1)
            else:
                meas = 0.5 * np.linalg.norm(np.cross(Pf[:, 1] - Pf[:, 0], Pf[:, 2] - Pf[:, 0]), axis=1)
            f = fv[on]
            rows.append(np.repeat(f, d, axis=1).ravel())
            cols.append(np.tile(f, (1, d)).ravel())
            vals.append((meas[:, None, None] * base[None]).ravel())
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n, self.n)).tocsr()

    def local_mass(self) -> np.ndarray:
        """Consistent element mass |e| (1 + delta_ab) / ((d+1)(d+2))."""
        vol, _ = self.geometry
        d = self.dim
        base = (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
        return vol[:, None, None] * base[None]

    def assemble(self, local: np.ndarray, weight: np.ndarray | None = None) -> sp.csr_matrix:
        """Sum_e weight_e * G_e^T local_e G_e as CSR."""
        el = self.elements
        vals = local if weight is None else local * weight[:, None, None]
        rows = np.repeat(el, el.shape[1], axis=1).ravel()
        cols = np.tile(el, (1, el.shape[1])).ravel()
        return sp.coo_matrix((vals.ravel(), (rows, cols)), shape=(self.n, self.n)).tocsr()

    def stiffness(self, kappa_e: np.ndarray) -> sp.csr_matrix:
        return self.assemble(self.local_stiffness(), kappa_e)

    @cached_property
    def mass(self) -> sp.csr_matrix:
        return self.assemble(self.local_mass())

    def elem_mean(self, nodal: np.ndarray) -> np.ndarray:
        """Element average of a nodal field: the exact element integral of its P1
        interpolant divided by |e|.  Works on (n,) or (n, s)."""
        return nodal[self.elements].mean(axis=1)

    # ---- boundary ---------------------------------------------------------
    @cached_property
    def dirichlet_mask(self) -> np.ndarray:
        """Nodes on the bottom (last coordinate 0) and top (last coordinate 1) faces."""
        last = self.coords[:, -1]
        return (np.abs(last) < 1e-12) | (np.abs(last - 1.0) < 1e-12)

    @cached_property
    def top_mask(self) -> np.ndarray:
        return np.abs(self.coords[:, -1] - 1.0) < 1e-12

    # ---- observation operator --------------------------------------------
    def locate(self, x: np.ndarray):
        """Element containing point x and its barycentric coordinates.

        The cell is floor(x/h) clamped to the mesh; within the cell the first
        element (local order) whose barycentric coordinates are all >= -1e-12
        is taken."""
        N, h = self.N, self.h
        c = np.minimum(np.floor(x / h).astype(int), N - 1)
        c = np.maximum(c, 0)
        ncell_elems = len(self.local_offsets)
        cell_lin = 0
        stride = 1
        for a in range(self.dim):
            cell_lin += c[a] * stride
            stride *= N
        vol, G = self.geometry
        for loc in range(ncell_elems):
            e = cell_lin * ncell_elems + loc
            X0 = self.coords[self.elements[e, 0]]
            lam_rest = G[e, 1:, :] @ (x - X0)
            lam = np.concatenate([[1.0 - lam_rest.sum()], lam_rest])
            if np.all(lam >= -1e-12):
                return e, lam
        raise ValueError("point outside mesh")

    def observation_operator(self, pts: np.ndarray) -> sp.csr_matrix:
        """B: (q, n) P1 interpolation at the points (sum of point evaluations)."""
        rows, cols, vals = [], [], []
        for i, x in enumerate(pts):
            e, lam = self.locate(np.asarray(x, dtype=float))
            for a, v in enumerate(self.elements[e]):
                rows.append(i)
                cols.append(v)
                vals.append(lam[a])
        return sp.coo_matrix((vals, (rows, cols)), shape=(len(pts), self.n)).tocsr()

    # ---- rectangular factor of the mass matrix (Appendix C) ---------------
    @cached_property
    def quadrature(self):
        """Per-element degree-2 rule: barycentric points (nq, d+1) and weights / |e|."""
        if self.dim == 2:
            pts = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
            wts = np.full(3, 1.0 / 3.0)
        else:
            a = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
            b = (5.0 - np.sqrt(5.0)) / 20.0
            pts = np.array([[a, b, b, b], [b, a, b, b], [b, b, a, b], [b, b, b, a]])
            wts = np.full(4, 0.25)
        return pts, wts

    def mass_factor_apply(self, eta: np.ndarray) -> np.ndarray:
        """w = C_M eta with C_M C_M^T = M (Appendix C): per element e and quadrature
        point q, sqrt(w_q |e|) * phi_a(x_q) * eta_{e,q} is added to node a.
        eta: (nelems*(d+1),) or (nelems*(d+1), s), element-major."""
        pts, wts = self.quadrature
        vol, _ = self.geometry
        ne, nq = self.nelems, len(wts)
        eta2 = eta.reshape(ne, nq, -1)
        scale = np.sqrt(wts[None, :] * vol[:, None])          # (ne, nq)
        contrib = np.einsum("qa,eq,eqs->eas", pts, scale, eta2)  # (ne, d+1, s)
        out = np.zeros((self.n, eta2.shape[2]))
        np.add.at(out, self.elements, contrib)
        return out if eta.ndim == 2 else out[:, 0]

    def mass_factor_dense(self) -> np.ndarray:
        """C_M as a dense (n, nelems*(d+1)) matrix (tiny meshes only)."""
        I = np.eye(self.nelems * (self.dim + 1))
        return self.mass_factor_apply(I)


def rotated_theta(theta1: float, theta2: float, alpha: float) -> np.ndarray:
    """2D anisotropy tensor with eigenvalues theta1, theta2 and the theta1-axis at angle alpha
    from the x axis: R(alpha) diag(theta1, theta2) R(alpha)^T (the s.p.d. reading of the
    printed tensor of Section 5.1.1)."""
    c, s = np.cos(alpha), np.sin(alpha)
    Rm = np.array([[c, -s], [s, c]])
    return Rm @ np.diag([theta1, theta2]) @ Rm.T

