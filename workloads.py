"""Seeded synthetic workloads for the log-coefficient Poisson inverse problem.

This module only draws random numbers and fixes problem sizes; it holds none
of the method's arithmetic.  Both the CPU oracle (``oracle/``) and the CUDA
path (``paper_1909_03948_gb300``) take their inputs from here, so that a
parity test feeds identical draws to both sides.

Workloads (Section 5.1 of the paper sets the shape: a unit-square/cube
domain, a bilaplacian Gaussian prior, pointwise observations with 1 % noise):

* ``small2d``   2D, 32x32 cells, 50 observations, k=20, p=10
* ``medium2d``  2D, 256x256 cells, 400 observations, k=50, p=10
* ``cube3d``    3D, 64^3 cells (Kuhn tetrahedra), 1000 observations, k=100, p=20

Observation points are uniform in [0.05, 0.95]^d.  The true parameter is a
prior draw; the standard normals that define it (one per element quadrature
point, Appendix C) are drawn here and the prior solve is done by each side.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1909_03948


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    N: int            # cells per axis; nodes per axis = N + 1
    nobs: int
    gamma: float
    delta: float
    k: int
    p: int
    nsamples: int = 0
    seed: int = SEED_BASE
    noise_level: float = 0.01   # sigma = noise_level * max|u_true|

    @property
    def nnodes(self) -> int:
        return (self.N + 1) ** self.dim

    @property
    def nelems(self) -> int:
        return self.N ** self.dim * (2 if self.dim == 2 else 6)


WORKLOADS = {
    "small2d": Workload("small2d", 2, 32, 50, 0.1, 0.5, 20, 10, seed=SEED_BASE + 0),
    "medium2d": Workload("medium2d", 2, 256, 400, 0.1, 0.5, 50, 10, seed=SEED_BASE + 1),
    "cube3d": Workload("cube3d", 3, 64, 1000, 0.05, 0.5, 100, 20, nsamples=1000,
                       seed=SEED_BASE + 2),
}


def batch_workloads(nprob: int = 64, seed: int = SEED_BASE + 3) -> list:
    """Uneven batch: nprob independent 2D problems, N log-uniform in [64, 512] rounded to a
    multiple of 32 (so that the multigrid hierarchy ends on a grid of at most 17^2
    nodes), q uniform in {100..800}, gamma in [0.05, 0.2], delta in [0.2, 1.0], k=30, p=10."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nprob):
        N = int(np.clip(32 * np.round(np.exp(rng.uniform(np.log(64), np.log(512))) / 32), 64, 512))
        q = int(rng.integers(100, 801))
        gamma = float(rng.uniform(0.05, 0.2))
        delta = float(rng.uniform(0.2, 1.0))
        out.append(Workload(f"batch{i:02d}", 2, N, q, gamma, delta, 30, 10, seed=seed + 1000 + i))
    return out


def make_workload(dim: int, N: int, nobs: int, gamma: float = 0.1, delta: float = 0.5,
                  k: int = 10, p: int = 5, seed: int = SEED_BASE + 100) -> Workload:
    """Ad-hoc workload (test sizes)."""
    return Workload(f"d{dim}n{N}q{nobs}", dim, N, nobs, gamma, delta, k, p, seed=seed)


@dataclass
class Draws:
    """All random inputs of one inverse-problem instance."""
    obs_xyz: np.ndarray      # (nobs, dim) observation locations
    eta_true: np.ndarray     # (nelems, dim+1) standard normals for the true-parameter prior draw
    xi_noise: np.ndarray     # (nobs,) standard normals for the data noise
    extra: dict = field(default_factory=dict)


def draws(w: Workload) -> Draws:
    rng = np.random.default_rng(w.seed)
    obs = rng.uniform(0.05, 0.95, size=(w.nobs, w.dim))
    eta = rng.standard_normal((w.nelems, w.dim + 1))
    xi = rng.standard_normal(w.nobs)
    return Draws(obs, eta, xi)


def omega(w: Workload, ncols: int | None = None, seed_offset: int = 1) -> np.ndarray:
    """Gaussian test matrix Omega (n x (k+p)), column-major as returned (shape n, s)."""
    s = (w.k + w.p) if ncols is None else ncols
    rng = np.random.default_rng(w.seed + 7919 * seed_offset)
    return np.asfortranarray(rng.standard_normal((w.nnodes, s)))


def sample_normals(w: Workload, nsamples: int, seed_offset: int = 2) -> np.ndarray:
    """Per-element quadrature normals for ``nsamples`` Laplace samples, shape (nelems*(dim+1), nsamples)."""
    rng = np.random.default_rng(w.seed + 7919 * seed_offset)
    return np.asfortranarray(rng.standard_normal((w.nelems * (w.dim + 1), nsamples)))


def random_block(n: int, s: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, s)))
