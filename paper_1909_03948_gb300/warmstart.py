"""Training data and training of the learned warm start (2D problems).

The network (``hp.UNet``) learns the solution of the stiffness system K(m) x = b
from (m, b) on the padded nodal grid.  Its training samples are the method's own
solves, recorded by the library while it runs:

* one state solve per log-coefficient m (``hp_set_point``), and
* one block of ``ncols`` Gauss-Newton Hessian actions at m on Philox normal
  directions: ``ncols`` incremental forward and ``ncols`` incremental adjoint solves.

The log-coefficients are prior draws (the prior leg of the Laplace sampler with
device Philox normals), so the training set covers the parameters the method meets
in Newton-CG and in the eigensolver.  Every step here runs in the library's CUDA
kernels; this module only schedules the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from .hp import UNet, philox_normals

_LAYERS = (  # (c_in, c_out, kernel) in the packed order of the library
    (3, 16, 3), (16, 16, 3), (16, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3), (64, 128, 3),
    (128, 128, 3), (192, 64, 3), (64, 64, 3), (96, 32, 3), (32, 32, 3), (48, 16, 3), (16, 16, 3),
    (16, 1, 1),
)


def he_init(seed: int = 0, out_scale: float = 1.0) -> np.ndarray:
    """Packed float32 parameters: He-normal weights (std sqrt(2 / fan_in)), zero biases;
    the 1x1 output layer's weights are multiplied by ``out_scale``."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (ci, co, k) in enumerate(_LAYERS):
        w = rng.standard_normal(co * ci * k * k) * np.sqrt(2.0 / (ci * k * k))
        if li == len(_LAYERS) - 1:
            w *= out_scale
        parts += [w, np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def prior_draws(problem, nsamples: int, seed: int) -> torch.Tensor:
    """(nsamples, n) prior samples m ~ N(m_prior, R^-1) drawn on the device."""
    prior, _, _ = problem.laplace_sample(None, None, None, None, want_prior=True, want_post=False,
                                         seed=seed, nsamples=nsamples)
    return prior


def generate(problem, ms: torch.Tensor, ncols: int, seed: int, with_solutions: bool = False):
    """Records 1 + 2 ncols solves per row of ``ms``; returns (X, A) -- or (X, A, T) with
    the scaled solutions -- as CUDA float32 tensors."""
    H, W = problem.warmstart_grid()
    cap = ms.shape[0] * (1 + 2 * ncols)
    dev = ms.device
    X = torch.empty((cap, 3, H, W), dtype=torch.float32, device=dev)
    A = torch.empty((cap, 4, H, W), dtype=torch.float32, device=dev)
    T = torch.empty((cap, 1, H, W), dtype=torch.float32, device=dev) if with_solutions else None
    problem.warmstart_record(X, A, T)
    try:
        for i in range(ms.shape[0]):
            problem.set_point(ms[i].contiguous())
            D = philox_normals(seed, i * ncols, ncols, problem.n, device=dev)
            problem.hessian_apply(D)
        count = problem.warmstart_counts()["recorded"]
    finally:
        problem.warmstart_record()
    if with_solutions:
        return X[:count], A[:count], T[:count]
    return X[:count], A[:count]


def train(X, A, epochs: int, batch: int = 16, lr: float = 1e-3, seed: int = 0, init_seed: int = 0,
          net: UNet | None = None):
    """Trains a network (a new He-initialised one unless ``net`` is given) with Adam on
    the samples; returns (net, mean loss per epoch)."""
    if net is None:
        net = UNet(X.shape[2], X.shape[3], batch_cap=batch)
        net.set_params(he_init(init_seed, out_scale=0.1))
    losses = net.train(X, A, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return net, losses
