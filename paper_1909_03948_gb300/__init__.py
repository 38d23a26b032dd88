"""GB300-native Gauss-Newton Hessian-action engine for the log-coefficient
Poisson inverse problem (hIPPYlib, Part I).

The engine is the C-ABI library ``libhp.so`` (declared in include/hp.h, built
from ``csrc/`` by ``build.py``); ``hp`` is its ctypes binding.  Importing the
package does not load the library; the first call does, and raises if it is
missing.  ``warmstart`` generates training data for, and trains, the learned
initial guess of the 2D stiffness solves (``UNet``).
"""
from .hp import (Batch, Problem, UNet, HPError, lib, kernel_launches, tiled_kernel_launches,  # noqa: F401
                 algorithmic_bytes, philox_normals, EXPORTED, LIB_PATH)

__all__ = ["Batch", "Problem", "UNet", "HPError", "lib", "kernel_launches", "tiled_kernel_launches",
           "algorithmic_bytes", "philox_normals", "EXPORTED", "LIB_PATH"]
