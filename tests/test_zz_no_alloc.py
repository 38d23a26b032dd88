"""hp_mass_solve_noalloc: the mass-matrix solve for callers that cannot allocate
device memory when they solve -- an application that reserves all device memory up
front, or must keep its device footprint fixed while it runs.  The entry point
keeps its temporaries in one fixed device array inside the library.

Checked here through the C ABI: two calls in a row with different right-hand sides
each agree with the allocating hp_mass_solve and with the oracle's M^{-1} B to the
solve tolerance used by the other parity tests (relative 1e-8 per column), and,
after a first call that may trigger lazy loading of the library's device module,
further calls leave the device's free memory unchanged.  An output block of the
wrong shape is refused before the library is called.  This file is collected last
so that a failure here cannot hide failures elsewhere; it also passes when run on
its own.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle.fem import Mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _colrel(A, B):
    return max(np.linalg.norm(A[j] - B[j]) / np.linalg.norm(B[j]) for j in range(B.shape[0]))


def test_noalloc_mass_solve_matches_allocating_solve():
    from paper_1909_03948_gb300 import Problem
    w = W.make_workload(2, 32, 10, seed=W.SEED_BASE + 900)
    dr = W.draws(w)
    P = Problem(2, w.N, w.gamma, w.delta, 0.01, dr.obs_xyz, rtol=1e-10)
    dev = torch.device("cuda", 0)
    out = torch.empty((3, P.n), dtype=torch.float64, device=dev)
    M = Mesh(2, w.N).mass.tocsc()
    for call in range(2):
        Bh = W.random_block(P.n, 3, 70 + call)
        B = torch.tensor(np.ascontiguousarray(Bh.T), device=dev)
        ref, _ = P.mass_solve(B)
        got, st = P.mass_solve_noalloc(B, out)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert _colrel(got, ref.cpu().numpy()) < 1e-8
        assert _colrel(got, spla.splu(M).solve(Bh).T) < 1e-8      # the oracle's M^{-1} B
        assert st["iterations"] > 0
    # no device allocation by the call: free memory is unchanged across more calls
    B = torch.tensor(np.ascontiguousarray(W.random_block(P.n, 3, 99).T), device=dev)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        P.mass_solve_noalloc(B, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    P.close()


def test_noalloc_rejects_oversized_blocks():
    from paper_1909_03948_gb300 import HPError, Problem
    P = Problem(2, 8, 0.1, 0.5, 0.01, np.array([[0.5, 0.5]]))
    dev = torch.device("cuda", 0)
    B = torch.zeros((65, P.n), dtype=torch.float64, device=dev)
    with pytest.raises(HPError):
        P.mass_solve_noalloc(B, torch.empty_like(B))
    B = torch.zeros((3, P.n), dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):                  # fewer output columns than B has
        P.mass_solve_noalloc(B, torch.empty((2, P.n), dtype=torch.float64, device=dev))
    P.close()
